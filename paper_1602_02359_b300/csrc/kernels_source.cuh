// Source step (flow-chart cell 7): sub-step 1, artificial viscosity with
// compression heating, and the viscous stress tensor.
//
// Every kernel runs one thread per cell of the augmented mesh (ghosts and the
// extra face row, plus the extra face plane when Z is active) and writes its
// output velocity buffer completely: interior faces get the update, every
// other face is copied, so the buffers can ping-pong without stale values.
// Without a Z direction v_z is not a variable of the method: it is neither
// read nor written.  The bodies take the cell (i, j, k) with 0 <= i < nx; the
// kernel wrappers map their launch shape onto cells.
#pragma once
#include "fargo_internal.cuh"

namespace fk {

// Planes of the augmented mesh the per-cell kernels visit: the extra face
// plane only holds v_z of the last ghost's upper face.
__device__ __host__ __forceinline__ int cell_planes(const MeshD &m) { return m.nzt + (m.hasZ ? 1 : 0); }
// Rows j0..j1 and planes k0..k1 of the stress pass (the upper ones only with
// that direction).
__device__ __host__ __forceinline__ int tau_rows(const MeshD &m) { return m.j1 - m.j0 + (m.hasY ? 1 : 0); }
__device__ __host__ __forceinline__ int tau_planes(const MeshD &m) { return m.k1 - m.k0 + (m.hasZ ? 1 : 0); }

// Pressure from the equation of state (Eqs. eos1, eos2).
template <typename T, class F = CfgRun>
__device__ __forceinline__ T pressure(const MeshD &m, const Tab<T> &tb, const Fld<T> &f, idx_t c, int ring)
{
    if (F::iso(m)) {
        T cs = tb.cs[ring];
        return cs * cs * f.rho[c];
    }
    return tb.gm1 * f.e[c];
}

// Planet part of the potential at the centre of cell (i, ring): Plummer
// potential of the planet and the indirect term.  The squared distance is
// written without cancellation, d^2 = (R - a)^2 + 4 R a sin^2(dphi/2) + Z^2,
// from per-ring tables (R - a formed in FP64) and the per-step azimuth
// tables, so the hot loop needs no FP64 arithmetic.  The star term, which has
// no azimuthal dependence, enters through precomputed FP64 face gradients.
template <typename T, class F = CfgRun>
__device__ __forceinline__ T phi_planet(const MeshD &m, const Tab<T> &tb, int i, int ring)
{
    if (F::live(m)) {   // planets read on the device, each with its own tables
        const int NR = m.nyt * m.nzt;
        T v = T(0);
        for (int p = 0; p < m.pl_n; p++) {
            const T *tp = tb.mring + (size_t)p * 5 * NR;
            const T rm = tp[ring];
            const T d2 = rm * rm + tp[NR + ring] * tb.ps[p * m.nx + i] + tp[2 * NR + ring] + tb.peps2;
            const T qp = tb.mq[p];
            if (sizeof(T) == 8) v -= qp / sqrt(d2);
            else v -= qp * rsqrtf((float)d2);
            if (F::indirect(m)) v += tp[3 * NR + ring] * tb.pc[p * m.nx + i] + tp[4 * NR + ring];
        }
        return v;
    }
    const T rm = tb.rma[ring];
    const T d2 = rm * rm + tb.fra[ring] * tb.ps[i] + tb.z2[ring] + tb.peps2;
    T v;
    if (sizeof(T) == 8) v = -tb.pq / sqrt(d2);
    else v = -tb.pq * rsqrtf((float)d2);
    if (F::indirect(m)) v += tb.qar[ring] * tb.pc[i];
    return v;
}

// ---------------------------------------------------------------------------
// Sub-step 1 (Sec. 3.3): pressure gradient with the two-point face density
// (Eq. 20), potential gradient, centrifugal and geometric terms with the
// four-face average of Eq. 12.  Jacobi: reads `in`, writes `out`.
// ---------------------------------------------------------------------------
template <typename T, class F = CfgRun>
__device__ __forceinline__ void substep1_body(const MeshD &m, const Tab<T> &tb, const Fld<T> &in, const Fld<T> &out,
                                              const Scal *sc, int i, int j, int k)
{
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    const idx_t c = IX(m, i, j, k);
    const bool jact = j >= m.j0 && j < m.j1, kact = k >= m.k0 && k < m.k1;
    const int ring = k * m.nyt + j;
    const T om = tb.omega;
    const int im = i == 0 ? m.nx - 1 : i - 1;
    const int ip = i + 1 == m.nx ? 0 : i + 1;
    // the three face values are stored at the end: no store sits between the
    // loads, so the compiler may keep every loaded value for all three faces
    T ox = T(0), oy = T(0), oz = T(0);
    bool wx = false, wy = false, wz = false;
    if (j < m.nyt && k < m.nzt) {
        T v = in.vx[c];
        if (F::hasX(m) && jact && kact) {
            const idx_t cm = c - i + im;
            const T id = tb.ilenx[ring];
            const T P0 = pressure<T, F>(m, tb, in, c, ring), Pm = pressure<T, F>(m, tb, in, cm, ring);
            T acc = div_fast(T(-2) * (P0 - Pm) * id, in.rho[c] + in.rho[cm]);
            if (F::planet(m))
                acc -= (phi_planet<T, F>(m, tb, i, ring) - phi_planet<T, F>(m, tb, im, ring)) * id;
            v = v + dt * acc;
        }
        ox = v;
        wx = true;
    }
    if (k < m.nzt) {
        T v = in.vy[c];
        if (F::hasY(m) && j >= m.jf && j < m.j1 && kact) {
            const idx_t cm = c - m.sj;
            const T id = tb.idyc[j];
            const T P0 = pressure<T, F>(m, tb, in, c, ring), Pm = pressure<T, F>(m, tb, in, cm, ring - 1);
            T acc = div_fast(T(-2) * (P0 - Pm) * id, in.rho[c] + in.rho[cm]);
            if (F::planet(m))
                acc -= (phi_planet<T, F>(m, tb, i, ring) - phi_planet<T, F>(m, tb, i, ring - 1)) * id;
            if (F::star(m)) acc -= tb.gphy[ring];
            if (F::geom(m) != CART) {
                // (the reference velocity of the reference form joins the frame's R Omega)
                const T Rj = tb.R[ring], Rm = tb.R[ring - 1];
                const T uj = Rj * om + vref_at(tb, ring), um = Rm * om + vref_at(tb, ring - 1);
                const idx_t cp = c - i + ip, cmp = cm - i + ip;
                const T vt = T(0.25) * ((in.vx[c] + uj) + (in.vx[cp] + uj) + (in.vx[cm] + um) + (in.vx[cmp] + um));
                T cen = vt * vt;
                if (F::geom(m) == SPH && F::hasZ(m)) {
                    const T vth = T(0.25) * (in.vz[c] + in.vz[c + m.sk] + in.vz[cm] + in.vz[cm + m.sk]);
                    cen += vth * vth;
                }
                acc += cen * tb.iyf[j];
            } else if (F::shearing(m)) {
                // shearing sheet: Coriolis 2 Omega_f v_x (v_x averaged over the four
                // faces around the Y face) and the tide -4 A Omega_f y
                const idx_t cp = c - i + ip, cmp = cm - i + ip;
                const T vxa = T(0.25) * (in.vx[c] + in.vx[cp] + in.vx[cm] + in.vx[cmp]) +
                              T(0.5) * (vref_at(tb, ring) + vref_at(tb, ring - 1));
                acc += T(2) * om * vxa - tb.tid[j];
            }
            v = v + dt * acc;
        }
        oy = v;
        wy = true;
    }
    if (F::hasZ(m) && j < m.nyt) {
        T v = in.vz[c];
        if (k >= m.kf && k < m.k1 && jact) {
            const idx_t cm = c - m.sk;
            const int rm = ring - m.nyt;
            const T id = tb.idzc[ring];
            const T P0 = pressure<T, F>(m, tb, in, c, ring), Pm = pressure<T, F>(m, tb, in, cm, rm);
            T acc = div_fast(T(-2) * (P0 - Pm) * id, in.rho[c] + in.rho[cm]);
            if (F::planet(m))
                acc -= (phi_planet<T, F>(m, tb, i, ring) - phi_planet<T, F>(m, tb, i, rm)) * id;
            if (F::star(m)) acc -= tb.gphz[ring];
            if (F::geom(m) == SPH) {
                const T Rk = tb.R[ring], Rm = tb.R[rm];
                const T uk = Rk * om + vref_at(tb, ring), um = Rm * om + vref_at(tb, rm);
                const idx_t cp = c - i + ip, cmp = cm - i + ip;
                const T vt = T(0.25) * ((in.vx[c] + uk) + (in.vx[cp] + uk) + (in.vx[cm] + um) + (in.vx[cmp] + um));
                acc += vt * vt * tb.cotzf[k] * tb.iym[j];
            }
            v = v + dt * acc;
        }
        oz = v;
        wz = true;
    }
    if (wx) out.vx[c] = ox;
    if (wy) out.vy[c] = oy;
    if (wz) out.vz[c] = oz;
}

// ---------------------------------------------------------------------------
// Sub-steps 2 and 3: von Neumann-Richtmyer artificial viscosity applied
// component-wise, q_d = C_q^2 rho (Delta v_d)^2 for compressions, its
// gradient on interior faces (two-point density), the heating -q Delta v /
// Delta, then the compression heating e (1 - theta)/(1 + theta),
// theta = dt (gamma-1) div v / 2, with div v from the post-viscosity
// velocities.  q of a neighbour is recomputed locally instead of stored, so
// the two passes of the paper become one kernel without races.
// ---------------------------------------------------------------------------
template <typename T, class F = CfgRun>
__device__ __forceinline__ T qvisc(T c2, T rho, T dv)
{
    return dv < T(0) ? c2 * rho * dv * dv : T(0);
}

template <typename T, class F = CfgRun>
__device__ __forceinline__ void artvisc_body(const MeshD &m, const Tab<T> &tb, const Fld<T> &in, const Fld<T> &out,
                                             const Scal *sc, int i, int j, int k)
{
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    const T c2 = tb.cq2;
    const bool av = F::av(m) != 0;
    const idx_t c = IX(m, i, j, k);
    const bool jact = j >= m.j0 && j < m.j1, kact = k >= m.k0 && k < m.k1;
    const int ring = k * m.nyt + j;
    const int im = i == 0 ? m.nx - 1 : i - 1;
    const int ip = i + 1 == m.nx ? 0 : i + 1;
    const int ipp = ip + 1 == m.nx ? 0 : ip + 1;
    const T *vx = in.vx, *vy = in.vy, *vz = in.vz, *rho = in.rho;
    const idx_t sj = m.sj, sk = m.sk;
    // own lower faces (stored at the end: no store sits between the loads,
    // so the compiler may keep every loaded value for all faces and e)
    T vxl = 0, vyl = 0, vzl = 0;
    bool wx = false, wy = false, wz = false;
    auto store_v = [&]() {
        if (wx) out.vx[c] = vxl;
        if (wy) out.vy[c] = vyl;
        if (wz) out.vz[c] = vzl;
    };
    if (j < m.nyt && k < m.nzt) {
        T v = vx[c];
        if (av && F::hasX(m) && jact && kact) {
            const idx_t cm = c - i + im, cp = c - i + ip;
            const T q0 = qvisc(c2, rho[c], vx[cp] - vx[c]);
            const T qm = qvisc(c2, rho[cm], vx[c] - vx[cm]);
            v -= div_fast(dt * T(2) * (q0 - qm) * tb.ilenx[ring], rho[c] + rho[cm]);
        }
        vxl = v;
        wx = true;
    }
    if (k < m.nzt) {
        T v = vy[c];
        if (av && F::hasY(m) && j >= m.jf && j < m.j1 && kact) {
            const idx_t cm = c - sj;
            const T q0 = qvisc(c2, rho[c], vy[c + sj] - vy[c]);
            const T qm = qvisc(c2, rho[cm], vy[c] - vy[cm]);
            v -= div_fast(dt * T(2) * (q0 - qm) * tb.idyc[j], rho[c] + rho[cm]);
        }
        vyl = v;
        wy = true;
    }
    if (F::hasZ(m) && j < m.nyt) {
        T v = vz[c];
        if (av && k >= m.kf && k < m.k1 && jact) {
            const idx_t cm = c - sk;
            const T q0 = qvisc(c2, rho[c], vz[c + sk] - vz[c]);
            const T qm = qvisc(c2, rho[cm], vz[c] - vz[cm]);
            v -= div_fast(dt * T(2) * (q0 - qm) * tb.idzc[ring], rho[c] + rho[cm]);
        }
        vzl = v;
        wz = true;
    }
    if (F::iso(m) || !(jact && kact)) {
        store_v();
        return;
    }
    // heating by the artificial viscosity of the cell itself
    T e = in.e[c];
    T h = 0;
    if (av) {
        if (F::hasX(m)) {
            const T dv = vx[c - i + ip] - vx[c];
            h += qvisc(c2, rho[c], dv) * dv * tb.ilenx[ring];
        }
        if (F::hasY(m)) {
            const T dv = vy[c + sj] - vy[c];
            h += qvisc(c2, rho[c], dv) * dv * tb.idy[j];
        }
        if (F::hasZ(m)) {
            const T dv = vz[c + sk] - vz[c];
            h += qvisc(c2, rho[c], dv) * dv * tb.ilenz[ring];
        }
    }
    e -= dt * h;
    // post-viscosity velocities on the upper faces (owned by the neighbours)
    T div = 0;
    if (F::hasX(m)) {
        const idx_t cp = c - i + ip, cpp = c - i + ipp;
        T vxu = vx[cp];
        if (av) {
            const T qp = qvisc(c2, rho[cp], vx[cpp] - vx[cp]);
            const T q0 = qvisc(c2, rho[c], vx[cp] - vx[c]);
            vxu -= div_fast(dt * T(2) * (qp - q0) * tb.ilenx[ring], rho[cp] + rho[c]);
        }
        div += tb.sx[ring] * (vxu - vxl);
    }
    const int fr = k * (m.nyt + 1) + j;
    if (F::hasY(m)) {
        T vyu = vy[c + sj];
        // (on a periodic axis face j1 is face j0, an interior face)
        if (av && (j + 1 < m.j1 || m.pery)) {
            const T qp = qvisc(c2, rho[c + sj], vy[c + 2 * sj] - vy[c + sj]);
            const T q0 = qvisc(c2, rho[c], vy[c + sj] - vy[c]);
            vyu -= div_fast(dt * T(2) * (qp - q0) * tb.idyc[j + 1], rho[c + sj] + rho[c]);
        }
        div += tb.sy[fr + 1] * vyu - tb.sy[fr] * vyl;
    }
    if (F::hasZ(m)) {
        T vzu = vz[c + sk];
        if (av && (k + 1 < m.k1 || m.perz)) {
            const T qp = qvisc(c2, rho[c + sk], vz[c + 2 * sk] - vz[c + sk]);
            const T q0 = qvisc(c2, rho[c], vz[c + sk] - vz[c]);
            vzu -= div_fast(dt * T(2) * (qp - q0) * tb.idzc[ring + m.nyt], rho[c + sk] + rho[c]);
        }
        div += tb.sz[fr + (m.nyt + 1)] * vzu - tb.sz[fr] * vzl;
    }
    div *= tb.vinv[ring];
    const T th = tb.half_gm1 * dt * div;
    store_v();
    out.e[c] = e * (T(1) - th) / (T(1) + th);
}

// ---------------------------------------------------------------------------
// Viscous stress tensor and velocity update (Appendix B, Eqs. 72-77).
// Diagonal stresses at cell centres, off-diagonal ones on the lowest edges;
// edge density and viscosity are the means over the cells sharing the edge.
// Each thread recomputes the stresses its faces need from the velocities at
// sub-step entry (Jacobi), so no stress array is stored.
// ---------------------------------------------------------------------------
template <typename T, class F = CfgRun>
struct ViscCtx {
    const MeshD &m;
    const Tab<T> &tb;
    const T *rho, *vx, *vy, *vz;
    __device__ ViscCtx(const MeshD &m_, const Tab<T> &tb_, const Fld<T> &f)
        : m(m_), tb(tb_), rho(f.rho), vx(f.vx), vy(f.vy), vz(f.vz) {}
    // azimuthal velocity of face q on ring `ring` (in the reference form the
    // stored value plus the ring's reference)
    __device__ T vxa(int q, int ring) const { return sizeof(T) == 4 && tb.vref ? vx[q] + tb.vref[ring] : vx[q]; }
    __device__ int wrap(int i) const { return i < 0 ? i + m.nx : (i >= m.nx ? i - m.nx : i); }
    __device__ idx_t at(int i, int j, int k) const { return IX(m, wrap(i), j, k); }
    __device__ T nu(int j, int k) const { return tb.nu[k * m.nyt + j]; }

    __device__ T divv(int i, int j, int k) const
    {
        const idx_t c = at(i, j, k);
        const int ring = k * m.nyt + j, fr = k * (m.nyt + 1) + j;
        T f = 0;
        if (F::hasX(m)) f += tb.sx[ring] * (vx[at(i + 1, j, k)] - vx[c]);
        if (F::hasY(m)) f += tb.sy[fr + 1] * vy[c + m.sj] - tb.sy[fr] * vy[c];
        if (F::hasZ(m)) f += tb.sz[fr + m.nyt + 1] * vz[c + m.sk] - tb.sz[fr] * vz[c];
        return f * tb.vinv[ring];
    }
    // diagonal components at the centre of cell (i,j,k)
    __device__ void diag(int i, int j, int k, T &txx, T &tyy, T &tzz) const
    {
        const idx_t c = at(i, j, k);
        const int ring = k * m.nyt + j;
        const T dv = divv(i, j, k);
        const T rn = rho[c] * nu(j, k);
        const T dxx = (vx[at(i + 1, j, k)] - vx[c]) * tb.ilenx[ring];
        const T dyy = F::hasY(m) ? (vy[c + m.sj] - vy[c]) * tb.idy[j] : T(0);
        const T dzz = F::hasZ(m) ? (vz[c + m.sk] - vz[c]) * tb.ilenz[ring] : T(0);
        const T tw = T(2.0 / 3.0) * dv;
        if (F::geom(m) == CART) {
            txx = -rn * (T(2) * dxx - tw);
            tyy = -rn * (T(2) * dyy - tw);
            tzz = -rn * (T(2) * dzz - tw);
        } else if (F::geom(m) == CYL) {
            const T ir = tb.iym[j];
            const T vr = T(0.5) * (vy[c] + vy[c + m.sj]);
            txx = -rn * (T(2) * (dxx + vr * ir) - tw);
            tyy = -rn * (T(2) * dyy - tw);
            tzz = -rn * (T(2) * dzz - tw);
        } else {
            const T ir = tb.iym[j], ct = tb.cotzm[k];
            const T vr = T(0.5) * (vy[c] + vy[c + m.sj]);
            const T vt = T(0.5) * (vz[c] + vz[c + m.sk]);
            txx = -rn * (T(2) * (dxx + vr * ir + vt * ct * ir) - tw);
            tyy = -rn * (T(2) * dyy - tw);
            tzz = -rn * (T(2) * (dzz + vr * ir) - tw);
        }
    }
    // tau_xy on the edge (i-1/2, j-1/2, k)
    __device__ T txy(int i, int j, int k) const
    {
        const idx_t c = at(i, j, k), cm = at(i - 1, j, k);
        const int ring = k * m.nyt + j;
        const T rb = T(0.25) * (rho[c] + rho[cm] + rho[c - m.sj] + rho[cm - m.sj]);
        const T nb = T(0.5) * (nu(j, k) + nu(j - 1, k));
        const T v0 = vxa(c, ring), v1 = vxa(c - m.sj, ring - 1);
        const T dvx_dy = (v0 - v1) * tb.idyc[j];
        T t;
        if (F::geom(m) == CART) {
            t = (vy[c] - vy[cm]) * tb.idx + dvx_dy;
        } else if (F::geom(m) == CYL) {
            const T irf = tb.iyf[j];
            t = dvx_dy - T(0.5) * (v0 + v1) * irf + (vy[c] - vy[cm]) * (irf * tb.idx);
        } else {
            const T irf = tb.iyf[j], isn = tb.iszm[k];
            t = (vy[c] - vy[cm]) * (irf * isn * tb.idx) + dvx_dy - T(0.5) * (v0 + v1) * irf;
        }
        return -rb * nb * t;
    }
    // tau_xz on the edge (i-1/2, j, k-1/2)
    __device__ T txz(int i, int j, int k) const
    {
        const idx_t c = at(i, j, k), cm = at(i - 1, j, k);
        const int ring = k * m.nyt + j;
        const T rb = T(0.25) * (rho[c] + rho[cm] + rho[c - m.sk] + rho[cm - m.sk]);
        const T nb = T(0.5) * (nu(j, k) + nu(j, k - 1));
        const T idzm = tb.idzm[k];
        const T v0 = vxa(c, ring), v1 = vxa(c - m.sk, ring - m.nyt);
        T t;
        if (F::geom(m) == CART) {
            t = (vz[c] - vz[cm]) * tb.idx + (v0 - v1) * idzm;
        } else if (F::geom(m) == CYL) {
            t = (v0 - v1) * idzm + (vz[c] - vz[cm]) * (tb.iym[j] * tb.idx);
        } else {
            const T ir = tb.iym[j], sf = tb.szf[k];
            t = sf * ir * (v0 * tb.iszm[k] - v1 * tb.iszm[k - 1]) * idzm +
                div_fast((vz[c] - vz[cm]) * (ir * tb.idx), sf);
        }
        return -rb * nb * t;
    }
    // tau_yz on the edge (i, j-1/2, k-1/2)
    __device__ T tyz(int i, int j, int k) const
    {
        const idx_t c = at(i, j, k);
        const T rb = T(0.25) * (rho[c] + rho[c - m.sj] + rho[c - m.sk] + rho[c - m.sj - m.sk]);
        const T nb = T(0.25) * (nu(j, k) + nu(j - 1, k) + nu(j, k - 1) + nu(j - 1, k - 1));
        const T idzm = tb.idzm[k];
        T t;
        if (F::geom(m) == SPH) {
            const T irf = tb.iyf[j];
            t = (vz[c] - vz[c - m.sj]) * tb.idyc[j] - T(0.5) * (vz[c] + vz[c - m.sj]) * irf +
                (vy[c] - vy[c - m.sk]) * (irf * idzm);
        } else {
            t = (vz[c] - vz[c - m.sj]) * tb.idyc[j] + (vy[c] - vy[c - m.sk]) * idzm;
        }
        return -rb * nb * t;
    }
};

template <typename T, class F, typename S>
__device__ __forceinline__ void visc_apply(const MeshD &m, const Tab<T> &tb, const Fld<T> &in, const Fld<T> &out,
                                           T dt, int i, int j, int k, const S &V)
{
    const idx_t c = IX(m, i, j, k);
    const bool jact = j >= m.j0 && j < m.j1, kact = k >= m.k0 && k < m.k1;
    const T idx = tb.idx;
    const T *rho = in.rho;
    if (j < m.nyt && k < m.nzt) {
        T v = in.vx[c];
        if (jact && kact) {
            const idx_t cm = V.at(i - 1, j, k);
            T a0, a1, a2, b0, b1, b2;
            V.diag(i, j, k, a0, a1, a2);
            V.diag(i - 1, j, k, b0, b1, b2);
            T f = 0;
            if (F::geom(m) == CART) {
                f += (a0 - b0) * idx;
                if (F::hasY(m)) f += (V.txy(i, j + 1, k) - V.txy(i, j, k)) * tb.idy[j];
                if (F::hasZ(m)) f += (V.txz(i, j, k + 1) - V.txz(i, j, k)) * tb.idz[k];
            } else if (F::geom(m) == CYL) {
                const T ir = tb.iym[j];
                if (F::hasY(m))
                    f += (tb.yf[j + 1] * tb.yf[j + 1] * V.txy(i, j + 1, k) - tb.yf[j] * tb.yf[j] * V.txy(i, j, k)) *
                         (ir * ir * tb.idy[j]);
                f += (a0 - b0) * (ir * idx);
                if (F::hasZ(m)) f += (V.txz(i, j, k + 1) - V.txz(i, j, k)) * tb.idz[k];
            } else {
                const T ir = tb.iym[j], isn = tb.iszm[k], ct = tb.cotzm[k];
                T ty0 = 0, ty1 = 0, tz0 = 0, tz1 = 0;
                if (F::hasY(m)) {
                    ty0 = V.txy(i, j, k);
                    ty1 = V.txy(i, j + 1, k);
                    f += (tb.yf[j + 1] * tb.yf[j + 1] * ty1 - tb.yf[j] * tb.yf[j] * ty0) * (ir * ir * tb.idy[j]);
                }
                if (F::hasZ(m)) {
                    tz0 = V.txz(i, j, k);
                    tz1 = V.txz(i, j, k + 1);
                    f += (tz1 - tz0) * (ir * tb.idz[k]);
                }
                f += (a0 - b0) * (ir * isn * idx);
                if (F::hasY(m)) f += T(0.5) * (ty0 + ty1) * ir;
                if (F::hasZ(m)) f += T(2) * T(0.5) * (tz0 + tz1) * ct * ir;
            }
            v = v - div_fast(T(2) * dt * f, rho[c] + rho[cm]);
        }
        out.vx[c] = v;
    }
    if (k < m.nzt) {
        T v = in.vy[c];
        if (F::hasY(m) && j >= m.jf && j < m.j1 && kact) {
            const idx_t cjm = c - m.sj;
            T a0, a1, a2, b0, b1, b2;
            V.diag(i, j, k, a0, a1, a2);
            V.diag(i, j - 1, k, b0, b1, b2);
            T f = 0;
            if (F::geom(m) == CART) {
                f += (V.txy(i + 1, j, k) - V.txy(i, j, k)) * idx;
                f += (a1 - b1) * tb.idyc[j];
                if (F::hasZ(m)) f += (V.tyz(i, j, k + 1) - V.tyz(i, j, k)) * tb.idz[k];
            } else if (F::geom(m) == CYL) {
                const T irf = tb.iyf[j];
                f += (tb.ym[j] * a1 - tb.ym[j - 1] * b1) * (irf * tb.idyc[j]);
                f += (V.txy(i + 1, j, k) - V.txy(i, j, k)) * (irf * idx);
                f -= T(0.5) * (a0 + b0) * irf;
                if (F::hasZ(m)) f += (V.tyz(i, j, k + 1) - V.tyz(i, j, k)) * tb.idz[k];
            } else {
                const T irf = tb.iyf[j], isn = tb.iszm[k];
                f += (tb.ym[j] * tb.ym[j] * a1 - tb.ym[j - 1] * tb.ym[j - 1] * b1) * (irf * irf * tb.idyc[j]);
                if (F::hasZ(m))
                    f += (V.tyz(i, j, k + 1) * tb.szf[k + 1] - V.tyz(i, j, k) * tb.szf[k]) * (irf * isn * tb.idz[k]);
                f += (V.txy(i + 1, j, k) - V.txy(i, j, k)) * (irf * isn * idx);
                f -= T(0.5) * (a2 + b2 + a0 + b0) * irf;
            }
            v = v - div_fast(T(2) * dt * f, rho[c] + rho[cjm]);
        }
        out.vy[c] = v;
    }
    if (F::hasZ(m) && j < m.nyt) {
        T v = in.vz[c];
        if (k >= m.kf && k < m.k1 && jact) {
            const idx_t ckm = c - m.sk;
            T a0, a1, a2, b0, b1, b2;
            V.diag(i, j, k, a0, a1, a2);
            V.diag(i, j, k - 1, b0, b1, b2);
            const T idzm = tb.idzm[k];
            T f = 0;
            if (F::geom(m) == CART) {
                f += (V.txz(i + 1, j, k) - V.txz(i, j, k)) * idx;
                if (F::hasY(m)) f += (V.tyz(i, j + 1, k) - V.tyz(i, j, k)) * tb.idy[j];
                f += (a2 - b2) * idzm;
            } else if (F::geom(m) == CYL) {
                const T ir = tb.iym[j];
                if (F::hasY(m)) f += (tb.yf[j + 1] * V.tyz(i, j + 1, k) - tb.yf[j] * V.tyz(i, j, k)) * (ir * tb.idy[j]);
                f += (V.txz(i + 1, j, k) - V.txz(i, j, k)) * (ir * idx);
                f += (a2 - b2) * idzm;
            } else {
                const T ir = tb.iym[j], sf = tb.szf[k], isf = div_fast(T(1), sf), ctf = tb.cotzf[k];
                if (F::hasY(m)) {
                    const T y1 = tb.yf[j + 1], y0 = tb.yf[j];
                    f += (y1 * y1 * y1 * V.tyz(i, j + 1, k) - y0 * y0 * y0 * V.tyz(i, j, k)) * (ir * ir * ir * tb.idy[j]);
                }
                f += (a2 * tb.szm[k] - b2 * tb.szm[k - 1]) * (ir * isf * idzm);
                f += (V.txz(i + 1, j, k) - V.txz(i, j, k)) * (ir * isf * idx);
                f -= T(0.5) * (a0 + b0) * ctf * ir;
            }
            v = v - div_fast(T(2) * dt * f, rho[c] + rho[ckm]);
        }
        out.vz[c] = v;
    }
}

// Stresses read back from the arrays written by k_visc_tau.
template <typename T, class F = CfgRun>
struct TauArr {
    const MeshD &m;
    const T *xx, *yy, *zz, *xy, *xz, *yz;
    __device__ idx_t at(int i, int j, int k) const
    {
        return IX(m, i < 0 ? i + m.nx : (i >= m.nx ? i - m.nx : i), j, k);
    }
    __device__ void diag(int i, int j, int k, T &a, T &b, T &c) const
    {
        const idx_t o = at(i, j, k);
        a = xx[o];
        b = yy[o];
        c = F::hasZ(m) ? zz[o] : T(0);
    }
    __device__ T txy(int i, int j, int k) const { return xy[at(i, j, k)]; }
    __device__ T txz(int i, int j, int k) const { return xz[at(i, j, k)]; }
    __device__ T tyz(int i, int j, int k) const { return yz[at(i, j, k)]; }
};

// Pass 1: every stress component once, diagonal ones on active cells and
// the edge ones on the edges that interior and boundary faces need
// (rows j0..j1, planes k0..k1).
template <typename T, class F = CfgRun>
__device__ __forceinline__ void visc_tau_body(const MeshD &m, const Tab<T> &tb, const Fld<T> &in, const QSet<T> &tau,
                                              const Scal *sc, int i, int j, int k)
{
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    // rows j0..j1, planes k0..k1 (the upper one only with that direction)
    if (j < m.j0 || j > m.j1 - (F::hasY(m) ? 0 : 1) || k < m.k0 || k > m.k1 - (F::hasZ(m) ? 0 : 1)) return;
    const ViscCtx<T, F> V(m, tb, in);
    const idx_t c = IX(m, i, j, k);
    const bool jin = j < m.j1, kin = k < m.k1;
    if (jin && kin) {
        T a, b, d;
        V.diag(i, j, k, a, b, d);
        tau.q[0][c] = a;
        tau.q[1][c] = b;
        if (F::hasZ(m)) tau.q[2][c] = d;
    }
    if (F::hasY(m) && kin) tau.q[3][c] = V.txy(i, j, k);
    if (F::hasZ(m) && jin) tau.q[4][c] = V.txz(i, j, k);
    if (F::hasY(m) && F::hasZ(m)) tau.q[5][c] = V.tyz(i, j, k);
}

// Pass 2: the velocity update of Eqs. 75-77 from the stored stresses.
template <typename T, class F = CfgRun>
__device__ __forceinline__ void visc_apply_body(const MeshD &m, const Tab<T> &tb, const Fld<T> &in,
                                                const Fld<T> &out, const QSet<T> &tau, const Scal *sc, int i,
                                                int j, int k)
{
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    const TauArr<T, F> S{m, tau.q[0], tau.q[1], tau.q[2], tau.q[3], tau.q[4], tau.q[5]};
    visc_apply<T, F>(m, tb, in, out, dt, i, j, k, S);
}

// Single-instance wrappers: a 3D grid, x over the azimuth (blockDim.x
// cells per block), y over the rows, z over the planes.
// (eight blocks per SM: a 32-register budget, full occupancy)
template <typename T, class F = CfgRun>
__global__ void __launch_bounds__(256, 8) k_substep1(MeshD m, Tab<T> tb, Fld<T> in, Fld<T> out, const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) substep1_body<T, F>(m, tb, in, out, sc, i, blockIdx.y, blockIdx.z);
}
template <typename T, class F = CfgRun>
__global__ void __launch_bounds__(256) k_artvisc(MeshD m, Tab<T> tb, Fld<T> in, Fld<T> out, const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) artvisc_body<T, F>(m, tb, in, out, sc, i, blockIdx.y, blockIdx.z);
}
// grid rows and planes start at j0 and k0
template <typename T, class F = CfgRun>
__global__ void __launch_bounds__(256) k_visc_tau(MeshD m, Tab<T> tb, Fld<T> in, QSet<T> tau, const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) visc_tau_body<T, F>(m, tb, in, tau, sc, i, m.j0 + blockIdx.y, m.k0 + blockIdx.z);
}
template <typename T, class F = CfgRun>
__global__ void __launch_bounds__(256) k_visc_apply(MeshD m, Tab<T> tb, Fld<T> in, Fld<T> out, QSet<T> tau,
                                                    const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) visc_apply_body<T, F>(m, tb, in, out, tau, sc, i, blockIdx.y, blockIdx.z);
}

// Launches with the configuration class cfg_of(m) selects.
template <typename T, class F>
static void launch_source_cfg(int which, const MeshD &m, dim3 g, dim3 b, cudaStream_t s, const Tab<T> &tb,
                              const Fld<T> &in, const Fld<T> &out, const QSet<T> &tau, const Scal *sc)
{
    switch (which) {
    case 0: k_substep1<T, F><<<g, b, 0, s>>>(m, tb, in, out, sc); break;
    case 1: k_artvisc<T, F><<<g, b, 0, s>>>(m, tb, in, out, sc); break;
    case 2: k_visc_tau<T, F><<<g, b, 0, s>>>(m, tb, in, tau, sc); break;
    default: k_visc_apply<T, F><<<g, b, 0, s>>>(m, tb, in, out, tau, sc); break;
    }
}
enum { SRC_SUB1 = 0, SRC_AV = 1, SRC_TAU = 2, SRC_VAPPLY = 3 };
// which: SRC_*; out is unused by SRC_TAU, tau by SRC_SUB1 and SRC_AV
template <typename T>
static void launch_source(int which, const MeshD &m, dim3 g, dim3 b, cudaStream_t s, const Tab<T> &tb,
                          const Fld<T> &in, const Fld<T> &out, const QSet<T> &tau, const Scal *sc)
{
    switch (cfg_of(m)) {
    case CFG_DISK3D: launch_source_cfg<T, CfgDisk3D>(which, m, g, b, s, tb, in, out, tau, sc); break;
    case CFG_DISK2D: launch_source_cfg<T, CfgDisk2D>(which, m, g, b, s, tb, in, out, tau, sc); break;
    case CFG_DISK3D_LIVE: launch_source_cfg<T, CfgDisk3DLive>(which, m, g, b, s, tb, in, out, tau, sc); break;
    case CFG_DISK2D_LIVE: launch_source_cfg<T, CfgDisk2DLive>(which, m, g, b, s, tb, in, out, tau, sc); break;
    default: launch_source_cfg<T, CfgRun>(which, m, g, b, s, tb, in, out, tau, sc); break;
    }
}

}  // namespace fk
