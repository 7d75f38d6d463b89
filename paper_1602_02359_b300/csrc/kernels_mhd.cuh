// Magnetohydrodynamics on Cartesian meshes (Sec. 3.5: the method of
// characteristics with constrained transport, MOCCT), mu_0 = 1.
//
// B is face centred like v (Sec. 2.3).  EMF component o lives on the edges
// along o; the one stored at index (i, j, k) is at the lower a-face and the
// lower b-face of cell (i, j, k), a = o + 1, b = o + 2 (mod 3).  Directions
// are X = 0, Y = 1, Z = 2; X is periodic; along an absent direction (a single
// cell) every difference vanishes and every average is the value itself.
//
// The kernels, in the order of the step:
//   k_mhd_pressure (cell 7a, after sub-step 1): minus the gradient of the
//     transverse magnetic pressure, from zone-centred two-point averages of
//     B, on every interior face velocity, in place;
//   k_mhd_edges (cells 8a-8d): the three EMFs of every edge (Eq. 45, with
//     the star values of Eqs. 41-44) minus eta curl B, and the magnetic
//     tension of Eq. 47 on every interior face velocity, out of place
//     (every component from the velocities on entry), from one set of
//     reconstructions per edge;
//   k_mhd_ct (cell 10, after the ghost fill of cell 9): the constrained
//     transport B_a += dt (d_b e_o - d_o e_b) for the cyclic (a, b, o) on
//     every interior face, in place.  Eq. 39 is printed with the signs of
//     e = B x v; the update follows the induction equation for e = v x B.
// Every kernel returns at once on a void step (dt <= 0).
#pragma once
#include "fargo_internal.cuh"
#include "kernels_bc_cfl.cuh"
#include "kernels_transport.cuh"

namespace fk {

__device__ __forceinline__ bool mh_has(const MeshD &m, int d) { return d == 0 ? m.hasX : (d == 1 ? m.hasY : m.hasZ); }
__device__ __forceinline__ int mh_pos(int i, int j, int k, int d) { return d == 0 ? i : (d == 1 ? j : k); }

// (i, j, k) moved by off cells along d, |off| <= 2 (X periodic; no move
// along an absent direction).
__device__ __forceinline__ void mh_shift(const MeshD &m, int &i, int &j, int &k, int d, int off)
{
    if (d == 0) {
        if (m.hasX) {
            i += off;
            i = i < 0 ? i + m.nx : (i >= m.nx ? i - m.nx : i);
        }
    } else if (d == 1) {
        if (m.hasY) j += off;
    } else if (m.hasZ) {
        k += off;
    }
}
__device__ __forceinline__ idx_t mh_nb(const MeshD &m, int i, int j, int k, int d, int off)
{
    mh_shift(m, i, j, k, d, off);
    return IX(m, i, j, k);
}

// Width of cell n along d, and the inverse of the distance between the
// centres of cells n - 1 and n (X uniform).
template <typename T>
__device__ __forceinline__ T mh_width(const Tab<T> &tb, int d, int n)
{
    return d == 0 ? tb.dx : (d == 1 ? tb.dy[n] : tb.dz[n]);
}
template <typename T>
__device__ __forceinline__ T mh_idc(const Tab<T> &tb, int d, int n)
{
    return d == 0 ? tb.idx : (d == 1 ? tb.mh_idcy[n] : tb.mh_idcz[n]);
}

// The reconstructions of one quantity q, cell centred along e, at the face
// between cells n - 1 and n: the upwind cell's value plus its van Leer
// slope times half the distance from the face to the point that reaches
// it at dt/2 (the interface value of Eq. 15), for any speed w: the flow
// speed (the upwind estimates "u" of Eq. 45) or an Alfven characteristic
// speed (the foot values of Eqs. 41-44).  The two slopes are formed once
// and serve every speed.  Along an absent direction the value is q itself.
template <typename T>
struct MhLine {
    T qm, q0, sm, s0, wm, w0;   // cells n - 1 and n: values, slopes, widths
    __device__ __forceinline__ T at(T w, T dt) const
    {
        return w >= T(0) ? qm + T(0.5) * sm * (wm - w * dt) : q0 - T(0.5) * s0 * (w0 + w * dt);
    }
};

// Line of q along e at the face of cell (i, j, k) (cell n); with `up` the
// face of the next cell along e as well (cells n .. n + 1), sharing the
// slope of cell n.
template <typename T>
__device__ __forceinline__ void mh_lines(const MeshD &m, const Tab<T> &tb, const T *q, int i, int j, int k, int e,
                                         MhLine<T> &L, MhLine<T> *up = nullptr)
{
    const idx_t c = IX(m, i, j, k);
    if (!mh_has(m, e)) {
        L = {q[c], q[c], T(0), T(0), T(0), T(0)};
        if (up) *up = L;
        return;
    }
    const int n = mh_pos(i, j, k, e);
    const T qm2 = q[mh_nb(m, i, j, k, e, -2)], qm1 = q[mh_nb(m, i, j, k, e, -1)], q0 = q[c],
            qp1 = q[mh_nb(m, i, j, k, e, 1)];
    const int nn = e == 0 ? 2 : n;   // X is uniform: any index serves
    const T im1 = mh_idc(tb, e, nn - 1), i0 = mh_idc(tb, e, nn), ip1 = mh_idc(tb, e, nn + 1);
    L.qm = qm1;
    L.q0 = q0;
    L.sm = vl_slope_i(qm2, qm1, q0, im1, i0);
    L.s0 = vl_slope_i(qm1, q0, qp1, i0, ip1);
    L.wm = mh_width(tb, e, nn - 1);
    L.w0 = mh_width(tb, e, nn);
    if (up) {
        const T qp2 = q[mh_nb(m, i, j, k, e, 2)];
        up->qm = q0;
        up->q0 = qp1;
        up->sm = L.s0;
        up->s0 = vl_slope_i(q0, qp1, qp2, ip1, mh_idc(tb, e, nn + 2));
        up->wm = L.w0;
        up->w0 = mh_width(tb, e, nn + 1);
    }
}

// Density at the edge at the lower a- and b-faces of cell (i, j, k): the
// mean of the four cells around it.
template <typename T>
__device__ __forceinline__ T mh_rho_edge(const MeshD &m, const T *rho, int i, int j, int k, int a, int b)
{
    const idx_t c00 = IX(m, i, j, k), c10 = mh_nb(m, i, j, k, a, -1), c01 = mh_nb(m, i, j, k, b, -1);
    int ia = i, ja = j, ka = k;
    mh_shift(m, ia, ja, ka, a, -1);
    const idx_t c11 = mh_nb(m, ia, ja, ka, b, -1);
    return T(0.25) * (rho[c00] + rho[c10] + rho[c01] + rho[c11]);
}

// Star values at an edge of the pair (v_p, B_p) from the 1.5D problem along
// the lines' direction (Eqs. 41-44): psi+- = v_p +- B_p / sqrt(rho), carried
// at C+- = U -+ W / sqrt(rho), taken at their feet.
template <typename T>
__device__ __forceinline__ void mh_star(const MhLine<T> &Lv, const MhLine<T> &Lb, T U, T W, T sq, T isq, T dt,
                                        T &vs, T &bs)
{
    const T cp = U - W * isq, cm = U + W * isq;
    const T vp = Lv.at(cp, dt), bp = Lb.at(cp, dt), vm = Lv.at(cm, dt), bm = Lb.at(cm, dt);
    vs = T(0.5) * (vp + vm + (bp - bm) * isq);
    bs = T(0.5) * (bp + bm + sq * (vp - vm));
}

// Faces of component a that the sub-steps update: every azimuth, the
// active rows and planes, along a its interior faces (from jf / kf).
__device__ __forceinline__ bool mh_face(const MeshD &m, int a, int j, int k)
{
    const bool y = m.hasY ? (j >= (a == 1 ? m.jf : m.j0) && j < m.j1) : j == 0;
    const bool z = m.hasZ ? (k >= (a == 2 ? m.kf : m.k0) && k < m.k1) : k == 0;
    return y && z;
}

// Transverse magnetic pressure (B_b^2 + B_c^2) / 2 at the centre of (i, j, k)
// for the gradient along a.
template <typename T>
__device__ __forceinline__ T mh_pmag(const MeshD &m, const Tab<T> &tb, int i, int j, int k, int a)
{
    T pb = T(0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
        if (b == a) continue;
        const T *B = tb.bfield[b];
        const T bc = T(0.5) * (B[IX(m, i, j, k)] + B[mh_nb(m, i, j, k, b, 1)]);
        pb += T(0.5) * bc * bc;
    }
    return pb;
}

// Grid of the face kernels: every row and plane of the arrays.
template <typename T>
__global__ void __launch_bounds__(256) k_mhd_pressure(MeshD m, Tab<T> tb, Fld<T> f, const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const T dt = step_dt<T>(sc);
    if (i >= m.nx || !(dt > T(0))) return;
    T *V[3] = {f.vx, f.vy, f.vz};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (!mh_has(m, a) || !mh_face(m, a, j, k)) continue;
        const idx_t c = IX(m, i, j, k), cm = mh_nb(m, i, j, k, a, -1);
        int ia = i, ja = j, ka = k;
        mh_shift(m, ia, ja, ka, a, -1);
        const T g = (mh_pmag(m, tb, i, j, k, a) - mh_pmag(m, tb, ia, ja, ka, a)) *
                    mh_idc(tb, a, a == 0 ? 1 : mh_pos(i, j, k, a));
        V[a][c] = V[a][c] - dt * T(2) * g / (f.rho[c] + f.rho[cm]);
    }
}

// Cells 8a-8d in one pass: per cell, for each edge orientation O (a = O + 1,
// b = O + 2) the four lines (v_a, B_a along b; v_b, B_b along a) are formed
// once and serve the EMF of the edge (Eq. 45) and the tension stars of
// both faces that meet there (Eq. 47: face a across b, face b across a,
// each with the star of the next edge along its direction as well).  The
// tension terms of a face are summed over its two directions in ascending
// order; every velocity component comes from the values on entry (out of
// place).  emf / tension switch the two parts (the debug phases run one).
// Under orbital advection f holds the residual v_x (Sec. 3.6) and vxb the
// velocity the tension updates; otherwise vxb is null.
// (FP32: four blocks per SM at 64 registers, no spills; against three at 72
// the edge kernel went 0.59 -> 0.54 ms on the 256 x 128 x 128 box)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_mhd_edges(MeshD m, Tab<T> tb, Fld<T> f, Fld<T> out, T *ex, T *ey, T *ez,
                                                   const Scal *sc, int emf, int tension, const T *vxb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const T dt = step_dt<T>(sc);
    if (i >= m.nx || !(dt > T(0))) return;
    const T *V[3] = {f.vx, f.vy, f.vz};
    T *VO[3] = {out.vx, out.vy, out.vz};
    T *E[3] = {ex, ey, ez};
    const T *rho = f.rho;
    const idx_t c = IX(m, i, j, k);
    const bool edge = emf && (m.hasY ? (j >= 2 && j <= m.nyt - 2) : j == 0) &&
                      (m.hasZ ? (k >= 2 && k <= m.nzt - 2) : k == 0);
    bool face[3];
#pragma unroll
    for (int a = 0; a < 3; a++) face[a] = tension && mh_has(m, a) && mh_face(m, a, j, k);
    T term[3][3];   // term[a][b]: the tension on face a across direction b
#pragma unroll
    for (int O = 0; O < 3; O++) {
        const int a = (O + 1) % 3, b = (O + 2) % 3;
        term[a][b] = T(0);
        term[b][a] = T(0);
        const bool ta = face[a] && mh_has(m, b), tb2 = face[b] && mh_has(m, a);
        if (!edge && !ta && !tb2) continue;
        const T *va = V[a], *vb = V[b], *ba = tb.bfield[a], *bb = tb.bfield[b];
        const idx_t ca = mh_nb(m, i, j, k, a, -1), cb = mh_nb(m, i, j, k, b, -1);
        MhLine<T> Lva, Lba, Lvb, Lbb, Uva, Uba, Uvb, Ubb;
        mh_lines(m, tb, va, i, j, k, b, Lva, ta ? &Uva : nullptr);
        mh_lines(m, tb, ba, i, j, k, b, Lba, ta ? &Uba : nullptr);
        mh_lines(m, tb, vb, i, j, k, a, Lvb, tb2 ? &Uvb : nullptr);
        mh_lines(m, tb, bb, i, j, k, a, Lbb, tb2 ? &Ubb : nullptr);
        const T r = mh_rho_edge(m, rho, i, j, k, a, b);
        const T sq = sqrt(r), isq = div_fast(T(1), sq);
        T vs, lo, hi;
        if (edge) {
            const T ub = T(0.5) * (vb[c] + vb[ca]);
            const T ua = T(0.5) * (va[c] + va[cb]);
            const T vau = Lva.at(ub, dt), bau = Lba.at(ub, dt);
            const T vbu = Lvb.at(ua, dt), bbu = Lbb.at(ua, dt);
            T vas, bas, vbs, bbs;
            mh_star(Lva, Lba, vbu, bbu, sq, isq, dt, vas, bas);
            mh_star(Lvb, Lbb, vau, bau, sq, isq, dt, vbs, bbs);
            T e = T(0.5) * (vas * bbu + bbs * vau - vbs * bau - bas * vbu);
            if (m.eta > 0.0) {
                T cur = T(0);
                if (mh_has(m, a)) cur += (bb[c] - bb[ca]) * mh_idc(tb, a, a == 0 ? 1 : mh_pos(i, j, k, a));
                if (mh_has(m, b)) cur -= (ba[c] - ba[cb]) * mh_idc(tb, b, b == 0 ? 1 : mh_pos(i, j, k, b));
                e -= (T)m.eta * cur;
            }
            // on the edges in a wall's plane (a non-periodic Y or Z boundary)
            // the EMF vanishes: the flux through the wall and the net flux out
            // of every cell next to it are held
            const bool wy = O != 1 && m.hasY && !m.pery && (j == m.j0 || j == m.j1);
            const bool wz = O != 2 && m.hasZ && !m.perz && (k == m.k0 || k == m.k1);
            E[O][c] = wy || wz ? T(0) : e;
        }
        if (ta) {   // face a across b: stars of B_a at this edge and the next along b
            mh_star(Lva, Lba, T(0), T(0.5) * (bb[c] + bb[ca]), sq, isq, dt, vs, lo);
            int ib = i, jb = j, kb = k;
            mh_shift(m, ib, jb, kb, b, 1);
            const idx_t cn = IX(m, ib, jb, kb), cna = mh_nb(m, ib, jb, kb, a, -1);
            const T r1 = mh_rho_edge(m, rho, ib, jb, kb, a, b), s1 = sqrt(r1);
            mh_star(Uva, Uba, T(0), T(0.5) * (bb[cn] + bb[cna]), s1, div_fast(T(1), s1), dt, vs, hi);
            const T bbar = T(0.25) * (bb[c] + bb[cn] + bb[ca] + bb[cna]);
            term[a][b] = bbar * (hi - lo) / mh_width(tb, b, mh_pos(i, j, k, b));
        }
        if (tb2) {  // face b across a
            mh_star(Lvb, Lbb, T(0), T(0.5) * (ba[c] + ba[cb]), sq, isq, dt, vs, lo);
            int ia = i, ja = j, ka = k;
            mh_shift(m, ia, ja, ka, a, 1);
            const idx_t cn = IX(m, ia, ja, ka), cnb = mh_nb(m, ia, ja, ka, b, -1);
            const T r1 = mh_rho_edge(m, rho, ia, ja, ka, a, b), s1 = sqrt(r1);
            mh_star(Uvb, Ubb, T(0), T(0.5) * (ba[cn] + ba[cnb]), s1, div_fast(T(1), s1), dt, vs, hi);
            const T bbar = T(0.25) * (ba[c] + ba[cn] + ba[cb] + ba[cnb]);
            term[b][a] = bbar * (hi - lo) / mh_width(tb, a, mh_pos(i, j, k, a));
        }
    }
    if (!tension) return;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        // (under orbital advection f carries the residual v_x; vxb the velocity itself)
        T v = a == 0 && vxb ? vxb[c] : V[a][c];
        if (face[a]) {
            T fa = T(0);
#pragma unroll
            for (int b = 0; b < 3; b++)
                if (b != a && mh_has(m, b)) fa += term[a][b];
            v = v + dt * T(2) / (rho[c] + rho[mh_nb(m, i, j, k, a, -1)]) * fa;
        }
        VO[a][c] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mhd_ct(MeshD m, Tab<T> tb, const T *ex, const T *ey, const T *ez,
                                                const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const T dt = step_dt<T>(sc);
    if (i >= m.nx || !(dt > T(0))) return;
    const T *E[3] = {ex, ey, ez};
    const idx_t c = IX(m, i, j, k);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (!mh_face(m, a, j, k)) continue;
        const int b = (a + 1) % 3, o = (a + 2) % 3;
        T d = T(0);
        if (mh_has(m, b)) d += (E[o][mh_nb(m, i, j, k, b, 1)] - E[o][c]) / mh_width(tb, b, mh_pos(i, j, k, b));
        if (mh_has(m, o)) d -= (E[b][mh_nb(m, i, j, k, o, 1)] - E[b][c]) / mh_width(tb, o, mh_pos(i, j, k, o));
        T *B = tb.bfield[a];
        B[c] = B[c] + dt * d;
    }
}

// ---------------------------------------------------------------------------
// Orbital advection of the field (Sec. 3.6).
// ---------------------------------------------------------------------------

// Eq. 37 on every ring, ghost rings included (cell 3): the ring velocities
// whose residual the MHD sub-steps see.  One warp per ring; exact maximum
// and minimum, so the active rings get the v0 of the X sweep.
template <typename T>
__global__ void __launch_bounds__(256) k_mhd_v0all(MeshD m, const T *vx, double *v0all)
{
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = (int)(threadIdx.x & 31);
    if (w >= m.nyt * m.nzt) return;   // (warp-uniform)
    const T *row = vx + IX(m, 0, w % m.nyt, w / m.nyt);
    T mx = row[0], mn = row[0];
    for (int i = lane; i < m.nx; i += 32) {
        mx = row[i] > mx ? row[i] : mx;
        mn = row[i] < mn ? row[i] : mn;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const T a = __shfl_xor_sync(0xffffffffu, mx, o), b = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = a > mx ? a : mx;
        mn = b < mn ? b : mn;
    }
    if (lane == 0) v0all[w] = 0.5 * ((double)mx + (double)mn);
}

// The residual azimuthal velocity v_x - v0 of every cell's ring (cells 8a-8d
// under orbital advection), rounded once.
template <typename T>
__global__ void __launch_bounds__(256) k_mhd_dvx(MeshD m, const T *vx, const double *v0all, T *dvx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= m.nx || j >= m.nyt || k >= m.nzt) return;
    const idx_t c = IX(m, i, j, k);
    dvx[c] = (T)((double)vx[c] - v0all[k * m.nyt + j]);
}

// The arc of one ring row: X = v0f dt / dX = N + xi (N the nearest integer,
// FP64), N modulo the ring, and whether the row takes part.  An arc beyond 16
// turns of the ring, or not finite, records FARGO_ERR_NONFINITE and the row
// takes no part.
struct OrbArc {
    long long N;
    int Nm, on;
    double xs;
};
__device__ __forceinline__ OrbArc mh_orbital_arc(const MeshD &m, double v0f, double dt, Scal *sc)
{
    OrbArc a{0, 0, 0, 0.0};
    const double X = __ddiv_rn(__dmul_rn(v0f, dt), m.dx);
    if (!(fabs(X) <= 16.0 * m.nx)) {
        atomicOr(&sc->err, 1);
        return a;
    }
    a.N = llround(X);
    a.xs = __dsub_rn(X, (double)a.N);
    a.Nm = (int)(((a.N % m.nx) + m.nx) % m.nx);
    a.on = 1;
    return a;
}

// Upstream average of the orbital EMF at the edge at the lower X face of
// cell i, for the ring row of B (B_y at a Y face, or B_z at a Z face) and
// the row's arc (Eq. 54): (1/dt) times the integral of B over the arc, i.e.
// (dX/dt) (sum of the N whole cells upstream + xi times the PPA face value N
// cells upstream).
template <typename T>
__device__ __forceinline__ T mh_orbital_emf(const MeshD &m, const T *row, int i, const OrbArc &a, double dt)
{
    const int nx = m.nx;
    const long long N = a.N;
    T w = T(0);
    if (N > 0) {
        int q = i;
        for (long long n = 0; n < N; n++) {   // cells i-1, i-2, ... (the order of the sum)
            q = q == 0 ? nx - 1 : q - 1;
            w += row[q];
        }
    } else {
        int q = i;
        for (long long n = 0; n < -N; n++) {  // cells i, i+1, ...
            w -= row[q];
            q = q + 1 == nx ? 0 : q + 1;
        }
    }
    T st = T(0);
    if (a.xs != 0.0) {
        int f = i - a.Nm;
        if (f < 0) f += nx;
        const bool pos = a.xs >= 0.0;
        const int d = pos ? f - 1 : f;   // the donor cell of face f, -1 .. nx-1
        T q5[5];
#pragma unroll
        for (int s = 0; s < 5; s++) {
            int q = d - 2 + s;           // -3 .. nx+1
            while (q < 0) q += nx;       // (at most three turns, for rings of one cell)
            while (q >= nx) q -= nx;
            q5[s] = row[q];
        }
        st = ppa_face(q5, (T)(pos ? a.xs : -a.xs), pos);
    }
    return (T)(m.dx / dt) * (w + (T)a.xs * st);
}

// Cell 11: e_z = v0 B_y and e_y = -v0 B_z averaged upstream on every edge
// (e_x = 0), v0 the two-point mean of the rings across the face carrying
// B_y (B_z), or the ring's own along an absent direction; zero on the edges
// in a wall's plane (non-periodic Y or Z) and off the active range.  The
// constrained transport k_mhd_ct then applies them.  Grid: every row and
// plane of the arrays (the face kernels' grid); a block's threads share one
// row (j, k), whose two arcs thread 0 forms once in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_mhd_fargo_emf(MeshD m, Tab<T> tb, const double *v0all, T *ex, T *ey,
                                                       T *ez, Scal *sc)
{
    __shared__ OrbArc arc[2];   // e_z's row, e_y's row
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const double dt = sc->dt;
    if (threadIdx.x == 0) {
        arc[0] = OrbArc{0, 0, 0, 0.0};
        arc[1] = OrbArc{0, 0, 0, 0.0};
        if (dt > 0.0 && j <= m.nyt && k <= m.nzt) {
            // e_z: Y-face rows j0..j1 (walls excluded), active planes
            const bool jz = m.hasY ? (j >= m.j0 && j <= m.j1 && (m.pery || (j != m.j0 && j != m.j1))) : j == 0;
            const bool kz = m.hasZ ? (k >= m.k0 && k < m.k1) : k == 0;
            if (jz && kz) {
                const int r = k * m.nyt + j;
                arc[0] = mh_orbital_arc(m, m.hasY ? 0.5 * (v0all[r - 1] + v0all[r]) : v0all[r], dt, sc);
            }
            // e_y: active rows, Z-face planes k0..k1 (walls excluded)
            const bool jy = m.hasY ? (j >= m.j0 && j < m.j1) : j == 0;
            const bool ky = m.hasZ ? (k >= m.k0 && k <= m.k1 && (m.perz || (k != m.k0 && k != m.k1))) : k == 0;
            if (jy && ky) {
                const int r = k * m.nyt + j;
                arc[1] = mh_orbital_arc(m, m.hasZ ? 0.5 * (v0all[r - m.nyt] + v0all[r]) : v0all[r], dt, sc);
            }
        }
    }
    __syncthreads();
    if (i >= m.nx || j > m.nyt || k > m.nzt) return;
    const idx_t c = IX(m, i, j, k);
    const OrbArc az = arc[0], ay = arc[1];
    ex[c] = T(0);
    ey[c] = ay.on ? -mh_orbital_emf(m, tb.bfield[2] + IX(m, 0, j, k), i, ay, dt) : T(0);
    ez[c] = az.on ? mh_orbital_emf(m, tb.bfield[1] + IX(m, 0, j, k), i, az, dt) : T(0);
}

// Periodic images of the field (periodic Y / Z axes): B_y face-centred
// along Y, B_z along Z.
template <typename T>
static PerSet<T> per_field(const MeshD &m, const Tab<T> &tb)
{
    PerSet<T> p{};
    for (int d = 0; d < 3; d++) {
        p.dst[d] = tb.bfield[d];
        p.src[d] = tb.bfield[d];
        p.fy[d] = (unsigned char)(d == 1 && m.hasY);
        p.fz[d] = (unsigned char)(d == 2 && m.hasZ);
    }
    p.n = 3;
    return p;
}

}  // namespace fk
