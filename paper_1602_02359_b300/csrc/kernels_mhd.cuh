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
//   k_mhd_emf (cells 8a-8c): the three EMFs of every edge (Eq. 45, with the
//     star values of Eqs. 41-44), minus eta curl B;
//   k_mhd_tension (cell 8d): the magnetic tension of Eq. 47 on every
//     interior face velocity, out of place (every component from the
//     velocities on entry);
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

// EMF of orientation O at the edge of cell (i, j, k) (Eq. 45):
//   e_O = (v_a* B_b^u + B_b* v_a^u - v_b* B_a^u - B_a* v_b^u) / 2,
// v_a^u, B_a^u upwind along b at the mean flow speed along b of the edge's
// two b-faces, (v_a*, B_a*) from the problem along b at C+- = v_b^u -+
// B_b^u / sqrt(rho) (and a, b swapped); then the resistive part
// -eta (curl B)_O, each derivative the difference of the two face values
// across the edge over their centre-to-centre distance.
template <typename T, int O>
__device__ __forceinline__ T mh_emf_edge(const MeshD &m, const Tab<T> &tb, const T *va, const T *vb, const T *ba,
                                         const T *bb, const T *rho, int i, int j, int k, T dt)
{
    constexpr int a = (O + 1) % 3, b = (O + 2) % 3;
    const idx_t c00 = IX(m, i, j, k), ca = mh_nb(m, i, j, k, a, -1), cb = mh_nb(m, i, j, k, b, -1);
    const T r = mh_rho_edge(m, rho, i, j, k, a, b);
    const T sq = sqrt(r), isq = div_fast(T(1), sq);
    const T ub = T(0.5) * (vb[c00] + vb[ca]);
    const T ua = T(0.5) * (va[c00] + va[cb]);
    MhLine<T> Lva, Lba, Lvb, Lbb;
    mh_lines(m, tb, va, i, j, k, b, Lva);
    mh_lines(m, tb, ba, i, j, k, b, Lba);
    mh_lines(m, tb, vb, i, j, k, a, Lvb);
    mh_lines(m, tb, bb, i, j, k, a, Lbb);
    const T vau = Lva.at(ub, dt), bau = Lba.at(ub, dt);
    const T vbu = Lvb.at(ua, dt), bbu = Lbb.at(ua, dt);
    T vas, bas, vbs, bbs;
    mh_star(Lva, Lba, vbu, bbu, sq, isq, dt, vas, bas);
    mh_star(Lvb, Lbb, vau, bau, sq, isq, dt, vbs, bbs);
    T e = T(0.5) * (vas * bbu + bbs * vau - vbs * bau - bas * vbu);
    if (m.eta > 0.0) {
        T cur = T(0);
        if (mh_has(m, a)) cur += (bb[c00] - bb[ca]) * mh_idc(tb, a, a == 0 ? 1 : mh_pos(i, j, k, a));
        if (mh_has(m, b)) cur -= (ba[c00] - ba[cb]) * mh_idc(tb, b, b == 0 ? 1 : mh_pos(i, j, k, b));
        e -= (T)m.eta * cur;
    }
    return e;
}

// Faces of component a that the sub-steps update: every azimuth, the
// active rows and planes, along a its interior faces (from jf / kf).
__device__ __forceinline__ bool mh_face(const MeshD &m, int a, int j, int k)
{
    const bool y = m.hasY ? (j >= (a == 1 ? m.jf : m.j0) && j < m.j1) : j == 0;
    const bool z = m.hasZ ? (k >= (a == 2 ? m.kf : m.k0) && k < m.k1) : k == 0;
    return y && z;
}

// Launch shapes: one thread per azimuth, one block row per (j, k).
// Edges: rows and planes 2 .. n - 2 of a present direction (the stencil
// reaches two cells down and one up), the single one of an absent one.
__host__ __device__ __forceinline__ int mh_edge_rows(const MeshD &m) { return m.hasY ? m.nyt - 3 : 1; }
__host__ __device__ __forceinline__ int mh_edge_planes(const MeshD &m) { return m.hasZ ? m.nzt - 3 : 1; }

template <typename T>
__global__ void __launch_bounds__(256) k_mhd_emf(MeshD m, Tab<T> tb, Fld<T> f, T *ex, T *ey, T *ez, const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y + (m.hasY ? 2 : 0), k = blockIdx.z + (m.hasZ ? 2 : 0);
    const T dt = step_dt<T>(sc);
    if (i >= m.nx || !(dt > T(0))) return;
    const idx_t c = IX(m, i, j, k);
    const T *bx = tb.bfield[0], *by = tb.bfield[1], *bz = tb.bfield[2];
    ex[c] = mh_emf_edge<T, 0>(m, tb, f.vy, f.vz, by, bz, f.rho, i, j, k, dt);
    ey[c] = mh_emf_edge<T, 1>(m, tb, f.vz, f.vx, bz, bx, f.rho, i, j, k, dt);
    ez[c] = mh_emf_edge<T, 2>(m, tb, f.vx, f.vy, bx, by, f.rho, i, j, k, dt);
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

// B_a* at the edges of cell (i, j, k) and of the next cell along b, at
// their lower a- and b-faces, from the problem along b with no flow speed
// and W the mean of each edge's two b-faces (Eq. 47).
template <typename T>
__device__ __forceinline__ void mh_tension_stars(const MeshD &m, const Tab<T> &tb, const T *va, const T *ba,
                                                 const T *bb, const T *rho, int i, int j, int k, int a, int b, T dt,
                                                 T &lo, T &hi)
{
    MhLine<T> Lv, Lb, Lv1, Lb1;
    mh_lines(m, tb, va, i, j, k, b, Lv, &Lv1);
    mh_lines(m, tb, ba, i, j, k, b, Lb, &Lb1);
    int ib = i, jb = j, kb = k;
    mh_shift(m, ib, jb, kb, b, 1);
    T vs;
    {
        const T r = mh_rho_edge(m, rho, i, j, k, a, b), sq = sqrt(r);
        const T W = T(0.5) * (bb[IX(m, i, j, k)] + bb[mh_nb(m, i, j, k, a, -1)]);
        mh_star(Lv, Lb, T(0), W, sq, div_fast(T(1), sq), dt, vs, lo);
    }
    {
        const T r = mh_rho_edge(m, rho, ib, jb, kb, a, b), sq = sqrt(r);
        const T W = T(0.5) * (bb[IX(m, ib, jb, kb)] + bb[mh_nb(m, ib, jb, kb, a, -1)]);
        mh_star(Lv1, Lb1, T(0), W, sq, div_fast(T(1), sq), dt, vs, hi);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mhd_tension(MeshD m, Tab<T> tb, Fld<T> f, Fld<T> out, const Scal *sc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    const T dt = step_dt<T>(sc);
    if (i >= m.nx || !(dt > T(0))) return;
    const T *V[3] = {f.vx, f.vy, f.vz};
    T *VO[3] = {out.vx, out.vy, out.vz};
    const idx_t c = IX(m, i, j, k);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T v = V[a][c];
        if (mh_has(m, a) && mh_face(m, a, j, k)) {
            const idx_t cm = mh_nb(m, i, j, k, a, -1);
            int ia = i, ja = j, ka = k;
            mh_shift(m, ia, ja, ka, a, -1);
            T fa = T(0);
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (b == a || !mh_has(m, b)) continue;
                const T *bb = tb.bfield[b];
                const T bbar = T(0.25) * (bb[c] + bb[mh_nb(m, i, j, k, b, 1)] + bb[cm] + bb[mh_nb(m, ia, ja, ka, b, 1)]);
                T lo, up;
                mh_tension_stars(m, tb, V[a], tb.bfield[a], bb, f.rho, i, j, k, a, b, dt, lo, up);
                fa += bbar * (up - lo) / mh_width(tb, b, mh_pos(i, j, k, b));
            }
            v = v + dt * T(2) / (f.rho[c] + f.rho[cm]) * fa;
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
