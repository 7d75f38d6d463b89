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

// (i, j, k) moved by off cells along d (X periodic; no move along an absent
// direction).
__device__ __forceinline__ void mh_shift(const MeshD &m, int &i, int &j, int &k, int d, int off)
{
    if (d == 0) {
        i = (i + off) % m.nx;
        if (i < 0) i += m.nx;
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

// Width of cell n along d, and the distance between the centres of cells
// n - 1 and n (X uniform).
template <typename T>
__device__ __forceinline__ T mh_width(const Tab<T> &tb, int d, int n)
{
    return d == 0 ? tb.dx : (d == 1 ? tb.dy[n] : tb.dz[n]);
}
template <typename T>
__device__ __forceinline__ T mh_dc(const Tab<T> &tb, int d, int n)
{
    return d == 0 ? tb.dx : T(0.5) * (mh_width(tb, d, n - 1) + mh_width(tb, d, n));
}

// Value at the face between cells n - 1 and n along e (cell (i, j, k) is n)
// of a quantity q cell centred along e, carried at speed w over dt: the
// upwind cell's value plus its van Leer slope times half the distance from
// the face to the point that reaches it at dt/2 (the interface value of
// Eq. 15), with w the flow speed (the upwind estimates "u") or an Alfven
// characteristic speed (the foot values of Eqs. 41-44).
template <typename T>
__device__ __forceinline__ T mh_recon(const MeshD &m, const Tab<T> &tb, const T *q, int i, int j, int k, int e, T w,
                                      T dt)
{
    const idx_t c = IX(m, i, j, k);
    if (!mh_has(m, e)) return q[c];
    const int n = e == 0 ? 2 : mh_pos(i, j, k, e);   // X is uniform: any index serves
    if (w >= T(0)) {
        const T qm1 = q[mh_nb(m, i, j, k, e, -1)];
        const T sl = vl_slope(q[mh_nb(m, i, j, k, e, -2)], qm1, q[c], mh_dc(tb, e, n - 1), mh_dc(tb, e, n));
        return qm1 + T(0.5) * sl * (mh_width(tb, e, n - 1) - w * dt);
    }
    const T q0 = q[c];
    const T sl = vl_slope(q[mh_nb(m, i, j, k, e, -1)], q0, q[mh_nb(m, i, j, k, e, 1)], mh_dc(tb, e, n),
                          mh_dc(tb, e, n + 1));
    return q0 - T(0.5) * sl * (mh_width(tb, e, n) + w * dt);
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

// Star values at that edge of the pair (v_p, B_p) from the 1.5D problem
// along q (Eqs. 41-44): psi+- = v_p +- B_p / sqrt(rho), carried at
// C+- = U -+ W / sqrt(rho), taken at their feet.
template <typename T>
__device__ __forceinline__ void mh_star(const MeshD &m, const Tab<T> &tb, const T *v, const T *bf, int i, int j, int k,
                                        int q, T U, T W, T rho, T dt, T &vs, T &bs)
{
    const T sq = sqrt(rho);
    const T cp = U - W / sq, cm = U + W / sq;
    const T vp = mh_recon(m, tb, v, i, j, k, q, cp, dt), bp = mh_recon(m, tb, bf, i, j, k, q, cp, dt);
    const T vm = mh_recon(m, tb, v, i, j, k, q, cm, dt), bm = mh_recon(m, tb, bf, i, j, k, q, cm, dt);
    vs = T(0.5) * (vp + vm + (bp - bm) / sq);
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
    const T ub = T(0.5) * (vb[c00] + vb[ca]);
    const T ua = T(0.5) * (va[c00] + va[cb]);
    const T vau = mh_recon(m, tb, va, i, j, k, b, ub, dt), bau = mh_recon(m, tb, ba, i, j, k, b, ub, dt);
    const T vbu = mh_recon(m, tb, vb, i, j, k, a, ua, dt), bbu = mh_recon(m, tb, bb, i, j, k, a, ua, dt);
    T vas, bas, vbs, bbs;
    mh_star(m, tb, va, ba, i, j, k, b, vbu, bbu, r, dt, vas, bas);
    mh_star(m, tb, vb, bb, i, j, k, a, vau, bau, r, dt, vbs, bbs);
    T e = T(0.5) * (vas * bbu + bbs * vau - vbs * bau - bas * vbu);
    if (m.eta > 0.0) {
        T cur = T(0);
        if (mh_has(m, a)) cur += (bb[c00] - bb[ca]) / mh_dc(tb, a, a == 0 ? 1 : mh_pos(i, j, k, a));
        if (mh_has(m, b)) cur -= (ba[c00] - ba[cb]) / mh_dc(tb, b, b == 0 ? 1 : mh_pos(i, j, k, b));
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
        const T g = (mh_pmag(m, tb, i, j, k, a) - mh_pmag(m, tb, ia, ja, ka, a)) /
                    mh_dc(tb, a, a == 0 ? 1 : mh_pos(i, j, k, a));
        V[a][c] = V[a][c] - dt * T(2) * g / (f.rho[c] + f.rho[cm]);
    }
}

// B_a* at the edge of cell (i, j, k) at its lower a- and b-faces, from the
// problem along b with no flow speed and W the mean of the edge's two
// b-faces (Eq. 47).
template <typename T>
__device__ __forceinline__ T mh_tension_star(const MeshD &m, const Tab<T> &tb, const T *va, const T *ba, const T *bb,
                                             const T *rho, int i, int j, int k, int a, int b, T dt)
{
    const T r = mh_rho_edge(m, rho, i, j, k, a, b);
    const T W = T(0.5) * (bb[IX(m, i, j, k)] + bb[mh_nb(m, i, j, k, a, -1)]);
    T vs, bs;
    mh_star(m, tb, va, ba, i, j, k, b, T(0), W, r, dt, vs, bs);
    return bs;
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
                int ib = i, jb = j, kb = k;
                mh_shift(m, ib, jb, kb, b, 1);
                const T up = mh_tension_star(m, tb, V[a], tb.bfield[a], bb, f.rho, ib, jb, kb, a, b, dt);
                const T lo = mh_tension_star(m, tb, V[a], tb.bfield[a], bb, f.rho, i, j, k, a, b, dt);
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
