// Ghost fill (flow-chart cells 2 and 9) and the Courant reduction (cells 3-6).
#pragma once
#include "fargo_internal.cuh"

namespace fk {

// ---------------------------------------------------------------------------
// Ghost fill.  Reflecting walls mirror scalars and tangential velocities and
// set the wall-normal face velocity to zero with odd mirroring beyond; frozen
// ghosts keep their values; zero gradient copies the last active cell (and
// the first interior normal face).  One thread per (i, transverse index,
// side).  mode 0 = cell 2 (skipped once the run is done or failed),
// mode 1 = cell 9 (skipped when the current step is void).
// ---------------------------------------------------------------------------
//
// `ref` (v_x in the reference form of FP32, else null) is the reference
// velocity of the ring at line position p, ref[p * rs]: a value copied from
// position s to position d keeps its v_x, so its stored value gains
// ref[s] - ref[d].  Periodic rings share their images' references.
template <typename T>
__device__ __forceinline__ T ref_shift(const T *ref, int rs, int s, int d)
{
    return ref ? ref[s * rs] - ref[d * rs] : T(0);
}
template <typename T>
__device__ void fill_line(T *a, idx_t base, idx_t stride, int lo, int hi, int g, int normal, int side,
                          int bc, const T *ref = nullptr, int rs = 0)
{
    if (bc == BC_FROZEN) return;
    if (bc == BC_PERIODIC) {
        // ghosts hold the values one period away; the upper normal face hi is face lo
        const int n = hi - lo;
        if (side == 0)
            for (int mm = 1; mm <= g; mm++) a[base + (lo - mm) * stride] = a[base + (lo - mm + n) * stride];
        else
            for (int mm = 0; mm < g + (normal ? 1 : 0); mm++) a[base + (hi + mm) * stride] = a[base + (lo + mm) * stride];
        return;
    }
    if (!normal) {
        for (int mm = 0; mm < g; mm++) {
            int dst = side == 0 ? lo - 1 - mm : hi + mm;
            int src = bc == BC_REFLECT ? (side == 0 ? lo + mm : hi - 1 - mm) : (side == 0 ? lo : hi - 1);
            if (ref) a[base + dst * stride] = a[base + src * stride] + ref_shift(ref, rs, src, dst);
            else a[base + dst * stride] = a[base + src * stride];
        }
    } else if (bc == BC_REFLECT) {
        int w = side == 0 ? lo : hi;
        a[base + w * stride] = T(0);
        for (int mm = 1; mm <= g; mm++) {
            if (side == 0) a[base + (w - mm) * stride] = -a[base + (w + mm) * stride];
            else a[base + (w + mm) * stride] = -a[base + (w - mm) * stride];
        }
    } else {
        if (side == 0) {
            T v = a[base + (lo + 1) * stride];
            for (int mm = 0; mm <= g; mm++) a[base + (lo - mm) * stride] = v;
        } else {
            T v = a[base + (hi - 1) * stride];
            for (int mm = 0; mm <= g; mm++) a[base + (hi + mm) * stride] = v;
        }
    }
}

// Ghosts of one magnetic-field component (MHD) along one line across a Y
// or Z boundary.  A wall's own face of the normal component is never
// written: the constrained transport holds the flux through it (the EMFs
// tangential to a wall vanish there).  Reflecting wall: every component
// mirrored evenly about the wall; zero gradient: the ghosts take the wall
// face's value (normal) or the last active cell's (tangential); frozen:
// kept; periodic: the images one period away.
template <typename T>
__device__ void fill_bline(T *a, idx_t base, idx_t stride, int lo, int hi, int g, int normal, int side, int bc)
{
    if (bc == BC_FROZEN) return;
    if (bc == BC_PERIODIC) {
        fill_line(a, base, stride, lo, hi, g, normal, side, bc);
        return;
    }
    for (int mm = 1; mm <= g; mm++) {
        int dst, src;
        if (normal) {
            dst = side == 0 ? lo - mm : hi + mm;
            src = bc == BC_REFLECT ? (side == 0 ? lo + mm : hi - mm) : (side == 0 ? lo : hi);
        } else {
            dst = side == 0 ? lo - mm : hi - 1 + mm;
            src = bc == BC_REFLECT ? (side == 0 ? lo + mm - 1 : hi - mm) : (side == 0 ? lo : hi - 1);
        }
        a[base + dst * stride] = a[base + src * stride];
    }
}

__device__ __forceinline__ bool bc_skip(const Scal *sc, int mode)
{
    if (mode == 0) return sc->err != 0 || (!sc->fixed && sc->t >= sc->t_end);
    return !(sc->dt > 0.0);
}

// The magnetic field (MagF, MHD) is filled by fill_bline, component d
// staggered like v_d, along every present axis: B_z, B_y stay transverse
// fields of a mesh without Z or Y, where v_z, v_y are unused.
template <typename T>
__device__ __forceinline__ void bc_y_body(const MeshD &m, const Fld<T> &f, const Scal *sc, int mode, long long tid,
                                          const T *vref = nullptr, MagF<T> mb = MagF<T>{})
{
    long long n = (long long)m.nx * (m.nzt + 1) * 2;
    if (tid >= n || bc_skip(sc, mode)) return;
    int i = (int)(tid % m.nx);
    long long r = tid / m.nx;
    int k = (int)(r % (m.nzt + 1));
    int side = (int)(r / (m.nzt + 1));
    int bc = m.bcy[side];
    T *fl[5] = {f.rho, m.iso ? nullptr : f.e, f.vx, f.vy, f.vz};
    for (int q = 0; q < 5; q++) {
        if (!fl[q]) continue;
        if (q == 4 && !m.hasZ) continue;
        int kmax = q == 4 ? m.nzt + 1 : m.nzt;
        if (k >= kmax) continue;
        fill_line(fl[q], k * m.sk + i, m.sj, m.j0, m.j1, m.g, q == 3, side, bc,
                  q == 2 && vref ? vref + k * m.nyt : (const T *)nullptr, 1);
    }
    if (mb.b[0])
        for (int d = 0; d < 3; d++) {
            if (k >= (d == 2 ? m.nzt + 1 : m.nzt)) continue;
            fill_bline(mb.b[d], k * m.sk + i, m.sj, m.j0, m.j1, m.g, d == 1, side, bc);
        }
}

template <typename T>
__device__ __forceinline__ void bc_z_body(const MeshD &m, const Fld<T> &f, const Scal *sc, int mode, long long tid,
                                          const T *vref = nullptr, MagF<T> mb = MagF<T>{})
{
    long long n = (long long)m.nx * (m.nyt + 1) * 2;
    if (tid >= n || bc_skip(sc, mode)) return;
    int i = (int)(tid % m.nx);
    long long r = tid / m.nx;
    int j = (int)(r % (m.nyt + 1));
    int side = (int)(r / (m.nyt + 1));
    int bc = m.bcz[side];
    T *fl[5] = {f.rho, m.iso ? nullptr : f.e, f.vx, f.vy, f.vz};
    for (int q = 0; q < 5; q++) {
        if (!fl[q]) continue;
        if (q == 3 && !m.hasY) continue;
        int jmax = q == 3 ? m.nyt + 1 : m.nyt;
        if (j >= jmax) continue;
        fill_line(fl[q], j * m.sj + i, m.sk, m.k0, m.k1, m.g, q == 4, side, bc,
                  q == 2 && vref ? vref + j : (const T *)nullptr, m.nyt);
    }
    if (mb.b[0])
        for (int d = 0; d < 3; d++) {
            if (j >= (d == 1 ? m.nyt + 1 : m.nyt)) continue;
            fill_bline(mb.b[d], j * m.sj + i, m.sk, m.k0, m.k1, m.g, d == 2, side, bc);
        }
}

// ---------------------------------------------------------------------------
// Periodic images between the sub-steps: on a periodic axis every value read
// across the boundary is the value one period away, so after a sub-step or a
// sweep changes values next to the boundary, the ghosts that mirror them are
// rewritten (the fills of cells 2 and 9 cover the other boundaries).  Up to
// eight arrays, each with its own source (dst ghosts <- src active values,
// the same array or the one a later kernel reads its ghosts from) and its
// staggering (face-centred along Y for v_y, along Z for v_z).  One thread per
// (azimuth, transverse index, side, array); Y before Z, so that the Z
// images copy rows whose Y ghosts are already filled.  Skipped on void steps.
// ---------------------------------------------------------------------------
template <typename T>
struct PerSet {
    T *dst[8];
    const T *src[8];
    unsigned char fy[8], fz[8];   // face-centred along Y / along Z
    int n;
};

template <typename T>
__global__ void k_periodic(MeshD m, PerSet<T> p, const Scal *sc, int axis)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ntr = axis == 1 ? m.nzt + 1 : m.nyt + 1;
    const long long n = (long long)m.nx * ntr * 2 * p.n;
    if (tid >= n || !(sc->dt > 0.0)) return;
    const int i = (int)(tid % m.nx);
    long long r = tid / m.nx;
    const int t = (int)(r % ntr);
    r /= ntr;
    const int side = (int)(r % 2), a = (int)(r / 2);
    T *dst = p.dst[a];
    const T *src = p.src[a];
    if (axis == 1) {
        if (t >= (p.fz[a] ? m.nzt + 1 : m.nzt)) return;
        const idx_t base = t * m.sk + i;
        const int lo = m.j0, hi = m.j1, len = hi - lo;
        if (side == 0)
            for (int mm = 1; mm <= m.g; mm++) dst[base + (lo - mm) * m.sj] = src[base + (lo - mm + len) * m.sj];
        else
            for (int mm = 0; mm < m.g + p.fy[a]; mm++) dst[base + (hi + mm) * m.sj] = src[base + (lo + mm) * m.sj];
    } else {
        if (t >= (p.fy[a] ? m.nyt + 1 : m.nyt)) return;
        const idx_t base = t * m.sj + i;
        const int lo = m.k0, hi = m.k1, len = hi - lo;
        if (side == 0)
            for (int mm = 1; mm <= m.g; mm++) dst[base + (lo - mm) * m.sk] = src[base + (lo - mm + len) * m.sk];
        else
            for (int mm = 0; mm < m.g + p.fz[a]; mm++) dst[base + (hi + mm) * m.sk] = src[base + (lo + mm) * m.sk];
    }
}

// Queue the images of p on the periodic axes among `axes` (bit 0 = Y, bit 1 = Z).
template <typename T>
static int launch_periodic(const MeshD &m, const PerSet<T> &p, const Scal *sc, cudaStream_t s, int axes = 3)
{
    int nl = 0;
    if ((axes & 1) && m.pery) {
        const long long n = (long long)m.nx * (m.nzt + 1) * 2 * p.n;
        k_periodic<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, p, sc, 1);
        nl++;
    }
    if ((axes & 2) && m.perz) {
        const long long n = (long long)m.nx * (m.nyt + 1) * 2 * p.n;
        k_periodic<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, p, sc, 2);
        nl++;
    }
    return nl;
}

// Image sets of the common cases: the velocities (and e) of a field set, a
// quantity set (every member cell-centred), the diagonal viscous stresses.
template <typename T>
static PerSet<T> per_fields(const MeshD &m, const Fld<T> &f, bool vel, bool energy)
{
    PerSet<T> p{};
    auto add = [&](T *a, int fy, int fz) {
        p.dst[p.n] = a;
        p.src[p.n] = a;
        p.fy[p.n] = (unsigned char)fy;
        p.fz[p.n] = (unsigned char)fz;
        p.n++;
    };
    if (vel) {
        add(f.vx, 0, 0);
        if (m.hasY) add(f.vy, 1, 0);
        if (m.hasZ) add(f.vz, 0, 1);
    }
    if (energy && !m.iso) add(f.e, 0, 0);
    return p;
}
template <typename T>
static PerSet<T> per_quantities(const QSet<T> &dst, const QSet<T> &src)
{
    PerSet<T> p{};
    for (int q = 0; q < dst.nq; q++) {
        p.dst[q] = dst.q[q];
        p.src[q] = src.q[q];
    }
    p.n = dst.nq;
    return p;
}

template <typename T>
__global__ void k_bc_y(MeshD m, Fld<T> f, const Scal *sc, int mode, const T *vref, MagF<T> mb)
{
    bc_y_body(m, f, sc, mode, (long long)blockIdx.x * blockDim.x + threadIdx.x, vref, mb);
}
template <typename T>
__global__ void k_bc_z(MeshD m, Fld<T> f, const Scal *sc, int mode, const T *vref, MagF<T> mb)
{
    bc_z_body(m, f, sc, mode, (long long)blockIdx.x * blockDim.x + threadIdx.x, vref, mb);
}

// ---------------------------------------------------------------------------
// Courant reduction, Eq. cfl2 with the items of Sec. 3.4 and the FARGO
// amendments of Sec. 3.4.2, in two launches.
//
// Per active cell s = sum_i (Delta t_i)^-2 (four rates, summed in the order
// 1..4); the step is C / sqrt(max s), which equals C min(1/sqrt(s)) exactly
// because sqrt and division are correctly rounded and monotone.  The FP64
// value of s must be bit-identical to a plain IEEE evaluation, and FP64
// division and square root are slow on this part, so:
//  k_cfl_screen: one warp per active ring computes v0 = (max + min)/2 of the
//    ring exactly (Eq. 37) and an FP32 estimate of s per cell (relative error
//    below 2e-6), keeps the ring maximum of the estimate, and the last block
//    reduces the global estimate M and the FP64 shear limit of Eq. 38.
//  k_cfl_exact: every ring whose estimate reaches M (1 - 2^-12) is evaluated
//    exactly in FP64 with round-to-nearest intrinsics (no fused multiply-add),
//    by a whole block (all four sub-partitions' FP64 units); the ring holding
//    the true maximum always qualifies.  The last block publishes dt, clipped
//    to t_end.
// The screening launch also fills the per-step planet angle tables (sin^2 of
// half the azimuth offset to the planet and its cosine) used by sub-step 1.
// With a magnetic field (Sec. 3.5) the sound speed becomes the fast speed
// sqrt(c_s^2 + B^2 / rho), B^2 from zone-centred two-point averages of the
// face values, and the Ohmic rate 4 eta / dmin^2 joins the sum of squares
// after the four others (the paper prints no MHD time-step condition).
// ---------------------------------------------------------------------------
// |B|^2 at the centre of cell c = (i, j, k): each component the mean of its
// two faces (the single value along an absent direction), summed X, Y, Z;
// FP64 round-to-nearest, or FP32 for the screen.
template <typename T>
__device__ __forceinline__ double mhd_b2(const MeshD &m, const Tab<T> &tb, idx_t c, int i)
{
    const idx_t n1[3] = {c - i + (i + 1 == m.nx ? 0 : i + 1), m.hasY ? c + m.sj : c, m.hasZ ? c + m.sk : c};
    double b2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double bc = __dmul_rn(0.5, __dadd_rn((double)tb.bfield[d][c], (double)tb.bfield[d][n1[d]]));
        b2 = __dadd_rn(b2, __dmul_rn(bc, bc));
    }
    return b2;
}
template <typename T>
__device__ __forceinline__ float mhd_b2f(const MeshD &m, const Tab<T> &tb, idx_t c, int i)
{
    const idx_t n1[3] = {c - i + (i + 1 == m.nx ? 0 : i + 1), m.hasY ? c + m.sj : c, m.hasZ ? c + m.sk : c};
    float b2 = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float bc = 0.5f * ((float)tb.bfield[d][c] + (float)tb.bfield[d][n1[d]]);
        b2 += bc * bc;
    }
    return b2;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_maxf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double av_rate(const MeshD &m, double dv, double len)
{
    if (m.av_lit) return __ddiv_rn(fabs(dv), __dmul_rn(m.av_c2, len));
    if (dv < 0.0) return __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(4.0, m.cq), m.cq), -dv), len);
    return 0.0;
}
// FP32 estimate of the artificial-viscosity rate from the reciprocal of the
// cell length; k4 = 4 C_q^2 (ZEUS form) or 1/(4 sqrt 2) (printed form), both
// rounded to FP32 on the host side.
__device__ __forceinline__ float av_ratef(bool lit, float k4, float dv, float ilen)
{
    if (lit) return fabsf(dv) * k4 * ilen;
    if (dv < 0.0f) return k4 * (-dv) * ilen;
    return 0.0f;
}

// 16 bytes of a field row: 4 FP32 or 2 FP64 values, loaded with one
// 128-bit access (the address is 16-byte aligned).
template <typename T>
struct alignas(16) Pack {
    static constexpr int W = 16 / sizeof(T);
    T v[W];
};
template <typename T>
__device__ __forceinline__ Pack<T> ldpack(const T *p)
{
    return *reinterpret_cast<const Pack<T> *>(p);
}

__device__ __forceinline__ bool cfl_skip(const Scal *sc)
{
    return sc->err != 0 || (!sc->fixed && sc->t >= sc->t_end);
}

template <typename T>
__device__ __forceinline__ void cfl_screen_body(const MeshD &m, const Tab<T> &tb, const Fld<T> &f, double *v0,
                                                float *ringmax, double *part, Scal *sc, int nrings, int bid,
                                                int nblk)
{
    __shared__ float s_red[8];
    __shared__ double s_m[8];
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = bid * 8 + warp;
    const bool skip = cfl_skip(sc);
    // planet tables for this step (time t^n): the planet on its circular
    // orbit, or the planets read from pl_pos (integrated on the device), each
    // with its azimuth and per-ring tables
    if (m.has_planet) {
        const int gt = bid * blockDim.x + threadIdx.x, gs = nblk * blockDim.x;
        const int np = m.pl_pos ? m.pl_n : 1, NR = m.nyt * m.nzt;
        for (int p = 0; p < np; p++) {
            double php = m.php0 + m.om_rel * sc->t, ap = 0.0, zp = 0.0, irp3 = 0.0, qp = m.pq;
            if (m.pl_pos) {
                const double *pos = m.pl_pos + (size_t)p * m.pl_stride;
                const double px = pos[0], py = pos[1];
                zp = pos[2];
                ap = sqrt(px * px + py * py);
                // the integrator's axes turned to the mesh's by the frame angle
                php = (ap > 0.0 ? atan2(py, px) : 0.0) - (m.fr0 + m.omega * sc->t);
                const double r2 = ap * ap + zp * zp;
                irp3 = 1.0 / (r2 * sqrt(r2));
                if (m.pl_mass) qp = m.pl_mass[p];
                if (gt == 0) tb.mq[p] = (T)qp;
            }
            for (int i = gt; i < m.nx; i += gs) {
                const double dphi = (m.xmin + (i + 0.5) * m.dx) - php;
                const double sh = sin(0.5 * dphi);
                tb.ps[p * m.nx + i] = (T)(sh * sh);
                tb.pc[p * m.nx + i] = (T)cos(dphi);
            }
            if (m.pl_pos) {
                T *tp = tb.mring + (size_t)p * 5 * NR;
                for (int r = gt; r < NR; r += gs) {
                    const double R = tb.Rd[r], Z = tb.zcd[r], dz = Z - zp;
                    tp[r] = (T)(R - ap);
                    tp[NR + r] = (T)(4.0 * R * ap);
                    tp[2 * NR + r] = (T)(dz * dz);
                    tp[3 * NR + r] = (T)(qp * R * ap * irp3);
                    tp[4 * NR + r] = (T)(qp * Z * zp * irp3);
                }
            }
        }
    }
    float smax = 0.0f;
    int bad = 0;
    if (!skip && r < nrings) {
        const int ny = m.j1 - m.j0;
        const int j = m.j0 + r % ny, k = m.k0 + r / ny;
        const int ring = k * m.nyt + j;
        const idx_t base = IX(m, 0, j, k);
        // 16-byte loads: W cells per lane (rows start on 128-byte boundaries;
        // the last pack of a ragged row reads into the row padding, and
        // only cells i < nx count)
        constexpr int W = Pack<T>::W;
        const int nx = m.nx;
        double v0r = 0.0;
        // the stored v_x is v_x - vref in the reference form (FP32); sums of
        // an FP32 value and vref are exact in FP64 whenever v_x itself is an
        // FP32 value (as it is right after the field was set)
        const double vrr = sizeof(T) == 4 && tb.vrefd ? tb.vrefd[ring] : 0.0;
        if (m.fargo) {
            // max and min are exact in the field precision
            T mx = f.vx[base], mn = mx;
            // (unrolled: several loads of a lane in flight at once)
#pragma unroll 4
            for (int i0 = lane * W; i0 < nx; i0 += 32 * W) {
                const Pack<T> pv = ldpack(f.vx + base + i0);
#pragma unroll
                for (int u = 0; u < W; u++)
                    if (i0 + u < nx) {
                        mx = pv.v[u] > mx ? pv.v[u] : mx;
                        mn = pv.v[u] < mn ? pv.v[u] : mn;
                    }
            }
            v0r = __dmul_rn(0.5, __dadd_rn(__dadd_rn(vrr, warp_max((double)mx)), __dadd_rn(vrr, warp_min((double)mn))));
            if (lane == 0) {
                v0[ring] = v0r;
                // the ring's bulk angular rate v0 / (R dx) for the shear limit (Eq. 38),
                // kept after the nyt*nzt v0 values
                v0[(size_t)m.nyt * m.nzt + ring] = __ddiv_rn(v0r, tb.lx[ring]);
            }
        }
        const double v0s = __dsub_rn(v0r, vrr);   // v0 against the stored values
        const T v0hi = (T)v0s, v0lo = (T)(v0s - (double)v0hi);
        // per-ring reciprocals: the estimate needs no division per cell and no
        // square root (the sound-speed rate enters squared)
        const float ilx = 1.0f / (float)tb.lenx[ring], ily = 1.0f / (float)tb.dy[j];
        const float ilz = 1.0f / (float)tb.lenz[ring];
        const float dmin = (float)tb.dminT[ring];
        const float idm2 = 1.0f / (dmin * dmin);
        const float r4 = m.has_nu ? (float)tb.r4[ring] : 0.0f;
        const float r5 = m.mhd ? 4.0f * (float)m.eta * idm2 : 0.0f;
        const float csr = m.iso ? (float)tb.cs[ring] : 0.0f;
        const float c1 = m.iso ? csr * csr * idm2 : (float)tb.g1 * idm2;
        const bool lit = m.av_lit != 0;
        const float k4 = (float)tb.k4;
        const bool avon = m.has_av != 0;
        const T vx0 = f.vx[base];   // right neighbour of the ring's last cell
        for (int i0 = lane * W; i0 < nx; i0 += 32 * W) {
            const idx_t c = base + i0;
            const Pack<T> prho = ldpack(f.rho + c);
            Pack<T> pe{}, px{}, py{}, pyu{}, pz{}, pzu{};
            if (!m.iso) pe = ldpack(f.e + c);
            T xnext = vx0;
            if (m.hasX) {
                px = ldpack(f.vx + c);
                if (i0 + W < nx) xnext = f.vx[c + W];
            }
            if (m.hasY) {
                py = ldpack(f.vy + c);
                pyu = ldpack(f.vy + c + m.sj);
            }
            if (m.hasZ) {
                pz = ldpack(f.vz + c);
                pzu = ldpack(f.vz + c + m.sk);
            }
#pragma unroll
            for (int u = 0; u < W; u++) {
                if (i0 + u >= nx) break;
                const float rho = (float)prho.v[u];
                float r1s;   // (c_s / dmin)^2
                if (m.iso) {
                    r1s = c1;
                } else {
                    const float e = (float)pe.v[u];
                    if (!isfinite(e) || e < 0.0f) bad = 1;
                    r1s = c1 * __fdividef(e, rho);
                }
                if (!isfinite(rho) || rho <= 0.0f) bad = 1;
                float r2 = 0.0f, r3 = 0.0f;
                if (m.hasX) {
                    const T vc = px.v[u];
                    const T vp = i0 + u + 1 < nx ? (u + 1 < W ? px.v[u + 1 < W ? u + 1 : u] : xnext) : vx0;
                    const float a = fabsf((float)sub_split(vc, v0hi, v0lo));
                    const float b = fabsf((float)sub_split(vp, v0hi, v0lo));
                    r2 = fmaxf(r2, fmaxf(a, b) * ilx);
                    if (avon) r3 = fmaxf(r3, av_ratef(lit, k4, (float)(vp - vc), ilx));
                    if (!isfinite((float)vc)) bad = 1;
                }
                if (m.hasY) {
                    const T vc = py.v[u], vp = pyu.v[u];
                    r2 = fmaxf(r2, fmaxf(fabsf((float)vc), fabsf((float)vp)) * ily);
                    if (avon) r3 = fmaxf(r3, av_ratef(lit, k4, (float)(vp - vc), ily));
                    if (!isfinite((float)vc)) bad = 1;
                }
                if (m.hasZ) {
                    const T vc = pz.v[u], vp = pzu.v[u];
                    r2 = fmaxf(r2, fmaxf(fabsf((float)vc), fabsf((float)vp)) * ilz);
                    if (avon) r3 = fmaxf(r3, av_ratef(lit, k4, (float)(vp - vc), ilz));
                    if (!isfinite((float)vc)) bad = 1;
                }
                float s = r1s + r2 * r2 + r3 * r3 + r4 * r4;
                if (m.mhd) s += __fdividef(mhd_b2f(m, tb, c + u, i0 + u), rho) * idm2 + r5 * r5;
                smax = fmaxf(smax, s);
            }
        }
        smax = warp_maxf(smax);
        if (lane == 0) ringmax[r] = smax;
    }
    smax = warp_maxf(smax);
    if (lane == 0) s_red[warp] = smax;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&sc->err, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = s_red[0];
        for (int w = 1; w < 8; w++) b = fmaxf(b, s_red[w]);
        part[bid] = (double)b;
        __threadfence();
        s_last = atomicAdd(&sc->counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double mx = 0.0;
    for (int b = threadIdx.x; b < (int)nblk; b += blockDim.x) mx = fmax(mx, __ldcg(&part[b]));
    mx = warp_max(mx);
    if (lane == 0) s_m[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) mx = fmax(mx, s_m[w]);
        sc->m32 = mx;
        sc->counter = 0u;
    }
}

template <typename T>
__device__ __forceinline__ void cfl_exact_body(const MeshD &m, const Tab<T> &tb, const Fld<T> &f, const double *v0,
                                               const float *ringmax, double *part, Scal *sc, int nrings, int bid,
                                               int nblk)
{
    __shared__ double s_red[8];
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool skip = cfl_skip(sc);
    const double M = sc->m32;
    const double thr = M < 1e-30 ? -1.0 : M * (1.0 - 1.0 / 4096.0);
    double smax = 0.0, wsh = 0.0;
    // chunks of eight rings, chunk ch for block ch mod nblk (the launch has an
    // eighth of the screen's blocks: the per-block overhead dominated); each
    // candidate ring is evaluated by the whole block (its FP64 divisions then
    // use every sub-partition's FP64 unit)
    const int nchunks = (nrings + 7) / 8;
    for (int ch = bid; ch < nchunks; ch += nblk) {
    for (int w = 0; w < 8 && !skip; w++) {
        const int r = ch * 8 + w;
        if (r >= nrings || !((double)ringmax[r] >= thr)) continue;
        const int ny = m.j1 - m.j0;
        const int j = m.j0 + r % ny, k = m.k0 + r / ny;
        const int ring = k * m.nyt + j;
        const idx_t base = IX(m, 0, j, k);
        // v0 against the stored values (the reference form's vref subtracted)
        const double v0r = __dsub_rn(m.fargo ? v0[ring] : 0.0, sizeof(T) == 4 && tb.vrefd ? tb.vrefd[ring] : 0.0);
        const double lx = tb.lx[ring], ly = tb.ly[ring], lz = tb.lz[ring], dmin = tb.dmin[ring];
        const double nu = m.has_nu ? tb.nud[ring] : 0.0;
        const double r4 = nu > 0.0 ? __ddiv_rn(__dmul_rn(4.0, nu), __dmul_rn(dmin, dmin)) : 0.0;
        const double csr = m.iso ? tb.csd[ring] : 0.0;
        // the screen's FP32 estimate per cell (same terms; per-ring factors in
        // FP32): a cell whose estimate falls below thr cannot hold the exact
        // maximum, by the argument that admits the ring (the estimate errs by
        // about 1e-6, the margin is 2^-12), so only the others are evaluated
        // in FP64
        const float ilx = 1.0f / (float)tb.lenx[ring], ily = 1.0f / (float)tb.dy[j];
        const float ilz = 1.0f / (float)tb.lenz[ring];
        const float dmf = (float)tb.dminT[ring];
        const float idm2 = 1.0f / (dmf * dmf);
        const float r4f = m.has_nu ? (float)tb.r4[ring] : 0.0f;
        const float r5f = m.mhd ? 4.0f * (float)m.eta * idm2 : 0.0f;
        const double r5 = m.mhd && m.eta > 0.0 ? __ddiv_rn(__dmul_rn(4.0, m.eta), __dmul_rn(dmin, dmin)) : 0.0;
        const float c1 = m.iso ? (float)csr * (float)csr * idm2 : (float)tb.g1 * idm2;
        const bool lit = m.av_lit != 0, avon = m.has_av != 0;
        const float k4 = (float)tb.k4;
        const T v0hi = (T)v0r, v0lo = (T)(v0r - (double)v0hi);
        for (int i = threadIdx.x; i < m.nx; i += blockDim.x) {
            const idx_t c = base + i;
            const int ip = i + 1 == m.nx ? 0 : i + 1;
            {
                const float rf = (float)f.rho[c];
                float est = m.iso ? c1 : c1 * __fdividef((float)f.e[c], rf);
                float e2 = 0.0f, e3 = 0.0f;
                if (m.hasX) {
                    const T vc = f.vx[c], vp = f.vx[base + ip];
                    const float a = fabsf((float)sub_split(vc, v0hi, v0lo));
                    const float b = fabsf((float)sub_split(vp, v0hi, v0lo));
                    e2 = fmaxf(e2, fmaxf(a, b) * ilx);
                    if (avon) e3 = fmaxf(e3, av_ratef(lit, k4, (float)(vp - vc), ilx));
                }
                if (m.hasY) {
                    const T vc = f.vy[c], vp = f.vy[c + m.sj];
                    e2 = fmaxf(e2, fmaxf(fabsf((float)vc), fabsf((float)vp)) * ily);
                    if (avon) e3 = fmaxf(e3, av_ratef(lit, k4, (float)(vp - vc), ily));
                }
                if (m.hasZ) {
                    const T vc = f.vz[c], vp = f.vz[c + m.sk];
                    e2 = fmaxf(e2, fmaxf(fabsf((float)vc), fabsf((float)vp)) * ilz);
                    if (avon) e3 = fmaxf(e3, av_ratef(lit, k4, (float)(vp - vc), ilz));
                }
                est += e2 * e2 + e3 * e3 + r4f * r4f;
                if (m.mhd) est += __fdividef(mhd_b2f(m, tb, c, i), rf) * idm2 + r5f * r5f;
                if ((double)est < thr) continue;
            }
            const double rho = (double)f.rho[c];
            const double cs = m.iso ? csr : __dsqrt_rn(__ddiv_rn(__dmul_rn(m.g1, (double)f.e[c]), rho));
            const double r1 = m.mhd ? __ddiv_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(cs, cs),
                                                                     __ddiv_rn(mhd_b2(m, tb, c, i), rho))), dmin)
                                    : __ddiv_rn(cs, dmin);
            double r2 = 0.0, r3 = 0.0;
            if (m.hasX) {
                const double vc = (double)f.vx[c], vp = (double)f.vx[base + ip];
                const double a = fabs(__dsub_rn(vc, v0r)), b = fabs(__dsub_rn(vp, v0r));
                r2 = fmax(r2, __ddiv_rn(a > b ? a : b, lx));
                r3 = fmax(r3, av_rate(m, __dsub_rn(vp, vc), lx));
            }
            if (m.hasY) {
                const double vc = (double)f.vy[c], vp = (double)f.vy[c + m.sj];
                const double a = fabs(vc), b = fabs(vp);
                r2 = fmax(r2, __ddiv_rn(a > b ? a : b, ly));
                r3 = fmax(r3, av_rate(m, __dsub_rn(vp, vc), ly));
            }
            if (m.hasZ) {
                const double vc = (double)f.vz[c], vp = (double)f.vz[c + m.sk];
                const double a = fabs(vc), b = fabs(vp);
                r2 = fmax(r2, __ddiv_rn(a > b ? a : b, lz));
                r3 = fmax(r3, av_rate(m, __dsub_rn(vp, vc), lz));
            }
            if (m.cq <= 0.0) r3 = 0.0;
            double s = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(r1, r1), __dmul_rn(r2, r2)),
                                           __dmul_rn(r3, r3)),
                                 __dmul_rn(r4, r4));
            if (r5 > 0.0) s = __dadd_rn(s, __dmul_rn(r5, r5));
            smax = fmax(smax, s);
        }
    }
    // shear limit (Eq. 38) of the chunk's eight rings and their outer
    // neighbours, from the bulk angular rates the screen stored after v0
    if (warp == 0 && lane < 8 && m.fargo && m.hasY && !skip) {
        const int r = ch * 8 + lane;
        const int ny = m.j1 - m.j0;
        // (on a periodic Y axis the last ring's outer neighbour is the first)
        if (r < nrings && (r % ny < ny - 1 || m.pery)) {
            const int ring = (m.k0 + r / ny) * m.nyt + m.j0 + r % ny;
            const int next = r % ny < ny - 1 ? ring + 1 : ring - (ny - 1);
            const double *om = v0 + (size_t)m.nyt * m.nzt;
            wsh = fmax(wsh, fabs(__dsub_rn(__ldcg(&om[ring]), __ldcg(&om[next]))));
        }
    }
    }
    smax = warp_max(smax);
    if (warp == 0) wsh = warp_max(wsh);
    if (lane == 0) s_red[warp] = smax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = s_red[0];
        for (int w = 1; w < 8; w++) b = fmax(b, s_red[w]);
        part[bid] = b;
        part[nblk + bid] = wsh;
        __threadfence();
        s_last = atomicAdd(&sc->counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double mx = 0.0, ws = 0.0;
    for (int b = threadIdx.x; b < (int)nblk; b += blockDim.x) {
        mx = fmax(mx, __ldcg(&part[b]));
        ws = fmax(ws, __ldcg(&part[nblk + b]));
    }
    mx = warp_max(mx);
    ws = warp_max(ws);
    __shared__ double s_ws[8];
    if (lane == 0) {
        s_red[warp] = mx;
        s_ws[warp] = ws;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) {
            mx = fmax(mx, s_red[w]);
            ws = fmax(ws, s_ws[w]);
        }
        int err = atomicOr(&sc->err, 0);
        const double t = sc->t, te = sc->t_end, wsh = ws;
        double dt = 0.0;
        if (!skip) {
            if (sc->fixed) {
                dt = sc->dt_fixed;
            } else {
                dt = __dmul_rn(m.cfl, __ddiv_rn(1.0, __dsqrt_rn(mx)));
                if (wsh > 0.0) {
                    const double ds = __ddiv_rn(m.cfl, wsh);
                    if (ds < dt) dt = ds;
                }
                if (__dadd_rn(t, dt) > te) dt = __dsub_rn(te, t);
                if (!(dt > 0.0) || !isfinite(dt)) err |= 2;
            }
        }
        if (err) dt = 0.0;
        sc->err = err;
        sc->dt = dt;
        sc->dtf = (float)dt;
        sc->counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// Reference form of v_x (FP32): one warp per ring r of the nyt * nzt rings.
//   VREF_ABS:    dst <- v' + vref[r] (the stored values back to v_x; dst may
//                be the field itself)
//   VREF_CHOOSE: vref[r] <- m, the mid-range of the v_x values of ring img(r)
//                (the ring itself, or its image one period away on a
//                periodic axis, so that images share a reference), when
//                every value v of that ring has (v - m) + m == v in FP32
//                (v - m then holds v exactly); otherwise 0
//   VREF_APPLY:  v' <- v - vref[r]; lane 0 also writes the frame shifts dAy,
//                dAz of the X momenta from A = R vref + w (FP64, rounded once)
//   VREF_TABLES: the frame shifts alone (after a change of the frame rate)
// CHOOSE reads v_x values only, so the whole field may be in v_x form while
// it runs; APPLY runs after it (a separate launch).
// ---------------------------------------------------------------------------
enum { VREF_ABS = 0, VREF_CHOOSE = 1, VREF_APPLY = 2, VREF_TABLES = 3 };

template <typename T>
__device__ void vref_ring(const MeshD &m, const Tab<T> &tb, T *vx, T *dst, int ring, int mode)
{
    const int lane = threadIdx.x & 31;
    const int j = ring % m.nyt, k = ring / m.nyt;
    const idx_t base = IX(m, 0, j, k);
    if (mode == VREF_ABS) {
        const T r = tb.vref[ring];
        for (int i = lane; i < m.nx; i += 32) dst[base + i] = vx[base + i] + r;
        return;
    }
    if (mode == VREF_APPLY || mode == VREF_TABLES) {
        const T r = tb.vref[ring];
        if (mode == VREF_APPLY)
            for (int i = lane; i < m.nx; i += 32) vx[base + i] = vx[base + i] - r;
        if (lane == 0) {
            auto A = [&](int q) {
                const double R = tb.Rd[q];
                const double w = m.geom == CART ? tb.wfrd[q] : R * R * m.omega;
                return R * tb.vrefd[q] + w;
            };
            const double a = A(ring);
            tb.dAy[ring] = j >= 1 ? (T)(a - A(ring - 1)) : T(0);
            tb.dAz[ring] = k >= 1 ? (T)(a - A(ring - m.nyt)) : T(0);
        }
        return;
    }
    int ji = j, ki = k;
    if (m.pery && m.hasY) ji = j < m.j0 ? j + (m.j1 - m.j0) : (j >= m.j1 ? j - (m.j1 - m.j0) : j);
    if (m.perz && m.hasZ) ki = k < m.k0 ? k + (m.k1 - m.k0) : (k >= m.k1 ? k - (m.k1 - m.k0) : k);
    const idx_t bi = IX(m, 0, ji, ki);
    double mx = -INFINITY, mn = INFINITY;
    bool fin = true;
    for (int i = lane; i < m.nx; i += 32) {
        const double v = (double)vx[bi + i];
        fin = fin && isfinite(v);
        mx = fmax(mx, v);
        mn = fmin(mn, v);
    }
    mx = warp_max(mx);
    mn = warp_min(mn);
    // (no reference with a magnetic field: the MHD kernels read v_x itself)
    T r = fin && !m.mhd ? (T)(0.5 * (mx + mn)) : T(0);
    bool exact = fin;
    for (int i = lane; i < m.nx && exact; i += 32) {
        const T v = vx[bi + i];
        exact = (v - r) + r == v;
    }
    if (!__all_sync(0xffffffffu, exact)) r = T(0);
    if (lane == 0) {
        tb.vref[ring] = r;
        tb.vrefd[ring] = (double)r;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_vref(MeshD m, Tab<T> tb, T *vx, T *dst, int mode)
{
    const int ring = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (ring < m.nyt * m.nzt) vref_ring(m, tb, vx, dst, ring, mode);
}

// Blocks of the exact pass for a screen of cfl_blocks blocks (eight rings each).
__host__ __device__ __forceinline__ int cfl_exact_grid(int cfl_blocks) { return (cfl_blocks + 7) / 8; }

// (four blocks per SM at 64 registers: at 40 the screen spilled, and the
// batched screen measured 0.66 ms against 0.53 ms with no spills)
template <typename T>
__global__ void __launch_bounds__(256, 4) k_cfl_screen(MeshD m, Tab<T> tb, Fld<T> f, double *v0, float *ringmax,
                                                    double *part, Scal *sc, int nrings)
{
    cfl_screen_body(m, tb, f, v0, ringmax, part, sc, nrings, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(256) k_cfl_exact(MeshD m, Tab<T> tb, Fld<T> f, const double *v0,
                                                   const float *ringmax, double *part, Scal *sc, int nrings)
{
    cfl_exact_body(m, tb, f, v0, ringmax, part, sc, nrings, blockIdx.x, gridDim.x);
}

}  // namespace fk
