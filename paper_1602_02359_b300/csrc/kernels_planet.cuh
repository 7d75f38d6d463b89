// Force of the gas on a planet (Sec. 3.7, orbital integrator: the force of
// the disk on the planets, evaluated once per hydrodynamical step), per unit
// planet mass, G = 1, Plummer softening eps:
//   a = sum over active cells of m_c (r_c - r_p) / (|r_c - r_p|^2 + eps^2)^(3/2),
// m_c = rho_c V_c, optionally with each ring's mean density removed first
// (the BM08 option of the same section: an axisymmetric disk then exerts no
// force).  Cylindrical and spherical meshes.
//
// The sum runs in the frame turned to the planet's azimuth: a cell at
// cylindrical radius R, height Z and azimuth offset dphi from the planet sits
// at X' = (R - R_p) - 2 R sin^2(dphi/2), Y' = R sin(dphi), Z' = Z - z_p, with
// R - R_p and Z - z_p formed in FP64 per ring and the sines evaluated per
// azimuth in FP64 (both then rounded to the field precision), so no difference of nearby large coordinates is formed in
// the field precision.  Per-cell arithmetic is in the field precision: the
// B300's FP64 rate is a small fraction of its FP32 rate, so FP64 appears only
// in the per-call tables and the final reduction.  A warp takes a ring: each
// lane sums its cells of the ring in the field precision and adds that into
// a compensated (TwoSum) total; lanes, warps and blocks are then summed in
// FP64, the block partials in a fixed order by the last block
// (deterministic for a given grid).
#pragma once
#include "fargo_internal.cuh"
#include "kernels_bc_cfl.cuh"

namespace fk {

// The planet's position: by value, or read from device memory (x, y, z at
// dev) when dev is set, so that a planet integrated on the device needs no
// round trip through the host.  With sc set, the position is in the
// planetary integrator's non-rotating axes, which the mesh's axes make the
// angle fr0 + om t with (t the device time); the force comes out in the
// integrator's axes.  Without, position and force are in the mesh's axes.
struct PfPlanet {
    double x, y, z;
    const double *dev;
    double fr0 = 0.0, om = 0.0;
    const Scal *sc = nullptr;
    __device__ __forceinline__ double frame_angle() const { return sc ? fr0 + om * sc->t : 0.0; }
    __device__ __forceinline__ void get(double &px, double &py, double &pz) const
    {
        if (dev) {
            px = dev[0];
            py = dev[1];
            pz = dev[2];
        } else {
            px = x;
            py = y;
            pz = z;
        }
    }
};

template <typename T>
struct PForceArgs {
    const T *rho;
    const T *tab;                   // sin^2(dphi/2) [nx], sin(dphi) [nx] (each padded to the row pitch sj),
                                    // then per active ring R, R - R_p, Z - z_p, V
    PfPlanet pl;                    // the planet's position
    T eps2;                         // squared softening
    double *ring_fy;                // with the profile option: each active ring's planet-frame y force
    int nx, j0, j1, k0, k1, nyt, sj, sk;
};

// Tables of one call, evaluated in FP64 and rounded to the field precision:
// per azimuth, sin^2((x_i - php)/2) and sin(x_i - php) for the cell centres
// x_i; per active ring r, the cylindrical radius R, R - R_p and Z - z_p
// (formed in FP64, so no nearby large numbers are subtracted in the field
// precision) and the cell volume.  One thread per azimuth or ring.
template <typename T>
__global__ void __launch_bounds__(256) k_pforce_tables(T *tab, int nx, int sj, double xmin, double dx, PfPlanet pl,
                                                       const double *Rd, const double *zcd, const double *vol,
                                                       int j0, int j1, int k0, int k1, int nyt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double px, py, pz;
    pl.get(px, py, pz);
    const double Rp = sqrt(px * px + py * py);
    if (t < nx) {
        // the planet's azimuth on the mesh; the force is turned back by the
        // azimuth in the planet's own axes (k_planet_force), so it comes out
        // in those axes
        const double php = (Rp > 0.0 ? atan2(py, px) : 0.0) - pl.frame_angle();
        const double d = (xmin + (t + 0.5) * dx) - php;
        const double h = sin(0.5 * d);
        tab[t] = (T)(h * h);
        tab[sj + t] = (T)sin(d);
    }
    const int nyA = j1 - j0, nr = nyA * (k1 - k0);
    if (t < nr) {
        const int j = j0 + t % nyA, k = k0 + t / nyA, ring = k * nyt + j;
        T *rt = tab + 2 * (size_t)sj + 4 * (size_t)t;
        rt[0] = (T)Rd[ring];
        rt[1] = (T)(Rd[ring] - Rp);
        rt[2] = (T)(zcd[ring] - pz);
        rt[3] = (T)vol[ring];
    }
}

// Error-free sum of two values (Knuth's TwoSum): s + e = a + b exactly.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e)
{
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// compensated accumulator: (s, c) += x
template <typename T>
__device__ __forceinline__ void csum_add(T &s, T &c, T x)
{
    T e;
    two_sum(s, x, s, e);
    c += e;
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// Contribution of one cell, of mass density mc, at (X, Y, dZ) from the
// planet in its frame, added to (tx, ty, tz).
template <typename T>
__device__ __forceinline__ void pforce_cell(T mc, T s2, T sn, T R, T dR, T dZ, T eps2, T &tx, T &ty, T &tz)
{
    const T X = dR - T(2) * R * s2;
    const T Y = R * sn;
    const T iv = rsqrt_t<T>(X * X + Y * Y + dZ * dZ + eps2);
    const T w = mc * iv * iv * iv;
    tx += w * X;
    ty += w * Y;
    tz += w * dZ;
}

// One warp per active ring (warp-stride); lanes take 16-byte packs of the
// ring's cells, kPfU density packs loaded before any is used (the DRAM
// loads of a lane overlap; the azimuth tables stay in L1), and the ring's
// last nx mod W cells one by one.
// part: 3 partials per block; out: (a_x, a_y, a_z, specific z torque).
// Resident blocks per SM: the hoisted packs and the unrolled cells want
// 85 (FP32) or 128 (FP64) registers a thread.
constexpr int kPfU = 4;
template <typename T>
constexpr int pforce_blocks_per_sm()
{
    return sizeof(T) == 4 ? 3 : 2;
}
template <typename T, bool BM08, bool PROF = false>
__global__ void __launch_bounds__(256, pforce_blocks_per_sm<T>()) k_planet_force(PForceArgs<T> a, double *part, unsigned *counter, double *out)
{
    constexpr int W = Pack<T>::W;
    __shared__ double s_red[3][8];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nyA = a.j1 - a.j0, nrings = nyA * (a.k1 - a.k0);
    const int nv = a.nx / W, itail = nv * W;
    const T *s2t = a.tab, *snt = s2t + a.sj;
    const T *rt = s2t + 2 * (size_t)a.sj;
    T sx = 0, cx = 0, sy = 0, cy = 0, sz = 0, cz = 0;   // compensated totals of the lane
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp, nw = gridDim.x * (blockDim.x >> 5);
    for (int r = gw; r < nrings; r += nw) {
        const int j = a.j0 + r % nyA, k = a.k0 + r / nyA;
        const T *row = a.rho + (size_t)k * a.sk + (size_t)j * a.sj;
        const T R = rt[4 * r], dR = rt[4 * r + 1], dZ = rt[4 * r + 2], V = rt[4 * r + 3];
        T mu_hi = 0, mu_lo = 0;
        if (BM08) {
            // the ring's mean density as an unevaluated pair hi + lo
            T s = 0, c = 0;
            for (int v0 = lane; v0 < nv; v0 += 32 * kPfU) {
                Pack<T> p[kPfU];
#pragma unroll
                for (int u = 0; u < kPfU; u++)
                    if (v0 + 32 * u < nv) p[u] = ldpack(row + (v0 + 32 * u) * W);
#pragma unroll
                for (int u = 0; u < kPfU; u++)
                    if (v0 + 32 * u < nv) {
#pragma unroll
                        for (int e = 0; e < W; e++) csum_add(s, c, p[u].v[e]);
                    }
            }
            for (int i = itail + lane; i < a.nx; i += 32) csum_add(s, c, row[i]);
            for (int o = 16; o > 0; o >>= 1) {
                const T s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
                T e;
                two_sum(s, s2, s, e);
                c += c2 + e;
            }
            const T inv = T(1) / (T)a.nx;
            T e;
            two_sum(s, c, s, e);   // renormalise: s carries the sum, e what it lost
            mu_hi = s * inv;
            mu_lo = ((s - mu_hi * (T)a.nx) + e) * inv;
        }
        T tx = 0, ty = 0, tz = 0;
        for (int v0 = lane; v0 < nv; v0 += 32 * kPfU) {
            Pack<T> pr[kPfU];
#pragma unroll
            for (int u = 0; u < kPfU; u++)
                if (v0 + 32 * u < nv) pr[u] = ldpack(row + (v0 + 32 * u) * W);
#pragma unroll
            for (int u = 0; u < kPfU; u++)
                if (v0 + 32 * u < nv) {
                    const int o = (v0 + 32 * u) * W;
                    const Pack<T> ps = ldpack(s2t + o), pn = ldpack(snt + o);   // L1-resident tables
#pragma unroll
                    for (int e = 0; e < W; e++)
                        pforce_cell((BM08 ? sub_split(pr[u].v[e], mu_hi, mu_lo) : pr[u].v[e]) * V, ps.v[e], pn.v[e],
                                    R, dR, dZ, a.eps2, tx, ty, tz);
                }
        }
        for (int i = itail + lane; i < a.nx; i += 32)
            pforce_cell((BM08 ? sub_split(row[i], mu_hi, mu_lo) : row[i]) * V, s2t[i], snt[i], R, dR, dZ, a.eps2,
                        tx, ty, tz);
        if (PROF) {   // the ring's share of the planet-frame y force, summed over lanes in FP64
            double ry = (double)ty;
            for (int o = 16; o > 0; o >>= 1) ry += __shfl_xor_sync(0xffffffffu, ry, o);
            if (lane == 0) a.ring_fy[r] = ry;
        }
        csum_add(sx, cx, tx);
        csum_add(sy, cy, ty);
        csum_add(sz, cz, tz);
    }
    // FP64 from here: lanes, warps, blocks (the last in block order)
    double vx = (double)sx + (double)cx, vy = (double)sy + (double)cy, vz = (double)sz + (double)cz;
    for (int o = 16; o > 0; o >>= 1) {
        vx += __shfl_xor_sync(0xffffffffu, vx, o);
        vy += __shfl_xor_sync(0xffffffffu, vy, o);
        vz += __shfl_xor_sync(0xffffffffu, vz, o);
    }
    if (lane == 0) {
        s_red[0][warp] = vx;
        s_red[1][warp] = vy;
        s_red[2][warp] = vz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bx = 0.0, by = 0.0, bz = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            bx += s_red[0][w];
            by += s_red[1][w];
            bz += s_red[2][w];
        }
        part[3 * blockIdx.x] = bx;
        part[3 * blockIdx.x + 1] = by;
        part[3 * blockIdx.x + 2] = bz;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the block partials, by the whole last block in a fixed order: thread t
    // takes blocks t, t + 256, ...; then lanes and warps as above
    {
        double bx = 0.0, by = 0.0, bz = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            bx += __ldcg(&part[3 * b]);
            by += __ldcg(&part[3 * b + 1]);
            bz += __ldcg(&part[3 * b + 2]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            bx += __shfl_xor_sync(0xffffffffu, bx, o);
            by += __shfl_xor_sync(0xffffffffu, by, o);
            bz += __shfl_xor_sync(0xffffffffu, bz, o);
        }
        __syncthreads();   // s_red was read by thread 0 above
        if (lane == 0) {
            s_red[0][warp] = bx;
            s_red[1][warp] = by;
            s_red[2][warp] = bz;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double bx = 0.0, by = 0.0, bz = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            bx += s_red[0][w];
            by += s_red[1][w];
            bz += s_red[2][w];
        }
        // back from the planet's frame; the torque is R_p a_y' (z component of r_p x a)
        double px, py, pz;
        a.pl.get(px, py, pz);
        const double Rp = sqrt(px * px + py * py);
        const double cph = Rp > 0.0 ? px / Rp : 1.0, sph = Rp > 0.0 ? py / Rp : 0.0;
        out[0] = bx * cph - by * sph;
        out[1] = bx * sph + by * cph;
        out[2] = bz;
        out[3] = Rp * by;
        *counter = 0u;
    }
}

}  // namespace fk
