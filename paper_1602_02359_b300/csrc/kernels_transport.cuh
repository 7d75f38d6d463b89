// Transport step (flow-chart cell 12): left/right momenta, the X sweep with
// orbital advection, the Y and Z sweeps, and the new face velocities.
#pragma once
#include <algorithm>
#include "fargo_internal.cuh"
#include "kernels_source.cuh"
#include "tma.cuh"

namespace fk {

// van Leer slope (Sec. 3.5, below Eq. 15): harmonic mean of the one-sided
// differences over the centre-to-centre distances, zero across an extremum.
template <typename T>
__device__ __forceinline__ T vl_slope(T qm, T q0, T qp, T dxm, T dxp)
{
    const T dp = (qp - q0) / dxp, dm = (q0 - qm) / dxm;
    return dp * dm > T(0) ? T(2) * dp * dm / (dp + dm) : T(0);
}


// The same slope with the inverse centre distances given.
template <typename T>
__device__ __forceinline__ T vl_slope_i(T qm, T q0, T qp, T idm, T idp)
{
    const T dp = (qp - q0) * idp, dm = (q0 - qm) * idm;
    const T pr = dp * dm;
    return pr > T(0) ? div_fast(T(2) * pr, dp + dm) : T(0);
}
// A product rounded on its own (never contracted into a later addition), and
// a fused multiply-add: the Y/Z sweeps form a face flux in two places (a
// segment's first face, and every later face), which must round alike.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// The same slope from the two differences q0 - qm and qp - q0.
template <typename T>
__device__ __forceinline__ T vl_slope_d(T dqm, T dqp, T idm, T idp)
{
    const T dp = dqp * idp, dm = dqm * idm;
    const T pr = dp * dm;
    return pr > T(0) ? div_fast(T(2) * pr, dp + dm) : T(0);
}

// PPA (Sec. 3.4.1): monotonised-centred slope of Eq. 34 for cell values
// (qm, q0, qp).
template <typename T>
__device__ __forceinline__ T ppa_dm(T qm, T q0, T qp)
{
    if (!((qp - q0) * (q0 - qm) > T(0))) return T(0);
    const T d = T(0.5) * (qp - qm);
    T mn = fmin(T(2) * fabs(q0 - qm), T(2) * fabs(qp - q0));
    mn = fmin(mn, fabs(d));
    return d > T(0) ? mn : -mn;
}

// PPA interface value through the face whose donor cell is the centre of
// a[0..4] (cells d-2..d+2): parabolic interface values (Eq. 35), the
// monotonisation of Eq. 36, then the xi-weighted average over the donor
// region (pos: the face above the donor; otherwise the face below).
template <typename T>
__device__ __forceinline__ T ppa_face(const T a[5], T xi, bool pos)
{
    const T sixth = T(1.0 / 6.0);
    const T dmm = ppa_dm(a[0], a[1], a[2]), dm0 = ppa_dm(a[1], a[2], a[3]), dmp = ppa_dm(a[2], a[3], a[4]);
    const T q0 = a[2];
    T l = a[1] + T(0.5) * (a[2] - a[1]) - (dm0 - dmm) * sixth;
    T r = a[2] + T(0.5) * (a[3] - a[2]) - (dmp - dm0) * sixth;
    if ((a[3] - q0) * (q0 - a[1]) <= T(0)) {
        l = q0;
        r = q0;
    } else {
        const T D = r - l, C = q0 - T(0.5) * (l + r);
        if (D * C > D * D * sixth) l = T(3) * q0 - T(2) * r;
        else if (-D * D * sixth > D * C) r = T(3) * q0 - T(2) * l;
    }
    const T w = xi * (T(1) - xi) * (T(2) * q0 - r - l);
    return pos ? r + xi * (q0 - r) + w : l + xi * (q0 - l) + w;
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// Ring kernels.  Persistent CTAs walk the rings (j,k) with a stride of the
// grid and keep two ring buffers in shared memory: while the threads
// compute ring r from one buffer, thread 0 has already issued the 1D bulk
// copies (cp.async.bulk, completed on that buffer's mbarrier) of the CTA's
// next ring into the other, so the staging latency hides behind compute.
// Every thread owns C consecutive cells of a ring.  For each quantity it
// rebuilds, in registers, the ratios to the density of its cells and their
// stencil halo, the slopes, the interface values and the fluxes through its
// C+1 faces, and writes its C updated cells straight to global memory.
// Consistent transport: quantity q > 0 moves with the mass flux times the
// interface ratio, all fluxes from the pre-sweep ring.
// ---------------------------------------------------------------------------

// Bytes of one staged row: nx values rounded up to 16 bytes (rows are
// pitch-aligned, 128-byte boundaries, so the rounding stays in the padding).
template <typename T>
__device__ __forceinline__ unsigned row_bytes(int nx)
{
    return (unsigned)(((size_t)nx * sizeof(T) + 15) / 16 * 16);
}

// Shared-memory layout of a staged ring row: the nx values start kRingLead
// values in (16-byte aligned for the bulk copies) and the row takes the
// field pitch plus kRingPad values.  After a ring lands, ring_frame copies
// its last kRingLead values in front of it and its first kRingTail values
// behind it, so every stencil window of a thread (at most kRingLead cells
// to the left of the ring, kRingTail to the right, or a window of up to
// nx + kRingTail cells starting anywhere on the ring) is one contiguous run
// of shared memory addressed at constant offsets from one base.
constexpr int kRingLead = 4, kRingTail = 16, kRingPad = 32;
__host__ __device__ __forceinline__ int ring_row(int pitch) { return pitch + kRingPad; }

template <typename T>
__device__ __forceinline__ void ring_frame(T *buf, int rows, int rp, int nx)
{
    constexpr int H = kRingLead + kRingTail;
    for (int t = threadIdx.x; t < rows * H; t += blockDim.x) {
        const int r = t / H, h = t - r * H;
        const int x = h < kRingLead ? h - kRingLead : nx + (h - kRingLead);
        int src = x % nx;
        if (src < 0) src += nx;
        T *row = buf + (size_t)r * rp + kRingLead;
        row[x] = row[src];
    }
    __syncthreads();
}

// Per-iteration facts of a ring, computed by all threads in parallel before
// the loop (so no FP64 division or member search sits on the loop's
// critical path): the member and local ring (batched launches), the integer
// shift (orbital step, -1: nothing to do) and two values in the field
// precision (v0 split hi/lo for the X sweep; xi and the fractional
// velocity for the orbital step).
template <typename T>
struct RingMeta {
    int id, local, N;
    T a, b;
    // orbital step: first cell of the ring, its X face area and dt over its
    // cell volume, so the ring's loop reads no table
    idx_t base;
    T S, dtVi;
};

// Persistent double-buffered loop over items first, first+step, ... < n.
// Op provides prepare(it, item) (any thread: fill meta[it]), issue(it, dst,
// bar) (thread 0 only: start the copies of iteration it into dst completed
// on bar, or a plain arrive when it needs no data), compute(it, src) (all
// threads) and fail(it).  bar[0..1] are initialised by the caller with an
// arrival count of one.  Every wait is bounded and the decision to stop is
// block-uniform; on timeout the error is recorded and the copies still in
// flight land before the CTA exits.
template <typename T, class Op>
__device__ __forceinline__ void ring_pipeline(Op &op, T *buf, size_t stride, uint64_t *bar, int first, int step,
                                              int n, int nbuf)
{
    if (first >= n) return;
    const int K = (n - first + step - 1) / step;
    for (int it = threadIdx.x; it < K; it += blockDim.x) op.prepare(it, first + it * step);
    __syncthreads();
    if (threadIdx.x == 0) op.issue(0, buf, &bar[0]);
    if (nbuf == 1) {
        // one buffer (rings too long for two): the next copy is issued once
        // the current ring has been computed
        unsigned use = 0u;
        for (int it = 0; it < K; it++) {
            const bool ok = __syncthreads_and(mbar_wait(&bar[0], use & 1u));
            use++;
            if (!ok) {
                if (threadIdx.x == 0) op.fail(it);
                return;
            }
            op.compute(it, buf);
            __syncthreads();
            if (threadIdx.x == 0 && it + 1 < K) {
                fence_proxy_async_smem();
                op.issue(it + 1, buf, &bar[0]);
            }
        }
        return;
    }
    for (int it = 0; it < K; it++) {
        const int b = it & 1;
        if (threadIdx.x == 0 && it + 1 < K) {
            // the other buffer was last read and framed through the generic proxy
            fence_proxy_async_smem();
            op.issue(it + 1, buf + (size_t)(1 - b) * stride, &bar[1 - b]);
        }
        // iteration it is the (it / 2)-th use of buffer b
        const bool ok = __syncthreads_and(mbar_wait(&bar[b], (unsigned)(it >> 1) & 1u));
        if (!ok) {
            if (threadIdx.x == 0) {
                op.fail(it);
                if (it + 1 < K) mbar_wait(&bar[1 - b], (unsigned)((it + 1) >> 1) & 1u);
            }
            return;
        }
        op.compute(it, buf + (size_t)b * stride);
        __syncthreads();
    }
}

// Iterations of one persistent CTA (the metadata entries it needs).
__host__ __device__ __forceinline__ int ring_iters(int n, int grid) { return (n + grid - 1) / grid; }

__device__ __forceinline__ void ring_bars_init(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
}

// X sweep, residual part (Sec. 3.4.1, Eq. fargo1; Eq. 15 with van Leer
// slopes).  The rows rho, e, v_x and the v_y / v_z rows of the cell's lower
// and upper faces are staged; the momenta of Eqs. 16-17 (Tab. "momenta")
// are formed from them, and so are their consistent-transport ratios, which
// are just the face velocities times the geometric factors (Pi-_x / rho =
// R v_x + R^2 Omega_f, Pi+_y / rho = v_y of the upper face, ...).  The face
// velocity is delta v = v_x - v0 (v0 = 0 for STANDARD transport).  Ghost
// rings only get their momenta written (the Y/Z sweeps read them).
struct TxRows {
    int n, rE, rVX, rVY, rVZ;   // staged rows: rho, e, vx, vy(j), vy(j+1), vz(k), vz(k+1)
};
__device__ __forceinline__ TxRows tx_rows(const MeshD &m)
{
    TxRows r{0, -1, -1, -1, -1};
    r.n = 1;
    if (!m.iso) r.rE = r.n++;
    r.rVX = r.n++;
    if (m.hasY) {
        r.rVY = r.n;
        r.n += 2;
    }
    if (m.hasZ) {
        r.rVZ = r.n;
        r.n += 2;
    }
    return r;
}

// v0 of ring `ring` split as hi + lo in the field precision (0 off the
// active rings and for STANDARD transport).
template <typename T>
__device__ __forceinline__ void tx_v0(const MeshD &m, const Tab<T> &tb, const double *v0, int ring, T &hi, T &lo)
{
    const int j = ring % m.nyt, k = ring / m.nyt;
    const bool active = j >= m.j0 && j < m.j1 && k >= m.k0 && k < m.k1;
    double v0r = m.fargo && active && m.hasX ? v0[ring] : 0.0;
    // the stored v_x is relative to vref in the reference form
    if (sizeof(T) == 4 && tb.vrefd && active) v0r -= tb.vrefd[ring];
    hi = (T)v0r;
    lo = (T)(v0r - (double)hi);
}

// Thread 0: copies of ring `ring` of the X sweep's input into dst (row r of
// the staging at dst + r * ring_row(pitch) + kRingLead).
template <typename T>
__device__ __forceinline__ void tx_issue(const MeshD &m, const Fld<T> &in, int ring, T *dst, uint64_t *bar)
{
    const TxRows r = tx_rows(m);
    const int j = ring % m.nyt, k = ring / m.nyt;
    const idx_t base = IX(m, 0, j, k);
    const size_t rp = (size_t)ring_row(m.sj);
    const unsigned bytes = row_bytes<T>(m.nx);
    dst += kRingLead;
    mbar_expect_tx(bar, bytes * (unsigned)r.n);
    bulk_load(dst, in.rho + base, bytes, bar);
    if (r.rE >= 0) bulk_load(dst + r.rE * rp, in.e + base, bytes, bar);
    bulk_load(dst + r.rVX * rp, in.vx + base, bytes, bar);
    if (r.rVY >= 0) {
        bulk_load(dst + r.rVY * rp, in.vy + base, bytes, bar);
        bulk_load(dst + (r.rVY + 1) * rp, in.vy + base + m.sj, bytes, bar);
    }
    if (r.rVZ >= 0) {
        bulk_load(dst + r.rVZ * rp, in.vz + base, bytes, bar);
        bulk_load(dst + (r.rVZ + 1) * rp, in.vz + base + m.sk, bytes, bar);
    }
}

template <typename T, int C>
__device__ __forceinline__ void tx_compute(const MeshD &m, const Tab<T> &tb, const QSet<T> &out, int ring, T *buf,
                                           T v0hi, T v0lo, T dt)
{
    const int nx = m.nx, nq = out.nq, rp = ring_row(m.sj);
    const TxRows rw = tx_rows(m);
    ring_frame(buf, rw.n, rp, nx);
    const T *sm = buf + kRingLead;   // cell i of staged row r: sm[r * rp + i], -kRingLead <= i < nx + kRingTail
    const int j = ring % m.nyt, k = ring / m.nyt;
    const bool active = j >= m.j0 && j < m.j1 && k >= m.k0 && k < m.k1;
    const idx_t base = IX(m, 0, j, k);
    const bool adi = !m.iso;
    const bool sweep = active && m.hasX;
    // the frame term of the X momentum: R^2 Omega_f, or the Cartesian table (shearing sheet)
    const T R = tb.R[ring], fz = tb.fz[ring];
    // the X momenta's frame term, or none in the reference form (they are
    // then held as rho R (v_x - vref), with v_x - vref the stored value)
    const T w = sizeof(T) == 4 && tb.vref ? T(0) : (m.geom == CART ? tb.wfr[ring] : R * R * tb.omega);
    const T *Rho = sm, *Vx = sm + (size_t)rw.rVX * rp;
    // ratio of quantity q to the density at cell i, as scale * row[i + off] +
    // shift (or e / rho), for the order rho, e, Pi-x, Pi+x, Pi-y, Pi+y,
    // Pi-z, Pi+z of the present components
    struct RatioSpec {
        const T *row;
        int off, div;
        T a, b;
    };
    auto spec = [&](int q) -> RatioSpec {
        if (q == 0) return {Rho, 0, 0, T(1), T(0)};
        int o = q - 1;
        if (adi) {
            if (o == 0) return {sm + (size_t)rw.rE * rp, 0, 1, T(1), T(0)};
            o -= 1;
        }
        if (o == 0) return {Vx, 0, 0, R, w};
        if (o == 1) return {Vx, 1, 0, R, w};
        if (m.hasY) {
            if (o == 2) return {sm + (size_t)rw.rVY * rp, 0, 0, T(1), T(0)};
            if (o == 3) return {sm + (size_t)(rw.rVY + 1) * rp, 0, 0, T(1), T(0)};
            o -= 2;
        }
        if (o == 2) return {sm + (size_t)rw.rVZ * rp, 0, 0, fz, T(0)};
        return {sm + (size_t)(rw.rVZ + 1) * rp, 0, 0, fz, T(0)};
    };
    if (!sweep) {
        for (int q = 0; q < nq; q++) {
            const RatioSpec sp = spec(q);
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const T v = sp.row[i + sp.off];
                out.q[q][base + i] = q == 0 ? v : (sp.div ? v : Rho[i] * (sp.a * v + sp.b));
            }
        }
        return;
    }
    const T dX = tb.lenx[ring], S = tb.sx[ring];
    const T idX = T(1) / dX;
    const T dtVi = dt * tb.vinv[ring];
    const int i0 = threadIdx.x * C;
    if (i0 >= nx) return;
    const int cnt = min(C, nx - i0);
    T vf[C + 1], F0[C + 1];
#pragma unroll
    for (int u = 0; u <= C; u++) vf[u] = sub_split(Vx[i0 + u], v0hi, v0lo);
    T rho[C + 4];
#pragma unroll
    for (int s = 0; s < C + 4; s++) rho[s] = Rho[i0 - 2 + s];
    // unrolled over the largest quantity count: every row and output pointer
    // index is then a compile-time constant
    #pragma unroll
    for (int q = 0; q < 8; q++) {
        if (q >= nq) break;
        const RatioSpec sp = spec(q);
        const T *win = sp.row + (i0 - 2 + sp.off);
        T a[C + 4];   // ratios of cells i0-2 .. i0+C+1
#pragma unroll
        for (int s = 0; s < C + 4; s++) {
            const T v = win[s];
            a[s] = sp.div ? v / rho[s] : sp.a * v + sp.b;
        }
        T sl[C + 2];  // van Leer slopes of cells i0-1 .. i0+C
#pragma unroll
        for (int s = 0; s < C + 2; s++) sl[s] = vl_slope_i(a[s], a[s + 1], a[s + 2], idX, idX);
        T F[C + 1];
#pragma unroll
        for (int u = 0; u <= C; u++) {
            const T v = vf[u];
            const T stv = v >= T(0) ? a[u + 1] + sl[u] * (dX - v * dt) * T(0.5)
                                    : a[u + 2] - sl[u + 1] * (dX + v * dt) * T(0.5);
            if (q == 0) F0[u] = v * stv * S;
            F[u] = q == 0 ? F0[u] : F0[u] * stv;
        }
#pragma unroll
        for (int u = 0; u < C; u++)
            if (u < cnt) {
                // the stored value itself for e; the momenta are formed here (Eqs. 16-17)
                const T old = q == 0 ? a[u + 2] : (sp.div ? win[u + 2] : rho[u + 2] * a[u + 2]);
                out.q[q][base + i0 + u] = old - dtVi * (F[u + 1] - F[u]);
            }
    }
}

// Uniform orbital step of each active ring (Sec. 3.4.1, Eqs. fargo2, 28-33),
// applied after the Y and Z sweeps, in place:
//  (ii)  circular shift by N = E(v0 dt / dX) (Eq. 32): the ring is staged
//        unrotated and read at the shifted index;
//  (iii) fractional step at xi = v0 dt/dX - N with PPA interface values
//        (Eqs. 34-36 and the xi-weighted value of Sec. 3.4.1), consistent
//        transport, in the same pass.
// N and xi are FP64 (round-to-nearest intrinsics), once per ring by thread 0
// when it issues the ring's copies; a ring with N = 0 and xi = 0 is skipped.
// Shift N (modulo nx; -1 when the ring needs no work), xi in the field
// precision and the fractional velocity xi dX / dt of active ring r.
template <typename T>
__device__ __forceinline__ void orb_prepare(const MeshD &m, const Tab<T> &tb, const double *v0, const Scal *sc,
                                            int r, int &Nm, T &xs, T &vR)
{
    const int nx = m.nx, ny = m.j1 - m.j0;
    const int j = m.j0 + r % ny, k = m.k0 + r / ny;
    const int ring = k * m.nyt + j;
    const double dtd = sc->dt;
    const double X = __ddiv_rn(__dmul_rn(v0[ring], dtd), tb.lx[ring]);
    const long long N = llround(X);
    const double x = __dsub_rn(X, (double)N);
    Nm = (int)(((N % nx) + nx) % nx);
    xs = (T)x;
    vR = (T)(x * tb.lx[ring] / dtd);
    if (Nm == 0 && xs == T(0)) Nm = -1;
}

// Per-ring constants of the orbital step: the ring's first cell, its X face
// area and dt over its cell volume.
template <typename T>
__device__ __forceinline__ void orb_ring_consts(const MeshD &m, const Tab<T> &tb, T dtT, int r, RingMeta<T> &e)
{
    const int ny = m.j1 - m.j0;
    const int j = m.j0 + r % ny, k = m.k0 + r / ny;
    const int ring = k * m.nyt + j;
    e.base = IX(m, 0, j, k);
    e.S = tb.sx[ring];
    e.dtVi = dtT * tb.vinv[ring];
}

// Thread 0: copies of the nq rows of active ring r into dst (row q at
// dst + q * ring_row(pitch) + kRingLead), or a plain arrive when the ring
// needs no work (Nm < 0).
template <typename T>
__device__ __forceinline__ void orb_issue(const MeshD &m, const QSet<T> &qs, int r, int Nm, T *dst, uint64_t *bar)
{
    if (Nm < 0) {
        mbar_arrive(bar);
        return;
    }
    const int ny = m.j1 - m.j0;
    const int j = m.j0 + r % ny, k = m.k0 + r / ny;
    const idx_t base = IX(m, 0, j, k);
    const size_t rp = (size_t)ring_row(m.sj);
    const unsigned bytes = row_bytes<T>(m.nx);
    mbar_expect_tx(bar, bytes * (unsigned)qs.nq);
    for (int q = 0; q < qs.nq; q++) bulk_load(dst + kRingLead + q * rp, qs.q[q] + base, bytes, bar);
}

// Upwind PPA value through each of a thread's C+1 faces (Sec. 3.4.1, Eqs.
// 34-36 and the xi-weighted value): for xi >= 0 (POS) the donor of face u
// is the cell left of it, else the cell right of it.  a holds the ratios of
// cells i0-3 .. i0+C+2, qr the right interface values of cells i0-2 ..
// i0+C.  The donor offset is a template constant, so every array index is a
// compile-time constant and the arrays stay in registers.
template <typename T, int C, bool POS>
__device__ __forceinline__ void ppa_face_values(const T *a, const T *qr, T xi, T *stv)
{
    const T sixth = T(1.0 / 6.0);
#pragma unroll
    for (int u = 0; u <= C; u++) {
        // donor cell d = i0+u-1 (POS) or i0+u; its value a[d-(i0-3)], its
        // left value qr[d-1-(i0-2)], its right value qr[d-(i0-2)]
        constexpr int sh = POS ? -1 : 0;
        const int dd = u + sh;
        const T q0 = a[dd + 3], qm = a[dd + 2], qp = a[dd + 4];
        T l = qr[dd + 1], rr = qr[dd + 2];
        if ((qp - q0) * (q0 - qm) <= T(0)) {
            l = q0;
            rr = q0;
        } else {
            const T D = rr - l, Cc = q0 - T(0.5) * (l + rr);
            if (D * Cc > D * D * sixth) l = T(3) * q0 - T(2) * rr;
            else if (-D * D * sixth > D * Cc) rr = T(3) * q0 - T(2) * l;
        }
        const T wgt = xi * (T(1) - xi) * (T(2) * q0 - rr - l);
        stv[u] = POS ? rr + xi * (q0 - rr) + wgt : l + xi * (q0 - l) + wgt;
    }
}

template <typename T, int C>
__device__ __forceinline__ void orb_compute(const MeshD &m, const Tab<T> &tb, const QSet<T> &qs, int r, T *buf,
                                            int Nm, T xsT, T vR, T dtT)
{
    if (Nm < 0) return;
    const int nx = m.nx, nq = qs.nq, rp = ring_row(m.sj);
    ring_frame(buf, nq, rp, nx);
    const T *sm = buf + kRingLead;
    const int ny = m.j1 - m.j0;
    const int j = m.j0 + r % ny, k = m.k0 + r / ny;
    const int ring = k * m.nyt + j;
    const idx_t base = IX(m, 0, j, k);
    // cell i after the shift holds the staged cell i - N
    if (xsT == T(0)) {   // a pure shift
        for (int q = 0; q < nq; q++)
            for (int i = threadIdx.x; i < nx; i += blockDim.x)
                qs.q[q][base + i] = sm[(size_t)q * rp + wrapi(i - Nm, nx)];
        return;
    }
    const int i0 = threadIdx.x * C;
    if (i0 >= nx) return;
    const int cnt = min(C, nx - i0);
    // the thread's window, cells i0-3 .. i0+C+2 after the shift, is the
    // staged run starting at cell (i0 - 3 - N) mod nx (framed rows: no wrap)
    int b = (i0 - 3 - Nm) % nx;
    if (b < 0) b += nx;
    const T *win = sm + b;
    const T S = tb.sx[ring];
    const T dtVi = dtT * tb.vinv[ring];
    const bool pos = xsT >= T(0);
    const T xi = pos ? xsT : -xsT;
    const T sixth = T(1.0 / 6.0);
    T rinv[C + 6], rho[C + 6];
#pragma unroll
    for (int s = 0; s < C + 6; s++) {
        rho[s] = win[s];
        rinv[s] = T(1) / rho[s];
    }
    T F0[C + 1];
    // unrolled over the largest quantity count: every row and output pointer
    // index is then a compile-time constant
    #pragma unroll
    for (int q = 0; q < 8; q++) {
        if (q >= nq) break;
        const T *wq = win + (size_t)q * rp;
        T a[C + 6];   // ratios of cells i0-3 .. i0+C+2
#pragma unroll
        for (int s = 0; s < C + 6; s++) a[s] = q == 0 ? rho[s] : wq[s] * rinv[s];
        T dm[C + 4];  // Eq. 34 slopes of cells i0-2 .. i0+C+1
#pragma unroll
        for (int s = 0; s < C + 4; s++) dm[s] = ppa_dm(a[s], a[s + 1], a[s + 2]);
        T qr[C + 3];  // Eq. 35 right interface value of cells i0-2 .. i0+C
#pragma unroll
        for (int s = 0; s < C + 3; s++) qr[s] = a[s + 1] + T(0.5) * (a[s + 2] - a[s + 1]) - (dm[s + 1] - dm[s]) * sixth;
        T stv[C + 1];
        if (pos) ppa_face_values<T, C, true>(a, qr, xi, stv);
        else ppa_face_values<T, C, false>(a, qr, xi, stv);
        T F[C + 1];
#pragma unroll
        for (int u = 0; u <= C; u++) {
            if (q == 0) F0[u] = vR * stv[u] * S;
            F[u] = q == 0 ? F0[u] : F0[u] * stv[u];
        }
#pragma unroll
        for (int u = 0; u < C; u++)
            if (u < cnt) qs.q[q][base + i0 + u] = wq[3 + u] - dtVi * (F[u + 1] - F[u]);
    }
}

// The same step with the stencil halo exchanged between lanes (C >= 3).  A
// warp covers 30 C consecutive cells: lane l in 1..30 owns C of them and
// lanes 0 and 31 own the C cells just outside, only so that their
// neighbours find the halo values in registers.  Every lane evaluates its
// cells' ratios, Eq. 34 slopes and Eq. 35 interface values once; the two
// values left of a lane's cells and one right of them arrive by shuffle, and
// so does the flux through its right face, so no value is computed twice
// inside a warp.
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_dn1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Quantity loop of orb_compute_w for one upwind direction (POS: xi >= 0,
// the donor of a face is the cell left of it).
template <typename T, int C, bool POS>
__device__ __forceinline__ void orb_lanes(const QSet<T> &qs, int nq, int rp, const T *win, idx_t base, int i0,
                                          bool owner, int nx, T xi, T vR, T S, T dtVi)
{
    const T sixth = T(1.0 / 6.0);
    T rho[C], rinv[C];
#pragma unroll
    for (int s = 0; s < C; s++) {
        rho[s] = win[s];
        rinv[s] = T(1) / rho[s];
    }
    T F0[C];
    #pragma unroll
    for (int q = 0; q < 8; q++) {
        if (q >= nq) break;
        const T *wq = win + (size_t)q * rp;
        // A[x + 2]: ratio of cell x = -2 .. C (own cells 0 .. C-1)
        T A[C + 3];
#pragma unroll
        for (int s = 0; s < C; s++) A[s + 2] = q == 0 ? rho[s] : wq[s] * rinv[s];
        A[0] = shfl_up1(A[C]);
        A[1] = shfl_up1(A[C + 1]);
        A[C + 2] = shfl_dn1(A[2]);
        T dm[C + 1];   // Eq. 34 slopes of cells 0 .. C
#pragma unroll
        for (int s = 0; s < C; s++) dm[s] = ppa_dm(A[s + 1], A[s + 2], A[s + 3]);
        dm[C] = shfl_dn1(dm[0]);
        // QR[x + 2]: Eq. 35 right interface value of cell x = -2 .. C-1
        T QR[C + 2];
#pragma unroll
        for (int s = 0; s < C; s++)
            QR[s + 2] = A[s + 2] + T(0.5) * (A[s + 3] - A[s + 2]) - (dm[s + 1] - dm[s]) * sixth;
        QR[0] = shfl_up1(QR[C]);
        QR[1] = shfl_up1(QR[C + 1]);
        // upwind PPA value through the left face u of each own cell: donor
        // cell d = u-1 (POS) or u, its value, neighbours and interface values
        T F[C];
#pragma unroll
        for (int u = 0; u < C; u++) {
            constexpr int sh = POS ? -1 : 0;
            const int d = u + sh;
            const T q0 = A[d + 2], qm = A[d + 1], qp = A[d + 3];
            T l = QR[d + 1], rr = QR[d + 2];
            if ((qp - q0) * (q0 - qm) <= T(0)) {
                l = q0;
                rr = q0;
            } else {
                const T D = rr - l, Cc = q0 - T(0.5) * (l + rr);
                if (D * Cc > D * D * sixth) l = T(3) * q0 - T(2) * rr;
                else if (-D * D * sixth > D * Cc) rr = T(3) * q0 - T(2) * l;
            }
            const T wgt = xi * (T(1) - xi) * (T(2) * q0 - rr - l);
            const T stv = POS ? rr + xi * (q0 - rr) + wgt : l + xi * (q0 - l) + wgt;
            if (q == 0) F0[u] = vR * stv * S;
            F[u] = q == 0 ? F0[u] : F0[u] * stv;
        }
        const T Fr = shfl_dn1(F[0]);   // flux through the right face of the last own cell
#pragma unroll
        for (int u = 0; u < C; u++) {
            const T fr = u + 1 < C ? F[u + 1 < C ? u + 1 : u] : Fr;
            if (owner && i0 + u < nx) qs.q[q][base + i0 + u] = wq[u] - dtVi * (fr - F[u]);
        }
    }
}

// FP32 form of orb_lanes for even C, on the packed two-lane FP32 units of
// sm_100+ (one instruction adds, multiplies or fuses two pairs).  The pairs
// are the cells (s, s + C/2) of a lane: every stencil neighbour of a pair is
// then the pair at the neighbouring index, so the ratios, Eq. 34 slopes,
// Eq. 35 interface values, the monotonised face values and the fluxes are
// formed two cells per instruction with no register moves between pairs;
// comparisons and selections stay per cell.  Each value is the same IEEE
// operation sequence as in orb_lanes, rounded to nearest.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b (a + (-1) b, exact before the one rounding)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Eq. 34 slope of one cell from the pair values of its stencil.
__device__ __forceinline__ float ppa_dm_pick(float pr, float dl, float dr, float d)
{
    if (!(pr > 0.f)) return 0.f;
    const float mn = fminf(2.f * fminf(fabsf(dl), fabsf(dr)), fabsf(d));
    return d > 0.f ? mn : -mn;
}
__device__ __forceinline__ float2 ppa_dm2(float2 qm, float2 q0, float2 qp)
{
    const float2 dr = sub2(qp, q0), dl = sub2(q0, qm);
    const float2 pr = mul2(dr, dl);
    const float2 d = mul2(pk(0.5f), sub2(qp, qm));
    return pk(ppa_dm_pick(pr.x, dl.x, dr.x, d.x), ppa_dm_pick(pr.y, dl.y, dr.y, d.y));
}

template <int C, bool POS>
__device__ __forceinline__ void orb_lanes2(const QSet<float> &qs, int nq, int rp, const float *win, idx_t base,
                                           int i0, bool owner, int nx, float xi, float vR, float S, float dtVi)
{
    static_assert(C % 2 == 0 && C >= 4, "pairs (s, s + C/2) need an even chunk of at least 4");
    constexpr int H = C / 2;
    const float2 sixth2 = pk(1.f / 6.f), half2 = pk(0.5f), nhalf2 = pk(-0.5f);
    const float2 ntwo2 = pk(-2.f), three2 = pk(3.f);
    const float2 xi2 = pk(xi), xx2 = pk(xi * (1.f - xi)), vR2 = pk(vR), S2 = pk(S), ndt2 = pk(-dtVi);
    float2 RI[H];   // reciprocal densities of the pairs
#pragma unroll
    for (int s = 0; s < H; s++) RI[s] = pk(1.f / win[s], 1.f / win[s + H]);
    float2 F0[H];
    #pragma unroll
    for (int q = 0; q < 8; q++) {
        if (q >= nq) break;
        const float *wq = win + (size_t)q * rp;
        // AA[k] = (A[k], A[k + H]): ratios of cells k-2 and k-2+H, k = 0 .. H+2
        float2 AA[H + 3];
#pragma unroll
        for (int s = 0; s < H; s++) {
            const float2 w = pk(wq[s], wq[s + H]);
            AA[s + 2] = q == 0 ? w : mul2(w, RI[s]);
        }
        AA[0] = pk(shfl_up1(AA[H].y), AA[H].x);
        AA[1] = pk(shfl_up1(AA[H + 1].y), AA[H + 1].x);
        AA[H + 2] = pk(AA[2].y, shfl_dn1(AA[2].x));
        // DM[k] = (dm[k], dm[k + H]): Eq. 34 slopes of cells k and k+H
        float2 DM[H + 1];
#pragma unroll
        for (int k = 0; k < H; k++) DM[k] = ppa_dm2(AA[k + 1], AA[k + 2], AA[k + 3]);
        DM[H] = pk(DM[0].y, shfl_dn1(DM[0].x));
        // QQ[k] = (QR[k], QR[k + H]): Eq. 35 right interface values of cells k-2, k-2+H
        float2 QQ[H + 2];
#pragma unroll
        for (int k = 2; k < H + 2; k++)
            QQ[k] = fma2(sub2(DM[k - 2], DM[k - 1]), sixth2, fma2(half2, sub2(AA[k + 1], AA[k]), AA[k]));
        QQ[0] = pk(shfl_up1(QQ[H].y), QQ[H].x);
        QQ[1] = pk(shfl_up1(QQ[H + 1].y), QQ[H + 1].x);
        // upwind PPA values through the left faces u and u+H of the pair
        float2 FF[H];
#pragma unroll
        for (int u = 0; u < H; u++) {
            constexpr int sh = POS ? 0 : 1;
            const float2 q0 = AA[u + 1 + sh], qm = AA[u + sh], qp = AA[u + 2 + sh];
            const float2 l = QQ[u + sh], rr = QQ[u + 1 + sh];
            const float2 pr = mul2(sub2(qp, q0), sub2(q0, qm));
            const float2 D = sub2(rr, l);
            const float2 Cc = fma2(nhalf2, add2(l, rr), q0);
            const float2 DC = mul2(D, Cc), DD6 = mul2(mul2(D, D), sixth2);
            const float2 q3 = mul2(three2, q0);
            const float2 ln = fma2(ntwo2, rr, q3), rn = fma2(ntwo2, l, q3);
            float2 L, R;
            {
                const bool ext = pr.x <= 0.f, c1 = DC.x > DD6.x, c2 = -DD6.x > DC.x;
                L.x = ext ? q0.x : (c1 ? ln.x : l.x);
                R.x = ext ? q0.x : (!c1 && c2 ? rn.x : rr.x);
            }
            {
                const bool ext = pr.y <= 0.f, c1 = DC.y > DD6.y, c2 = -DD6.y > DC.y;
                L.y = ext ? q0.y : (c1 ? ln.y : l.y);
                R.y = ext ? q0.y : (!c1 && c2 ? rn.y : rr.y);
            }
            const float2 wgt = mul2(xx2, sub2(sub2(add2(q0, q0), R), L));
            const float2 stv = POS ? add2(fma2(xi2, sub2(q0, R), R), wgt) : add2(fma2(xi2, sub2(q0, L), L), wgt);
            if (q == 0) F0[u] = mul2(mul2(vR2, stv), S2);
            FF[u] = q == 0 ? F0[u] : mul2(F0[u], stv);
        }
        const float Fr = shfl_dn1(FF[0].x);   // flux through the right face of the last own cell
        float *out = qs.q[q] + base + i0;
#pragma unroll
        for (int u = 0; u < H; u++) {
            const float2 fr = u + 1 < H ? FF[u + 1 < H ? u + 1 : u] : pk(FF[0].y, Fr);
            // (the staged values again: they are the cells' old values)
            const float2 v = fma2(ndt2, sub2(fr, FF[u]), pk(wq[u], wq[u + H]));
            if (owner && i0 + u < nx) out[u] = v.x;
            if (owner && i0 + u + H < nx) out[u + H] = v.y;
        }
    }
}

// The orbital step's form per cells-per-thread class: the lane-exchange form
// for C = 3, 4, 6; the per-thread form for C = 1, 2 (too few cells for the
// halo lanes) and C = 8 (rings beyond 2880 cells, too long for the halo
// lanes' thread count).
template <int C>
__host__ __device__ constexpr bool orb_uses_lanes()
{
    return C >= 3 && C <= 6;
}

// Launch bounds of the orbital kernels per chunk: the FP32 lane form's
// packed stencils of C = 4 and 6 get 72 registers (no spills) under a lower
// thread cap that keeps the CTAs per SM of the 64-register budget; ring_chunk
// keeps every ring within its chunk's cap.
__host__ __device__ constexpr int orb_max_threads(int C) { return C == 6 ? 288 : (C == 4 ? 416 : 512); }
__host__ __device__ constexpr int orb_min_blocks(int C) { return C == 6 ? 3 : 2; }
__host__ __device__ constexpr int orb_regs(int C) { return C == 4 || C == 6 ? 72 : 64; }

template <typename T, int C>
__device__ __forceinline__ void orb_compute_w(const QSet<T> &qs, int nx, int rp, const RingMeta<T> &e, T *buf)
{
    // the left halo of a lane's interface values reaches three cells back,
    // and the halo lanes must own those cells: C >= 3
    static_assert(orb_uses_lanes<C>(), "the halo lanes need three cells");
    const int Nm = e.N;
    if (Nm < 0) return;
    const int nq = qs.nq;
    ring_frame(buf, nq, rp, nx);
    const T *sm = buf + kRingLead;
    const idx_t base = e.base;
    const T xsT = e.a, vR = e.b;
    if (xsT == T(0)) {   // a pure shift
        for (int q = 0; q < nq; q++)
            for (int i = threadIdx.x; i < nx; i += blockDim.x)
                qs.q[q][base + i] = sm[(size_t)q * rp + wrapi(i - Nm, nx)];
        return;
    }
    const int lane = threadIdx.x & 31;
    const int i0 = (int)(threadIdx.x >> 5) * (30 * C) + (lane - 1) * C;
    const bool owner = lane >= 1 && lane <= 30;
    // cells i0 .. i0+C-1 after the shift: the staged run from (i0 - N) mod nx
    int b = (i0 - Nm) % nx;
    if (b < 0) b += nx;
    const bool pos = xsT >= T(0);
    const T xi = pos ? xsT : -xsT;
    if constexpr (sizeof(T) == 4 && C % 2 == 0) {
        if (pos) orb_lanes2<C, true>(qs, nq, rp, sm + b, base, i0, owner, nx, xi, vR, e.S, e.dtVi);
        else orb_lanes2<C, false>(qs, nq, rp, sm + b, base, i0, owner, nx, xi, vR, e.S, e.dtVi);
    } else {
        if (pos) orb_lanes<T, C, true>(qs, nq, rp, sm + b, base, i0, owner, nx, xi, vR, e.S, e.dtVi);
        else orb_lanes<T, C, false>(qs, nq, rp, sm + b, base, i0, owner, nx, xi, vR, e.S, e.dtVi);
    }
}

// Single-instance ring operations for ring_pipeline (meta: the per-iteration
// table in shared memory).
template <typename T, int C>
struct TxOp {
    const MeshD &m;
    const Tab<T> &tb;
    const Fld<T> &in;
    const QSet<T> &out;
    const double *v0;
    Scal *sc;
    T dt;
    RingMeta<T> *meta;
    __device__ void prepare(int it, int ring)
    {
        meta[it].local = ring;
        tx_v0(m, tb, v0, ring, meta[it].a, meta[it].b);
    }
    __device__ void issue(int it, T *dst, uint64_t *bar) { tx_issue(m, in, meta[it].local, dst, bar); }
    __device__ void compute(int it, T *src)
    {
        tx_compute<T, C>(m, tb, out, meta[it].local, src, meta[it].a, meta[it].b, dt);
    }
    __device__ void fail(int) { atomicOr(&sc->err, kErrTimeout); }
};

template <typename T, int C>
struct OrbOp {
    const MeshD &m;
    const Tab<T> &tb;
    const QSet<T> &qs;
    const double *v0;
    Scal *sc;
    T dt;
    RingMeta<T> *meta;
    __device__ void prepare(int it, int r)
    {
        meta[it].local = r;
        orb_prepare(m, tb, v0, sc, r, meta[it].N, meta[it].a, meta[it].b);
        orb_ring_consts(m, tb, dt, r, meta[it]);
    }
    __device__ void issue(int it, T *dst, uint64_t *bar) { orb_issue(m, qs, meta[it].local, meta[it].N, dst, bar); }
    __device__ void compute(int it, T *src)
    {
        const RingMeta<T> &e = meta[it];
        if constexpr (orb_uses_lanes<C>()) orb_compute_w<T, C>(qs, m.nx, ring_row(m.sj), e, src);
        else orb_compute<T, C>(m, tb, qs, e.local, src, e.N, e.a, e.b, dt);
    }
    __device__ void fail(int) { atomicOr(&sc->err, kErrTimeout); }
};

// Dynamic shared memory of a ring kernel: nbuf (2, or 1 for rings too long
// for two) ring buffers of `stride` values, then the per-iteration table.
template <typename T>
__device__ __forceinline__ RingMeta<T> *ring_meta(unsigned char *smem, int stride, int nbuf)
{
    return reinterpret_cast<RingMeta<T> *>(smem + (size_t)nbuf * stride * sizeof(T));
}

// The parameters are __grid_constant__: the ring operations hold references
// to them, which then point into the parameter bank instead of a local copy.
template <typename T, int C>
__global__ void __launch_bounds__(512, 2)
    k_transport_x(const __grid_constant__ MeshD m, const __grid_constant__ Tab<T> tb, const __grid_constant__ Fld<T> in,
                  const __grid_constant__ QSet<T> out, const double *v0, Scal *sc, int stride, int nbuf)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    ring_bars_init(bar);
    TxOp<T, C> op{m, tb, in, out, v0, sc, dt, ring_meta<T>(smem_raw, stride, nbuf)};
    ring_pipeline<T>(op, reinterpret_cast<T *>(smem_raw), (size_t)stride, bar, blockIdx.x, gridDim.x,
                     m.nyt * m.nzt, nbuf);
}

template <typename T, int C>
__global__ void __launch_bounds__(orb_max_threads(C), orb_min_blocks(C))
    k_orbital(const __grid_constant__ MeshD m, const __grid_constant__ Tab<T> tb, const __grid_constant__ QSet<T> qs,
              const double *v0, Scal *sc, int nrings, int stride, int nbuf)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    ring_bars_init(bar);
    OrbOp<T, C> op{m, tb, qs, v0, sc, dt, ring_meta<T>(smem_raw, stride, nbuf)};
    ring_pipeline<T>(op, reinterpret_cast<T *>(smem_raw), (size_t)stride, bar, blockIdx.x, gridDim.x, nrings,
                     nbuf);
}

// Cells per thread of a ring kernel whose CTA stages `rows` rows of `pitch`
// values of esz bytes in two buffers.  Larger chunks recompute less of the
// stencil halo per cell but leave fewer threads per ring, and the staging
// decides how many CTAs share an SM: take the largest of 1, 2, 3, 4, 6 that
// keeps the ring within 512 threads, at 192 threads or more (below that the
// per-ring staging and barriers dominate), and at least 24 warps resident per
// SM (228 KB of shared memory, 64 registers a thread), else the smallest
// that fits; 8 (which spills) only for rings above 3072 cells.
// Threads of a ring kernel with C cells per thread: C cells per lane, or
// (halo, C = 3..6) warps of 30 C cells, lanes 0 and 31 holding the
// neighbours' halo (the orbital step's lane-exchange form).
static inline int ring_threads(int nx, int C, bool halo)
{
    return halo && C >= 3 && C <= 6 ? 32 * ((nx + 30 * C - 1) / (30 * C)) : ((nx + C - 1) / C + 31) / 32 * 32;
}

static inline int ring_chunk(int nx, int rows, int pitch, int esz, bool halo, int nbuf)
{
    const int cs[6] = {1, 2, 3, 4, 6, 8};
    const size_t smem = (size_t)nbuf * rows * ring_row(pitch) * esz + 2048;
    int best = 0;
    for (int c : cs) {
        const int th = ring_threads(nx, c, halo);
        if (th > (halo ? orb_max_threads(c) : 512)) continue;
        if (c == 8 && best) break;
        if (th < 192 && best) break;
        int per = (int)(233472 / smem);
        per = std::min(per, 2048 / th);
        per = std::min(per, 65536 / ((halo ? orb_regs(c) : 64) * th));
        per = std::min(per, 32);
        if (best == 0 || per * th >= 768) best = c;
    }
    return best;
}

// Launch shape of a ring kernel: threads per CTA, values per ring buffer,
// dynamic shared memory (two buffers) and the persistent grid.
struct RingShape {
    int threads, stride, grid;
    size_t smem;
    int chunk;   // cells per thread (ring_chunk)
    int nbuf;    // ring buffers: 2 (double buffering), 1 when two do not fit
};

// Ring buffers of a ring kernel staging `stride` values of esz bytes.  The
// orbital step (halo: the heavier per-cell work) double-buffers while two
// buffers and the per-iteration table fit the 227 KB a CTA can have: its
// CTAs need their own prefetch.  The X sweep stages one ring at a time: its
// lighter work leaves the copy latency to the other CTAs on the SM, which
// the halved staging admits (measured on the 3D disk: 1.37 -> 1.19 ms; on
// the 256-disk sweep 1.27 -> 1.21 ms; the orbital step there went
// 1.54 -> 2.09 ms with one buffer).
static inline int ring_nbuf(int stride, int esz, bool halo)
{
    return halo && 2 * (size_t)stride * esz + 4096 <= 232448 ? 2 : 1;
}

template <typename T, int C>
static void launch_tx_c(const MeshD &m, const Tab<T> &tb, const Fld<T> &in, const QSet<T> &out, const double *v0,
                        Scal *sc, const RingShape &rs, cudaStream_t s)
{
    k_transport_x<T, C><<<rs.grid, rs.threads, rs.smem, s>>>(m, tb, in, out, v0, sc, rs.stride, rs.nbuf);
}
template <typename T, int C>
static void launch_orb_c(const MeshD &m, const Tab<T> &tb, const QSet<T> &qs, const double *v0, Scal *sc,
                         int nrings, const RingShape &rs, cudaStream_t s)
{
    k_orbital<T, C><<<rs.grid, rs.threads, rs.smem, s>>>(m, tb, qs, v0, sc, nrings, rs.stride, rs.nbuf);
}

template <typename T>
static void launch_tx(const MeshD &m, const Tab<T> &tb, const Fld<T> &in, const QSet<T> &out, const double *v0,
                      Scal *sc, const RingShape &rs, cudaStream_t s)
{
    switch (rs.chunk) {
    case 1: launch_tx_c<T, 1>(m, tb, in, out, v0, sc, rs, s); break;
    case 2: launch_tx_c<T, 2>(m, tb, in, out, v0, sc, rs, s); break;
    case 3: launch_tx_c<T, 3>(m, tb, in, out, v0, sc, rs, s); break;
    case 4: launch_tx_c<T, 4>(m, tb, in, out, v0, sc, rs, s); break;
    case 6: launch_tx_c<T, 6>(m, tb, in, out, v0, sc, rs, s); break;
    default: launch_tx_c<T, 8>(m, tb, in, out, v0, sc, rs, s); break;
    }
}
// Threads, buffer stride and shared memory of a ring kernel for rings of up
// to nx cells staged as `rows` rows of `pitch` values (halo: the thread
// count of ring_threads); the persistent grid is filled in by ring_grid.
template <typename T>
static RingShape ring_shape(int nx, int rows, int pitch, bool halo)
{
    RingShape rs{};
    rs.stride = rows * ring_row(pitch);
    rs.nbuf = ring_nbuf(rs.stride, (int)sizeof(T), halo);
    const int C = ring_chunk(nx, rows, pitch, (int)sizeof(T), halo, rs.nbuf);
    rs.chunk = C;
    rs.threads = C ? ring_threads(nx, C, halo) : 0;
    rs.smem = (size_t)rs.nbuf * rs.stride * sizeof(T);
    return rs;
}

// Raise (never lower) a kernel's dynamic shared-memory cap: the cap is per
// function and process-wide, so lowering it for one context would break
// another context's launches.
template <typename F>
static cudaError_t raise_smem_cap(F *func, size_t bytes)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Persistent grid of a ring kernel: the CTAs resident on the whole GPU, at
// most one per item.  The dynamic shared memory is the two ring buffers
// plus the per-iteration table, whose length depends on the grid, so the
// grid and the memory are settled together (the memory only grows as the
// grid shrinks).  The kernel's shared-memory cap is raised accordingly.
template <typename T, typename K>
static cudaError_t ring_grid(K *kernel, RingShape &rs, int nitems)
{
    int dev = 0, sms = 0, maxsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t bufs = (size_t)rs.nbuf * rs.stride * sizeof(T);
    const int n = nitems > 0 ? nitems : 1;
    int grid = n;
    for (int pass = 0; pass < 4; pass++) {
        const size_t smem = bufs + (size_t)ring_iters(n, grid) * sizeof(RingMeta<T>);
        if (smem > (size_t)maxsm) return cudaErrorInvalidValue;
        if ((e = raise_smem_cap(kernel, smem)) != cudaSuccess) return e;
        int per = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, rs.threads, smem)) != cudaSuccess)
            return e;
        const long long g = (long long)(per > 0 ? per : 1) * sms;
        if (g >= grid) break;
        grid = (int)g;
    }
    rs.grid = grid;
    rs.smem = bufs + (size_t)ring_iters(n, grid) * sizeof(RingMeta<T>);
    if (rs.smem > (size_t)maxsm) return cudaErrorInvalidValue;
    return raise_smem_cap(kernel, rs.smem);
}

template <typename T>
static void launch_orb(const MeshD &m, const Tab<T> &tb, const QSet<T> &qs, const double *v0, Scal *sc,
                       int nrings, const RingShape &rs, cudaStream_t s)
{
    switch (rs.chunk) {
    case 1: launch_orb_c<T, 1>(m, tb, qs, v0, sc, nrings, rs, s); break;
    case 2: launch_orb_c<T, 2>(m, tb, qs, v0, sc, nrings, rs, s); break;
    case 3: launch_orb_c<T, 3>(m, tb, qs, v0, sc, nrings, rs, s); break;
    case 4: launch_orb_c<T, 4>(m, tb, qs, v0, sc, nrings, rs, s); break;
    case 6: launch_orb_c<T, 6>(m, tb, qs, v0, sc, nrings, rs, s); break;
    default: launch_orb_c<T, 8>(m, tb, qs, v0, sc, nrings, rs, s); break;
    }
}

// ---------------------------------------------------------------------------
// Y and Z sweeps (Eqs. 1D-advection-Y/Z) with TMA staging.  A CTA owns a tile
// of TW consecutive azimuths (one 512-byte row segment per quantity) of one
// transverse index and a segment of the sweep axis.  A producer thread
// streams the rows of the segment and its 2+2 halo rows, every quantity plus
// the face velocity, into an S-stage ring of shared memory with 3D
// tensor-map loads completed on an mbarrier.  The TW consumer threads own one
// column each and march it with a register window: at cell p a thread holds
// the ratios Q/rho of rows p..p+2, the van Leer slope of cell p and the flux
// through its lower face; it forms the slope of cell p+1 and the flux through
// the upper face, updates cell p, slides the window and releases the row's
// stage through a second mbarrier.  Each face flux and slope is computed
// once; consistent transport (ratio to density times the mass flux), all
// fluxes from the pre-sweep values.  Rows outside the active range come from
// `maps.qg` (the ghost source).  Every wait is bounded: on timeout the CTA
// records kErrTimeout and returns after its copies in flight have landed.
// ---------------------------------------------------------------------------
struct SweepMaps {
    CUtensorMap qin[8];
    CUtensorMap qg[8];
    CUtensorMap vel;
};

template <typename T>
struct TmaTile {
    static constexpr int TW = 512 / (int)sizeof(T);   // 128 floats or 64 doubles per row segment
    static constexpr int S = 8;                       // pipeline stages
};

template <typename T, int AXIS, int NQ>
__device__ __forceinline__ void sweep_body(const MeshD &m, const Tab<T> &tb, const SweepMaps &maps,
                                           const QSet<T> &out, Scal *sc, int seglen, int bid)
{
    constexpr int TW = TmaTile<T>::TW, S = TmaTile<T>::S, NW = TW / 32;
    constexpr int ROW = (NQ + 1) * TW;                // values per stage
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *stage = reinterpret_cast<T *>(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    const T dt = step_dt<T>(sc);
    if (!(dt > T(0))) return;
    const int p0 = AXIS == 1 ? m.j0 : m.k0, pN = AXIS == 1 ? m.j1 : m.k1;
    const int n2 = AXIS == 1 ? m.k1 - m.k0 : m.j1 - m.j0;
    const int ntx = (m.nx + TW - 1) / TW;
    const int bx = bid % ntx;
    const int rest = bid / ntx;
    const int c2 = (AXIS == 1 ? m.k0 : m.j0) + rest % n2;
    const int seg = rest / n2;
    const int ps = p0 + seg * seglen, pe = min(ps + seglen, pN);
    const int nrows = pe - ps + 4;                    // rows ps-2 .. pe+1
    const int x0 = bx * TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (warp == NW) {
        // ---------------- producer ----------------
        if (lane != 0) return;
        for (int q = 0; q < NQ; q++) prefetch_tensormap(&maps.qin[q]);
        prefetch_tensormap(&maps.vel);
        bool ok = true;
        int issued = 0;
        for (int r = 0; r < nrows && ok; r++) {
            const int slot = r % S;
            if (r >= S && !mbar_wait(&empty[slot], ((r / S) - 1) & 1)) {
                ok = false;
                break;
            }
            const int p = ps - 2 + r;
            const bool ghost = p < p0 || p >= pN;
            mbar_expect_tx(&full[slot], (unsigned)(ROW * sizeof(T)));
            T *dst = stage + (size_t)slot * ROW;
            const int y = AXIS == 1 ? p : c2, z = AXIS == 1 ? c2 : p;
#pragma unroll
            for (int q = 0; q < NQ; q++) tma_load_3d(dst + q * TW, ghost ? &maps.qg[q] : &maps.qin[q], x0, y, z, &full[slot]);
            tma_load_3d(dst + NQ * TW, &maps.vel, x0, y, z, &full[slot]);
            issued = r + 1;
        }
        if (!ok) atomicOr(&sc->err, kErrTimeout);
        // let every copy in flight land before the CTA can exit
        for (int r = issued > S ? issued - S : 0; r < issued; r++) mbar_wait(&full[r % S], (r / S) & 1);
        return;
    }
    // ---------------- consumers: one column each ----------------
    const int i = x0 + threadIdx.x;
    const bool col = i < m.nx;
    const idx_t st = AXIS == 1 ? m.sj : m.sk;
    const idx_t base = AXIS == 1 ? IX(m, col ? i : 0, 0, c2) : IX(m, col ? i : 0, c2, 0);
    auto ring_of = [&](int p) { return AXIS == 1 ? c2 * m.nyt + p : p * m.nyt + c2; };
    auto icd = [&](int f) -> T { return AXIS == 1 ? tb.idyc[f] : tb.idzc[f * m.nyt + c2]; };
    auto width = [&](int d) -> T { return AXIS == 1 ? tb.dy[d] : tb.lenz[d * m.nyt + c2]; };
    auto area = [&](int f) -> T { return AXIS == 1 ? tb.sy[c2 * (m.nyt + 1) + f] : tb.sz[f * (m.nyt + 1) + c2]; };
    // Reference form of the X momenta (FP32): row p holds Pi - rho A(p).  The
    // cell update of row p works in the frame of row p: the ratios of rows
    // p +- 1, 2 are shifted by the differences of A across the faces between
    // (dA(f) = A(f) - A(f - 1) at face f), and a face flux computed in the
    // frame of the row below moves to the frame of the row above by
    // subtracting the mass flux times dA.  Other quantities are not shifted.
    // The X momenta are quantities QX and QX + 1: after rho and, for an
    // adiabatic gas, e; the quantity count is odd exactly when the gas is
    // isothermal (rho, then pairs of momenta).
    constexpr int QX = NQ % 2 == 1 ? 1 : 2;
    const bool rf = sizeof(T) == 4 && tb.dAy != nullptr;
    auto dA = [&](int f) -> T { return !rf ? T(0) : (AXIS == 1 ? tb.dAy[c2 * m.nyt + f] : tb.dAz[f * m.nyt + c2]); };
    auto isx = [](int q) { return q == QX || q == QX + 1; };
    auto sh = [&](int q, T d) -> T { return isx(q) ? d : T(0); };
    bool ok = true;
    // fetch row r into ratios + face velocity, then release the stage (the
    // update starts from ratio x density: measured against the stored value
    // itself, the FP32 error after 10 orbits of the 768 x 256 disk is the
    // same, and holding the stages until the update slowed the sweeps)
    auto fetch = [&](int r, T *rat, T &vface) {
        const int slot = r % S;
        if (!mbar_wait(&full[slot], (r / S) & 1)) {
            ok = false;
            return;
        }
        const T *src = stage + (size_t)slot * ROW + threadIdx.x;
        const T rho = src[0];
        const T ri = T(1) / rho;
        rat[0] = rho;
#pragma unroll
        for (int q = 1; q < NQ; q++) rat[q] = src[q * TW] * ri;
        vface = src[NQ * TW];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    };
    T Rm2[NQ], Rm1[NQ], R0[NQ], R1[NQ], R2[NQ], aP[NQ], Flo[NQ];
    T vm2, vm1, v0f, v1f, v2f;
    fetch(0, Rm2, vm2);
    fetch(1, Rm1, vm1);
    fetch(2, R0, v0f);
    fetch(3, R1, v1f);
    fetch(4, R2, v2f);
    if (!ok) {
        atomicOr(&sc->err, kErrTimeout);
        return;
    }
    (void)vm2;
    (void)vm1;
    {
        const T d0 = icd(ps - 1), d1 = icd(ps), d2 = icd(ps + 1);
        const T v = v0f;   // face ps
        const T wl = width(ps - 1), wr = width(ps);
        const T Sa = area(ps);
        T F0 = 0;
        const T e0 = dA(ps - 1), e1 = dA(ps), e2 = dA(ps + 1);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const T s0 = sh(q, e0), s1 = sh(q, e1), s2 = sh(q, e2);
            const T am = vl_slope_d((Rm1[q] - Rm2[q]) + s0, (R0[q] - Rm1[q]) + s1, d0, d1);
            const T a0 = vl_slope_d((R0[q] - Rm1[q]) + s1, (R1[q] - R0[q]) + s2, d1, d2);
            aP[q] = a0;
            // interface value in the frame of row ps - 1
            const T stv = v >= T(0) ? Rm1[q] + am * (wl - v * dt) * T(0.5) : (R0[q] + s1) - a0 * (wr + v * dt) * T(0.5);
            if (q == 0) F0 = v * stv * Sa;
            const T Fup = q == 0 ? F0 : mul_rn(F0, stv);
            Flo[q] = rf && isx(q) ? fma_rn(-F0, s1, Fup) : Fup;   // in the frame of row ps
        }
    }
    // frame shifts of faces p + 1 and p + 2; the next ones are loaded two
    // iterations ahead (a load per row, off the critical path)
    T e1 = dA(ps + 1), e2 = dA(ps + 2), e3 = ps + 2 <= pe ? dA(ps + 3) : T(0);
    for (int p = ps; p < pe; p++) {
        const T e4 = p + 3 <= pe ? dA(p + 4) : T(0);   // face p + 4 <= pe + 1, inside the table
        const T v = v1f;   // face p+1
        const T dn = icd(p + 1), dnn = icd(p + 2);
        const T wp = width(p), wn = width(p + 1);
        const T Sa = area(p + 1);
        const T dtVi = dt * tb.vinv[ring_of(p)];
        const T rho = R0[0];
        const idx_t c = base + p * st;
        T F0 = 0;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const T s1 = sh(q, e1), s2 = sh(q, e2);
            const T aN = vl_slope_d((R1[q] - R0[q]) + s1, (R2[q] - R1[q]) + s2, dn, dnn);
            // interface value and flux in the frame of row p
            const T stv = v >= T(0) ? R0[q] + aP[q] * (wp - v * dt) * T(0.5) : (R1[q] + s1) - aN * (wn + v * dt) * T(0.5);
            if (q == 0) F0 = v * stv * Sa;
            const T Fup = q == 0 ? F0 : mul_rn(F0, stv);
            const T Q = q == 0 ? rho : R0[q] * rho;
            if (col) out.q[q][c] = Q - dtVi * (Fup - Flo[q]);
            Flo[q] = rf && isx(q) ? fma_rn(-F0, s1, Fup) : Fup;   // in the frame of row p + 1
            aP[q] = aN;
        }
        e1 = e2;
        e2 = e3;
        e3 = e4;
        if (p + 1 < pe) {
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                R0[q] = R1[q];
                R1[q] = R2[q];
            }
            v0f = v1f;
            v1f = v2f;
            fetch(p - ps + 5, R2, v2f);   // row p+3
            if (!ok) {
                atomicOr(&sc->err, kErrTimeout);
                return;
            }
        }
    }
}

template <typename T, int AXIS, int NQ>
__global__ void __launch_bounds__(TmaTile<T>::TW + 32) k_sweep_tma(MeshD m, Tab<T> tb,
                                                                    const __grid_constant__ SweepMaps maps,
                                                                    QSet<T> out, Scal *sc, int seglen)
{
    sweep_body<T, AXIS, NQ>(m, tb, maps, out, sc, seglen, blockIdx.x);
}

// Segment length of a sweep over np active rows.
static inline int sweep_seglen(int np) { return np > 96 ? 64 : np; }

template <typename T, int AXIS>
static size_t sweep_tma_smem(int nq)
{
    return (size_t)TmaTile<T>::S * (nq + 1) * TmaTile<T>::TW * sizeof(T);
}

template <typename T, int AXIS>
static void launch_sweep_tma(const MeshD &m, const Tab<T> &tb, const SweepMaps &maps, const QSet<T> &out,
                             Scal *sc, int nq, cudaStream_t s, int seglen = 0)
{
    constexpr int TW = TmaTile<T>::TW;
    const int np = AXIS == 1 ? m.j1 - m.j0 : m.k1 - m.k0;
    const int n2 = AXIS == 1 ? m.k1 - m.k0 : m.j1 - m.j0;
    if (seglen <= 0) seglen = sweep_seglen(np);
    const int nseg = (np + seglen - 1) / seglen;
    const int ntx = (m.nx + TW - 1) / TW;
    const unsigned g = (unsigned)ntx * n2 * nseg;
    const size_t sm = sweep_tma_smem<T, AXIS>(nq);
    switch (nq) {
    case 3: k_sweep_tma<T, AXIS, 3><<<g, TW + 32, sm, s>>>(m, tb, maps, out, sc, seglen); break;
    case 4: k_sweep_tma<T, AXIS, 4><<<g, TW + 32, sm, s>>>(m, tb, maps, out, sc, seglen); break;
    case 5: k_sweep_tma<T, AXIS, 5><<<g, TW + 32, sm, s>>>(m, tb, maps, out, sc, seglen); break;
    case 6: k_sweep_tma<T, AXIS, 6><<<g, TW + 32, sm, s>>>(m, tb, maps, out, sc, seglen); break;
    case 7: k_sweep_tma<T, AXIS, 7><<<g, TW + 32, sm, s>>>(m, tb, maps, out, sc, seglen); break;
    default: k_sweep_tma<T, AXIS, 8><<<g, TW + 32, sm, s>>>(m, tb, maps, out, sc, seglen); break;
    }
}

template <typename T, int AXIS>
static cudaError_t sweep_tma_attrs(int nq)
{
    const int a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int sm = (int)sweep_tma_smem<T, AXIS>(nq);
    switch (nq) {
    case 3: return cudaFuncSetAttribute(k_sweep_tma<T, AXIS, 3>, (cudaFuncAttribute)a, sm);
    case 4: return cudaFuncSetAttribute(k_sweep_tma<T, AXIS, 4>, (cudaFuncAttribute)a, sm);
    case 5: return cudaFuncSetAttribute(k_sweep_tma<T, AXIS, 5>, (cudaFuncAttribute)a, sm);
    case 6: return cudaFuncSetAttribute(k_sweep_tma<T, AXIS, 6>, (cudaFuncAttribute)a, sm);
    case 7: return cudaFuncSetAttribute(k_sweep_tma<T, AXIS, 7>, (cudaFuncAttribute)a, sm);
    default: return cudaFuncSetAttribute(k_sweep_tma<T, AXIS, 8>, (cudaFuncAttribute)a, sm);
    }
}

// Pointer n of a quantity set through constant indices (a runtime index into
// the parameter array would copy it to local memory).
template <typename T>
__device__ __forceinline__ T *qsel(const QSet<T> &s, int n)
{
    switch (n) {
    case 0: return s.q[0];
    case 1: return s.q[1];
    case 2: return s.q[2];
    case 3: return s.q[3];
    case 4: return s.q[4];
    case 5: return s.q[5];
    case 6: return s.q[6];
    default: return s.q[7];
    }
}

// ---------------------------------------------------------------------------
// New face velocities from the new momenta and densities (Eq. 18), undoing
// the geometric factors of Tab. "momenta", on interior faces; every other
// face is copied from the post-source velocities.  When the last sweep left
// density and energy in the scratch set, they are copied back too.  Thread 0
// advances the device time.
// ---------------------------------------------------------------------------
template <typename T, class F = CfgRun>
__device__ __forceinline__ void newvel_body(const MeshD &m, const Tab<T> &tb, const QSet<T> &fin, const Fld<T> &vsrc,
                                            const Fld<T> &state, Scal *sc, int copy_scalars, int i, int j, int k)
{
    const T dtT = step_dt<T>(sc);
    if (!(dtT > T(0))) return;
    if (i == 0 && j == 0 && k == 0) {
        sc->t = sc->t + sc->dt;
        sc->nstep += 1;
    }
    const idx_t c = IX(m, i, j, k);
    const bool jact = j >= m.j0 && j < m.j1, kact = k >= m.k0 && k < m.k1;
    const int ring = k * m.nyt + j;
    const T *rho = fin.q[0];
    const int o = F::iso(m) ? 1 : 2;   // index of Pi-x in the quantity set
    const T *pmx = F::iso(m) ? fin.q[1] : fin.q[2], *ppx = F::iso(m) ? fin.q[2] : fin.q[3];
    const int oy = o + 2, oz = o + (F::hasY(m) ? 4 : 2);
    const T *pmy = qsel(fin, oy), *ppy = qsel(fin, oy + 1);
    const T *pmz = qsel(fin, oz), *ppz = qsel(fin, oz + 1);
    // interior faces from the momenta; every other face from the post-source
    // velocities, read only there (and not at all when they are the state).
    // The three values are stored at the end: no store sits between the loads.
    T nvx = T(0), nvy = T(0), nvz = T(0);
    bool wx = false, wy = false, wz = false;
    if (j < m.nyt && k < m.nzt) {
        if (jact && kact) {
            const idx_t cm = c - i + (i == 0 ? m.nx - 1 : i - 1);
            const T R = tb.R[ring];
            // divisions, not reciprocal products: v_x is rebuilt from R v_x every
            // step, and a rounded 1/R would bias it by R (1/R) - 1 each time.
            // In the reference form the momenta hold rho (R v_x + w) - rho A with
            // A = R vref + w, so the quotient is R (v_x - vref), the stored value.
            if (sizeof(T) == 4 && tb.vref) {
                nvx = ((ppx[cm] + pmx[c]) / (rho[cm] + rho[c])) / R;
                wx = true;
            } else {
                const T w = F::geom(m) == CART ? tb.wfr[ring] : R * R * tb.omega;
                nvx = ((ppx[cm] + pmx[c]) / (rho[cm] + rho[c]) - w) / R;
                wx = true;
            }
        } else if (vsrc.vx != state.vx) {
            nvx = vsrc.vx[c];
            wx = true;
        }
    }
    if (k < m.nzt) {
        if (F::hasY(m) && j >= m.jf && j < m.j1 && kact) {
            const idx_t cm = c - m.sj;
            nvy = (ppy[cm] + pmy[c]) / (rho[cm] + rho[c]);
            wy = true;
        } else if (vsrc.vy != state.vy) {
            nvy = vsrc.vy[c];
            wy = true;
        }
    }
    if (F::hasZ(m) && j < m.nyt) {
        if (k >= m.kf && k < m.k1 && jact) {
            const idx_t cm = c - m.sk;
            nvz = (ppz[cm] + pmz[c]) / (rho[cm] + rho[c]) / tb.fz[ring];
            wz = true;
        } else if (vsrc.vz != state.vz) {
            nvz = vsrc.vz[c];
            wz = true;
        }
    }
    if (copy_scalars && j < m.nyt && k < m.nzt) {
        state.rho[c] = rho[c];
        if (!F::iso(m)) state.e[c] = fin.q[1][c];
    }
    if (wx) state.vx[c] = nvx;
    if (wy) state.vy[c] = nvy;
    if (wz) state.vz[c] = nvz;
}


template <typename T, class F = CfgRun>
__global__ void __launch_bounds__(256) k_newvel(MeshD m, Tab<T> tb, QSet<T> fin, Fld<T> vsrc, Fld<T> state,
                                                Scal *sc, int copy_scalars)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) newvel_body<T, F>(m, tb, fin, vsrc, state, sc, copy_scalars, i, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Conserved totals with compensated (Neumaier) FP64 sums: per thread, then a
// fixed-shape block tree, then a fixed-order pass over the block partials by
// the last block.  Deterministic for a given launch shape.
// ---------------------------------------------------------------------------
struct KB {
    double s, c;
};
__device__ __forceinline__ void kb_add(KB &a, double x)
{
    const double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}
__device__ __forceinline__ void kb_merge(KB &a, const KB &b)
{
    kb_add(a, b.s);
    a.c += b.c;
}

// What the sums need of a state: density, internal energy (NULL when
// isothermal), azimuthal velocity, and per ring the volume and lever arm.
template <typename T>
struct SumInput {
    const T *rho, *e, *vx;
    const double *vol, *R;
    double omega;
    int nx, j0, j1, k0, k1, nyt;
    long long sj, sk;
    const double *wfr;   // the frame term of the X momentum per ring, or null for R^2 omega
    const double *vref;  // the reference velocity per ring of the reference form (FP32), or null
};

// Per-block compensated partials of the three totals, then the last block to
// finish (ticket counter) folds the partials in block order.  `part` holds
// 6 doubles per block; `counter` starts at zero and is left at zero.
template <typename T>
__device__ void sums_reduce(const SumInput<T> &in, double *part, unsigned *counter, double *result)
{
    __shared__ KB sh[3][256];
    __shared__ int s_last;
    KB acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    const int ny = in.j1 - in.j0, nz = in.k1 - in.k0;
    const long long n = (long long)in.nx * ny * nz;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % in.nx);
        const long long r = t / in.nx;
        const int j = in.j0 + (int)(r % ny), k = in.k0 + (int)(r / ny);
        const int ring = k * in.nyt + j;
        const long long c = (long long)k * in.sk + (long long)j * in.sj + i;
        const double V = in.vol[ring];
        const double rho = (double)in.rho[c];
        kb_add(acc[0], rho * V);
        if (in.e) kb_add(acc[1], (double)in.e[c] * V);
        const double R = in.R[ring];
        const double w = (in.wfr ? in.wfr[ring] : R * R * in.omega) + (in.vref ? R * in.vref[ring] : 0.0);
        const int ip = i + 1 == in.nx ? 0 : i + 1;
        const double pm = rho * (R * (double)in.vx[c] + w), pp = rho * (R * (double)in.vx[c - i + ip] + w);
        kb_add(acc[2], 0.5 * (pm + pp) * V);
    }
    for (int q = 0; q < 3; q++) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 3; q++) kb_merge(sh[q][threadIdx.x], sh[q][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; q++) {
            part[(blockIdx.x * 3 + q) * 2] = sh[q][0].s;
            part[(blockIdx.x * 3 + q) * 2 + 1] = sh[q][0].c;
        }
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the block partials, by the whole last block in a fixed order: thread t
    // merges blocks t, t + blockDim, ..., then the same tree as above
    for (int q = 0; q < 3; q++) {
        KB a = {0, 0};
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            KB x = {__ldcg(&part[(b * 3 + q) * 2]), __ldcg(&part[(b * 3 + q) * 2 + 1])};
            kb_merge(a, x);
        }
        sh[q][threadIdx.x] = a;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 3; q++) kb_merge(sh[q][threadIdx.x], sh[q][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; q++) result[q] = sh[q][0].s + sh[q][0].c;
    *counter = 0u;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sums(SumInput<T> in, double *part, unsigned *counter, double *result)
{
    sums_reduce<T>(in, part, counter, result);
}

// k_newvel with the configuration class cfg_of(m) selects.
template <typename T>
static void launch_newvel(const MeshD &m, dim3 g, dim3 b, cudaStream_t s, const Tab<T> &tb, const QSet<T> &fin,
                          const Fld<T> &vsrc, const Fld<T> &state, Scal *sc, int copy_scalars)
{
    switch (cfg_of(m)) {
    case CFG_DISK3D: k_newvel<T, CfgDisk3D><<<g, b, 0, s>>>(m, tb, fin, vsrc, state, sc, copy_scalars); break;
    case CFG_DISK2D: k_newvel<T, CfgDisk2D><<<g, b, 0, s>>>(m, tb, fin, vsrc, state, sc, copy_scalars); break;
    case CFG_DISK3D_LIVE: k_newvel<T, CfgDisk3DLive><<<g, b, 0, s>>>(m, tb, fin, vsrc, state, sc, copy_scalars); break;
    case CFG_DISK2D_LIVE: k_newvel<T, CfgDisk2DLive><<<g, b, 0, s>>>(m, tb, fin, vsrc, state, sc, copy_scalars); break;
    default: k_newvel<T, CfgRun><<<g, b, 0, s>>>(m, tb, fin, vsrc, state, sc, copy_scalars); break;
    }
}

}  // namespace fk
