// Transport step (flow-chart cell 12): left/right momenta, the X sweep with
// orbital advection, the Y and Z sweeps, and the new face velocities.
#pragma once
#include "fargo_internal.cuh"
#include "kernels_source.cuh"

namespace fk {

// van Leer slope (Sec. 3.5, below Eq. 15): harmonic mean of the one-sided
// differences over the centre-to-centre distances, zero across an extremum.
template <typename T>
__device__ __forceinline__ T vl_slope(T qm, T q0, T qp, T dxm, T dxp)
{
    const T dp = (qp - q0) / dxp, dm = (q0 - qm) / dxm;
    return dp * dm > T(0) ? T(2) * dp * dm / (dp + dm) : T(0);
}

// ---------------------------------------------------------------------------
// X sweep, residual part, one CTA per ring (j,k), the ring staged in shared
// memory:
//  12a  momenta Pi-/+ of Eqs. 16-17 with the factors of Tab. "momenta";
//  (i)  van Leer sweep at delta v = v_x - v0 (Eq. fargo1, Eq. 15; v0 = 0 for
//       STANDARD transport), consistent transport (ratio to the density times
//       the mass flux), all fluxes from the pre-sweep ring.
// Ghost rings only get their momenta (the Y/Z sweeps read them).
// Shared memory: nq ring arrays + 5 work arrays of nx values.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_transport_x(MeshD m, Tab<T> tb, Fld<T> in, QSet<T> out, const double *v0,
                                                     const Scal *sc)
{
    extern __shared__ unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const double dtd = sc->dt;
    if (!(dtd > 0.0)) return;
    const int nx = m.nx, nq = out.nq;
    const int ring = blockIdx.x;
    const int j = ring % m.nyt, k = ring / m.nyt;
    const bool active = j >= m.j0 && j < m.j1 && k >= m.k0 && k < m.k1;
    T *Q = sm;                       // nq * nx
    T *Fr = sm + (size_t)nq * nx;    // mass flux on faces
    T *Ft = Fr + nx;                 // flux of the current quantity
    T *A = Ft + nx, *Cw = A + 2 * nx;
    const long long base = IX(m, 0, j, k);
    const T R = tb.R[ring], w = R * R * T(m.omega), fz = tb.fz[ring];
    const bool adi = !m.iso;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const long long c = base + i;
        const int ip = i + 1 == nx ? 0 : i + 1;
        const T rho = in.rho[c];
        int q = 0;
        Q[(q++) * nx + i] = rho;
        if (adi) Q[(q++) * nx + i] = in.e[c];
        Q[(q++) * nx + i] = rho * (R * in.vx[c] + w);
        Q[(q++) * nx + i] = rho * (R * in.vx[base + ip] + w);
        if (m.hasY) {
            Q[(q++) * nx + i] = rho * in.vy[c];
            Q[(q++) * nx + i] = rho * in.vy[c + m.sj];
        }
        if (m.hasZ) {
            Q[(q++) * nx + i] = rho * (fz * in.vz[c]);
            Q[(q++) * nx + i] = rho * (fz * in.vz[c + m.sk]);
        }
    }
    __syncthreads();
    if (active && m.hasX) {
        const double v0r = m.fargo ? v0[ring] : 0.0;
        const T dt = (T)dtd;
        const T dX = tb.lenx[ring], S = tb.sx[ring], Vi = tb.vinv[ring];
        for (int i = threadIdx.x; i < nx; i += blockDim.x) Cw[i] = (T)((double)in.vx[base + i] - v0r);
        __syncthreads();
        for (int q = 0; q < nq; q++) {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) A[i] = q == 0 ? Q[i] : Q[q * nx + i] / Q[i];
            __syncthreads();
            T *F = q == 0 ? Fr : Ft;
            for (int f = threadIdx.x; f < nx; f += blockDim.x) {
                const T v = Cw[f];
                const int d = v >= T(0) ? (f == 0 ? nx - 1 : f - 1) : f;
                const int dm = d == 0 ? nx - 1 : d - 1, dp = d + 1 == nx ? 0 : d + 1;
                const T a = vl_slope(A[dm], A[d], A[dp], dX, dX);
                const T st = v >= T(0) ? A[d] + a * (dX - v * dt) / T(2) : A[d] - a * (dX + v * dt) / T(2);
                F[f] = q == 0 ? v * st * S : Fr[f] * st;
            }
            __syncthreads();
            if (q > 0) {
                for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                    const int ip = i + 1 == nx ? 0 : i + 1;
                    Q[q * nx + i] -= dt * Vi * (Ft[ip] - Ft[i]);
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int ip = i + 1 == nx ? 0 : i + 1;
            Q[i] -= dt * Vi * (Fr[ip] - Fr[i]);
        }
        __syncthreads();
    }
    for (int q = 0; q < nq; q++)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) out.q[q][base + i] = Q[q * nx + i];
}

// ---------------------------------------------------------------------------
// Uniform orbital step of each active ring (Sec. 3.4.1, Eqs. fargo2, 28-33),
// applied after the Y and Z sweeps, in place, one CTA per ring:
//  (ii)  circular shift by N = E(v0 dt / dX) (Eq. 32): the ring is rotated
//        while it is copied into shared memory;
//  (iii) fractional step at xi = v0 dt/dX - N with PPA interface values
//        (Eqs. 34-36 and the xi-weighted value of Sec. 3.4.1), consistent
//        transport, in the same pass.
// N and xi are FP64, evaluated with round-to-nearest intrinsics.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_orbital(MeshD m, Tab<T> tb, QSet<T> qs, const double *v0, const Scal *sc)
{
    extern __shared__ unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const double dtd = sc->dt;
    if (!(dtd > 0.0)) return;
    const int nx = m.nx, nq = qs.nq;
    const int r = blockIdx.x;
    const int ny = m.j1 - m.j0;
    const int j = m.j0 + r % ny, k = m.k0 + r / ny;
    const int ring = k * m.nyt + j;
    const long long base = IX(m, 0, j, k);
    const double v0r = v0[ring];
    const double X = __ddiv_rn(__dmul_rn(v0r, dtd), tb.lx[ring]);
    const long long N = llround(X);
    const double xs = __dsub_rn(X, (double)N);
    const int Nm = (int)(((N % nx) + nx) % nx);
    if (Nm == 0 && xs == 0.0) return;
    T *Q = sm;
    T *Fr = sm + (size_t)nq * nx;
    T *Ft = Fr + nx;
    T *A = Ft + nx, *B = A + nx, *Cw = B + nx;
    for (int q = 0; q < nq; q++)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            int s = i - Nm;
            if (s < 0) s += nx;
            Q[q * nx + i] = qs.q[q][base + s];
        }
    __syncthreads();
    if (xs != 0.0) {
        const T dt = (T)dtd;
        const T S = tb.sx[ring], Vi = tb.vinv[ring];
        const T vR = (T)(xs * tb.lx[ring] / dtd);
        const T xi = (T)fabs(xs);
        const bool pos = xs >= 0.0;
        for (int q = 0; q < nq; q++) {
            for (int i = threadIdx.x; i < nx; i += blockDim.x) A[i] = q == 0 ? Q[i] : Q[q * nx + i] / Q[i];
            __syncthreads();
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const T qm = A[i == 0 ? nx - 1 : i - 1], q0 = A[i], qp = A[i + 1 == nx ? 0 : i + 1];
                T dmv = T(0);
                if ((qp - q0) * (q0 - qm) > T(0)) {
                    const T d = T(0.5) * (qp - qm);
                    T mn = fmin(T(2) * fabs(q0 - qm), T(2) * fabs(qp - q0));
                    mn = fmin(mn, fabs(d));
                    dmv = d > T(0) ? mn : -mn;
                }
                B[i] = dmv;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                const int ip = i + 1 == nx ? 0 : i + 1;
                Cw[i] = A[i] + T(0.5) * (A[ip] - A[i]) - (B[ip] - B[i]) / T(6);
            }
            __syncthreads();
            T *F = q == 0 ? Fr : Ft;
            for (int f = threadIdx.x; f < nx; f += blockDim.x) {
                const int d = pos ? (f == 0 ? nx - 1 : f - 1) : f;
                const int dm = d == 0 ? nx - 1 : d - 1, dp = d + 1 == nx ? 0 : d + 1;
                const T qm = A[dm], q0 = A[d], qp = A[dp];
                T l = Cw[dm], rr = Cw[d];
                if ((qp - q0) * (q0 - qm) <= T(0)) {
                    l = q0;
                    rr = q0;
                } else {
                    const T D = rr - l, C = q0 - T(0.5) * (l + rr);
                    if (D * C > D * D / T(6)) l = T(3) * q0 - T(2) * rr;
                    else if (-D * D / T(6) > D * C) rr = T(3) * q0 - T(2) * l;
                }
                const T st = pos ? rr + xi * (q0 - rr) + xi * (T(1) - xi) * (T(2) * q0 - rr - l)
                                 : l + xi * (q0 - l) + xi * (T(1) - xi) * (T(2) * q0 - rr - l);
                F[f] = q == 0 ? vR * st * S : Fr[f] * st;
            }
            __syncthreads();
            if (q > 0) {
                for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                    const int ip = i + 1 == nx ? 0 : i + 1;
                    Q[q * nx + i] -= dt * Vi * (Ft[ip] - Ft[i]);
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int ip = i + 1 == nx ? 0 : i + 1;
            Q[i] -= dt * Vi * (Fr[ip] - Fr[i]);
        }
        __syncthreads();
    }
    for (int q = 0; q < nq; q++)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) qs.q[q][base + i] = Q[q * nx + i];
}

// ---------------------------------------------------------------------------
// Y and Z sweeps (Eqs. 1D-advection-Y/Z): one thread per cell, fluxes through
// its lower and upper face recomputed from the five cells around it.  Reads
// `in` (the values of the previous sweep, ghosts included) and writes `out`;
// with copy_ghosts set, cells outside the active box are copied so that the
// next sweep finds every ghost it needs.
// ---------------------------------------------------------------------------
template <typename T, int AXIS>
__global__ void __launch_bounds__(256) k_transport_yz(MeshD m, Tab<T> tb, QSet<T> in, QSet<T> out, const T *vel,
                                                      const Scal *sc, int copy_ghosts)
{
    const double dtd = sc->dt;
    if (!(dtd > 0.0)) return;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)m.nx * m.nyt * m.nzt;
    if (tid >= n) return;
    const int i = (int)(tid % m.nx);
    const long long rr = tid / m.nx;
    const int j = (int)(rr % m.nyt), k = (int)(rr / m.nyt);
    const long long c = IX(m, i, j, k);
    const int nq = in.nq;
    const bool active = j >= m.j0 && j < m.j1 && k >= m.k0 && k < m.k1;
    if (!active) {
        if (copy_ghosts)
            for (int q = 0; q < nq; q++) out.q[q][c] = in.q[q][c];
        return;
    }
    const T dt = (T)dtd;
    const int ring = k * m.nyt + j;
    const long long st = AXIS == 1 ? m.sj : m.sk;
    const int p = AXIS == 1 ? j : k;      // index along the sweep
    // centre distance across face f and width of cell d along the sweep
    auto cdist = [&](int f) -> T {
        if (AXIS == 1) return tb.dyc[f];
        return tb.dzc[f * m.nyt + j];
    };
    auto width = [&](int d) -> T {
        if (AXIS == 1) return tb.dy[d];
        return tb.lenz[d * m.nyt + j];
    };
    const int fr = k * (m.nyt + 1) + j;
    const T Slo = AXIS == 1 ? tb.sy[fr] : tb.sz[fr];
    const T Sup = AXIS == 1 ? tb.sy[fr + 1] : tb.sz[fr + m.nyt + 1];
    const T vlo = vel[c], vup = vel[c + st];
    const T Vi = tb.vinv[ring];
    // stencil cells p-2 .. p+2 -> s = 0..4
    T r5[5];
    for (int s = 0; s < 5; s++) r5[s] = in.q[0][c + (s - 2) * st];
    // donor index (0..4) for each face, and its slope/width
    const int dlo = vlo >= T(0) ? 1 : 2, dup = vup >= T(0) ? 2 : 3;
    const T cdlo_m = cdist(p - 2 + dlo), cdlo_p = cdist(p - 1 + dlo);
    const T cdup_m = cdist(p - 2 + dup), cdup_p = cdist(p - 1 + dup);
    const T wlo = width(p - 2 + dlo), wup = width(p - 2 + dup);
    auto face = [&](const T *f5, int d, T v, T cdm, T cdp, T wd) -> T {
        const T a = vl_slope(f5[d - 1], f5[d], f5[d + 1], cdm, cdp);
        return v >= T(0) ? f5[d] + a * (wd - v * dt) / T(2) : f5[d] - a * (wd + v * dt) / T(2);
    };
    const T F0lo = vlo * face(r5, dlo, vlo, cdlo_m, cdlo_p, wlo) * Slo;
    const T F0up = vup * face(r5, dup, vup, cdup_m, cdup_p, wup) * Sup;
    out.q[0][c] = r5[2] - dt * Vi * (F0up - F0lo);
    for (int q = 1; q < nq; q++) {
        T f5[5];
        for (int s = 0; s < 5; s++) f5[s] = in.q[q][c + (s - 2) * st] / r5[s];
        const T Flo = F0lo * face(f5, dlo, vlo, cdlo_m, cdlo_p, wlo);
        const T Fup = F0up * face(f5, dup, vup, cdup_m, cdup_p, wup);
        out.q[q][c] = in.q[q][c] - dt * Vi * (Fup - Flo);
    }
}

// ---------------------------------------------------------------------------
// New face velocities from the new momenta and densities (Eq. 18), undoing
// the geometric factors of Tab. "momenta", on interior faces; every other
// face is copied from the post-source velocities.  When the last sweep left
// density and energy in the scratch set, they are copied back too.  Thread 0
// advances the device time.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_newvel(MeshD m, Tab<T> tb, QSet<T> fin, Fld<T> vsrc, Fld<T> state,
                                                Scal *sc, int copy_scalars)
{
    const double dtd = sc->dt;
    if (!(dtd > 0.0)) return;
    CellIdx ci;
    if (!decode(m, ci)) return;
    const int i = ci.i, j = ci.j, k = ci.k;
    if (i == 0 && j == 0 && k == 0) {
        sc->t = sc->t + dtd;
        sc->nstep += 1;
    }
    const long long c = IX(m, i, j, k);
    const bool jact = j >= m.j0 && j < m.j1, kact = k >= m.k0 && k < m.k1;
    const int ring = k * m.nyt + j;
    const T *rho = fin.q[0];
    const int o = m.iso ? 1 : 2;   // index of Pi-x in the quantity set
    if (j < m.nyt && k < m.nzt) {
        T v = vsrc.vx[c];
        if (jact && kact) {
            const long long cm = c - i + (i == 0 ? m.nx - 1 : i - 1);
            const T R = tb.R[ring], w = R * R * T(m.omega);
            v = ((fin.q[o + 1][cm] + fin.q[o][c]) / (rho[cm] + rho[c]) - w) / R;
        }
        state.vx[c] = v;
        if (copy_scalars) {
            state.rho[c] = rho[c];
            if (!m.iso) state.e[c] = fin.q[1][c];
        }
    }
    const int oy = o + 2, oz = o + (m.hasY ? 4 : 2);
    if (k < m.nzt) {
        T v = vsrc.vy[c];
        if (m.hasY && j > m.j0 && j < m.j1 && kact) {
            const long long cm = c - m.sj;
            v = (fin.q[oy + 1][cm] + fin.q[oy][c]) / (rho[cm] + rho[c]);
        }
        state.vy[c] = v;
    }
    if (j < m.nyt) {
        T v = vsrc.vz[c];
        if (m.hasZ && k > m.k0 && k < m.k1 && jact) {
            const long long cm = c - m.sk;
            v = (fin.q[oz + 1][cm] + fin.q[oz][c]) / (rho[cm] + rho[c]) / tb.fz[ring];
        }
        state.vz[c] = v;
    }
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

template <typename T>
__global__ void __launch_bounds__(256) k_sums(MeshD m, Tab<T> tb, Fld<T> f, const double *vol, double *part,
                                              Scal *sc, double *result)
{
    __shared__ KB sh[3][256];
    __shared__ int s_last;
    KB acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    const int ny = m.j1 - m.j0, nz = m.k1 - m.k0;
    const long long n = (long long)m.nx * ny * nz;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % m.nx);
        const long long r = t / m.nx;
        const int j = m.j0 + (int)(r % ny), k = m.k0 + (int)(r / ny);
        const int ring = k * m.nyt + j;
        const long long c = IX(m, i, j, k);
        const double V = vol[ring];
        const double rho = (double)f.rho[c];
        kb_add(acc[0], rho * V);
        if (!m.iso) kb_add(acc[1], (double)f.e[c] * V);
        const double R = tb.Rd[ring], w = R * R * m.omega;
        const int ip = i + 1 == m.nx ? 0 : i + 1;
        const double pm = rho * (R * (double)f.vx[c] + w), pp = rho * (R * (double)f.vx[c - i + ip] + w);
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
        s_last = atomicAdd(&sc->counter2, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    for (int q = 0; q < 3; q++) {
        KB a = {0, 0};
        for (unsigned b = 0; b < gridDim.x; b++) {
            KB x = {__ldcg(&part[(b * 3 + q) * 2]), __ldcg(&part[(b * 3 + q) * 2 + 1])};
            kb_merge(a, x);
        }
        result[q] = a.s + a.c;
    }
    sc->counter2 = 0u;
}

}  // namespace fk
