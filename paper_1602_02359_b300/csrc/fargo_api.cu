// C ABI of the B300 hydro step: context, geometry tables, step driver and
// CUDA-graph capture.  See include/fargo.h for the contract of each call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "context.cuh"

using namespace fk;

// cuTensorMapEncodeTiled through the runtime's driver entry point.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3D map of one field array (nx, ny_t+1, nz_t+1; row pitch in bytes), box =
// one row segment of 512 bytes.  Out-of-range azimuths read as zero.
template <typename T>
static int encode_field_map(const fargo_ctx *c, CUtensorMap *map, const T *ptr)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return FARGO_ERR_CUDA;
    const cuuint64_t dims[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->nyt + 1, (cuuint64_t)c->nzt + 1};
    const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * sizeof(T), (cuuint64_t)c->m.sk * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)TmaTile<T>::TW, 1, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    (void *)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FARGO_OK : FARGO_ERR_CUDA;
}

template <typename T>
static int encode_sweep_maps(const fargo_ctx *c, SweepMaps *mp, const QSet<T> &in, const QSet<T> &ghost,
                             const T *vel)
{
    int rc;
    for (int q = 0; q < in.nq; q++) {
        if ((rc = encode_field_map<T>(c, &mp->qin[q], in.q[q]))) return rc;
        if ((rc = encode_field_map<T>(c, &mp->qg[q], ghost.q[q]))) return rc;
    }
    return encode_field_map<T>(c, &mp->vel, vel);
}

static const char *g_errstr[] = {"ok", "bad argument", "out of memory", "CUDA error", "non-finite state",
                                 "Courant step not positive", "size mismatch or kernel limit", "barrier timeout",
                                 "CUDA device or kernel image unavailable"};

extern "C" const char *fargo_strerror(int code)
{
    if (code > 0 || code < -8) return "unknown error";
    return g_errstr[-code];
}

static int dalloc(fargo_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? FARGO_ERR_OOM : FARGO_ERR_CUDA;
    }
    c->allocs.push_back(*p);
    e = cudaMemsetAsync(*p, 0, bytes < 16 ? 16 : bytes, c->stream);
    return e == cudaSuccess ? FARGO_OK : FARGO_ERR_CUDA;
}

template <typename T>
static int upload(fargo_ctx *c, const T **dst, const std::vector<double> &src)
{
    std::vector<T> h(src.size() ? src.size() : 1);
    for (size_t i = 0; i < src.size(); i++) h[i] = (T)src[i];
    void *p;
    int rc = dalloc(c, &p, h.size() * sizeof(T));
    if (rc) return rc;
    CK(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *dst = (const T *)p;
    return FARGO_OK;
}

// ---------------------------------------------------------------------------
// Geometry of Appendix A (Tab. "geom", Eqs. 70-71), built in FP64 on the host.
// ---------------------------------------------------------------------------
static void build_geometry(fargo_ctx *c, const fargo_params *p, double gamma, const fargo_planet *pl)
{
    HostGeom &h = c->hg;
    const int nx = c->nx, nyt = c->nyt, nzt = c->nzt, geom = c->geom;
    const double *yf = p->yfaces, *zf = p->zfaces;
    const double dx = (p->xmax - p->xmin) / nx;
    const bool hasX = nx > 1, hasY = c->ny > 1, hasZ = c->nz > 1;
    h.ym.assign(nyt + 1, 0.0); h.dy.assign(nyt + 1, 0.0); h.dyc.assign(nyt + 1, 0.0);
    h.zm.assign(nzt + 1, 0.0); h.dz.assign(nzt + 1, 0.0);
    for (int j = 0; j < nyt; j++) {
        h.ym[j] = 0.5 * (yf[j] + yf[j + 1]);
        h.dy[j] = yf[j + 1] - yf[j];
    }
    for (int j = 1; j < nyt; j++) h.dyc[j] = h.ym[j] - h.ym[j - 1];
    for (int k = 0; k < nzt; k++) {
        h.zm[k] = 0.5 * (zf[k] + zf[k + 1]);
        h.dz[k] = zf[k + 1] - zf[k];
    }
    const size_t nr = (size_t)nzt * nyt, nf = (size_t)(nzt + 1) * (nyt + 1);
    h.lx.assign(nr, 0); h.ly.assign(nr, 0); h.lz.assign(nr, 0); h.dmin.assign(nr, 0); h.R.assign(nr, 0);
    h.zc.assign(nr, 0); h.vol.assign(nr, 0); h.fz.assign(nr, 0); h.dzc.assign(nr, 0); h.sx.assign(nr, 0);
    h.vinv.assign(nr, 0); h.lenz.assign(nr, 0); h.gphy.assign(nr, 0); h.gphz.assign(nr, 0);
    h.cs.assign(nr, 0); h.nu.assign(nr, 0);
    h.rma.assign(nr, 0); h.fra.assign(nr, 0); h.z2.assign(nr, 0); h.qar.assign(nr, 0);
    h.wfr.assign(nr, 0); h.tid.assign(nyt + 1, 0);
    if (p->shearing)   // the shearing sheet's tide per Y face, 4 A Omega_f y (subtracted)
        for (int j = 0; j <= nyt; j++) h.tid[j] = 4.0 * p->oort_a * p->omega_frame * yf[j];
    h.sy.assign(nf, 0); h.sz.assign(nf, 0);
    auto syk = [&](int k) {
        if (geom == FARGO_CYL) return zf[k + 1] - zf[k];
        if (geom == FARGO_SPH) return cos(zf[k]) - cos(zf[k + 1]);
        return dx * (zf[k + 1] - zf[k]);
    };
    auto syj = [&](int j) {
        if (geom == FARGO_CYL) return yf[j] * dx;
        if (geom == FARGO_SPH) return yf[j] * yf[j] * dx;
        return 1.0;
    };
    auto szj = [&](int j) {
        if (geom == FARGO_CART) return dx * (yf[j + 1] - yf[j]);
        return 0.5 * dx * (yf[j + 1] * yf[j + 1] - yf[j] * yf[j]);
    };
    auto szk = [&](int k) { return geom == FARGO_SPH ? sin(zf[k]) : 1.0; };
    auto sxj = [&](int j) {
        if (geom == FARGO_SPH) return 0.5 * (yf[j + 1] * yf[j + 1] - yf[j] * yf[j]);
        return yf[j + 1] - yf[j];
    };
    auto vjinv = [&](int j) {
        if (geom == FARGO_CYL) return 2.0 / ((yf[j + 1] * yf[j + 1] - yf[j] * yf[j]) * dx);
        if (geom == FARGO_SPH) return 3.0 / ((yf[j + 1] * yf[j + 1] * yf[j + 1] - yf[j] * yf[j] * yf[j]) * dx);
        return 1.0 / (yf[j + 1] - yf[j]);
    };
    const double M = p->star_mass;
    auto phis = [&](int j, int k) {
        if (M <= 0.0 || geom == FARGO_CART) return 0.0;
        if (geom == FARGO_CYL) return -M / sqrt(h.ym[j] * h.ym[j] + h.zm[k] * h.zm[k]);
        return -M / h.ym[j];
    };
    for (int k = 0; k < nzt; k++)
        for (int j = 0; j < nyt; j++) {
            const size_t r = (size_t)k * nyt + j;
            double R = 1.0;
            if (geom == FARGO_CYL) R = h.ym[j];
            else if (geom == FARGO_SPH) R = h.ym[j] * sin(h.zm[k]);
            h.R[r] = R;
            // the frame's share of the X momentum (Tab. momenta)
            if (geom != FARGO_CART) h.wfr[r] = R * R * p->omega_frame;
            else if (p->shearing) h.wfr[r] = 2.0 * p->omega_frame * h.ym[j];
            h.lx[r] = R * dx;
            h.ly[r] = h.dy[j];
            h.lz[r] = geom == FARGO_SPH ? h.ym[j] * h.dz[k] : h.dz[k];
            double dmin = INFINITY;
            if (hasX && h.lx[r] < dmin) dmin = h.lx[r];
            if (hasY && h.ly[r] < dmin) dmin = h.ly[r];
            if (hasZ && h.lz[r] < dmin) dmin = h.lz[r];
            h.dmin[r] = dmin;
            h.lenz[r] = h.lz[r];
            h.zc[r] = geom == FARGO_SPH ? h.ym[j] * cos(h.zm[k]) : h.zm[k];
            h.fz[r] = geom == FARGO_SPH ? h.ym[j] : 1.0;
            if (k > 0) h.dzc[r] = geom == FARGO_SPH ? h.ym[j] * (h.zm[k] - h.zm[k - 1]) : h.zm[k] - h.zm[k - 1];
            h.sx[r] = sxj(j) * (zf[k + 1] - zf[k]);
            h.vinv[r] = vjinv(j) / syk(k);
            h.vol[r] = 1.0 / h.vinv[r];
            if (j > 0) h.gphy[r] = (phis(j, k) - phis(j - 1, k)) / h.dyc[j];
            if (k > 0) h.gphz[r] = (phis(j, k) - phis(j, k - 1)) / h.dzc[r];
            if (p->cs) h.cs[r] = p->cs[r];
            if (p->nu) h.nu[r] = p->nu[r];
            if (pl && pl->q > 0.0) {
                h.rma[r] = R - pl->a;
                h.fra[r] = 4.0 * R * pl->a;
                h.z2[r] = h.zc[r] * h.zc[r];
                h.qar[r] = pl->q / (pl->a * pl->a) * R;
            }
        }
    for (int k = 0; k <= nzt; k++)
        for (int j = 0; j <= nyt; j++) {
            const size_t f = (size_t)k * (nyt + 1) + j;
            if (k < nzt) h.sy[f] = syj(j) * syk(k);
            if (j < nyt) h.sz[f] = szj(j) * szk(k);
        }
    h.cosx.assign(nx, 0);
    h.sinx.assign(nx, 0);
    for (int i = 0; i < nx; i++) {
        const double x = p->xmin + (i + 0.5) * dx;
        h.cosx[i] = cos(x);
        h.sinx[i] = sin(x);
    }
    MeshD &m = c->m;
    m.dx = dx;
    m.xmin = p->xmin;
    (void)gamma;
}

template <typename T>
static int build_tables(fargo_ctx *c, Tab<T> &t)
{
    HostGeom &h = c->hg;
    const int nyt = c->nyt, nzt = c->nzt;
    int rc;
#define UP(dst, src) \
    if ((rc = upload<T>(c, &t.dst, src))) return rc
#define UPD(dst, src) \
    if ((rc = upload<double>(c, &t.dst, src))) return rc
    std::vector<double> szm(nzt + 1, 0), szf(nzt + 1, 0), cotzm(nzt + 1, 0), cotzf(nzt + 1, 0), zf(nzt + 1, 0),
        yf(nyt + 1, 0);
    for (int k = 0; k <= nzt; k++) {
        zf[k] = c->zfaces_store[k];
        szf[k] = sin(zf[k]);
        cotzf[k] = cos(zf[k]) / sin(zf[k]);
        if (k < nzt) {
            szm[k] = sin(h.zm[k]);
            cotzm[k] = cos(h.zm[k]) / sin(h.zm[k]);
        }
    }
    for (int j = 0; j <= nyt; j++) yf[j] = c->yfaces_store[j];
    UP(ym, h.ym); UP(dy, h.dy); UP(yf, yf); UP(dyc, h.dyc);
    UP(zm, h.zm); UP(dz, h.dz); UP(zf, zf); UP(szm, szm); UP(szf, szf); UP(cotzm, cotzm); UP(cotzf, cotzf);
    UP(R, h.R); UP(lenx, h.lx); UP(lenz, h.lenz); UP(dzc, h.dzc); UP(sx, h.sx); UP(vinv, h.vinv);
    UP(cs, h.cs); UP(nu, h.nu); UP(gphy, h.gphy); UP(gphz, h.gphz); UP(fz, h.fz);
    UP(sy, h.sy); UP(sz, h.sz);
    UP(wfr, h.wfr); UP(tid, h.tid); UPD(wfrd, h.wfr);
    UPD(lx, h.lx); UPD(ly, h.ly); UPD(lz, h.lz); UPD(dmin, h.dmin); UPD(csd, h.cs); UPD(nud, h.nu);
    UPD(Rd, h.R); UPD(zcd, h.zc); UPD(cosx, h.cosx); UPD(sinx, h.sinx);
    UP(rma, h.rma); UP(fra, h.fra); UP(z2, h.z2); UP(qar, h.qar);
    {
        const MeshD &m = c->m;
        t.gm1 = (T)(m.gamma - 1.0);
        t.half_gm1 = (T)(0.5 * (m.gamma - 1.0));
        t.cq2 = (T)(m.cq * m.cq);
        t.omega = (T)m.omega;
        t.pq = (T)m.pq;
        t.peps2 = (T)m.peps2;
        t.dx = (T)m.dx;
        t.g1 = (T)m.g1;
        t.k4 = (T)(m.av_lit ? 1.0 / m.av_c2 : 4.0 * m.cq * m.cq);
    }
    {
        std::vector<double> r4(h.dmin.size(), 0.0);
        for (size_t r = 0; r < r4.size(); r++)
            if (h.nu[r] > 0.0) r4[r] = 4.0 * h.nu[r] / (h.dmin[r] * h.dmin[r]);
        UP(r4, r4);
        UP(dminT, h.dmin);
        std::vector<double> idyc(h.dyc.size(), 0.0), idzc(h.dzc.size(), 0.0);
        for (size_t q = 0; q < idyc.size(); q++) idyc[q] = h.dyc[q] > 0.0 ? 1.0 / h.dyc[q] : 0.0;
        for (size_t q = 0; q < idzc.size(); q++) idzc[q] = h.dzc[q] > 0.0 ? 1.0 / h.dzc[q] : 0.0;
        UP(idyc, idyc);
        UP(idzc, idzc);
        auto inv = [](const std::vector<double> &a) {
            std::vector<double> r(a.size(), 0.0);
            for (size_t q = 0; q < a.size(); q++) r[q] = a[q] != 0.0 ? 1.0 / a[q] : 0.0;
            return r;
        };
        UP(ilenx, inv(h.lx));
        UP(ilenz, inv(h.lenz));
        UP(iR, inv(h.R));
        UP(idy, inv(h.dy));
        UP(iyf, inv(yf));
        UP(iym, inv(h.ym));
        UP(idz, inv(h.dz));
        UP(iszm, inv(szm));
        std::vector<double> dzm(nzt + 1, 0.0);
        for (int k = 1; k < nzt; k++) dzm[k] = h.zm[k] - h.zm[k - 1];
        UP(idzm, inv(dzm));
        t.idx = (T)(1.0 / c->m.dx);
    }
    {
        // azimuth tables of up to kPotPlanets planets (planet p at p * nx),
        // and the live planets' per-ring tables and masses
        const int np = c->m.has_planet ? kPotPlanets : 1;
        void *q;
        if ((rc = dalloc(c, &q, sizeof(T) * (size_t)np * c->nx))) return rc;
        t.ps = (T *)q;
        if ((rc = dalloc(c, &q, sizeof(T) * (size_t)np * c->nx))) return rc;
        t.pc = (T *)q;
        if ((rc = dalloc(c, &q, sizeof(T) * (size_t)np * 5 * nyt * nzt))) return rc;
        t.mring = (T *)q;
        if ((rc = dalloc(c, &q, sizeof(T) * kPotPlanets))) return rc;
        t.mq = (T *)q;
    }
    if (sizeof(T) == 4) {
        // the reference form of v_x: per-ring references (zero until v_x is
        // set) and the X momenta's frame shifts, filled by vref_refresh
        const size_t nr = (size_t)nyt * nzt;
        void *q;
        if ((rc = dalloc(c, &q, sizeof(T) * nr))) return rc;
        t.vref = (T *)q;
        if ((rc = dalloc(c, &q, sizeof(double) * nr))) return rc;
        t.vrefd = (double *)q;
        if ((rc = dalloc(c, &q, sizeof(T) * nr))) return rc;
        t.dAy = (T *)q;
        if ((rc = dalloc(c, &q, sizeof(T) * nr))) return rc;
        t.dAz = (T *)q;
    }
#undef UP
#undef UPD
    return FARGO_OK;
}

// ---------------------------------------------------------------------------
// Reference form of v_x (FP32 contexts; see Tab::vref).  vref_launch runs one
// mode of k_vref over every ring; the state's v_x goes to v_x form before a
// field write (VREF_ABS in place), and back to the reference form after it
// with references chosen afresh (vref_refresh: VREF_CHOOSE, then VREF_APPLY).
// ---------------------------------------------------------------------------
template <typename T>
static int vref_launch(fargo_ctx *c, Buffers<T> &b, int mode, T *dst, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (!b.tab.vref) return FARGO_OK;
        const int nr = c->m.nyt * c->m.nzt;
        k_vref<T><<<(nr + 7) / 8, 256, 0, s>>>(c->m, b.tab, b.A.vx, dst ? dst : b.A.vx, mode);
        CK(cudaGetLastError());
    }
    return FARGO_OK;
}
template <typename T>
static int vref_refresh(fargo_ctx *c, Buffers<T> &b, cudaStream_t s)
{
    int rc = vref_launch<T>(c, b, VREF_CHOOSE, nullptr, s);
    return rc ? rc : vref_launch<T>(c, b, VREF_APPLY, nullptr, s);
}

template <typename T>
static int alloc_fields(fargo_ctx *c, Buffers<T> &b)
{
    const size_t n = (size_t)c->m.ntot * sizeof(T);
    void *p;
    int rc;
    T **slots[] = {&b.A.rho, &b.A.e, &b.A.vx, &b.A.vy, &b.A.vz, &b.vB[0], &b.vB[1], &b.vB[2], &b.rhoB, &b.eB};
    for (T **s : slots) {
        if ((rc = dalloc(c, &p, n))) return rc;
        *s = (T *)p;
    }
    for (int q = 0; q < 6; q++) {
        if ((rc = dalloc(c, &p, n))) return rc;
        b.piA[q] = (T *)p;
        if ((rc = dalloc(c, &p, n))) return rc;
        b.piB[q] = (T *)p;
    }
    int rc2 = build_tables<T>(c, b.tab);
    return rc2 ? rc2 : vref_refresh<T>(c, b, c->stream);
}

// ---------------------------------------------------------------------------
// The launch sequence of one full update (flow chart cells 2-12).
// Velocity buffers ping-pong A -> B -> A (-> B); the Y and Z sweeps are
// out of place, and the X sweep is in place or not so that the last sweep
// lands in the state buffers.
// ---------------------------------------------------------------------------
// Optional per-launch event marks (fargo_profile_step).
constexpr int kProfMax = 64;   // launches of one step, periodic images included
struct Prof {
    cudaEvent_t ev[kProfMax + 1];
    const char *name[kProfMax];
    int n;
};

template <typename T>
static int enqueue_step(fargo_ctx *c, Buffers<T> &b, Prof *prof = nullptr)
{
    const StepPlan<T> P = make_plan<T>(c, b);
    const MeshD &m = P.m;
    cudaStream_t s = c->stream;
    const int bs = 256;
    int nl = 0;
#define MARK(nm)                                                    \
    do {                                                            \
        if (prof) {                                                 \
            prof->name[nl] = nm;                                    \
            cudaEventRecord(prof->ev[nl + 1], s);                   \
        }                                                           \
        nl++;                                                       \
    } while (0)
    const dim3 cb = cell_block(m, c->cell_bs), cg = cell_grid_all(m, c->cell_bs);
    // cell 2
    if (m.hasY) { k_bc_y<T><<<grid_for((long long)m.nx * (m.nzt + 1) * 2, bs), bs, 0, s>>>(m, P.A, P.sc, 0, P.tb.vref, P.B); MARK("bc_y"); }
    if (m.hasZ) { k_bc_z<T><<<grid_for((long long)m.nx * (m.nyt + 1) * 2, bs), bs, 0, s>>>(m, P.A, P.sc, 0, P.tb.vref, P.B); MARK("bc_z"); }
    // cells 3-6
    k_cfl_screen<T><<<P.cfl_blocks, 256, 0, s>>>(m, P.tb, P.A, P.v0, P.ringmax, P.part, P.sc, P.nrings_active);
    MARK("cfl_screen");
    const bool mfargo = m.mhd && m.fargo && m.hasX;   // orbital advection of the field (Sec. 3.6)
    if (mfargo) {
        k_mhd_v0all<T><<<(m.nyt * m.nzt + 7) / 8, 256, 0, s>>>(m, P.A.vx, P.v0all);
        MARK("mhd_v0all");
    }
    k_cfl_exact<T><<<cfl_exact_grid(P.cfl_blocks), 256, 0, s>>>(m, P.tb, P.A, P.v0, P.ringmax, P.part, P.sc, P.nrings_active);
    MARK("cfl_exact");
    // periodic images between the phases (periodic Y/Z axes only)
    const bool per = m.pery || m.perz;
#define PERIODIC(set, nm)                                                      \
    do {                                                                       \
        if (per) {                                                             \
            const int k_ = launch_periodic<T>(m, set, P.sc, s);                \
            for (int q_ = 0; q_ < k_; q_++) MARK(nm);                          \
        }                                                                      \
    } while (0)
    // cell 7
    launch_source<T>(SRC_SUB1, m, cg, cb, s, P.tb, P.A, P.VB, P.tau, P.sc); MARK("substep1");
    // the magnetic pressure of the transverse field, with B at time t (cell 7a)
    const dim3 fgrid(cg.x, m.nyt + 1, m.nzt + 1);
    if (m.mhd && !m.mhd_passive) { k_mhd_pressure<T><<<fgrid, cb, 0, s>>>(m, P.tb, P.VB, P.sc); MARK("mhd_pressure"); }
    PERIODIC(per_fields<T>(m, P.VB, true, false), "periodic");
    launch_source<T>(SRC_AV, m, cg, cb, s, P.tb, P.VB, P.A, P.tau, P.sc); MARK("artvisc");
    PERIODIC(per_fields<T>(m, P.A, true, true), "periodic");
    if (m.has_nu) {
        // stresses once into the scratch momenta of set B (unused until the transport step)
        launch_source<T>(SRC_TAU, m, tau_grid(m, c->cell_bs), cb, s, P.tb, P.A, P.VB, P.tau, P.sc); MARK("visc_tau");
        QSet<T> diag = P.tau;
        diag.nq = m.hasZ ? 3 : 2;
        PERIODIC(per_quantities<T>(diag, diag), "periodic");
        launch_source<T>(SRC_VAPPLY, m, cg, cb, s, P.tb, P.A, P.VB, P.tau, P.sc); MARK("visc_apply");
        PERIODIC(per_fields<T>(m, P.VB, true, false), "periodic");
    }
    // cells 8a-8d: the EMFs and the magnetic tension, both from the velocities
    // after the source sub-steps
    if (m.mhd) {
        if (mfargo) {   // the EMFs and the tension's stars from the residual v_x
            k_mhd_dvx<T><<<dim3(cg.x, m.nyt, m.nzt), cb, 0, s>>>(m, P.vpre.vx, P.v0all, P.dvx);
            MARK("mhd_dvx");
            const Fld<T> res = {P.vpre.rho, P.vpre.e, P.dvx, P.vpre.vy, P.vpre.vz};
            k_mhd_edges<T><<<fgrid, cb, 0, s>>>(m, P.tb, res, P.VM, P.E[0], P.E[1], P.E[2], P.sc, 1,
                                                !m.mhd_passive, P.vpre.vx);
        } else {
            k_mhd_edges<T><<<fgrid, cb, 0, s>>>(m, P.tb, P.vpre, P.VM, P.E[0], P.E[1], P.E[2], P.sc, 1,
                                                !m.mhd_passive, (const T *)nullptr);
        }
        MARK("mhd_edges");
        if (!m.mhd_passive) PERIODIC(per_fields<T>(m, P.VM, true, false), "periodic");
    }
    // cell 9
    if (m.hasY) { k_bc_y<T><<<grid_for((long long)m.nx * (m.nzt + 1) * 2, bs), bs, 0, s>>>(m, P.vsrc, P.sc, 1, P.tb.vref, P.B); MARK("bc_y9"); }
    if (m.hasZ) { k_bc_z<T><<<grid_for((long long)m.nx * (m.nyt + 1) * 2, bs), bs, 0, s>>>(m, P.vsrc, P.sc, 1, P.tb.vref, P.B); MARK("bc_z9"); }
    // cell 10: constrained transport of the field
    if (m.mhd) {
        k_mhd_ct<T><<<fgrid, cb, 0, s>>>(m, P.tb, P.E[0], P.E[1], P.E[2], P.sc);
        MARK("mhd_ct");
        PERIODIC(per_field<T>(m, P.tb), "periodic");
        // cell 11: the field's orbital advection, the upstream-averaged EMFs
        // of the orbital motion through the same constrained transport
        if (mfargo) {
            k_mhd_fargo_emf<T><<<fgrid, cb, 0, s>>>(m, P.tb, P.v0all, P.E[0], P.E[1], P.E[2], P.sc);
            MARK("mhd_fargo_emf");
            k_mhd_ct<T><<<fgrid, cb, 0, s>>>(m, P.tb, P.E[0], P.E[1], P.E[2], P.sc);
            MARK("mhd_ct11");
            PERIODIC(per_field<T>(m, P.tb), "periodic");
        }
    }
    // cell 12
    launch_tx<T>(m, P.tb, P.txin, P.qx, P.v0, P.sc, c->tx_rs, s);
    MARK("transport_x");
    PERIODIC(per_quantities<T>(P.qx, P.qx), "periodic");
    if (m.hasY) {
        launch_sweep_tma<T, 1>(m, P.tb, c->mapsY, P.qy, P.sc, P.qx.nq, s, P.seg_y);
        MARK("transport_y");
        // the Z sweep reads its ghost planes from the Y sweep's input
        if (per && m.hasZ && m.perz) {
            const int k_ = launch_periodic<T>(m, per_quantities<T>(P.qx, P.qy), P.sc, s, 2);
            for (int q_ = 0; q_ < k_; q_++) MARK("periodic");
        }
    }
    if (m.hasZ) {
        launch_sweep_tma<T, 2>(m, P.tb, c->mapsZ, P.qz, P.sc, P.qx.nq, s, P.seg_z);
        MARK("transport_z");
    }
    // the uniform orbital step comes last, in place on the state set
    if (m.fargo && m.hasX) {
        launch_orb<T>(m, P.tb, P.qfin, P.v0, P.sc, P.nrings_active, c->orb_rs, s);
        MARK("orbital");
    }
    PERIODIC(per_quantities<T>(P.qfin, P.qfin), "periodic");
    launch_newvel<T>(m, cg, cb, s, P.tb, P.qfin, P.vsrc, P.A, P.sc, 0); MARK("newvel");
    PERIODIC(per_fields<T>(m, P.A, true, false), "periodic");
#undef PERIODIC
#undef MARK
    c->launches = nl;
    if (prof) prof->n = nl;
    CK(cudaGetLastError());
    return FARGO_OK;
}

static int enqueue(fargo_ctx *c)
{
    return c->prec == FARGO_F64 ? enqueue_step<double>(c, c->b64) : enqueue_step<float>(c, c->b32);
}

static int launch_step(fargo_ctx *c)
{
    if (!c->use_graph) return enqueue(c);
    if (!c->gexec) {
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue(c);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc) return rc;
        if (e != cudaSuccess) return FARGO_ERR_CUDA;
        c->graph = g;
        CK(cudaGraphInstantiate(&c->gexec, g, 0));
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    return FARGO_OK;
}

// Tensor maps of the step's Y and Z sweeps, following the buffer routing of
// enqueue_step: the X sweep is in place when an even number of Y/Z sweeps
// follows it; the Z sweep after a Y sweep reads its ghost planes from the
// Y sweep's input (the Y sweep writes active cells only).
// Tensor maps of the step's Y and Z sweeps, following the plan's buffer
// routing; the Z sweep after a Y sweep reads its ghost planes from the Y
// sweep's input (the Y sweep writes active cells only).
template <typename T>
static int build_sweep_maps(fargo_ctx *c, Buffers<T> &b)
{
    const StepPlan<T> P = make_plan<T>(c, b);
    const MeshD &m = P.m;
    int rc;
    if (m.hasY && (rc = encode_sweep_maps<T>(c, &c->mapsY, P.qx, P.qx, P.vsrc.vy))) return rc;
    if (m.hasZ) {
        const QSet<T> &zin = m.hasY ? P.qy : P.qx;
        if ((rc = encode_sweep_maps<T>(c, &c->mapsZ, zin, P.qx, P.vsrc.vz))) return rc;
    }
    const int nq = P.qx.nq;
    CK((sweep_tma_attrs<T, 1>(nq)));
    CK((sweep_tma_attrs<T, 2>(nq)));
    return FARGO_OK;
}

template <typename T, int C>
static cudaError_t ring_attrs_c(RingShape &rs, int n, bool orb)
{
    return orb ? ring_grid<T>(k_orbital<T, C>, rs, n) : ring_grid<T>(k_transport_x<T, C>, rs, n);
}
template <typename T>
static cudaError_t ring_attrs(RingShape &rs, int n, bool orb)
{
    switch (rs.chunk) {
    case 1: return ring_attrs_c<T, 1>(rs, n, orb);
    case 2: return ring_attrs_c<T, 2>(rs, n, orb);
    case 3: return ring_attrs_c<T, 3>(rs, n, orb);
    case 4: return ring_attrs_c<T, 4>(rs, n, orb);
    case 6: return ring_attrs_c<T, 6>(rs, n, orb);
    default: return ring_attrs_c<T, 8>(rs, n, orb);
    }
}

template <typename T>
static int set_kernel_attrs(fargo_ctx *c)
{
    int dev;
    CK(cudaGetDevice(&dev));
    int maxsm = 0;
    CK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int nq = 3 + (c->m.iso ? 0 : 1) + (c->m.hasY ? 2 : 0) + (c->m.hasZ ? 2 : 0);
    const int txrows = 2 + (c->m.iso ? 0 : 1) + (c->m.hasY ? 2 : 0) + (c->m.hasZ ? 2 : 0);
    // two ring buffers per CTA (double buffering)
    c->tx_rs = ring_shape<T>(c->nx, txrows, c->pitch, false);
    c->orb_rs = ring_shape<T>(c->nx, nq, c->pitch, true);
    const size_t smem = c->tx_rs.smem > c->orb_rs.smem ? c->tx_rs.smem : c->orb_rs.smem;
    if (smem > (size_t)maxsm - 1024 || c->tx_rs.chunk == 0 || c->orb_rs.chunk == 0) return FARGO_ERR_SIZE;
    if (ring_attrs<T>(c->tx_rs, c->nyt * c->nzt, false) != cudaSuccess ||
        ring_attrs<T>(c->orb_rs, c->nrings_active, true) != cudaSuccess)
        return FARGO_ERR_SIZE;
    return FARGO_OK;
}

// A periodic axis (Sec. 4.1): both sides periodic, a geometry that does not
// change along the axis, more active cells than ghost layers, ghost widths
// and per-ring tables (cs, nu) equal to their images one period away.
static bool close_rel(double a, double b) { return fabs(a - b) <= 1e-12 * fmax(fabs(a), fabs(b)); }
static bool periodic_ok(int geom, int nx, int ny, int nz, int g, const fargo_params *p)
{
    for (int ax = 0; ax < 2; ax++) {
        const int *bc = ax == 0 ? p->bc_y : p->bc_z;
        const int n = ax == 0 ? ny : nz;
        if ((bc[0] == FARGO_BC_PERIODIC) != (bc[1] == FARGO_BC_PERIODIC)) return false;
        if (bc[0] != FARGO_BC_PERIODIC || n == 1) continue;
        if (ax == 0 && geom != FARGO_CART) return false;
        if (ax == 1 && geom == FARGO_SPH) return false;
        if (n <= g) return false;
        const double *f = ax == 0 ? p->yfaces : p->zfaces;
        const int lo = g, hi = g + n;
        for (int mm = 1; mm <= g; mm++) {
            if (!close_rel(f[lo - mm + 1] - f[lo - mm], f[hi - mm + 1] - f[hi - mm])) return false;
            if (!close_rel(f[hi + mm - 1 + 1] - f[hi + mm - 1], f[lo + mm - 1 + 1] - f[lo + mm - 1])) return false;
        }
        const int nyt = ny > 1 ? ny + 2 * g : 1, nzt = nz > 1 ? nz + 2 * g : 1;
        for (const double *tab : {p->cs, p->nu}) {
            if (!tab) continue;
            for (int a = 0; a < (ax == 0 ? nzt : nyt); a++)
                for (int mm = 1; mm <= g; mm++) {
                    auto at = [&](int b) { return ax == 0 ? tab[(size_t)a * nyt + b] : tab[(size_t)b * nyt + a]; };
                    if (!close_rel(at(lo - mm), at(hi - mm)) || !close_rel(at(hi + mm - 1), at(lo + mm - 1)))
                        return false;
                }
        }
    }
    return true;
}

extern "C" int fargo_create(fargo_ctx **out, int geom, int nx, int ny, int nz, int ghost, double gamma,
                            const fargo_planet *planet, const fargo_params *prm)
{
    if (!out || !prm) return FARGO_ERR_BADARG;
    *out = nullptr;
    if (geom < 0 || geom > 2 || nx < 1 || ny < 1 || nz < 1) return FARGO_ERR_BADARG;
    if ((ny > 1 || nz > 1) && ghost < 2) return FARGO_ERR_BADARG;
    if (!prm->yfaces || !prm->zfaces || !(prm->xmax > prm->xmin)) return FARGO_ERR_BADARG;
    if (prm->precision != FARGO_F64 && prm->precision != FARGO_F32) return FARGO_ERR_BADARG;
    if (prm->shearing && (geom != FARGO_CART || !isfinite(prm->oort_a))) return FARGO_ERR_BADARG;
    if (gamma <= 0.0 && !prm->cs) return FARGO_ERR_BADARG;
    if (!(prm->cfl > 0.0)) return FARGO_ERR_BADARG;
    for (int s = 0; s < 2; s++)
        if (prm->bc_y[s] < 0 || prm->bc_y[s] > 3 || prm->bc_z[s] < 0 || prm->bc_z[s] > 3) return FARGO_ERR_BADARG;
    if (!periodic_ok(geom, nx, ny, nz, ghost, prm)) return FARGO_ERR_BADARG;
    if (planet && planet->q > 0.0 && !(planet->a > 0.0)) return FARGO_ERR_BADARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return FARGO_ERR_NOTBUILT;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_cfl_exact<double>) != cudaSuccess) return FARGO_ERR_NOTBUILT;

    fargo_ctx *c = new fargo_ctx();
    c->prec = prm->precision;
    c->nx = nx; c->ny = ny; c->nz = nz; c->g = ghost; c->geom = geom;
    c->star_mass = prm->star_mass;
    c->nyt = ny > 1 ? ny + 2 * ghost : 1;
    c->nzt = nz > 1 ? nz + 2 * ghost : 1;
    c->pitch = (nx + 31) / 32 * 32;
    c->esz = c->prec == FARGO_F64 ? 8 : 4;
    c->yfaces_store.assign(prm->yfaces, prm->yfaces + c->nyt + 1);
    c->zfaces_store.assign(prm->zfaces, prm->zfaces + c->nzt + 1);
    if (prm->stream) {
        c->stream = (cudaStream_t)prm->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return FARGO_ERR_CUDA;
        }
        c->own_stream = true;
    }
    MeshD &m = c->m;
    m.nx = nx; m.nyt = c->nyt; m.nzt = c->nzt;
    m.gy = ny > 1 ? ghost : 0; m.gz = nz > 1 ? ghost : 0; m.g = ghost;
    m.j0 = m.gy; m.j1 = m.gy + ny; m.k0 = m.gz; m.k1 = m.gz + nz;
    m.hasX = nx > 1; m.hasY = ny > 1; m.hasZ = nz > 1;
    m.geom = geom;
    m.iso = gamma <= 0.0;
    m.fargo = prm->fargo ? 1 : 0;
    m.av_lit = prm->av_dt_literal ? 1 : 0;
    m.has_nu = prm->nu ? 1 : 0;
    m.has_av = prm->cq > 0.0 ? 1 : 0;
    m.has_planet = planet && planet->q > 0.0;
    m.indirect = m.has_planet && planet->indirect;
    m.has_star = prm->star_mass > 0.0 && geom != FARGO_CART;
    for (int s = 0; s < 2; s++) { m.bcy[s] = prm->bc_y[s]; m.bcz[s] = prm->bc_z[s]; }
    m.pery = m.hasY && m.bcy[0] == BC_PERIODIC;
    m.perz = m.hasZ && m.bcz[0] == BC_PERIODIC;
    m.jf = m.j0 + (m.pery ? 0 : 1);
    m.kf = m.k0 + (m.perz ? 0 : 1);
    if ((long long)(c->nzt + 1) * (c->nyt + 1) * c->pitch >= (1LL << 31)) {
        // field indices are 32-bit in the kernels
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return FARGO_ERR_SIZE;
    }
    m.sj = c->pitch;
    m.sk = (c->nyt + 1) * c->pitch;
    m.ntot = (long long)(c->nzt + 1) * m.sk;
    m.gamma = gamma > 0.0 ? gamma : 1.0;
    m.g1 = m.gamma * (m.gamma - 1.0);
    m.cq = prm->cq;
    m.cfl = prm->cfl;
    m.omega = prm->omega_frame;
    m.shearing = prm->shearing ? 1 : 0;
    m.av_c2 = 4.0 * sqrt(2.0);
    if (m.has_planet) {
        m.pq = planet->q; m.pa = planet->a; m.pa3 = planet->a * planet->a * planet->a;
        m.peps = planet->eps; m.peps2 = planet->eps * planet->eps;
        const double om = sqrt((prm->star_mass + planet->q) / (planet->a * planet->a * planet->a));
        m.om_rel = om - prm->omega_frame;
    }
    fargo_params p2 = *prm;
    p2.yfaces = c->yfaces_store.data();
    p2.zfaces = c->zfaces_store.data();
    build_geometry(c, &p2, gamma, planet);
    int rc = FARGO_OK;
    void *p;
    if ((rc = dalloc(c, &p, sizeof(Scal)))) goto fail;
    c->sc = (Scal *)p;
    c->nrings_active = ny * nz;
    c->cfl_blocks = (c->nrings_active + 7) / 8;
    // v0 per ring, then the bulk angular rate v0 / (R dx) per ring (shear limit)
    if ((rc = dalloc(c, &p, sizeof(double) * 2 * (size_t)c->nyt * c->nzt))) goto fail;
    c->v0 = (double *)p;
    // Courant partials per block: the rate maximum, then the shear maximum
    if ((rc = dalloc(c, &p, sizeof(double) * 2 * c->cfl_blocks))) goto fail;
    c->part = (double *)p;
    if ((rc = dalloc(c, &p, sizeof(float) * c->nrings_active))) goto fail;
    c->ringmax = (float *)p;
    c->sum_blocks = 4 * 148;
    if ((rc = dalloc(c, &p, sizeof(double) * 6 * c->sum_blocks))) goto fail;
    c->part2 = (double *)p;
    if ((rc = dalloc(c, &p, sizeof(double) * 4))) goto fail;
    c->sums = (double *)p;
    // planet force: result, then the azimuth and ring tables of one call
    if ((rc = dalloc(c, &p, sizeof(double) * (4 + 2 * (size_t)c->pitch + 4 * (size_t)c->nrings_active)))) goto fail;
    c->pf = (double *)p;
    if ((rc = dalloc(c, &p, sizeof(double) * 4 * (kNbMax + 1)))) goto fail;
    c->pacc = (double *)p;
    if ((rc = dalloc(c, &p, sizeof(double) * (size_t)c->nrings_active))) goto fail;
    c->pprof = (double *)p;
    if ((rc = upload<double>(c, (const double **)&c->vol, c->hg.vol))) goto fail;
    if (c->prec == FARGO_F64) {
        if ((rc = alloc_fields<double>(c, c->b64))) goto fail;
        if ((rc = set_kernel_attrs<double>(c))) goto fail;
        if ((rc = build_sweep_maps<double>(c, c->b64))) goto fail;
    } else {
        if ((rc = alloc_fields<float>(c, c->b32))) goto fail;
        if ((rc = set_kernel_attrs<float>(c))) goto fail;
        if ((rc = build_sweep_maps<float>(c, c->b32))) goto fail;
    }
    {
        Scal s0{};
        s0.t = 0.0;
        s0.t_end = 1e300;
        if (cudaMemcpyAsync(c->sc, &s0, sizeof(Scal), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            rc = FARGO_ERR_CUDA;
            goto fail;
        }
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { rc = FARGO_ERR_CUDA; goto fail; }
    *out = c;
    return FARGO_OK;
fail:
    fargo_destroy(c);
    return rc;
}

extern "C" void fargo_destroy(fargo_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (void *p : c->allocs) cudaFree(p);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

// pointer of a state field
static void *field_ptr(fargo_ctx *c, int field)
{
    if (c->prec == FARGO_F64) {
        Fld<double> &A = c->b64.A;
        double *const *B = c->b64.tab.bfield;
        void *p[8] = {A.rho, A.e, A.vx, A.vy, A.vz, B[0], B[1], B[2]};
        return p[field];
    }
    Fld<float> &A = c->b32.A;
    float *const *B = c->b32.tab.bfield;
    void *p[8] = {A.rho, A.e, A.vx, A.vy, A.vz, B[0], B[1], B[2]};
    return p[field];
}

// Fields a context holds: the five of the gas, and B_x, B_y, B_z once a
// magnetic field is enabled.
static bool field_ok(const fargo_ctx *c, int field)
{
    return field >= 0 && (field <= 4 || (field <= 7 && c->m.mhd));
}

// Queue the copies of one field region on `stream` (no synchronisation).
static int queue_region(fargo_ctx *c, void *dev, void *host, int region, size_t bytes, int to_dev,
                        cudaStream_t stream)
{
    const size_t es = c->esz;
    const size_t pitchb = (size_t)c->pitch * es, rowb = (size_t)c->nx * es;
    cudaMemcpyKind kind = cudaMemcpyDefault;
    if (region == FARGO_FULL) {
        const size_t rows = (size_t)(c->nzt + 1) * (c->nyt + 1);
        if (bytes != rows * rowb) return FARGO_ERR_SIZE;
        if (to_dev) CK(cudaMemcpy2DAsync(dev, pitchb, host, rowb, rowb, rows, kind, stream));
        else CK(cudaMemcpy2DAsync(host, rowb, dev, pitchb, rowb, rows, kind, stream));
    } else if (region == FARGO_ACTIVE) {
        if (bytes != (size_t)c->nx * c->ny * c->nz * es) return FARGO_ERR_SIZE;
        const int gy = c->m.gy, gz = c->m.gz;
        for (int k = 0; k < c->nz; k++) {
            char *d = (char *)dev + ((size_t)(k + gz) * c->m.sk + (size_t)gy * c->pitch) * es;
            char *h = (char *)host + (size_t)k * c->ny * rowb;
            if (to_dev) CK(cudaMemcpy2DAsync(d, pitchb, h, rowb, rowb, c->ny, kind, stream));
            else CK(cudaMemcpy2DAsync(h, rowb, d, pitchb, rowb, c->ny, kind, stream));
        }
    } else {
        return FARGO_ERR_BADARG;
    }
    return FARGO_OK;
}

static int copy_region(fargo_ctx *c, void *dev, void *host, int region, size_t bytes, int to_dev)
{
    const int rc = queue_region(c, dev, host, region, bytes, to_dev, c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

// Batch field transfers (fargo_batch_set_field / fargo_batch_get_field in
// fargo_batch.cu): one field of member c queued on the batch's stream.
int fargo_queue_field(fargo_ctx *c, int field, int region, void *buf, size_t bytes, int to_dev, cudaStream_t s)
{
    if (!c || !buf || !field_ok(c, field)) return FARGO_ERR_BADARG;
    if (c->prec == FARGO_F32 && field == FARGO_VX) {
        // v_x crosses the boundary in v_x form (the stored values are v_x - vref)
        Buffers<float> &b = c->b32;
        int rc;
        if (to_dev) {
            if ((rc = vref_launch<float>(c, b, VREF_ABS, nullptr, s))) return rc;
            if ((rc = queue_region(c, b.A.vx, buf, region, bytes, 1, s))) return rc;
            return vref_refresh<float>(c, b, s);
        }
        // through the scratch increment buffer (free between steps); the copy
        // first brings the rows that belong to no ring
        CK(cudaMemcpyAsync(b.vB[0], b.A.vx, (size_t)c->m.ntot * sizeof(float), cudaMemcpyDeviceToDevice, s));
        if ((rc = vref_launch<float>(c, b, VREF_ABS, b.vB[0], s))) return rc;
        return queue_region(c, b.vB[0], buf, region, bytes, 0, s);
    }
    return queue_region(c, field_ptr(c, field), buf, region, bytes, to_dev, s);
}

extern "C" int fargo_set_field(fargo_ctx *c, int field, int region, const void *src, size_t bytes, int on_device)
{
    (void)on_device;
    if (!c || !src || !field_ok(c, field)) return FARGO_ERR_BADARG;
    const int rc = fargo_queue_field(c, field, region, (void *)src, bytes, 1, c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_get_field(fargo_ctx *c, int field, int region, void *dst, size_t bytes, int on_device)
{
    (void)on_device;
    if (!c || !dst || !field_ok(c, field)) return FARGO_ERR_BADARG;
    const int rc = fargo_queue_field(c, field, region, dst, bytes, 0, c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

static int read_scal(fargo_ctx *c, Scal *s)
{
    CK(cudaMemcpyAsync(s, c->sc, sizeof(Scal), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_set_time(fargo_ctx *c, double t, double t_end)
{
    if (!c || !(t_end >= t)) return FARGO_ERR_BADARG;
    Scal s;
    int rc = read_scal(c, &s);
    if (rc) return rc;
    s.t = t;
    s.t_end = t_end;
    s.nstep = 0;
    s.err = 0;
    s.fixed = 0;
    s.counter = 0;
    s.counter2 = 0;
    CK(cudaMemcpyAsync(c->sc, &s, sizeof(Scal), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_get_scalars(fargo_ctx *c, double *t, double *dt_last, long long *nsteps, int *err)
{
    if (!c) return FARGO_ERR_BADARG;
    Scal s;
    int rc = read_scal(c, &s);
    if (rc) return rc;
    if (t) *t = s.t;
    if (dt_last) *dt_last = s.dt;
    if (nsteps) *nsteps = s.nstep;
    if (err) *err = err_code(s.err);
    return FARGO_OK;
}

extern "C" int fargo_step(fargo_ctx *c, double *dt_out)
{
    if (!c) return FARGO_ERR_BADARG;
    int rc = launch_step(c);
    if (rc) return rc;
    if (dt_out) {
        Scal s;
        if ((rc = read_scal(c, &s))) return rc;
        *dt_out = s.dt;
        return err_code(s.err);
    }
    return FARGO_OK;
}

static int set_fixed(fargo_ctx *c, int fixed, double dt)
{
    // fixed and dt_fixed are adjacent ints/doubles of Scal; write the fields one by one
    CK(cudaMemcpyAsync(&c->sc->fixed, &fixed, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(&c->sc->dt_fixed, &dt, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_step_fixed(fargo_ctx *c, double dt)
{
    if (!c || !(dt > 0.0)) return FARGO_ERR_BADARG;
    int rc = set_fixed(c, 1, dt);
    if (rc) return rc;
    rc = launch_step(c);
    int rc2 = set_fixed(c, 0, 0.0);
    if (rc) return rc;
    if (rc2) return rc2;
    Scal s;
    if ((rc = read_scal(c, &s))) return rc;
    return err_code(s.err);
}

extern "C" int fargo_run_to(fargo_ctx *c, double t_end, long long max_steps, int poll, long long *steps_done)
{
    if (!c || poll < 1) return FARGO_ERR_BADARG;
    Scal s;
    int rc = read_scal(c, &s);
    if (rc) return rc;
    s.t_end = t_end;
    CK(cudaMemcpyAsync(&c->sc->t_end, &s.t_end, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const long long n0 = s.nstep;
    long long launched = 0;
    while (launched < max_steps) {
        const long long k = max_steps - launched < poll ? max_steps - launched : poll;
        for (long long q = 0; q < k; q++)
            if ((rc = launch_step(c))) return rc;
        launched += k;
        if ((rc = read_scal(c, &s))) return rc;
        if (s.err || s.t >= t_end) break;
    }
    if (steps_done) *steps_done = s.nstep - n0;
    return err_code(s.err);
}

template <typename T>
static int sums_impl(fargo_ctx *c, Buffers<T> &b, double out[3])
{
    const MeshD &m = c->m;
    SumInput<T> in{b.A.rho, m.iso ? nullptr : b.A.e, b.A.vx, c->vol, b.tab.Rd, m.omega,
                   m.nx, m.j0, m.j1, m.k0, m.k1, m.nyt, m.sj, m.sk};
    if (c->geom == FARGO_CART) in.wfr = b.tab.wfrd;   // the shearing sheet's 2 Omega_f y (0 otherwise)
    in.vref = b.tab.vrefd;                             // the reference form (FP32), else null
    k_sums<T><<<c->sum_blocks, 256, 0, c->stream>>>(in, c->part2, &c->sc->counter2, c->sums);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, c->sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

// ---------------------------------------------------------------------------
// Conserved totals without any device allocation: the block partials and
// the ticket counter of the sums kernel live in a file-scope device array
// instead of context memory.  The array is looked up once per device with
// cudaGetSymbolAddress (its name is only a host-side stand-in in host code);
// the lookup is guarded by a mutex so that host threads can make their first
// calls concurrently.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoallocMaxBlocks = 1184;                            // 8 blocks per SM on 148 SMs
constexpr int kNoallocScratch = 6 * kNoallocMaxBlocks + 2;         // partials + ticket word
constexpr int kNoallocMaxDevices = 64;
double *g_noalloc_ptr[kNoallocMaxDevices] = {};
std::mutex g_noalloc_mu;
}  // namespace
static __device__ __align__(256) double g_sums_scratch[kNoallocScratch];

template <typename T>
static int sums_noalloc_impl(const void *rho, const void *e, const void *vx, int nx, int ny, int nz, int ghost,
                             const double *vol, const double *R, const double *wframe, double omega, int nblocks,
                             double *out, cudaStream_t s, double *scratch)
{
    const int nyt = ny > 1 ? ny + 2 * ghost : 1;
    const int gy = ny > 1 ? ghost : 0, gz = nz > 1 ? ghost : 0;
    SumInput<T> in{(const T *)rho, (const T *)e, (const T *)vx, vol, R, omega,
                   nx, gy, gy + ny, gz, gz + nz, nyt, (long long)nx, (long long)(nyt + 1) * nx, wframe};
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + 6 * kNoallocMaxBlocks);
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));   // the ticket must start at zero
    k_sums<T><<<nblocks, 256, 0, s>>>(in, scratch, counter, out);
    CK(cudaGetLastError());
    return FARGO_OK;
}

extern "C" int fargo_sums_noalloc(const void *rho, const void *e, const void *vx, int precision, int nx, int ny,
                                  int nz, int ghost, const double *vol, const double *R, const double *wframe,
                                  double omega_frame, int nblocks, double *out, void *stream)
{
    if (!rho || !vx || !vol || !R || !out) return FARGO_ERR_BADARG;
    if (precision != FARGO_F64 && precision != FARGO_F32) return FARGO_ERR_BADARG;
    if (nx < 1 || ny < 1 || nz < 1 || ghost < 0) return FARGO_ERR_BADARG;
    if (nblocks < 0 || nblocks > kNoallocMaxBlocks) return FARGO_ERR_SIZE;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return FARGO_ERR_SIZE;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // first call on this device (with it current): resolve the array's device address
            double *p = nullptr;
            CK(cudaGetSymbolAddress((void **)&p, g_sums_scratch));
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    if (nblocks == 0) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        nblocks = 4 * sms < kNoallocMaxBlocks ? 4 * sms : kNoallocMaxBlocks;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == FARGO_F64)
        return sums_noalloc_impl<double>(rho, e, vx, nx, ny, nz, ghost, vol, R, wframe, omega_frame, nblocks, out,
                                         st, scratch);
    return sums_noalloc_impl<float>(rho, e, vx, nx, ny, nz, ghost, vol, R, wframe, omega_frame, nblocks, out, st,
                                    scratch);
}

// ---------------------------------------------------------------------------
// Force of the gas on a planet (kernels_planet.cuh).
// ---------------------------------------------------------------------------
template <typename T>
static int pforce_impl(fargo_ctx *c, Buffers<T> &b, PfPlanet pl, double eps, int bm08, double *out,
                       double *ring_fy = nullptr)
{
    const MeshD &m = c->m;
    cudaStream_t s = c->stream;
    T *tab = reinterpret_cast<T *>(c->pf + 4);
    const int nt = std::max(m.nx, c->nrings_active);
    k_pforce_tables<T><<<grid_for(nt, 256), 256, 0, s>>>(tab, m.nx, m.sj, m.xmin, m.dx, pl, b.tab.Rd, b.tab.zcd,
                                                          c->vol, m.j0, m.j1, m.k0, m.k1, m.nyt);
    PForceArgs<T> a{};
    a.rho = b.A.rho;
    a.tab = tab;
    a.pl = pl;
    a.eps2 = (T)(eps * eps);
    a.nx = m.nx;
    a.j0 = m.j0;
    a.j1 = m.j1;
    a.k0 = m.k0;
    a.k1 = m.k1;
    a.nyt = m.nyt;
    a.sj = m.sj;
    a.sk = m.sk;
    // one resident wave; part2 holds 3 partials for up to 2 * sum_blocks blocks
    const int grid = std::min(148 * pforce_blocks_per_sm<T>(), 2 * c->sum_blocks);
    a.ring_fy = ring_fy;
    if (ring_fy && bm08)
        k_planet_force<T, true, true><<<grid, 256, 0, s>>>(a, c->part2, &c->sc->counter2, out);
    else if (ring_fy)
        k_planet_force<T, false, true><<<grid, 256, 0, s>>>(a, c->part2, &c->sc->counter2, out);
    else if (bm08)
        k_planet_force<T, true><<<grid, 256, 0, s>>>(a, c->part2, &c->sc->counter2, out);
    else
        k_planet_force<T, false><<<grid, 256, 0, s>>>(a, c->part2, &c->sc->counter2, out);
    CK(cudaGetLastError());
    return FARGO_OK;
}

static int pforce_any(fargo_ctx *c, PfPlanet pl, double eps, int bm08, double *out)
{
    return c->prec == FARGO_F64 ? pforce_impl<double>(c, c->b64, pl, eps, bm08, out)
                                : pforce_impl<float>(c, c->b32, pl, eps, bm08, out);
}

static bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

static int pforce_check(fargo_ctx *c, const double rp[3], double eps, const double *out)
{
    if (!c || !rp || !out || !(eps >= 0.0) || !isfinite(eps) || !isfinite(rp[0]) || !isfinite(rp[1]) ||
        !isfinite(rp[2]))
        return FARGO_ERR_BADARG;
    if (c->geom == FARGO_CART) return FARGO_ERR_BADARG;
    if (!aligned8(out)) return FARGO_ERR_BADARG;
    return FARGO_OK;
}

extern "C" int fargo_planet_force_async(fargo_ctx *c, const double rp[3], double eps, int bm08, double *out)
{
    int rc = pforce_check(c, rp, eps, out);
    if (rc) return rc;
    return pforce_any(c, PfPlanet{rp[0], rp[1], rp[2], nullptr}, eps, bm08, out);
}

extern "C" int fargo_planet_force(fargo_ctx *c, const double rp[3], double eps, int bm08, double out[4])
{
    int rc = pforce_check(c, rp, eps, out);
    if (rc) return rc;
    if ((rc = pforce_any(c, PfPlanet{rp[0], rp[1], rp[2], nullptr}, eps, bm08, c->pf))) return rc;
    CK(cudaMemcpyAsync(out, c->pf, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_planet_torque_profile(fargo_ctx *c, const double rp[3], double eps, int bm08, double *ring,
                                           double out[4])
{
    int rc = pforce_check(c, rp, eps, ring);
    if (rc) return rc;
    rc = c->prec == FARGO_F64
             ? pforce_impl<double>(c, c->b64, PfPlanet{rp[0], rp[1], rp[2], nullptr}, eps, bm08, c->pf, c->pprof)
             : pforce_impl<float>(c, c->b32, PfPlanet{rp[0], rp[1], rp[2], nullptr}, eps, bm08, c->pf, c->pprof);
    if (rc) return rc;
    CK(cudaMemcpyAsync(ring, c->pprof, sizeof(double) * (size_t)c->nrings_active, cudaMemcpyDeviceToHost,
                       c->stream));
    double tot[4];
    CK(cudaMemcpyAsync(tot, c->pf, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double Rp = sqrt(rp[0] * rp[0] + rp[1] * rp[1]);
    for (int r = 0; r < c->nrings_active; r++) ring[r] *= Rp;
    if (out)
        for (int q = 0; q < 4; q++) out[q] = tot[q];
    return FARGO_OK;
}

extern "C" int fargo_planets_force_async(fargo_ctx *c, int n, const double *y, int stride, double eps, int bm08,
                                         double *out)
{
    if (!c || !y || !out || n < 1 || stride < 3 || !(eps >= 0.0) || !isfinite(eps)) return FARGO_ERR_BADARG;
    if (c->geom == FARGO_CART || !aligned8(y) || !aligned8(out)) return FARGO_ERR_BADARG;
    if (n > kNbMax) return FARGO_ERR_SIZE;
    for (int i = 0; i < n; i++) {
        // positions and forces in the integrator's axes (the mesh turned by its frame angle)
        const int rc = pforce_any(c, PfPlanet{0.0, 0.0, 0.0, y + (size_t)stride * i, c->m.fr0, c->m.omega, c->sc},
                                  eps, bm08, out + 4 * i);
        if (rc) return rc;
    }
    return FARGO_OK;
}

static int nbody_launch(int n, double *y, const double *mass, double mstar, double h, const double *h_dev,
                        const double *kick, int kick_stride, const double *kick_star, int indirect,
                        cudaStream_t s)
{
    NbArgs a{};
    a.y = y;
    a.mass = mass;
    a.kick = kick;
    a.kick_star = kick_star;
    a.h_dev = h_dev;
    a.mstar = mstar;
    a.h = h;
    a.n = n;
    a.kick_stride = kick_stride;
    a.indirect = indirect ? 1 : 0;
    k_nbody_rk5<<<1, 32, 0, s>>>(a);
    CK(cudaGetLastError());
    return FARGO_OK;
}

extern "C" int fargo_nbody_rk5_async(int n, double *y, const double *mass, double mstar, double h,
                                     const double *h_dev, const double *kick, int kick_stride,
                                     const double *kick_star, int indirect, void *stream)
{
    if (!y || !mass || n < 1 || !(mstar >= 0.0) || !isfinite(mstar) || !isfinite(h)) return FARGO_ERR_BADARG;
    if (kick && kick_stride < 3) return FARGO_ERR_BADARG;
    if (kick_star && !kick) return FARGO_ERR_BADARG;
    if (!aligned8(y) || !aligned8(mass) || !aligned8(h_dev) || !aligned8(kick) || !aligned8(kick_star))
        return FARGO_ERR_BADARG;
    if (n > kNbMax) return FARGO_ERR_SIZE;
    return nbody_launch(n, y, mass, mstar, h, h_dev, kick, kick_stride, kick_star, indirect,
                        static_cast<cudaStream_t>(stream));
}

extern "C" int fargo_planets_advance_async(fargo_ctx *c, int n, double *y, const double *mass, double eps, int bm08,
                                           int indirect)
{
    if (!c || !y || !mass || n < 1 || !(eps >= 0.0) || !isfinite(eps)) return FARGO_ERR_BADARG;
    if (c->geom == FARGO_CART || !aligned8(y) || !aligned8(mass)) return FARGO_ERR_BADARG;
    if (n > kNbMax) return FARGO_ERR_SIZE;
    int rc = fargo_planets_force_async(c, n, y, 6, eps, bm08, c->pacc);
    if (rc) return rc;
    const double *star = nullptr;
    if (indirect) {
        // the star sits at the origin, which no cell of a cylindrical or spherical mesh contains
        if ((rc = pforce_any(c, PfPlanet{0.0, 0.0, 0.0, nullptr, c->m.fr0, c->m.omega, c->sc}, 0.0, 0,
                             c->pacc + 4 * kNbMax)))
            return rc;
        star = c->pacc + 4 * kNbMax;
    }
    return nbody_launch(n, y, mass, c->star_mass, 0.0, &c->sc->dt, c->pacc, 4, star, indirect, c->stream);
}

// Frame change (Sec. 3.2, Eq. 13): v_phi -= (Omega' - Omega) R at every
// v_phi point of the array, ghosts included (frozen ghosts hold state in the
// frame too).  R is the ring's lever arm at the face centre where v_phi
// lives (cylindrical radius).  Formed in FP64 and rounded once.
template <typename T>
__global__ void __launch_bounds__(256) k_change_frame(T *vx, const double *Rd, double dom, int nx, int nyt, int nzt,
                                                      int sj, int sk)
{
    const long long n = (long long)nx * nyt * nzt;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx);
        const long long r = t / nx;
        const int j = (int)(r % nyt), k = (int)(r / nyt);
        const long long c = (long long)k * sk + (long long)j * sj + i;
        vx[c] = (T)((double)vx[c] - dom * Rd[(size_t)k * nyt + j]);
    }
}

// rebase: in FP32, go through the v_x form and choose the references afresh
// in the new frame (a change of any size); otherwise correct the stored
// v_x - vref directly and refresh the frame shifts only (small changes, as
// when the frame tracks a planet: the stored values stay small).
template <typename T>
static int change_frame_impl(fargo_ctx *c, Buffers<T> &b, double omega_new, bool rebase)
{
    Scal sh;
    int rc = read_scal(c, &sh);   // the current time (synchronises)
    if (rc) return rc;
    MeshD &m = c->m;
    const double dom = omega_new - m.omega;
    const long long n = (long long)m.nx * m.nyt * m.nzt;
    if (rebase && (rc = vref_launch<T>(c, b, VREF_ABS, nullptr, c->stream))) return rc;
    k_change_frame<T><<<grid_for(n, 256), 256, 0, c->stream>>>(b.A.vx, b.tab.Rd, dom, m.nx, m.nyt, m.nzt, m.sj,
                                                                 m.sk);
    CK(cudaGetLastError());
    // the planet keeps its azimuth: php0 + om_rel t is continuous at t
    if (m.has_planet) {
        m.php0 += dom * sh.t;
        m.om_rel -= dom;
    }
    // and so does the mesh's angle to the planetary integrator's axes
    m.fr0 -= dom * sh.t;
    m.omega = omega_new;
    b.tab.omega = (T)omega_new;
    if (rebase) rc = vref_refresh<T>(c, b, c->stream);
    else rc = vref_launch<T>(c, b, VREF_TABLES, nullptr, c->stream);
    if (rc) return rc;
    if (c->gexec) {   // the captured step holds the old frame
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_change_frame(fargo_ctx *c, double omega_new)
{
    if (!c || !isfinite(omega_new) || c->geom == FARGO_CART) return FARGO_ERR_BADARG;
    if (c->batch_refs > 0) return FARGO_ERR_BADARG;
    return c->prec == FARGO_F64 ? change_frame_impl<double>(c, c->b64, omega_new, true)
                                : change_frame_impl<float>(c, c->b32, omega_new, true);
}

extern "C" int fargo_track_frame(fargo_ctx *c, const double *y, int index, double *omega_out)
{
    if (!c || !y || index < 0 || index >= kNbMax || c->geom == FARGO_CART || c->batch_refs > 0 || !aligned8(y))
        return FARGO_ERR_BADARG;
    double s[6];
    CK(cudaMemcpyAsync(s, y + 6 * (size_t)index, sizeof(s), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // the body's angular velocity about the polar axis (Sec. 3.2: the x axis tracks it)
    const double r2 = s[0] * s[0] + s[1] * s[1];
    const double rate = (s[0] * s[4] - s[1] * s[3]) / r2;
    if (!(r2 > 0.0) || !isfinite(rate)) return FARGO_ERR_BADARG;
    const int rc = c->prec == FARGO_F64 ? change_frame_impl<double>(c, c->b64, rate, false)
                                        : change_frame_impl<float>(c, c->b32, rate, false);
    if (!rc && omega_out) *omega_out = rate;
    return rc;
}

// ---------------------------------------------------------------------------
// Magnetic field (Sec. 3.5): B, the EMFs and the tension's output
// velocities, allocated once and zero.  FP32 contexts switch the reference
// form of v_x off (every vref 0), since the MHD kernels read v_x itself.
// ---------------------------------------------------------------------------
template <typename T>
static int enable_mhd_impl(fargo_ctx *c, Buffers<T> &b)
{
    const size_t n = (size_t)c->m.ntot * sizeof(T);
    int rc;
    void *p;
    if (!b.tab.bfield[0]) {
        for (int d = 0; d < 3; d++) {
            if ((rc = dalloc(c, &p, n))) return rc;
            b.tab.bfield[d] = (T *)p;
            if ((rc = dalloc(c, &p, n))) return rc;
            b.ef[d] = (T *)p;
            if ((rc = dalloc(c, &p, n))) return rc;
            b.vM[d] = (T *)p;
        }
        // inverse centre-to-centre distances along Y and Z, (w[n-1] + w[n]) / 2
        auto idc = [](const std::vector<double> &w) {
            std::vector<double> o(w.size(), 0.0);
            for (size_t q = 1; q < w.size(); q++) o[q] = 1.0 / (0.5 * (w[q - 1] + w[q]));
            return o;
        };
        if ((rc = upload<T>(c, &b.tab.mh_idcy, idc(c->hg.dy)))) return rc;
        if ((rc = upload<T>(c, &b.tab.mh_idcz, idc(c->hg.dz)))) return rc;
    }
    if (c->m.fargo && !b.v0all) {   // orbital advection of the field (Sec. 3.6)
        if ((rc = dalloc(c, &p, sizeof(double) * (size_t)c->nyt * c->nzt))) return rc;
        b.v0all = (double *)p;
        if ((rc = dalloc(c, &p, n))) return rc;
        b.dvx = (T *)p;
    }
    if ((rc = vref_launch<T>(c, b, VREF_ABS, nullptr, c->stream))) return rc;
    c->m.mhd = 1;
    if ((rc = vref_refresh<T>(c, b, c->stream))) return rc;
    // the Y / Z sweeps read v_y, v_z through tensor maps: with magnetic
    // forces they read the tension's output
    return build_sweep_maps<T>(c, b);
}

extern "C" int fargo_enable_mhd(fargo_ctx *c, int passive, double eta)
{
    if (!c || c->geom != FARGO_CART || c->batch_refs > 0) return FARGO_ERR_BADARG;
    if (!(eta >= 0.0) || !isfinite(eta)) return FARGO_ERR_BADARG;
    c->m.mhd_passive = passive ? 1 : 0;
    c->m.eta = eta;
    const int rc = c->prec == FARGO_F64 ? enable_mhd_impl<double>(c, c->b64) : enable_mhd_impl<float>(c, c->b32);
    if (rc) return rc;
    if (c->gexec) {   // the captured step has no MHD launches
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_set_planet_source(fargo_ctx *c, const double *pos, int n, int stride, const double *mass)
{
    if (!c || !c->m.has_planet || c->geom == FARGO_CART) return FARGO_ERR_BADARG;
    if (c->batch_refs > 0 || !aligned8(pos) || !aligned8(mass)) return FARGO_ERR_BADARG;
    if (pos && (n < 1 || stride < 3 || (n > 1 && !mass))) return FARGO_ERR_BADARG;
    if (pos && n > kPotPlanets) return FARGO_ERR_SIZE;
    c->m.pl_pos = pos;
    c->m.pl_n = pos ? n : 0;
    c->m.pl_stride = pos ? stride : 0;
    c->m.pl_mass = pos ? mass : nullptr;
    if (c->gexec) {   // the captured step holds the old mesh record
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return FARGO_OK;
}

extern "C" int fargo_sums(fargo_ctx *c, double out[3])
{
    if (!c || !out) return FARGO_ERR_BADARG;
    return c->prec == FARGO_F64 ? sums_impl<double>(c, c->b64, out) : sums_impl<float>(c, c->b32, out);
}

// ---------------------------------------------------------------------------
// Single sub-steps for kernel-level parity tests.
// ---------------------------------------------------------------------------
template <typename T>
static int debug_impl(fargo_ctx *c, Buffers<T> &b, int phase, double dt)
{
    const MeshD &m = c->m;
    cudaStream_t s = c->stream;
    const int bs = 256;
    const size_t nbytes = (size_t)m.ntot * sizeof(T);
    Fld<T> A = b.A;
    Fld<T> VB = {A.rho, A.e, b.vB[0], b.vB[1], b.vB[2]};
    QSet<T> qa = qset<T>(c, A.rho, A.e, b.piA), qb = qset<T>(c, b.rhoB, b.eB, b.piB);
    Scal sh;
    int rc = read_scal(c, &sh);
    if (rc) return rc;
    sh.dt = dt;
    sh.dtf = (float)dt;
    sh.err = 0;
    sh.fixed = phase == 1 ? 0 : 1;
    sh.dt_fixed = dt;
    sh.counter = 0;
    if (m.has_planet) {
        const double ph = m.php0 + m.om_rel * sh.t;
        sh.xp = m.pa * cos(ph);
        sh.yp = m.pa * sin(ph);
    }
    CK(cudaMemcpyAsync(c->sc, &sh, sizeof(Scal), cudaMemcpyHostToDevice, s));
    auto copyv = [&](T *const *dst, T *const *src) -> int {
        // v_z only exists with a Z direction
        for (int q = 0; q < (m.hasZ ? 3 : 2); q++)
            CK(cudaMemcpyAsync(dst[q], src[q], nbytes, cudaMemcpyDeviceToDevice, s));
        return FARGO_OK;
    };
    T *va[3] = {A.vx, A.vy, A.vz};
    MagF<T> MB{};
    if (m.mhd)
        for (int d = 0; d < 3; d++) MB.b[d] = b.tab.bfield[d];
    if (phase >= 10 && !m.mhd) return FARGO_ERR_BADARG;
    const dim3 fg(cell_grid_all(m, c->cell_bs).x, m.nyt + 1, m.nzt + 1);
    const dim3 fb = cell_block(m, c->cell_bs);
    switch (phase) {
    case 0:
        if (m.hasY) k_bc_y<T><<<grid_for((long long)m.nx * (m.nzt + 1) * 2, bs), bs, 0, s>>>(m, A, c->sc, 1, b.tab.vref, MB);
        if (m.hasZ) k_bc_z<T><<<grid_for((long long)m.nx * (m.nyt + 1) * 2, bs), bs, 0, s>>>(m, A, c->sc, 1, b.tab.vref, MB);
        break;
    case 1:
        k_cfl_screen<T><<<c->cfl_blocks, 256, 0, s>>>(m, b.tab, A, c->v0, c->ringmax, c->part, c->sc,
                                                      c->nrings_active);
        k_cfl_exact<T><<<cfl_exact_grid(c->cfl_blocks), 256, 0, s>>>(m, b.tab, A, c->v0, c->ringmax, c->part, c->sc,
                                                     c->nrings_active);
        break;
    case 2:
        // the screening launch fills the per-step planet angle tables
        k_cfl_screen<T><<<c->cfl_blocks, 256, 0, s>>>(m, b.tab, A, c->v0, c->ringmax, c->part, c->sc,
                                                      c->nrings_active);
        launch_source<T>(SRC_SUB1, m, cell_grid_all(m, c->cell_bs), cell_block(m, c->cell_bs), s, b.tab, A, VB,
                         QSet<T>{}, c->sc);
        if ((rc = copyv(va, b.vB))) return rc;
        launch_periodic<T>(m, per_fields<T>(m, A, true, false), c->sc, s);
        break;
    case 3:
        if ((rc = copyv(b.vB, va))) return rc;
        launch_source<T>(SRC_AV, m, cell_grid_all(m, c->cell_bs), cell_block(m, c->cell_bs), s, b.tab, VB, A,
                         QSet<T>{}, c->sc);
        launch_periodic<T>(m, per_fields<T>(m, A, true, true), c->sc, s);
        break;
    case 4: {
        if (!m.has_nu) break;
        QSet<T> tau{};
        for (int q = 0; q < 6; q++) tau.q[q] = b.piB[q];
        tau.nq = 6;
        launch_source<T>(SRC_TAU, m, tau_grid(m, c->cell_bs), cell_block(m, c->cell_bs), s, b.tab, A, VB, tau, c->sc);
        QSet<T> diag = tau;
        diag.nq = m.hasZ ? 3 : 2;
        launch_periodic<T>(m, per_quantities<T>(diag, diag), c->sc, s);
        launch_source<T>(SRC_VAPPLY, m, cell_grid_all(m, c->cell_bs), cell_block(m, c->cell_bs), s, b.tab, A, VB, tau,
                         c->sc);
        if ((rc = copyv(va, b.vB))) return rc;
        launch_periodic<T>(m, per_fields<T>(m, A, true, false), c->sc, s);
        break;
    }
    case 5:
        launch_tx<T>(m, b.tab, A, qa, c->v0, c->sc, c->tx_rs, s);
        launch_periodic<T>(m, per_quantities<T>(qa, qa), c->sc, s);
        break;
    case 6:
    case 7: {
        if ((phase == 6 && !m.hasY) || (phase == 7 && !m.hasZ)) break;
        for (int q = 0; q < qa.nq; q++) CK(cudaMemcpyAsync(qb.q[q], qa.q[q], nbytes, cudaMemcpyDeviceToDevice, s));
        SweepMaps mp{};
        if ((rc = encode_sweep_maps<T>(c, &mp, qa, qa, phase == 6 ? A.vy : A.vz))) return rc;
        if (phase == 6) launch_sweep_tma<T, 1>(m, b.tab, mp, qb, c->sc, qa.nq, s);
        else launch_sweep_tma<T, 2>(m, b.tab, mp, qb, c->sc, qa.nq, s);
        for (int q = 0; q < qa.nq; q++) CK(cudaMemcpyAsync(qa.q[q], qb.q[q], nbytes, cudaMemcpyDeviceToDevice, s));
        launch_periodic<T>(m, per_quantities<T>(qa, qa), c->sc, s);
        break;
    }
    case 8:
        launch_newvel<T>(m, cell_grid_all(m, c->cell_bs), cell_block(m, c->cell_bs), s, b.tab, qa, A, A, c->sc, 0);
        launch_periodic<T>(m, per_fields<T>(m, A, true, false), c->sc, s);
        break;
    case 9:
        if (m.fargo && m.hasX) {
            launch_orb<T>(m, b.tab, qa, c->v0, c->sc, c->nrings_active, c->orb_rs, s);
            launch_periodic<T>(m, per_quantities<T>(qa, qa), c->sc, s);
        }
        break;
    case 10:   // the magnetic pressure (cell 7a), in place on the state's velocities
        if (!m.mhd_passive) k_mhd_pressure<T><<<fg, fb, 0, s>>>(m, b.tab, A, c->sc);
        launch_periodic<T>(m, per_fields<T>(m, A, true, false), c->sc, s);
        break;
    case 11: {  // the EMFs (cells 8a-8c) of the state, into the aux arrays 7-9
        Fld<T> VM = {A.rho, A.e, b.vM[0], b.vM[1], b.vM[2]};
        k_mhd_edges<T><<<fg, fb, 0, s>>>(m, b.tab, A, VM, b.ef[0], b.ef[1], b.ef[2], c->sc, 1, 0, (const T *)nullptr);
        break;
    }
    case 12: {  // the magnetic tension (cell 8d), back into the state's velocities
        if (m.mhd_passive) break;
        Fld<T> VM = {A.rho, A.e, b.vM[0], b.vM[1], b.vM[2]};
        k_mhd_edges<T><<<fg, fb, 0, s>>>(m, b.tab, A, VM, b.ef[0], b.ef[1], b.ef[2], c->sc, 0, 1, (const T *)nullptr);
        if ((rc = copyv(va, b.vM))) return rc;
        if (!m.hasZ) CK(cudaMemcpyAsync(va[2], b.vM[2], nbytes, cudaMemcpyDeviceToDevice, s));
        launch_periodic<T>(m, per_fields<T>(m, A, true, false), c->sc, s);
        break;
    }
    case 13:   // the constrained transport (cell 10) with the aux EMFs
        k_mhd_ct<T><<<fg, fb, 0, s>>>(m, b.tab, b.ef[0], b.ef[1], b.ef[2], c->sc);
        launch_periodic<T>(m, per_field<T>(m, b.tab), c->sc, s);
        break;
    default:
        return FARGO_ERR_BADARG;
    }
    CK(cudaGetLastError());
    // restore time and flags (phase 8 advances t)
    Scal s2;
    if ((rc = read_scal(c, &s2))) return rc;
    if (phase != 1) {
        s2.t = sh.t;
        s2.nstep = sh.nstep;
    }
    s2.fixed = 0;
    CK(cudaMemcpyAsync(c->sc, &s2, sizeof(Scal), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return err_code(s2.err);
}

extern "C" int fargo_debug_phase(fargo_ctx *c, int phase, double dt)
{
    if (!c) return FARGO_ERR_BADARG;
    if (phase != 0 && phase != 1 && !(dt > 0.0)) return FARGO_ERR_BADARG;
    if (phase == 0 || phase == 1) dt = dt > 0.0 ? dt : 1.0;
    return c->prec == FARGO_F64 ? debug_impl<double>(c, c->b64, phase, dt) : debug_impl<float>(c, c->b32, phase, dt);
}

static int aux_ptr(fargo_ctx *c, int which, void **p, size_t *bytes, int *pitched)
{
    if (which >= 0 && which < 6) {
        *p = c->prec == FARGO_F64 ? (void *)c->b64.piA[which] : (void *)c->b32.piA[which];
        *bytes = (size_t)(c->nzt + 1) * (c->nyt + 1) * c->nx * c->esz;
        *pitched = 1;
        return FARGO_OK;
    }
    if (which == 6) {
        *p = c->v0;
        *bytes = (size_t)c->nzt * c->nyt * sizeof(double);
        *pitched = 0;
        return FARGO_OK;
    }
    if (which >= 7 && which < 10 && c->m.mhd) {   // the EMFs e_x, e_y, e_z
        *p = c->prec == FARGO_F64 ? (void *)c->b64.ef[which - 7] : (void *)c->b32.ef[which - 7];
        *bytes = (size_t)(c->nzt + 1) * (c->nyt + 1) * c->nx * c->esz;
        *pitched = 1;
        return FARGO_OK;
    }
    return FARGO_ERR_BADARG;
}

extern "C" int fargo_get_aux(fargo_ctx *c, int which, void *dst, size_t bytes)
{
    if (!c || !dst) return FARGO_ERR_BADARG;
    void *p;
    size_t want;
    int pitched;
    int rc = aux_ptr(c, which, &p, &want, &pitched);
    if (rc) return rc;
    if (bytes != want) return FARGO_ERR_SIZE;
    if (pitched) return copy_region(c, p, dst, FARGO_FULL, bytes, 0);
    CK(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_set_aux(fargo_ctx *c, int which, const void *src, size_t bytes)
{
    if (!c || !src) return FARGO_ERR_BADARG;
    void *p;
    size_t want;
    int pitched;
    int rc = aux_ptr(c, which, &p, &want, &pitched);
    if (rc) return rc;
    if (bytes != want) return FARGO_ERR_SIZE;
    if (pitched) return copy_region(c, p, (void *)src, FARGO_FULL, bytes, 1);
    CK(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FARGO_OK;
}

extern "C" int fargo_profile_step(fargo_ctx *c, int max_kernels, float *ms, int *n_out, const char **names)
{
    if (!c || !ms || !n_out || max_kernels < 1) return FARGO_ERR_BADARG;
    Prof prof{};
    for (int i = 0; i <= kProfMax; i++) CK(cudaEventCreate(&prof.ev[i]));
    CK(cudaEventRecord(prof.ev[0], c->stream));
    int rc = c->prec == FARGO_F64 ? enqueue_step<double>(c, c->b64, &prof) : enqueue_step<float>(c, c->b32, &prof);
    if (rc == FARGO_OK) {
        CK(cudaStreamSynchronize(c->stream));
        const int n = prof.n < max_kernels ? prof.n : max_kernels;
        for (int i = 0; i < n; i++) {
            CK(cudaEventElapsedTime(&ms[i], prof.ev[i], prof.ev[i + 1]));
            if (names) names[i] = prof.name[i];
        }
        *n_out = n;
    }
    for (int i = 0; i <= kProfMax; i++) cudaEventDestroy(prof.ev[i]);
    return rc;
}

// ---------------------------------------------------------------------------
// Autotuner of the launch shapes that do not change results: the azimuths
// per block of the per-cell kernels (the same compiled kernel on any block
// width) and the segment lengths of the Y / Z sweeps (each column marches
// the same arithmetic whatever the segmentation).  Coordinate search with
// per-launch CUDA events on `reps` steps per candidate, the state restored
// from a snapshot before every trial step and at the end.
// ---------------------------------------------------------------------------
namespace {
struct Snapshot {
    std::vector<void *> bufs;
    ~Snapshot()
    {
        for (void *p : bufs) cudaFree(p);
    }
};
}  // namespace

template <typename T>
static int snapshot_copy(fargo_ctx *c, Buffers<T> &b, Snapshot &sn, bool save)
{
    const size_t nbytes = (size_t)c->m.ntot * sizeof(T);
    T *f[5] = {b.A.rho, b.A.e, b.A.vx, b.A.vy, b.A.vz};
    void *aux[2] = {c->sc, c->v0};
    const size_t auxb[2] = {sizeof(Scal), sizeof(double) * (size_t)c->nyt * c->nzt};
    if (save && sn.bufs.empty()) {
        for (int q = 0; q < 7; q++) {
            void *p = nullptr;
            CK(cudaMalloc(&p, q < 5 ? nbytes : auxb[q - 5]));
            sn.bufs.push_back(p);
        }
    }
    for (int q = 0; q < 7; q++) {
        void *live = q < 5 ? (void *)f[q] : aux[q - 5];
        const size_t n = q < 5 ? nbytes : auxb[q - 5];
        if (save) CK(cudaMemcpyAsync(sn.bufs[q], live, n, cudaMemcpyDeviceToDevice, c->stream));
        else CK(cudaMemcpyAsync(live, sn.bufs[q], n, cudaMemcpyDeviceToDevice, c->stream));
    }
    return FARGO_OK;
}

// Summed device time (ms) of the launches named in `names` over `reps`
// steps of the current configuration, the state restored before each.
template <typename T>
static int time_step_kernels(fargo_ctx *c, Buffers<T> &b, Snapshot &sn, int reps, const char *const *names,
                             int nnames, double *ms_out)
{
    double tot = 0.0;
    for (int r = 0; r < reps; r++) {
        int rc = snapshot_copy<T>(c, b, sn, false);
        if (rc) return rc;
        Prof prof{};
        for (int i = 0; i <= kProfMax; i++) CK(cudaEventCreate(&prof.ev[i]));
        CK(cudaEventRecord(prof.ev[0], c->stream));
        rc = enqueue_step<T>(c, b, &prof);
        if (rc == FARGO_OK) {
            CK(cudaStreamSynchronize(c->stream));
            for (int i = 0; i < prof.n; i++)
                for (int q = 0; q < nnames; q++)
                    if (!strcmp(prof.name[i], names[q])) {
                        float ms = 0.0f;
                        CK(cudaEventElapsedTime(&ms, prof.ev[i], prof.ev[i + 1]));
                        if (r > 0) tot += ms;   // the first repetition warms up
                    }
        }
        for (int i = 0; i <= kProfMax; i++) cudaEventDestroy(prof.ev[i]);
        if (rc) return rc;
    }
    *ms_out = tot;
    return FARGO_OK;
}

template <typename T>
static int autotune_impl(fargo_ctx *c, Buffers<T> &b, int reps, int *cfg)
{
    Snapshot sn;
    int rc = snapshot_copy<T>(c, b, sn, true);
    if (rc) return rc;
    const MeshD &m = c->m;
    const char *cell_names[] = {"substep1", "artvisc", "visc_tau", "visc_apply", "newvel"};
    // the per-cell kernels are compiled for at most 256 threads per block
    const int cand_bs[] = {64, 128, 256};
    double best = 1e300;
    int best_bs = c->cell_bs;
    for (int bs : cand_bs) {
        if ((m.nx + 31) / 32 * 32 < bs && bs != cand_bs[0]) continue;   // wider than a row
        c->cell_bs = bs;
        double t;
        if ((rc = time_step_kernels<T>(c, b, sn, reps, cell_names, 5, &t))) return rc;
        if (t < best) {
            best = t;
            best_bs = bs;
        }
    }
    c->cell_bs = best_bs;
    const int cand_seg[] = {16, 32, 64, 128, 256};
    for (int axis = 1; axis <= 2; axis++) {
        if ((axis == 1 && !m.hasY) || (axis == 2 && !m.hasZ)) continue;
        const int np = axis == 1 ? m.j1 - m.j0 : m.k1 - m.k0;
        int &seg = axis == 1 ? c->seg_y : c->seg_z;
        const char *nm[] = {axis == 1 ? "transport_y" : "transport_z"};
        best = 1e300;
        int best_seg = seg;
        for (int sl : cand_seg) {
            if (sl > np && sl != cand_seg[0]) continue;
            seg = sl < np ? sl : np;
            double t;
            if ((rc = time_step_kernels<T>(c, b, sn, reps, nm, 1, &t))) return rc;
            if (t < best) {
                best = t;
                best_seg = seg;
            }
        }
        seg = best_seg;
    }
    if ((rc = snapshot_copy<T>(c, b, sn, false))) return rc;
    CK(cudaStreamSynchronize(c->stream));
    // the captured step used the old shapes
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    if (cfg) {
        cfg[0] = c->cell_bs;
        cfg[1] = c->seg_y;
        cfg[2] = c->seg_z;
    }
    return FARGO_OK;
}

extern "C" int fargo_autotune(fargo_ctx *c, int reps, int *cfg)
{
    if (!c || reps < 2) return FARGO_ERR_BADARG;
    return c->prec == FARGO_F64 ? autotune_impl<double>(c, c->b64, reps, cfg)
                                : autotune_impl<float>(c, c->b32, reps, cfg);
}

extern "C" int fargo_set_launch_shape(fargo_ctx *c, int cell_bs, int seg_y, int seg_z)
{
    if (!c || (cell_bs != 64 && cell_bs != 128 && cell_bs != 256) || seg_y < 0 || seg_z < 0)
        return FARGO_ERR_BADARG;
    c->cell_bs = cell_bs;
    c->seg_y = seg_y;
    c->seg_z = seg_z;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    return FARGO_OK;
}

// ---------------------------------------------------------------------------
// Failure-detection check of the bounded waits: an mbarrier that expects one
// arrival which never comes, waited on with a given poll budget.
// ---------------------------------------------------------------------------
__global__ void k_wait_probe(unsigned limit, int *flag)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool done = mbar_wait(&bar, 0, limit);
    if (!done && threadIdx.x == 0) atomicOr(flag, kErrTimeout);
}

extern "C" int fargo_debug_wait_timeout(unsigned spin_limit)
{
    if (spin_limit < 1 || spin_limit > (1u << 22)) return FARGO_ERR_BADARG;
    int *d = nullptr, h = 0;
    CK(cudaMalloc(&d, sizeof(int)));
    int rc = FARGO_OK;
    if (cudaMemset(d, 0, sizeof(int)) != cudaSuccess) rc = FARGO_ERR_CUDA;
    if (!rc) {
        k_wait_probe<<<1, 64>>>(spin_limit, d);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = FARGO_ERR_CUDA;
    }
    cudaFree(d);
    return rc ? rc : err_code(h);
}

// ---------------------------------------------------------------------------
// Arithmetic peaks of the device, for the rooflines of the ALU-bound kernels
// (the FP64 step): every thread runs 8 independent multiply-add chains, so
// the units stay busy whatever their latency; the grid is 8 blocks of 256
// threads per SM.  FP32 is measured in the scalar form the step's kernels
// use and in the packed two-lane form of this architecture.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *sink, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int c = 0; c < 8; c++) x[c] = fma(x[c], a, b);
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += x[c];
    if (s == (T)-12345) sink[threadIdx.x] = s;   // keeps the chains alive; never true for |a| < 1
}
__global__ void __launch_bounds__(256) k_fma2_chains(float *sink, int iters, float a, float b)
{
    float2 x[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x + c + 1));
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int c = 0; c < 8; c++) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) s += x[c].x + x[c].y;
    if (s == -12345.f) sink[threadIdx.x] = s;
}

template <typename K, typename... A>
static int time_chains(K kernel, int blocks, double flops, cudaStream_t st, double *tflops, A... args)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    kernel<<<blocks, 256, 0, st>>>(args...);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; r++) {
        CK(cudaEventRecord(e0, st));
        kernel<<<blocks, 256, 0, st>>>(args...);
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    *tflops = flops / (best * 1e-3) / 1e12;
    return FARGO_OK;
}

extern "C" int fargo_alu_peaks(double out[3], void *stream)
{
    if (!out) return FARGO_ERR_BADARG;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    void *sink = nullptr;
    CK(cudaMalloc(&sink, 256 * sizeof(double)));
    const int blocks = 8 * sms;
    const double threads = (double)blocks * 256;
    const int it64 = 1 << 12, it32 = 1 << 15;
    int rc = time_chains(k_fma_chains<double>, blocks, 2.0 * 8 * it64 * threads, st, &out[0], (double *)sink, it64,
                         0.999999, 1e-7);
    if (!rc)
        rc = time_chains(k_fma_chains<float>, blocks, 2.0 * 8 * it32 * threads, st, &out[1], (float *)sink, it32,
                         0.999999f, 1e-7f);
    if (!rc)
        rc = time_chains(k_fma2_chains, blocks, 4.0 * 8 * it32 * threads, st, &out[2], (float *)sink, it32,
                         0.999999f, 1e-7f);
    cudaFree(sink);
    return rc;
}

extern "C" int fargo_use_graph(fargo_ctx *c, int enable)
{
    if (!c) return FARGO_ERR_BADARG;
    c->use_graph = enable != 0;
    return FARGO_OK;
}

extern "C" int fargo_launches_per_step(fargo_ctx *c)
{
    if (!c) return FARGO_ERR_BADARG;
    int n = 0;
    const MeshD &m = c->m;
    n += m.hasY + m.hasZ;        // cell 2
    n += 2;                      // Courant (screen + exact)
    n += 2 + (m.has_nu ? 2 : 0); // sources (viscosity: stresses + update)
    n += m.hasY + m.hasZ;        // cell 9
    n += 1 + m.hasY + m.hasZ;    // sweeps
    n += (m.fargo && m.hasX) ? 1 : 0;  // orbital step
    n += 1;                      // new velocities
    return n;
}
