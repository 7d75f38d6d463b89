// Batched engine: many independent hydro instances (uneven meshes and
// parameters) advanced together.  Each phase of the step is ONE launch
// whose blocks cover every member's work for that phase; a block finds its
// member by a binary search over the launch's block offsets and runs the
// same device body as the single-instance kernel on that member's mesh,
// tables and buffers.  Every member keeps its own Courant step and time
// (its own two-stage reduction and device scalars), so members that reached
// their end time or failed drop out on the device without host involvement.
// The sequence of launches is captured once as a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "context.cuh"

using namespace fk;

namespace fk {

// The members that share one launch of a phase kernel.
struct Group {
    const int *ids;   // member index of each entry
    const int *off;   // first block of each entry; off[n] = blocks of the launch
    int n;
};

// Member of block b and the block's index within that member's work.
__device__ __forceinline__ int group_member(const Group &g, int b, int &local)
{
    int lo = 0, hi = g.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&g.off[mid]) <= b) lo = mid;
        else hi = mid - 1;
    }
    local = b - __ldg(&g.off[lo]);
    return __ldg(&g.ids[lo]);
}

// A member's plan copied into shared memory by the whole block: the per-cell
// kernels read its mesh constants and table pointers many times per cell, and
// from shared memory these are short-latency loads instead of dependent
// global ones (the single-instance kernels find them in the constant bank).
// The ring kernels and the exact Courant pass keep reading the plan from
// global memory: a copy per ring costs them more than it saves.
template <typename T>
struct PlanSmem {
    long long w[(sizeof(StepPlan<T>) + 7) / 8];
};
template <typename T>
__device__ __forceinline__ const StepPlan<T> &plan_to_smem(const StepPlan<T> *P, int id, PlanSmem<T> &s)
{
    const long long *src = reinterpret_cast<const long long *>(&P[id]);
    for (int t = threadIdx.x; t < (int)(sizeof(s.w) / 8); t += blockDim.x) s.w[t] = src[t];
    __syncthreads();
    return *reinterpret_cast<const StepPlan<T> *>(s.w);
}

enum { PH_SUB1, PH_AV, PH_TAU, PH_VAPPLY, PH_NEWVEL };

template <typename T>
__global__ void __launch_bounds__(256) kb_bc(const StepPlan<T> *__restrict__ P, Group g, int axis, int mode)
{
    int local;
    __shared__ PlanSmem<T> sp;
    const StepPlan<T> &p = plan_to_smem(P, group_member(g, blockIdx.x, local), sp);
    const long long tid = (long long)local * blockDim.x + threadIdx.x;
    if (axis == 1) bc_y_body(p.m, mode == 0 ? p.A : p.vsrc, p.sc, mode, tid, p.tb.vref);
    else bc_z_body(p.m, mode == 0 ? p.A : p.vsrc, p.sc, mode, tid, p.tb.vref);
}

// (64 registers: no spills; see k_cfl_screen)
template <typename T>
__global__ void __launch_bounds__(256, 4) kb_cfl_screen(const StepPlan<T> *__restrict__ P, Group g)
{
    int local;
    __shared__ PlanSmem<T> sp;
    const StepPlan<T> &p = plan_to_smem(P, group_member(g, blockIdx.x, local), sp);
    cfl_screen_body(p.m, p.tb, p.A, p.v0, p.ringmax, p.part, p.sc, p.nrings_active, local, p.cfl_blocks);
}

template <typename T>
__global__ void __launch_bounds__(256) kb_cfl_exact(const StepPlan<T> *__restrict__ P, Group g)
{
    int local;
    const StepPlan<T> &p = P[group_member(g, blockIdx.x, local)];
    cfl_exact_body(p.m, p.tb, p.A, p.v0, p.ringmax, p.part, p.sc, p.nrings_active, local,
                   cfl_exact_grid(p.cfl_blocks));
}

// Per-cell phases: a member's cells of the augmented mesh (rows, planes as
// in the single-instance grid) are numbered row by row; a block takes
// cpt * blockDim.x consecutive cells, each thread every blockDim.x-th of
// them, so the member lookup is paid once per block for several cells and
// no block is padded to a row's end.  cpt (cells per thread, 16 by default)
// is a launch shape the batch autotuner may change: every cell runs the same
// body whatever the grouping.
constexpr int kCellsPerThread = 16;

// Register budgets (measured): 32 per thread for sub-step 1 (eight 256-thread
// blocks per SM), 48 for the viscous update (five blocks), 40 for the other
// phases (six blocks).
template <typename T, int PH, class F>
__global__ void __launch_bounds__(256, PH == PH_VAPPLY ? 5 : (PH == PH_SUB1 ? 8 : 6)) kb_cell(const StepPlan<T> *__restrict__ P, Group g,
                                                                                                int cpt)
{
    int local;
    __shared__ PlanSmem<T> sp;
    const StepPlan<T> &p = plan_to_smem(P, group_member(g, blockIdx.x, local), sp);
    const MeshD &m = p.m;
    const unsigned nyr = PH == PH_TAU ? tau_rows(m) : m.nyt + 1;
    const unsigned rows = nyr * (PH == PH_TAU ? tau_planes(m) : cell_planes(m));
    const unsigned nx = (unsigned)m.nx;
    const unsigned lin = (unsigned)local * (cpt * blockDim.x) + threadIdx.x;
    unsigned row = lin / nx;
    unsigned i = lin - row * nx;
    for (int u = 0; u < cpt && row < rows; u++) {
        // one plane without a Z direction: the row is the Y index
        int j = F::hasZ(m) ? (int)(row % nyr) : (int)row, k = F::hasZ(m) ? (int)(row / nyr) : 0;
        if constexpr (PH == PH_TAU) {
            j += m.j0;
            k += m.k0;
        }
        if constexpr (PH == PH_SUB1) substep1_body<T, F>(m, p.tb, p.A, p.VB, p.sc, (int)i, j, k);
        else if constexpr (PH == PH_AV) artvisc_body<T, F>(m, p.tb, p.VB, p.A, p.sc, (int)i, j, k);
        else if constexpr (PH == PH_TAU) visc_tau_body<T, F>(m, p.tb, p.A, p.tau, p.sc, (int)i, j, k);
        else if constexpr (PH == PH_VAPPLY) visc_apply_body<T, F>(m, p.tb, p.A, p.VB, p.tau, p.sc, (int)i, j, k);
        else newvel_body<T, F>(m, p.tb, p.qfin, p.vsrc, p.A, p.sc, 0, (int)i, j, k);
        i += blockDim.x;
        while (i >= nx) {
            i -= nx;
            row++;
        }
    }
}

// Ring operations over the items (member, ring) of a group: the member and
// local ring of every iteration are found in parallel before the loop.  A
// member that takes a void step gets a plain arrive instead of copies.
template <typename T, int C>
struct BTxOp {
    const StepPlan<T> *P;
    Group g;
    RingMeta<T> *meta;
    __device__ void prepare(int it, int item)
    {
        RingMeta<T> &e = meta[it];
        e.id = group_member(g, item, e.local);
        const StepPlan<T> &p = P[e.id];
        e.N = step_dt<T>(p.sc) > T(0) ? 0 : -1;
        tx_v0(p.m, p.tb, p.v0, e.local, e.a, e.b);
    }
    __device__ void issue(int it, T *dst, uint64_t *bar)
    {
        const RingMeta<T> &e = meta[it];
        if (e.N < 0) {
            mbar_arrive(bar);
            return;
        }
        const StepPlan<T> &p = P[e.id];
        tx_issue(p.m, p.txin, e.local, dst, bar);
    }
    __device__ void compute(int it, T *src)
    {
        const RingMeta<T> &e = meta[it];
        if (e.N < 0) return;
        const StepPlan<T> &p = P[e.id];
        tx_compute<T, C>(p.m, p.tb, p.qx, e.local, src, e.a, e.b, step_dt<T>(p.sc));
    }
    __device__ void fail(int it) { atomicOr(&P[meta[it].id].sc->err, kErrTimeout); }
};

template <typename T, int C>
struct BOrbOp {
    const StepPlan<T> *P;
    Group g;
    RingMeta<T> *meta;
    __device__ void prepare(int it, int item)
    {
        RingMeta<T> &e = meta[it];
        e.id = group_member(g, item, e.local);
        const StepPlan<T> &p = P[e.id];
        const T dt = step_dt<T>(p.sc);
        if (!(dt > T(0))) {
            e.N = -1;
            return;
        }
        orb_prepare(p.m, p.tb, p.v0, p.sc, e.local, e.N, e.a, e.b);
        orb_ring_consts(p.m, p.tb, dt, e.local, e);
    }
    __device__ void issue(int it, T *dst, uint64_t *bar)
    {
        const RingMeta<T> &e = meta[it];
        const StepPlan<T> &p = P[e.id];
        orb_issue(p.m, p.qfin, e.local, e.N, dst, bar);
    }
    __device__ void compute(int it, T *src)
    {
        const RingMeta<T> &e = meta[it];
        if (e.N < 0) return;
        const StepPlan<T> &p = P[e.id];
        if constexpr (orb_uses_lanes<C>())
            orb_compute_w<T, C>(p.qfin, p.m.nx, ring_row(p.m.sj), e, src);
        else
            orb_compute<T, C>(p.m, p.tb, p.qfin, e.local, src, e.N, e.a, e.b, step_dt<T>(p.sc));
    }
    __device__ void fail(int it) { atomicOr(&P[meta[it].id].sc->err, kErrTimeout); }
};

template <typename T, int C>
__global__ void __launch_bounds__(512, 2) kb_tx(const StepPlan<T> *__restrict__ P, Group g, int stride, int nitems,
                                                 int nbuf)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    ring_bars_init(bar);
    BTxOp<T, C> op{P, g, ring_meta<T>(smem_raw, stride, nbuf)};
    ring_pipeline<T>(op, reinterpret_cast<T *>(smem_raw), (size_t)stride, bar, blockIdx.x, gridDim.x, nitems,
                     nbuf);
}

template <typename T, int C>
__global__ void __launch_bounds__(orb_max_threads(C), orb_min_blocks(C)) kb_orb(const StepPlan<T> *__restrict__ P, Group g, int stride, int nitems,
                                                 int nbuf)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    ring_bars_init(bar);
    BOrbOp<T, C> op{P, g, ring_meta<T>(smem_raw, stride, nbuf)};
    ring_pipeline<T>(op, reinterpret_cast<T *>(smem_raw), (size_t)stride, bar, blockIdx.x, gridDim.x, nitems,
                     nbuf);
}

// Tensor maps of every member live in global memory (64-byte aligned).
template <typename T, int AXIS, int NQ>
__global__ void __launch_bounds__(TmaTile<T>::TW + 32) kb_sweep(const StepPlan<T> *__restrict__ P,
                                                                 const SweepMaps *__restrict__ maps, Group g)
{
    int local;
    const int id = group_member(g, blockIdx.x, local);
    __shared__ PlanSmem<T> sp;
    const StepPlan<T> &p = plan_to_smem(P, id, sp);
    sweep_body<T, AXIS, NQ>(p.m, p.tb, maps[id], AXIS == 1 ? p.qy : p.qz, p.sc, AXIS == 1 ? p.seg_y : p.seg_z,
                            local);
}

// Packed field transfers: the active cells of one field of every member,
// concatenated in member order (X fastest within a member), between the
// members' padded field arrays and one contiguous staging buffer.  A block
// covers 1024 consecutive cells of one member (found by the group search).
constexpr int kPackCells = 1024;
template <typename T>
__global__ void __launch_bounds__(256) kb_pack(const StepPlan<T> *__restrict__ P, Group g,
                                               const long long *__restrict__ pk, int field, T *stage, int to_fields)
{
    int local;
    const int id = group_member(g, blockIdx.x, local);
    const StepPlan<T> &p = P[id];
    const MeshD &m = p.m;
    T *const fl[5] = {p.A.rho, p.A.e, p.A.vx, p.A.vy, p.A.vz};
    T *f = fl[field];
    const int nx = m.nx, ny = m.j1 - m.j0, nz = m.k1 - m.k0;
    const long long nact = (long long)nx * ny * nz;
    T *s = stage + __ldg(&pk[id]);
    // v_x leaves in v_x form (FP32: stored v_x - vref); it arrives in v_x form
    // and kb_vref rebases it afterwards
    const T *ref = field == 2 && sizeof(T) == 4 ? p.tb.vref : nullptr;
    for (int u = 0; u < kPackCells / 256; u++) {
        const long long t = (long long)local * kPackCells + u * 256 + threadIdx.x;
        if (t >= nact) return;
        const int i = (int)(t % nx);
        const long long r = t / nx;
        const int j = m.j0 + (int)(r % ny), k = m.k0 + (int)(r / ny);
        const idx_t c = IX(m, i, j, k);
        if (to_fields) f[c] = s[t];
        else s[t] = ref ? f[c] + ref[k * m.nyt + j] : f[c];
    }
}

// The reference form of v_x for every member (FP32): mode VREF_ABS, _CHOOSE
// or _APPLY of vref_ring over all rings of all members, eight rings a block.
template <typename T>
__global__ void __launch_bounds__(256) kb_vref(const StepPlan<T> *__restrict__ P, Group g, int mode)
{
    int local;
    const int id = group_member(g, blockIdx.x, local);
    const StepPlan<T> &p = P[id];
    const int ring = local * 8 + (threadIdx.x >> 5);
    if (ring < p.m.nyt * p.m.nzt) vref_ring(p.m, p.tb, p.A.vx, p.A.vx, ring, mode);
}

// out[0] = members still running, out[1] = OR of their error flags,
// out[2] = lowest index of a failed member (n if none).
__global__ void __launch_bounds__(256) kb_status(Scal *const *sc, int n, int *out)
{
    __shared__ int s_run, s_err, s_first;
    if (threadIdx.x == 0) {
        s_run = 0;
        s_err = 0;
        s_first = n;
    }
    __syncthreads();
    int run = 0, err = 0, first = n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Scal *s = sc[i];
        const int e = s->err;
        err |= e;
        if (e && i < first) first = i;
        if (!e && (s->fixed || s->t < s->t_end)) run++;
    }
    atomicAdd(&s_run, run);
    atomicOr(&s_err, err);
    atomicMin(&s_first, first);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = s_run;
        out[1] = s_err;
        out[2] = s_first;
    }
}

}  // namespace fk

namespace {

enum LaunchKind { L_BC, L_SCREEN, L_EXACT, L_CELL, L_TX, L_SWEEP, L_ORB };

// One launch of the batched step: a phase over a group of members.
struct BLaunch {
    LaunchKind kind;
    int arg = 0;       // BC: axis; CELL: phase; SWEEP: axis
    int mode = 0;      // BC: 0 = cell 2, 1 = cell 9
    int key = 0;       // ring kernels: cells per thread; sweeps: quantities
    std::vector<int> ids, off;
    int *d = nullptr;  // device copy: ids, then off
    int threads = 256;
    size_t smem = 0;
    RingShape rs{};    // ring kernels: threads, values per ring buffer, shared memory, persistent grid
    const char *name = "";
    Group dev() const { return Group{d, d + ids.size(), (int)ids.size()}; }
    int blocks() const { return off.empty() ? 0 : off.back(); }
};

}  // namespace

struct fargo_batch {
    int n = 0, prec = FARGO_F32;
    std::vector<fargo_ctx *> mem;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *plans = nullptr;                    // StepPlan<T>[n]
    SweepMaps *mapsY = nullptr, *mapsZ = nullptr;
    Scal **scs = nullptr;
    int *status = nullptr;                    // device: run, err, first failed
    int *hstatus = nullptr;                   // pinned host copy
    std::vector<void *> allocs;
    std::vector<BLaunch> seq;                 // the launches of one step, in order
    // packed field transfers: staging buffer (all members' active cells of
    // one field), per-member packed offsets and the group of the pack launch
    void *stage = nullptr;
    long long *pk = nullptr;
    int *pack_grp = nullptr;
    int pack_blocks = 0;
    int *vref_grp = nullptr;     // kb_vref's launch: member ids and block offsets (eight rings a block)
    int vref_blocks = 0;
    size_t packed_bytes = 0;
    int cpt = kCellsPerThread;                // cells per thread of the per-cell phases
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    long long steps = 0;
};

static int balloc(fargo_batch *b, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? FARGO_ERR_OOM : FARGO_ERR_CUDA;
    }
    b->allocs.push_back(*p);
    return FARGO_OK;
}

// Group the eligible members of a phase by `key` (one launch per key value)
// with `blocks(member)` blocks each.
template <typename Elig, typename Key, typename Blocks>
static void add_phase(fargo_batch *b, BLaunch proto, Elig elig, Key key, Blocks blocks)
{
    std::map<int, BLaunch> by;
    for (int i = 0; i < b->n; i++) {
        if (!elig(b->mem[i])) continue;
        const int k = key(b->mem[i]);
        auto it = by.find(k);
        if (it == by.end()) {
            BLaunch L = proto;
            L.key = k;
            L.off.push_back(0);
            it = by.emplace(k, L).first;
        }
        BLaunch &L = it->second;
        L.ids.push_back(i);
        L.off.push_back(L.off.back() + blocks(b->mem[i]));
    }
    for (auto &kv : by) b->seq.push_back(kv.second);
}

template <typename T>
static const Buffers<T> &bufs(const fargo_ctx *c);
template <>
const Buffers<double> &bufs<double>(const fargo_ctx *c) { return c->b64; }
template <>
const Buffers<float> &bufs<float>(const fargo_ctx *c) { return c->b32; }

template <typename T, int C>
static cudaError_t ring_attrs(BLaunch &x)
{
    cudaError_t e;
    if (x.kind == L_TX) e = ring_grid<T>(kb_tx<T, C>, x.rs, x.blocks());
    else e = ring_grid<T>(kb_orb<T, C>, x.rs, x.blocks());
    x.smem = x.rs.smem;
    return e;
}

template <typename T, int AXIS>
static cudaError_t sweep_attrs(int nq)
{
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int sm = (int)sweep_tma_smem<T, AXIS>(nq);
    switch (nq) {
    case 3: return cudaFuncSetAttribute(kb_sweep<T, AXIS, 3>, a, sm);
    case 4: return cudaFuncSetAttribute(kb_sweep<T, AXIS, 4>, a, sm);
    case 5: return cudaFuncSetAttribute(kb_sweep<T, AXIS, 5>, a, sm);
    case 6: return cudaFuncSetAttribute(kb_sweep<T, AXIS, 6>, a, sm);
    case 7: return cudaFuncSetAttribute(kb_sweep<T, AXIS, 7>, a, sm);
    default: return cudaFuncSetAttribute(kb_sweep<T, AXIS, 8>, a, sm);
    }
}

// Build the launch sequence (the same phase order as the single-instance
// step) and upload the plans, tensor maps and groups.
template <typename T>
static int batch_setup(fargo_batch *b)
{
    const int n = b->n;
    std::vector<StepPlan<T>> plans(n);
    std::vector<SweepMaps> my(n), mz(n);
    std::vector<Scal *> scs(n);
    for (int i = 0; i < n; i++) {
        plans[i] = make_plan<T>(b->mem[i], bufs<T>(b->mem[i]));
        my[i] = b->mem[i]->mapsY;
        mz[i] = b->mem[i]->mapsZ;
        scs[i] = b->mem[i]->sc;
    }
    auto all = [](const fargo_ctx *) { return true; };
    auto one = [](const fargo_ctx *) { return 0; };
    const int cpt = b->cpt;
    auto cells = [cpt](const fargo_ctx *c) {
        return (int)grid_for((long long)c->nx * (c->nyt + 1) * cell_planes(c->m), 256 * cpt);
    };
    auto tau_cells = [cpt](const fargo_ctx *c) {
        return (int)grid_for((long long)c->nx * tau_rows(c->m) * tau_planes(c->m), 256 * cpt);
    };
    auto hasY = [](const fargo_ctx *c) { return c->m.hasY != 0; };
    auto hasZ = [](const fargo_ctx *c) { return c->m.hasZ != 0; };
    auto hasNu = [](const fargo_ctx *c) { return c->m.has_nu != 0; };
    auto bcy = [](const fargo_ctx *c) { return (int)grid_for((long long)c->nx * (c->nzt + 1) * 2, 256); };
    auto bcz = [](const fargo_ctx *c) { return (int)grid_for((long long)c->nx * (c->nyt + 1) * 2, 256); };
    auto tx_chunk = [](const fargo_ctx *c) { return c->tx_rs.chunk; };
    auto orb_chunk = [](const fargo_ctx *c) { return c->orb_rs.chunk; };
    auto nqk = [](const fargo_ctx *c) { return 3 + (c->m.iso ? 0 : 1) + (c->m.hasY ? 2 : 0) + (c->m.hasZ ? 2 : 0); };
    auto sweep_blocks = [](int axis) {
        return [axis](const fargo_ctx *c) {
            const MeshD &m = c->m;
            const int np = axis == 1 ? m.j1 - m.j0 : m.k1 - m.k0;
            const int n2 = axis == 1 ? m.k1 - m.k0 : m.j1 - m.j0;
            const int set = axis == 1 ? c->seg_y : c->seg_z;   // as make_plan
            const int sl = set > 0 ? set : sweep_seglen(np);
            const int ntx = (m.nx + TmaTile<T>::TW - 1) / TmaTile<T>::TW;
            return ntx * n2 * ((np + sl - 1) / sl);
        };
    };
    BLaunch L;
    b->seq.clear();
    L = BLaunch{L_BC}; L.arg = 1; L.mode = 0; L.name = "bc_y";
    add_phase(b, L, hasY, one, bcy);
    L = BLaunch{L_BC}; L.arg = 2; L.mode = 0; L.name = "bc_z";
    add_phase(b, L, hasZ, one, bcz);
    L = BLaunch{L_SCREEN}; L.name = "cfl_screen";
    add_phase(b, L, all, one, [](const fargo_ctx *c) { return c->cfl_blocks; });
    L = BLaunch{L_EXACT}; L.name = "cfl_exact";
    add_phase(b, L, all, one, [](const fargo_ctx *c) { return cfl_exact_grid(c->cfl_blocks); });
    // the per-cell phases launch once per configuration class (cfg_of)
    auto cfg = [](const fargo_ctx *c) { return cfg_of(c->m); };
    L = BLaunch{L_CELL}; L.arg = PH_SUB1; L.name = "substep1";
    add_phase(b, L, all, cfg, cells);
    L = BLaunch{L_CELL}; L.arg = PH_AV; L.name = "artvisc";
    add_phase(b, L, all, cfg, cells);
    L = BLaunch{L_CELL}; L.arg = PH_TAU; L.name = "visc_tau";
    add_phase(b, L, hasNu, cfg, tau_cells);
    L = BLaunch{L_CELL}; L.arg = PH_VAPPLY; L.name = "visc_apply";
    add_phase(b, L, hasNu, cfg, cells);
    L = BLaunch{L_BC}; L.arg = 1; L.mode = 1; L.name = "bc_y9";
    add_phase(b, L, hasY, one, bcy);
    L = BLaunch{L_BC}; L.arg = 2; L.mode = 1; L.name = "bc_z9";
    add_phase(b, L, hasZ, one, bcz);
    L = BLaunch{L_TX}; L.name = "transport_x";
    add_phase(b, L, all, tx_chunk, [](const fargo_ctx *c) { return c->nyt * c->nzt; });
    L = BLaunch{L_SWEEP}; L.arg = 1; L.name = "transport_y";
    add_phase(b, L, hasY, nqk, sweep_blocks(1));
    L = BLaunch{L_SWEEP}; L.arg = 2; L.name = "transport_z";
    add_phase(b, L, hasZ, nqk, sweep_blocks(2));
    L = BLaunch{L_ORB}; L.name = "orbital";
    add_phase(b, L, [](const fargo_ctx *c) { return c->m.fargo && c->m.hasX; }, orb_chunk,
              [](const fargo_ctx *c) { return c->nrings_active; });
    L = BLaunch{L_CELL}; L.arg = PH_NEWVEL; L.name = "newvel";
    add_phase(b, L, all, cfg, cells);

    // launch shapes of the ring and sweep groups
    int rc;
    for (BLaunch &x : b->seq) {
        if (x.kind == L_TX || x.kind == L_ORB) {
            int threads = 0, stride = 0;
            for (int id : x.ids) {
                const RingShape &rs = x.kind == L_TX ? b->mem[id]->tx_rs : b->mem[id]->orb_rs;
                threads = std::max(threads, rs.threads);
                stride = std::max(stride, rs.stride);
            }
            x.rs.threads = x.threads = threads;
            x.rs.stride = stride;
            x.rs.chunk = x.key;
            x.rs.nbuf = ring_nbuf(stride, (int)sizeof(T), x.kind == L_ORB);
            x.rs.smem = x.smem = (size_t)x.rs.nbuf * stride * sizeof(T);
        } else if (x.kind == L_SWEEP) {
            x.threads = TmaTile<T>::TW + 32;
            x.smem = x.arg == 1 ? sweep_tma_smem<T, 1>(x.key) : sweep_tma_smem<T, 2>(x.key);
        }
        const size_t nb = (x.ids.size() + x.off.size()) * sizeof(int);
        if ((rc = balloc(b, (void **)&x.d, nb))) return rc;
        CK(cudaMemcpyAsync(x.d, x.ids.data(), x.ids.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(x.d + x.ids.size(), x.off.data(), x.off.size() * sizeof(int), cudaMemcpyHostToDevice,
                           b->stream));
    }
    // ring kernels: one dynamic shared-memory limit per variant (the largest member)
    for (BLaunch &x : b->seq) {
        if (x.kind != L_TX && x.kind != L_ORB) continue;
        switch (x.key) {
        case 1: CK((ring_attrs<T, 1>(x))); break;
        case 2: CK((ring_attrs<T, 2>(x))); break;
        case 3: CK((ring_attrs<T, 3>(x))); break;
        case 4: CK((ring_attrs<T, 4>(x))); break;
        case 6: CK((ring_attrs<T, 6>(x))); break;
        default: CK((ring_attrs<T, 8>(x))); break;
        }
    }
    for (const BLaunch &x : b->seq)
        if (x.kind == L_SWEEP) CK(x.arg == 1 ? (sweep_attrs<T, 1>(x.key)) : (sweep_attrs<T, 2>(x.key)));

    if ((rc = balloc(b, &b->plans, sizeof(StepPlan<T>) * n))) return rc;
    if ((rc = balloc(b, (void **)&b->mapsY, sizeof(SweepMaps) * n))) return rc;
    if ((rc = balloc(b, (void **)&b->mapsZ, sizeof(SweepMaps) * n))) return rc;
    if ((rc = balloc(b, (void **)&b->scs, sizeof(Scal *) * n))) return rc;
    if ((rc = balloc(b, (void **)&b->status, sizeof(int) * 4))) return rc;
    CK(cudaMemcpyAsync(b->plans, plans.data(), sizeof(StepPlan<T>) * n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->mapsY, my.data(), sizeof(SweepMaps) * n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->mapsZ, mz.data(), sizeof(SweepMaps) * n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->scs, scs.data(), sizeof(Scal *) * n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return FARGO_OK;
}

template <typename T, class F>
static void launch_cell_cfg(int ph, int nb, const StepPlan<T> *P, Group g, int cpt, cudaStream_t s)
{
    switch (ph) {
    case PH_SUB1: kb_cell<T, PH_SUB1, F><<<nb, 256, 0, s>>>(P, g, cpt); break;
    case PH_AV: kb_cell<T, PH_AV, F><<<nb, 256, 0, s>>>(P, g, cpt); break;
    case PH_TAU: kb_cell<T, PH_TAU, F><<<nb, 256, 0, s>>>(P, g, cpt); break;
    case PH_VAPPLY: kb_cell<T, PH_VAPPLY, F><<<nb, 256, 0, s>>>(P, g, cpt); break;
    default: kb_cell<T, PH_NEWVEL, F><<<nb, 256, 0, s>>>(P, g, cpt); break;
    }
}

template <typename T>
static void launch_ring(const BLaunch &x, const StepPlan<T> *P, cudaStream_t s)
{
    const Group g = x.dev();
    const int n = x.blocks();
    const RingShape &r = x.rs;
    if (x.kind == L_TX) {
        switch (x.key) {
        case 1: kb_tx<T, 1><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 2: kb_tx<T, 2><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 3: kb_tx<T, 3><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 4: kb_tx<T, 4><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 6: kb_tx<T, 6><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        default: kb_tx<T, 8><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        }
    } else {
        switch (x.key) {
        case 1: kb_orb<T, 1><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 2: kb_orb<T, 2><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 3: kb_orb<T, 3><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 4: kb_orb<T, 4><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        case 6: kb_orb<T, 6><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        default: kb_orb<T, 8><<<r.grid, r.threads, r.smem, s>>>(P, g, r.stride, n, r.nbuf); break;
        }
    }
}

template <typename T, int AXIS>
static void launch_bsweep(const BLaunch &x, const StepPlan<T> *P, const SweepMaps *maps, cudaStream_t s)
{
    const Group g = x.dev();
    const unsigned nb = (unsigned)x.blocks();
    switch (x.key) {
    case 3: kb_sweep<T, AXIS, 3><<<nb, x.threads, x.smem, s>>>(P, maps, g); break;
    case 4: kb_sweep<T, AXIS, 4><<<nb, x.threads, x.smem, s>>>(P, maps, g); break;
    case 5: kb_sweep<T, AXIS, 5><<<nb, x.threads, x.smem, s>>>(P, maps, g); break;
    case 6: kb_sweep<T, AXIS, 6><<<nb, x.threads, x.smem, s>>>(P, maps, g); break;
    case 7: kb_sweep<T, AXIS, 7><<<nb, x.threads, x.smem, s>>>(P, maps, g); break;
    default: kb_sweep<T, AXIS, 8><<<nb, x.threads, x.smem, s>>>(P, maps, g); break;
    }
}

template <typename T>
static int batch_enqueue(fargo_batch *b, cudaEvent_t *marks = nullptr)
{
    const StepPlan<T> *P = (const StepPlan<T> *)b->plans;
    cudaStream_t s = b->stream;
    int nl = 0;
    for (const BLaunch &x : b->seq) {
        const unsigned nb = (unsigned)x.blocks();
        if (nb == 0) continue;
        const Group g = x.dev();
        switch (x.kind) {
        case L_BC: kb_bc<T><<<nb, 256, 0, s>>>(P, g, x.arg, x.mode); break;
        case L_SCREEN: kb_cfl_screen<T><<<nb, 256, 0, s>>>(P, g); break;
        case L_EXACT: kb_cfl_exact<T><<<nb, 256, 0, s>>>(P, g); break;
        case L_CELL:
            if (x.key == CFG_DISK3D) launch_cell_cfg<T, CfgDisk3D>(x.arg, nb, P, g, b->cpt, s);
            else if (x.key == CFG_DISK2D) launch_cell_cfg<T, CfgDisk2D>(x.arg, nb, P, g, b->cpt, s);
            else if (x.key == CFG_DISK3D_LIVE) launch_cell_cfg<T, CfgDisk3DLive>(x.arg, nb, P, g, b->cpt, s);
            else if (x.key == CFG_DISK2D_LIVE) launch_cell_cfg<T, CfgDisk2DLive>(x.arg, nb, P, g, b->cpt, s);
            else launch_cell_cfg<T, CfgRun>(x.arg, nb, P, g, b->cpt, s);
            break;
        case L_TX:
        case L_ORB: launch_ring<T>(x, P, s); break;
        case L_SWEEP:
            if (x.arg == 1) launch_bsweep<T, 1>(x, P, b->mapsY, s);
            else launch_bsweep<T, 2>(x, P, b->mapsZ, s);
            break;
        }
        if (marks) cudaEventRecord(marks[nl + 1], s);
        nl++;
    }
    CK(cudaGetLastError());
    return FARGO_OK;
}

static int benqueue(fargo_batch *b)
{
    return b->prec == FARGO_F64 ? batch_enqueue<double>(b) : batch_enqueue<float>(b);
}

static int batch_launch(fargo_batch *b)
{
    if (!b->use_graph) return benqueue(b);
    if (!b->gexec) {
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = benqueue(b);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc) return rc;
        if (e != cudaSuccess) return FARGO_ERR_CUDA;
        b->graph = g;
        CK(cudaGraphInstantiate(&b->gexec, g, 0));
    }
    CK(cudaGraphLaunch(b->gexec, b->stream));
    return FARGO_OK;
}

extern "C" int fargo_batch_create(fargo_batch **out, fargo_ctx *const *members, int n, void *stream)
{
    if (!out || !members || n < 1) return FARGO_ERR_BADARG;
    *out = nullptr;
    const int prec = members[0] ? members[0]->prec : -1;
    for (int i = 0; i < n; i++) {
        if (!members[i] || members[i]->prec != prec) return FARGO_ERR_BADARG;
        // the batched phases have no periodic-image launches between them
        if (members[i]->m.pery || members[i]->m.perz) return FARGO_ERR_BADARG;
        if (members[i]->m.mhd) return FARGO_ERR_BADARG;   // no magnetic field in the batched engine
        for (int k = 0; k < i; k++)
            if (members[k] == members[i]) return FARGO_ERR_BADARG;
    }
    fargo_batch *b = new fargo_batch();
    b->n = n;
    b->prec = prec;
    b->mem.assign(members, members + n);
    for (fargo_ctx *m : b->mem) m->batch_refs++;   // released by fargo_batch_destroy
    int rc = FARGO_OK;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        b->stream = nullptr;
        fargo_batch_destroy(b);
        return FARGO_ERR_CUDA;
    } else {
        b->own_stream = true;
    }
    // the members' own streams may still hold work (uploads of their state)
    for (int i = 0; i < n; i++)
        if (cudaStreamSynchronize(members[i]->stream) != cudaSuccess) rc = FARGO_ERR_CUDA;
    if (!rc && cudaMallocHost((void **)&b->hstatus, sizeof(int) * 4) != cudaSuccess) rc = FARGO_ERR_OOM;
    if (!rc) rc = prec == FARGO_F64 ? batch_setup<double>(b) : batch_setup<float>(b);
    if (rc) {
        fargo_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FARGO_OK;
}

extern "C" void fargo_batch_destroy(fargo_batch *b)
{
    if (!b) return;
    for (fargo_ctx *m : b->mem) m->batch_refs--;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *p : b->allocs) cudaFree(p);
    if (b->stage) cudaFree(b->stage);
    if (b->pk) cudaFree(b->pk);
    if (b->pack_grp) cudaFree(b->pack_grp);
    if (b->vref_grp) cudaFree(b->vref_grp);
    if (b->hstatus) cudaFreeHost(b->hstatus);
    // a stream handed in by the caller stays theirs; the member contexts too
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

int fargo_queue_field(fargo_ctx *c, int field, int region, void *buf, size_t bytes, int to_dev, cudaStream_t s);

extern "C" int fargo_batch_set_field(fargo_batch *b, int field, int region, const void *const *src,
                                     const size_t *bytes)
{
    if (!b || !src || !bytes) return FARGO_ERR_BADARG;
    for (int i = 0; i < b->n; i++) {
        const int rc = fargo_queue_field(b->mem[i], field, region, (void *)src[i], bytes[i], 1, b->stream);
        if (rc) return rc;
    }
    return FARGO_OK;
}

extern "C" int fargo_batch_get_field(fargo_batch *b, int field, int region, void *const *dst, const size_t *bytes)
{
    if (!b || !dst || !bytes) return FARGO_ERR_BADARG;
    for (int i = 0; i < b->n; i++) {
        const int rc = fargo_queue_field(b->mem[i], field, region, dst[i], bytes[i], 0, b->stream);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(b->stream));
    return FARGO_OK;
}

// The staging buffer and the pack launch's tables, made at the first packed
// transfer and kept until the batch is destroyed.
static int pack_setup(fargo_batch *b)
{
    if (b->stage) return FARGO_OK;
    std::vector<long long> pk(b->n);
    std::vector<int> ids(b->n), off(b->n + 1, 0), voff(b->n + 1, 0);
    long long tot = 0;
    for (int i = 0; i < b->n; i++) {
        const fargo_ctx *c = b->mem[i];
        const long long nact = (long long)c->nx * c->ny * c->nz;
        pk[i] = tot;
        tot += nact;
        ids[i] = i;
        off[i + 1] = off[i] + (int)((nact + kPackCells - 1) / kPackCells);
        voff[i + 1] = voff[i] + (c->m.nyt * c->m.nzt + 7) / 8;
    }
    CK(cudaMalloc(&b->vref_grp, sizeof(int) * (2 * b->n + 1)));
    CK(cudaMemcpyAsync(b->vref_grp, ids.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->vref_grp + b->n, voff.data(), sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice, b->stream));
    b->vref_blocks = voff[b->n];
    const size_t esz = b->mem[0]->esz;
    b->packed_bytes = (size_t)tot * esz;
    CK(cudaMalloc(&b->stage, b->packed_bytes));
    CK(cudaMalloc(&b->pk, sizeof(long long) * b->n));
    CK(cudaMalloc(&b->pack_grp, sizeof(int) * (2 * b->n + 1)));
    CK(cudaMemcpyAsync(b->pk, pk.data(), sizeof(long long) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->pack_grp, ids.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->pack_grp + b->n, off.data(), sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice, b->stream));
    b->pack_blocks = off[b->n];
    return FARGO_OK;
}

static int pack_launch(fargo_batch *b, int field, int to_fields)
{
    const Group g{b->pack_grp, b->pack_grp + b->n, b->n};
    if (b->prec == FARGO_F64)
        kb_pack<double><<<b->pack_blocks, 256, 0, b->stream>>>((const StepPlan<double> *)b->plans, g, b->pk, field,
                                                               (double *)b->stage, to_fields);
    else
        kb_pack<float><<<b->pack_blocks, 256, 0, b->stream>>>((const StepPlan<float> *)b->plans, g, b->pk, field,
                                                              (float *)b->stage, to_fields);
    CK(cudaGetLastError());
    return FARGO_OK;
}

static bool field_ok(const fargo_batch *b, int field)
{
    if (field < 0 || field > 4) return false;
    for (const fargo_ctx *c : b->mem) {
        if (field == FARGO_ENERGY && c->m.iso) return false;
        if ((field == FARGO_VY && !c->m.hasY) || (field == FARGO_VZ && !c->m.hasZ)) return false;
    }
    return true;
}

static int vref_batch(fargo_batch *b, int mode)
{
    const Group g{b->vref_grp, b->vref_grp + b->n, b->n};
    kb_vref<float><<<b->vref_blocks, 256, 0, b->stream>>>((const StepPlan<float> *)b->plans, g, mode);
    CK(cudaGetLastError());
    return FARGO_OK;
}

extern "C" int fargo_batch_set_field_packed(fargo_batch *b, int field, const void *src, size_t bytes)
{
    if (!b || !src || !field_ok(b, field)) return FARGO_ERR_BADARG;
    int rc = pack_setup(b);
    if (rc) return rc;
    if (bytes != b->packed_bytes) return FARGO_ERR_SIZE;
    // FP32 v_x: the members' ghost rings to v_x form, the active cells
    // written, then every ring rebased on fresh references
    const bool ref = b->prec == FARGO_F32 && field == FARGO_VX;
    if (ref && (rc = vref_batch(b, VREF_ABS))) return rc;
    CK(cudaMemcpyAsync(b->stage, src, bytes, cudaMemcpyDefault, b->stream));
    if ((rc = pack_launch(b, field, 1))) return rc;
    if (ref && ((rc = vref_batch(b, VREF_CHOOSE)) || (rc = vref_batch(b, VREF_APPLY)))) return rc;
    return FARGO_OK;
}

extern "C" int fargo_batch_get_field_packed(fargo_batch *b, int field, void *dst, size_t bytes)
{
    if (!b || !dst || !field_ok(b, field)) return FARGO_ERR_BADARG;
    int rc = pack_setup(b);
    if (rc) return rc;
    if (bytes != b->packed_bytes) return FARGO_ERR_SIZE;
    if ((rc = pack_launch(b, field, 0))) return rc;
    CK(cudaMemcpyAsync(dst, b->stage, bytes, cudaMemcpyDefault, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return FARGO_OK;
}

extern "C" int fargo_batch_step(fargo_batch *b)
{
    if (!b) return FARGO_ERR_BADARG;
    int rc = batch_launch(b);
    if (!rc) b->steps++;
    return rc;
}

extern "C" int fargo_batch_status(fargo_batch *b, int *n_running, int *first_failed)
{
    if (!b) return FARGO_ERR_BADARG;
    kb_status<<<1, 256, 0, b->stream>>>(b->scs, b->n, b->status);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(b->hstatus, b->status, sizeof(int) * 3, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (n_running) *n_running = b->hstatus[0];
    if (first_failed) *first_failed = b->hstatus[2] < b->n ? b->hstatus[2] : -1;
    return err_code(b->hstatus[1]);
}

extern "C" int fargo_batch_run(fargo_batch *b, long long max_steps, int poll, long long *steps_done,
                               int *n_running)
{
    if (!b || poll < 1 || max_steps < 0) return FARGO_ERR_BADARG;
    long long launched = 0;
    int run = 0, first = -1;
    int rc = fargo_batch_status(b, &run, &first);
    while (rc == FARGO_OK && run > 0 && launched < max_steps) {
        const long long k = max_steps - launched < poll ? max_steps - launched : poll;
        for (long long q = 0; q < k; q++) {
            int r2 = fargo_batch_step(b);
            if (r2) return r2;
        }
        launched += k;
        rc = fargo_batch_status(b, &run, &first);
    }
    if (steps_done) *steps_done = launched;
    if (n_running) *n_running = run;
    return rc;
}

extern "C" int fargo_batch_use_graph(fargo_batch *b, int enable)
{
    if (!b) return FARGO_ERR_BADARG;
    b->use_graph = enable != 0;
    return FARGO_OK;
}

extern "C" int fargo_batch_launches_per_step(const fargo_batch *b)
{
    if (!b) return FARGO_ERR_BADARG;
    int n = 0;
    for (const BLaunch &x : b->seq) n += x.blocks() > 0;
    return n;
}

extern "C" int fargo_batch_profile_step(fargo_batch *b, int max_kernels, float *ms, int *n_out, const char **names)
{
    if (!b || !ms || !n_out || max_kernels < 1) return FARGO_ERR_BADARG;
    const int nseq = (int)b->seq.size();
    std::vector<cudaEvent_t> ev(nseq + 1);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(ev[0], b->stream));
    int rc = b->prec == FARGO_F64 ? batch_enqueue<double>(b, ev.data()) : batch_enqueue<float>(b, ev.data());
    if (rc == FARGO_OK) {
        CK(cudaStreamSynchronize(b->stream));
        int n = 0;
        for (const BLaunch &x : b->seq) {
            if (x.blocks() == 0) continue;
            if (n < max_kernels) {
                CK(cudaEventElapsedTime(&ms[n], ev[n], ev[n + 1]));
                if (names) names[n] = x.name;
            }
            n++;
        }
        *n_out = n < max_kernels ? n : max_kernels;
        b->steps++;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

// ---------------------------------------------------------------------------
// Autotuner of the batch's launch shapes that leave every result unchanged:
// the cells per thread of the per-cell phases (each cell runs the same body
// whatever the grouping) and the segment length of the Y/Z sweeps (each
// column marches the same arithmetic whatever the segmentation), the latter
// set for every member.  Coordinate search: each candidate rebuilds the
// launch sequence and is timed over `reps` profiled steps (per-launch CUDA
// events, summed), every trial step starting from a device snapshot of the
// members' states and times, which is restored at the end, so the run is
// unchanged.  The paper's code searches block sizes per kernel in a similar
// way (Sec. 4.2); the batch has no counterpart there.
// ---------------------------------------------------------------------------
namespace {
struct BSnap {
    std::vector<void *> dst;
    std::vector<const void *> src;
    std::vector<size_t> bytes;
    void *mem = nullptr;
};
}  // namespace

static int bsnap_copy(fargo_batch *b, BSnap &sn, bool save)
{
    for (size_t i = 0; i < sn.dst.size(); i++) {
        void *to = save ? sn.dst[i] : const_cast<void *>(sn.src[i]);
        const void *from = save ? sn.src[i] : sn.dst[i];
        CK(cudaMemcpyAsync(to, from, sn.bytes[i], cudaMemcpyDeviceToDevice, b->stream));
    }
    return FARGO_OK;
}

static int bsnap_make(fargo_batch *b, BSnap &sn)
{
    size_t tot = 0;
    std::vector<std::pair<const void *, size_t>> parts;
    for (fargo_ctx *c : b->mem) {
        const size_t nb = (size_t)c->m.ntot * c->esz;
        void *f[5];
        if (c->prec == FARGO_F64) {
            const Fld<double> &A = c->b64.A;
            f[0] = A.rho; f[1] = A.e; f[2] = A.vx; f[3] = A.vy; f[4] = A.vz;
        } else {
            const Fld<float> &A = c->b32.A;
            f[0] = A.rho; f[1] = A.e; f[2] = A.vx; f[3] = A.vy; f[4] = A.vz;
        }
        for (int q = 0; q < 5; q++) {
            if (q == 1 && c->m.iso) continue;
            if ((q == 3 && !c->m.hasY) || (q == 4 && !c->m.hasZ)) continue;
            parts.push_back({f[q], nb});
            tot += (nb + 255) / 256 * 256;
        }
        parts.push_back({c->sc, sizeof(Scal)});
        tot += 256;
    }
    CK(cudaMalloc(&sn.mem, tot));
    size_t o = 0;
    for (auto &p : parts) {
        sn.src.push_back(p.first);
        sn.dst.push_back((char *)sn.mem + o);
        sn.bytes.push_back(p.second);
        o += (p.second + 255) / 256 * 256;
    }
    return FARGO_OK;
}

// Rebuild the launch sequence (after a shape change) and drop the graph.
static int batch_rebuild(fargo_batch *b)
{
    CK(cudaStreamSynchronize(b->stream));
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    b->seq.clear();
    return b->prec == FARGO_F64 ? batch_setup<double>(b) : batch_setup<float>(b);
}

// Summed device time (ms) of one profiled step, averaged over reps steps,
// each from the snapshot.
static int btime(fargo_batch *b, BSnap &sn, int reps, float *ms)
{
    std::vector<float> t(b->seq.size() + 1);
    double tot = 0.0;
    int rc;
    for (int r = 0; r < reps; r++) {
        if ((rc = bsnap_copy(b, sn, false))) return rc;
        int n = 0;
        if ((rc = fargo_batch_profile_step(b, (int)t.size(), t.data(), &n, nullptr))) return rc;
        if (r == 0 && reps > 1) continue;   // warm-up
        for (int i = 0; i < n; i++) tot += t[i];
    }
    *ms = (float)(tot / (reps > 1 ? reps - 1 : 1));
    return FARGO_OK;
}

extern "C" int fargo_batch_autotune(fargo_batch *b, int reps, int *cfg, float *ms_default, float *ms_tuned)
{
    if (!b || reps < 2) return FARGO_ERR_BADARG;
    BSnap sn;
    int rc = bsnap_make(b, sn);
    if (rc) return rc;
    const long long steps0 = b->steps;
    if ((rc = bsnap_copy(b, sn, true)) == FARGO_OK) {
        const int cpt0 = b->cpt;
        std::vector<int> seg0(b->n), segz0(b->n);
        for (int i = 0; i < b->n; i++) {
            seg0[i] = b->mem[i]->seg_y;
            segz0[i] = b->mem[i]->seg_z;
        }
        float base = 0.f, best = 0.f;
        rc = btime(b, sn, reps, &base);
        best = base;
        int best_cpt = cpt0, best_seg = -1;   // -1: the members' own segment settings
        const int cpts[4] = {4, 8, 16, 32};
        for (int k = 0; k < 4 && !rc; k++) {
            if (cpts[k] == cpt0) continue;
            b->cpt = cpts[k];
            float t = 0.f;
            if ((rc = batch_rebuild(b)) || (rc = btime(b, sn, reps, &t))) break;
            if (t < best) {
                best = t;
                best_cpt = cpts[k];
            }
        }
        b->cpt = best_cpt;
        const int segs[5] = {0, 16, 32, 64, 128};
        for (int k = 0; k < 5 && !rc; k++) {
            for (fargo_ctx *c : b->mem) c->seg_y = c->seg_z = segs[k];
            float t = 0.f;
            if ((rc = batch_rebuild(b)) || (rc = btime(b, sn, reps, &t))) break;
            if (t < best) {
                best = t;
                best_seg = segs[k];
            }
        }
        for (int i = 0; i < b->n; i++) {
            b->mem[i]->seg_y = best_seg >= 0 ? best_seg : seg0[i];
            b->mem[i]->seg_z = best_seg >= 0 ? best_seg : segz0[i];
        }
        if (!rc) rc = batch_rebuild(b);
        const int rc2 = bsnap_copy(b, sn, false);
        if (!rc) rc = rc2;
        if (cfg) {
            cfg[0] = b->cpt;
            cfg[1] = best_seg;
        }
        if (ms_default) *ms_default = base;
        if (ms_tuned) *ms_tuned = best;
    }
    cudaStreamSynchronize(b->stream);
    b->steps = steps0;
    cudaFree(sn.mem);
    return rc;
}
