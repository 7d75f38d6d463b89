// Host-side state of one hydro instance (the opaque fargo_ctx of the C ABI)
// and the buffer routing of its step, shared by the single-instance entry
// points (fargo_api.cu) and the batched engine (fargo_batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "../../include/fargo.h"
#include "fargo_internal.cuh"
#include "kernels_bc_cfl.cuh"
#include "kernels_source.cuh"
#include "kernels_transport.cuh"
#include "kernels_planet.cuh"
#include "kernels_nbody.cuh"
#include "kernels_mhd.cuh"

namespace fk {

template <typename T>
struct Buffers {
    Fld<T> A{};                 // state: rho, e, vx, vy, vz
    T *vB[3] = {nullptr, nullptr, nullptr};
    T *piA[6] = {}, *piB[6] = {};
    T *rhoB = nullptr, *eB = nullptr;
    Tab<T> tab{};
    // MHD (fargo_enable_mhd): the EMFs of the edges and the velocities after
    // the magnetic tension (the field itself is tab.bfield)
    T *ef[3] = {nullptr, nullptr, nullptr};
    T *vM[3] = {nullptr, nullptr, nullptr};
    // MHD with orbital advection: Eq. 37 on every ring, and the residual v_x
    double *v0all = nullptr;
    T *dvx = nullptr;
};

struct HostGeom {
    // FP64 tables, computed with the same expressions as a plain evaluation
    std::vector<double> ym, dy, zm, dz, dyc, lx, ly, lz, dmin, R, zc, vol, fz, dzc;
    std::vector<double> sx, vinv, sy, sz, lenz, gphy, gphz, cosx, sinx, cs, nu;
    std::vector<double> rma, fra, z2, qar;
    std::vector<double> wfr, tid;   // frame term of the X momentum per ring; shearing-sheet tide per Y face
};

// Everything one step of one instance needs on the device: the mesh, its
// tables, and the routing of the step, i.e. which buffers each phase reads
// and writes.  Velocity buffers go A -> B -> A (-> B); the Y and Z sweeps are
// out of place, and the X sweep is in place or not so that the last sweep
// lands in the state buffers.
template <typename T>
struct StepPlan {
    MeshD m;
    Tab<T> tb;
    Fld<T> A, VB;      // state and the scratch velocities of the source step
    Fld<T> vsrc;       // post-source velocities (VB with viscosity, else A; with magnetic
                       // forces, the tension's output VM)
    Fld<T> vpre;       // the velocities the EMFs and the tension read (VB with viscosity, else A)
    Fld<T> VM;         // the tension's output (MHD)
    MagF<T> B;         // the field (null without MHD)
    T *E[3];           // the EMFs (MHD)
    double *v0all;     // MHD with orbital advection: every ring's v0
    T *dvx;            //   and the residual v_x the EMFs and the tension read
    Fld<T> txin;       // input of the X sweep: state scalars, post-source velocities
    QSet<T> qx, qy, qz;   // outputs of the X, Y and Z sweeps
    QSet<T> qfin;      // quantity set after the sweeps (orbital step in place, new velocities)
    QSet<T> tau;       // viscous stresses (the scratch momenta of set B)
    Scal *sc;
    double *v0, *part;
    float *ringmax;
    int nrings_active, cfl_blocks, seg_y, seg_z;
};

}  // namespace fk

struct fargo_ctx {
    int prec;  // FARGO_F64 / FARGO_F32
    fk::MeshD m{};
    int nx, ny, nz, g, geom;
    int nyt, nzt, pitch;
    size_t esz;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    fk::Scal *sc = nullptr;
    double *v0 = nullptr, *part = nullptr, *part2 = nullptr, *sums = nullptr, *vol = nullptr;
    double *pf = nullptr;   // planet force: result (4), then the azimuth and ring tables of one call
    double *pacc = nullptr; // planetary step: gas accelerations of up to kNbMax planets and of the star (4 each)
    double *pprof = nullptr; // torque profile: each active ring's planet-frame y force
    double star_mass = 0.0;
    int batch_refs = 0;     // batches holding this context (their plans snapshot its frame)
    float *ringmax = nullptr;
    int nrings_active = 0, cfl_blocks = 0, sum_blocks = 0;
    fk::Buffers<double> b64;
    fk::Buffers<float> b32;
    std::vector<void *> allocs;
    fk::HostGeom hg;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    int launches = 0;
    fk::RingShape tx_rs{}, orb_rs{};   // launch shapes of the two ring kernels
    std::vector<double> yfaces_store, zfaces_store;
    fk::SweepMaps mapsY{}, mapsZ{};   // tensor maps of the Y and Z sweeps of the step
    // launch shapes (fargo_autotune): azimuths per block of the per-cell
    // kernels, and segment lengths of the Y / Z sweeps (0 = the default rule)
    int cell_bs = 256, seg_y = 0, seg_z = 0;
};

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            fprintf(stderr, "fargo: %s failed: %s\n", #call, cudaGetErrorString(e_));           \
            return e_ == cudaErrorMemoryAllocation ? FARGO_ERR_OOM : FARGO_ERR_CUDA;              \
        }                                                                                        \
    } while (0)

namespace fk {

// Quantity sets (Sec. 3.2): rho, e (adiabatic), Pi-/+ of each active direction.
template <typename T>
static QSet<T> qset(const fargo_ctx *c, T *rho, T *e, T *const *pi)
{
    QSet<T> s{};
    int n = 0;
    s.q[n++] = rho;
    if (!c->m.iso) s.q[n++] = e;
    s.q[n++] = pi[0];
    s.q[n++] = pi[1];
    if (c->m.hasY) {
        s.q[n++] = pi[2];
        s.q[n++] = pi[3];
    }
    if (c->m.hasZ) {
        s.q[n++] = pi[4];
        s.q[n++] = pi[5];
    }
    s.nq = n;
    return s;
}

template <typename T>
static StepPlan<T> make_plan(const fargo_ctx *c, const Buffers<T> &b)
{
    StepPlan<T> p{};
    const MeshD &m = c->m;
    p.m = m;
    p.tb = b.tab;
    p.A = b.A;
    p.VB = {b.A.rho, b.A.e, b.vB[0], b.vB[1], b.vB[2]};
    p.vsrc = m.has_nu ? p.VB : p.A;
    p.vpre = p.vsrc;
    for (int d = 0; d < 3; d++) {
        p.B.b[d] = m.mhd ? b.tab.bfield[d] : nullptr;
        p.E[d] = b.ef[d];
    }
    p.VM = {b.A.rho, b.A.e, b.vM[0], b.vM[1], b.vM[2]};
    p.v0all = b.v0all;
    p.dvx = b.dvx;
    if (m.mhd && !m.mhd_passive) p.vsrc = p.VM;
    p.txin = {b.A.rho, b.A.e, p.vsrc.vx, p.vsrc.vy, p.vsrc.vz};
    for (int q = 0; q < 6; q++) p.tau.q[q] = b.piB[q];
    p.tau.nq = 6;
    QSet<T> qa = qset<T>(c, b.A.rho, b.A.e, b.piA), qb = qset<T>(c, b.rhoB, b.eB, b.piB);
    const bool x_out = ((m.hasY + m.hasZ) % 2) == 1;
    p.qx = x_out ? qb : qa;
    QSet<T> cur = p.qx, oth = x_out ? qa : qb;
    if (m.hasY) {
        p.qy = oth;
        QSet<T> t = cur; cur = oth; oth = t;
    }
    if (m.hasZ) {
        p.qz = oth;
        QSet<T> t = cur; cur = oth; oth = t;
    }
    p.qfin = cur;   // the state set qa again
    p.sc = c->sc;
    p.v0 = c->v0;
    p.part = c->part;
    p.ringmax = c->ringmax;
    p.nrings_active = c->nrings_active;
    p.cfl_blocks = c->cfl_blocks;
    p.seg_y = c->seg_y > 0 ? c->seg_y : sweep_seglen(m.j1 - m.j0);
    p.seg_z = c->seg_z > 0 ? c->seg_z : sweep_seglen(m.k1 - m.k0);
    return p;
}

static inline int err_code(int flags)
{
    if (flags & 1) return FARGO_ERR_NONFINITE;
    if (flags & 2) return FARGO_ERR_DT;
    if (flags & kErrTimeout) return FARGO_ERR_BARRIER_TIMEOUT;
    return FARGO_OK;
}

// 3D launch shape of the per-cell kernels: x = azimuth (at most bs per
// block), y = rows, z = planes.
static inline dim3 cell_block(const MeshD &m, int bs)
{
    int bx = (m.nx + 31) / 32 * 32;
    return dim3(bx < bs ? bx : bs, 1, 1);
}
static inline dim3 cell_grid(const MeshD &m, int ny, int nz, int bs)
{
    const dim3 b = cell_block(m, bs);
    return dim3((m.nx + b.x - 1) / b.x, ny, nz);
}
// every row (extra face row included) and the planes of cell_planes()
static inline dim3 cell_grid_all(const MeshD &m, int bs) { return cell_grid(m, m.nyt + 1, cell_planes(m), bs); }
static inline dim3 tau_grid(const MeshD &m, int bs) { return cell_grid(m, tau_rows(m), tau_planes(m), bs); }

static inline unsigned grid_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace fk
