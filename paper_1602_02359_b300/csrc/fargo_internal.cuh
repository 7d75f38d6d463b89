// Device-side data structures shared by the kernels of the hydro step.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fk {

enum { CART = 0, CYL = 1, SPH = 2 };
enum { BC_REFLECT = 0, BC_FROZEN = 1, BC_ZEROGRAD = 2 };

// Mesh description and run constants, passed by value to every kernel.
struct MeshD {
    int nx, nyt, nzt, gy, gz, j0, j1, k0, k1, g;
    int hasX, hasY, hasZ, geom, iso, fargo, av_lit, has_nu, has_planet, indirect, has_star, has_av;
    int bcy[2], bcz[2];
    int sj, sk;                  // row pitch, plane stride (elements)
    long long ntot;              // elements per field (below 2^31, checked at creation)
    double dx, xmin, gamma, g1, cq, cfl, omega, pq, pa, pa3, peps, peps2, av_c2, om_rel;
};

// Geometry tables (Appendix A) in the field precision T, plus the FP64
// tables that the Courant reduction and the orbital advection need bit for bit.
template <typename T>
struct Tab {
    // per Y index j (nyt + 1 entries)
    const T *ym, *dy, *yf, *dyc;
    // per Z index k (nzt + 1 entries)
    const T *zm, *dz, *zf, *szm, *szf, *cotzm, *cotzf;
    // per ring (j,k): index k * nyt + j
    const T *R, *lenx, *lenz, *dzc, *sx, *vinv, *cs, *nu, *gphy, *gphz, *fz;
    // per face (j,k): index k * (nyt + 1) + j
    const T *sy, *sz;
    // FP64 per ring
    const double *lx, *ly, *lz, *dmin, *csd, *nud, *Rd, *zcd;
    // FP64 per azimuthal index i: cos and sin of the cell-centre azimuth
    const double *cosx, *sinx;
    // planet: per ring R - a, 4 R a, Z^2 and (q/a^2) R (the indirect term's
    // coefficient); per azimuth, rewritten every step, sin^2(dphi/2) and
    // cos(dphi) of the offset to the planet
    const T *rma, *fra, *z2, *qar;
    T *ps, *pc;
    // run constants in the field precision (no FP64 work in FP32 kernels)
    T gm1, cq2, omega, pq, peps2, dx, half_gm1, g1, k4;
    // Courant screening: 4 nu / dmin^2 and dmin per ring
    const T *r4, *dminT;
    // inverse centre-to-centre distances across Y faces (per j) and Z faces (per ring)
    const T *idyc, *idzc;
    // reciprocals of mesh lengths: per ring 1/lenx, 1/lenz, 1/R; per j 1/dy,
    // 1/yf, 1/ym; per k 1/dz, 1/sin(zm), 1/(zm[k] - zm[k-1]); scalar 1/dx
    const T *ilenx, *ilenz, *iR, *idy, *iyf, *iym, *idz, *iszm, *idzm;
    T idx;
};

template <typename T>
struct Fld {
    T *rho, *e, *vx, *vy, *vz;
};

// Up to eight transported quantities: rho, e, Pi-x, Pi+x, Pi-y, Pi+y, Pi-z, Pi+z.
template <typename T>
struct QSet {
    T *q[8];
    int nq;
};

// Device scalars of the run.  `counter` serves the last-block reductions.
struct Scal {
    double t, t_end, dt, xp, yp, dt_fixed, m32, wsh;
    long long nstep;
    int err, fixed;
    unsigned int counter, counter2;
    float dtf;     // dt rounded to FP32, published with dt
};

// The step in the field precision.
template <typename T>
__device__ __forceinline__ T step_dt(const Scal *sc);
template <>
__device__ __forceinline__ double step_dt<double>(const Scal *sc) { return sc->dt; }
template <>
__device__ __forceinline__ float step_dt<float>(const Scal *sc) { return sc->dtf; }

// v - v0 for a field value v and an FP64 v0 split as v0 = hi + lo (hi, lo in
// the field precision): (v - hi) is formed exactly with TwoSum, then lo is
// subtracted, so the result is within about one ulp of the exact difference
// without FP64 arithmetic.
__device__ __forceinline__ float sub_split(float v, float hi, float lo)
{
    const float s = v - hi;
    const float bb = s - v;
    const float err = (v - (s - bb)) + (-hi - bb);
    return s + (err - lo);
}
__device__ __forceinline__ double sub_split(double v, double hi, double lo) { return v - hi - lo; }

// Element index of cell (i, j, k) in a field array.  32-bit: a context's
// fields hold fewer than 2^31 elements, so no index overflows and each
// neighbour address costs one integer multiply-add.
typedef int idx_t;
__device__ __forceinline__ idx_t IX(const MeshD &m, int i, int j, int k) { return k * m.sk + j * m.sj + i; }

}  // namespace fk
