// Device-side data structures shared by the kernels of the hydro step.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fk {

enum { CART = 0, CYL = 1, SPH = 2 };
enum { BC_REFLECT = 0, BC_FROZEN = 1, BC_ZEROGRAD = 2, BC_PERIODIC = 3 };

// Mesh description and run constants, passed by value to every kernel.
struct MeshD {
    int nx, nyt, nzt, gy, gz, j0, j1, k0, k1, g;
    int hasX, hasY, hasZ, geom, iso, fargo, av_lit, has_nu, has_planet, indirect, has_star, has_av;
    int bcy[2], bcz[2];
    int pery, perz;              // periodic Y / Z (both sides)
    int jf, kf;                  // first interior Y / Z face: j0 + 1 and k0 + 1, or j0 / k0 when periodic
    int sj, sk;                  // row pitch, plane stride (elements)
    long long ntot;              // elements per field (below 2^31, checked at creation)
    double dx, xmin, gamma, g1, cq, cfl, omega, pq, pa, pa3, peps, peps2, av_c2, om_rel;
    double php0;                 // planet azimuth at t = 0 in the current frame (moved by frame changes)
    double fr0;                  // the mesh's angle to the planetary integrator's non-rotating axes is
                                 // fr0 + omega t (the frame rate piecewise constant; moved by frame changes)
    int shearing;                // Cartesian shearing sheet
    const double *pl_pos;        // planets' positions read on the device each step (x, y, z at pl_pos +
                                 // p * pl_stride), or null for the fixed circular orbit
    const double *pl_mass;       // their masses (device), or null: the planet of creation's q
    int pl_n, pl_stride;
    int mhd;                     // magnetic field (Sec. 3.5): Cartesian, standard transport
    int mhd_passive;             // the field is transported but exerts no force on the gas
    double eta;                  // Ohmic diffusivity
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
    // planets whose positions are read each step (pl_pos), rebuilt at the
    // step's start: per planet p, five per-ring tables at mring + (5 p + t) *
    // nyt * nzt (R - a_p, 4 R a_p, (Z - z_p)^2, q_p R a_p / |r_p|^3 and
    // q_p Z z_p / |r_p|^3), its azimuth tables at ps / pc + p * nx, its mass
    T *mring, *mq;
    // run constants in the field precision (no FP64 work in FP32 kernels)
    T gm1, cq2, omega, pq, peps2, dx, half_gm1, g1, k4;
    // Courant screening: 4 nu / dmin^2 and dmin per ring
    const T *r4, *dminT;
    // the frame's share of the X momentum per unit mass, per ring: R^2 Omega_f
    // (cylindrical, spherical), 2 Omega_f y (shearing sheet), 0 (Cartesian);
    // and the shearing sheet's tidal acceleration -4 A Omega_f y per Y face
    const T *wfr, *tid;
    const double *wfrd;
    // inverse centre-to-centre distances across Y faces (per j) and Z faces (per ring)
    const T *idyc, *idzc;
    // reciprocals of mesh lengths: per ring 1/lenx, 1/lenz, 1/R; per j 1/dy,
    // 1/yf, 1/ym; per k 1/dz, 1/sin(zm), 1/(zm[k] - zm[k-1]); scalar 1/dx
    const T *ilenx, *ilenz, *iR, *idy, *iyf, *iym, *idz, *iszm, *idzm;
    T idx;
    // Reference form of the azimuthal velocity (FP32 only; null in FP64).
    // The stored v_x of ring r is v_x - vref[r], a per-ring constant chosen
    // when v_x is set (the ring's mid-range, or 0), so that the slow changes
    // of a nearly Keplerian flow are not rounded away against |v_x| ~ v_K.
    // The transported X momenta are held as Pi - rho A(r), A = R vref + w
    // (w the frame term above), and the Y / Z sweeps move them between the
    // rings' frames with dAy[r] = A(r) - A(r - 1), dAz[r] = A(r) - A(r - nyt).
    T *vref, *dAy, *dAz;
    double *vrefd;
    // MHD: the face-centred field B_x, B_y, B_z (stored like v_x, v_y, v_z;
    // null without a field), and per Y index j / Z index k the inverse of
    // the distance (dy[j-1] + dy[j]) / 2 between cell centres (0 at j = 0)
    T *bfield[3];
    const T *mh_idcy, *mh_idcz;
};

// The magnetic field's three components (null: no field).
template <typename T>
struct MagF {
    T *b[3];
};

template <typename T>
__device__ __forceinline__ T vref_at(const Tab<T> &tb, int ring)
{
    return sizeof(T) == 4 && tb.vref ? tb.vref[ring] : T(0);
}

// The fields a kernel reads or writes.
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
    double t, t_end, dt, xp, yp, dt_fixed, m32;
    long long nstep;
    int err, fixed;
    unsigned int counter, counter2;
    float dtf;     // dt rounded to FP32, published with dt
};

// Mesh facts the per-cell source kernels branch on.  CfgRun reads them from
// the mesh at run time; CfgDisk fixes them at compile time for a disk (the
// azimuth and the radius present, a planet with the indirect term, the
// star, artificial viscosity), which turns those uniform branches into
// straight-line code.  cfg_of picks the class a mesh runs with.
// Planets that a step's potential can feel when their positions are read on
// the device (fargo_set_planet_source).
constexpr int kPotPlanets = 8;

struct CfgRun {
    __host__ __device__ static int geom(const MeshD &m) { return m.geom; }
    __host__ __device__ static bool hasX(const MeshD &m) { return m.hasX; }
    __host__ __device__ static bool hasY(const MeshD &m) { return m.hasY; }
    __host__ __device__ static bool hasZ(const MeshD &m) { return m.hasZ; }
    __host__ __device__ static bool iso(const MeshD &m) { return m.iso; }
    __host__ __device__ static bool planet(const MeshD &m) { return m.has_planet; }
    __host__ __device__ static bool indirect(const MeshD &m) { return m.indirect; }
    __host__ __device__ static bool star(const MeshD &m) { return m.has_star; }
    __host__ __device__ static bool av(const MeshD &m) { return m.has_av; }
    __host__ __device__ static bool shearing(const MeshD &m) { return m.shearing; }
    __host__ __device__ static bool live(const MeshD &m) { return m.pl_pos != nullptr; }
};
template <int GEOM, bool Z, bool ISO, bool LIVE = false>
struct CfgDisk {
    __host__ __device__ static constexpr int geom(const MeshD &) { return GEOM; }
    __host__ __device__ static constexpr bool hasX(const MeshD &) { return true; }
    __host__ __device__ static constexpr bool hasY(const MeshD &) { return true; }
    __host__ __device__ static constexpr bool hasZ(const MeshD &) { return Z; }
    __host__ __device__ static constexpr bool iso(const MeshD &) { return ISO; }
    __host__ __device__ static constexpr bool planet(const MeshD &) { return true; }
    __host__ __device__ static constexpr bool indirect(const MeshD &) { return true; }
    __host__ __device__ static constexpr bool star(const MeshD &) { return true; }
    __host__ __device__ static constexpr bool av(const MeshD &) { return true; }
    __host__ __device__ static constexpr bool shearing(const MeshD &) { return false; }
    __host__ __device__ static constexpr bool live(const MeshD &) { return LIVE; }
};
typedef CfgDisk<SPH, true, false> CfgDisk3D;   // spherical, adiabatic
typedef CfgDisk<CYL, false, true> CfgDisk2D;   // cylindrical, isothermal
// the same disks with their planets read on the device (fargo_set_planet_source)
typedef CfgDisk<SPH, true, false, true> CfgDisk3DLive;
typedef CfgDisk<CYL, false, true, true> CfgDisk2DLive;
enum { CFG_RUN = 0, CFG_DISK3D = 1, CFG_DISK2D = 2, CFG_DISK3D_LIVE = 3, CFG_DISK2D_LIVE = 4 };

template <class F>
inline bool cfg_matches(const MeshD &m)
{
    return F::geom(m) == m.geom && F::hasX(m) == (m.hasX != 0) && F::hasY(m) == (m.hasY != 0) &&
           F::hasZ(m) == (m.hasZ != 0) && F::iso(m) == (m.iso != 0) && F::planet(m) == (m.has_planet != 0) &&
           F::indirect(m) == (m.indirect != 0) && F::star(m) == (m.has_star != 0) && F::av(m) == (m.has_av != 0) &&
           F::shearing(m) == (m.shearing != 0) && F::live(m) == (m.pl_pos != nullptr);
}
inline int cfg_of(const MeshD &m)
{
    if (cfg_matches<CfgDisk3D>(m)) return CFG_DISK3D;
    if (cfg_matches<CfgDisk2D>(m)) return CFG_DISK2D;
    if (cfg_matches<CfgDisk3DLive>(m)) return CFG_DISK3D_LIVE;
    if (cfg_matches<CfgDisk2DLive>(m)) return CFG_DISK2D_LIVE;
    return CFG_RUN;
}

// The step in the field precision.
template <typename T>
__device__ __forceinline__ T step_dt(const Scal *sc);
template <>
__device__ __forceinline__ double step_dt<double>(const Scal *sc) { return sc->dt; }
template <>
__device__ __forceinline__ float step_dt<float>(const Scal *sc) { return sc->dtf; }

// a / b: IEEE division in FP64, the fast reciprocal-based division in FP32
// (within 2 ulp for |b| below 2^126, and branch-free: the IEEE FP32 division
// carries a slow-path branch).  Used where the quotient is an increment
// (an acceleration, a slope), never where a state value is rebuilt every
// step, since its error is not centred and would accumulate there.
__device__ __forceinline__ double div_fast(double a, double b) { return a / b; }
__device__ __forceinline__ float div_fast(float a, float b) { return __fdividef(a, b); }

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
