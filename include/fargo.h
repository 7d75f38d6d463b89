/*
 * fargo.h — C ABI of a B300 (sm_103a) implementation of one explicit
 * hydrodynamic time step of the FARGO3D method (Benitez-Llambay & Masset
 * 2016): Courant reduction, source sub-steps, dimensionally split van Leer
 * transport with left/right momenta, and FARGO orbital advection.
 *
 * Conventions
 *  - Every call returns FARGO_OK (0) or a negative FARGO_ERR_* code; no C++
 *    exception crosses the ABI.  fargo_strerror() names a code.
 *  - A context owns all device memory it allocates (state, scratch, tables).
 *    Caller buffers are borrowed for the duration of a call only.
 *  - Fields are stored in the context precision (FARGO_F64 -> double,
 *    FARGO_F32 -> float).  Field arrays exchanged with the caller are dense,
 *    X fastest, in the context precision:
 *      region FARGO_ACTIVE: nz * ny * nx values (active cells only);
 *      region FARGO_FULL  : (nz_t+1) * (ny_t+1) * nx values, ghosts included,
 *        with ny_t = ny + 2*ghost when ny > 1 else 1 (nz_t likewise).  The
 *        extra row / plane holds the face velocity v_y / v_z on the upper
 *        face of the last ghost cell (staggered mesh, Sec. 2.3).
 *    Scalars (density, energy) are cell centred; velocity component v_d sits
 *    on the lower d-face of its cell.
 *  - FP32 contexts hold the azimuthal velocity internally as v_x - vref,
 *    with one reference vref per ring (the ring's mid-range when v_x is
 *    set, or 0 where that would not be exact), so that the slow changes of
 *    a nearly Keplerian flow are not rounded away against |v_x| ~ v_K.  The
 *    field calls convert: v_x is written and read as v_x itself.  Writing
 *    v_x (any region) chooses the references afresh; the values of rings
 *    outside the written region are kept (rounded once to FP32).
 *  - A context is thread-compatible, not thread-safe.  Work is queued on the
 *    stream given at creation (NULL = the legacy default stream).
 *  - Errors found on the device (non-finite state, Courant step not
 *    positive) are latched in a device flag; the step that meets one leaves
 *    the state unchanged and later calls that synchronise report the code.
 */
#ifndef FARGO_H
#define FARGO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fargo_ctx fargo_ctx;

/* Mesh geometries (Sec. 2.2, Tab. "corresp"): X = azimuth, Y = radius,
 * Z = z (cylindrical) or colatitude (spherical). */
enum { FARGO_CART = 0, FARGO_CYL = 1, FARGO_SPH = 2 };
enum { FARGO_F64 = 0, FARGO_F32 = 1 };
/* Y/Z boundary conditions (X is periodic, Sec. 3.4.1): reflecting wall,
 * frozen ghosts (keep the values given), zero gradient, periodic (Sec. 4.1,
 * ghost zones: every value read across the boundary is the value one period
 * away).  Periodic goes on both sides of an axis or neither; Y may be
 * periodic on Cartesian meshes, Z on Cartesian and cylindrical ones (the
 * geometry does not change along those axes).  On a periodic axis the first
 * face (j0 / k0) is interior and updated by every sub-step, the ghosts are
 * refreshed with their images after each sub-step and sweep that changes
 * the values they copy, the ghost cells' widths must equal those of their
 * images, and so must the per-ring tables cs and nu (fargo_create checks
 * both, to 1e-12 relative), and the axis needs more active cells than
 * ghost layers. */
enum { FARGO_BC_REFLECT = 0, FARGO_BC_FROZEN = 1, FARGO_BC_ZEROGRAD = 2, FARGO_BC_PERIODIC = 3 };
/* Fields: the gas's five, and the magnetic field's face-centred components
 * (stored like v_x, v_y, v_z; only once fargo_enable_mhd was called). */
enum { FARGO_RHO = 0, FARGO_ENERGY = 1, FARGO_VX = 2, FARGO_VY = 3, FARGO_VZ = 4,
       FARGO_BX = 5, FARGO_BY = 6, FARGO_BZ = 7 };
enum { FARGO_ACTIVE = 0, FARGO_FULL = 1 };

enum {
    FARGO_OK = 0,
    FARGO_ERR_BADARG = -1,        /* invalid argument or parameter */
    FARGO_ERR_OOM = -2,           /* device or host allocation failed */
    FARGO_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    FARGO_ERR_NONFINITE = -4,     /* NaN/Inf, rho <= 0 or e < 0 met by the Courant reduction */
    FARGO_ERR_DT = -5,            /* Courant step not positive and finite */
    FARGO_ERR_SIZE = -6,          /* buffer size mismatch or mesh beyond a kernel limit */
    FARGO_ERR_BARRIER_TIMEOUT = -7,
    FARGO_ERR_NOTBUILT = -8       /* CUDA device absent or kernel image missing */
};

/* Planet on a fixed circular orbit (Sec. 3.7, with the orbit fixed): mass
 * ratio q, orbital radius a, Plummer smoothing length eps, indirect term on
 * or off.  The planet phase is (Omega_p - Omega_f) t, Omega_p = sqrt((M+q)/a^3). */
typedef struct {
    double q, a, eps;
    int indirect;
} fargo_planet;

/* Run parameters.  Host pointers are copied at creation. */
typedef struct {
    double xmin, xmax;          /* X extent; the azimuth spans 2 pi in cyl/sph */
    const double *yfaces;       /* ny_t + 1 Y face coordinates (ghost faces included) */
    const double *zfaces;       /* nz_t + 1 Z face coordinates */
    const double *cs;           /* isothermal sound speed per ring, nz_t*ny_t (j fastest), Eq. eos1 */
    const double *nu;           /* kinematic viscosity per ring, nz_t*ny_t, or NULL (App. B) */
    double cfl;                 /* Courant number C of Eq. cfl2 (paper default 0.44) */
    double cq;                  /* artificial-viscosity coefficient C_q (<= 0 disables it) */
    int av_dt_literal;          /* 1: Courant AV term 4 sqrt2 |Delta/Delta v| as printed */
    double omega_frame;         /* constant frame rotation Omega_f */
    int fargo;                  /* 1: orbital advection (Sec. 3.4.1); 0: STANDARD transport */
    int bc_y[2], bc_z[2];       /* lower / upper boundary condition per axis */
    double star_mass;           /* central mass M (cyl/sph); 0 = none */
    int precision;              /* FARGO_F64 or FARGO_F32 */
    void *stream;               /* cudaStream_t, NULL = legacy default stream */
    int shearing;               /* 1: Cartesian shearing sheet (Sec. 2): X along the shear flow, Y
                                   across it; X momentum rho (v_x + 2 Omega_f y) (Tab. momenta), and
                                   the Y source 2 Omega_f v_x - 4 A Omega_f y; Cartesian meshes only */
    double oort_a;              /* the sheet's shear rate A (unperturbed flow v_x = 2 A y) */
} fargo_params;

/* Create a context for an nx * ny * nz active mesh with `ghost` ghost layers
 * in each active Y/Z direction (Sec. 4.1; >= 2).  gamma > 0 selects the
 * adiabatic EOS P = (gamma-1) e (Eq. eos2); gamma <= 0 the locally isothermal
 * P = cs^2 rho (Eq. eos1), which needs prm->cs.  planet may be NULL.
 * Allocates every device buffer and uploads the 1D/2D geometry tables of
 * Appendix A.  Fields start at zero.  Errors: BADARG, OOM, CUDA, NOTBUILT,
 * SIZE (a ring does not fit the orbital-advection kernel's shared memory). */
int fargo_create(fargo_ctx **out, int geom, int nx, int ny, int nz, int ghost,
                 double gamma, const fargo_planet *planet, const fargo_params *prm);
void fargo_destroy(fargo_ctx *ctx);

/* Copy one field in or out (region FARGO_ACTIVE or FARGO_FULL, see above).
 * `bytes` must equal the region's element count times the element size.
 * on_device = 1: src/dst is a device pointer on the context's device.
 * Synchronises the context stream.  Errors: BADARG, SIZE, CUDA. */
int fargo_set_field(fargo_ctx *ctx, int field, int region, const void *src, size_t bytes, int on_device);
int fargo_get_field(fargo_ctx *ctx, int field, int region, void *dst, size_t bytes, int on_device);

/* Simulation time t (FP64, kept on the device) and the end time that clips
 * the last Courant step (Sec. 3.4).  Setting t also clears the step counter
 * and the latched error flag. */
int fargo_set_time(fargo_ctx *ctx, double t, double t_end);

/* One full update (flow chart Fig. 2, cells 2-12): queued on the context
 * stream as one CUDA graph launch, no host synchronisation.  dt_out (may be
 * NULL) receives the step taken, which synchronises.  A step after t has
 * reached t_end does nothing.  Errors: CUDA, and when dt_out is given the
 * latched NONFINITE / DT. */
int fargo_step(fargo_ctx *ctx, double *dt_out);

/* Steps with dt fixed by the caller (no Courant reduction; v0 is still
 * computed).  Used to compare sub-domains at one common step. */
int fargo_step_fixed(fargo_ctx *ctx, double dt);

/* Advance until t = t_end (the last step lands on it) or max_steps steps,
 * polling the device time every `poll` graph launches (>= 1).  t_end
 * becomes the context's end time: later fargo_step calls at t >= t_end are
 * void steps (dt = 0) until fargo_set_time or another fargo_run_to moves it.
 * steps_done may be NULL.  Errors: CUDA, NONFINITE, DT. */
int fargo_run_to(fargo_ctx *ctx, double t_end, long long max_steps, int poll, long long *steps_done);

/* t, last dt, steps taken, latched error code (0 or FARGO_ERR_*). Synchronises. */
int fargo_get_scalars(fargo_ctx *ctx, double *t, double *dt_last, long long *nsteps, int *err);

/* Force of the gas on a planet at rp (Sec. 3.7, orbital integrator: the
 * force of the disk on the planets, evaluated once per hydrodynamical step),
 * per unit planet mass, G = 1:
 *   a = sum over active cells of rho V (r_c - r_p) / (|r_c - r_p|^2 + eps^2)^(3/2)
 * with r_c the cell centre (Cartesian coordinates, the star at the origin)
 * and eps the Plummer softening.  bm08 = 1 removes each ring's mean density
 * before the sum (the option of the same section: an axisymmetric disk then
 * exerts no force).  out (host, 4 values) = (a_x, a_y, a_z, the z component
 * of r_p x a, the specific torque).  Reads the current state; per-cell
 * arithmetic in the field precision, each lane's per-ring sums in the field
 * precision added into a compensated total, lanes and blocks summed in
 * FP64; deterministic.  Cylindrical and spherical meshes.  Synchronises.
 * Errors: BADARG (NULL, eps < 0 or not finite, non-finite rp, Cartesian
 * mesh), CUDA. */
int fargo_planet_force(fargo_ctx *ctx, const double rp[3], double eps, int bm08, double out[4]);

/* The torque diagnostic's radial profile (Sec. 3.7): each active ring's share
 * of the specific torque of fargo_planet_force, written to ring (host,
 * ny * nz doubles, ring (j, k) of the active mesh at (k - k0) * ny + (j -
 * j0), j fastest); the shares sum to the total.  Per ring, the lanes' sums
 * in the field precision are added in FP64.  out (host, 4 values, may be
 * NULL) receives fargo_planet_force's result for the same call.
 * Synchronises.  Errors: as fargo_planet_force. */
int fargo_planet_torque_profile(fargo_ctx *ctx, const double rp[3], double eps, int bm08, double *ring,
                                double out[4]);

/* fargo_planet_force without the synchronisation: the work is queued on the
 * context's stream after whatever is queued there (a step, a field upload),
 * and the 4 FP64 results are written to out, memory the device can write
 * (device memory, or mapped pinned host memory), 8-byte aligned, owned by
 * the caller.  Read out after synchronising the stream.  Calls on one
 * context share its scratch and are ordered by its stream.  Errors: as
 * fargo_planet_force, plus BADARG for a misaligned out. */
int fargo_planet_force_async(fargo_ctx *ctx, const double rp[3], double eps, int bm08, double *out);

/* Planets per call of the planetary entry points below (one lane each). */
#define FARGO_MAX_PLANETS 32

/* fargo_planet_force_async for n planets whose positions are on the device:
 * planet i at y + i*stride (x, y, z; stride >= 3 doubles, e.g. 6 for the
 * state rows of fargo_nbody_rk5_async), its 4 results at out + 4*i.  y and
 * out are device memory, 8-byte aligned, owned by the caller; nothing is
 * read on the host, so the call can follow a step with no synchronisation.
 * Errors: BADARG (NULL, n < 1, stride < 3, eps < 0 or not finite,
 * misaligned pointer, Cartesian mesh), SIZE (n > FARGO_MAX_PLANETS), CUDA. */
int fargo_planets_force_async(fargo_ctx *ctx, int n, const double *y, int stride, double eps, int bm08,
                              double *out);

/* One step of the planetary integrator (Sec. 3.7, orbital integrator for
 * planets): the fifth-order Cash-Karp Runge-Kutta method with the Butcher
 * tableau of Tab. rk, fixed step h, for n planets orbiting a star of mass
 * mstar, G = 1, FP64, in the star's frame:
 *   d2r_i/dt2 = -(mstar + m_i) r_i/|r_i|^3
 *               + sum_{j != i} m_j [(r_j - r_i)/|r_j - r_i|^3 - r_j/|r_j|^3]
 * (with indirect = 0 the frame terms are dropped: the m_i beside mstar and
 * the bracket's second term).  No softening between planets.  Before the
 * stages, when kick is given, the gas force updates the velocities:
 * v_i += h (kick_i - kick_star), kick_i = kick + i*kick_stride (3 values
 * used; kick_stride >= 3, 4 for the output of fargo_planets_force_async),
 * kick_star (3 values, may be NULL) the star's gas acceleration.
 * y: [n][6] = (x, y, z, vx, vy, vz) per planet, updated in place; mass: [n].
 * h_dev, when not NULL, holds h on the device (the argument h is then
 * ignored).  All pointers are device memory, 8-byte aligned, owned by the
 * caller.  Queued on `stream` (NULL = legacy default stream); synchronise
 * it before reading y.  Errors: BADARG (NULL y or mass, n < 1, mstar < 0,
 * non-finite mstar or h, kick_stride < 3 with a kick, kick_star without a
 * kick, misaligned pointer), SIZE (n > FARGO_MAX_PLANETS), CUDA. */
int fargo_nbody_rk5_async(int n, double *y, const double *mass, double mstar, double h, const double *h_dev,
                          const double *kick, int kick_stride, const double *kick_star, int indirect,
                          void *stream);

/* The planets' update after a hydrodynamical step, queued on the context's
 * stream behind it (Sec. 3.7: the gas force, evaluated once per step,
 * updates the velocities; then the planets move by the step's dt):
 *   1. the gas force on each planet at its position in y (softening eps,
 *      BM08 option as fargo_planet_force);
 *   2. with indirect = 1, the gas force on the star at the origin
 *      (unsoftened), subtracted from each planet's (the star's frame);
 *   3. fargo_nbody_rk5_async with h = the dt of the context's last step,
 *      read on the device, and the context's star mass.
 * y ([n][6]) and mass ([n]) are device memory owned by the caller; y is
 * updated in place.  The force scratch belongs to the context.  y is in the
 * integrator's star-centred, non-rotating axes; the mesh's axes make the
 * frame angle theta(t) with them (theta = 0 at t = 0 and in a frame that
 * has never rotated; theta advances at Omega_f and stays continuous through
 * fargo_change_frame and fargo_track_frame), so positions are turned by
 * -theta onto the mesh and the forces back by +theta (fargo_planets_force_async
 * likewise).  Errors: as fargo_planets_force_async. */
int fargo_planets_advance_async(fargo_ctx *ctx, int n, double *y, const double *mass, double eps, int bm08,
                                int indirect);

/* Where the step's planets are (Sec. 3.7: the planets interact with the gas;
 * cell 5a feeding cell 5).  pos, when not NULL, is a device address: planet
 * p's (x, y, z) at pos + p * stride (stride >= 3 doubles, 6 for the state
 * rows of fargo_nbody_rk5_async), p < n <= FARGO_MAX_POT_PLANETS, read at
 * the start of every later step.  The potential then sums the n planets'
 * softened potentials (the context's softening) and indirect terms, each
 * planet's azimuth and per-ring tables rebuilt on the device, the indirect
 * term's z part included; mass (device, n values) gives their masses, and
 * may be NULL only for n = 1 (the planet of creation's mass).  So the
 * integrator (fargo_planets_advance_async on the same rows) and the step
 * alternate on the stream with no host round trip.  NULL pos returns to
 * the fixed circular orbit.  The positions are in the integrator's
 * non-rotating axes and are turned onto the mesh by the frame angle at the
 * step's time (see fargo_planets_advance_async).  Requires a planet at
 * creation and a cylindrical or spherical mesh; pos and mass 8-byte
 * aligned, owned by the caller and valid while set.  Errors: BADARG (no
 * planet, Cartesian mesh, context held by a batch, n < 1, stride < 3,
 * n > 1 without masses, misaligned pointer), SIZE (n > FARGO_MAX_POT_PLANETS). */
#define FARGO_MAX_POT_PLANETS 8
int fargo_set_planet_source(fargo_ctx *ctx, const double *pos, int n, int stride, const double *mass);

/* Magnetic field (Sec. 3.5, the method of characteristics with constrained
 * transport, MOCCT), mu_0 = 1, on Cartesian meshes, with standard transport
 * or with orbital advection (FARGO on, e.g. the shearing sheet; Sec. 3.6).
 * Allocates B_x, B_y, B_z (face centred like the velocity, all zero until
 * set with fargo_set_field(FARGO_BX..FARGO_BZ)), the edge EMFs and a third
 * velocity set; from then on every step adds, in the flow chart's order:
 * the gradient of the transverse magnetic pressure after sub-step 1 (cell
 * 7a, B at time t), the EMFs of Eq. 45 minus eta curl B (cells 8a-8c) and
 * the magnetic tension of Eq. 47 (cell 8d), both from the velocities after
 * the source sub-steps, and after the ghost fill of cell 9 the constrained
 * transport dB_a/dt = d_b e_o - d_o e_b for the cyclic (a, b, o), with
 * e = v x B - eta curl B (cell 10; the paper prints Eq. 39 with the signs
 * of B x v).  The Courant step takes the fast speed sqrt(c_s^2 + B^2/rho)
 * for the sound speed and adds the Ohmic rate 4 eta / dmin^2.  B's ghosts
 * are filled like the velocity's (zero gradient, reflection, images on a
 * periodic axis), along every present axis.  passive != 0: the field is
 * transported but the gas feels no magnetic force.  eta: the uniform Ohmic
 * diffusivity (>= 0).  A second call changes passive and eta and keeps B.
 * In an FP32 context the reference form of v_x is switched off (every vref
 * is 0).  With orbital advection the EMFs and the tension's characteristic
 * values take the residual azimuthal velocity v_x - v0 (v0 of Eq. 37 on
 * every ring, ghost rings included), and after cell 10 the field's orbital
 * share is applied (cell 11): the EMFs e_z = v0 B_y and e_y = -v0 B_z
 * averaged upstream over the arc v0 dt of each edge (Eq. 54: the whole
 * cells upstream plus the PPA value of the residual arc), v0 the mean of
 * the rings on both sides of the face, zero on wall edges, through the same
 * constrained transport.  The net flux of B out of every cell is kept to
 * round-off.  Errors: BADARG (not Cartesian, eta negative or not finite,
 * context held by a batch), OOM, CUDA; a step whose orbital arc exceeds 16
 * turns of a ring latches NONFINITE. */
int fargo_enable_mhd(fargo_ctx *ctx, int passive, double eta);

/* Change the frame's rotation rate to omega_new at the current time (Sec.
 * 3.2, Eq. 13): every azimuthal velocity, ghosts included, becomes
 * v_phi - (omega_new - Omega_f) R, R the cylindrical radius of its ring (the
 * lever arm at the face where v_phi is stored), formed in FP64 and rounded
 * once, so the inertial velocity and the angular momentum are unchanged.
 * The planet keeps its azimuth: its phase is continuous at the current time
 * and then advances at the new relative rate.  Later steps use the new
 * rate in the Coriolis and centrifugal terms and in the momenta.  Cylindrical
 * and spherical meshes; a context held by a batch cannot change frame (the
 * batch holds its members' frames).  In FP32 the per-ring references of v_x
 * are chosen afresh in the new frame.  Synchronises.  Errors: BADARG (NULL,
 * non-finite omega_new, Cartesian mesh, context held by a batch), CUDA. */
int fargo_change_frame(fargo_ctx *ctx, double omega_new);

/* Frame tracking (Sec. 3.2, cell 5b of Fig. 2: the x axis follows a planet),
 * called before a step: the frame rate becomes the angular velocity about
 * the polar axis of body `index` of the planetary state y (rows of 6
 * doubles x, y, z, vx, vy, vz in the integrator's non-rotating axes, device
 * memory, as for fargo_nbody_rk5_async), (x vy - y vx) / (x^2 + y^2), and
 * the azimuthal velocities are corrected by Eq. 13 as in fargo_change_frame
 * (the frame's time derivative enters the method only through this
 * correction).  In FP32 the stored v_x - vref is corrected in place and the
 * references are kept.  The frame angle stays continuous.  Synchronises
 * (reads the body's six values).  omega_out, when not NULL, receives the new
 * rate.  Errors: BADARG (NULL y, index outside 0..31, body on the polar
 * axis, Cartesian mesh, context held by a batch, misaligned y), CUDA. */
int fargo_track_frame(fargo_ctx *ctx, const double *y, int index, double *omega_out);

/* Conserved totals over active cells with compensated FP64 sums:
 * out[0] = sum rho V, out[1] = sum e V, out[2] = sum (Pi-_x + Pi+_x)/2 V
 * (X momentum, angular momentum in cyl/sph; Eqs. 16-17, Tab. momenta).
 * Synchronises. */
int fargo_sums(fargo_ctx *ctx, double out[3]);

/* Conserved totals of fargo_sums for a state held in caller buffers, with no
 * device memory allocated by the call.  The paper has no counterpart; this
 * exists for callers that cannot allocate device memory themselves: an
 * application whose device memory belongs to another allocator (a framework
 * pool or a fixed arena with a preset budget), or a latency-critical loop
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.
 * Such a caller hands over its own buffers and needs no fargo_ctx.
 *
 * Inputs (device pointers, precision FARGO_F64 or FARGO_F32): rho, e (NULL
 * when isothermal: out[1] = 0) and v_x in the FULL layout with a dense row
 * pitch of nx values, i.e. shape (nz_t+1, ny_t+1, nx) for the mesh
 * nx*ny*nz with `ghost` ghost layers; vol and R, the cell volume and the
 * azimuthal lever arm (1 Cartesian, r cylindrical, r sin(theta) spherical)
 * per ring, nz_t*ny_t FP64 values (j fastest).  The X momentum carries the
 * frame's share w per unit mass (Tab. momenta): wframe, when not NULL, gives
 * it per ring (nz_t*ny_t FP64 values on the device); NULL means
 * w = R^2 omega_frame, the cylindrical and spherical term.  A Cartesian
 * caller must pass wframe to match fargo_sums: zeros for a plain box (the
 * context adds no frame term there whatever its Omega_f), 2 Omega_f y at the
 * cell-centre Y for the shearing sheet; with NULL, R = 1 would add
 * omega_frame times the mass.  Output: out, a device pointer to 3 FP64
 * values, written on `stream` (NULL = legacy default stream) in the order
 * of fargo_sums.  The call returns once the work is queued; synchronise the
 * stream before reading out.
 *
 * Scratch: a library-wide device array of 1184 * 6 + 2 doubles (about
 * 57 KB).  The CUDA runtime creates it with the library's device code in
 * each context that uses the library (at load or, with lazy module loading,
 * at first use), and every GPU that holds it keeps it until the process
 * exits.  nblocks (0 = four per SM) is the number of thread blocks, at most
 * 1184; a larger value returns FARGO_ERR_SIZE.  The first call on each
 * device (with that device current) looks up the array's device address
 * and caches it for the process; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset, or a reset of the primary
 * context) invalidates the cached address: do not call this entry point
 * after one.  Every call shares the one array and the call clears its
 * counter itself, so calls that overlap on the GPU race and must be
 * serialised by the caller: two streams at once, and equally graph replays
 * of a captured call that may run concurrently (on different streams, or
 * several such nodes in one graph without a dependency between them).
 * Errors: BADARG, SIZE, CUDA. */
int fargo_sums_noalloc(const void *rho, const void *e, const void *vx, int precision, int nx, int ny, int nz,
                       int ghost, const double *vol, const double *R, const double *wframe, double omega_frame,
                       int nblocks, double *out, void *stream);

/* Kernel-level access, for parity tests of single sub-steps.
 * phase: 0 ghost fill, 1 v0 + Courant reduction (the caller's dt is
 * ignored), 2 sub-step 1, 3 artificial viscosity + compression heating,
 * 4 viscosity, 5 momenta + residual X sweep, 6 Y sweep, 7 Z sweep,
 * 8 new velocities, 9 uniform orbital step (integer shift + PPA); with a
 * magnetic field: 10 magnetic pressure (cell 7a), 11 EMFs (cells 8a-8c,
 * into aux 7-9), 12 magnetic tension (cell 8d), 13 constrained transport
 * (cell 10, with the EMFs of aux 7-9).
 * Phases 2-13 use the given dt.  Results land in the state fields; phases
 * 5-9 read and write the momenta, accessible with fargo_get_aux/set_aux;
 * phases 5 and 9 read v0 (fargo_set_aux(6) or phase 1). */
int fargo_debug_phase(fargo_ctx *ctx, int phase, double dt);

/* Auxiliary arrays: which = 0..5 momenta Pi-_x, Pi+_x, Pi-_y, Pi+_y, Pi-_z,
 * Pi+_z (FULL region, context precision); 6 = v0 per ring (nz_t*ny_t FP64);
 * 7..9 = the EMFs e_x, e_y, e_z of the last step (FULL region, with a
 * magnetic field; e_o at index (i, j, k) lies on the edge along o at the
 * lower faces of cell (i, j, k) across the two other directions).
 * In an FP32 context the X momenta are held as Pi - rho (R vref + w), w the
 * frame term of Tab. "momenta" (R^2 Omega_f, or 2 Omega_f y on the shearing
 * sheet), and are exchanged in that form.  Host buffers.  Errors: BADARG,
 * SIZE, CUDA. */
int fargo_get_aux(fargo_ctx *ctx, int which, void *dst, size_t bytes);
int fargo_set_aux(fargo_ctx *ctx, int which, const void *src, size_t bytes);

/* One full update launched kernel by kernel with a CUDA event between
 * launches on the context stream; ms[i] receives the device time of launch
 * i and names[i] (may be NULL) a static string naming its kernel.  At most
 * max_kernels entries; *n_out receives the count.  Synchronises. */
int fargo_profile_step(fargo_ctx *ctx, int max_kernels, float *ms, int *n_out, const char **names);

/* Autotuner of the launch shapes that leave every result unchanged: the
 * azimuths per block of the per-cell source kernels (64, 128, 256) and the
 * segment lengths of the Y and Z sweeps (16 .. 256 rows).  Each candidate is
 * timed with CUDA events on `reps` (>= 2, the first one warming up) full
 * steps, coordinate by coordinate; the state and time are restored from a
 * device snapshot before every trial step and at the end, so the run is
 * unchanged.  cfg (may be NULL) receives {cell block, Y segment, Z segment}.
 * Allocates a temporary snapshot of the state; synchronises.  The paper's
 * own code searches block sizes per kernel in a similar way (Sec. 4.2).  Errors:
 * BADARG, OOM, CUDA. */
int fargo_autotune(fargo_ctx *ctx, int reps, int *cfg);

/* Set those launch shapes directly: cell_bs in {64, 128, 256}; seg_y, seg_z
 * rows per sweep segment (0 = the default: the whole axis up to 96 rows,
 * else 64). */
int fargo_set_launch_shape(fargo_ctx *ctx, int cell_bs, int seg_y, int seg_z);

/* Failure-detection check of the kernels' bounded waits: one block waits on
 * an mbarrier whose arrival never comes, for at most spin_limit polls
 * (1 .. 2^22; the kernels use 2^22), and records the timeout as the step
 * kernels do.  Returns FARGO_ERR_BARRIER_TIMEOUT, the expected outcome:
 * no hang and no fault.  Synchronises the legacy default stream. */
int fargo_debug_wait_timeout(unsigned spin_limit);

/* Arithmetic peaks of the current device, measured (a measurement aid; the
 * paper has no counterpart): out[0] FP64, out[1] FP32 and out[2] packed
 * two-lane FP32 multiply-add throughput in TFLOP/s (2 flops per lane and
 * multiply-add), each the best of three timed launches of independent
 * multiply-add chains filling every SM, after a warm-up launch.  Queued on
 * `stream` (NULL = legacy default stream) and synchronised; allocates 2 KB
 * for the duration of the call; changes no device setting.  The FP64 path
 * of the step is bound by out[0], not by memory.  Errors: BADARG, CUDA. */
int fargo_alu_peaks(double out[3], void *stream);

/* Use (1) or bypass (0) the CUDA graph for fargo_step (default 1). */
int fargo_use_graph(fargo_ctx *ctx, int enable);

/* Number of kernel launches one fargo_step queues (for accounting). */
int fargo_launches_per_step(fargo_ctx *ctx);

const char *fargo_strerror(int code);

/* ------------------------------------------------------------------------
 * Batched engine: n independent contexts (uneven meshes, parameters,
 * geometries and boundary conditions; one precision) advanced together.
 * Each member takes the step of Fig. 2 (cells 2-12) with its OWN Courant
 * step (Sec. 3.4, Eq. 38) and time, exactly as fargo_step would take it:
 * the batched kernels run the single-instance kernels' per-cell and
 * per-ring code on every member, one launch per phase covering all
 * members' blocks, and the step is captured once as a CUDA graph.  A member
 * whose t reached its t_end (fargo_set_time) or whose error flag is set
 * takes void steps.  The paper runs one problem at a time; the batch has
 * no counterpart there.
 *
 * The batch borrows the members: it holds pointers to their device state,
 * tables and tensor maps.  Destroy the batch before any member, and do not
 * step a member on its own while batch work is in flight (call
 * fargo_batch_status first, which synchronises).  Field and time accessors
 * of a member (fargo_set_field, fargo_get_field, fargo_set_time,
 * fargo_get_scalars) are valid between batch calls once
 * fargo_batch_status has returned.
 * ------------------------------------------------------------------------ */
typedef struct fargo_batch fargo_batch;

/* members: n distinct contexts of one precision, none with a periodic Y or
 * Z boundary.  stream: cudaStream_t of the batch (NULL = a stream the batch
 * creates and owns).  Synchronises the members' streams.  Errors: BADARG
 * (NULL, duplicate, mixed precision, a periodic member), OOM, CUDA. */
int fargo_batch_create(fargo_batch **out, fargo_ctx *const *members, int n, void *stream);
void fargo_batch_destroy(fargo_batch *b);

/* One field (FARGO_FIELD_*) of every member in or out in one call, region
 * FARGO_ACTIVE or FARGO_FULL as for fargo_set_field.  src[i] / dst[i] is
 * member i's buffer (host memory, pinned for asynchronous copies, or device
 * memory on the batch's device) of bytes[i] bytes, which must equal that
 * member's region size.  The copies are queued on the batch's stream, so
 * they are ordered with the batch's steps:
 *  - fargo_batch_set_field returns without synchronising; the source
 *    buffers must stay unchanged until the next synchronising batch call
 *    (fargo_batch_get_field or fargo_batch_status);
 *  - fargo_batch_get_field synchronises once, after the last copy.
 * An upload, a step and a download thus cost one host synchronisation per
 * step instead of one per member and field.  Errors: BADARG, SIZE (a
 * member's byte count), CUDA. */
int fargo_batch_set_field(fargo_batch *b, int field, int region, const void *const *src, const size_t *bytes);
int fargo_batch_get_field(fargo_batch *b, int field, int region, void *const *dst, const size_t *bytes);

/* One field of every member in or out as ONE contiguous buffer: the active
 * cells (FARGO_ACTIVE layout) of member 0, then member 1, ..., each nz*ny*nx
 * values X fastest, in the batch's precision; bytes must be the sum of the
 * members' active sizes.  The buffer is host memory (pinned for an
 * asynchronous copy) or device memory.  The batch stages it through a
 * device buffer of the same size (allocated at the first packed transfer,
 * freed with the batch) with one copy and one scatter (gather) kernel, so a
 * field crosses the host link in a single transfer instead of one per row.
 * set: queued on the batch's stream, no synchronisation (keep src unchanged
 * until the next synchronising batch call); get: synchronises.  Errors:
 * BADARG (a field some member does not have), SIZE, OOM, CUDA. */
int fargo_batch_set_field_packed(fargo_batch *b, int field, const void *src, size_t bytes);
int fargo_batch_get_field_packed(fargo_batch *b, int field, void *dst, size_t bytes);

/* Queue one step of every member (one graph launch); no host sync. */
int fargo_batch_step(fargo_batch *b);

/* Synchronise; n_running (may be NULL) = members with no error and t < t_end;
 * first_failed (may be NULL) = lowest index of a member with an error, or -1.
 * Returns that member's latched error (NONFINITE, DT, BARRIER_TIMEOUT) or OK. */
int fargo_batch_status(fargo_batch *b, int *n_running, int *first_failed);

/* Step until no member is running or max_steps batch steps were queued,
 * checking fargo_batch_status every `poll` steps (>= 1).  steps_done and
 * n_running may be NULL.  Errors as fargo_batch_status, BADARG. */
int fargo_batch_run(fargo_batch *b, long long max_steps, int poll, long long *steps_done, int *n_running);

/* Use (1) or bypass (0) the CUDA graph of the batched step (default 1). */
int fargo_batch_use_graph(fargo_batch *b, int enable);

/* Number of kernel launches one batched step queues. */
int fargo_batch_launches_per_step(const fargo_batch *b);

/* Autotuner of the batch's launch shapes that leave every result unchanged:
 * the cells per thread of the per-cell phases (4, 8, 16, 32) and the
 * segment length of the Y/Z sweeps for every member (the members' own
 * setting, 0 = the default rule, 16 .. 128 rows).  Each candidate is timed
 * by per-launch CUDA events over `reps` (>= 2, the first one warming up)
 * batched steps, each started from a device snapshot of every member's state
 * and time; the snapshot is restored at the end, so the run is unchanged.
 * cfg (may be NULL) receives {cells per thread, segment length (-1: the
 * members' own)}; ms_default and ms_tuned (may be NULL) the summed device
 * time of one step with the shapes at entry and with the chosen ones.  The
 * paper's code searches block sizes in a similar way (Sec. 4.2).  Allocates
 * the snapshot (the members' state fields) for the duration of the call;
 * synchronises.  Errors: BADARG, OOM, CUDA. */
int fargo_batch_autotune(fargo_batch *b, int reps, int *cfg, float *ms_default, float *ms_tuned);

/* One batched step launched kernel by kernel with CUDA events between
 * launches; as fargo_profile_step.  Synchronises. */
int fargo_batch_profile_step(fargo_batch *b, int max_kernels, float *ms, int *n_out, const char **names);

#ifdef __cplusplus
}
#endif
#endif /* FARGO_H */
