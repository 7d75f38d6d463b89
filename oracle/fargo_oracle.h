/*
 * Plain, slow FP64 CPU oracle of one FARGO3D hydrodynamic time step
 * (Benitez-Llambay & Masset 2016, Sec. 3 and Appendices A-B).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Every field is a full array of shape (nz_t + 1, ny_t + 1, nx), X fastest,
 * ny_t = ny + 2g (ny > 1) else 1, nz_t likewise.  Scalars are cell centred;
 * v_x, v_y, v_z live on the lower X, Y, Z face of their cell (Sec. 2.3).
 */
#ifndef FARGO_ORACLE_H
#define FARGO_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_CART = 0, OR_CYL = 1, OR_SPH = 2 };
enum { OR_BC_REFLECT = 0, OR_BC_FROZEN = 1, OR_BC_ZEROGRAD = 2, OR_BC_PERIODIC = 3 };

typedef struct {
    int geom, nx, ny, nz, g;
    double xmin, xmax;
    const double *yf, *zf;      /* face coordinates, ny_t+1 and nz_t+1 entries */
    double gamma;
    int iso;                    /* 1: P = cs^2 rho (Eq. eos1); 0: P = (gamma-1) e (Eq. eos2) */
    const double *cs;           /* isothermal sound speed per ring [nz_t][ny_t] */
    const double *nu;           /* kinematic viscosity per ring [nz_t][ny_t], NULL = inviscid */
    double cfl, cq;
    int av_dt_literal;          /* 1: Delta t_3 = 4 sqrt2 |Delta/Delta v| as printed in Sec. 3.4 */
    double omega_f;             /* constant frame rotation rate */
    int fargo;                  /* 0: STANDARD transport */
    int bc_ylo, bc_yhi, bc_zlo, bc_zhi;
    double star_mass, planet_q, planet_a, planet_eps;
    int indirect;
    double planet_phase0;       /* planet azimuth at t = 0 in the current frame (moved by frame changes) */
    int shearing;               /* Cartesian shearing sheet (Sec. 2): X along the shear flow, Y across it */
    double oort_a;              /* its shear rate A (the unperturbed flow is v_x = 2 A y) */
    int planet_live;            /* n > 0: n integrated planets at planet_pos, masses planet_mass */
    double planet_pos[8][3];    /* their positions (x, y, z) */
    double planet_mass[8];      /* their masses */
    int mhd;                    /* 1: magnetic field B (Sec. 3.5), Cartesian meshes, STANDARD transport */
    int mhd_passive;            /* 1: B evolves passively: no magnetic force on the gas */
    double eta;                 /* Ohmic diffusivity (uniform) */
} or_params;

/* bx, by, bz: face-centred like vx, vy, vz (NULL without MHD). */
typedef struct { double *rho, *e, *vx, *vy, *vz, *bx, *by, *bz; } or_state;

/* Full step: cells 2..12 of the flow chart (Fig. 2).  dt_fixed > 0 skips the
 * Courant reduction and uses the given step.  Returns 0 or a negative code. */
/* Threads of the OpenMP loops (no effect without OpenMP), and their number. */
void or_set_threads(int n);
int  or_get_threads(void);

int  or_step(const or_params *p, or_state *s, double t, double t_end, double dt_fixed, double *dt_out);

/* Individual sub-steps (each cites its section inside the source). */
void or_bc_fill(const or_params *p, or_state *s);
/* Frame change at time t to the rotation rate omega_new (Sec. 3.2, Eq. 13):
 * corrects v_x everywhere and updates p (omega_f, planet_phase0). */
void or_change_frame(or_params *p, or_state *s, double omega_new, double t);
void or_v0(const or_params *p, const or_state *s, double *v0 /* [nz_t][ny_t] */);
void or_v0_all(const or_params *p, const or_state *s, double *v0 /* [nz_t][ny_t], every ring */);
int  or_cfl(const or_params *p, const or_state *s, const double *v0, double t, double t_end, double *dt);
void or_potential(const or_params *p, double t, double *phi /* full cell array */);
void or_substep1(const or_params *p, or_state *s, const double *phi, double dt);
void or_artificial_viscosity(const or_params *p, or_state *s, double dt);
void or_compression_heating(const or_params *p, or_state *s, double dt);
void or_viscosity(const or_params *p, or_state *s, double dt);
void or_momenta(const or_params *p, const or_state *s, double *pi[6]);
void or_transport_x(const or_params *p, or_state *s, double *pi[6], const double *v0, double dt);
void or_orbital_shift(const or_params *p, or_state *s, double *pi[6], const double *v0, double dt);
void or_transport_y(const or_params *p, or_state *s, double *pi[6], double dt);
void or_transport_z(const or_params *p, or_state *s, double *pi[6], double dt);
void or_new_velocities(const or_params *p, or_state *s, double *pi[6]);

/* MHD (Sec. 3.5), Cartesian meshes, mu_0 = 1.  Cell 7a's magnetic pressure
 * gradient; cells 8a-8c: the edge EMFs, e_x at (i, j-1/2, k-1/2), e_y at
 * (i-1/2, j, k-1/2), e_z at (i-1/2, j-1/2, k) stored at index (i, j, k)
 * (full arrays); cell 8d: the magnetic tension; cell 10: the constrained
 * transport of the face fields. */
void or_mhd_pressure(const or_params *p, or_state *s, double dt);
void or_mhd_emf(const or_params *p, const or_state *s, double dt, double *ex, double *ey, double *ez);
void or_mhd_tension(const or_params *p, or_state *s, double dt);
void or_mhd_ct(const or_params *p, or_state *s, const double *ex, const double *ey, const double *ez, double dt);
void or_mhd_fargo_emf(const or_params *p, const or_state *s, const double *v0all, double dt, double *ex,
                      double *ey, double *ez);
/* Discrete divergence of B of active cell (i, j, k) times its volume. */
double or_mhd_divb(const or_params *p, const or_state *s, int i, int j, int k);

/* Geometry of Appendix A, per ring (j,k): face areas, inverse volume,
 * volume and azimuthal cell length. Arrays [nz_t][ny_t] (sy, sz also use the
 * extra row / plane: [nz_t+1][ny_t+1]). */
void or_geometry(const or_params *p, double *sx, double *sy, double *sz, double *vinv, double *vol, double *dxr);

/* Force of the active cells' gas on a planet at rp (per unit planet mass),
 * Plummer softening eps; bm08 = 1 subtracts each ring's mean density first.
 * out = (a_x, a_y, a_z, specific torque z). */
/* The specific torque of each active ring on the planet (the torque
 * diagnostic's radial profile): ring[(k - k0) * ny + (j - j0)], summing to
 * or_planet_force's out[3]. */
void or_planet_torque_profile(const or_params *p, const or_state *st, const double rp[3], double eps, int bm08,
                              double *ring);
void or_planet_force(const or_params *p, const or_state *st, const double rp[3], double eps, int bm08,
                     double out[4]);

/* 1D building blocks, exposed for the special-case tests. */
double or_vanleer_slope(double qm, double q0, double qp, double dxm, double dxp);
void or_ppa_faces(int n, const double *q, double xi_signed, double *qstar /* face i = between i-1 and i */);
void or_shift_ring(int n, double *q, long long nshift);
long long or_nearest_int(double x);

#ifdef __cplusplus
}
#endif
#endif
