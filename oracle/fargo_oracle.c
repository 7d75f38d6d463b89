/*
 * Plain FP64 CPU oracle of one FARGO3D hydrodynamic time step, with the
 * magnetohydrodynamics of Sec. 3.5 (MOCCT) on Cartesian meshes.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Written from the
 * paper (Benitez-Llambay & Masset 2016): every loop is a plain triple loop
 * over the mesh in the order of the flow chart (Fig. 2), with no blocking or
 * fusion.  Where the paper is silent the reading taken is stated at the spot.
 * Pins: tests/test_oracle_pins.py, tests/test_bruteforce_pins.py (the
 * hydrodynamic step), tests/test_mhd_oracle.py (the MHD functions).
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused: the
 * Courant step, the mean azimuthal velocity and the integer shift must be
 * reproducible bit for bit.
 *
 * Built with OpenMP, the loops over rings (or lines) are shared among
 * threads (PAR2 below, or a parallel region around the ring loop).  Every
 * ring's arithmetic is unchanged and each iteration writes only its own
 * cells; the one reduction, the Courant minimum, is exact in any order, so
 * the results are bit-identical to a single thread.  Without OpenMP the
 * pragmas are ignored.
 */
#include "fargo_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PAR2 _Pragma("omp parallel for collapse(2) schedule(static)")

/* Threads used by the loops above (1 when built without OpenMP). */
void or_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Mesh bookkeeping                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_params *p;
    int nx, nyt, nzt, gy, gz, j0, j1, k0, k1;
    int hasX, hasY, hasZ;
    int pery, perz;      /* periodic Y / Z (both sides) */
    int jf, kf;          /* first interior Y / Z face: j0 + 1, or j0 on a periodic axis */
    size_t sj, sk, n;
    double dx;
    double *ym, *dy, *zm, *dz;
} mesh;

static void mesh_init(mesh *m, const or_params *p)
{
    m->p = p;
    m->nx = p->nx;
    m->nyt = p->ny > 1 ? p->ny + 2 * p->g : 1;
    m->nzt = p->nz > 1 ? p->nz + 2 * p->g : 1;
    m->gy = p->ny > 1 ? p->g : 0;
    m->gz = p->nz > 1 ? p->g : 0;
    m->j0 = m->gy; m->j1 = m->gy + p->ny;
    m->k0 = m->gz; m->k1 = m->gz + p->nz;
    m->hasX = p->nx > 1; m->hasY = p->ny > 1; m->hasZ = p->nz > 1;
    m->pery = m->hasY && p->bc_ylo == OR_BC_PERIODIC;
    m->perz = m->hasZ && p->bc_zlo == OR_BC_PERIODIC;
    m->jf = m->j0 + (m->pery ? 0 : 1);
    m->kf = m->k0 + (m->perz ? 0 : 1);
    m->sj = (size_t)p->nx;
    m->sk = (size_t)(m->nyt + 1) * p->nx;
    m->n = (size_t)(m->nzt + 1) * m->sk;
    m->dx = (p->xmax - p->xmin) / p->nx;
    m->ym = malloc(sizeof(double) * m->nyt);
    m->dy = malloc(sizeof(double) * m->nyt);
    m->zm = malloc(sizeof(double) * m->nzt);
    m->dz = malloc(sizeof(double) * m->nzt);
    for (int j = 0; j < m->nyt; j++) {
        m->ym[j] = 0.5 * (p->yf[j] + p->yf[j + 1]);
        m->dy[j] = p->yf[j + 1] - p->yf[j];
    }
    for (int k = 0; k < m->nzt; k++) {
        m->zm[k] = 0.5 * (p->zf[k] + p->zf[k + 1]);
        m->dz[k] = p->zf[k + 1] - p->zf[k];
    }
}

static void mesh_free(mesh *m)
{
    free(m->ym); free(m->dy); free(m->zm); free(m->dz);
}

#define IDX(m, i, j, k) ((size_t)(k) * (m)->sk + (size_t)(j) * (m)->sj + (size_t)(i))
#define IP(m, i) (((i) + 1) % (m)->nx)
#define IM(m, i) (((i) - 1 + (m)->nx) % (m)->nx)

static double *zalloc(size_t n) { return calloc(n, sizeof(double)); }
/* (MHD helpers, defined with the MHD sub-steps below) */
static size_t mh_nb(const mesh *m, int i, int j, int k, int d, int off);
static double *mh_b(const or_state *s, int d);
static void mhd_tension_from(const or_params *p, const or_state *chr, or_state *s, double dt);
static double *dup(const double *a, size_t n)
{
    double *b = malloc(sizeof(double) * n);
    memcpy(b, a, sizeof(double) * n);
    return b;
}

/* ------------------------------------------------------------------------ */
/* Geometry (Appendix A, Tab. "geom", Eqs. 70-71)                            */
/* ------------------------------------------------------------------------ */
/* Cylindrical radius of ring (j,k): the lever arm of the azimuthal motion. */
static double ring_R(const mesh *m, int j, int k)
{
    switch (m->p->geom) {
    case OR_CYL: return m->ym[j];
    case OR_SPH: return m->ym[j] * sin(m->zm[k]);
    default: return 1.0;
    }
}
/* The frame's share of the X momentum per unit mass of ring (j,k) (Tab.     */
/* momenta): R^2 Omega_f in cylindrical and spherical geometry, 2 Omega_f y  */
/* in the shearing sheet (y the cell-centre Y), none in plain Cartesian.     */
static double frame_w(const mesh *m, int j, int k)
{
    const or_params *p = m->p;
    if (p->geom == OR_CART) return p->shearing ? 2.0 * p->omega_f * m->ym[j] : 0.0;
    double R = ring_R(m, j, k);
    return R * R * p->omega_f;
}
/* Azimuthal (X) cell length of ring (j,k). */
static double len_x(const mesh *m, int j, int k) { return ring_R(m, j, k) * m->dx; }
/* Z cell length and centre-to-centre distance across Z face k. */
static double len_z(const mesh *m, int j, int k)
{
    return m->p->geom == OR_SPH ? m->ym[j] * m->dz[k] : m->dz[k];
}
static double dist_z(const mesh *m, int j, int k)
{
    return m->p->geom == OR_SPH ? m->ym[j] * (m->zm[k] - m->zm[k - 1]) : m->zm[k] - m->zm[k - 1];
}
static double dist_y(const mesh *m, int j) { return m->ym[j] - m->ym[j - 1]; }

static double sxj(const mesh *m, int j)
{
    const double *yf = m->p->yf;
    if (m->p->geom == OR_SPH) return 0.5 * (yf[j + 1] * yf[j + 1] - yf[j] * yf[j]);
    return yf[j + 1] - yf[j];
}
static double sxk(const mesh *m, int k) { return m->p->zf[k + 1] - m->p->zf[k]; }
static double syj(const mesh *m, int j)
{
    const double *yf = m->p->yf;
    switch (m->p->geom) {
    case OR_CYL: return yf[j] * m->dx;
    case OR_SPH: return yf[j] * yf[j] * m->dx;
    default: return 1.0;
    }
}
static double syk(const mesh *m, int k)
{
    const double *zf = m->p->zf;
    switch (m->p->geom) {
    case OR_CYL: return zf[k + 1] - zf[k];
    case OR_SPH: return cos(zf[k]) - cos(zf[k + 1]);
    default: return m->dx * (zf[k + 1] - zf[k]);
    }
}
static double szj(const mesh *m, int j)
{
    const double *yf = m->p->yf;
    if (m->p->geom == OR_CART) return m->dx * (yf[j + 1] - yf[j]);
    return 0.5 * m->dx * (yf[j + 1] * yf[j + 1] - yf[j] * yf[j]);
}
static double szk(const mesh *m, int k)
{
    return m->p->geom == OR_SPH ? sin(m->p->zf[k]) : 1.0;
}
static double vjinv(const mesh *m, int j)
{
    const double *yf = m->p->yf;
    switch (m->p->geom) {
    case OR_CYL: return 2.0 / ((yf[j + 1] * yf[j + 1] - yf[j] * yf[j]) * m->dx);
    case OR_SPH: return 3.0 / ((yf[j + 1] * yf[j + 1] * yf[j + 1] - yf[j] * yf[j] * yf[j]) * m->dx);
    default: return 1.0 / (yf[j + 1] - yf[j]);
    }
}
static double area_x(const mesh *m, int j, int k) { return sxj(m, j) * sxk(m, k); }
static double area_y(const mesh *m, int j, int k) { return syj(m, j) * syk(m, k); }
static double area_z(const mesh *m, int j, int k) { return szj(m, j) * szk(m, k); }
static double inv_vol(const mesh *m, int j, int k) { return vjinv(m, j) / syk(m, k); }

void or_geometry(const or_params *p, double *sx, double *sy, double *sz, double *vinv, double *vol, double *dxr)
{
    mesh m;
    mesh_init(&m, p);
    for (int k = 0; k <= m.nzt; k++)
        for (int j = 0; j <= m.nyt; j++) {
            size_t o = (size_t)k * (m.nyt + 1) + j;
            if (j < m.nyt) sz[o] = area_z(&m, j, k);
            if (k < m.nzt) sy[o] = area_y(&m, j, k);
            if (j < m.nyt && k < m.nzt) {
                sx[o] = area_x(&m, j, k);
                vinv[o] = inv_vol(&m, j, k);
                vol[o] = 1.0 / vinv[o];
                dxr[o] = len_x(&m, j, k);
            }
        }
    mesh_free(&m);
}

/* Pressure from the equation of state (Eqs. eos1, eos2; flow-chart cell 4). */
static double pressure(const mesh *m, const or_state *s, size_t c, int j, int k)
{
    if (m->p->iso) {
        double cs = m->p->cs[(size_t)k * m->nyt + j];
        return cs * cs * s->rho[c];
    }
    return (m->p->gamma - 1.0) * s->e[c];
}

/* ------------------------------------------------------------------------ */
/* Cell 2 / 9: ghost fill.  Reading: reflecting walls mirror scalars and     */
/* tangential velocities about the wall and set the wall-normal velocity to  */
/* zero on the wall face with odd mirroring beyond; frozen boundaries keep   */
/* the values the ghosts were given; zero-gradient copies the last active    */
/* cell (and the first interior normal face).  Periodic (both sides of the   */
/* axis): every ghost value is the value one period away, so the ghost      */
/* layers below the first active cell hold the last active cells, and the   */
/* normal face j1 (the upper face of the last active cell) is face j0.      */
/* ------------------------------------------------------------------------ */
static void fill_periodic(double *a, size_t base, size_t stride, int lo, int hi, int g, int normal, int side)
{
    int n = hi - lo;
    if (side == 0)
        for (int mm = 1; mm <= g; mm++) a[base + (size_t)(lo - mm) * stride] = a[base + (size_t)(lo - mm + n) * stride];
    else
        for (int mm = 0; mm < g + (normal ? 1 : 0); mm++)
            a[base + (size_t)(hi + mm) * stride] = a[base + (size_t)(lo + mm) * stride];
}

static void fill_y(const mesh *m, double *a, int normal, int side, int bc, int k, int i)
{
    int g = m->p->g, j0 = m->j0, j1 = m->j1;
    if (bc == OR_BC_FROZEN) return;
    if (bc == OR_BC_PERIODIC) {
        fill_periodic(a, IDX(m, i, 0, k), m->sj, j0, j1, g, normal, side);
        return;
    }
    for (int mm = 0; mm < g; mm++) {
        if (!normal) {
            int dst = side == 0 ? j0 - 1 - mm : j1 + mm;
            int src;
            if (bc == OR_BC_REFLECT) src = side == 0 ? j0 + mm : j1 - 1 - mm;
            else src = side == 0 ? j0 : j1 - 1;
            a[IDX(m, i, dst, k)] = a[IDX(m, i, src, k)];
        }
    }
    if (normal) {
        if (bc == OR_BC_REFLECT) {
            int w = side == 0 ? j0 : j1;
            a[IDX(m, i, w, k)] = 0.0;
            for (int mm = 1; mm <= g; mm++) {
                if (side == 0) a[IDX(m, i, w - mm, k)] = -a[IDX(m, i, w + mm, k)];
                else a[IDX(m, i, w + mm, k)] = -a[IDX(m, i, w - mm, k)];
            }
        } else { /* zero gradient */
            if (side == 0)
                for (int mm = 0; mm <= g; mm++) a[IDX(m, i, j0 - mm, k)] = a[IDX(m, i, j0 + 1, k)];
            else
                for (int mm = 0; mm <= g; mm++) a[IDX(m, i, j1 + mm, k)] = a[IDX(m, i, j1 - 1, k)];
        }
    }
}

static void fill_z(const mesh *m, double *a, int normal, int side, int bc, int j, int i)
{
    int g = m->p->g, k0 = m->k0, k1 = m->k1;
    if (bc == OR_BC_FROZEN) return;
    if (bc == OR_BC_PERIODIC) {
        fill_periodic(a, IDX(m, i, j, 0), m->sk, k0, k1, g, normal, side);
        return;
    }
    if (!normal) {
        for (int mm = 0; mm < g; mm++) {
            int dst = side == 0 ? k0 - 1 - mm : k1 + mm;
            int src;
            if (bc == OR_BC_REFLECT) src = side == 0 ? k0 + mm : k1 - 1 - mm;
            else src = side == 0 ? k0 : k1 - 1;
            a[IDX(m, i, j, dst)] = a[IDX(m, i, j, src)];
        }
    } else {
        if (bc == OR_BC_REFLECT) {
            int w = side == 0 ? k0 : k1;
            a[IDX(m, i, j, w)] = 0.0;
            for (int mm = 1; mm <= g; mm++) {
                if (side == 0) a[IDX(m, i, j, w - mm)] = -a[IDX(m, i, j, w + mm)];
                else a[IDX(m, i, j, w + mm)] = -a[IDX(m, i, j, w - mm)];
            }
        } else {
            if (side == 0)
                for (int mm = 0; mm <= g; mm++) a[IDX(m, i, j, k0 - mm)] = a[IDX(m, i, j, k0 + 1)];
            else
                for (int mm = 0; mm <= g; mm++) a[IDX(m, i, j, k1 + mm)] = a[IDX(m, i, j, k1 - 1)];
        }
    }
}

/* Ghosts of one magnetic-field component along one line across a Y or Z  */
/* boundary (MHD; reading M11).  A wall's own face of the normal component */
/* is never written: the constrained transport holds the flux through it   */
/* (the EMFs tangential to a wall vanish on it).  Reflecting wall: every   */
/* component mirrored evenly about the wall; zero gradient: the ghosts take */
/* the wall face's value (normal) or the last active cell's (tangential);  */
/* frozen: kept; periodic: the images one period away.                     */
static void fill_b(double *a, size_t base, size_t stride, int lo, int hi, int g, int normal, int side, int bc)
{
    if (bc == OR_BC_FROZEN) return;
    if (bc == OR_BC_PERIODIC) {
        fill_periodic(a, base, stride, lo, hi, g, normal, side);
        return;
    }
    for (int mm = 1; mm <= g; mm++) {
        int dst, src;
        if (normal) {   /* faces: the wall at lo (side 0) or hi (side 1) */
            dst = side == 0 ? lo - mm : hi + mm;
            src = bc == OR_BC_REFLECT ? (side == 0 ? lo + mm : hi - mm) : (side == 0 ? lo : hi);
        } else {        /* cells: lo .. hi - 1 active */
            dst = side == 0 ? lo - mm : hi - 1 + mm;
            src = bc == OR_BC_REFLECT ? (side == 0 ? lo + mm - 1 : hi - mm) : (side == 0 ? lo : hi - 1);
        }
        a[base + (size_t)dst * stride] = a[base + (size_t)src * stride];
    }
}

void or_bc_fill(const or_params *p, or_state *s)
{
    mesh m;
    mesh_init(&m, p);
    double *f[8] = { s->rho, p->iso ? NULL : s->e, s->vx, s->vy, s->vz, NULL, NULL, NULL };
    /* the magnetic field (MHD): each component along every present axis    */
    /* (B_z, B_y stay transverse fields of a mesh without Z or Y)           */
    double *bf[3] = { p->mhd ? s->bx : NULL, p->mhd ? s->by : NULL, p->mhd ? s->bz : NULL };
    if (m.hasY && bf[0]) {
        int bcs[2] = { p->bc_ylo, p->bc_yhi };
        for (int side = 0; side < 2; side++)
            for (int d = 0; d < 3; d++)
                for (int k = 0; k < (d == 2 ? m.nzt + 1 : m.nzt); k++)
                    for (int i = 0; i < m.nx; i++)
                        fill_b(bf[d], IDX(&m, i, 0, k), m.sj, m.j0, m.j1, m.p->g, d == 1, side, bcs[side]);
    }
    if (m.hasZ && bf[0]) {
        int bcs[2] = { p->bc_zlo, p->bc_zhi };
        for (int side = 0; side < 2; side++)
            for (int d = 0; d < 3; d++)
                for (int j = 0; j < (d == 1 ? m.nyt + 1 : m.nyt); j++)
                    for (int i = 0; i < m.nx; i++)
                        fill_b(bf[d], IDX(&m, i, j, 0), m.sk, m.k0, m.k1, m.p->g, d == 2, side, bcs[side]);
    }
    if (m.hasY) {
        int bcs[2] = { p->bc_ylo, p->bc_yhi };
        for (int side = 0; side < 2; side++)
            for (int q = 0; q < 8; q++) {
                if (!f[q]) continue;
                int zn = q == 4 || q == 7, yn = q == 3 || q == 6;
                if (q == 4 && !m.hasZ) continue;
                int kmax = zn ? m.nzt + 1 : m.nzt;
                for (int k = 0; k < kmax; k++)
                    for (int i = 0; i < m.nx; i++)
                        fill_y(&m, f[q], yn, side, bcs[side], k, i);
            }
    }
    if (m.hasZ) {
        int bcs[2] = { p->bc_zlo, p->bc_zhi };
        for (int side = 0; side < 2; side++)
            for (int q = 0; q < 8; q++) {
                if (!f[q]) continue;
                int zn = q == 4 || q == 7, yn = q == 3 || q == 6;
                if (q == 3 && !m.hasY) continue;
                int jmax = yn ? m.nyt + 1 : m.nyt;
                for (int j = 0; j < jmax; j++)
                    for (int i = 0; i < m.nx; i++)
                        fill_z(&m, f[q], zn, side, bcs[side], j, i);
            }
    }
    mesh_free(&m);
}

/* Periodic images of one array on the periodic axes only (the other       */
/* boundaries are filled at cells 2 and 9 alone).  On a periodic axis the    */
/* method reads across the boundary the values one period away, so every    */
/* sub-step that changes values near it refreshes their images before the   */
/* next one reads them: the velocities after each source sub-step, the      */
/* transported quantities after each sweep.  normal: a face-centred array   */
/* along that axis (v_y for Y, v_z for Z).                                   */
static void periodic_images(const mesh *m, double *a, int normal_y, int normal_z)
{
    int g = m->p->g;
    if (m->pery) {
        int kmax = normal_z ? m->nzt + 1 : m->nzt;
        for (int k = 0; k < kmax; k++)
            for (int i = 0; i < m->nx; i++)
                for (int side = 0; side < 2; side++)
                    fill_periodic(a, IDX(m, i, 0, k), m->sj, m->j0, m->j1, g, normal_y, side);
    }
    if (m->perz) {
        int jmax = normal_y ? m->nyt + 1 : m->nyt;
        for (int j = 0; j < jmax; j++)
            for (int i = 0; i < m->nx; i++)
                for (int side = 0; side < 2; side++)
                    fill_periodic(a, IDX(m, i, j, 0), m->sk, m->k0, m->k1, g, normal_z, side);
    }
}

static void periodic_state(const mesh *m, or_state *s, int velocities, int energy)
{
    if (!m->pery && !m->perz) return;
    if (velocities) {
        periodic_images(m, s->vx, 0, 0);
        if (m->hasY) periodic_images(m, s->vy, 1, 0);
        if (m->hasZ) periodic_images(m, s->vz, 0, 1);
    }
    if (energy && !m->p->iso) periodic_images(m, s->e, 0, 0);
}

/* The magnetic field's periodic images (MHD). */
static void periodic_field(const mesh *m, or_state *s)
{
    if (!m->pery && !m->perz) return;
    periodic_images(m, s->bx, 0, 0);
    periodic_images(m, s->by, m->hasY, 0);
    periodic_images(m, s->bz, 0, m->hasZ);
}

/* ------------------------------------------------------------------------ */
/* Cell 3: bulk azimuthal velocity of each ring, Eq. 37 (minimises the L_inf */
/* norm of the residual).  Zero for every ring when FARGO is off.            */
/* ------------------------------------------------------------------------ */
void or_v0(const or_params *p, const or_state *s, double *v0)
{
    mesh m;
    mesh_init(&m, p);
    for (size_t o = 0; o < (size_t)m.nzt * m.nyt; o++) v0[o] = 0.0;
    if (p->fargo)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++) {
                double mx = s->vx[IDX(&m, 0, j, k)], mn = mx;
                for (int i = 1; i < m.nx; i++) {
                    double v = s->vx[IDX(&m, i, j, k)];
                    if (v > mx) mx = v;
                    if (v < mn) mn = v;
                }
                v0[(size_t)k * m.nyt + j] = 0.5 * (mx + mn);
            }
    mesh_free(&m);
}

/* Eq. 37 on every ring, ghost rings included: the velocity whose residual  */
/* the MHD sub-steps see when the field is advected orbitally (reading M13); */
/* on the active rings it is the v0 of or_v0.                                */
void or_v0_all(const or_params *p, const or_state *s, double *v0)
{
    mesh m;
    mesh_init(&m, p);
    for (int k = 0; k < m.nzt; k++)
        for (int j = 0; j < m.nyt; j++) {
            double mx = s->vx[IDX(&m, 0, j, k)], mn = mx;
            for (int i = 1; i < m.nx; i++) {
                double v = s->vx[IDX(&m, i, j, k)];
                if (v > mx) mx = v;
                if (v < mn) mn = v;
            }
            v0[(size_t)k * m.nyt + j] = 0.5 * (mx + mn);
        }
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Cell 6: Courant time step, Eq. cfl2, with the items of Sec. 3.4 and the   */
/* FARGO amendments of Sec. 3.4.2 (residual velocity, shear limit Eq. 38).   */
/* Readings: each Delta t_i is the minimum over the active directions; the   */
/* fluid-motion term uses the larger |v| of the two faces of the cell; the   */
/* artificial-viscosity term is the ZEUS limit Delta/(4 C_q^2 |Delta v|) for  */
/* compressions (printed form 4 sqrt2 |Delta/Delta v| under av_dt_literal);  */
/* C_0 of Eq. 38 is the Courant number.  Terms are summed as inverse squares */
/* in the order 1..4, and the last step is clipped to land on t_end.         */
/* ------------------------------------------------------------------------ */
int or_cfl(const or_params *p, const or_state *s, const double *v0, double t, double t_end, double *dt_out)
{
    mesh m;
    mesh_init(&m, p);
    double best = INFINITY;
    int bad = 0;
    const double g1 = p->gamma * (p->gamma - 1.0);
    _Pragma("omp parallel for collapse(2) schedule(static) reduction(min:best) reduction(|:bad)")
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++) {
            double v0r = p->fargo ? v0[(size_t)k * m.nyt + j] : 0.0;
            double lx = len_x(&m, j, k), ly = m.dy[j], lz = len_z(&m, j, k);
            double dmin = INFINITY;
            if (m.hasX && lx < dmin) dmin = lx;
            if (m.hasY && ly < dmin) dmin = ly;
            if (m.hasZ && lz < dmin) dmin = lz;
            double nu = p->nu ? p->nu[(size_t)k * m.nyt + j] : 0.0;
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k);
                double rho = s->rho[c];
                double cs;
                if (p->iso) cs = p->cs[(size_t)k * m.nyt + j];
                else {
                    double e = s->e[c];
                    if (!isfinite(e) || e < 0.0) bad = 1;
                    cs = sqrt(g1 * e / rho);
                }
                if (!isfinite(rho) || rho <= 0.0) bad = 1;
                double r1 = cs / dmin;
                if (p->mhd) {
                    /* fast magnetosonic speed: c_s^2 + B^2/rho, B from zone-centred
                       two-point averages of the face fields (reading M5) */
                    double b2 = 0.0;
                    for (int a = 0; a < 3; a++) {
                        const double *B = mh_b(s, a);
                        double bc = 0.5 * (B[c] + B[mh_nb(&m, i, j, k, a, 1)]);
                        b2 += bc * bc;
                    }
                    r1 = sqrt(cs * cs + b2 / rho) / dmin;
                }
                double r2 = 0.0, r3 = 0.0;
                if (m.hasX) {
                    double a = fabs(s->vx[c] - v0r), b = fabs(s->vx[IDX(&m, IP(&m, i), j, k)] - v0r);
                    double v = a > b ? a : b;
                    double r = v / lx;
                    if (r > r2) r2 = r;
                    double dv = s->vx[IDX(&m, IP(&m, i), j, k)] - s->vx[c];
                    double ra = p->av_dt_literal ? fabs(dv) / (4.0 * sqrt(2.0) * lx)
                                                  : (dv < 0.0 ? 4.0 * p->cq * p->cq * (-dv) / lx : 0.0);
                    if (ra > r3) r3 = ra;
                    if (!isfinite(s->vx[c])) bad = 1;
                }
                if (m.hasY) {
                    double a = fabs(s->vy[c]), b = fabs(s->vy[c + m.sj]);
                    double v = a > b ? a : b;
                    double r = v / ly;
                    if (r > r2) r2 = r;
                    double dv = s->vy[c + m.sj] - s->vy[c];
                    double ra = p->av_dt_literal ? fabs(dv) / (4.0 * sqrt(2.0) * ly)
                                                  : (dv < 0.0 ? 4.0 * p->cq * p->cq * (-dv) / ly : 0.0);
                    if (ra > r3) r3 = ra;
                    if (!isfinite(s->vy[c])) bad = 1;
                }
                if (m.hasZ) {
                    double a = fabs(s->vz[c]), b = fabs(s->vz[c + m.sk]);
                    double v = a > b ? a : b;
                    double r = v / lz;
                    if (r > r2) r2 = r;
                    double dv = s->vz[c + m.sk] - s->vz[c];
                    double ra = p->av_dt_literal ? fabs(dv) / (4.0 * sqrt(2.0) * lz)
                                                  : (dv < 0.0 ? 4.0 * p->cq * p->cq * (-dv) / lz : 0.0);
                    if (ra > r3) r3 = ra;
                    if (!isfinite(s->vz[c])) bad = 1;
                }
                if (p->cq <= 0.0) r3 = 0.0;
                double r4 = nu > 0.0 ? 4.0 * nu / (dmin * dmin) : 0.0;
                double sum = r1 * r1 + r2 * r2 + r3 * r3 + r4 * r4;
                if (p->mhd && p->eta > 0.0) {   /* Ohmic diffusion, as the viscosity */
                    double r5 = 4.0 * p->eta / (dmin * dmin);
                    sum += r5 * r5;
                }
                double local = 1.0 / sqrt(sum);
                if (local < best) best = local;
            }
        }
    double dt = p->cfl * best;
    /* Shear limit, Eq. 38, between radially adjacent rings. */
    /* (on a periodic Y axis the last ring's outer neighbour is the first) */
    if (p->fargo && m.hasY)
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j < m.j1 - (m.pery ? 0 : 1); j++) {
                int jn = j + 1 < m.j1 ? j + 1 : m.j0;
                double a = v0[(size_t)k * m.nyt + j] / len_x(&m, j, k);
                double b = v0[(size_t)k * m.nyt + jn] / len_x(&m, jn, k);
                double w = fabs(a - b);
                if (w > 0.0) {
                    double ds = p->cfl / w;
                    if (ds < dt) dt = ds;
                }
            }
    if (t + dt > t_end) dt = t_end - t;
    mesh_free(&m);
    *dt_out = dt;
    if (bad) return -4;
    if (!(dt > 0.0) || !isfinite(dt)) return -5;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cell 5: gravitational potential at cell centres at time t.  Reading: a    */
/* central mass (Phi = -M/r with r the spherical radius), a planet of mass q */
/* on a fixed circular orbit of radius a in the midplane at phase            */
/* phi_0 + (Omega_p - Omega_f) t, Omega_p = sqrt((M+q)/a^3) (phi_0 = 0 until  */
/* a frame change moves it), or at the given position of an integrated      */
/* planet (Sec. 3.7, cell 5a), Plummer smoothing eps,                         */
/* and the indirect term q (r . r_p)/a^3.                                     */
/* ------------------------------------------------------------------------ */
void or_potential(const or_params *p, double t, double *phi)
{
    mesh m;
    mesh_init(&m, p);
    double M = p->star_mass, q = p->planet_q, a = p->planet_a;
    double om = q > 0.0 ? sqrt((M + q) / (a * a * a)) : 0.0;
    double ph = p->planet_phase0 + (om - p->omega_f) * t;
    /* the planets: one on the circular orbit, or the integrated ones */
    int np = p->planet_live > 0 ? p->planet_live : 1;
    double xs[8], ys[8], zs[8], qs[8], r3s[8];
    for (int n = 0; n < np; n++) {
        if (p->planet_live > 0) {
            xs[n] = p->planet_pos[n][0]; ys[n] = p->planet_pos[n][1]; zs[n] = p->planet_pos[n][2];
            qs[n] = p->planet_mass[n];
        } else {
            xs[n] = a * cos(ph); ys[n] = a * sin(ph); zs[n] = 0.0;
            qs[n] = q;
        }
        double r2 = xs[n] * xs[n] + ys[n] * ys[n] + zs[n] * zs[n];
        r3s[n] = p->planet_live > 0 ? r2 * sqrt(r2) : a * a * a;
    }
    PAR2
    for (int k = 0; k < m.nzt; k++)
        for (int j = 0; j < m.nyt; j++)
            for (int i = 0; i < m.nx; i++) {
                double x = p->xmin + (i + 0.5) * m.dx;
                double X, Y, Z, rs;
                if (p->geom == OR_CYL) {
                    double r = m.ym[j];
                    X = r * cos(x); Y = r * sin(x); Z = m.zm[k];
                    rs = sqrt(r * r + Z * Z);
                } else if (p->geom == OR_SPH) {
                    double r = m.ym[j], st = sin(m.zm[k]);
                    X = r * st * cos(x); Y = r * st * sin(x); Z = r * cos(m.zm[k]);
                    rs = r;
                } else {
                    X = x; Y = m.ym[j]; Z = m.zm[k];
                    rs = 0.0;
                }
                double v = 0.0;
                if (M > 0.0 && p->geom != OR_CART) v -= M / rs;
                if (q > 0.0)
                    for (int n = 0; n < np; n++) {
                        double dx = X - xs[n], dy = Y - ys[n], dz = Z - zs[n];
                        double d2 = dx * dx + dy * dy + dz * dz;
                        v -= qs[n] / sqrt(d2 + p->planet_eps * p->planet_eps);
                        if (p->indirect) v += qs[n] * (X * xs[n] + Y * ys[n] + Z * zs[n]) / r3s[n];
                    }
                phi[IDX(&m, i, j, k)] = v;
            }
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Cell 7a, sub-step 1 (Sec. 3.3): pressure gradient with the two-point face */
/* density of Eq. 20, potential gradient and the centrifugal / geometric     */
/* terms, the inertial-frame velocity averaged over four faces before        */
/* squaring (Eq. 12).  All components read the state at sub-step entry.     */
/* Interior faces only: boundary faces belong to the boundary condition.     */
/* ------------------------------------------------------------------------ */
void or_substep1(const or_params *p, or_state *s, const double *phi, double dt)
{
    mesh m;
    mesh_init(&m, p);
    double *P = zalloc(m.n);
    PAR2
    for (int k = 0; k < m.nzt; k++)
        for (int j = 0; j < m.nyt; j++)
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k);
                P[c] = pressure(&m, s, c, j, k);
            }
    double *vx = dup(s->vx, m.n), *vy = dup(s->vy, m.n), *vz = dup(s->vz, m.n);
    const double *rho = s->rho;
    double om = p->omega_f;
    if (m.hasX)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = IDX(&m, IM(&m, i), j, k);
                    double d = len_x(&m, j, k);
                    double acc = -2.0 * (P[c] - P[cm]) / (d * (rho[c] + rho[cm]));
                    if (phi) acc -= (phi[c] - phi[cm]) / d;
                    s->vx[c] = vx[c] + dt * acc;
                }
    if (m.hasY)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.jf; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = c - m.sj;
                    double d = dist_y(&m, j);
                    double acc = -2.0 * (P[c] - P[cm]) / (d * (rho[c] + rho[cm]));
                    if (phi) acc -= (phi[c] - phi[cm]) / d;
                    if (p->geom != OR_CART) {
                        int ip = IP(&m, i);
                        double Rj = ring_R(&m, j, k), Rm = ring_R(&m, j - 1, k);
                        double vt = 0.25 * ((vx[c] + Rj * om) + (vx[IDX(&m, ip, j, k)] + Rj * om)
                                            + (vx[cm] + Rm * om) + (vx[IDX(&m, ip, j - 1, k)] + Rm * om));
                        double cen = vt * vt;
                        if (p->geom == OR_SPH && m.hasZ) {
                            double vth = 0.25 * (vz[c] + vz[c + m.sk] + vz[cm] + vz[cm + m.sk]);
                            cen += vth * vth;
                        }
                        acc += cen / p->yf[j];
                    } else if (p->shearing) {
                        /* shearing sheet (Sec. 3.3, its Y equation): Coriolis 2 Omega_f v_x with
                           v_x averaged over the four faces around the Y face, and the tidal
                           term -4 A Omega_f y at the face */
                        int ip = IP(&m, i);
                        double vxa = 0.25 * (vx[c] + vx[IDX(&m, ip, j, k)] + vx[cm] + vx[IDX(&m, ip, j - 1, k)]);
                        acc += 2.0 * om * vxa - 4.0 * p->oort_a * om * p->yf[j];
                    }
                    s->vy[c] = vy[c] + dt * acc;
                }
    if (m.hasZ)
        PAR2
        for (int k = m.kf; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = c - m.sk;
                    double d = dist_z(&m, j, k);
                    double acc = -2.0 * (P[c] - P[cm]) / (d * (rho[c] + rho[cm]));
                    if (phi) acc -= (phi[c] - phi[cm]) / d;
                    if (p->geom == OR_SPH) {
                        int ip = IP(&m, i);
                        double Rk = ring_R(&m, j, k), Rm = ring_R(&m, j, k - 1);
                        double vt = 0.25 * ((vx[c] + Rk * om) + (vx[IDX(&m, ip, j, k)] + Rk * om)
                                            + (vx[cm] + Rm * om) + (vx[IDX(&m, ip, j, k - 1)] + Rm * om));
                        acc += vt * vt * (cos(p->zf[k]) / sin(p->zf[k])) / m.ym[j];
                    }
                    s->vz[c] = vz[c] + dt * acc;
                }
    periodic_state(&m, s, 1, 0);
    free(P); free(vx); free(vy); free(vz);
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Cell 7b, sub-step 2: von Neumann-Richtmyer artificial viscosity, applied  */
/* component-wise (Sec. 3.3).  The paper defers the formula to ZEUS-2D;      */
/* reading: q_d = C_q^2 rho (Delta v_d)^2 for a compression Delta v_d < 0    */
/* (else 0), its gradient accelerates the faces with the two-point density   */
/* of Eq. 20, and it heats the gas by -q_d Delta v_d / Delta_d.  q is first  */
/* computed everywhere (first pass), then applied (second pass).             */
/* ------------------------------------------------------------------------ */
void or_artificial_viscosity(const or_params *p, or_state *s, double dt)
{
    if (p->cq <= 0.0) return;
    mesh m;
    mesh_init(&m, p);
    double c2 = p->cq * p->cq;
    double *qx = zalloc(m.n), *qy = zalloc(m.n), *qz = zalloc(m.n);
    double *dvx = zalloc(m.n), *dvy = zalloc(m.n), *dvz = zalloc(m.n);
    const double *rho = s->rho;
    PAR2
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++)
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k);
                if (m.hasX) {
                    double dv = s->vx[IDX(&m, IP(&m, i), j, k)] - s->vx[c];
                    dvx[c] = dv;
                    qx[c] = dv < 0.0 ? c2 * rho[c] * dv * dv : 0.0;
                }
                if (m.hasY) {
                    double dv = s->vy[c + m.sj] - s->vy[c];
                    dvy[c] = dv;
                    qy[c] = dv < 0.0 ? c2 * rho[c] * dv * dv : 0.0;
                }
                if (m.hasZ) {
                    double dv = s->vz[c + m.sk] - s->vz[c];
                    dvz[c] = dv;
                    qz[c] = dv < 0.0 ? c2 * rho[c] * dv * dv : 0.0;
                }
            }
    /* on a periodic axis the first face reads q one period away */
    periodic_images(&m, qy, 0, 0);
    periodic_images(&m, qz, 0, 0);
    if (!p->iso)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k);
                    double h = 0.0;
                    if (m.hasX) h += qx[c] * dvx[c] / len_x(&m, j, k);
                    if (m.hasY) h += qy[c] * dvy[c] / m.dy[j];
                    if (m.hasZ) h += qz[c] * dvz[c] / len_z(&m, j, k);
                    s->e[c] -= dt * h;
                }
    if (m.hasX)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = IDX(&m, IM(&m, i), j, k);
                    s->vx[c] -= dt * 2.0 * (qx[c] - qx[cm]) / (len_x(&m, j, k) * (rho[c] + rho[cm]));
                }
    if (m.hasY)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.jf; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = c - m.sj;
                    s->vy[c] -= dt * 2.0 * (qy[c] - qy[cm]) / (dist_y(&m, j) * (rho[c] + rho[cm]));
                }
    if (m.hasZ)
        PAR2
        for (int k = m.kf; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = c - m.sk;
                    s->vz[c] -= dt * 2.0 * (qz[c] - qz[cm]) / (dist_z(&m, j, k) * (rho[c] + rho[cm]));
                }
    periodic_state(&m, s, 1, 1);
    free(qx); free(qy); free(qz); free(dvx); free(dvy); free(dvz);
    mesh_free(&m);
}

/* Geometry-exact velocity divergence of cell (i,j,k): V^-1 sum of S v over */
/* the six faces (Gauss theorem with the areas of Appendix A).               */
static double divergence(const mesh *m, const or_state *s, int i, int j, int k)
{
    size_t c = IDX(m, i, j, k);
    double f = 0.0;
    if (m->hasX) f += area_x(m, j, k) * (s->vx[IDX(m, IP(m, i), j, k)] - s->vx[c]);
    if (m->hasY) f += area_y(m, j + 1, k) * s->vy[c + m->sj] - area_y(m, j, k) * s->vy[c];
    if (m->hasZ) f += area_z(m, j, k + 1) * s->vz[c + m->sk] - area_z(m, j, k) * s->vz[c];
    return f * inv_vol(m, j, k);
}

/* ------------------------------------------------------------------------ */
/* Cell 7c, sub-step 3: compression heating -P div v for a gamma-law gas.    */
/* Reading of "Eq. (40) of Stone & Norman": the time-centred implicit form   */
/* e' = e (1 - theta)/(1 + theta), theta = dt (gamma - 1) div v / 2.         */
/* ------------------------------------------------------------------------ */
void or_compression_heating(const or_params *p, or_state *s, double dt)
{
    if (p->iso) return;
    mesh m;
    mesh_init(&m, p);
    PAR2
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++)
            for (int i = 0; i < m.nx; i++) {
                double th = 0.5 * dt * (p->gamma - 1.0) * divergence(&m, s, i, j, k);
                size_t c = IDX(&m, i, j, k);
                s->e[c] = s->e[c] * (1.0 - th) / (1.0 + th);
            }
    periodic_state(&m, s, 0, 1);
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Cell 7d: viscous stress tensor and velocity update (Appendix B, Eqs.      */
/* 72-77).  Diagonal components at cell centres, off-diagonal ones on the    */
/* edges with the lowest coordinates (Fig. "stress"); derivatives are plain  */
/* centred differences on the staggered mesh.  Readings: the density (and   */
/* viscosity) of an edge is the mean over the cells sharing it; Eq. 75 is   */
/* divided by the face density like Eqs. 76-77.  Every stress is computed    */
/* from the velocities at sub-step entry, then all faces are updated.        */
/* ------------------------------------------------------------------------ */
void or_viscosity(const or_params *p, or_state *s, double dt)
{
    if (!p->nu) return;
    mesh m;
    mesh_init(&m, p);
    const double *rho = s->rho;
    const double *yf = p->yf, *zf = p->zf;
    const double *ym = m.ym, *zm = m.zm, *dy = m.dy, *dz = m.dz;
    double dx = m.dx;
    int geom = p->geom;
    or_state v0s = { s->rho, s->e, dup(s->vx, m.n), dup(s->vy, m.n), dup(s->vz, m.n) };
    const double *vx = v0s.vx, *vy = v0s.vy, *vz = v0s.vz;
    double *txx = zalloc(m.n), *tyy = zalloc(m.n), *tzz = zalloc(m.n);
    double *txy = zalloc(m.n), *txz = zalloc(m.n), *tyz = zalloc(m.n);
#define NU(j, k) (p->nu[(size_t)(k) * m.nyt + (j)])
    /* diagonal components at active cell centres */
    PAR2
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++)
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k), cxp = IDX(&m, IP(&m, i), j, k);
                double dv = divergence(&m, &v0s, i, j, k);
                double rn = rho[c] * NU(j, k);
                double dxx = (vx[cxp] - vx[c]) / len_x(&m, j, k);
                double dyy = m.hasY ? (vy[c + m.sj] - vy[c]) / dy[j] : 0.0;
                double dzz = m.hasZ ? (vz[c + m.sk] - vz[c]) / len_z(&m, j, k) : 0.0;
                if (geom == OR_CART) {
                    txx[c] = -rn * (2.0 * dxx - 2.0 / 3.0 * dv);
                    tyy[c] = -rn * (2.0 * dyy - 2.0 / 3.0 * dv);
                    tzz[c] = -rn * (2.0 * dzz - 2.0 / 3.0 * dv);
                } else if (geom == OR_CYL) {
                    double r = ym[j];
                    double vr = 0.5 * (vy[c] + vy[c + m.sj]);
                    txx[c] = -rn * (2.0 * (dxx + vr / r) - 2.0 / 3.0 * dv);
                    tyy[c] = -rn * (2.0 * dyy - 2.0 / 3.0 * dv);
                    tzz[c] = -rn * (2.0 * dzz - 2.0 / 3.0 * dv);
                } else {
                    double r = ym[j], ct = cos(zm[k]) / sin(zm[k]);
                    double vr = 0.5 * (vy[c] + vy[c + m.sj]);
                    double vt = 0.5 * (vz[c] + vz[c + m.sk]);
                    txx[c] = -rn * (2.0 * (dxx + vr / r + vt * ct / r) - 2.0 / 3.0 * dv);
                    tyy[c] = -rn * (2.0 * dyy - 2.0 / 3.0 * dv);
                    tzz[c] = -rn * (2.0 * (dzz + vr / r) - 2.0 / 3.0 * dv);
                }
            }
    /* on a periodic axis the faces next to the boundary read the diagonal */
    /* stresses one period away */
    periodic_images(&m, txx, 0, 0);
    periodic_images(&m, tyy, 0, 0);
    periodic_images(&m, tzz, 0, 0);
    /* tau_xy on the z-directed edge (i-1/2, j-1/2, k) */
    if (m.hasY)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j <= m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    int im = IM(&m, i);
                    size_t c = IDX(&m, i, j, k), cm = IDX(&m, im, j, k);
                    double rb = 0.25 * (rho[c] + rho[cm] + rho[c - m.sj] + rho[cm - m.sj]);
                    double nb = 0.5 * (NU(j, k) + NU(j - 1, k));
                    double dvx_dy = (vx[c] - vx[c - m.sj]) / (ym[j] - ym[j - 1]);
                    double t;
                    if (geom == OR_CART) {
                        t = (vy[c] - vy[cm]) / dx + dvx_dy;
                    } else if (geom == OR_CYL) {
                        double rf = yf[j];
                        t = dvx_dy - 0.5 * (vx[c] + vx[c - m.sj]) / rf + (vy[c] - vy[cm]) / (rf * dx);
                    } else {
                        double rf = yf[j], sn = sin(zm[k]);
                        t = (vy[c] - vy[cm]) / (rf * sn * dx) + dvx_dy - 0.5 * (vx[c] + vx[c - m.sj]) / rf;
                    }
                    txy[c] = -rb * nb * t;
                }
    /* tau_xz on the y-directed edge (i-1/2, j, k-1/2) */
    if (m.hasZ)
        PAR2
        for (int k = m.k0; k <= m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    int im = IM(&m, i);
                    size_t c = IDX(&m, i, j, k), cm = IDX(&m, im, j, k);
                    double rb = 0.25 * (rho[c] + rho[cm] + rho[c - m.sk] + rho[cm - m.sk]);
                    double nb = 0.5 * (NU(j, k) + NU(j, k - 1));
                    double t;
                    if (geom == OR_CART) {
                        t = (vz[c] - vz[cm]) / dx + (vx[c] - vx[c - m.sk]) / (zm[k] - zm[k - 1]);
                    } else if (geom == OR_CYL) {
                        t = (vx[c] - vx[c - m.sk]) / (zm[k] - zm[k - 1]) + (vz[c] - vz[cm]) / (ym[j] * dx);
                    } else {
                        double r = ym[j], sf = sin(zf[k]);
                        t = sf / r * (vx[c] / sin(zm[k]) - vx[c - m.sk] / sin(zm[k - 1])) / (zm[k] - zm[k - 1])
                            + (vz[c] - vz[cm]) / (r * sf * dx);
                    }
                    txz[c] = -rb * nb * t;
                }
    /* tau_yz on the x-directed edge (i, j-1/2, k-1/2) */
    if (m.hasY && m.hasZ)
        PAR2
        for (int k = m.k0; k <= m.k1; k++)
            for (int j = m.j0; j <= m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k);
                    double rb = 0.25 * (rho[c] + rho[c - m.sj] + rho[c - m.sk] + rho[c - m.sj - m.sk]);
                    double nb = 0.25 * (NU(j, k) + NU(j - 1, k) + NU(j, k - 1) + NU(j - 1, k - 1));
                    double t;
                    if (geom == OR_SPH) {
                        double rf = yf[j];
                        t = (vz[c] - vz[c - m.sj]) / (ym[j] - ym[j - 1]) - 0.5 * (vz[c] + vz[c - m.sj]) / rf
                            + (vy[c] - vy[c - m.sk]) / (rf * (zm[k] - zm[k - 1]));
                    } else {
                        t = (vz[c] - vz[c - m.sj]) / (ym[j] - ym[j - 1]) + (vy[c] - vy[c - m.sk]) / (zm[k] - zm[k - 1]);
                    }
                    tyz[c] = -rb * nb * t;
                }
    /* v_x update on faces (i-1/2, j, k) */
    PAR2
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++)
            for (int i = 0; i < m.nx; i++) {
                int im = IM(&m, i), ip = IP(&m, i);
                size_t c = IDX(&m, i, j, k), cm = IDX(&m, im, j, k);
                (void)ip;
                double rf = 0.5 * (rho[c] + rho[cm]);
                double f = 0.0;
                if (geom == OR_CART) {
                    f += (txx[c] - txx[cm]) / dx;
                    if (m.hasY) f += (txy[c + m.sj] - txy[c]) / dy[j];
                    if (m.hasZ) f += (txz[c + m.sk] - txz[c]) / dz[k];
                } else if (geom == OR_CYL) {
                    double r = ym[j];
                    if (m.hasY) f += (yf[j + 1] * yf[j + 1] * txy[c + m.sj] - yf[j] * yf[j] * txy[c]) / (r * r * dy[j]);
                    f += (txx[c] - txx[cm]) / (r * dx);
                    if (m.hasZ) f += (txz[c + m.sk] - txz[c]) / dz[k];
                } else {
                    double r = ym[j], sn = sin(zm[k]), ct = cos(zm[k]) / sin(zm[k]);
                    if (m.hasY) f += (yf[j + 1] * yf[j + 1] * txy[c + m.sj] - yf[j] * yf[j] * txy[c]) / (r * r * dy[j]);
                    if (m.hasZ) f += (txz[c + m.sk] - txz[c]) / (r * dz[k]);
                    f += (txx[c] - txx[cm]) / (r * sn * dx);
                    if (m.hasY) f += 0.5 * (txy[c] + txy[c + m.sj]) / r;
                    if (m.hasZ) f += 2.0 * 0.5 * (txz[c] + txz[c + m.sk]) * ct / r;
                }
                s->vx[c] = vx[c] - dt * f / rf;
            }
    /* v_y update on interior faces (i, j-1/2, k) */
    if (m.hasY)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.jf; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    int ip = IP(&m, i);
                    size_t c = IDX(&m, i, j, k), cjm = c - m.sj, cp = IDX(&m, ip, j, k);
                    double rf = 0.5 * (rho[c] + rho[cjm]);
                    double f = 0.0;
                    if (geom == OR_CART) {
                        f += (txy[cp] - txy[c]) / dx;
                        f += (tyy[c] - tyy[cjm]) / (ym[j] - ym[j - 1]);
                        if (m.hasZ) f += (tyz[c + m.sk] - tyz[c]) / dz[k];
                    } else if (geom == OR_CYL) {
                        double r = yf[j];
                        f += (ym[j] * tyy[c] - ym[j - 1] * tyy[cjm]) / (r * (ym[j] - ym[j - 1]));
                        f += (txy[cp] - txy[c]) / (r * dx);
                        f -= 0.5 * (txx[c] + txx[cjm]) / r;
                        if (m.hasZ) f += (tyz[c + m.sk] - tyz[c]) / dz[k];
                    } else {
                        double r = yf[j], sn = sin(zm[k]);
                        f += (ym[j] * ym[j] * tyy[c] - ym[j - 1] * ym[j - 1] * tyy[cjm]) / (r * r * (ym[j] - ym[j - 1]));
                        if (m.hasZ) f += (tyz[c + m.sk] * sin(zf[k + 1]) - tyz[c] * sin(zf[k])) / (r * sn * dz[k]);
                        f += (txy[cp] - txy[c]) / (r * sn * dx);
                        f -= 0.5 * (tzz[c] + tzz[cjm] + txx[c] + txx[cjm]) / r;
                    }
                    s->vy[c] = vy[c] - dt * f / rf;
                }
    /* v_z update on interior faces (i, j, k-1/2) */
    if (m.hasZ)
        PAR2
        for (int k = m.kf; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    int ip = IP(&m, i);
                    size_t c = IDX(&m, i, j, k), ckm = c - m.sk, cp = IDX(&m, ip, j, k);
                    double rf = 0.5 * (rho[c] + rho[ckm]);
                    double f = 0.0;
                    if (geom == OR_CART) {
                        f += (txz[cp] - txz[c]) / dx;
                        if (m.hasY) f += (tyz[c + m.sj] - tyz[c]) / dy[j];
                        f += (tzz[c] - tzz[ckm]) / (zm[k] - zm[k - 1]);
                    } else if (geom == OR_CYL) {
                        double r = ym[j];
                        if (m.hasY) f += (yf[j + 1] * tyz[c + m.sj] - yf[j] * tyz[c]) / (r * dy[j]);
                        f += (txz[cp] - txz[c]) / (r * dx);
                        f += (tzz[c] - tzz[ckm]) / (zm[k] - zm[k - 1]);
                    } else {
                        double r = ym[j], sf = sin(zf[k]), ctf = cos(zf[k]) / sin(zf[k]);
                        if (m.hasY) f += (yf[j + 1] * yf[j + 1] * yf[j + 1] * tyz[c + m.sj] - yf[j] * yf[j] * yf[j] * tyz[c]) / (r * r * r * dy[j]);
                        f += (tzz[c] * sin(zm[k]) - tzz[ckm] * sin(zm[k - 1])) / (r * sf * (zm[k] - zm[k - 1]));
                        f += (txz[cp] - txz[c]) / (r * sf * dx);
                        f -= 0.5 * (txx[c] + txx[ckm]) * ctf / r;
                    }
                    s->vz[c] = vz[c] - dt * f / rf;
                }
#undef NU
    periodic_state(&m, s, 1, 0);
    free(txx); free(tyy); free(tzz); free(txy); free(txz); free(tyz);
    free(v0s.vx); free(v0s.vy); free(v0s.vz);
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Cell 12a: left and right momenta (Eqs. 16-17) with the geometric factors  */
/* of Tab. "momenta": X carries rho (R v + R^2 Omega_f), Z in spherical       */
/* geometry carries rho r v_theta.  Computed on every cell that has both     */
/* faces in storage, ghosts included (the sweeps read ghost values).         */
/* pi = { Pi-_x, Pi+_x, Pi-_y, Pi+_y, Pi-_z, Pi+_z }.                          */
/* ------------------------------------------------------------------------ */
void or_momenta(const or_params *p, const or_state *s, double *pi[6])
{
    mesh m;
    mesh_init(&m, p);
    for (int q = 0; q < 6; q++) memset(pi[q], 0, sizeof(double) * m.n);
    PAR2
    for (int k = 0; k < m.nzt; k++)
        for (int j = 0; j < m.nyt; j++) {
            double R = ring_R(&m, j, k);
            double w = frame_w(&m, j, k);
            double fz = p->geom == OR_SPH ? m.ym[j] : 1.0;
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k);
                double r = s->rho[c];
                pi[0][c] = r * (R * s->vx[c] + w);
                pi[1][c] = r * (R * s->vx[IDX(&m, IP(&m, i), j, k)] + w);
                if (m.hasY) { pi[2][c] = r * s->vy[c]; pi[3][c] = r * s->vy[c + m.sj]; }
                if (m.hasZ) { pi[4][c] = r * (fz * s->vz[c]); pi[5][c] = r * (fz * s->vz[c + m.sk]); }
            }
        }
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* van Leer slope (Sec. 3.5, below Eq. 15): the harmonic mean of the two     */
/* one-sided differences divided by the centre-to-centre distances, zero     */
/* when they differ in sign or one vanishes.                                 */
/* ------------------------------------------------------------------------ */
double or_vanleer_slope(double qm, double q0, double qp, double dxm, double dxp)
{
    double dp = (qp - q0) / dxp, dm = (q0 - qm) / dxm;
    if (dp * dm > 0.0) return 2.0 * dp * dm / (dp + dm);
    return 0.0;
}

/* One conservative 1D upwind sweep (Eqs. 1D-advection-X/Y/Z, flux Eq. 14,   */
/* interface value Eq. 15) over one line of cells.  q[0] is the density;     */
/* the other quantities are transported consistently (their ratio to the    */
/* density is interpolated and multiplied by the mass flux).  Face f lies    */
/* between cells f-1 and f; faces c0..c1 are used, cells c0..c1-1 updated.  */
typedef struct {
    int n, nq;
    double **q;          /* nq lines of n values */
    const double *cen;   /* centre coordinate of each cell */
    const double *wid;   /* width of each cell */
    const double *vel;   /* face velocity, face f at index f */
    const double *area;  /* face area, face f at index f */
    const double *vinv;  /* inverse volume per cell */
} line_t;

static double vl_face(const line_t *L, const double *f, int face, double v, double dt)
{
    if (v >= 0.0) {
        int c = face - 1;
        double a = or_vanleer_slope(f[c - 1], f[c], f[c + 1], L->cen[c] - L->cen[c - 1], L->cen[c + 1] - L->cen[c]);
        return f[c] + a * (L->wid[c] - v * dt) / 2.0;
    } else {
        int c = face;
        double a = or_vanleer_slope(f[c - 1], f[c], f[c + 1], L->cen[c] - L->cen[c - 1], L->cen[c + 1] - L->cen[c]);
        return f[c] - a * (L->wid[c] + v * dt) / 2.0;
    }
}

static void sweep_line(const line_t *L, int c0, int c1, double dt)
{
    int n = L->n, nq = L->nq;
    double **ratio = malloc(sizeof(double *) * nq);
    double **flux = malloc(sizeof(double *) * nq);
    for (int q = 0; q < nq; q++) {
        flux[q] = zalloc(n + 1);
        ratio[q] = zalloc(n);
        for (int c = 0; c < n; c++) ratio[q][c] = q == 0 ? L->q[0][c] : L->q[q][c] / L->q[0][c];
    }
    for (int f = c0; f <= c1; f++) {
        double v = L->vel[f];
        double fr = v * vl_face(L, ratio[0], f, v, dt) * L->area[f];
        flux[0][f] = fr;
        for (int q = 1; q < nq; q++) flux[q][f] = fr * vl_face(L, ratio[q], f, v, dt);
    }
    for (int q = 0; q < nq; q++)
        for (int c = c0; c < c1; c++)
            L->q[q][c] -= dt * L->vinv[c] * (flux[q][c + 1] - flux[q][c]);
    for (int q = 0; q < nq; q++) { free(flux[q]); free(ratio[q]); }
    free(flux); free(ratio);
}

/* Nearest integer E(X) of Sec. 3.4.1, ties away from zero. */
long long or_nearest_int(double x) { return llround(x); }

/* Integer shift, Eq. 32: circular permutation Q_i <- Q_{i-N}. */
void or_shift_ring(int n, double *q, long long nshift)
{
    double *t = malloc(sizeof(double) * n);
    long long N = ((nshift % n) + n) % n;
    for (int i = 0; i < n; i++) t[i] = q[(i - N + n) % n];
    memcpy(q, t, sizeof(double) * n);
    free(t);
}

/* PPA interface values on a periodic ring (Eqs. 34-36 and the xi-weighted  */
/* interface value of Sec. 3.4.1).  qstar[i] is the value on the face        */
/* between cells i-1 and i for the uniform signed Courant number xi_signed. */
void or_ppa_faces(int n, const double *q, double xs, double *qstar)
{
    double *dm = zalloc(n), *qr = zalloc(n), *L = zalloc(n), *R = zalloc(n);
    for (int i = 0; i < n; i++) {
        double qm = q[(i - 1 + n) % n], q0 = q[i], qp = q[(i + 1) % n];
        double d = 0.5 * (qp - qm);
        if ((qp - q0) * (q0 - qm) <= 0.0) dm[i] = 0.0;
        else {
            double a = 2.0 * fabs(q0 - qm), b = 2.0 * fabs(qp - q0), c = fabs(d);
            double mn = a < b ? a : b;
            if (c < mn) mn = c;
            dm[i] = d > 0.0 ? mn : -mn;
        }
    }
    for (int i = 0; i < n; i++) {
        int ip = (i + 1) % n;
        qr[i] = q[i] + 0.5 * (q[ip] - q[i]) - (dm[ip] - dm[i]) / 6.0;   /* Eq. 35 */
    }
    for (int i = 0; i < n; i++) {
        double qm = q[(i - 1 + n) % n], q0 = q[i], qp = q[(i + 1) % n];
        double l = qr[(i - 1 + n) % n], r = qr[i];
        if ((qp - q0) * (q0 - qm) <= 0.0) { l = q0; r = q0; }            /* Eq. 36 */
        else {
            double D = r - l, C = q0 - 0.5 * (l + r);
            if (D * C > D * D / 6.0) l = 3.0 * q0 - 2.0 * r;
            else if (-D * D / 6.0 > D * C) r = 3.0 * q0 - 2.0 * l;
        }
        L[i] = l; R[i] = r;
    }
    for (int f = 0; f < n; f++) {
        if (xs >= 0.0) {
            int d = (f - 1 + n) % n;
            double xi = xs;
            qstar[f] = R[d] + xi * (q[d] - R[d]) + xi * (1.0 - xi) * (2.0 * q[d] - R[d] - L[d]);
        } else {
            int d = f;
            double xi = -xs;
            qstar[f] = L[d] + xi * (q[d] - L[d]) + xi * (1.0 - xi) * (2.0 * q[d] - R[d] - L[d]);
        }
    }
    free(dm); free(qr); free(L); free(R);
}

/* Quantities carried by the transport step (Sec. 3.2): density, internal   */
/* energy (adiabatic), and the left/right momenta of each active direction. */
static int gather_quantities(const mesh *m, or_state *s, double *pi[6], double **out)
{
    int nq = 0;
    out[nq++] = s->rho;
    if (!m->p->iso) out[nq++] = s->e;
    out[nq++] = pi[0]; out[nq++] = pi[1];
    if (m->hasY) { out[nq++] = pi[2]; out[nq++] = pi[3]; }
    if (m->hasZ) { out[nq++] = pi[4]; out[nq++] = pi[5]; }
    return nq;
}

/* The transported quantities' periodic images after a sweep. */
static void periodic_quantities(const mesh *m, double **fld, int nq)
{
    if (!m->pery && !m->perz) return;
    for (int q = 0; q < nq; q++) periodic_images(m, fld[q], 0, 0);
}

/* ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------ */
/* Cells 12b-c along X, residual part (Sec. 3.4.1, Eq. fargo1): upwind       */
/* transport at delta v = v - v0 with van Leer interface values (Eq. 15).    */
/* With FARGO off, v0 = 0 and this is the whole STANDARD X transport.        */
/* The X length of ring (j,k) is R dx.  Active rings only.                   */
/* ------------------------------------------------------------------------ */
void or_transport_x(const or_params *p, or_state *s, double *pi[6], const double *v0, double dt)
{
    mesh m;
    mesh_init(&m, p);
    if (!m.hasX) { mesh_free(&m); return; }
    double *fld[8];
    int nq = gather_quantities(&m, s, pi, fld);
    int nx = m.nx, n = nx + 4;
    _Pragma("omp parallel")
    {
        /* line buffers of this thread */
        double **lq = malloc(sizeof(double *) * nq);
        for (int q = 0; q < nq; q++) lq[q] = zalloc(n);
        double *cen = zalloc(n), *wid = zalloc(n), *vel = zalloc(n), *area = zalloc(n), *vinv = zalloc(n);
        _Pragma("omp for collapse(2) schedule(static)")
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++) {
                double dX = len_x(&m, j, k);
                double vr0 = p->fargo ? v0[(size_t)k * m.nyt + j] : 0.0;
                double S = area_x(&m, j, k), Vi = inv_vol(&m, j, k);
                /* the ring padded by two periodic images on each side */
                for (int c = 0; c < n; c++) {
                    int i = ((c - 2) % nx + nx) % nx;
                    cen[c] = c * dX; wid[c] = dX; area[c] = S; vinv[c] = Vi;
                    vel[c] = s->vx[IDX(&m, i, j, k)] - vr0;
                    for (int q = 0; q < nq; q++) lq[q][c] = fld[q][IDX(&m, i, j, k)];
                }
                line_t L = { n, nq, lq, cen, wid, vel, area, vinv };
                sweep_line(&L, 2, nx + 2, dt);
                for (int q = 0; q < nq; q++)
                    for (int i = 0; i < nx; i++) fld[q][IDX(&m, i, j, k)] = lq[q][i + 2];
            }
        for (int q = 0; q < nq; q++) free(lq[q]);
        free(lq); free(cen); free(wid); free(vel); free(area); free(vinv);
    }
    periodic_quantities(&m, fld, nq);
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Uniform orbital step of each ring (Sec. 3.4.1, Eqs. fargo2, 28-33): the   */
/* integer shift by N = E(v0 dt / dX) (Eq. 32), then the fractional step at  */
/* xi = v0 dt/dX - N with PPA interface values (Eqs. 34-36).  Reading: this  */
/* uniform step is split off and applied after the Y and Z sweeps, so that   */
/* the radial and vertical fluxes move each cell's content with the face     */
/* velocities of the same azimuth; applied before them, the multi-cell shift */
/* decorrelates the two and the scheme is unstable at C = 0.44.              */
/* ------------------------------------------------------------------------ */
void or_orbital_shift(const or_params *p, or_state *s, double *pi[6], const double *v0, double dt)
{
    mesh m;
    mesh_init(&m, p);
    if (!m.hasX || !p->fargo) { mesh_free(&m); return; }
    double *fld[8];
    int nq = gather_quantities(&m, s, pi, fld);
    int nx = m.nx;
    _Pragma("omp parallel")
    {
    double *ring = zalloc(nx), *fs = zalloc(nx);    /* buffers of this thread */
    _Pragma("omp for collapse(2) schedule(static)")
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++) {
            double dX = len_x(&m, j, k);
            double vr0 = v0[(size_t)k * m.nyt + j];
            double S = area_x(&m, j, k), Vi = inv_vol(&m, j, k);
            double X = vr0 * dt / dX;
            long long N = or_nearest_int(X);
            double xs = X - (double)N;
            for (int q = 0; q < nq; q++) {
                for (int i = 0; i < nx; i++) ring[i] = fld[q][IDX(&m, i, j, k)];
                or_shift_ring(nx, ring, N);
                for (int i = 0; i < nx; i++) fld[q][IDX(&m, i, j, k)] = ring[i];
            }
            if (xs == 0.0) continue;
            double vR = xs * dX / dt;
            double *flux0 = zalloc(nx + 1), **fl = malloc(sizeof(double *) * nq);
            for (int i = 0; i < nx; i++) ring[i] = fld[0][IDX(&m, i, j, k)];
            or_ppa_faces(nx, ring, xs, fs);
            for (int f = 0; f < nx; f++) flux0[f] = vR * fs[f] * S;
            for (int q = 0; q < nq; q++) {
                fl[q] = zalloc(nx + 1);
                if (q == 0) { memcpy(fl[0], flux0, sizeof(double) * nx); continue; }
                for (int i = 0; i < nx; i++) ring[i] = fld[q][IDX(&m, i, j, k)] / fld[0][IDX(&m, i, j, k)];
                or_ppa_faces(nx, ring, xs, fs);
                for (int f = 0; f < nx; f++) fl[q][f] = flux0[f] * fs[f];
            }
            for (int q = 0; q < nq; q++) {
                for (int i = 0; i < nx; i++)
                    fld[q][IDX(&m, i, j, k)] -= dt * Vi * (fl[q][(i + 1) % nx] - fl[q][i]);
                free(fl[q]);
            }
            free(fl); free(flux0);
        }
    free(ring); free(fs);
    }
    periodic_quantities(&m, fld, nq);
    mesh_free(&m);
}

/* Cells 12b-c along Y (Eq. 1D-advection-Y): non-uniform radial spacing,     */
/* face areas S_y(j,k) and inverse volumes of Appendix A.  Face velocities   */
/* are the post-source v_y, unchanged during the transport step.           */
void or_transport_y(const or_params *p, or_state *s, double *pi[6], double dt)
{
    mesh m;
    mesh_init(&m, p);
    if (!m.hasY) { mesh_free(&m); return; }
    double *fld[8];
    int nq = gather_quantities(&m, s, pi, fld);
    int n = m.nyt;
    _Pragma("omp parallel")
    {
    double **lq = malloc(sizeof(double *) * nq);    /* line buffers of this thread */
    for (int q = 0; q < nq; q++) lq[q] = zalloc(n);
    double *vel = zalloc(n + 1), *area = zalloc(n + 1), *vinv = zalloc(n);
    _Pragma("omp for collapse(2) schedule(static)")
    for (int k = m.k0; k < m.k1; k++)
        for (int i = 0; i < m.nx; i++) {
            for (int j = 0; j < n; j++) {
                size_t c = IDX(&m, i, j, k);
                vel[j] = s->vy[c];
                area[j] = area_y(&m, j, k);
                vinv[j] = inv_vol(&m, j, k);
                for (int q = 0; q < nq; q++) lq[q][j] = fld[q][c];
            }
            line_t L = { n, nq, lq, m.ym, m.dy, vel, area, vinv };
            sweep_line(&L, m.j0, m.j1, dt);
            for (int q = 0; q < nq; q++)
                for (int j = m.j0; j < m.j1; j++) fld[q][IDX(&m, i, j, k)] = lq[q][j];
        }
    for (int q = 0; q < nq; q++) free(lq[q]);
    free(lq); free(vel); free(area); free(vinv);
    }
    periodic_quantities(&m, fld, nq);
    mesh_free(&m);
}

/* Cells 12b-c along Z (Eq. 1D-advection-Z); in spherical geometry the       */
/* colatitude lengths are r dtheta.                                          */
void or_transport_z(const or_params *p, or_state *s, double *pi[6], double dt)
{
    mesh m;
    mesh_init(&m, p);
    if (!m.hasZ) { mesh_free(&m); return; }
    double *fld[8];
    int nq = gather_quantities(&m, s, pi, fld);
    int n = m.nzt;
    _Pragma("omp parallel")
    {
    double **lq = malloc(sizeof(double *) * nq);    /* line buffers of this thread */
    for (int q = 0; q < nq; q++) lq[q] = zalloc(n);
    double *vel = zalloc(n + 1), *area = zalloc(n + 1), *vinv = zalloc(n), *cen = zalloc(n), *wid = zalloc(n);
    _Pragma("omp for schedule(static)")
    for (int j = m.j0; j < m.j1; j++) {
        double f = p->geom == OR_SPH ? m.ym[j] : 1.0;
        for (int k = 0; k < n; k++) { cen[k] = f * m.zm[k]; wid[k] = f * m.dz[k]; }
        for (int i = 0; i < m.nx; i++) {
            for (int k = 0; k < n; k++) {
                size_t c = IDX(&m, i, j, k);
                vel[k] = s->vz[c];
                area[k] = area_z(&m, j, k);
                vinv[k] = inv_vol(&m, j, k);
                for (int q = 0; q < nq; q++) lq[q][k] = fld[q][c];
            }
            line_t L = { n, nq, lq, cen, wid, vel, area, vinv };
            sweep_line(&L, m.k0, m.k1, dt);
            for (int q = 0; q < nq; q++)
                for (int k = m.k0; k < m.k1; k++) fld[q][IDX(&m, i, j, k)] = lq[q][k];
        }
    }
    for (int q = 0; q < nq; q++) free(lq[q]);
    free(lq); free(vel); free(area); free(vinv); free(cen); free(wid);
    }
    periodic_quantities(&m, fld, nq);
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Cell 12d: new face velocities from the new momenta and densities, Eq. 18, */
/* undoing the geometric factors of Tab. "momenta".  Interior faces only.    */
/* ------------------------------------------------------------------------ */
void or_new_velocities(const or_params *p, or_state *s, double *pi[6])
{
    mesh m;
    mesh_init(&m, p);
    const double *rho = s->rho;
    PAR2
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++) {
            double R = ring_R(&m, j, k), w = frame_w(&m, j, k);
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k), cm = IDX(&m, IM(&m, i), j, k);
                s->vx[c] = ((pi[1][cm] + pi[0][c]) / (rho[cm] + rho[c]) - w) / R;
            }
        }
    if (m.hasY)
        PAR2
        for (int k = m.k0; k < m.k1; k++)
            for (int j = m.jf; j < m.j1; j++)
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = c - m.sj;
                    s->vy[c] = (pi[3][cm] + pi[2][c]) / (rho[cm] + rho[c]);
                }
    if (m.hasZ)
        PAR2
        for (int k = m.kf; k < m.k1; k++)
            for (int j = m.j0; j < m.j1; j++) {
                double f = p->geom == OR_SPH ? m.ym[j] : 1.0;
                for (int i = 0; i < m.nx; i++) {
                    size_t c = IDX(&m, i, j, k), cm = c - m.sk;
                    s->vz[c] = (pi[5][cm] + pi[4][c]) / (rho[cm] + rho[c]) / f;
                }
            }
    periodic_state(&m, s, 1, 0);
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* One full update, in the order of the flow chart (Fig. 2).                 */
/* ------------------------------------------------------------------------ */
int or_step(const or_params *p, or_state *s, double t, double t_end, double dt_fixed, double *dt_out)
{
    mesh m;
    mesh_init(&m, p);
    size_t nr = (size_t)m.nzt * m.nyt;
    double *v0 = zalloc(nr), *v0all = NULL;
    double dt;
    int rc = 0;
    /* with orbital advection the MHD sub-steps see the residual velocity    */
    /* and the field's orbital share is cell 11 (Sec. 3.6; reading M13)     */
    int mfargo = p->mhd && p->fargo && m.hasX;
    or_bc_fill(p, s);                                     /* cell 2 */
    or_v0(p, s, v0);                                      /* cell 3 */
    if (mfargo) {
        v0all = zalloc(nr);
        or_v0_all(p, s, v0all);
    }
    if (dt_fixed > 0.0) dt = dt_fixed;
    else rc = or_cfl(p, s, v0, t, t_end, &dt);            /* cells 4-6 */
    if (rc) { free(v0); free(v0all); mesh_free(&m); *dt_out = dt; return rc; }
    double *phi = NULL;
    if (p->planet_q > 0.0 || (p->star_mass > 0.0 && p->geom != OR_CART)) {
        phi = zalloc(m.n);
        or_potential(p, t, phi);                          /* cell 5 */
    }
    or_substep1(p, s, phi, dt);                           /* cell 7a */
    if (p->mhd) or_mhd_pressure(p, s, dt);                /* cell 7a, magnetic pressure */
    or_artificial_viscosity(p, s, dt);                    /* cell 7b */
    or_compression_heating(p, s, dt);                     /* cell 7c */
    or_viscosity(p, s, dt);                               /* cell 7d */
    double *em[3] = { NULL, NULL, NULL };
    if (p->mhd) {
        for (int o = 0; o < 3; o++) em[o] = zalloc(m.n);
        if (mfargo) {
            /* the residual state: v_x - v0 of its ring, every ring */
            or_state r = *s;
            double *dvx = dup(s->vx, m.n);
            for (int k = 0; k < m.nzt; k++)
                for (int j = 0; j < m.nyt; j++)
                    for (int i = 0; i < m.nx; i++) dvx[IDX(&m, i, j, k)] -= v0all[(size_t)k * m.nyt + j];
            r.vx = dvx;
            or_mhd_emf(p, &r, dt, em[0], em[1], em[2]);  /* cells 8a-8c */
            mhd_tension_from(p, &r, s, dt);               /* cell 8d */
            free(dvx);
        } else {
            or_mhd_emf(p, s, dt, em[0], em[1], em[2]);   /* cells 8a-8c */
            or_mhd_tension(p, s, dt);                     /* cell 8d */
        }
    }
    or_bc_fill(p, s);                                     /* cell 9 */
    if (p->mhd) {
        or_mhd_ct(p, s, em[0], em[1], em[2], dt);         /* cell 10 */
        if (mfargo) {
            or_mhd_fargo_emf(p, s, v0all, dt, em[0], em[1], em[2]);
            or_mhd_ct(p, s, em[0], em[1], em[2], dt);     /* cell 11 */
        }
        for (int o = 0; o < 3; o++) free(em[o]);
    }
    double *pi[6];
    for (int q = 0; q < 6; q++) pi[q] = zalloc(m.n);
    or_momenta(p, s, pi);                                 /* cell 12a */
    or_transport_x(p, s, pi, v0, dt);                     /* cells 12b-c */
    or_transport_y(p, s, pi, dt);
    or_transport_z(p, s, pi, dt);
    or_orbital_shift(p, s, pi, v0, dt);
    or_new_velocities(p, s, pi);                          /* cell 12d */
    for (int q = 0; q < 6; q++) free(pi[q]);
    free(phi); free(v0); free(v0all);
    mesh_free(&m);
    *dt_out = dt;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Force of the gas on a planet (Sec. 3.7, orbital integrator: the force of  */
/* the disk on the planets, evaluated once per hydrodynamical step), per     */
/* unit planet mass, G = 1:                                                   */
/*   a = sum over active cells of  m_c (r_c - r_p) / (|r_c - r_p|^2 + eps^2)^(3/2) */
/* with m_c = rho_c V_c and r_c the cell centre in Cartesian coordinates.    */
/* bm08 = 1 removes the axisymmetric part of the density first: rho_c minus  */
/* the mean of rho over the cell's ring (the option of the same section, so */
/* that an axisymmetric disk exerts no force).  out = (a_x, a_y, a_z, the z  */
/* component of r_p x a, the specific torque).  Compensated (Neumaier) sums. */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

void or_planet_force(const or_params *p, const or_state *st, const double rp[3], double eps, int bm08,
                     double out[4])
{
    mesh m;
    mesh_init(&m, p);
    nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0};
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++) {
            double mean = 0.0;
            if (bm08) {
                nsum r = {0, 0};
                for (int i = 0; i < m.nx; i++) nsum_add(&r, st->rho[IDX(&m, i, j, k)]);
                mean = (r.s + r.c) / m.nx;
            }
            double V = 1.0 / inv_vol(&m, j, k);
            for (int i = 0; i < m.nx; i++) {
                double x = p->xmin + (i + 0.5) * m.dx;
                double X, Y, Z;
                if (p->geom == OR_CYL) {
                    double r = m.ym[j];
                    X = r * cos(x); Y = r * sin(x); Z = m.zm[k];
                } else if (p->geom == OR_SPH) {
                    double r = m.ym[j], sn = sin(m.zm[k]);
                    X = r * sn * cos(x); Y = r * sn * sin(x); Z = r * cos(m.zm[k]);
                } else {
                    X = x; Y = m.ym[j]; Z = m.zm[k];
                }
                double mc = (st->rho[IDX(&m, i, j, k)] - mean) * V;
                double dx = X - rp[0], dy = Y - rp[1], dz = Z - rp[2];
                double d2 = dx * dx + dy * dy + dz * dz + eps * eps;
                double w = mc / (d2 * sqrt(d2));
                nsum_add(&ax, w * dx);
                nsum_add(&ay, w * dy);
                nsum_add(&az, w * dz);
            }
        }
    out[0] = ax.s + ax.c;
    out[1] = ay.s + ay.c;
    out[2] = az.s + az.c;
    out[3] = rp[0] * out[1] - rp[1] * out[0];
    mesh_free(&m);
}

/* Radial profile of the torque (Sec. 3.7, the torque of the gas on the     */
/* planet resolved by ring): each active ring's share of the specific       */
/* torque r_p x a (z component), summed like or_planet_force.               */
void or_planet_torque_profile(const or_params *p, const or_state *st, const double rp[3], double eps, int bm08,
                              double *ring)
{
    mesh m;
    mesh_init(&m, p);
    int ny = m.j1 - m.j0;
    for (int k = m.k0; k < m.k1; k++)
        for (int j = m.j0; j < m.j1; j++) {
            double mean = 0.0;
            if (bm08) {
                nsum r = {0, 0};
                for (int i = 0; i < m.nx; i++) nsum_add(&r, st->rho[IDX(&m, i, j, k)]);
                mean = (r.s + r.c) / m.nx;
            }
            double V = 1.0 / inv_vol(&m, j, k);
            nsum tq = {0, 0};
            for (int i = 0; i < m.nx; i++) {
                double x = p->xmin + (i + 0.5) * m.dx;
                double X, Y, Z;
                if (p->geom == OR_CYL) {
                    double r = m.ym[j];
                    X = r * cos(x); Y = r * sin(x); Z = m.zm[k];
                } else if (p->geom == OR_SPH) {
                    double r = m.ym[j], sn = sin(m.zm[k]);
                    X = r * sn * cos(x); Y = r * sn * sin(x); Z = r * cos(m.zm[k]);
                } else {
                    X = x; Y = m.ym[j]; Z = m.zm[k];
                }
                double mc = (st->rho[IDX(&m, i, j, k)] - mean) * V;
                double dx = X - rp[0], dy = Y - rp[1], dz = Z - rp[2];
                double d2 = dx * dx + dy * dy + dz * dz + eps * eps;
                double w = mc / (d2 * sqrt(d2));
                nsum_add(&tq, rp[0] * (w * dy) - rp[1] * (w * dx));
            }
            ring[(size_t)(k - m.k0) * ny + (j - m.j0)] = tq.s + tq.c;
        }
    mesh_free(&m);
}

/* ------------------------------------------------------------------------ */
/* Frame change, Sec. 3.2, Eq. 13: when the frame's rotation rate changes   */
/* from Omega_f to Omega_f', every azimuthal velocity becomes               */
/* v_phi - (Omega_f' - Omega_f) R, R the lever arm at the face where v_phi  */
/* is stored (the ring's cylindrical radius), so the inertial velocity is   */
/* unchanged.  Ghost cells are corrected too.  The planet keeps its azimuth */
/* at time t: its phase offset moves by (Omega_f' - Omega_f) t.             */
/* ------------------------------------------------------------------------ */
void or_change_frame(or_params *p, or_state *s, double omega_new, double t)
{
    mesh m;
    mesh_init(&m, p);
    double dom = omega_new - p->omega_f;
    for (int k = 0; k < m.nzt; k++)
        for (int j = 0; j < m.nyt; j++) {
            double R = ring_R(&m, j, k);
            for (int i = 0; i < m.nx; i++) {
                size_t c = IDX(&m, i, j, k);
                s->vx[c] = s->vx[c] - dom * R;
            }
        }
    p->planet_phase0 += dom * t;
    p->omega_f = omega_new;
    mesh_free(&m);
}

/* ======================================================================== */
/* Magnetohydrodynamics (Sec. 3.5, "Magnetohydrodynamics": the method of    */
/* characteristics and constrained transport, MOCCT), Cartesian meshes,     */
/* mu_0 = 1.  B is face centred like v (Sec. 2.3); the EMF of orientation o */
/* lives on the edges along o (Fig. "cell").  Directions are numbered       */
/* X = 0, Y = 1, Z = 2; an absent direction (one cell) has no neighbours:   */
/* every difference along it vanishes and every average over it is the     */
/* value itself.                                                             */
/* ======================================================================== */

/* Index of the cell `off` cells away from (i, j, k) along direction d (X    */
/* periodic; an absent direction maps onto the cell itself).                */
static size_t mh_nb(const mesh *m, int i, int j, int k, int d, int off)
{
    if (d == 0) return IDX(m, ((i + off) % m->nx + m->nx) % m->nx, j, k);
    if (d == 1) return IDX(m, i, m->hasY ? j + off : j, k);
    return IDX(m, i, j, m->hasZ ? k + off : k);
}
static int mh_has(const mesh *m, int d) { return d == 0 ? m->hasX : (d == 1 ? m->hasY : m->hasZ); }
/* Index of (i, j, k) along d, and the cell width there (Cartesian). */
static int mh_pos(int i, int j, int k, int d) { return d == 0 ? i : (d == 1 ? j : k); }
static double mh_width(const mesh *m, int d, int n) { return d == 0 ? m->dx : (d == 1 ? m->dy[n] : m->dz[n]); }
/* Centre-to-centre distance between cells n - 1 and n along d. */
static double mh_dc(const mesh *m, int d, int n)
{
    return d == 0 ? m->dx : 0.5 * (mh_width(m, d, n - 1) + mh_width(m, d, n));
}
static double *mh_v(const or_state *s, int d) { return d == 0 ? s->vx : (d == 1 ? s->vy : s->vz); }
static double *mh_b(const or_state *s, int d) { return d == 0 ? s->bx : (d == 1 ? s->by : s->bz); }

/* Value at the face between cells n - 1 and n along e (cell (i, j, k) is n)  */
/* of a quantity q that is cell centred along e, carried by the speed w     */
/* over dt: the donor cell's value plus its van Leer slope times half the   */
/* distance from the face to the point that reaches it at dt/2 - the        */
/* interface value of Eq. 15 with w for the flow speed (the upwind estimate */
/* "u" of Sec. 3.5) or for a characteristic speed C+- (the foot values of   */
/* Eqs. 41-44).                                                              */
static double mh_recon(const mesh *m, const double *q, int i, int j, int k, int e, double w, double dt)
{
    size_t c = IDX(m, i, j, k);
    if (!mh_has(m, e)) return q[c];
    int n = mh_pos(i, j, k, e);
    double qm2 = q[mh_nb(m, i, j, k, e, -2)], qm1 = q[mh_nb(m, i, j, k, e, -1)], q0 = q[c],
           qp1 = q[mh_nb(m, i, j, k, e, 1)];
    int nn = e == 0 ? 2 : n;   /* X is uniform: any index serves for its widths */
    if (w >= 0.0) {
        double sl = or_vanleer_slope(qm2, qm1, q0, mh_dc(m, e, nn - 1), mh_dc(m, e, nn));
        return qm1 + 0.5 * sl * (mh_width(m, e, nn - 1) - w * dt);
    }
    double sl = or_vanleer_slope(qm1, q0, qp1, mh_dc(m, e, nn), mh_dc(m, e, nn + 1));
    return q0 - 0.5 * sl * (mh_width(m, e, nn) + w * dt);
}

/* Density at the edge at the lower a- and lower b-face of cell (i, j, k):   */
/* the mean of the four cells around it (Sec. 3.5).                         */
static double mh_rho_edge(const mesh *m, const double *rho, int i, int j, int k, int a, int b)
{
    size_t c00 = IDX(m, i, j, k), c10 = mh_nb(m, i, j, k, a, -1), c01 = mh_nb(m, i, j, k, b, -1);
    int ia = a == 0 ? ((i - 1) % m->nx + m->nx) % m->nx : i, ja = a == 1 && m->hasY ? j - 1 : j,
        ka = a == 2 && m->hasZ ? k - 1 : k;
    size_t c11 = mh_nb(m, ia, ja, ka, b, -1);
    return 0.25 * (rho[c00] + rho[c10] + rho[c01] + rho[c11]);
}

/* Star values at that edge of the pair (v_p, B_p), p one of the edge's two  */
/* transverse directions, from the 1.5D problem along the other one, q      */
/* (Eqs. 41-44): the Alfven characteristics C+- = U -+ W / sqrt(rho) carry   */
/* psi+- = v_p +- B_p / sqrt(rho), taken at their feet from the van Leer     */
/* reconstructions of v_p and B_p along q.  U, W: the velocity and field     */
/* along q at the edge (U = 0 for the magnetic tension, Eq. 47).            */
static void mh_star(const mesh *m, const or_state *s, int i, int j, int k, int p, int q, double U, double W,
                    double rho, double dt, double *vs, double *bs)
{
    double sq = sqrt(rho);
    double cp = U - W / sq, cm = U + W / sq;
    const double *v = mh_v(s, p), *bf = mh_b(s, p);
    double vp = mh_recon(m, v, i, j, k, q, cp, dt), bp = mh_recon(m, bf, i, j, k, q, cp, dt);
    double vm = mh_recon(m, v, i, j, k, q, cm, dt), bm = mh_recon(m, bf, i, j, k, q, cm, dt);
    *vs = 0.5 * (vp + vm + (bp - bm) / sq);
    *bs = 0.5 * (bp + bm + sq * (vp - vm));
}

/* Cells 8a-8c.  EMF of orientation o, a = o + 1, b = o + 2 (mod 3), at the  */
/* edge at the lower a- and b-face of cell (i, j, k) (Eq. 45):              */
/*   e_o = (v_a* B_b^u + B_b* v_a^u - v_b* B_a^u - B_a* v_b^u) / 2,          */
/* with v_a^u, B_a^u the upwind estimates along b at the mean flow speed    */
/* along b of the edge's two b-faces, and v_a*, B_a* from the problem along */
/* b at C+- = v_b^u -+ B_b^u / sqrt(rho) (and a, b swapped).  Then the      */
/* resistive part: e_o -= eta (curl B)_o, by finite differences at the edge.*/
static double mh_emf_edge(const mesh *m, const or_params *p, const or_state *s, int o, int i, int j, int k,
                          double dt)
{
    int a = (o + 1) % 3, b = (o + 2) % 3;
    double *va = mh_v(s, a), *vb = mh_v(s, b), *ba = mh_b(s, a), *bb = mh_b(s, b);
    size_t c00 = IDX(m, i, j, k), ca = mh_nb(m, i, j, k, a, -1), cb = mh_nb(m, i, j, k, b, -1);
    double rho = mh_rho_edge(m, s->rho, i, j, k, a, b);
    double ub = 0.5 * (vb[c00] + vb[ca]);   /* mean speed along b at the edge (the b-faces at a and a-1) */
    double ua = 0.5 * (va[c00] + va[cb]);   /* mean speed along a (the a-faces at b and b-1) */
    double vau = mh_recon(m, va, i, j, k, b, ub, dt), bau = mh_recon(m, ba, i, j, k, b, ub, dt);
    double vbu = mh_recon(m, vb, i, j, k, a, ua, dt), bbu = mh_recon(m, bb, i, j, k, a, ua, dt);
    double vas, bas, vbs, bbs;
    mh_star(m, s, i, j, k, a, b, vbu, bbu, rho, dt, &vas, &bas);   /* (v_a*, B_a*): along b */
    mh_star(m, s, i, j, k, b, a, vau, bau, rho, dt, &vbs, &bbs);   /* (v_b*, B_b*): along a */
    double e = 0.5 * (vas * bbu + bbs * vau - vbs * bau - bas * vbu);
    if (p->eta > 0.0) {
        double cur = 0.0;   /* (curl B)_o = d_a B_b - d_b B_a */
        if (mh_has(m, a)) cur += (bb[c00] - bb[ca]) / mh_dc(m, a, a == 0 ? 1 : mh_pos(i, j, k, a));
        if (mh_has(m, b)) cur -= (ba[c00] - ba[cb]) / mh_dc(m, b, b == 0 ? 1 : mh_pos(i, j, k, b));
        e -= p->eta * cur;
    }
    return e;
}

/* Range of cell indices along d whose neighbours -2..+1 exist (the EMF     */
/* stencil): the whole of an absent direction (its single index 0) and the  */
/* whole periodic X.                                                         */
static void mh_edge_range(const mesh *m, int d, int *lo, int *hi)
{
    int n = d == 0 ? m->nx : (d == 1 ? m->nyt : m->nzt);
    if (d == 0 || !mh_has(m, d)) { *lo = 0; *hi = n; return; }
    *lo = 2; *hi = n - 1;
}

void or_mhd_emf(const or_params *p, const or_state *s, double dt, double *ex, double *ey, double *ez)
{
    mesh m;
    mesh_init(&m, p);
    double *E[3] = { ex, ey, ez };
    int jl, jh, kl, kh, il, ih;
    mh_edge_range(&m, 0, &il, &ih);
    mh_edge_range(&m, 1, &jl, &jh);
    mh_edge_range(&m, 2, &kl, &kh);
    for (int o = 0; o < 3; o++) {
        for (size_t q = 0; q < m.n; q++) E[o][q] = 0.0;
        PAR2
        for (int k = kl; k < kh; k++)
            for (int j = jl; j < jh; j++)
                for (int i = il; i < ih; i++)
                    E[o][IDX(&m, i, j, k)] = mh_emf_edge(&m, p, s, o, i, j, k, dt);
    }
    /* Walls (every non-periodic Y or Z boundary; reading M11): the EMFs on  */
    /* the edges that lie in a wall's plane vanish, the antisymmetric        */
    /* condition on the tangential EMF, so that the flux through the wall   */
    /* and the net flux out of every cell next to it are held.               */
    if (m.hasY && !m.pery)
        for (int w = 0; w < 2; w++) {
            int j = w == 0 ? m.j0 : m.j1;
            for (int k = 0; k < m.nzt + 1; k++)
                for (int i = 0; i < m.nx; i++) {
                    E[0][IDX(&m, i, j, k)] = 0.0;
                    E[2][IDX(&m, i, j, k)] = 0.0;
                }
        }
    if (m.hasZ && !m.perz)
        for (int w = 0; w < 2; w++) {
            int k = w == 0 ? m.k0 : m.k1;
            for (int j = 0; j < m.nyt + 1; j++)
                for (int i = 0; i < m.nx; i++) {
                    E[0][IDX(&m, i, j, k)] = 0.0;
                    E[1][IDX(&m, i, j, k)] = 0.0;
                }
        }
    mesh_free(&m);
}

/* Face ranges the update of component d covers: active cells along the    */
/* other directions; along d its interior faces (jf.., kf..), or the single */
/* index of an absent direction.                                             */
static void mh_face_range(const mesh *m, int d, int e, int *lo, int *hi)
{
    if (e == 0) { *lo = 0; *hi = m->nx; return; }
    if (!mh_has(m, e)) { *lo = 0; *hi = 1; return; }
    if (e == 1) { *lo = d == 1 ? m->jf : m->j0; *hi = m->j1; return; }
    *lo = d == 2 ? m->kf : m->k0; *hi = m->k1;
}

/* Cell 10: constrained transport (Eq. 39 with the circulation of e = v x B */
/* taken counterclockwise about each face's normal, Stokes' theorem: the    */
/* printed signs are those of e = B x v; reading M3).  On the Cartesian     */
/* mesh: dB_a/dt = d_b e_o - d_o e_b for the cyclic (a, b, o).              */
void or_mhd_ct(const or_params *p, or_state *s, const double *ex, const double *ey, const double *ez, double dt)
{
    mesh m;
    mesh_init(&m, p);
    const double *E[3] = { ex, ey, ez };
    for (int a = 0; a < 3; a++) {
        int b = (a + 1) % 3, o = (a + 2) % 3;   /* dB_a/dt = d_b e_o - d_o e_b */
        double *B = mh_b(s, a);
        int il, ih, jl, jh, kl, kh;
        mh_face_range(&m, a, 0, &il, &ih);
        mh_face_range(&m, a, 1, &jl, &jh);
        mh_face_range(&m, a, 2, &kl, &kh);
        double *nb = dup(B, m.n);
        PAR2
        for (int k = kl; k < kh; k++)
            for (int j = jl; j < jh; j++)
                for (int i = il; i < ih; i++) {
                    size_t c = IDX(&m, i, j, k);
                    double d = 0.0;
                    if (mh_has(&m, b))
                        d += (E[o][mh_nb(&m, i, j, k, b, 1)] - E[o][c]) / mh_width(&m, b, mh_pos(i, j, k, b));
                    if (mh_has(&m, o))
                        d -= (E[b][mh_nb(&m, i, j, k, o, 1)] - E[b][c]) / mh_width(&m, o, mh_pos(i, j, k, o));
                    nb[c] = B[c] + dt * d;
                }
        memcpy(B, nb, sizeof(double) * m.n);
        free(nb);
    }
    periodic_field(&m, s);
    mesh_free(&m);
}

/* Cell 11: orbital advection of the field (Sec. 3.6).  The field's share   */
/* of the orbital motion v0 x (uniform along each ring) is the induction    */
/* equation dB/dt = curl(v0 x B) (Eq. 50), whose EMF has the components     */
/* e_z = v0 B_y and e_y = -v0 B_z.  Over the step each edge takes the        */
/* upstream average of that EMF along the arc v0 dt that reaches it (Eq. 54):*/
/*   Ebar_z(i-1/2, j-1/2, k) = (1/dt) int_{x - v0 dt}^{x} B_y(x') dx',        */
/*   Ebar_y(i-1/2, j, k-1/2) = -(1/dt) int_{x - v0 dt}^{x} B_z(x') dx',       */
/* x the edge's azimuth, v0 the two-point mean of the ring velocities on     */
/* both sides of the face that carries B_y (B_z), or the ring's own along an */
/* absent direction.  With X = v0 dt / dX = N + xi (N = E(X), the nearest    */
/* integer of Sec. 3.4.1), the integral in units of dX is the sum of the N   */
/* whole cells upstream (with the opposite sign for N < 0) plus xi times     */
/* the PPA value of Sec. 3.4.1 on the face N cells upstream: the parabolic  */
/* interpolation of the residual arc.  For a uniform v0 and xi = 0 the       */
/* constrained transport of these EMFs is the shift B_i <- B_{i-N} (Eqs.     */
/* 60, 64) up to the round-off of the sums.  Ebar_x = 0.  Edges in a wall's  */
/* plane (non-periodic Y or Z) get zero, as in the residual step (M11).     */
/* ex, ey, ez are written on every edge of the arrays (zero where no arc).  */
static void mhd_fargo_ring(int nx, const double *ring, double X, double *out)
{
    long long N = or_nearest_int(X);
    double xs = X - (double)N;
    double *fs = zalloc(nx);
    if (xs != 0.0) or_ppa_faces(nx, ring, xs, fs);
    for (int i = 0; i < nx; i++) {
        double w = 0.0;
        if (N > 0)
            for (long long q = 1; q <= N; q++) w += ring[(int)((((long long)i - q) % nx + nx) % nx)];
        else
            for (long long q = 0; q < -N; q++) w -= ring[(int)((((long long)i + q) % nx + nx) % nx)];
        int f = (int)((((long long)i - N) % nx + nx) % nx);
        out[i] = w + xs * fs[f];
    }
    free(fs);
}

void or_mhd_fargo_emf(const or_params *p, const or_state *s, const double *v0all, double dt, double *ex,
                      double *ey, double *ez)
{
    mesh m;
    mesh_init(&m, p);
    for (size_t q = 0; q < m.n; q++) ex[q] = ey[q] = ez[q] = 0.0;
    if (m.hasX && p->fargo) {
        int nx = m.nx;
        double dX = m.dx;
        double *ring = zalloc(nx), *out = zalloc(nx);
        /* Ebar_z from B_y: edge rows j0..j1 (Y faces), active planes */
        int jl = m.hasY ? m.j0 : 0, jh = m.hasY ? m.j1 + 1 : 1;
        int kl = m.hasZ ? m.k0 : 0, kh = m.hasZ ? m.k1 : 1;
        for (int k = kl; k < kh; k++)
            for (int j = jl; j < jh; j++) {
                if (m.hasY && !m.pery && (j == m.j0 || j == m.j1)) continue;   /* wall */
                double v0f = m.hasY ? 0.5 * (v0all[(size_t)k * m.nyt + j - 1] + v0all[(size_t)k * m.nyt + j])
                                    : v0all[(size_t)k * m.nyt + j];
                for (int i = 0; i < nx; i++) ring[i] = s->by[IDX(&m, i, j, k)];
                mhd_fargo_ring(nx, ring, v0f * dt / dX, out);
                for (int i = 0; i < nx; i++) ez[IDX(&m, i, j, k)] = dX / dt * out[i];
            }
        /* Ebar_y from B_z: active rows, edge planes k0..k1 (Z faces) */
        jl = m.hasY ? m.j0 : 0; jh = m.hasY ? m.j1 : 1;
        kl = m.hasZ ? m.k0 : 0; kh = m.hasZ ? m.k1 + 1 : 1;
        for (int k = kl; k < kh; k++)
            for (int j = jl; j < jh; j++) {
                if (m.hasZ && !m.perz && (k == m.k0 || k == m.k1)) continue;   /* wall */
                double v0f = m.hasZ ? 0.5 * (v0all[(size_t)(k - 1) * m.nyt + j] + v0all[(size_t)k * m.nyt + j])
                                    : v0all[(size_t)k * m.nyt + j];
                for (int i = 0; i < nx; i++) ring[i] = s->bz[IDX(&m, i, j, k)];
                mhd_fargo_ring(nx, ring, v0f * dt / dX, out);
                for (int i = 0; i < nx; i++) ey[IDX(&m, i, j, k)] = -dX / dt * out[i];
            }
        free(ring); free(out);
    }
    mesh_free(&m);
}

double or_mhd_divb(const or_params *p, const or_state *s, int i, int j, int k)
{
    mesh m;
    mesh_init(&m, p);
    double w[3] = { m.dx, m.dy[j], m.dz[k] }, d = 0.0;
    for (int a = 0; a < 3; a++) {
        if (!mh_has(&m, a)) continue;
        const double *B = mh_b(s, a);
        double area = 1.0;
        for (int e = 0; e < 3; e++)
            if (e != a) area *= w[e];
        d += (B[mh_nb(&m, i, j, k, a, 1)] - B[IDX(&m, i, j, k)]) * area;
    }
    mesh_free(&m);
    return d;
}

/* Cell 8d: the magnetic tension (Eq. 47 and its permutations), for every   */
/* interior face of v_a:                                                     */
/*   dv_a = dt 2/(rho + rho_{-a}) sum_b Bbar_b (B_a*(b+1/2) - B_a*(b-1/2)) / D_b */
/* over the other present directions b; Bbar_b the mean of the four b-faces */
/* around the a-face; B_a* at the edges from the problem along b with no    */
/* flow speed (U = 0, W the mean of the edge's two b-faces: reading M4).   */
/* Jacobi: every component from the velocities on entry.                    */
static double mh_tension_star(const mesh *m, const or_state *s, int i, int j, int k, int a, int b, double dt)
{
    const double *bb = mh_b(s, b);
    double rho = mh_rho_edge(m, s->rho, i, j, k, a, b);
    double W = 0.5 * (bb[IDX(m, i, j, k)] + bb[mh_nb(m, i, j, k, a, -1)]);
    double vs, bs;
    mh_star(m, s, i, j, k, a, b, 0.0, W, rho, dt, &vs, &bs);
    return bs;
}

/* The tension's velocity update of s, its star values from the state chr  */
/* (chr = s in the plain step; with orbital advection chr carries the       */
/* residual velocity, reading M13).                                          */
void or_mhd_tension(const or_params *p, or_state *s, double dt) { mhd_tension_from(p, s, s, dt); }

static void mhd_tension_from(const or_params *p, const or_state *chr, or_state *s, double dt)
{
    if (!p->mhd || p->mhd_passive) return;
    mesh m;
    mesh_init(&m, p);
    double *nv[3] = { NULL, NULL, NULL };
    for (int a = 0; a < 3; a++) {
        if (!mh_has(&m, a)) continue;
        double *v = mh_v(s, a);
        nv[a] = dup(v, m.n);
        int il, ih, jl, jh, kl, kh;
        mh_face_range(&m, a, 0, &il, &ih);
        mh_face_range(&m, a, 1, &jl, &jh);
        mh_face_range(&m, a, 2, &kl, &kh);
        PAR2
        for (int k = kl; k < kh; k++)
            for (int j = jl; j < jh; j++)
                for (int i = il; i < ih; i++) {
                    size_t c = IDX(&m, i, j, k), cm = mh_nb(&m, i, j, k, a, -1);
                    double f = 0.0;
                    for (int b = 0; b < 3; b++) {
                        if (b == a || !mh_has(&m, b)) continue;
                        const double *bb = mh_b(s, b);
                        int ia = a == 0 ? ((i - 1) % m.nx + m.nx) % m.nx : i, ja = a == 1 ? j - 1 : j,
                            ka = a == 2 ? k - 1 : k;
                        double bbar = 0.25 * (bb[c] + bb[mh_nb(&m, i, j, k, b, 1)] + bb[cm] +
                                              bb[mh_nb(&m, ia, ja, ka, b, 1)]);
                        int ib = b == 0 ? (i + 1) % m.nx : i, jb = b == 1 ? j + 1 : j, kb = b == 2 ? k + 1 : k;
                        double up = mh_tension_star(&m, chr, ib, jb, kb, a, b, dt);
                        double lo = mh_tension_star(&m, chr, i, j, k, a, b, dt);
                        f += bbar * (up - lo) / mh_width(&m, b, mh_pos(i, j, k, b));
                    }
                    nv[a][c] = v[c] + dt * 2.0 / (s->rho[c] + s->rho[cm]) * f;
                }
    }
    for (int a = 0; a < 3; a++)
        if (nv[a]) {
            memcpy(mh_v(s, a), nv[a], sizeof(double) * m.n);
            free(nv[a]);
        }
    periodic_state(&m, s, 1, 0);
    mesh_free(&m);
}

/* Cell 7a, the magnetic part: the gradient of the magnetic pressure of the */
/* transverse field, -(1/rho) d_a (B_b^2 + B_c^2)/2, with zone-centred two-  */
/* point averages of B_b, B_c and the two-point face density, as the        */
/* thermal pressure gradient (Sec. 3.5; Eq. 20).                            */
static double mh_pmag(const mesh *m, const or_state *s, int i, int j, int k, int a)
{
    double pb = 0.0;
    for (int b = 0; b < 3; b++) {
        if (b == a) continue;
        const double *B = mh_b(s, b);
        double bc = 0.5 * (B[IDX(m, i, j, k)] + B[mh_nb(m, i, j, k, b, 1)]);
        pb += 0.5 * bc * bc;
    }
    return pb;
}

void or_mhd_pressure(const or_params *p, or_state *s, double dt)
{
    if (!p->mhd || p->mhd_passive) return;
    mesh m;
    mesh_init(&m, p);
    double *nv[3] = { NULL, NULL, NULL };
    for (int a = 0; a < 3; a++) {
        if (!mh_has(&m, a)) continue;
        double *v = mh_v(s, a);
        nv[a] = dup(v, m.n);
        int il, ih, jl, jh, kl, kh;
        mh_face_range(&m, a, 0, &il, &ih);
        mh_face_range(&m, a, 1, &jl, &jh);
        mh_face_range(&m, a, 2, &kl, &kh);
        PAR2
        for (int k = kl; k < kh; k++)
            for (int j = jl; j < jh; j++)
                for (int i = il; i < ih; i++) {
                    size_t c = IDX(&m, i, j, k), cm = mh_nb(&m, i, j, k, a, -1);
                    int ia = a == 0 ? ((i - 1) % m.nx + m.nx) % m.nx : i, ja = a == 1 ? j - 1 : j,
                        ka = a == 2 ? k - 1 : k;
                    double g = (mh_pmag(&m, s, i, j, k, a) - mh_pmag(&m, s, ia, ja, ka, a)) /
                               mh_dc(&m, a, a == 0 ? 1 : mh_pos(i, j, k, a));
                    nv[a][c] = v[c] - dt * 2.0 * g / (s->rho[c] + s->rho[cm]);
                }
    }
    for (int a = 0; a < 3; a++)
        if (nv[a]) {
            memcpy(mh_v(s, a), nv[a], sizeof(double) * m.n);
            free(nv[a]);
        }
    periodic_state(&m, s, 1, 0);
    mesh_free(&m);
}
