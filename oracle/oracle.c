/*
 * oracle.c -- plain, slow FP64 restatement of the two-range
 * pseudopotential lattice Boltzmann method for binary mixtures with tunable
 * viscosity ratio (Fei, Scagliarini, Montessori, Lauricella, Succi, Luo,
 * "Mesoscopic model for soft flowing systems with tunable viscosity ratio",
 * arXiv:1806.06943).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Equation numbers are the paper's printed numbers, counted in order of
 * appearance: (1) evolution, (2) equilibrium, (3) common velocity u^eq,
 * (4) velocity-shift forcing, (5) Guo forcing, (6) moments, (7) barycentric
 * velocity, (8) competing intra-species force, (9) inter-species repulsion,
 * (11) bulk equation of state, (19) layered Poiseuille profile.
 *
 * Build: cc -O2 -ffp-contract=off -std=c99 -fPIC -shared [-fopenmp] oracle.c -lm
 * (no fused multiply-add, libm exp), so every operation below rounds once,
 * in the order it is written.  With OpenMP the row loops of a time step run
 * on several threads; no sum crosses rows, so the results do not depend on
 * the thread count.
 *
 * Readings where the paper is silent or garbled (each listed with its reason
 * in the design notes):
 *  - Eq. (2) is printed without the 1/2 on the quadratic term; the standard
 *    second-order equilibrium w rho [1 + e.u/cs2 + (e.u)^2/(2 cs4) - u.u/(2 cs2)]
 *    is used (the printed form breaks the second moment rho cs2 I + rho u u).
 *  - The component momentum entering Eq. (3) is Eq. (6), i.e. includes F/2.
 *  - The body force acts on both species as F^b_k = rho_k g (Sec. III A: the
 *    body force "acts on both components").
 *  - Wall interaction for the stencil: ghost rows y=-1,-2 and y=ny,ny+1 are
 *    either mirrored from the fluid (neutral walls) or held at fixed ghost
 *    densities (non-wetting walls, Sec. III D).
 *  - The second-belt sum of Eq. (8) runs over all 25 vectors of D2Q25,
 *    nearest belt included, as printed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---- lattice tables (Sec. II A, Fig. 1; Sec. II B after Eq. (8)) ---------- */

/* D2Q9 velocities: rest, 4 axis, 4 diagonal. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* w(|e|^2): w(0)=4/9, w(1)=1/9, w(2)=1/36 (Sec. II A, after Eq. (2)). */
static double w_of(int e2)
{
    if (e2 == 0) return 4.0 / 9.0;
    if (e2 == 1) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* D2Q25 weights p(|e|^2) (Sec. II B, after Eq. (8)). */
static double p_of(int e2)
{
    switch (e2) {
    case 0: return 247.0 / 420.0;
    case 1: return 4.0 / 63.0;
    case 2: return 4.0 / 135.0;
    case 4: return 1.0 / 180.0;
    case 5: return 2.0 / 945.0;
    case 8: return 1.0 / 15120.0;
    default: return 0.0;
    }
}

/* D2Q25 vectors in raster order: dy = -2..2 (outer), dx = -2..2 (inner). */
static int JX(int j) { return j % 5 - 2; }
static int JY(int j) { return j / 5 - 2; }

/* ---- simulation state ------------------------------------------------------ */

typedef struct orc_params {
    int32_t nx, ny;
    double tau[2];
    double G_AB, G1, G2;
    double g[2];
    int32_t walls;      /* 0: periodic in y; 1: half-way bounce-back at y=-1/2 and y=ny-1/2 */
    int32_t wall_mode;  /* 0: mirrored ghost densities; 1: fixed ghost densities */
    double wall_rho[2]; /* ghost densities for wall_mode 1 */
    int32_t forcing;    /* 0: Guo forcing, Eqs. (5)-(6), the present model;
                           1: velocity-shift forcing, Eq. (4), the original model */
    int32_t pad;
} orc_params;

typedef struct orc_sim {
    orc_params p;
    long t;
    double *f, *fn;     /* [2][9][ny][nx] */
    double *rho;        /* [2][ny][nx] */
    double *rho_ext;    /* [2][ny+4][nx]: rows -2..ny+1 */
    double *psi_ext;    /* [2][ny+4][nx] */
    double *force;      /* [2][2][ny][nx]: species, component */
    int *xw;            /* periodic x index for x = -2..nx+1, stored at xw[x + 2] */
    int *yw;            /* periodic y index for y = -1..ny, stored at yw[y + 1] */
} orc_sim;

#define FIDX(s, k, i, x, y) ((((size_t)(k) * 9 + (i)) * (s)->p.ny + (y)) * (s)->p.nx + (x))
#define RIDX(s, k, x, y) (((size_t)(k) * (s)->p.ny + (y)) * (s)->p.nx + (x))
#define EIDX(s, k, x, y) (((size_t)(k) * ((s)->p.ny + 4) + ((y) + 2)) * (s)->p.nx + (x))
#define FOIDX(s, k, c, x, y) ((((size_t)(k) * 2 + (c)) * (s)->p.ny + (y)) * (s)->p.nx + (x))

static int wrap(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
#define XW(s, x) ((s)->xw[(x) + 2])
#define YW(s, y) ((s)->yw[(y) + 1])

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->f); free(s->fn); free(s->rho); free(s->rho_ext); free(s->psi_ext); free(s->force);
    free(s->xw); free(s->yw);
    free(s);
}

orc_sim *orc_create(const orc_params *p)
{
    if (p->nx < 5 || p->ny < 5 || !(p->tau[0] > 0.5) || !(p->tau[1] > 0.5)) return NULL;
    if (p->forcing != 0 && p->forcing != 1) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    size_t n = (size_t)p->nx * p->ny;
    size_t ne = (size_t)p->nx * (p->ny + 4);
    s->f = (double *)calloc(18 * n, sizeof(double));
    s->fn = (double *)calloc(18 * n, sizeof(double));
    s->rho = (double *)calloc(2 * n, sizeof(double));
    s->rho_ext = (double *)calloc(2 * ne, sizeof(double));
    s->psi_ext = (double *)calloc(2 * ne, sizeof(double));
    s->force = (double *)calloc(4 * n, sizeof(double));
    s->xw = (int *)calloc((size_t)p->nx + 4, sizeof(int));
    s->yw = (int *)calloc((size_t)p->ny + 2, sizeof(int));
    if (!s->f || !s->fn || !s->rho || !s->rho_ext || !s->psi_ext || !s->force || !s->xw || !s->yw) {
        orc_destroy(s);
        return NULL;
    }
    for (int x = -2; x < p->nx + 2; ++x) s->xw[x + 2] = wrap(x, p->nx);
    for (int y = -1; y < p->ny + 1; ++y) s->yw[y + 1] = wrap(y, p->ny);
    return s;
}

/* ---- model pieces, one lattice site at a time ------------------------------ */

/* Pseudopotential psi(rho) = rho0 (1 - exp(-rho/rho0)), rho0 = 1 (Sec. II B). */
double orc_psi(double rho)
{
    return 1.0 - exp(-rho);
}

/* Second-order equilibrium, Eq. (2) with the 1/2 restored, cs^2 = 1/3. */
void orc_equilibrium(double rho, double ux, double uy, double feq[9])
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = w_of(EX[i] * EX[i] + EY[i] * EY[i]) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Guo forcing term, Eq. (5): (1 - 1/(2 tau)) w_i [(e_i - u)/cs^2 + (e_i.u) e_i / cs^4] . F,
 * with u the common velocity u^eq. */
void orc_guo(double tau, double ux, double uy, double Fx, double Fy, double C[9])
{
    double omega = 1.0 / tau;
    for (int i = 0; i < 9; ++i) {
        double ex = EX[i], ey = EY[i];
        double eu = ex * ux + ey * uy;
        double cx = 3.0 * (ex - ux) + 9.0 * eu * ex;
        double cy = 3.0 * (ey - uy) + 9.0 * eu * ey;
        C[i] = (1.0 - 0.5 * omega) * w_of(EX[i] * EX[i] + EY[i] * EY[i]) * (cx * Fx + cy * Fy);
    }
}

/* Copies of the lattice tables, for the table tests. */
void orc_tables(double w[9], int32_t ex[9], int32_t ey[9], double p[25], int32_t jx[25], int32_t jy[25])
{
    for (int i = 0; i < 9; ++i) {
        w[i] = w_of(EX[i] * EX[i] + EY[i] * EY[i]);
        ex[i] = EX[i];
        ey[i] = EY[i];
    }
    for (int j = 0; j < 25; ++j) {
        p[j] = p_of(JX(j) * JX(j) + JY(j) * JY(j));
        jx[j] = JX(j);
        jy[j] = JY(j);
    }
}

/* ---- whole-lattice passes ---------------------------------------------------- */

/* rho_k = sum_i f_k,i, Eq. (6). */
static void density(orc_sim *s)
{
    for (int k = 0; k < 2; ++k)
#pragma omp parallel for schedule(static)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                double r = 0.0;
                for (int i = 0; i < 9; ++i) r += s->f[FIDX(s, k, i, x, y)];
                s->rho[RIDX(s, k, x, y)] = r;
            }
}

/* Densities seen by the interaction stencils, rows -2..ny+1: periodic copies,
 * or wall ghosts (mirror: row -1 <- 0, -2 <- 1 and symmetrically at the top;
 * fixed: the prescribed wall densities). */
static void fill_extended(orc_sim *s)
{
    int nx = s->p.nx, ny = s->p.ny;
    for (int k = 0; k < 2; ++k)
#pragma omp parallel for schedule(static)
        for (int y = -2; y < ny + 2; ++y)
            for (int x = 0; x < nx; ++x) {
                double r;
                if (y >= 0 && y < ny) {
                    r = s->rho[RIDX(s, k, x, y)];
                } else if (!s->p.walls) {
                    r = s->rho[RIDX(s, k, x, wrap(y, ny))];
                } else if (s->p.wall_mode == 1) {
                    r = s->p.wall_rho[k];
                } else {
                    int ys = y < 0 ? -1 - y : 2 * ny - 1 - y;
                    r = s->rho[RIDX(s, k, x, ys)];
                }
                s->rho_ext[EIDX(s, k, x, y)] = r;
                s->psi_ext[EIDX(s, k, x, y)] = orc_psi(r);
            }
}

/* Total force on species k at (x, y): F^c (Eq. 8) + F^r (Eq. 9) + F^b. */
static void force_at(const orc_sim *s, int k, int x, int y, double *Fx, double *Fy)
{
    int kb = 1 - k;
    double psi = s->psi_ext[EIDX(s, k, x, y)];
    double rho = s->rho_ext[EIDX(s, k, x, y)];
    /* short range, D2Q9 weights w (Eq. 8, first sum) */
    double s1x = 0.0, s1y = 0.0;
    for (int i = 0; i < 9; ++i) {
        double wp = w_of(EX[i] * EX[i] + EY[i] * EY[i]) * s->psi_ext[EIDX(s, k, XW(s, x + EX[i]), y + EY[i])];
        s1x += wp * EX[i];
        s1y += wp * EY[i];
    }
    /* mid range, D2Q25 weights p (Eq. 8, second sum) */
    double s2x = 0.0, s2y = 0.0;
    for (int j = 0; j < 25; ++j) {
        int dx = JX(j), dy = JY(j);
        double pp = p_of(dx * dx + dy * dy) * s->psi_ext[EIDX(s, k, XW(s, x + dx), y + dy)];
        s2x += pp * dx;
        s2y += pp * dy;
    }
    /* inter-species repulsion on densities of the other species (Eq. 9) */
    double s3x = 0.0, s3y = 0.0;
    for (int i = 0; i < 9; ++i) {
        double wr = w_of(EX[i] * EX[i] + EY[i] * EY[i]) * s->rho_ext[EIDX(s, kb, XW(s, x + EX[i]), y + EY[i])];
        s3x += wr * EX[i];
        s3y += wr * EY[i];
    }
    const double G1 = s->p.G1, G2 = s->p.G2, GAB = s->p.G_AB;
    *Fx = -G1 * psi * s1x - G2 * psi * s2x - GAB * rho * s3x + rho * s->p.g[0];
    *Fy = -G1 * psi * s1y - G2 * psi * s2y - GAB * rho * s3y + rho * s->p.g[1];
}

static void forces(orc_sim *s)
{
    density(s);
    fill_extended(s);
    for (int k = 0; k < 2; ++k)
#pragma omp parallel for schedule(static)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x)
                force_at(s, k, x, y, &s->force[FOIDX(s, k, 0, x, y)], &s->force[FOIDX(s, k, 1, x, y)]);
}

/* Component momentum with half force, Eq. (6); common velocity, Eq. (3). */
static void site_moments(const orc_sim *s, int x, int y, double rho[2], double m[2][2], double ueq[2])
{
    for (int k = 0; k < 2; ++k) {
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            double fi = s->f[FIDX(s, k, i, x, y)];
            jx += fi * EX[i];
            jy += fi * EY[i];
        }
        rho[k] = s->rho[RIDX(s, k, x, y)];
        m[k][0] = jx + 0.5 * s->force[FOIDX(s, k, 0, x, y)];
        m[k][1] = jy + 0.5 * s->force[FOIDX(s, k, 1, x, y)];
    }
    double om0 = 1.0 / s->p.tau[0], om1 = 1.0 / s->p.tau[1];
    double den = om0 * rho[0] + om1 * rho[1];
    ueq[0] = (om0 * m[0][0] + om1 * m[1][0]) / den;
    ueq[1] = (om0 * m[0][1] + om1 * m[1][1]) / den;
}

/* Velocity-shift forcing term of the original model, Eq. (4):
 * C^SC_i = (1/tau) [f^eq_i(rho, u + F tau / rho) - f^eq_i(rho, u)], u = u^eq. */
void orc_shift_forcing(double tau, double rho, double ux, double uy, double Fx, double Fy, double C[9])
{
    double omega = 1.0 / tau;
    double feq[9], feqs[9];
    orc_equilibrium(rho, ux, uy, feq);
    orc_equilibrium(rho, ux + tau * Fx / rho, uy + tau * Fy / rho, feqs);
    for (int i = 0; i < 9; ++i) C[i] = omega * (feqs[i] - feq[i]);
}

/* Common velocity of the original model: Eq. (3) with the component momenta
 * sum_i f e_i, without the force (Sec. II A, after Eq. 4). */
static void site_moments_shift(const orc_sim *s, int x, int y, double rho[2], double ueq[2])
{
    double m[2][2];
    for (int k = 0; k < 2; ++k) {
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            double fi = s->f[FIDX(s, k, i, x, y)];
            jx += fi * EX[i];
            jy += fi * EY[i];
        }
        rho[k] = s->rho[RIDX(s, k, x, y)];
        m[k][0] = jx;
        m[k][1] = jy;
    }
    double om0 = 1.0 / s->p.tau[0], om1 = 1.0 / s->p.tau[1];
    double den = om0 * rho[0] + om1 * rho[1];
    ueq[0] = (om0 * m[0][0] + om1 * m[1][0]) / den;
    ueq[1] = (om0 * m[0][1] + om1 * m[1][1]) / den;
}

/* One time step: collide with Guo forcing (Eqs. 1, 2, 5), or with the
 * velocity-shift forcing of the original model (Eqs. 1, 2, 4), then stream;
 * a population that would cross a wall returns to its own node reversed
 * (half-way bounce-back, Sec. III A). */
static void step_once(orc_sim *s)
{
    int nx = s->p.nx, ny = s->p.ny;
    forces(s);
    /* every (species, direction, node) of fn is written by exactly one site */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double rho[2], m[2][2], ueq[2];
            if (s->p.forcing == 1) site_moments_shift(s, x, y, rho, ueq);
            else site_moments(s, x, y, rho, m, ueq);
            for (int k = 0; k < 2; ++k) {
                double omega = 1.0 / s->p.tau[k];
                double feq[9], C[9];
                double Fx = s->force[FOIDX(s, k, 0, x, y)], Fy = s->force[FOIDX(s, k, 1, x, y)];
                orc_equilibrium(rho[k], ueq[0], ueq[1], feq);
                if (s->p.forcing == 1) orc_shift_forcing(s->p.tau[k], rho[k], ueq[0], ueq[1], Fx, Fy, C);
                else orc_guo(s->p.tau[k], ueq[0], ueq[1], Fx, Fy, C);
                for (int i = 0; i < 9; ++i) {
                    double fi = s->f[FIDX(s, k, i, x, y)];
                    double fpost = fi - omega * (fi - feq[i]) + C[i];
                    int xd = x + EX[i], yd = y + EY[i];
                    if (s->p.walls && (yd < 0 || yd >= ny)) {
                        s->fn[FIDX(s, k, OPP[i], x, y)] = fpost;
                    } else {
                        s->fn[FIDX(s, k, i, XW(s, xd), YW(s, yd))] = fpost;
                    }
                }
            }
        }
    double *tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
    s->t += 1;
}

/* Threads of the row loops (OpenMP, when the library was built with it):
 * each node's arithmetic is the same whatever thread runs it, so the results
 * are bitwise those of one thread.  Returns the count in use (1 without
 * OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void orc_step(orc_sim *s, long n)
{
    for (long t = 0; t < n; ++t) step_once(s);
}

long orc_time(const orc_sim *s) { return s->t; }

/* f = f^eq(rho_k, u) from given densities [2][ny][nx] and an optional common
 * initial velocity [2][ny][nx] (component-major: ux field then uy field). */
void orc_set_fields(orc_sim *s, const double *rho, const double *u)
{
    int nx = s->p.nx, ny = s->p.ny;
    size_t n = (size_t)nx * ny;
    for (int k = 0; k < 2; ++k)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = (size_t)y * nx + x;
                double ux = u ? u[c] : 0.0, uy = u ? u[n + c] : 0.0;
                double feq[9];
                orc_equilibrium(rho[k * n + c], ux, uy, feq);
                for (int i = 0; i < 9; ++i) s->f[FIDX(s, k, i, x, y)] = feq[i];
            }
    s->t = 0;
}

void orc_get_f(const orc_sim *s, double *f)
{
    memcpy(f, s->f, sizeof(double) * 18 * (size_t)s->p.nx * s->p.ny);
}

void orc_set_f(orc_sim *s, const double *f, long t)
{
    memcpy(s->f, f, sizeof(double) * 18 * (size_t)s->p.nx * s->p.ny);
    s->t = t;
}

/* Diagnostic fields at the current time, from the pre-collision populations
 * and the forces recomputed from them.  Any output pointer may be NULL.
 *   rho  [2][ny][nx]      component densities (Eq. 6)
 *   mom  [2][2][ny][nx]   component momenta with half force (Eq. 6)
 *   force[2][2][ny][nx]   total force per component
 *   ueq  [2][ny][nx]      common velocity (Eq. 3)
 *   ubar [2][ny][nx]      barycentric velocity (Eq. 7) */
void orc_fields(orc_sim *s, double *rho, double *mom, double *force, double *ueq, double *ubar)
{
    int nx = s->p.nx, ny = s->p.ny;
    size_t n = (size_t)nx * ny;
    forces(s);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double r[2], m[2][2], ue[2];
            site_moments(s, x, y, r, m, ue);
            for (int k = 0; k < 2; ++k) {
                if (rho) rho[k * n + c] = r[k];
                for (int a = 0; a < 2; ++a) {
                    if (mom) mom[(k * 2 + a) * n + c] = m[k][a];
                    if (force) force[(k * 2 + a) * n + c] = s->force[FOIDX(s, k, a, x, y)];
                }
            }
            if (ueq) { ueq[c] = ue[0]; ueq[n + c] = ue[1]; }
            if (ubar) {
                double rt = r[0] + r[1];
                ubar[c] = (m[0][0] + m[1][0]) / rt;
                ubar[n + c] = (m[0][1] + m[1][1]) / rt;
            }
        }
}

/* Bulk equation of state, Eq. (11), with G_k,1 = G1, G_k,2 = G2 for both species. */
double orc_bulk_pressure(const orc_params *p, double rhoA, double rhoB)
{
    double psiA = orc_psi(rhoA), psiB = orc_psi(rhoB);
    double Gs = p->G1 + p->G2;
    return (rhoA + 0.5 * Gs * psiA * psiA) / 3.0 + (rhoB + 0.5 * Gs * psiB * psiB) / 3.0
         + p->G_AB * rhoA * rhoB / 3.0;
}

/* Observables at the current time.
 * out[0..1]  mass of A, B
 * out[2..5]  total momentum of A (x, y), B (x, y), half force included
 * out[6]     Q = (1/nx) sum_{x,y} ubar_x   (channel flux, Sec. III D)
 * out[7]     mu_r = Q0/Q with Q0 = g_x (H^3 + H/2) / (12 nu_B), H = ny, walls only
 * out[8]     dp = <p_b>_in - <p_b>_out around the probe (Laplace test)
 * out[9]     R_eff, equimolar radius of species A around the probe
 * out[10]    max |ubar|
 * out[11]    1 if every density and velocity is finite, else 0
 * The probe is the disk centre (cx, cy) and nominal radius R: inside means
 * r < R/2, outside means r > R + 6 (minimum-image distances on periodic axes).
 * With R <= 0, out[8] and out[9] are NaN. */
void orc_observables(orc_sim *s, double cx, double cy, double R, double out[12])
{
    int nx = s->p.nx, ny = s->p.ny;
    size_t n = (size_t)nx * ny;
    double *rho = (double *)malloc(sizeof(double) * 2 * n);
    double *mom = (double *)malloc(sizeof(double) * 4 * n);
    double *ub = (double *)malloc(sizeof(double) * 2 * n);
    orc_fields(s, rho, mom, NULL, NULL, ub);
    double mass[2] = {0.0, 0.0}, mt[4] = {0.0, 0.0, 0.0, 0.0}, sumux = 0.0, umax = 0.0;
    double pin = 0.0, pout = 0.0, ain = 0.0, aout = 0.0, nin = 0.0, nout = 0.0;
    int finite = 1;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            for (int k = 0; k < 2; ++k) {
                mass[k] += rho[k * n + c];
                mt[2 * k] += mom[(2 * k) * n + c];
                mt[2 * k + 1] += mom[(2 * k + 1) * n + c];
            }
            double ux = ub[c], uy = ub[n + c];
            if (!isfinite(rho[c]) || !isfinite(rho[n + c]) || !isfinite(ux) || !isfinite(uy)) finite = 0;
            sumux += ux;
            double um = sqrt(ux * ux + uy * uy);
            if (um > umax) umax = um;
            if (R > 0.0) {
                double dx = fabs(x - cx), dy = fabs(y - cy);
                if (dx > 0.5 * nx) dx = nx - dx;
                if (!s->p.walls && dy > 0.5 * ny) dy = ny - dy;
                double r = sqrt(dx * dx + dy * dy);
                double pb = orc_bulk_pressure(&s->p, rho[c], rho[n + c]);
                if (r < 0.5 * R) { pin += pb; ain += rho[c]; nin += 1.0; }
                if (r > R + 6.0) { pout += pb; aout += rho[c]; nout += 1.0; }
            }
        }
    out[0] = mass[0];
    out[1] = mass[1];
    for (int a = 0; a < 4; ++a) out[2 + a] = mt[a];
    out[6] = sumux / nx;
    if (s->p.walls && s->p.g[0] != 0.0) {
        double H = ny, nuB = (s->p.tau[1] - 0.5) / 3.0;
        double Q0 = s->p.g[0] * (H * H * H + 0.5 * H) / (12.0 * nuB);
        out[7] = Q0 / out[6];
    } else {
        out[7] = NAN;
    }
    if (R > 0.0 && nin > 0.0 && nout > 0.0) {
        double rin = ain / nin, rout = aout / nout;
        out[8] = pin / nin - pout / nout;
        out[9] = sqrt((mass[0] - rout * (double)n) / (ORC_PI * (rin - rout)));
    } else {
        out[8] = NAN;
        out[9] = NAN;
    }
    out[10] = umax;
    out[11] = finite ? 1.0 : 0.0;
    free(rho); free(mom); free(ub);
}

/* Pressure tensor at the current time, per node (Sec. II B, Eq. 10):
 *   P_ab = P^kin_ab + P^int_ab
 *   P^kin_ab = sum_k sum_i f_k,i e_ia e_ib                          Eq. (13)
 *   P^int_ab = 1/2 sum_k [ G1 psi_k(x) sum_i w_i psi_k(x + e_i) e_ia e_ib
 *                        + G2 psi_k(x) sum_j p_j psi_k(x + e_j) e_ja e_jb
 *                        + G_AB rho_k(x) sum_i w_i rho_kbar(x + e_i) e_ia e_ib ]
 * The paper defines P^int only through its divergence, Eq. (12), and refers
 * elsewhere for the lattice form.  This is the form that gives each pair of
 * interacting nodes' contribution half to each node (the force of Eqs. 8-9
 * is a sum of such pair forces): in a uniform state it is the bulk pressure
 * of Eq. (11) minus sum_k rho_k cs^2, and summed over the nodes of a profile
 * it equals the sum of the momentum flux through the planes between the
 * nodes, whose differences are -sum_k F_k (Eq. 12), so the surface-tension
 * integral of Eq. (15) does not depend on how the pair contributions are
 * shared out.  Ghost densities and periodic copies are those of the forces.
 *   out [2][3][ny][nx]: kinetic then interaction part; components xx, yy, xy */
void orc_pressure_tensor(orc_sim *s, double *out)
{
    int nx = s->p.nx, ny = s->p.ny;
    size_t n = (size_t)nx * ny;
    forces(s);    /* densities, ghost rows and psi of the current populations */
    const double G1 = s->p.G1, G2 = s->p.G2, GAB = s->p.G_AB;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double kin[3] = {0.0, 0.0, 0.0}, pint[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < 2; ++k) {
                for (int i = 0; i < 9; ++i) {
                    double fi = s->f[FIDX(s, k, i, x, y)];
                    kin[0] += fi * EX[i] * EX[i];
                    kin[1] += fi * EY[i] * EY[i];
                    kin[2] += fi * EX[i] * EY[i];
                }
                int kb = 1 - k;
                double psi = s->psi_ext[EIDX(s, k, x, y)], rho = s->rho_ext[EIDX(s, k, x, y)];
                double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0}, s3[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < 9; ++i) {
                    double w = w_of(EX[i] * EX[i] + EY[i] * EY[i]);
                    double a = w * s->psi_ext[EIDX(s, k, XW(s, x + EX[i]), y + EY[i])];
                    double b = w * s->rho_ext[EIDX(s, kb, XW(s, x + EX[i]), y + EY[i])];
                    s1[0] += a * EX[i] * EX[i]; s1[1] += a * EY[i] * EY[i]; s1[2] += a * EX[i] * EY[i];
                    s3[0] += b * EX[i] * EX[i]; s3[1] += b * EY[i] * EY[i]; s3[2] += b * EX[i] * EY[i];
                }
                for (int j = 0; j < 25; ++j) {
                    int dx = JX(j), dy = JY(j);
                    double a = p_of(dx * dx + dy * dy) * s->psi_ext[EIDX(s, k, XW(s, x + dx), y + dy)];
                    s2[0] += a * dx * dx; s2[1] += a * dy * dy; s2[2] += a * dx * dy;
                }
                for (int c3 = 0; c3 < 3; ++c3)
                    pint[c3] += 0.5 * (G1 * psi * s1[c3] + G2 * psi * s2[c3] + GAB * rho * s3[c3]);
            }
            for (int c3 = 0; c3 < 3; ++c3) {
                out[(size_t)c3 * n + c] = kin[c3];
                out[(size_t)(3 + c3) * n + c] = pint[c3];
            }
        }
}

/* ===========================================================================
 * Three-dimensional extension (not in the paper, which is 2-D; Sec. II A).
 * The same method on D3Q19 for the fluid, with the short-range sums of
 * Eqs. (8), (9) over the D3Q19 neighbours (weights w: 1/3, 1/18, 1/36) and
 * the mid-range sum of Eq. (8) over the 5 x 5 x 5 neighbourhood with weights
 * q(|e|^2) isotropic to eighth order, normalised like the 2-D D2Q25 weights
 * (sum q = 1, sum q e_x^2 = 1/3) and sharing their fourth moment
 * (sum q e_x^4 = 4/7), the outermost shells |e|^2 = 9, 12 unweighted.
 * Projected onto one axis both stencils are the 2-D ones, so a profile that
 * varies along x only evolves exactly as in 2-D.  Periodic in x, y, z.
 * ======================================================================== */

static const int EX3[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY3[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ3[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

/* w(|e|^2) of D3Q19 */
static double w3_of(int e2)
{
    if (e2 == 0) return 1.0 / 3.0;
    if (e2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* q(|e|^2) of the 5 x 5 x 5 mid-range stencil */
static double q3_of(int e2)
{
    switch (e2) {
    case 0: return 47.0 / 90.0;
    case 1: return 4.0 / 135.0;
    case 2: return 1.0 / 63.0;
    case 3: return 2.0 / 315.0;
    case 4: return 5.0 / 1512.0;
    case 5: return 1.0 / 945.0;
    case 6: return 1.0 / 1890.0;
    case 8: return 1.0 / 15120.0;
    default: return 0.0;
    }
}

typedef struct orc3_params {
    int32_t nx, ny, nz, pad;
    double tau[2];
    double G_AB, G1, G2;
    double g[3];
} orc3_params;

typedef struct orc3_sim {
    orc3_params p;
    long t;
    double *f, *fn;     /* [2][19][nz][ny][nx] */
    double *rho, *psi;  /* [2][nz][ny][nx] */
    double *force;      /* [2][3][nz][ny][nx] */
} orc3_sim;

#define N3(s) ((size_t)(s)->p.nx * (s)->p.ny * (s)->p.nz)
#define C3(s, x, y, z) ((((size_t)(z)) * (s)->p.ny + (y)) * (s)->p.nx + (x))

void orc3_destroy(orc3_sim *s)
{
    if (!s) return;
    free(s->f); free(s->fn); free(s->rho); free(s->psi); free(s->force);
    free(s);
}

orc3_sim *orc3_create(const orc3_params *p)
{
    if (p->nx < 5 || p->ny < 5 || p->nz < 5 || !(p->tau[0] > 0.5) || !(p->tau[1] > 0.5)) return NULL;
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return NULL;
    s->p = *p;
    size_t n = N3(s);
    s->f = (double *)calloc(38 * n, sizeof(double));
    s->fn = (double *)calloc(38 * n, sizeof(double));
    s->rho = (double *)calloc(2 * n, sizeof(double));
    s->psi = (double *)calloc(2 * n, sizeof(double));
    s->force = (double *)calloc(6 * n, sizeof(double));
    if (!s->f || !s->fn || !s->rho || !s->psi || !s->force) {
        orc3_destroy(s);
        return NULL;
    }
    return s;
}

/* Copies of the 3-D tables, for the table tests. */
void orc3_tables(double w[19], int32_t e[57], double q[13])
{
    for (int i = 0; i < 19; ++i) {
        w[i] = w3_of(EX3[i] * EX3[i] + EY3[i] * EY3[i] + EZ3[i] * EZ3[i]);
        e[3 * i] = EX3[i];
        e[3 * i + 1] = EY3[i];
        e[3 * i + 2] = EZ3[i];
    }
    for (int k = 0; k < 13; ++k) q[k] = q3_of(k);
}

/* Eq. (2) in 3-D, cs^2 = 1/3 */
static void eq3(double rho, const double u[3], double feq[19])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double eu = EX3[i] * u[0] + EY3[i] * u[1] + EZ3[i] * u[2];
        feq[i] = w3_of(EX3[i] * EX3[i] + EY3[i] * EY3[i] + EZ3[i] * EZ3[i]) * rho
               * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Eq. (5) in 3-D */
static void guo3(double tau, const double u[3], const double F[3], double C[19])
{
    double omega = 1.0 / tau;
    for (int i = 0; i < 19; ++i) {
        double e[3] = {EX3[i], EY3[i], EZ3[i]};
        double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (3.0 * (e[a] - u[a]) + 9.0 * eu * e[a]) * F[a];
        C[i] = (1.0 - 0.5 * omega) * w3_of(EX3[i] * EX3[i] + EY3[i] * EY3[i] + EZ3[i] * EZ3[i]) * s;
    }
}

static int wrap3(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* densities (Eq. 6), psi (Sec. II B) and the total force on each species
 * (Eqs. 8, 9 and rho_k g) at every node */
static void forces3(orc3_sim *s)
{
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    size_t n = N3(s);
    for (int k = 0; k < 2; ++k)
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t c = C3(s, x, y, z);
                    double r = 0.0;
                    for (int i = 0; i < 19; ++i) r += s->f[(k * 19 + i) * n + c];
                    s->rho[k * n + c] = r;
                    s->psi[k * n + c] = orc_psi(r);
                }
    const double G1 = s->p.G1, G2 = s->p.G2, GAB = s->p.G_AB;
    for (int k = 0; k < 2; ++k)
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t c = C3(s, x, y, z);
                    int kb = 1 - k;
                    double s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0}, s3[3] = {0, 0, 0};
                    for (int i = 0; i < 19; ++i) {
                        size_t d = C3(s, wrap3(x + EX3[i], nx), wrap3(y + EY3[i], ny), wrap3(z + EZ3[i], nz));
                        double w = w3_of(EX3[i] * EX3[i] + EY3[i] * EY3[i] + EZ3[i] * EZ3[i]);
                        double a = w * s->psi[k * n + d], b = w * s->rho[kb * n + d];
                        s1[0] += a * EX3[i]; s1[1] += a * EY3[i]; s1[2] += a * EZ3[i];
                        s3[0] += b * EX3[i]; s3[1] += b * EY3[i]; s3[2] += b * EZ3[i];
                    }
                    for (int dz = -2; dz <= 2; ++dz)
                        for (int dy = -2; dy <= 2; ++dy)
                            for (int dx = -2; dx <= 2; ++dx) {
                                size_t d = C3(s, wrap3(x + dx, nx), wrap3(y + dy, ny), wrap3(z + dz, nz));
                                double a = q3_of(dx * dx + dy * dy + dz * dz) * s->psi[k * n + d];
                                s2[0] += a * dx; s2[1] += a * dy; s2[2] += a * dz;
                            }
                    double psi = s->psi[k * n + c], rho = s->rho[k * n + c];
                    for (int a = 0; a < 3; ++a)
                        s->force[(k * 3 + a) * n + c] = -G1 * psi * s1[a] - G2 * psi * s2[a] - GAB * rho * s3[a]
                                                      + rho * s->p.g[a];
                }
}

/* Eq. (6) momenta with half force and the common velocity of Eq. (3) */
static void moments3(const orc3_sim *s, size_t c, double rho[2], double m[2][3], double ueq[3])
{
    size_t n = N3(s);
    for (int k = 0; k < 2; ++k) {
        double j[3] = {0, 0, 0};
        for (int i = 0; i < 19; ++i) {
            double fi = s->f[(k * 19 + i) * n + c];
            j[0] += fi * EX3[i]; j[1] += fi * EY3[i]; j[2] += fi * EZ3[i];
        }
        rho[k] = s->rho[k * n + c];
        for (int a = 0; a < 3; ++a) m[k][a] = j[a] + 0.5 * s->force[(k * 3 + a) * n + c];
    }
    double om0 = 1.0 / s->p.tau[0], om1 = 1.0 / s->p.tau[1];
    double den = om0 * rho[0] + om1 * rho[1];
    for (int a = 0; a < 3; ++a) ueq[a] = (om0 * m[0][a] + om1 * m[1][a]) / den;
}

static void step3_once(orc3_sim *s)
{
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    size_t n = N3(s);
    forces3(s);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = C3(s, x, y, z);
                double rho[2], m[2][3], ueq[3];
                moments3(s, c, rho, m, ueq);
                for (int k = 0; k < 2; ++k) {
                    double omega = 1.0 / s->p.tau[k], feq[19], C[19];
                    double F[3] = {s->force[(k * 3) * n + c], s->force[(k * 3 + 1) * n + c], s->force[(k * 3 + 2) * n + c]};
                    eq3(rho[k], ueq, feq);
                    guo3(s->p.tau[k], ueq, F, C);
                    for (int i = 0; i < 19; ++i) {
                        double fi = s->f[(k * 19 + i) * n + c];
                        size_t d = C3(s, wrap3(x + EX3[i], nx), wrap3(y + EY3[i], ny), wrap3(z + EZ3[i], nz));
                        s->fn[(k * 19 + i) * n + d] = fi - omega * (fi - feq[i]) + C[i];
                    }
                }
            }
    double *tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
    s->t += 1;
}

void orc3_step(orc3_sim *s, long n)
{
    for (long t = 0; t < n; ++t) step3_once(s);
}

/* f = f^eq(rho_k, u) from rho [2][nz][ny][nx] and an optional u [3][nz][ny][nx] */
void orc3_set_fields(orc3_sim *s, const double *rho, const double *u)
{
    size_t n = N3(s);
    for (size_t c = 0; c < n; ++c)
        for (int k = 0; k < 2; ++k) {
            double uu[3] = {u ? u[c] : 0.0, u ? u[n + c] : 0.0, u ? u[2 * n + c] : 0.0};
            double feq[19];
            eq3(rho[k * n + c], uu, feq);
            for (int i = 0; i < 19; ++i) s->f[(k * 19 + i) * n + c] = feq[i];
        }
    s->t = 0;
}

void orc3_get_f(const orc3_sim *s, double *f) { memcpy(f, s->f, sizeof(double) * 38 * N3(s)); }

/* rho [2][nz][ny][nx], force [2][3][..], ubar [3][..] (Eq. 7); NULL skips */
void orc3_fields(orc3_sim *s, double *rho, double *force, double *ubar)
{
    size_t n = N3(s);
    forces3(s);
    for (size_t c = 0; c < n; ++c) {
        double r[2], m[2][3], ue[3];
        moments3(s, c, r, m, ue);
        if (rho) { rho[c] = r[0]; rho[n + c] = r[1]; }
        if (force)
            for (int q = 0; q < 6; ++q) force[q * n + c] = s->force[q * n + c];
        if (ubar)
            for (int a = 0; a < 3; ++a) ubar[a * n + c] = (m[0][a] + m[1][a]) / (r[0] + r[1]);
    }
}

/* Observables: out[0..1] mass of A, B; out[2..7] momentum of A (x, y, z), B
 * (x, y, z) with half force; out[8] dp = <p_b>_in - <p_b>_out around the
 * probe sphere (inside r < R/2, outside r > R + 6, minimum image); out[9]
 * R_eff = (3 (M_A - rho_out N) / (4 pi (rho_in - rho_out)))^(1/3), the
 * equimolar radius; out[10] max |ubar|; out[11] 1 if every density and
 * velocity is finite.  R <= 0: out[8], out[9] NaN. */
void orc3_observables(orc3_sim *s, double cx, double cy, double cz, double R, double out[12])
{
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    size_t n = N3(s);
    double *rho = (double *)malloc(sizeof(double) * 2 * n), *ub = (double *)malloc(sizeof(double) * 3 * n);
    orc3_fields(s, rho, NULL, ub);
    double mass[2] = {0, 0}, mom[6] = {0, 0, 0, 0, 0, 0}, umax = 0.0;
    double pin = 0, pout = 0, ain = 0, aout = 0, nin = 0, nout = 0;
    int finite = 1;
    orc_params pp;
    memset(&pp, 0, sizeof pp);
    pp.G1 = s->p.G1; pp.G2 = s->p.G2; pp.G_AB = s->p.G_AB;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = C3(s, x, y, z);
                double r[2], m[2][3], ue[3];
                moments3(s, c, r, m, ue);
                for (int k = 0; k < 2; ++k) {
                    mass[k] += rho[k * n + c];
                    for (int a = 0; a < 3; ++a) mom[3 * k + a] += m[k][a];
                }
                double u2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    if (!isfinite(ub[a * n + c])) finite = 0;
                    u2 += ub[a * n + c] * ub[a * n + c];
                }
                if (!isfinite(rho[c]) || !isfinite(rho[n + c])) finite = 0;
                if (sqrt(u2) > umax) umax = sqrt(u2);
                if (R > 0.0) {
                    double d[3] = {fabs(x - cx), fabs(y - cy), fabs(z - cz)};
                    int L[3] = {nx, ny, nz};
                    double r2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        if (d[a] > 0.5 * L[a]) d[a] = L[a] - d[a];
                        r2 += d[a] * d[a];
                    }
                    double rr = sqrt(r2), pb = orc_bulk_pressure(&pp, rho[c], rho[n + c]);
                    if (rr < 0.5 * R) { pin += pb; ain += rho[c]; nin += 1.0; }
                    if (rr > R + 6.0) { pout += pb; aout += rho[c]; nout += 1.0; }
                }
            }
    out[0] = mass[0];
    out[1] = mass[1];
    for (int a = 0; a < 6; ++a) out[2 + a] = mom[a];
    if (R > 0.0 && nin > 0.0 && nout > 0.0) {
        double rin = ain / nin, rout = aout / nout;
        out[8] = pin / nin - pout / nout;
        out[9] = cbrt(3.0 * (mass[0] - rout * (double)n) / (4.0 * ORC_PI * (rin - rout)));
    } else {
        out[8] = NAN;
        out[9] = NAN;
    }
    out[10] = umax;
    out[11] = finite ? 1.0 : 0.0;
    free(rho);
    free(ub);
}
