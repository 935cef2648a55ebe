/*
 * lb.h -- C-ABI of the GB300 two-range pseudopotential lattice Boltzmann
 * library for binary mixtures with tunable viscosity ratio
 * (Fei, Scagliarini, Montessori, Lauricella, Succi, Luo, arXiv:1806.06943).
 *
 * The method (Sec. II of the paper), per time step and for both species
 * k in {A, B}:
 *   rho_k = sum_i f_k,i                                 Eq. (6)
 *   psi_k = 1 - exp(-rho_k)                             Sec. II B
 *   F_k   = F^c_k (Eq. 8, D2Q9 + D2Q25 stencils) + F^r_k (Eq. 9) + rho_k g
 *   rho_k u_k = sum_i f_k,i e_i + F_k / 2               Eq. (6)
 *   u^eq  = sum_k (rho_k u_k / tau_k) / sum_k (rho_k / tau_k)     Eq. (3)
 *   f_k,i(x + e_i, t + 1) = f - (f - f^eq(rho_k, u^eq)) / tau_k + C^Guo_k,i
 *                                                      Eqs. (1), (2), (5)
 * with half-way bounce-back walls at y = -1/2 and y = ny - 1/2 (Sec. III A)
 * and periodic boundaries otherwise.
 *
 * Conventions shared by every call:
 *  - Host arrays are row-major, x fastest: a field is [ny][nx] doubles and a
 *    species-resolved field is [2][ny][nx] (species A first).  A vector field
 *    stores its x component block before its y component block.
 *  - Calls return LB_OK (0) or a negative error code; the message of the
 *    last failure on the calling thread is returned by lb_last_error().  No
 *    call aborts, traps or exits the process.
 *  - Work is enqueued on lb_params.stream when it is not NULL (a stream the
 *    caller created on the current device; not the legacy default stream,
 *    since the time loop is replayed as a captured CUDA graph), otherwise on
 *    a non-blocking stream the handle creates and owns.  Calls that return
 *    host data synchronise that stream.
 *  - The handle owns all device memory it uses; the caller owns every
 *    pointer it passes and may reuse it as soon as the call returns.
 *  - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define LB_OK 0
#define LB_EINVAL (-1)    /* invalid argument: tau <= 1/2, nx or ny < 5, non-finite parameter, bad pointer */
#define LB_ENOMEM (-2)    /* device or host allocation failed */
#define LB_ECUDA (-3)     /* a CUDA runtime call failed (message names it) */
#define LB_EUNSTABLE (-4) /* a density or velocity became non-finite */
#define LB_ETIMEOUT (-5)  /* a bounded device-side wait expired */

/* Number formats of the populations. */
#define LB_FP64 0         /* plain populations f in IEEE double */
#define LB_FP32 1         /* offset populations h_i = f_i - w_i R in IEEE single, R the node's
                             density at the previous step; sums of the observables in FP64 */

/* Wall configurations. */
#define LB_PERIODIC 0     /* periodic in x and y */
#define LB_WALLS_Y 1      /* half-way bounce-back walls at y = -1/2 and y = ny - 1/2, periodic in x */

/* Execution modes of the time loop (lb_set_config, lb_batch_set_config).
 * LB_MODE_LAUNCH: each time step is a density-pass launch and a fused-kernel
 *   launch over the tiles of all lattices, replayed 32 steps per CUDA graph.
 * LB_MODE_PERSISTENT: one launch advances 64 time steps of all lattices; its
 *   blocks take (step, phase, tile) work items from an atomic queue and wait,
 *   with a bounded spin, only for the tiles of their own lattice that an item
 *   depends on; replayed as a CUDA graph.  A wait that runs out (default 2 s)
 *   ends the launch and the next synchronising call returns LB_ETIMEOUT.
 * LB_MODE_FUSED: each time step is one launch: every block forms the
 *   densities of its tile and 2-node halo from the populations itself (no
 *   separate density pass), then runs the fused force / collision / push;
 *   replayed 32 steps per CUDA graph.
 * LB_MODE_TMA (LB_FP32 only): LB_MODE_FUSED with every full tile of a
 *   lattice of at least 40 x (tile height + 4) nodes brought into shared
 *   memory by tensor-memory-accelerator copies of its box (the tile, 4
 *   columns each side, 2 rows above and below; 18 population planes and 2
 *   reference-density planes), completed on an mbarrier; each block also
 *   prefetches into L2 the box of a tile about a wave of blocks later.  Halo
 *   nodes across a periodic edge or on wall ghost rows, ragged tiles and
 *   smaller lattices load as in LB_MODE_FUSED.  Same arithmetic as
 *   LB_MODE_FUSED, same results.  A copy not complete within the wait limit
 *   (default 2 s) ends its block and the next synchronising call returns
 *   LB_ETIMEOUT. */
#define LB_MODE_LAUNCH 0
#define LB_MODE_PERSISTENT 1
#define LB_MODE_FUSED 2
#define LB_MODE_TMA 3

/* How the force enters the collision (lb_params.forcing).
 * LB_FORCING_GUO: the method of the paper: Guo forcing term of Eq. (5),
 *   component momenta with half the force (Eq. 6) in u^eq of Eq. (3).
 * LB_FORCING_SHIFT: the original two-range model the paper compares with:
 *   u^eq of Eq. (3) from the momenta sum_i f e_i without force, and the
 *   velocity-shift forcing term of Eq. (4), i.e. species k relaxes to
 *   f^eq(rho_k, u^eq + tau_k F_k / rho_k), which needs rho_k > 0 at every
 *   node (a vanishing species makes the shift non-finite, reported as
 *   LB_EUNSTABLE by the observables).  LB_FP64 populations only; no adjoint
 *   (lb_grad) for it.  The observables and fields keep the
 *   half-force momenta of Eq. (6) in both forms. */
#define LB_FORCING_GUO 0
#define LB_FORCING_SHIFT 1

/* Densities the interaction stencils see beyond a wall (ghost rows
 * y = -1, -2 and y = ny, ny + 1). */
#define LB_WALL_MIRROR 0  /* row -1 <- row 0, row -2 <- row 1, and symmetrically at the top */
#define LB_WALL_FIXED 1   /* wall_rho[k] for species k (non-wetting walls, Sec. III D) */

/* Parameters of one lattice (Sec. II A-B; Sec. III for the walls).
 *   nx, ny     lattice size, both >= 5
 *   tau[k]     relaxation times tau_A, tau_B > 1/2; nu_k = (tau_k - 1/2)/3
 *   G_AB       inter-species repulsion strength (Eq. 9), G_AB = G_BA
 *   G1, G2     short-range and mid-range intra-species strengths (Eq. 8),
 *              the same for both species
 *   g[2]       body acceleration; the body force on species k is rho_k g
 *   walls      LB_PERIODIC or LB_WALLS_Y
 *   wall_mode  LB_WALL_MIRROR or LB_WALL_FIXED (ignored without walls)
 *   wall_rho   ghost densities for LB_WALL_FIXED
 *   precision  LB_FP64 or LB_FP32
 *   forcing    LB_FORCING_GUO (the method) or LB_FORCING_SHIFT (the original
 *              model's velocity shift, LB_FP64 only)
 *   stream     the cudaStream_t to run on (see above), or NULL */
typedef struct lb_params {
    int32_t nx, ny;
    double tau[2];
    double G_AB, G1, G2;
    double g[2];
    int32_t walls;
    int32_t wall_mode;
    double wall_rho[2];
    int32_t precision;
    int32_t forcing;
    void *stream;
} lb_params;

/* Observables at the current time t, computed from the pre-collision
 * populations and the forces recomputed from them; sums in FP64.
 *   mass[k]      sum_x rho_k
 *   mom[k][a]    sum_x rho_k u_k,a (half force included, Eq. 6)
 *   flux_Q       (1/nx) sum_x ubar_x, ubar the barycentric velocity (Eq. 7)
 *   mu_r         Q0 / flux_Q, Q0 = g_x (ny^3 + ny/2) / (12 nu_B) the flux of
 *                the pure continuous phase (Sec. III D); NaN without walls
 *                or with g_x = 0
 *   dp_laplace   <p_b>_in - <p_b>_out around the probe (Eq. 11 bulk
 *                pressure; inside r < R/2, outside r > R + 6); NaN without probe
 *   R_eff        equimolar radius of species A around the probe; NaN without probe
 *   umax         max_x |ubar|
 *   finite       1 if every density and velocity is finite, else 0 */
typedef struct lb_obs {
    int64_t t;
    double mass[2];
    double mom[2][2];
    double flux_Q;
    double mu_r;
    double dp_laplace;
    double R_eff;
    double umax;
    int32_t finite;
    int32_t reserved;
} lb_obs;

typedef struct lb_handle lb_handle;
typedef struct lb_batch lb_batch;

/* Message of the last failed call on this thread ("" if none). */
const char *lb_last_error(void);

/* ---- one lattice ----------------------------------------------------------- */

/* Create a lattice on the current CUDA device.  The parameters are copied.
 * Populations start at f = f^eq(rho = 0, u = 0); set them with
 * lb_set_fields before stepping.  Returns LB_EINVAL, LB_ENOMEM or LB_ECUDA on
 * failure, with *out set to NULL. */
int lb_create(const lb_params *p, lb_handle **out);

/* Free the lattice and all its device memory.  NULL is ignored. */
void lb_destroy(lb_handle *h);

/* Set f_k,i = f^eq_i(rho_k, u) (Eq. 2) at every node and t = 0.
 *   rho  host [2][ny][nx] species densities
 *   u    host [2][ny][nx] initial velocity (x block, then y block), or NULL for rest
 * Synchronous with respect to the host buffers. */
int lb_set_fields(lb_handle *h, const double *rho, const double *u);

/* As lb_set_fields, with rho and u in device memory of the handle's device;
 * the copy is ordered on the handle's stream. */
int lb_set_fields_device(lb_handle *h, const double *rho, const double *u);

/* Advance n >= 0 time steps.  Asynchronous: returns once the work is
 * enqueued; a failure detected on the device surfaces on the next
 * synchronising call (lb_observables, lb_get_fields, lb_synchronize). */
int lb_step(lb_handle *h, int64_t n);

/* Block until the handle's queued work has finished.  Returns LB_ETIMEOUT
 * (once) if a bounded device-side wait of a persistent launch, or of a TMA
 * copy in LB_MODE_TMA, expired. */
int lb_synchronize(lb_handle *h);

/* Execution configuration: mode (LB_MODE_LAUNCH, LB_MODE_PERSISTENT,
 * LB_MODE_FUSED, or LB_MODE_TMA for LB_FP32 lattices) and tile height (2, 4
 * or 8 nodes; tiles are 32 nodes wide, one thread per node).  Default:
 * LB_MODE_LAUNCH, 4.  Results do not depend on it beyond the rounding order of
 * FP32 sums.  LB_EINVAL for an unknown mode or height, or LB_MODE_TMA on an
 * LB_FP64 handle or where the driver offers no tensor-map encoder. */
int lb_set_config(lb_handle *h, int32_t mode, int32_t tile_height);
int lb_get_config(const lb_handle *h, int32_t *mode, int32_t *tile_height);

/* Autotuner: times every mode and tile height on trial_steps time steps of
 * the current state (the state is restored after each trial, so the lattice
 * does not advance) and keeps the fastest.  With cache_path != NULL the
 * choice is read from / appended to that text file, keyed by device name,
 * precision and lattice shapes; a cached key skips the trials.  *best_ms
 * (may be NULL) receives the time per step of the chosen configuration.
 * Needs device memory for one copy of the state while it runs. */
int lb_autotune(lb_handle *h, int32_t trial_steps, const char *cache_path, double *best_ms);

/* Current time step count. */
int64_t lb_time(const lb_handle *h);

/* Probe for the Laplace observables: disk centre (cx, cy) and nominal
 * radius R > 0 (R <= 0 removes the probe). */
int lb_set_probe(lb_handle *h, double cx, double cy, double R);

/* Compute the observables at the current time into *o.  Synchronises.
 * Returns LB_EUNSTABLE (with *o filled) if a value is non-finite. */
int lb_observables(lb_handle *h, lb_obs *o);

/* Copy diagnostic fields at the current time to host memory; NULL skips one.
 *   rho   [2][ny][nx]       species densities
 *   mom   [2][2][ny][nx]    species momenta rho_k u_k with half force (Eq. 6)
 *   ubar  [2][ny][nx]       barycentric velocity (Eq. 7)
 * Synchronises. */
int lb_get_fields(lb_handle *h, double *rho, double *mom, double *ubar);

/* Pressure tensor at the current time (Sec. II B, Eq. 10), in FP64, from the
 * pre-collision populations and the densities they give:
 *   kinetic part      P^kin_ab = sum_k sum_i f_k,i e_ia e_ib             Eq. (13)
 *   interaction part  P^int_ab = 1/2 sum_k [G1 psi_k(x) sum_i w_i psi_k(x + e_i) e_ia e_ib
 *                                + G2 psi_k(x) sum_j p_j psi_k(x + e_j) e_ja e_jb
 *                                + G_AB rho_k(x) sum_i w_i rho_kbar(x + e_i) e_ia e_ib]
 * The paper defines P^int by its divergence (Eq. 12) only; this per-node form
 * shares each pair interaction of Eqs. (8), (9) equally between its two
 * nodes: uniform states give the bulk pressure of Eq. (11), and the sum over
 * a flat interface, which the surface tension of Eq. (15) integrates, equals
 * that of any other sharing.  Ghost rows and periodic copies are those of
 * the forces.
 *   P     host [2][3][ny][nx] (kinetic, interaction; components xx, yy, xy),
 *         or NULL
 *   sums  host [6]: the lattice sums of the six fields (same order), or NULL
 * For a flat interface normal to x in a periodic lattice (two interfaces),
 * gamma = (sums[0] + sums[3] - sums[1] - sums[4]) / (2 ny).  Synchronises. */
int lb_pressure_tensor(lb_handle *h, double *P, double sums[6]);

/* Copy the populations f_k,i (as FP64; for LB_FP32 with w_i R added back) to
 * host [2][9][ny][nx], direction order: rest, (1,0), (0,1), (-1,0), (0,-1),
 * (1,1), (-1,1), (-1,-1), (1,-1).  Synchronises. */
int lb_get_populations(lb_handle *h, double *f);

/* Overwrite the populations from host [2][9][ny][nx] (same order) and set the
 * time counter to t (LB_FP32: R becomes sum_i f_k,i rounded to single). */
int lb_set_populations(lb_handle *h, const double *f, int64_t t);

/* Checkpoint: with buf == NULL store the byte size needed in *len; otherwise
 * write the time counter and the raw state (populations, and for LB_FP32 the
 * reference densities; bitwise, native format) into buf of *len bytes.
 * Synchronises. */
int lb_save(lb_handle *h, void *buf, size_t *len);

/* Restore a checkpoint written by lb_save on a lattice of the same size and
 * precision. */
int lb_load(lb_handle *h, const void *buf, size_t len);

/* Time nsteps time steps kernel by kernel with CUDA events on the handle's
 * stream (direct launches, no graph):
 *   ms[0]  mean duration of one density-pass launch (0 in LB_MODE_FUSED)
 *   ms[1]  mean duration of one fused force/collide/stream launch (in
 *          LB_MODE_FUSED the one-pass kernel; LB_MODE_PERSISTENT is timed as
 *          LB_MODE_LAUNCH)
 *   ms[2]  mean duration of one whole time step (both launches)
 * If flush_bytes > 0, the caller's device buffer flush_buf of that size is
 * overwritten before every step, outside the timed intervals, so that each
 * step starts with no population data in L2.  The lattice advances by
 * nsteps.  Synchronises. */
int lb_profile(lb_handle *h, int32_t nsteps, void *flush_buf, size_t flush_bytes, double ms[3]);

/* Objectives of lb_grad. */
#define LB_OBJ_MU_R 0     /* relative effective viscosity mu_r = Q0 / Q (walls, g_x != 0) */
#define LB_OBJ_DP 1       /* Laplace pressure jump dp_laplace around the probe */

/* Gradient of an observable J of the state reached after nsteps time steps,
 * with respect to theta = (G_AB, G1, G2, tau_A, tau_B), by the discrete
 * adjoint of the time step (reverse of Eqs. 1-3, 5, 6, 8, 9 with streaming and
 * bounce-back): a forward sweep stores the populations every ckpt_every steps;
 * each segment is then recomputed from its checkpoint and stepped backwards.
 * On return the lattice holds the state after nsteps steps (as lb_step would
 * leave it), *J the observable there and dJ[5] its gradient; parameter
 * gradients are accumulated in FP64.  An LB_FP32 lattice runs the forward
 * sweep and the recomputation in FP32 (checkpoints hold offsets and reference
 * densities) and hands the adjoint FP64 populations f = h + w R of each step;
 * the adjoint populations and the gradients stay FP64.  LB_OBJ_DP needs a
 * probe.  Device memory, allocated for the call: nsteps/ckpt_every + 1
 * states of the lattice's precision, ckpt_every + 2 (FP32: + 3) FP64
 * population copies, plus 22 FP64 planes.  Synchronises. */
int lb_grad(lb_handle *h, int64_t nsteps, int32_t ckpt_every, int32_t objective, double *J, double dJ[5]);

/* One step of the discrete adjoint at the current state (the transpose of
 * the linearised time step, Eqs. 1-3, 5, 6, 8, 9 with streaming and
 * bounce-back): for host w[2][9][ny][nx] (population order of
 * lb_get_populations), out = (dStep/df)^T w and dtheta = <w, dStep/dtheta>
 * for theta = (G_AB, G1, G2, tau_A, tau_B), Step the map from the
 * populations at time t to those at t + 1.  Either output may be NULL.
 * LB_FP64 lattices with Guo forcing only (else LB_EINVAL).  The state is
 * not changed.  Device memory: two FP64 population copies and 22 FP64
 * planes, allocated for the call.  Synchronises. */
int lb_step_vjp(lb_handle *h, const double *w, double *out, double dtheta[5]);

/* ---- many independent lattices advanced together ------------------------- */

/* Create n >= 1 lattices of possibly different sizes and parameters that
 * are stepped together: each time step is one launch of each kernel over the
 * tiles of all lattices.  All p[i].precision must agree; the stream of p[0]
 * is used.  With n >= 2, lb_batch_step runs the lattices as two chains
 * (groups of about equal node counts, each launch over one group's tiles):
 * the second on a non-blocking stream the batch creates and owns, forked
 * from and joined back to the batch's stream by events inside each step
 * call, so work the caller enqueues on that stream afterwards still sees
 * every lattice stepped.  The populations are the same bit for bit as with
 * one launch per step.  lb_batch_profile times single launches over all
 * tiles. */
int lb_batch_create(const lb_params *p, int32_t n, lb_batch **out);
void lb_batch_destroy(lb_batch *b);
int lb_batch_size(const lb_batch *b);
int lb_batch_set_fields(lb_batch *b, int32_t i, const double *rho, const double *u);
int lb_batch_step(lb_batch *b, int64_t n);
int lb_batch_synchronize(lb_batch *b);
int lb_batch_set_probe(lb_batch *b, int32_t i, double cx, double cy, double R);
/* o points to n lb_obs, one per lattice.  Synchronises. */
int lb_batch_observables(lb_batch *b, lb_obs *o);
int lb_batch_get_fields(lb_batch *b, int32_t i, double *rho, double *mom, double *ubar);
/* As lb_pressure_tensor, for lattice i of the batch (the sums of every
 * lattice are formed by one launch). */
int lb_batch_pressure_tensor(lb_batch *b, int32_t i, double *P, double sums[6]);
/* As lb_profile, over all lattices of the batch (one launch covers them all). */
int lb_batch_profile(lb_batch *b, int32_t nsteps, void *flush_buf, size_t flush_bytes, double ms[3]);
/* As lb_set_config, lb_get_config and lb_autotune, for the whole batch. */
int lb_batch_set_config(lb_batch *b, int32_t mode, int32_t tile_height);
int lb_batch_get_config(const lb_batch *b, int32_t *mode, int32_t *tile_height);
int lb_batch_autotune(lb_batch *b, int32_t trial_steps, const char *cache_path, double *best_ms);
/* Limit of every bounded wait of the persistent kernel and of the TMA copies
 * of LB_MODE_TMA, in seconds (default 2).  drop_tile >= 0 is a test hook:
 * that tile of the batch's tile list (for the configured tile height) never
 * reports completion in LB_MODE_PERSISTENT, or never has its copy started in
 * LB_MODE_TMA, so the waits on it run out and the launch ends with
 * LB_ETIMEOUT; -1 turns the hook off. */
int lb_batch_set_wait_limit(lb_batch *b, double seconds, int32_t drop_tile);

/* ---- three-dimensional extension ------------------------------------------- */

/* The method in 3-D (the paper is 2-D): D3Q19 fluid (weights 1/3, 1/18,
 * 1/36) with the BGK + Guo step of Eqs. (1)-(3), (5), (6); the short-range
 * sums of Eqs. (8), (9) over the D3Q19 neighbours; the mid-range sum of
 * Eq. (8) over the 5 x 5 x 5 neighbourhood with weights q(|e|^2) = 47/90,
 * 4/135, 1/63, 2/315, 5/1512, 1/945, 1/1890, 1/15120 for |e|^2 = 0..6, 8 (0
 * for 9, 12): isotropic to eighth order, with the D2Q25 weights' second and
 * fourth moments, so that a profile varying along one axis evolves exactly
 * as in 2-D.  Periodic in x, y and z; no walls.  Host arrays are
 * [..][nz][ny][nx], x fastest; a species field is [2][nz][ny][nx], a vector
 * field [3][nz][ny][nx], populations [2][19][nz][ny][nx] with the direction
 * order rest, (+-1,0,0), (0,+-1,0), (0,0,+-1), (1,1,0), (-1,-1,0), (1,-1,0),
 * (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1),
 * (0,1,-1), (0,-1,1).  One time step is two launches (density pass, fused
 * force / collision / push); LB_FP32 stores offsets from the node's previous
 * density as the 2-D form does.  Same error conventions as above. */
typedef struct lb3_params {
    int32_t nx, ny, nz;   /* each >= 5 */
    int32_t precision;    /* LB_FP64 or LB_FP32 */
    double tau[2];        /* > 1/2 */
    double G_AB, G1, G2;  /* Eqs. (8), (9) */
    double g[3];          /* body acceleration; the force on species k is rho_k g */
    void *stream;         /* cudaStream_t, or NULL for a stream of its own */
} lb3_params;

/* mass[k], mom[k][a] (half force, Eq. 6), dp_laplace and R_eff (equimolar
 * sphere radius, (3 V / 4 pi)^(1/3)) around the probe (inside r < R/2,
 * outside r > R + 6; NaN without probe), umax = max |ubar| (Eq. 7), finite. */
typedef struct lb3_obs {
    int64_t t;
    double mass[2];
    double mom[2][3];
    double dp_laplace;
    double R_eff;
    double umax;
    int32_t finite;
    int32_t reserved;
} lb3_obs;

typedef struct lb3_handle lb3_handle;

int lb3_create(const lb3_params *p, lb3_handle **out);
void lb3_destroy(lb3_handle *h);
/* f = f^eq(rho_k, u) (Eq. 2) and t = 0; rho host [2][nz][ny][nx], u host
 * [3][nz][ny][nx] or NULL.  Synchronous. */
int lb3_set_fields(lb3_handle *h, const double *rho, const double *u);
/* Advance n >= 0 steps (asynchronous, as lb_step). */
int lb3_step(lb3_handle *h, int64_t n);
int64_t lb3_time(const lb3_handle *h);
/* Sphere probe for the Laplace observables (R <= 0 removes it). */
int lb3_set_probe(lb3_handle *h, double cx, double cy, double cz, double R);
/* Observables at the current time, sums in FP64.  Synchronises; LB_EUNSTABLE
 * (with *o filled) if a value is not finite. */
int lb3_observables(lb3_handle *h, lb3_obs *o);
/* rho host [2][nz][ny][nx] and ubar host [3][nz][ny][nx]; NULL skips one. */
int lb3_get_fields(lb3_handle *h, double *rho, double *ubar);
/* Populations as FP64 host [2][19][nz][ny][nx] (LB_FP32: w_i R added back). */
int lb3_get_populations(lb3_handle *h, double *f);
/* As lb_profile: ms[0] density pass, ms[1] fused kernel, ms[2] whole step. */
int lb3_profile(lb3_handle *h, int32_t nsteps, void *flush_buf, size_t flush_bytes, double ms[3]);

/* ---- device diagnostics ------------------------------------------------------ */

/* Measured FP64 fused multiply-add throughput of the current device in
 * TFLOP/s (2 flops per FMA): independent FMA chains on every SM at full
 * occupancy, trips x 128 FMAs per thread, best of five timed launches after
 * a warm-up, CUDA events on a stream of its own.  Not part of the method: it
 * is the denominator of the FP64 step's roofline, which is bound by the FP64
 * pipe rather than by memory.  Allocates and frees a few KB; synchronises.
 * LB_EINVAL for trips < 1 or a NULL tflops, LB_ECUDA on a failed CUDA call. */
int lb_device_fp64_peak(int32_t trips, double *tflops);

/* ---- observables without any allocation ------------------------------------ */

/* Largest lattice lb_observables_static accepts, in tiles of 32 x 4 nodes
 * (32768 tiles: 4,194,304 nodes, e.g. 2048 x 2048). */
#define LB_STATIC_MAX_TILES 32768

/* Observables of an LB_FP64 lattice whose populations live in the caller's
 * device memory, computed without allocating memory.  No counterpart in the
 * paper: this is a service for callers that may not call cudaMalloc (or
 * anything else that allocates) once they run, e.g. an application that owns
 * a fixed device-memory budget, or a solver step that must stay out of the
 * driver's allocator.
 *   p     lattice parameters, checked as lb_create checks them (precision
 *         must be LB_FP64; p->stream is the stream the two kernels are
 *         launched on, NULL for the default stream)
 *   f     device [2][9][ny][nx] FP64 populations, direction order as for
 *         lb_get_populations
 *   cx, cy, R   Laplace probe as for lb_set_probe (R <= 0: none)
 *   obs   device array of 16 doubles receiving, in order: mass A, mass B,
 *         momentum A (x, y), momentum B (x, y), flux_Q, mu_r, dp_laplace,
 *         R_eff, umax, finite (1.0 or 0.0), then four zeros; the definitions
 *         are those of lb_obs
 * The scratch is a file-scope device array of LB_STATIC_MAX_TILES x 16
 * doubles (4 MiB).  CUDA loads the part of the library that holds it on
 * first use on each device; that is when the driver places the array, which
 * the device then keeps until the process exits.  Only that first use can
 * allocate: call lb_observables_static(NULL, NULL, 0, 0, 0, NULL) (f and obs
 * both NULL: set-up only, nothing is launched, p is ignored) on each device,
 * with that device current, before the phase in which nothing may be
 * allocated and before any stream capture; every later call allocates
 * nothing.  Each call looks the array's device address up again (no
 * allocation once loaded), so a context reset in between is harmless.
 * Every call shares the array and leaves its contents behind; calls whose
 * kernels overlap on the GPU race on it, so serialise them (one stream, or
 * events).  Asynchronous: obs is written when the stream reaches the
 * kernels.  Returns LB_EINVAL for a NULL p, f or obs (other than the set-up
 * form), invalid parameters, a precision other than LB_FP64, a non-finite
 * probe, or a lattice of more than LB_STATIC_MAX_TILES tiles; LB_ECUDA if
 * the address lookup or a launch fails. */
int lb_observables_static(const lb_params *p, const double *f, double cx, double cy, double R, double *obs);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
