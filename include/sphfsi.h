/*
 * sphfsi — GB300 (sm_103a) library for one coarse time step of the
 * multi-resolution SPH fluid-structure interaction method of Zhang, Rezavand
 * & Hu, "A multi-resolution SPH method for fluid-structure interactions"
 * (arXiv 1911.13255).
 *
 * One step (sphfsi_step) is, in order (Section 3, Alg. 1):
 *   a1  inflow buffer and fluid first half drift of rho and r
 *       (Eq. verlet-first-half)
 *   a2  cell-linked-list neighbour build (counting sort by cell), fluid grid
 *       with cell edge >= 2 h_F; solid and wall particles binned in it
 *   a3  every n_reinit steps: density reinitialisation from the number
 *       density and solid normal update (Alg. 1, outer loop)
 *   a4  equation of state (Eq. eqeos), fluid momentum with the Riemann
 *       pressure and viscous terms at h_F plus the fluid-solid/wall ghost
 *       forces (Eqs. fluid-model-mr-mom, fs-force-mr-sp, fs-force-mr-sv,
 *       fs-coupling-mr) and the velocity kick (Eq. verlet-first-mediate)
 *   a5  fluid force on the solid from the same pair terms (Eqs. F:p, F:v)
 *   a6  fluid continuity (Eq. fluid-model-mr-con) and second half drift
 *       (Eq. verlet-first-final)
 *   a7  K solid sub-steps at h_S, dt_S = dt_F / K: corrected deformation
 *       gradient, neo-Hookean PK1 stress and force loop, position-based
 *       Verlet (Eqs. correctmatrix, solid-model-mr, Neo-Hookean-energy,
 *       verlet-first-half-solid .. verlet-first-final-solid)
 *   a8  time-averaged solid velocity and acceleration for the next step's
 *       coupling (Eq. fs-coupling-mr), max-speed reductions for the next
 *       time step (Eqs. dt-relax, dts-advection), FP64 momentum sums.
 *
 * Precision: pair loops in FP32; particle positions, solid displacement,
 * the time-averaged sums and the momentum reductions in FP64.
 *
 * Conventions for every entry point:
 *   - Return 0 on success or a negative SPHFSI_E_* code; nothing aborts.
 *   - Vectors are row-major n x dim, tensors n x dim x dim, in the caller's
 *     original particle order (the library keeps the permutation).
 *   - Array arguments may be host pointers or CUDA device pointers (unified
 *     addressing decides); the caller owns them; the library copies.
 *   - All work is issued on the stream given to sphfsi_create; getters and
 *     sphfsi_sync wait for it.
 *   - A context is used by one host thread at a time.
 */
#ifndef SPHFSI_H
#define SPHFSI_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPHFSI_OK 0
#define SPHFSI_E_INVAL (-1)    /* bad argument or out-of-range size         */
#define SPHFSI_E_NOMEM (-2)    /* device allocation failed                   */
#define SPHFSI_E_CUDA (-3)     /* a CUDA runtime call failed                 */
#define SPHFSI_E_STATE (-4)    /* call out of order (e.g. step before finalize) */
#define SPHFSI_E_UNSTABLE (-5) /* run-away (non-finite) state on the device  */
#define SPHFSI_E_TIMEOUT (-6)  /* a bounded device-side wait ran out         */
#define SPHFSI_E_CAPACITY (-7) /* problem exceeds a documented device limit  */

typedef struct sphfsi_ctx sphfsi_ctx;

/* Global parameters.  gravity is an acceleration (body force per unit
 * mass).  The fixed cell grid covers [domain_lo, domain_hi]; particles that
 * leave it are clamped into the border cells (still correct, slower).
 * periodic_x wraps fluid particles in x over [x_lo, x_lo + Lx); the grid's
 * x extent is then that period.  free_surface selects the density
 * reinitialisation rho = max(rho0 sigma / sigma0, rho0).  n_reinit is the
 * cadence of density reinitialisation and normal update in steps (0 = off).
 * cell_reach (no counterpart in the paper) sets the cell grid of the pair
 * loops: 1 (or 0) cells of edge >= 2 h_F, the 3^d cells around a particle's
 * cell hold its neighbours; 2 cells of edge >= h_F and the 5^d cells around
 * it, which test fewer candidates per particle (a volume of (5 h_F)^d
 * instead of (6 h_F)^d) in more, smaller cells.  With 2 the pair loops run
 * in the cell form without tiles.  Results agree to rounding. */
typedef struct {
    int32_t dim; /* 2 or 3 */
    int32_t periodic_x;
    double gravity[3];
    double x_lo, Lx;
    int32_t free_surface;
    int32_t n_reinit;
    double domain_lo[3], domain_hi[3];
    int32_t cell_reach; /* 0 or 1: cells of >= 2 h_F; 2: cells of >= h_F */
} sphfsi_params;

/* Velocity-imposing inflow buffer (Section 4.1): fluid particles with
 * x in [x_lo, x_lo + width) get v = (U(y, t), 0, 0) at the start of a step.
 * profile 0: U = 6 Ubar (y - y0)(H - (y - y0)) / H^2 (mean Ubar, clamped to
 * [y0, y0 + H]); profile 1: uniform Ubar.  Ubar(t) = U (1 - cos(pi t /
 * t_ramp)) / 2 for t < t_ramp, else U.  profile 2 (Section 4.3, Appendix
 * A): the Womersley flow of a channel of height H under the pressure
 * gradient dp/dx = -A cos(2 pi t / period), with U = A / rho_F (m/s^2, ramped
 * like Ubar) and womersley = (H / 2) sqrt(2 pi / (period nu)); with
 * b = womersley / sqrt(2), s = 2 (y - y0) / H - 1, f1,2 = b (1 +- s),
 * g = cosh 2b + cos 2b, w = 2 pi / period:
 * u = U / (w g) [(sinh f1 sin f2 + sinh f2 sin f1) cos wt
 *                + (g - cosh f1 cos f2 - cosh f2 cos f1) sin wt].
 * profile 3 (3-D ducts; the channel profile of Section 4.1 across both
 * walls' directions, no counterpart in the paper): U = 36 Ubar (y - y0)
 * (H - (y - y0)) (z - z0) (Hz - (z - z0)) / (H^2 Hz^2), y and z clamped to
 * the cross-section [y0, y0 + H] x [z0, z0 + Hz]: zero on its four walls,
 * mean Ubar.  SPHFSI_E_INVAL (when on) for width <= 0, an unknown profile,
 * H <= 0 with profile 0, 2 or 3, period or womersley <= 0 with profile 2,
 * or Hz <= 0 or a non-finite z0 with profile 3. */
typedef struct {
    int32_t on, profile;
    double width, y0, H, U, t_ramp;
    double period, womersley;   /* profile 2 only */
    double z0, Hz;              /* profile 3 only */
} sphfsi_inflow;

/* Counters and last-step diagnostics of the selected instance. */
typedef struct {
    int64_t n_fluid, n_solid, n_wall, n_cells;
    int64_t step;            /* completed steps                                  */
    double t;                /* simulated time                                   */
    double last_dt;          /* dt_F of the last step                            */
    int32_t last_K;          /* solid sub-steps of the last step                 */
    int32_t status;          /* device status bits of the last sync (0 = fine)   */
    int64_t pairs_ff, pairs_fw, pairs_fs, pairs_sf; /* in-support pairs, last step */
    int64_t pairs_ss;        /* static solid neighbour entries (per loop)        */
    int64_t pairs_total;     /* all pair interactions since creation             */
    double vmax_f, vmax_s, amax_s;  /* reductions of the last step               */
    double mom_fs_fluid[3];  /* sum of fluid-side fluid-solid forces, last step  */
    double mom_fs_solid[3];  /* sum of solid-side fluid forces, last step        */
    int32_t solid_path;      /* 1 = cluster-resident sub-steps, 2 = cooperative grid,
                                3 = cluster-resident, one cluster barrier per sub-step */
    int32_t kernels_per_step; /* this library's kernel launches per step        */
    int64_t learned_accepted; /* steps whose learned solid step was accepted    */
    int64_t learned_rejected; /* steps that fell back to the plain sub-steps    */
    double learned_residual;  /* residual R of the last learned step            */
} sphfsi_info;

/* Create an empty context bound to a CUDA stream (cudaStream_t, may be 0
 * for the legacy default stream) on the current device.  *out receives the
 * context; the caller frees it with sphfsi_destroy. */
int sphfsi_create(sphfsi_ctx **out, const sphfsi_params *p, void *cuda_stream);

/* Batched context of n >= 1 independent instances (the paper has no
 * counterpart: many small problems of the kind of Section 4 advanced by the
 * same launches).  p points to n parameter blocks, all of the same dim.
 * Every instance has its own particles, grid, constants, time, dt_F and K;
 * one sphfsi_step / sphfsi_run advances all of them.  The set-up calls
 * (add_fluid, set_walls, add_solid, set_inflow), the getters and setters,
 * sphfsi_set_time, sphfsi_get_info and sphfsi_debug_neighbors act on the
 * instance chosen by sphfsi_select (0 after creation).  Each instance's
 * body must fit one thread-block cluster (sphfsi_set_solid_path); a batch
 * whose body does not gets SPHFSI_E_CAPACITY from the first step.
 * sphfsi_create(out, p, s) is sphfsi_create_batch(out, 1, p, s).  n outside
 * [1, 2^20] or mixed dim: SPHFSI_E_INVAL. */
int sphfsi_create_batch(sphfsi_ctx **out, int32_t n, const sphfsi_params *p, void *cuda_stream);

/* Choose the instance that the per-instance calls address (0 <= inst < n,
 * else SPHFSI_E_INVAL). */
int sphfsi_select(sphfsi_ctx *c, int32_t inst);

/* Pair interactions of all instances since creation (sum of
 * sphfsi_info.pairs_total over the instances); waits for the stream. */
int sphfsi_pairs_total(sphfsi_ctx *c, int64_t *total);

/* Fluid particles (Section 2.1): positions r (n x dim, FP64), velocities v
 * (n x dim), initial pressure p_init (n; the density follows from the
 * inverse of Eq. eqeos; NULL means rho = rho0), spacing dp (h_F = 1.3 dp,
 * mass rho0 dp^dim), reference density rho0, sound speed c0, dynamic
 * viscosity eta.  Called once, before sphfsi_finalize. */
int sphfsi_add_fluid(sphfsi_ctx *c, int64_t n, const double *r, const double *v, const double *p_init,
                     double dp, double rho0, double c0, double eta);

/* Static wall particles (v = 0) with outward unit normals nrm pointing into
 * the fluid, spacing dp (volume dp^dim).  Optional; once, before finalize. */
int sphfsi_set_walls(sphfsi_ctx *c, int64_t n, const double *r, const double *nrm, double dp);

/* One elastic body (Section 2.1, total Lagrangian, neo-Hookean): reference
 * positions r0, initial velocities v0, outward unit normals n0 (solid ->
 * fluid) in the reference configuration, constrained flags (1 = position
 * fixed at r0, velocity 0), spacing dp (h_S = 1.3 dp, volume dp^dim),
 * density rho0, Young's modulus E, Poisson ratio nu.  Optional; once. */
int sphfsi_add_solid(sphfsi_ctx *c, int64_t n, const double *r0, const double *v0, const double *n0,
                     const uint8_t *constrained, double dp, double rho0, double E, double nu);

/* Inflow buffer (see sphfsi_inflow).  Optional; before finalize. */
int sphfsi_set_inflow(sphfsi_ctx *c, const sphfsi_inflow *f);

/* Build the device state: the solid's static reference neighbour list and
 * correction matrices B0 (Eq. correctmatrix), F = I, the wall bins, the
 * lattice number density sigma0 for reinitialisation. */
int sphfsi_finalize(sphfsi_ctx *c);

/* Fix the number of solid sub-steps K per fluid step (K >= 1), or 0 for
 * the paper's kappa = [dt_F / dt_S] + 1 from the previous step's maxima
 * (Section 3.2).  SPHFSI_E_INVAL for K < 0. */
int sphfsi_set_substeps(sphfsi_ctx *c, int32_t K);

/* Time stepping of fluid and solid (the paper's comparison of multiple and
 * single time steps, Tables 1 and 2).  mode 0: multiple time steps, the
 * setting of sphfsi_set_substeps (the default, kappa sub-steps).  mode 1:
 * one time step for both, K = 1, dt = min(0.25 min(h_F / (c_F + |v|max),
 * h_F^2 / nu), 0.6 min(h_S / (c_S + |v|max), sqrt(h_S / |dv/dt|max))), the
 * single-step criterion of Section 2.2 with |v|max over fluid and solid,
 * |dv/dt|max over the solid, nu = eta / rho0 and each phase's own h, from the
 * previous step's maxima.  mode 2: K = 1, dt = min(dt_ac^F, dt^S), the solid
 * step taken as the step of both (Section 3.2).  In modes 1 and 2 a step
 * called with dt_F <= 0 takes that dt; dt_F > 0 still fixes it.  The last
 * call of sphfsi_set_substeps or this one decides.  SPHFSI_E_INVAL for any
 * other mode.  Applies to every instance of a batch. */
int sphfsi_set_time_stepping(sphfsi_ctx *c, int32_t mode);

/* Advection cadence of the pair configuration (Algorithm 1: the neighbour
 * lists and the kernel values W_ij and gradients grad W_ij are updated once
 * per advection step and held over its acoustic steps).  n = 1 (the
 * default): rebuilt every coarse step from the step's mid positions.  n > 1:
 * rebuilt at steps whose index (instance 0's) is a multiple of n.  n = 0:
 * the advection steps of Algorithm 1 (reading F3): an advection step starts
 * with a rebuild and lasts while the coarse steps taken in it sum to at most
 * dt_ad = 0.25 min(h_F / |v|max, h_F^2 / nu) (Eq. dtf-advection, nu =
 * eta / rho0), evaluated at the fluid speed maximum each of its steps starts
 * from, the smallest of those values counting (instance 0's values decide
 * for a batch).  Every cadence also rebuilds at the next step after any of
 * sphfsi_set_fluid_state, sphfsi_set_solid_state, sphfsi_set_time or this
 * call.  On the steps between rebuilds every pair term takes its W and
 * grad W at the fluid and solid positions of the last rebuild (the same
 * pairs, in the same order), with current densities, pressures, velocities,
 * time-averaged solid velocities and accelerations and normals.  All
 * instances of a batch rebuild together.  While n != 1,
 * sphfsi_debug_neighbors returns SPHFSI_E_STATE (its binning would replace
 * the held configuration).  SPHFSI_E_INVAL for n < 0. */
int sphfsi_set_advection_cadence(sphfsi_ctx *c, int32_t n);

/* One coarse step a1..a8.  dt_F > 0 fixes the step; dt_F <= 0 uses the
 * acoustic criterion 0.6 h_F / (c0 + |v|max) (Eq. dt-relax) from the
 * previous step's maximum fluid speed.  Asynchronous on the context stream;
 * errors detected on the device surface at the next sphfsi_sync. */
int sphfsi_step(sphfsi_ctx *c, double dt_F);

/* nsteps steps replayed from one captured CUDA graph of a step (the first
 * call captures it); same semantics as nsteps calls of sphfsi_step. */
int sphfsi_run(sphfsi_ctx *c, int64_t nsteps, double dt_F);

/* Wait for the stream; return SPHFSI_E_UNSTABLE / SPHFSI_E_TIMEOUT if the
 * device flagged a run-away state or a bounded wait ran out in any
 * instance.  After SPHFSI_E_TIMEOUT the state is not a valid step of the
 * method (the step that gave up was not completed, and when the cell-list
 * scan gave up, that step's and later steps' kernels returned without
 * work): sphfsi_step and sphfsi_run return SPHFSI_E_TIMEOUT without doing
 * anything until sphfsi_set_state restores a checkpoint taken before.
 * A run-away state (no counterpart in the paper) is a step that ended with
 * a non-finite maximum fluid speed, solid speed or solid acceleration, a
 * fluid particle faster than the artificial sound speed c0 (outside the
 * weakly-compressible model), or a solid step more than 10^6 times shorter
 * than the fluid step.  The steps enqueued after it (in the same graph
 * replay, or before the sync that reports it) do no work, and from that
 * sync on sphfsi_step and sphfsi_run return SPHFSI_E_UNSTABLE until
 * sphfsi_set_state restores a checkpoint taken before; in a batch this
 * stops every instance. */
int sphfsi_sync(sphfsi_ctx *c);

/* Bounded device waits (no counterpart in the paper): the grid barrier of the
 * cooperative sub-step kernel and the decoupled look-back of the cell-list
 * scan give up after this many polling iterations, set SPHFSI_E_TIMEOUT and
 * return, so a stalled wait never hangs the device.  0 restores the default
 * (2^22 iterations, about 0.5 to 2 s); a small value makes waits give up
 * almost at once (for checking how a time-out is reported).  Applies to the
 * steps issued after the call.  SPHFSI_E_INVAL for a negative value. */
int sphfsi_set_wait_limit(sphfsi_ctx *c, int64_t iterations);

/* Fluid state in original order: r (n x dim FP64), v (n x dim FP32),
 * rho (n FP64: rho0 plus the FP32 deviation the library stores), drho_dt
 * (n FP32, the last density rate), dvdt (n x dim
 * FP32, the last step's accelerations, a4).  Any pointer may be NULL. */
int sphfsi_get_fluid(sphfsi_ctx *c, double *r, float *v, double *rho, float *drho_dt, float *dvdt);

/* Solid state in original order: r (FP64), v (FP32), F (n x dim x dim
 * FP64: I plus the FP32 displacement gradient the library stores), vbar and abar (FP64, the time averages of the last step), fF (the
 * fluid force of the last step, FP32), nrm (current normals, FP32). */
int sphfsi_get_solid(sphfsi_ctx *c, double *r, float *v, double *F, double *vbar, double *abar, float *fF,
                     float *nrm);

/* Solid positions of every instance (original order within each instance,
 * instances in order, n_total x dim FP64); one device read for the batch. */
int sphfsi_get_solid_positions_all(sphfsi_ctx *c, double *r);

/* The same rows, read without waiting: a gather kernel and a copy into r are
 * enqueued on the context's stream after the steps enqueued so far, and the
 * call returns at once.  r (n_total x dim FP64, host or device; pinned host
 * memory for a copy that overlaps later steps) must stay valid, and is
 * complete only once the stream has reached the copy (sphfsi_sync, or an
 * event recorded on the stream after this call).  Returns SPHFSI_E_INVAL for
 * a NULL r, SPHFSI_E_STATE before sphfsi_finalize. */
int sphfsi_get_solid_positions_async(sphfsi_ctx *c, double *r);

/* Overwrite the dynamic state (original order, FP64 inputs; NULL keeps a
 * field).  Used for checkpoint/resume and for parity at a given state. */
int sphfsi_set_fluid_state(sphfsi_ctx *c, const double *r, const double *v, const double *rho,
                           const double *drho_dt);
int sphfsi_set_solid_state(sphfsi_ctx *c, const double *r, const double *v, const double *F,
                           const double *vbar, const double *abar, const double *nrm);
int sphfsi_set_time(sphfsi_ctx *c, double t, int64_t step);

int sphfsi_get_info(sphfsi_ctx *c, sphfsi_info *out);

/* Time-step criteria of the selected instance at its current state, from
 * the maxima of the last finished step (the initial velocities before the
 * first step): dt_ac = 0.6 h_F / (c0 + |v|max,F) (Eq. dt-relax, the step a
 * call with dt_F <= 0 takes); dt_ad = 0.25 min(h_F / |v|max,F, h_F^2 / nu)
 * (advection and viscous limit); dt_S = 0.6 min(h_S / (c_S + |v|max,S),
 * sqrt(h_S / |a|max,S)) (Eq. dts-advection; 1e300 without a solid).  The
 * automatic sub-step count is K = floor(dt_F / dt_S) + 1. */
int sphfsi_suggest_dt(sphfsi_ctx *c, double *dt_ac, double *dt_ad, double *dt_S);

/* Checkpoint (no counterpart in the paper): the whole device state of a
 * finalised context (every instance: particles, records, static lists,
 * control blocks with time, step and counters) as one host blob.
 * sphfsi_state_size gives its size; sphfsi_get_state writes it into
 * caller-owned host memory of at least that size; sphfsi_set_state restores
 * it into a context built by the same creation calls (same sizes; else
 * SPHFSI_E_INVAL and nothing changes).  Both wait for the context's work.
 * The learned sub-stepper's network is not part of the state. */
int sphfsi_state_size(sphfsi_ctx *c, int64_t *bytes);
int sphfsi_get_state(sphfsi_ctx *c, void *blob, int64_t bytes);
int sphfsi_set_state(sphfsi_ctx *c, const void *blob, int64_t bytes);

/* Neighbour sets from the device cell list at the current positions with the
 * FP64 in-support test r^2 < (2 h_F)^2 (dx*dx + dy*dy (+ dz*dz), no FMA).
 * which: 0 fluid-fluid, 1 fluid-wall, 2 fluid-solid, 3 solid-fluid.
 * Two-phase: with idx == NULL, *nnz receives the total count and ptr
 * (n_rows + 1, may be NULL) the row offsets; then call again with idx of
 * *nnz entries.  Rows in original order, columns sorted ascending. */
int sphfsi_debug_neighbors(sphfsi_ctx *c, int which, int64_t *ptr, int64_t *idx, int64_t *nnz);

/* Solid sub-step kernel selection: 0 automatic (a cluster-resident kernel
 * when the body fits one thread-block cluster of at most 16 CTAs x 128
 * particles and the device can launch it -- in 2-D with at most 24 static
 * neighbours per particle the one-thread-per-particle variant, otherwise the
 * four-lanes-per-particle variant -- else the cooperative grid kernel);
 * 1 the four-lane cluster variant where it fits; 2 always the cooperative
 * grid kernel (single-instance contexts only; SPHFSI_E_INVAL in a batch).
 * All compute the same sub-steps (Section 3.3); the choice exists to test
 * and compare them.  In a batch the cluster kernels are persistent: as many
 * clusters as fit on the device take instances from a device queue. */
int sphfsi_set_solid_path(sphfsi_ctx *c, int path);

/* Per-stage device timing.  With on != 0 every later step records CUDA
 * events on the context stream at its stage boundaries (also inside the
 * captured graph of sphfsi_run).  sphfsi_stage_times waits for the stream
 * and writes the durations in ms of the last step's 8 stages into ms[0..7]:
 * 0 step control, normal update, fluid drift, fluid and solid binning, sort
 * and records, 1 density reinitialisation, 2 momentum (a4), 3 solid-side
 * coupling force (a5), 4 continuity + drift (a6), 5 solid sub-steps (a7,
 * a8), 6 finish, 7 neighbour rows (sphfsi_tuning.list; 0 without).  Stages 3
 * and 5 run on a side stream concurrently with stages 2 and 4; finish
 * follows the join of both streams.
 * Returns the number of stages, SPHFSI_E_INVAL if n < 8, SPHFSI_E_STATE if
 * profiling is off. */
int sphfsi_set_profiling(sphfsi_ctx *c, int on);
int sphfsi_stage_times(sphfsi_ctx *c, float *ms, int n);
/* Device ms of the whole last step (first to last event of the step). */
int sphfsi_step_time(sphfsi_ctx *c, float *ms);

/* Launch shape of the pair loops and the solid kernel variant.  None of
 * these changes what is computed; the summation order of a particle's pair
 * terms follows the lane count, so results agree to rounding across
 * settings and bit for bit at equal settings. */
typedef struct {
    int32_t lanes;         /* threads per target particle in the fluid pair loops:
                              2, 4 or 8 in 2-D (default 8 below 262 144 particles in the
                              context, else 4); 4, 8 or 16 in 3-D (default 8 below 200 000
                              fluid particles in the context, else 4) */
    int32_t block;         /* threads per block of those loops: 64, 128 (default) or 256 */
    int32_t solid_variant; /* 2-D cluster sub-step kernel: 0 one thread per particle;
                              1 four lanes per particle (sphfsi_set_solid_path 1);
                              2 two threads per particle; 3 one thread per particle reading
                              the neighbours across the cluster in every phase; 4 one thread
                              per particle whose halo copies (below) are refreshed by
                              asynchronous remote stores that each CTA awaits on its own
                              mbarriers instead of cluster barriers (measured slower); 5 (a
                              single body, else as 0) one cluster barrier per sub-step instead
                              of two: each CTA also evolves copies of the particles its own
                              particles read (one extra thread each) and computes their
                              stresses itself, so only velocities cross the cluster.  0 and
                              2 keep copies of the neighbours from other CTAs in each CTA,
                              refreshed by their owners' remote stores and ordered by the
                              cluster barrier between phases, where they fit, else they read
                              across the cluster.  All compute the same values. */
    float step_ms;         /* sphfsi_autotune: device ms per step measured for this setting */
    int32_t compact;       /* fluid-fluid pair loops: 0 evaluate each pair inside the
                              candidate loop; 1 first collect each thread's in-support
                              neighbours in shared memory, then evaluate them densely
                              (default 1 in 2-D from 262 144 particles in the context, else 0) */
    int32_t tile;          /* fluid pair loops: 0 one group of lanes per target particle
                              over the whole grid; 1 one block per tile of grid cells (16 of a
                              row in 2-D, 4 in 3-D) whose neighbour records are first staged in
                              shared memory by bulk copies (default 0) */
    int32_t records;       /* binning: 0 four kernels (keys and histograms, scan, scatter, then a
                              group of lanes per non-empty cell ranks the cell's entries and
                              writes their records); 1 the same, but the groups only rank and
                              one thread per slot writes the records (one more launch); 2 the
                              four phases of 0 in one cooperative kernel with grid barriers
                              (one launch; falls back to 0 where it cannot be co-resident).
                              Default 1 from 262 144 particles in the context, else 0 */
    int32_t rows;          /* fluid pair loops without tiles: 0 visit the neighbour cells one at a
                              time; 1 a row of three cells at a time, the cell starts of the row
                              (fluid, walls, solid) loaded together: fewer dependent loads, a few
                              more instructions per candidate (default 1 below 262 144 particles
                              in the context, else 0) */
    int32_t list;          /* fluid pair loops: 0 test the candidates of the neighbour cells in
                              every loop; 1 test them once per rebuild of the pair configuration,
                              keeping each fluid particle's in-support fluid and wall neighbours in
                              a row (at most 64 in 2-D, 128 in 3-D; a fuller row falls back to the
                              cell visit for that particle), and stream the rows in momentum,
                              continuity and reinitialisation; not with tiles or cell_reach 2
                              (default 1 in 3-D from 262 144 particles in the context, else 0) */
    int32_t list_lanes;    /* threads per fluid particle of the row build: 1 (one warp per cell,
                              each candidate loaded once for the cell's particles), 8, 16 or 32
                              (default 8 in 2-D, 1 in 3-D; 0 keeps the current value); all build
                              the same rows */
} sphfsi_tuning;

/* Set or read the launch shape (SPHFSI_E_INVAL for values outside the lists). */
int sphfsi_set_tuning(sphfsi_ctx *c, const sphfsi_tuning *t);
int sphfsi_get_tuning(sphfsi_ctx *c, sphfsi_tuning *t);

/* Autotuner (no counterpart in the paper).  Times the context's own
 * workload: for each candidate setting, `steps` graph-replayed steps of size
 * dt_F (as sphfsi_run) to warm up, then `steps` timed with CUDA events.  The
 * search goes over the lane count (block 128), then the pair-loop form,
 * then neighbour rows on or off (with rows: the row build's lane count),
 * then (without rows) tiles on or off and the row form, then the block
 * size, then the
 * records form, then (2-D with a solid) the solid kernel variant, keeping the
 * fastest of each.
 * Every device allocation of the context is saved before and restored after
 * each trial and at the end, so the simulation state, time and counters are
 * exactly as before the call; the best setting stays selected and is
 * written to *best.  Needs a non-default stream, and free device memory for
 * one copy of the context's state (else SPHFSI_E_NOMEM). */
int sphfsi_autotune(sphfsi_ctx *c, double dt_F, int32_t steps, sphfsi_tuning *best);

/* Allocation-free neighbour counting.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (a framework's
 * caching allocator owns the device memory, a latency-critical loop cannot
 * take the implicit synchronisation of cudaMalloc/cudaFree, or plug-in code
 * that is only handed input and output buffers).  It allocates nothing.
 *
 * For each of the n points r (device pointer, n x dim FP64, row-major) it
 * writes to counts (device pointer, n int32) the number of other points j
 * with |r_i - r_j|^2 < (2 h)^2, h = 1.3 dp, computed in FP64 as dx*dx + dy*dy
 * (+ dz*dz) with the minimal image in x when p->periodic_x (the same test as
 * sphfsi_debug_neighbors); with periodic_x, x is first brought into
 * [x_lo, x_lo + Lx) (points already inside keep their value bit for bit),
 * so points may be given outside the period.  The cell grid follows p (dim,
 * domain box, periodic x) as a context built from p with cell_reach 1 would
 * (the counts do not depend on the cell grid; points outside the box fall
 * into its border cells).  Work is issued on cuda_stream and is
 * asynchronous.
 *
 * Scratch (cell keys, the permutation, the cell histogram) is one
 * file-scope device array sized for at most SPHFSI_NOALLOC_MAX_PARTICLES
 * points and SPHFSI_NOALLOC_MAX_CELLS cells (about 4 MB per GPU, held by
 * every GPU that loads the library until the process exits); larger inputs
 * return SPHFSI_E_CAPACITY.  The first call on a device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture.  Every call shares the one array, so calls
 * whose work overlaps on the GPU (other streams, other host threads) race:
 * serialise them.  Returns SPHFSI_E_INVAL for bad arguments (including a
 * non-finite dp, box or period) and SPHFSI_E_CAPACITY when the box holds
 * more cells of edge 2 h than the maximum; both checks run before any
 * device work. */
#define SPHFSI_NOALLOC_MAX_PARTICLES (1 << 18)
#define SPHFSI_NOALLOC_MAX_CELLS (1 << 18)
int sphfsi_neighbor_counts_noalloc(const sphfsi_params *p, int64_t n, const double *r, double dp, int32_t *counts,
                                   void *cuda_stream);

/* ---------------------------------------------------------------------
 * Learned sub-stepper building blocks (the paper has no learned form; the
 * network is the message-passing model described with sphfsi_mpnn_*).
 * ------------------------------------------------------------------- */

/* Tensor-core GEMM: C[M x N] = A[M x K] . B[N x K]^T (+ bias[N] if not
 * NULL), A and B bfloat16 (raw 16-bit patterns) row-major with K contiguous,
 * C FP32 row-major, all device pointers, 16-byte aligned.  M % 128 == 0,
 * N % 16 == 0, K % 64 == 0 (callers pad with zeros), else SPHFSI_E_INVAL.
 * Asynchronous on cuda_stream; the FP32 accumulation order over K is fixed
 * (ascending chunks of 16). */
int sphfsi_gemm_bf16(const void *A, const void *B, const float *bias, float *C, int64_t M, int64_t N, int64_t K,
                     void *cuda_stream);

/* Status of the bounded tensor-core waits since the last reset: *status
 * bit 0 set if one ran out (the affected outputs were not written). */
int sphfsi_tc_status(int32_t *status, int32_t reset);

/* The graph the learned sub-stepper works on, for the selected instance in
 * original order: ptr (n_solid + 1), idx, w (pairs_ss entries each, see
 * sphfsi_info) and g (pairs_ss x dim): the static reference neighbour list of
 * the solid with w_ab = V0 W(|r0_a - r0_b|, h_S) and g_ab = h_S V0 grad0_a W_ab.
 * Host pointers; any may be NULL. */
int sphfsi_solid_graph(sphfsi_ctx *c, int64_t *ptr, int64_t *idx, double *w, double *g);

/* Learned sub-stepper (no counterpart in the paper): every later step runs,
 * after the coupling force, the network of sphfsi_mpnn_* (parameters theta)
 * on each body's graph with the features
 *   [u / s_u, v / s_v, (F - I) / s_H (row-major), f^F / s_f, constrained, dt_F / s_t]
 * (u = r - r0; scales = {s_u, s_v, s_f, s_t, s_du, s_dv, s_H}) and proposes
 *   du = dt_F v + s_du out[0:dim],  dv = dt_F (f^F / m + g) + s_dv out[dim:2 dim]
 * (0 for constrained particles).  The proposal of an instance is accepted
 * when its residual
 *   R = |m (v' - v) - dt_F (f_int(r + du/2) + f^F + m g)| / |m v'|
 * (norms over the free particles; f_int one plain force evaluation with F
 * from the positions, Eq. correctmatrix) is at most tol: positions,
 * velocities, F (from the new positions) and the time averages
 * (du / dt_F, dv / dt_F) are then committed and the K sub-steps skipped;
 * otherwise the plain sub-steps run from the unchanged state.  tol < 0
 * switches the learned path off. */
int sphfsi_set_learned(sphfsi_ctx *c, const float *theta, const double *scales, double tol);

/* The network's input rows of the selected instance from the last step that
 * ran the learned sub-stepper (the feature rows described with
 * sphfsi_set_learned, 64 FP32 columns, zero-padded), in original particle
 * order: x receives n_solid x 64 floats (host or device pointer).  For
 * checking training features against the ones a step feeds the network.
 * SPHFSI_E_STATE before sphfsi_set_learned. */
int sphfsi_get_learned_features(sphfsi_ctx *c, float *x);

/* Message-passing network over one body's static neighbour graph (the
 * learned solid sub-stepper).  With x the N x 64 feature matrix (FP32):
 *   h = silu(x W_enc^T + b_enc)                                 (N x 128)
 *   3 times: z = [h, sum_b w_ab (h_b - h_a), sum_b g_ab,k (h_b - h_a)]_{k<dim}
 *            h = h + silu(z W_l^T + b_l)                (W_l: 128 x 128 (2+dim))
 *   out = h W_dec^T + b_dec                                      (N x 16)
 * Parameters are one FP32 vector [W_enc (128x64), b_enc, (W_l, b_l) x 3,
 * W_dec (16x128), b_dec], weights row-major [out][in]; its length is
 * sphfsi_mpnn_n_params(dim).  GEMMs run on the tensor cores with bfloat16
 * operands and FP32 accumulation; everything else in FP32.
 *
 * The graph (ptr n+1, idx nnz, w nnz, g nnz x dim; host or device) must be a
 * symmetric relation without self entries, with w_ab = w_ba and
 * g_ab = -g_ba (one body at one spacing), else SPHFSI_E_INVAL.  The context
 * holds `replicas` copies of the graph side by side, so a batch of replicas
 * samples is one network evaluation over replicas x n nodes (node r n + a is
 * node a of sample r).  All work is issued on cuda_stream. */
typedef struct sphfsi_mpnn sphfsi_mpnn;
int64_t sphfsi_mpnn_n_params(int32_t dim);
int sphfsi_mpnn_create(sphfsi_mpnn **out, int32_t dim, int64_t n, int64_t nnz, const int64_t *ptr,
                       const int64_t *idx, const double *w, const double *g, int32_t replicas, void *cuda_stream);
/* Load parameters (resets the Adam moments and step count) / read them. */
int sphfsi_mpnn_set_params(sphfsi_mpnn *m, const float *theta);
int sphfsi_mpnn_get_params(sphfsi_mpnn *m, float *theta);
/* out (replicas n x 16, may be NULL) = network(x (replicas n x 64)). */
int sphfsi_mpnn_forward(sphfsi_mpnn *m, const float *x, float *out);
/* After sphfsi_mpnn_forward: grad (n_params) = gradient of
 * sum(dout * out) with respect to the parameters. */
int sphfsi_mpnn_backward(sphfsi_mpnn *m, const float *dout, float *grad);
/* One training step: forward on x, loss = mean over the masked nodes (mask
 * NULL = all) of the squared error of the first 2 dim outputs against
 * target (replicas n x 16), backward, one Adam step (b1 0.9, b2 0.999,
 * eps 1e-8, learning rate lr).  *loss (may be NULL) receives the loss. */
int sphfsi_mpnn_train_step(sphfsi_mpnn *m, const float *x, const float *target, const uint8_t *mask, float lr,
                           float *loss);
/* Wait for the context's stream; SPHFSI_E_TIMEOUT if a bounded tensor-core
 * wait ran out. */
int sphfsi_mpnn_sync(sphfsi_mpnn *m);
void sphfsi_mpnn_destroy(sphfsi_mpnn *m);

void sphfsi_destroy(sphfsi_ctx *c);
const char *sphfsi_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
