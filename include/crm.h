/*
 * crm.h -- C ABI of the B300 (sm_103a) SPH continuum terrain library.
 *
 * The library advances the per-step particle loop of the continuum
 * representation model of "A Physics-Based Continuum Model for Versatile,
 * Scalable, and Fast Terramechanics Simulation" (arXiv 2507.05643):
 *   - cell binning of SPH particles and boundary (BCE) markers by key sort and
 *     the neighbour sets of Sec. 3.1 / Alg. 1,
 *   - the pairwise continuity, momentum (stress divergence + artificial
 *     viscosity) and Jaumann stress-rate sums of Sec. 2.1-2.2,
 *   - the explicit-midpoint (RK2) update of Sec. 2.2 and the cohesive return
 *     map of Sec. 2.3, restricted to the active-domain particles of Sec. 3.2,
 *   - the BCE extrapolation and body force/torque of Sec. 2.4.
 *
 * Conventions
 *   - Every call returns an int status: CRM_OK (0) or a negative CRM_E* code.
 *     No C++ exception crosses the ABI.  crm_last_error() gives a message.
 *   - A terrain handle is opaque, owns all of its device memory, and is bound
 *     to one CUDA stream given at creation (NULL = the legacy default
 *     stream).  A handle is not thread-safe; use one handle per host thread.
 *   - Host arrays passed in are copied before the call returns; host arrays
 *     passed out are written before the call returns (such calls synchronise
 *     the stream).  crm_step() only enqueues work; device-side failures
 *     (capacity, escaped particle, non-finite state, device wait timeout) are
 *     latched on the device and reported by the next synchronising call
 *     (crm_sync, crm_get_*).
 *   - Units are SI.  Stresses are 6-vectors (xx, yy, zz, xy, xz, yz),
 *     compression negative.  Poses are (x, y, z, qw, qx, qy, qz); twists are
 *     (vx, vy, vz, wx, wy, wz) with the angular velocity in the world frame.
 *   - Particle indices in the query calls are the order of insertion: SPH
 *     particles in crm_add_sph order, markers in crm_add_fixed_bce /
 *     crm_add_rigid_body order (fixed markers and body markers share one
 *     marker index space, in call order).
 */
#ifndef CRM_H
#define CRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRM_OK          0
#define CRM_EINVAL     -1   /* bad argument (null pointer, size, value range) */
#define CRM_ENOMEM     -2   /* a device or host allocation failed */
#define CRM_ECAPACITY  -3   /* a neighbour list exceeded max_neighbors */
#define CRM_EESCAPED   -4   /* a particle or marker left the grid domain */
#define CRM_ENONFINITE -5   /* the state became non-finite */
#define CRM_ETIMEOUT   -6   /* a bounded device-side wait gave up */
#define CRM_ECUDA      -7   /* a CUDA runtime call failed */
#define CRM_ESTATE     -8   /* call made in the wrong state (e.g. add after step) */

#define CRM_AV_NONE        0
#define CRM_AV_BILATERAL   1  /* Eq. artificial_viscosity_bilateral */
#define CRM_AV_UNILATERAL  2  /* Eq. artificial_viscosity_unilateral */

#define CRM_KERNEL_CUBIC    0  /* cubic spline, support 2h (Sec. 3.1) */
#define CRM_KERNEL_WENDLAND 1  /* quintic Wendland, support 2h (Sec. 3.1):
                                  W = 21/(16 pi h^3) (1 - q/2)^4 (2q + 1) */

#define CRM_DOF_RX 8   /* angular velocity components (world frame), integrated */
#define CRM_DOF_RY 16  /* from I w' = T - w x I w when set (crm_set_body_inertia) */
#define CRM_DOF_RZ 32
#define CRM_DOF_X 1
#define CRM_DOF_Y 2
#define CRM_DOF_Z 4

/* Material and numerical parameters (Sec. 2.1-2.3, Table tab:sph_params,
 * Sec. 3.1-3.2).  Fill with crm_default_params() and override. */
typedef struct crm_params {
    double rho0;           /* reference (bulk) density, kg/m^3, > 0 */
    double E, nu;          /* Young's modulus (Pa, > 0), Poisson ratio in (-1, 0.5):
                              G = E / (2(1+nu)), K = E / (3(1-2nu)) */
    double mu_s, mu_2;     /* static and limiting friction coefficients of mu(I);
                              mu_s = tan(friction angle) (Sec. 4.4); mu_2 = mu_s
                              gives the rate-independent cohesive cone */
    double I0, grain_d;    /* mu(I) constants: I0 and particle diameter d (m) */
    double cohesion;       /* cohesive intercept c of the yield cone, Pa, >= 0 */
    double d0, h;          /* initial spacing and smoothing length (m); cells are 2h */
    int32_t kernel;        /* CRM_KERNEL_CUBIC or CRM_KERNEL_WENDLAND */
    int32_t av_mode;       /* CRM_AV_* */
    double av_gamma;       /* gamma_a of the artificial viscosity */
    double av_xi2_over_h2; /* xi^2 / h^2 in the viscosity denominator (default 0.01) */
    double gravity[3];     /* body force per unit mass, m/s^2 */
    int32_t ps_freq;       /* neighbour lists rebuilt every ps_freq steps (Alg. 2), >= 1 */
    int32_t max_neighbors; /* per-particle neighbour list capacity, 8..1024 */
    double domain_min[3];  /* axis-aligned grid extent; every particle and marker */
    double domain_max[3];  /* must stay inside it (else CRM_EESCAPED) */
    double growth;         /* active-set capacity growth factor G (Sec. 3.2), >= 1 */
    double shrink_ratio;   /* shrink threshold S (Sec. 3.2), in (0, 1] */
    int32_t shrink_interval; /* shrink check interval S_I in steps (Sec. 3.2), >= 1 */
    int32_t pair_lanes;    /* lanes per fluid particle in the pair kernels on exact lists:
                              1, 2, 4, or 0 = the library default (4 while four threads
                              per particle fit the GPU's resident threads, else 2); a
                              pure speed knob (crm_batch_autotune picks it per terrain) */
    double skin;           /* Verlet skin as a fraction of 2h, in [0, 1): with skin > 0
                              the cell sort and the 27-cell search run with radius
                              2h (1 + skin) only when some particle has moved skin * h
                              since the last search, and at every Alg. 2 rebuild the
                              first-stage kernels filter those lists down to the exact
                              2h sets (the same sets a fresh search gives) while they
                              compute the stage.  0 = a fresh 2h search every rebuild.
                              With active boxes the Alg. 3 working set is gathered
                              4 skin h beyond the boxes grown by 2h and kept until the
                              search is due (also when a point of a grown box may
                              have moved 0.95 of that margin); every step re-flags it
                              against the current boxes. */
} crm_params;

typedef struct crm_terrain crm_terrain;

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int crm_version(void);

/* Human-readable name of a status code (static string). */
const char *crm_status_string(int status);

/* Defaults: rho0 1700, E 1e6, nu 0.3, mu_s = mu_2 = tan 30 deg, I0 0.08,
 * grain_d 0.002, c 0, d0 0.01, h 0.012, cubic kernel, unilateral AV 0.02,
 * xi^2 = 0.01 h^2, g = (0, 0, -9.81), ps_freq 1, max_neighbors 96, domain
 * [0,1]^3, G 1.2, S 0.75, S_I 50 (Sec. 3.2), skin 0.1. */
void crm_default_params(crm_params *p);

/* Create a terrain.  `cuda_stream` is a cudaStream_t (NULL for the default
 * stream); all work is ordered on it.  Validates the parameters (CRM_EINVAL).
 * On success *out receives the handle; on failure *out is NULL. */
int crm_create(const crm_params *p, void *cuda_stream, crm_terrain **out);

/* Release every device and host resource of the handle (NULL is a no-op). */
int crm_destroy(crm_terrain *t);

/* Message of the last error on this handle ("" if none).  Valid until the
 * next call on the handle. */
const char *crm_last_error(const crm_terrain *t);

/* Add n SPH particles (Sec. 2.2).  xyz: n*3 positions (required); vel: n*3
 * velocities, stress6: n*6 stresses, rho: n densities -- each nullable
 * (zero velocity, zero stress, rho0).  Host arrays, copied.  Only before the
 * first crm_step / crm_eval_rates (else CRM_ESTATE).  A terrain holds fewer than
 * 2^29 SPH particles and markers together (the first step returns CRM_EINVAL
 * otherwise: a slot's id keeps three flag bits). */
int crm_add_sph(crm_terrain *t, int64_t n, const double *xyz, const double *vel,
                const double *stress6, const double *rho);

/* Add n fixed BCE wall markers at world positions xyz (n*3), Sec. 2.4. */
int crm_add_fixed_bce(crm_terrain *t, int64_t n, const double *xyz);

/* Add a rigid body carrying n_markers BCE markers given in the body frame
 * (marker_xyz_local, n*3), with pose[7], twist[6], mass (kg, > 0) and a DOF
 * mask: bit k of CRM_DOF_X/Y/Z set = that linear velocity component is
 * integrated from the soil force (plus the external load) and gravity by
 * symplectic Euler; bit k of CRM_DOF_RX/RY/RZ set = that angular velocity
 * component is integrated from I w' = T - w x I w (needs crm_set_body_inertia);
 * unset components are prescribed.  The body's pose is taken at its centre of
 * mass.  *body_id receives the body index (0, 1, ... in call order).  The
 * paper couples bodies through a multibody solver (Sec. 2.4); this built-in
 * 6-DOF update is the library's own stand-in for it. */
int crm_add_rigid_body(crm_terrain *t, int64_t n_markers, const double *marker_xyz_local,
                       const double pose[7], const double twist[6], double mass,
                       int32_t dof_mask, int32_t *body_id);

/* Prescribe a body's pose and twist (the FSI exchange of Sec. 2.4): takes
 * effect at the next step.  Host arrays, copied (enqueued on the stream).  The
 * quaternion is normalised; CRM_EINVAL if its norm is outside (0.5, 2) or an
 * entry is not finite. */
int crm_set_body_motion(crm_terrain *t, int32_t body, const double pose[7],
                        const double twist[6]);

/* Principal moments of inertia (kg m^2, body frame, all > 0) of a body; needed
 * before the first step when any angular DOF of the body is free.  Host array,
 * copied; CRM_EINVAL on a bad body or a non-positive moment. */
int crm_set_body_inertia(crm_terrain *t, int32_t body, const double inertia[3]);

/* External force (N) and torque about the centre (N m), world frame, added to
 * the soil wrench in the body update of every following step (e.g. a drive
 * torque); zero by default.  Host arrays, copied. */
int crm_set_body_load(crm_terrain *t, int32_t body, const double force[3],
                      const double torque[3]);

/* Current pose and twist of a body (synchronises the stream). */
int crm_get_body_state(crm_terrain *t, int32_t body, double pose[7], double twist[6]);

/* Attach an active box (Sec. 3.2) to `body`: an oriented box with the given
 * half extents and centre offset in the body frame.  Once any box exists the
 * terrain runs in active-domain mode: after t_delay (the largest delay of any
 * box) only SPH particles inside a box are integrated, particles within 2h of
 * a box are read-only neighbours and the rest are frozen. */
int crm_add_active_box(crm_terrain *t, int32_t body, const double half_extents[3],
                       const double offset[3], double t_delay);

/* Advance n_steps steps of size dt (Sec. 2.2 RK2 with the return map of
 * Sec. 2.3 at the end of each step).  Enqueues on the stream and returns. */
int crm_step(crm_terrain *t, double dt, int32_t n_steps);

/* Wait for the stream and report any latched device-side failure.  After
 * CRM_ETIMEOUT (a bounded device wait gave up) the terrain is frozen: the
 * kernels enqueued after the failed wait returned at once, its state is
 * unspecified, and the calls that advance or evaluate it (crm_step,
 * crm_cosim_step, crm_eval_rates, the adjoint calls) return CRM_ESTATE until
 * crm_load_state restores a checkpoint. */
int crm_sync(crm_terrain *t);

/* Copy the SPH state out in insertion order: xyz (double, n*3), vel (n*3),
 * stress6 (n*6), rho (n); each nullable.  cap = room in particles; fewer
 * than n particles of room is CRM_EINVAL.  *n_out (nullable) receives n. */
int crm_get_particles(crm_terrain *t, int64_t cap, double *xyz, float *vel, float *stress6,
                      float *rho, int64_t *n_out);

/* Body force and torque (about the body centre) of the last step, FP64. */
int crm_get_body_wrench(crm_terrain *t, int32_t body, double force[3], double torque[3]);

/* Global FP64 diagnostics of the SPH particles (every particle of the terrain,
 * Active or not; the precision pattern: FP32 state, FP64 global sums), with the
 * particle mass m = rho0 d0^3 of the readings (Sec. 2.2):
 *   out[CRM_DIAG_COUNT]     number of SPH particles
 *   out[CRM_DIAG_MASS]      sum m
 *   out[CRM_DIAG_VOLUME]    sum m / rho (rho the particle's density)
 *   out[CRM_DIAG_MOMENTUM]  sum m u (3 entries, x y z)
 *   out[CRM_DIAG_ANGULAR]   sum m x (x) u about the world origin (3 entries), x the
 *                           absolute FP64 position rebuilt from the cell-relative one
 *   out[CRM_DIAG_KINETIC]   sum m |u|^2 / 2
 * out: caller-owned host array of CRM_NUM_DIAG doubles.  Summed on the device in
 * FP64 in a fixed order: the same state gives the same bits.  Before the first
 * step the sums come from the host copies of the inputs.  Synchronises the
 * terrain's stream.  CRM_EINVAL for a null handle or output. */
#define CRM_DIAG_COUNT 0
#define CRM_DIAG_MASS 1
#define CRM_DIAG_VOLUME 2
#define CRM_DIAG_MOMENTUM 3
#define CRM_DIAG_ANGULAR 6
#define CRM_DIAG_KINETIC 9
#define CRM_NUM_DIAG 10
int crm_get_diagnostics(crm_terrain *t, double *out);

/* Active / extended-active SPH particles and BCE markers processed in the
 * last step (without active boxes every SPH particle is active). */
int crm_get_counts(crm_terrain *t, int64_t *n_active, int64_t *n_extended, int64_t *n_bce);

/* One co-simulation exchange with a multibody code (the FSI loop of Sec.
 * 2.4): set every body's motion from pose_in (n_bodies*7) and twist_in
 * (n_bodies*6) -- both or neither (nullptr: keep the current motion) -- then
 * advance n_steps steps of dt (0: none), then return every body's soil wrench
 * (wrench_out, n_bodies*6, as crm_get_body_wrench), pose and twist (each
 * nullable), with a single synchronisation (the transfers go through pinned
 * staging kept with the terrain; an exchange of one step with a new motion
 * replays one graph holding the upload, the step and the read-back).  Errors as
 * crm_set_body_motion, crm_step and crm_sync. */
int crm_cosim_step(crm_terrain *t, const double *pose_in, const double *twist_in, double dt,
                   int32_t n_steps, double *wrench_out, double *pose_out, double *twist_out);

/* Evaluate the rates f(y) at the current state without advancing it (the
 * first RK2 stage: rebuilds the lists, extrapolates the BCE state and sums the
 * pairs).  Outputs in insertion order, each nullable: drho (n_sph),
 * dvel (n_sph*3), dstress (n_sph*6), marker_acc (n_markers*3; every marker),
 * marker_vel (n_markers*3) and marker_stress (n_markers*6): the extrapolated
 * marker state.  cap_sph / cap_markers = room in elements of each kind. */
int crm_eval_rates(crm_terrain *t, int64_t cap_sph, float *drho, float *dvel, float *dstress,
                   int64_t cap_markers, float *marker_acc, float *marker_vel,
                   float *marker_stress);

/* The neighbour lists of the last rebuild in CSR form over insertion indices
 * (SPH particles 0..n_sph-1, then markers n_sph..): offset[n_sph+n_markers+1],
 * list[nnz] (ascending within a row).  cap = room in list; *nnz receives the
 * total.  Rows of inactive particles are empty. */
int crm_get_neighbors(crm_terrain *t, int64_t cap, int64_t *offset, int32_t *list,
                      int64_t *nnz);

/* Bytes needed by crm_save_state. */
int crm_state_bytes(crm_terrain *t, size_t *bytes);

/* Checkpoint: copy the complete dynamic state (particles, bodies, step
 * counter) into a caller device buffer of `cap` bytes; *used receives the
 * size.  crm_load_state restores it into a terrain built from the same
 * inputs. */
int crm_save_state(crm_terrain *t, void *dev_buf, size_t cap, size_t *used);
int crm_load_state(crm_terrain *t, const void *dev_buf, size_t used);

/* ---- Reverse sweep (adjoint) --------------------------------------------
 * The paper differentiates nothing; these calls are this library's
 * hand-derived adjoint of the discrete method of Sec. 2.1-2.4 (pair sums,
 * Jaumann rate, artificial viscosity, BCE extrapolation, return map of Sec. 2.3
 * with mu(I), midpoint step, body update of Sec. 2.4), in FP32 on the device with FP64 sums of the parameter and body
 * adjoints.  Neighbour lists are those of the forward evaluation, held fixed,
 * and every branch is the one the forward took (the adjoint is that of the
 * piecewise-smooth map at the evaluated point).  Bodies: centre, velocity,
 * acceleration, orientation, angular velocity and acceleration, through the
 * markers' kinematics, the wrench and the 6-DOF update (Euler's equations in the
 * world frame).  Not differentiated (CRM_EINVAL): active domains; in runs also
 * a Verlet skin or ps_freq > 1.  With mu(I) off (mu_2 = mu_s) the gradient for
 * mu_s is the one with mu_2 moving along (mu_2's is zero). */

/* Indices of the parameter gradients. */
#define CRM_GRAD_E          0
#define CRM_GRAD_NU         1
#define CRM_GRAD_RHO0       2   /* with the particle mass m = rho0 d0^3 and the
                                 * marker density following rho0; the particles'
                                 * own densities are state */
#define CRM_GRAD_MU_S       3
#define CRM_GRAD_COHESION   4
#define CRM_GRAD_AV_GAMMA   5
#define CRM_GRAD_MU_2       6
#define CRM_GRAD_I0         7
#define CRM_GRAD_GRAIN_D    8
#define CRM_NUM_GRADS       9
#define CRM_BODY_GRADS      18  /* per body: centre 3, velocity 3, acceleration 3,
                                 * orientation 3, angular velocity 3, angular
                                 * acceleration 3 */

/* Vector-Jacobian product of crm_eval_rates at the current state.  Inputs,
 * insertion order, each nullable (= zero): l_drho (n_sph), l_dvel (n_sph*3),
 * l_dstress (n_sph*6), l_macc (n_markers*3, the marker accelerations that
 * crm_eval_rates returns).  Outputs, each nullable: the adjoints of the SPH
 * positions (g_xyz, n_sph*3), velocities (g_vel), stresses (g_stress, n_sph*6,
 * xx yy zz xy xz yz as independent entries), densities (g_rho, n_sph); of each
 * body's centre, linear velocity, linear acceleration, orientation (as a
 * world-frame rotation vector: the gradient with respect to a small turn
 * applied to the body), angular velocity and angular acceleration (g_body,
 * CRM_BODY_GRADS per body, in that order);
 * of the parameters (g_params, CRM_NUM_GRADS).  The output of
 * crm_eval_rates is sum(l . rates); the returned adjoints are its gradient.
 * Rebuilds the lists like crm_eval_rates; allocates its workspace once (kept
 * with the terrain).  Synchronises the stream. */
int crm_eval_rates_vjp(crm_terrain *t, int64_t cap_sph, const float *l_drho, const float *l_dvel,
                       const float *l_dstress, int64_t cap_markers, const float *l_macc,
                       double *g_xyz, double *g_vel, double *g_stress, double *g_rho,
                       double *g_body, double *g_params);

/* Differentiable run, forward half: n_steps steps of dt (as crm_step) with a
 * checkpoint of the state every `every` steps and after the last, and the
 * bodies after each step; every = 0 keeps the whole run's tape resident
 * instead (no checkpoints, and no re-run in the backward half: about
 * 35 MB per step for 30,000 particles -- HBM traded for time).  wrench_hist (n_steps*n_bodies*6: the soil force and
 * torque of each step, as crm_get_body_wrench) and pose_hist
 * (n_steps*n_bodies*7: the pose after each step) are nullable.  Device memory:
 * the checkpoints (ceil(n_steps / every) + 1 states of crm_state_bytes) and the
 * tape of one segment (`every` steps of stage arrays and lists), freed by the
 * next call or crm_destroy.  Synchronises the stream. */
int crm_adjoint_forward(crm_terrain *t, double dt, int64_t n_steps, int32_t every,
                        double *wrench_hist, double *pose_hist);

/* Differentiable run, backward half: for an objective J of the recorded run
 * with dJ / d wrench given as l_wrench (n_steps*n_bodies*6), dJ / d centre
 * after each step as l_center (n_steps*n_bodies*3), and dJ / d final SPH state
 * as l_xyz, l_vel (n_sph*3), l_stress (n_sph*6), l_rho (n_sph), insertion
 * order, all nullable (= zero), returns dJ / d parameters (g_params,
 * CRM_NUM_GRADS) and the adjoints of the run's initial state: SPH positions,
 * velocities, stresses, densities (insertion order, as crm_eval_rates_vjp) and
 * bodies (g_body, CRM_BODY_GRADS per body, as crm_eval_rates_vjp: their state
 * at the start; a prescribed velocity is constant over the run, so its entry is
 * the gradient with respect to it);
 * each output nullable.  Re-runs every segment from its checkpoint (with
 * direct launches) and sweeps it in reverse; leaves the terrain in the state
 * after the recorded run.  CRM_ESTATE without a recorded run.  Synchronises
 * the stream. */
int crm_adjoint_backward(crm_terrain *t, const double *l_wrench, const double *l_center,
                         const double *l_xyz, const double *l_vel, const double *l_stress,
                         const double *l_rho, double *g_params, double *g_xyz, double *g_vel,
                         double *g_stress, double *g_rho, double *g_body);

/* Array-capacity policy of ManageArrayMemory (Sec. 3.2): the capacity that
 * follows `cap` when `need` elements are required at step `step`: grown to
 * ceil(need * growth) when need > cap; shrunk to need when step is a multiple
 * of shrink_interval and need / cap < shrink_ratio; else unchanged.  Pure
 * host function (the active-domain stepper applies it to the working set).
 * CRM_EINVAL on a null output or out-of-range argument. */
int crm_capacity_policy(int64_t need, int64_t cap, int64_t step, double growth,
                        double shrink_ratio, int32_t shrink_interval, int64_t *new_cap);

/* Lanes per fluid particle in the exact-list pair kernels (1, 2 or 4; 0 = the
 * default): a speed knob with no effect on the method (the sums of a particle
 * are split between the lanes and combined, so only their order changes). */
int crm_set_pair_lanes(crm_terrain *t, int32_t lanes);

/* Cell tiles of the sort order (Sec. 3.1 steps 1-2): cells are keyed tile by
 * tile, tiles of nx x ny x nz cells (powers of two up to 8 x 4 x 4; 1 x 1 x 1 =
 * the row-major order c = (z Y + y) X + x), so that consecutive sorted slots
 * form compact 3-D pieces of the terrain.  Takes effect at the next step (which
 * re-sorts).  A speed knob with no effect on the method: neighbour sets are
 * unchanged, only the slot order and the order of the pair sums. */
int crm_set_cell_tile(crm_terrain *t, int32_t nx, int32_t ny, int32_t nz);

/* Comparison layout for the precision pattern (a test hook): on = 1 stores
 * every position as an absolute FP32 coordinate would be stored -- the inputs
 * and, after every stage, each SPH particle's and BCE marker's position are
 * rounded to the nearest FP32 value of the absolute coordinate -- so that a run
 * shows what the cell-relative FP32 layout (the default) avoids: the spacing
 * of FP32 values grows with the distance from the origin (4.9e-4 m at 5 km).
 * Before the first step only (CRM_ESTATE after); CRM_EINVAL for other values. */
int crm_debug_absolute_fp32(crm_terrain *t, int32_t on);

/* Test hook of the failure detection for device-side waits (CRM_ETIMEOUT), on
 * the current device: on = 1 makes every look-back scan (the cell sort of a
 * terrain, its active-set compaction, the stateless binning) started from now
 * on hold back the prefix of its first tile and give up each wait after 1,000
 * polls, so the waits of its later tiles run out and report the timeout --
 * nothing hangs and nothing faults, every wait being bounded; on = 0 restores
 * normal operation.  Scans of a single tile (4,096 cells or fewer) have no
 * wait.  CRM_EINVAL for other values, CRM_ECUDA if the device copy fails. */
int crm_debug_wait_fault(int32_t on);


/* ------------------------------------------------------------------------
 * Batches (an ensemble of independent terrains, e.g. many single-wheel bins of
 * uneven size; the paper runs one terrain at a time, this is the library's own
 * addition).  Two forms:
 *   - streams (the default): each member runs on its own non-default CUDA
 *     stream (members that share a stream run one after the other); a batch step
 *     enqueues one step of every member on its stream (one replayed step graph
 *     each), so members on different streams run concurrently, bracketed by a
 *     fork from and a join to the batch's stream;
 *   - persistent (crm_batch_set_persistent): one CUDA graph per batch step on
 *     the batch's stream: every member's search decision and gated cell search
 *     as parallel branches, then one persistent launch per stage over all
 *     members (marker state, pair sums of stage 1, midpoint marker state, pair
 *     sums of stage 2 beside the wrench pass and the body updates) whose blocks
 *     take the members' blocks off a work queue; the per-member arithmetic is
 *     that of the members' own steps, so both forms give the same bits.
 * The batch does not own its members. */
typedef struct crm_batch crm_batch;

/* Batch of n members (distinct handles, each on a non-default stream) joined on
 * `stream` (nullable: the legacy default stream).  CRM_EINVAL on a null or
 * repeated member or a member on the legacy default stream. */
int crm_batch_create(int32_t n, crm_terrain *const *members, void *stream, crm_batch **out);

/* n_steps steps of every member, member i with time step dt[i]; step-major
 * order (step k of all members is enqueued before any step k + 1).  Returns the
 * first member error. */
int crm_batch_step(crm_batch *b, const double *dt, int32_t n_steps);

/* Per-member tuning of crm_set_pair_lanes (1, 2, 4) and crm_set_cell_tile
 * (1 x 1 x 1 or 4 x 2 x 2 cells): each member runs 1 + trial_steps steps with
 * each of the six choices, timed on its own stream, and keeps the fastest; the
 * trial steps are ordinary steps (the simulation advances).  choice (nullable,
 * n entries) receives the picks as lanes | nx << 4 | ny << 8 | nz << 12.
 * Synchronises the members' streams. */
int crm_batch_autotune(crm_batch *b, const double *dt, int32_t trial_steps, int32_t *choice);

/* Select the form of crm_batch_step: on = 1 persistent, 0 streams (the
 * default).  The persistent form needs every member with a Verlet skin
 * (skin > 0), ps_freq = 1 and no active boxes (crm_batch_step returns
 * CRM_EINVAL otherwise); its graph is built at the first step and rebuilt
 * when the time steps or a member's tuning change.  CRM_EINVAL for a null
 * batch or another value of on. */
int crm_batch_set_persistent(crm_batch *b, int32_t on);

int crm_batch_destroy(crm_batch *b);

/* Per-kernel launch counts and CUDA-event timings of one handle (for
 * measurement).  Kernel ids 0..CRM_NUM_KERNELS-1, names from crm_kernel_name:
 * keys, scan, scatter, reorder, neighbors (cell search), compact (markers with
 * fluid in reach), bce (with the body wrench and update), pair_stage1,
 * pair_stage2 (with a skin, the first-stage kernels after a rebuild also filter
 * the exact lists), skin (search decision, copy-back and, with active boxes, the
 * per-step activity flags), export, adjoint (the
 * reverse-sweep kernels of crm_eval_rates_vjp and crm_adjoint_backward). */
#define CRM_NUM_KERNELS 12
typedef struct crm_profile {
    int64_t launches[CRM_NUM_KERNELS]; /* kernels enqueued since the last reset */
    double ms[CRM_NUM_KERNELS];        /* summed event-timed durations (timing on) */
    int64_t steps;                     /* steps enqueued since the last reset */
    int64_t rebuilds;                  /* neighbour-list rebuilds since the last reset */
} crm_profile;

/* Name of kernel id k (static string; "" when out of range). */
const char *crm_kernel_name(int32_t k);

/* Zero the counters.  timing != 0: from now on every kernel launch is
 * bracketed by two CUDA events recorded on the handle's stream. */
int crm_profile_reset(crm_terrain *t, int32_t timing);

/* Synchronise the stream and return the counters (and the summed event
 * durations of the launches timed since the reset). */
int crm_profile_read(crm_terrain *t, crm_profile *out);

/* Stateless cell binning of n points (Sec. 3.1 steps 1-3: hash, sort,
 * cellStart/cellEnd).  All pointers are device pointers.
 *   xyz        n*3 floats, coordinates relative to the grid origin (m)
 *   cell_size  edge of a cubic cell (2h in the method), > 0
 *   dims       grid size in cells (X, Y, Z), each >= 1, product < 2^31
 *   cell_out   n uint32: c = z (Y X) + y X + x of each point's cell; points
 *              outside the grid are clamped into the nearest boundary cell
 *   perm_out   n uint32: the point stored at sorted slot s is perm_out[s];
 *              the sort is stable (equal cells keep ascending input order)
 *   cell_start_out  X*Y*Z + 1 uint32: the points of cell c occupy sorted
 *              slots [cell_start[c], cell_start[c+1]) (cellStart/cellEnd of
 *              the paper folded into one array)
 *   scratch    caller buffer of at least crm_bin_scratch_bytes(n, X*Y*Z)
 *              bytes, 256-byte aligned; its contents are overwritten
 * Enqueues on `cuda_stream` (NULL = default stream) and returns without
 * synchronising.  CRM_EINVAL for null pointers, n < 0, n >= 2^31, a
 * non-positive cell size, a bad grid, or too small a scratch buffer.
 * Cost: O(n + X*Y*Z) per call for any distribution of the points over the cells
 * (the sort is a least-significant-digit radix sort, one pass per 8 bits of the
 * largest cell index).  Device-side failure: a bounded wait of the scans that
 * gives up leaves cell_start_out[X*Y*Z] = 0xFFFFFFFF (a successful call leaves n
 * there) and the other outputs unspecified; the call itself has returned
 * CRM_OK by then, so a caller that must detect it reads that entry. */
size_t crm_bin_scratch_bytes(int64_t n, int64_t ncell);
int crm_bin_points(const float *xyz, int64_t n, float cell_size, const int32_t dims[3],
                   uint32_t *cell_out, uint32_t *perm_out, uint32_t *cell_start_out,
                   void *scratch, size_t scratch_bytes, void *cuda_stream);

/* crm_bin_points without a scratch argument, for callers that cannot
 * allocate device memory when they bin (code in a host callback or a
 * real-time loop where cudaMalloc would block or is not allowed, or a caller
 * whose device memory is entirely owned by its own allocator).  The paper has
 * no counterpart: this is a packaging of the same binning.
 *   Arguments, outputs and results are those of crm_bin_points.
 *   Limits: n <= 1,048,576 points and X*Y*Z <= 1,048,575 cells; larger
 *   inputs return CRM_EINVAL (with a message on stderr) -- use
 *   crm_bin_points with a caller buffer instead.
 *   Scratch: one built-in device array of 22 MiB, shared by every call on a
 *   device and held by every GPU that loads the library until the process
 *   exits.  Each call clears the parts that must start at zero, so results
 *   never depend on the previous call; but calls whose work can overlap on a
 *   GPU (different streams, or host threads) race on that array: serialise
 *   them.
 *   Set-up: the first call on each device -- and the first call after the
 *   device's context was reset -- looks up the array's device address with
 *   that device current (cudaGetSymbolAddress); make that call before any
 *   stream capture.
 *   Device-side failure: as crm_bin_points (cell_start_out[X*Y*Z] =
 *   0xFFFFFFFF).
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
int crm_bin_points_noalloc(const float *xyz, int64_t n, float cell_size, const int32_t dims[3],
                           uint32_t *cell_out, uint32_t *perm_out, uint32_t *cell_start_out,
                           void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CRM_H */
