/*
 * hweno.h - C ABI of the GB300 (sm_103a) L-HWENO library.
 *
 * The library advances u_t + f(u)_x (+ g(u)_y) = 0 together with its
 * derivative equations v = u_x (and w = u_y) by the fifth-order
 * finite-difference HWENO scheme with limiter of Zhang & Zhao,
 * arXiv:2207.05258 (Sec. 2): global Lax-Friedrichs flux splitting, the
 * nonlinear HWENO reconstruction of the governing-equation flux (one quintic
 * and two quadratics, Sec. 2.1; characteristic-wise for Euler, remarks of
 * Sec. 2.1 and 2.2), the linear p_0' fluxes of the derivative equations, the
 * central mixed-derivative fluxes (Eq. mixed), the HWENO limiter that
 * modifies the derivatives used only in time stepping (Sec. 2.2) and the
 * SSP-RK3 stages of the fully discrete scheme.
 *
 * Conventions for every call:
 *  - Arrays named U, V, W, dU, ... are DEVICE pointers owned by the caller,
 *    laid out [instance][component][j][i] with i contiguous, interior points
 *    only (ghost values are produced inside the library from the boundary
 *    conditions). Elements are double (HWENO_FP64) or float (HWENO_FP32) as
 *    chosen at create time. Components: Burgers m = 1 (u); Euler 1D m = 3
 *    (rho, rho u, E); Euler 2D m = 4 (rho, rho u, rho v, E). Instance k of a
 *    1D batch starts at element m * sum_{l<k} nx[l]. V is u_x, W is u_y (2D).
 *  - Times t are DEVICE arrays of `batch` doubles (one time per instance).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy stream); all
 *    work is enqueued on it and the calls return without synchronising,
 *    except hweno_sync_status and hweno_step_host.
 *  - The library allocates all of its device scratch in hweno_create and
 *    frees it in hweno_destroy: the stage buffers, the stored limited
 *    derivative, per-instance wave speeds and time steps, a status word, the
 *    persistent run's counters (1D), the device copies, streams and events of
 *    hweno_step_host, and (FP64 Burgers and Euler contexts) the adjoint's
 *    scratch. No other call allocates device memory, so the calls that only
 *    enqueue work (hweno_rhs, hweno_step, hweno_run_persistent without a
 *    point-update count, hweno_totals, hweno_adjoint_step and the record
 *    calls) can be recorded into a CUDA graph by the caller. hweno_run
 *    instantiates a graph of its own (driver objects), hweno_profile_start
 *    creates events, and hweno_measure_fp64_peak allocates and frees a small
 *    buffer of its own (no context).
 *  - Every call returns an int status: HWENO_OK (0) or a negative code; a
 *    readable message is kept in the context (hweno_last_error). Errors the
 *    device detects (a non-finite wave speed) are latched into the context's
 *    device status word and returned by hweno_sync_status (which
 *    hweno_step_host calls). No call aborts the process or throws across the
 *    ABI.
 */
#ifndef HWENO_H
#define HWENO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define HWENO_OK 0
#define HWENO_EINVAL (-1)     /* invalid argument: grid, BC, option, pointer */
#define HWENO_ENOMEM (-2)     /* device or host allocation failed */
#define HWENO_ECUDA (-3)      /* a CUDA runtime call failed */
#define HWENO_ENONFINITE (-4) /* a wave speed (alpha) became NaN or Inf */
#define HWENO_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define HWENO_ENOTSUP (-6)    /* not implemented for this configuration */
#define HWENO_EBOUNDS (-7)    /* a device-side index check failed (checked builds
                                 only: compiled with -DHWENO_CHECKS=1) */

/* Equations (Sec. 3: Burgers, Eq. 1dbugers / 2dbugers; Euler, Eq. euler1 /
 * euler2 with E = p/(gamma-1) + rho |u|^2 / 2; Buckley-Leverett, Example 3.4,
 * f(u) = 4u^2 / (4u^2 + (1-u)^2), 1D only, whose alpha is the maximum of
 * |f'| over the admissible states [0, 1] and over grid values outside it). */
#define HWENO_BURGERS 0
#define HWENO_EULER 1
#define HWENO_BUCKLEY 2

/* Precision of state arrays and of the reconstruction arithmetic. Wave
 * speeds, time steps and times are always FP64. */
#define HWENO_FP64 0
#define HWENO_FP32 1

/* Boundary conditions (Sec. 3). Ghost derivatives: periodic wraps; outflow
 * copies U and its derivatives; reflective mirrors U with the normal momentum
 * odd (Burgers: u odd), the normal derivative of opposite parity and the
 * tangential one of the same parity; imposed states carry zero derivatives.
 * HWENO_BC_DMR_BOTTOM (y-low only): imposed state `inflow` for x < dmr_x0,
 * reflective wall beyond; HWENO_BC_DMR_TOP (y-high only): `inflow` left of the
 * exact shock position x_s(y, t) = dmr_x0 + y / tan(dmr_angle)
 * + dmr_speed t / sin(dmr_angle), `pre` right of it (Example 3.11). */
#define HWENO_BC_PERIODIC 0
#define HWENO_BC_OUTFLOW 1
#define HWENO_BC_REFLECTIVE 2
#define HWENO_BC_INFLOW 3
#define HWENO_BC_DMR_BOTTOM 4
#define HWENO_BC_DMR_TOP 5

typedef struct hweno_bc {
  int xlo, xhi, ylo, yhi; /* HWENO_BC_* per side (y sides ignored in 1D) */
  double inflow[4];       /* imposed conserved state (inflow, DMR post-shock) */
  double pre[4];          /* DMR pre-shock conserved state */
  double dmr_x0;          /* DMR: x where the shock meets y = 0 at t = 0 */
  double dmr_speed;       /* DMR: normal speed of the shock */
  double dmr_angle;       /* DMR: angle of the shock to the x axis, radians */
} hweno_bc;

/* Uniform cell-centred grid (Sec. 2.1: x_i the centre of I_i,
 * dx = (x1 - x0) / nx). A 1D batch holds `batch` independent instances on
 * the same [x0, x1] with nx_per_instance[k] points each (host array, read
 * only during hweno_create; NULL means nx for all). 2D requires batch = 1.
 * Every nx, ny must be >= 4. */
typedef struct hweno_grid {
  int dim;                    /* 1 or 2 */
  int nx, ny;                 /* points per direction (ny ignored in 1D) */
  double x0, x1, y0, y1;      /* domain */
  int batch;                  /* number of instances, >= 1 */
  const int* nx_per_instance; /* host, [batch], or NULL */
  int precision;              /* HWENO_FP64 or HWENO_FP32 */
} hweno_grid;

/* Scheme options. hweno_default_options fills the paper's values (Sec. 3):
 * lin_w = lim_d = {0.98, 0.01, 0.01}, eps = 1e-6, cfl = 0.6,
 * dt_mode = 0, limiter = 1, eig_avg = 0, tile_variant = 0, fused_small = 0,
 * adj_frozen_weights = 0 and fused_2d = 0. */
typedef struct hweno_options {
  double lin_w[3]; /* gamma_0..2 of the reconstruction: >= 1e-6 each, sum 1 (Sec. 2.1) */
  double lim_d[3]; /* d_0..2 of the limiter: >= 1e-6 each, sum 1 (Sec. 2.2) */
  double eps;      /* epsilon of the nonlinear weights, in [1e-20, 1e6]. The
                      FP64 kernels resolve the nonlinear weights of two sides
                      and two fields over one common denominator, a product
                      of up to sixteen factors of the size of beta + eps; the
                      bounds on eps and the linear weights keep it above the
                      FP64 underflow limit. Large data (beta grows like the
                      square of the split-flux jumps) would push it past the
                      overflow limit, so each side's numerator and
                      denominator are rescaled by an exact power of two; this
                      holds for split-flux jumps up to about 1e35 (tested
                      against the CPU oracle with Euler states scaled by 1e6,
                      1e12, 1e20 and Burgers by 1e4, 1e8). Other eps values
                      are HWENO_EINVAL. */
  double cfl;      /* CFL number, > 0 */
  int dt_mode;     /* 0: dt = cfl / sum(alpha_d / h_d) with h = dx;
                      1: h = dx^{5/3} (accuracy runs); 2: dt = dt_fixed.
                      The last step of a run is clipped to land on t_end. */
  double dt_fixed;
  int limiter;     /* 0: off; 1: on characteristic variables (eigenvectors at
                      U_i of the sweep direction); 2: component-wise */
  int eig_avg;     /* eigenvectors at x_{i+1/2}: 0 Roe average of U_i, U_{i+1};
                      1 arithmetic mean */
  int tile_variant; /* 1D tile shape 0 .. HWENO_TILE_VARIANTS - 1 (see
                       hweno_autotune; results do not depend on it); ignored
                       in 2D */
  int fused_small;  /* 1D: 1 = when every instance has at most
                       HWENO_FUSED_MAX_POINTS points, hweno_step runs the whole
                       step (wave speed, three stages, time update) in one
                       launch with one CTA per instance; 0 (default) = the
                       tiled kernels. Results agree to rounding. One CTA has
                       1/152 of the GPU's FP64 pipe, so for a few FP64
                       instances the tiled kernels are faster (Burgers N = 400:
                       133 vs 81 us per step); the fused step pays off in FP32
                       or for batches of many small instances.
                       2 = when every instance has at most
                       HWENO_CLUSTER_MAX_POINTS points, one launch per step
                       on thread-block clusters: one cluster per instance,
                       one tile per CTA, each CTA on an SM of its own (it
                       reserves 116 KB of shared memory), the stages
                       separated by cluster barriers. Up to 448 points the
                       tiles have 28 points and the work of a point is
                       divided over the CTA's four warps (up to 16 CTAs per
                       cluster, where the device allows it); otherwise 124
                       points (up to 8); a device that cannot hold the
                       cluster gets the tiled kernels. Meant for a few small
                       instances, where the latency of a step matters. */
  int adj_frozen_weights; /* hweno_adjoint_step: 0 = differentiate the
                       nonlinear weights of the reconstruction and the
                       limiter; 1 = hold them at their forward values (the
                       adjoint of the scheme linearised with frozen weights) */
  int fused_2d;     /* 2D steps: 0 = per stage an x-sweep and a y-sweep launch
                       (the x parts pass through library scratch); 1 = one
                       fused launch per stage, one CTA per 16 x 7 block doing
                       both directions (the x-interfaces on block edges are
                       computed by both neighbours). Results agree to
                       rounding; hweno_autotune picks the faster form for the
                       caller's grid. hweno_rhs always uses the sweeps. */
} hweno_options;

/* Largest instance of the cluster step (fused_small = 2): 8 tiles of 124. */
#define HWENO_CLUSTER_MAX_POINTS 992

/* Number of 1D tile shapes (hweno_options.tile_variant, hweno_autotune). */
#define HWENO_TILE_VARIANTS 5

/* Largest instance of the fused single-launch step (one 508-point tile). */
#define HWENO_FUSED_MAX_POINTS 508

typedef struct hweno_ctx hweno_ctx; /* opaque, library-owned */

/* Fill *opt with the paper's defaults (Sec. 3). */
int hweno_default_options(hweno_options* opt);

/* Create a solver for `equation` (HWENO_BURGERS / HWENO_EULER /
 * HWENO_BUCKLEY) on `grid` with ratio of specific heats `gamma` (Euler;
 * ignored otherwise) and
 * boundary conditions `bc` (the problem statement of Sec. 2.1 and Sec. 3).
 * Allocates all device scratch on the current device. On success *out holds
 * the context and HWENO_OK is returned; on failure *out is NULL and the code
 * says why: HWENO_EINVAL for an invalid grid, equation, gamma or boundary
 * set (nx, ny < 4; batch < 1; 2D with batch > 1; periodic on one side only;
 * DMR kinds outside y-low/y-high or with Burgers; Buckley-Leverett in 2D or
 * with reflective walls), HWENO_ENOMEM / HWENO_ECUDA
 * for allocation or runtime failures. Options start at hweno_default_options. */
int hweno_create(hweno_ctx** out, int equation, const hweno_grid* grid, double gamma,
                 const hweno_bc* bc);

/* Replace the scheme options (validated; HWENO_EINVAL leaves them unchanged).
 * A graph that hweno_run recorded is dropped, so that the next hweno_run
 * records the new options. No device memory is written: the tile tables of
 * every tile variant and the step sizes of every dt_mode are made by
 * hweno_create, so work still running on any stream is not disturbed. */
int hweno_set_options(hweno_ctx* ctx, const hweno_options* opt);

/* The context's current options into *out (host): those of the last
 * hweno_set_options, with the tile variant (1D) or the stage form (2D, field
 * fused_2d) that hweno_autotune, hweno_autotune_classes or
 * hweno_set_class_variants chose since. A caller changes one option by
 * reading, editing and setting them back. HWENO_EINVAL for a null pointer. */
int hweno_get_options(const hweno_ctx* ctx, hweno_options* out);

/* Spatial operator of one stage (Eq. odeH in 1D, Eq. ode2H in 2D):
 * dU = L^1(U, V[, W]), dV = L^2, dW = L^3 (2D), each -(flux difference)/h,
 * with alpha the maximum of |f'(u)| (Euler: |u| + c per direction) over each
 * instance's grid and boundary data at time t[k]. Vlim / Wlim (nullable)
 * receive the limited derivatives of Sec. 2.2. W, dW, Wlim must be NULL in
 * 1D. All array arguments are device pointers of the state's size. */
int hweno_rhs(hweno_ctx* ctx, const void* U, const void* V, const void* W, void* dU,
              void* dV, void* dW, void* Vlim, void* Wlim, const double* t, void* stream);

/* One SSP-RK3 step of the fully discrete scheme (Sec. 2.2) in place on
 * U, V (, W): stage k evaluates L at the unlimited stage state and combines
 * with the limited derivatives. dt per instance from the wave speed of U^n
 * (dt_mode), clipped so that t lands on t_end; instances with t >= t_end
 * are left unchanged. t (device, [batch]) is advanced; dt_used (device,
 * [batch], nullable) receives each instance's dt (0 when inactive). */
int hweno_step(hweno_ctx* ctx, void* U, void* V, void* W, double* t, double t_end,
               double* dt_used, void* stream);

/* Advance until every instance has reached t_end or `max_steps` steps have
 * been taken. The steps are recorded once into a CUDA graph of
 * `steps_per_launch` SSP-RK3 steps, kept in the context for these arrays and
 * t_end (re-recorded when they change), and the graph is replayed on
 * `stream`; after each replay the host reads the number of active instances.
 * Steps of finished instances are no-ops, so up to steps_per_launch - 1
 * extra (empty) steps can run after the last instance lands. `stream` must
 * not be NULL (graphs are recorded from a stream). max_steps = 0 only records
 * the graph. On return (stream synchronised) *steps_taken (host, nullable)
 * holds the steps launched and *point_updates (host, nullable) the number of
 * grid points advanced through a full step, summed over instances and steps.
 * Recording a graph creates driver objects but no device buffer. */
int hweno_run(hweno_ctx* ctx, void* U, void* V, void* W, double* t, double t_end,
              long long max_steps, int steps_per_launch, long long* steps_taken,
              long long* point_updates, void* stream);

/* As hweno_step with HOST arrays: copies U, V (, W) and t (host, [batch]) to
 * library-owned device buffers, takes `nsteps` steps, copies them back and
 * synchronises the stream. Pinned host memory makes the copies asynchronous.
 * A 1D batch (fused_small = 0) is cut into up to eight ranges of whole
 * instances with about equal points, each copied in, stepped and copied out
 * on a library stream of its own, so that the copies of one range overlap
 * the kernels of the others; the results are those of hweno_step bit for bit
 * and hweno_active_instances counts after the call. The device copies, the
 * streams and their events are made by hweno_create. */
int hweno_step_host(hweno_ctx* ctx, void* U, void* V, void* W, double* t, double t_end,
                    int nsteps, void* stream);

/* Persistent run of a 1D batch: `steps` SSP-RK3 steps (Sec. 2.2) of every
 * instance in ONE kernel launch (after a wave-speed launch for the first
 * step). The CTAs stay resident and take work items (step, stage, tile) from
 * a device counter in that order; a tile waits only for the previous stage
 * of its own instance, so instances of different sizes and step counts flow
 * through the stages without grid-wide barriers. Results agree with `steps`
 * calls of hweno_step to rounding (the same stage code, compiled into another
 * kernel, may fuse a*b + c*d differently); instances reaching t_end stop
 * stepping. U, V, t (device) are updated in
 * place. If point_updates (host) is not NULL the call synchronises `stream`
 * and stores the point-updates of stepping instances there, then returns the
 * latched device status; otherwise it returns after enqueueing. Waits are
 * bounded (about two seconds); a wait that gives up latches HWENO_ETIMEOUT,
 * and every CTA then stops: tiles whose inputs were ready have run, the rest
 * have not, so after HWENO_ETIMEOUT the contents of U, V and t are
 * undefined. 1D only (2D: HWENO_ENOTSUP). Library scratch (counters, alpha
 * slots, tiles per instance of every tile variant) is made by hweno_create;
 * with point_updates NULL the
 * call only enqueues work, so it can be recorded into a CUDA graph and
 * replayed (each replay resets the counters first). With fused_small = 2 and instances within
 * HWENO_CLUSTER_MAX_POINTS, the steps run instead as one launch of the
 * cluster step (one cluster per instance, cluster barriers between stages and
 * steps); it gives the bits of `steps` calls of hweno_step with that option. */
int hweno_run_persistent(hweno_ctx* ctx, void* U, void* V, double* t, double t_end, int steps,
                         long long* point_updates, void* stream);

/* Test hook for failure detection (no counterpart in the paper). kind = 1:
 * the next hweno_run_persistent expects one tile too many for instance 0, so
 * the waits for that instance cannot be satisfied; they give up after about
 * two seconds, every CTA then stops, and the call returns HWENO_ETIMEOUT
 * (latched status). The injection travels as an argument of that one
 * launch; the context stays usable and the following runs are normal.
 * kind = 0 clears a pending injection. kind = 2 (builds compiled with
 * -DHWENO_CHECKS=1, whose kernels check their shared-memory and global
 * indices): a one-CTA self-test kernel on the legacy stream reads one row
 * and one column past the end of a checked shared-memory view; the check
 * redirects both reads to element 0 (nothing outside the array is read) and
 * latches HWENO_EBOUNDS, which the next hweno_sync_status returns (other
 * builds: HWENO_ENOTSUP). Nothing faults or hangs the device. */
int hweno_test_inject(hweno_ctx* ctx, int kind);

/* Tile-shape autotuner (1D): times the fused stage kernel of every tile
 * variant (CTA sizes 64, 128, 256 threads, one or two points per thread) on
 * the given state U, V at times t (device) with t_end, and keeps the fastest
 * for the following calls of this context. Only library scratch is written
 * (U, V, W, t are read). Synchronises `stream` and drops a graph that
 * hweno_run recorded for another variant. *chosen (host, nullable)
 * receives the variant index (0 = the default 128 x 1; variants 1..4 are
 * 64 x 1, 256 x 1, 128 x 2 and 64 x 2, threads x points per thread);
 * ms (host, nullable, HWENO_TILE_VARIANTS doubles) the best measured time of
 * each variant in milliseconds. In 2D the two forms of a stage are timed
 * instead (the x- and y-sweep launches, and the fused launch; stage 1 on
 * the given state) and the faster is kept as fused_2d: *chosen receives 0
 * or 1 and ms[0], ms[1] their times. */
int hweno_autotune(hweno_ctx* ctx, const void* U, const void* V, const void* W, const double* t,
                   double t_end, int* chosen, double* ms, void* stream);

/* Largest number of instance-size classes of a 1D batch. */
#define HWENO_MAX_SIZE_CLASSES 16

/* Size classes of a 1D batch (no counterpart in the paper; a tuning aid):
 * the distinct instance sizes when there are at most HWENO_MAX_SIZE_CLASSES
 * of them, else octaves of the size above the smallest instance. Returns the
 * number of classes (0 in 2D, HWENO_EINVAL for a NULL context) and writes
 * each class's smallest and largest instance size to lo, hi (host, nullable,
 * HWENO_MAX_SIZE_CLASSES ints each). */
int hweno_size_classes(const hweno_ctx* ctx, int* lo, int* hi);

/* Tile-shape autotuner per size class (1D batches; no counterpart in the
 * paper): times the stage-1 kernel of every tile variant on each class's
 * instances alone (U, V, t device, read only; library scratch written) and
 * keeps the fastest variant per class. When the classes choose different
 * variants, hweno_step (and the graph of hweno_run) launches each stage once
 * per run of consecutive classes with the same variant, over tile tables
 * ordered by class that hweno_create made; the results are the bits of any
 * single variant. When all classes agree this is hweno_autotune's choice.
 * hweno_rhs, hweno_step_host and hweno_run_persistent keep one variant (the
 * one in force before). hweno_set_options and hweno_autotune end the
 * per-class choice. chosen (host, nullable, one int per class) receives the
 * variants, ms (host, nullable, classes x HWENO_TILE_VARIANTS doubles) the
 * best time of each class and variant. Synchronises `stream`; drops a graph
 * that hweno_run recorded. 2D: HWENO_ENOTSUP. */
int hweno_autotune_classes(hweno_ctx* ctx, const void* U, const void* V, const double* t,
                           double t_end, int* chosen, double* ms, void* stream);

/* Set the tile variant of every size class directly (host array of
 * hweno_size_classes(ctx) ints in [0, HWENO_TILE_VARIANTS)), for example a
 * choice hweno_autotune_classes made in an earlier run; the same rules as
 * there. When all entries are equal this selects that tile_variant for every
 * call. No device memory is written; a graph that hweno_run recorded is
 * dropped. HWENO_EINVAL for a variant out of range, HWENO_ENOTSUP in 2D. */
int hweno_set_class_variants(hweno_ctx* ctx, const int* variants);

/* Conserved totals in FP64 (the discrete integrals conserved by the flux
 * form of Eq. odeH / ode2H): totals[k * m + c] = sum_i U_c(x_i) dx (2D:
 * times dy) for every instance k and component c, accumulated in FP64 in a
 * fixed order (the same bits on every call), also for FP32 states. totals is
 * a device array of batch * m doubles. */
int hweno_totals(hweno_ctx* ctx, const void* U, double* totals, void* stream);

/* Discrete adjoint of one hweno_step (the fully discrete scheme of Sec. 2.2,
 * 1D Eq. odeH and 2D Eq. ode2H with the mixed fluxes of Eq. mixed,
 * differentiated stage by stage): given the step's input state U, V (, W)
 * (device), the time at the start of the step t (device, [batch]) and the
 * time step it took dt (device, [batch], the dt_used of hweno_step; 0 = the
 * instance did not step), replaces lamU, lamV (, lamW) (device, in: the
 * gradient of a functional with respect to the step's output, out: with
 * respect to its input). The wave speeds of each stage and dt are frozen
 * (constants of the step) and the |.| in the smoothness differences keeps the
 * branch of the forward state; the nonlinear weights, the characteristic
 * eigenvectors (Roe average) and the limiter are differentiated. FP64 states
 * only, Roe-averaged eigenvectors (eig_avg = 0), and in each direction both
 * boundaries periodic or neither (else HWENO_ENOTSUP). 1D: W and lamW must be
 * NULL and t is not read (may be NULL). 2D: W and lamW are required; t is
 * read by the double-Mach top boundary and may be NULL otherwise. Library
 * scratch holds the replayed stages and the stage cotangents (made by
 * hweno_create for FP64 Burgers and Euler contexts: 6 fields of m x points
 * doubles in 1D, 12 in 2D). */
int hweno_adjoint_step(hweno_ctx* ctx, const void* U, const void* V, const void* W,
                       const double* t, const double* dt, void* lamU, void* lamV, void* lamW,
                       void* stream);

/* Step records: the same forward step and adjoint without the adjoint's
 * replay of stages 1 and 2. hweno_step_record takes one hweno_step (same
 * arguments and results) and then copies that step's stage states (U, V
 * [, W] after stages 1 and 2) and per-stage wave speeds into `record`, a
 * device buffer of hweno_adjoint_record_bytes(ctx) bytes owned by the caller
 * (for 2D Euler 6 x 4 x points doubles). hweno_adjoint_step_recorded is
 * hweno_adjoint_step for that step reading the stages from its record instead
 * of recomputing them: the same results (the record holds the bits the
 * replay would produce when the forward step ran the tiled kernels), two
 * fewer stages of work. FP64 states only (else HWENO_ENOTSUP); a null record
 * is HWENO_EINVAL. hweno_adjoint_record_bytes returns -1 for a null ctx. */
long long hweno_adjoint_record_bytes(const hweno_ctx* ctx);
int hweno_step_record(hweno_ctx* ctx, void* U, void* V, void* W, double* t, double t_end,
                      double* dt_used, void* record, void* stream);
int hweno_adjoint_step_recorded(hweno_ctx* ctx, const void* U, const void* V, const void* W,
                                const void* record, const double* t, const double* dt,
                                void* lamU, void* lamV, void* lamW, void* stream);

/* Synchronise `stream`, read the device status word and return the latched
 * device error (HWENO_OK if none); clears the latch. */
int hweno_sync_status(hweno_ctx* ctx, void* stream);

/* Number of grid points summed over instances (-1 for a NULL context). */
long long hweno_num_points(const hweno_ctx* ctx);

/* Number of instances with t < t_end after the last hweno_step enqueued on
 * `stream` (synchronises the stream; negative on error). */
int hweno_active_instances(hweno_ctx* ctx, void* stream);

/* Kernel launches enqueued by the most recent hweno_step / hweno_rhs call. */
int hweno_launches_last_call(const hweno_ctx* ctx);

/* Kernel timing for measurement. hweno_profile_start(ctx, capacity) makes the
 * following hweno_step / hweno_rhs calls bracket each kernel launch with CUDA
 * events on the call's stream, for up to `capacity` launches (0 stops it).
 * hweno_profile_read synchronises `stream` and writes, per kernel kind
 * (0: wave-speed reduction, 1: fused stage, 2: step finalisation), the summed
 * device time in milliseconds ms[3] and the launch count n[3] recorded since
 * the start; it then clears the record. Events are host-side objects created
 * in hweno_profile_start; no device memory is allocated. */
int hweno_profile_start(hweno_ctx* ctx, int capacity);
int hweno_profile_read(hweno_ctx* ctx, double* ms, int* n, void* stream);

/* Measured FP64 ceiling (no counterpart in the paper; a measurement aid):
 * times a loop of independent DFMA chains with eight warps per SM, no memory
 * traffic, and stores the rate in *tflops (host) as FP64 TFLOP/s (2 flops per
 * DFMA) on the current device at its current clocks. Allocates and frees a
 * small output buffer; synchronises `stream`. HWENO_EINVAL for a null
 * pointer, HWENO_ENOMEM / HWENO_ECUDA on CUDA failures. */
int hweno_measure_fp64_peak(double* tflops, void* stream);

/* Allocation-free step (this entry point has no counterpart in the paper; it
 * serves callers that cannot allocate device memory: code inside a host
 * framework that owns all device allocations through its own pool, code that
 * must not pay cudaMalloc's implicit synchronisation, plug-ins that are only
 * handed pre-allocated buffers).
 *
 * One SSP-RK3 step, as hweno_step, of a single 1D instance in FP64, with no
 * context: the problem is passed in full (`opt` NULL = the paper's defaults),
 * U, V (device, [m][nx]) are advanced in place, t (device, one double)
 * advances and dt_used (device, one double, nullable) receives the step.
 * All scratch lives in one fixed device array built into the library (about
 * 2 MB, enough for nx <= HWENO_NOALLOC_MAX_POINTS points), present on every
 * GPU that loads the library until the process exits; the call performs no
 * cudaMalloc, cudaFree or other allocation. The first call on a device looks
 * up that array's address for the device (with the device current). The
 * call synchronises `stream` and returns HWENO_ENONFINITE if a wave speed was
 * not finite. HWENO_EINVAL: nx outside [4, HWENO_NOALLOC_MAX_POINTS], an invalid
 * equation, gamma, boundary set or option. Every call shares the one array,
 * so calls whose GPU work overlaps (other streams, other host threads) race:
 * serialise them. */
#define HWENO_NOALLOC_MAX_POINTS 16384
int hweno_step_1d_noalloc(int equation, int nx, double x0, double x1, double gamma,
                          const hweno_bc* bc, const hweno_options* opt, double* U, double* V,
                          double* t, double t_end, double* dt_used, void* stream);

/* Message describing the last error on this context ("" if none). */
const char* hweno_last_error(const hweno_ctx* ctx);

/* Free all device and host resources of the context (NULL is a no-op). */
int hweno_destroy(hweno_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HWENO_H */
