/*
 * plan.h -- C ABI of the GB300 batched bi-level trajectory planner.
 *
 * The library implements the data-parallel hot path of "Bi-Level Optimization
 * Augmented with Conditional Variational Autoencoder for Autonomous Driving in
 * Dense Traffic" (Singh, Shrestha, Albarella): for each of B sampled
 * behavioural inputs p_j it solves the lower-level trajectory problem (Step 1
 * QP of Alg. 1 via the shared KKT inverse of Eq. over_3, then the batch
 * projection of Alg. 2), scores every solution (Alg. 1 line 9 and the
 * upper-level cost of Sec. V-A) and runs the gradient-free outer loop of
 * Alg. 1 (elite sets, distribution update of Eqs. mean_update / cov_update /
 * s_formula, re-sampling).
 *
 * Conventions shared by every call:
 *   - Every function returns a plan_status; none aborts, throws or exits.
 *     On an error return no device work has been enqueued by that call and
 *     plan_last_error() describes the failure.
 *   - Floating-point buffers at this boundary are IEEE float64, row-major.
 *   - "device" pointers are CUDA global memory of the device that was current
 *     when plan_init ran; "host" pointers are ordinary process memory
 *     (pinned memory makes the copies asynchronous).
 *   - Work is enqueued on the caller's stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) and is asynchronous unless the
 *     function says otherwise; results are valid after the stream is
 *     synchronised.
 *   - Inputs are copied into the context before the call returns; callers keep
 *     ownership of every buffer they pass.
 *   - A context is not thread-safe: use one per host thread, or lock.
 *
 * Coordinates: a scene is expressed in a frame where the road's lanes run
 * along +x, lane i spans y in [i w, (i+1) w] and the lane-boundary
 * constraint of Table I is y_lb <= y <= y_ub with y_lb = lane_margin and
 * y_ub = n_lanes w - lane_margin.
 */
#ifndef PLAN_H_
#define PLAN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct plan_ctx plan_ctx;   /* opaque; owns all device memory it uses */

typedef enum {
    PLAN_OK = 0,
    PLAN_EINVAL = -1,      /* an argument is out of range or inconsistent      */
    PLAN_ENOMEM = -2,      /* a device or pinned-host allocation failed        */
    PLAN_ECAPACITY = -3,   /* request exceeds the capacities given to plan_init */
    PLAN_ETIMEOUT = -4,    /* a bounded wait expired                            */
    PLAN_ECUDA = -5,       /* a CUDA runtime call failed (see plan_last_error) */
    PLAN_ESTATE = -6,      /* call not valid in the context's current state    */
    PLAN_ENONFINITE = -7   /* a result is not finite                            */
} plan_status;

/* Arithmetic of the lower-level solve.  FP64: one kernel per step of Alg. 2
 * with intermediates in HBM, float64 throughout (the reference GPU path).
 * FP32: the fused multi-iteration kernel, float32 projections and
 * contractions with constants formed and inverted in float64.
 * TF32, BF16, TF32X3: the fused iteration with the two n-wide contractions of
 * Alg. 2 (the forward evaluation W xi of Eq. param and the transposed
 * contraction F^T h, G^T (e - s) of the xi-step, Eq. split_xy) on the tensor
 * cores with float32 accumulation; the projections stay float32.  TF32 and
 * BF16 round the operands once (about 2^-11 and 2^-8 relative); TF32X3
 * splits every operand into a TF32 head and tail and sums three products,
 * which is float32-level accuracy.  These modes need m <= 128. */
typedef enum {
    PLAN_PREC_FP64 = 0,
    PLAN_PREC_FP32 = 1,
    PLAN_PREC_TF32 = 2,
    PLAN_PREC_BF16 = 3,
    PLAN_PREC_TF32X3 = 4
} plan_prec;

/* Planner configuration (plan_init).  Symbols follow the paper.
 *   m            timesteps t_i = i dt of the horizon (Eq. param), 8..256
 *   n_coef       polynomial coefficients per axis (degree + 1), 4..16; the
 *                paper uses a 10th-order polynomial, n_coef = 11 (Sec. V-A)
 *   n_seg        set-point segments of p (Eq. behaviour_param), 1..4;
 *                p = [y_d,1..y_d,n_seg, v_d,1..v_d,n_seg] has d_p = 2 n_seg entries
 *   goal         0 or 1.  With 1, p also carries the goal positions of
 *                Eq. behaviour_param, p = [y_d.., v_d.., x_f, y_f]
 *                (d_p = 2 n_seg + 2), and the lower level adds the final
 *                boundary rows of Eq. final_boundary, (x(t_f), y(t_f),
 *                ydot(t_f)) = (x_f, y_f, 0), to its equality constraints
 *                A_eq xi = b(p) (Eq. lower_eq: the goal positions enter b,
 *                the set-points the cost).  x_f is in the scene's frame.
 *                In the first iteration of a fresh episode x_f = x0 + v t_f
 *                with v ~ U[v_des_lo, v_des_hi] (t_f = (m - 1) dt) and y_f is
 *                a lane centre drawn uniformly.
 *   inner_iters  K, iterations of Alg. 2 (>= 1)
 *   outer_iters  L, iterations of Alg. 1 (>= 1)
 *   n_elite_c    size of ConstraintEliteSet (Alg. 1 line 10); <= 0 means
 *                min(B, 3 n_elite); at most 2048
 *   n_elite      size q of EliteSet (Alg. 1 line 13), 1..n_elite_c
 *   prec         a plan_prec value
 *   max_obs      capacity: obstacles per scene (<= 64)
 *   max_samples  capacity: samples per call, summed over scenes
 *   max_scenes   capacity: scenes per call
 *   dt           time step [s]
 *   rho          penalty of the augmented Lagrangian, Eq. (aug_lag)
 *   kp_lat, kv_lat, kp_lon   PD / P gains of the tracking costs c_l, c_v
 *   gamma, eta   s_formula scaling and learning rate of the distribution update
 *   cov_eps      jitter added to Sigma before its Cholesky factorisation
 *   v_min, v_max, a_max, kappa_max, c_max   bounds of Table I and Eq. d_reform_1
 *   lane_margin  distance kept from the road edges [m]
 *   v_des_lo, v_des_hi   range of v_d in the first iteration of a fresh episode
 */
typedef struct {
    int m, n_coef, n_seg, inner_iters, outer_iters, n_elite_c, n_elite;
    int prec;
    int max_obs, max_samples, max_scenes;
    int goal;
    double dt, rho, kp_lat, kv_lat, kp_lon, gamma, eta, cov_eps;
    double v_min, v_max, a_max, kappa_max, c_max, lane_margin, v_des_lo, v_des_hi;
} plan_config;

/* Ego state at t0: the vector b0 of Eq. (boundary_cond_initial). */
typedef struct { double x, y, vx, vy, ax, ay; } plan_ego;

/* A neighbouring vehicle moving at constant velocity: centre
 * (x0 + vx t, y0 + vy t), ellipse semi-axes a (along x) and b (along y) of
 * Table I's collision constraint. */
typedef struct { double x0, y0, vx, vy, a, b; } plan_obstacle;

/* A knot of the road profile along the reference centre line (Frenet frame,
 * Sec. III-C: x is arc length, y the lateral offset): road curvature kappa of
 * Eq. (cent_bounds) and the road edges lb < ub of Table I's lane-boundary row
 * at arc length s. */
typedef struct { double s, kappa, lb, ub; } plan_road_knot;

/* One driving scene; `obs` is host memory with n_obs entries (may be NULL
 * when n_obs == 0).
 * Road: with n_road == 0 the road is straight-laned with constant curvature
 * kappa_road (0 for a straight road) and lane limits [lane_margin,
 * n_lanes lane_width - lane_margin].  With n_road in 1..8 knots (host, s
 * strictly increasing), kappa(x) and the edges are interpolated linearly in
 * x + road_origin and held constant beyond the end knots; the lane limits are
 * the edges moved inwards by lane_margin.  As the paper prescribes, the
 * projection evaluates kappa and the limits at the positions of the current
 * iterate (Alg. 2, analysis of step split_xy). */
typedef struct {
    plan_ego ego;
    int n_lanes;
    double lane_width;
    double kappa_road;
    int n_obs;
    const plan_obstacle* obs;
    int n_road;
    const plan_road_knot* road;
    double road_origin;   /* arc length of x = 0 along the road profile */
} plan_scene;

/* Largest d_p: four set-point segments per axis plus the two goal entries. */
#define PLAN_MAX_DP 10

/* Sampling distribution of p carried between MPC cycles (Alg. 1 lines 2, 14).
 * mu[0..d_p-1] and sigma (d_p x d_p, row-major, leading dimension
 * PLAN_MAX_DP) are used when fresh == 0; when fresh != 0 the first iteration
 * draws y_d uniformly over lane centres and v_d ~ U[v_des_lo, v_des_hi] (and
 * the goal entries as described at plan_config.goal) and mu, sigma start at
 * that distribution's moments.  seed and episode_step select the
 * Philox4x32-10 stream (key = seed, counter = (j, l | c << 16, step)).
 * With goal entries, a warm start carries x_f as a position in the scene's
 * frame; plan_advance re-centres the frame on the ego, so a caller that
 * keeps an absolute goal across cycles shifts mu[x_f] by the distance
 * travelled. */
typedef struct {
    double mu[PLAN_MAX_DP];
    double sigma[PLAN_MAX_DP * PLAN_MAX_DP];
    uint64_t seed;
    uint64_t episode_step;
    int fresh;
    int reserved0;
} plan_cem_state;

/* Best pair of the final EliteSet (the return line of Alg. 1). */
typedef struct {
    double p[PLAN_MAX_DP]; /* d_p entries                                    */
    double xi[32];       /* 2 n_coef entries: (c_x, c_y)                      */
    double cost;         /* c_u + r_j                                         */
    double resid;        /* r_j, Alg. 1 line 9                                */
    double cu;           /* c_u, upper-level driving cost                     */
    int index;           /* sample index within the last outer iteration      */
    int reserved0;
} plan_result;

/* ---------------------------------------------------------------- lifecycle */

/* Create a context on the current CUDA device: validates `cfg`, allocates the
 * device arena sized by max_obs / max_samples / max_scenes, and builds in
 * float64 on the GPU the Bernstein basis (Eq. param) and the inverted KKT
 * systems of Step 1 (Eq. over_2) and of the projection xi-step (Eq. split_xy)
 * for every obstacle count 0..max_obs.  Synchronous.  On failure *out is NULL. */
int plan_init(const plan_config* cfg, plan_ctx** out);

/* Release the context and everything it allocated.  NULL is accepted. */
int plan_destroy(plan_ctx* ctx);

/* Static description of a status code. */
const char* plan_status_str(int status);

/* Copy the context's last error message (NUL-terminated, truncated to len). */
int plan_last_error(const plan_ctx* ctx, char* buf, size_t len);

/* ------------------------------------------------------ lower level (Alg. 1 l.6-9) */

/* Solve the lower-level problem for B given behavioural inputs of one scene:
 * Step 1 (Eq. over_3), inner_iters iterations of Alg. 2, then the residual
 * r_j = sum max(0, g(xi*_j)) over Table I (Alg. 1 line 9) and the driving
 * cost c_u = sum_t (|v(t)| - v_max)^2 (Sec. V-A).
 *   p       device, B x d_p
 *   xi      device, B x 2 n_coef, or NULL
 *   resid   device, B
 *   cu      device, B
 *   status  device, B ints, or NULL: per sample PLAN_OK when its solution
 *           xi*_j (all 2 n_coef coefficients, written or not), r_j and c_u
 *           are finite, PLAN_ENONFINITE otherwise.  A non-finite input p_j
 *           (or a solve that overflows) affects only its own sample.
 * Errors: EINVAL (bad scene or B < 0), ECAPACITY (B > max_samples or
 * n_obs > max_obs).  B == 0 is a no-op.  Per-sample failures are reported
 * only through `status` (the call itself does not wait for the result). */
int plan_solve(plan_ctx* ctx, const plan_scene* scene, const double* p, int B,
               double* xi, double* resid, double* cu, int* status, void* stream);

/* As plan_solve for S scenes in one launch.  Scene s owns samples
 * [off_s, off_s + B[s]) of the concatenated p / xi / resid / cu / status,
 * with off_s = B[0] + ... + B[s-1].  `B` is host memory. */
int plan_solve_batch(plan_ctx* ctx, const plan_scene* scenes, const int* B, int S,
                     const double* p, double* xi, double* resid, double* cu,
                     int* status, void* stream);

/* ---------------------------------------------------------- Alg. 1 (MPC cycle) */

/* Copy S scenes into the context's device-resident scene slots 0..S-1 (the
 * per-cycle inputs of plan_step_resident).  Asynchronous on `stream`. */
int plan_upload_scenes(plan_ctx* ctx, const plan_scene* scenes, int S, void* stream);

/* Load (host -> device) or read back (device -> host, synchronous) the
 * sampling distribution of scene slot `slot`.  A loaded covariance is factored
 * on the device by the routine of the selection kernels, so that an episode
 * exported after some cycles and loaded into a new context continues bit for
 * bit as it would have without the interruption. */
int plan_set_state(plan_ctx* ctx, int slot, const plan_cem_state* st, void* stream);
int plan_get_state(plan_ctx* ctx, int slot, plan_cem_state* st, void* stream);

/* Run Alg. 1 (outer_iters iterations: sample, solve, select, update) for the
 * resident scene slots 0..S-1 with B[s] samples each, entirely on the device.
 * Afterwards each slot holds its updated distribution (fresh cleared,
 * episode_step incremented) and its best pair.  The first call for a given
 * (S, B[]) captures the work into a CUDA graph that later calls replay; the
 * first call must therefore not itself be inside a stream capture.
 * Errors: EINVAL, ECAPACITY (sum B > max_samples, S > max_scenes, or a slot
 * that was never uploaded). */
int plan_step_resident(plan_ctx* ctx, const int* B, int S, void* stream);

/* Read back (synchronous) the best pair of slot `slot` from the last
 * plan_step_resident. */
int plan_get_result(plan_ctx* ctx, int slot, plan_result* out, void* stream);

/* One MPC cycle through host memory: upload `scene` and `*st` to slot 0, run
 * Alg. 1 with B samples, and write the best pair to *out and the updated
 * distribution back to *st.  Synchronous on `stream`. */
int plan_step(plan_ctx* ctx, const plan_scene* scene, plan_cem_state* st, int B,
              plan_result* out, void* stream);

/* ------------------------------------------------------ MPC receding horizon */

/* Advance one MPC cycle (Sec. V-A, MPC-Bi-Level: the ego executes the first
 * `steps` elements of the plan, then replans): the new ego state is the
 * trajectory xi (2 n_coef coefficients, host) at t = steps dt, obstacles move
 * on at constant velocity, and the frame is shifted so that the ego is again at
 * x = 0 (road_origin grows by the distance travelled; the road knots are
 * shared with `in`).  out->obs points to out_obs (host, in->n_obs entries,
 * caller-owned).
 * Host-only arithmetic in float64; no device work. */
int plan_advance(const plan_config* cfg, const plan_scene* in, const double* xi, int steps,
                 plan_scene* out, plan_obstacle* out_obs);

/* ------------------------------------------------------------------ serving */

/* A serving loop batches planning requests of many scenes continuously: a
 * library thread admits pending requests into waves of executors (one planner
 * context per horizon m, own stream and arena) as scene slots and samples free
 * up, creates executors while `device_budget` bytes and `max_executors` allow,
 * and runs waves of different executors concurrently.  Each request is one
 * MPC cycle (Alg. 1, outer_iters iterations) of an episode; the episode's
 * sampling distribution stays in a device table between its cycles (the
 * warm start of Sec. V-A / Alg. 1 line 2).  A scene's result does not depend
 * on the other scenes of its wave: every sample, selection and update is per
 * scene, and the kernel shape is fixed per executor.
 * The configuration's max_samples / max_scenes / max_obs are the capacities
 * of one executor's wave. */
typedef struct plan_server plan_server;

typedef struct {
    plan_scene scene;     /* host; copied at submission                          */
    int B;                /* samples, 1..max_samples                             */
    int m;                /* horizon in timesteps; 0 = the configuration's m     */
    uint64_t episode;     /* warm-start key; a new key starts a fresh episode    */
    uint64_t seed;        /* Philox key of a fresh episode                       */
    int fresh;            /* restart a known episode from the uniform draw       */
    int reserved0;
} plan_request;

typedef struct {
    int executors, busy, pending, max_wave;
    uint64_t waves, completed;
    size_t device_bytes;
} plan_server_stats;

/* Create a serving loop on the current device.  Errors: EINVAL (bad config),
 * ENOMEM (budget below one executor or allocation failure). */
int plan_server_create(const plan_config* cfg, int max_executors, size_t device_budget,
                       int max_episodes, plan_server** out);

/* Stop the loop, wait for work in flight, release everything.  NULL accepted. */
int plan_server_destroy(plan_server* srv);

/* Queue one request; returns at once with a ticket.  Requests of one episode
 * must be submitted one at a time (after the previous one was polled).
 * Errors: ECAPACITY (B, n_obs or the episode table), EINVAL. */
int plan_submit(plan_server* srv, const plan_request* req, uint64_t* ticket);

/* Wait up to timeout_us for a ticket.  OK: *out holds the best pair and
 * *latency_us (may be NULL) the time from submission to completion; the ticket
 * is released.  ETIMEOUT: not done yet (poll again).  ENONFINITE / ECUDA: the
 * request failed.  EINVAL: unknown ticket. */
int plan_poll(plan_server* srv, uint64_t ticket, plan_result* out, double* latency_us,
              int timeout_us);

/* Wait up to timeout_us for any ticket to complete and take the one that
 * completed first: *ticket names it, and *out / *latency_us / the return
 * value are those plan_poll would give for it.  ETIMEOUT: none completed in
 * time (*ticket is untouched).  EINVAL: srv or ticket is NULL.  Lets a client
 * serve many episodes from one wait instead of polling each ticket. */
int plan_poll_any(plan_server* srv, uint64_t* ticket, plan_result* out, double* latency_us,
                  int timeout_us);

/* Release an episode's warm-start row (no request of it may be pending). */
int plan_end_episode(plan_server* srv, uint64_t episode);

/* Counters of the loop. */
int plan_server_info(plan_server* srv, plan_server_stats* out);

/* ------------------------------------------------------------------- tuning */

/* Shape of the fused FP32 kernel: warps_per_sample (the warps that share one
 * sample's timesteps) and samples_per_cta; valid shapes are (1, 1..8),
 * (2, 1), (2, 2), (2, 4) and (4, 1).  (0, 0) restores the built-in choice.  Clears the captured graphs of plan_step_resident.  Not a stage of
 * the paper's method: it only changes how the work is laid out on the GPU. */
int plan_set_tuning(plan_ctx* ctx, int warps_per_sample, int samples_per_cta);

/* Launch form of the fused FP32 kernel.  With one CTA per tile of
 * samples_per_cta samples, a CTA holds its SM until its slowest sample has
 * finished, and every CTA stages the basis again.  The persistent form
 * launches one wave of CTAs (as many as fit on the SMs at once); each CTA
 * stages the basis once and each sample group takes the next unsolved sample
 * from a device counter until none is left, so no group waits for the other
 * groups of its CTA.  Results are bit-identical between the two forms.  The
 * persistent form exists for the shapes with one warp per sample, and for two
 * warps per sample when m > 128; the other shapes always run one CTA per tile.
 *   PLAN_PERSIST_AUTO (the default): the persistent form when the launch
 *                      holds one scene whose tiles need more than one wave
 *                      of CTAs,
 *   PLAN_PERSIST_OFF:  always one CTA per tile,
 *   PLAN_PERSIST_ON:   the persistent form whenever the shape has one.
 * The counter belongs to the context, so solves of one context must not run
 * concurrently on different streams.  Clears the captured graphs of
 * plan_step_resident.  Errors: EINVAL (unknown mode).  Like plan_set_tuning,
 * it changes only how the work is laid out on the GPU. */
enum { PLAN_PERSIST_AUTO = 0, PLAN_PERSIST_OFF = 1, PLAN_PERSIST_ON = 2 };
int plan_set_persistent(plan_ctx* ctx, int mode);

/* Time every fused-kernel shape on B samples of `scene` (drawn from the
 * uniform first-iteration distribution), keep the fastest for this context and
 * return it.  Synchronous on `stream`; must not overlap other work of the
 * context.  When the environment variable PLAN_TUNE_CACHE names a file, a
 * result for the same (n_coef, m, n_obs, B) is read from it instead of timing
 * and new results are appended to it.  With prec = FP64 it returns (0, 0). */
int plan_autotune(plan_ctx* ctx, const plan_scene* scene, int B, int* warps_per_sample,
                  int* samples_per_cta, void* stream);

/* ------------------------------------------------------------- single stages */

/* Alg. 1 lines 10-13 for one set of B scores: ConstraintEliteSet = the n_c
 * samples with the lowest resid, EliteSet = the q of those with the lowest
 * resid + cu, ties to the lower index.  Writes the q EliteSet indices in
 * ascending order of cost to `elite` (device int, q entries).  All buffers
 * are device memory. */
int plan_select_elites(plan_ctx* ctx, const double* resid, const double* cu, int B,
                       int n_c, int q, int* elite, void* stream);

/* Eqs. (mean_update, cov_update, s_formula) from q elites: p_elite (device,
 * q x d_p) with costs (device, q), mu (device, d_p) and sigma (device,
 * d_p x d_p) updated in place. */
int plan_update_distribution(plan_ctx* ctx, const double* p_elite, const double* cost,
                             int q, double* mu, double* sigma, void* stream);

/* Alg. 1 line 4: draw B samples (device, B x d_p) for outer iteration l
 * (1-based) from N(mu, sigma + cov_eps I) or, when fresh != 0 and l == 1,
 * from the uniform initial distribution of `scene`'s lanes.  mu, sigma are
 * host memory (d_p and d_p x d_p). */
int plan_sample(plan_ctx* ctx, const plan_scene* scene, const double* mu,
                const double* sigma, int fresh, int l, uint64_t seed,
                uint64_t episode_step, int B, double* p, void* stream);

/* ------------------------------------------------ differentiable Step-1 layer */

/* The Step-1 QP of Alg. 1 line 7 as a differentiable layer: the optimization
 * layer of the learned sampler (Sec. IV, "choice of differentiable
 * optimizer"), which keeps the convex cost of Eq. (lower_cost) and the
 * equality constraints and ignores the inequalities.  Each row has its own
 * initial state, as the training trajectories of a sampler do.
 *   p   device, B x d_p   behavioural inputs (Eq. behaviour_param)
 *   b0  device, B x 6     initial state (x, y, vx, vy, ax, ay) per row
 *   xi  device, B x 2 n   output: [c_x | c_y], float64
 * The solution is affine in (p, b0) through the float64 KKT inverse formed at
 * plan_init.  Asynchronous on `stream`.  Errors: EINVAL (NULL buffer, B < 0),
 * ECAPACITY (B > max_samples). */
int plan_qp_forward(plan_ctx* ctx, const double* p, const double* b0, int B, double* xi,
                    void* stream);

/* Vector-Jacobian product of plan_qp_forward: given g = dL/dxi (device,
 * B x 2 n) writes dL/dp (device, B x d_p) and, when grad_b0 is not NULL,
 * dL/db0 (device, B x 6).  The layer is affine, so the product does not
 * depend on the forward inputs.  Errors as plan_qp_forward. */
int plan_qp_backward(plan_ctx* ctx, const double* g, int B, double* grad_p, double* grad_b0,
                     void* stream);

/* ------------------------------------------------ arithmetic ceilings */

/* Measured throughput of the arithmetic the fused kernel is bound by, on the
 * current device: out[0] float32 FMA TFLOP/s, out[1] packed float32x2 FMA
 * TFLOP/s, out[2] float64 FMA TFLOP/s, out[3] MUFU reciprocal square roots
 * (10^12 per s), out[4] the SM count.  Independent FMA chains over 8 CTAs of
 * 256 threads per SM, best of three timed launches.  Synchronous on `stream`;
 * allocates a small sink buffer.  The paper has no counterpart: this measures
 * the roofline's denominators.  Errors: EINVAL (NULL out), ECUDA. */
int plan_probe_alu(double* out, void* stream);

/* Diagnostic of the bounded waits of the tensor-core solve; the paper has no
 * counterpart.  Every mbarrier wait of that kernel gives up after a bound;
 * the kernel then raises an error flag, and the solve calls return
 * PLAN_ETIMEOUT while the device and every context stay usable.  This call
 * runs the same wait on an mbarrier that expects one arrival and gets none,
 * with a bound of wait_us microseconds (1..100000) of SM clock cycles at
 * 2.1 GHz.  It returns PLAN_ETIMEOUT when the wait gave up, which is the
 * expected outcome, and PLAN_OK only if the wait completed.  Synchronous on
 * `stream`; allocates and frees a 4-byte flag.  Errors: EINVAL (wait_us out
 * of range), ECUDA. */
int plan_probe_wait_timeout(int wait_us, void* stream);

/* Issue cost of the two contractions of one Alg. 2 iteration on the tensor
 * cores at a wide N: a CTA of 64 samples of the m = 200, n = 16 workload
 * (N = 128 columns = 64 samples x 2 axes), TF32 MMAs with `passes` 1 (TF32)
 * or 3 (split TF32, the TF32X3 mode), operands staged in shared memory and
 * accumulators in tensor memory; one CTA per SM, `iters` iterations
 * (1..10000).  Only the MMAs are timed (zero operands, results not read).
 * out[0]: SM cycles per iteration of the forward product (3 derivatives x 2
 * row tiles of 128 timesteps x K = 16, M = N = 128); out[1]: the transposed
 * product over K = 768 as M = 128 columns x N = 16 coefficients; out[2]: the
 * same as M = 64 (coefficients, padded) x N = 128 columns; out[3], out[4]:
 * out[1], out[2] with the K steps dealt round-robin to four accumulators;
 * medians over the CTAs; out[5]: the number of CTAs (out holds 6 doubles).  The paper has no counterpart: this is the
 * evidence for where B x (basis) is dense enough for the tensor cores.  Every
 * wait is bounded.  Synchronous on `stream`; allocates small buffers.
 * Errors: EINVAL (NULL out, passes, iters), ETIMEOUT (a wait gave up), ECUDA. */
int plan_probe_tc_wide(int passes, int iters, double* out, void* stream);

/* ------------------------------------------------ allocation-free lower level */

/* The float64 lower-level solve of plan_solve (same kernels, same results) for
 * callers that cannot allocate device memory: code embedded in a host
 * application that owns every device allocation (a fixed, pre-reserved pool
 * that a cudaMalloc would fragment or exceed), and real-time control loops that
 * after start-up must not enter an allocator, whose latency is unbounded and
 * which may synchronise the device.  The paper has no counterpart; this is an
 * integration entry point, not a step of the method.
 *
 * No context is needed and nothing is allocated: no cudaMalloc / cudaFree and
 * no allocating library routine.  The basis, the KKT inverses, a copy of the
 * scene and the per-iteration intermediates live in one fixed __device__ array
 * of about 4.7 MB in the library, which every GPU that loads the library holds
 * until the process exits.  Limits: B <= 256 samples, 8 <= m <= 128 timesteps,
 * n_obs <= 32 obstacles, n_coef <= 16, n_seg <= 4; larger requests return
 * PLAN_ECAPACITY.  Of `cfg` only m, n_coef, n_seg, inner_iters, dt, rho, the
 * gains, the bounds and lane_margin are used (prec and the capacities are
 * ignored; the arithmetic is float64).
 *
 *   p      device, B x d_p        xi     device, B x 2 n_coef, or NULL
 *   resid  device, B              cu     device, B
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every call
 * uses the same array and leaves its contents behind, so two calls whose work
 * overlaps on the GPU (different streams, or concurrent threads) race and give
 * wrong results; serialise them, e.g. on one stream.  Errors are described by
 * plan_last_error(NULL, ...).  Asynchronous on `stream`. */
int plan_solve_fp64_noalloc(const plan_config* cfg, const plan_scene* scene, const double* p,
                            int B, double* xi, double* resid, double* cu, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PLAN_H_ */
