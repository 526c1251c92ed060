/*
 * gpmppi.h -- C ABI of the GB300 chance-constrained GP-MPPI rollout library.
 *
 * The library implements the data-parallel hot path of the chance-constrained
 * GP-MPPI controller of Trivedi et al. (Sec. IV, Alg. 1): K sampled control
 * sequences are propagated over a horizon of T steps through the dynamic
 * unicycle plus a GP residual mean (Eq. 1-3, Eq. 6, Eq. 10), the GP variance is
 * propagated into the state covariance (Eq. 10), every trajectory is scored
 * against lane and obstacle chance constraints tightened by that covariance
 * (Eq. 11-16), and the nominal control is updated by a log-sum-exp stabilised
 * softmax-weighted sum of the sampled controls (Alg. 1, Step 1).
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: GPMPPI_OK (0) or a negative error
 *    code; gpmppi_last_error() returns a thread-local message for the last
 *    failure on the calling thread.  No C++ exception crosses the ABI.
 *  - The caller owns every array argument.  Arrays documented as "device" must
 *    be CUDA device (or managed) memory of the current device; the library
 *    checks the pointer kind and returns GPMPPI_ERR_INVALID_ARG for host
 *    pointers, but it cannot check a device array's length: the caller must
 *    provide at least the documented number of elements.
 *  - Arrays documented as "host" are read or written synchronously before the
 *    function returns (gp_fit, mppi_create, gp_factors, state vectors).
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it and the call returns without
 *    synchronising, except where noted.
 *  - A failed call leaves its outputs unspecified and the handles usable.
 *  - Row-major layouts throughout; float is IEEE binary32, double binary64.
 */
#ifndef GPMPPI_H
#define GPMPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GPMPPI_OK 0
#define GPMPPI_ERR_INVALID_ARG (-1)   /* bad shape, value, pointer kind or handle */
#define GPMPPI_ERR_NOT_PD (-2)        /* K_XX + noise I not positive definite     */
#define GPMPPI_ERR_CUDA (-3)          /* a CUDA runtime call failed               */
#define GPMPPI_ERR_OOM (-4)           /* device allocation failed                 */
#define GPMPPI_ERR_TIMEOUT (-5)       /* a bounded device wait gave up            */
#define GPMPPI_ERR_NONFINITE (-6)     /* NaN or Inf in an input                   */
#define GPMPPI_ERR_UNSUPPORTED (-7)   /* valid request this library does not serve */

/* variance modes (where the tightening covariance comes from) */
#define GPMPPI_VAR_PER_SAMPLE 0   /* each sample's own propagated Sigma (Eq. 10)     */
#define GPMPPI_VAR_NOMINAL 1      /* Alg. 1 Step 2: Sigma along the previous update */

/* arithmetic of the GP variance contraction |L^-1 k*|^2 */
#define GPMPPI_FP32 0         /* FP32 on the CUDA cores                                   */
#define GPMPPI_BF16_SPLIT 1   /* tensor cores: BF16 hi/lo operands, 3 products, FP32 sums */
#define GPMPPI_FP16_SPLIT 2   /* tensor cores: FP16 hi/lo operands, 3 products, FP32 sums */
#define GPMPPI_BF16_SPLIT3 3  /* tensor cores: BF16 hi/mid/lo operands, 6 products, FP32 sums
                                 (the streaming rollout at every N; 24 operand bits)     */

/* limits of this library */
#define GPMPPI_MAX_N 4096         /* GP training points      */
#define GPMPPI_MAX_T 1024         /* horizon                 */
#define GPMPPI_MAX_K (1 << 24)    /* samples                 */
#define GPMPPI_MAX_OBSTACLES 4096
#define GPMPPI_MAX_PATH 65536     /* polyline vertices       */

typedef struct gpmppi_gp_s* gpmppi_gp;       /* opaque, owned by the library */
typedef struct gpmppi_ctrl_s* gpmppi_ctrl;   /* opaque, owned by the library */
typedef struct gpmppi_batch_s* gpmppi_batch; /* opaque, owned by the library */

/* SE-ARD hyper-parameters of one GP output (Sec. III-A; Sec. V-A trains
 * them with GPyTorch, here they are supplied):
 * k(a,b) = signal_var * exp(-1/2 sum_d (a_d - b_d)^2 / lengthscale_d^2),
 * observation noise variance noise_var. */
typedef struct gpmppi_hyper {
    double lengthscale[4];
    double signal_var;
    double noise_var;
} gpmppi_hyper;

/* Controller parameters (Alg. 1 inputs; Eq. 5-9, Eq. 11-16). */
typedef struct gpmppi_params {
    int32_t K;               /* samples per iteration (S in Alg. 1), >= 1           */
    int32_t T;               /* horizon (N in Eq. 5), >= 1                          */
    float dt;                /* Euler step [s]                                      */
    float tau_v, tau_w;      /* first-order lag time constants of f_v, f_omega      */
    float sigma[2];          /* std of the control noise Sigma_sim (v, omega), >= 0 */
    float lambda;            /* MPPI temperature, > 0                               */
    float p_x;               /* chance level of Eq. 7, in (0, 1)                    */
    float u_min[2], u_max[2];/* control box of Eq. 8                                */
    float alpha[5];          /* Eq. 11 weights; alpha[2] (slip) must be 0           */
    float beta[4];           /* Eq. 12 weights: variance, collision, goal distance,
                                terminal miss                                        */
    float P_lane, P_coll;    /* penalties multiplying the two indicators            */
    float lane_half_width;   /* r of Eq. 13, > 0                                    */
    float v_desired;         /* v_desired of Eq. 11                                 */
    uint64_t seed;           /* Philox key                                          */
    int32_t variance_mode;   /* GPMPPI_VAR_*                                        */
    int32_t precision;       /* GPMPPI_FP32, GPMPPI_BF16_SPLIT, GPMPPI_FP16_SPLIT or
                                GPMPPI_BF16_SPLIT3                                  */
    float goal[2];           /* goal position of the Eq. 12 goal terms              */
    float goal_radius;       /* terminal term: penalty when |mu_XY(T) - goal| > this */
    float P_goal;            /* penalty multiplying the terminal indicator          */
} gpmppi_params;

/* Fit the two residual GPs of Sec. III-A (outputs delta_v and delta_omega)
 * on the current CUDA device, in FP64: K_j = k_j(X,X) + noise_var_j I,
 * L_j = chol(K_j), alpha_j = K_j^-1 Y[:,j], and L_j^-1; the rollout uses
 * FP32 copies of alpha_j and L_j^-1 (and BF16 hi/lo parts when requested).
 *   X     host, N x 4 doubles (v, omega, v_cmd, omega_cmd) per row
 *   Y     host, N x 2 doubles (delta_v, delta_omega)
 *   N     0 <= N <= GPMPPI_MAX_N (N = 0 gives the prior: mean 0, var signal_var)
 *   hyper host, two entries (output 0 = delta_v, output 1 = delta_omega)
 *   out   receives the new handle (owned by the library; free with gp_destroy)
 * Blocking: returns after the factorisation finished.
 * Errors: INVALID_ARG, NONFINITE, NOT_PD (Cholesky pivot <= 0), OOM, CUDA. */
int gp_fit(const double* X, const double* Y, int32_t N, const gpmppi_hyper hyper[2],
           gpmppi_gp* out);

/* Release a GP handle.  A controller created from it must be destroyed first. */
int gp_destroy(gpmppi_gp gp);

/* Copy the FP64 factors of output j (0 or 1) to the host (the Cholesky
 * quantities of Sec. III-A that the GP mean and variance are formed from):
 *   Linv  host, N x N doubles, lower triangular L_j^-1 (upper part zero); may be NULL
 *   alpha host, N doubles, K_j^-1 Y[:,j]; may be NULL
 * Blocking. */
int gp_factors(gpmppi_gp gp, int32_t j, double* Linv, double* alpha);

/* GP posterior of the latent residual at M query points (Eq. 3 with one
 * terrain): mean_j = k_j(z,X) alpha_j, var_j = max(0, sf2_j - |L_j^-1 k_j(X,z)|^2).
 *   Z     device, M x 4 floats
 *   mean  device, M x 2 floats (output)
 *   var   device, M x 2 floats (output)
 * FP32 arithmetic on the FP32 factors. */
int gp_predict(gpmppi_gp gp, const float* Z, int32_t M, float* mean, float* var, void* stream);

/* Create a controller for one robot.  The radius tightening factors of the
 * chance constraints (Eq. 13-16: sqrt(chi^2_2(p_x)) for the lane, Phi^-1(p_x)
 * for obstacles) are computed here in double.
 *   p          host, parameters (validated; copied)
 *   obstacles  host, O x 3 floats (centre x, centre y, radius > 0); NULL if O = 0
 *   path       host, P x 2 floats, lane-centre polyline (P >= 1); copied
 *   gp         fitted GP on the current device; must outlive the controller.
 *              Both outputs must share their hyper-parameters (the rollout
 *              evaluates one kernel row and one variance per query).
 * Allocates the controller's device buffers on the current device.
 * Errors: INVALID_ARG, NONFINITE, UNSUPPORTED, OOM, CUDA. */
int mppi_create(const gpmppi_params* p, const float* obstacles, int32_t O, const float* path,
                int32_t P, gpmppi_gp gp, gpmppi_ctrl* out);

/* One MPPI iteration (Alg. 1 Step 1, plus Step 2 in GPMPPI_VAR_NOMINAL mode):
 * sample K perturbed control sequences with Philox4x32-10 (key = seed,
 * counter = (k, s, it_lo, it_hi)), roll each out for T steps with the GP
 * mean and variance, score it, and return the softmax-weighted update.
 *   state    host, 5 floats (X, Y, theta, v, omega): mu_x(0); Sigma_x(0) = 0
 *   U_nom    device, T x 2 floats: nominal controls u(0..T-1)
 *   U_new    device, T x 2 floats (output): U + sum_s w_s (u~_s - U)
 *   weights  device, K floats (output) or NULL
 *   costs    device, K floats (output) or NULL
 * The iteration counter advances by one per successful call.  Calls on one
 * controller must not overlap on the GPU (they share its scratch buffers). */
int mppi_step(gpmppi_ctrl c, const float state[5], const float* U_nom, float* U_new,
              float* weights, float* costs, void* stream);

/* The same iteration with every array on the host, as a receding-horizon
 * controller calls it (Alg. 1 once per control period): copies U_nom in,
 * runs mppi_step on the controller's own staging buffers, copies the results
 * out and returns once they are on the host (the stream is synchronised).
 *   state    host, 5 floats
 *   U_nom    host, T x 2 floats (pinned memory makes the copy asynchronous)
 *   U_new    host, T x 2 floats (output)
 *   weights  host, K floats (output) or NULL
 *   costs    host, K floats (output) or NULL
 * The staging buffers (2 T x 2 floats, plus K floats once weights are asked
 * for) are allocated by the first call and freed with the controller.
 * Errors: as mppi_step; INVALID_ARG for device pointers; OOM; CUDA. */
int mppi_step_host(gpmppi_ctrl c, const float state[5], const float* U_nom, float* U_new,
                   float* weights, float* costs, void* stream);

/* The rollout of mppi_step for the current iteration (Alg. 1 Step 1),
 * recording every sample's trajectory: the mean and covariance of Eq. 6 and
 * Eq. 10 and the stage costs and margins of Eq. 11-16 (does not update U and
 * does not advance the counter):
 *   mu      device, K x T x 5 floats: state after step k (mu(k+1)), or NULL
 *   sigma   device, K x T x 15 floats: upper triangle of Sigma(k+1), row by row
 *           (00,01,02,03,04,11,12,13,14,22,23,24,33,34,44), or NULL
 *   stage   device, K x T floats: stage cost of step k, or NULL
 *   margins device, K x T x 2 floats: (e - r_bar, min_j d_bar_j); the lane
 *           indicator fires when the first is > 0, the collision indicator
 *           when the second is <= 0 (+inf without obstacles), or NULL
 *   costs   device, K floats: summed costs, or NULL */
int mppi_rollout_trace(gpmppi_ctrl c, const float state[5], const float* U_nom, float* mu,
                       float* sigma, float* stage, float* margins, float* costs, void* stream);

/* Set / read the MPPI iteration counter (Philox counter words 2 and 3). */
int mppi_set_iteration(gpmppi_ctrl c, uint64_t it);
int mppi_get_iteration(gpmppi_ctrl c, uint64_t* it);

/* GPMPPI_VAR_NOMINAL: the tightening covariance carried to the next call
 * (Alg. 1 Step 2), T x 3 floats (Sxx, Sxy, Syy) of Sigma_XY(k+1), device. */
int mppi_nominal_sxy(gpmppi_ctrl c, float* sxy, void* stream);

/* Which rollout kernel mppi_step runs for this controller (host int32):
 * GPMPPI_KERNEL_FP32 (CUDA cores), GPMPPI_KERNEL_TC_STREAM (tensor cores,
 * factor tiles streamed per step), GPMPPI_KERNEL_TC_CLUSTER (tensor cores,
 * factor resident in a CTA cluster; split precisions with N <= 512 when the
 * cluster fits the device) or GPMPPI_KERNEL_ENSEMBLE (FP32 terrain ensemble;
 * a terrain ensemble in the split precisions reports GPMPPI_KERNEL_TC_STREAM). */
#define GPMPPI_KERNEL_FP32 0
#define GPMPPI_KERNEL_TC_STREAM 1
#define GPMPPI_KERNEL_TC_CLUSTER 2
#define GPMPPI_KERNEL_ENSEMBLE 3
int mppi_rollout_kind(gpmppi_ctrl c, int32_t* kind);

/* Per-kernel timing of mppi_step.  When enabled, mppi_step records CUDA
 * events on its stream around the rollout kernel and around the update
 * kernel(s); mppi_last_profile waits for the last step's events and returns
 * the two durations in milliseconds (host floats).  mppi_grad records the
 * same pair around its adjoint kernel and around the rest (Gram trace and
 * reductions); the last call of either is reported.  Off by default. */
int mppi_set_profiling(gpmppi_ctrl c, int32_t on);
int mppi_last_profile(gpmppi_ctrl c, float* rollout_ms, float* update_ms);

/* Device-side status of the controller's kernels since the last check:
 * GPMPPI_OK, or GPMPPI_ERR_TIMEOUT when a rollout kernel gave up a bounded
 * wait for one of its shared-memory tile copies (its outputs are then
 * invalid).  Synchronises the device; clears the status. */
int mppi_device_status(gpmppi_ctrl c);

/* Release a controller and its device buffers (synchronises its device). */
int mppi_destroy(gpmppi_ctrl c);

/* Terrain ensemble (Eq. 3): a controller whose residual model is the
 * mixture of M terrain GP pairs, mean sum_i w_i m_i(z) and variance
 * sum_i w_i^2 var_i(z) per output.  gps: M fitted GPs (host array of
 * handles; each terrain's two outputs must share hyper-parameters; the
 * controller keeps them alive as mppi_create does), weights: host, M floats
 * (any finite values; Eq. 4 keeps them on the simplex).  2 <= M <= 8, or
 * M = 1 (weight 1 gives the single-GP controller of mppi_create).  Needs
 * the per-sample variance mode (else GPMPPI_ERR_UNSUPPORTED).  In FP32 the
 * ensemble rollout runs on the CUDA cores; in the split precisions the
 * streaming tensor-core rollout runs over the GPs' factors stacked
 * block-diagonally (each GP's block count rounded up to even; UNSUPPORTED
 * when the GPs' training sets do not fit shared memory together).
 * mppi_step and mppi_rollout_trace use it; mppi_grad rejects it; the batch
 * API takes it in the split precisions only.
 * mppi_set_terrain_weights replaces the weights (host, M floats) for the
 * following steps, e.g. with the result of terrain_weights. */
int mppi_create_ensemble(const gpmppi_params* p, const float* obstacles, int32_t O, const float* path,
                         int32_t P, const gpmppi_gp* gps, int32_t M, const float* weights,
                         gpmppi_ctrl* out);
int mppi_set_terrain_weights(gpmppi_ctrl c, const float* weights, int32_t M);

/* Terrain-weight estimation, Eq. 4 (Alg. 1 Step 3), on the host:
 *   w* = argmin |Yv - Fv w|^2 + |Yw - Fw w|^2 + gamma |w - w_prev|_1
 *        s.t. 0 <= w_i <= 1, sum w_i = 1.
 *   Yv, Yw   host, H doubles: observed velocity residuals over the last H steps
 *   Fv, Fw   host, H x M doubles row-major: the terrains' GP mean predictions
 *            (e.g. from gp_predict) at the same inputs
 *   w_prev   host, M doubles; gamma >= 0; w_out host, M doubles (output)
 * Exact: every pattern of active bounds and L1 kinks is solved as a small KKT
 * system (4^M of them, 1 <= M <= 8) and the feasible candidate of least
 * objective returned.  Pure host computation; no device is touched.
 * Errors: INVALID_ARG, NONFINITE. */
int terrain_weights(const double* Yv, const double* Yw, const double* Fv, const double* Fw, int32_t H,
                    int32_t M, const double* w_prev, double gamma, double* w_out);

/* Gradient of the smoothed chance-constrained rollout cost (adjoint rollout).
 * J(U, l) = sum_s w_s S_s, where S_s is the cost of sample s over the horizon
 * (Alg. 1 Step 1: Eq. 6 and 10 for mean and covariance, Eq. 11-16 for the
 * stage cost) with the lane and collision indicators of Eq. 11-12 replaced by
 * logistic sigmoids of slope * (e - r_bar) and -slope * min_j d_bar_j, and the
 * control noise fixed at the draws of the controller's current iteration
 * (the counter is not advanced).  The gradient is exact for that smoothed
 * cost up to FP32 rounding, taken by a reverse pass over the horizon that
 * stores the state every ceil(sqrt(T)) steps and recomputes each segment;
 * derivatives of sqrt(lambda_max) and sqrt(n^T Sigma n) are taken as zero
 * where their argument is zero (Sigma_XY(1) = 0), and those of the clamps
 * (Eq. 8, the variance at zero) as zero outside the box.
 *   state          host, 5 floats (x0)
 *   U_nom          device, T x 2 floats
 *   sample_weights device, K floats w_s, or NULL for w_s = 1/K
 *   slope          sigmoid slope > 0 (20 in the differentiable workload)
 *   J              device, 1 float (output)
 *   dU             device, T x 2 floats dJ/dU (output), or NULL to evaluate J only
 *   dlengthscale   device, 2 x 4 floats dJ/dl_{o,d} for output o (v, omega) and
 *                  GP input d (output), or NULL.  It includes the dependence of
 *                  alpha = K^-1 y and K^-1 on the lengthscales (one more kernel
 *                  and T * K * N floats of scratch)
 * Needs variance mode GPMPPI_VAR_PER_SAMPLE (else GPMPPI_ERR_UNSUPPORTED) and
 * enough shared memory for 2 x 8 x N floats (GPMPPI_ERR_UNSUPPORTED beyond).
 * The first call, and the first call asking for dlengthscale, allocate
 * device scratch owned by the controller (freed by mppi_destroy) and may
 * synchronise.  Runs on the controller's FP32 path whatever its precision. */
int mppi_grad(gpmppi_ctrl c, const float state[5], const float* U_nom, const float* sample_weights,
              float slope, float* J, float* dU, float* dlengthscale, void* stream);

/* Allocation-free weights-and-update step (the paper has no counterpart;
 * this is a deployment aid).  Some callers cannot allocate device memory
 * once running: a controller in a real-time loop whose memory is fixed at
 * start-up (cudaMalloc may synchronise the device and has no latency bound),
 * or a framework that owns all device memory and forbids plug-ins from
 * allocating.  This call runs the same softmax weights and control update as
 * mppi_step's second kernel (Alg. 1: w_s = exp(-(S_s - rho)/lambda) / Z with
 * rho = min_s S_s, then the weighted sum of the perturbations), with its
 * scratch (per-CTA partial sums, per-block softmax statistics and a
 * completion ticket) in a fixed static device array of 1 MiB that every GPU
 * loading the library holds until the process exits.  It allocates nothing.
 *   costs    device, K floats: the samples' total costs S_s
 *   u_tilde  device, T x K x 2 floats, step-major: the clamped sampled
 *            controls u~ of sample s at step k at [(k*K + s)*2 + {0,1}]
 *   U_nom    device, T x 2 floats; U_new device, T x 2 floats (output,
 *            U_nom + sum_s w_s (u~_s - U_nom)); weights device, K floats or NULL
 *   lambda   temperature > 0
 * Limit: ceil(K / 256) * T <= 65536 (and T <= GPMPPI_MAX_T); larger sizes
 * return GPMPPI_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  All calls share the one array, so calls that overlap
 * on the GPU (other streams, other host threads) race: serialise them. */
int mppi_update_noalloc(const float* costs, const float* u_tilde, const float* U_nom,
                        float* U_new, float* weights, int32_t K, int32_t T, float lambda,
                        void* stream);

/* ---- Batched iterations of many independent controllers (Alg. 1 run for
 * several robots at once; each controller keeps its own GP, scene, sizes
 * K, T, N, obstacles and precision). ---------------------------------------
 *
 * mppi_batch_create groups B distinct controllers of the current device
 * (per-sample variance mode only).  The batch owns device buffers for every
 * controller's state (5 floats), nominal controls U_nom (T x 2), result U_new
 * (T x 2) and weights (K); mppi_batch_buffers returns their device addresses
 * (and that of the controller's cost array, K floats).  The caller writes
 * states and U_nom there (e.g. cudaMemcpyAsync) before a step and reads the
 * results after it.  The Philox iteration counter of each controller lives in
 * device memory while batched: it starts from the controller's counter at
 * creation, advances by one per batched step, and is read back with
 * mppi_batch_get_iteration (the controller's own counter is not updated).
 * A step = ONE persistent rollout launch (one CTA per SM) whose CTAs take
 * (controller, sample tile) items from an atomic work queue - FP32 tiles and
 * FP16- or BF16-split tensor-core tiles alike, longest first - then one update
 * launch for all controllers.  Controllers whose own mppi_step would use the
 * cluster rollout (N <= 512) run the streaming tensor-core body here; terrain
 * ensembles in the split precisions are items like single-GP controllers
 * (their weights as set on the controller when a step is enqueued); FP32
 * terrain ensembles give GPMPPI_ERR_UNSUPPORTED. */
int mppi_batch_create(const gpmppi_ctrl* ctrls, int32_t B, gpmppi_batch* out);
int mppi_batch_buffers(gpmppi_batch b, int32_t i, float** state, float** U_nom, float** U_new,
                       float** weights, float** costs);
/* One iteration of every controller, enqueued on stream (NULL = legacy). */
int mppi_batch_step(gpmppi_batch b, void* stream);
/* The same iteration through a CUDA graph: captured on first use (stream
 * must be a created stream, not NULL) and replayed by every later call. */
int mppi_batch_graph(gpmppi_batch b, void* stream);
/* Autotuner, per controller shape (precision, K, T, N, lane segments,
 * obstacles): times one wave of the controller's tiles for each tensor-core
 * tile layout (2, 4 or 8 producer threads per sample, i.e. 128, 64 or 32
 * samples per tile; FP32 controllers have one layout), keeps the layout with
 * the least SM time (tiles x time per tile) and orders the work queue by the
 * measured time per tile.  Results are kept for the process and reused for
 * the same shape.  Runs rollouts only (their outputs are scratch; iteration
 * counters do not move).  Blocking.  *chosen = number of controllers whose
 * layout changed. */
int mppi_batch_autotune(gpmppi_batch b, void* stream, int32_t* chosen);
/* The tile layout of controller i in the batch: producer threads per sample of
 * its tensor-core tiles (0 for an FP32 controller) and the time per tile that
 * orders the work queue (microseconds: measured by the autotuner, else an
 * estimate). */
int mppi_batch_layout(gpmppi_batch b, int32_t i, int32_t* threads_per_sample, float* tile_us);
int mppi_batch_get_iteration(gpmppi_batch b, int32_t i, uint64_t* it);
int mppi_batch_destroy(gpmppi_batch b);

/* Raw Philox4x32-10 blocks as the kernels draw them (Salmon et al., SC'11):
 *   ctr  device, M x 4 uint32 counters; out device, M x 4 uint32 words. */
int gpmppi_philox(uint64_t seed, const uint32_t* ctr, int32_t M, uint32_t* out, void* stream);

/* The control perturbations eps (K x T x 2 floats, device) of one iteration,
 * as the rollout draws them before clamping (Alg. 1 "Sample eps^s"). */
int gpmppi_control_noise(uint64_t seed, int32_t K, int32_t T, uint64_t it, const float sigma[2],
                         float* eps, void* stream);

/* Tensor-core self-test (diagnostic): D = A B^T on one CTA with the
 * library's tcgen05 operand layout, descriptors and TMEM path.
 *   fmt      0 = FP16, 1 = BF16 (A and B share it)
 *   N        64, 128 or 256 (rows of B, columns of D); K 16, 32, 48 or 64
 *   variant  0 = the library's descriptor convention; 1 = leading and stride
 *            byte offsets exchanged (N <= 128), to show which one the
 *            hardware expects; 2 = A written to tensor memory (one row per
 *            lane, tcgen05.st) and read from there by the MMA
 *   A device 128 x K, B device N x K (16-bit, row-major), D device 128 x N floats
 * Blocking; GPMPPI_ERR_TIMEOUT if the MMA completion did not arrive. */
int gpmppi_mma_selftest(int32_t fmt, int32_t N, int32_t K, int32_t variant, const uint16_t* A,
                        const uint16_t* B, float* D);

/* Throughput probe of one arithmetic unit (measurement tool for roofline
 * denominators; no counterpart in the paper): blocks x 256 threads each run
 * iters iterations of 16 independent chains of one instruction,
 *   kind 0  fma.rn.f32 (FP32 FMA pipe), kind 1  fma.rn.f32x2 (packed pairs,
 *           counted as two FMAs each), kind 2  ex2.approx.ftz.f32 (SFU);
 * i.e. blocks * 256 * iters * 16 operations.  out: device, blocks * 256
 * floats (one result per thread, so that nothing is optimised away).
 * Asynchronous on stream; time it with events on that stream. */
int gpmppi_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float* out, void* stream);

/* Failure-detection hook (no counterpart in the paper) for the FP32
 * CUDA-core rollout of this controller:
 *   ns            time limit of each bounded wait for a tile copy of L^-T, in
 *                 nanoseconds (default 2e9)
 *   expire_first  non-zero: before any copy, one warp of every CTA waits,
 *                 bounded by ns, on an mbarrier that nothing arrives on, so
 *                 that the wait runs out
 * A wait that runs out records GPMPPI_ERR_TIMEOUT in the controller's status
 * word (mppi_device_status reports and clears it) and stops that warp's copies;
 * the copies in flight land (bounded) before the CTA exits and the kernel ends
 * normally, so the context stays usable; that step's outputs are unspecified.
 * A host-side setting of this controller only (not applied in batches); no GPU
 * setting is changed. */
int mppi_set_wait_limit(gpmppi_ctrl c, uint64_t ns, int32_t expire_first);

/* Thread-local message describing the last failed call ("" if none). */
const char* gpmppi_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int gpmppi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GPMPPI_H */
