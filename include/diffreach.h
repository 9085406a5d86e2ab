/*
 * diffreach.h -- C ABI of the B300 (sm_103a) reachability library.
 *
 * The library bounds the reachable sets of the discrete-time closed loop
 *     x_{t+1} = A x_t + B pi(x_t) + e,      pi = ReLU MLP with L affine layers,
 * over a horizon H, for D independent domains (input sub-boxes or branch domains),
 * with the paper's fixed-shape linear Taylor model (TM) x = c + P zeta + r,
 * zeta in [-1,1]^n, r in [I_lo, I_hi] (Sec. IV-A), certified through the
 * controller by shared-slope CROWN back-substitution (Thm. 2, Sec. IV-C) over a
 * TM input (Thm. 3 and its proof in App. B), propagated stepwise as in Alg. 2
 * with the closed-loop remark of Sec. IV-E, and concretised with EvalInt
 * (Alg. 2).  The differentiable objective is the tube-volume proxy
 * V_d = sum_{t=1..H} sum_i width(box_{t,i}) of Sec. V-A; slopes are refined by
 * projected gradient ("gradient-based refinement", Sec. VI-A, Table I).
 *
 * Conventions for every entry point:
 *  - The return value is DR_OK (0) or a negative DR_ERR_* code; dr_last_error()
 *    returns a message for the last failing call on that context.
 *  - Host inputs are copied during the call; the caller keeps ownership.
 *    Device pointers (flag on_device != 0) must be device memory of the context's
 *    device, stay valid until the context's stream has completed the call, and are
 *    only read (inputs) or written (outputs).
 *  - All device work is ordered on the context's CUDA stream.  Calls that return
 *    results into host memory synchronise that stream before returning.
 *  - Arrays are dense, C order, without padding.  Shapes are given in brackets.
 *  - There is no CPU fallback: without a usable sm_103a device dr_create fails.
 */
#ifndef DIFFREACH_H
#define DIFFREACH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DR_OK 0
#define DR_ERR_ARG (-1)       /* invalid argument (null pointer, negative size, bad enum) */
#define DR_ERR_SHAPE (-2)     /* shapes inconsistent or beyond the supported limits       */
#define DR_ERR_STATE (-3)     /* call order: e.g. bounds before controller/dynamics/boxes  */
#define DR_ERR_OOM (-4)       /* device allocation failed or the memory cap was exceeded   */
#define DR_ERR_CUDA (-5)      /* a CUDA runtime call failed                                */
#define DR_ERR_TIMEOUT (-6)   /* a bounded device-side wait expired                        */
#define DR_ERR_NONFINITE (-7) /* non-finite input values                                   */

/* element types of controller parameters */
#define DR_F32 0
#define DR_F64 1

/* slope rules for unstable ReLUs, lower alpha*z, upper alpha*z + max(-alpha*l, (1-alpha)*u) */
#define DR_SLOPE_ADAPTIVE 0 /* alpha = 1 if u >= -l else 0                          */
#define DR_SLOPE_CHORD 1    /* alpha = u / (u - l)                                   */
#define DR_SLOPE_ZERO 2     /* alpha = 0                                             */
#define DR_SLOPE_USER 3     /* alpha from dr_set_alpha / dr_optimize_slopes          */

/* arithmetic of the back-substitution chain Lambda <- Lambda diag(s) W */
#define DR_PREC_AUTO 0   /* fused FP32 kernel for narrow controllers, tensor cores otherwise */
#define DR_PREC_SIMT 1   /* FP32 on CUDA cores                                              */
#define DR_PREC_TF32X3 2 /* FP32-accurate 3xTF32 split on tcgen05 tensor cores              */

/* per-domain status bits written by dr_compute_bounds */
#define DR_STATUS_NONFINITE 1u  /* some bound is inf/nan                                     */
#define DR_STATUS_INFEASIBLE 2u /* a split left l > u: the domain is empty, bounds vacuous   */
#define DR_STATUS_MARGIN 4u     /* a row of the controller pass summed terms of more than 256x
                                   the Taylor model's scale (max_i |c_i| + sum_k |P_ik| + max |I_i|):
                                   beyond the range the default box_margin was calibrated on, so
                                   its FP32 rounding may exceed the margin; dr_options.rigorous
                                   gives guaranteed boxes (never set in rigorous mode)          */

typedef struct dr_ctx dr_ctx;

/* One ReLU split of a branch domain: at step t (0-based), hidden layer `layer`
 * (1-based, 1..L-1) and neuron `neuron` (0-based) the domain only contains states
 * with sign * z >= 0 (sign = +1 or -1). */
typedef struct dr_split {
    int32_t t;
    int32_t layer;
    int32_t neuron;
    int32_t sign;
} dr_split;

typedef struct dr_options {
    int32_t slope_mode;    /* DR_SLOPE_*, default DR_SLOPE_CHORD                                */
    int32_t precision;     /* DR_PREC_*, default DR_PREC_AUTO                                   */
    double margin_rho;     /* optional outward margin inside the pass: every FP32 concretisation
                              (pre-activation bounds, controller remainder, split constraint)
                              is widened by rho * S, S the L1 magnitude of its summed terms.
                              Default 0: such margins compound through the closed loop.      */
    int64_t chunk_domains; /* domains per device pass of the staged path (bounds its scratch) and
                              at most this many per launch of the reverse sweep;
                              0 = automatic: the fewest equal chunks per lane that 24 GiB of
                              scratch holds, at most a quarter
                              of the free device memory and within mem_cap_bytes              */
    int64_t mem_cap_bytes; /* cap on library-owned device memory; 0 = no cap                    */
    double box_margin;     /* outward margin of every reported box: lo -= b*S_box, hi += b*S_box,
                              S_box = |c| + sum|P| + |I| + |w| + sum|v| of the FP64 Taylor model;
                              default 2^-18, calibrated to cover the measured deviation of the
                              FP32 controller pass from FP64 arithmetic (it does not feed back
                              into the Taylor model)                                        */
    int32_t tuning;        /* 0 = pick the fused kernel's launch shape by timing the candidates on
                              first use (cached per architecture and widths; file DR_TUNE_CACHE
                              if set), and the tensor-core GEMM's launch shape per GEMM shape
                              (persistent or one tile per CTA, 128/64/32 columns; timed on the
                              first pass outside a graph capture, cached per process and in the
                              file DR_GEMM_TUNE_CACHE if set; see dr_gemm_tuning_report),
                              1 = no search (first candidate that fits;
                              the GEMM heuristic), 2 + v = use
                              candidate v (0..9; DR_ERR_SHAPE if it does not fit the controller):
                              0..2 one warp per domain (16/8/4 warps per CTA; two hidden layers,
                              n, m <= 8, hidden widths <= 128), 3..9 several domains per CTA;
                              100 + g = the tensor-core GEMM's launch shape g (1..6, see
                              dr_gemm_tuning_report) for every GEMM, the fused kernels untuned */
    int32_t graphs;        /* 0 = dr_compute_bounds captures its launch sequence in a CUDA graph on
                              the second call with unchanged buffers, options and slope mode, and
                              replays it afterwards (needs a stream other than the legacy default
                              stream; any capture failure falls back to plain launches); 1 = never */
    int32_t timing;        /* 1 = time every tensor-core GEMM launch with a pair of CUDA events on the
                              stream it is launched on (read with dr_kernel_timing); passes then run
                              as plain launches, not graph replays.  0 (default) = off            */
    int32_t rigorous;      /* 1 = rigorous rounding for dr_compute_bounds: every FP32 product and sum
                              of the controller pass carries a worst-case error bound (gamma(K)
                              times the sum of its terms' magnitudes, IEEE round-to-nearest), summed
                              with the intercepts and added outward to the pre-activation bounds and
                              the controller TM's remainder; intercepts round up; the FP64 dynamics
                              widen the remainder by 2^-47 of their terms' magnitude.  The chain then
                              runs on CUDA cores (the tensor cores' accumulation rounding is not
                              documented) on the staged path.  The boxes enclose the reachable sets
                              of the real-number closed loop; they are wider than FP64 arithmetic
                              without error terms gives.  The reverse sweep and refinement ignore
                              it.  0 (default) = the calibrated box_margin only                  */
    int32_t weight_grad;   /* 1 = dr_backward also forms the gradient with respect to the controller's
                              weights and biases (read with dr_get_weight_gradient); costs about one
                              more product per chain level in the reverse sweep and a per-domain
                              slice of the parameters (at most 512 MiB, the sweep runs in chunks of
                              domains).  0 (default) = off                                        */
    int32_t reverse;       /* engine of the reverse sweep (dr_backward, dr_optimize_slopes) for controllers
                              too wide for the fused kernels' shared memory: 0 (default) = staged: the
                              forward pass of a chunk of domains keeps every step's chain levels,
                              bounds and Taylor models in device memory (chunks sized to a memory
                              budget), and the reverse chain products run on the tensor cores (3xTF32;
                              targets of width not a multiple of 32, and DR_PREC_SIMT, on CUDA cores);
                              1 = the fused kernels (out of per-domain global-memory slabs for wide
                              controllers, levels recomputed per step); 2 = the staged sweep for any
                              controller width.  The weight gradient always uses the fused kernels;
                              under 0, narrow controllers use them too.                           */
} dr_options;

/* Paper: no passage; the engine of Sec. IV runs batched on a single GPU (Sec. VI), and a context
 * is this library's handle for that device and its stream.
 * Create a context on `device` whose work is ordered on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Fails with DR_ERR_CUDA if the device is missing
 * or is not compute capability 10.3.  *out receives the context. */
int dr_create(dr_ctx** out, int device, void* cuda_stream);

/* Paper: no passage (resource management).
 * Release the context and all device memory it owns (after draining its stream). */
void dr_destroy(dr_ctx* ctx);

/* Paper: the neural component that CROWN certifies (Thm. 2, Sec. IV-C), here the ReLU feedback
 * controller of the discrete-time loop (closing remark of Sec. IV-E).
 * Controller pi: L affine layers; widths[0..L] = (n, n_1, ..., n_{L-1}, m).
 * W[l] points to n_{l+1} x n_l row-major values (layer l+1), b[l] to n_{l+1} values,
 * both host memory of element type `dtype` (DR_F32 or DR_F64).  The device computes in
 * FP32 (values are rounded once).  ReLU follows every layer but the last. */
int dr_load_controller(dr_ctx* ctx, int L, const int32_t* widths, const void* const* W,
                       const void* const* b, int dtype);

/* Paper: the one-step map x_{k+1} = f(x_k, u_k) of Sec. IV-E and Alg. 2, read here as linear
 * dynamics driven by the controller output u_k = pi(x_k).
 * Dynamics x' = A x + B u + e: A [n x n], B [n x m], e [n] (NULL = 0), host FP64.
 * n and m must match the controller's input and output widths. */
int dr_load_dynamics(dr_ctx* ctx, int n, int m, const double* A, const double* B, const double* e);

/* Paper: the initial box X_0 = [x_lo, x_hi] of Alg. 2 (B_eps(x_hat) of Sec. III-A), one per domain;
 * many sub-boxes of one initial set are the input splitting of Sec. VI-A (Table I).  Each box is
 * turned into a linear TM by BuildLinearTM (Alg. 2) inside dr_compute_bounds.
 * D initial boxes [lo, hi] (each [D x n], FP64, lo <= hi), host (on_device = 0) or device.
 * Resets the slopes (alpha), the split list and the multipliers (beta). */
int dr_set_boxes(dr_ctx* ctx, int64_t D, const double* lo, const double* hi, int on_device);

/* Paper: no passage.  Split constraints and their multipliers beta come from beta-CROWN, which the
 * paper only cites; the Lagrangian dual used here is this library's reading of how a split enters
 * a shared-slope TM bound.
 * Branch-domain splits in CSR form: domain d owns s[row_ptr[d] .. row_ptr[d+1]), sorted
 * by (t, layer).  row_ptr [D+1] (row_ptr[0] = 0, non-decreasing), s [nnz], beta [nnz]
 * multipliers >= 0 (NULL = all 0); host memory.  Every concretisation after a split's own
 * layer uses the Lagrangian dual min_zeta p^T zeta >= -|p - sum beta_k g_k|_1 - sum beta_k h_k
 * of the split constraints g_k^T zeta + h_k >= 0. */
int dr_set_splits(dr_ctx* ctx, const int64_t* row_ptr, const dr_split* s, const float* beta);

/* Paper: the planned or exogenous inputs {u_k} of Alg. 2 and the sampled action sequences of
 * reachability-aware MPC (Sec. V-B).  Per-domain, per-step offsets of the dynamics,
 *     x_{t+1} = A x_t + B pi(x_t) + e + e_off[d, t],
 * e_off [D x H x n] FP64, host (on_device = 0) or device memory; NULL removes them.  With the state
 * augmented by the planned input, y = [x; u], A = [[0 (or I), 0], [0, 0]], B = [[I], [0]] and
 * e_off[d, t] = [0; u_{d,t+1}], the loop is the neural dynamics y_{t+1} = f(x_t, u_t) of Alg. 2 (the
 * initial box carries u_{d,0} as a point), each domain one action sequence.  Set after the boxes and
 * horizon; dr_set_boxes and a new horizon remove them.  DR_ERR_NONFINITE for a non-finite host value. */
int dr_set_step_offsets(dr_ctx* ctx, const double* e_off, int on_device);

/* Paper: the gradient of the reachable-set objective with respect to the planned inputs, which the
 * planner of Sec. V-B refines.  After dr_backward: g [D x (H+1) x n] FP64, the gradient of the
 * objective dr_backward differentiated with respect to a shift of the Taylor-model centre at step t
 * (t = 0: the initial box centre; t >= 1: an offset added after step t-1).  For the augmented
 * neural-dynamics form above, g[d, t, n_x:] is dV/du_{d,t} for t = 0..H-1.  DR_ERR_STATE if no
 * dr_backward ran since the problem changed. */
int dr_get_shift_gradient(dr_ctx* ctx, double* g, int on_device);

/* Paper: the horizon H of Alg. 2.
 * Horizon H >= 1 (number of controller/dynamics steps). */
int dr_set_horizon(dr_ctx* ctx, int H);

/* Paper: slope_mode selects the relaxation under the shared-slope constraint of Sec. IV-C (the
 * paper fixes no rule); the other fields are numerics and resource limits with no passage.
 * Options (copied).  NULL restores the defaults. */
int dr_set_options(dr_ctx* ctx, const dr_options* opt);

/* Paper: Alg. 2 (BuildLinearTM, then per step the CROWN certification of Thm. 3 and EvalInt),
 * with the closed loop of Sec. IV-E; the hull is the union over input splits of Sec. VI-A.
 * Bounds for all domains and steps (Alg. 2):
 *   lo, hi          [D x (H+1) x n]  box of every domain and step (step 0 = the input box)
 *   hull_lo/hull_hi [(H+1) x n]      min/max over domains without DR_STATUS_INFEASIBLE
 *   status          [D]              DR_STATUS_* bits
 * Any output may be NULL.  out_on_device selects device (1) or host (0) outputs.
 * Boxes are FP64, concretised in FP64 from the FP64 TM and pushed outward by box_margin. */
int dr_compute_bounds(dr_ctx* ctx, double* lo, double* hi, double* hull_lo, double* hull_hi,
                      uint32_t* status, int out_on_device);

/* Per-domain tube-volume proxy V_d of the last dr_compute_bounds / dr_optimize_slopes
 * (Sec. V-A), [D] FP64. */
int dr_get_objective(dr_ctx* ctx, double* V, int on_device);

/* Paper: "gradient-based refinement" of Sec. VI-A (Table I, 20 iterations), minimising the
 * tube-volume proxy of Sec. V-A; the update rule and keep-best are this library's reading.
 * Projected-gradient refinement: alpha <- clip(alpha - lr_alpha dV/dalpha, 0, 1),
 * beta <- max(beta - lr_beta dV/dbeta, 0), keeping per domain the best (alpha, beta, V).
 * If no slopes were set, they start at the CHORD slopes.  V_out [steps+1] (host, may be
 * NULL) receives sum_d best V_d after each evaluation.  Afterwards the context holds the
 * best slopes and multipliers and slope mode DR_SLOPE_USER.  The first step runs as plain launches;
 * the others replay one captured CUDA graph of a step when dr_options.graphs is 0 and the context
 * has a stream other than the legacy default stream. */
int dr_optimize_slopes(dr_ctx* ctx, int steps, double lr_alpha, double lr_beta, double* V_out);

/* Paper: the gradient of a reachable-set objective that Sec. V-A (L_reach) and the refinement of
 * Sec. VI-A differentiate, taken here with respect to the relaxation slopes and split multipliers.
 * Reverse-mode gradient of the scalar sum_{d,t,i} (g_lo[d,t,i] * lo[d,t,i] + g_hi[d,t,i] * hi[d,t,i])
 * at the current slopes (DR_SLOPE_USER; the slopes of the current mode otherwise, with dalpha 0):
 *   dV_dlo, dV_dhi [D x (H+1) x n] FP64 upstream gradients g_lo, g_hi of the boxes (NULL for both =
 *   the tube-volume proxy V, i.e. g_lo = -1 and g_hi = +1 on steps 1..H; one NULL = zeros);
 *   dalpha [D x H x hidden] FP32; dbeta [nnz] FP32.  Step 0 (the input box) carries no gradient.
 * Pointers are host memory unless on_device != 0.  Recomputes the forward pass with a per-step tape
 * (library-owned, D*H*(n^2+4n+2) doubles) and runs the fused reverse sweep, which recomputes each
 * step's back-substitution levels from the tape.  Controllers whose per-domain working set exceeds
 * shared memory run the same kernels out of library-owned per-CTA global-memory slabs (up to 2 GiB). */
int dr_backward(dr_ctx* ctx, const double* dV_dlo, const double* dV_dhi, float* dalpha, float* dbeta,
                int on_device);

/* Paper: the certified-training loss of Sec. V-A differentiates the reachable-set objective with
 * respect to the model's parameters; here the controller's parameters theta = (W_l, b_l).
 * The gradient of the same scalar as the last dr_backward (which must have run with
 * dr_options.weight_grad = 1), summed over all domains, with respect to the FP32 weights and biases
 * the device computes with, through every path: the controller TM of each step, the pre-activation
 * bounds that set the relaxation offsets (and, outside DR_SLOPE_USER, the slopes), and the split
 * constraints.  dW [sum_l n_{l+1} n_l] FP64 packed as dr_static_args.W (layer after layer, row-major
 * n_{l+1} x n_l), db [sum_l n_{l+1}] FP64 packed likewise; either may be NULL.  Host memory unless
 * on_device != 0.  DR_ERR_STATE when no such dr_backward ran since the controller, dynamics, domains,
 * horizon or splits changed. */
int dr_get_weight_gradient(dr_ctx* ctx, double* dW, double* db, int on_device);

/* Paper: the shared slope of each unstable ReLU under the shared-slope constraint (Sec. IV-C).
 * Slopes alpha [D x H x hidden] FP32 (hidden = n_1 + ... + n_{L-1}, layers concatenated);
 * only unstable neurons read them.  dr_set_alpha switches the slope mode to DR_SLOPE_USER. */
int dr_get_alpha(dr_ctx* ctx, float* alpha, int on_device);
int dr_set_alpha(dr_ctx* ctx, const float* alpha, int on_device);

/* Paper: no passage (beta-CROWN multipliers, only cited by the paper; see dr_set_splits).
 * Split multipliers beta [nnz] FP32 (>= 0). */
int dr_get_beta(dr_ctx* ctx, float* beta, int on_device);
int dr_set_beta(dr_ctx* ctx, const float* beta, int on_device);

/* ---- allocation-free slope gradient ----------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory, e.g. code running inside a custom memory pool or a real-time loop that forbids
 * cudaMalloc/cudaFree (which may synchronise the device), or a host that owns all GPU memory
 * itself.  It computes the same gradient as dr_backward (dV/dalpha of the tube-volume proxy at
 * user slopes, without split constraints) using only caller-owned inputs and outputs plus a
 * fixed scratch array that the library reserves statically on every device that loads it.
 *
 * All pointers in dr_static_args are device memory of the current device; nothing is copied and
 * nothing is allocated.  Layouts: W packs the L layers one after another, layer l+1 as an
 * n_{l+1} x n_l row-major FP32 block; b packs the biases the same way; A [n x n], B [n x m],
 * e [n] (may be NULL) FP64; lo/hi [D x n] FP64; alpha and dalpha [D x H x hidden] FP32; V [D]
 * FP64 (may be NULL).  Work is ordered on `stream` (NULL = legacy default stream).
 *
 * Limits: D*H*(n^2 + 4n + 2) doubles of scratch must fit DR_STATIC_SCRATCH_BYTES (8 MiB), and
 * the controller must fit the fused kernels (widths up to a few hundred); larger problems are
 * rejected with DR_ERR_SHAPE and a message, before any device work.
 * Every call made outside stream capture looks up the scratch address (cudaGetSymbolAddress,
 * which loads the library's device code on first use); a call made while `stream` is being
 * captured reuses the address of the last call on that device, so make a first call before
 * capturing a stream into a graph.  Every call shares the same scratch array:
 * calls that overlap on the GPU (other streams, other threads) race and must be serialised by
 * the caller.  Each call overwrites the scratch before reading it, so no clearing is needed. */
#define DR_STATIC_SCRATCH_BYTES (8u << 20)

typedef struct dr_static_args {
    int32_t L;
    int32_t widths[9]; /* n_0 .. n_L */
    const float* W;
    const float* b;
    const double* A;
    const double* B;
    const double* e;
    int64_t D;
    int32_t H;
    const double* lo;
    const double* hi;
    const float* alpha;
    double margin_rho; /* same meaning as dr_options.margin_rho (0 = none) */
    float* dalpha;
    double* V;
    void* stream;
} dr_static_args;

int dr_slope_gradient_static(const dr_static_args* args);

/* FP32-accurate matrix product on the tensor cores: C [M x N] = A [M x K] * BT [N x K]^T, all FP32
 * row-major device arrays, computed as the 3xTF32 split A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32
 * accumulation (tcgen05.mma kind::tf32, TMA-staged operands).  This is the contraction the chain
 * Lambda <- (Lambda diag(s)) W of Thm. 2 runs on; exposed for testing and reuse.  Uses temporary
 * device memory; synchronises `stream`.  DR_ERR_TIMEOUT if a bounded pipeline wait expired. */
int dr_tf32x3_gemm(int M, int N, int K, const float* A, const float* BT, float* C, void* stream);

/* Paper: no passage (device-side safety of this library's tensor-core pipelines).
 * Check of the bounded device-side waits behind DR_ERR_TIMEOUT: one thread on the current device
 * waits, through the same bounded mbarrier wait the tensor-core pipelines use, on a barrier phase
 * that nothing completes, with a budget of `seconds` (0 < seconds <= 2) of SM clock cycles at the
 * device's rated clock.  Returns DR_ERR_TIMEOUT when the wait gave up and reported it (the designed
 * outcome; the device stays usable), DR_OK if the phase completed (it cannot), DR_ERR_ARG for a
 * budget outside the range, DR_ERR_CUDA / DR_ERR_OOM on a device error.  Synchronises the device. */
int dr_check_wait_expiry(double seconds);

/* Paper: no passage (accounting).
 * Number of kernels this context has launched (monotone counter, for accounting; a graph replay
 * counts the kernels of the captured pass). */
int64_t dr_kernel_launches(const dr_ctx* ctx);

/* Paper: no passage (measurement).
 * Launch classes of dr_kernel_timing: */
#define DR_KT_GEMM_ALL 0   /* every tcgen05 3xTF32 GEMM launch of the staged path                      */
#define DR_KT_GEMM_CHAIN 1 /* persistent chain-level GEMM, next left operand formed in the epilogue     */
#define DR_KT_GEMM_FINAL 2 /* persistent GEMM whose epilogue also multiplies by W_1 (last chain level) */
#define DR_KT_GEMM_OTHER 3 /* the remaining GEMMs (one tile per CTA; target-2 products)                */
#define DR_KT_GEMM_REVERSE 4 /* persistent reverse chain-level GEMM of the staged reverse sweep: adjoint
                                times W_m^T, slope/intercept column sums and the next adjoint operand */
/* Totals over the launches of class `which` with at least `min_rows` rows R (stacked Lambda rows, the
 * M dimension) timed since timing was switched on by dr_set_options (options.timing = 1):
 * *launches, *ms (sum of the per-launch CUDA-event durations, each measured on the stream the launch
 * went to) and *flop (algorithmic FP32-equivalent FLOP: 2 R K N per product of an R x K by K x N
 * operand pair, plus 2 R N n for the fused x W_1 of the last level).  Waits for the recorded events.
 * Any output pointer may be NULL. */
int dr_kernel_timing(dr_ctx* ctx, int which, int64_t min_rows, int64_t* launches, double* ms, double* flop);

/* Paper: no passage (accounting).
 * Number of dr_compute_bounds calls and dr_optimize_slopes steps served by replaying a captured CUDA
 * graph (dr_options.graphs). */
int64_t dr_graph_replays(const dr_ctx* ctx);

/* Paper: no passage (accounting).  The tensor-core GEMM autotuner's choices so far in this process
 * (dr_options.tuning = 0), one line per shape: "epi<e> R<rows> K<k> N<n> sm<SMs>: variant <v> (ms:
 * v<i>=<time> ...)", variants 1 = persistent 128 x 128 tiles in clusters of two CTAs that share the
 * right operand's tiles (TMA multicast), 5 = the same without clusters, 6 = the pair form (one
 * cta_group::2 MMA of M = 256 over two CTAs, B's columns split between them), 2 / 3 / 4 = one
 * 128 x 128 / 64 / 32 tile per CTA.  Writes at most cap bytes including the terminating NUL into buf (truncating; buf may
 * be NULL) and returns the length the whole report needs. */
int64_t dr_gemm_tuning_report(char* buf, int64_t cap);

/* Paper: no passage (error reporting).
 * Message of the last failing call on ctx (or of the last failing dr_create when ctx is
 * NULL).  The pointer stays valid until the next call on the same context. */
const char* dr_last_error(const dr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DIFFREACH_H */
