/*
 * qg.h -- C ABI of libqg, the GB300 (sm_103a) implementation of the QuasiGrad
 * hot path: one full evaluation of the penalized, multi-period, security- and
 * reserve-constrained AC unit-commitment objective and its gradient
 * (Chevalier, "A Parallelized, Adam-Based Solver for Reserve and Security
 * Constrained AC Unit Commitment", Sec. II), chained with the projected Adam
 * update that consumes it (Alg. 3).
 *
 * Conventions shared by every entry point
 *  - Return value: QG_OK (0) or a negative QG_ERR_* code; qg_last_error() gives
 *    a one-line message for the last failing call on a handle.
 *  - Host arrays passed to qg_create, qg_create_batch and qg_eval_grad_host are read during the
 *    call only; the caller keeps ownership.  Device pointers (x, g, m, v, obj)
 *    belong to the caller; the library never frees them.  Everything else the
 *    handle allocates is freed by qg_destroy.
 *  - Device arrays are contiguous; their element type is double in QG_FP64
 *    mode and float in QG_MIXED mode (obj is always double).
 *  - All device work is ordered on the stream set by qg_set_stream (default:
 *    the legacy default stream).  The calls that return host data or re-plan
 *    wait for that stream: qg_eval_grad_host, qg_breakdown, qg_get_step,
 *    qg_set_step, qg_get_state, qg_set_state, qg_phase_times,
 *    qg_ctg_select, qg_ctg_scores, qg_autotune and qg_round_batch;
 *    qg_create*, qg_destroy and the MLP set-up and
 *    destroy calls wait for the device.
 *    Every other call only enqueues work.
 *  - Variable layout of one instance (qg_layout): period-major blocks
 *        x = [ v (T x n) | theta (T x n) | p (T x G) | q (T x G) | r (T x G)
 *              | tau (T x X) | phi (T x X) | u (T x G) ]
 *    (the transformer blocks are empty when X = 0, the on-status block u when
 *    commit = 0), and batched instances are concatenated in creation order.
 *  - Per-unit quantities, periods of dt hours.
 */
#ifndef QG_H
#define QG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QG_OK 0
#define QG_ERR_INVALID_ARG (-1)   /* a size, index, pointer or parameter is out of range      */
#define QG_ERR_ISLANDING (-2)     /* an outage disconnects the grid (1 - PTDF_kk ~ 0)          */
#define QG_ERR_CUDA (-3)          /* a CUDA runtime call failed (message has the CUDA error)   */
#define QG_ERR_NOT_CONVERGED (-4) /* reserved: no call of this build returns it (the DC solves
                                   * are direct, nothing iterates to a tolerance)              */
#define QG_ERR_TIMEOUT (-5)       /* reserved: no call of this build returns it (no kernel
                                   * waits on another block or launch)                         */
#define QG_ERR_NONFINITE (-6)     /* qg_eval_grad_host: an objective came back NaN or Inf      */
#define QG_ERR_NO_DEVICE (-7)     /* no CUDA device, or not an sm_103 device                   */
#define QG_ERR_UNSUPPORTED (-8)   /* a valid request this build does not implement             */

enum { QG_FP64 = 0, QG_MIXED = 1 };                              /* qg_options.precision */
enum { QG_LODF_F32 = 0, QG_LODF_BF16 = 1, QG_LODF_BF16X2 = 2 };  /* qg_options.lodf_dtype (mixed) */
enum { QG_DC_AUTO = 0, QG_DC_DENSE = 1, QG_DC_SPARSE = 2 };      /* qg_options.dc_solver */
enum { QG_CTG_BOUND_AUTO = 0, QG_CTG_BOUND_OFF = 1,               /* qg_options.ctg_bound */
       QG_CTG_BOUND_EAGER = 2, QG_CTG_BOUND_LAZY = 3 };

typedef struct qg_ctx qg_ctx; /* opaque handle; owns all device memory it allocates */

/* Network of one instance (Sec. II-B reduced to v, theta, p, q, r, the
 * transformer variables tau, phi and, optionally, relaxed on-status variables u).
 *   br_from/br_to [M]  bus indices in [0, n), from != to
 *   br_r, br_x [M]     series impedance r + jx (x > 0); g + jb = 1/(r + jx)
 *   br_b [M]           total line charging b_ch (pi model, b_ch/2 per end)
 *   s_max [M]          base-case apparent power limit (thermal, Example 1)
 *   s_max_ctg [M]      post-contingency limit (Eqs. sfr_pen-zctg)
 *   gen_bus, gen_zone [G], cost_a, cost_b [G] (cost d_t (a p^2 + b p)),
 *   cost_r [G] (reserve offer), pmin, pmax, qmin, qmax [G], ramp [G] (pu/h)
 *   vmin, vmax [n]; ref_bus in [0, n) (angle reference, theta_ref clipped to 0)
 *   n_xf, xf_branch [X]  branches that are transformers (distinct ids in [0, M); X = 0 allowed,
 *                       with NULL arrays): an ideal transformer of tap ratio tau and phase
 *                       shift phi at the "fr" end (Sec. II-F line-flow example; the AC flows
 *                       use v_f / tau and delta = theta_f - theta_o - phi) whose DC contingency
 *                       flow is -b_sr (theta_f - theta_o - phi) (Sec. II-E); tau, phi are
 *                       per-period variables in [tau_min, tau_max] (> 0), [phi_min, phi_max]
 * Devices ("generators" above; every field below is optional: 0 / NULL keeps every device a
 * producer with the quadratic cost that is always on):
 *   dev_cons [G]        nonzero marks a consumer: its p, q are drawn from its bus (Example 4 adds
 *                       them to the bus's consumption) and its cost curve is a value that the
 *                       objective subtracts (market surplus); its reserve r is held at 0
 *   n_blk, blk_price, blk_width [G x n_blk] row-major: bid blocks of Example 3; the energy cost
 *                       (value) per hour is sum_l c_l max(min(p - P_{l-1}, w_l), 0) with
 *                       P_{l-1} = w_1 + ... + w_{l-1}, its p-derivative the price of the block that
 *                       p is entering (0 past the last block).  Widths >= 0; a device whose widths
 *                       are all 0 keeps the quadratic cost a p^2 + b p
 *   commit              1: per-period on-status u in [0, 1] (relaxed binaries) with the on cost
 *                       d_t c_on u, startup c_su max(u_t - u_{t-1}, 0) and shutdown
 *                       c_sd max(u_{t-1} - u_t, 0) (Example 2; u_{-1} = u_init in [0, 1]); the limits
 *                       p + r <= pmax u, p >= pmin u, qmin u <= q <= qmax u become penalized linear
 *                       constraints (weight rho beta, soft-ReLU), and the box keeps p in [0, pmax],
 *                       q in [min(qmin, 0), max(qmax, 0)].  c_on, c_su, c_sd >= 0 and u_init [G]
 *                       are required when commit = 1 */
typedef struct {
  int32_t n_bus, n_branch, n_gen, n_zone, ref_bus;
  const int32_t *br_from, *br_to;
  const double *br_r, *br_x, *br_b, *s_max, *s_max_ctg;
  const int32_t *gen_bus, *gen_zone;
  const double *cost_a, *cost_b, *cost_r, *pmin, *pmax, *qmin, *qmax, *ramp;
  const double *vmin, *vmax;
  int32_t n_xf;
  const int32_t *xf_branch;
  const double *tau_min, *tau_max, *phi_min, *phi_max;
  const int32_t *dev_cons;
  int32_t n_blk;
  const double *blk_price, *blk_width;
  int32_t commit;
  const double *c_on, *c_su, *c_sd, *u_init;
} qg_network;

/* Horizon: T periods of dt[t] hours; load_p, load_q are T x n period-major;
 * reserve_req is T x Z (zonal up-reserve requirement). */
typedef struct {
  int32_t T;
  const double *dt, *load_p, *load_q, *reserve_req;
} qg_horizon;

/* Single-branch outages (Sec. II-E): K distinct branch ids in [0, M). */
typedef struct {
  int32_t K;
  const int32_t *branch;
} qg_contingencies;

/* Penalty prices and numerics.  c_p, c_q: balance ($/pu h, Example 4); c_s:
 * thermal and contingency overload (Example 1, Eq. zctg); c_rz: zonal reserve
 * shortfall; rho: penalized linear constraints (headroom, ramps; Eq.
 * nlp_updated); eps: soft-abs / soft-ReLU smoothing (Sec. II-C footnote); beta:
 * homotopy scale on every penalty (Sec. II-F); adam_eps: Adam epsilon. */
typedef struct {
  double c_p, c_q, c_s, c_rz, rho, eps, beta, adam_eps;
  int32_t precision;   /* QG_FP64 or QG_MIXED                                   */
  int32_t lodf_dtype;  /* QG_LODF_*; QG_FP64 always stores the LODF in FP64     */
  int32_t adam_paper_eps; /* 1: numerator (mhat + eps) exactly as printed in Alg. 3 */
  int32_t dc_solver;   /* how the DC solves of Sec. II-E run on the device:
                        * QG_DC_DENSE: products with the PTDF rows of the generator buses
                        *   (set-up holds Yhat^-1 densely; n <= 8192);
                        * QG_DC_SPARSE: the sparse factor Yhat = L diag(D_S, S) L^T with a dense
                        *   tail, two gathers and one dense product per solve, for the base flows
                        *   (Eq. Yb_solve) and the adjoint (Eq. 2nd_lin_sys); no PTDF is formed.
                        *   One instance per handle (QG_ERR_UNSUPPORTED otherwise);
                        * QG_DC_AUTO (0, the default): sparse for a single instance of more
                        *   than 4096 buses, dense otherwise.
                        * Both compute the same quantities (the results agree to rounding). */
  double ctg_frac;     /* contingency screening (Alg. 2): 0 (the default) or >= 1 evaluates every
                        * outage; in (0, 1) each evaluation covers a selected subset of
                        * Ks = ceil(ctg_frac K) outages per instance (qg_ctg_select; initially the
                        * first Ks), through a compacted line-outage block, and records their
                        * scores (qg_ctg_scores) */
  int32_t ctg_bound;   /* bound test ahead of the contingency screen (Sec. II-E): each warp of the
                        * contingency kernel first bounds its 8 branches x 64 outages over 8 periods by
                        * max|L| max|f_k| against the branches' clearance, and screens elements only
                        * where that bound fails.  The classification, and so every result, is
                        * bitwise the same with or without it.  QG_CTG_BOUND_OFF: no bound test;
                        * QG_CTG_BOUND_EAGER: the test, with the line-outage tile loaded up front;
                        * QG_CTG_BOUND_LAZY: the tests of a batch of tiles first, from per-branch
                        * clearances computed once per evaluation (one more kernel), and tiles staged,
                        * loaded and screened only where the test fails; QG_CTG_BOUND_AUTO (0, the
                        * default): lazy where instances with M Ks >= 2^22 hold at least half of the
                        * handle's T M Ks elements (large grids, where most of it passes), no test
                        * otherwise (small grids, where too little passes to pay).  Device memory: 1,024 ceil(M/64) ceil(Ks/64) + 256 T
                        * ceil(M/64) bytes per instance. */
} qg_options;

/* Fill *opt with the defaults: c_p = c_q = 1e4, c_s = c_rz = rho = 1e3,
 * eps = 1e-3, beta = 1, adam_eps = 1e-8, QG_FP64, QG_LODF_F32. */
void qg_default_options(qg_options *opt);

/* Build a handle for one instance: validates the inputs, factors the reduced DC
 * Laplacian E^T Y_x E (Sec. II-E, Eq. Yb_solve; reference bus removed), builds
 * the line-outage block L[m,k] = PTDF_mk / (1 - PTDF_kk) of the rank-1 (SMW)
 * correction (Eq. rank_correct, in flow space) with the denominators in FP64,
 * and uploads everything to the current CUDA device.  Returns
 * QG_ERR_ISLANDING if an outage has |1 - PTDF_kk| < 1e-9, and QG_ERR_INVALID_ARG
 * for an instance whose T (2n + 4G + 2X), T M, T Z or G n_blk reaches 2^31
 * (per-instance element counts are indexed in 32 bits). */
int qg_create(qg_ctx **out, const qg_network *net, const qg_horizon *hor, const qg_contingencies *ctg,
              const qg_options *opt);

/* Same for n_inst independent instances (arrays of n_inst structs) evaluated
 * together by every later call; instance sizes may differ.  1 <= n_inst <= 32
 * (QG_ERR_UNSUPPORTED above: the instance table travels as a kernel parameter). */
int qg_create_batch(qg_ctx **out, int32_t n_inst, const qg_network *net, const qg_horizon *hor,
                    const qg_contingencies *ctg, const qg_options *opt);

void qg_destroy(qg_ctx *h);

/* Total variable count of the handle (all instances). */
int64_t qg_num_vars(const qg_ctx *h);

/* Layout of instance `inst`: its first variable in the concatenated x, its
 * n_x = T (2n + 3G + 2X + commit G), and the starts of the v, theta, p, q, r, tau,
 * phi, u blocks relative to that first variable. */
int qg_layout(const qg_ctx *h, int32_t inst, int64_t *first, int64_t *n_x, int64_t offsets[8]);

/* Order all later device work on `stream` (a cudaStream_t; NULL = default). */
int qg_set_stream(qg_ctx *h, void *stream);

/* One full evaluation (Eq. grads): obj[b] = Phi_b(x) for every instance b
 * (device, n_inst doubles) and g = grad Phi(x) (device, qg_num_vars elements),
 * covering every period and every contingency (Alg. 2 with K_t = all, zeta = 0).
 * g may be NULL (objective only).  x is not modified. */
int qg_eval_grad(qg_ctx *h, const void *x, double *obj, void *g);

/* qg_eval_grad without any allocation, for callers that cannot call cudaMalloc at this point
 * (for example code running under an allocator lock, inside a host callback, or in a process
 * whose memory pool is already sized and frozen).  The paper has no counterpart: it is an
 * interface addition.  The handle's set-up data (made by qg_create) is reused; every
 * per-evaluation work buffer comes from one file-scope static device array of 16 MiB that every
 * GPU loading the library holds from load until the process exits.  The caller passes the inputs
 * and outputs: x (device, qg_num_vars elements), obj (device, n_inst doubles) and g (device,
 * qg_num_vars elements, required).  Results equal those of qg_eval_grad.
 *  - Handles whose work buffers need more than 16 MiB (e.g. large batches) are rejected with
 *    QG_ERR_UNSUPPORTED and a message giving the size needed; so are handles on the sparse DC
 *    solver (QG_DC_SPARSE), whose solve buffers are not carved from the array, and handles with
 *    contingency screening (0 < ctg_frac < 1), whose compacted line-outage block is not either.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress); make
 *    that first call before any stream capture on that device.  The address is kept per device
 *    ordinal for the device's primary context (the one the CUDA runtime uses): it does not follow
 *    a cudaDeviceReset, after which this library's handles are not valid anyway.
 *  - All calls share the one array, which keeps the last call's contents: calls that overlap on
 *    the GPU (other streams, other handles, other threads) race and must be serialized by the
 *    caller.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine. */
int qg_eval_grad_noalloc(qg_ctx *h, const void *x, double *obj, void *g);

/* qg_eval_grad on host buffers: moves x (qg_num_vars doubles) to the device,
 * evaluates, and moves obj (n_inst doubles) and g (qg_num_vars doubles, may be
 * NULL) back; synchronizes.  In QG_MIXED mode the moves convert to/from float.
 * With page-locked buffers the evaluation replays from a graph cached for those
 * buffers (re-captured when they change), in which kernels read x and write obj
 * and g through the buffers' device mappings (copies when a buffer has none).  Returns
 * QG_ERR_NONFINITE when an instance's objective is NaN or Inf (x holds one, or
 * a term overflowed); obj and g are written as computed all the same. */
int qg_eval_grad_host(qg_ctx *h, const double *x, double *obj, double *g);

/* One projected Adam step (Alg. 3) on every variable, using the gradient of the
 * last qg_eval_grad on this handle (kept internally):
 *   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; x -= lr mhat/(sqrt(vhat)+eps);
 *   x = clip(x, box) with v in [vmin, vmax], theta_ref = 0, p in [pmin, pmax],
 *   q in [qmin, qmax], r in [0, pmax] (0 for consumers), tau, phi in their
 *   ranges, u in [0, 1] (with commit, p in [0, pmax], q in [min(qmin, 0),
 *   max(qmax, 0)]).  The step counter i (bias correction) is kept in the handle
 *   and advanced by one. */
int qg_adam_step(qg_ctx *h, void *x, void *m, void *v, double lr, double beta1, double beta2);

/* iters iterations of (qg_eval_grad; qg_adam_step) on x in place, with Adam
 * moments kept inside the handle (zero after qg_create and after
 * qg_set_step(h, 0)), replayed from a CUDA graph that is captured on the first
 * call and re-captured when x, lr, beta1, beta2, obj_trace or (with a trace) iters change.  Does not
 * synchronize.  obj_trace (device, iters x n_inst doubles, may be NULL) receives the objective
 * evaluated at the start of each iteration.  Long runs replay a graph of 8 iterations (bitwise the
 * same result).  Without a trace the objective is summed once per graph replay, for its last
 * iteration (what qg_breakdown then reports). */
int qg_solve(qg_ctx *h, void *x, int32_t iters, double lr, double beta1, double beta2, double *obj_trace);

/* qg_solve with the schedules of Sec. II-F: iteration i of a scheduled run takes its Adam step size,
 * soft-abs / soft-ReLU epsilon and homotopy scale beta from sched[3 i .. 3 i + 2] (device array of
 * sched_len x 3 doubles: lr, eps, beta; e.g. written by qg_schedule; rows past the end repeat the
 * last), in place of lr and of the handle's eps and beta options.  A run starts at a call with
 * restart != 0 (i = 0 at its first iteration); calls with restart = 0 continue the run, so it can
 * be driven in chunks.  obj_trace (device, sched_len x n_inst doubles, may be NULL) receives each
 * iteration's objective at its own eps and beta, indexed by i.  The graph is re-captured when x,
 * sched, sched_len, beta1, beta2 or obj_trace change; a changed iters or restart does not. */
int qg_solve_schedule(qg_ctx *h, void *x, int32_t iters, const double *sched, int32_t sched_len, int32_t restart,
                      double beta1, double beta2, double *obj_trace);

/* The per-iteration schedule of Sec. II-F for `iters` iterations, written to out (host, iters x 3
 * doubles).  Time is the iteration fraction (reading of the wall-clock time of Eq. norm_t):
 * t_i = 2 i / (iters - 1) - 1 (t = -1 for iters = 1), s(t) = e^{4t} / (0.6 + e^{4t}) (Eq. mag_scale):
 *   lr_i   = lr0 10^{s(t_i) log10(lrf / lr0)}                (Eq. step_size)
 *   eps_i  = eps0 10^{s(t_i - lag) log10(epsf / eps0)}       (soft-abs / soft-ReLU tightening, which
 *                                                             lags the step-size decay by `lag`)
 *   beta_i = beta0 + (beta1 - beta0) (t_i + 1) / 2           (homotopy scale, linear)
 * Host-only (no device needed).  Returns QG_ERR_INVALID_ARG for iters < 1, non-positive lr0, lrf,
 * eps0, epsf or non-finite beta0, beta1, lag. */
int qg_schedule(double *out, int32_t iters, double lr0, double lrf, double eps0, double epsf, double beta0,
                double beta1, double lag);

/* Per-instance penalty breakdown of the last evaluation, host array of
 * 8 x n_inst doubles: cost, z_p, z_q, z_s, z_rz, z_headroom, z_ramp, z_ctg.
 * cost is energy cost minus consumer value plus reserve cost, and with commit the
 * on, startup and shutdown costs; z_headroom holds every device-limit penalty
 * (with commit the four u-scaled limits).  Synchronizes the stream. */
int qg_breakdown(qg_ctx *h, double *out);

/* The base DC flows f_t of the last evaluation (Eq. p_flow with the uniform slack of Sec. II-E and
 * the phase shifters' own flows), as the FP32 values the contingency screen reads: host array of
 * sum over instances of T M floats, instance-major, each instance [T][M].  On the mixed path they
 * are the double-FP32 products rounded once to FP32, on the FP64 path the FP64 flows rounded once.
 * Synchronizes the stream. */
int qg_dc_flows(qg_ctx *h, float *out);

/* Adam step counter (for checkpoint/resume together with x, m, v);
 * qg_set_step(h, 0) also zeroes the moments that qg_solve keeps in the handle. */
int qg_get_step(qg_ctx *h, int64_t *step);
int qg_set_step(qg_ctx *h, int64_t step);

/* Checkpoint and resume of a solve.  Alg. 3's iteration carries (x, m, v, i); a run on the
 * schedules of Sec. II-F also carries its position in the schedule, contingency screening (Alg. 2)
 * the current outage selection of every instance, and batch rounding (Alg. 1) the fixed pairs and
 * the clip box they pinned.  x belongs to the caller; everything else is in the handle and travels
 * in one opaque state blob:
 *   header (magic "QGS1", version, precision, n_inst, qg_num_vars, step counter i, step count at the
 *   start of the current scheduled run), the moments m and v that qg_solve / qg_solve_schedule keep
 *   in the handle (qg_num_vars elements each, float in QG_MIXED, double in QG_FP64), then, when the
 *   handle screens contingencies, the selection of every instance (int32), and, once qg_round_batch
 *   has run, the fixed flags of the (period, device) pairs and the current clip box.
 * qg_state_size returns the blob's size in bytes now (it grows once rounding starts), or a negative
 * error code.  qg_get_state writes it to buf (host memory, size bytes; QG_ERR_INVALID_ARG if size
 * is too small).  qg_set_state restores a blob written by a handle created from the same inputs and
 * options (QG_ERR_INVALID_ARG when the header does not match this handle: precision, instance
 * count, variable count, selection sizes).  A run continued from a restored blob with the restored
 * x produces bitwise the iterates of the uninterrupted run (same kernels, same order).
 * qg_get_state and qg_set_state wait for the handle's stream; qg_set_state may allocate the
 * rounding buffers, and a blob written before any rounding round unfixes every pair. */
int64_t qg_state_size(qg_ctx *h);
int qg_get_state(qg_ctx *h, void *buf, int64_t size);
int qg_set_state(qg_ctx *h, const void *buf, int64_t size);

/* Per-kernel timing (CUDA events, no profiler): when on, every evaluation and
 * Adam step records an event after each stage, also inside qg_solve's graph.
 * qg_phase_times writes the durations in ms of the last evaluation's five
 * stages in launch order (s1: branch flows, bus balances, zonal sums and base
 * DC flows; s2: contingencies; s3: contingency sums and branch adjoints; s4:
 * bus adjoint gather and adjoint DC products, and on the mixed path with the
 * dense DC products also the device gradients; s5: the device gradients where
 * stage 4 does not update them, then the closing kernel that sums the
 * objective; with the sparse DC solver s1 includes the forward solve and s4
 * the adjoint solve), then that of a stand-alone qg_adam_step if one
 * followed, up to cap entries; returns how many it wrote or a negative error
 * code.  Waits for those events. */
int qg_set_profiling(qg_ctx *h, int on);
int qg_phase_times(qg_ctx *h, float *ms, int32_t cap);

/* Contingency screening (Alg. 2; handles created with 0 < ctg_frac < 1).  qg_ctg_select makes the
 * n outages ids[0 .. n - 1] (host array of distinct indices into the instance's contingency list,
 * n = its Ks) the ones later evaluations of instance `inst` cover: their columns of the line-outage
 * block are gathered on the device and the instance's contingency term and gradient become those of
 * the subset.  The reading of Alg. 2 here: one subset for all periods of the instance (the union of
 * the per-period sets K_t and S_t).  Synchronizes the handle's stream.
 * qg_ctg_scores copies to `z` (host, sum over instances of T x Ks doubles, period-major per
 * instance, instances in order) the score of every evaluated (period, outage) of the last
 * evaluation: z_tk of Eq. zctg without the soft-ReLU floor, i.e. sum_m d_t c_s beta
 * (sigma_s(s - s_ctg) - eps) over the monitored branches, in the order of the current selection.
 * Both return QG_ERR_UNSUPPORTED on a handle without screening. */
int qg_ctg_select(qg_ctx *h, int32_t inst, const int32_t *ids, int32_t n);
int qg_ctg_scores(qg_ctx *h, double *z);

/* Autotuner of the contingency-block shape (stage 2, Eqs. rank_correct-zctg): for each candidate
 * shape (periods per block x 64-branch tiles per block, deduplicated per handle) re-plans the
 * handle and times `reps` evaluations at x (device, qg_num_vars elements; the point matters: the
 * overload screen skips work); the heuristic shape and the four fastest are timed twice more, and a
 * shape replaces the heuristic only when it is more than 2% faster.  cold != 0 writes a 256 MB
 * buffer (allocated for the call) before every timed evaluation, so that the timing is that of an
 * evaluation starting from an L2 without its data; cold = 0 times back-to-back evaluations (a long
 * Adam run).  Only the order of the outage sums depends on the shape (results agree to rounding).
 * shape (host, may be NULL) receives instance 0's periods per block and tiles per block.
 * Synchronizes; a graph captured by qg_solve is dropped and re-captured on the next call.
 * qg_tile_shape reports the shape in use for an instance. */
int qg_autotune(qg_ctx *h, const void *x, int32_t reps, int32_t cold, int32_t shape[2]);
int qg_tile_shape(const qg_ctx *h, int32_t inst, int32_t shape[2]);

/* Batch rounding (Alg. 1) with a device projection stand-in, for handles whose instances have
 * on-status variables (commit = 1; other instances are skipped).  One call is one round after a
 * solve: every unfixed (period, device) pair is projected on its own (the paper's per-device MILP of
 * Proj. bin_proj needs a MILP solver): u in {0, 1} with the nearer of (u = 1: p, q, r moved to the
 * nearest point of pmin <= p <= pmax, 0 <= r <= rcap, p + r <= pmax, qmin <= q <= qmax, rcap = pmax
 * for producers and 0 for consumers) and (u = 0: p = q = r = 0), ties to u = 1, ramp limits left to
 * the penalized objective; then ceil(frac x unfixed) pairs of each instance whose projection moved
 * them least (squared distance over p, q, r, u; ties by pair index) are fixed: x (device,
 * qg_num_vars elements) takes their projected values and the clip box pins them (u, and with u = 0
 * also p, q, r, at their values; with u = 1 the box becomes the u = 1 limits).  n_fixed and
 * n_binaries (host, may be NULL) receive the fixed and total pair counts over the handle.  frac in
 * (0, 1].  Synchronizes.  qg_round_reset unfixes every pair and restores the original box. */
int qg_round_batch(qg_ctx *h, void *x, double frac, int64_t *n_fixed, int64_t *n_binaries);
int qg_round_reset(qg_ctx *h);

/* Kernel launches of one evaluation (with or without the fused Adam update) on this handle, the
 * closing kernel that sums the objective included: 4 stage kernels on the mixed path with the
 * dense DC products (stage 4 updates the devices), 5 on the FP64 path, 5 plus 3 to 7 solve kernels
 * with the sparse DC solver, one fewer without contingencies, one more on the on-demand contingency
 * path (the clearance kernel, qg_ctg_path = 2); plus 1.  qg_solve without a trace
 * runs its iterations in graphs of 8 that share one closing kernel, so there an iteration costs
 * one launch less, plus 1/8.  Returns a negative error code for a NULL handle. */
int32_t qg_launches_per_eval(const qg_ctx *h);

/* The contingency stage's path on this handle (qg_options.ctg_bound after QG_CTG_BOUND_AUTO is
 * resolved): 0 no bound test, 1 the bound test with every tile staged and loaded (eager), 2 the
 * on-demand path.  Returns a negative error code for a NULL handle. */
int32_t qg_ctg_path(const qg_ctx *h);

const char *qg_last_error(const qg_ctx *h);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start (an AI-systems addition; the paper's future-work remark in Sec. V motivates
 * it): an MLP  Y = W3 relu(W2 relu(W1 X + b1) + b2) + b3  mapping a load profile to an initial
 * point, trained on the GPU by the library's own BF16 tensor-core GEMMs (tcgen05.mma with a TMEM
 * accumulator and TMA-staged operands; FP32 accumulation) and an Adam step.  GEMM operands (X, the weights, the hidden activations, and the back-propagated
 * dY, dZ2, dZ1) are rounded to BF16 where they enter a GEMM; the master weights, biases, bias
 * gradients and Adam moments are FP32.  Parameters are laid out as W1 (H x I, row-major), b1
 * (H), W2 (H x H), b2, W3 (O x H), b3 (O).  All pointers are device pointers; x is batch x I
 * row-major, y and target batch x O.  Weights start from seeded He-scaled normal draws.
 * ------------------------------------------------------------------------------------------- */
typedef struct qg_mlp qg_mlp;

/* max_batch <= 64 (the batch is one 64-column tile of the tensor-core GEMMs); QG_ERR_UNSUPPORTED
 * above that, and when the driver does not provide the TMA descriptor encoder. */
int qg_mlp_create(qg_mlp **out, int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, uint64_t seed);
void qg_mlp_destroy(qg_mlp *m);
int64_t qg_mlp_num_params(const qg_mlp *m);
int qg_mlp_set_stream(qg_mlp *m, void *stream);

/* Inference: y = MLP(x) for `batch` rows (batch <= max_batch). */
int qg_mlp_forward(qg_mlp *m, const float *x, int32_t batch, float *y);

/* One training step on the mean squared error mean((Y - target)^2): forward, backward, and (if
 * lr > 0) an Adam update with the given lr, beta1, beta2 (eps 1e-8).  loss (device double, may
 * be NULL) receives the batch loss before the update. */
int qg_mlp_train_step(qg_mlp *m, const float *x, const float *target, int32_t batch, double lr, double beta1,
                      double beta2, double *loss);

/* FP32 master parameters and the gradient of the last training step (device arrays of
 * qg_mlp_num_params floats). */
int qg_mlp_get_params(qg_mlp *m, float *w);
int qg_mlp_set_params(qg_mlp *m, const float *w);
int qg_mlp_get_grads(qg_mlp *m, float *g);
const char *qg_mlp_last_error(const qg_mlp *m);

/* Synchronizes the MLP's stream and reports whether a tensor-core GEMM since the handle was
 * created gave up on a pipeline wait (each wait is bounded at 1 s; the block then drains its
 * copies in flight, frees its tensor memory and exits, leaving its output invalid): QG_ERR_CUDA
 * with a message if so, else QG_OK. */
int qg_mlp_check(qg_mlp *m);

/* Index-checked builds (the library compiled with QG_CHECK_BOUNDS, `python -m
 * paper_2310_06650_gb300.build --check-bounds`): every access of the stage kernels to one of the
 * library's device arrays (or to a caller's array a handle was given) is checked against the
 * address ranges of those arrays; an access that falls outside all of them reads or writes a
 * dummy word instead, and the first one is recorded.  qg_bounds_report synchronizes the device and
 * returns 1 with that access's source line (of qg_kernels.cu) and address (host pointers, may be
 * NULL), or 0 if none was seen; QG_ERR_UNSUPPORTED in the normal build. */
int qg_bounds_report(int64_t *line, uint64_t *addr);

/* Build identification: major*10000 + minor*100 + patch. */
int qg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QG_H */
