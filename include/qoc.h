/*
 * qoc.h -- C ABI of the GB300 forward + gradient evaluation of a piecewise-constant
 * quantum-control cost (Leung, Abdelhafez, Koch, Schuster, arXiv:1612.04929).
 *
 * One evaluation computes, for controls u[k][j] (k = 1..M controls, j = 1..N slices):
 *   H_j   = H_0 + sum_k u[k][j] H_k (+ delta_e H_det per ensemble member)        Sec. II, Eq. 1
 *   U_j   = exp(-i H_j dt) by a truncated Taylor series of order p after scaling
 *           by 2^-n, then n squarings, with one global (p, n) per evaluation       Sec. III, Eqs. 3, 9, 10
 *   Psi_j = U_j Psi_{j-1} for a d x S block of columns (S = d, Psi_0 = I: gates)  Sec. II, Eqs. 2, 4
 *   C     = a_fid C_fid + a_amp C3 + a_var C4 + a_forbid C5 + a_time C67          Sec. II, Table I
 *   dC/du by a backward (adjoint) sweep that differentiates the truncated series
 *   exactly                                                                       Sec. II.B, Appendix A
 * The cost terms (Table I, with column weights w_s, W = sum_s w_s):
 *   O_j   = sum_s w_s <PsiT^s(j)|Psi_j^s> / W
 *   C_fid = 1 - |O_N|^2                          (C1 gate, C2 state, C2-Sigma subspace)
 *   C3    = sum_{k,j} u[k][j]^2
 *   C4    = sum_k sum_{j=2..N} (u[k][j] - u[k][j-1])^2
 *   C5    = sum_{j=1..N} sum_s w_s sum_{f in F} |Psi_j[f][s]|^2   (forbidden basis states F)
 *   C67   = 1 - (1/N) sum_{j=1..N} |O_j|^2        (C6 gate / C7 state; PsiT(j) may vary with j)
 * State-dependent terms are averaged over ensemble members.
 *
 * Conventions for every entry point:
 *   - Complex arrays are complex128 interleaved (re, im) and row-major: a d x d matrix A has
 *     A[a][b] at doubles [2*(a*d + b)], [2*(a*d + b) + 1]; a d x S block likewise with S columns.
 *   - Host input arrays are copied before the call returns; the library never keeps caller
 *     pointers.  Output arrays are owned by the caller.
 *   - Every call returns a qoc_status; no C++ exception crosses this boundary.  On an error the
 *     context keeps its previous valid state and qoc_last_error() describes the failure.
 *   - A context owns all of its device memory and runs on one CUDA stream; use one context per
 *     host thread.
 */
#ifndef QOC_H
#define QOC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qoc_ctx qoc_ctx;

typedef enum qoc_status {
    QOC_OK = 0,
    QOC_ERR_ARG = 1,            /* NULL pointer where one is required, or an invalid option */
    QOC_ERR_SHAPE = 2,          /* d, M, N, S, E, or an index out of range */
    QOC_ERR_NOT_HERMITIAN = 3,  /* H_0, H_k or H_det deviates from Hermitian by > 1e-12 max|H| */
    QOC_ERR_NONFINITE = 4,      /* NaN or Inf in an input */
    QOC_ERR_STATE = 5,          /* call order: set_system before set_targets before evaluate */
    QOC_ERR_OOM = 6,            /* device allocation failed */
    QOC_ERR_CUDA = 7,           /* a CUDA runtime call or kernel launch failed */
    QOC_ERR_TIMEOUT = 8,        /* a bounded device wait ran out (kernel returned early) */
    QOC_ERR_UNSUPPORTED = 9,    /* size / precision combination this build does not provide */
    QOC_ERR_RANGE = 10,         /* the (p, n) heuristic needs p above its maximum (huge |H dt|) */
    QOC_ERR_STALE = 11          /* a captured batch's frozen (p, n) no longer cover the controls */
} qoc_status;

/* Arithmetic of the Taylor, squaring and propagation products.  Reductions of overlaps,
 * traces, costs and gradient sums are FP64 in every mode; so is the norm bound that picks n. */
typedef enum qoc_precision {
    QOC_PREC_FP64 = 0,          /* plain FP64 form: parity anchor */
    QOC_PREC_FP32 = 1,          /* FP32 adjoint and stored states; slice exponentials and the
                                   carried recursions in extended FP32 (values as hi + lo pairs,
                                   products of grid-split operands: exact FP32 sums of products
                                   of parts of at most 13 significant bits, plus rounded cross
                                   terms; see qoc_options.plain_fp32_exp) */
    QOC_PREC_TF32_SPLIT = 2,    /* the FP32 form, with the products of the large-d adjoint (d > 68)
                                   on tcgen05 tensor cores: TF32 hi + mid + lo split, six MMAs per
                                   real product, FP32 accumulation in tensor memory (the
                                   accumulator's truncation leaves ~2e-5 relative gradient error on
                                   long evolutions) */
    QOC_PREC_BF16_SPLIT = 3     /* the FP32 form, with the products of the large-d adjoint (d > 68)
                                   on tcgen05 tensor cores with exact accumulation: four six-bit
                                   integer slices per value in BF16, per-row / per-column
                                   power-of-two scales, every accumulator an exact integer */
} qoc_precision;

typedef struct qoc_options {
    int precision;        /* qoc_precision */
    double tol;           /* bound on the Taylor remainder per slice after squaring; <= 0: default
                             (1e-15 FP64, 1e-8 otherwise) */
    double theta_max;     /* n is the least n >= 0 with theta / 2^n <= theta_max; <= 0: default
                             (0.25 FP64; FP32 forms: 2 with the Paterson-Stockmeyer form on the
                             per-slice path (d <= 57), 0.5 with Horner there (d <= 68), 1.0 for
                             larger d) */
    int ckpt_stride;      /* slices between stored checkpoints of the propagated block Psi
                             (0: ceil(sqrt(N))).  The backward sweep regenerates Psi_j and U_j
                             between checkpoints instead of storing all N of them. */
    int device;           /* CUDA device ordinal */
    void* stream;         /* cudaStream_t to run on (cudaStreamLegacy = (void*)1 selects the legacy
                             default stream); NULL: the context creates its own stream */
    int p_override;       /* >= 1 forces the Taylor order p, at most 40 (diagnostics); <= 0: heuristic */
    int n_override;       /* >= 0 forces the squaring count n (diagnostics); < 0: heuristic */
    int profile;          /* != 0: bracket every kernel launch with CUDA events (qoc_get_profile) */
    int wave_slices;      /* slices whose propagators are held at once (one parallel launch),
                             rounded up to a multiple of ckpt_stride.  0: half the evolution when
                             two waves fit 1/8 of the free device memory (clamped to 1..32 GiB),
                             so that nothing is recomputed, else the largest wave that fits.
                             Device memory is O(wave d^2 + N / ckpt_stride d S). */
    int plain_fp32_exp;   /* FP32 form only.  0 (default): the slice exponentials (forward and
                             recomputation) use extended FP32 arithmetic (X_j from s H_k held as
                             FP32 pairs, grid-split products), which keeps the coherent rounding of
                             H_j dt out of long evolutions; != 0: plain FP32 exponentials
                             (faster, diagnostics) */
    int sweep;            /* form of the two recursions Psi_j = U_j Psi_{j-1} and the costate:
                             QOC_SWEEP_AUTO (0), QOC_SWEEP_SERIAL (1: one step per slice), or
                             QOC_SWEEP_SCAN (2: products of the U_j over each checkpoint segment by
                             a parallel tree, a scan over segments, then all segments in parallel) */
    int gradient;         /* QOC_GRAD_EXACT (0): the exact derivative of the truncated series;
                             QOC_GRAD_FIRST_ORDER (1): the paper's approximate gradient (Eq. 11,
                             dU_j/du_kj ~ -i dt H_k U_j), O(M d^2 S) per slice instead of an adjoint
                             exponential; its error is O(dt ||[H_j, H_k]||) */
    int adjoint;          /* QOC_ADJ_AUTO (0): the exact adjoint runs in reverse mode over the stored
                             operands of the forward products (two products per step) when the store
                             fits, else by the block recursion; QOC_ADJ_RECOMPUTE (1): always the
                             block recursion (three products per step, nothing stored) */
    int graph;            /* != 0: on the per-slice path (d <= 68 FP32, <= 48 FP64), where every decision
                             of an evaluation is taken on the device, qoc_evaluate_device captures its
                             launches once into a CUDA graph (per (u_dev, grad_dev, out_dev) triple) and
                             replays it on later calls with the same pointers; a new triple or a new
                             plan captures again.  qoc_evaluate_cost_and_grad replays the graph of its
                             own device buffers between its copies.  Ignored with profile != 0 and on
                             the batched path. */
    int fault_inject;     /* test of the failure path, 0 (default) off.  1: the tensor-core adjoint
                             kernels (TF32_SPLIT, BF16_SPLIT, d > 68) withhold their first operand
                             copy, so their bounded mbarrier wait (shortened to 4096 polls) runs
                             out; later kernels of the evaluation skip their work, the evaluation
                             reports QOC_ERR_TIMEOUT and the context and device stay usable.
                             Nothing faults or hangs. */
    int reversal;         /* 0 (default): the backward pass regenerates the states Psi_j from
                             checkpoints (every ckpt_stride slices); 1: by reversal, Psi_{j-1} =
                             U_j^dag Psi_j from the last state of each wave backwards (the paper's
                             Algorithms 1-3, Appendix A), with checkpoints only at wave boundaries
                             and no parallel segment replay.  FP64 form only (QOC_ERR_UNSUPPORTED
                             otherwise): in FP32 the rounding of the stored U_j would accumulate
                             over the backward pass. */
    int propagation;      /* QOC_PROP_UNITARY (0, default): each slice propagator U_j is formed
                             (Taylor + squaring matrix products) and applied to the block;
                             QOC_PROP_STATE (1): state mode (Sec. IV, Eq. 12), the truncated series
                             is applied to the propagated columns by Horner matrix-vector products,
                             T_p(X_j)^(2^n) Psi, without forming U_j: O(p 2^n d^2 S) per slice
                             instead of O((p + n) d^3).  The same truncated map, so the same exact
                             gradient (adjoint_form 4).  At most 8 weighted columns (S); one CTA
                             per (column panel, member) runs the serial recursion, so it pays for
                             few columns with many ensemble members or large d. */
    int exponential;      /* QOC_EXP_TAYLOR (0, default): the truncated Taylor series with scaling
                             and squaring (Sec. III, Eqs. 9, 10); QOC_EXP_CHEBYSHEV (1): the
                             Chebyshev expansion of exp(-i dt H_j) (the Jacobi-Anger series in
                             T_k(dt H_j / theta), theta the FP64 bound of dt ||H_j||) with no
                             scaling, its degree the least whose tail bound is below tol; about
                             theta + O(log 1/tol) matrix-vector products per slice instead of
                             p 2^n.  State mode only (QOC_ERR_UNSUPPORTED otherwise); the gradient is
                             the exact derivative of that polynomial map; qoc_info.p reports the
                             degree.  QOC_ERR_RANGE if the degree would exceed 96. */
    int taylor_scheme;    /* how the Taylor polynomial of Eq. 10 is evaluated.  QOC_TAYLOR_AUTO (0,
                             default): the Paterson-Stockmeyer form (blocks of three terms,
                             T = B_0 + X^3 (B_1 + X^3 (B_2 + ...)), about p / 3 + 2 matrix products
                             instead of p - 1) on the FP32 per-slice path (d <= 57), whose default
                             theta_max is then 2 (fewer squarings), with its reverse-mode adjoints;
                             Horner everywhere else.  QOC_TAYLOR_HORNER (1): Horner on every path
                             (theta_max default 0.5 there).  The polynomial, its truncation and the
                             gradient's definition are the same; qoc_info.taylor_scheme reports the
                             form used. */
    int autotune;         /* 0 (default): the built-in choices.  1: before the first evaluation of a
                             context (unitary propagation only), time candidate configurations on
                             the caller's own inputs and keep the fastest: the Taylor scheme (if
                             taylor_scheme is auto), theta_max x {1/2, 1, 2} (if theta_max is
                             left at 0), the sweep form (if sweep is auto) and, on the per-slice
                             path with two waves, the wave size (up to three checkpoint strides
                             either side of the planner's, if wave_slices is 0), one after another,
                             each candidate run as the context runs it (graph replay included):
                             one warm-up and four (per-slice path) or two timed evaluations.  Every
                             candidate computes the same cost and gradient to the form's tolerance.
                             The choice is cached per process for the same form, dimensions and
                             columns, so later contexts of that shape skip the timing.  The
                             evaluation that triggers it synchronises the context stream and may
                             not be captured into a graph (a qoc_options.graph context tunes
                             before it captures). */
} qoc_options;

enum { QOC_SWEEP_AUTO = 0, QOC_SWEEP_SERIAL = 1, QOC_SWEEP_SCAN = 2 };
enum { QOC_GRAD_EXACT = 0, QOC_GRAD_FIRST_ORDER = 1 };
enum { QOC_ADJ_AUTO = 0, QOC_ADJ_RECOMPUTE = 1 };
enum { QOC_PROP_UNITARY = 0, QOC_PROP_STATE = 1 };
enum { QOC_EXP_TAYLOR = 0, QOC_EXP_CHEBYSHEV = 1 };
enum { QOC_TAYLOR_AUTO = 0, QOC_TAYLOR_HORNER = 1 };

/* Information about the last evaluation (reading it synchronises the context stream). */
typedef struct qoc_info {
    int p, n;             /* Taylor order and squaring count used */
    double theta;         /* dt * max_j ||H_j||_1 bound that picked n (FP64) */
    int ckpt_stride;      /* slices per checkpoint segment */
    int wave_slices;      /* slices per parallel launch (multiple of ckpt_stride) */
    int n_waves;          /* number of waves */
    int launches_per_eval;/* kernels launched by one evaluation */
    int kernel_path;      /* 0: fused per-slice kernels (small d); 1: batched tiled GEMM (large d);
                             2: state mode (matrix-vector Horner chains) */
    long long device_bytes; /* device memory held by the context */
    int adjoint_form;     /* gradient of the last evaluation: 0 reverse mode over the stored products
                             (2 products per forward product), 1 block recursion (3), 2 first-order
                             (Eq. 11, no adjoint exponential), 3 low-rank reverse mode (the cotangent
                             kept as d x r factors, r = 2^n S; small S, per-slice kernels), 4 the
                             state mode's reverse pass over its matrix-vector chain */
    int taylor_scheme;    /* 0 Horner, 1 Paterson-Stockmeyer (see qoc_options.taylor_scheme) */
    int autotune_candidates; /* configurations timed by the autotuner for this context (0: none, or
                             the choice came from the process cache) */
} qoc_info;

/* Per-kernel timings gathered while qoc_options.profile is set: for each kernel class the number
 * of launches and the summed CUDA-event duration (ms) on the context stream. */
#define QOC_PROFILE_SLOTS 16
typedef struct qoc_profile {
    int count;                           /* classes filled */
    char name[QOC_PROFILE_SLOTS][32];
    long long launches[QOC_PROFILE_SLOTS];
    double total_ms[QOC_PROFILE_SLOTS];
} qoc_profile;

/* Fills *opt with the defaults (FP64, heuristic p and n, sqrt(N) checkpoints, device 0, own
 * stream). */
void qoc_default_options(qoc_options* opt);

/* Creates a context on opt->device (opt may be NULL for the defaults).  *out receives the
 * context, or NULL on failure.  Errors: QOC_ERR_ARG (out NULL, bad precision), QOC_ERR_CUDA. */
qoc_status qoc_create(qoc_ctx** out, const qoc_options* opt);

/* Releases every device buffer and the stream the context created.  NULL is a no-op. */
void qoc_destroy(qoc_ctx* ctx);

/* Text of the last error of this context (never NULL; "" after a successful call).  The pointer
 * stays valid until the next call on the same context. */
const char* qoc_last_error(const qoc_ctx* ctx);

/* Static name of a status code. */
const char* qoc_status_string(qoc_status s);

/* The system of Eq. 1.  H0: d x d complex; Hk: M consecutive d x d complex matrices (may be
 * NULL when M = 0); dt > 0; N >= 1 slices; 1 <= d <= 512; 0 <= M <= 64.  The matrices are
 * copied; the caller keeps its buffers.  Resets the targets and the ensemble (a later evaluate
 * needs qoc_set_targets again).  Errors, all raised before any device work: QOC_ERR_ARG (NULL
 * matrix, dt not finite and positive), QOC_ERR_SHAPE (d, M or N out of range),
 * QOC_ERR_NONFINITE, QOC_ERR_NOT_HERMITIAN (|H_ab - conj(H_ba)| above 1e-12 max(1, max|H|));
 * then QOC_ERR_CUDA / QOC_ERR_OOM from the device copies. */
qoc_status qoc_set_system(qoc_ctx* ctx, int d, int M, const double* H0, const double* Hk,
                          double dt, int N);

/* Initial columns and costs (Table I).  psi0, psiT: d x S complex (1 <= S <= d); forbidden: nF
 * basis indices in [0, d) (may be NULL when nF = 0); col_weight: S non-negative weights with a
 * positive sum (NULL: all 1); psiT_path: N consecutive d x S targets for the per-slice time cost
 * C67 (NULL: psiT at every slice); alpha: 5 weights [fid, C3 amplitude, C4 variation,
 * C5 forbidden, C67 time].  Everything is copied.  Requires qoc_set_system (else
 * QOC_ERR_STATE).  Other errors: QOC_ERR_ARG (NULL argument, a negative or non-finite weight,
 * weights summing to 0), QOC_ERR_SHAPE (S or nF out of range, a forbidden index outside
 * [0, d)), QOC_ERR_NONFINITE.  No device work. */
qoc_status qoc_set_targets(qoc_ctx* ctx, int S, const double* psi0, const double* psiT, int nF,
                           const int* forbidden, const double* col_weight,
                           const double* psiT_path, const double* alpha);

/* Detuning ensemble for robust control: member e propagates H_j + delta[e] Hdet; the
 * state-dependent cost terms and their gradients are averaged over the E members.
 * 1 <= E <= 65535; delta: E doubles; Hdet: d x d complex Hermitian (may be NULL when every
 * delta is 0); both are copied.  Requires qoc_set_system (else QOC_ERR_STATE).  Other errors:
 * QOC_ERR_SHAPE (E), QOC_ERR_ARG (delta NULL, or Hdet NULL with a non-zero delta),
 * QOC_ERR_NONFINITE, QOC_ERR_NOT_HERMITIAN; then QOC_ERR_CUDA / QOC_ERR_OOM. */
qoc_status qoc_set_ensemble(qoc_ctx* ctx, int E, const double* delta, const double* Hdet);

/* One forward + gradient evaluation from host memory: the cost C of Table I (Sec. II) and its
 * exact gradient dC/du (Sec. II.B, Appendix A).  u: M x N doubles (row k holds control k
 * over the N slices); *cost receives C; grad (M x N doubles) receives dC/du; terms (5 doubles,
 * may be NULL) receives the unweighted [C_fid, C3, C4, C5, C67].  Copies u to the device, runs,
 * copies the results back and synchronises the stream.  Requires set_system and set_targets. */
qoc_status qoc_evaluate_cost_and_grad(qoc_ctx* ctx, const double* u, double* cost, double* grad,
                                      double* terms);

/* The same evaluation (Table I cost, Sec. II.B / Appendix A gradient) on device memory,
 * asynchronous on the context stream: u_dev (M x N doubles), grad_dev (M x N doubles) and
 * out_dev (6 doubles: C then the 5 terms) are device pointers owned by the caller.  Returns
 * after enqueueing; errors raised inside kernels are reported by the next synchronising call
 * (qoc_sync, qoc_get_info or a host evaluation). */
qoc_status qoc_evaluate_device(qoc_ctx* ctx, const double* u_dev, double* grad_dev,
                               double* out_dev);

/* Batched evaluation of `count` independent problems (for example many control problems of
 * uneven d, N, M and ensemble size): ctxs[i] is a context set up for problem i, and u_dev[i],
 * grad_dev[i], out_dev[i] are its device buffers as in qoc_evaluate_device.  Every context's
 * (p, n) is picked first (FP64, on the GPU); if some problem uses the large-d kernels, the call
 * waits once to read those choices.  Then every evaluation is enqueued on its own context's
 * streams, so the problems run concurrently on the GPU; all of them start after the work
 * already enqueued on `stream` and the work enqueued on `stream` after this call waits for all
 * of them (NULL: the legacy default stream).  Contexts created with their own streams
 * (qoc_options.stream = NULL) run concurrently; a context may appear only once.  Errors of one
 * context are reported through its qoc_last_error. */
qoc_status qoc_evaluate_batch(int count, qoc_ctx* const* ctxs, const double* const* u_dev,
                              double* const* grad_dev, double* const* out_dev, void* stream);

/* A batch captured into one CUDA graph (independent problems, Sec. II.A: every slice, problem and
 * ensemble member is independent until the sweeps).  qoc_batch_create takes the arguments of
 * qoc_evaluate_batch, runs one evaluation of the batch as that call does (planning, device
 * allocations, qoc_options.autotune, the (p, n) of every problem; its results are in grad_dev and
 * out_dev when the call returns, which synchronises `stream`), then freezes the Taylor orders and
 * grid exponents of the problems on the batched large-d path at those of this evaluation and
 * captures a second evaluation of every problem, fork and join included, into one graph on a
 * stream of its own.  *out receives the batch.  qoc_batch_launch replays the graph on `stream`
 * (NULL: the legacy default stream): every problem is evaluated on the device buffers given at
 * creation (the caller rewrites u_dev[i] in place between launches), with no host work per
 * problem.  A replay whose controls need a larger (p, n) or grid exponents than the frozen ones
 * still runs, with the frozen orders, and is flagged: qoc_batch_sync (which waits for the last
 * launch) then reports QOC_ERR_STALE for that problem; frozen orders that are larger than needed
 * only cost time.  While a batch holds a context, the context's own evaluations use the frozen
 * orders too, and qoc_set_system / qoc_set_targets / qoc_set_ensemble refuse with QOC_ERR_STATE;
 * qoc_destroy of a held context is deferred until the last batch holding it is destroyed.  Not in a batch (QOC_ERR_UNSUPPORTED): contexts in state
 * mode (qoc_options.propagation), profiled contexts, contexts on different devices; contexts on
 * the legacy default stream cannot be captured (QOC_ERR_CUDA from the capture).  Errors of
 * one context are reported through its qoc_last_error (launch and graph errors through the first
 * context's); count < 1 or a NULL out is QOC_ERR_ARG. */
typedef struct qoc_batch qoc_batch;
qoc_status qoc_batch_create(int count, qoc_ctx* const* ctxs, const double* const* u_dev,
                            double* const* grad_dev, double* const* out_dev, void* stream,
                            qoc_batch** out);
qoc_status qoc_batch_launch(qoc_batch* batch, void* stream);
/* Waits for the last launch and returns the first device-side error of the batch's problems
 * (QOC_ERR_STALE, QOC_ERR_NONFINITE, QOC_ERR_TIMEOUT, QOC_ERR_RANGE), each also recorded in its
 * context's qoc_last_error. */
qoc_status qoc_batch_sync(qoc_batch* batch);
/* Waits for the last launch, releases the graph, unfreezes the contexts it held and completes a
 * qoc_destroy deferred while it held them. */
void qoc_batch_destroy(qoc_batch* batch);

/* Waits for the context stream and reports a device-side error of earlier evaluations. */
qoc_status qoc_sync(qoc_ctx* ctx);

/* Fills *info (synchronises). */
qoc_status qoc_get_info(qoc_ctx* ctx, qoc_info* info);

/* Synchronises and returns the per-kernel timings accumulated since the last reset (all zero
 * when the context was created without qoc_options.profile). */
qoc_status qoc_get_profile(qoc_ctx* ctx, qoc_profile* out);

/* Clears the accumulated per-kernel timings. */
qoc_status qoc_reset_profile(qoc_ctx* ctx);

/* Measured multiply-add throughput of a device, the peak against which the FP32 (fp64 = 0) or
 * FP64 (fp64 != 0) arithmetic of the products is reported: one launch of independent FMA chains
 * on every SM, best of three CUDA-event timings on a stream of its own.  *tflops receives
 * 2 x FMAs / second / 1e12; *sms (may be NULL) the device's SM count.  No device setting is read
 * or changed.  Not a step of the paper's method.  Errors: QOC_ERR_ARG (tflops NULL),
 * QOC_ERR_CUDA (no device, or a failed launch). */
qoc_status qoc_measure_fma_peak(int device, int fp64, double* tflops, int* sms);

/* Bytes of the device array that qoc_evaluate_static works in (32 MiB).  Every GPU that loads
 * the library holds this array until the process exits. */
#define QOC_STATIC_ARENA_BYTES (32u << 20)

/* One evaluation that allocates no memory, for callers that may not allocate at the time they
 * evaluate: code running while a stream is captured into a CUDA graph (allocation is not
 * permitted there), real-time loops that forbid allocator calls because they can block, or
 * programs whose device memory belongs to a pool that must not be bypassed.  The paper has no
 * counterpart; this is a packaging of the same computation.
 *
 * It computes what qoc_evaluate_device computes for the FP64 form with no ensemble, no
 * per-slice targets and unit column weights, keeping every intermediate in a fixed device array
 * of QOC_STATIC_ARENA_BYTES instead of context-owned buffers.  There is no context.
 *   d (1..48), M (0..64), N (>= 1), S (1..d); dt > 0.
 *   H0_dev: d x d complex128 (interleaved, row-major), Hk_dev: M such matrices, u_dev: M x N
 *   doubles, psi0_dev / psiT_dev: d x S complex128, fmask_dev: d ints, 1 for a forbidden basis
 *   state (NULL: none) -- all device pointers owned by the caller and not validated.
 *   alpha: 5 host doubles [fid, C3, C4, C5, C67], read before the call returns.
 *   grad_dev (M x N doubles) and out_dev (6 doubles: C then the 5 terms) receive the results.
 *   stream: cudaStream_t to enqueue on (NULL: the legacy default stream).
 * The call enqueues its kernels and returns without synchronising.  Its status covers the
 * argument checks, the size check and launch errors only.  Conditions found on the device (a
 * NaN or Inf in the controls or the results, a Taylor order at its cap) are not returned; they
 * leave out_dev[0] = NaN, so a caller checks that value after synchronising.
 * QOC_ERR_SHAPE also means that the problem does not fit the array, and that check comes before
 * any CUDA call.  With Spad = S rounded up to a multiple of min(S, 8) and d2 = d^2 rounded up to
 * a multiple of 16, the array holds, each piece rounded up to 256 bytes: U_j and U_j^dag
 * (32 N d2 bytes), the states (16 (N + 1) d Spad), costates and sources (16 N d Spad each),
 * three d x Spad blocks, per-slice overlaps and occupations (24 N), the gradient parts
 * (8 (M N + 1)) and a few small pieces: about 32 N d^2 + 48 N d Spad + 8 M N bytes in all.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before capturing a stream.  All calls share the
 * one array and every call overwrites it: calls that may overlap on the GPU (different streams
 * without ordering between them, or different host threads) race and give wrong results. */
qoc_status qoc_evaluate_static(int d, int M, int N, int S, double dt, const double* H0_dev,
                               const double* Hk_dev, const double* u_dev, const double* psi0_dev,
                               const double* psiT_dev, const int* fmask_dev, const double* alpha,
                               double* grad_dev, double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QOC_H */
