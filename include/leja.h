/*
 * leja.h — C ABI of the GB300 (sm_103a) Léja-point log-determinant library.
 *
 * The library estimates log det A for a sparse symmetric positive definite matrix A (CSR) by
 * the method of Mbingui, Tambue & Karambal, "Novel technique based on Léja Points Approximation
 * for Log-determinant Estimation of Large matrices" (arXiv 2603.02207):
 *   log det A = n log sigma + tr log(A / sigma)                       (Section 4, Eq. scaled_sigma_matrix)
 *   log(A / sigma) V ~ p_m(A / sigma) V, p_m the Newton interpolant of log at m+1 fast Léja
 *   points mapped to the spectral interval                             (Section 3, Algorithms 1-2)
 *   tr is estimated by Hutch++ (sketch, QR, deterministic part, deflated Hutchinson part)
 *                                                                      (Section 4.1, Algorithm 3)
 * Every compute step runs in the library's own CUDA kernels on the device.
 *
 * Conventions for every entry point:
 *   - Matrix and block pointers are DEVICE pointers unless the parameter says "host". They are
 *     owned by the caller and only read (inputs) or written (outputs) during the call.
 *   - Dense blocks are row-major: element (i, j) of an n x b block X with leading dimension ldx
 *     is X[i * ldx + j], ldx >= b.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that return a host value
 *     synchronise that stream before returning; the others only enqueue work.
 *   - Every call returns an ll_status. On failure the outputs are left unchanged (except device
 *     outputs of calls that only enqueue work, which are unspecified) and ll_last_error(h)
 *     describes the failure.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef LEJA_H_
#define LEJA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LL_OK = 0,
    LL_ERR_INVALID_ARG = 1,       /* a null pointer, a negative size, an unknown enum value      */
    LL_ERR_BAD_CSR = 2,           /* rowptr not monotone, rowptr[0] != 0, rowptr[n] != nnz,
                                     or a column index outside [0, n)                            */
    LL_ERR_BAD_BOUNDS = 3,        /* lmin <= 0 or lmin >= lmax, or non-finite bounds             */
    LL_ERR_DD_NOT_CONVERGED = 4,  /* the Taylor series of Algorithm 1 did not converge           */
    LL_ERR_QR_BREAKDOWN = 5,      /* CholeskyQR met a non-positive pivot (rank-deficient sketch) */
    LL_ERR_NONFINITE = 6,         /* a NaN or Inf appeared in the traces                         */
    LL_ERR_TIMEOUT = 7,           /* a bounded device-side wait ran out                          */
    LL_ERR_OOM = 8,               /* device workspace allocation failed                          */
    LL_ERR_CUDA = 9,              /* a CUDA runtime error                                        */
    LL_ERR_UNSUPPORTED = 10,      /* a valid but unimplemented option combination                */
    LL_ERR_NO_FORWARD = 11        /* no kept forward (backward) or no forward yet                 */
} ll_status;

/* Storage type of the CSR values. */
enum { LL_F64 = 0, LL_F32 = 1 };

/* Arithmetic of the Léja recurrence (a12):
 *   LL_PREC_F64        W_j, P and the traces in IEEE FP64 on the FP64 pipe.
 *   LL_PREC_DF64       W_j, P and V stored as float pairs (hi, lo) and updated in double-float
 *                      arithmetic on the FP32 pipes (about 46-48 significant bits); trace sums
 *                      are finished in FP64; the QR products run in double-float with FP64
 *                      accumulation and an FP64 Cholesky. Same 8 bytes per element as FP64.
 *   LL_PREC_F32_MIXED  matrix values and W_j in FP32; P = sum_j d_j W_j and the traces accumulated
 *                      in double-float (exact FP32 products, TwoSum accumulation: FP64-class);
 *                      QR as in LL_PREC_DF64.                                                       */
enum { LL_PREC_F64 = 0, LL_PREC_DF64 = 1, LL_PREC_F32_MIXED = 2 };

enum { LL_PROBE_RADEMACHER = 0, LL_PROBE_GAUSSIAN = 1 };

/* Trace estimator of ll_logdet_forward:
 *   LL_EST_HUTCHPP     Hutch++ (Section 4.1, Algorithm 3): probes/3 sketch columns, a QR, and
 *                      the deflated Hutchinson part;
 *   LL_EST_HUTCHINSON  plain Hutchinson (Eq. Léja8): estimate = n log sigma +
 *                      (1/m) sum_i g_i^T p(A~) g_i over m = probes vectors from stream
 *                      LL_STREAM_G (1 <= m <= 192), with no sketch and no QR. */
enum { LL_EST_HUTCHPP = 0, LL_EST_HUTCHINSON = 1 };

/* s_val of Algorithm 1: the Lemma 3.1 optimum c = (lmin+lmax)/2, or lmax/2. */
enum { LL_SVAL_CENTER = 0, LL_SVAL_HALF_LMAX = 1 };
/* How the Newton coefficients d_j are computed (ll_options.dd_scheme):
 *   LL_DD_AUTO     Algorithm 1 (Section 3.1), or the FP64 divided-difference table in the xi
 *                  variable (Eq. Léja7) when the series would need more than 1e6 terms;
 *   LL_DD_TABLE_Q  the divided-difference table in the xi variable in binary128 arithmetic on the
 *                  host (a second scheme for very large condition numbers), rounded to FP64. */
enum { LL_DD_AUTO = 0, LL_DD_TABLE_Q = 1 };
/* Kernel of CholeskyQR2's Gram products Y^T Y, Q1^T Q1 and Q^T G (ll_options.qr_gram, ll_gram):
 *   LL_GRAM_AUTO    the faster of the two for the shape (element type, widths, symmetry, rows):
 *                   both are timed on the first product of a shape on the handle and the choice
 *                   is cached (the chosen kernel runs last, so every call of the shape gives the
 *                   same result); LL_GRAM_DFLOAT above width 42;
 *   LL_GRAM_TENSOR  tcgen05 MMAs on BF16 digit slices: each column is written in fixed point as
 *                   seven 7-bit digits (six for widths above 36) below its scale 2^E (max |x| <
 *                   2^(E-1), from a maximum pre-pass), every slice product summed over up to 4096
 *                   rows is exact in the FP32 accumulators, and the products are scaled and summed
 *                   in double-float (Ozaki, Ogita & Oishi 2012): 49 (42) bits below each column's
 *                   maximum; widths up to 42;
 *   LL_GRAM_DFLOAT  double-float products on the FP32 pipes (any width up to 96).            */
enum { LL_GRAM_AUTO = 0, LL_GRAM_TENSOR = 1, LL_GRAM_DFLOAT = 2 };
/* ll_set_adjoint_fusion modes */
enum { LL_FUSE_AUTO = 0, LL_FUSE_ON = 1, LL_FUSE_OFF = 2 };
/* Row order of the forward (ll_options.reorder):
 *   LL_REORDER_AUTO    the degree order below for irregular matrices (the longest row above four
 *                      times the mean plus 16, most entries outside the tile windows, not banded)
 *                      in a forward that keeps nothing for a backward; else the matrix's order;
 *   LL_REORDER_NONE    the matrix's order;
 *   LL_REORDER_DEGREE  the passes run on P A P^T with the rows ordered by entry count, descending
 *                      (ties by row index): a power-law graph's hubs come first and the rows most
 *                      entries gather stay together in L2. The probe rows keep the probe values
 *                      of their original rows, so the estimate equals the unpermuted one up to the
 *                      order of its sums. The permuted structure is built on the device once per
 *                      structure (a checksum of rowptr and colind tells a changed one) and cached
 *                      on the handle; the values are gathered through it at every call. Not with
 *                      keep_for_backward (LL_ERR_UNSUPPORTED). */
enum { LL_REORDER_AUTO = 0, LL_REORDER_NONE = 1, LL_REORDER_DEGREE = 2 };

/* Step kernel of the m-step passes:
 *   LL_KERNEL_AUTO    banded matrices (every row's columns strictly increasing and within 2 of
 *                     the diagonal) take LL_KERNEL_BAND; otherwise autotuned: the kernel and its
 *                     launch shape are timed once per (precision, pass, n, nnz, block width) on
 *                     the handle and the fastest is kept;
 *   LL_KERNEL_GATHER  neighbour rows gathered into registers by each thread (k_leja_step);
 *   LL_KERNEL_TMA     neighbour rows gathered into shared memory by TMA (tile::gather4) in a
 *                     multi-stage mbarrier pipeline (k_leja_tma); falls back to LL_KERNEL_GATHER
 *                     when a block row is wider than 256 elements;
 *   LL_KERNEL_BAND    banded matrices only (else as LL_KERNEL_AUTO): up to four steps per launch
 *                     on row tiles with halos, W_j between the steps in shared memory
 *                     (k_leja_band); W_{j+1} and P equal the one-step kernels' bit for bit. Not
 *                     with the stopping rule (tol > 0), the adjoint or the batched call, which
 *                     run the one-step kernels.                                                  */
enum { LL_KERNEL_AUTO = 0, LL_KERNEL_GATHER = 1, LL_KERNEL_TMA = 2, LL_KERNEL_BAND = 3 };

/* Probe streams of the counter-based generator (see ll_probes). */
enum { LL_STREAM_S = 0, LL_STREAM_G = 1, LL_STREAM_POWER = 2 };

typedef struct {
    int64_t n;                 /* order of the square matrix                                    */
    int64_t nnz;               /* stored entries                                                 */
    const int32_t* rowptr;     /* device, n+1 entries, rowptr[0] = 0, rowptr[n] = nnz           */
    const int32_t* colind;     /* device, nnz entries in [0, n)                                  */
    const void* values;        /* device, nnz entries of type `dtype`                            */
    int dtype;                 /* LL_F64 or LL_F32                                               */
} ll_csr;

typedef struct {
    double lmin, lmax;         /* spectral interval [lambda_min, lambda_max], 0 < lmin < lmax    */
} ll_bounds;

typedef struct {
    int degree;                /* m: m+1 Léja points, m operator applications per pass          */
    int probes;                /* m_vec: Hutch++, a positive multiple of 3 (k = m_vec / 3);
                                  Hutchinson, the number of probe vectors (1 to 192)            */
    uint64_t seed;             /* probe seed                                                     */
    int probe_kind;            /* LL_PROBE_RADEMACHER or LL_PROBE_GAUSSIAN                      */
    int precision;             /* LL_PREC_*                                                      */
    int sval_mode;             /* LL_SVAL_*                                                      */
    int keep_for_backward;     /* 1: keep [Q | G'] and the coefficients for ll_logdet_backward   */
    int rows_per_thread;       /* LL_KERNEL_GATHER: rows each thread handles per tile (0 = 8);
                                  LL_KERNEL_TMA: 2 = two column pairs per thread (FP32-mixed)   */
    int threads_per_block;     /* CTA size of the step kernel (0 = kernel default: 384 or 512
                                  for LL_KERNEL_GATHER, 512 for LL_KERNEL_TMA; a TMA CTA of at
                                  most 256 threads runs two per SM). Ignored by LL_KERNEL_AUTO.  */
    int ckpt_stride;           /* backward: 0 (default) = the forward's trace pass keeps W_1 ..
                                  W_m for the backward when they take at most half of the
                                  free device memory (ll_set_keep_budget), else the trace pass
                                  writes checkpoints at the smallest stride that fits
                                  (<= ceil(sqrt(m))), else none are kept and the backward
                                  checkpoints itself; > 0 = the backward checkpoints every
                                  ckpt_stride steps itself                                     */
    int use_graph;             /* 1: capture the m-step passes in a CUDA graph (default 1)       */
    int64_t timeout_cycles;    /* batched launch: clock cycles a dependency wait may spin before
                                  the call fails with LL_ERR_TIMEOUT; 0 = about 2 s. Also bounds
                                  the pipeline waits of the TMA step kernel.                     */
    int step_kernel;           /* LL_KERNEL_* (default LL_KERNEL_AUTO)                           */
    int estimator;             /* LL_EST_HUTCHPP (default) or LL_EST_HUTCHINSON                  */
    double tol;                /* Algorithm 2's stopping rule (Section 3.1): 0 (default) = fixed
                                  degree; > 0: in each pass every column stops at the first m
                                  with |d_m| ||w_m||_2 <= tol (w_m the Newton basis vector of
                                  the scaled operator), degree being the cap. Not with
                                  keep_for_backward nor ll_logdet_batched (LL_ERR_UNSUPPORTED).  */
    int dd_scheme;             /* LL_DD_AUTO (default) or LL_DD_TABLE_Q                          */
    int qr_gram;               /* LL_GRAM_AUTO (default), LL_GRAM_TENSOR or LL_GRAM_DFLOAT: the
                                  Gram kernel of the CholeskyQR2 of Algorithm 3 step 4 and of
                                  Q^T G in step 6 (the backward uses the kept forward's)        */
    int reorder;               /* LL_REORDER_AUTO (default), LL_REORDER_NONE or LL_REORDER_DEGREE */
} ll_options;

typedef struct ll_handle ll_handle;

/* Diagnostics of the last forward call on a handle. */
typedef struct {
    double sigma, c, gamma;          /* normalisation and affine map of the scaled interval       */
    double trace_q, trace_res;       /* tr(Q^T F Q) and the Hutchinson part                       */
    double estimate;                 /* n log sigma + trace_q + trace_res                         */
    int taylor_terms;                /* p used by Algorithm 1                                     */
    int k;                           /* sketch columns used (min(m_vec/3, n))                     */
    int kernel_launches;             /* library kernels launched by the call                      */
    float ms_probes, ms_pass1, ms_qr, ms_pass2, ms_total;   /* device times (CUDA events)         */
    int kernel_pass1, kernel_pass2;  /* LL_KERNEL_GATHER, _TMA or _BAND used by each pass          */
    int threads_pass1, threads_pass2;   /* CTA size used by each pass                             */
    int deg_max_pass1, deg_max_pass2;   /* largest final degree over the columns of each pass
                                           (the degree itself under a fixed degree)              */
    double deg_mean_pass2;              /* mean final degree over the trace pass's columns        */
    int kept_w_steps;                   /* W_j blocks the trace pass kept for the backward: m
                                           (W_1 .. W_m), or the checkpoint count when only
                                           W_s, W_2s, ... fit; 0: none                           */
    int kept_w_steps_pass1;             /* the same for pass 1 (W_0 = S), used by the through-QR
                                           adjoint; 0 for a banded matrix or when they do not fit */
    int kept_w_stride;                  /* 1: the trace pass kept every W_j (kept_w_steps = m);
                                           s > 1: it kept the checkpoints W_s, W_2s, ...
                                           (kept_w_steps = ceil(m/s) - 1); 0: none kept        */
    int64_t forward_id;                 /* 1 + the number of earlier successful forwards on the
                                           handle: a caller that keeps it can tell whether the
                                           handle's kept state is still that of its forward     */
    int pairs_pass1, pairs_pass2;       /* column pairs per thread of each pass's step kernel (2:
                                           the FP32-mixed TMA kernel with 16-byte row accesses)  */
    int rows_pass1, rows_pass2;         /* rows per tile of each pass's step kernel               */
    int batch_tuned;                    /* ll_logdet_batched: 1 when the autotuner chose the launch
                                           shape (step kernel, threads and rows per pass)        */
    int reordered;                      /* 1 when the passes ran on the degree-ordered matrix    */
    int adjoint_fused;                  /* ll_logdet_backward(_qr): 1 when the reverse steps of its
                                           last adjoint recurrence ran with the gradient
                                           contraction fused in, 0 with it separate              */
} ll_info;

/* ---- handle -------------------------------------------------------------------------------- */

/* Create a handle on the current CUDA device. The handle owns the device workspace and the
 * kept forward state. */
ll_status ll_create(ll_handle** out);
void ll_destroy(ll_handle* h);
const char* ll_status_string(ll_status s);
/* Text of the last failure on this handle (empty when none). Owned by the handle. */
const char* ll_last_error(const ll_handle* h);
/* Fill *opts with defaults: degree 40, probes 30, seed 0, Rademacher, LL_PREC_DF64, s_val = c,
 * no backward, autotuned step kernel, ckpt_stride 0, CUDA graphs on. */
void ll_default_options(ll_options* opts);
/* Step kernel and launch shape used by ll_apply_poly and ll_logdet_backward on this handle
 * (LL_KERNEL_*, with threads_per_block and rows_per_thread as in ll_options; the default is
 * LL_KERNEL_AUTO). LL_ERR_INVALID_ARG for an unknown kernel or a negative shape. */
ll_status ll_set_step_config(ll_handle* h, int step_kernel, int threads_per_block, int rows_per_thread);
/* Device memory that ll_logdet_forward with keep_for_backward may spend on the trace pass's W_j
 * for the backward (every W_j, else the checkpoints at the smallest stride <= ceil(sqrt(m)) that
 * fits, else none). 0 (default): half of the free device memory at the call. Lets a caller
 * leave memory to other work, and lets tests reach the checkpointed layout on small matrices.
 * LL_ERR_INVALID_ARG for a negative value. */
ll_status ll_set_keep_budget(ll_handle* h, int64_t bytes);
/* The gradient contraction of ll_logdet_backward(_qr) (the sum over j of
 * Lambda_{j+1}[r_e, :] . W_j[c_e, :] for every stored entry e) fused into the reverse step of the
 * adjoint recurrence: the TMA step kernel with one column pair per thread, on a matrix whose
 * rows hold strictly increasing columns, adds each tile's entries from the rows it stages.
 *   LL_FUSE_AUTO (default): the first backward of a shape (precision, n, nnz, width) times the
 *                           fused step against the reverse step plus the separate contraction
 *                           and keeps the faster on the handle;
 *   LL_FUSE_ON:  fused wherever it applies;
 *   LL_FUSE_OFF: always the separate contraction.
 * Both forms give the same gradient up to the order of each entry's sum. ll_info.adjoint_fused
 * reports the form the last backward took. LL_ERR_INVALID_ARG for another mode. */
ll_status ll_set_adjoint_fusion(ll_handle* h, int mode);
/* Free the handle's device workspace: every block the calls allocated (probe and W blocks, the
 * kept W_j, tile descriptors, the cached degree order) and the captured CUDA graphs, so that other
 * work can use the memory. The kept forward state is dropped (ll_logdet_backward then returns
 * LL_ERR_NO_FORWARD); the autotuners' choices stay. The next call allocates afresh. Synchronises
 * the device. */
ll_status ll_trim_workspace(ll_handle* h);

/* Test hook for failure detection. LL_INJECT_STALL: from now on, the TMA step kernel launched by
 * this handle expects 16 bytes for its first tile that no copy delivers, so that tile's pipeline
 * waits run out after the options' timeout_cycles; the kernel then records the error, stops
 * issuing copies, waits (bounded) for the copies it issued, and returns, and the call fails with
 * LL_ERR_TIMEOUT while the context stays usable. LL_INJECT_NONE clears it. No other kernel is
 * affected. LL_ERR_INVALID_ARG for an unknown value. */
enum { LL_INJECT_NONE = 0, LL_INJECT_STALL = 1 };
ll_status ll_debug_inject(ll_handle* h, int what);

/* ---- host-side method pieces (FP64 on the host: their stability needs it) ------------------ */

/* First `count` fast Léja points on [-2, 2] into xi_out (host, count doubles).
 * Section 3, Eq. (Léja5), fast variant (Baglama, Calvetti & Reichel 1998) as used in
 * Section 3.1: xi_0 = 2, xi_1 = -2, candidates are midpoints of neighbouring chosen points,
 * score prod_k |x - xi_k| (FP64, k ascending), scores within a relative 1e-10 of the best are
 * ties and the smallest tied x wins. */
ll_status ll_leja_points(int count, double* xi_out);

/* Scaled divided differences d_j = gamma^j log[z_0..z_j], j = 0..degree, of log at
 * z_i = c + gamma xi_i with c = (lmin+lmax)/2 and gamma = (lmax-lmin)/4, by Algorithm 1
 * (Section 3.1): d = log(Q_m) e_1 with Q_m = c I + gamma Qhat_m and a Taylor series of
 * log(I + (Q_m - s I)/s). The series stops when a term's max-norm falls below 1e-18 times the
 * sum's (after >= 10 terms). When the series would need more than 1e6 terms (its factor
 * q = max_i |z_i/s - 1| gives ln(1e-18)/ln(q) > 1e6: condition numbers above ~1e5 at s = c, and
 * every s = lmax/2), the coefficients come from the textbook divided-difference table (Eq. Léja7)
 * of log(c + gamma xi) in the xi variable instead, and *terms_out is 0. A series that still fails
 * within 5e6 terms gives LL_ERR_DD_NOT_CONVERGED.
 * d_out: host, degree+1 doubles. terms_out: host, may be NULL. */
ll_status ll_divided_differences(ll_bounds bounds, int degree, int sval_mode, double* d_out, int* terms_out);

/* The same d_j (j = 0..degree) by the textbook divided-difference table of log(c + gamma xi)
 * over the Léja points xi_j (Eq. Léja7) carried out in binary128 arithmetic on the host and
 * rounded to FP64 (LL_DD_TABLE_Q). Every node and difference is exact or rounded at 113 bits, so
 * the table's cancellation leaves the FP64 coefficients accurate at any degree <= 100000 and any
 * condition number. c and gamma are the FP64 values (lmin+lmax)/2 and (lmax-lmin)/4.
 * d_out: host, degree+1 doubles. Errors: LL_ERR_INVALID_ARG, LL_ERR_BAD_BOUNDS (lmin <= 0,
 * lmin >= lmax, non-finite), LL_ERR_UNSUPPORTED (degree > 100000). */
ll_status ll_divided_differences_q(ll_bounds bounds, int degree, double* d_out);

/* ---- device kernels exposed for parity checks ---------------------------------------------- */

/* Gershgorin interval [min_i (a_ii - R_i), max_i (a_ii + R_i)], R_i = sum_{j!=i} |a_ij|
 * (Section 3 and Algorithm 1 step 1). Host result; synchronises `stream`. A non-positive lower
 * bound is returned as is: the caller decides (the Remark in Section 3 replaces it by an
 * epsilon > 0). Validates the CSR first. */
ll_status ll_gershgorin(ll_handle* h, const ll_csr* A, ll_bounds* out, void* stream);

/* Rayleigh quotient of A after `iters` normalised power steps from the Rademacher vector of
 * stream LL_STREAM_POWER (a cheap lambda_max estimate in the spirit of Appendix A).
 * lmax_out: host; synchronises `stream`. */
ll_status ll_power_lmax(ll_handle* h, const ll_csr* A, int iters, uint64_t seed, double* lmax_out, void* stream);

/* Largest matrix order accepted by ll_power_lmax_noalloc. */
#define LL_NOALLOC_MAX_ROWS (1 << 18)

/* The same estimate as ll_power_lmax (identical kernels, grid and reduction order, so identical
 * results on any part with at most 1024 SMs), for callers that cannot allocate device memory: code running inside an application
 * whose device memory belongs to another allocator (a framework's caching pool or a fixed arena
 * that forbids raw cudaMalloc), or latency-sensitive code that cannot accept the implicit device
 * synchronisation of cudaMalloc/cudaFree. No handle is needed and nothing is allocated: the
 * working vectors and reduction scratch live in one device array of about 4.2 MB that the library
 * reserves on every GPU that loads it, until the process exits. The paper has no counterpart.
 *   - A: device CSR with at most LL_NOALLOC_MAX_ROWS (262,144) rows; larger -> LL_ERR_UNSUPPORTED
 *     (also on a part with more than 1024 SMs).
 *   - lmax_out: host; the call synchronises `stream`.
 *   - The first call on a device looks up the array's address with that device current; make
 *     that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents (the call clears what must
 *     start at zero). Calls that overlap on the GPU race with each other: serialise them. */
ll_status ll_power_lmax_noalloc(const ll_csr* A, int iters, uint64_t seed, double* lmax_out, void* stream);

/* Probe block: out[i * ld + j] = probe(kind, seed, stream_id, row i, column j) for i < n,
 * j < cols, FP64, by the counter-based generator
 *   mix(z) = SplitMix64 output function of z + 0x9E3779B97F4A7C15 (Steele, Lea & Flood 2014),
 *   x = mix(seed ^ mix(stream_id * 2^56 + j * 2^32 + i)),
 *   Rademacher: 1 - 2 * (x >> 63);  Gaussian: Box-Muller of u1 = ((x >> 11) + 1) 2^-53 and
 *   u2 = (mix(x) >> 11) 2^-53.
 * Algorithm 3 steps 2 and 6. Requires n < 2^32, cols < 2^24. Enqueue only. */
ll_status ll_probes(ll_handle* h, int kind, uint64_t seed, int stream_id, int64_t n, int cols,
                    double* out, int64_t ld, void* stream);

/* PV = p_m(A) V: the degree-m Newton-Léja interpolant of log on [lmin, lmax] applied to the
 * n x b block V (Algorithm 2 with a fixed degree, all b columns at once):
 *   W_0 = V, W_{j+1} = (B - xi_j I) W_j with B = (A - c I) / gamma, PV = sum_j d_j W_j.
 * V, PV: device FP64, row-major, leading dimensions ldv, ldp (>= b). PV must not alias V.
 * precision: LL_PREC_*; the matrix values may be LL_F64 or LL_F32. Enqueue only (the host
 * coefficient set-up is synchronous). */
ll_status ll_apply_poly(ll_handle* h, const ll_csr* A, ll_bounds bounds, int degree, int precision,
                        const double* V, int64_t ldv, int b, double* PV, int64_t ldp, void* stream);

/* Algorithm 2 with its stopping rule (Section 3.1), column by column, on the same block as
 * ll_apply_poly: for every column c, m_c is the first m with |d_m| ||W_m[:, c]||_2 <= tol (m_c =
 * degree when none), and PV[:, c] = sum_{j <= m_c} d_j W_j[:, c]. The kernels reduce the norms
 * of every W_{j+1} with the step, retire the columns that meet the rule, and skip the remaining
 * steps once no column is left. degrees_out: host, b ints, receives m_c. tol > 0 (else
 * LL_ERR_INVALID_ARG), degree >= 1. Synchronises `stream`. */
ll_status ll_apply_poly_tol(ll_handle* h, const ll_csr* A, ll_bounds bounds, int degree, double tol, int precision,
                            const double* V, int64_t ldv, int b, double* PV, int64_t ldp, int* degrees_out,
                            void* stream);

/* ---- the estimator ------------------------------------------------------------------------- */

/* logdet_leja(csr, bounds, degree, probes, seed): Algorithm 3.
 *   sigma = lmin if lmin < 1 else 1; A~ = A / sigma on [lmin/sigma, lmax/sigma];
 *   S, G: n x k probes (k = probes/3; streams LL_STREAM_S, LL_STREAM_G);
 *   Y = p(A~) S; Q = CholeskyQR2(Y) (FP64); G' = G - Q (Q^T G);
 *   estimate = n log sigma + tr(Q^T p(A~) Q) + (1/k) tr(G'^T p(A~) G').
 * With opts->estimator = LL_EST_HUTCHINSON the call skips S, pass 1 and the QR and applies p(A~)
 * to G (probes columns) in the trace pass: estimate = n log sigma + (1/m) tr(G^T p(A~) G).
 * The matrix is device-resident (A). *estimate: host; synchronises `stream`.
 * With opts->keep_for_backward the handle keeps [Q | G'] (Hutchinson: G) for ll_logdet_backward;
 * ll_kept_basis returns LL_ERR_UNSUPPORTED after a Hutchinson forward. */
ll_status ll_logdet_forward(ll_handle* h, const ll_csr* A, ll_bounds bounds, const ll_options* opts,
                            double* estimate, void* stream);

/* The same estimate for a HOST-resident CSR (rowptr/colind/values are host pointers): the call
 * copies the matrix to the device (host-to-device copies inside the call), runs
 * ll_logdet_forward, and returns the estimate on the host. */
ll_status ll_logdet_forward_host(ll_handle* h, const ll_csr* A_host, ll_bounds bounds,
                                 const ll_options* opts, double* estimate, void* stream);

/* Derivative of the last kept forward estimate with respect to every stored value of A,
 * with [Q | G'], the bounds, sigma and the coefficients held fixed (stop-gradient through the
 * QR and the bounds; not in the paper):
 *   grad_values[e] += grad_output * (1/gamma) sum_{j<m} Lambda_{j+1}[r_e, :] . W_j[c_e, :],
 *   Lambda_m = d_m U, Lambda_j = d_j U + (B - xi_j I)^T Lambda_{j+1}, U = [Q | G'/k].
 * A must be symmetric (B^T = B is used; the call checks that every stored (r, c) has a stored
 * (c, r) of the same value, else LL_ERR_INVALID_ARG) and the same matrix (pattern and values) as
 * in the forward (only n and nnz are checked; ll_info.forward_id tells a caller whether another
 * forward ran on the handle since its own). The W_j come from the forward's trace pass when it kept them (ll_info.kept_w_steps),
 * else from checkpoints every ckpt_stride steps, recomputed. The contraction over the entries
 * runs inside the reverse steps or after each of them (ll_set_adjoint_fusion,
 * ll_info.adjoint_fused); the first backward of a shape may time both forms.
 * grad_values: device, nnz doubles, overwritten. Enqueue only. */
ll_status ll_logdet_backward(ll_handle* h, const ll_csr* A, double grad_output, double* grad_values, void* stream);

/* Derivative of the last kept forward estimate through the sketch's QR as well (Algorithm 3
 * step 4: Q = orth(Y), Y = p(A~) S, and G' = (I - Q Q^T) G move with A; the bounds, sigma and the
 * coefficients stay fixed): ll_logdet_backward's gradient plus the term
 *   grad_output * d/da_e tr(Gamma^T p(A~) S),  Gamma = 2 (I - Q Q^T) Z Q R^-T,
 *   Z Q = F Q - (1/k) G (G'^T F Q) - (1/k) (F G') (G^T Q),  F = p(A~),  Y = Q R,
 * which is the derivative of tr(dPi Z) for the projector Pi = Q Q^T onto span(Y). F [Q | G'] is
 * recomputed by one pass-1 sweep, the n x k products run on the GPU in FP64, R^-1 = R1^-1 R2^-1
 * (the two CholeskyQR factors) is formed on the host, and the second term runs the same reverse
 * recurrence with W_0 = S and U = Gamma. After a Hutchinson forward, or with k >= n (Q spans
 * R^n, so Gamma = 0), it equals ll_logdet_backward. Same arguments and requirements as
 * ll_logdet_backward; synchronises `stream`. */
ll_status ll_logdet_backward_qr(ll_handle* h, const ll_csr* A, double grad_output, double* grad_values, void* stream);

/* Chain to model parameters theta_p of a parameterised matrix A(theta) (e.g. the tau and kappa of a
 * Matérn GMRF): out[p] = sum_e grad_values[e] * dvalues[p * ld + e], p < nparams, where
 * dvalues[p * ld + e] = d a_e / d theta_p for every stored entry e < nnz. grad_values and
 * dvalues are device FP64 arrays; out is host (nparams doubles); synchronises `stream`. With
 * grad_values from ll_logdet_backward this is d estimate / d theta (chain rule; not in the paper). */
ll_status ll_param_grad(ll_handle* h, const double* grad_values, const double* dvalues, int64_t ld, int64_t nnz,
                        int nparams, double* out, void* stream);

/* Many independent estimates in one persistent launch per pass (batching, a11): count matrices
 * mats[0..count-1] (device CSR each), bounds b[i], per-matrix degree degrees[i] (NULL = from the
 * bound ratio: m = clamp(ceil(ln 1e6 / ln rho), 10, 250), rho = (sqrt(kappa)+1)/(sqrt(kappa)-1),
 * Proposition 3.1). opts->probes, seed, kind and precision apply to every matrix; matrix i uses
 * seed + i. estimates: host, count doubles; synchronises `stream`.
 * With opts->step_kernel = LL_KERNEL_AUTO the first call for a batch shape (precision, count, k,
 * total rows and entries, largest degree) times the candidate launch shapes on the real operands
 * (the TMA kernel with 512, 384 and 256 consumer threads per pass, i.e. rows per tile, and the
 * register kernel), keeps the fastest shape of each pass on the handle, and runs with it;
 * ll_info reports the shape (threads_pass1/2, rows_pass1/2, batch_tuned). */
ll_status ll_logdet_batched(ll_handle* h, const ll_csr* mats, const ll_bounds* b, int count,
                            const ll_options* opts, const int* degrees, double* estimates, void* stream);

/* Log-determinants along a matrix pencil (Section 5's GMRF likelihood over a theta grid, where
 * Q(theta) = I + theta Adj): estimates[g] ~ log det A_g for A_g = diag(D) + thetas[g] O, g < t,
 * every A_g symmetric positive definite with spectrum inside bounds[g] (the Léja interval of its
 * own scaling, Section 4) and run at degrees[g] (NULL: opts->degree for every theta). O: device
 * CSR (FP32 or FP64 values; its diagonal entries, if stored, are part of O); D: device, n FP64
 * values; thetas, bounds, degrees, estimates: host arrays of t entries.
 * All t estimates come from one pass pair over a block of t column groups, one per theta: each
 * step reads the shared sparsity structure once for every theta (a multi-value SpMM: one operand
 * offset per stored entry, then the t matrices' prepared values A_g / (sigma_g gamma_g), each
 * group with its own step scalars), and the block shrinks to the groups still running once a
 * theta's degree is reached (the groups are ordered by degree). Every theta takes the same probes
 * (opts->seed): estimates[g] equals ll_logdet_forward on A_g assembled in FP64 with the same
 * options, up to rounding. Where D_r != 0, O must store exactly one diagonal entry of row r
 * (LL_ERR_INVALID_ARG otherwise, after the passes).
 * opts as for ll_logdet_forward, with tol = 0 and keep_for_backward = 0 (LL_ERR_UNSUPPORTED
 * otherwise); TMA step kernel only (step_kernel AUTO or TMA); t x (probe columns of one theta,
 * rounded up to 16 bytes of a row) <= 1024, t n < 2^31 and k < n, else LL_ERR_UNSUPPORTED. ll_info reports the
 * phases (ms_*), the launch shapes and deg_max_pass2 = the largest degree. Synchronises
 * `stream`. */
ll_status ll_logdet_sweep(ll_handle* h, const ll_csr* O, const double* D, int t, const double* thetas,
                          const ll_bounds* bounds, const int* degrees, const ll_options* opts, double* estimates,
                          void* stream);

/* The Gram product X^T Z as CholeskyQR2 forms it (Algorithm 3 step 4: G = Y^T Y; step 6: C = Q^T G):
 * a parity hook for the Gram kernels. X: device, n x kx, row-major with leading dimension ldx, in
 * `layout` LL_PREC_F64 (FP64 elements) or LL_PREC_DF64 (the library's double-float blocks: the 16
 * bytes of columns (2q, 2q+1) of a row hold (hi_2q, hi_2q+1, lo_2q, lo_2q+1); ldx even). Z: device
 * FP64 n x kz (ldz), or NULL for X^T X. method: LL_GRAM_*. out: device kx x kz FP64 row-major.
 * 1 <= kx, kz <= 96; LL_GRAM_TENSOR with a width above 42 gives LL_ERR_UNSUPPORTED. Synchronises
 * `stream` (the kernel's bounded waits are checked: LL_ERR_TIMEOUT). */
ll_status ll_gram(ll_handle* h, int layout, const void* X, int64_t ldx, int kx, const double* Z, int64_t ldz, int kz,
                  int64_t n, int method, double* out, void* stream);

/* Diagnostics of the last ll_logdet_forward on this handle. */
ll_status ll_get_info(const ll_handle* h, ll_info* out);

/* Final degree of every column of one pass of the last ll_logdet_forward (pass 1: the k sketch
 * columns; pass 2: the columns of [Q | G'], or the Hutchinson probes), as fixed by Algorithm 2's
 * stopping rule (ll_options.tol), or the degree for every column under a fixed degree. out: host,
 * up to cap ints (may be NULL with cap 0); *count (host, may be NULL) receives the column count.
 * LL_ERR_NO_FORWARD before a forward; LL_ERR_INVALID_ARG for a pass other than 1 or 2. */
ll_status ll_stop_degrees(const ll_handle* h, int pass, int* out, int cap, int* count);

/* Copy the kept basis [Q | G'] of the last forward with keep_for_backward (FP64, n x (kq + kg):
 * columns [0, kq) hold Q, columns [kq, kq + kg) hold G' = (I - Q Q^T) G) into `out` (device,
 * leading dimension ld >= kq + kg). With out == NULL only the sizes are returned.
 * Sizes: host pointers, each may be NULL. Enqueue only (the copy runs on `stream`).
 * LL_ERR_NO_FORWARD when nothing is kept. */
ll_status ll_kept_basis(const ll_handle* h, double* out, int64_t ld, int64_t* n_out, int* kq_out, int* kg_out,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LEJA_H_ */
