// Kernel launch interfaces of the Léja log-determinant library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "leja.h"

namespace ll {

enum StepMode { MODE_PLAIN = 0, MODE_ACCUM = 1, MODE_DOT = 2, MODE_ADJ = 3 };
// Algorithm 2's stopping rule on top of ACCUM or DOT: the step also reduces ||W_{j+1} col||^2,
// the last CTA retires every column with |d_{j+1}| ||W_{j+1} col|| <= tol, P stops growing in
// retired columns, and once no column is left the following steps of the pass (all but the
// first) return at once.
constexpr int MODE_STOP = 4;
constexpr int MODE_ACCUM_STOP = MODE_ACCUM | MODE_STOP;
constexpr int MODE_DOT_STOP = MODE_DOT | MODE_STOP;
// A sweep over t matrices A_g that share one sparsity pattern (a theta grid of a parametric
// matrix), on top of ACCUM or DOT, on the TMA step kernel: the blocks stack one n x (2 sw_gpairs)
// block per group (ldw = 2 sw_gpairs; group g's row r is row g n + r; b = the columns of all
// groups), group g for A_g, with its own prepared values (each tile record holds one operand
// offset and the values of every group) and its own step scalars (beta_{g,j}, d_{g,j+1},
// d_{g,0}). A tile loads its operand rows once per group.
constexpr int MODE_SWEEP = 8;
constexpr int MODE_ACCUM_SWEEP = MODE_ACCUM | MODE_SWEEP;
constexpr int MODE_DOT_SWEEP = MODE_DOT | MODE_SWEEP;
// The adjoint step fused with the gradient contraction (TMA step kernel, on top of ADJ): besides
// Lambda_j = (B - xi_j I) Lambda_{j+1} + d_j U, a tile also adds, for every stored entry e = (r, c)
// of its rows, gscale <Lambda_{j+1}[c, :], W_j[r, :]> to grad[e]: the term of the transposed entry
// (c, r) (B symmetric), from the staged neighbour rows of Lambda_{j+1} and the tile's own W_j rows
// (staged beside them). grad is therefore in transposed order; the caller maps it back once, after
// the last step (launch_gather_add through the transposed-entry map).
constexpr int MODE_GRAD = 16;
constexpr int MODE_ADJ_GRAD = MODE_ADJ | MODE_GRAD;
constexpr int NUM_MODES = 32;
__host__ __device__ constexpr int base_mode(int mode) { return mode & 3; }
__host__ __device__ constexpr bool grad_mode(int mode) { return (mode & MODE_GRAD) != 0; }
__host__ __device__ constexpr bool stop_mode(int mode) { return (mode & MODE_STOP) != 0; }
__host__ __device__ constexpr bool sweep_mode(int mode) { return (mode & MODE_SWEEP) != 0; }
// per group and step of a sweep: beta_{g,j}, d_{g,j+1}, d_{g,0}
constexpr int SWEEP_SCALARS = 3;

// One Léja step over an n x b block, all columns at once (Algorithm 2 loop body):
//   Wout = B Win - xi_j Win   with B = (A - c I)/gamma folded into prepared values a_e / gamma
//          and beta = -(c/gamma + xi_j) applied to the row's own entry,
//   ACCUM: P = (first ? d0 * Win : P) + dn * Wout
//   DOT:   dots_next[col] = sum_i V[i, col] * Wout[i, col]   (and dots_first = V . Win if first)
//   ADJ:   Wout += coef(col) * V[i, col] with coef = adj_q for col < adj_split, adj_g otherwise
//          (the reverse recurrence Lambda_j = (B - xi_j I) Lambda_{j+1} + d_j U, B symmetric)
//   ACCUM_STOP / DOT_STOP: ACCUM / DOT with Algorithm 2's stopping rule (dn is applied only to
//          live columns; see MODE_STOP)
struct StepParams {
    const int32_t* rowptr;
    const int32_t* colind;
    const void* vals;        // prepared values (storage type of the precision)
    const void* win;
    void* wout;
    const void* v;
    void* p;
    double* partials;        // DOT: 2 * grid * b doubles
    unsigned int* ticket;    // DOT: zero-initialised counter, reset by the last block
    double* dots_next;
    double* dots_first;
    long long ldw, ldv, ldp;     // leading dimensions in columns (even: blocks are stored in column pairs)
    int n, b, tp, rl, rpt, num_tiles, smem_cap;
    int first;
    double beta, d0, dn;
    float2 beta_df, d0_df, dn_df;
    int adj_split;               // ADJ: first column using adj_g
    double adj_q, adj_g;         // ADJ: coefficients of V (FP64)
    float2 adj_q_df, adj_g_df;   // ADJ: the same as double-float pairs
    // STOP modes (partials then hold 3 * grid * b doubles: the norms are quantity 2)
    int* live;                   // per column (b rounded up to even): 1 while the column runs
    int* stop_deg;               // per column: the degree at which the column stopped
    int* done;                   // 1 once no column runs: the step returns at once
    double tol;                  // Algorithm 2's tolerance
    int jnext;                   // j + 1: the index of the W this step writes
    // SWEEP modes: the step's SWEEP_SCALARS scalars of every group (FP64 and double-float), the
    // column pairs of one group, and the elements between the groups' value arrays (vals holds
    // group g's prepared values at g * sw_vstride)
    const double* sw_scal;
    const float2* sw_scal_df;
    int sw_gpairs;
    long long sw_vstride;
    long long hub_bytes;         // TMA step: L2 bytes for the rows of the first (hub) rows of W_j
                                 // gathered with an evict-last policy (0: none)
    // ADJ_GRAD: W_j (W type, ldw), the gradient in transposed-entry order and its scale
    const void* wj;
    double* grad;
    double gscale;
};

struct StepLaunch {
    int threads;      // CTA size (multiple of 32, >= rl * b)
    int grid;
    size_t smem;
};

// Shape of the step launch for a block width b (threads_target: CTA size target; rpt: rows per
// thread per tile); fills p.rl, p.rpt, p.num_tiles, p.smem_cap.
StepLaunch plan_step(int precision, int mode, int n, int64_t nnz, int b, int threads_target, int rpt,
                     StepParams& p, int sm_count);
cudaError_t launch_step(int precision, int mode, const StepLaunch& L, const StepParams& p, cudaStream_t s);

// probes into columns [0, cols) of an n x ld block of element type out_type; columns
// [cols, pad) are set to zero (pad = cols for none). rowmap (optional, device, n entries): row i of
// the block holds the probe values of row rowmap[i] (a reordered matrix keeps its rows' probes)
cudaError_t launch_probes(int out_type, int kind, uint64_t seed, int stream_id, int n, int cols, int pad,
                          void* out, long long ld, cudaStream_t s, const int32_t* rowmap = nullptr);

// Locality reordering (reorder.cu): perm[i] = the old row of new row i, rows by entry count,
// descending (ties by row index; counts from 1023 on share one bucket), inv its inverse; the
// matrix P A P^T as rowptr_new (n + 1), colind_new (nnz; columns relabelled by inv, in the old
// row's order) and src (nnz; the old entry of each new entry). work: reorder_work_bytes(n).
size_t reorder_work_bytes(int n);
cudaError_t launch_reorder(const int32_t* rowptr, const int32_t* colind, int n, int32_t* perm, int32_t* inv,
                           int32_t* rowptr_new, int32_t* colind_new, int32_t* src, void* work, cudaStream_t s);
// *out = an order-independent 64-bit checksum of (rowptr, colind)
cudaError_t launch_structure_hash(const int32_t* rowptr, const int32_t* colind, int n, int64_t nnz,
                                  unsigned long long* out, cudaStream_t s);
// rows of halo on each side of a TMA step tile's window (entries with |col - row| <= TMA_HALO are
// always served from the window)
constexpr int TMA_HALO = 2;
// flag[0]: error bits (1 rowptr decreasing, 2 column out of range, 4 rowptr[0] != 0 or rowptr[n] != nnz);
// flag[1]: stored entries with |col - row| > TMA_HALO (int32; saturates nowhere below 2^31)
// rowmax (optional): atomicMax of the longest row's entry count
// unsorted (optional): rows whose column indices are not strictly increasing
// runs (optional): entries of flag[1] on a diagonal run ((i - 1, c - 1) or (i + 1, c + 1) stored,
// found by binary search: exact for rows with increasing columns, a hint otherwise)
cudaError_t launch_validate_csr(const int32_t* rowptr, const int32_t* colind, int n, int64_t nnz,
                                int* flag, cudaStream_t s, int* rowmax = nullptr, int* unsorted = nullptr,
                                int* runs = nullptr);
// flag[0] |= 1 when some stored entry (r, c) has no stored (c, r) of the same value; sorted: every
// row's columns strictly increase (the search is then binary)
cudaError_t launch_check_symmetric(const int32_t* rowptr, const int32_t* colind, const void* vals, int dtype, int n,
                                   int sorted, int* flag, cudaStream_t s);
cudaError_t launch_gershgorin(const int32_t* rowptr, const int32_t* colind, const void* vals, int dtype,
                              int n, double* partials, unsigned int* ticket, double* out, int grid, cudaStream_t s);
// out[e] = convert(values[src ? src[e] : e] * scale) into the storage type of `precision`
cudaError_t launch_prepare_values(const void* vals, int dtype, int64_t nnz, double scale, int precision,
                                  void* out, cudaStream_t s, const int32_t* src = nullptr);
// out[e] = convert((theta * o_e + [c_e == r_e] D_{r_e}) * scale) into the storage type of `precision`
// (one matrix of a pencil sweep diag(D) + theta O, prepared as launch_prepare_values would prepare
// it assembled in FP64); flag[0] |= 1 where D_r != 0 and row r stores no single diagonal entry
cudaError_t launch_prepare_pencil(const int32_t* rowptr, const int32_t* colind, const void* o, int dtype, const double* D,
                                  int n, double theta, double scale, int precision, void* out, int* flag,
                                  cudaStream_t s);
// out (type of `precision` W storage, ld_out) <- in (FP64, ld_in), n x b; columns [b, pad) of out
// are set to zero
cudaError_t launch_convert_block(const double* in, long long ld_in, int precision, void* out,
                                 long long ld_out, int n, int b, int pad, cudaStream_t s);
// out (FP64, ld_out) <- in (type of `precision` P storage, ld_in)
cudaError_t launch_block_to_f64(int precision, const void* in, long long ld_in, double* out,
                                long long ld_out, int n, int b, cudaStream_t s);

// out[r, c] = coef(c) * V[r, c] for c < b (coef = cq for c < split, cg otherwise), pad columns zero;
// V and out in the W storage type of `precision`, leading dimension ld
cudaError_t launch_scale_cols(int precision, const void* V, long long ld, int n, int b, int split, double cq, double cg,
                              void* out, cudaStream_t s);
// rowidx[e] = row of stored entry e
cudaError_t launch_row_index(const int32_t* rowptr, int n, int32_t* rowidx, cudaStream_t s);
// tmap[e] = the index of entry (c, r) for every entry e = (r, c) (rows with strictly increasing
// columns); flag[0] |= 1 where the transposed entry is not stored
cudaError_t launch_transpose_map(const int32_t* rowptr, const int32_t* colind, int n, int32_t* tmap, int* flag,
                                 cudaStream_t s);
// dst[e] += src[map[e]] for e < nnz
cudaError_t launch_gather_add(const int32_t* map, const double* src, int64_t nnz, double* dst, cudaStream_t s);
// P = sum_{j<=m} d_j W_j over W_0 = w0 and the m blocks W_1 .. W_m at wk (blk bytes apart), with the
// P-axpy step's arithmetic and order (same P as the pass); b columns, W and P leading dims ld, ldp
cudaError_t launch_weighted_sum(int precision, const void* w0, const void* wk, size_t blk, long long ld, int n, int b,
                                int m, const double* d, const float2* ddf, void* P, long long ldp, cudaStream_t s);
// g[e] += scale * <Lam[r_e, :], W[c_e, :]> over b columns for every stored entry (W storage type of
// `precision`, ld even; rowidx[e] = r_e from launch_row_index)
cudaError_t launch_sddmm(int precision, const int32_t* rowidx, const int32_t* colind, int64_t nnz, const void* lam,
                         const void* w, long long ld, int b, double scale, double* g, cudaStream_t s);
// out[p] = sum_e g[e] * dv[p * ldd + e], p < np; partials: np * grid doubles; result in out (device)
cudaError_t launch_param_dot(const double* g, const double* dv, long long ldd, int64_t nnz, int np, double* partials,
                             unsigned int* ticket, double* out, int grid, cudaStream_t s);

// out[r, c] = in[r, c0 + c], c < b, for blocks of W storage type t (the element's bits; both
// parts of a double-float pair); columns [b, pad) of out set to zero
cudaError_t launch_copy_cols(int t, const void* in, long long ld_in, int c0, void* out, long long ld_out, int n, int b,
                             int pad, cudaStream_t s);
// out (FP32, ld_out) <- hi + lo of a double-float column-pair block (ld_in), n x b; columns
// [b, pad) of out are set to zero
cudaError_t launch_dfp_to_f32(const void* in, long long ld_in, float* out, long long ld_out, int n, int b, int pad,
                              cudaStream_t s);
// out = alpha * in (FP64 blocks)
cudaError_t launch_scaled_copy_f64(const double* in, long long ld_in, double* out, long long ld_out, int n, int b,
                                   double alpha, cudaStream_t s);

// out[i * ld + i] = 1 for i < n (type t); the rest of `out` is left as is
cudaError_t launch_unit_diag(int t, void* out, long long ld, int n, cudaStream_t s);

// Banded Léja steps (band.cu): matrices whose entries all lie within BAND_H of the diagonal,
// stored as BAND_H * 2 + 1 diagonals (DIA layout of the prepared values), s <= BAND_SMAX steps
// per launch over row tiles with halos, the intermediate W in shared memory.
constexpr int BAND_H = 2;
constexpr int BAND_SMAX = 4;
constexpr int BAND_THREADS = 256;
struct BandParams {
    const void* dia;     // n x (2 BAND_H + 1) prepared values (the precision's raw value type)
    const void* win;     // W_{j0} (W type, ldw columns)
    void* wout;          // W_{j0+s}
    const void* v;       // pass 2: V (W type, ldw)
    void* p;             // pass 1: P (P type, ldp), read (j0 > 0) and written
    double* partials;    // pass 2: (BAND_SMAX + 1) x grid x b doubles
    unsigned int* ticket;   // pass 2: zero-initialised counter, reset by the last CTA
    double* dots;        // pass 2: (m + 1) x b traces; writes rows j0 + 1 .. j0 + s (and 0 if j0 = 0)
    long long ldw, ldp;
    int n, b, tp, R, num_tiles, s, j0;
    double beta[BAND_SMAX], dn[BAND_SMAX], d0;    // beta_{j0+q}, d_{j0+q+1}, d_0
    float2 beta_df[BAND_SMAX], dn_df[BAND_SMAX], d0_df;
};
struct BandLaunch {
    int R = 0, tp = 0, num_tiles = 0, grid = 0;
    size_t smem = 0;
};
// launch shape for (precision, MODE_ACCUM or MODE_DOT, n, b); false when not applicable
bool plan_band(int precision, int mode, int n, int b, int sm_count, BandLaunch& L);
cudaError_t launch_band(int precision, int mode, const BandLaunch& L, const BandParams& p, cudaStream_t s);
// dia[r * (2 BAND_H + 1) + (c - r + BAND_H)] = vals[e] for every entry e = (r, c) (rows with
// strictly increasing columns within BAND_H of the diagonal), zero elsewhere
cudaError_t launch_to_dia(int precision, const int32_t* rowptr, const int32_t* colind, const void* vals, int n, void* dia,
                          cudaStream_t s);

// Start of a pass under Algorithm 2's stopping rule: e_0 = |d_0| ||W_0 col||_2 for every column
// c < b of the n x b block W0 (element type of `precision`'s W blocks, ld columns); live[c] =
// (e_0 > tol), stop_deg[c] = live ? mmax : 0, live[b] = 0 when b is odd, *done = no column live.
// partials holds grid * b doubles (grid = STOP_INIT_GRID), ticket a zeroed counter (left zeroed).
constexpr int STOP_INIT_GRID = 304;
cudaError_t launch_stop_init(int precision, const void* W0, long long ld, int n, int b, double d0, double tol,
                             int mmax, double* partials, unsigned int* ticket, int* live, int* stop_deg, int* done,
                             cudaStream_t s);

// Power iteration helpers (FP64): y = A x; and reductions
cudaError_t launch_spmv_f64(const int32_t* rowptr, const int32_t* colind, const void* vals, int dtype, int n,
                            const double* x, double* y, cudaStream_t s);
cudaError_t launch_dot_f64(const double* x, const double* y, int n, double* partials, unsigned int* ticket,
                           double* out, int grid, cudaStream_t s);
cudaError_t launch_scale_f64(double* x, const double* num, int n, int mode, cudaStream_t s);

// CholeskyQR pieces. Each launch takes one job by value or, for a batch of matrices with the same
// widths and leading dimensions, a device array of jobs (one matrix per blockIdx.z for the Gram and
// row-product kernels, per CTA for the Cholesky).
struct GramJob {
    const void* X;            // n x kx (type tx)
    const void* Z;            // n x kz (FP64); unused when symmetric
    int n;
    int gx;                   // row blocks of this matrix (<= the launch's gridDim.x)
    double* partials;         // gx * OT * 16 doubles
    unsigned int* ticket;     // zero-initialised; reset by the last CTA
    double* out;              // kx x kz
};
struct CholJob {
    const double* G;          // k x k
    double* Rinv;             // k x k
    int* status;
};
struct RowJob {
    const void* X;            // n x kx rows (type tx): Y or Q1 (apply_rinv), Q (project)
    const double* M;          // kx x kc: R^{-1} or C
    const double* G;          // project: the residual probes (FP64)
    double* out64;            // FP64 output
    void* out2;               // optional second output (type t2); may be null
    int n;
};
// row blocks the Gram kernel uses for n rows under a budget of `grid` CTAs
int gram_blocks(int kx, int kz, bool sym, int n, int grid);
cudaError_t launch_gram_jobs(int tx, long long ldx, int kx, int tz, long long ldz, int kz, bool sym, const GramJob& one,
                             const GramJob* jobs, int count, int gx_max, cudaStream_t s);
cudaError_t launch_chol_jobs(int k, const CholJob& one, const CholJob* jobs, int count, cudaStream_t s);
cudaError_t launch_apply_rinv_jobs(int tx, long long ldx, int k, long long ld64, int t2, long long ld2, const RowJob& one,
                                   const RowJob* jobs, int count, int n_max, cudaStream_t s);
cudaError_t launch_project_jobs(long long ldq, int k, long long ldg, int kg, long long ld64, int t2, long long ld2,
                                int zero_pad, int col2, const RowJob& one, const RowJob* jobs, int count, int n_max,
                                cudaStream_t s);
// out = X M for an n x kx FP64 block X and a full kx x kc matrix M (row-major, device), the
// products in double-float as in apply_rinv; out64 FP64 (ld64), out2 (type t2, ld2) optional
cudaError_t launch_mul_small(const double* X, long long ldx, int n, int kx, int kc, const double* M, double* out64,
                             long long ld64, int t2, void* out2, long long ld2, cudaStream_t s);
// doubles of Gram partials needed for a launch with `grid` CTAs
size_t gram_partials_doubles(int kx, int kz, bool sym, int grid);
// The same Gram X^T Z on the tensor cores (gram_tc.cu): BF16 fixed-point digit slices of both
// operands (per-column scales from a maximum pre-pass), exact FP32 products in TMEM, double-float
// sums. X of type T_F64 or T_DF64 (column pairs, even ldx), Z FP64 (ignored when sym); widths up to
// 42 (gram_tc_digits: 7 digits up to 36, 6 up to 42, 0 = unsupported); partials:
// gram_tc_partials_doubles(kx, kz, sm_count) doubles; work: gram_tc_workspace_bytes(kx, kz,
// sm_count) bytes; ticket zero-initialised (reset by the last CTA); err set to 1 when a bounded wait
// runs out. One CTA per SM.
int gram_tc_digits(int kx, int kz);
bool gram_tc_supported(int tx, int kx, int kz, bool sym);
size_t gram_tc_partials_doubles(int kx, int kz, int grid);
size_t gram_tc_workspace_bytes(int kx, int kz, int grid);
cudaError_t launch_gram_tc(int tx, const void* X, long long ldx, int kx, const double* Z, long long ldz, int kz, long long n,
                           bool sym, double* partials, unsigned int* ticket, double* out, void* work, int* err,
                           long long spin_budget, int sm_count, cudaStream_t s);

// out (kx x kz, row-major) = X^T Z, X: n x kx (type tx), Z: n x kz (type tz); sym: X == Z
cudaError_t launch_gram(int tx, const void* X, long long ldx, int kx, int tz, const void* Z, long long ldz, int kz,
                        int n, bool sym, double* partials, unsigned int* ticket, double* out, int grid, cudaStream_t s);
// Cholesky G = R^T R (upper R) and Rinv = R^{-1}; status[0] = 1 on a non-positive pivot
cudaError_t launch_chol_rinv(const double* G, int k, double* Rinv, int* status, cudaStream_t s);
// Out = X * Rinv (upper triangular k x k), X type tx; writes FP64 (out64; may be null) and
// optionally out2 (type t2)
cudaError_t launch_apply_rinv(int tx, const void* X, long long ldx, int n, int k, const double* Rinv,
                              double* out64, long long ld64, int t2, void* out2, long long ld2, cudaStream_t s);
// G' = G - Q C in double-float arithmetic, G: FP64 (ldg), Q: type tq (T_F64 or T_DF64 column
// pairs, ldq), C k x kg; writes FP64 (out64, columns [0, kg); may be null) and optionally out2
// (type t2, columns [col2, col2 + kg)); zero_pad: also write 0 to the zero_pad columns after the
// last one (the pad columns of a pair layout)
cudaError_t launch_project(int tq, const void* Q, long long ldq, int k, const double* G, long long ldg, int kg,
                           const double* C, int n, double* out64, long long ld64, int t2, void* out2,
                           long long ld2, int zero_pad, int col2, cudaStream_t s);

// ---- batched passes (many matrices, one persistent launch per pass) ----------------------------
struct BatchMat {
    const int32_t* rowptr;
    const int32_t* colind;
    const void* vals;         // prepared values (storage type of the precision)
    const void* w0;           // W_0: the probe block S (pass 1) or V = [Q | G'] (pass 2)
    void* wa;                 // ping-pong blocks
    void* wb;
    void* p;                  // pass 1: P (P storage type), leading dimension as W
    double* partials;         // pass 2: 2 * T * b per-tile trace partials
    double* dots;             // pass 2: (m + 1) * b traces
    const double* coef;       // (beta_j, d_j) for j = 0..m
    int n, T, m;
};

constexpr int BATCH_THREADS = 256;   // CTA size of the register-gather persistent kernel

struct BatchParams {
    const BatchMat* mats;          // sorted by degree, descending
    const int* step_off;           // first item of each step (max_m + 1 entries)
    const int* step_active;        // matrices still active at each step (a prefix)
    const int* tile_prefix;        // tile prefix sums over the sorted matrices (count + 1)
    unsigned int* ticket;          // zero-initialised item counter
    int* error;                    // set when a bounded wait runs out
    unsigned long long* arrived;   // per matrix: tiles finished
    unsigned long long* released;  // per matrix: tiles of fully completed steps
    long long spin_budget;         // clock64 cycles a wait may spin
    long long ld;                  // leading dimension (columns, even) of every block
    int total_items, max_m, tp, rl, rpt, R, b, smem_cap;
};

// ---- TMA-fed step (k_leja_tma): geometry of the shared-memory pipeline -------------------------
struct TmaParams {
    int R;             // rows per tile (one row lane each)
    int ecap;          // entries per tile with a record; later entries load directly
    int fcap;          // far entries per tile gathered by TMA (multiple of 4)
    int nst;           // pipeline stages (tiles in flight + 1)
    int nprod;         // producer warps (divides nst)
    int slot;          // bytes of one gather4 slot (4 rows, 128-byte aligned)
    int wslots;        // gather slots taken by one extra window (R + 2 HALO rows)
    int rowbytes;      // bytes of one W row (ld * element size)
    int auxbytes;      // bytes of one V (pass 2, adjoint) or P (pass 1) row; 0 without
    int wjbytes;       // bytes of one staged W_j row (the reverse step with the gradient contraction); 0 without
    int gsp;           // lanes per entry of the gradient contraction (1, 2 or 4)
    int recbytes;      // bytes of one entry record (prepared value, operand offset)
    int hdr_bytes;     // descriptor header: R + 1 row offsets, z0, record count (16-byte padded)
    int desc_stride;   // bytes per tile of the descriptor array (header and ecap records)
    int gcol_stride;   // bytes per tile of the gather-column array (4 window rows, then fcap columns)
    int stage_bytes;   // bytes per stage: window, aux rows, gathered rows, descriptor
    int off_aux, off_wj, off_gat, off_desc;   // the window is at offset 0
    int hub_rows;      // gathered rows below this index (a degree-ordered matrix's hubs) are kept in
                       // L2 in preference to the others (0: no cache policy)
    int ngrp, gsz;     // a sweep's groups per tile and bytes of one group's part of a stage (its
                       // window, V or P rows and gathered rows at offsets off_aux, off_gat from
                       // g gsz; the shared descriptor at off_desc); 1, 0 otherwise
    int ring_base;     // gather-column rings of the producer warps, after the stages
    const unsigned char* desc;   // per-tile descriptors (built once per pass)
    const int* gcol;             // per-tile gather columns
    const int4* meta;            // per tile: (records, gathered rows, extra windows, 0)
    unsigned char* desc_w;       // the same arrays, writable (for the describe kernel)
    int* gcol_w;
    int4* meta_w;
    int* error;                                  // TMA_ERR_* where a bounded wait ran out (the first)
    long long spin_budget;                       // clock64 cycles a wait may spin
    int inject;                                  // test hook: tile 0 expects bytes no copy delivers
};
struct TmaLaunch {
    TmaParams q;
    int np = 1;       // column pairs per consumer thread (2: FP32-mixed, 16-byte row accesses)
    int threads, grid;
    size_t smem;
    size_t desc_bytes, gcol_bytes, meta_bytes;   // global descriptor arrays of the pass
};
// Shape of a TMA-fed step launch; false when the block layout does not allow TMA (a row wider than
// 256 elements or not a multiple of 16 bytes) or the pipeline does not fit in shared memory.
// ctas_per_sm: 1 (one 512-thread CTA with ~223 KB of stages) or 2 (two of half the size).
// nfar: entries with |col - row| > TMA_HALO, nrun: those of them on a diagonal run (the extra
// windows take them); maxrow: the longest row (all three size the per-tile record and gather
// capacities; hints, not bounds)
bool plan_step_tma(int precision, int mode, int n, int64_t nnz, int64_t nfar, int64_t nrun, int maxrow, int b,
                   int threads_target, int ctas_per_sm, StepParams& p, TmaLaunch& L, int sm_count, int np = 1);
cudaError_t launch_step_tma(int precision, int mode, const TmaLaunch& L, const StepParams& p, cudaStream_t s);
// builds the tile descriptors of a plan (L.q.desc_w, gcol_w, meta_w) from the CSR and the prepared
// values in p; once per pass, before its steps
cudaError_t launch_tma_describe(int precision, const TmaLaunch& L, const StepParams& p, cudaStream_t s);

void plan_batched(int b, double avg_nnz_per_row, BatchParams& bp, size_t* smem);
cudaError_t launch_batched(int precision, int mode, const BatchParams& bp, int grid, size_t smem, cudaStream_t s);

// element types used by the typed helpers above; T_DF64 blocks are double-float in column pairs
enum ElemType { T_F64 = 0, T_F32 = 1, T_DF64 = 2 };
// even leading dimension of a block of b columns
inline int even_ld(int b) { return b + (b & 1); }
// leading dimension of an n x b block in the W storage of `precision`: column pairs (even), and
// for FP32 a multiple of 4 so that a row is a whole number of 16-byte units (the TMA row stride).
// (Padding DF64 blocks to 4 columns as well, so that every width could take two column pairs per
// thread, cost 6% more bytes in pass 1 and the autotuner kept one pair: measured on the 128^3
// Laplacian, pass 1 30.7 -> 32.4 ms.)
inline int block_ld(int precision, int b) { return precision == LL_PREC_F32_MIXED ? (b + 3) & ~3 : b + (b & 1); }
inline int w_type_of(int precision) {
    return precision == LL_PREC_F64 ? T_F64 : (precision == LL_PREC_DF64 ? T_DF64 : T_F32);
}
inline int p_type_of(int precision) {
    return precision == LL_PREC_F64 ? T_F64 : T_DF64;
}
inline size_t elem_size(int t) { return t == T_F32 ? 4 : 8; }

}  // namespace ll
