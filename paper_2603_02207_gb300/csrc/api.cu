// C ABI of the Léja log-determinant library: handle and workspace, argument checks, the host
// coefficient set-up, and the orchestration of the device passes of Algorithm 3.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "common.cuh"
#include "host_math.h"
#include "kernels.cuh"
#include "leja.h"
#include "tma_common.cuh"

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    uint64_t gen = 0;   // the handle's ws_gen when the block was allocated
};

}  // namespace

struct ll_handle {
    int device = 0;
    int sm_count = 152;
    std::string err;
    std::map<std::string, Buf> ws;
    ll_info info{};
    cudaEvent_t ev[8] = {};
    int launches = 0;
    // step kernel of ll_apply_poly and ll_logdet_backward (ll_set_step_config)
    int cfg_kernel = LL_KERNEL_AUTO, cfg_threads = 0, cfg_rpt = 0;
    // autotuned step launches: (precision, mode, n, nnz, b, ld) -> (kernel, threads, rows per thread)
    std::map<std::tuple<int, int, int, int64_t, int, long long>, std::tuple<int, int, int>> tuned;
    long long spin_budget = 4000000000LL;   // clock cycles a TMA pipeline wait may spin (about 2 s)
    int inject = LL_INJECT_NONE;            // ll_debug_inject
    bool tma_used = false;                  // a TMA step ran since the last error-flag check
    int last_kernel = 0, last_threads = 0;  // choice of the last run_pass
    int last_np = 1;                        // and its column pairs per thread
    int last_rows = 0;                      // and its rows per tile
    // CUDA graph of the last forward's device work (replayed when the next call is identical)
    uint64_t ws_gen = 0;                    // bumped whenever a workspace buffer moves
    cudaStream_t cap_stream = nullptr;      // capture stream (the caller's may be the legacy stream)
    struct Graph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;
        int launches = 0, k1 = 0, t1 = 0, k2 = 0, t2 = 0, np1 = 1, np2 = 1, r1 = 0, r2 = 0;
        bool tma = false;
    } gfwd;
    // CUDA graph of the last batched call's device work, with what the host combine needs
    struct BatchGraph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;
        int launches = 0, kq = 0, kg = 0;
        std::vector<std::vector<double>> d;   // per matrix: d_0 .. d_m
        std::vector<double> sigma;
        std::vector<double*> dots;            // per matrix: device (m + 1) x 2k traces
        unsigned long long* ctr = nullptr;    // counters (error flag at 2 count + 2)
        int* qrstat = nullptr;
        int kernel = 0, threads1 = 0, threads2 = 0;   // step kernel of both passes, CTA sizes
        int rows1 = 0, rows2 = 0;                     // rows per tile of both passes
    } gbat;
    // autotuned batched launch shapes: (precision, count, k, total rows, total entries, largest degree)
    // -> (kernel, consumer-thread targets of both passes)
    std::map<std::tuple<int, int, int, int64_t, int64_t, int>, std::tuple<int, int, int>> tuned_batch;
    int64_t far_entries = 0;  // entries with |col - row| > TMA_HALO of the last validated matrix
    int64_t far_runs = 0;     // those of them on a diagonal run (a stencil's far diagonals)
    bool band_ok = false;     // the last validated matrix suits the banded kernel
    int max_row = 0;          // longest row of the last validated matrix
    bool sorted = false;      // every row of the last validated matrix has strictly increasing columns
    int64_t keep_budget = 0;  // ll_set_keep_budget: bytes the forward may keep for the backward (0: half the free memory)
    int fuse_mode = LL_FUSE_AUTO;   // ll_set_adjoint_fusion
    int64_t forward_id = 0;   // count of successful forwards on the handle (ll_info.forward_id)
    int gram_method = LL_GRAM_AUTO;   // CholeskyQR2 Gram kernel of the running call (ll_options.qr_gram)
    // the structure last reordered (LL_REORDER_DEGREE) and the allocation generations of the
    // workspace blocks that hold its permuted copy
    struct Reorder {
        const void* rp = nullptr;
        const void* ci = nullptr;
        int64_t n = -1, nnz = -1;
        unsigned long long hash = 0;
        uint64_t gens = 0;
    } ro;
    // L2 bytes for the hub rows of a degree-ordered matrix's passes (set by the forward that runs
    // on one; 0 otherwise)
    long long hub_bytes = 0;
    // LL_GRAM_AUTO: the faster Gram kernel per (element type, kx, kz, sym, n), timed on first use
    std::map<std::tuple<int, int, int, int, int>, int> gram_choice;
    // the adjoint's reverse step with the gradient contraction fused in (1) or followed by the
    // separate contraction (0), per (precision, n, nnz, width, ld): timed on first use
    std::map<std::tuple<int, int, long long, int, long long>, int> adj_fuse_choice;
    int kept_gram = LL_GRAM_AUTO;     // and of the kept forward (its backward uses the same)
    // cached coefficients of the last set-up
    double dd_lmin = 0, dd_lmax = 0;
    int dd_degree = -1, dd_sval = -1, dd_scheme = -1, dd_terms = 0;
    std::vector<double> dd;
    // kept forward state (for the backward)
    bool kept = false;
    int64_t kept_n = 0, kept_nnz = 0;
    int kept_kq = 0, kept_kg = 0, kept_m = 0, kept_prec = 0, kept_ckpt = 0;
    bool kept_hutch = false;  // the kept forward used plain Hutchinson (V = G, no basis)
    bool kept_qr = false;     // the kept forward ran the sketch and its CholeskyQR2 (S, G, R1^-1, R2^-1 kept)
    bool kept_band = false;   // the kept forward's matrix suits the banded kernel
    int kept_stride = 0;      // the kept forward's trace pass left W_1 .. W_m (1) or the checkpoints
                              // W_s, W_2s, ... (s > 1) in "bw_ckpt"; 0: none
    bool kept_wall_s = false; // and its pass 1 (W_0 = S) left them in "bw_ckpt_s"
    int64_t kept_far = 0;     // its far-entry count and longest row (TMA plans of the adjoint)
    int64_t kept_runs = 0;
    int kept_max_row = 0;
    bool kept_sorted = false; // its rows have strictly increasing columns (the symmetry check)
    // final degree of every column of both passes of the last forward (Algorithm 2's rule)
    bool have_forward = false;
    std::vector<int> last_deg1, last_deg2;
    double kept_sigma = 1, kept_c = 0, kept_gamma = 1;
    std::vector<double> kept_d, kept_xi;
};

namespace ll {
namespace {

ll_status fail(ll_handle* h, ll_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

#define LL_CK(expr)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail(h, LL_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void* ws_get(ll_handle* h, const char* name, size_t bytes, cudaError_t* err) {
    Buf& b = h->ws[name];
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return b.p;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    b.gen = ++h->ws_gen;
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = e;
        return nullptr;
    }
    b.bytes = bytes;
    return b.p;
}

// Frees a workspace block (if any); the next ws_get of the name allocates afresh.
void ws_release(ll_handle* h, const char* name) {
    auto it = h->ws.find(name);
    if (it == h->ws.end()) return;
    if (it->second.p) cudaFree(it->second.p);
    h->ws.erase(it);
    h->ws_gen++;
}

#define WS(ptr, type, name, bytes)                                                               \
    type ptr = nullptr;                                                                          \
    do {                                                                                         \
        cudaError_t e_ = cudaSuccess;                                                            \
        ptr = (type)ws_get(h, name, (bytes), &e_);                                               \
        if (!ptr) return fail(h, LL_ERR_OOM, std::string("workspace ") + name + ": " + cudaGetErrorString(e_)); \
    } while (0)

ll_status check_csr_args(ll_handle* h, const ll_csr* A) {
    if (!A) return fail(h, LL_ERR_INVALID_ARG, "null matrix");
    if (A->n < 0 || A->nnz < 0) return fail(h, LL_ERR_INVALID_ARG, "negative size");
    if (A->n >= (int64_t)1 << 31 || A->nnz >= (int64_t)1 << 31) return fail(h, LL_ERR_UNSUPPORTED, "n and nnz must be < 2^31 (int32 CSR)");
    if (A->dtype != LL_F64 && A->dtype != LL_F32) return fail(h, LL_ERR_INVALID_ARG, "unknown value dtype");
    if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && (!A->colind || !A->values))))
        return fail(h, LL_ERR_INVALID_ARG, "null CSR array");
    return LL_OK;
}

ll_status check_bounds(ll_handle* h, ll_bounds b) {
    if (!std::isfinite(b.lmin) || !std::isfinite(b.lmax) || !(b.lmin > 0.0) || !(b.lmin < b.lmax))
        return fail(h, LL_ERR_BAD_BOUNDS, "bounds must satisfy 0 < lmin < lmax (finite)");
    return LL_OK;
}

// Validates the device CSR (synchronises the stream).
ll_status validate_csr(ll_handle* h, const ll_csr* A, cudaStream_t s) {
    if (A->n == 0) return LL_OK;
    WS(flag, int*, "csr_flag", 5 * sizeof(int));
    LL_CK(cudaMemsetAsync(flag, 0, 5 * sizeof(int), s));
    LL_CK(launch_validate_csr(A->rowptr, A->colind, (int)A->n, A->nnz, flag, s, flag + 2, flag + 3, flag + 4));
    h->launches++;
    int hv[5] = {0, 0, 0, 0, 0};
    LL_CK(cudaMemcpyAsync(hv, flag, sizeof hv, cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    const int hf = hv[0];
    h->far_entries = hv[1];
    h->far_runs = hv[4];
    h->max_row = hv[2];
    // the banded kernel takes matrices whose rows hold strictly increasing columns within
    // BAND_H (= TMA_HALO) of the diagonal
    h->band_ok = hv[1] == 0 && hv[3] == 0;
    h->sorted = hv[3] == 0;
    if (hf) {
        char buf[160];
        snprintf(buf, sizeof buf, "invalid CSR:%s%s%s", (hf & 4) ? " rowptr[0]!=0 or rowptr[n]!=nnz;" : "",
                 (hf & 1) ? " rowptr decreasing;" : "", (hf & 2) ? " column index out of range;" : "");
        return fail(h, LL_ERR_BAD_CSR, buf);
    }
    return LL_OK;
}

// Léja points and Algorithm 1 coefficients for [lmin, lmax] (cached on the handle).
// d[0..degree] on the scaled interval [lmin, lmax] by the chosen scheme; the Taylor terms used
// (0 for either table), -1 if Algorithm 1 did not converge.
int coefficients_by_scheme(double lmin, double lmax, int degree, int sval, int scheme, double* d) {
    if (scheme == LL_DD_TABLE_Q) {
        divided_differences_table_q(lmin, lmax, degree, d);
        return 0;
    }
    return scaled_divided_differences(lmin, lmax, degree, sval, d);
}

ll_status setup_coefficients(ll_handle* h, double lmin, double lmax, int degree, int sval, std::vector<double>& xi,
                             std::vector<double>& d, int scheme = LL_DD_AUTO) {
    xi.resize(degree + 1);
    leja_points(degree + 1, xi.data());
    if (!(h->dd_degree == degree && h->dd_sval == sval && h->dd_scheme == scheme && h->dd_lmin == lmin &&
          h->dd_lmax == lmax)) {
        std::vector<double> dn(degree + 1);
        const int terms = coefficients_by_scheme(lmin, lmax, degree, sval, scheme, dn.data());
        if (terms < 0) return fail(h, LL_ERR_DD_NOT_CONVERGED, "Algorithm 1 Taylor series did not converge within 5e6 terms");
        h->dd = dn;
        h->dd_degree = degree;
        h->dd_sval = sval;
        h->dd_scheme = scheme;
        h->dd_lmin = lmin;
        h->dd_lmax = lmax;
        h->dd_terms = terms;
    }
    d = h->dd;
    return LL_OK;
}

int64_t pad_elems(int64_t x) { return (x + 31) & ~(int64_t)31; }

// A planned step launch: the register-gather kernel (k_leja_step) or the TMA-fed one (k_leja_tma).
struct StepExec {
    int kind = LL_KERNEL_GATHER;
    int threads = 0, rpt = 0;   // requested shape (0 = kernel default)
    StepLaunch gl{};
    TmaLaunch tl{};
    int grid() const { return kind == LL_KERNEL_TMA ? tl.grid : gl.grid; }
    int cta() const { return kind == LL_KERNEL_TMA ? tl.threads : gl.threads; }
};

// Plans a launch of the given kind (shape fields of p are filled); false when not applicable.
bool plan_exec(ll_handle* h, int kind, int precision, int mode, int n, int64_t nnz, int b, int threads, int rpt,
               StepParams& p, StepExec& E) {
    E.kind = kind;
    E.threads = threads;
    E.rpt = rpt;
    if (kind == LL_KERNEL_TMA) {
        // rpt = 2 selects two column pairs per consumer thread (FP32-mixed blocks)
        const int ctas = (threads > 0 && threads <= 256) ? 2 : 1;
        if (!plan_step_tma(precision, mode, n, nnz, h->far_entries, h->far_runs, h->max_row, b, threads, ctas, p, E.tl, h->sm_count,
                           rpt == 2 ? 2 : 1))
            return false;
        E.tl.q.spin_budget = h->spin_budget;
        E.tl.q.inject = h->inject;
        return true;
    }
    E.gl = plan_step(precision, mode, n, nnz, b, threads, rpt, p, h->sm_count);
    return true;
}

cudaError_t exec_step(ll_handle* h, int precision, int mode, const StepExec& E, const StepParams& p, cudaStream_t s) {
    h->launches++;
    if (E.kind == LL_KERNEL_TMA) {
        h->tma_used = true;
        return launch_step_tma(precision, mode, E.tl, p, s);
    }
    return launch_step(precision, mode, E.gl, p, s);
}

// Workspace of a step launch: DOT partials for the plan's grid, and the TMA error flag.
// Workspace of a step launch: DOT partials for the plan's grid; for the TMA kernel the error flag
// and the pass's tile descriptors (one set per mode, built here from the CSR and the prepared
// values in p, on the stream, before the pass's steps).
ll_status bind_exec(ll_handle* h, int precision, int mode, int b, StepExec& E, StepParams& p, cudaStream_t s) {
    if (base_mode(mode) == MODE_DOT || stop_mode(mode)) {
        WS(partials, double*, "dot_partials", (size_t)3 * E.grid() * b * sizeof(double));
        p.partials = partials;
    }
    if (E.kind == LL_KERNEL_TMA) {
        WS(err, int*, "tma_error", sizeof(int));
        E.tl.q.error = err;
        // one descriptor set per mode (a pass's steps and the adjoint's reverse steps interleave)
        static const char* mname[] = {"plain", "accum", "dot", "adj", "4", "accum_stop", "dot_stop", "7",
                                      "8", "accum_sweep", "dot_sweep", "11", "12", "13", "14", "15",
                                      "16", "17", "18", "adj_grad"};
        const std::string mnm = mode < (int)(sizeof mname / sizeof mname[0]) ? mname[mode] : std::to_string(mode);
        WS(desc, unsigned char*, ("tma_desc_" + mnm).c_str(), E.tl.desc_bytes);
        WS(gcol, int*, ("tma_gcol_" + mnm).c_str(), E.tl.gcol_bytes);
        WS(meta, int4*, ("tma_meta_" + mnm).c_str(), E.tl.meta_bytes);
        E.tl.q.desc = desc;
        E.tl.q.gcol = gcol;
        E.tl.q.meta = meta;
        E.tl.q.desc_w = desc;
        E.tl.q.gcol_w = gcol;
        E.tl.q.meta_w = meta;
        LL_CK(launch_tma_describe(precision, E.tl, p, s));
        h->launches++;
    }
    return LL_OK;
}

// Reads and clears the TMA pipeline's error flag (synchronises the stream); LL_ERR_TIMEOUT if set.
ll_status check_tma_flag(ll_handle* h, cudaStream_t s) {
    if (!h->tma_used) return LL_OK;
    h->tma_used = false;
    WS(err, int*, "tma_error", sizeof(int));
    int v = 0;
    LL_CK(cudaMemcpyAsync(&v, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    if (v) {
        LL_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
        return fail(h, LL_ERR_TIMEOUT, "step kernel: a bounded pipeline wait ran out (code " + std::to_string(v) + ")");
    }
    return LL_OK;
}

// X^T Z (Z = X when sym) for CholeskyQR2 and the through-QR adjoint: on the tensor cores (k_gram_tc)
// when h->gram_method allows and the widths and element type fit, else in double-float on the FP32
// pipes (k_gram). The tensor-core kernel's bounded waits report through the pipeline error flag.
ll_status run_gram(ll_handle* h, int tx, const void* X, long long ldx, int kx, const double* Z, long long ldz, int kz,
                   int n, bool sym, double* partials, unsigned int* ticket, double* out, int ggrid, cudaStream_t s) {
    bool tc = h->gram_method != LL_GRAM_DFLOAT && gram_tc_supported(tx, kx, kz, sym) && (tx != T_DF64 || ldx % 2 == 0);
    if (h->gram_method == LL_GRAM_TENSOR && !tc)
        return fail(h, LL_ERR_UNSUPPORTED, "tensor-core Gram: widths up to 42 and FP64 or double-float operands");
    auto launch = [&](bool on_tc) -> ll_status {
        if (on_tc) {
            WS(err, int*, "tma_error", sizeof(int));
            WS(work, void*, "gram_tc_work", gram_tc_workspace_bytes(kx, sym ? kx : kz, h->sm_count));
            h->tma_used = true;
            LL_CK(launch_gram_tc(tx, X, ldx, kx, Z, ldz, kz, n, sym, partials, ticket, out, work, err, h->spin_budget,
                                 h->sm_count, s));
            h->launches += sym ? 2 : 3;
        } else {
            LL_CK(launch_gram(tx, X, ldx, kx, T_F64, sym ? nullptr : Z, ldz, kz, n, sym, partials, ticket, out, ggrid, s));
            h->launches++;
        }
        return LL_OK;
    };
    if (tc && h->gram_method == LL_GRAM_AUTO) {
        // both kernels timed once per shape (not inside a stream capture, where the tensor-core
        // kernel is taken), the faster cached; the chosen one runs last, so its result is the one
        // every later call of the shape reproduces
        const auto key = std::make_tuple(tx, kx, sym ? kx : kz, (int)sym, n);
        auto it = h->gram_choice.find(key);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        LL_CK(cudaStreamIsCapturing(s, &cs));
        if (it != h->gram_choice.end()) {
            tc = it->second == LL_GRAM_TENSOR;
        } else if (cs == cudaStreamCaptureStatusNone) {
            float ms[2] = {0.f, 0.f};
            const int counted = h->launches;   // the timing runs are not the call's launches
            // each kernel once untimed (a kernel's first launch may also load its module), then timed
            for (int rep = 0; rep < 2; ++rep) {
                for (int v = 0; v < 2; ++v) {
                    LL_CK(cudaEventRecord(h->ev[6], s));
                    ll_status st = launch(v == 0);
                    if (st != LL_OK) return st;
                    LL_CK(cudaEventRecord(h->ev[7], s));
                    LL_CK(cudaEventSynchronize(h->ev[7]));
                    LL_CK(cudaEventElapsedTime(&ms[v], h->ev[6], h->ev[7]));
                }
            }
            h->launches = counted;
            tc = ms[0] <= ms[1];
            h->gram_choice[key] = tc ? LL_GRAM_TENSOR : LL_GRAM_DFLOAT;
        }
    }
    return launch(tc);
}

// doubles of Gram partials for either kernel (kx x kz, grid ggrid for k_gram)
size_t gram_partials_any(const ll_handle* h, int kx, int kz, bool sym, int ggrid) {
    return std::max(gram_partials_doubles(kx, kz, sym, ggrid), gram_tc_partials_doubles(kx, kz, h->sm_count));
}

// The degree-ordered copy P A P^T of A for the passes (LL_REORDER_DEGREE): built on the device
// when A's structure differs from the cached one (pointers, sizes and a checksum of rowptr and
// colind) or a block holding it was reallocated; Aw then describes it (A's values, gathered
// through *src by the value preparation), *perm maps its rows to A's (the probes' row map), and
// the handle's matrix statistics are the permuted matrix's.
ll_status prepare_reorder(ll_handle* h, const ll_csr* A, ll_csr& Aw, const int32_t** perm_out, const int32_t** src_out,
                          cudaStream_t s) {
    const int n = (int)A->n;
    WS(perm, int32_t*, "ro_perm", (size_t)n * sizeof(int32_t));
    WS(inv, int32_t*, "ro_inv", (size_t)n * sizeof(int32_t));
    WS(rp2, int32_t*, "ro_rowptr", (size_t)(n + 1) * sizeof(int32_t));
    WS(ci2, int32_t*, "ro_colind", (size_t)A->nnz * sizeof(int32_t));
    WS(src, int32_t*, "ro_src", (size_t)A->nnz * sizeof(int32_t));
    WS(work, void*, "ro_work", reorder_work_bytes(n));
    WS(hash, unsigned long long*, "ro_hash", sizeof(unsigned long long));
    uint64_t gens = 0;
    for (const char* nm : {"ro_perm", "ro_inv", "ro_rowptr", "ro_colind", "ro_src"}) gens = gens * 1000003u + h->ws[nm].gen;
    LL_CK(launch_structure_hash(A->rowptr, A->colind, n, A->nnz, hash, s));
    h->launches++;
    unsigned long long hv = 0;
    LL_CK(cudaMemcpyAsync(&hv, hash, sizeof hv, cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    ll_handle::Reorder& R = h->ro;
    if (!(R.rp == A->rowptr && R.ci == A->colind && R.n == A->n && R.nnz == A->nnz && R.hash == hv && R.gens == gens)) {
        LL_CK(launch_reorder(A->rowptr, A->colind, n, perm, inv, rp2, ci2, src, work, s));
        h->launches += 8;
        R.rp = A->rowptr;
        R.ci = A->colind;
        R.n = A->n;
        R.nnz = A->nnz;
        R.hash = hv;
        R.gens = gens;
    }
    Aw = *A;
    Aw.rowptr = rp2;
    Aw.colind = ci2;
    *perm_out = perm;
    *src_out = src;
    return validate_csr(h, &Aw, s);
}

// The blocks of Algorithm 3 steps 4 and 6 for one sketch (leading dimensions in columns; typed
// pointers already offset to the sketch's columns where several share a block)
struct QrBlocks {
    const void* P;       // Y: n x kq, P storage type of the precision
    long long lp;
    void* q1;            // Q1 of the first CholeskyQR (FP64; double-float pairs outside the F64 mode)
    long long lq1;
    const double* G;     // the residual probes, n x kg FP64 (ld kg)
    void* V;             // the trace block [Q | G'] (W storage type)
    double* basis;       // [Q | G'] in FP64 (F64 mode) or as double-float pairs (FP32-mixed); unused in DF64
    long long lv;        // leading dimension of V and basis
    int vpad;            // columns of V written (from column 0): b2 and zeros up to vpad
    double* gpart;
    unsigned int* gticket;
    double* gram;
    double* rinv1;
    double* rinv;
    int* qrstat;
    int ggrid;
};

// Algorithm 3 step 4, Q = CholeskyQR2(Y), and step 6, G' = G - Q (Q^T G), forming V = [Q | G'].
// Outside the F64 mode Q1 and Q stay double-float column pairs: the products are double-float
// anyway, and FP64 intermediates would only add conversions on GB300's slow FP64 pipe. In the DF64
// mode Q lives in V itself; in the FP32-mixed mode [Q | G'] is formed as pairs in the basis block
// and V (FP32) is written from it; the F64 mode keeps FP64 Q1 and Q (the basis block, which is V).
ll_status qr_project(ll_handle* h, int prec, int n, int kq, int kg, const QrBlocks& B, cudaStream_t q) {
    ll_status st;
    const int b2 = kq + kg;
    const int pt = p_type_of(prec);
    const bool dfq = prec != LL_PREC_F64;
    const bool qv = prec == LL_PREC_DF64;
    const int tq = dfq ? T_DF64 : T_F64;
    void* Qb = qv ? B.V : static_cast<void*>(B.basis);
    const long long l2 = B.lv;
    if ((st = run_gram(h, pt, B.P, B.lp, kq, nullptr, 0, kq, n, true, B.gpart, B.gticket, B.gram, B.ggrid, q)) != LL_OK)
        return st;
    LL_CK(launch_chol_rinv(B.gram, kq, B.rinv1, B.qrstat, q));
    if (dfq) LL_CK(launch_apply_rinv(pt, B.P, B.lp, n, kq, B.rinv1, nullptr, 0, T_DF64, B.q1, B.lq1, q));
    else LL_CK(launch_apply_rinv(pt, B.P, B.lp, n, kq, B.rinv1, static_cast<double*>(B.q1), B.lq1, T_F64, nullptr, 0, q));
    if ((st = run_gram(h, tq, B.q1, B.lq1, kq, nullptr, 0, kq, n, true, B.gpart, B.gticket, B.gram, B.ggrid, q)) != LL_OK)
        return st;
    LL_CK(launch_chol_rinv(B.gram, kq, B.rinv, B.qrstat, q));
    if (dfq) LL_CK(launch_apply_rinv(tq, B.q1, B.lq1, n, kq, B.rinv, nullptr, l2, T_DF64, Qb, l2, q));
    else LL_CK(launch_apply_rinv(tq, B.q1, B.lq1, n, kq, B.rinv, B.basis, l2, T_F64, nullptr, l2, q));
    if ((st = run_gram(h, tq, Qb, l2, kq, B.G, kg, kg, n, false, B.gpart, B.gticket, B.gram, B.ggrid, q)) != LL_OK)
        return st;
    // G' into columns [kq, kq + kg); the pad columns up to the leading dimension are zeroed by the
    // same kernel.
    // The typed block pointer is offset by kq elements: element index r * l2 + kq + c.
    LL_CK(launch_project(tq, Qb, l2, kq, B.G, kg, kg, B.gram, n, dfq ? nullptr : B.basis + kq, l2, T_DF64,
                         dfq ? Qb : nullptr, l2, (int)(l2 - b2), kq, q));
    h->launches += 5;   // (run_gram counts its own)
    if (dfq && !qv) {
        LL_CK(launch_dfp_to_f32(B.basis, l2, static_cast<float*>(B.V), l2, n, b2, B.vpad, q));
        h->launches++;
    }
    return LL_OK;
}

// Chooses the step launch for (precision, mode, n, nnz, b). kernel = LL_KERNEL_AUTO times the
// candidates on the real operands once (p holds a representative non-first step: its outputs are
// overwritten by the pass) and caches the fastest on the handle.
ll_status choose_exec(ll_handle* h, int precision, int mode, int n, int64_t nnz, int b, int kernel, int threads,
                      int rpt, StepParams& p, StepExec& E, cudaStream_t s) {
    ll_status st;
    if (kernel == LL_KERNEL_TMA) {
        StepParams q = p;
        if (plan_exec(h, LL_KERNEL_TMA, precision, mode, n, nnz, b, threads, rpt, q, E)) {
            p = q;
            return bind_exec(h, precision, mode, b, E, p, s);
        }
        kernel = LL_KERNEL_GATHER;
        threads = 0;
        rpt = 0;
    }
    if (kernel == LL_KERNEL_GATHER) {
        plan_exec(h, LL_KERNEL_GATHER, precision, mode, n, nnz, b, threads, rpt, p, E);
        return bind_exec(h, precision, mode, b, E, p, s);
    }
    const auto key = std::make_tuple(precision, mode, n, nnz, b, p.ldw);
    auto it = h->tuned.find(key);
    if (it != h->tuned.end()) {
        const int kind = std::get<0>(it->second);
        plan_exec(h, kind, precision, mode, n, nnz, b, std::get<1>(it->second), std::get<2>(it->second), p, E);
        return bind_exec(h, precision, mode, b, E, p, s);
    }
    struct Cand { int kind, threads, rpt; };
    // (TMA candidates with rpt = 2 take two column pairs per thread; FP32-mixed only)
    const Cand cands[] = {{LL_KERNEL_TMA, 512, 0}, {LL_KERNEL_TMA, 256, 0}, {LL_KERNEL_TMA, 512, 2},
                          {LL_KERNEL_TMA, 256, 2}, {LL_KERNEL_GATHER, 0, 8}, {LL_KERNEL_GATHER, 0, 4},
                          {LL_KERNEL_GATHER, 0, 2}, {LL_KERNEL_GATHER, 256, 2}};
    float best_ms = 0.f;
    Cand best{LL_KERNEL_GATHER, 0, 8};
    bool have = false;
    for (const Cand& c : cands) {
        StepParams q = p;
        StepExec C;
        if (!plan_exec(h, c.kind, precision, mode, n, nnz, b, c.threads, c.rpt, q, C)) continue;
        if ((st = bind_exec(h, precision, mode, b, C, q, s)) != LL_OK) return st;
        LL_CK(exec_step(h, precision, mode, C, q, s));
        LL_CK(cudaEventRecord(h->ev[6], s));
        LL_CK(exec_step(h, precision, mode, C, q, s));
        LL_CK(exec_step(h, precision, mode, C, q, s));
        LL_CK(cudaEventRecord(h->ev[7], s));
        LL_CK(cudaEventSynchronize(h->ev[7]));
        if ((st = check_tma_flag(h, s)) != LL_OK) return st;
        float ms = 0.f;
        LL_CK(cudaEventElapsedTime(&ms, h->ev[6], h->ev[7]));
        if (!have || ms < best_ms) {
            best_ms = ms;
            best = c;
            have = true;
        }
    }
    h->tuned[key] = std::make_tuple(best.kind, best.threads, best.rpt);
    plan_exec(h, best.kind, precision, mode, n, nnz, b, best.threads, best.rpt, p, E);
    return bind_exec(h, precision, mode, b, E, p, s);
}

// Per-column state of a pass under Algorithm 2's stopping rule (device; live and stop_deg hold
// b rounded up to even ints). tol = 0: fixed degree.
struct StopState {
    double tol = 0.0;
    int* live = nullptr;
    int* stop_deg = nullptr;
    int* done = nullptr;
};

// Runs m Léja steps over an n x b block.
//   mode ACCUM: W_0 = win0 (ld = ldw), P accumulates sum_j d_j W_j (P type, ld = ldp)
//   mode DOT:   W_0 = V = win0, dots[(j) * b + col] = <V_col, W_j col> for j = 0..m
// With stop.tol > 0 the pass runs the STOP variant of the mode: the launch that starts it sets
// the column state from ||W_0||, each step retires the columns that meet the rule (P stops
// growing there; the dots of later steps are still written for the columns that run), and once
// no column runs the remaining steps return at once. stop.stop_deg then holds each column's
// final degree. The step kernel is the one chosen for the plain mode.
// The pass on the banded kernel: the prepared values in DIA layout, then ceil(m / BAND_SMAX)
// launches of up to BAND_SMAX steps each (W_j in and W_{j+s} out alternate between wa and wb).
ll_status run_band_pass(ll_handle* h, const ll_csr* A, const void* vals_prep, int precision, int mode, int n, int b,
                        const BandLaunch& BL, const void* win0, long long ldw, void* wa, void* wb, void* P,
                        long long ldp, double* dots, const std::vector<double>& beta, const std::vector<double>& d,
                        cudaStream_t s) {
    static_assert(BAND_H == TMA_HALO, "the band test of the validation uses TMA_HALO");
    const int m = (int)d.size() - 1;
    const size_t raw = precision == LL_PREC_F32_MIXED ? 4 : 8;
    WS(dia, void*, "band_dia", (size_t)n * (2 * BAND_H + 1) * raw);
    LL_CK(launch_to_dia(precision, A->rowptr, A->colind, vals_prep, n, dia, s));
    h->launches++;
    BandParams bp{};
    bp.dia = dia;
    bp.ldw = ldw;
    bp.ldp = ldp;
    bp.n = n;
    bp.b = b;
    bp.tp = BL.tp;
    bp.R = BL.R;
    bp.num_tiles = BL.num_tiles;
    bp.d0 = d[0];
    bp.d0_df = df_split(d[0]);
    if (mode == MODE_DOT) {
        WS(partials, double*, "band_partials", (size_t)(BAND_SMAX + 1) * BL.grid * b * sizeof(double));
        WS(ticket, unsigned int*, "dot_ticket", sizeof(unsigned int));
        LL_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
        bp.v = win0;
        bp.partials = partials;
        bp.ticket = ticket;
        bp.dots = dots;
    } else {
        bp.p = P;
    }
    const void* cur = win0;
    int flip = 0;
    for (int j = 0; j < m;) {
        const int sn = std::min(BAND_SMAX, m - j);
        bp.j0 = j;
        bp.s = sn;
        for (int q = 0; q < sn; ++q) {
            bp.beta[q] = beta[j + q];
            bp.dn[q] = d[j + q + 1];
            bp.beta_df[q] = df_split(beta[j + q]);
            bp.dn_df[q] = df_split(d[j + q + 1]);
        }
        void* out = flip ? wb : wa;
        bp.win = cur;
        bp.wout = out;
        LL_CK(launch_band(precision, mode, BL, bp, s));
        h->launches++;
        cur = out;
        flip ^= 1;
        j += sn;
    }
    h->last_kernel = LL_KERNEL_BAND;
    h->last_threads = BAND_THREADS;
    h->last_np = 1;
    h->last_rows = BL.R;
    return LL_OK;
}

ll_status run_pass(ll_handle* h, const ll_csr* A, const void* vals_prep, int precision, int mode, int n, int b,
                   const void* win0, long long ldw, void* wa, void* wb, void* P, long long ldp, double* dots,
                   const std::vector<double>& beta, const std::vector<double>& d, int kernel, int threads_target,
                   int rpt, cudaStream_t s, const StopState& stop = StopState{}, void* store = nullptr,
                   int store_stride = 1) {
    const int m = (int)d.size() - 1;
    // with store and store_stride 1, W_1 .. W_m are written to m consecutive n x ldw blocks there
    // instead of the ping-pong pair; with store_stride s > 1, W_s, W_2s, ..., W_{(ceil(m/s)-1)s}
    // (the backward's checkpoints) go there and the others to the ping-pong pair
    const size_t sblk = (size_t)n * ldw * elem_size(w_type_of(precision));
    char* const sb = static_cast<char*>(store);
    // banded matrices: several steps per launch (the stopping rule runs on the one-step kernels;
    // a stored pass needs every W_j in memory)
    if (stop.tol <= 0.0 && !store && (mode == MODE_ACCUM || mode == MODE_DOT) && h->band_ok && m > 0 &&
        (kernel == LL_KERNEL_AUTO || kernel == LL_KERNEL_BAND)) {
        BandLaunch BL;
        if (plan_band(precision, mode, n, b, h->sm_count, BL))
            return run_band_pass(h, A, vals_prep, precision, mode, n, b, BL, win0, ldw, wa, wb, P, ldp, dots, beta, d, s);
    }
    if (kernel == LL_KERNEL_BAND) kernel = LL_KERNEL_AUTO;
    StepParams p{};
    p.rowptr = A->rowptr;
    p.colind = A->colind;
    p.vals = vals_prep;
    p.ldw = ldw;
    p.ldv = ldw;
    p.ldp = ldp;
    p.p = P;
    p.hub_bytes = h->hub_bytes;
    const bool adaptive = stop.tol > 0.0;
    if (mode == MODE_DOT || adaptive) {
        WS(ticket, unsigned int*, "dot_ticket", sizeof(unsigned int));
        LL_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
        p.ticket = ticket;
    }
    if (mode == MODE_DOT) p.v = win0;
    {
        WS(err, int*, "tma_error", sizeof(int));
        LL_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    }
    // a representative non-first step for the autotuner (the pass overwrites what it writes)
    const int jt = m > 1 ? 1 : 0;
    p.win = win0;
    p.wout = wa;
    p.first = 0;
    p.beta = beta[jt];
    p.d0 = d[0];
    p.dn = d[jt + 1];
    p.beta_df = df_split(beta[jt]);
    p.d0_df = df_split(d[0]);
    p.dn_df = df_split(d[jt + 1]);
    if (mode == MODE_DOT) {
        p.dots_next = dots + (size_t)(jt + 1) * b;
        p.dots_first = dots;
    }
    StepExec E;
    ll_status st = choose_exec(h, precision, mode, n, A->nnz, b, kernel, threads_target, rpt, p, E, s);
    if (st != LL_OK) return st;
    int run_mode = mode;
    if (adaptive) {
        // the same kernel and shape in the STOP variant (the gather kernel when a TMA plan of it
        // does not fit), then the column state from W_0
        run_mode = mode | MODE_STOP;
        StepExec ES;
        if (!plan_exec(h, E.kind, precision, run_mode, n, A->nnz, b, E.threads, E.rpt, p, ES))
            plan_exec(h, LL_KERNEL_GATHER, precision, run_mode, n, A->nnz, b, 0, 0, p, ES);
        if ((st = bind_exec(h, precision, run_mode, b, ES, p, s)) != LL_OK) return st;
        E = ES;
        p.live = stop.live;
        p.stop_deg = stop.stop_deg;
        p.done = stop.done;
        p.tol = stop.tol;
        WS(ipart, double*, "stop_init_partials", (size_t)STOP_INIT_GRID * b * sizeof(double));
        LL_CK(launch_stop_init(precision, win0, ldw, n, b, d[0], stop.tol, m, ipart, p.ticket, stop.live,
                               stop.stop_deg, stop.done, s));
        h->launches++;
    }
    h->last_kernel = E.kind;
    h->last_threads = E.cta();
    h->last_np = E.kind == LL_KERNEL_TMA ? E.tl.np : 1;
    h->last_rows = E.kind == LL_KERNEL_TMA ? E.tl.q.R : p.rl * p.rpt;
    const int nslot = store_stride > 1 ? (m + store_stride - 1) / store_stride - 1 : m;
    const void* cur = win0;
    for (int j = 0; j < m; ++j) {
        if (sb) {
            const int k = j + 1;   // this step writes W_k
            void* out;
            if (store_stride <= 1) out = sb + (size_t)j * sblk;
            else if (k % store_stride == 0 && k / store_stride <= nslot) out = sb + (size_t)(k / store_stride - 1) * sblk;
            else out = (cur == wa) ? wb : wa;
            p.win = cur;
            p.wout = out;
            cur = out;
        } else {
            p.win = (j == 0) ? win0 : ((j & 1) ? wa : wb);
            p.wout = (j & 1) ? wb : wa;
        }
        p.first = (j == 0);
        p.beta = beta[j];
        p.d0 = d[0];
        p.dn = d[j + 1];
        p.beta_df = df_split(beta[j]);
        p.d0_df = df_split(d[0]);
        p.dn_df = df_split(d[j + 1]);
        if (mode == MODE_DOT) {
            p.dots_next = dots + (size_t)(j + 1) * b;
            p.dots_first = dots;
        }
        p.jnext = j + 1;
        LL_CK(exec_step(h, precision, run_mode, E, p, s));
    }
    return LL_OK;
}

// Adds grad_output * d/da_e sum_j d_j <U_w, W_j> to grad_values for the kept forward's coefficients,
// with W_0 = W0 and U_w = coef(col) U (coef = cq for col < split, 1 / gdiv otherwise); W0 and U are
// n x b blocks of the W storage type with leading dimension l. Reverse recurrence of the adjoint,
// Lambda_m = d_m U_w, Lambda_j = (B - xi_j I) Lambda_{j+1} + d_j U_w (B symmetric); vprep holds the
// values prepared for B, rowidx the row of every stored entry. The W_j come from the workspace
// block ckpt_name: with stored, it already holds W_1 .. W_m (the forward's trace pass wrote
// them) and no forward step runs here; otherwise they are recomputed from checkpoints kept there
// every ckpt_stride (default ceil(sqrt(m))) steps.
ll_status adjoint_accumulate(ll_handle* h, const ll_csr* A, const void* vprep, const int32_t* rowidx, const int32_t* tmap,
                             const void* W0, const void* U, long long l, int b, int split, double cq, double gdiv,
                             double grad_output, double* grad_values, cudaStream_t s, const char* ckpt_name,
                             int stored_stride) {
    const bool stored = stored_stride > 0;   // the forward wrote the checkpoints at this stride
    const int n = (int)A->n;
    const int prec = h->kept_prec, m = h->kept_m;
    const int wt = w_type_of(prec);
    const size_t ew = elem_size(wt), blk = (size_t)n * l * ew;
    const double sigma = h->kept_sigma, c = h->kept_c, gamma = h->kept_gamma;
    const std::vector<double>& d = h->kept_d;
    std::vector<double> beta(m + 1);
    for (int j = 0; j <= m; ++j) beta[j] = -(c / gamma + h->kept_xi[j]);
    // checkpoints W_{k s} (k >= 1) and a segment buffer for W_{j0+1} .. W_{j1-1}
    const int sck = stored ? stored_stride : h->kept_ckpt > 0 ? h->kept_ckpt : (int)std::ceil(std::sqrt((double)m));
    const int nseg = (m + sck - 1) / sck;
    WS(ckpt, char*, ckpt_name, blk * (size_t)(nseg > 1 ? nseg - 1 : 1));
    WS(lam, char*, "bw_lam", 2 * blk);
    char* seg = nullptr;
    char* tmp = nullptr;
    if (sck > 1) {
        WS(seg_, char*, "bw_seg", blk * (size_t)(sck - 1));
        seg = seg_;
    }
    if (!stored) {
        WS(tmp_, char*, "bw_tmp", 2 * blk);
        tmp = tmp_;
    }

    StepParams pp{};
    pp.rowptr = A->rowptr;
    pp.colind = A->colind;
    pp.vals = vprep;
    pp.ldw = l;
    pp.ldv = l;
    pp.ldp = l;
    pp.v = U;
    pp.adj_split = split;
    {
        WS(err, int*, "tma_error", sizeof(int));
        LL_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    }
    StepParams pa = pp;
    // representative steps for the autotuner: W_1 from W_0 into the segment buffer, and one
    // reverse step between the two Lambda buffers (both rewritten below)
    pp.win = W0;
    pp.wout = tmp;
    pp.beta = beta[0];
    pp.beta_df = df_split(beta[0]);
    pa.win = lam;
    pa.wout = lam + blk;
    pa.beta = beta[0];
    pa.beta_df = df_split(beta[0]);
    pa.adj_q = d[0] * cq;
    pa.adj_g = d[0] / gdiv;
    pa.adj_q_df = df_split(d[0] * cq);
    pa.adj_g_df = df_split(d[0] / gdiv);
    StepExec Ep, Ea;
    ll_status cs = LL_OK;
    if (!stored || sck > 1) {
        if (!tmp) pp.wout = seg;   // the autotuner's representative step (rewritten below)
        cs = choose_exec(h, prec, MODE_PLAIN, n, A->nnz, b, h->cfg_kernel, h->cfg_threads, h->cfg_rpt, pp, Ep, s);
    }
    if (cs != LL_OK) return cs;
    cs = choose_exec(h, prec, MODE_ADJ, n, A->nnz, b, h->cfg_kernel, h->cfg_threads, h->cfg_rpt, pa, Ea, s);
    if (cs != LL_OK) return cs;
    const double scale = grad_output / (sigma * gamma);
    // the reverse step fused with the gradient contraction (TMA kernel, one column pair per
    // thread, the shape the autotuner chose for the plain reverse step): no separate SDDMM. The
    // step accumulates each entry's term in transposed order (gt[e] holds the term of entry
    // tmap[e]), mapped into grad_values after the last step.
    StepParams pg = pa;
    StepExec Eg;
    bool fused = false;
    double* gt = nullptr;
    if (h->fuse_mode != LL_FUSE_OFF && tmap && Ea.kind == LL_KERNEL_TMA && Ea.tl.np == 1) {
        WS(gtw, double*, "bw_gt", (size_t)A->nnz * sizeof(double));
        gt = gtw;
        pg.wj = W0;
        pg.grad = gt;
        pg.gscale = scale;
        if (plan_exec(h, LL_KERNEL_TMA, prec, MODE_ADJ_GRAD, n, A->nnz, b, Ea.threads, 0, pg, Eg)) {
            if ((cs = bind_exec(h, prec, MODE_ADJ_GRAD, b, Eg, pg, s)) != LL_OK) return cs;
            fused = true;
            // the fused step against the reverse step followed by the separate contraction, both
            // timed once per shape on the representative operands (Lambda buffers rewritten below,
            // gt cleared after) and the faster cached: fusing gains where rows are long (13-point
            // stencil) and can lose where they are short and the step is cheap
            const auto key = std::make_tuple(prec, n, (long long)A->nnz, b, l);
            auto it = h->adj_fuse_choice.find(key);
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            LL_CK(cudaStreamIsCapturing(s, &cap));
            if (h->fuse_mode == LL_FUSE_ON) {
                fused = true;
            } else if (it != h->adj_fuse_choice.end()) {
                fused = it->second != 0;
            } else if (cap == cudaStreamCaptureStatusNone) {
                float ms[2] = {0.f, 0.f};
                const int counted = h->launches;   // the timing runs are not the call's launches
                // each form once untimed (a kernel's first launch may also load its module), then timed
                for (int rep = 0; rep < 2; ++rep) {
                    for (int v = 0; v < 2; ++v) {
                        LL_CK(cudaEventRecord(h->ev[6], s));
                        if (v == 0) {
                            LL_CK(exec_step(h, prec, MODE_ADJ_GRAD, Eg, pg, s));
                        } else {
                            LL_CK(exec_step(h, prec, MODE_ADJ, Ea, pa, s));
                            LL_CK(launch_sddmm(prec, rowidx, A->colind, A->nnz, lam, W0, l, b, scale, gt, s));
                        }
                        LL_CK(cudaEventRecord(h->ev[7], s));
                        LL_CK(cudaEventSynchronize(h->ev[7]));
                        LL_CK(cudaEventElapsedTime(&ms[v], h->ev[6], h->ev[7]));
                    }
                }
                h->launches = counted;
                fused = ms[0] < ms[1];
                h->adj_fuse_choice[key] = fused ? 1 : 0;
            }
            if (fused) LL_CK(cudaMemsetAsync(gt, 0, (size_t)A->nnz * sizeof(double), s));
        }
    }
    auto plain_step = [&](int j, const void* win, void* wout) -> cudaError_t {
        pp.win = win;
        pp.wout = wout;
        pp.beta = beta[j];
        pp.beta_df = df_split(beta[j]);
        return exec_step(h, prec, MODE_PLAIN, Ep, pp, s);
    };
    // phase A: W_1 .. W_{(nseg-1) sck}, keeping W_{k sck} in the checkpoint slots (stored: there)
    const void* cur = W0;
    for (int j = 0; !stored && j < (nseg - 1) * sck; ++j) {
        void* out = ((j + 1) % sck == 0) ? (void*)(ckpt + (size_t)((j + 1) / sck - 1) * blk)
                                         : (void*)(tmp + (cur == tmp ? blk : 0));
        LL_CK(plain_step(j, cur, out));
        cur = out;
    }
    // phase B: Lambda_m = d_m U, then segments in reverse
    char* lam_cur = lam;
    LL_CK(launch_scale_cols(prec, U, l, n, b, split, d[m] * cq, d[m] / gdiv, lam_cur, s));
    h->launches++;
    for (int kk = nseg - 1; kk >= 0; --kk) {
        const int j0 = kk * sck, j1 = std::min(j0 + sck, m);
        const void* wj0 = kk == 0 ? W0 : (const void*)(ckpt + (size_t)(kk - 1) * blk);
        const void* w = wj0;
        for (int t = 1; t < j1 - j0; ++t) {
            void* out = seg + (size_t)(t - 1) * blk;
            LL_CK(plain_step(j0 + t - 1, w, out));
            w = out;
        }
        for (int j = j1 - 1; j >= j0; --j) {
            const void* wj = (j == j0) ? wj0 : (const void*)(seg + (size_t)(j - j0 - 1) * blk);
            if (fused) {
                // Lambda_j and g_e += (1 / (sigma gamma)) <Lambda_{j+1}[r, :], W_j[c, :]> in one step
                // (Lambda_0, written at j = 0, is not used)
                char* lam_next = (lam_cur == lam) ? lam + blk : lam;
                pg.win = lam_cur;
                pg.wout = lam_next;
                pg.wj = wj;
                pg.beta = beta[j];
                pg.beta_df = df_split(beta[j]);
                pg.adj_q = d[j] * cq;
                pg.adj_g = d[j] / gdiv;
                pg.adj_q_df = df_split(d[j] * cq);
                pg.adj_g_df = df_split(d[j] / gdiv);
                LL_CK(exec_step(h, prec, MODE_ADJ_GRAD, Eg, pg, s));
                lam_cur = lam_next;
                continue;
            }
            // g_e += (1 / (sigma gamma)) <Lambda_{j+1}[r, :], W_j[c, :]>
            LL_CK(launch_sddmm(prec, rowidx, A->colind, A->nnz, lam_cur, wj, l, b, scale, grad_values, s));
            h->launches++;
            if (j == 0) break;
            // Lambda_j = (B - xi_j I) Lambda_{j+1} + d_j U
            char* lam_next = (lam_cur == lam) ? lam + blk : lam;
            pa.win = lam_cur;
            pa.wout = lam_next;
            pa.beta = beta[j];
            pa.beta_df = df_split(beta[j]);
            pa.adj_q = d[j] * cq;
            pa.adj_g = d[j] / gdiv;
            pa.adj_q_df = df_split(d[j] * cq);
            pa.adj_g_df = df_split(d[j] / gdiv);
            LL_CK(exec_step(h, prec, MODE_ADJ, Ea, pa, s));
            lam_cur = lam_next;
        }
    }
    if (fused) {
        LL_CK(launch_gather_add(tmap, gt, A->nnz, grad_values, s));
        h->launches++;
    }
    h->info.adjoint_fused = fused ? 1 : 0;
    LL_CK(cudaGetLastError());
    return check_tma_flag(h, s);
}


// The adjoint of the kept forward: the frozen-basis gradient, and with through_qr the derivative
// through the sketch's CholeskyQR2 as well (Algorithm 3 step 4; bounds, sigma and d fixed):
//   E = tr(F Pi) + (1/k) tr(F (I - Pi) G G^T (I - Pi)),  Pi = Q Q^T,  Y = F S = Q R,
//   dE = tr(dF [Q Q^T + G' G'^T / k]) + tr(Gamma^T dF S),  Gamma = 2 (I - Pi) Z Q R^-T,
//   Z Q = F Q - (1/k) G (G'^T F Q) - (1/k) (F G') (G^T Q).
// The second term is the same reverse recurrence with W_0 = S and U = Gamma.
ll_status backward_impl(ll_handle* h, const ll_csr* A, double grad_output, double* grad_values, void* stream,
                        bool through_qr) {
    if (!h) return LL_ERR_INVALID_ARG;
    if (!h->kept) return fail(h, LL_ERR_NO_FORWARD, "no kept forward (call ll_logdet_forward with keep_for_backward = 1)");
    ll_status st = check_csr_args(h, A);
    if (st != LL_OK) return st;
    if (A->n != h->kept_n || A->nnz != h->kept_nnz) return fail(h, LL_ERR_INVALID_ARG, "matrix shape differs from the kept forward");
    if (A->nnz > 0 && !grad_values) return fail(h, LL_ERR_INVALID_ARG, "null grad_values");
    cudaStream_t s = (cudaStream_t)stream;
    h->launches = 0;
    const int n = (int)A->n;
    const int prec = h->kept_prec, kq = h->kept_kq, kg = h->kept_kg, m = h->kept_m;
    const int b2 = kq + kg, l2 = block_ld(prec, b2);
    const int wt = w_type_of(prec);
    const size_t ew = elem_size(wt), blk = (size_t)n * l2 * ew;
    if (n == 0 || A->nnz == 0) {
        if (A->nnz > 0) LL_CK(cudaMemsetAsync(grad_values, 0, (size_t)A->nnz * sizeof(double), s));
        return LL_OK;
    }
    {
        // the reverse recurrence uses B^T = B: refuse a matrix that is not symmetric
        WS(sflag, int*, "bw_sym_flag", sizeof(int));
        LL_CK(cudaMemsetAsync(sflag, 0, sizeof(int), s));
        LL_CK(launch_check_symmetric(A->rowptr, A->colind, A->values, A->dtype, n, h->kept_sorted ? 1 : 0, sflag, s));
        h->launches++;
        int hs = 0;
        LL_CK(cudaMemcpyAsync(&hs, sflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        LL_CK(cudaStreamSynchronize(s));
        if (hs) return fail(h, LL_ERR_INVALID_ARG, "A is not symmetric (the adjoint uses A^T = A)");
    }
    // the transposed-entry map of the fused adjoint step (rows with strictly increasing columns)
    const int32_t* tmap = nullptr;
    if (h->kept_sorted && A->nnz > 0) {
        WS(tm, int32_t*, "bw_tmap", (size_t)A->nnz * sizeof(int32_t));
        WS(tflag, int*, "bw_tmap_flag", sizeof(int));
        LL_CK(cudaMemsetAsync(tflag, 0, sizeof(int), s));
        LL_CK(launch_transpose_map(A->rowptr, A->colind, n, tm, tflag, s));
        h->launches++;
        int ht = 0;
        LL_CK(cudaMemcpyAsync(&ht, tflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        LL_CK(cudaStreamSynchronize(s));
        if (!ht) tmap = tm;
    }
    LL_CK(cudaMemsetAsync(grad_values, 0, (size_t)A->nnz * sizeof(double), s));
    auto it_v = h->ws.find(wt == T_F64 ? "fw_basis" : "fw_V");
    if (it_v == h->ws.end()) return fail(h, LL_ERR_NO_FORWARD, "kept basis missing");
    const void* V = it_v->second.p;
    const double sigma = h->kept_sigma, c = h->kept_c, gamma = h->kept_gamma;
    // the step plans below describe the kept forward's matrix (it is not revalidated here)
    h->band_ok = h->kept_band;
    h->far_entries = h->kept_far;
    h->far_runs = h->kept_runs;
    h->max_row = h->kept_max_row;
    WS(vprep, void*, "bw_vals", (size_t)A->nnz * ew);
    LL_CK(launch_prepare_values(A->values, A->dtype, A->nnz, 1.0 / (sigma * gamma), prec, vprep, s));
    h->launches++;
    // row of every stored entry, for the gradient contraction
    WS(rowidx, int32_t*, "bw_rowidx", (size_t)A->nnz * sizeof(int32_t));
    LL_CK(launch_row_index(A->rowptr, n, rowidx, s));
    h->launches++;
    // frozen basis: W_0 = [Q | G'], U = [Q | G' / k]
    st = adjoint_accumulate(h, A, vprep, rowidx, tmap, V, V, l2, b2, kq, 1.0, (double)kg, grad_output, grad_values, s,
                            "bw_ckpt", h->kept_stride);
    if (st != LL_OK || !through_qr || !h->kept_qr) return st;

    // ---- through the QR: F [Q | G'] by the pass-1 arithmetic on the kept block
    auto kept_buf = [&](const char* name) -> void* {
        auto it = h->ws.find(name);
        return it == h->ws.end() ? nullptr : it->second.p;
    };
    void* S = kept_buf("fw_S");
    const double* Gb = static_cast<const double*>(kept_buf("fw_G"));
    const double* basis = static_cast<const double*>(kept_buf("fw_basis"));
    if (prec != LL_PREC_F64) {
        // the DF64 forward keeps [Q | G'] as double-float column pairs in V, the FP32-mixed one in
        // the basis block
        WS(b64, double*, "bw_basis64", (size_t)n * l2 * sizeof(double));
        LL_CK(launch_block_to_f64(prec, prec == LL_PREC_DF64 ? V : static_cast<const void*>(basis), l2, b64, l2, n, b2, s));
        h->launches++;
        basis = b64;
    }
    const double* rinv1 = static_cast<const double*>(kept_buf("fw_rinv1"));
    const double* rinv2 = static_cast<const double*>(kept_buf("fw_rinv"));
    if (!S || !Gb || !basis || !rinv1 || !rinv2) return fail(h, LL_ERR_NO_FORWARD, "kept sketch missing");
    const int l1 = block_ld(prec, kq);
    const size_t ep = elem_size(p_type_of(prec));
    std::vector<double> beta(m + 1);
    for (int j = 0; j <= m; ++j) beta[j] = -(c / gamma + h->kept_xi[j]);
    WS(FV, void*, "bw_FV", (size_t)n * l2 * ep);
    WS(FV64, double*, "bw_FV64", (size_t)n * b2 * sizeof(double));
    void* wk = h->kept_stride == 1 ? kept_buf("bw_ckpt") : nullptr;
    if (wk) {
        // the trace pass kept W_1 .. W_m of W_0 = [Q | G']: F [Q | G'] = sum_j d_j W_j, the same
        // numbers as the P-axpy sweep below
        std::vector<float2> ddf(m + 1);
        for (int j = 0; j <= m; ++j) ddf[j] = df_split(h->kept_d[j]);
        WS(dco, double*, "bw_dcoef", (size_t)(m + 1) * sizeof(double));
        WS(dcf, float2*, "bw_dcoef_df", (size_t)(m + 1) * sizeof(float2));
        LL_CK(cudaMemcpyAsync(dco, h->kept_d.data(), (size_t)(m + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
        LL_CK(cudaMemcpyAsync(dcf, ddf.data(), (size_t)(m + 1) * sizeof(float2), cudaMemcpyHostToDevice, s));
        LL_CK(cudaStreamSynchronize(s));   // the host vectors go out of scope
        LL_CK(launch_weighted_sum(prec, V, wk, blk, l2, n, b2, m, dco, dcf, FV, l2, s));
        h->launches++;
    } else {
        WS(scratch, char*, "bw_tmp", 2 * blk);
        st = run_pass(h, A, vprep, prec, MODE_ACCUM, n, b2, V, l2, scratch, scratch + blk, FV, l2, nullptr, beta, h->kept_d,
                      h->cfg_kernel, h->cfg_threads, h->cfg_rpt, s);
        if (st != LL_OK) return st;
    }
    LL_CK(launch_block_to_f64(prec, FV, l2, FV64, b2, n, b2, s));
    h->launches++;

    // ---- Gamma = 2 (I - Pi) Z Q R^-T (tall-skinny FP64 products)
    const int ggrid = h->sm_count * 2;
    const size_t gpn = gram_partials_any(h, kg > kq ? kg : kq, kq, false, ggrid);
    h->gram_method = h->kept_gram;
    WS(gpart, double*, "bw_gram_partials", gpn * sizeof(double));
    WS(gticket, unsigned int*, "bw_gram_ticket", sizeof(unsigned int));
    WS(small, double*, "bw_small", (size_t)5 * (kg > kq ? kg : kq) * kq * sizeof(double));
    double* C1 = small;                              // G'^T F Q / k   (kg x kq)
    double* C2 = small + (size_t)kg * kq;            // G^T Q / k      (kg x kq)
    double* C3 = small + (size_t)2 * kg * kq;        // Q^T Z Q        (kq x kq)
    double* Mt = C3 + (size_t)kq * kq;               // 2 R^-T         (kq x kq)
    WS(zq, double*, "bw_zq", (size_t)3 * n * kq * sizeof(double));
    double* ZQa = zq;
    double* ZQ = zq + (size_t)n * kq;
    double* Xb = zq + (size_t)2 * n * kq;
    LL_CK(cudaMemsetAsync(gticket, 0, sizeof(unsigned int), s));
    if ((st = run_gram(h, T_F64, basis + kq, l2, kg, FV64, b2, kq, n, false, gpart, gticket, C1, ggrid, s)) != LL_OK) return st;
    if ((st = run_gram(h, T_F64, Gb, kg, kg, basis, l2, kq, n, false, gpart, gticket, C2, ggrid, s)) != LL_OK) return st;
    LL_CK(launch_scaled_copy_f64(C1, kq, C1, kq, 2 * kg, kq, 1.0 / kg, s));
    LL_CK(launch_project(T_F64, Gb, kg, kg, FV64, b2, kq, C1, n, ZQa, kq, T_F64, nullptr, 0, 0, 0, s));
    LL_CK(launch_project(T_F64, FV64 + kq, b2, kg, ZQa, kq, kq, C2, n, ZQ, kq, T_F64, nullptr, 0, 0, 0, s));
    if ((st = run_gram(h, T_F64, basis, l2, kq, ZQ, kq, kq, n, false, gpart, gticket, C3, ggrid, s)) != LL_OK) return st;
    LL_CK(launch_project(T_F64, basis, l2, kq, ZQ, kq, kq, C3, n, Xb, kq, T_F64, nullptr, 0, 0, 0, s));
    h->launches += 4;   // (run_gram counts its own)
    // R^-1 = R1^-1 R2^-1 (Y R1^-1 = Q1, Q1 R2^-1 = Q), and M = 2 R^-T, on the host (kq x kq)
    std::vector<double> r1((size_t)kq * kq), r2((size_t)kq * kq), mt((size_t)kq * kq, 0.0);
    LL_CK(cudaMemcpyAsync(r1.data(), rinv1, r1.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaMemcpyAsync(r2.data(), rinv2, r2.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    for (int a = 0; a < kq; ++a)
        for (int b = 0; b < kq; ++b) {
            double t = 0.0;
            for (int x = 0; x < kq; ++x) t += r1[(size_t)a * kq + x] * r2[(size_t)x * kq + b];
            mt[(size_t)b * kq + a] = 2.0 * t;   // (R^-1)^T
        }
    LL_CK(cudaMemcpyAsync(Mt, mt.data(), mt.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    WS(gam, void*, "bw_gamma", (size_t)n * l1 * ew);
    WS(gam64, double*, "bw_gamma64", (size_t)n * kq * sizeof(double));
    LL_CK(cudaMemsetAsync(gam, 0, (size_t)n * l1 * ew, s));
    LL_CK(launch_mul_small(Xb, kq, n, kq, kq, Mt, gam64, kq, wt, gam, l1, s));
    h->launches++;
    LL_CK(cudaStreamSynchronize(s));   // the host copy of mt stays alive until the upload is done

    // ---- the QR term: W_0 = S, U = Gamma
    // pass 1's W_j as the forward kept them, or checkpoints in a block of their own, so that the
    // trace pass's kept W_j stay valid for the next backward
    return adjoint_accumulate(h, A, vprep, rowidx, tmap, S, gam, l1, kq, kq, 1.0, 1.0, grad_output, grad_values, s,
                              h->kept_stride > 0 ? "bw_ckpt_s" : "bw_ckpt", h->kept_wall_s ? 1 : 0);
}


}  // namespace
}  // namespace ll

using namespace ll;

extern "C" {

ll_status ll_create(ll_handle** out) {
    if (!out) return LL_ERR_INVALID_ARG;
    ll_handle* h = new ll_handle();
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LL_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    for (auto& e : h->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return LL_ERR_CUDA;
        }
    }
    *out = h;
    return LL_OK;
}

void ll_destroy(ll_handle* h) {
    if (!h) return;
    for (auto& kv : h->ws)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->gfwd.exec) cudaGraphExecDestroy(h->gfwd.exec);
    if (h->gbat.exec) cudaGraphExecDestroy(h->gbat.exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

const char* ll_status_string(ll_status s) {
    switch (s) {
        case LL_OK: return "LL_OK";
        case LL_ERR_INVALID_ARG: return "LL_ERR_INVALID_ARG";
        case LL_ERR_BAD_CSR: return "LL_ERR_BAD_CSR";
        case LL_ERR_BAD_BOUNDS: return "LL_ERR_BAD_BOUNDS";
        case LL_ERR_DD_NOT_CONVERGED: return "LL_ERR_DD_NOT_CONVERGED";
        case LL_ERR_QR_BREAKDOWN: return "LL_ERR_QR_BREAKDOWN";
        case LL_ERR_NONFINITE: return "LL_ERR_NONFINITE";
        case LL_ERR_TIMEOUT: return "LL_ERR_TIMEOUT";
        case LL_ERR_OOM: return "LL_ERR_OOM";
        case LL_ERR_CUDA: return "LL_ERR_CUDA";
        case LL_ERR_UNSUPPORTED: return "LL_ERR_UNSUPPORTED";
        case LL_ERR_NO_FORWARD: return "LL_ERR_NO_FORWARD";
    }
    return "LL_ERR_UNKNOWN";
}

const char* ll_last_error(const ll_handle* h) { return h ? h->err.c_str() : ""; }

void ll_default_options(ll_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->degree = 40;
    o->probes = 30;
    o->seed = 0;
    o->probe_kind = LL_PROBE_RADEMACHER;
    o->precision = LL_PREC_DF64;
    o->sval_mode = LL_SVAL_CENTER;
    o->dd_scheme = LL_DD_AUTO;
    o->keep_for_backward = 0;
    o->rows_per_thread = 0;
    o->threads_per_block = 0;
    o->ckpt_stride = 0;
    o->use_graph = 1;
    o->timeout_cycles = 0;
    o->step_kernel = LL_KERNEL_AUTO;
    o->estimator = LL_EST_HUTCHPP;
    o->tol = 0.0;
    o->qr_gram = LL_GRAM_AUTO;
}

ll_status ll_debug_inject(ll_handle* h, int what) {
    if (!h || what < LL_INJECT_NONE || what > LL_INJECT_STALL) return LL_ERR_INVALID_ARG;
    h->inject = what;
    return LL_OK;
}

ll_status ll_set_adjoint_fusion(ll_handle* h, int mode) {
    if (!h) return LL_ERR_INVALID_ARG;
    if (mode != LL_FUSE_AUTO && mode != LL_FUSE_ON && mode != LL_FUSE_OFF)
        return fail(h, LL_ERR_INVALID_ARG, "unknown adjoint fusion mode");
    h->fuse_mode = mode;
    return LL_OK;
}

ll_status ll_set_keep_budget(ll_handle* h, int64_t bytes) {
    if (!h) return LL_ERR_INVALID_ARG;
    if (bytes < 0) return fail(h, LL_ERR_INVALID_ARG, "negative keep budget");
    h->keep_budget = bytes;
    return LL_OK;
}

ll_status ll_trim_workspace(ll_handle* h) {
    if (!h) return LL_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(h, LL_ERR_CUDA, std::string("cudaDeviceSynchronize: ") + cudaGetErrorString(e));
    for (auto& kv : h->ws)
        if (kv.second.p) cudaFree(kv.second.p);
    h->ws.clear();
    h->ws_gen++;
    if (h->gfwd.exec) cudaGraphExecDestroy(h->gfwd.exec);
    h->gfwd.exec = nullptr;
    h->gfwd.key.clear();
    if (h->gbat.exec) cudaGraphExecDestroy(h->gbat.exec);
    h->gbat.exec = nullptr;
    h->gbat.key.clear();
    h->ro = ll_handle::Reorder{};
    h->kept = false;
    h->have_forward = false;
    return LL_OK;
}

ll_status ll_set_step_config(ll_handle* h, int step_kernel, int threads_per_block, int rows_per_thread) {
    if (!h || step_kernel < LL_KERNEL_AUTO || step_kernel > LL_KERNEL_BAND || threads_per_block < 0 || rows_per_thread < 0)
        return LL_ERR_INVALID_ARG;
    h->cfg_kernel = step_kernel;
    h->cfg_threads = threads_per_block;
    h->cfg_rpt = rows_per_thread;
    return LL_OK;
}

ll_status ll_leja_points(int count, double* xi_out) {
    if (count < 0 || (count > 0 && !xi_out)) return LL_ERR_INVALID_ARG;
    if (count > 100000) return LL_ERR_UNSUPPORTED;
    leja_points(count, xi_out);
    return LL_OK;
}

ll_status ll_divided_differences(ll_bounds b, int degree, int sval_mode, double* d_out, int* terms_out) {
    if (degree < 0 || !d_out) return LL_ERR_INVALID_ARG;
    if (sval_mode != LL_SVAL_CENTER && sval_mode != LL_SVAL_HALF_LMAX) return LL_ERR_INVALID_ARG;
    if (!std::isfinite(b.lmin) || !std::isfinite(b.lmax) || !(b.lmin > 0.0) || !(b.lmin < b.lmax)) return LL_ERR_BAD_BOUNDS;
    const int terms = scaled_divided_differences(b.lmin, b.lmax, degree, sval_mode, d_out);
    if (terms < 0) return LL_ERR_DD_NOT_CONVERGED;
    if (terms_out) *terms_out = terms;
    return LL_OK;
}

ll_status ll_divided_differences_q(ll_bounds b, int degree, double* d_out) {
    if (degree < 0 || !d_out) return LL_ERR_INVALID_ARG;
    if (degree > 100000) return LL_ERR_UNSUPPORTED;
    if (!std::isfinite(b.lmin) || !std::isfinite(b.lmax) || !(b.lmin > 0.0) || !(b.lmin < b.lmax)) return LL_ERR_BAD_BOUNDS;
    divided_differences_table_q(b.lmin, b.lmax, degree, d_out);
    return LL_OK;
}

ll_status ll_gershgorin(ll_handle* h, const ll_csr* A, ll_bounds* out, void* stream) {
    if (!h || !out) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, A);
    if (st != LL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (A->n == 0) return fail(h, LL_ERR_INVALID_ARG, "empty matrix has no spectrum");
    st = validate_csr(h, A, s);
    if (st != LL_OK) return st;
    const int grid = h->sm_count * 4;
    WS(partials, double*, "gg_partials", (size_t)2 * grid * sizeof(double));
    WS(ticket, unsigned int*, "gg_ticket", sizeof(unsigned int));
    WS(res, double*, "gg_out", 2 * sizeof(double));
    LL_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
    LL_CK(launch_gershgorin(A->rowptr, A->colind, A->values, A->dtype, (int)A->n, partials, ticket, res, grid, s));
    h->launches++;
    double hres[2];
    LL_CK(cudaMemcpyAsync(hres, res, sizeof hres, cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    out->lmin = hres[0];
    out->lmax = hres[1];
    return LL_OK;
}

ll_status ll_power_lmax(ll_handle* h, const ll_csr* A, int iters, uint64_t seed, double* lmax_out, void* stream) {
    if (!h || !lmax_out || iters < 0) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, A);
    if (st != LL_OK) return st;
    if (A->n == 0) return fail(h, LL_ERR_INVALID_ARG, "empty matrix has no spectrum");
    cudaStream_t s = (cudaStream_t)stream;
    st = validate_csr(h, A, s);
    if (st != LL_OK) return st;
    const int n = (int)A->n;
    const int grid = h->sm_count * 4;
    WS(x, double*, "pw_x", (size_t)n * sizeof(double));
    WS(y, double*, "pw_y", (size_t)n * sizeof(double));
    WS(partials, double*, "pw_partials", (size_t)grid * sizeof(double));
    WS(ticket, unsigned int*, "pw_ticket", sizeof(unsigned int));
    WS(nrm, double*, "pw_nrm", sizeof(double));
    LL_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
    LL_CK(launch_probes(T_F64, LL_PROBE_RADEMACHER, seed, LL_STREAM_POWER, n, 1, 1, x, 1, s));
    LL_CK(launch_dot_f64(x, x, n, partials, ticket, nrm, grid, s));
    LL_CK(launch_scale_f64(x, nrm, n, 0, s));
    h->launches += 3;
    for (int it = 0; it < iters; ++it) {
        LL_CK(launch_spmv_f64(A->rowptr, A->colind, A->values, A->dtype, n, x, y, s));
        LL_CK(launch_dot_f64(y, y, n, partials, ticket, nrm, grid, s));
        LL_CK(launch_scale_f64(y, nrm, n, 0, s));
        h->launches += 3;
        double* t = x; x = y; y = t;
    }
    LL_CK(launch_spmv_f64(A->rowptr, A->colind, A->values, A->dtype, n, x, y, s));
    LL_CK(launch_dot_f64(x, y, n, partials, ticket, nrm, grid, s));
    h->launches += 2;
    double hn = 0;
    LL_CK(cudaMemcpyAsync(&hn, nrm, sizeof hn, cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    *lmax_out = hn;
    return LL_OK;
}

ll_status ll_probes(ll_handle* h, int kind, uint64_t seed, int stream_id, int64_t n, int cols, double* out,
                    int64_t ld, void* stream) {
    if (!h) return LL_ERR_INVALID_ARG;
    if (kind != LL_PROBE_RADEMACHER && kind != LL_PROBE_GAUSSIAN) return fail(h, LL_ERR_INVALID_ARG, "unknown probe kind");
    if (n < 0 || cols < 0 || ld < cols || stream_id < 0 || stream_id > 255) return fail(h, LL_ERR_INVALID_ARG, "bad probe shape");
    if (n >= ((int64_t)1 << 31) || cols >= (1 << 24)) return fail(h, LL_ERR_UNSUPPORTED, "probe block too large");
    if (n * cols == 0) return LL_OK;
    if (!out) return fail(h, LL_ERR_INVALID_ARG, "null output");
    LL_CK(launch_probes(T_F64, kind, seed, stream_id, (int)n, cols, cols, out, ld, (cudaStream_t)stream));
    h->launches++;
    return LL_OK;
}

ll_status ll_apply_poly(ll_handle* h, const ll_csr* A, ll_bounds bounds, int degree, int precision, const double* V,
                        int64_t ldv, int b, double* PV, int64_t ldp, void* stream) {
    if (!h) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, A);
    if (st != LL_OK) return st;
    if ((st = check_bounds(h, bounds)) != LL_OK) return st;
    if (degree < 0 || b < 0 || ldv < b || ldp < b) return fail(h, LL_ERR_INVALID_ARG, "bad degree or block shape");
    if (precision < LL_PREC_F64 || precision > LL_PREC_F32_MIXED) return fail(h, LL_ERR_INVALID_ARG, "unknown precision");
    const int n = (int)A->n;
    if (n == 0 || b == 0) return LL_OK;
    if (b > 512) return fail(h, LL_ERR_UNSUPPORTED, "block width above 512");
    if (!V || !PV) return fail(h, LL_ERR_INVALID_ARG, "null block");
    cudaStream_t s = (cudaStream_t)stream;
    h->launches = 0;
    if ((st = validate_csr(h, A, s)) != LL_OK) return st;
    std::vector<double> xi, d;
    if ((st = setup_coefficients(h, bounds.lmin, bounds.lmax, degree, LL_SVAL_CENTER, xi, d)) != LL_OK) return st;
    const double c = (bounds.lmin + bounds.lmax) / 2.0, gamma = (bounds.lmax - bounds.lmin) / 4.0;
    std::vector<double> beta(degree + 1);
    for (int j = 0; j <= degree; ++j) beta[j] = -(c / gamma + xi[j]);
    const int wt = w_type_of(precision), pt = p_type_of(precision);
    const int lb = block_ld(precision, b);     // blocks are stored in column pairs
    const size_t nb = (size_t)n * lb;
    WS(vprep, void*, "ap_vals", (size_t)A->nnz * elem_size(wt));
    WS(w0, void*, "ap_w0", nb * elem_size(wt));
    WS(wa, void*, "ap_wa", nb * elem_size(wt));
    WS(wb, void*, "ap_wb", nb * elem_size(wt));
    WS(pp, void*, "ap_p", nb * elem_size(pt));
    LL_CK(launch_prepare_values(A->values, A->dtype, A->nnz, 1.0 / gamma, precision, vprep, s));
    LL_CK(launch_convert_block(V, ldv, precision, w0, lb, n, b, lb, s));
    h->launches += 2;
    if (degree == 0) {
        // p_0 = d_0: PV = d_0 V
        LL_CK(launch_scaled_copy_f64(V, ldv, PV, ldp, n, b, d[0], s));
        h->launches++;
        return LL_OK;
    }
    st = run_pass(h, A, vprep, precision, MODE_ACCUM, n, b, w0, lb, wa, wb, pp, lb, nullptr, beta, d, h->cfg_kernel,
                  h->cfg_threads, h->cfg_rpt, s);
    if (st != LL_OK) return st;
    h->info = ll_info{};
    h->info.kernel_pass1 = h->last_kernel;
    h->info.threads_pass1 = h->last_threads;
    h->info.pairs_pass1 = h->last_np;
    h->info.rows_pass1 = h->last_rows;
    LL_CK(launch_block_to_f64(precision, pp, lb, PV, ldp, n, b, s));
    h->launches++;
    return check_tma_flag(h, s);
}

ll_status ll_apply_poly_tol(ll_handle* h, const ll_csr* A, ll_bounds bounds, int degree, double tol, int precision,
                            const double* V, int64_t ldv, int b, double* PV, int64_t ldp, int* degrees_out,
                            void* stream) {
    if (!h) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, A);
    if (st != LL_OK) return st;
    if ((st = check_bounds(h, bounds)) != LL_OK) return st;
    if (degree < 1 || b < 0 || ldv < b || ldp < b) return fail(h, LL_ERR_INVALID_ARG, "bad degree or block shape");
    if (!std::isfinite(tol) || !(tol > 0.0)) return fail(h, LL_ERR_INVALID_ARG, "tol must be finite and > 0");
    if (precision < LL_PREC_F64 || precision > LL_PREC_F32_MIXED) return fail(h, LL_ERR_INVALID_ARG, "unknown precision");
    const int n = (int)A->n;
    if (n == 0 || b == 0) return LL_OK;
    if (b > 512) return fail(h, LL_ERR_UNSUPPORTED, "block width above 512");
    if (!V || !PV || !degrees_out) return fail(h, LL_ERR_INVALID_ARG, "null block or degree array");
    cudaStream_t s = (cudaStream_t)stream;
    h->launches = 0;
    if ((st = validate_csr(h, A, s)) != LL_OK) return st;
    std::vector<double> xi, d;
    if ((st = setup_coefficients(h, bounds.lmin, bounds.lmax, degree, LL_SVAL_CENTER, xi, d)) != LL_OK) return st;
    const double c = (bounds.lmin + bounds.lmax) / 2.0, gamma = (bounds.lmax - bounds.lmin) / 4.0;
    std::vector<double> beta(degree + 1);
    for (int j = 0; j <= degree; ++j) beta[j] = -(c / gamma + xi[j]);
    const int wt = w_type_of(precision), pt = p_type_of(precision);
    const int lb = block_ld(precision, b);
    const size_t nb = (size_t)n * lb;
    WS(vprep, void*, "ap_vals", (size_t)A->nnz * elem_size(wt));
    WS(w0, void*, "ap_w0", nb * elem_size(wt));
    WS(wa, void*, "ap_wa", nb * elem_size(wt));
    WS(wb, void*, "ap_wb", nb * elem_size(wt));
    WS(pp, void*, "ap_p", nb * elem_size(pt));
    WS(sst, int*, "ap_stop_state", (size_t)(2 * (b + 2) + 1) * sizeof(int));
    LL_CK(launch_prepare_values(A->values, A->dtype, A->nnz, 1.0 / gamma, precision, vprep, s));
    LL_CK(launch_convert_block(V, ldv, precision, w0, lb, n, b, lb, s));
    h->launches += 2;
    const StopState stop{tol, sst, sst + (b + 2), sst + 2 * (b + 2)};
    st = run_pass(h, A, vprep, precision, MODE_ACCUM, n, b, w0, lb, wa, wb, pp, lb, nullptr, beta, d, h->cfg_kernel,
                  h->cfg_threads, h->cfg_rpt, s, stop);
    if (st != LL_OK) return st;
    h->info = ll_info{};
    h->info.kernel_pass1 = h->last_kernel;
    h->info.threads_pass1 = h->last_threads;
    h->info.pairs_pass1 = h->last_np;
    h->info.rows_pass1 = h->last_rows;
    LL_CK(launch_block_to_f64(precision, pp, lb, PV, ldp, n, b, s));
    h->launches++;
    LL_CK(cudaMemcpyAsync(degrees_out, stop.stop_deg, (size_t)b * sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    return check_tma_flag(h, s);
}

ll_status ll_logdet_forward(ll_handle* h, const ll_csr* A0, ll_bounds bounds, const ll_options* opts, double* estimate,
                            void* stream) {
    const ll_csr* A = A0;   // the matrix the passes run on: A0, or its degree-ordered copy
    if (!h || !opts || !estimate) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, A0);
    if (st != LL_OK) return st;
    if ((st = check_bounds(h, bounds)) != LL_OK) return st;
    const ll_options& o = *opts;
    if (o.degree < 1) return fail(h, LL_ERR_INVALID_ARG, "degree must be >= 1");
    if (o.estimator != LL_EST_HUTCHPP && o.estimator != LL_EST_HUTCHINSON) return fail(h, LL_ERR_INVALID_ARG, "unknown estimator");
    const bool hutch = o.estimator == LL_EST_HUTCHINSON;   // plain Hutchinson: no sketch, no QR
    if (hutch ? o.probes <= 0 : (o.probes <= 0 || o.probes % 3 != 0))
        return fail(h, LL_ERR_INVALID_ARG, hutch ? "probes must be positive" : "probes must be a positive multiple of 3");
    if (o.probe_kind != LL_PROBE_RADEMACHER && o.probe_kind != LL_PROBE_GAUSSIAN) return fail(h, LL_ERR_INVALID_ARG, "unknown probe kind");
    if (o.precision < LL_PREC_F64 || o.precision > LL_PREC_F32_MIXED) return fail(h, LL_ERR_INVALID_ARG, "unknown precision");
    if (o.sval_mode != LL_SVAL_CENTER && o.sval_mode != LL_SVAL_HALF_LMAX) return fail(h, LL_ERR_INVALID_ARG, "unknown s_val mode");
    if (o.dd_scheme != LL_DD_AUTO && o.dd_scheme != LL_DD_TABLE_Q) return fail(h, LL_ERR_INVALID_ARG, "unknown divided-difference scheme");
    if (!std::isfinite(o.tol) || o.tol < 0.0) return fail(h, LL_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (o.qr_gram < LL_GRAM_AUTO || o.qr_gram > LL_GRAM_DFLOAT) return fail(h, LL_ERR_INVALID_ARG, "unknown Gram method");
    if (o.reorder < LL_REORDER_AUTO || o.reorder > LL_REORDER_DEGREE) return fail(h, LL_ERR_INVALID_ARG, "unknown row order");
    if (o.reorder == LL_REORDER_DEGREE && o.keep_for_backward)
        return fail(h, LL_ERR_UNSUPPORTED, "the degree order is for forwards that keep nothing for a backward");
    h->gram_method = o.qr_gram;
    const bool adaptive = o.tol > 0.0;   // Algorithm 2's stopping rule in both passes
    if (adaptive && o.keep_for_backward)
        return fail(h, LL_ERR_UNSUPPORTED, "the backward needs a fixed degree (tol = 0)");
    cudaStream_t s = (cudaStream_t)stream;
    h->launches = 0;
    h->kept = false;
    h->have_forward = false;
    h->spin_budget = o.timeout_cycles > 0 ? o.timeout_cycles : 4000000000LL;
    const int n = (int)A->n;
    if (n == 0) {
        *estimate = 0.0;
        return LL_OK;
    }
    const int kg = hutch ? o.probes : o.probes / 3;
    const int kq = hutch ? 0 : (kg < n ? kg : n);
    const int b2 = kq + kg;
    if (hutch && kg > 192) return fail(h, LL_ERR_UNSUPPORTED, "more than 192 Hutchinson probes are not supported");
    if (b2 > 512 || kq > 96) return fail(h, LL_ERR_UNSUPPORTED, "m_vec / 3 above 96 is not supported");
    if ((st = validate_csr(h, A0, s)) != LL_OK) return st;
    // the degree order for irregular matrices (power-law graphs: hubs first, their rows together in L2)
    ll_csr Aw{};
    const int32_t* rowmap = nullptr;   // probe row map of the permuted passes
    const int32_t* vsrc = nullptr;     // value gather map of the permuted passes
    {
        const double avg = (double)A0->nnz / (double)n;
        const bool irregular = !h->band_ok && (double)h->max_row > 4.0 * avg + 16.0 && 2 * h->far_entries > A0->nnz;
        const bool reorder = o.reorder == LL_REORDER_DEGREE || (o.reorder == LL_REORDER_AUTO && !o.keep_for_backward && irregular);
        if (reorder) {
            if ((st = prepare_reorder(h, A0, Aw, &rowmap, &vsrc, s)) != LL_OK) return st;
            A = &Aw;
            h->far_runs = 0;   // (the order breaks the diagonal runs: gather capacity for every far entry)
        }
    }
    // the gathered hub rows of the degree order kept in L2 (about half of it), for this call's passes
    struct HubScope {
        ll_handle* h;
        ~HubScope() { h->hub_bytes = 0; }
    } hub_scope{h};
    h->hub_bytes = A != A0 ? (long long)64 << 20 : 0;

    // host set-up: sigma, the scaled interval, Léja points, Algorithm 1 coefficients
    const double sigma = sigma_of(bounds.lmin);
    const double lt = bounds.lmin / sigma, ut = bounds.lmax / sigma;
    std::vector<double> xi, d;
    if ((st = setup_coefficients(h, lt, ut, o.degree, o.sval_mode, xi, d, o.dd_scheme)) != LL_OK) return st;
    const double c = (lt + ut) / 2.0, gamma = (ut - lt) / 4.0;
    const int m = o.degree;
    std::vector<double> beta(m + 1);
    for (int j = 0; j <= m; ++j) beta[j] = -(c / gamma + xi[j]);

    const int prec = o.precision;
    const int wt = w_type_of(prec), pt = p_type_of(prec);
    const size_t ew = elem_size(wt), ep = elem_size(pt);
    const int l1 = block_ld(prec, kq), l2 = block_ld(prec, b2);   // pass-1 and pass-2 blocks (column pairs)
    // workspace
    WS(vprep, void*, "fw_vals", (size_t)A->nnz * ew);
    WS(S, void*, "fw_S", (size_t)n * l1 * ew);
    WS(G, double*, "fw_G", (size_t)n * kg * sizeof(double));
    WS(P, void*, "fw_P", (size_t)n * l1 * ep);
    WS(wa, void*, "fw_wa", (size_t)n * l2 * ew);
    WS(wb, void*, "fw_wb", (size_t)n * l2 * ew);
    WS(basis, double*, "fw_basis", (size_t)n * l2 * sizeof(double));
    WS(q1, double*, "fw_q1", (size_t)n * (l1 > kq ? l1 : kq) * sizeof(double));   // FP64, or DF64 column pairs
    void* V = basis;
    if (wt != T_F64) {
        WS(vv, void*, "fw_V", (size_t)n * l2 * ew);
        V = vv;
    }
    const int ggrid = h->sm_count * 2;
    const size_t gp1 = gram_partials_any(h, kq, kq, true, ggrid), gp2 = gram_partials_any(h, kq, kg, false, ggrid);
    WS(gpart, double*, "fw_gram_partials", (gp1 > gp2 ? gp1 : gp2) * sizeof(double));
    WS(gticket, unsigned int*, "fw_gram_ticket", sizeof(unsigned int));
    WS(gram, double*, "fw_gram", (size_t)kq * (kq > kg ? kq : kg) * sizeof(double));
    WS(rinv1, double*, "fw_rinv1", (size_t)kq * kq * sizeof(double));   // R1^-1 (first CholeskyQR)
    WS(rinv, double*, "fw_rinv", (size_t)kq * kq * sizeof(double));     // R2^-1 (second)
    WS(qrstat, int*, "fw_qr_status", sizeof(int));
    WS(dots, double*, "fw_dots", (size_t)(m + 1) * b2 * sizeof(double));
    WS(tma_err, int*, "tma_error", sizeof(int));
    // column state of both passes under the stopping rule: live and final degree (b rounded up
    // to even), and the done flag
    StopState stop1, stop2, stop2g;
    // Under the rule, Hutch++'s trace pass runs as two passes, [Q] then [G']: the columns of Q
    // (unit norm) stop long before those of G' (norm about sqrt n), and a pass costs its whole
    // width until its last column stops
    const bool split2 = adaptive && !hutch && kq > 0 && kq < n && kg > 0;
    const int lg = block_ld(prec, kg);
    if (adaptive) {
        WS(sst, int*, "fw_stop_state", (size_t)(2 * (kq + 2) + 2 * (b2 + 2) + 2 * (kg + 2) + 3) * sizeof(int));
        int* z = sst;
        stop1 = StopState{o.tol, z, z + (kq + 2), nullptr};
        z += 2 * (kq + 2);
        stop2 = StopState{o.tol, z, z + (b2 + 2), nullptr};
        z += 2 * (b2 + 2);
        stop2g = StopState{o.tol, z, z + (kg + 2), nullptr};
        z += 2 * (kg + 2);
        stop1.done = z;
        stop2.done = z + 1;
        stop2g.done = z + 2;
    }
    void* Vq = nullptr;
    void* Vg = nullptr;
    if (split2) {
        WS(vq_, void*, "fw_Vq", (size_t)n * l1 * ew);
        WS(vg_, void*, "fw_Vg", (size_t)n * lg * ew);
        Vq = vq_;
        Vg = vg_;
    }
    // The backward needs W_0 .. W_{m-1} of the trace pass (and W_m for the through-QR term's
    // F [Q | G']). With GB300's HBM they usually fit: the trace pass then writes W_1 .. W_m into
    // the backward's checkpoint block, and the adjoint runs no forward steps. Taken when they need
    // at most half of the free device memory (counting the backward blocks this makes
    // unnecessary); otherwise the trace pass writes the backward's checkpoints at the smallest
    // stride that fits (at most ceil(sqrt(m))). Not under an explicit checkpoint stride.
    // Pass 1's W_j (W_0 = S), which the through-QR adjoint's second recurrence needs, are kept
    // as well when both fit, except for a banded matrix, whose pass 1 keeps its multi-step kernel.
    void* wall = nullptr;
    void* wall_s = nullptr;
    int wstride = 0, wblocks = 0;
    if (o.keep_for_backward && o.ckpt_stride == 0 && m >= 2 && !split2) {
        const size_t blk2 = (size_t)n * l2 * ew;
        const bool sketch = !hutch && kq > 0 && kq < n && !h->band_ok;
        const size_t need_s = sketch ? (size_t)m * n * l1 * ew : 0;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        size_t have = 0;
        for (const char* nm : {"bw_ckpt", "bw_ckpt_s", "bw_seg", "bw_tmp"}) {
            auto it = h->ws.find(nm);
            if (it != h->ws.end()) have += it->second.bytes;
        }
        const double budget = h->keep_budget > 0 ? (double)h->keep_budget : 0.5 * (double)(fr + have);
        // every W_j if they fit; else the checkpoints at the smallest stride that fits, at most the
        // backward's own ceil(sqrt(m)): written here, they spare the backward its first sweep
        // (when not even that fits, the forward keeps none and the backward checkpoints itself)
        const int smax = std::max(2, (int)std::ceil(std::sqrt((double)m)));
        if ((double)m * (double)blk2 <= budget) {
            wstride = 1;
            wblocks = m;
        } else {
            for (int st_ = 2; st_ <= smax; ++st_) {
                const int nb = (m + st_ - 1) / st_ - 1;
                if ((double)nb * (double)blk2 <= budget) {
                    wstride = st_;
                    wblocks = nb;
                    break;
                }
            }
        }
        if (wstride > 0 && wblocks > 0) {
            ws_release(h, "bw_tmp");
            if (wstride == 1) ws_release(h, "bw_seg");
            WS(wall_, void*, "bw_ckpt", (size_t)wblocks * blk2);
            wall = wall_;
            if (wstride == 1 && sketch && (double)(wblocks * blk2 + need_s) <= budget) {
                WS(wall_s_, void*, "bw_ckpt_s", need_s);
                wall_s = wall_s_;
            }
        } else {
            wstride = 0;
        }
    }
    int k1 = 0, t1 = 0, np1 = 1, rw1 = 0;   // step kernel, CTA size, column pairs per thread, rows per tile of pass 1

    // the device work of the call (Algorithm 3 steps 2-6), enqueued on q; with capture, the
    // phase events become event-record nodes of the graph
    bool capturing = false;
    auto rec = [&](cudaEvent_t ev, cudaStream_t q) {
        return capturing ? cudaEventRecordWithFlags(ev, q, cudaEventRecordExternal) : cudaEventRecord(ev, q);
    };
    auto enqueue = [&](cudaStream_t q) -> ll_status {
        LL_CK(rec(h->ev[0], q));
        LL_CK(cudaMemsetAsync(gticket, 0, sizeof(unsigned int), q));
        LL_CK(cudaMemsetAsync(qrstat, 0, sizeof(int), q));
        // matrix values scaled by 1 / (sigma gamma): B = (A/sigma - c I)/gamma = prepared - (c/gamma) I
        LL_CK(launch_prepare_values(A->values, A->dtype, A->nnz, 1.0 / (sigma * gamma), prec, vprep, q, vsrc));
        if (hutch) {
            // plain Hutchinson (Eq. Léja8): G straight into the trace pass's block (the pad
            // column zeroed); no pass 1 and no QR
            LL_CK(launch_probes(wt, o.probe_kind, o.seed, LL_STREAM_G, n, kg, l2, V, l2, q, rowmap));
            h->launches += 2;
            LL_CK(rec(h->ev[1], q));
            LL_CK(rec(h->ev[2], q));
            LL_CK(rec(h->ev[3], q));
        } else {
            // Algorithm 3 step 2 (S) and step 6 (G)
            LL_CK(launch_probes(wt, o.probe_kind, o.seed, LL_STREAM_S, n, kq, l1, S, l1, q, rowmap));
            LL_CK(launch_probes(T_F64, o.probe_kind, o.seed, LL_STREAM_G, n, kg, kg, G, kg, q, rowmap));
            h->launches += 3;
            LL_CK(rec(h->ev[1], q));
        }

        if (hutch) {
            // the trace pass below is the whole estimator
        } else if (kq == n) {
            // k >= n: the sketch spans R^n, so Q = I is an orthonormal basis of span(Y) and
            // G' = (I - Q Q^T) G = 0; the estimate is the exact trace of p(A~)
            LL_CK(rec(h->ev[2], q));
            LL_CK(cudaMemsetAsync(basis, 0, (size_t)n * l2 * sizeof(double), q));
            // the basis block holds FP64 (F64, DF64) or double-float pairs (FP32-mixed)
            LL_CK(launch_unit_diag(prec == LL_PREC_F32_MIXED ? T_DF64 : T_F64, basis, l2, n, q));
            h->launches++;
            if (wt != T_F64) {
                LL_CK(cudaMemsetAsync(V, 0, (size_t)n * l2 * ew, q));
                LL_CK(launch_unit_diag(wt, V, l2, n, q));
                h->launches++;
            }
            LL_CK(rec(h->ev[3], q));
        } else {
            // step 3: Y = p(A~) S
            st = run_pass(h, A, vprep, prec, MODE_ACCUM, n, kq, S, l1, wa, wb, P, l1, nullptr, beta, d, o.step_kernel,
                          o.threads_per_block, o.rows_per_thread, q, stop1, wall_s);
            if (st != LL_OK) return st;
            k1 = h->last_kernel;
            t1 = h->last_threads;
            np1 = h->last_np;
            rw1 = h->last_rows;
            LL_CK(rec(h->ev[2], q));

            // step 4: Q = CholeskyQR2(Y); step 6: G' = G - Q (Q^T G); V = [Q | G']
            const QrBlocks qb{P,     l1,      q1,   prec != LL_PREC_F64 ? l1 : kq, G,    V,      basis, l2, l2,
                              gpart, gticket, gram, rinv1, rinv, qrstat, ggrid};
            if ((st = qr_project(h, prec, n, kq, kg, qb, q)) != LL_OK) return st;
            LL_CK(rec(h->ev[3], q));
        }

        // steps 5-6: traces t_j[col] = <V_col, W_j col> for j = 0..m
        if (split2) {
            // [Q] and [G'] as two blocks; their traces land in dots as (m+1) x kq, then (m+1) x kg
            LL_CK(launch_copy_cols(wt, V, l2, 0, Vq, l1, n, kq, l1, q));
            LL_CK(launch_copy_cols(wt, V, l2, kq, Vg, lg, n, kg, lg, q));
            h->launches += 2;
            st = run_pass(h, A, vprep, prec, MODE_DOT, n, kq, Vq, l1, wa, wb, nullptr, 0, dots, beta, d, o.step_kernel,
                          o.threads_per_block, o.rows_per_thread, q, stop2);
            if (st != LL_OK) return st;
            st = run_pass(h, A, vprep, prec, MODE_DOT, n, kg, Vg, lg, wa, wb, nullptr, 0, dots + (size_t)(m + 1) * kq, beta,
                          d, o.step_kernel, o.threads_per_block, o.rows_per_thread, q, stop2g);
        } else {
            st = run_pass(h, A, vprep, prec, MODE_DOT, n, b2, V, l2, wa, wb, nullptr, 0, dots, beta, d, o.step_kernel,
                          o.threads_per_block, o.rows_per_thread, q, stop2, wall, wstride);
        }
        if (st != LL_OK) return st;
        LL_CK(rec(h->ev[4], q));
        return LL_OK;
    };

    // graph key: every input the enqueued work depends on (operands, coefficients, options, workspace)
    struct Key {
        const void* rp; const void* ci; const void* va;
        int64_t n, nnz;
        int dtype;
        double lmin, lmax;
        ll_options o;
        uint64_t ws_gen;
        int inject;
        int reordered;
    };
    Key key;
    memset(&key, 0, sizeof key);
    key.rp = A0->rowptr; key.ci = A0->colind; key.va = A0->values;
    key.n = A->n; key.nnz = A->nnz; key.dtype = A->dtype;
    key.lmin = bounds.lmin; key.lmax = bounds.lmax;
    key.o = o;
    key.o.keep_for_backward = (wall ? 1 + wstride * 4 : 0) + (wall_s ? 2 : 0);   // the passes write into the backward's blocks
    key.ws_gen = h->ws_gen;
    key.inject = h->inject;
    key.reordered = A != A0;
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&key);
    ll_handle::Graph& gr = h->gfwd;
    const bool hit = o.use_graph && gr.exec && gr.key.size() == sizeof key && memcmp(gr.key.data(), kb, sizeof key) == 0;
    if (hit) {
        LL_CK(cudaGraphLaunch(gr.exec, s));
        h->launches += gr.launches;
        k1 = gr.k1;
        t1 = gr.t1;
        np1 = gr.np1;
        rw1 = gr.r1;
        h->last_kernel = gr.k2;
        h->last_threads = gr.t2;
        h->last_np = gr.np2;
        h->last_rows = gr.r2;
        h->tma_used = gr.tma;
    } else {
        const int before = h->launches;
        if ((st = enqueue(s)) != LL_OK) return st;
        if (o.use_graph) {
            // capture the same work for the next identical call (tuning is cached by now and the
            // workspace allocated, so the capture only records launches and memsets); the key
            // takes the workspace as the eager run left it
            key.ws_gen = h->ws_gen;
            const int launched = h->launches - before;
            const bool tma = h->tma_used;
            if (gr.exec) {
                cudaGraphExecDestroy(gr.exec);
                gr.exec = nullptr;
            }
            if (!h->cap_stream) LL_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            LL_CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
            capturing = true;
            const int kk1 = k1, tt1 = t1, kk2 = h->last_kernel, tt2 = h->last_threads, nn1 = np1, nn2 = h->last_np;
            const int rr1 = rw1, rr2 = h->last_rows;
            const int cap0 = h->launches;
            ll_status cst = enqueue(h->cap_stream);
            const int in_graph = h->launches - cap0;   // without the autotuner's launches of the eager run
            capturing = false;
            cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
            if (cst == LL_OK && ce == cudaSuccess && graph && h->ws_gen == key.ws_gen &&
                cudaGraphInstantiate(&gr.exec, graph, 0) == cudaSuccess) {
                gr.key.assign(kb, kb + sizeof key);
                gr.launches = in_graph;
                gr.k1 = kk1;
                gr.t1 = tt1;
                gr.k2 = kk2;
                gr.t2 = tt2;
                gr.np1 = nn1;
                gr.np2 = nn2;
                gr.r1 = rr1;
                gr.r2 = rr2;
                gr.tma = tma;
            } else {
                gr.exec = nullptr;
                gr.key.clear();
            }
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            h->launches = before + launched;
            k1 = kk1;
            t1 = tt1;
            h->last_kernel = kk2;
            h->last_threads = tt2;
            np1 = nn1;
            h->last_np = nn2;
            rw1 = rr1;
            h->last_rows = rr2;
            h->tma_used = tma;
        }
    }

    std::vector<double> hd((size_t)(m + 1) * b2);
    int hstat = 0, herr = 0;
    // final degrees: the pass-1 columns (not run: Hutchinson, or k >= n) count as 0
    std::vector<int> deg1(kq, (hutch || kq == n) ? 0 : m), deg2(b2, m);
    LL_CK(cudaMemcpyAsync(hd.data(), dots, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (adaptive) {
        if (kq > 0 && !hutch && kq < n)
            LL_CK(cudaMemcpyAsync(deg1.data(), stop1.stop_deg, kq * sizeof(int), cudaMemcpyDeviceToHost, s));
        if (split2) {
            LL_CK(cudaMemcpyAsync(deg2.data(), stop2.stop_deg, kq * sizeof(int), cudaMemcpyDeviceToHost, s));
            LL_CK(cudaMemcpyAsync(deg2.data() + kq, stop2g.stop_deg, kg * sizeof(int), cudaMemcpyDeviceToHost, s));
        } else {
            LL_CK(cudaMemcpyAsync(deg2.data(), stop2.stop_deg, b2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        }
    }
    LL_CK(cudaMemcpyAsync(&hstat, qrstat, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (h->tma_used) LL_CK(cudaMemcpyAsync(&herr, tma_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    h->tma_used = false;
    if (herr) return fail(h, LL_ERR_TIMEOUT, "step kernel: a bounded pipeline wait ran out");
    if (hstat) return fail(h, LL_ERR_QR_BREAKDOWN, "CholeskyQR2: non-positive pivot (rank-deficient sketch)");

    if (split2) {
        // the two passes' traces, (m+1) x kq then (m+1) x kg, into the (m+1) x b2 layout
        std::vector<double> two(hd);
        for (int j = 0; j <= m; ++j) {
            for (int col = 0; col < kq; ++col) hd[(size_t)j * b2 + col] = two[(size_t)j * kq + col];
            for (int col = 0; col < kg; ++col) hd[(size_t)j * b2 + kq + col] = two[(size_t)(m + 1) * kq + (size_t)j * kg + col];
        }
    }
    // step 7 and output: n log sigma + tr(Q^T F Q) + (1/k) tr(G'^T F G'); under the stopping
    // rule, column col takes the terms j <= deg2[col] (the later dots are not its terms)
    double tq = 0.0, tr = 0.0;
    for (int j = 0; j <= m; ++j) {
        double sq = 0.0, sr = 0.0;
        for (int col = 0; col < kq; ++col)
            if (deg2[col] >= j) sq += hd[(size_t)j * b2 + col];
        for (int col = kq; col < b2; ++col)
            if (deg2[col] >= j) sr += hd[(size_t)j * b2 + col];
        tq += d[j] * sq;
        tr += d[j] * sr;
    }
    tr /= (double)kg;
    if (!std::isfinite(tq) || !std::isfinite(tr)) return fail(h, LL_ERR_NONFINITE, "non-finite trace");
    const double est = (double)n * std::log(sigma) + tq + tr;

    ll_info& I = h->info;
    I.sigma = sigma;
    I.c = c;
    I.gamma = gamma;
    I.trace_q = tq;
    I.trace_res = tr;
    I.estimate = est;
    I.taylor_terms = h->dd_terms;
    I.k = kq;
    I.kernel_launches = h->launches;
    cudaEventElapsedTime(&I.ms_probes, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&I.ms_pass1, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&I.ms_qr, h->ev[2], h->ev[3]);
    cudaEventElapsedTime(&I.ms_pass2, h->ev[3], h->ev[4]);
    cudaEventElapsedTime(&I.ms_total, h->ev[0], h->ev[4]);
    I.kernel_pass1 = k1;
    I.threads_pass1 = t1;
    I.kernel_pass2 = h->last_kernel;
    I.threads_pass2 = h->last_threads;
    I.pairs_pass1 = np1;
    I.pairs_pass2 = h->last_np;
    I.rows_pass1 = rw1;
    I.rows_pass2 = h->last_rows;
    I.batch_tuned = 0;
    I.reordered = A != A0;
    I.deg_max_pass1 = 0;
    for (int v : deg1) I.deg_max_pass1 = v > I.deg_max_pass1 ? v : I.deg_max_pass1;
    I.deg_max_pass2 = 0;
    double dsum = 0.0;
    for (int v : deg2) {
        I.deg_max_pass2 = v > I.deg_max_pass2 ? v : I.deg_max_pass2;
        dsum += v;
    }
    I.deg_mean_pass2 = b2 > 0 ? dsum / b2 : 0.0;
    I.kept_w_steps = wall ? wblocks : 0;
    I.kept_w_steps_pass1 = wall_s ? m : 0;
    I.kept_w_stride = wall ? wstride : 0;
    I.forward_id = ++h->forward_id;
    h->last_deg1 = deg1;
    h->last_deg2 = deg2;
    h->have_forward = true;

    if (o.keep_for_backward) {
        h->kept = true;
        h->kept_n = n;
        h->kept_nnz = A->nnz;
        h->kept_kq = kq;
        h->kept_kg = kg;
        h->kept_hutch = hutch;
        h->kept_qr = !hutch && kq < n;
        h->kept_band = h->band_ok;
        h->kept_stride = wall ? wstride : 0;
        h->kept_wall_s = wall_s != nullptr;
        h->kept_far = h->far_entries;
        h->kept_runs = h->far_runs;
        h->kept_max_row = h->max_row;
        h->kept_sorted = h->sorted;
        h->kept_m = m;
        h->kept_prec = prec;
        h->kept_ckpt = o.ckpt_stride;
        h->kept_gram = o.qr_gram;
        h->kept_sigma = sigma;
        h->kept_c = c;
        h->kept_gamma = gamma;
        h->kept_d = d;
        h->kept_xi = xi;
    }
    *estimate = est;
    return LL_OK;
}

ll_status ll_logdet_forward_host(ll_handle* h, const ll_csr* Ah, ll_bounds bounds, const ll_options* opts,
                                 double* estimate, void* stream) {
    if (!h) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, Ah);
    if (st != LL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vs = Ah->dtype == LL_F64 ? 8 : 4;
    WS(rp, int32_t*, "host_rowptr", (size_t)(Ah->n + 1) * sizeof(int32_t));
    WS(ci, int32_t*, "host_colind", (size_t)Ah->nnz * sizeof(int32_t));
    WS(va, void*, "host_values", (size_t)Ah->nnz * vs);
    LL_CK(cudaMemcpyAsync(rp, Ah->rowptr, (size_t)(Ah->n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (Ah->nnz > 0) {
        LL_CK(cudaMemcpyAsync(ci, Ah->colind, (size_t)Ah->nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        LL_CK(cudaMemcpyAsync(va, Ah->values, (size_t)Ah->nnz * vs, cudaMemcpyHostToDevice, s));
    }
    ll_csr Ad = *Ah;
    Ad.rowptr = rp;
    Ad.colind = ci;
    Ad.values = va;
    return ll_logdet_forward(h, &Ad, bounds, opts, estimate, stream);
}

ll_status ll_logdet_backward(ll_handle* h, const ll_csr* A, double grad_output, double* grad_values, void* stream) {
    return backward_impl(h, A, grad_output, grad_values, stream, false);
}

ll_status ll_logdet_backward_qr(ll_handle* h, const ll_csr* A, double grad_output, double* grad_values, void* stream) {
    return backward_impl(h, A, grad_output, grad_values, stream, true);
}

ll_status ll_param_grad(ll_handle* h, const double* grad_values, const double* dvalues, int64_t ld, int64_t nnz,
                        int nparams, double* out, void* stream) {
    if (!h || nparams < 0 || nnz < 0 || ld < nnz || (nparams > 0 && !out)) return LL_ERR_INVALID_ARG;
    if (nparams == 0) return LL_OK;
    if (nnz > 0 && (!grad_values || !dvalues)) return fail(h, LL_ERR_INVALID_ARG, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = h->sm_count * 4;
    WS(partials, double*, "pg_partials", (size_t)nparams * grid * sizeof(double));
    WS(ticket, unsigned int*, "pg_ticket", sizeof(unsigned int));
    WS(res, double*, "pg_out", (size_t)nparams * sizeof(double));
    LL_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
    LL_CK(launch_param_dot(grad_values, dvalues, ld, nnz, nparams, partials, ticket, res, grid, s));
    h->launches++;
    std::vector<double> hv(nparams);
    LL_CK(cudaMemcpyAsync(hv.data(), res, nparams * sizeof(double), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    for (int p = 0; p < nparams; ++p) out[p] = hv[p];
    return LL_OK;
}

}  // extern "C"

namespace {

// Graph key of a batched call: every input its device work depends on.
std::vector<unsigned char> batched_key(const ll_handle* h, const ll_csr* mats, const ll_bounds* bnd, int count,
                                       const ll_options& o, const int* degrees) {
    std::vector<unsigned char> k;
    auto put = [&](const void* p, size_t bytes) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        k.insert(k.end(), c, c + bytes);
    };
    put(&count, sizeof count);
    for (int i = 0; i < count; ++i) {
        put(&mats[i].n, sizeof mats[i].n);
        put(&mats[i].nnz, sizeof mats[i].nnz);
        put(&mats[i].rowptr, sizeof mats[i].rowptr);
        put(&mats[i].colind, sizeof mats[i].colind);
        put(&mats[i].values, sizeof mats[i].values);
        put(&mats[i].dtype, sizeof mats[i].dtype);
        put(&bnd[i].lmin, sizeof bnd[i].lmin);
        put(&bnd[i].lmax, sizeof bnd[i].lmax);
        const int m = degrees ? degrees[i] : -1;
        put(&m, sizeof m);
    }
    ll_options oo;
    memset(&oo, 0, sizeof oo);
    oo = o;
    oo.keep_for_backward = 0;
    put(&oo.degree, sizeof oo.degree);
    put(&oo.probes, sizeof oo.probes);
    put(&oo.seed, sizeof oo.seed);
    put(&oo.probe_kind, sizeof oo.probe_kind);
    put(&oo.precision, sizeof oo.precision);
    put(&oo.sval_mode, sizeof oo.sval_mode);
    put(&oo.dd_scheme, sizeof oo.dd_scheme);
    put(&oo.timeout_cycles, sizeof oo.timeout_cycles);
    put(&oo.step_kernel, sizeof oo.step_kernel);
    put(&h->ws_gen, sizeof h->ws_gen);
    put(&h->inject, sizeof h->inject);
    return k;
}

// Reads the traces, error flag and QR status of the last batched device work and combines the
// estimates (Section 4.1) from the coefficients kept with it.
ll_status batched_finish(ll_handle* h, const ll_csr* mats, int count, double* estimates, cudaStream_t s) {
    const ll_handle::BatchGraph& G = h->gbat;
    const int kq = G.kq, kg = G.kg, b2 = kq + kg;
    int herr = 0;
    std::vector<int> hqr(count);
    LL_CK(cudaMemcpyAsync(&herr, G.ctr + 2 * count + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaMemcpyAsync(hqr.data(), G.qrstat, count * sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<std::vector<double>> hd(count);
    for (int i = 0; i < count; ++i) {
        hd[i].resize(G.d[i].size() * b2);
        LL_CK(cudaMemcpyAsync(hd[i].data(), G.dots[i], hd[i].size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    LL_CK(cudaStreamSynchronize(s));
    if (herr) return fail(h, LL_ERR_TIMEOUT, "batched launch: a bounded wait ran out");
    for (int i = 0; i < count; ++i)
        if (hqr[i]) return fail(h, LL_ERR_QR_BREAKDOWN, "CholeskyQR2 breakdown in batch entry " + std::to_string(i));
    std::vector<double> est(count);
    for (int i = 0; i < count; ++i) {
        double tq = 0.0, tr = 0.0;
        for (size_t j = 0; j < G.d[i].size(); ++j) {
            double sq = 0.0, sr = 0.0;
            for (int col = 0; col < kq; ++col) sq += hd[i][j * b2 + col];
            for (int col = kq; col < b2; ++col) sr += hd[i][j * b2 + col];
            tq += G.d[i][j] * sq;
            tr += G.d[i][j] * sr;
        }
        tr /= (double)kg;
        if (!std::isfinite(tq) || !std::isfinite(tr)) return fail(h, LL_ERR_NONFINITE, "non-finite trace in batch entry " + std::to_string(i));
        est[i] = (double)mats[i].n * std::log(G.sigma[i]) + tq + tr;
    }
    for (int i = 0; i < count; ++i) estimates[i] = est[i];
    ll_info& I = h->info;
    I = ll_info{};
    I.k = kq;
    I.kernel_launches = h->launches;
    I.kernel_pass1 = G.kernel;
    I.kernel_pass2 = G.kernel;
    I.threads_pass1 = G.threads1;
    I.threads_pass2 = G.threads2;
    I.rows_pass1 = G.rows1;
    I.rows_pass2 = G.rows2;
    I.pairs_pass1 = I.pairs_pass2 = 1;
    cudaEventElapsedTime(&I.ms_probes, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&I.ms_pass1, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&I.ms_qr, h->ev[2], h->ev[3]);
    cudaEventElapsedTime(&I.ms_pass2, h->ev[3], h->ev[4]);
    cudaEventElapsedTime(&I.ms_total, h->ev[0], h->ev[4]);
    return LL_OK;
}

// Launch shape of a batched call: the step kernel of both passes (LL_KERNEL_TMA or LL_KERNEL_GATHER)
// and, for the TMA kernel, the consumer-thread target of each pass (rows per tile = target / column
// pairs); graph: capture / replay the device work.
struct BatchCfg {
    int kernel = LL_KERNEL_TMA;
    int threads1 = 512, threads2 = 512;
    bool graph = true;
};

ll_status batched_run(ll_handle* h, const ll_csr* mats, const ll_bounds* bnd, int count, const ll_options* opts,
                      const int* degrees, double* estimates, void* stream, const BatchCfg& cfg) {
    if (!h || !opts || count < 0 || (count > 0 && (!mats || !bnd || !estimates))) return LL_ERR_INVALID_ARG;
    if (count == 0) return LL_OK;
    const ll_options& o = *opts;
    if (o.probes <= 0 || o.probes % 3 != 0) return fail(h, LL_ERR_INVALID_ARG, "probes must be a positive multiple of 3");
    if (o.estimator != LL_EST_HUTCHPP) return fail(h, LL_ERR_UNSUPPORTED, "the batched call runs Hutch++ only");
    if (o.tol != 0.0) return fail(h, LL_ERR_UNSUPPORTED, "the batched call runs a fixed degree per matrix (tol = 0)");
    if (o.probe_kind != LL_PROBE_RADEMACHER && o.probe_kind != LL_PROBE_GAUSSIAN) return fail(h, LL_ERR_INVALID_ARG, "unknown probe kind");
    if (o.precision < LL_PREC_F64 || o.precision > LL_PREC_F32_MIXED) return fail(h, LL_ERR_INVALID_ARG, "unknown precision");
    cudaStream_t s = (cudaStream_t)stream;
    h->launches = 0;
    h->kept = false;
    const int kg = o.probes / 3;
    const int prec = o.precision;
    const int wt = w_type_of(prec), pt = p_type_of(prec);
    const size_t ew = elem_size(wt), ep = elem_size(pt);
    for (int i = 0; i < count; ++i) {
        ll_status st = check_csr_args(h, &mats[i]);
        if (st != LL_OK) return st;
        if ((st = check_bounds(h, bnd[i])) != LL_OK) return st;
        if (mats[i].n <= kg) return fail(h, LL_ERR_UNSUPPORTED, "batched matrices need more rows than m_vec / 3");
        if (degrees && degrees[i] < 1) return fail(h, LL_ERR_INVALID_ARG, "degree must be >= 1");
    }
    if (2 * kg > 512 || kg > 96) return fail(h, LL_ERR_UNSUPPORTED, "m_vec / 3 above 96 is not supported");
    const int kq = kg, b1 = kq, b2 = kq + kg, l1 = block_ld(prec, b1), l2 = block_ld(prec, b2);

    // validation of every CSR (one synchronisation); the far-entry counts size the TMA gather capacity
    std::vector<int> hfar(count, 0);
    {
        WS(flags, int*, "bt_flags", (size_t)2 * count * sizeof(int));
        LL_CK(cudaMemsetAsync(flags, 0, (size_t)2 * count * sizeof(int), s));
        for (int i = 0; i < count; ++i)
            if (mats[i].n > 0) { LL_CK(launch_validate_csr(mats[i].rowptr, mats[i].colind, (int)mats[i].n, mats[i].nnz, flags + 2 * i, s)); h->launches++; }
        std::vector<int> hf(2 * count);
        LL_CK(cudaMemcpyAsync(hf.data(), flags, hf.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        LL_CK(cudaStreamSynchronize(s));
        for (int i = 0; i < count; ++i)
            if (hf[2 * i]) return fail(h, LL_ERR_BAD_CSR, "invalid CSR in batch entry " + std::to_string(i));
        for (int i = 0; i < count; ++i) hfar[i] = hf[2 * i + 1];
    }
    // an identical call replays the captured device work (the descriptors, tables and
    // coefficients it reads are still on the device)
    const bool use_graph = o.use_graph && cfg.graph;
    if (use_graph && h->gbat.exec && h->gbat.key == batched_key(h, mats, bnd, count, o, degrees)) {
        LL_CK(cudaGraphLaunch(h->gbat.exec, s));
        h->launches += h->gbat.launches;
        return batched_finish(h, mats, count, estimates, s);
    }
    // host set-up per matrix: sigma, interval, degree, coefficients
    struct Host { double sigma, c, gamma; int m; std::vector<double> d, coef; };
    std::vector<Host> hs(count);
    int max_m = 0;
    for (int i = 0; i < count; ++i) {
        Host& x = hs[i];
        x.sigma = sigma_of(bnd[i].lmin);
        const double lt = bnd[i].lmin / x.sigma, ut = bnd[i].lmax / x.sigma;
        x.m = degrees ? degrees[i] : degree_from_bounds(lt, ut);
        x.c = (lt + ut) / 2.0;
        x.gamma = (ut - lt) / 4.0;
        x.d.resize(x.m + 1);
        if (coefficients_by_scheme(lt, ut, x.m, o.sval_mode, o.dd_scheme, x.d.data()) < 0)
            return fail(h, LL_ERR_DD_NOT_CONVERGED, "Algorithm 1 did not converge for batch entry " + std::to_string(i));
        std::vector<double> xi(x.m + 1);
        leja_points(x.m + 1, xi.data());
        x.coef.resize(2 * (x.m + 1));
        for (int j = 0; j <= x.m; ++j) { x.coef[2 * j] = -(x.c / x.gamma + xi[j]); x.coef[2 * j + 1] = x.d[j]; }
        max_m = std::max(max_m, x.m);
    }
    // order by degree (descending): the matrices active at a step are then a prefix
    std::vector<int> ord(count);
    for (int i = 0; i < count; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hs[a].m > hs[b].m; });

    BatchParams bp1{}, bp2{};
    size_t smem1 = 0, smem2 = 0;
    double avg = 0.0, tot_n = 0.0;
    for (int i = 0; i < count; ++i) { avg += (double)mats[i].nnz; tot_n += (double)mats[i].n; }
    avg /= tot_n;
    plan_batched(b1, avg, bp1, &smem1);
    plan_batched(b2, avg, bp2, &smem2);
    // TMA-fed persistent passes, unless the register-gather kernel is asked for or no layout fits
    BatchTmaLaunch tl1, tl2;
    bool use_tma = false;
    if (cfg.kernel != LL_KERNEL_GATHER) {
        int n_min = INT32_MAX;
        double far = 0.0;
        for (int i = 0; i < count; ++i) {
            n_min = std::min(n_min, (int)mats[i].n);
            far += (double)hfar[i];
        }
        use_tma = plan_batched_tma(prec, MODE_ACCUM, n_min, avg, far / tot_n, b1, l1, l1, max_m, count, h->sm_count, tl1,
                                   cfg.threads1) &&
                  plan_batched_tma(prec, MODE_DOT, n_min, avg, far / tot_n, b2, l2, l2, max_m, count, h->sm_count, tl2,
                                   cfg.threads2);
    }
    const int R1 = use_tma ? tl1.q.R : bp1.R, R2 = use_tma ? tl2.q.R : bp2.R;
    const int tstride = bt_table_ints(max_m, count);   // per pass: step offsets, active counts, tile prefix, coef offsets

    // one workspace for every per-matrix buffer (256-byte aligned regions)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    struct Off { size_t vals, S, G, P, wa, wb, basis, q1, V, part, dots, coef, qpart, gram, rinv; int T1, T2, gxs, gxc; };
    const int ggrid = h->sm_count * 2;
    std::vector<Off> off(count);
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        const size_t n = (size_t)mats[i].n, nnz = (size_t)mats[i].nnz;
        Off& f = off[i];
        f.T1 = (int)((n + R1 - 1) / R1);
        f.T2 = (int)((n + R2 - 1) / R2);
        f.vals = total; total += al(nnz * ew);
        f.S = total; total += al(n * l1 * ew);
        f.G = total; total += al(n * kg * sizeof(double));
        f.P = total; total += al(n * l1 * ep);
        f.wa = total; total += al(n * l2 * ew);
        f.wb = total; total += al(n * l2 * ew);
        f.basis = total; total += al(n * l2 * sizeof(double));
        f.q1 = total; total += al(n * kq * sizeof(double));
        f.V = total; total += al(n * l2 * ew);
        // trace partials: per step and tile (TMA passes, reduced after the pass), else two slots per tile
        f.part = total;
        total += al((use_tma ? (size_t)(hs[i].m + 1) * f.T2 : (size_t)2 * std::max(f.T1, f.T2)) * b2 * sizeof(double));
        f.dots = total; total += al((size_t)(hs[i].m + 1) * b2 * sizeof(double));
        f.coef = total; total += al((size_t)2 * (hs[i].m + 1) * sizeof(double));
        // CholeskyQR2 of this matrix: Gram partials of its row blocks, ticket, Gram and R^{-1}
        // Gram row blocks: this matrix's share of about four CTAs per SM over the whole batch (a
        // grid sized for one matrix, 64 times over, spent the time in per-CTA reductions)
        const int gshare = (int)std::max(1.0, std::ceil(4.0 * ggrid * (double)n / tot_n));
        f.gxs = gram_blocks(kq, kq, true, (int)n, gshare);
        f.gxc = gram_blocks(kq, kg, false, (int)n, gshare);
        const size_t qp = std::max(gram_partials_doubles(kq, kq, true, f.gxs), gram_partials_doubles(kq, kg, false, f.gxc));
        f.qpart = total; total += al(qp * sizeof(double));
        f.gram = total; total += al((size_t)kq * kg * sizeof(double));
        f.rinv = total; total += al((size_t)kq * kq * sizeof(double));
    }
    WS(base, char*, "bt_all", total);
    WS(qrstat, int*, "bt_qr_status", (size_t)count * sizeof(int));
    WS(qticks, unsigned int*, "bt_qr_tickets", (size_t)count * sizeof(unsigned int));
    WS(gjobs, GramJob*, "bt_gram_jobs", (size_t)3 * count * sizeof(GramJob));
    WS(cjobs, CholJob*, "bt_chol_jobs", (size_t)count * sizeof(CholJob));
    WS(rjobs, RowJob*, "bt_row_jobs", (size_t)3 * count * sizeof(RowJob));
    WS(ctr, unsigned long long*, "bt_counters", (size_t)(2 * count + 8) * sizeof(unsigned long long));
    WS(dmats, BatchMat*, "bt_mats", (size_t)2 * count * sizeof(BatchMat));
    WS(dtab, int*, "bt_tables", (size_t)2 * tstride * sizeof(int));
    // TMA passes: per-pass tile descriptors of every matrix (by batch tile), the matrices with
    // their tensor maps, and the coefficient tables concatenated
    size_t ntiles[2] = {0, 0}, ncoef = 0;
    for (int i = 0; i < count; ++i) {
        ntiles[0] += (size_t)off[i].T1;
        ntiles[1] += (size_t)off[i].T2;
        ncoef += (size_t)2 * (hs[i].m + 1);
    }
    unsigned char* tdesc[2] = {nullptr, nullptr};
    int* tgcol[2] = {nullptr, nullptr};
    int4* tmeta[2] = {nullptr, nullptr};
    BatchTmaMat* dtm = nullptr;
    double* coef_all = nullptr;
    float2* coef_df_all = nullptr;
    if (use_tma) {
        WS(d1, unsigned char*, "bt_tma_desc1", ntiles[0] * tl1.q.desc_stride);
        WS(d2, unsigned char*, "bt_tma_desc2", ntiles[1] * tl2.q.desc_stride);
        WS(g1, int*, "bt_tma_gcol1", ntiles[0] * tl1.q.gcol_stride);
        WS(g2, int*, "bt_tma_gcol2", ntiles[1] * tl2.q.gcol_stride);
        WS(m1, int4*, "bt_tma_meta1", ntiles[0] * sizeof(int4));
        WS(m2, int4*, "bt_tma_meta2", ntiles[1] * sizeof(int4));
        WS(tm, BatchTmaMat*, "bt_tma_mats", (size_t)2 * count * sizeof(BatchTmaMat));
        WS(ca, double*, "bt_tma_coef", ncoef * sizeof(double));
        WS(cd, float2*, "bt_tma_coef_df", ncoef * sizeof(float2));
        coef_df_all = cd;
        tdesc[0] = d1; tdesc[1] = d2;
        tgcol[0] = g1; tgcol[1] = g2;
        tmeta[0] = m1; tmeta[1] = m2;
        dtm = tm;
        coef_all = ca;
    }

    // descriptors and item tables of both passes
    std::vector<BatchMat> hm(2 * count);
    std::vector<int> tabs((size_t)2 * tstride);
    BatchTmaParams bt1{}, bt2{};
    std::vector<BatchTmaMat> htm(use_tma ? 2 * count : 0);
    std::vector<double> hcoef;
    std::vector<int> coef_off(count);
    for (int q = 0; q < count; ++q) {
        coef_off[q] = (int)hcoef.size();
        hcoef.insert(hcoef.end(), hs[ord[q]].coef.begin(), hs[ord[q]].coef.end());
    }
    for (int pass = 0; pass < 2; ++pass) {
        int* t_off = tabs.data() + pass * tstride;
        int* t_act = t_off + (max_m + 1);
        int* t_pre = t_act + (max_m + 1);
        int* t_cof = t_pre + (count + 1);
        for (int q = 0; q < count; ++q) t_cof[q] = coef_off[q];
        t_pre[0] = 0;
        for (int q = 0; q < count; ++q) {
            const int i = ord[q];
            const Off& f = off[i];
            BatchMat& M = hm[pass * count + q];
            M.rowptr = mats[i].rowptr;
            M.colind = mats[i].colind;
            M.vals = base + f.vals;
            M.w0 = base + (pass == 0 ? f.S : f.V);
            M.wa = base + f.wa;
            M.wb = base + f.wb;
            M.p = base + f.P;
            M.partials = (double*)(base + f.part);
            M.dots = (double*)(base + f.dots);
            M.coef = (const double*)(base + f.coef);
            M.n = (int)mats[i].n;
            M.T = pass == 0 ? f.T1 : f.T2;
            M.m = hs[i].m;
            t_pre[q + 1] = t_pre[q] + M.T;
        }
        int acc = 0;
        for (int j = 0; j < max_m; ++j) {
            int a = 0;
            while (a < count && hs[ord[a]].m > j) ++a;
            t_act[j] = a;
            t_off[j] = acc;
            acc += t_pre[a];
        }
        t_off[max_m] = acc;
        BatchParams& bp = pass == 0 ? bp1 : bp2;
        bp.mats = dmats + pass * count;
        bp.step_off = dtab + pass * tstride;
        bp.step_active = bp.step_off + (max_m + 1);
        bp.tile_prefix = bp.step_active + (max_m + 1);
        bp.ticket = (unsigned int*)(ctr + 2 * count) + pass;
        bp.error = (int*)(ctr + 2 * count + 2);
        bp.arrived = ctr;
        bp.released = ctr + count;
        bp.spin_budget = o.timeout_cycles > 0 ? o.timeout_cycles : 4000000000LL;   // default: about 2 s at 2 GHz
        bp.ld = pass == 0 ? l1 : l2;
        bp.total_items = acc;
        bp.max_m = max_m;
        if (use_tma) {
            const BatchTmaLaunch& TL = pass == 0 ? tl1 : tl2;
            const int ld = pass == 0 ? l1 : l2;
            const int Rt = TL.q.R;
            for (int q = 0; q < count; ++q) {
                const BatchMat& M = hm[pass * count + q];
                BatchTmaMat& X = htm[pass * count + q];
                X.colind = M.colind;
                X.vals = M.vals;
                X.w[0] = const_cast<void*>(M.w0);
                X.w[1] = M.wa;
                X.w[2] = M.wb;
                X.p = M.p;
                X.partials = M.partials;
                X.dots = M.dots;
                X.n = M.n;
                X.T = M.T;
                X.m = M.m;
                bool ok = true;
                for (int x = 0; x < 3; ++x)
                    ok = ok && encode_rows(&X.gat[x], X.w[x], (int)ew, ld, X.n, 1) &&
                         encode_rows(&X.win[x], X.w[x], (int)ew, ld, X.n, Rt + 2 * TMA_HALO);
                // pass 1 reads P rows (8-byte elements), pass 2 the V rows
                ok = ok && (pass == 0 ? encode_rows(&X.aux, M.p, 8, ld, X.n, Rt) : encode_rows(&X.aux, M.w0, (int)ew, ld, X.n, Rt));
                if (!ok) return fail(h, LL_ERR_CUDA, "tensor map encoding failed for batch entry " + std::to_string(ord[q]));
            }
            BatchTmaParams& B = pass == 0 ? bt1 : bt2;
            B.mats = dtm + pass * count;
            B.tables = bp.step_off;
            B.coef = coef_all;
            B.coef_df = coef_df_all;
            B.desc = tdesc[pass];
            B.gcol = tgcol[pass];
            B.meta = tmeta[pass];
            B.ticket = bp.ticket;
            B.error = bp.error;
            B.arrived = bp.arrived;
            B.spin_budget = bp.spin_budget;
            B.total_items = acc;
            B.max_m = max_m;
            B.count = count;
            B.b = pass == 0 ? b1 : b2;
            B.ldw = ld;
            B.ldp = ld;
            B.q = TL.q;
            B.q.inject = h->inject;
        }
    }
    if (use_tma) {
        LL_CK(cudaMemcpyAsync(dtm, htm.data(), htm.size() * sizeof(BatchTmaMat), cudaMemcpyHostToDevice, s));
        LL_CK(cudaMemcpyAsync(coef_all, hcoef.data(), hcoef.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        std::vector<float2> hcoef_df(hcoef.size());
        for (size_t x = 0; x < hcoef.size(); ++x) hcoef_df[x] = df_split(hcoef[x]);
        LL_CK(cudaMemcpyAsync(coef_df_all, hcoef_df.data(), hcoef_df.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    }
    LL_CK(cudaMemcpyAsync(dmats, hm.data(), hm.size() * sizeof(BatchMat), cudaMemcpyHostToDevice, s));
    LL_CK(cudaMemcpyAsync(dtab, tabs.data(), tabs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int i = 0; i < count; ++i)
        LL_CK(cudaMemcpyAsync(base + off[i].coef, hs[i].coef.data(), hs[i].coef.size() * sizeof(double), cudaMemcpyHostToDevice, s));

    // QR job lists of every matrix (pointers only), copied before the device work
    std::vector<GramJob> gj(3 * count);
    std::vector<CholJob> cj(count);
    std::vector<RowJob> rj(3 * count);
    int gxs_max = 1, gxc_max = 1, n_max = 1;
    for (int i = 0; i < count; ++i) {
        const Off& f = off[i];
        const int n = (int)mats[i].n;
        double* part = (double*)(base + f.qpart);
        unsigned int* tick = qticks + i;
        double* gram = (double*)(base + f.gram);
        double* rinv = (double*)(base + f.rinv);
        void* P = base + f.P;
        double* q1 = (double*)(base + f.q1);
        double* basis = (double*)(base + f.basis);
        double* G = (double*)(base + f.G);
        void* V = base + f.V;
        gj[i] = GramJob{P, nullptr, n, f.gxs, part, tick, gram};
        gj[count + i] = GramJob{q1, nullptr, n, f.gxs, part, tick, gram};
        gj[2 * count + i] = GramJob{basis, G, n, f.gxc, part, tick, gram};
        cj[i] = CholJob{gram, rinv, qrstat + i};
        rj[i] = RowJob{P, rinv, nullptr, q1, nullptr, n};
        rj[count + i] = RowJob{q1, rinv, nullptr, basis, V, n};
        // G' into columns [kq, kq + kg) of [Q | G']; the typed block is offset by kq elements
        rj[2 * count + i] = RowJob{basis, gram, G, basis + kq, V, n};
        gxs_max = std::max(gxs_max, f.gxs);
        gxc_max = std::max(gxc_max, f.gxc);
        n_max = std::max(n_max, n);
    }
    LL_CK(cudaMemcpyAsync(gjobs, gj.data(), gj.size() * sizeof(GramJob), cudaMemcpyHostToDevice, s));
    LL_CK(cudaMemcpyAsync(cjobs, cj.data(), cj.size() * sizeof(CholJob), cudaMemcpyHostToDevice, s));
    LL_CK(cudaMemcpyAsync(rjobs, rj.data(), rj.size() * sizeof(RowJob), cudaMemcpyHostToDevice, s));

    // the device work of the call, enqueued on q (captured into a graph for identical calls)
    bool capturing = false;
    auto rec = [&](cudaEvent_t ev, cudaStream_t q) {
        return capturing ? cudaEventRecordWithFlags(ev, q, cudaEventRecordExternal) : cudaEventRecord(ev, q);
    };
    auto enqueue = [&](cudaStream_t q) -> ll_status {
        LL_CK(rec(h->ev[0], q));
        LL_CK(cudaMemsetAsync(ctr, 0, (size_t)(2 * count + 8) * sizeof(unsigned long long), q));
        LL_CK(cudaMemsetAsync(qrstat, 0, (size_t)count * sizeof(int), q));
        LL_CK(cudaMemsetAsync(qticks, 0, (size_t)count * sizeof(unsigned int), q));
        for (int i = 0; i < count; ++i) {
            const Off& f = off[i];
            const int n = (int)mats[i].n;
            const uint64_t seed = o.seed + (uint64_t)i;
            LL_CK(launch_prepare_values(mats[i].values, mats[i].dtype, mats[i].nnz, 1.0 / (hs[i].sigma * hs[i].gamma), prec, base + f.vals, q));
            LL_CK(launch_probes(wt, o.probe_kind, seed, LL_STREAM_S, n, kq, l1, base + f.S, l1, q));
            LL_CK(launch_probes(T_F64, o.probe_kind, seed, LL_STREAM_G, n, kg, kg, base + f.G, kg, q));
            h->launches += 3;
        }
        int per_sm = 2;
        const int grid1 = h->sm_count * per_sm, grid2 = h->sm_count * per_sm;
        // tile descriptors of every matrix for a TMA pass (built from the prepared values)
        auto describe = [&](int pass) -> ll_status {
            const BatchTmaLaunch& TL = pass == 0 ? tl1 : tl2;
            const int* t_pre = tabs.data() + pass * tstride + 2 * (max_m + 1);
            for (int qq = 0; qq < count; ++qq) {
                const int i = ord[qq];
                TmaLaunch D{};
                D.q = TL.q;
                D.q.desc_w = tdesc[pass] + (size_t)t_pre[qq] * TL.q.desc_stride;
                D.q.gcol_w = tgcol[pass] + (size_t)t_pre[qq] * (TL.q.gcol_stride / 4);
                D.q.meta_w = tmeta[pass] + t_pre[qq];
                StepParams pd{};
                pd.rowptr = mats[i].rowptr;
                pd.colind = mats[i].colind;
                pd.vals = base + off[i].vals;
                pd.n = (int)mats[i].n;
                pd.num_tiles = pass == 0 ? off[i].T1 : off[i].T2;
                LL_CK(launch_tma_describe(prec, D, pd, q));
                h->launches++;
            }
            return LL_OK;
        };
        LL_CK(rec(h->ev[1], q));
        // pass 1 of every matrix: one persistent launch
        if (use_tma) {
            ll_status ds = describe(0);
            if (ds != LL_OK) return ds;
            LL_CK(launch_batched_tma(prec, MODE_ACCUM, bt1, tl1, q));
        } else {
            LL_CK(launch_batched(prec, MODE_ACCUM, bp1, grid1, smem1, q));
        }
        h->launches++;
        LL_CK(rec(h->ev[2], q));
        // CholeskyQR2 and deflation of every matrix: eight launches over per-matrix job lists
        // (Gram of Y, Cholesky, Y R^{-1}; Gram of Q1, Cholesky, Q1 R^{-1}; C = Q^T G; G' = G - Q C)
        {
            const GramJob g0 = gj[0];
            const CholJob c0 = cj[0];
            const RowJob r0 = rj[0];
            LL_CK(launch_gram_jobs(pt, l1, kq, T_F64, 0, kq, true, g0, gjobs, count, gxs_max, q));
            LL_CK(launch_chol_jobs(kq, c0, cjobs, count, q));
            LL_CK(launch_apply_rinv_jobs(pt, l1, kq, kq, T_F64, 0, r0, rjobs, count, n_max, q));
            LL_CK(launch_gram_jobs(T_F64, kq, kq, T_F64, 0, kq, true, g0, gjobs + count, count, gxs_max, q));
            LL_CK(launch_chol_jobs(kq, c0, cjobs, count, q));
            LL_CK(launch_apply_rinv_jobs(T_F64, kq, kq, l2, wt, l2, r0, rjobs + count, count, n_max, q));
            LL_CK(launch_gram_jobs(T_F64, l2, kq, T_F64, kg, kg, false, g0, gjobs + 2 * count, count, gxc_max, q));
            LL_CK(launch_project_jobs(l2, kq, kg, kg, l2, wt, l2, l2 - b2, kq, r0, rjobs + 2 * count, count, n_max, q));
            h->launches += 8;
        }
        LL_CK(rec(h->ev[3], q));
        // pass 2 of every matrix: one persistent launch (arrival / release counters start at zero)
        LL_CK(cudaMemsetAsync(ctr, 0, (size_t)2 * count * sizeof(unsigned long long), q));
        if (use_tma) {
            ll_status ds = describe(1);
            if (ds != LL_OK) return ds;
            LL_CK(launch_batched_tma(prec, MODE_DOT, bt2, tl2, q));
            // traces of every matrix and step: the tile partials summed in tile order
            LL_CK(launch_batched_dots(prec, dtm + count, count, b2, (max_m + 1) * b2, q));
            h->launches++;
        } else {
            LL_CK(launch_batched(prec, MODE_DOT, bp2, grid2, smem2, q));
        }
        h->launches++;
        LL_CK(rec(h->ev[4], q));
        return LL_OK;
    };
    const int before = h->launches;
    ll_status st = enqueue(s);
    if (st != LL_OK) return st;
    const int launched = h->launches - before;
    ll_handle::BatchGraph& G = h->gbat;
    G.d.resize(count);
    G.sigma.resize(count);
    G.dots.resize(count);
    for (int i = 0; i < count; ++i) {
        G.d[i] = hs[i].d;
        G.sigma[i] = hs[i].sigma;
        G.dots[i] = (double*)(base + off[i].dots);
    }
    G.kq = kq;
    G.kg = kg;
    G.ctr = ctr;
    G.qrstat = qrstat;
    G.launches = launched;
    G.kernel = use_tma ? LL_KERNEL_TMA : LL_KERNEL_GATHER;
    G.threads1 = use_tma ? tl1.threads : BATCH_THREADS;
    G.threads2 = use_tma ? tl2.threads : BATCH_THREADS;
    G.rows1 = R1;
    G.rows2 = R2;
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    G.key.clear();
    if (use_graph) {
        if (!h->cap_stream) LL_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        LL_CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
        capturing = true;
        const ll_status cst = enqueue(h->cap_stream);
        capturing = false;
        const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
        if (cst == LL_OK && ce == cudaSuccess && graph && cudaGraphInstantiate(&G.exec, graph, 0) == cudaSuccess)
            G.key = batched_key(h, mats, bnd, count, o, degrees);
        else
            G.exec = nullptr;
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        h->launches = before + launched;
    }
    return batched_finish(h, mats, count, estimates, s);
}

}  // namespace

extern "C" {

ll_status ll_logdet_batched(ll_handle* h, const ll_csr* mats, const ll_bounds* bnd, int count, const ll_options* opts,
                            const int* degrees, double* estimates, void* stream) {
    if (!h || !opts || count < 0 || (count > 0 && (!mats || !bnd || !estimates))) return LL_ERR_INVALID_ARG;
    if (count == 0) return LL_OK;
    const ll_options& o = *opts;
    BatchCfg cfg;
    if (o.step_kernel == LL_KERNEL_GATHER) cfg.kernel = LL_KERNEL_GATHER;
    if (o.step_kernel != LL_KERNEL_AUTO) {
        const ll_status st = batched_run(h, mats, bnd, count, opts, degrees, estimates, stream, cfg);
        h->info.batch_tuned = 0;
        return st;
    }
    // LL_KERNEL_AUTO: the first call for a batch shape times the candidate launch shapes (the TMA
    // kernel with 512, 384 and 256 consumer threads per pass, and the register kernel) on the real
    // operands, picks the fastest pass 1 and pass 2 shapes, and caches them on the handle
    int64_t ntot = 0, nnztot = 0;
    int maxdeg = 0;
    for (int i = 0; i < count; ++i) {
        ntot += mats[i].n;
        nnztot += mats[i].nnz;
        if (degrees) maxdeg = std::max(maxdeg, degrees[i]);
    }
    const auto key = std::make_tuple(o.precision, count, o.probes / 3, ntot, nnztot, maxdeg);
    auto it = h->tuned_batch.find(key);
    if (it == h->tuned_batch.end()) {
        const int cand[3] = {512, 384, 256};
        float best1 = 0.f, best2 = 0.f, best_tma = 0.f;
        int t1 = 512, t2 = 512;
        bool have = false;
        for (int c : cand) {
            BatchCfg x;
            x.threads1 = x.threads2 = c;
            x.graph = false;
            ll_status st = batched_run(h, mats, bnd, count, opts, degrees, estimates, stream, x);
            if (st != LL_OK) return st;
            if (h->gbat.kernel != LL_KERNEL_TMA) break;   // no TMA layout fits: the register kernel ran
            const float p1 = h->info.ms_pass1, p2 = h->info.ms_pass2;
            if (!have || p1 < best1) { best1 = p1; t1 = c; }
            if (!have || p2 < best2) { best2 = p2; t2 = c; }
            have = true;
        }
        best_tma = best1 + best2;
        BatchCfg g;
        g.kernel = LL_KERNEL_GATHER;
        g.graph = false;
        ll_status st = batched_run(h, mats, bnd, count, opts, degrees, estimates, stream, g);
        if (st != LL_OK) return st;
        const float pg = h->info.ms_pass1 + h->info.ms_pass2;
        const int kern = (have && best_tma <= pg) ? LL_KERNEL_TMA : LL_KERNEL_GATHER;
        it = h->tuned_batch.emplace(key, std::make_tuple(kern, t1, t2)).first;
    }
    cfg.kernel = std::get<0>(it->second);
    cfg.threads1 = std::get<1>(it->second);
    cfg.threads2 = std::get<2>(it->second);
    const ll_status st = batched_run(h, mats, bnd, count, opts, degrees, estimates, stream, cfg);
    h->info.batch_tuned = 1;
    return st;
}

ll_status ll_gram(ll_handle* h, int layout, const void* X, int64_t ldx, int kx, const double* Z, int64_t ldz, int kz,
                  int64_t n, int method, double* out, void* stream) {
    if (!h) return LL_ERR_INVALID_ARG;
    if (layout != LL_PREC_F64 && layout != LL_PREC_DF64) return fail(h, LL_ERR_INVALID_ARG, "layout must be LL_PREC_F64 or LL_PREC_DF64");
    if (method < LL_GRAM_AUTO || method > LL_GRAM_DFLOAT) return fail(h, LL_ERR_INVALID_ARG, "unknown Gram method");
    const bool sym = Z == nullptr;
    if (sym) kz = kx, ldz = 0;
    if (n < 0 || kx < 1 || kz < 1 || kx > 96 || kz > 96 || ldx < kx || (!sym && ldz < kz)) return fail(h, LL_ERR_INVALID_ARG, "bad Gram shape");
    if (layout == LL_PREC_DF64 && (ldx & 1)) return fail(h, LL_ERR_INVALID_ARG, "double-float column pairs need an even ldx");
    if (n >= ((int64_t)1 << 31)) return fail(h, LL_ERR_UNSUPPORTED, "n must be < 2^31");
    if (!out || (n > 0 && !X)) return fail(h, LL_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        LL_CK(cudaMemsetAsync(out, 0, (size_t)kx * kz * sizeof(double), s));
        return LL_OK;
    }
    const int tx = layout == LL_PREC_F64 ? T_F64 : T_DF64;
    const int ggrid = h->sm_count * 2;
    WS(part, double*, "gram_partials", gram_partials_any(h, kx, kz, sym, ggrid) * sizeof(double));
    WS(tick, unsigned int*, "gram_ticket", sizeof(unsigned int));
    WS(err, int*, "tma_error", sizeof(int));
    LL_CK(cudaMemsetAsync(tick, 0, sizeof(unsigned int), s));
    LL_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    h->gram_method = method;
    h->launches = 0;
    ll_status st = run_gram(h, tx, X, ldx, kx, Z, ldz, kz, (int)n, sym, part, tick, out, ggrid, s);
    h->gram_method = LL_GRAM_AUTO;
    if (st != LL_OK) return st;
    h->tma_used = true;
    return check_tma_flag(h, s);
}

}  // extern "C"

// One pass of a sweep (MODE_ACCUM_SWEEP or MODE_DOT_SWEEP) over t groups of gw columns, sorted by
// degree (deg[0] >= deg[1] >= ...). Every block stacks the groups' n x gw blocks (group g's rows at
// g n, leading dimension gw: W_0 = win0, the ping-pong pair wa / wb, P); step j runs on the groups
// with deg[g] > j, the first ones of the stack, through a TMA plan for that many groups
// (re-planned, with its tile descriptors, where the count drops). vals: the t matrices' prepared
// values, group g's at g * O->nnz; dots: (deg[0] + 1) x (t gw) traces, column g gw + c for group
// g; tab / tab_df: SWEEP_SCALARS per group for every step (device, t * SWEEP_SCALARS per step).
// The launch shape (CTA size, column pairs per thread) is timed on all t groups once per
// (precision, mode, n, nnz, t gw) and cached on the handle.
ll_status run_sweep_pass(ll_handle* h, const ll_csr* O, const void* vals, int prec, int mode, int n, int t, int gw,
                         const std::vector<int>& deg, const void* win0, void* wa, void* wb, void* P, double* dots,
                         const double* tab, const float2* tab_df, int threads, int rpt, cudaStream_t s) {
    const int mmax = deg[0];
    const long long dld = (long long)t * gw;   // columns of a row of dots
    StepParams p{};
    p.rowptr = O->rowptr;
    p.colind = O->colind;
    p.vals = vals;
    p.ldw = gw;
    p.ldv = gw;
    p.ldp = gw;
    p.p = P;
    p.sw_gpairs = gw / 2;
    p.sw_vstride = O->nnz;
    if (base_mode(mode) == MODE_DOT) {
        WS(ticket, unsigned int*, "dot_ticket", sizeof(unsigned int));
        LL_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
        p.ticket = ticket;
        p.v = win0;
    }
    {
        WS(err, int*, "tma_error", sizeof(int));
        LL_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    }
    ll_status st;
    const int bfull = t * gw;
    if (threads <= 0 && rpt <= 0) {
        const auto key = std::make_tuple(prec, mode, n, O->nnz, bfull, (long long)gw);
        auto it = h->tuned.find(key);
        if (it != h->tuned.end()) {
            threads = std::get<1>(it->second);
            rpt = std::get<2>(it->second);
        } else {
            // a representative non-first step on all groups (its outputs are overwritten by the pass)
            const int jt = mmax > 1 ? 1 : 0;
            p.win = win0;
            p.wout = wa;
            p.first = 0;
            p.sw_scal = tab + (size_t)jt * t * SWEEP_SCALARS;
            p.sw_scal_df = tab_df + (size_t)jt * t * SWEEP_SCALARS;
            if (base_mode(mode) == MODE_DOT) {
                p.dots_next = dots + (size_t)(jt + 1) * dld;
                p.dots_first = dots;
            }
            const int cands[4][2] = {{512, 0}, {256, 0}, {512, 2}, {256, 2}};
            float best_ms = 0.f;
            bool have = false;
            for (const auto& c : cands) {
                StepParams q = p;
                StepExec C;
                if (!plan_exec(h, LL_KERNEL_TMA, prec, mode, n, O->nnz, bfull, c[0], c[1], q, C)) continue;
                if ((st = bind_exec(h, prec, mode, bfull, C, q, s)) != LL_OK) return st;
                LL_CK(exec_step(h, prec, mode, C, q, s));
                LL_CK(cudaEventRecord(h->ev[6], s));
                LL_CK(exec_step(h, prec, mode, C, q, s));
                LL_CK(exec_step(h, prec, mode, C, q, s));
                LL_CK(cudaEventRecord(h->ev[7], s));
                LL_CK(cudaEventSynchronize(h->ev[7]));
                if ((st = check_tma_flag(h, s)) != LL_OK) return st;
                float ms = 0.f;
                LL_CK(cudaEventElapsedTime(&ms, h->ev[6], h->ev[7]));
                if (!have || ms < best_ms) {
                    best_ms = ms;
                    threads = c[0];
                    rpt = c[1];
                    have = true;
                }
            }
            if (!have) return fail(h, LL_ERR_UNSUPPORTED, "sweep: no TMA step plan fits the block");
            h->tuned[key] = std::make_tuple((int)LL_KERNEL_TMA, threads, rpt);
        }
    }
    StepExec E;
    int act = -1;
    for (int j = 0; j < mmax; ++j) {
        int a = 0;
        while (a < t && deg[a] > j) ++a;
        if (a != act) {
            StepParams q = p;
            // two pairs per thread need an even number of pairs per group: otherwise one pair
            if (!plan_exec(h, LL_KERNEL_TMA, prec, mode, n, O->nnz, a * gw, threads, rpt, q, E)) {
                q = p;
                if (!plan_exec(h, LL_KERNEL_TMA, prec, mode, n, O->nnz, a * gw, threads, 0, q, E))
                    return fail(h, LL_ERR_UNSUPPORTED, "sweep: no TMA step plan fits the block");
            }
            p = q;
            if ((st = bind_exec(h, prec, mode, a * gw, E, p, s)) != LL_OK) return st;
            if (act < 0) {
                h->last_kernel = E.kind;
                h->last_threads = E.cta();
                h->last_np = E.tl.np;
                h->last_rows = E.tl.q.R;
            }
            act = a;
        }
        p.win = j == 0 ? win0 : ((j & 1) ? wa : wb);
        p.wout = (j & 1) ? wb : wa;
        p.first = j == 0;
        p.sw_scal = tab + (size_t)j * t * SWEEP_SCALARS;
        p.sw_scal_df = tab_df + (size_t)j * t * SWEEP_SCALARS;
        if (base_mode(mode) == MODE_DOT) {
            p.dots_next = dots + (size_t)(j + 1) * dld;
            p.dots_first = dots;
        }
        p.jnext = j + 1;
        LL_CK(exec_step(h, prec, mode, E, p, s));
    }
    return LL_OK;
}

extern "C" {

ll_status ll_logdet_sweep(ll_handle* h, const ll_csr* O, const double* D, int t, const double* thetas,
                          const ll_bounds* bounds, const int* degrees, const ll_options* opts, double* estimates,
                          void* stream) {
    if (!h || !opts || !estimates || !thetas || !bounds || t < 1) return LL_ERR_INVALID_ARG;
    ll_status st = check_csr_args(h, O);
    if (st != LL_OK) return st;
    const ll_options& o = *opts;
    if (o.estimator != LL_EST_HUTCHPP && o.estimator != LL_EST_HUTCHINSON) return fail(h, LL_ERR_INVALID_ARG, "unknown estimator");
    const bool hutch = o.estimator == LL_EST_HUTCHINSON;
    if (hutch ? o.probes <= 0 : (o.probes <= 0 || o.probes % 3 != 0))
        return fail(h, LL_ERR_INVALID_ARG, hutch ? "probes must be positive" : "probes must be a positive multiple of 3");
    if (o.probe_kind != LL_PROBE_RADEMACHER && o.probe_kind != LL_PROBE_GAUSSIAN) return fail(h, LL_ERR_INVALID_ARG, "unknown probe kind");
    if (o.precision < LL_PREC_F64 || o.precision > LL_PREC_F32_MIXED) return fail(h, LL_ERR_INVALID_ARG, "unknown precision");
    if (o.sval_mode != LL_SVAL_CENTER && o.sval_mode != LL_SVAL_HALF_LMAX) return fail(h, LL_ERR_INVALID_ARG, "unknown s_val mode");
    if (o.dd_scheme != LL_DD_AUTO && o.dd_scheme != LL_DD_TABLE_Q) return fail(h, LL_ERR_INVALID_ARG, "unknown divided-difference scheme");
    if (o.qr_gram < LL_GRAM_AUTO || o.qr_gram > LL_GRAM_DFLOAT) return fail(h, LL_ERR_INVALID_ARG, "unknown Gram method");
    if (o.tol != 0.0 || o.keep_for_backward)
        return fail(h, LL_ERR_UNSUPPORTED, "a sweep runs fixed degrees (tol = 0) and keeps nothing for a backward");
    if (o.step_kernel != LL_KERNEL_AUTO && o.step_kernel != LL_KERNEL_TMA)
        return fail(h, LL_ERR_UNSUPPORTED, "a sweep runs on the TMA step kernel");
    for (int g = 0; g < t; ++g) {
        if (!std::isfinite(thetas[g])) return fail(h, LL_ERR_INVALID_ARG, "non-finite theta");
        if ((st = check_bounds(h, bounds[g])) != LL_OK) return st;
        const int m = degrees ? degrees[g] : o.degree;
        if (m < 1) return fail(h, LL_ERR_INVALID_ARG, "degree must be >= 1");
    }
    cudaStream_t s = (cudaStream_t)stream;
    h->launches = 0;
    h->kept = false;
    h->have_forward = false;
    h->gram_method = o.qr_gram;
    h->spin_budget = o.timeout_cycles > 0 ? o.timeout_cycles : 4000000000LL;
    const int n = (int)O->n;
    if (n == 0) {
        for (int g = 0; g < t; ++g) estimates[g] = 0.0;
        return LL_OK;
    }
    if (!D) return fail(h, LL_ERR_INVALID_ARG, "null diagonal");
    const int kg = hutch ? o.probes : o.probes / 3;
    const int kq = hutch ? 0 : kg;
    const int b2 = kq + kg;
    if (!hutch && kq >= n) return fail(h, LL_ERR_UNSUPPORTED, "a sweep needs k < n");
    const int prec = o.precision;
    // group widths: whole 16-byte units of a W row (4 FP32 columns, 2 otherwise); every block stacks
    // the t groups' n x wg blocks (group g's rows from g n)
    const int al = prec == LL_PREC_F32_MIXED ? 4 : 2;
    const int wg1 = (kq + al - 1) / al * al, wg2 = (b2 + al - 1) / al * al;
    const long long L2 = (long long)t * wg2;   // columns of a row of the traces
    if (L2 > 1024 || kq > 96)
        return fail(h, LL_ERR_UNSUPPORTED, "a sweep takes at most 1024 trace columns (theta count x probe columns)");
    if ((long long)t * n >= (1LL << 31)) return fail(h, LL_ERR_UNSUPPORTED, "theta count x n must be < 2^31");
    if ((st = validate_csr(h, O, s)) != LL_OK) return st;

    // per theta: sigma, the scaled interval, Léja points, coefficients; groups by degree, descending
    struct Grp { int idx, m; double sigma, c, gamma; std::vector<double> xi, d; };
    std::vector<Grp> gs(t);
    for (int g = 0; g < t; ++g) {
        Grp& x = gs[g];
        x.idx = g;
        x.m = degrees ? degrees[g] : o.degree;
        x.sigma = sigma_of(bounds[g].lmin);
        const double lt = bounds[g].lmin / x.sigma, ut = bounds[g].lmax / x.sigma;
        if ((st = setup_coefficients(h, lt, ut, x.m, o.sval_mode, x.xi, x.d, o.dd_scheme)) != LL_OK) return st;
        x.c = (lt + ut) / 2.0;
        x.gamma = (ut - lt) / 4.0;
    }
    std::stable_sort(gs.begin(), gs.end(), [](const Grp& a, const Grp& b) { return a.m > b.m; });
    std::vector<int> deg(t);
    for (int g = 0; g < t; ++g) deg[g] = gs[g].m;
    const int mmax = deg[0];
    // step scalars of group g at step j: beta_{g,j} = -(c_g / gamma_g + xi_j), d_{g,j+1}, d_{g,0}
    // (B_g = (A_g / sigma_g - c_g I) / gamma_g, its values A_g / (sigma_g gamma_g) prepared below)
    std::vector<double> tab((size_t)mmax * t * SWEEP_SCALARS, 0.0);
    for (int j = 0; j < mmax; ++j)
        for (int g = 0; g < t; ++g) {
            const Grp& x = gs[g];
            if (j >= x.m) continue;
            double* e = &tab[((size_t)j * t + g) * SWEEP_SCALARS];
            e[0] = -(x.c / x.gamma + x.xi[j]);
            e[1] = x.d[j + 1];
            e[2] = x.d[0];
        }
    std::vector<float2> tab_df(tab.size());
    for (size_t x = 0; x < tab.size(); ++x) tab_df[x] = df_split(tab[x]);

    const int wt = w_type_of(prec), pt = p_type_of(prec);
    const size_t ew = elem_size(wt), ep = elem_size(pt);
    WS(vals, void*, "sw_vals", (size_t)t * O->nnz * ew);
    WS(vflag, int*, "sw_value_flag", sizeof(int));
    WS(dtab, double*, "sw_tab", tab.size() * sizeof(double));
    WS(dtab_df, float2*, "sw_tab_df", tab_df.size() * sizeof(float2));
    WS(G, double*, "sw_G", (size_t)n * kg * sizeof(double));
    const size_t blk1 = (size_t)n * wg1, blk2 = (size_t)n * wg2;   // elements of one group's block
    WS(wa, void*, "sw_wa", (size_t)t * blk2 * ew);
    WS(wb, void*, "sw_wb", (size_t)t * blk2 * ew);
    WS(V, void*, "sw_V", (size_t)t * blk2 * ew);
    WS(dots, double*, "sw_dots", (size_t)(mmax + 1) * L2 * sizeof(double));
    WS(qrstat, int*, "sw_qr_status", sizeof(int));
    WS(tma_err, int*, "tma_error", sizeof(int));
    void* S = nullptr;
    void* P = nullptr;
    void* q1 = nullptr;
    double* basis = nullptr;
    double* gpart = nullptr;
    unsigned int* gticket = nullptr;
    double* gram = nullptr;
    double* rinv1 = nullptr;
    double* rinv = nullptr;
    const int ggrid = h->sm_count * 2;
    if (!hutch) {
        WS(S_, void*, "sw_S", (size_t)t * blk1 * ew);
        WS(P_, void*, "sw_P", (size_t)t * blk1 * ep);
        WS(q1_, void*, "sw_q1", blk1 * sizeof(double));
        S = S_;
        P = P_;
        q1 = q1_;
        if (prec != LL_PREC_DF64) {
            WS(basis_, double*, "sw_basis", (size_t)t * blk2 * sizeof(double));
            basis = basis_;
        }
        const size_t gp1 = gram_partials_any(h, kq, kq, true, ggrid), gp2 = gram_partials_any(h, kq, kg, false, ggrid);
        WS(gpart_, double*, "sw_gram_partials", (gp1 > gp2 ? gp1 : gp2) * sizeof(double));
        WS(gticket_, unsigned int*, "sw_gram_ticket", sizeof(unsigned int));
        WS(gram_, double*, "sw_gram", (size_t)kq * kg * sizeof(double));
        WS(rinv1_, double*, "sw_rinv1", (size_t)kq * kq * sizeof(double));
        WS(rinv_, double*, "sw_rinv", (size_t)kq * kq * sizeof(double));
        gpart = gpart_;
        gticket = gticket_;
        gram = gram_;
        rinv1 = rinv1_;
        rinv = rinv_;
    }
    // the F64 mode's trace block is the FP64 basis itself
    if (prec == LL_PREC_F64 && !hutch) V = basis;

    LL_CK(cudaEventRecord(h->ev[0], s));
    LL_CK(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    LL_CK(cudaMemcpyAsync(dtab_df, tab_df.data(), tab_df.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    LL_CK(cudaMemsetAsync(qrstat, 0, sizeof(int), s));
    if (gticket) LL_CK(cudaMemsetAsync(gticket, 0, sizeof(unsigned int), s));
    // every group's matrix A_g = diag(D) + theta_g O, prepared as A_g / (sigma_g gamma_g)
    LL_CK(cudaMemsetAsync(vflag, 0, sizeof(int), s));
    for (int g = 0; g < t; ++g) {
        const Grp& x = gs[g];
        LL_CK(launch_prepare_pencil(O->rowptr, O->colind, O->values, O->dtype, D, n, thetas[x.idx],
                                    1.0 / (x.sigma * x.gamma), prec, static_cast<char*>(vals) + (size_t)g * O->nnz * ew,
                                    vflag, s));
        h->launches++;
    }
    // the same probes for every theta (common random numbers across the sweep): each group's
    // columns get the block ll_logdet_forward draws with this seed
    for (int g = 0; g < t; ++g) {
        if (hutch) {
            LL_CK(launch_probes(wt, o.probe_kind, o.seed, LL_STREAM_G, n, kg, wg2, static_cast<char*>(V) + g * blk2 * ew, wg2, s));
        } else {
            LL_CK(launch_probes(wt, o.probe_kind, o.seed, LL_STREAM_S, n, kq, wg1, static_cast<char*>(S) + g * blk1 * ew, wg1, s));
        }
        h->launches++;
    }
    if (!hutch) {
        LL_CK(launch_probes(T_F64, o.probe_kind, o.seed, LL_STREAM_G, n, kg, kg, G, kg, s));
        h->launches++;
    }
    LL_CK(cudaEventRecord(h->ev[1], s));
    int k1 = 0, t1 = 0, np1 = 1, rw1 = 0;
    if (!hutch) {
        // step 3 for every theta: Y_g = p_g(A_g~) S, then steps 4 and 6 per group
        st = run_sweep_pass(h, O, vals, prec, MODE_ACCUM_SWEEP, n, t, wg1, deg, S, wa, wb, P, nullptr, dtab, dtab_df,
                            o.threads_per_block, o.rows_per_thread, s);
        if (st != LL_OK) return st;
        k1 = h->last_kernel;
        t1 = h->last_threads;
        np1 = h->last_np;
        rw1 = h->last_rows;
        LL_CK(cudaEventRecord(h->ev[2], s));
        for (int g = 0; g < t; ++g) {
            const QrBlocks qb{static_cast<char*>(P) + g * blk1 * ep,
                              wg1,
                              q1,
                              wg1,
                              G,
                              static_cast<char*>(V) + g * blk2 * ew,
                              basis ? basis + g * blk2 : nullptr,
                              wg2,
                              wg2,
                              gpart,
                              gticket,
                              gram,
                              rinv1,
                              rinv,
                              qrstat,
                              ggrid};
            if ((st = qr_project(h, prec, n, kq, kg, qb, s)) != LL_OK) return st;
        }
    } else {
        LL_CK(cudaEventRecord(h->ev[2], s));
    }
    LL_CK(cudaEventRecord(h->ev[3], s));
    // steps 5-6 for every theta: traces t_j[col] = <V_col, W_j col>
    st = run_sweep_pass(h, O, vals, prec, MODE_DOT_SWEEP, n, t, wg2, deg, V, wa, wb, nullptr, dots, dtab, dtab_df,
                        o.threads_per_block, o.rows_per_thread, s);
    if (st != LL_OK) return st;
    LL_CK(cudaEventRecord(h->ev[4], s));

    std::vector<double> hd((size_t)(mmax + 1) * L2);
    int hstat = 0, herr = 0, hflag = 0;
    LL_CK(cudaMemcpyAsync(hd.data(), dots, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaMemcpyAsync(&hflag, vflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaMemcpyAsync(&hstat, qrstat, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaMemcpyAsync(&herr, tma_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LL_CK(cudaStreamSynchronize(s));
    h->tma_used = false;
    if (hflag) return fail(h, LL_ERR_INVALID_ARG, "O must store one diagonal entry in every row where D is non-zero");
    if (herr) return fail(h, LL_ERR_TIMEOUT, "step kernel: a bounded pipeline wait ran out");
    if (hstat) return fail(h, LL_ERR_QR_BREAKDOWN, "CholeskyQR2: non-positive pivot (rank-deficient sketch)");
    // step 7 per theta: n log sigma_g + tr(Q_g^T F_g Q_g) + (1/k) tr(G_g'^T F_g G_g')
    for (int g = 0; g < t; ++g) {
        const Grp& x = gs[g];
        const size_t c0 = (size_t)g * wg2;
        double tq = 0.0, tr = 0.0;
        for (int j = 0; j <= x.m; ++j) {
            double sq = 0.0, sr = 0.0;
            for (int col = 0; col < kq; ++col) sq += hd[(size_t)j * L2 + c0 + col];
            for (int col = kq; col < b2; ++col) sr += hd[(size_t)j * L2 + c0 + col];
            tq += x.d[j] * sq;
            tr += x.d[j] * sr;
        }
        tr /= (double)kg;
        if (!std::isfinite(tq) || !std::isfinite(tr)) return fail(h, LL_ERR_NONFINITE, "non-finite trace");
        estimates[x.idx] = (double)n * std::log(x.sigma) + tq + tr;
    }
    ll_info& I = h->info;
    I = ll_info{};
    I.k = kq;
    I.kernel_launches = h->launches;
    cudaEventElapsedTime(&I.ms_probes, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&I.ms_pass1, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&I.ms_qr, h->ev[2], h->ev[3]);
    cudaEventElapsedTime(&I.ms_pass2, h->ev[3], h->ev[4]);
    cudaEventElapsedTime(&I.ms_total, h->ev[0], h->ev[4]);
    I.kernel_pass1 = k1;
    I.threads_pass1 = t1;
    I.pairs_pass1 = np1;
    I.rows_pass1 = rw1;
    I.kernel_pass2 = h->last_kernel;
    I.threads_pass2 = h->last_threads;
    I.pairs_pass2 = h->last_np;
    I.rows_pass2 = h->last_rows;
    I.deg_max_pass1 = hutch ? 0 : mmax;
    I.deg_max_pass2 = mmax;
    double dsum = 0.0;
    for (int g = 0; g < t; ++g) dsum += deg[g];
    I.deg_mean_pass2 = dsum / t;
    return LL_OK;
}

ll_status ll_get_info(const ll_handle* h, ll_info* out) {
    if (!h || !out) return LL_ERR_INVALID_ARG;
    *out = h->info;
    return LL_OK;
}

ll_status ll_stop_degrees(const ll_handle* h, int pass, int* out, int cap, int* count) {
    if (!h || (pass != 1 && pass != 2) || cap < 0 || (cap > 0 && !out)) return LL_ERR_INVALID_ARG;
    if (!h->have_forward) return LL_ERR_NO_FORWARD;
    const std::vector<int>& v = pass == 1 ? h->last_deg1 : h->last_deg2;
    if (count) *count = (int)v.size();
    for (int i = 0; i < cap && i < (int)v.size(); ++i) out[i] = v[i];
    return LL_OK;
}

ll_status ll_kept_basis(const ll_handle* h, double* out, int64_t ld, int64_t* n_out, int* kq_out, int* kg_out,
                        void* stream) {
    if (!h) return LL_ERR_INVALID_ARG;
    if (!h->kept) return LL_ERR_NO_FORWARD;
    if (h->kept_hutch) return LL_ERR_UNSUPPORTED;   // no sketch basis in a Hutchinson forward
    auto it = h->ws.find("fw_basis");
    if (it == h->ws.end()) return LL_ERR_NO_FORWARD;
    const int b2 = h->kept_kq + h->kept_kg;
    const int l2 = block_ld(h->kept_prec, b2);
    if (n_out) *n_out = h->kept_n;
    if (kq_out) *kq_out = h->kept_kq;
    if (kg_out) *kg_out = h->kept_kg;
    if (!out) return LL_OK;
    if (ld < b2) return LL_ERR_INVALID_ARG;
    if (h->kept_prec != LL_PREC_F64) {
        // [Q | G'] is kept as double-float column pairs: in V (DF64) or in the basis block
        // (FP32-mixed)
        auto iv = h->ws.find(h->kept_prec == LL_PREC_DF64 ? "fw_V" : "fw_basis");
        if (iv == h->ws.end()) return LL_ERR_NO_FORWARD;
        cudaError_t e = launch_block_to_f64(h->kept_prec, iv->second.p, l2, out, ld, (int)h->kept_n, b2, (cudaStream_t)stream);
        return e == cudaSuccess ? LL_OK : LL_ERR_CUDA;
    }
    cudaError_t e = cudaMemcpy2DAsync(out, (size_t)ld * sizeof(double), it->second.p, (size_t)l2 * sizeof(double),
                                      (size_t)b2 * sizeof(double), (size_t)h->kept_n, cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream);
    return e == cudaSuccess ? LL_OK : LL_ERR_CUDA;
}

}  // extern "C"
