// ll_power_lmax_noalloc: the power-iteration lambda_max estimate without any device allocation.
//
// Some callers cannot allocate device memory themselves: code embedded in an application whose
// device memory is owned by another allocator (a framework's caching pool or a fixed arena that
// forbids raw cudaMalloc), and latency-sensitive callers that cannot accept the implicit device
// synchronisation of cudaMalloc/cudaFree. This entry point serves them: its working vectors,
// reduction partials, ticket and validation flag live in one file-scope device array that the
// library reserves when it is loaded.
//
// Contract:
//   * at most LL_NOALLOC_MAX_ROWS rows (the array holds two FP64 vectors of that length plus the
//     reduction scratch: 2 * 262,144 * 8 B + 32 KB, about 4.2 MB, held on every GPU that loads the
//     library until the process exits); larger matrices are rejected with LL_ERR_UNSUPPORTED, and
//     so are parts with more than 1024 SMs;
//   * the first call on a device looks up the array's device address (cudaGetSymbolAddress) with
//     that device current; make that first call before any stream capture;
//   * every call reuses the same array and leaves its last contents there; the ticket and the
//     validation flag are cleared at the start of each call. Calls that overlap on the GPU
//     (different streams, or different host threads on one device) race on the array;
//   * no cudaMalloc, cudaFree or allocating library routine is called.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "leja.h"

namespace ll {
namespace {

// The reduction kernels run 4 CTAs per SM, the grid of ll_power_lmax, so both entry points sum
// their partials in the same order on any part; the partials slot is sized for up to 1024 SMs.
constexpr int kNoAllocMaxSms = 1024;
constexpr int kNoAllocGrid = 4 * kNoAllocMaxSms;
// layout in doubles: x[MAX_ROWS] | y[MAX_ROWS] | partials[kNoAllocGrid] | nrm | ticket+flags
constexpr size_t kNoAllocDoubles = 2 * (size_t)LL_NOALLOC_MAX_ROWS + kNoAllocGrid + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace ll

extern "C" ll_status ll_power_lmax_noalloc(const ll_csr* A, int iters, uint64_t seed, double* lmax_out, void* stream) {
    using namespace ll;
    if (!A || !lmax_out || iters < 0) return LL_ERR_INVALID_ARG;
    if (A->n <= 0 || A->nnz < 0 || A->dtype < LL_F64 || A->dtype > LL_F32) return LL_ERR_INVALID_ARG;
    if (!A->rowptr || (A->nnz > 0 && (!A->colind || !A->values))) return LL_ERR_INVALID_ARG;
    if (A->n > LL_NOALLOC_MAX_ROWS || A->nnz >= ((int64_t)1 << 31)) return LL_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    double* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return LL_ERR_CUDA;
    const int n = (int)A->n;
    double* x = base;
    double* y = base + LL_NOALLOC_MAX_ROWS;
    double* partials = base + 2 * (size_t)LL_NOALLOC_MAX_ROWS;
    double* nrm = partials + kNoAllocGrid;
    unsigned int* ticket = reinterpret_cast<unsigned int*>(nrm + 2);
    int* flag = reinterpret_cast<int*>(nrm + 4);
    int sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LL_ERR_CUDA;
    }
    if (sms < 1 || sms > kNoAllocMaxSms) return LL_ERR_UNSUPPORTED;
    const int grid = 4 * sms;   // as ll_power_lmax

#define NA_CK(expr) do { if ((expr) != cudaSuccess) { cudaGetLastError(); return LL_ERR_CUDA; } } while (0)
    // start-of-call state: ticket and validation flags at zero
    NA_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
    NA_CK(cudaMemsetAsync(flag, 0, 2 * sizeof(int), s));
    NA_CK(launch_validate_csr(A->rowptr, A->colind, n, A->nnz, flag, s));
    int hflag[2] = {0, 0};
    NA_CK(cudaMemcpyAsync(hflag, flag, sizeof hflag, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (hflag[0]) return LL_ERR_BAD_CSR;
    // the same sequence of kernels as ll_power_lmax, on the static scratch
    NA_CK(launch_probes(T_F64, LL_PROBE_RADEMACHER, seed, LL_STREAM_POWER, n, 1, 1, x, 1, s));
    NA_CK(launch_dot_f64(x, x, n, partials, ticket, nrm, grid, s));
    NA_CK(launch_scale_f64(x, nrm, n, 0, s));
    for (int it = 0; it < iters; ++it) {
        NA_CK(launch_spmv_f64(A->rowptr, A->colind, A->values, A->dtype, n, x, y, s));
        NA_CK(launch_dot_f64(y, y, n, partials, ticket, nrm, grid, s));
        NA_CK(launch_scale_f64(y, nrm, n, 0, s));
        double* t = x; x = y; y = t;
    }
    NA_CK(launch_spmv_f64(A->rowptr, A->colind, A->values, A->dtype, n, x, y, s));
    NA_CK(launch_dot_f64(x, y, n, partials, ticket, nrm, grid, s));
    double hn = 0.0;
    NA_CK(cudaMemcpyAsync(&hn, nrm, sizeof hn, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
    *lmax_out = hn;
    return LL_OK;
}
