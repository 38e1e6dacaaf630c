// Tall-skinny QR of the Hutch++ sketch by CholeskyQR2, and the deflation of the residual probes
// (Algorithm 3 steps 4 and 6: Q = orth(Y), G' = G - Q (Q^T G)). FP64 arithmetic throughout.
//   Gram:   X^T Z over n rows, per-CTA partials reduced by the last CTA in a fixed order;
//   chol:   G = R^T R (upper R) and R^{-1} in one CTA, with a breakdown flag;
//   apply:  X R^{-1} row by row (R^{-1} in shared memory);
//   project: G - Q C row by row (C in shared memory).
#include "common.cuh"
#include "kernels.cuh"

namespace ll {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_E = 8;       // entries per thread per CTA
constexpr int GRAM_TR = 16;     // rows per shared tile

template <typename TX, typename TZ>
__global__ void __launch_bounds__(GRAM_THREADS) k_gram(const TX* X, long long ldx, int kx, const TZ* Z, long long ldz, int kz,
                                                       int n, int sym, double* partials, unsigned int* ticket, double* out) {
    extern __shared__ __align__(16) double sg[];
    double* xs = sg;                       // GRAM_TR x kx
    double* zs = sg + GRAM_TR * kx;        // GRAM_TR x kz
    __shared__ bool s_last;
    const int count = sym ? kx * (kx + 1) / 2 : kx * kz;
    const int chunk0 = blockIdx.y * GRAM_THREADS * GRAM_E;
    int ea[GRAM_E], ec[GRAM_E];
    double acc[GRAM_E];
#pragma unroll
    for (int q = 0; q < GRAM_E; ++q) {
        const int e = chunk0 + q * GRAM_THREADS + threadIdx.x;
        acc[q] = 0.0;
        ea[q] = -1; ec[q] = 0;
        if (e < count) {
            if (sym) {
                int a = 0, rem = e;
                while (rem >= kx - a) { rem -= kx - a; ++a; }
                ea[q] = a; ec[q] = a + rem;
            } else {
                ea[q] = e / kz; ec[q] = e - (e / kz) * kz;
            }
        }
    }
    const int ntiles = (n + GRAM_TR - 1) / GRAM_TR;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * GRAM_TR;
        const int rows = min(GRAM_TR, n - r0);
        for (int i = threadIdx.x; i < GRAM_TR * kx; i += blockDim.x) {
            const int rr = i / kx, c = i - rr * kx;
            xs[i] = rr < rows ? load_f64<TX>(X, (size_t)(r0 + rr) * ldx + c) : 0.0;
        }
        if (!sym) {
            for (int i = threadIdx.x; i < GRAM_TR * kz; i += blockDim.x) {
                const int rr = i / kz, c = i - rr * kz;
                zs[i] = rr < rows ? load_f64<TZ>(Z, (size_t)(r0 + rr) * ldz + c) : 0.0;
            }
        }
        __syncthreads();
        const double* zsrc = sym ? xs : zs;
        const int ldzs = sym ? kx : kz;
#pragma unroll
        for (int q = 0; q < GRAM_E; ++q) {
            if (ea[q] >= 0) {
                double s = acc[q];
                for (int rr = 0; rr < GRAM_TR; ++rr) s = fma(xs[rr * kx + ea[q]], zsrc[rr * ldzs + ec[q]], s);
                acc[q] = s;
            }
        }
        __syncthreads();
    }
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int q = 0; q < GRAM_E; ++q) {
        const int e = chunk0 + q * GRAM_THREADS + threadIdx.x;
        if (e < count) partials[(size_t)blockIdx.x * count + e] = acc[q];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)nblk - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int e = threadIdx.x; e < count; e += blockDim.x) {
            double s = 0.0;
            for (int g = 0; g < (int)gridDim.x; ++g) s += __ldcg(&partials[(size_t)g * count + e]);
            if (sym) {
                int a = 0, rem = e;
                while (rem >= kx - a) { rem -= kx - a; ++a; }
                const int c = a + rem;
                out[a * kx + c] = s;
                out[c * kx + a] = s;
            } else {
                out[e] = s;
            }
        }
        if (threadIdx.x == 0) *ticket = 0u;
    }
    (void)bid;
}

template <typename TX, typename TZ>
static cudaError_t gram_typed(const void* X, long long ldx, int kx, const void* Z, long long ldz, int kz, int n, bool sym,
                              double* partials, unsigned int* ticket, double* out, int grid, cudaStream_t s) {
    const int count = sym ? kx * (kx + 1) / 2 : kx * kz;
    const int chunks = (count + GRAM_THREADS * GRAM_E - 1) / (GRAM_THREADS * GRAM_E);
    const size_t smem = (size_t)GRAM_TR * (kx + (sym ? 0 : kz)) * sizeof(double);
    dim3 g(grid, chunks);
    k_gram<TX, TZ><<<g, GRAM_THREADS, smem, s>>>((const TX*)X, ldx, kx, (const TZ*)Z, ldz, kz, n, sym ? 1 : 0, partials, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_gram(int tx, const void* X, long long ldx, int kx, int tz, const void* Z, long long ldz, int kz,
                        int n, bool sym, double* partials, unsigned int* ticket, double* out, int grid, cudaStream_t s) {
    if (tz != T_F64) return cudaErrorInvalidValue;
    switch (tx) {
        case T_F64: return gram_typed<double, double>(X, ldx, kx, Z, ldz, kz, n, sym, partials, ticket, out, grid, s);
        case T_F32: return gram_typed<float, double>(X, ldx, kx, Z, ldz, kz, n, sym, partials, ticket, out, grid, s);
        default: return gram_typed<float2, double>(X, ldx, kx, Z, ldz, kz, n, sym, partials, ticket, out, grid, s);
    }
}

// ---------------------------------------------------------------- Cholesky + triangular inverse
__global__ void k_chol_rinv(const double* G, int k, double* Rinv, int* status) {
    extern __shared__ __align__(16) double sc[];
    double* a = sc;            // k x k working copy; its upper triangle becomes R
    double* ri = sc + k * k;   // k x k R^{-1}
    __shared__ double s_piv;
    __shared__ int s_bad;
    __shared__ double s_maxdiag;
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) { a[i] = G[i]; ri[i] = 0.0; }
    if (threadIdx.x == 0) {
        s_bad = 0;
        double md = 0.0;
        for (int j = 0; j < k; ++j) md = fmax(md, G[j * k + j]);
        s_maxdiag = md;
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            const double d = a[j * k + j];
            if (!(d > 1e-14 * s_maxdiag)) { s_bad = 1; s_piv = 1.0; }
            else s_piv = sqrt(d);
            a[j * k + j] = s_piv;
        }
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < k; c += blockDim.x) a[j * k + c] /= s_piv;
        __syncthreads();
        const int m = k - j - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int r = j + 1 + idx / m, c = j + 1 + idx % m;
            if (c >= r) a[r * k + c] -= a[j * k + r] * a[j * k + c];
        }
        __syncthreads();
    }
    // R^{-1}: column c solved by back substitution
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        ri[c * k + c] = 1.0 / a[c * k + c];
        for (int i = c - 1; i >= 0; --i) {
            double s = 0.0;
            for (int l = i + 1; l <= c; ++l) s = fma(a[i * k + l], ri[l * k + c], s);
            ri[i * k + c] = -s / a[i * k + i];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) Rinv[i] = ri[i];
    if (threadIdx.x == 0 && s_bad) *status = 1;
}

cudaError_t launch_chol_rinv(const double* G, int k, double* Rinv, int* status, cudaStream_t s) {
    const size_t smem = (size_t)2 * k * k * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_chol_rinv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_chol_rinv<<<1, 256, smem, s>>>(G, k, Rinv, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- row-wise small products
// mode 0: out[r, col] = sum_{a <= col} X[r, a] M[a, col]           (X R^{-1}, M upper triangular)
// mode 1: out[r, col] = G[r, col] - sum_{a < kx} X[r, a] M[a, col]  (G - Q C)
template <typename TX, typename T2, int MODE>
__global__ void k_rowprod(const TX* X, long long ldx, int kx, const double* M, int kc, const double* G, long long ldg,
                          int n, int rl, double* out64, long long ld64, T2* out2, long long ld2) {
    extern __shared__ __align__(16) double sm[];   // kx x kc
    for (int i = threadIdx.x; i < kx * kc; i += blockDim.x) sm[i] = M[i];
    __syncthreads();
    const int rlane = threadIdx.x / kc;
    const int col = threadIdx.x - rlane * kc;
    if (rlane >= rl) return;
    for (int r = blockIdx.x * rl + rlane; r < n; r += gridDim.x * rl) {
        const size_t xo = (size_t)r * ldx;
        double s = 0.0;
        const int amax = (MODE == 0) ? col + 1 : kx;
        for (int a = 0; a < amax; ++a) s = fma(load_f64<TX>(X, xo + a), sm[a * kc + col], s);
        const double v = (MODE == 0) ? s : G[(size_t)r * ldg + col] - s;
        out64[(size_t)r * ld64 + col] = v;
        if (out2) store_f64<T2>(out2, (size_t)r * ld2 + col, v);
    }
}

template <typename TX, int MODE>
static cudaError_t rowprod_dispatch(int t2, const TX* X, long long ldx, int kx, const double* M, int kc, const double* G,
                                    long long ldg, int n, double* out64, long long ld64, void* out2, long long ld2, cudaStream_t s) {
    int rl = 256 / kc;
    if (rl < 1) rl = 1;
    const int threads = ((rl * kc + 31) / 32) * 32;
    int blocks = (n + rl - 1) / rl;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) return cudaSuccess;
    const size_t smem = (size_t)kx * kc * sizeof(double);
    switch (t2) {
        case T_F32:
            cudaFuncSetAttribute(k_rowprod<TX, float, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            k_rowprod<TX, float, MODE><<<blocks, threads, smem, s>>>(X, ldx, kx, M, kc, G, ldg, n, rl, out64, ld64, (float*)out2, ld2);
            break;
        case T_DF64:
            cudaFuncSetAttribute(k_rowprod<TX, float2, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            k_rowprod<TX, float2, MODE><<<blocks, threads, smem, s>>>(X, ldx, kx, M, kc, G, ldg, n, rl, out64, ld64, (float2*)out2, ld2);
            break;
        default:
            cudaFuncSetAttribute(k_rowprod<TX, double, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            k_rowprod<TX, double, MODE><<<blocks, threads, smem, s>>>(X, ldx, kx, M, kc, G, ldg, n, rl, out64, ld64, (double*)out2, ld2);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_apply_rinv(int tx, const void* X, long long ldx, int n, int k, const double* Rinv,
                              double* out64, long long ld64, int t2, void* out2, long long ld2, cudaStream_t s) {
    switch (tx) {
        case T_F64: return rowprod_dispatch<double, 0>(t2, (const double*)X, ldx, k, Rinv, k, nullptr, 0, n, out64, ld64, out2, ld2, s);
        case T_F32: return rowprod_dispatch<float, 0>(t2, (const float*)X, ldx, k, Rinv, k, nullptr, 0, n, out64, ld64, out2, ld2, s);
        default: return rowprod_dispatch<float2, 0>(t2, (const float2*)X, ldx, k, Rinv, k, nullptr, 0, n, out64, ld64, out2, ld2, s);
    }
}

cudaError_t launch_project(const double* Q, long long ldq, int k, const double* G, long long ldg, int kg,
                           const double* C, int n, double* out64, long long ld64, int t2, void* out2,
                           long long ld2, cudaStream_t s) {
    return rowprod_dispatch<double, 1>(t2, Q, ldq, k, C, kg, G, ldg, n, out64, ld64, out2, ld2, s);
}

}  // namespace ll
