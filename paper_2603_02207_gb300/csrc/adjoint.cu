// Kernels of the adjoint (derivative of the frozen-basis estimator with respect to the stored
// values of A): the gradient contraction g_e += <Lambda_{j+1}[r_e, :], W_j[c_e, :]> (an SDDMM over
// the sparsity pattern), the initial Lambda_m = d_m U, the row index of every stored entry, and the
// chain to model parameters sum_e g_e da_e/dtheta_p.
#include "common.cuh"
#include "kernels.cuh"

namespace ll {

__global__ void k_row_index(const int32_t* rowptr, int n, int32_t* rowidx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) rowidx[e] = i;
}

cudaError_t launch_row_index(const int32_t* rowptr, int n, int32_t* rowidx, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_row_index<<<152 * 4, 256, 0, s>>>(rowptr, n, rowidx);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_scale_cols(const T* V, long long ld, int n, int b, int split, double cq, double cg, T* out) {
    const int bp = (int)ld;
    const long long total = (long long)n * bp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / bp), c = (int)(e - (long long)r * bp);
        const size_t i = (size_t)r * ld + c;
        const double v = c < b ? (c < split ? cq : cg) * load_f64<T>(V, i) : 0.0;
        store_f64<T>(out, i, v);
    }
}

cudaError_t launch_scale_cols(int precision, const void* V, long long ld, int n, int b, int split, double cq, double cg,
                              void* out, cudaStream_t s) {
    const int grid = 152 * 8, threads = 256;
    switch (w_type_of(precision)) {
        case T_F64: k_scale_cols<double><<<grid, threads, 0, s>>>((const double*)V, ld, n, b, split, cq, cg, (double*)out); break;
        case T_F32: k_scale_cols<float><<<grid, threads, 0, s>>>((const float*)V, ld, n, b, split, cq, cg, (float*)out); break;
        default: k_scale_cols<dfp><<<grid, threads, 0, s>>>((const dfp*)V, ld, n, b, split, cq, cg, (dfp*)out); break;
    }
    return cudaGetLastError();
}

// Warp-wide sum of a double-float value (TwoSum at every level), result in lane 0.
__device__ __forceinline__ void warp_df_sum(float& h, float& l) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, h, off);
        const float ol = __shfl_down_sync(0xffffffffu, l, off);
        const float s = __fadd_rn(h, oh);
        const float bb = __fsub_rn(s, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(oh, bb));
        h = s;
        l = __fadd_rn(l, __fadd_rn(ol, err));
    }
}

// One warp per row r: each lane holds column pairs of Lambda_{j+1}[r, :]; for every stored entry
// (r, c) the lanes multiply it with W_j[c, :] (coalesced pair loads), the warp sums, lane 0 adds
// scale * sum to g[e]. Double-float products and sums for the F32 and DF64 storage, FP64 for F64.
template <int PREC>
__global__ void __launch_bounds__(256) k_sddmm(const int32_t* rowptr, const int32_t* colind, int n, const void* lam_,
                                               const void* w_, long long ld, int b, double scale, double* g) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const long long ldq = ld >> 1;
    const int npairs = (b + 1) / 2;
    constexpr int MAXP = 4;   // pairs per lane (b <= 256)
    for (int r = warp; r < n; r += nwarps) {
        const int e0 = rowptr[r], e1 = rowptr[r + 1];
        if (e0 == e1) continue;
        if constexpr (PREC == LL_PREC_F64) {
            const double2* lam = static_cast<const double2*>(lam_);
            const double2* w = static_cast<const double2*>(w_);
            double2 lr[MAXP];
#pragma unroll
            for (int q = 0; q < MAXP; ++q) {
                const int pq = lane + 32 * q;
                lr[q] = pq < npairs ? lam[(size_t)r * ldq + pq] : make_double2(0.0, 0.0);
            }
            for (int e = e0; e < e1; ++e) {
                const size_t cb = (size_t)colind[e] * ldq;
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < MAXP; ++q) {
                    const int pq = lane + 32 * q;
                    if (pq < npairs) {
                        const double2 x = w[cb + pq];
                        acc = fma(lr[q].x, x.x, acc);
                        acc = fma(lr[q].y, x.y, acc);
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
                if (lane == 0) g[e] += scale * acc;
            }
        } else if constexpr (PREC == LL_PREC_DF64) {
            const ulonglong2* lam = static_cast<const ulonglong2*>(lam_);
            const ulonglong2* w = static_cast<const ulonglong2*>(w_);
            ulonglong2 lr[MAXP];
            f2x nlh[MAXP];
#pragma unroll
            for (int q = 0; q < MAXP; ++q) {
                const int pq = lane + 32 * q;
                lr[q] = pq < npairs ? lam[(size_t)r * ldq + pq] : make_ulonglong2(0ull, 0ull);
                nlh[q] = f2_sub(0ull, lr[q].x);
            }
            for (int e = e0; e < e1; ++e) {
                const size_t cb = (size_t)colind[e] * ldq;
                f2x sh = 0ull, sl = 0ull;
#pragma unroll
                for (int q = 0; q < MAXP; ++q) {
                    const int pq = lane + 32 * q;
                    if (pq < npairs) {
                        const ulonglong2 x = w[cb + pq];
                        df2_mac_pp(sh, sl, lr[q].x, lr[q].y, nlh[q], x.x, x.y);
                    }
                }
                float h0, h1, l0, l1;
                f2_unpack(sh, h0, h1);
                f2_unpack(sl, l0, l1);
                float h = 0.f, l = 0.f;
                df_mac(h, l, h0, l0, 1.f, 0.f);
                df_mac(h, l, h1, l1, 1.f, 0.f);
                warp_df_sum(h, l);
                if (lane == 0) g[e] += scale * ((double)h + (double)l);
            }
        } else {  // LL_PREC_F32_MIXED
            const f2x* lam = static_cast<const f2x*>(lam_);
            const f2x* w = static_cast<const f2x*>(w_);
            f2x lr[MAXP], nlr[MAXP];
#pragma unroll
            for (int q = 0; q < MAXP; ++q) {
                const int pq = lane + 32 * q;
                lr[q] = pq < npairs ? lam[(size_t)r * ldq + pq] : 0ull;
                nlr[q] = f2_sub(0ull, lr[q]);
            }
            for (int e = e0; e < e1; ++e) {
                const size_t cb = (size_t)colind[e] * ldq;
                f2x sh = 0ull, sl = 0ull;
#pragma unroll
                for (int q = 0; q < MAXP; ++q) {
                    const int pq = lane + 32 * q;
                    if (pq < npairs) df2_mac_f(sh, sl, lr[q], 0ull, nlr[q], w[cb + pq]);
                }
                float h0, h1, l0, l1;
                f2_unpack(sh, h0, h1);
                f2_unpack(sl, l0, l1);
                float h = 0.f, l = 0.f;
                df_mac(h, l, h0, l0, 1.f, 0.f);
                df_mac(h, l, h1, l1, 1.f, 0.f);
                warp_df_sum(h, l);
                if (lane == 0) g[e] += scale * ((double)h + (double)l);
            }
        }
    }
}

cudaError_t launch_sddmm(int precision, const int32_t* rowptr, const int32_t* colind, int n, const void* lam,
                         const void* w, long long ld, int b, double scale, double* g, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (b > 256) return cudaErrorInvalidValue;
    const int threads = 256;
    const int grid = 152 * 8;
    switch (precision) {
        case LL_PREC_F64: k_sddmm<LL_PREC_F64><<<grid, threads, 0, s>>>(rowptr, colind, n, lam, w, ld, b, scale, g); break;
        case LL_PREC_DF64: k_sddmm<LL_PREC_DF64><<<grid, threads, 0, s>>>(rowptr, colind, n, lam, w, ld, b, scale, g); break;
        default: k_sddmm<LL_PREC_F32_MIXED><<<grid, threads, 0, s>>>(rowptr, colind, n, lam, w, ld, b, scale, g); break;
    }
    return cudaGetLastError();
}

// out[p] = sum_e g[e] * dv[p * ldd + e]: per-CTA partials, reduced in a fixed order by the last CTA.
__global__ void k_param_dot(const double* g, const double* dv, long long ldd, int64_t nnz, int np, double* partials,
                            unsigned int* ticket, double* out) {
    __shared__ double red[256];
    __shared__ bool s_last;
    for (int p = 0; p < np; ++p) {
        double acc = 0.0;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
            acc = fma(g[e], dv[(size_t)p * ldd + e], acc);
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)p * gridDim.x + blockIdx.x] = red[0];
        __syncthreads();
    }
    __threadfence();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            double t = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&partials[(size_t)p * gridDim.x + b]);
            out[p] = t;
        }
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

cudaError_t launch_param_dot(const double* g, const double* dv, long long ldd, int64_t nnz, int np, double* partials,
                             unsigned int* ticket, double* out, int grid, cudaStream_t s) {
    k_param_dot<<<grid, 256, 0, s>>>(g, dv, ldd, nnz, np, partials, ticket, out);
    return cudaGetLastError();
}

}  // namespace ll
