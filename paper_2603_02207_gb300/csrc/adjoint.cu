// Kernels of the adjoint (derivative of the frozen-basis estimator with respect to the stored
// values of A): the gradient contraction g_e += <Lambda_{j+1}[r_e, :], W_j[c_e, :]> (an SDDMM over
// the sparsity pattern), the initial Lambda_m = d_m U, the row index of every stored entry, and the
// chain to model parameters sum_e g_e da_e/dtheta_p.
#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"

namespace ll {

__global__ void k_row_index(const int32_t* rowptr, int n, int32_t* rowidx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) rowidx[e] = i;
}

// tmap[e] = the index of entry (c, r) for every stored entry e = (r, c) of a pattern whose rows hold
// strictly increasing columns (binary search in row c); flag[0] |= 1 where (c, r) is not stored
__global__ void k_transpose_map(const int32_t* rowptr, const int32_t* colind, int n, int32_t* tmap, int* flag) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const int c = colind[e];
            int lo = rowptr[c], hi = rowptr[c + 1];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (colind[mid] < r) lo = mid + 1; else hi = mid;
            }
            if (lo < rowptr[c + 1] && colind[lo] == r) {
                tmap[e] = lo;
            } else {
                tmap[e] = e;
                atomicOr(flag, 1);
            }
        }
    }
}

cudaError_t launch_transpose_map(const int32_t* rowptr, const int32_t* colind, int n, int32_t* tmap, int* flag,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_transpose_map<<<152 * 8, 256, 0, s>>>(rowptr, colind, n, tmap, flag);
    return cudaGetLastError();
}

__global__ void k_gather_add(const int32_t* map, const double* src, int64_t nnz, double* dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] += src[map[e]];
}

cudaError_t launch_gather_add(const int32_t* map, const double* src, int64_t nnz, double* dst, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    k_gather_add<<<152 * 8, 256, 0, s>>>(map, src, nnz, dst);
    return cudaGetLastError();
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


// g[e] += scale * <Lambda_{j+1}[r_e, :], W_j[c_e, :]> for every stored entry e = (r_e, c_e): one
// thread per entry walks the column pairs of both rows (Lambda's row is shared by the entries of a
// row, so it is an L1 hit for all but the first) and accumulates in double-float (FP64 for F64),
// column pairs in order, the two lanes of a pair added at the end. Each g[e] is written by one
// thread: no reduction across threads, deterministic.
template <int PREC>
__global__ void __launch_bounds__(256) k_sddmm(const int32_t* rowidx, const int32_t* colind, int64_t nnz, const void* lam_,
                                               const void* w_, long long ld, int b, double scale, double* g) {
    const long long ldq = ld >> 1;
    const int npairs = (b + 1) / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const size_t rb = (size_t)rowidx[e] * ldq, cb = (size_t)colind[e] * ldq;
        double acc;
        if constexpr (PREC == LL_PREC_F64) {
            const double2* lam = static_cast<const double2*>(lam_) + rb;
            const double2* w = static_cast<const double2*>(w_) + cb;
            double a0 = 0.0, a1 = 0.0;
#pragma unroll 4
            for (int q = 0; q < npairs; ++q) {
                const double2 l = __ldg(&lam[q]), x = __ldg(&w[q]);
                a0 = fma(l.x, x.x, a0);
                a1 = fma(l.y, x.y, a1);
            }
            acc = a0 + a1;
        } else if constexpr (PREC == LL_PREC_DF64) {
            const ulonglong2* lam = static_cast<const ulonglong2*>(lam_) + rb;
            const ulonglong2* w = static_cast<const ulonglong2*>(w_) + cb;
            f2x sh = 0ull, sl = 0ull;
#pragma unroll 4
            for (int q = 0; q < npairs; ++q) {
                const ulonglong2 l = __ldg(&lam[q]), x = __ldg(&w[q]);
                df2_mac_pp(sh, sl, l.x, l.y, f2_sub(0ull, l.x), x.x, x.y);
            }
            float h0, h1, l0, l1;
            f2_unpack(sh, h0, h1);
            f2_unpack(sl, l0, l1);
            float h = 0.f, lo = 0.f;
            df_mac(h, lo, h0, l0, 1.f, 0.f);
            df_mac(h, lo, h1, l1, 1.f, 0.f);
            acc = (double)h + (double)lo;
        } else {  // LL_PREC_F32_MIXED: exact FP32 products accumulated in double-float
            const f2x* lam = static_cast<const f2x*>(lam_) + rb;
            const f2x* w = static_cast<const f2x*>(w_) + cb;
            f2x sh = 0ull, sl = 0ull;
#pragma unroll 4
            for (int q = 0; q < npairs; ++q) {
                const f2x l = __ldg(reinterpret_cast<const unsigned long long*>(&lam[q]));
                const f2x x = __ldg(reinterpret_cast<const unsigned long long*>(&w[q]));
                df2_mac_f(sh, sl, l, 0ull, f2_sub(0ull, l), x);
            }
            float h0, h1, l0, l1;
            f2_unpack(sh, h0, h1);
            f2_unpack(sl, l0, l1);
            float h = 0.f, lo = 0.f;
            df_mac(h, lo, h0, l0, 1.f, 0.f);
            df_mac(h, lo, h1, l1, 1.f, 0.f);
            acc = (double)h + (double)lo;
        }
        g[e] += scale * acc;
    }
}

cudaError_t launch_sddmm(int precision, const int32_t* rowidx, const int32_t* colind, int64_t nnz, const void* lam,
                         const void* w, long long ld, int b, double scale, double* g, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t grid = (nnz + threads - 1) / threads;
    if (grid > 152 * 16) grid = 152 * 16;
    switch (precision) {
        case LL_PREC_F64: k_sddmm<LL_PREC_F64><<<(int)grid, threads, 0, s>>>(rowidx, colind, nnz, lam, w, ld, b, scale, g); break;
        case LL_PREC_DF64: k_sddmm<LL_PREC_DF64><<<(int)grid, threads, 0, s>>>(rowidx, colind, nnz, lam, w, ld, b, scale, g); break;
        default: k_sddmm<LL_PREC_F32_MIXED><<<(int)grid, threads, 0, s>>>(rowidx, colind, nnz, lam, w, ld, b, scale, g); break;
    }
    return cudaGetLastError();
}

// P = sum_{j=0..m} d_j W_j for the first npairs column pairs of W_0 (w0) and W_1 .. W_m
// (consecutive n x ld blocks, blk bytes apart, from wk), by the P-axpy step epilogue's operations
// in its order: d_0 W_0 and d_1 W_1 accumulated and renormalised, then one accumulation and one
// renormalisation per further step. P therefore equals the P-axpy pass over the same W_j bit for
// bit. d: FP64 coefficients, ddf: their double-float splits (device, m + 1 each).
template <int PREC>
__global__ void k_weighted_sum(const void* w0, const char* wk, size_t blk, long long ld, int n, int npairs, int m,
                               const double* d, const float2* ddf, void* P, long long ldp) {
    using WP = typename PairT<PREC>::W;
    using PP = typename PairT<PREC>::P;
    const long long ldq = ld >> 1, ldpq = ldp >> 1;
    const long long total = (long long)n * npairs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / npairs, q = e - r * npairs;
        const size_t off = (size_t)r * ldq + q;
        auto W = [&](int j) -> WP {
            const WP* b = j == 0 ? static_cast<const WP*>(w0) : reinterpret_cast<const WP*>(wk + (size_t)(j - 1) * blk);
            return b[off];
        };
        PP out;
        if constexpr (PREC == LL_PREC_F64) {
            const WP a = W(0), b = W(1);
            double p0 = fma(d[1], b.x, d[0] * a.x), p1 = fma(d[1], b.y, d[0] * a.y);
            for (int j = 2; j <= m; ++j) {
                const WP w = W(j);
                p0 = fma(d[j], w.x, p0);
                p1 = fma(d[j], w.y, p1);
            }
            out = make_double2(p0, p1);
        } else {
            f2x ph = 0ull, pl = 0ull;
            for (int j = 0; j <= m; ++j) {
                const float2 c = ddf[j];
                const f2x ch = f2_pack(c.x, c.x), cl = f2_pack(c.y, c.y), nch = f2_pack(-c.x, -c.x);
                const WP w = W(j);
                if constexpr (PREC == LL_PREC_DF64) df2_mac(ph, pl, ch, cl, nch, w.x, w.y);
                else df2_mac_f(ph, pl, ch, cl, nch, w);
                if (j >= 1) {   // the first step adds d_0 W_0 and d_1 W_1 before its renormalisation
                    f2x oh, ol;
                    df2_norm(ph, pl, oh, ol);
                    ph = oh;
                    pl = ol;
                }
            }
            out = make_ulonglong2(ph, pl);
        }
        static_cast<PP*>(P)[(size_t)r * ldpq + q] = out;
    }
}

cudaError_t launch_weighted_sum(int precision, const void* w0, const void* wk, size_t blk, long long ld, int n, int b,
                                int m, const double* d, const float2* ddf, void* P, long long ldp, cudaStream_t s) {
    if (n <= 0 || b <= 0 || m < 1) return cudaSuccess;
    const int npairs = (b + 1) / 2;
    const long long total = (long long)n * npairs;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    const char* k = static_cast<const char*>(wk);
    switch (precision) {
        case LL_PREC_F64: k_weighted_sum<LL_PREC_F64><<<grid, 256, 0, s>>>(w0, k, blk, ld, n, npairs, m, d, ddf, P, ldp); break;
        case LL_PREC_DF64: k_weighted_sum<LL_PREC_DF64><<<grid, 256, 0, s>>>(w0, k, blk, ld, n, npairs, m, d, ddf, P, ldp); break;
        default: k_weighted_sum<LL_PREC_F32_MIXED><<<grid, 256, 0, s>>>(w0, k, blk, ld, n, npairs, m, d, ddf, P, ldp); break;
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
