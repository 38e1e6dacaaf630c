// Probe generation, CSR validation, Gershgorin bounds, value preparation, block conversions and
// the FP64 pieces of the power iteration.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace ll {

// ---------------------------------------------------------------------------- probes (Alg. 3)
// A Rademacher value (+-1, or 0 in a pad column) stored without FP64 arithmetic: exact in every
// storage type, the double-float pair being (+-1, 0). Gaussian values go through store_f64.
__device__ __forceinline__ void store_sign(double* p, size_t i, float v) { p[i] = (double)v; }
__device__ __forceinline__ void store_sign(float* p, size_t i, float v) { p[i] = v; }
__device__ __forceinline__ void store_sign(dfp* p, size_t i, float v) {
    float* f = reinterpret_cast<float*>(p) + dfp_hi(i);
    f[0] = v;
    f[2] = 0.f;
}

// Narrow blocks (pad <= blockDim): thread t owns column t % pad of rows t / pad + k * (blockDim /
// pad) of the CTA's share. Wide blocks: a CTA takes one row at a time, its threads striding over
// the columns. 32-bit index arithmetic per element.
template <typename T>
__global__ void k_probes(int kind, uint64_t seed, int stream_id, int n, int cols, int pad, T* out, long long ld,
                         const int32_t* rowmap) {
    const int nt = (int)blockDim.x;
    const bool narrow = pad <= nt;
    const int rpb = narrow ? nt / pad : 1;                 // rows per CTA pass
    const int roff = narrow ? (int)threadIdx.x / pad : 0;
    const int col0 = (int)threadIdx.x - roff * (narrow ? pad : 0);
    const int cstep = narrow ? pad : nt;
    if (roff >= rpb) return;
    for (int row = blockIdx.x * rpb + roff; row < n; row += gridDim.x * rpb) {
        const uint32_t prow = (uint32_t)(rowmap ? rowmap[row] : row);   // the row whose probe values these are
        for (int col = col0; col < pad; col += cstep) {
            const size_t idx = (size_t)row * ld + col;
            if (kind == LL_PROBE_RADEMACHER) {
                const float v = col < cols ? ((probe_bits(seed, (uint32_t)stream_id, (uint32_t)col, prow) >> 63) ? -1.f : 1.f)
                                           : 0.f;
                store_sign(out, idx, v);
            } else {
                const double v = col < cols ? probe_value(kind, seed, (uint32_t)stream_id, (uint32_t)col, prow) : 0.0;
                store_f64<T>(out, idx, v);
            }
        }
    }
}

cudaError_t launch_probes(int out_type, int kind, uint64_t seed, int stream_id, int n, int cols, int pad,
                          void* out, long long ld, cudaStream_t s, const int32_t* rowmap) {
    if (pad < cols) pad = cols;
    const long long total = (long long)n * pad;
    if (total <= 0) return cudaSuccess;
    const int threads = 256;
    const int rpb = pad <= threads ? threads / pad : 1;
    long long blocks = ((long long)n + rpb - 1) / rpb;
    if (blocks > 152 * 16) blocks = 152 * 16;
    switch (out_type) {
        case T_F64: k_probes<double><<<(int)blocks, threads, 0, s>>>(kind, seed, stream_id, n, cols, pad, (double*)out, ld, rowmap); break;
        case T_F32: k_probes<float><<<(int)blocks, threads, 0, s>>>(kind, seed, stream_id, n, cols, pad, (float*)out, ld, rowmap); break;
        default: k_probes<dfp><<<(int)blocks, threads, 0, s>>>(kind, seed, stream_id, n, cols, pad, (dfp*)out, ld, rowmap); break;
    }
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------- CSR validation
// flag[0] bits: 1 = rowptr decreasing, 2 = column index out of range, 4 = rowptr[0] != 0 or
// rowptr[n] != nnz. flag[1]: entries farther than TMA_HALO from the diagonal. unsorted (optional):
// rows whose columns are not strictly increasing.
// (i, c) is stored in row i (a row of increasing columns; false for a row whose offsets are not in
// [0, nnz] or decrease)
__device__ __forceinline__ bool csr_has(const int32_t* rowptr, const int32_t* colind, int64_t nnz, int i, int c) {
    int lo = rowptr[i], hi = rowptr[i + 1];
    if (lo < 0 || hi < lo || (int64_t)hi > nnz) return false;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (colind[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo < rowptr[i + 1] && colind[lo] == c;
}

__global__ void k_validate_csr(const int32_t* rowptr, const int32_t* colind, int n, int64_t nnz, int* flag, int* rowmax,
                               int* unsorted, int* runs) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (tid == 0 && (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz)) atomicOr(flag, 4);
    int far = 0, longest = 0, unsort = 0, run = 0;
    for (int i = tid; i < n; i += stride) {
        const int a = rowptr[i], e = rowptr[i + 1];
        if (e < a) { atomicOr(flag, 1); continue; }
        longest = max(longest, e - a);
        if (a < 0 || (int64_t)e > nnz) { atomicOr(flag, 4); continue; }
        int prev = -1;
        bool inc = true;
        for (int k = a; k < e; ++k) {
            const int c = colind[k];
            if (c < 0 || c >= n) {
                atomicOr(flag, 2);
            } else if (c - i > TMA_HALO || i - c > TMA_HALO) {
                ++far;
                if (runs && ((i > 0 && c > 0 && csr_has(rowptr, colind, nnz, i - 1, c - 1)) ||
                             (i + 1 < n && c + 1 < n && csr_has(rowptr, colind, nnz, i + 1, c + 1))))
                    ++run;
            }
            inc = inc && c > prev;
            prev = c;
        }
        unsort += inc ? 0 : 1;
    }
    if (far > 0) atomicAdd(flag + 1, far);
    if (rowmax && longest > 0) atomicMax(rowmax, longest);
    if (unsorted && unsort > 0) atomicAdd(unsorted, unsort);
    if (runs && run > 0) atomicAdd(runs, run);
}

cudaError_t launch_validate_csr(const int32_t* rowptr, const int32_t* colind, int n, int64_t nnz, int* flag, cudaStream_t s,
                                int* rowmax, int* unsorted, int* runs) {
    k_validate_csr<<<152 * 4, 256, 0, s>>>(rowptr, colind, n, nnz, flag, rowmax, unsorted, runs);
    return cudaGetLastError();
}

// --------------------------------------------------------------- symmetry of a CSR matrix
// flag[0] = 1 when some stored entry (r, c, v) has no stored partner (c, r) with the same value
// (bit for bit). sorted: every row's columns strictly increase (binary search), else a scan.
template <typename T>
__global__ void k_check_symmetric(const int32_t* rowptr, const int32_t* colind, const T* vals, int n, int sorted,
                                  int* flag) {
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += gridDim.x * (blockDim.x >> 5)) {
        const int k0 = rowptr[r], k1 = rowptr[r + 1];
        bool bad = false;
        for (int k = k0 + (threadIdx.x & 31); k < k1; k += 32) {
            const int c = colind[k];
            const T v = vals[k];
            int lo = rowptr[c], hi = rowptr[c + 1];
            bool found = false;
            if (sorted) {
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const int cm = colind[mid];
                    if (cm == r) { found = vals[mid] == v; break; }
                    if (cm < r) lo = mid + 1; else hi = mid;
                }
            } else {
                for (int t = lo; t < hi && !found; ++t) found = colind[t] == r && vals[t] == v;
            }
            bad = bad || !found;
        }
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
    }
}

cudaError_t launch_check_symmetric(const int32_t* rowptr, const int32_t* colind, const void* vals, int dtype, int n,
                                   int sorted, int* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (dtype == LL_F64)
        k_check_symmetric<double><<<152 * 8, 256, 0, s>>>(rowptr, colind, static_cast<const double*>(vals), n, sorted, flag);
    else
        k_check_symmetric<float><<<152 * 8, 256, 0, s>>>(rowptr, colind, static_cast<const float*>(vals), n, sorted, flag);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- Gershgorin (Section 3)
template <typename T>
__global__ void k_gershgorin(const int32_t* rowptr, const int32_t* colind, const T* vals, int n,
                             double* partials, unsigned int* ticket, double* out) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a_ii = 0.0, r_i = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const double v = (double)vals[k];
            if (colind[k] == i) a_ii += v; else r_i += fabs(v);
        }
        lo = fmin(lo, a_ii - r_i);
        hi = fmax(hi, a_ii + r_i);
    }
    __shared__ double s_lo[256], s_hi[256];
    __shared__ bool s_last;
    s_lo[threadIdx.x] = lo;
    s_hi[threadIdx.x] = hi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + w]);
            s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s_lo[0];
        partials[2 * blockIdx.x + 1] = s_hi[0];
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double L = INFINITY, H = -INFINITY;
        for (int g = 0; g < (int)gridDim.x; ++g) {
            L = fmin(L, __ldcg(&partials[2 * g]));
            H = fmax(H, __ldcg(&partials[2 * g + 1]));
        }
        out[0] = L;
        out[1] = H;
        *ticket = 0u;
    }
}

cudaError_t launch_gershgorin(const int32_t* rowptr, const int32_t* colind, const void* vals, int dtype,
                              int n, double* partials, unsigned int* ticket, double* out, int grid, cudaStream_t s) {
    if (dtype == LL_F64) k_gershgorin<double><<<grid, 256, 0, s>>>(rowptr, colind, (const double*)vals, n, partials, ticket, out);
    else k_gershgorin<float><<<grid, 256, 0, s>>>(rowptr, colind, (const float*)vals, n, partials, ticket, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ value preparation
template <typename TI, typename TO>
__global__ void k_prepare(const TI* in, int64_t nnz, double scale, TO* out, const int32_t* src) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        store_f64<TO>(out, (size_t)e, (double)in[src ? (int64_t)src[e] : e] * scale);
}

cudaError_t launch_prepare_values(const void* vals, int dtype, int64_t nnz, double scale, int precision,
                                  void* out, cudaStream_t s, const int32_t* src) {
    if (nnz <= 0) return cudaSuccess;
    const int grid = 152 * 8, threads = 256;
    const int t = w_type_of(precision);
    if (dtype == LL_F64) {
        if (t == T_F64) k_prepare<double, double><<<grid, threads, 0, s>>>((const double*)vals, nnz, scale, (double*)out, src);
        else if (t == T_F32) k_prepare<double, float><<<grid, threads, 0, s>>>((const double*)vals, nnz, scale, (float*)out, src);
        else k_prepare<double, float2><<<grid, threads, 0, s>>>((const double*)vals, nnz, scale, (float2*)out, src);
    } else {
        if (t == T_F64) k_prepare<float, double><<<grid, threads, 0, s>>>((const float*)vals, nnz, scale, (double*)out, src);
        else if (t == T_F32) k_prepare<float, float><<<grid, threads, 0, s>>>((const float*)vals, nnz, scale, (float*)out, src);
        else k_prepare<float, float2><<<grid, threads, 0, s>>>((const float*)vals, nnz, scale, (float2*)out, src);
    }
    return cudaGetLastError();
}

// Values of one matrix of a pencil sweep, A = diag(D) + theta O, prepared like k_prepare: out[e] =
// convert((theta * o_e + [c_e == r] D_r) * scale), the product and the sum rounded separately (no
// FMA), as the same matrix assembled in FP64 and prepared on its own. One thread per row; flag[0]
// |= 1 where D_r != 0 and row r stores no diagonal entry or more than one.
template <typename TI, typename TO>
__global__ void k_prepare_pencil(const int32_t* rowptr, const int32_t* colind, const TI* o, const double* D, int n,
                                 double theta, double scale, TO* out, int* flag) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const double dr = D[r];
        int nd = 0;
        for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            double v = __dmul_rn(theta, (double)o[e]);
            if (colind[e] == r) {
                v = __dadd_rn(v, dr);
                ++nd;
            }
            store_f64<TO>(out, (size_t)e, __dmul_rn(v, scale));
        }
        if (nd != 1 && dr != 0.0) atomicOr(flag, 1);
    }
}

cudaError_t launch_prepare_pencil(const int32_t* rowptr, const int32_t* colind, const void* o, int dtype, const double* D,
                                  int n, double theta, double scale, int precision, void* out, int* flag,
                                  cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int grid = (int)std::min<int64_t>(((int64_t)n + threads - 1) / threads, 152 * 16);
    const int t = w_type_of(precision);
#define PP_(TI, TO) k_prepare_pencil<TI, TO><<<grid, threads, 0, s>>>(rowptr, colind, (const TI*)o, D, n, theta, scale, (TO*)out, flag)
    if (dtype == LL_F64) {
        if (t == T_F64) PP_(double, double);
        else if (t == T_F32) PP_(double, float);
        else PP_(double, float2);
    } else {
        if (t == T_F64) PP_(float, double);
        else if (t == T_F32) PP_(float, float);
        else PP_(float, float2);
    }
#undef PP_
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ block conversions
// columns [0, b) converted, columns [b, pad) of `out` set to zero
template <typename TI, typename TO>
__global__ void k_convert(const TI* in, long long ld_in, TO* out, long long ld_out, int n, int b, int pad) {
    const long long total = (long long)n * pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / pad);
        const int c = (int)(e - (long long)r * pad);
        store_f64<TO>(out, (size_t)r * ld_out + c, c < b ? load_f64<TI>(in, (size_t)r * ld_in + c) : 0.0);
    }
}

cudaError_t launch_convert_block(const double* in, long long ld_in, int precision, void* out,
                                 long long ld_out, int n, int b, int pad, cudaStream_t s) {
    if (pad < b) pad = b;
    if ((long long)n * pad <= 0) return cudaSuccess;
    const int grid = 152 * 8, threads = 256;
    switch (w_type_of(precision)) {
        case T_F64: k_convert<double, double><<<grid, threads, 0, s>>>(in, ld_in, (double*)out, ld_out, n, b, pad); break;
        case T_F32: k_convert<double, float><<<grid, threads, 0, s>>>(in, ld_in, (float*)out, ld_out, n, b, pad); break;
        default: k_convert<double, dfp><<<grid, threads, 0, s>>>(in, ld_in, (dfp*)out, ld_out, n, b, pad); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_block_to_f64(int precision, const void* in, long long ld_in, double* out,
                                long long ld_out, int n, int b, cudaStream_t s) {
    if ((long long)n * b <= 0) return cudaSuccess;
    const int grid = 152 * 8, threads = 256;
    if (p_type_of(precision) == T_DF64)
        k_convert<dfp, double><<<grid, threads, 0, s>>>((const dfp*)in, ld_in, out, ld_out, n, b, b);
    else
        k_convert<double, double><<<grid, threads, 0, s>>>((const double*)in, ld_in, out, ld_out, n, b, b);
    return cudaGetLastError();
}

// out[r, c] = in[r, c0 + c] for c < b, raw (the element's bits, both parts of a double-float
// pair); columns [b, pad) of out set to zero
template <typename T>
__global__ void k_copy_cols(const T* in, long long ld_in, int c0, T* out, long long ld_out, int n, int b, int pad) {
    const long long total = (long long)n * pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / pad);
        const int c = (int)(e - (long long)r * pad);
        out[(size_t)r * ld_out + c] = c < b ? in[(size_t)r * ld_in + c0 + c] : T(0);
    }
}
__global__ void k_copy_cols_dfp(const float* in, long long ld_in, int c0, float* out, long long ld_out, int n, int b, int pad) {
    const long long total = (long long)n * pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / pad);
        const int c = (int)(e - (long long)r * pad);
        const size_t o = dfp_hi((size_t)r * ld_out + c);
        if (c < b) {
            const size_t i = dfp_hi((size_t)r * ld_in + c0 + c);
            out[o] = in[i];
            out[o + 2] = in[i + 2];
        } else {
            out[o] = 0.f;
            out[o + 2] = 0.f;
        }
    }
}

cudaError_t launch_copy_cols(int t, const void* in, long long ld_in, int c0, void* out, long long ld_out, int n, int b,
                             int pad, cudaStream_t s) {
    if (pad < b) pad = b;
    if ((long long)n * pad <= 0) return cudaSuccess;
    const int grid = 152 * 8, threads = 256;
    switch (t) {
        case T_F64: k_copy_cols<double><<<grid, threads, 0, s>>>((const double*)in, ld_in, c0, (double*)out, ld_out, n, b, pad); break;
        case T_F32: k_copy_cols<float><<<grid, threads, 0, s>>>((const float*)in, ld_in, c0, (float*)out, ld_out, n, b, pad); break;
        default: k_copy_cols_dfp<<<grid, threads, 0, s>>>((const float*)in, ld_in, c0, (float*)out, ld_out, n, b, pad); break;
    }
    return cudaGetLastError();
}

// out[r, c] = hi + lo (FP32) of a double-float column-pair block, columns [b, pad) zero
__global__ void k_dfp_to_f32(const dfp* in, long long ld_in, float* out, long long ld_out, int n, int b, int pad) {
    const long long total = (long long)n * pad;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / pad);
        const int c = (int)(e - (long long)r * pad);
        float v = 0.f;
        if (c < b) {
            const float* f = reinterpret_cast<const float*>(in) + dfp_hi((size_t)r * ld_in + c);
            v = f[0] + f[2];
        }
        out[(size_t)r * ld_out + c] = v;
    }
}

cudaError_t launch_dfp_to_f32(const void* in, long long ld_in, float* out, long long ld_out, int n, int b, int pad,
                              cudaStream_t s) {
    if (pad < b) pad = b;
    if ((long long)n * pad <= 0) return cudaSuccess;
    k_dfp_to_f32<<<152 * 8, 256, 0, s>>>(static_cast<const dfp*>(in), ld_in, out, ld_out, n, b, pad);
    return cudaGetLastError();
}

__global__ void k_scaled_copy(const double* in, long long ld_in, double* out, long long ld_out, int n, int b, double alpha) {
    const long long total = (long long)n * b;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / b);
        const int c = (int)(e - (long long)r * b);
        out[(size_t)r * ld_out + c] = alpha * in[(size_t)r * ld_in + c];
    }
}

cudaError_t launch_scaled_copy_f64(const double* in, long long ld_in, double* out, long long ld_out, int n, int b,
                                   double alpha, cudaStream_t s) {
    if ((long long)n * b <= 0) return cudaSuccess;
    k_scaled_copy<<<152 * 8, 256, 0, s>>>(in, ld_in, out, ld_out, n, b, alpha);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_unit_diag(T* out, long long ld, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        store_f64<T>(out, (size_t)i * ld + i, 1.0);
}

cudaError_t launch_unit_diag(int t, void* out, long long ld, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    switch (t) {
        case T_F64: k_unit_diag<double><<<152, 256, 0, s>>>((double*)out, ld, n); break;
        case T_F32: k_unit_diag<float><<<152, 256, 0, s>>>((float*)out, ld, n); break;
        default: k_unit_diag<dfp><<<152, 256, 0, s>>>((dfp*)out, ld, n); break;
    }
    return cudaGetLastError();
}

// ----------------------------------------------------------------- power iteration (FP64)
template <typename T>
__global__ void k_spmv(const int32_t* rowptr, const int32_t* colind, const T* vals, int n, const double* x, double* y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) acc = fma((double)vals[k], x[colind[k]], acc);
        y[i] = acc;
    }
}

cudaError_t launch_spmv_f64(const int32_t* rowptr, const int32_t* colind, const void* vals, int dtype, int n,
                            const double* x, double* y, cudaStream_t s) {
    if (dtype == LL_F64) k_spmv<double><<<152 * 8, 256, 0, s>>>(rowptr, colind, (const double*)vals, n, x, y);
    else k_spmv<float><<<152 * 8, 256, 0, s>>>(rowptr, colind, (const float*)vals, n, x, y);
    return cudaGetLastError();
}

__global__ void k_dot(const double* x, const double* y, int n, double* partials, unsigned int* ticket, double* out) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc = fma(x[i], y[i], acc);
    __shared__ double s[256];
    __shared__ bool s_last;
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s[0];
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int g = 0; g < (int)gridDim.x; ++g) t += __ldcg(&partials[g]);
        *out = t;
        *ticket = 0u;
    }
}

cudaError_t launch_dot_f64(const double* x, const double* y, int n, double* partials, unsigned int* ticket,
                           double* out, int grid, cudaStream_t s) {
    k_dot<<<grid, 256, 0, s>>>(x, y, n, partials, ticket, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------- Algorithm 2's stopping rule, m = 0
// Thread t of a 512-thread CTA owns column t % b of rows (t / b) + lanes * i of the CTA's share,
// accumulating squares in FP64; the lanes are summed in lane order, the CTAs in CTA order by the
// last CTA to finish, which takes the decision for every column.
template <typename T>
__global__ void __launch_bounds__(512) k_stop_init(const T* W, long long ld, int n, int b, double d0, double tol,
                                                   int mmax, double* partials, unsigned int* ticket, int* live,
                                                   int* stop_deg, int* done) {
    __shared__ double red[512];
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    const int lanes = (int)blockDim.x / b;
    const int rlane = tid / b, c = tid - rlane * b;
    double acc = 0.0;
    if (rlane < lanes)
        for (long long r = (long long)blockIdx.x * lanes + rlane; r < n; r += (long long)gridDim.x * lanes) {
            const double x = load_f64<T>(W, (size_t)r * ld + c);
            acc = fma(x, x, acc);
        }
    red[tid] = acc;
    __syncthreads();
    for (int cc = tid; cc < b; cc += blockDim.x) {
        double sum = 0.0;
        for (int l = 0; l < lanes; ++l) sum += red[l * b + cc];
        partials[(size_t)blockIdx.x * b + cc] = sum;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    int any = 0;
    for (int cc = tid; cc < b; cc += blockDim.x) {
        double sum = 0.0;
        for (int g = 0; g < (int)gridDim.x; ++g) sum += __ldcg(&partials[(size_t)g * b + cc]);
        const int l = fabs(d0) * sqrt(sum) > tol ? 1 : 0;
        live[cc] = l;
        stop_deg[cc] = l ? mmax : 0;
        any |= l;
    }
    if (tid == 0 && (b & 1)) {
        live[b] = 0;
        stop_deg[b] = 0;
    }
    any = __syncthreads_or(any);
    if (tid == 0) {
        *done = any ? 0 : 1;
        *ticket = 0u;
    }
}

cudaError_t launch_stop_init(int precision, const void* W0, long long ld, int n, int b, double d0, double tol,
                             int mmax, double* partials, unsigned int* ticket, int* live, int* stop_deg, int* done,
                             cudaStream_t s) {
    if (b <= 0 || b > 512 || n < 0) return cudaErrorInvalidValue;
    const int G = STOP_INIT_GRID;
    switch (w_type_of(precision)) {
        case T_F64:
            k_stop_init<double><<<G, 512, 0, s>>>((const double*)W0, ld, n, b, d0, tol, mmax, partials, ticket, live, stop_deg, done);
            break;
        case T_F32:
            k_stop_init<float><<<G, 512, 0, s>>>((const float*)W0, ld, n, b, d0, tol, mmax, partials, ticket, live, stop_deg, done);
            break;
        default:
            k_stop_init<dfp><<<G, 512, 0, s>>>((const dfp*)W0, ld, n, b, d0, tol, mmax, partials, ticket, live, stop_deg, done);
            break;
    }
    return cudaGetLastError();
}

// mode 0: x /= sqrt(*num)
__global__ void k_scale(double* x, const double* num, int n, int mode) {
    const double f = 1.0 / sqrt(*num);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] *= f;
}

cudaError_t launch_scale_f64(double* x, const double* num, int n, int mode, cudaStream_t s) {
    k_scale<<<152 * 8, 256, 0, s>>>(x, num, n, mode);
    return cudaGetLastError();
}

}  // namespace ll
