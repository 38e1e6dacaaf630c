// Tall-skinny QR of the Hutch++ sketch by CholeskyQR2, and the deflation of the residual probes
// (Algorithm 3 steps 4 and 6: Q = orth(Y), G' = G - Q (Q^T G)).
//   Gram:   X^T Z over n rows, per-CTA partials reduced by the last CTA in a fixed order;
//   chol:   G = R^T R (upper R) and R^{-1} in one CTA (FP64, k <= 96), with a breakdown flag;
//   apply:  X R^{-1} row by row (R^{-1} in shared memory);
//   project: G - Q C row by row (C in shared memory).
// The O(n k^2) products run in double-float arithmetic on the FP32 pipes (about 46-48 bits per
// product, FP64 accumulation across row blocks); the k x k Cholesky stays in FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace ll {

constexpr int QR_THREADS = 256;
// Rows per shared-memory tile of the Gram kernel: about 1152 staged elements (32 rows at k = 33),
// more rows for narrow blocks so that a tile carries enough loads and products to hide its
// latency (k = 10: 96 rows), between 32 and 256 in multiples of 16.
__host__ __device__ inline int gram_tile_rows(int kxp, int kzp, bool sym) {
    const int cols = kxp + (sym ? 0 : kzp);
    int tr = (4608 / cols) / 16 * 16;
    return tr < 32 ? 32 : (tr > 512 ? 512 : tr);
}
constexpr int QR_FLUSH = 8;     // tiles summed in double-float before they join the running sum

// Element (i) of a block as an unevaluated float pair hi + lo.
__device__ __forceinline__ void ld_split(const double* p, size_t i, float& h, float& l) { split_bits(p[i], h, l); }

// Asynchronous staging of block tiles in shared memory (cp.async, completion waited for by the
// hardware): one copy unit is an element (double, float) or a column pair (dfp, 16 bytes).
template <typename T> struct Stg;
template <> struct Stg<double> { static constexpr int cp = 8, per = 1; };
template <> struct Stg<float> { static constexpr int cp = 4, per = 1; };
template <> struct Stg<dfp> { static constexpr int cp = 16, per = 2; };

template <int CP>
__device__ __forceinline__ void cp_async_unit(void* sdst, const void* gsrc, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc),
                 "n"(CP), "r"(valid ? CP : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// global address of the copy unit holding element a of row `row`
__device__ __forceinline__ const void* unit_src(const double* X, long long ld, long long row, int a) { return X + row * ld + a; }
__device__ __forceinline__ const void* unit_src(const float* X, long long ld, long long row, int a) { return X + row * ld + a; }
__device__ __forceinline__ const void* unit_src(const dfp* X, long long ld, long long row, int a) {
    return reinterpret_cast<const float*>(X) + ((row * ld + a) >> 1) * 4;   // a and ld are even
}
// element `sub` of a staged unit as a float pair
__device__ __forceinline__ void unit_split(const double* u, int, float& h, float& l) { split_bits(*u, h, l); }
__device__ __forceinline__ void unit_split(const float* u, int, float& h, float& l) { h = *u; l = 0.f; }
__device__ __forceinline__ void unit_split(const dfp* u, int sub, float& h, float& l) {
    const float* f = reinterpret_cast<const float*>(u);
    h = f[sub];
    l = f[2 + sub];
}

// Issues the copies of rows [tile * TR, tile * TR + TR) x columns [0, kp) of X (ld) into `stage`
// (TR x kp / per units); rows >= n and columns >= k are zero-filled.
template <typename T> __host__ __device__ constexpr size_t stage_bytes(int TR, int kp) { return (size_t)TR * (kp / Stg<T>::per) * Stg<T>::cp; }
template <typename T>
__device__ __forceinline__ void stage_tile(unsigned char* stage, const T* X, long long ld, int k, int kp, int n, int tile, int TR) {
    constexpr int CP = Stg<T>::cp, PER = Stg<T>::per;
    const int U = kp / PER;
    for (int u = threadIdx.x; u < TR * U; u += blockDim.x) {
        const int r = u / U, a = (u - r * U) * PER;
        const long long row = (long long)tile * TR + r;
        const bool valid = row < n && a < k;
        cp_async_unit<CP>(stage + (size_t)u * CP, valid ? unit_src(X, ld, row, a) : (const void*)X, valid);
    }
}
// Splits a staged tile into float pairs: h[r * ks + a], l[r * ks + a] for a < kp (columns >= k
// are zero; ks >= kp is the row stride, kp when 0)
template <typename T>
__device__ __forceinline__ void split_tile(const unsigned char* stage, int k, int kp, float* h, float* l, int TR,
                                           int ks = 0) {
    constexpr int CP = Stg<T>::cp, PER = Stg<T>::per;
    if (ks <= 0) ks = kp;
    for (int i = threadIdx.x; i < TR * kp; i += blockDim.x) {
        const int r = i / kp, a = i - r * kp;
        float hh = 0.f, ll = 0.f;
        if (a < k) unit_split(reinterpret_cast<const T*>(stage + ((size_t)r * (kp / PER) + a / PER) * CP), a % PER, hh, ll);
        h[(size_t)r * ks + a] = hh;
        l[(size_t)r * ks + a] = ll;
    }
}
__device__ __forceinline__ void ld_split(const float2* p, size_t i, float& h, float& l) {
    const float2 v = p[i];
    h = v.x;
    l = v.y;
}
__device__ __forceinline__ void ld_split(const float* p, size_t i, float& h, float& l) {
    h = p[i];
    l = 0.f;
}
__device__ __forceinline__ void ld_split(const dfp* p, size_t i, float& h, float& l) {
    const float* f = reinterpret_cast<const float*>(p) + dfp_hi(i);
    h = f[0];
    l = f[2];
}

// X^T Z over n rows in double-float arithmetic on the FP32 pipes (GB300's FP64 pipe runs at 1/62
// of FP32). Each thread owns a 4x4 register tile of the output and a group of rows; per-thread
// double-float sums cover QR_FLUSH tiles (at most 2048 rows) before they are added (TwoSum, still
// on the FP32 pipes) into a running double-float sum, converted to FP64 once at the end, so the
// error stays near FP64's. Per-CTA partials are reduced by the last CTA in a fixed order. sym:
// Z == X and only the upper-triangular 4x4 tiles are computed.
template <typename TX, typename TZ>
__global__ void __launch_bounds__(QR_THREADS) k_gram(long long ldx, int kx, long long ldz, int kz, int sym, GramJob one,
                                                     const GramJob* jobs) {
    extern __shared__ __align__(16) float sgf[];
    __shared__ bool s_last;
    // one matrix per blockIdx.z in a batch; CTAs beyond the matrix's row-block count leave
    const GramJob J = jobs ? jobs[blockIdx.z] : one;
    if ((int)blockIdx.x >= J.gx) return;
    const TX* X = static_cast<const TX*>(J.X);
    const TZ* Z = static_cast<const TZ*>(J.Z);
    const int n = J.n;
    double* partials = J.partials;
    unsigned int* ticket = J.ticket;
    double* out = J.out;
    const int kxp = (kx + 3) & ~3;
    const int kzp = sym ? kxp : ((kz + 3) & ~3);
    const int trows = gram_tile_rows(kxp, kzp, sym != 0);
    // double-float X is read straight from its staged column pairs (hi, hi, lo, lo): no split
    // arrays for it (and none at all when Z = X)
    constexpr bool XRAW = std::is_same<TX, dfp>::value;
    const int xrows = XRAW ? 0 : trows;
    float* xh = sgf;
    float* xl = xh + xrows * kxp;
    float* zh = sym ? xh : xl + xrows * kxp;
    float* zl = sym ? xl : zh + trows * kzp;
    const int ta = kxp / 4, tc = kzp / 4;
    const int OT = sym ? ta * (ta + 1) / 2 : ta * tc;
    const int otc = min(OT, QR_THREADS);
    const int G = QR_THREADS / otc;
    const int t = threadIdx.x;
    const int g = t / otc;
    const int ot = blockIdx.y * otc + (t - g * otc);
    const bool act = (g < G) && (ot < OT) && (t - g * otc < otc);
    int ia = 0, ic = 0;
    if (act) {
        if (sym) {
            int rem = ot;
            while (rem >= ta - ia) { rem -= ta - ia; ++ia; }
            ic = ia + rem;
        } else {
            ia = ot / tc;
            ic = ot - ia * tc;
        }
    }
    // 4 x 4 output tile as 4 rows x 2 column pairs of double-float sums (f32x2: both columns of a
    // pair per instruction, the same operations per lane as the scalar double-float MAC)
    f2x h2[8], l2[8], H2[8], L2[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) { h2[e] = 0ull; l2[e] = 0ull; H2[e] = 0ull; L2[e] = 0ull; }
    const int ntiles = (n + trows - 1) / trows;
    // raw tiles staged asynchronously one tile ahead (two buffers after the split arrays), so that
    // the next tile's loads are in flight while this one is computed
    unsigned char* stg = reinterpret_cast<unsigned char*>(sym ? xl + xrows * kxp : zl + trows * kzp);
    const size_t sxb = stage_bytes<TX>(trows, kxp), szb = sym ? 0 : stage_bytes<TZ>(trows, kzp);
    auto stage = [&](int tile, int b) {
        unsigned char* sb = stg + (size_t)b * (sxb + szb);
        stage_tile<TX>(sb, X, ldx, kx, kxp, n, tile, trows);
        if (!sym) stage_tile<TZ>(sb + sxb, Z, ldz, kz, kzp, n, tile, trows);
        cp_async_commit();
    };
    int cnt = 0, buf = 0;
    stage(blockIdx.x, 0);
    for (int tile = blockIdx.x; tile < ntiles; tile += J.gx) {
        if (tile + J.gx < ntiles) stage(tile + J.gx, buf ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();   // this thread's copies of `tile`
        __syncthreads();
        const unsigned char* sb = stg + (size_t)buf * (sxb + szb);
        if (!XRAW) split_tile<TX>(sb, kx, kxp, xh, xl, trows);
        if (!sym) split_tile<TZ>(sb + sxb, kz, kzp, zh, zl, trows);
        buf ^= 1;
        if (!XRAW || !sym) __syncthreads();   // the split arrays are complete
        // four columns 4 q .. 4 q + 3 of staged row rr of X as hi and lo parts (columns at or past
        // kx are zero: the pad column of a staged pair may hold anything)
        auto raw4 = [&](int rr, int q, float4& h4, float4& l4) {
            const float4* u = reinterpret_cast<const float4*>(sb + ((size_t)rr * (kxp / 2) + 2 * q) * 16);
            const float4 v0 = u[0], v1 = u[1];
            h4 = make_float4(v0.x, v0.y, v1.x, v1.y);
            l4 = make_float4(v0.z, v0.w, v1.z, v1.w);
            if (4 * q + 4 > kx) {
                const int c = kx - 4 * q;   // valid columns of the group (1 .. 3)
                if (c < 4) { h4.w = 0.f; l4.w = 0.f; }
                if (c < 3) { h4.z = 0.f; l4.z = 0.f; }
                if (c < 2) { h4.y = 0.f; l4.y = 0.f; }
            }
        };
        if (act) {
            for (int rr = g; rr < trows; rr += G) {
                float4 a4h, a4l, c4h, c4l;
                if constexpr (XRAW) {
                    raw4(rr, ia, a4h, a4l);
                } else {
                    a4h = *reinterpret_cast<const float4*>(&xh[rr * kxp + ia * 4]);
                    a4l = *reinterpret_cast<const float4*>(&xl[rr * kxp + ia * 4]);
                }
                if (XRAW && sym) {
                    raw4(rr, ic, c4h, c4l);
                } else {
                    c4h = *reinterpret_cast<const float4*>(&zh[rr * kzp + ic * 4]);
                    c4l = *reinterpret_cast<const float4*>(&zl[rr * kzp + ic * 4]);
                }
                const float ah[4] = {a4h.x, a4h.y, a4h.z, a4h.w}, al[4] = {a4l.x, a4l.y, a4l.z, a4l.w};
                const f2x c0h = f2_pack(c4h.x, c4h.y), c1h = f2_pack(c4h.z, c4h.w);
                const f2x c0l = f2_pack(c4l.x, c4l.y), c1l = f2_pack(c4l.z, c4l.w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const f2x a2h = f2_pack(ah[i], ah[i]), a2l = f2_pack(al[i], al[i]), na2h = f2_pack(-ah[i], -ah[i]);
                    df2_mac(h2[2 * i], l2[2 * i], a2h, a2l, na2h, c0h, c0l);
                    df2_mac(h2[2 * i + 1], l2[2 * i + 1], a2h, a2l, na2h, c1h, c1l);
                }
            }
        }
        __syncthreads();
        if (++cnt == QR_FLUSH) {
            cnt = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                df2_add(H2[e], L2[e], h2[e], l2[e]);
                h2[e] = 0ull;
                l2[e] = 0ull;
            }
        }
    }
    double a64[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        df2_add(H2[e], L2[e], h2[e], l2[e]);
        float h0, h1, l0, l1;
        f2_unpack(H2[e], h0, h1);
        f2_unpack(L2[e], l0, l1);
        a64[2 * e] = (double)h0 + (double)l0;
        a64[2 * e + 1] = (double)h1 + (double)l1;
    }
    // reduce the row groups (fixed order) and write this CTA's partial
    double* red = reinterpret_cast<double*>(sgf);
    cp_async_wait<0>();
    __syncthreads();
    if (act) {
#pragma unroll
        for (int e = 0; e < 16; ++e) red[((size_t)g * otc + (t - g * otc)) * 16 + e] = a64[e];
    }
    __syncthreads();
    if (t < otc && blockIdx.y * otc + t < OT) {
        const int o = blockIdx.y * otc + t;
        for (int e = 0; e < 16; ++e) {
            double sacc = 0.0;
            for (int gg = 0; gg < G; ++gg) sacc += red[((size_t)gg * otc + t) * 16 + e];
            partials[((size_t)blockIdx.x * OT + o) * 16 + e] = sacc;
        }
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)J.gx * gridDim.y - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int q = t; q < OT * 16; q += QR_THREADS) {
            const int o = q / 16, e = q - o * 16;
            // eight running sums over the CTAs (CTA bx into sum bx % 8), added in a fixed order
            double s8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int bx = 0;
            for (; bx + 8 <= J.gx; bx += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) s8[u] += __ldcg(&partials[((size_t)(bx + u) * OT + o) * 16 + e]);
            }
            for (int u = 0; bx < J.gx; ++bx, ++u) s8[u] += __ldcg(&partials[((size_t)bx * OT + o) * 16 + e]);
            const double sacc = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
            int oa, oc;
            if (sym) {
                int rem = o;
                oa = 0;
                while (rem >= ta - oa) { rem -= ta - oa; ++oa; }
                oc = oa + rem;
            } else {
                oa = o / tc;
                oc = o - oa * tc;
            }
            const int a = oa * 4 + e / 4, c = oc * 4 + e % 4;
            if (a < kx && c < kz) {
                if (sym) {
                    if (a <= c) { out[a * kx + c] = sacc; out[c * kx + a] = sacc; }
                } else {
                    out[a * kz + c] = sacc;
                }
            }
        }
        if (t == 0) *ticket = 0u;
    }
}

template <typename TX, typename TZ>
static cudaError_t gram_typed(long long ldx, int kx, long long ldz, int kz, bool sym, const GramJob& one,
                              const GramJob* jobs, int count, int gx, cudaStream_t s) {
    const int kxp = (kx + 3) & ~3, kzp = sym ? kxp : ((kz + 3) & ~3);
    const int ta = kxp / 4, tc = kzp / 4;
    const int OT = sym ? ta * (ta + 1) / 2 : ta * tc;
    const int chunks = (OT + QR_THREADS - 1) / QR_THREADS;
    const int trows = gram_tile_rows(kxp, kzp, sym);
    const int xrows = std::is_same<TX, dfp>::value ? 0 : trows;   // (double-float X: no split arrays)
    size_t smem = ((size_t)xrows * kxp + (sym ? 0 : (size_t)trows * kzp)) * 2 * sizeof(float) +
                  2 * (stage_bytes<TX>(trows, kxp) + (sym ? 0 : stage_bytes<TZ>(trows, kzp)));
    const size_t red = (size_t)QR_THREADS * 16 * sizeof(double);
    if (smem < red) smem = red;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gram<TX, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 gd(gx, chunks, count);
    k_gram<TX, TZ><<<gd, QR_THREADS, smem, s>>>(ldx, kx, ldz, kz, sym ? 1 : 0, one, jobs);
    return cudaGetLastError();
}

// row blocks of a Gram launch over n rows: at most grid / chunks, and at least four row tiles each
int gram_blocks(int kx, int kz, bool sym, int n, int grid) {
    const int kxp = (kx + 3) & ~3, kzp = sym ? kxp : ((kz + 3) & ~3);
    const int ta = kxp / 4, tc = kzp / 4;
    const int OT = sym ? ta * (ta + 1) / 2 : ta * tc;
    const int chunks = (OT + QR_THREADS - 1) / QR_THREADS;
    int gx = grid / chunks;
    const int trows = gram_tile_rows(kxp, kzp, sym);
    const int ntiles = (n + trows - 1) / trows;
    const int by_rows = (ntiles + 3) / 4;
    if (gx > by_rows) gx = by_rows;
    return gx < 1 ? 1 : gx;
}

size_t gram_partials_doubles(int kx, int kz, bool sym, int grid) {
    const int kxp = (kx + 3) & ~3, kzp = sym ? kxp : ((kz + 3) & ~3);
    const int ta = kxp / 4, tc = kzp / 4;
    const size_t OT = sym ? (size_t)ta * (ta + 1) / 2 : (size_t)ta * tc;
    return (size_t)grid * OT * 16;
}

cudaError_t launch_gram_jobs(int tx, long long ldx, int kx, int tz, long long ldz, int kz, bool sym, const GramJob& one,
                             const GramJob* jobs, int count, int gx_max, cudaStream_t s) {
    if (tz != T_F64 || count < 1 || gx_max < 1) return cudaErrorInvalidValue;
    switch (tx) {
        case T_F64: return gram_typed<double, double>(ldx, kx, ldz, kz, sym, one, jobs, count, gx_max, s);
        case T_F32: return gram_typed<float, double>(ldx, kx, ldz, kz, sym, one, jobs, count, gx_max, s);
        default: return gram_typed<dfp, double>(ldx, kx, ldz, kz, sym, one, jobs, count, gx_max, s);
    }
}

cudaError_t launch_gram(int tx, const void* X, long long ldx, int kx, int tz, const void* Z, long long ldz, int kz,
                        int n, bool sym, double* partials, unsigned int* ticket, double* out, int grid, cudaStream_t s) {
    GramJob one{X, Z, n, gram_blocks(kx, kz, sym, n, grid), partials, ticket, out};
    return launch_gram_jobs(tx, ldx, kx, tz, ldz, kz, sym, one, nullptr, 1, one.gx, s);
}

// ---------------------------------------------------------------- Cholesky + triangular inverse
__global__ void k_chol_rinv(int k, CholJob one, const CholJob* jobs) {
    extern __shared__ __align__(16) double sc[];
    const CholJob J = jobs ? jobs[blockIdx.x] : one;
    const double* G = J.G;
    double* Rinv = J.Rinv;
    int* status = J.status;
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

cudaError_t launch_chol_jobs(int k, const CholJob& one, const CholJob* jobs, int count, cudaStream_t s) {
    const size_t smem = (size_t)2 * k * k * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_chol_rinv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (count < 1) return cudaErrorInvalidValue;
    k_chol_rinv<<<count, 256, smem, s>>>(k, one, jobs);
    return cudaGetLastError();
}

cudaError_t launch_chol_rinv(const double* G, int k, double* Rinv, int* status, cudaStream_t s) {
    return launch_chol_jobs(k, CholJob{G, Rinv, status}, nullptr, 1, s);
}

// ------------------------------------------------------------------- row-wise small products
// mode 0: out[r, c] = sum_{a <= c} X[r, a] M[a, c]           (X R^{-1}, M upper triangular)
// mode 1: out[r, c] = G[r, c] - sum_{a < kx} X[r, a] M[a, c]  (G - Q C)
// Double-float products on the FP32 pipes; each thread computes 4 consecutive columns of a row.
__device__ __forceinline__ void st_out2(double* p, size_t i, float h, float l) { p[i] = (double)h + (double)l; }
__device__ __forceinline__ void st_out2(float* p, size_t i, float h, float l) { p[i] = h + l; }
__device__ __forceinline__ void st_out2(dfp* p, size_t i, float h, float l) {
    const float2 v = df_norm(h, l);
    float* f = reinterpret_cast<float*>(p) + dfp_hi(i);
    f[0] = v.x;
    f[2] = v.y;
}

// Thread layout: warp w takes the four columns 4 (w mod CG) .. + 3 of the 32 rows 32 (w / CG) ..
// + 31 of each tile of TR = 32 RB rows (CG = kcp / 4 column groups, RB row blocks, 32 CG RB
// threads): a warp's lanes share their column group, so the triangular loop of mode 0 runs
// without divergence. The split rows have an odd stride (kxs = kxp + 1): the lanes' loads of their
// rows' element a fall in distinct banks.
__host__ __device__ inline int rowprod_row_blocks(int CG) { return CG >= 8 ? 1 : (8 + CG - 1) / CG; }
constexpr int ROWPROD_MAX_THREADS = 1024;
// bytes of the split M and row arrays (16-byte multiple: the staging buffers follow)
__host__ __device__ inline size_t rowprod_split_bytes(int kx, int kcp, int RG, int kxs) {
    return (((size_t)2 * kx * kcp + (size_t)2 * RG * kxs) * sizeof(float) + 15) & ~(size_t)15;
}

template <typename TX, typename T2, int MODE>
__global__ void __launch_bounds__(ROWPROD_MAX_THREADS) k_rowprod(long long ldx, int kx, int kc, long long ldg, long long ld64,
                                                        long long ld2, int col2, int zero_pad, RowJob one,
                                                        const RowJob* jobs) {
    extern __shared__ __align__(16) float srp[];
    const RowJob J = jobs ? jobs[blockIdx.z] : one;
    const TX* X = static_cast<const TX*>(J.X);
    const double* M = J.M;
    const double* G = J.G;
    const int n = J.n;
    double* out64 = J.out64;
    T2* out2 = static_cast<T2*>(J.out2);
    const int kxp = (kx + 3) & ~3, kcp = (kc + 3) & ~3, kxs = kxp + 1;
    const int CG = kcp / 4;
    const int RG = 32 * rowprod_row_blocks(CG);   // rows per tile
    float* mh = srp;                    // kx x kcp
    float* ml = mh + (size_t)kx * kcp;
    float* xh = ml + (size_t)kx * kcp;  // RG x kxs
    float* xl = xh + (size_t)RG * kxs;
    for (int i = threadIdx.x; i < kx * kcp; i += blockDim.x) {
        const int a = i / kcp, c = i - a * kcp;
        float hh = 0.f, ll = 0.f;
        if (c < kc) ld_split(M, (size_t)a * kc + c, hh, ll);
        mh[i] = hh;
        ml[i] = ll;
    }
    const int warp = threadIdx.x >> 5;
    const int cg = warp % CG;
    const int rr = (warp / CG) * 32 + (threadIdx.x & 31);
    const bool act = rr < RG;
    const int ntiles = (n + RG - 1) / RG;
    // raw row tiles staged asynchronously one tile ahead (two buffers after the split arrays,
    // 16-byte aligned)
    unsigned char* stg = reinterpret_cast<unsigned char*>(srp) + rowprod_split_bytes(kx, kcp, RG, kxs);
    const size_t sxb = stage_bytes<TX>(RG, kxp);
    int buf = 0;
    if ((int)blockIdx.x < ntiles) stage_tile<TX>(stg, X, ldx, kx, kxp, n, blockIdx.x, RG);
    cp_async_commit();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tile + (int)gridDim.x < ntiles) stage_tile<TX>(stg + (size_t)(buf ^ 1) * sxb, X, ldx, kx, kxp, n, tile + gridDim.x, RG);
        cp_async_commit();
        cp_async_wait<1>();   // this thread's copies of `tile`
        __syncthreads();      // ... everyone's, and every thread is done with the previous tile
        split_tile<TX>(stg + (size_t)buf * sxb, kx, kxp, xh, xl, RG, kxs);
        buf ^= 1;
        __syncthreads();
        const int row = tile * RG + rr;
        if (!act || row >= n) continue;
        if (zero_pad > 0 && cg == 0) {
            for (int z = 0; z < zero_pad; ++z) {
                if (out64) out64[(size_t)row * ld64 + kc + z] = 0.0;
                if (out2) store_f64<T2>(out2, (size_t)row * ld2 + col2 + kc + z, 0.0);
            }
        }
        // the four columns as two f32x2 pairs: df2_mac runs df_mac's operations on both lanes
        f2x h01 = 0ull, l01 = 0ull, h23 = 0ull, l23 = 0ull;
        const int amax = (MODE == 0) ? min(kx, cg * 4 + 4) : kx;
        for (int a = 0; a < amax; ++a) {
            const float x_h = xh[rr * kxs + a], x_l = xl[rr * kxs + a];
            const f2x ah2 = f2_pack(x_h, x_h), al2 = f2_pack(x_l, x_l), nah2 = f2_pack(-x_h, -x_h);
            const ulonglong2 m4h = *reinterpret_cast<const ulonglong2*>(&mh[(size_t)a * kcp + cg * 4]);
            const ulonglong2 m4l = *reinterpret_cast<const ulonglong2*>(&ml[(size_t)a * kcp + cg * 4]);
            df2_mac(h01, l01, ah2, al2, nah2, m4h.x, m4l.x);
            df2_mac(h23, l23, ah2, al2, nah2, m4h.y, m4l.y);
        }
        float h[4], l[4];
        f2_unpack(h01, h[0], h[1]);
        f2_unpack(h23, h[2], h[3]);
        f2_unpack(l01, l[0], l[1]);
        f2_unpack(l23, l[2], l[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = cg * 4 + j;
            if (c >= kc) break;
            if (MODE != 1) {
                if (out64) out64[(size_t)row * ld64 + c] = (double)h[j] + (double)l[j];
                if (out2) st_out2(out2, (size_t)row * ld2 + col2 + c, h[j], l[j]);
            } else {
                // G - (h + l) in double-float on the FP32 pipes: G split from its bits, TwoSum of
                // the leading parts, the trailing parts added to the error, renormalised
                float gh, gl;
                split_bits(G[(size_t)row * ldg + c], gh, gl);
                const float sd = gh - h[j];
                const float bb = sd - gh;
                float e = (gh - (sd - bb)) + (-h[j] - bb);
                e += gl - l[j];
                const float2 r = df_norm(sd, e);
                if (out64) out64[(size_t)row * ld64 + c] = (double)r.x + (double)r.y;
                if (out2) st_out2(out2, (size_t)row * ld2 + col2 + c, r.x, r.y);
            }
        }
    }
}

template <typename TX, typename T2, int MODE>
static cudaError_t rowprod_launch(long long ldx, int kx, int kc, long long ldg, long long ld64, long long ld2, int col2,
                                  int zero_pad, const RowJob& one, const RowJob* jobs, dim3 gd, int threads, size_t smem,
                                  cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_rowprod<TX, T2, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_rowprod<TX, T2, MODE><<<gd, threads, smem, s>>>(ldx, kx, kc, ldg, ld64, ld2, col2, zero_pad, one, jobs);
    return cudaGetLastError();
}

// n_max: the largest row count of the jobs (sizes the grid); count: jobs (blockIdx.z)
template <typename TX, int MODE>
static cudaError_t rowprod_dispatch(int t2, long long ldx, int kx, int kc, long long ldg, long long ld64, long long ld2,
                                    int col2, int zero_pad, const RowJob& one, const RowJob* jobs, int count, int n_max,
                                    cudaStream_t s) {
    const int kxp = (kx + 3) & ~3, kcp = (kc + 3) & ~3, kxs = kxp + 1;
    const int CG = kcp / 4;
    const int RB = rowprod_row_blocks(CG);
    const int RG = 32 * RB;
    const int threads = 32 * CG * RB;
    if (CG < 1 || threads > ROWPROD_MAX_THREADS || count < 1) return cudaErrorInvalidValue;
    int blocks = (n_max + RG - 1) / RG;
    const int cap = 152 * 8;   // per matrix: the largest matrix of a batch sets the time; CTAs past a matrix's tiles leave
    if (blocks > cap) blocks = cap;
    if (blocks < 1) return cudaSuccess;
    const size_t smem = rowprod_split_bytes(kx, kcp, RG, kxs) + 2 * stage_bytes<TX>(RG, kxp);
    const dim3 gd(blocks, 1, count);
    switch (t2) {
        case T_F32:
            return rowprod_launch<TX, float, MODE>(ldx, kx, kc, ldg, ld64, ld2, col2, zero_pad, one, jobs, gd, threads, smem, s);
        case T_DF64:
            return rowprod_launch<TX, dfp, MODE>(ldx, kx, kc, ldg, ld64, ld2, col2, zero_pad, one, jobs, gd, threads, smem, s);
        default:
            return rowprod_launch<TX, double, MODE>(ldx, kx, kc, ldg, ld64, ld2, col2, zero_pad, one, jobs, gd, threads, smem, s);
    }
}

cudaError_t launch_apply_rinv_jobs(int tx, long long ldx, int k, long long ld64, int t2, long long ld2, const RowJob& one,
                                   const RowJob* jobs, int count, int n_max, cudaStream_t s) {
    switch (tx) {
        case T_F64: return rowprod_dispatch<double, 0>(t2, ldx, k, k, 0, ld64, ld2, 0, 0, one, jobs, count, n_max, s);
        case T_F32: return rowprod_dispatch<float, 0>(t2, ldx, k, k, 0, ld64, ld2, 0, 0, one, jobs, count, n_max, s);
        default: return rowprod_dispatch<dfp, 0>(t2, ldx, k, k, 0, ld64, ld2, 0, 0, one, jobs, count, n_max, s);
    }
}

cudaError_t launch_apply_rinv(int tx, const void* X, long long ldx, int n, int k, const double* Rinv,
                              double* out64, long long ld64, int t2, void* out2, long long ld2, cudaStream_t s) {
    const RowJob one{X, Rinv, nullptr, out64, out2, n};
    return launch_apply_rinv_jobs(tx, ldx, k, ld64, t2, ld2, one, nullptr, 1, n, s);
}

cudaError_t launch_mul_small(const double* X, long long ldx, int n, int kx, int kc, const double* M, double* out64,
                             long long ld64, int t2, void* out2, long long ld2, cudaStream_t s) {
    const RowJob one{X, M, nullptr, out64, out2, n};
    return rowprod_dispatch<double, 2>(t2, ldx, kx, kc, 0, ld64, ld2, 0, 0, one, nullptr, 1, n, s);
}

cudaError_t launch_project_jobs(long long ldq, int k, long long ldg, int kg, long long ld64, int t2, long long ld2,
                                int zero_pad, int col2, const RowJob& one, const RowJob* jobs, int count, int n_max,
                                cudaStream_t s) {
    return rowprod_dispatch<double, 1>(t2, ldq, k, kg, ldg, ld64, ld2, col2, zero_pad, one, jobs, count, n_max, s);
}

cudaError_t launch_project(int tq, const void* Q, long long ldq, int k, const double* G, long long ldg, int kg,
                           const double* C, int n, double* out64, long long ld64, int t2, void* out2,
                           long long ld2, int zero_pad, int col2, cudaStream_t s) {
    const RowJob one{Q, C, G, out64, out2, n};
    if (tq == T_DF64) return rowprod_dispatch<dfp, 1>(t2, ldq, k, kg, ldg, ld64, ld2, col2, zero_pad, one, nullptr, 1, n, s);
    return launch_project_jobs(ldq, k, ldg, kg, ld64, t2, ld2, zero_pad, col2, one, nullptr, 1, n, s);
}

}  // namespace ll
