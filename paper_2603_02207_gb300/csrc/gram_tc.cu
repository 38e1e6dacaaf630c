// The Gram products X^T Z of CholeskyQR2 (Algorithm 3 step 4: Y^T Y and Q1^T Q1; step 6: Q^T G) on
// the tensor cores, in FP64-class accuracy.
//
// tcgen05 multiplies BF16 operands into FP32 accumulators in tensor memory (TMEM). An FP64-class
// product is made of exact pieces by the error-free splitting of Ozaki, Ogita & Oishi (2012):
//   * rows are processed in batches of GT_BATCH_ROWS; within a batch, column j of X is scaled by
//     2^-E_j with max_i |x_ij| < 2^(E_j - 1) and written in fixed point as
//     x_ij = 2^E_j sum_{s < S} t_s[i, j] 2^(-8 (s + 1)), with integer digits |t_s| <= 128
//     (exact in BF16) and S = 6 (about 47 bits below the column's scale); Z likewise (F_l);
//   * then X^T Z = sum_{s, u} 2^(E_j + F_l - 8 (s + u + 2)) T_s^T U_u, and every T_s^T U_u over a
//     batch is a sum of at most 512 * 128^2 = 2^23 integer products: exact in FP32;
//   * one MMA computes all slice pairs at once: A holds [T_0; ...; T_5] (6 kx rows, K = the
//     batch's rows), B holds [U_0; ...; U_5] (6 kz rows), D = A B^T (6 kx x 6 kz) in TMEM;
//   * after each batch every thread reads its D row (s, j) from TMEM, scales each entry exactly by
//     powers of two and adds it into double-float sums per (s, j, l) in shared memory; at the end
//     the sums over s give the CTA's partial X^T Z, and the last CTA adds the partials in CTA order.
// The products carry no rounding; the only roundings are the digit truncation (below 2^-47 of a
// column's batch maximum) and the double-float sums (about 2^-48 relative).
//
// Operands go to shared memory in the canonical K-major layout without swizzle: 8 x 8 BF16 core
// matrices (8 rows of 16 bytes), K-adjacent core matrices GT_LBO bytes apart (128 + 16: the padding
// keeps the 16-byte digit stores free of bank conflicts), 8-row groups GT_SBO bytes apart. One
// thread issues the MMAs and commits them to an mbarrier; every wait is bounded, and a wait that
// runs out sets the error flag, waits (bounded) for the MMAs in flight, frees the TMEM and returns.
#include "common.cuh"
#include "kernels.cuh"
#include "tma_common.cuh"

namespace ll {
namespace {

constexpr int GT_S = 6;                        // digits per value
constexpr int GT_CH = 128;                     // rows per staged chunk (MMA K: 8 steps of 16)
constexpr int GT_BATCH = 4;                    // chunks per exact accumulation batch
constexpr int GT_BATCH_ROWS = GT_CH * GT_BATCH;
constexpr int GT_LBO = 144;                    // bytes between K-adjacent core matrices
constexpr int GT_SBO = (GT_CH / 8) * GT_LBO;   // bytes between 8-row groups (2304)
constexpr int GT_THREADS = 256;

// ---- tcgen05 / TMEM wrappers (inline PTX) ----------------------------------------------------
__device__ __forceinline__ void tc_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A B^T, BF16 operands from shared-memory descriptors, FP32 accumulators
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive on the mbarrier once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
// shared-memory matrix descriptor: K-major, no swizzle, start / leading / stride offsets in bytes
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- operands ----------------------------------------------------------------------------------
// columns (2 cp, 2 cp + 1) of row `row` as double-float pairs: hi = (h0, h1), lo = (l0, l1); columns
// at or past k read as zero
__device__ __forceinline__ void ld_cols(const dfp* X, long long ld, int k, long long row, int cp, f2x& hi, f2x& lo) {
    const float4 v = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + ((row * ld + 2 * cp) >> 1) * 4);
    hi = f2_pack(v.x, 2 * cp + 1 < k ? v.y : 0.f);
    lo = f2_pack(v.z, 2 * cp + 1 < k ? v.w : 0.f);
}
__device__ __forceinline__ void ld_cols(const double* X, long long ld, int k, long long row, int cp, f2x& hi, f2x& lo) {
    float h0, l0, h1 = 0.f, l1 = 0.f;
    split_bits(X[row * ld + 2 * cp], h0, l0);
    if (2 * cp + 1 < k) split_bits(X[row * ld + 2 * cp + 1], h1, l1);
    hi = f2_pack(h0, h1);
    lo = f2_pack(l0, l1);
}

// 2^e as a float, e clamped to the normal range [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(max(-126, min(127, e)) + 127) << 23); }
// x 2^e for e in [-252, 254] by two exact multiplications (exact unless the result leaves the
// float range)
__device__ __forceinline__ float scale2(float x, int e) {
    const int e1 = max(-126, min(127, e));
    return (x * pow2f(e1)) * pow2f(e - e1);
}

struct GtShape {
    int k;        // columns of the operand
    int kp2;      // column pairs
    int rows;     // slice rows: 6 k
    int base;     // shared-memory offset of the operand
};

// Maxima of |x_ij| over rows [r0, r0 + nr) into smax[j] (float bits, atomicMax), coalesced: thread t
// takes column pair t % kp2 of rows t / kp2, t / kp2 + rstride, ...
template <typename T>
__device__ __forceinline__ void batch_max(const T* X, long long ld, const GtShape& S, long long r0, int nr,
                                          unsigned int* smax) {
    const int rstride = GT_THREADS / S.kp2;
    const int cp = threadIdx.x % S.kp2, rg = threadIdx.x / S.kp2;
    if (rg >= rstride) return;
    float m0 = 0.f, m1 = 0.f;
    for (int i = rg; i < nr; i += rstride) {
        f2x hi, lo;
        ld_cols(X, ld, S.k, r0 + i, cp, hi, lo);
        float h0, h1;
        f2_unpack(hi, h0, h1);
        m0 = fmaxf(m0, fabsf(h0));
        m1 = fmaxf(m1, fabsf(h1));
    }
    atomicMax(&smax[2 * cp], __float_as_uint(m0));
    if (2 * cp + 1 < S.k) atomicMax(&smax[2 * cp + 1], __float_as_uint(m1));
}

// Digits of rows [c0, c0 + GT_CH) of X (rows at or past n are zero) into the operand's slice rows
// s k + j, K index = row - c0, scaled by sc[j] = 2^-E_j. One item = 8 rows x one column pair; per
// digit and column the 8 rows' BF16 digits form one 16-byte store (a core-matrix row).
template <typename T>
__device__ __forceinline__ void slice_chunk(const T* X, long long ld, const GtShape& S, long long c0, long long n,
                                            const int* ex, unsigned char* smem) {
    const f2x k256 = f2_pack(256.f, 256.f);
    const f2x magic = f2_pack(12582912.f, 12582912.f);   // 1.5 * 2^23: adding and subtracting it rounds to an integer
    for (int it = threadIdx.x; it < 16 * S.kp2; it += GT_THREADS) {
        const int g = it & 15, cp = it >> 4;
        const int j0 = 2 * cp;
        // 2^-E_j as the product of two floats (E_j may leave the normal range of one)
        const int e0 = ex[j0], e1 = j0 + 1 < S.k ? ex[j0 + 1] : 0;
        const int a0 = max(-126, min(127, -e0)), a1 = max(-126, min(127, -e1));
        const f2x sa = f2_pack(pow2f(a0), pow2f(a1)), sb = f2_pack(pow2f(-e0 - a0), pow2f(-e1 - a1));
        f2x vh[8], vl[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const long long row = c0 + 8 * g + r;
            f2x hi = 0ull, lo = 0ull;
            if (row < n) ld_cols(X, ld, S.k, row, cp, hi, lo);
            vh[r] = f2_mul(f2_mul(hi, sa), sb);
            vl[r] = f2_mul(f2_mul(lo, sa), sb);
        }
#pragma unroll
        for (int s = 0; s < GT_S; ++s) {
            uint32_t w0[4], w1[4];   // 8 rows of BF16 digits for columns j0 and j0 + 1
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const f2x h = f2_mul(vh[r], k256);
                const f2x l = f2_mul(vl[r], k256);
                const f2x t = f2_sub(f2_add(h, magic), magic);
                const f2x d = f2_sub(h, t);   // exact remainder in [-1/2, 1/2]
                // TwoSum(d, l): the remainder as a normalised double-float pair again
                const f2x sm = f2_add(d, l);
                const f2x bb = f2_sub(sm, d);
                vl[r] = f2_add(f2_sub(d, f2_sub(sm, bb)), f2_sub(l, bb));
                vh[r] = sm;
                float t0, t1;
                f2_unpack(t, t0, t1);
                // |t| <= 128: a BF16 holds it exactly in the float's upper 16 bits
                if (r & 1) {   // (row r - 1, row r) as the low and high halves of one word
                    asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w0[r >> 1]) : "r"(w0[r >> 1]), "r"(__float_as_uint(t0)));
                    asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w1[r >> 1]) : "r"(w1[r >> 1]), "r"(__float_as_uint(t1)));
                } else {
                    w0[r >> 1] = __float_as_uint(t0);
                    w1[r >> 1] = __float_as_uint(t1);
                }
            }
            // slice row m = s k + j, K offset 8 g: core matrix (m / 8, g), row m % 8
            const int m0 = s * S.k + j0;
            *reinterpret_cast<uint4*>(smem + S.base + (m0 >> 3) * GT_SBO + g * GT_LBO + (m0 & 7) * 16) =
                make_uint4(w0[0], w0[1], w0[2], w0[3]);
            if (j0 + 1 < S.k) {
                const int m1 = m0 + 1;
                *reinterpret_cast<uint4*>(smem + S.base + (m1 >> 3) * GT_SBO + g * GT_LBO + (m1 & 7) * 16) =
                    make_uint4(w1[0], w1[1], w1[2], w1[3]);
            }
        }
    }
}

struct GramTcArgs {
    const void* X;
    long long ldx;
    int kx;
    const double* Z;   // null: Z = X (symmetric)
    long long ldz;
    int kz;
    long long n;
    double* partials;  // grid x kx x kz
    unsigned int* ticket;
    double* out;       // kx x kz
    int* err;
    long long spin_budget;
    int mt, nb;        // M tiles (1 or 2) of A, N of B (a multiple of 16)
    int off_b, off_acc, off_sc, acc_stride, acc_copies, zero_bytes;
    uint32_t tmem_cols;
};

template <typename TX>
__global__ void __launch_bounds__(GT_THREADS, 1) k_gram_tc(const GramTcArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t s_tmem;
    __shared__ bool s_last;
    __shared__ int s_dead;
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const bool sym = a.Z == nullptr;
    const TX* X = static_cast<const TX*>(a.X);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GtShape SA{a.kx, (a.kx + 1) / 2, GT_S * a.kx, 0};
    const GtShape SB{a.kz, (a.kz + 1) / 2, GT_S * a.kz, sym ? 0 : a.off_b};
    // per-column exponents E of the batch (|x| < 2^(E - 1)), and the maxima they come from
    int* exx = reinterpret_cast<int*>(smem + a.off_sc);
    int* exz = exx + 64;
    unsigned int* mxx = reinterpret_cast<unsigned int*>(exz + 64);
    unsigned int* mxz = mxx + 64;
    float2* acc = reinterpret_cast<float2*>(smem + a.off_acc);

    // zero the operands (slice rows past 6 k stay zero) and the sums
    for (uint32_t i = tid * 16u; i < (uint32_t)a.zero_bytes; i += GT_THREADS * 16u) *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(smem_u32(&mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_dead = 0;
    }
    if (warp == 0) {
        tc_alloc(smem_u32(&s_tmem), a.tmem_cols);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc_idesc(128, a.nb);
    const uint32_t sbase = smem_u32(smem);
    uint32_t phase = 0;
    int pending = 0;   // MMA commits not yet waited for (0 or 1)
    bool dead = false;
    const long long nbat = (a.n + GT_BATCH_ROWS - 1) / GT_BATCH_ROWS;

    for (long long bt = blockIdx.x; bt < nbat && !dead; bt += gridDim.x) {
        const long long r0 = bt * GT_BATCH_ROWS;
        const int nr = (int)min((long long)GT_BATCH_ROWS, a.n - r0);
        // ---- column scales of the batch
        for (int j = tid; j < 64; j += GT_THREADS) { mxx[j] = 0u; mxz[j] = 0u; }
        __syncthreads();
        batch_max<TX>(X, a.ldx, SA, r0, nr, mxx);
        if (!sym) batch_max<double>(a.Z, a.ldz, SB, r0, nr, mxz);
        __syncthreads();
        for (int j = tid; j < 128; j += GT_THREADS) {
            const bool isx = j < 64;
            const int jj = isx ? j : j - 64;
            if (jj >= (isx ? a.kx : a.kz)) continue;
            const float mx = __uint_as_float(isx ? mxx[jj] : mxz[jj]);
            // E with mx < 2^(E - 1); all-zero columns take E = 0 (their digits are zero)
            (isx ? exx : exz)[jj] = mx > 0.f ? ilogbf(mx) + 2 : 0;
        }
        __syncthreads();
        // ---- the batch's chunks: digits into shared memory, then the MMAs of the chunk
        for (int c = 0; c < GT_BATCH; ++c) {
            const long long c0 = r0 + (long long)c * GT_CH;
            if (c0 >= a.n) break;
            if (pending) {   // the previous chunk's MMAs have read the operands
                const bool ok = mbar_wait_bounded(smem_u32(&mbar), phase, a.spin_budget);
                if (__syncthreads_or(ok ? 0 : 1)) { dead = true; break; }
                phase ^= 1u;
                pending = 0;
            }
            slice_chunk<TX>(X, a.ldx, SA, c0, a.n, exx, smem);
            if (!sym) slice_chunk<double>(a.Z, a.ldz, SB, c0, a.n, exz, smem);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll 1
                for (int t = 0; t < GT_CH / 16; ++t) {
                    // K step t: the core matrices 2t and 2t + 1 of every 8-row group
                    const uint64_t bd = tc_desc(sbase + (uint32_t)SB.base + (uint32_t)(2 * t) * GT_LBO, GT_LBO, GT_SBO);
                    for (int mt = 0; mt < a.mt; ++mt) {
                        const uint64_t ad = tc_desc(sbase + (uint32_t)SA.base + (uint32_t)(16 * mt) * GT_SBO + (uint32_t)(2 * t) * GT_LBO,
                                                    GT_LBO, GT_SBO);
                        tc_mma(tmem + (uint32_t)(256 * mt), ad, bd, idesc, (c > 0 || t > 0) ? 1u : 0u);
                    }
                }
                tc_commit(smem_u32(&mbar));
            }
            pending = 1;
        }
        if (dead) break;
        // ---- the batch's products: scaled into the double-float sums
        {
            const bool ok = mbar_wait_bounded(smem_u32(&mbar), phase, a.spin_budget);
            if (__syncthreads_or(ok ? 0 : 1)) { dead = true; break; }
            phase ^= 1u;
            pending = 0;
        }
        tc_fence_after();
        const int grp = warp >> 2;                        // two groups of four warps
        const int tile = a.mt == 2 ? grp : 0;
        const int m = tile * 128 + 32 * (warp & 3) + lane;   // slice row of A (this thread's TMEM lane)
        const int nblk = a.nb / 16;
        const int b0 = a.mt == 2 ? 0 : (grp == 0 ? 0 : (nblk + 1) / 2);
        const int b1 = a.mt == 2 ? nblk : (grp == 0 ? (nblk + 1) / 2 : nblk);
        const bool rowok = m < SA.rows;
        const int s = rowok ? m / a.kx : 0, j = rowok ? m - s * a.kx : 0;
        float2* accr = acc + ((size_t)(a.mt == 2 ? 0 : grp) * SA.rows + (rowok ? m : 0)) * a.acc_stride;
        const int* ez = sym ? exx : exz;
        const int ebase = rowok ? exx[j] - 16 - 8 * s : 0;
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * tile);
        for (int blk = b0; blk < b1; ++blk) {
            float v[16];
            tc_ld16(taddr + (uint32_t)(16 * blk), v);   // every lane of the warp takes part
            if (!rowok) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int col = 16 * blk + q;
                if (col >= SB.rows) continue;
                const int u = col / a.kz, l = col - u * a.kz;
                // the exact product D 2^(E_j + F_l - 8 (s + u + 2)) added into the (s, j, l) sum
                const float x = scale2(v[q], ebase + ez[l] - 8 * u);
                float2 r = accr[l];
                const float sm = r.x + x;
                const float bb = sm - r.x;
                r.y += (r.x - (sm - bb)) + (x - bb);
                r.x = sm;
                accr[l] = r;
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM read before the next batch's first MMA overwrites it
    }
    // ---- after a failed wait: the MMAs in flight finish before the TMEM is freed
    if (dead && tid == 0) {
        *((volatile int*)a.err) = 1;
        if (pending) mbar_wait_bounded(smem_u32(&mbar), phase, a.spin_budget > TMA_DRAIN_MIN ? a.spin_budget : TMA_DRAIN_MIN);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, a.tmem_cols);
    }
    // ---- the CTA's partial X^T Z: the (s, j, l) sums added over s (and over the two column halves)
    const int ncop = a.acc_copies;
    for (int o = tid; o < a.kx * a.kz; o += GT_THREADS) {
        const int j = o / a.kz, l = o - j * a.kz;
        float h = 0.f, lo = 0.f;
        for (int cpy = 0; cpy < ncop; ++cpy)
            for (int s = 0; s < GT_S; ++s) {
                const float2 r = acc[((size_t)cpy * SA.rows + s * a.kx + j) * a.acc_stride + l];
                // double-float add of (r.x, r.y) into (h, lo)
                const float sm = h + r.x;
                const float bb = sm - h;
                lo += ((h - (sm - bb)) + (r.x - bb)) + r.y;
                h = sm;
            }
        a.partials[(size_t)blockIdx.x * a.kx * a.kz + o] = (double)h + (double)lo;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int o = tid; o < a.kx * a.kz; o += GT_THREADS) {
            const int j = o / a.kz, l = o - j * a.kz;
            if (sym && l < j) continue;
            double s8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int bx = 0;
            for (; bx + 8 <= (int)gridDim.x; bx += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) s8[u] += __ldcg(&a.partials[(size_t)(bx + u) * a.kx * a.kz + o]);
            }
            for (int u = 0; bx < (int)gridDim.x; ++bx, ++u) s8[u] += __ldcg(&a.partials[(size_t)bx * a.kx * a.kz + o]);
            const double v = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
            a.out[o] = v;
            if (sym) a.out[(size_t)l * a.kz + j] = v;
        }
        if (tid == 0) *a.ticket = 0u;
    }
}

}  // namespace

size_t gram_tc_partials_doubles(int kx, int kz, int grid) { return (size_t)grid * kx * kz; }

bool gram_tc_supported(int tx, int kx, int kz, bool sym) {
    if (kx < 1 || kz < 1 || kx > GRAM_TC_KMAX || kz > GRAM_TC_KMAX) return false;
    if (sym && kx != kz) return false;
    return tx == T_F64 || tx == T_DF64;
}

cudaError_t launch_gram_tc(int tx, const void* X, long long ldx, int kx, const double* Z, long long ldz, int kz, long long n,
                           bool sym, double* partials, unsigned int* ticket, double* out, int* err, long long spin_budget,
                           int sm_count, cudaStream_t s) {
    if (!gram_tc_supported(tx, kx, kz, sym) || n < 1) return cudaErrorInvalidValue;
    if (tx == T_DF64 && (ldx & 1)) return cudaErrorInvalidValue;   // column pairs need an even leading dimension
    GramTcArgs a{};
    a.X = X;
    a.ldx = ldx;
    a.kx = kx;
    a.Z = sym ? nullptr : Z;
    a.ldz = ldz;
    a.kz = sym ? kx : kz;
    a.n = n;
    a.partials = partials;
    a.ticket = ticket;
    a.out = out;
    a.err = err;
    a.spin_budget = spin_budget;
    const int ma = GT_S * a.kx, mb = GT_S * a.kz;
    a.mt = ma > 128 ? 2 : 1;
    a.nb = (mb + 15) / 16 * 16;
    const size_t bytes_a = (size_t)a.mt * 16 * GT_SBO;
    const size_t bytes_b = sym ? 0 : (size_t)(a.nb / 8) * GT_SBO;
    a.off_b = (int)bytes_a;
    a.off_sc = (int)(bytes_a + bytes_b);
    a.off_acc = a.off_sc + 4 * 64 * 4;
    a.acc_stride = a.kz | 1;   // odd: the per-thread rows of the sums spread over the banks
    a.acc_copies = a.mt == 2 ? 1 : 2;
    a.zero_bytes = (int)(((size_t)a.off_acc + (size_t)a.acc_copies * ma * a.acc_stride * sizeof(float2) + 15) & ~(size_t)15);
    size_t smem = (size_t)a.zero_bytes + 128;
    // at least 116 KB: one CTA per SM, so that no second CTA waits for the TMEM it holds
    if (smem < 116 * 1024) smem = 116 * 1024;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    uint32_t cols = a.mt == 2 ? 512u : 32u;
    while (cols < (uint32_t)a.nb) cols <<= 1;
    a.tmem_cols = cols;
    const long long nbat = (n + GT_BATCH_ROWS - 1) / GT_BATCH_ROWS;
    const int grid = (int)std::min<long long>(nbat, (long long)sm_count);
    cudaError_t e;
    if (tx == T_DF64) {
        e = cudaFuncSetAttribute(k_gram_tc<dfp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gram_tc<dfp><<<grid, GT_THREADS, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_gram_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gram_tc<double><<<grid, GT_THREADS, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ll
