// The Gram products X^T Z of CholeskyQR2 (Algorithm 3 step 4: Y^T Y and Q1^T Q1; step 6: Q^T G) on
// the tensor cores, in FP64-class accuracy.
//
// tcgen05 multiplies BF16 operands into FP32 accumulators in tensor memory (TMEM). An FP64-class
// product is made of exact pieces by the error-free splitting of Ozaki, Ogita & Oishi (2012):
//   * a pre-pass takes each column's maximum; column j of X is scaled by 2^-E_j with
//     max_i |x_ij| < 2^(E_j - 1) and written in fixed point as
//     x_ij = 2^E_j sum_{s < S} t_s[i, j] 2^(-7 (s + 1)), integer digits |t_s| <= 64 (exact in
//     BF16); S = 7 digits for widths up to 36 (49 bits below the column's scale), 6 up to 42;
//     Z likewise (exponents F_l);
//   * then X^T Z = sum_{s, u} 2^(E_j + F_l - 7 (s + u + 2)) T_s^T U_u, and T_s^T U_u summed over
//     up to 4096 rows is a sum of integer products of at most 64^2 = 2^12 each: below 2^24, so
//     exact in FP32 whatever the order of the additions;
//   * one MMA computes all slice pairs at once: A holds [T_0; ...; T_{S-1}] (S kx rows, K = rows),
//     B holds [U_0; ...; U_{S-1}] (S kz rows), D = A B^T (S kx x S kz) in TMEM;
//   * every 4096 rows (and at the end of the CTA's rows) each thread reads its D row (s, j) from
//     TMEM, scales the entries exactly by powers of two and adds them into double-float sums per
//     (s, j, l) in global memory (the CTA's own slice of the workspace, an L2-resident region);
//     at the end the sums over s give the CTA's partial X^T Z, and the last CTA adds the
//     partials in CTA order.
// The products carry no rounding; the only roundings are the digit truncation (below 2^-49, or
// 2^-42, of each column's maximum) and the double-float sums (about 2^-48 relative).
//
// Pipeline of a CTA over its contiguous rows, in chunks of GT_CH rows: the raw rows of chunk c + 1
// are copied to shared memory (cp.async) while chunk c is split into digits (one thread per item
// of 4 rows x one column pair), and the digits of chunk c go to one of two operand buffers while
// the MMAs of chunk c - 1 read the other. Operands
// use the canonical K-major layout without swizzle: 8 x 8 BF16 core matrices (8 rows of 16 bytes),
// K-adjacent core matrices 128 bytes apart, 8-row groups GT_SBO = 1040 bytes apart (16 bytes of
// padding spread the digit stores over the banks). One thread issues the MMAs and commits each
// chunk to its buffer's mbarrier. Every wait is bounded: one that runs out sets the error flag,
// waits (bounded) for the MMAs in flight, frees the TMEM and returns.
#include "common.cuh"
#include "kernels.cuh"
#include "tma_common.cuh"

namespace ll {
namespace {

constexpr int GT_CH = 64;                      // rows per chunk (MMA K: 4 steps of 16)
constexpr int GT_BATCH_CHUNKS = 64;            // chunks summed exactly in TMEM (4096 rows)
constexpr int GT_LBO = 128;                    // bytes between K-adjacent core matrices
constexpr int GT_SBO = (GT_CH / 8) * GT_LBO + 16;   // bytes between 8-row groups (1040)
constexpr int GT_MAX_THREADS = 512;           // threads of a CTA: one per digit item of a chunk (at least 256)
constexpr int GT_SMAX = 7;

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

// 2^e as a float, e clamped to the normal range [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(max(-126, min(127, e)) + 127) << 23); }
// x 2^e for e in [-252, 254] by two exact multiplications (exact unless the result leaves the float range)
__device__ __forceinline__ float scale2(float x, int e) {
    const int e1 = max(-126, min(127, e));
    return (x * pow2f(e1)) * pow2f(e - e1);
}

// ---- operand element access ------------------------------------------------------------------
// Raw staging of an operand's chunk in shared memory: DF64 blocks by 16-byte column pairs, FP64
// blocks by 8-byte elements (their rows need not be 16-byte aligned); row stride `rs` bytes.
template <typename T> struct Raw;
template <> struct Raw<dfp> {
    static constexpr int unit = 16;
    __device__ static int units(int k) { return (k + 1) / 2; }
    __device__ static const void* src(const dfp* X, long long ld, long long row, int u) {
        return reinterpret_cast<const float*>(X) + ((row * ld + 2 * u) >> 1) * 4;
    }
    // columns (2 cp, 2 cp + 1) of a staged row as (hi pair, lo pair); a column at or past k is zero
    __device__ static void pair(const unsigned char* row, int cp, int k, f2x& hi, f2x& lo) {
        const float4 v = *reinterpret_cast<const float4*>(row + 16 * cp);
        hi = f2_pack(v.x, 2 * cp + 1 < k ? v.y : 0.f);
        lo = f2_pack(v.z, 2 * cp + 1 < k ? v.w : 0.f);
    }
};
template <> struct Raw<double> {
    static constexpr int unit = 8;
    __device__ static int units(int k) { return k; }
    __device__ static const void* src(const double* X, long long ld, long long row, int u) { return X + row * ld + u; }
    __device__ static void pair(const unsigned char* row, int cp, int k, f2x& hi, f2x& lo) {
        const double* r = reinterpret_cast<const double*>(row);
        float h0, l0, h1 = 0.f, l1 = 0.f;
        split_bits(r[2 * cp], h0, l0);
        if (2 * cp + 1 < k) split_bits(r[2 * cp + 1], h1, l1);
        hi = f2_pack(h0, h1);
        lo = f2_pack(l0, l1);
    }
};

template <int CP>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc),
                 "n"(CP), "r"(valid ? CP : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// rows [c0, c0 + GT_CH) of X into the raw stage (rows at or past `end` zero-filled)
template <typename T>
__device__ __forceinline__ void stage_raw(unsigned char* st, int rs, const T* X, long long ld, int k, long long c0, long long end,
                                          int t, int nthreads) {
    const int U = Raw<T>::units(k);
    for (int e = t; e < GT_CH * U; e += nthreads) {
        const int r = e / U, u = e - r * U;
        const long long row = c0 + r;
        const bool ok = row < end;
        cp_async<Raw<T>::unit>(st + r * rs + u * Raw<T>::unit, ok ? Raw<T>::src(X, ld, row, u) : (const void*)X, ok);
    }
}

// One item of the staged chunk's digits into the operand buffer `op`: rows 4 g4 .. 4 g4 + 3 of the
// chunk, columns 2 cp and 2 cp + 1; slice row m = s k + j, K index = the row within the chunk. Per
// digit and column the 4 rows' BF16 digits make one 8-byte store (half a core-matrix row).
// ex[j]: the column exponents E_j.
template <typename T>
__device__ __forceinline__ void slice_item(const unsigned char* st, int rs, int k, int S, const int* ex, unsigned char* op,
                                           int cp, int g4) {
    const f2x k128 = f2_pack(128.f, 128.f);
    const f2x magic = f2_pack(12582912.f, 12582912.f);   // 1.5 * 2^23: adding and subtracting it rounds to an integer
    const int j0 = 2 * cp;
    // 2^-E_j as the product of two floats (E_j may leave the normal range of one)
    const int e0 = ex[j0], e1 = j0 + 1 < k ? ex[j0 + 1] : 0;
    const int a0 = max(-126, min(127, -e0)), a1 = max(-126, min(127, -e1));
    const f2x sa = f2_pack(pow2f(a0), pow2f(a1)), sb = f2_pack(pow2f(-e0 - a0), pow2f(-e1 - a1));
    f2x vh[4], vl[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        f2x hi, lo;
        Raw<T>::pair(st + (4 * g4 + r) * rs, cp, k, hi, lo);
        vh[r] = f2_mul(f2_mul(hi, sa), sb);
        vl[r] = f2_mul(f2_mul(lo, sa), sb);
    }
    // K index 4 g4 .. 4 g4 + 3: core matrix g4 / 2 along K, bytes 8 (g4 & 1) .. + 7 of its row
    unsigned char* o0 = op + (g4 >> 1) * GT_LBO + (g4 & 1) * 8;
#pragma unroll
    for (int s = 0; s < GT_SMAX; ++s) {
        if (s >= S) break;
        uint32_t w0[2], w1[2];   // 4 rows of BF16 digits for columns j0 and j0 + 1
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const f2x h = f2_mul(vh[r], k128);
            const f2x l = f2_mul(vl[r], k128);
            const f2x t = f2_sub(f2_add(h, magic), magic);
            const f2x d = f2_sub(h, t);   // exact remainder in [-1/2, 1/2]
            // TwoSum(d, l): the remainder as a normalised double-float pair again
            const f2x sm = f2_add(d, l);
            const f2x bb = f2_sub(sm, d);
            vl[r] = f2_add(f2_sub(d, f2_sub(sm, bb)), f2_sub(l, bb));
            vh[r] = sm;
            float t0, t1;
            f2_unpack(t, t0, t1);
            // |t| <= 64: a BF16 holds it exactly in the float's upper 16 bits
            if (r & 1) {   // (row r - 1, row r) as the low and high halves of one word
                asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w0[r >> 1]) : "r"(w0[r >> 1]), "r"(__float_as_uint(t0)));
                asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w1[r >> 1]) : "r"(w1[r >> 1]), "r"(__float_as_uint(t1)));
            } else {
                w0[r >> 1] = __float_as_uint(t0);
                w1[r >> 1] = __float_as_uint(t1);
            }
        }
        const int m0 = s * k + j0;
        *reinterpret_cast<uint2*>(o0 + (m0 >> 3) * GT_SBO + (m0 & 7) * 16) = make_uint2(w0[0], w0[1]);
        if (j0 + 1 < k) {
            const int m1 = m0 + 1;
            *reinterpret_cast<uint2*>(o0 + (m1 >> 3) * GT_SBO + (m1 & 7) * 16) = make_uint2(w1[0], w1[1]);
        }
    }
}

struct GramTcArgs {
    const void* X;
    long long ldx;
    int kx;
    const double* Z;     // null: Z = X (symmetric)
    long long ldz;
    int kz;
    long long n;
    long long rows_per_cta;   // a multiple of GT_CH
    const unsigned int* mx;   // column maxima (float bits): kx of X, then kz of Z
    float2* acc;         // per CTA: S kx x kz double-float sums
    double* partials;    // grid x kx x kz
    unsigned int* ticket;
    double* out;         // kx x kz
    int* err;
    long long spin_budget;
    int S, mt, nb, nb1;  // digits, M tiles (1 or 2) of A, N of B (a multiple of 16), and N for M tile 1
    int off_a, off_b, off_rx, off_rz, rsx, rsz, opbytes_a, opbytes_b;
    uint32_t tmem_cols;
};

template <typename TX>
__global__ void __launch_bounds__(GT_MAX_THREADS, 1) k_gram_tc(const GramTcArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[2];    // slicer warps: buffer b holds a chunk's digits
    __shared__ __align__(8) unsigned long long empty[2];   // tcgen05.commit: the MMAs reading buffer b are done
    __shared__ __align__(8) unsigned long long fin;        // tcgen05.commit: every MMA issued is done
    __shared__ uint32_t s_tmem;
    __shared__ int s_dead;
    __shared__ bool s_last;
    __shared__ int s_ex[128];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const bool sym = a.Z == nullptr;
    const TX* X = static_cast<const TX*>(a.X);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = a.S;
    const int kz = sym ? a.kx : a.kz;
    int* exx = s_ex;
    int* exz = sym ? s_ex : s_ex + 64;
    // the CTA's (s, j, l) sums
    const size_t cset = (size_t)S * a.kx * kz;
    float2* accg = a.acc + (size_t)blockIdx.x * cset;
    // digit items of every chunk: 4 rows x one column pair of X, then of Z; thread t takes items
    // t, t + blockDim, ...
    const int kp2x = (a.kx + 1) / 2, kp2z = (kz + 1) / 2;
    const int itx = (GT_CH / 4) * kp2x, itz = sym ? 0 : (GT_CH / 4) * kp2z;

    // column exponents: max |x| < 2^(E - 1); all-zero columns take E = 0 (their digits are zero)
    const int nt = blockDim.x;
    for (int j = tid; j < a.kx + (sym ? 0 : a.kz); j += nt) {
        const float m = __uint_as_float(a.mx[j]);
        s_ex[j < a.kx ? j : 64 + (j - a.kx)] = m > 0.f ? ilogbf(m) + 2 : 0;
    }
    // zero both operand buffers (slice rows past S k stay zero) and this CTA's sums
    for (int i = tid * 16; i < a.off_rx; i += nt * 16) *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < (int)cset; i += nt) accg[i] = make_float2(0.f, 0.f);
    // the last warp issues the MMAs; the others (slicers) stage, split and drain
    const int nsl = nt - 32;
    const bool issuer = tid >= nsl;
    if (tid == 0) {
        mbar_init(smem_u32(&full[0]), nsl / 32);
        mbar_init(smem_u32(&full[1]), nsl / 32);
        mbar_init(smem_u32(&empty[0]), 1);
        mbar_init(smem_u32(&empty[1]), 1);
        mbar_init(smem_u32(&fin), 1);
        s_dead = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
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
    const uint32_t idesc1 = tc_idesc(128, a.nb1);   // M tile 1: only the columns u < S - s_min of its rows
    const long long r0 = (long long)blockIdx.x * a.rows_per_cta;
    const long long r1 = min(a.n, r0 + a.rows_per_cta);
    const int nch = r0 < r1 ? (int)((r1 - r0 + GT_CH - 1) / GT_CH) : 0;
    // named barrier of the slicer warps (the issuer warp does not take part)
    auto sl_sync = [&]() { asm volatile("bar.sync 1, %0;\n" ::"r"(nsl) : "memory"); };
    // the D rows of this thread's TMEM lane, scaled exactly, into the (s, j, l) sums
    auto drain = [&]() {
        tc_fence_after();
        // warps 4 t .. 4 t + 3 read M tile t (warp w reaches TMEM lanes 32 (w % 4) .. + 31)
        const int tile = warp >> 2;
        const int m = tile * 128 + 32 * (warp & 3) + lane;
        const int nblk = tile < a.mt ? (tile == 0 ? a.nb : a.nb1) / 16 : 0;
        const int ncols = tile == 0 ? S * kz : min(S * kz, a.nb1);
        const bool rowok = tile < a.mt && m < S * a.kx;
        const int s = rowok ? m / a.kx : 0, j = rowok ? m - s * a.kx : 0;
        // sums stored l-major (lanes = consecutive slice rows m: coalesced accesses)
        float2* accr = accg + (rowok ? m : 0);
        const int ms = S * a.kx;
        const int ebase = rowok ? exx[j] - 14 - 7 * s : 0;
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * tile);
        for (int blk = 0; blk < nblk; ++blk) {
            float v[16];
            tc_ld16(taddr + (uint32_t)(16 * blk), v);   // every lane of the warp takes part
            if (!rowok) continue;
            const int cb = 16 * blk;
            const int u0 = cb / kz, l0 = cb - u0 * kz;
            if (kz >= 16) {
                // the block's 16 columns have distinct l: their sums are read together, updated and
                // written back together
                float2 r[16];
                int u = u0, l = l0;   // (u, l) of column cb + q, advanced with q
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (cb + q < ncols) r[q] = accr[(size_t)l * ms];
                    if (++l == kz) { l = 0; ++u; }
                }
                u = u0;
                l = l0;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (cb + q < ncols) {
                        // the exact product D 2^(E_j + F_l - 7 (s + u + 2)) added into the (s, j, l) sum
                        const float x = scale2(v[q], ebase + exz[l] - 7 * u);
                        const float sm = r[q].x + x;
                        const float bb = sm - r[q].x;
                        r[q].y += (r[q].x - (sm - bb)) + (x - bb);
                        r[q].x = sm;
                        accr[(size_t)l * ms] = r[q];
                    }
                    if (++l == kz) { l = 0; ++u; }
                }
            } else {
                // narrow Z: one column after the other (columns of one block may share l)
                int u = u0, l = l0;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (cb + q < ncols) {
                        const float x = scale2(v[q], ebase + exz[l] - 7 * u);
                        float2 r = accr[(size_t)l * ms];
                        const float sm = r.x + x;
                        const float bb = sm - r.x;
                        r.y += (r.x - (sm - bb)) + (x - bb);
                        r.x = sm;
                        accr[(size_t)l * ms] = r;
                    }
                    if (++l == kz) { l = 0; ++u; }
                }
            }
        }
        tc_fence_before();
    };

    if (issuer) {
        // ---------------------------------------------------------------- the MMA issuer warp
        uint32_t pf[2] = {0u, 0u};
        int inbatch = 0;   // chunks accumulated in TMEM since the last drain
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(smem_u32(&full[b]), pf[b], a.spin_budget);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok || *((volatile int*)&s_dead)) {
                if (lane == 0) { s_dead = 1; atomicCAS(a.err, 0, TMA_ERR_GRAM); }
                break;
            }
            pf[b] ^= 1u;
            if (lane == 0) {
                tc_fence_after();
                const unsigned char* opa = smem + a.off_a + b * a.opbytes_a;
                const unsigned char* opb = sym ? opa : smem + a.off_b + b * a.opbytes_b;
#pragma unroll 1
                for (int t = 0; t < GT_CH / 16; ++t) {
                    // K step t: the core matrices 2t and 2t + 1 of every 8-row group
                    const uint64_t bd = tc_desc(smem_u32(opb) + (uint32_t)(2 * t) * GT_LBO, GT_LBO, GT_SBO);
                    for (int mt = 0; mt < a.mt; ++mt) {
                        const uint64_t ad = tc_desc(smem_u32(opa) + (uint32_t)(16 * mt) * GT_SBO + (uint32_t)(2 * t) * GT_LBO, GT_LBO, GT_SBO);
                        tc_mma(tmem + (uint32_t)(256 * mt), ad, bd, mt == 0 ? idesc : idesc1, (inbatch > 0 || t > 0) ? 1u : 0u);
                    }
                }
                tc_commit(smem_u32(&empty[b]));
            }
            __syncwarp();
            if (++inbatch == GT_BATCH_CHUNKS) inbatch = 0;
        }
        // every MMA issued has completed before the TMEM is freed (bounded: on a timeout elsewhere)
        if (lane == 0) {
            tc_commit(smem_u32(&fin));
            const long long bud = a.spin_budget > TMA_DRAIN_MIN ? a.spin_budget : TMA_DRAIN_MIN;
            if (!mbar_wait_bounded(smem_u32(&fin), 0u, bud)) atomicCAS(a.err, 0, TMA_ERR_GRAM);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- slicer warps
        uint32_t pe[2] = {0u, 0u};
        int waited[2] = {-1, -1};   // the last chunk on buffer b whose MMAs were waited for
        auto wait_empty = [&](int b, int c) {   // the MMAs of chunk c (on buffer b) are done
            if (waited[b] >= c) return;
            if (!mbar_wait_bounded(smem_u32(&empty[b]), pe[b], a.spin_budget)) {
                s_dead = 1;
                atomicCAS(a.err, 0, TMA_ERR_GRAM);
                return;
            }
            pe[b] ^= 1u;
            waited[b] = c;
        };
        if (nch > 0) {
            stage_raw<TX>(smem + a.off_rx, a.rsx, X, a.ldx, a.kx, r0, r1, tid, nsl);
            if (!sym) stage_raw<double>(smem + a.off_rz, a.rsz, a.Z, a.ldz, a.kz, r0, r1, tid, nsl);
            cp_async_commit();
        }
        int inbatch = 0;
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            const long long c0 = r0 + (long long)c * GT_CH;
            // next chunk's raw rows in flight while this one is split
            if (c + 1 < nch) {
                stage_raw<TX>(smem + a.off_rx + (b ^ 1) * GT_CH * a.rsx, a.rsx, X, a.ldx, a.kx, c0 + GT_CH, r1, tid, nsl);
                if (!sym)
                    stage_raw<double>(smem + a.off_rz + (b ^ 1) * GT_CH * a.rsz, a.rsz, a.Z, a.ldz, a.kz, c0 + GT_CH, r1, tid, nsl);
            }
            cp_async_commit();
            cp_async_wait<1>();
            // the MMAs of chunk c - 2 have read operand buffer b
            if (c >= 2) wait_empty(b, c - 2);
            sl_sync();
            if (*((volatile int*)&s_dead)) break;
            unsigned char* opa = smem + a.off_a + b * a.opbytes_a;
            unsigned char* opb = sym ? opa : smem + a.off_b + b * a.opbytes_b;
            for (int it = tid; it < itx + itz; it += nsl) {
                if (it < itx) slice_item<TX>(smem + a.off_rx + b * GT_CH * a.rsx, a.rsx, a.kx, S, exx, opa, it % kp2x, it / kp2x);
                else slice_item<double>(smem + a.off_rz + b * GT_CH * a.rsz, a.rsz, a.kz, S, exz, opb, (it - itx) % kp2z, (it - itx) / kp2z);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full[b]));
            // every slicer is done with raw stage b before the next iteration copies chunk c + 2 there
            sl_sync();
            if (++inbatch == GT_BATCH_CHUNKS || c + 1 == nch) {
                // the batch's MMAs done (chunk c's commit covers every earlier one): drain the sums
                inbatch = 0;
                wait_empty(b, c);
                sl_sync();
                if (*((volatile int*)&s_dead)) break;
                drain();
                // each warp arrives on full[] for the next chunk after its drain: the issuer's next
                // MMAs (which overwrite the accumulators) wait for every warp's arrival
            }
        }
    }
    cp_async_wait<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, a.tmem_cols);
    }
    // ---- the CTA's partial X^T Z: the (s, j, l) sums added over s
    __threadfence_block();
    for (int o = tid; o < a.kx * kz; o += nt) {
        const int j = o / kz, l = o - j * kz;
        float h = 0.f, lo = 0.f;
        for (int s = 0; s < S; ++s) {
            const float2 r = accg[(size_t)l * S * a.kx + s * a.kx + j];
            // double-float add of (r.x, r.y) into (h, lo)
            const float sm = h + r.x;
            const float bb = sm - h;
            lo += ((h - (sm - bb)) + (r.x - bb)) + r.y;
            h = sm;
        }
        a.partials[(size_t)blockIdx.x * a.kx * kz + o] = (double)h + (double)lo;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int o = tid; o < a.kx * kz; o += nt) {
            const int j = o / kz, l = o - j * kz;
            if (sym && l < j) continue;
            double s8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int bx = 0;
            for (; bx + 8 <= (int)gridDim.x; bx += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) s8[u] += __ldcg(&a.partials[(size_t)(bx + u) * a.kx * kz + o]);
            }
            double tail = 0.0;
            for (; bx < (int)gridDim.x; ++bx) tail += __ldcg(&a.partials[(size_t)bx * a.kx * kz + o]);
            const double v = (((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]))) + tail;
            a.out[o] = v;
            if (sym) a.out[(size_t)l * kz + j] = v;
        }
        if (tid == 0) *a.ticket = 0u;
    }
}

// Column maxima of |x| (hi parts) into mx[0..k) as float bits (atomicMax; mx zeroed before).
template <typename T>
__global__ void __launch_bounds__(256) k_colmax(const T* X, long long ld, int k, long long n, unsigned int* mx) {
    __shared__ unsigned int smx[64];
    for (int j = threadIdx.x; j < k; j += blockDim.x) smx[j] = 0u;
    __syncthreads();
    const int kp2 = (k + 1) / 2;
    const int rpb = blockDim.x / kp2;   // rows per pass of the block
    const int cp = threadIdx.x % kp2, rg = threadIdx.x / kp2;
    if (rg < rpb) {
        float m0 = 0.f, m1 = 0.f;
        if constexpr (sizeof(T) == 4) {   // dfp: the hi parts of the column pair
            for (long long i = (long long)blockIdx.x * rpb + rg; i < n; i += (long long)gridDim.x * rpb) {
                const float2 v = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(X) + ((i * ld + 2 * cp) >> 1) * 4);
                m0 = fmaxf(m0, fabsf(v.x));
                m1 = fmaxf(m1, fabsf(2 * cp + 1 < k ? v.y : 0.f));
            }
        } else {
            // FP64: the largest magnitude by its bits (an order-preserving integer compare, no FP64
            // instructions), then the hi float of that value
            const unsigned long long* B = reinterpret_cast<const unsigned long long*>(X);
            unsigned long long b0 = 0ull, b1 = 0ull;
            for (long long i = (long long)blockIdx.x * rpb + rg; i < n; i += (long long)gridDim.x * rpb) {
                b0 = max(b0, B[i * ld + 2 * cp] & 0x7FFFFFFFFFFFFFFFull);
                if (2 * cp + 1 < k) b1 = max(b1, B[i * ld + 2 * cp + 1] & 0x7FFFFFFFFFFFFFFFull);
            }
            float l;
            split_bits(__longlong_as_double((long long)b0), m0, l);
            split_bits(__longlong_as_double((long long)b1), m1, l);
        }
        atomicMax(&smx[2 * cp], __float_as_uint(m0));
        if (2 * cp + 1 < k) atomicMax(&smx[2 * cp + 1], __float_as_uint(m1));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) atomicMax(&mx[j], smx[j]);
}

}  // namespace

int gram_tc_digits(int kx, int kz) {
    const int k = kx > kz ? kx : kz;
    return k <= 36 ? 7 : (k <= 42 ? 6 : 0);
}

size_t gram_tc_partials_doubles(int kx, int kz, int grid) { return (size_t)grid * kx * kz; }

size_t gram_tc_workspace_bytes(int kx, int kz, int grid) {
    return (size_t)grid * GT_SMAX * kx * kz * sizeof(float2) + 128 * sizeof(unsigned int);
}

bool gram_tc_supported(int tx, int kx, int kz, bool sym) {
    if (kx < 1 || kz < 1 || gram_tc_digits(kx, kz) == 0) return false;
    if (sym && kx != kz) return false;
    return tx == T_F64 || tx == T_DF64;
}

cudaError_t launch_gram_tc(int tx, const void* X, long long ldx, int kx, const double* Z, long long ldz, int kz, long long n,
                           bool sym, double* partials, unsigned int* ticket, double* out, void* work, int* err,
                           long long spin_budget, int sm_count, cudaStream_t s) {
    if (sym) kz = kx;
    if (!gram_tc_supported(tx, kx, kz, sym) || n < 1 || !work) return cudaErrorInvalidValue;
    if (tx == T_DF64 && (ldx & 1)) return cudaErrorInvalidValue;   // column pairs need an even leading dimension
    GramTcArgs a{};
    a.X = X;
    a.ldx = ldx;
    a.kx = kx;
    a.Z = sym ? nullptr : Z;
    a.ldz = ldz;
    a.kz = kz;
    a.n = n;
    a.S = gram_tc_digits(kx, kz);
    const int ma = a.S * kx, mb = a.S * kz;
    a.mt = ma > 128 ? 2 : 1;
    a.nb = (mb + 15) / 16 * 16;
    if (a.nb > 256) return cudaErrorInvalidValue;
    // M tile 1 holds the slice rows s >= s1 = 128 / kx: pairs with s + u > S lie below the digits'
    // resolution (2^-7 of the truncation of the last digit) and are left out, so its MMAs take
    // N = (S - s1 + 1) kz columns
    a.nb1 = std::min(a.nb, ((a.S - 128 / kx + 1) * kz + 15) / 16 * 16);
    // shared memory: operand buffers (two each), then the raw stages (two each)
    a.opbytes_a = a.mt * 16 * GT_SBO;
    a.opbytes_b = sym ? 0 : (a.nb / 8) * GT_SBO;
    a.off_a = 0;
    a.off_b = 2 * a.opbytes_a;
    a.off_rx = a.off_b + 2 * a.opbytes_b;
    a.rsx = tx == T_DF64 ? ((kx + 1) / 2) * 16 : ((kx * 8 + 15) / 16) * 16;
    a.rsz = sym ? 0 : ((kz * 8 + 15) / 16) * 16;
    a.off_rz = a.off_rx + 2 * GT_CH * a.rsx;
    size_t smem = (size_t)a.off_rz + (size_t)2 * GT_CH * a.rsz + 128;
    // at least 116 KB: one CTA per SM, so that no second CTA waits for the TMEM one holds
    if (smem < 116 * 1024) smem = 116 * 1024;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    uint32_t cols = a.mt == 2 ? 512u : 32u;
    while (cols < (uint32_t)a.nb) cols <<= 1;
    a.tmem_cols = cols;
    // contiguous rows per CTA, whole chunks
    const long long nchunks = (n + GT_CH - 1) / GT_CH;
    int grid = (int)std::min<long long>(nchunks, (long long)sm_count);
    a.rows_per_cta = ((nchunks + grid - 1) / grid) * GT_CH;
    grid = (int)((n + a.rows_per_cta - 1) / a.rows_per_cta);
    unsigned int* mx = static_cast<unsigned int*>(work);
    a.mx = mx;
    a.acc = reinterpret_cast<float2*>(static_cast<unsigned char*>(work) + 128 * sizeof(unsigned int));
    a.partials = partials;
    a.ticket = ticket;
    a.out = out;
    a.err = err;
    a.spin_budget = spin_budget;
    // one thread per digit item of a chunk (4 rows x one column pair of X, then of Z), at least the
    // eight warps of the drain
    const int items = (GT_CH / 4) * ((kx + 1) / 2 + (sym ? 0 : (kz + 1) / 2));
    const int threads = 32 + std::min(GT_MAX_THREADS - 32, std::max(256, (items + 31) / 32 * 32));
    cudaError_t e = cudaMemsetAsync(mx, 0, 128 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int cgrid = sm_count * 2;
    if (tx == T_DF64) k_colmax<dfp><<<cgrid, 256, 0, s>>>(static_cast<const dfp*>(X), ldx, kx, n, mx);
    else k_colmax<double><<<cgrid, 256, 0, s>>>(static_cast<const double*>(X), ldx, kx, n, mx);
    if (!sym) k_colmax<double><<<cgrid, 256, 0, s>>>(Z, ldz, kz, n, mx + kx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (tx == T_DF64) {
        e = cudaFuncSetAttribute(k_gram_tc<dfp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gram_tc<dfp><<<grid, threads, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_gram_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gram_tc<double><<<grid, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ll
