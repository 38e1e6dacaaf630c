// TMA-fed Léja step kernel (Algorithm 2 loop body over a whole probe block).
//
// Same step as k_leja_step (W_{j+1} = (B - xi_j I) W_j on every column, fused with the P-axpy of
// pass 1, the traces of pass 2 or the adjoint's U term; the per-row arithmetic is shared), but the
// operand rows reach shared memory through the tensor memory accelerator instead of registers:
//   * the neighbour rows W_j[c_k, :] of a tile's entries by tile::gather4 (four rows of the
//     row-major block per instruction, rows given by the column indices),
//   * the tile's own rows W_j[r, :] and its V (pass 2, adjoint) or P (pass 1) rows by 2-D tile
//     loads,
// all completing on one mbarrier per pipeline stage. The CTA runs a software pipeline over its
// tiles (persistent, round robin): while tile i is computed, the copies of tiles i+1 .. i+D are in
// flight and the CSR segment of tile i+D+1 is staged with cp.async. A thread owns one row of the
// tile and one column pair, reads the gathered rows from shared memory, and writes W_{j+1} (and P)
// straight to global memory. Entries of a tile beyond the gather capacity (long rows) are read
// directly from global memory. Every wait on an mbarrier is bounded (clock64 budget); when one runs
// out the kernel records the error, stops issuing copies, drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"

namespace ll {

constexpr int TMA_MAX_STAGES = 6;
constexpr int TMA_MAX_THREADS = 512;
constexpr int TMA_CSR_SLOTS = 3;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// waits for the phase of parity `parity` to complete; false when `budget` clock cycles pass first.
// Budgets below 1e5 cycles poll with the non-blocking test_wait (try_wait may itself suspend the
// thread for longer than such a budget).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long budget) {
    const bool poll = budget < 100000;
    if (poll ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!(poll ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)))
        if (clock64() - t0 > budget) return false;
    return true;
}
// least cycles the drain after a timeout waits for each tile's copies (copies of valid rows
// complete in microseconds; this only bounds the wait)
constexpr long long TMA_DRAIN_MIN = 10000000LL;
__device__ __forceinline__ void tma_load_rows(uint32_t dst, const CUtensorMap* map, int row, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
        "l"(map), "r"(0), "r"(row), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, int r0, int r1, int r2, int r3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
        "l"(map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void cp_async4_(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8_(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(TMA_MAX_THREADS, 1)
    k_leja_tma(const __grid_constant__ CUtensorMap tm_gather, const __grid_constant__ CUtensorMap tm_own,
               const __grid_constant__ CUtensorMap tm_aux, const StepParams p, const TmaParams q) {
    using WP = typename PairT<PREC>::W;
    using PP = typename PairT<PREC>::P;
    using Raw = typename PairT<PREC>::Raw;
    using Ex = typename ExT<PREC>::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[TMA_MAX_STAGES];
    // TMA destinations are 128-byte aligned: the plan reserves 128 bytes for this offset
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ bool s_last;

    const int tid = threadIdx.x;
    const int tp = p.tp;
    const int R = q.R;
    const int NST = q.nst;
    const int D = NST - 1;
    const int rlane = tid / tp;
    const int cp = tid - rlane * tp;
    const bool active = rlane < R;
    const int n = p.n;
    const long long ldq = p.ldw >> 1;
    const long long ldpq = p.ldp >> 1;
    const WP* __restrict__ win = static_cast<const WP*>(p.win);
    WP* __restrict__ wout = static_cast<WP*>(p.wout);
    const Raw* __restrict__ vals = static_cast<const Raw*>(p.vals);
    PP* __restrict__ pblk = static_cast<PP*>(p.p);
    const int* __restrict__ rowptr = p.rowptr;
    const int* __restrict__ colind = p.colind;
    const bool has_aux = (MODE == MODE_DOT || MODE == MODE_ADJ) || (MODE == MODE_ACCUM && !p.first);

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(smem_u32(&full[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    const StepScalars<PREC> S(p, cp);
    TracePart T;

    const int nt = p.num_tiles;
    const int my = (int)blockIdx.x < nt ? (nt - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto row0_of = [&](int i) { return ((int)blockIdx.x + i * (int)gridDim.x) * R; };
    unsigned char* csr = smem + q.csr_base;

    // nnz range [zs0, zs1) of the next tile whose CSR segment is staged (loaded one iteration ahead)
    int zs0 = 0, zs1 = 0;
    if (my > 0) {
        const int r0 = row0_of(0);
        zs0 = rowptr[r0];
        zs1 = rowptr[min(r0 + R, n)];
    }

    bool dead = false;
    int issued = 0;   // tiles whose copies were issued (the same on every thread)
    int waited = 0;   // tiles this thread saw complete
    for (int i = -D - 1; i < my; ++i) {
        // (A) CSR segment (row pointers, the first gcap column indices and values) of tile i + D + 1
        const int js = i + D + 1;
        if (js < my) {
            unsigned char* slot = csr + (js % TMA_CSR_SLOTS) * q.csr_bytes;
            int* drp = reinterpret_cast<int*>(slot);
            int* dcol = reinterpret_cast<int*>(slot + q.csr_col);
            Raw* dval = reinterpret_cast<Raw*>(slot + q.csr_val);
            const int r0 = row0_of(js);
            const int nr = min(R, n - r0);
            const int g = min(zs1 - zs0, q.gcap);
            for (int e = tid; e <= nr; e += blockDim.x) cp_async4_(drp + e, rowptr + r0 + e);
            for (int e = tid; e < g; e += blockDim.x) {
                cp_async4_(dcol + e, colind + zs0 + e);
                if constexpr (sizeof(Raw) == 8) cp_async8_(dval + e, vals + zs0 + e);
                else cp_async4_(dval + e, vals + zs0 + e);
            }
            if (js + 1 < my) {
                const int r0n = row0_of(js + 1);
                zs0 = rowptr[r0n];
                zs1 = rowptr[min(r0n + R, n)];
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        // (B) every group but the newest has landed: the segment of tile i + D is here
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        // (C) publish it; every thread is done with tile i - 1 (its stage and CSR slot are free)
        const int any_dead = __syncthreads_or(dead ? 1 : 0);

        // (D) issue the copies of tile i + D into stage (i + D) % NST
        const int ji = i + D;
        if (!any_dead && ji >= 0 && ji < my) {
            unsigned char* st = smem + (ji % NST) * q.stage_bytes;
            const unsigned char* slot = csr + (ji % TMA_CSR_SLOTS) * q.csr_bytes;
            const int* crp = reinterpret_cast<const int*>(slot);
            const int* ccol = reinterpret_cast<const int*>(slot + q.csr_col);
            const Raw* cval = reinterpret_cast<const Raw*>(slot + q.csr_val);
            const int r0 = row0_of(ji);
            const int nr = min(R, n - r0);
            const int z0 = crp[0];
            const int g = min(crp[nr] - z0, q.gcap);
            const int ngr = (g + 3) >> 2;
            int* srp = reinterpret_cast<int*>(st + q.off_rp);
            for (int e = tid; e <= nr; e += blockDim.x) srp[e] = crp[e] - z0;
            if (tid == 0) {
                srp[R + 1] = z0;
                srp[R + 2] = g;
            }
            Ex* sex = reinterpret_cast<Ex*>(st + q.off_ex);
            for (int e = tid; e < g; e += blockDim.x) sex[e] = expand(cval[e]);
            const uint32_t bar = smem_u32(&full[ji % NST]);
            if (tid == 0) {
                // (the test hook adds 16 bytes to tile 0 that no copy delivers: its waits run out)
                const uint32_t bytes = (uint32_t)ngr * 4u * (uint32_t)q.rowbytes + (uint32_t)q.rbox * (uint32_t)q.rowbytes +
                                       (has_aux ? (uint32_t)q.rbox * (uint32_t)q.auxbytes : 0u) +
                                       ((q.inject && ji == 0) ? 16u : 0u);
                mbar_arrive_expect_tx(bar, bytes);
                tma_load_rows(smem_u32(st + q.off_own), &tm_own, r0, bar);
                if (has_aux) tma_load_rows(smem_u32(st + q.off_aux), &tm_aux, r0, bar);
            }
            for (int gi = tid; gi < ngr; gi += blockDim.x) {
                const int e = 4 * gi;
                tma_gather4(smem_u32(st + (size_t)gi * q.slot), &tm_gather, ccol[e], ccol[min(e + 1, g - 1)],
                            ccol[min(e + 2, g - 1)], ccol[min(e + 3, g - 1)], bar);
            }
            ++issued;
        }

        // (E) compute tile i
        if (i >= 0 && i < issued && !dead) {
            const int s = i % NST;
            if (mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((i / NST) & 1), q.spin_budget)) {
                waited = i + 1;
            } else {
                dead = true;
                *((volatile int*)q.error) = 1;
            }
            const int r0 = row0_of(i);
            const int r = r0 + rlane;
            if (!dead && active && r < n) {
                const unsigned char* st = smem + s * q.stage_bytes;
                const int* srp = reinterpret_cast<const int*>(st + q.off_rp);
                const Ex* sex = reinterpret_cast<const Ex*>(st + q.off_ex);
                const int k0 = srp[rlane], k1 = srp[rlane + 1];
                const int z0 = srp[R + 1], g = srp[R + 2];
                const WP wr = *reinterpret_cast<const WP*>(st + q.off_own + (size_t)rlane * q.rowbytes + cp * sizeof(WP));
                WP vr{};
                PP po{};
                if constexpr (MODE == MODE_DOT || MODE == MODE_ADJ)
                    vr = *reinterpret_cast<const WP*>(st + q.off_aux + (size_t)rlane * q.auxbytes + cp * sizeof(WP));
                if constexpr (MODE == MODE_ACCUM) {
                    if (!p.first) po = *reinterpret_cast<const PP*>(st + q.off_aux + (size_t)rlane * q.auxbytes + cp * sizeof(PP));
                }
                RowAcc A;
                const int kend = min(k1, g);
                const unsigned char* gcol = st + cp * sizeof(WP);
#pragma unroll 4
                for (int k = k0; k < kend; ++k) {
                    const WP x = *reinterpret_cast<const WP*>(gcol + (size_t)(k >> 2) * q.slot + (size_t)(k & 3) * q.rowbytes);
                    row_mac<PREC>(A, sex[k], x);
                }
                for (int k = max(k0, g); k < k1; ++k) {   // beyond the gather capacity: direct loads
                    const WP x = win[(size_t)colind[z0 + k] * ldq + cp];
                    row_mac<PREC>(A, expand(vals[z0 + k]), x);
                }
                row_epilogue<PREC, MODE>(p, S, A, wr, vr, po, wout + (size_t)r * ldq + cp, pblk + (size_t)r * ldpq + cp, T);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // after a timeout, wait (bounded, tile by tile) for the copies this CTA issued but did not
    // consume, so that none lands in shared memory after the CTA exits
    if (tid == 0 && dead) {
        const long long drain = q.spin_budget > TMA_DRAIN_MIN ? q.spin_budget : TMA_DRAIN_MIN;
        for (int j = waited; j < issued; ++j) mbar_wait_bounded(smem_u32(&full[j % NST]), (uint32_t)((j / NST) & 1), drain);
    }
    const int any_dead = __syncthreads_or(dead ? 1 : 0);
    if constexpr (MODE == MODE_DOT) {
        if (!any_dead) trace_reduce<PREC>(p, T, reinterpret_cast<double*>(smem), tp, R, &s_last);
    }
}

// ------------------------------------------------------------------------------------------ host

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult r{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &r) == cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D map over the rows of an n x ld block of `elem` bytes per element; a box is `box_rows` whole rows
bool encode_rows(CUtensorMap* m, const void* base, int elem, long long ld, int n, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !base || ((uintptr_t)base & 15) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)elem};
    const cuuint32_t box[2] = {(cuuint32_t)ld, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
size_t a128(size_t x) { return (x + 127) & ~(size_t)127; }

size_t raw_size(int precision) { return precision == LL_PREC_F64 ? 8 : (precision == LL_PREC_DF64 ? 8 : 4); }
size_t ex_size(int precision) { return precision == LL_PREC_F64 ? 8 : (precision == LL_PREC_DF64 ? 24 : 8); }

template <int PREC, int MODE>
int occupancy_tma(int threads, size_t smem) {
    cudaFuncSetAttribute(k_leja_tma<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leja_tma<PREC, MODE>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

template <int PREC, int MODE>
cudaError_t launch_tma_typed(const TmaLaunch& L, const CUtensorMap& g, const CUtensorMap& o, const CUtensorMap& a,
                             const StepParams& p, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_leja_tma<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_leja_tma<PREC, MODE><<<L.grid, L.threads, L.smem, s>>>(g, o, a, p, L.q);
    return cudaGetLastError();
}

}  // namespace

bool plan_step_tma(int precision, int mode, int n, int64_t nnz, int b, int threads_target, int ctas_per_sm,
                   StepParams& p, TmaLaunch& L, int sm_count) {
    L = TmaLaunch{};
    if (n <= 0 || b <= 0 || !encode_fn()) return false;
    if (ctas_per_sm < 1 || ctas_per_sm > 2) ctas_per_sm = 1;
    const int ew = (int)elem_size(w_type_of(precision));
    const long long ld = p.ldw;
    if (ld > 256 || (ld * ew) % 16 != 0) return false;
    int auxbytes = 0;
    if (mode == MODE_DOT || mode == MODE_ADJ) {
        if (p.ldv != ld) return false;
        auxbytes = (int)(ld * ew);
    } else if (mode == MODE_ACCUM) {
        if (p.ldp > 256 || (p.ldp * 8) % 16 != 0) return false;
        auxbytes = (int)(p.ldp * 8);
    }
    if (threads_target <= 0 || threads_target > TMA_MAX_THREADS) threads_target = TMA_MAX_THREADS / ctas_per_sm;
    const int tp = (b + 1) / 2;
    int R = threads_target / tp;
    if (R < 1) R = 1;
    if (R > 256) R = 256;
    if (R > n) R = n;
    if (R * tp > TMA_MAX_THREADS) return false;
    TmaParams& q = L.q;
    q.R = R;
    q.rbox = R;
    q.rowbytes = (int)(ld * ew);
    q.auxbytes = auxbytes;
    q.slot = (int)a128((size_t)4 * q.rowbytes);
    const double avg = (double)nnz / (double)n;
    const size_t budget = (ctas_per_sm == 2 ? 112 : 224) * 1024 - 1024;
    int gcap = (((int)(avg * R * 1.15) + 8) + 3) & ~3;
    if (gcap > 4096) gcap = 4096;
    for (int attempt = 0; attempt < 8; ++attempt) {
        q.gcap = gcap;
        q.off_own = (gcap / 4) * q.slot;
        q.off_aux = q.off_own + (int)a128((size_t)R * q.rowbytes);
        q.off_ex = q.off_aux + (int)a128((size_t)R * auxbytes);
        q.off_rp = q.off_ex + (int)a16((size_t)gcap * ex_size(precision));
        q.stage_bytes = (int)a128((size_t)q.off_rp + (size_t)(R + 3) * 4);
        q.csr_col = (int)a16((size_t)(R + 1) * 4);
        q.csr_val = q.csr_col + (int)a16((size_t)gcap * 4);
        q.csr_bytes = (int)a16((size_t)q.csr_val + (size_t)gcap * raw_size(precision));
        const size_t csr_total = (size_t)TMA_CSR_SLOTS * q.csr_bytes;
        const int nst = budget > csr_total ? (int)((budget - csr_total) / q.stage_bytes) : 0;
        q.nst = nst > TMA_MAX_STAGES ? TMA_MAX_STAGES : nst;
        if (q.nst >= 3 || (q.nst == 2 && gcap <= 64)) break;
        gcap = ((gcap * 3 / 4) + 3) & ~3;
        if (gcap < 16) break;
    }
    if (q.nst < 2) return false;
    q.csr_base = q.nst * q.stage_bytes;
    L.smem = (size_t)q.csr_base + (size_t)TMA_CSR_SLOTS * q.csr_bytes;
    L.threads = ((R * tp + 31) / 32) * 32;
    if (L.smem < (size_t)L.threads * 2 * sizeof(double)) L.smem = (size_t)L.threads * 2 * sizeof(double);
    L.smem += 128;
    p.tp = tp;
    p.rl = R;
    p.rpt = 1;
    p.b = b;
    p.n = n;
    p.num_tiles = (n + R - 1) / R;
    int per_sm = 0;
    switch (precision * NUM_MODES + mode) {
#define OCC(P_, M_) case P_ * NUM_MODES + M_: per_sm = occupancy_tma<P_, M_>(L.threads, L.smem); break;
#define OCC4(P_) OCC(P_, MODE_PLAIN) OCC(P_, MODE_ACCUM) OCC(P_, MODE_DOT) OCC(P_, MODE_ADJ)
        OCC4(LL_PREC_F64) OCC4(LL_PREC_DF64) OCC4(LL_PREC_F32_MIXED)
#undef OCC4
#undef OCC
        default: break;
    }
    if (per_sm < 1) return false;
    if (per_sm > ctas_per_sm) per_sm = ctas_per_sm;
    int grid = per_sm * sm_count;
    if (grid > p.num_tiles) grid = p.num_tiles;
    L.grid = grid < 1 ? 1 : grid;
    return true;
}

cudaError_t launch_step_tma(int precision, int mode, const TmaLaunch& L, const StepParams& p, cudaStream_t s) {
    if (p.num_tiles <= 0) return cudaSuccess;
    const int ew = (int)elem_size(w_type_of(precision));
    CUtensorMap g{}, o{}, a{};
    if (!encode_rows(&g, p.win, ew, p.ldw, p.n, 1) || !encode_rows(&o, p.win, ew, p.ldw, p.n, L.q.rbox))
        return cudaErrorInvalidValue;
    bool aux_ok = true;
    if (mode == MODE_DOT || mode == MODE_ADJ) aux_ok = encode_rows(&a, p.v, ew, p.ldv, p.n, L.q.rbox);
    else if (mode == MODE_ACCUM && !p.first) aux_ok = encode_rows(&a, p.p, 8, p.ldp, p.n, L.q.rbox);
    else a = o;
    if (!aux_ok) return cudaErrorInvalidValue;
    switch (precision * NUM_MODES + mode) {
#define LCH(P_, M_) case P_ * NUM_MODES + M_: return launch_tma_typed<P_, M_>(L, g, o, a, p, s);
#define LCH4(P_) LCH(P_, MODE_PLAIN) LCH(P_, MODE_ACCUM) LCH(P_, MODE_DOT) LCH(P_, MODE_ADJ)
        LCH4(LL_PREC_F64) LCH4(LL_PREC_DF64) LCH4(LL_PREC_F32_MIXED)
#undef LCH4
#undef LCH
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ll
