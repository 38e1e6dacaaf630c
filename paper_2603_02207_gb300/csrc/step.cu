// Fused Léja-step kernel (Algorithm 2 loop body over a whole probe block) and its launch plan.
//
// One launch applies W_{j+1} = (B - xi_j I) W_j to every column of an n x b row-major block,
// streaming the CSR matrix once, and fuses the per-step epilogue:
//   pass 1 (MODE_ACCUM): P += d_{j+1} W_{j+1}                (Algorithm 2, P_m = P_{m-1} + d_m w_m)
//   pass 2 (MODE_DOT):   t_{j+1}[col] = <V[:, col], W_{j+1}[:, col]>   (Algorithm 3 steps 5-6)
//   MODE_PLAIN:          W_{j+1} only (recomputation in the adjoint);
//   MODE_ACCUM_STOP / MODE_DOT_STOP: pass 1 / pass 2 under Algorithm 2's stopping rule (the
//                        norms of W_{j+1} are reduced with the traces; see MODE_STOP);
//   MODE_ADJ:            Lambda_j = (B - xi_j I) Lambda_{j+1} + d_j U, U = V with per-column
//                        weights (the reverse recurrence of the adjoint, B symmetric).
//
// Thread mapping: every thread owns a pair of adjacent columns (2cp, 2cp+1) of rows
// r0 + rlane + rl * t, t < rpt, of a CTA tile of R = rl * rpt consecutive rows; a warp touches
// consecutive pairs of the row-major block (coalesced own-row traffic, 8- or 16-byte accesses)
// and each thread keeps its pair for the whole launch (per-column trace partials stay in
// registers). Arithmetic on the pair uses the f32x2 instructions (both columns per instruction);
// double-float blocks are stored in column pairs (hi, hi, lo, lo) so a 16-byte load feeds them
// directly. The tile's row pointers, column indices and values are staged in shared memory with
// cp.async, double-buffered (the next tile's segment loads while the current one computes), and
// the values are expanded once per CTA into the broadcast pairs the f32x2 instructions take.
// Neighbour gathers of a row are issued in batches (gather_batch) before any is consumed. The
// grid is persistent: CTA i walks tiles i, i + grid, ..., so concurrently processed tiles form one
// contiguous row window and the gathered neighbour rows W_j[c, :] are L2 hits.
#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"

namespace ll {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// neighbour rows gathered per round trip and row: 8 for 8-byte pairs, 7 for 16-byte pairs (a
// 7-point stencil row in one round trip within the register budget of two CTAs per SM)
template <int PREC> __host__ __device__ constexpr int gather_batch() { return PREC == LL_PREC_F32_MIXED ? 8 : 7; }
// CTA size limit: two CTAs per SM at <= 85 registers (16-byte pairs) or <= 64 (8-byte pairs)
template <int PREC> __host__ __device__ constexpr int step_max_threads() { return PREC == LL_PREC_F32_MIXED ? 512 : 384; }
inline int step_max_threads_rt(int precision) { return precision == LL_PREC_F32_MIXED ? 512 : 384; }

// Shared memory: two staging buffers (raw row pointers, column indices, raw values) and one
// expanded-value area for the tile being computed.
template <int PREC>
struct StepSmem {
    using Raw = typename PairT<PREC>::Raw;
    using Ex = typename ExT<PREC>::T;
    unsigned char* base;
    size_t a, c, stride, ex_off;
    __device__ __host__ StepSmem(unsigned char* base_, int R, int cap) : base(base_) {
        a = align16((size_t)(R + 1) * 4);
        c = align16((size_t)cap * 4);
        stride = a + c + align16((size_t)cap * sizeof(Raw));
        ex_off = 2 * stride;
    }
    __device__ __host__ size_t bytes(int cap) const { return ex_off + align16((size_t)cap * sizeof(Ex)); }
    __device__ int* rp(int b) const { return reinterpret_cast<int*>(base + b * stride); }
    __device__ int* col(int b) const { return reinterpret_cast<int*>(base + b * stride + a); }
    __device__ Raw* raw(int b) const { return reinterpret_cast<Raw*>(base + b * stride + a + c); }
    __device__ Ex* ex() const { return reinterpret_cast<Ex*>(base + ex_off); }
};

template <int PREC, int MODE>
__global__ void __launch_bounds__(step_max_threads<PREC>(), 2) k_leja_step(const StepParams p) {
    using WP = typename PairT<PREC>::W;
    using PP = typename PairT<PREC>::P;
    using Raw = typename PairT<PREC>::Raw;
    using Ex = typename ExT<PREC>::T;
    constexpr int U = gather_batch<PREC>();
    constexpr int MB = base_mode(MODE);
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (stop_mode(MODE)) {
        // every column of the pass has met the stopping rule (the first step always runs: it
        // writes P = d_0 W_0 and the traces of W_0 that degree-0 columns keep)
        if (!p.first && *p.done) return;
    }

    const int tid = threadIdx.x;
    const int tp = p.tp;                  // column pairs per row = threads per row
    const int rlane = tid / tp;
    const int cp = tid - rlane * tp;
    const bool active = rlane < p.rl;
    const int R = p.rl * p.rpt;
    const int n = p.n;
    StepSmem<PREC> sm(smem, R, p.smem_cap);

    const long long ldq = p.ldw >> 1;     // pairs per row of W
    const long long ldvq = p.ldv >> 1;
    const long long ldpq = p.ldp >> 1;
    const WP* __restrict__ win = static_cast<const WP*>(p.win);
    WP* __restrict__ wout = static_cast<WP*>(p.wout);
    const Raw* __restrict__ vals = static_cast<const Raw*>(p.vals);
    const WP* __restrict__ vblk = static_cast<const WP*>(p.v);
    PP* __restrict__ pblk = static_cast<PP*>(p.p);
    const int* __restrict__ rowptr = p.rowptr;
    const int* __restrict__ colind = p.colind;

    const StepScalars<PREC> S(p, cp, stop_mode(MODE) && MB == MODE_ACCUM);

    auto stage = [&](int tile, int buf, int nz0, int nz1) {
        const int r0 = tile * R;
        const int nrows = min(R, n - r0);
        for (int i = tid; i <= nrows; i += blockDim.x) cp_async4(sm.rp(buf) + i, &rowptr[r0 + i]);
        const int cnt = nz1 - nz0;
        if (cnt <= p.smem_cap) {
            int* sc = sm.col(buf);
            Raw* sv = sm.raw(buf);
            for (int i = tid; i < cnt; i += blockDim.x) {
                cp_async4(sc + i, &colind[nz0 + i]);
                if constexpr (sizeof(Raw) == 8) cp_async8(sv + i, &vals[nz0 + i]);
                else cp_async4(sv + i, &vals[nz0 + i]);
            }
        }
        cp_async_commit();
    };

    TracePart T;

    int tile = blockIdx.x;
    int nz0 = rowptr[tile * R], nz1 = rowptr[min(tile * R + R, n)];
    stage(tile, 0, nz0, nz1);
    int ntile = tile + gridDim.x;
    int nnz0 = 0, nnz1 = 0;
    if (ntile < p.num_tiles) { nnz0 = rowptr[ntile * R]; nnz1 = rowptr[min(ntile * R + R, n)]; }

    for (int it = 0; tile < p.num_tiles; ++it) {
        const int buf = it & 1;
        if (ntile < p.num_tiles) {
            stage(ntile, buf ^ 1, nnz0, nnz1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int ftile = ntile + gridDim.x;
        int fz0 = 0, fz1 = 0;
        if (ftile < p.num_tiles) { fz0 = rowptr[ftile * R]; fz1 = rowptr[min(ftile * R + R, n)]; }

        const int r0 = tile * R;
        const int r1 = min(r0 + R, n);
        const bool in_smem = (nz1 - nz0) <= p.smem_cap;
        const int* rp = sm.rp(buf);
        const int* cols = in_smem ? sm.col(buf) : colind + nz0;
        Ex* ex = sm.ex();
        if constexpr (PREC != LL_PREC_F64) {
            if (in_smem) {
                const Raw* sr = sm.raw(buf);
                for (int i = tid; i < nz1 - nz0; i += blockDim.x) ex[i] = expand(sr[i]);
                __syncthreads();
            }
        }
        const Raw* rawv = in_smem ? sm.raw(buf) : vals + nz0;

        if (active) {
            for (int t = 0; t < p.rpt; ++t) {
                const int rr = rlane + p.rl * t;
                const int r = r0 + rr;
                if (r >= r1) break;
                const int k0 = rp[rr] - nz0;
                const int nk = rp[rr + 1] - rp[rr];
                const size_t own = (size_t)r * ldq + cp;
                const WP wr = win[own];
                PP po{};
                WP vr{};
                if constexpr (MB == MODE_ACCUM) {
                    if (!p.first) po = pblk[(size_t)r * ldpq + cp];
                }
                if constexpr (MB == MODE_DOT || MB == MODE_ADJ) vr = vblk[(size_t)r * ldvq + cp];

                // accumulate sum_k a_k W_j[c_k, pair]
                RowAcc A;
                for (int kb = 0; kb < nk; kb += U) {
                    WP x[U];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (kb + u < nk) x[u] = win[(size_t)cols[k0 + kb + u] * ldq + cp];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (kb + u < nk) {
                            const int k = k0 + kb + u;
                            if constexpr (PREC == LL_PREC_F64) row_mac<PREC>(A, rawv[k], x[u]);
                            else row_mac<PREC>(A, in_smem ? ex[k] : expand(rawv[k]), x[u]);
                        }
                    }
                }
                row_epilogue<PREC, MODE>(p, S, A, wr, vr, po, wout + own, pblk + (size_t)r * ldpq + cp, T);
            }
        }
        __syncthreads();
        tile = ntile;
        nz0 = nnz0;
        nz1 = nnz1;
        ntile = ftile;
        nnz0 = fz0;
        nnz1 = fz1;
    }

    if constexpr (MB == MODE_DOT || stop_mode(MODE)) {
        __shared__ bool s_last;
        trace_reduce<PREC, MODE>(p, &T, reinterpret_cast<double*>(smem), tp, p.rl, &s_last);
    }
}

template <int PREC, int MODE>
static cudaError_t launch_typed(const StepLaunch& L, const StepParams& p, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_leja_step<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_leja_step<PREC, MODE><<<L.grid, L.threads, L.smem, s>>>(p);
    return cudaGetLastError();
}

template <int PREC, int MODE>
static int occupancy(int threads, size_t smem) {
    cudaFuncSetAttribute(k_leja_step<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leja_step<PREC, MODE>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return per_sm;
}

template <int PREC>
static size_t smem_bytes(int R, int cap) {
    StepSmem<PREC> sm(nullptr, R, cap);
    return sm.bytes(cap);
}

StepLaunch plan_step(int precision, int mode, int n, int64_t nnz, int b, int threads_target, int rpt,
                     StepParams& p, int sm_count) {
    StepLaunch L{};
    const int tmax = step_max_threads_rt(precision);
    if (threads_target <= 0 || threads_target > tmax) threads_target = tmax;
    if (rpt <= 0) rpt = 8;
    const int tp = (b + 1) / 2;
    int rl = threads_target / tp;
    if (rl < 1) rl = 1;
    while (rl > 1 && rl * tp > tmax) --rl;
    L.threads = ((rl * tp + 31) / 32) * 32;
    const int R = rl * rpt;
    p.tp = tp;
    p.rl = rl;
    p.rpt = rpt;
    p.b = b;
    p.n = n;
    p.num_tiles = (n + R - 1) / R;
    // expected tile nnz with 25% headroom (+64), and at most ~80 KB of shared memory in all
    const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    int64_t cap = (int64_t)(avg * R * 1.25) + 64;
    auto bytes_of = [&](int64_t c) -> size_t {
        switch (precision) {
            case LL_PREC_F64: return smem_bytes<LL_PREC_F64>(R, (int)c);
            case LL_PREC_DF64: return smem_bytes<LL_PREC_DF64>(R, (int)c);
            default: return smem_bytes<LL_PREC_F32_MIXED>(R, (int)c);
        }
    };
    while (cap > 64 && bytes_of(cap) > 80 * 1024) cap = cap * 7 / 8;
    p.smem_cap = (int)cap;
    size_t smem = bytes_of(cap);
    const size_t red = (size_t)L.threads * 2 * sizeof(double);
    if ((base_mode(mode) == MODE_DOT || stop_mode(mode)) && smem < red) smem = red;
    L.smem = smem;
    int per_sm = 1;
    switch (precision * NUM_MODES + mode) {
#define OCC(P_, M_) case P_ * NUM_MODES + M_: per_sm = occupancy<P_, M_>(L.threads, smem); break;
#define OCC4(P_) OCC(P_, MODE_PLAIN) OCC(P_, MODE_ACCUM) OCC(P_, MODE_DOT) OCC(P_, MODE_ADJ) \
    OCC(P_, MODE_ACCUM_STOP) OCC(P_, MODE_DOT_STOP)
        OCC4(LL_PREC_F64) OCC4(LL_PREC_DF64) OCC4(LL_PREC_F32_MIXED)
#undef OCC4
#undef OCC
        default: break;
    }
    if (per_sm < 1) per_sm = 1;
    int grid = per_sm * sm_count;
    if (grid > p.num_tiles) grid = p.num_tiles;
    if (grid < 1) grid = 1;
    L.grid = grid;
    return L;
}

cudaError_t launch_step(int precision, int mode, const StepLaunch& L, const StepParams& p, cudaStream_t s) {
    if (p.num_tiles <= 0) return cudaSuccess;
    switch (precision * NUM_MODES + mode) {
#define LCH(P_, M_) case P_ * NUM_MODES + M_: return launch_typed<P_, M_>(L, p, s);
#define LCH4(P_) LCH(P_, MODE_PLAIN) LCH(P_, MODE_ACCUM) LCH(P_, MODE_DOT) LCH(P_, MODE_ADJ) \
    LCH(P_, MODE_ACCUM_STOP) LCH(P_, MODE_DOT_STOP)
        LCH4(LL_PREC_F64) LCH4(LL_PREC_DF64) LCH4(LL_PREC_F32_MIXED)
#undef LCH4
#undef LCH
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ll
