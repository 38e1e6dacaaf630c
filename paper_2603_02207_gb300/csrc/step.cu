// Fused Léja-step kernel (Algorithm 2 loop body over a whole probe block) and its launch plan.
//
// One launch applies W_{j+1} = (B - xi_j I) W_j to every column of an n x b row-major block,
// streaming the CSR matrix once, and fuses the per-step epilogue:
//   pass 1 (MODE_ACCUM): P += d_{j+1} W_{j+1}                (Algorithm 2, P_m = P_{m-1} + d_m w_m)
//   pass 2 (MODE_DOT):   t_{j+1}[col] = <V[:, col], W_{j+1}[:, col]>   (Algorithm 3 steps 5-6)
//
// Thread mapping: a CTA owns a tile of R = rl * rpt consecutive rows. Thread tid works on column
// col = tid % b of rows r0 + tid / b + rl * t, t < rpt, so a warp touches consecutive elements of
// the row-major block (coalesced own-row traffic), each thread keeps one column for the whole
// tile (per-column trace partials stay in registers), and the tile's column indices and values
// are staged once in shared memory and broadcast to the b threads of a row. The grid is
// persistent: CTA i walks tiles i, i + grid, ..., so concurrently processed tiles form one
// contiguous row window and the gathered neighbour rows W_j[c, :] are L2 hits.
#include "common.cuh"
#include "kernels.cuh"

namespace ll {

template <int PREC> struct Storage;
template <> struct Storage<LL_PREC_F64> { using W = double; using V = double; using P = double; };
template <> struct Storage<LL_PREC_DF64> { using W = float2; using V = float2; using P = float2; };
template <> struct Storage<LL_PREC_F32_MIXED> { using W = float; using V = float; using P = float2; };

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int PREC> struct Acc;
template <> struct Acc<LL_PREC_F64> { double v; };
template <> struct Acc<LL_PREC_F32_MIXED> { float v; };
template <> struct Acc<LL_PREC_DF64> { float h, l; };

__device__ __forceinline__ void mac(Acc<LL_PREC_F64>& a, double v, double x) { a.v = fma(v, x, a.v); }
__device__ __forceinline__ void mac(Acc<LL_PREC_F32_MIXED>& a, float v, float x) { a.v = fmaf(v, x, a.v); }
__device__ __forceinline__ void mac(Acc<LL_PREC_DF64>& a, float2 v, float2 x) { df_mac(a.h, a.l, v.x, v.y, x.x, x.y); }

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

constexpr int GATHER_BATCH = 8;   // neighbour rows gathered per round trip and row
constexpr int STEP_MAX_THREADS = 512;

// Two staging buffers, each holding a tile's raw row pointers, column indices and values.
template <int PREC>
struct StepSmem {
    using Val = typename Storage<PREC>::V;
    unsigned char* base;
    size_t a, c, stride;
    __device__ StepSmem(unsigned char* base_, int R, int cap) : base(base_) {
        a = align16((size_t)(R + 1) * 4);
        c = align16((size_t)cap * 4);
        stride = a + c + align16((size_t)cap * sizeof(Val));
    }
    __device__ int* rp(int b) const { return reinterpret_cast<int*>(base + b * stride); }
    __device__ int* col(int b) const { return reinterpret_cast<int*>(base + b * stride + a); }
    __device__ Val* val(int b) const { return reinterpret_cast<Val*>(base + b * stride + a + c); }
};

// L2 prefetch of rows [lo, hi) of a row-major block (TMA bulk prefetch, 16-byte granules,
// split into 4 KB requests over the lanes of warp 0). A hint only: ranges are clamped to the
// block and an unaligned base skips the prefetch.
__device__ __forceinline__ void prefetch_rows_l2(const void* base, long long ld, int es, long long lo, long long hi, int n) {
    if (!base || (((uintptr_t)base) & 15)) return;
    if (lo < 0) lo = 0;
    if (hi > n) hi = n;
    if (lo >= hi) return;
    const unsigned long long b0 = ((unsigned long long)lo * ld * es) & ~15ull;
    const unsigned long long b1 = ((unsigned long long)hi * ld * es) & ~15ull;
    const int lane = threadIdx.x;
    for (unsigned long long off = b0 + (unsigned long long)lane * 4096; off < b1; off += 32ull * 4096) {
        const unsigned long long len = (b1 - off < 4096) ? (b1 - off) : 4096;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"((uintptr_t)base + off), "r"((unsigned)len) : "memory");
    }
}

template <int PREC, int MODE, int RB>
__global__ void __launch_bounds__(STEP_MAX_THREADS, (RB == 1 ? 2 : 1)) k_leja_step(const StepParams p) {
    using W = typename Storage<PREC>::W;
    using Val = typename Storage<PREC>::V;
    using PS = typename Storage<PREC>::P;
    constexpr int U = GATHER_BATCH;
    extern __shared__ __align__(16) unsigned char smem[];

    const int tid = threadIdx.x;
    const int b = p.b;
    const int rlane = tid / b;
    const int col = tid - rlane * b;
    const bool active = rlane < p.rl;
    const int R = p.rl * p.rpt;
    const int n = p.n;
    StepSmem<PREC> sm(smem, R, p.smem_cap);

    const W* __restrict__ win = static_cast<const W*>(p.win);
    W* __restrict__ wout = static_cast<W*>(p.wout);
    const Val* __restrict__ vals = static_cast<const Val*>(p.vals);
    const W* __restrict__ vblk = static_cast<const W*>(p.v);
    PS* __restrict__ pblk = static_cast<PS*>(p.p);
    const int* __restrict__ rowptr = p.rowptr;
    const int* __restrict__ colind = p.colind;
    const long long ldw = p.ldw;

    // stage the CSR segment of a tile into shared buffer `buf` (asynchronous copies)
    auto stage = [&](int tile, int buf, int nz0, int nz1) {
        const int r0 = tile * R;
        const int nrows = min(R, n - r0);
        for (int i = tid; i <= nrows; i += blockDim.x) cp_async4(sm.rp(buf) + i, &rowptr[r0 + i]);
        const int cnt = nz1 - nz0;
        if (cnt <= p.smem_cap) {
            int* sc = sm.col(buf);
            Val* sv = sm.val(buf);
            for (int i = tid; i < cnt; i += blockDim.x) {
                cp_async4(sc + i, &colind[nz0 + i]);
                if constexpr (sizeof(Val) == 8) cp_async8(sv + i, &vals[nz0 + i]);
                else cp_async4(sv + i, &vals[nz0 + i]);
            }
        }
        cp_async_commit();
    };
    // prefetch into L2 the streamed operands of a tile ahead: its own W_j, V / P rows and the
    // far-neighbour rows W_j[r + F] that a banded matrix touches first
    auto prefetch_tile = [&](int tile) {
        if (p.pf_dist <= 0 || tile >= p.num_tiles || tid >= 32) return;
        const long long lo = (long long)tile * R, hi = lo + R;
        prefetch_rows_l2(win, ldw, (int)sizeof(W), lo, hi, n);
        if (p.pf_far > 0) prefetch_rows_l2(win, ldw, (int)sizeof(W), lo + p.pf_far, hi + p.pf_far, n);
        if constexpr (MODE == MODE_DOT) prefetch_rows_l2(vblk, p.ldv, (int)sizeof(W), lo, hi, n);
        if constexpr (MODE == MODE_ACCUM) {
            if (!p.first) prefetch_rows_l2(pblk, p.ldp, (int)sizeof(PS), lo, hi, n);
        }
    };

    // per-thread trace partials (one column per thread)
    Acc<LL_PREC_DF64> tq{}, t0q{};   // double-float trace partials (F32 and DF64 modes)
    double t_acc = 0.0, t0_acc = 0.0;

    int tile = blockIdx.x;
    int nz0 = rowptr[tile * R], nz1 = rowptr[min(tile * R + R, n)];
    stage(tile, 0, nz0, nz1);
    for (int d = 1; d <= p.pf_dist; ++d) prefetch_tile(tile + d * (int)gridDim.x);
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
        if (p.pf_dist > 0) prefetch_tile(tile + (p.pf_dist + 1) * (int)gridDim.x);
        // bounds of the tile after next, loaded now and consumed one iteration later
        const int ftile = ntile + gridDim.x;
        int fz0 = 0, fz1 = 0;
        if (ftile < p.num_tiles) { fz0 = rowptr[ftile * R]; fz1 = rowptr[min(ftile * R + R, n)]; }

        const int r0 = tile * R;
        const int r1 = min(r0 + R, n);
        const bool in_smem = (nz1 - nz0) <= p.smem_cap;
        const int* rp = sm.rp(buf);
        const int* cols = in_smem ? sm.col(buf) : colind + nz0;
        const Val* vv = in_smem ? sm.val(buf) : vals + nz0;

        if (active) {
            for (int t = 0; t < p.rpt; t += RB) {
                int kq0[RB], nk[RB], rr[RB];
                bool has[RB];
                W wr[RB], vr[RB];
                PS po[RB];
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    rr[q] = rlane + p.rl * (t + q);
                    has[q] = (t + q < p.rpt) && (r0 + rr[q] < r1);
                    kq0[q] = has[q] ? rp[rr[q]] - nz0 : 0;
                    nk[q] = has[q] ? rp[rr[q] + 1] - rp[rr[q]] : 0;
                }
                if (!has[0]) break;
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    wr[q] = W{};
                    vr[q] = W{};
                    po[q] = PS{};
                    if (has[q]) {
                        const size_t rq = (size_t)(r0 + rr[q]);
                        wr[q] = win[rq * ldw + col];
                        if constexpr (MODE == MODE_ACCUM) {
                            if (!p.first) po[q] = pblk[rq * p.ldp + col];
                        }
                        if constexpr (MODE == MODE_DOT) vr[q] = vblk[rq * p.ldv + col];
                    }
                }
                Acc<PREC> acc[RB];
#pragma unroll
                for (int q = 0; q < RB; ++q) acc[q] = Acc<PREC>{};
                int nmax = nk[0];
#pragma unroll
                for (int q = 1; q < RB; ++q) nmax = max(nmax, nk[q]);
                for (int kb = 0; kb < nmax; kb += U) {
                    W x[RB][U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            if (kb + u < nk[q]) x[q][u] = win[(size_t)cols[kq0[q] + kb + u] * ldw + col];
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            if (kb + u < nk[q]) mac(acc[q], vv[kq0[q] + kb + u], x[q][u]);
                    }
                }
                // epilogue: shift, store, P-axpy or trace
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    if (!has[q]) continue;
                    const size_t rq = (size_t)(r0 + rr[q]);
                    const size_t own = rq * ldw + col;
                    if constexpr (PREC == LL_PREC_F64) {
                        const double wn = fma(p.beta, wr[q], acc[q].v);
                        wout[own] = wn;
                        if constexpr (MODE == MODE_ACCUM) {
                            const double base = p.first ? p.d0 * wr[q] : po[q];
                            pblk[rq * p.ldp + col] = fma(p.dn, wn, base);
                        }
                        if constexpr (MODE == MODE_DOT) {
                            t_acc = fma(vr[q], wn, t_acc);
                            if (p.first) t0_acc = fma(vr[q], wr[q], t0_acc);
                        }
                    } else if constexpr (PREC == LL_PREC_F32_MIXED) {
                        const float wn = fmaf((float)p.beta, wr[q], acc[q].v);
                        wout[own] = wn;
                        if constexpr (MODE == MODE_ACCUM) {
                            // P (double-float) += d_{j+1} W_{j+1}, all on the FP32 pipes
                            float ph, pl;
                            if (p.first) {
                                ph = 0.f; pl = 0.f;
                                df_mac(ph, pl, p.d0_df.x, p.d0_df.y, wr[q], 0.f);
                            } else {
                                ph = po[q].x; pl = po[q].y;
                            }
                            df_mac(ph, pl, p.dn_df.x, p.dn_df.y, wn, 0.f);
                            pblk[rq * p.ldp + col] = df_norm(ph, pl);
                        }
                        if constexpr (MODE == MODE_DOT) {
                            // exact FP32 products accumulated in double-float
                            df_mac(tq.h, tq.l, vr[q], 0.f, wn, 0.f);
                            if (p.first) df_mac(t0q.h, t0q.l, vr[q], 0.f, wr[q], 0.f);
                        }
                    } else {  // LL_PREC_DF64
                        float sh = acc[q].h, sl = acc[q].l;
                        df_mac(sh, sl, p.beta_df.x, p.beta_df.y, wr[q].x, wr[q].y);
                        const float2 wn = df_norm(sh, sl);
                        wout[own] = wn;
                        if constexpr (MODE == MODE_ACCUM) {
                            float ph, pl;
                            if (p.first) {
                                ph = 0.f; pl = 0.f;
                                df_mac(ph, pl, p.d0_df.x, p.d0_df.y, wr[q].x, wr[q].y);
                            } else {
                                ph = po[q].x; pl = po[q].y;
                            }
                            df_mac(ph, pl, p.dn_df.x, p.dn_df.y, wn.x, wn.y);
                            pblk[rq * p.ldp + col] = df_norm(ph, pl);
                        }
                        if constexpr (MODE == MODE_DOT) {
                            df_mac(tq.h, tq.l, vr[q].x, vr[q].y, wn.x, wn.y);
                            if (p.first) df_mac(t0q.h, t0q.l, vr[q].x, vr[q].y, wr[q].x, wr[q].y);
                        }
                    }
                }
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

    if constexpr (MODE == MODE_DOT) {
        if constexpr (PREC != LL_PREC_F64) {
            t_acc = (double)tq.h + (double)tq.l;
            t0_acc = (double)t0q.h + (double)t0q.l;
        }
        // block reduction per column, in row-lane order (deterministic)
        double* red = reinterpret_cast<double*>(smem);
        __shared__ bool s_last;
        const int nred = p.first ? 2 : 1;
        for (int q = 0; q < nred; ++q) {
            red[tid] = (q == 0) ? t_acc : t0_acc;
            __syncthreads();
            if (tid < b) {
                double s = 0.0;
                for (int l = 0; l < p.rl; ++l) s += red[l * b + tid];
                p.partials[((size_t)q * gridDim.x + blockIdx.x) * b + tid] = s;
            }
            __syncthreads();
        }
        __threadfence();
        if (tid == 0) s_last = (atomicAdd(p.ticket, 1u) == gridDim.x - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int c = tid; c < nred * b; c += blockDim.x) {
                const int q = c / b, cc = c - q * b;
                double s = 0.0;
                for (int g = 0; g < (int)gridDim.x; ++g) s += __ldcg(&p.partials[((size_t)q * gridDim.x + g) * b + cc]);
                if (q == 0) p.dots_next[cc] = s; else p.dots_first[cc] = s;
            }
            if (tid == 0) *p.ticket = 0u;
        }
    }
}

template <int PREC, int MODE, int RB>
static cudaError_t launch_typed(const StepLaunch& L, const StepParams& p, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_leja_step<PREC, MODE, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_leja_step<PREC, MODE, RB><<<L.grid, L.threads, L.smem, s>>>(p);
    return cudaGetLastError();
}

template <int PREC, int MODE, int RB>
static int occupancy(int threads, size_t smem) {
    cudaFuncSetAttribute(k_leja_step<PREC, MODE, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leja_step<PREC, MODE, RB>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return per_sm;
}

template <int PREC, int MODE>
static int occupancy_rb(int rb, int threads, size_t smem) {
    return rb == 2 ? occupancy<PREC, MODE, 2>(threads, smem) : occupancy<PREC, MODE, 1>(threads, smem);
}

static size_t val_size(int precision) { return precision == LL_PREC_F32_MIXED ? 4 : 8; }

StepLaunch plan_step(int precision, int mode, int n, int64_t nnz, int b, int threads_target, int rpt,
                     StepParams& p, int sm_count) {
    StepLaunch L{};
    if (threads_target <= 0) threads_target = 512;
    if (rpt <= 0) rpt = 8;
    if (threads_target > STEP_MAX_THREADS) threads_target = STEP_MAX_THREADS;
    int rl = threads_target / b;
    if (rl < 1) rl = 1;
    while (rl > 1 && rl * b > STEP_MAX_THREADS) --rl;
    L.threads = ((rl * b + 31) / 32) * 32;
    if (p.rb != 1 && p.rb != 2) p.rb = 1;
    if (p.rb == 2 && (rpt & 1)) ++rpt;
    const int R = rl * rpt;
    p.rl = rl;
    p.rpt = rpt;
    p.b = b;
    p.n = n;
    p.num_tiles = (n + R - 1) / R;
    // shared staging (two buffers): expected tile nnz with 2x headroom, capped at 48 KB in all
    const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    int64_t cap = (int64_t)(avg * R * 2.0) + 64;
    const size_t vs = val_size(precision);
    const size_t fixed = align16((size_t)(R + 1) * 4);
    const int64_t cap_max = (int64_t)((24 * 1024 - fixed - 32) / (4 + vs));
    if (cap > cap_max) cap = cap_max;
    p.smem_cap = (int)cap;
    size_t smem = 2 * (fixed + align16((size_t)cap * 4) + align16((size_t)cap * vs));
    const size_t red = (size_t)L.threads * 8;
    if (mode == MODE_DOT && smem < red) smem = red;
    L.smem = smem;
    // persistent grid: resident CTAs per SM from the occupancy calculator
    int per_sm = 1;
    switch (precision * 3 + mode) {
#define OCC(P_, M_) case P_ * 3 + M_: per_sm = occupancy_rb<P_, M_>(p.rb, L.threads, smem); break;
        OCC(LL_PREC_F64, MODE_PLAIN) OCC(LL_PREC_F64, MODE_ACCUM) OCC(LL_PREC_F64, MODE_DOT)
        OCC(LL_PREC_DF64, MODE_PLAIN) OCC(LL_PREC_DF64, MODE_ACCUM) OCC(LL_PREC_DF64, MODE_DOT)
        OCC(LL_PREC_F32_MIXED, MODE_PLAIN) OCC(LL_PREC_F32_MIXED, MODE_ACCUM) OCC(LL_PREC_F32_MIXED, MODE_DOT)
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
    switch ((precision * 3 + mode) * 2 + (p.rb == 2 ? 1 : 0)) {
#define LCH(P_, M_) case (P_ * 3 + M_) * 2: return launch_typed<P_, M_, 1>(L, p, s); \
                    case (P_ * 3 + M_) * 2 + 1: return launch_typed<P_, M_, 2>(L, p, s);
        LCH(LL_PREC_F64, MODE_PLAIN) LCH(LL_PREC_F64, MODE_ACCUM) LCH(LL_PREC_F64, MODE_DOT)
        LCH(LL_PREC_DF64, MODE_PLAIN) LCH(LL_PREC_DF64, MODE_ACCUM) LCH(LL_PREC_DF64, MODE_DOT)
        LCH(LL_PREC_F32_MIXED, MODE_PLAIN) LCH(LL_PREC_F32_MIXED, MODE_ACCUM) LCH(LL_PREC_F32_MIXED, MODE_DOT)
#undef LCH
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ll
