// Fused Léja-step kernel (Algorithm 2 loop body over a whole probe block) and its launch plan.
//
// One launch applies W_{j+1} = (B - xi_j I) W_j to every column of an n x b row-major block,
// streaming the CSR matrix once, and fuses the per-step epilogue:
//   pass 1 (MODE_ACCUM): P += d_{j+1} W_{j+1}                (Algorithm 2, P_m = P_{m-1} + d_m w_m)
//   pass 2 (MODE_DOT):   t_{j+1}[col] = <V[:, col], W_{j+1}[:, col]>   (Algorithm 3 steps 5-6)
//   MODE_PLAIN:          W_{j+1} only (recomputation in the adjoint);
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

namespace ll {

template <int PREC> struct PairT;
// W / V pair, P pair, raw CSR value (as prepared in global memory)
template <> struct PairT<LL_PREC_F64> { using W = double2; using P = double2; using Raw = double; };
template <> struct PairT<LL_PREC_DF64> { using W = ulonglong2; using P = ulonglong2; using Raw = float2; };
template <> struct PairT<LL_PREC_F32_MIXED> { using W = f2x; using P = ulonglong2; using Raw = float; };

// value expanded for the f32x2 instructions: DF64 (ah2, al2, nah2), F32 (a2), F64 (a)
struct ExDF { f2x ah2, al2, nah2; };
template <int PREC> struct ExT;
template <> struct ExT<LL_PREC_F64> { using T = double; };
template <> struct ExT<LL_PREC_DF64> { using T = ExDF; };
template <> struct ExT<LL_PREC_F32_MIXED> { using T = f2x; };

__device__ __forceinline__ double expand(double a) { return a; }
__device__ __forceinline__ ExDF expand(float2 a) { return ExDF{f2_pack(a.x, a.x), f2_pack(a.y, a.y), f2_pack(-a.x, -a.x)}; }
__device__ __forceinline__ f2x expand(float a) { return f2_pack(a, a); }

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
    extern __shared__ __align__(16) unsigned char smem[];

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

    // per-step scalars broadcast to both lanes (beta_j, d_{j+1}, d_0 as double-float)
    const f2x bh2 = f2_pack(p.beta_df.x, p.beta_df.x), bl2 = f2_pack(p.beta_df.y, p.beta_df.y);
    const f2x nbh2 = f2_pack(-p.beta_df.x, -p.beta_df.x);
    const f2x beta2 = f2_pack((float)p.beta, (float)p.beta);
    const f2x dnh2 = f2_pack(p.dn_df.x, p.dn_df.x), dnl2 = f2_pack(p.dn_df.y, p.dn_df.y);
    const f2x ndnh2 = f2_pack(-p.dn_df.x, -p.dn_df.x);
    const f2x d0h2 = f2_pack(p.d0_df.x, p.d0_df.x), d0l2 = f2_pack(p.d0_df.y, p.d0_df.y);
    const f2x nd0h2 = f2_pack(-p.d0_df.x, -p.d0_df.x);
    const f2x zero2 = 0ull;
    // ADJ: lane-wise coefficients of the thread's two columns
    const bool q0 = 2 * cp < p.adj_split, q1 = 2 * cp + 1 < p.adj_split;
    const double cadj0 = q0 ? p.adj_q : p.adj_g, cadj1 = q1 ? p.adj_q : p.adj_g;
    const float2 cdf0 = q0 ? p.adj_q_df : p.adj_g_df, cdf1 = q1 ? p.adj_q_df : p.adj_g_df;
    const f2x ch2 = f2_pack(cdf0.x, cdf1.x), cl2 = f2_pack(cdf0.y, cdf1.y), nch2 = f2_pack(-cdf0.x, -cdf1.x);
    const f2x cf2 = f2_pack((float)cadj0, (float)cadj1);

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

    // trace partials of the thread's two columns (double-float; FP64 in the F64 mode)
    f2x th2 = 0ull, tl2 = 0ull, t0h2 = 0ull, t0l2 = 0ull;
    double td[2] = {0.0, 0.0}, t0d[2] = {0.0, 0.0};

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
                if constexpr (MODE == MODE_ACCUM) {
                    if (!p.first) po = pblk[(size_t)r * ldpq + cp];
                }
                if constexpr (MODE == MODE_DOT || MODE == MODE_ADJ) vr = vblk[(size_t)r * ldvq + cp];

                // accumulate sum_k a_k W_j[c_k, pair]
                double a0 = 0.0, a1 = 0.0;             // F64
                f2x ah = 0ull, al = 0ull;              // DF64 (hi, lo pairs); F32 uses ah
                for (int kb = 0; kb < nk; kb += U) {
                    WP x[U];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (kb + u < nk) x[u] = win[(size_t)cols[k0 + kb + u] * ldq + cp];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (kb + u < nk) {
                            const int k = k0 + kb + u;
                            if constexpr (PREC == LL_PREC_F64) {
                                const double v = rawv[k];
                                a0 = fma(v, x[u].x, a0);
                                a1 = fma(v, x[u].y, a1);
                            } else if constexpr (PREC == LL_PREC_DF64) {
                                const ExDF v = in_smem ? ex[k] : expand(rawv[k]);
                                df2_mac(ah, al, v.ah2, v.al2, v.nah2, x[u].x, x[u].y);
                            } else {
                                const f2x v = in_smem ? ex[k] : expand(rawv[k]);
                                ah = f2_fma(v, x[u], ah);
                            }
                        }
                    }
                }
                // epilogue: shift by beta_j, store W_{j+1}, then the P-axpy or the trace
                if constexpr (PREC == LL_PREC_F64) {
                    double w0 = fma(p.beta, wr.x, a0), w1 = fma(p.beta, wr.y, a1);
                    if constexpr (MODE == MODE_ADJ) {
                        w0 = fma(cadj0, vr.x, w0);
                        w1 = fma(cadj1, vr.y, w1);
                    }
                    wout[own] = make_double2(w0, w1);
                    if constexpr (MODE == MODE_ACCUM) {
                        const double b0 = p.first ? p.d0 * wr.x : po.x, b1 = p.first ? p.d0 * wr.y : po.y;
                        pblk[(size_t)r * ldpq + cp] = make_double2(fma(p.dn, w0, b0), fma(p.dn, w1, b1));
                    }
                    if constexpr (MODE == MODE_DOT) {
                        td[0] = fma(vr.x, w0, td[0]);
                        td[1] = fma(vr.y, w1, td[1]);
                        if (p.first) { t0d[0] = fma(vr.x, wr.x, t0d[0]); t0d[1] = fma(vr.y, wr.y, t0d[1]); }
                    }
                } else if constexpr (PREC == LL_PREC_DF64) {
                    df2_mac(ah, al, bh2, bl2, nbh2, wr.x, wr.y);
                    if constexpr (MODE == MODE_ADJ) df2_mac_pp(ah, al, ch2, cl2, nch2, vr.x, vr.y);
                    f2x wh, wl;
                    df2_norm(ah, al, wh, wl);
                    wout[own] = make_ulonglong2(wh, wl);
                    if constexpr (MODE == MODE_ACCUM) {
                        f2x ph = zero2, pl = zero2;
                        if (p.first) df2_mac(ph, pl, d0h2, d0l2, nd0h2, wr.x, wr.y);
                        else { ph = po.x; pl = po.y; }
                        df2_mac(ph, pl, dnh2, dnl2, ndnh2, wh, wl);
                        f2x oh, ol;
                        df2_norm(ph, pl, oh, ol);
                        pblk[(size_t)r * ldpq + cp] = make_ulonglong2(oh, ol);
                    }
                    if constexpr (MODE == MODE_DOT) {
                        const f2x nvh = f2_sub(zero2, vr.x);
                        df2_mac_pp(th2, tl2, vr.x, vr.y, nvh, wh, wl);
                        if (p.first) df2_mac_pp(t0h2, t0l2, vr.x, vr.y, nvh, wr.x, wr.y);
                    }
                } else {  // LL_PREC_F32_MIXED
                    f2x wn = f2_fma(beta2, wr, ah);
                    if constexpr (MODE == MODE_ADJ) wn = f2_fma(cf2, vr, wn);
                    wout[own] = wn;
                    if constexpr (MODE == MODE_ACCUM) {
                        f2x ph = zero2, pl = zero2;
                        if (p.first) df2_mac_f(ph, pl, d0h2, d0l2, nd0h2, wr);
                        else { ph = po.x; pl = po.y; }
                        df2_mac_f(ph, pl, dnh2, dnl2, ndnh2, wn);
                        f2x oh, ol;
                        df2_norm(ph, pl, oh, ol);
                        pblk[(size_t)r * ldpq + cp] = make_ulonglong2(oh, ol);
                    }
                    if constexpr (MODE == MODE_DOT) {
                        // exact FP32 products v * w accumulated in double-float
                        const f2x nv = f2_sub(zero2, vr);
                        df2_mac_f(th2, tl2, vr, zero2, nv, wn);
                        if (p.first) df2_mac_f(t0h2, t0l2, vr, zero2, nv, wr);
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
            float h0, h1, l0, l1;
            f2_unpack(th2, h0, h1);
            f2_unpack(tl2, l0, l1);
            td[0] = (double)h0 + (double)l0;
            td[1] = (double)h1 + (double)l1;
            f2_unpack(t0h2, h0, h1);
            f2_unpack(t0l2, l0, l1);
            t0d[0] = (double)h0 + (double)l0;
            t0d[1] = (double)h1 + (double)l1;
        }
        // block reduction per column, in row-lane order (deterministic)
        double* red = reinterpret_cast<double*>(smem);
        __shared__ bool s_last;
        const int b = p.b;
        const int nred = p.first ? 2 : 1;
        for (int q = 0; q < nred; ++q) {
            red[2 * tid] = q ? t0d[0] : td[0];
            red[2 * tid + 1] = q ? t0d[1] : td[1];
            __syncthreads();
            for (int c = tid; c < b; c += blockDim.x) {
                const int pc = c >> 1, lane = c & 1;
                double s = 0.0;
                for (int l = 0; l < p.rl; ++l) s += red[2 * (l * tp + pc) + lane];
                p.partials[((size_t)q * gridDim.x + blockIdx.x) * b + c] = s;
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
    if (mode == MODE_DOT && smem < red) smem = red;
    L.smem = smem;
    int per_sm = 1;
    switch (precision * NUM_MODES + mode) {
#define OCC(P_, M_) case P_ * NUM_MODES + M_: per_sm = occupancy<P_, M_>(L.threads, smem); break;
#define OCC4(P_) OCC(P_, MODE_PLAIN) OCC(P_, MODE_ACCUM) OCC(P_, MODE_DOT) OCC(P_, MODE_ADJ)
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
#define LCH4(P_) LCH(P_, MODE_PLAIN) LCH(P_, MODE_ACCUM) LCH(P_, MODE_DOT) LCH(P_, MODE_ADJ)
        LCH4(LL_PREC_F64) LCH4(LL_PREC_DF64) LCH4(LL_PREC_F32_MIXED)
#undef LCH4
#undef LCH
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ll
