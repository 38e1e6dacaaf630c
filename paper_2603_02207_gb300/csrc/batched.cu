// Batched Léja passes: many independent matrices, all their Léja steps, in one persistent launch.
//
// Work items are (step j, matrix i, row tile t), numbered step-major (all tiles of step 0 of every
// matrix, then step 1 of every matrix whose degree exceeds 1, ...); matrices are sorted by degree
// (descending) so the matrices still active at step j are a prefix. CTAs take item numbers from a
// global ticket counter. An item may start only when every tile of step j-1 of its own matrix has
// been released; a CTA takes a new ticket only after finishing its item, and every dependency of
// an item has a smaller ticket, so the smallest unfinished item can always proceed and the launch
// cannot deadlock whatever the residency. Waits spin on a per-matrix release counter with a
// clock64 budget; when it runs out (or another CTA reported a failure) the CTA sets the error flag
// and returns, and the host reports LL_ERR_TIMEOUT.
//
// The last tile of (i, j) to arrive (arrival counter) reduces the per-tile trace partials of the
// step in a fixed order and only then releases the step (release counter), so the partial slots
// and the ping-pong buffers of matrix i are never reused while still being read. Blocks written by
// other CTAs during the launch (W, P) are read through L2 (ld.global.cg): L1 is not coherent.
#include "common.cuh"
#include "kernels.cuh"

namespace ll {

namespace {

template <int PREC> struct BPair;
template <> struct BPair<LL_PREC_F64> { using W = double2; using P = double2; using Raw = double; };
template <> struct BPair<LL_PREC_DF64> { using W = ulonglong2; using P = ulonglong2; using Raw = float2; };
template <> struct BPair<LL_PREC_F32_MIXED> { using W = f2x; using P = ulonglong2; using Raw = float; };

__device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ ulonglong2 ldcg(const ulonglong2* p) { return __ldcg(p); }
__device__ __forceinline__ f2x ldcg(const f2x* p) { return __ldcg(reinterpret_cast<const unsigned long long*>(p)); }

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr int BATCH_U = 8;

}  // namespace

template <int PREC, int MODE>
__global__ void __launch_bounds__(BATCH_THREADS) k_leja_batched(const BatchParams bp) {
    using WP = typename BPair<PREC>::W;
    using PP = typename BPair<PREC>::P;
    using Raw = typename BPair<PREC>::Raw;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item[3];
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int tp = bp.tp;
    const int rlane = tid / tp;
    const int cp = tid - rlane * tp;
    const bool active = rlane < bp.rl;
    const int R = bp.rl * bp.rpt;
    const long long ldq = bp.ld >> 1;
    int* s_rp = reinterpret_cast<int*>(smem);
    int* s_col = s_rp + ((R + 1 + 3) & ~3);
    Raw* s_val = reinterpret_cast<Raw*>(s_col + ((bp.smem_cap + 3) & ~3));
    const f2x zero2 = 0ull;

    for (;;) {
        // take the next work item and decode it into (step, matrix, tile)
        if (tid == 0) {
            const int g = (int)atomicAdd(bp.ticket, 1u);
            int j = -1, i = 0, t = 0;
            if (g < bp.total_items && !*bp.error) {
                int lo = 0, hi = bp.max_m - 1;
                while (lo < hi) {                       // last step whose offset is <= g
                    const int mid = (lo + hi + 1) >> 1;
                    if (bp.step_off[mid] <= g) lo = mid; else hi = mid - 1;
                }
                j = lo;
                const int local = g - bp.step_off[j];
                int a = 0, b = bp.step_active[j] - 1;   // last active matrix whose tile prefix <= local
                while (a < b) {
                    const int mid = (a + b + 1) >> 1;
                    if (bp.tile_prefix[mid] <= local) a = mid; else b = mid - 1;
                }
                i = a;
                t = local - bp.tile_prefix[i];
            }
            s_item[0] = j;
            s_item[1] = i;
            s_item[2] = t;
            s_abort = 0;
            if (j > 0) {
                // wait until step j-1 of matrix i has been released (bounded)
                const unsigned long long need = (unsigned long long)j * bp.mats[i].T;
                const long long t0 = clock64();
                while (ld_acquire(&bp.released[i]) < need) {
                    if (*((volatile int*)bp.error) || clock64() - t0 > bp.spin_budget) {
                        atomicExch(bp.error, 1);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            __threadfence();
        }
        __syncthreads();
        const int j = s_item[0];
        if (j < 0 || s_abort) return;
        const int i = s_item[1], t = s_item[2];
        const BatchMat M = bp.mats[i];
        const int n = M.n;
        const int r0 = t * R, r1 = min(r0 + R, n);
        const WP* win = static_cast<const WP*>(j == 0 ? M.w0 : ((j & 1) ? M.wa : M.wb));
        WP* wout = static_cast<WP*>((j & 1) ? M.wb : M.wa);
        const WP* vblk = static_cast<const WP*>(M.w0);
        PP* pblk = static_cast<PP*>(M.p);
        const Raw* vals = static_cast<const Raw*>(M.vals);
        const double beta = M.coef[2 * j], dnext = M.coef[2 * (j + 1) + 1], d0 = M.coef[1];
        const float2 beta_df = df_split(beta), dn_df = df_split(dnext), d0_df = df_split(d0);
        const f2x bh2 = f2_pack(beta_df.x, beta_df.x), bl2 = f2_pack(beta_df.y, beta_df.y), nbh2 = f2_pack(-beta_df.x, -beta_df.x);
        const f2x beta2 = f2_pack((float)beta, (float)beta);
        const f2x dnh2 = f2_pack(dn_df.x, dn_df.x), dnl2 = f2_pack(dn_df.y, dn_df.y), ndnh2 = f2_pack(-dn_df.x, -dn_df.x);
        const f2x d0h2 = f2_pack(d0_df.x, d0_df.x), d0l2 = f2_pack(d0_df.y, d0_df.y), nd0h2 = f2_pack(-d0_df.x, -d0_df.x);
        const bool first = (j == 0);

        // stage the tile's CSR segment (synchronous; the item changes every tile)
        const int nz0 = M.rowptr[r0], nz1 = M.rowptr[r1];
        const bool in_smem = (nz1 - nz0) <= bp.smem_cap;
        for (int q = tid; q <= r1 - r0; q += blockDim.x) s_rp[q] = M.rowptr[r0 + q] - nz0;
        if (in_smem)
            for (int q = tid; q < nz1 - nz0; q += blockDim.x) { s_col[q] = M.colind[nz0 + q]; s_val[q] = vals[nz0 + q]; }
        __syncthreads();
        const int* cols = in_smem ? s_col : M.colind + nz0;
        const Raw* vv = in_smem ? s_val : vals + nz0;

        f2x th2 = 0ull, tl2 = 0ull, t0h2 = 0ull, t0l2 = 0ull;
        double td[2] = {0.0, 0.0}, t0d[2] = {0.0, 0.0};
        if (active && 2 * cp < bp.b) {
            for (int tt = 0; tt < bp.rpt; ++tt) {
                const int rr = rlane + bp.rl * tt;
                const int r = r0 + rr;
                if (r >= r1) break;
                const int k0 = s_rp[rr], nk = s_rp[rr + 1] - s_rp[rr];
                const size_t own = (size_t)r * ldq + cp;
                const WP wr = ldcg(&win[own]);
                PP po{};
                WP vr{};
                if constexpr (MODE == MODE_ACCUM) { if (!first) po = ldcg(&pblk[own]); }
                if constexpr (MODE == MODE_DOT) vr = vblk[own];
                double a0 = 0.0, a1 = 0.0;
                f2x ah = 0ull, al = 0ull;
                for (int kb = 0; kb < nk; kb += BATCH_U) {
                    WP x[BATCH_U];
#pragma unroll
                    for (int u = 0; u < BATCH_U; ++u)
                        if (kb + u < nk) x[u] = ldcg(&win[(size_t)cols[k0 + kb + u] * ldq + cp]);
#pragma unroll
                    for (int u = 0; u < BATCH_U; ++u) {
                        if (kb + u < nk) {
                            const Raw v = vv[k0 + kb + u];
                            if constexpr (PREC == LL_PREC_F64) {
                                a0 = fma(v, x[u].x, a0);
                                a1 = fma(v, x[u].y, a1);
                            } else if constexpr (PREC == LL_PREC_DF64) {
                                df2_mac(ah, al, f2_pack(v.x, v.x), f2_pack(v.y, v.y), f2_pack(-v.x, -v.x), x[u].x, x[u].y);
                            } else {
                                ah = f2_fma(f2_pack(v, v), x[u], ah);
                            }
                        }
                    }
                }
                if constexpr (PREC == LL_PREC_F64) {
                    const double w0 = fma(beta, wr.x, a0), w1 = fma(beta, wr.y, a1);
                    wout[own] = make_double2(w0, w1);
                    if constexpr (MODE == MODE_ACCUM) {
                        const double b0 = first ? d0 * wr.x : po.x, b1 = first ? d0 * wr.y : po.y;
                        pblk[own] = make_double2(fma(dnext, w0, b0), fma(dnext, w1, b1));
                    }
                    if constexpr (MODE == MODE_DOT) {
                        td[0] = fma(vr.x, w0, td[0]);
                        td[1] = fma(vr.y, w1, td[1]);
                        if (first) { t0d[0] = fma(vr.x, wr.x, t0d[0]); t0d[1] = fma(vr.y, wr.y, t0d[1]); }
                    }
                } else if constexpr (PREC == LL_PREC_DF64) {
                    df2_mac(ah, al, bh2, bl2, nbh2, wr.x, wr.y);
                    f2x wh, wl;
                    df2_norm(ah, al, wh, wl);
                    wout[own] = make_ulonglong2(wh, wl);
                    if constexpr (MODE == MODE_ACCUM) {
                        f2x ph = zero2, pl = zero2;
                        if (first) df2_mac(ph, pl, d0h2, d0l2, nd0h2, wr.x, wr.y);
                        else { ph = po.x; pl = po.y; }
                        df2_mac(ph, pl, dnh2, dnl2, ndnh2, wh, wl);
                        f2x oh, ol;
                        df2_norm(ph, pl, oh, ol);
                        pblk[own] = make_ulonglong2(oh, ol);
                    }
                    if constexpr (MODE == MODE_DOT) {
                        const f2x nvh = f2_sub(zero2, vr.x);
                        df2_mac_pp(th2, tl2, vr.x, vr.y, nvh, wh, wl);
                        if (first) df2_mac_pp(t0h2, t0l2, vr.x, vr.y, nvh, wr.x, wr.y);
                    }
                } else {
                    const f2x wn = f2_fma(beta2, wr, ah);
                    wout[own] = wn;
                    if constexpr (MODE == MODE_ACCUM) {
                        f2x ph = zero2, pl = zero2;
                        if (first) df2_mac_f(ph, pl, d0h2, d0l2, nd0h2, wr);
                        else { ph = po.x; pl = po.y; }
                        df2_mac_f(ph, pl, dnh2, dnl2, ndnh2, wn);
                        f2x oh, ol;
                        df2_norm(ph, pl, oh, ol);
                        pblk[own] = make_ulonglong2(oh, ol);
                    }
                    if constexpr (MODE == MODE_DOT) {
                        const f2x nv = f2_sub(zero2, vr);
                        df2_mac_f(th2, tl2, vr, zero2, nv, wn);
                        if (first) df2_mac_f(t0h2, t0l2, vr, zero2, nv, wr);
                    }
                }
            }
        }

        __shared__ bool s_last;
        if constexpr (MODE == MODE_DOT) {
            if constexpr (PREC != LL_PREC_F64) {
                float h0, h1, l0, l1;
                f2_unpack(th2, h0, h1); f2_unpack(tl2, l0, l1);
                td[0] = (double)h0 + (double)l0; td[1] = (double)h1 + (double)l1;
                f2_unpack(t0h2, h0, h1); f2_unpack(t0l2, l0, l1);
                t0d[0] = (double)h0 + (double)l0; t0d[1] = (double)h1 + (double)l1;
            }
            // per-tile partial of every column (row lanes summed in a fixed order)
            double* red = reinterpret_cast<double*>(smem);
            __syncthreads();
            const int nred = first ? 2 : 1;
            for (int q = 0; q < nred; ++q) {
                red[2 * tid] = q ? t0d[0] : td[0];
                red[2 * tid + 1] = q ? t0d[1] : td[1];
                __syncthreads();
                for (int c = tid; c < bp.b; c += blockDim.x) {
                    double sacc = 0.0;
                    for (int l = 0; l < bp.rl; ++l) sacc += red[2 * (l * tp + (c >> 1)) + (c & 1)];
                    M.partials[((size_t)q * M.T + t) * bp.b + c] = sacc;
                }
                __syncthreads();
            }
        }
        // arrival; the last tile of (i, j) reduces the step's partials, then releases the step
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned long long a = atomicAdd(&bp.arrived[i], 1ull);
            s_last = (a + 1 == (unsigned long long)(j + 1) * M.T);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if constexpr (MODE == MODE_DOT) {
                const int nred = first ? 2 : 1;
                for (int c = tid; c < nred * bp.b; c += blockDim.x) {
                    const int q = c / bp.b, cc = c - q * bp.b;
                    double sacc = 0.0;
                    for (int tt = 0; tt < M.T; ++tt) sacc += __ldcg(&M.partials[((size_t)q * M.T + tt) * bp.b + cc]);
                    if (q == 0) M.dots[(size_t)(j + 1) * bp.b + cc] = sacc; else M.dots[cc] = sacc;
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(&bp.released[i], (unsigned long long)M.T);
        }
        __syncthreads();
    }
}

template <int PREC, int MODE>
static cudaError_t launch_batched_typed(const BatchParams& bp, int grid, size_t smem, cudaStream_t s) {
    cudaFuncSetAttribute(k_leja_batched<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k_leja_batched<PREC, MODE><<<grid, BATCH_THREADS, smem, s>>>(bp);
    return cudaGetLastError();
}

void plan_batched(int b, double avg_nnz_per_row, BatchParams& bp, size_t* smem) {
    const int tp = (b + 1) / 2;
    int rl = BATCH_THREADS / tp;
    if (rl < 1) rl = 1;
    bp.tp = tp;
    bp.rl = rl;
    bp.rpt = 4;
    bp.b = b;
    const int R = rl * bp.rpt;
    bp.R = R;
    int cap = (int)(avg_nnz_per_row * R * 1.5) + 64;
    const size_t vs = 8;
    const size_t fixed = (size_t)((R + 1 + 3) & ~3) * 4;
    while (cap > 64 && fixed + (size_t)((cap + 3) & ~3) * 4 + (size_t)cap * vs > 40 * 1024) cap = cap * 7 / 8;
    bp.smem_cap = cap;
    size_t sm = fixed + (size_t)((cap + 3) & ~3) * 4 + (size_t)cap * vs + 16;
    const size_t red = (size_t)BATCH_THREADS * 2 * sizeof(double);
    if (sm < red) sm = red;
    *smem = sm;
}

cudaError_t launch_batched(int precision, int mode, const BatchParams& bp, int grid, size_t smem, cudaStream_t s) {
    switch (precision * NUM_MODES + mode) {
        case LL_PREC_F64 * NUM_MODES + MODE_ACCUM: return launch_batched_typed<LL_PREC_F64, MODE_ACCUM>(bp, grid, smem, s);
        case LL_PREC_F64 * NUM_MODES + MODE_DOT: return launch_batched_typed<LL_PREC_F64, MODE_DOT>(bp, grid, smem, s);
        case LL_PREC_DF64 * NUM_MODES + MODE_ACCUM: return launch_batched_typed<LL_PREC_DF64, MODE_ACCUM>(bp, grid, smem, s);
        case LL_PREC_DF64 * NUM_MODES + MODE_DOT: return launch_batched_typed<LL_PREC_DF64, MODE_DOT>(bp, grid, smem, s);
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_ACCUM: return launch_batched_typed<LL_PREC_F32_MIXED, MODE_ACCUM>(bp, grid, smem, s);
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_DOT: return launch_batched_typed<LL_PREC_F32_MIXED, MODE_DOT>(bp, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ll
