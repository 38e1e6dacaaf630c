// Banded Léja steps: several steps of Algorithm 2 per launch for matrices whose entries all lie
// within BAND_H = 2 of the diagonal (the paper's pentadiagonal family of Section 5.1, tridiagonal
// and 1-D operators).
//
// A CTA takes a tile of R rows. It loads W_j for the tile and a halo of s * BAND_H rows on each
// side, the five diagonals of the prepared matrix (DIA layout, zeros where the CSR row has no
// entry), and the tile's rows of V (pass 2) or P (pass 1). It then runs s steps in shared memory,
// each over the rows whose inputs are still in the buffer (the halo shrinks by BAND_H per step).
// It writes W_{j+s} and P once, or keeps the traces of every step in registers. Per s steps, W, P
// and V cross HBM once instead of s times; the halo rows are recomputed by both neighbouring
// tiles, with the same operations in the same order, so every row of W_{j+s} is the value the
// one-step kernels produce. The per-row arithmetic is that of step_common.cuh, and the
// diagonals are visited in ascending column order (the CSR order), so P and W match the
// one-step kernels bit for bit. The traces are summed over rows in another order.
#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"

namespace ll {

namespace {

constexpr int BAND_D = 2 * BAND_H + 1;

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout for R rows and tp column pairs (element sizes of the precision)
struct BandSmem {
    size_t w0, w1, dia, aux, bytes;
    __host__ __device__ BandSmem(int R, int tp, size_t wpair, size_t raw, size_t auxpair) {
        const size_t rb = (size_t)R + 2 * BAND_SMAX * BAND_H;
        const size_t rd = (size_t)R + 2 * (BAND_SMAX - 1) * BAND_H;
        w0 = 0;
        w1 = a16(rb * tp * wpair);
        dia = w1 + a16(rb * tp * wpair);
        aux = dia + a16(rd * BAND_D * raw);
        bytes = aux + a16((size_t)R * tp * auxpair);
    }
};

template <int PREC, int MODE>
__global__ void __launch_bounds__(BAND_THREADS) k_leja_band(const BandParams bp) {
    using WP = typename PairT<PREC>::W;
    using PP = typename PairT<PREC>::P;
    using Raw = typename PairT<PREC>::Raw;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int tp = bp.tp, R = bp.R, s = bp.s, n = bp.n;
    const BandSmem L(R, tp, sizeof(WP), sizeof(Raw), MODE == MODE_ACCUM ? sizeof(PP) : sizeof(WP));
    WP* const wbuf0 = reinterpret_cast<WP*>(smem + L.w0);
    WP* const wbuf1 = reinterpret_cast<WP*>(smem + L.w1);
    Raw* const ds = reinterpret_cast<Raw*>(smem + L.dia);
    WP* const vs = reinterpret_cast<WP*>(smem + L.aux);    // pass 2: the tile's V rows
    PP* const ps = reinterpret_cast<PP*>(smem + L.aux);    // pass 1: the tile's P rows
    const int rl = tid / tp, cp = tid - rl * tp;
    const int RL = BAND_THREADS / tp;
    const bool act = rl < RL;
    const long long ldq = bp.ldw >> 1, ldpq = bp.ldp >> 1;
    const WP* __restrict__ win = static_cast<const WP*>(bp.win);
    WP* __restrict__ wout = static_cast<WP*>(bp.wout);
    const Raw* __restrict__ dia = static_cast<const Raw*>(bp.dia);
    const WP* __restrict__ vg = static_cast<const WP*>(bp.v);
    PP* __restrict__ pg = static_cast<PP*>(bp.p);
    const int hs = s * BAND_H;   // input halo of this launch

    TracePart T[BAND_SMAX];
    for (int tile = blockIdx.x; tile < bp.num_tiles; tile += gridDim.x) {
        const int r0 = tile * R;
        const int wbase = r0 - hs;                    // row of buffer index 0
        const int nin = R + 2 * hs;
        for (int idx = tid; idx < nin * tp; idx += BAND_THREADS) {
            const int rr = idx / tp, c = idx - rr * tp;
            const int row = wbase + rr;
            wbuf0[idx] = (row >= 0 && row < n) ? win[(size_t)row * ldq + c] : WP{};
        }
        const int dbase = r0 - (s - 1) * BAND_H;      // row of diagonal index 0
        const int nd = R + 2 * (s - 1) * BAND_H;
        for (int idx = tid; idx < nd * BAND_D; idx += BAND_THREADS) {
            const int rr = idx / BAND_D;
            const int row = dbase + rr;
            ds[idx] = (row >= 0 && row < n) ? dia[(size_t)row * BAND_D + (idx - rr * BAND_D)] : Raw{};
        }
        for (int idx = tid; idx < R * tp; idx += BAND_THREADS) {
            const int rr = idx / tp, c = idx - rr * tp;
            const int row = r0 + rr;
            if constexpr (MODE == MODE_DOT) vs[idx] = row < n ? vg[(size_t)row * ldq + c] : WP{};
            else ps[idx] = (row < n && bp.j0 > 0) ? pg[(size_t)row * ldpq + c] : PP{};
        }
        __syncthreads();
        WP* bin = wbuf0;
        WP* bout = wbuf1;
#pragma unroll
        for (int q = 0; q < BAND_SMAX; ++q) {
            if (q < s) {
                StepParams p{};
                p.first = (bp.j0 + q == 0);
                p.beta = bp.beta[q];
                p.d0 = bp.d0;
                p.dn = bp.dn[q];
                p.beta_df = bp.beta_df[q];
                p.d0_df = bp.d0_df;
                p.dn_df = bp.dn_df[q];
                const StepScalars<PREC> S(p, cp);
                // rows computed at this step: the tile and a halo of (s - 1 - q) * BAND_H rows
                const int lo = r0 - (s - 1 - q) * BAND_H, hi = r0 + R + (s - 1 - q) * BAND_H;
                if (act) {
                    for (int row = lo + rl; row < hi; row += RL) {
                        const int bi = row - wbase;
                        const Raw* drow = ds + (size_t)(row - dbase) * BAND_D;
                        RowAcc A;
#pragma unroll
                        for (int o = 0; o < BAND_D; ++o) {
                            const WP x = bin[(size_t)(bi - BAND_H + o) * tp + cp];
                            if constexpr (PREC == LL_PREC_F64) row_mac<PREC>(A, drow[o], x);
                            else row_mac<PREC>(A, expand(drow[o]), x);
                        }
                        const WP wr = bin[(size_t)bi * tp + cp];
                        WP* wo = bout + (size_t)bi * tp + cp;
                        if (row >= r0 && row < r0 + R && row < n) {
                            const int ti = (row - r0) * tp + cp;
                            if constexpr (MODE == MODE_DOT)
                                row_epilogue<PREC, MODE_DOT>(p, S, A, wr, vs[ti], PP{}, wo, nullptr, T[q]);
                            else
                                row_epilogue<PREC, MODE_ACCUM>(p, S, A, wr, WP{}, ps[ti], wo, ps + ti, T[q]);
                        } else {
                            row_epilogue<PREC, MODE_PLAIN>(p, S, A, wr, WP{}, PP{}, wo, nullptr, T[q]);
                        }
                    }
                }
                __syncthreads();
                WP* t = bin;
                bin = bout;
                bout = t;
            }
        }
        // W_{j+s} (in bin now) and P of the tile's rows
        for (int idx = tid; idx < R * tp; idx += BAND_THREADS) {
            const int rr = idx / tp, c = idx - rr * tp;
            const int row = r0 + rr;
            if (row < n) {
                wout[(size_t)row * ldq + c] = bin[(size_t)(row - wbase) * tp + c];
                if constexpr (MODE == MODE_ACCUM) pg[(size_t)row * ldpq + c] = ps[idx];
            }
        }
        __syncthreads();
    }

    if constexpr (MODE == MODE_DOT) {
        // per-CTA column sums of every step's traces (row lanes in order), then the last CTA sums
        // the CTAs in order: slot q < s holds step q's W_{j+q+1} traces, slot s (first launch)
        // the W_0 traces
        __shared__ bool s_last;
        double* red = reinterpret_cast<double*>(smem);
        const int b = bp.b;
        const int nslot = s + (bp.j0 == 0 ? 1 : 0);
#pragma unroll
        for (int q = 0; q <= BAND_SMAX; ++q) {
            // slot q < s: step q's traces; slot s: the W_0 traces of the first launch (T[0].t0);
            // every index into T is a constant once the loop is unrolled (T stays in registers)
            const bool t0 = q == s;
            if (q < s || (t0 && nslot > s)) {
                const TracePart& Tq = T[q < BAND_SMAX ? q : BAND_SMAX - 1];
                const TracePart& T0 = T[0];
                double v0, v1;
                if constexpr (PREC == LL_PREC_F64) {
                    v0 = t0 ? T0.t0d[0] : Tq.td[0];
                    v1 = t0 ? T0.t0d[1] : Tq.td[1];
                } else {
                    float h0, h1, l0, l1;
                    f2_unpack(t0 ? T0.t0h2 : Tq.th2, h0, h1);
                    f2_unpack(t0 ? T0.t0l2 : Tq.tl2, l0, l1);
                    v0 = (double)h0 + (double)l0;
                    v1 = (double)h1 + (double)l1;
                }
                red[2 * tid] = act ? v0 : 0.0;
                red[2 * tid + 1] = act ? v1 : 0.0;
                __syncthreads();
                for (int c = tid; c < b; c += BAND_THREADS) {
                    const int pc = c >> 1, lane = c & 1;
                    double sum = 0.0;
                    for (int l = 0; l < RL; ++l) sum += red[2 * (l * tp + pc) + lane];
                    bp.partials[((size_t)q * gridDim.x + blockIdx.x) * b + c] = sum;
                }
                __syncthreads();
            }
        }
        __threadfence();
        if (tid == 0) s_last = (atomicAdd(bp.ticket, 1u) == gridDim.x - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int c = tid; c < nslot * b; c += BAND_THREADS) {
                const int q = c / b, cc = c - q * b;
                double sum = 0.0;
                for (int g = 0; g < (int)gridDim.x; ++g) sum += __ldcg(&bp.partials[((size_t)q * gridDim.x + g) * b + cc]);
                const int slot = q < s ? bp.j0 + q + 1 : 0;
                bp.dots[(size_t)slot * b + cc] = sum;
            }
            if (tid == 0) *bp.ticket = 0u;
        }
    }
}

// DIA layout of the prepared values: dia[r * 5 + (c - r + 2)] = a_rc, zero elsewhere. The rows
// have been checked to hold strictly increasing columns within two of the diagonal.
template <typename Raw>
__global__ void k_to_dia(const int32_t* rowptr, const int32_t* colind, const Raw* vals, int n, Raw* dia) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        Raw v[BAND_D];
#pragma unroll
        for (int d = 0; d < BAND_D; ++d) v[d] = Raw{};
        for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const int d = colind[k] - r + BAND_H;
            if (d >= 0 && d < BAND_D) v[d] = vals[k];
        }
#pragma unroll
        for (int d = 0; d < BAND_D; ++d) dia[(size_t)r * BAND_D + d] = v[d];
    }
}

template <int PREC, int MODE>
int band_occupancy(size_t smem) {
    cudaFuncSetAttribute(k_leja_band<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leja_band<PREC, MODE>, BAND_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

template <int PREC, int MODE>
cudaError_t band_launch(const BandLaunch& L, const BandParams& p, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_leja_band<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_leja_band<PREC, MODE><<<L.grid, BAND_THREADS, L.smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

bool plan_band(int precision, int mode, int n, int b, int sm_count, BandLaunch& L) {
    L = BandLaunch{};
    if (n <= 0 || b <= 0 || (mode != MODE_ACCUM && mode != MODE_DOT)) return false;
    const int tp = (b + 1) / 2;
    if (tp > BAND_THREADS) return false;
    const size_t wpair = precision == LL_PREC_F32_MIXED ? 8 : 16;
    const size_t raw = precision == LL_PREC_F32_MIXED ? 4 : 8;
    const size_t auxpair = mode == MODE_ACCUM ? 16 : wpair;
    // the most rows per tile (a multiple of 32, at most 512) within 72 KB of shared memory, so that
    // three CTAs share an SM and one loads while the others compute
    int R = 512;
    while (R > 32 && BandSmem(R, tp, wpair, raw, auxpair).bytes > 72 * 1024) R -= 32;
    const size_t red = (size_t)BAND_THREADS * 2 * sizeof(double);
    size_t smem = BandSmem(R, tp, wpair, raw, auxpair).bytes;
    if (smem < red) smem = red;
    if (smem > 200 * 1024) return false;
    int per_sm = 0;
    switch (precision * NUM_MODES + mode) {
        case LL_PREC_F64 * NUM_MODES + MODE_ACCUM: per_sm = band_occupancy<LL_PREC_F64, MODE_ACCUM>(smem); break;
        case LL_PREC_F64 * NUM_MODES + MODE_DOT: per_sm = band_occupancy<LL_PREC_F64, MODE_DOT>(smem); break;
        case LL_PREC_DF64 * NUM_MODES + MODE_ACCUM: per_sm = band_occupancy<LL_PREC_DF64, MODE_ACCUM>(smem); break;
        case LL_PREC_DF64 * NUM_MODES + MODE_DOT: per_sm = band_occupancy<LL_PREC_DF64, MODE_DOT>(smem); break;
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_ACCUM: per_sm = band_occupancy<LL_PREC_F32_MIXED, MODE_ACCUM>(smem); break;
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_DOT: per_sm = band_occupancy<LL_PREC_F32_MIXED, MODE_DOT>(smem); break;
        default: return false;
    }
    if (per_sm < 1) return false;
    L.R = R;
    L.tp = tp;
    L.num_tiles = (n + R - 1) / R;
    L.smem = smem;
    int grid = per_sm * sm_count;
    if (grid > L.num_tiles) grid = L.num_tiles;
    L.grid = grid < 1 ? 1 : grid;
    return true;
}

cudaError_t launch_band(int precision, int mode, const BandLaunch& L, const BandParams& p, cudaStream_t s) {
    if (p.s < 1 || p.s > BAND_SMAX) return cudaErrorInvalidValue;
    switch (precision * NUM_MODES + mode) {
        case LL_PREC_F64 * NUM_MODES + MODE_ACCUM: return band_launch<LL_PREC_F64, MODE_ACCUM>(L, p, s);
        case LL_PREC_F64 * NUM_MODES + MODE_DOT: return band_launch<LL_PREC_F64, MODE_DOT>(L, p, s);
        case LL_PREC_DF64 * NUM_MODES + MODE_ACCUM: return band_launch<LL_PREC_DF64, MODE_ACCUM>(L, p, s);
        case LL_PREC_DF64 * NUM_MODES + MODE_DOT: return band_launch<LL_PREC_DF64, MODE_DOT>(L, p, s);
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_ACCUM: return band_launch<LL_PREC_F32_MIXED, MODE_ACCUM>(L, p, s);
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_DOT: return band_launch<LL_PREC_F32_MIXED, MODE_DOT>(L, p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_to_dia(int precision, const int32_t* rowptr, const int32_t* colind, const void* vals, int n, void* dia,
                          cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = 152 * 8, threads = 256;
    switch (precision) {
        case LL_PREC_F64: k_to_dia<double><<<grid, threads, 0, s>>>(rowptr, colind, (const double*)vals, n, (double*)dia); break;
        case LL_PREC_DF64: k_to_dia<float2><<<grid, threads, 0, s>>>(rowptr, colind, (const float2*)vals, n, (float2*)dia); break;
        default: k_to_dia<float><<<grid, threads, 0, s>>>(rowptr, colind, (const float*)vals, n, (float*)dia); break;
    }
    return cudaGetLastError();
}

}  // namespace ll
