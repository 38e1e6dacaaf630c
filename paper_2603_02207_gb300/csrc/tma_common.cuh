// Pieces shared by the TMA-fed step kernels (single matrix and batched): mbarrier waits with a
// clock budget, the TMA copy wrappers (2-D tile loads, tile::gather4, 1-D bulk copies), the entry
// record of a tile descriptor and the kernel that builds the descriptors once per pass, and the
// host-side tensor-map encoding.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <climits>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"

namespace ll {

constexpr int TMA_MAX_STAGES = 6;
constexpr int TMA_MAX_THREADS = 608;   // up to 512 consumer threads and three producer warps
constexpr int TMA_MAX_PROD = 3;
constexpr int TMA_GRING = 3;           // gather-column blocks staged up to two tiles ahead
constexpr int TMA_MAX_WIN = 4;         // extra windows per tile (runs of far columns)
// error flag values of the TMA step kernel (the first failure is kept): a bounded wait that ran out
// on the gather-column ring, on a stage's release, on a stage's copies; a tile header out of range
constexpr int TMA_ERR_GCOL = 1, TMA_ERR_EMPTY = 2, TMA_ERR_FULL = 3, TMA_ERR_DESC = 4;
constexpr int TMA_ERR_GRAM = 8;   // a bounded wait of the tensor-core Gram

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
// the same with an L2 cache policy (createpolicy) for the four rows' lines
__device__ __forceinline__ void tma_gather4_hint(uint32_t dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                                 uint32_t bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;\n" ::"r"(dst),
        "l"(map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar), "l"(policy)
        : "memory");
}
// L2 policies: lines kept in preference to others (evict_last) or given up first (evict_first)
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
// 1-D bulk copy global -> shared (both 16-byte aligned, size a multiple of 16) completing on bar
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Entry record of a tile's descriptor: the matrix value as prepared (FP64, float pair, FP32) and
// the byte offset of its operand row W_j[c, :] in the stage (window or gather slot). One
// broadcast shared-memory load per entry in the consumer loop.
template <int PREC> struct Rec;
template <> struct __align__(16) Rec<LL_PREC_F64> { double a; int off, pad; };     // pad: the entry's row in the tile
template <> struct __align__(16) Rec<LL_PREC_DF64> { float2 a; int off, pad; };    // (hi, lo); pad as above
template <> struct __align__(8) Rec<LL_PREC_F32_MIXED> { float a; int off; };
__device__ __forceinline__ int rec_row(const Rec<LL_PREC_F64>& r) { return r.pad; }
__device__ __forceinline__ int rec_row(const Rec<LL_PREC_DF64>& r) { return r.pad; }
__device__ __forceinline__ int rec_row(const Rec<LL_PREC_F32_MIXED>&) { return 0; }   // (not carried)

// Tile descriptors, built once per pass (the matrix and the tile geometry do not change between
// the m steps). One warp per tile of R rows:
//   desc[t]: row offsets rowptr[r0 .. r0 + nr] - z0, then z0 and the record count g, padded to
//            16 bytes; then one record per entry e < g (the value and its operand row's offset in
//            the stage);
//   gcol[t]: the start rows of up to TMA_MAX_WIN extra windows, then the gathered columns in slot
//            order, padded with the last one to a multiple of 4;
//   meta[t]: (g, gathered rows, extra windows, 0).
// Columns inside the tile's own window [r0 - HALO, r0 + R + HALO) point into it. Far columns that
// form runs (a stencil's off-diagonal bands: row r0 + k meets column c + k) are loaded as extra
// windows of R + 2 HALO rows, one 2-D tile copy each instead of a gather per four rows: the
// candidates are the far columns of the tile's first and last rows, shifted to the first row, and
// a candidate is kept when it holds at least half a window of the tile's far entries. The
// windows occupy the first wslots gather slots each; the other far columns take the next gather
// slot in entry order. When the gather slots run out (or after ecap entries) the records stop, and
// that entry and every later entry of the tile load directly.
// ngv > 0 (a sweep over ngv matrices of one pattern): a record is the operand offset (padded to
// the value size, sweep_rec_head bytes), then the values of the ngv matrices, vals[v * vstride + e]
// for v < ngv (q.recbytes bytes per record).
template <int PREC>
__global__ void k_tma_describe(const int32_t* rowptr, const int32_t* colind, const typename PairT<PREC>::Raw* vals, int n,
                               int num_tiles, const TmaParams q, unsigned char* desc, int* gcol, int4* meta, int ngv = 0,
                               long long vstride = 0) {
    using Raw = typename PairT<PREC>::Raw;
    using RecT = Rec<PREC>;
    constexpr int NCAND = 8;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int R = q.R;
    const int WR = R + 2 * TMA_HALO;   // rows of a window
    const int gstride = q.gcol_stride >> 2;
    const int thresh = max(8, WR / 2);
    for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < num_tiles; t += (int)((gridDim.x * blockDim.x) >> 5)) {
        const int r0 = t * R;
        const int nr = min(R, n - r0);
        const int z0 = rowptr[r0];
        const int g = min(rowptr[r0 + nr] - z0, q.ecap);
        int* hdr = reinterpret_cast<int*>(desc + (size_t)t * q.desc_stride);
        RecT* rec = reinterpret_cast<RecT*>(desc + (size_t)t * q.desc_stride + q.hdr_bytes);
        int* gc = gcol + (size_t)t * gstride;
        for (int e = lane; e <= nr; e += 32) hdr[e] = rowptr[r0 + e] - z0;
        const int wlo = r0 - TMA_HALO, whi = r0 + R + TMA_HALO;
        // candidate windows (warp-uniform), from the far columns of the first and last rows in
        // increasing order: a window started HALO before a far column's diagonal d covers the
        // diagonals d .. d + 2 HALO of every row of the tile, so a column whose diagonal lies
        // within that reach of the previous candidate's starts none (a stencil's cluster of
        // neighbouring far diagonals takes one window)
        int cand[NCAND] = {0, 0, 0, 0, 0, 0, 0, 0};
        int nc = 0;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int rr = side ? r0 + nr - 1 : r0;
            const int k0 = rowptr[rr], k1 = rowptr[rr + 1];
            const int c = (k0 + lane < k1) ? colind[k0 + lane] : wlo;   // rows longer than 32: the first 32
            unsigned farm = __ballot_sync(0xffffffffu, c < wlo || c >= whi);
            long long reach = LLONG_MIN;   // the last diagonal the previous candidate covers
            while (farm && nc < NCAND) {
                const int src = __ffs(farm) - 1;
                farm &= farm - 1;
                const int cs = __shfl_sync(0xffffffffu, c, src);
                const long long dg = (long long)cs - rr;
                if (dg <= reach) continue;
                reach = dg + 2 * TMA_HALO;
                const int wsv = cs - (rr - r0) - TMA_HALO;
                bool dup = false;
#pragma unroll
                for (int y = 0; y < NCAND; ++y) dup = dup || (y < nc && cand[y] == wsv);
                if (!dup) {
#pragma unroll
                    for (int y = 0; y < NCAND; ++y)
                        if (y == nc) cand[y] = wsv;
                    ++nc;
                }
            }
        }
        // far entries of the tile inside each candidate
        int cnt[NCAND];
#pragma unroll
        for (int y = 0; y < NCAND; ++y) cnt[y] = 0;
        for (int e0 = 0; e0 < g; e0 += 32) {
            const int e = e0 + lane;
            const int c = e < g ? colind[z0 + e] : wlo;
            const bool far = c < wlo || c >= whi;
#pragma unroll
            for (int y = 0; y < NCAND; ++y)
                if (y < nc) cnt[y] += __popc(__ballot_sync(0xffffffffu, far && c >= cand[y] && c < cand[y] + WR));
        }
        int ws[TMA_MAX_WIN] = {0, 0, 0, 0};
        int nw = 0;
#pragma unroll
        for (int y = 0; y < NCAND; ++y) {
            if (y < nc && nw < TMA_MAX_WIN && cnt[y] >= thresh && (nw + 1) * q.wslots * 4 <= q.fcap) {
#pragma unroll
                for (int w = 0; w < TMA_MAX_WIN; ++w)
                    if (w == nw) ws[w] = cand[y];
                ++nw;
            }
        }
        const int gcap = q.fcap - nw * q.wslots * 4;   // gathered rows that still fit
        const int gbase = q.off_gat + nw * q.wslots * q.slot;
        int nfar = 0, gcut = g;
        for (int e0 = 0; e0 < gcut; e0 += 32) {
            const int e = e0 + lane;
            const bool valid = e < gcut;
            const int c = valid ? colind[z0 + e] : 0;
            const bool near = c >= wlo && c < whi;
            int woff = -1;   // offset in the first extra window holding c
#pragma unroll
            for (int w = TMA_MAX_WIN - 1; w >= 0; --w)
                if (w < nw && c >= ws[w] && c < ws[w] + WR) woff = q.off_gat + w * q.wslots * q.slot + (c - ws[w]) * q.rowbytes;
            const bool gath = valid && !near && woff < 0;
            const unsigned farm = __ballot_sync(0xffffffffu, gath);
            const int fs = nfar + __popc(farm & lt_mask);
            const unsigned over = __ballot_sync(0xffffffffu, gath && fs >= gcap);
            if (over) gcut = e0 + __ffs(over) - 1;   // first entry without a gather slot
            if (valid && e < gcut) {
                int off;
                if (near) {
                    off = (c - wlo) * q.rowbytes;
                } else if (woff >= 0) {
                    off = woff;
                } else {
                    off = gbase + (fs >> 2) * q.slot + (fs & 3) * q.rowbytes;
                    gc[TMA_MAX_WIN + fs] = c;
                }
                if (ngv == 0) {
                    RecT rr;
                    rr.a = vals[z0 + e];
                    rr.off = off;
                    if constexpr (PREC != LL_PREC_F32_MIXED) {
                        // (16-byte records: the entry's row in the tile, for the reverse step's
                        // gradient contraction)
                        int lo = 0, hi = nr;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (rowptr[r0 + mid] - z0 <= e) lo = mid; else hi = mid;
                        }
                        rr.pad = lo;
                    }
                    rec[e] = rr;
                } else {
                    unsigned char* rb = reinterpret_cast<unsigned char*>(rec) + (size_t)e * q.recbytes;
                    *reinterpret_cast<int*>(rb) = off;
                    Raw* rv = reinterpret_cast<Raw*>(rb + sizeof(Raw));
                    for (int v = 0; v < ngv; ++v) rv[v] = vals[(size_t)v * (size_t)vstride + z0 + e];
                }
            }
            nfar += __popc(farm);
        }
        const int ng = min(nfar, gcap);
        __syncwarp();
        if (ng > 0) {
            const int last = gc[TMA_MAX_WIN + ng - 1];
            for (int e = ng + lane; e < ((ng + 3) & ~3); e += 32) gc[TMA_MAX_WIN + e] = last;
        }
#pragma unroll
        for (int w = 0; w < TMA_MAX_WIN; ++w)
            if (lane == w) gc[w] = w < nw ? ws[w] : 0;
        if (lane == 0) {
            hdr[R + 1] = z0;
            hdr[R + 2] = gcut;
            meta[t] = make_int4(gcut, ng, nw, 0);
        }
    }
}


// ---------------------------------------------------------------------------------------- host

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2-D map over the rows of an n x ld block of `elem` bytes per element; a box is `box_rows` rows of
// the first box_cols columns (0: whole rows)
inline bool encode_rows(CUtensorMap* m, const void* base, int elem, long long ld, int n, int box_rows, long long box_cols = 0) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !base || ((uintptr_t)base & 15) != 0) return false;
    if (box_cols <= 0) box_cols = ld;
    if (box_cols > ld || (box_cols * elem) % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)elem};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
inline size_t a128(size_t x) { return (x + 127) & ~(size_t)127; }

// bytes of one prepared matrix value
__host__ __device__ constexpr int raw_size(int precision) { return precision == LL_PREC_F32_MIXED ? 4 : 8; }
// bytes of a sweep record's head (the operand offset, padded to the alignment of the values)
__host__ __device__ constexpr int sweep_rec_head(int precision) { return raw_size(precision); }

inline size_t rec_size(int precision) {
    return precision == LL_PREC_F64 ? sizeof(Rec<LL_PREC_F64>) : (precision == LL_PREC_DF64 ? sizeof(Rec<LL_PREC_DF64>) : sizeof(Rec<LL_PREC_F32_MIXED>));
}


// Per-stage layout of a tile of Rt rows (entry records, gather slots, operand window, V/P rows):
// sets ecap, fcap, hdr_bytes, desc_stride, gcol_stride, off_aux, off_wj, off_gat, off_desc,
// stage_bytes from rowbytes, auxbytes, wjbytes, slot and recbytes. `avg` / `avgfar` are the mean
// entries / far entries (outside the window) per row; `slack` the capacity margin over those means.
// `avgrun`: far entries per row on diagonal runs (a stencil's), which the extra windows take: the
// gather rows then cover TMA_MAX_WIN windows and the other far entries, where that is fewer.
inline void tma_stage_layout(TmaParams& q, int Rt, double avg, double avgfar, double slack, double avgrun = 0.0) {
    int ecap = (((int)(avg * Rt * slack) + 8) + 3) & ~3;
    if (ecap > 4096) ecap = 4096;
    q.wslots = (int)(((size_t)(Rt + 2 * TMA_HALO) * q.rowbytes + q.slot - 1) / q.slot);
    int fcap = (((int)(avgfar * Rt * slack) + 8) + 3) & ~3;
    if (avgrun > 0.0 && avgrun <= avgfar) {
        const int frun = TMA_MAX_WIN * q.wslots * 4 + ((((int)((avgfar - avgrun) * Rt * slack) + 8) + 3) & ~3);
        if (frun < fcap) fcap = frun;
    }
    if (fcap > ecap) fcap = ecap;
    q.R = Rt;
    q.ecap = ecap;
    q.fcap = fcap;
    q.hdr_bytes = (int)a16((size_t)(Rt + 3) * 4);
    q.desc_stride = (int)a16((size_t)q.hdr_bytes + (size_t)ecap * q.recbytes);
    q.gcol_stride = (int)a16((size_t)(TMA_MAX_WIN + fcap) * 4);
    q.off_aux = (int)a128((size_t)(Rt + 2 * TMA_HALO) * q.rowbytes);
    q.off_wj = q.off_aux + (int)a128((size_t)Rt * q.auxbytes);
    q.off_gat = q.off_wj + (int)a128((size_t)Rt * q.wjbytes);
    q.off_desc = q.off_gat + (fcap / 4) * q.slot;
    q.stage_bytes = (int)a128((size_t)q.off_desc + (size_t)q.desc_stride);
}

// ---- batched TMA passes ----------------------------------------------------------------------
constexpr int BT_IRING = 32;   // work items taken ahead of the one being issued
constexpr int BT_TAKE = 16;    // items taken per ticket increment (decoded by sixteen lanes)
constexpr int BT_NRB = 3;      // trace-term buffers of the consumer warps (a tile's terms are summed one tile later)
constexpr int BT_MAX_THREADS = 512 + 96;   // consumers, then the producer, freeing and releasing warps

// Per matrix of a batch, in degree order (device array; the tensor maps make it 128-byte aligned)
struct BatchTmaMat {
    CUtensorMap gat[3];          // gather maps (one-row box) over W_0 (S or V), wa, wb
    CUtensorMap win[3];          // window maps (R + 2 HALO rows) over the same buffers
    CUtensorMap aux;             // V (pass 2) or P (pass 1) rows (R rows)
    const int32_t* colind;
    const void* vals;            // prepared values (direct loads past the records)
    void* w[3];                  // W_0, wa, wb
    void* p;                     // pass 1: P
    double* partials;            // pass 2: per tile trace partials, (m + 1) * T * b (FP64; double-float
                                 // pairs, one float2 per 8 bytes, in the DF64 and FP32 modes)
    double* dots;                // pass 2: traces, (m + 1) * b (slot 0: W_0, slot j + 1: W_{j+1})
    int n, T, m, pad;
};

// Work item handed from the producer to the consumers (one per stage) and kept in the take-ahead
// ring: the step scalars and the matrix's pointers, so that no consumer reads global memory
// before its rows' operands.
struct BItem {
    double beta, d0, dn;         // beta_j, d_0, d_{j+1}
    float2 beta_df, d0_df, dn_df;   // the same as double-float pairs
    const void* win;             // W_j (direct loads)
    void* wout;                  // W_{j+1}
    void* aux;                   // pass 1: P; pass 2: the tile partials of the matrix
    const int32_t* colind;
    const void* vals;
    int j, i, t, gt;             // step (-1: no more items), matrix, tile, tile number in the batch
    int nrec, ng, n, T;          // records and gathered rows of the tile; rows and tiles of the matrix
    int nw, dep;                 // extra windows of the tile; 1: step j - 1 known finished when taken
};
static_assert(sizeof(BItem) == 128, "BItem is copied as 32 words");

struct BatchTmaParams {
    const BatchTmaMat* mats;     // sorted by degree, descending
    // tables (copied to shared memory): step_off[max_m + 1] (first item of each step),
    // step_active[max_m + 1] (matrices active at each step: a prefix), tile_prefix[count + 1]
    // (first batch tile of each matrix), coef_off[count] (offset of (beta_j, d_j) in coef)
    const int* tables;
    const double* coef;          // (beta_j, d_j), j = 0..m, of every matrix, concatenated
    const float2* coef_df;       // the same as double-float pairs
    const unsigned char* desc;   // tile descriptors of every matrix, by batch tile
    const int* gcol;
    const int4* meta;
    unsigned int* ticket;        // zero-initialised item counter
    int* error;                  // set when a bounded wait runs out
    unsigned long long* arrived; // per matrix: tiles finished (all steps)
    long long spin_budget;
    int total_items, max_m, count, b;
    long long ldw, ldp;          // leading dimensions of the W / V blocks and of P (columns)
    TmaParams q;                 // tile geometry shared by every matrix
};

__host__ __device__ inline int bt_table_ints(int max_m, int count) { return 2 * (max_m + 1) + (count + 1) + count; }

struct BatchTmaLaunch {
    TmaParams q;
    int threads = 0, grid = 0;
    size_t smem = 0;
    size_t off_red = 0, off_tab = 0;   // shared-memory offsets of the trace reduction area and the tables
};

// Plans one batched pass: rows per tile (about threads_target / ((b + 1) / 2) rows, fewer when three
// stages do not fit) and stages for b columns, the shared-memory layout, the launch shape (one CTA
// per SM). False when no layout fits (the register kernel is used then).
bool plan_batched_tma(int precision, int mode, int n_min, double avg_nnz, double avg_far, int b, long long ldw,
                      long long ldp, int max_m, int count, int sm_count, BatchTmaLaunch& L, int threads_target = 512);
cudaError_t launch_batched_tma(int precision, int mode, const BatchTmaParams& bp, const BatchTmaLaunch& L, cudaStream_t s);
cudaError_t launch_batched_dots(int precision, const BatchTmaMat* mats, int count, int b, int max_span, cudaStream_t s);

}  // namespace ll
