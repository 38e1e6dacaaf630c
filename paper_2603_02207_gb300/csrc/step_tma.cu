// TMA-fed Léja step kernel (Algorithm 2 loop body over a whole probe block).
//
// Same step as k_leja_step (W_{j+1} = (B - xi_j I) W_j on every column, fused with the P-axpy of
// pass 1, the traces of pass 2 or the adjoint's U term; the per-row arithmetic is shared), but the
// operand rows reach shared memory through the tensor memory accelerator instead of registers:
//   * a window of the tile's rows +-2 by a 2-D tile load (the diagonal and the near columns),
//   * runs of far columns (a stencil's off-diagonal bands) by further windows of the same size,
//   * the remaining (far) neighbour rows W_j[c_k, :] by tile::gather4 (four rows per instruction,
//     rows given by the column indices),
//   * the tile's V (pass 2, adjoint) or P (pass 1) rows by a 2-D tile load,
//   * the tile's descriptor (row offsets and one record per entry: prepared value and the
//     operand row's offset in the stage), built once per pass, by a 1-D bulk copy,
// all completing on one mbarrier per pipeline stage. The CTA is warp-specialised and persistent
// (tiles i, i + grid, ...): its last warps produce (stage each tile's gather columns two tiles
// ahead and issue the copies of a free stage), the other warps consume (a thread owns one row of
// the tile and one column pair, reads its operands from shared memory and writes W_{j+1} (and P)
// straight to global memory, then its warp releases the stage). Full and empty barriers per
// stage replace block-wide barriers. Entries past a tile's record or gather capacity (long rows)
// are read directly from global memory. Every wait on an mbarrier is bounded (clock64 budget);
// when one runs out the kernel records the error, stops issuing copies, waits (bounded) for the
// copies it issued and returns.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"
#include "tma_common.cuh"

namespace ll {

// NP consecutive column pairs of W to or from a 16-byte aligned address (one 16-byte access for two
// FP32 pairs)
template <int NP, typename WP>
__device__ __forceinline__ void ld_pairs(WP (&x)[NP], const void* a) {
    if constexpr (NP == 2 && sizeof(WP) == 8) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(a);
        x[0] = v.x;
        x[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) x[q] = reinterpret_cast<const WP*>(a)[q];
    }
}
template <int NP, typename WP>
__device__ __forceinline__ void st_pairs(WP* a, const WP (&x)[NP]) {
    if constexpr (NP == 2 && sizeof(WP) == 8) {
        *reinterpret_cast<ulonglong2*>(a) = make_ulonglong2(x[0], x[1]);
    } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) a[q] = x[q];
    }
}

// NP: column pairs per consumer thread (1; or 2 in the FP32-mixed mode, whose rows are whole
// 16-byte units: one 16-byte load feeds both pairs, and a tile holds twice the rows)
template <int PREC, int MODE, int NP>
__global__ void __launch_bounds__(TMA_MAX_THREADS, 1)
    k_leja_tma(const __grid_constant__ CUtensorMap tm_gather, const __grid_constant__ CUtensorMap tm_win,
               const __grid_constant__ CUtensorMap tm_aux, const StepParams p, const TmaParams q) {
    using WP = typename PairT<PREC>::W;
    using PP = typename PairT<PREC>::P;
    using Raw = typename PairT<PREC>::Raw;
    using RecT = Rec<PREC>;
    constexpr int MB = base_mode(MODE);
    if constexpr (stop_mode(MODE)) {
        // every column of the pass has met the stopping rule (the first step always runs: it
        // writes P = d_0 W_0 and the traces of W_0 that degree-0 columns keep)
        if (!p.first && *p.done) return;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[TMA_MAX_STAGES];
    __shared__ __align__(8) unsigned long long empty[TMA_MAX_STAGES];
    __shared__ __align__(8) unsigned long long gbar[TMA_MAX_PROD * TMA_GRING];
    __shared__ int4 gmeta[TMA_MAX_PROD * TMA_GRING];
    __shared__ bool s_last;
    // TMA destinations are 128-byte aligned: the plan reserves 128 bytes for this offset
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);

    const int tid = threadIdx.x;
    const int tp = p.tp;
    const int R = q.R;
    const int NST = q.nst;
    const int nprod = q.nprod;                           // producer warps (the last warps of the CTA)
    const int cthreads = (int)blockDim.x - 32 * nprod;   // consumer threads
    const int cwarps = cthreads >> 5;
    const int n = p.n;
    const bool has_aux = (MB == MODE_DOT || MB == MODE_ADJ) || (MB == MODE_ACCUM && !p.first);

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(smem_u32(&full[s]), 1);         // the issuing producer's lane 0 (with the byte count)
            mbar_init(smem_u32(&empty[s]), cwarps);   // one arrival per consumer warp
        }
        for (int s = 0; s < nprod * TMA_GRING; ++s) mbar_init(smem_u32(&gbar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    const int nt = p.num_tiles;
    const int my = (int)blockIdx.x < nt ? (nt - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int rstep = (int)gridDim.x * R;   // rows between this CTA's consecutive tiles
    bool dead = false;
    TracePart T[NP];

    if (tid >= cthreads) {
        // ------------------------------------------------------------------ producer warps
        // warp w of the nprod producers issues tiles w, w + nprod, ... (nprod <= nst: see the plan)
        const int pw = (tid - cthreads) >> 5;
        const int lane = (tid - cthreads) & 31;
        const int myp = my > pw ? (my - 1 - pw) / nprod + 1 : 0;   // tiles of this producer
        auto tile_of = [&](int t) { return (int)blockIdx.x + (pw + t * nprod) * (int)gridDim.x; };
        unsigned char* ring = smem + q.ring_base + pw * TMA_GRING * q.gcol_stride;
        unsigned long long* gb = gbar + pw * TMA_GRING;
        int4* gm = gmeta + pw * TMA_GRING;
        // per-tile (records, gathered rows, extra windows) of this producer's tiles, 32 per batch
        // (lane l holds tile zb + l), the next batch loaded one batch ahead
        auto meta_of = [&](int t) { return t < myp ? q.meta[tile_of(t)] : make_int4(0, 0, 0, 0); };
        int zb = 0;
        int4 mcur = meta_of(lane), mnext = meta_of(32 + lane);
        int cslot = 0;   // ring slot of the next gather-column block to stage
        // L2 policies of the gathered rows: a degree-ordered matrix's hub rows (the first
        // hub_rows) kept, the others given up first
        const uint64_t pol_hub = q.hub_rows > 0 ? l2_policy_evict_last() : 0ull;
        const uint64_t pol_rest = q.hub_rows > 0 ? l2_policy_evict_first() : 0ull;
        // stage the gather columns of this producer's tile t (t increasing by one per call)
        auto stage_gcol = [&](int t) {
            if (t >= zb + 32) {
                zb += 32;
                mcur = mnext;
                mnext = meta_of(zb + 32 + lane);
            }
            const int nrec = __shfl_sync(0xffffffffu, mcur.x, t - zb);
            const int ng = __shfl_sync(0xffffffffu, mcur.y, t - zb);
            const int nw = __shfl_sync(0xffffffffu, mcur.z, t - zb);
            if (lane == 0) {
                gm[cslot] = make_int4(nrec, ng, nw, 0);
                const uint32_t bar = smem_u32(&gb[cslot]);
                // the window start rows, then the gathered columns
                const uint32_t bytes = (ng > 0 || nw > 0) ? (uint32_t)(TMA_MAX_WIN + ((ng + 3) & ~3)) * 4u : 0u;
                if (bytes) {
                    mbar_arrive_expect_tx(bar, bytes);
                    bulk_copy(smem_u32(ring + cslot * q.gcol_stride), q.gcol + (size_t)tile_of(t) * (q.gcol_stride >> 2), bytes, bar);
                } else {
                    mbar_arrive(bar);
                }
            }
            if (++cslot == TMA_GRING) cslot = 0;
        };
        constexpr int LOOK = TMA_GRING - 1;
        for (int t = 0; t < LOOK && t < myp; ++t) stage_gcol(t);
        int gslot = 0, gph = 0;   // ring slot and phase of the tile being issued
        int issued = 0;
        for (int ii = 0; ii < myp; ++ii) {
            const int i = pw + ii * nprod;   // the CTA's tile index
            const int s = i % NST, ph = (i / NST) & 1;
            const int tile = tile_of(ii);
            const int r0 = tile * R;
            if (ii + LOOK < myp) stage_gcol(ii + LOOK);
            // this tile's gather columns, and a free stage (every consumer warp released the
            // stage's previous tile)
            bool ok = mbar_wait_bounded(smem_u32(&gb[gslot]), (uint32_t)gph, q.spin_budget);
            int where = ok ? 0 : TMA_ERR_GCOL;
            if (ok && i >= NST && lane == 0) {
                ok = mbar_wait_bounded(smem_u32(&empty[s]), (uint32_t)(ph ^ 1), q.spin_budget);
                if (!ok) where = TMA_ERR_EMPTY;
            }
            if (!__all_sync(0xffffffffu, ok)) {
                dead = true;
                if (!ok) atomicCAS(q.error, 0, where);
                break;
            }
            const int4 mt = gm[gslot];
            const int ngr = (mt.y + 3) >> 2;
            const int nw = mt.z;
            unsigned char* st = smem + s * q.stage_bytes;
            const uint32_t bar = smem_u32(&full[s]);
            // a sweep loads every operand region once per active group: group g's rows are rows
            // g n + r of the stacked blocks, its part of the stage starts at g gsz
            const int ngrp = sweep_mode(MODE) ? q.ngrp : 1;
            if (lane == 0) {
                // (the test hook adds 16 bytes to tile 0 that no copy delivers: its waits run out)
                const uint32_t dbytes = (uint32_t)q.hdr_bytes + (uint32_t)mt.x * (uint32_t)q.recbytes;
                const uint32_t dbytes16 = (dbytes + 15u) & ~15u;
                const uint32_t per_grp = (uint32_t)ngr * 4u * (uint32_t)q.rowbytes +
                                         (uint32_t)(1 + nw) * (uint32_t)(R + 2 * TMA_HALO) * (uint32_t)q.rowbytes +
                                         (has_aux ? (uint32_t)R * (uint32_t)q.auxbytes : 0u);
                // (the gradient contraction's W_j rows: the tile's rows of a contiguous block, one copy)
                const uint32_t wjb = grad_mode(MODE) ? (uint32_t)min(R, n - r0) * (uint32_t)q.rowbytes : 0u;
                const uint32_t bytes = dbytes16 + (uint32_t)ngrp * per_grp + wjb + ((q.inject && i == 0) ? 16u : 0u);
                mbar_arrive_expect_tx(bar, bytes);
                bulk_copy(smem_u32(st + q.off_desc), q.desc + (size_t)tile * q.desc_stride, dbytes16, bar);
                if constexpr (!sweep_mode(MODE)) {
                    // the window may start above row 0 or end below row n: those rows are zero-filled
                    tma_load_rows(smem_u32(st), &tm_win, r0 - TMA_HALO, bar);
                    if (has_aux) tma_load_rows(smem_u32(st + q.off_aux), &tm_aux, r0, bar);
                }
                if constexpr (grad_mode(MODE))
                    bulk_copy(smem_u32(st + q.off_wj), static_cast<const unsigned char*>(p.wj) + (size_t)r0 * q.rowbytes, wjb,
                              bar);
            }
            const int* gcs = reinterpret_cast<const int*>(ring + gslot * q.gcol_stride);
            const int gs0 = nw * q.wslots;
            if constexpr (sweep_mode(MODE)) {
                // (a window's halo rows past a group's ends hold the neighbouring group's rows, or
                // zeros past the stack: no record refers to them)
                for (int gi = lane; gi < ngrp; gi += 32) {
                    tma_load_rows(smem_u32(st + gi * q.gsz), &tm_win, gi * n + r0 - TMA_HALO, bar);
                    if (has_aux) tma_load_rows(smem_u32(st + gi * q.gsz + q.off_aux), &tm_aux, gi * n + r0, bar);
                }
                for (int x = lane; x < nw * ngrp; x += 32) {
                    const int gi = x / nw, w = x - gi * nw;
                    tma_load_rows(smem_u32(st + gi * q.gsz + q.off_gat + w * q.wslots * q.slot), &tm_win, gi * n + gcs[w], bar);
                }
                for (int x = lane; x < ngr * ngrp; x += 32) {
                    const int gi = x / ngr, q4 = x - gi * ngr;
                    const int4 c4 = *reinterpret_cast<const int4*>(gcs + TMA_MAX_WIN + 4 * q4);
                    const int o = gi * n;
                    tma_gather4(smem_u32(st + gi * q.gsz + q.off_gat + (gs0 + q4) * q.slot), &tm_gather, o + c4.x, o + c4.y,
                                o + c4.z, o + c4.w, bar);
                }
            } else {
                // extra windows (runs of far columns) in the first gather slots, then the gathers
                if (lane < nw) tma_load_rows(smem_u32(st + q.off_gat + lane * q.wslots * q.slot), &tm_win, gcs[lane], bar);
                for (int gi = lane; gi < ngr; gi += 32) {
                    const int4 c4 = *reinterpret_cast<const int4*>(gcs + TMA_MAX_WIN + 4 * gi);
                    const uint32_t dst = smem_u32(st + q.off_gat + (gs0 + gi) * q.slot);
                    if (q.hub_rows > 0) {
                        const int cmin = min(min(c4.x, c4.y), min(c4.z, c4.w));
                        tma_gather4_hint(dst, &tm_gather, c4.x, c4.y, c4.z, c4.w, bar, cmin < q.hub_rows ? pol_hub : pol_rest);
                    } else {
                        tma_gather4(dst, &tm_gather, c4.x, c4.y, c4.z, c4.w, bar);
                    }
                }
            }
            __syncwarp();   // the ring slot is read before the next copy into it
            ++issued;
            if (++gslot == TMA_GRING) {
                gslot = 0;
                gph ^= 1;
            }
        }
        // after a timeout, wait (bounded) for the copies this warp issued and the consumers did not
        // release (all among its last nst tiles: tile i was issued after tile i - nst was
        // released), and for the gather-column blocks staged ahead, so that none lands in shared
        // memory after the CTA exits
        if (dead && lane == 0) {
            const long long drain = q.spin_budget > TMA_DRAIN_MIN ? q.spin_budget : TMA_DRAIN_MIN;
            for (int jj = max(0, issued - NST); jj < issued; ++jj) {
                const int j = pw + jj * nprod;
                mbar_wait_bounded(smem_u32(&full[j % NST]), (uint32_t)((j / NST) & 1), drain);
            }
            for (int t = issued; t < min(myp, issued + LOOK + 1); ++t)
                mbar_wait_bounded(smem_u32(&gb[t % TMA_GRING]), (uint32_t)((t / TMA_GRING) & 1), drain);
        }
    } else {
        // ------------------------------------------------------------------ consumer warps
        const int rlane = tid / tp;
        const int cp = tid - rlane * tp;
        const bool active = rlane < R;
        const long long ldq = p.ldw >> 1;
        const long long ldpq = p.ldp >> 1;
        const WP* __restrict__ win = static_cast<const WP*>(p.win);
        WP* __restrict__ wout = static_cast<WP*>(p.wout);
        const Raw* __restrict__ vals = static_cast<const Raw*>(p.vals);
        PP* __restrict__ pblk = static_cast<PP*>(p.p);
        const int* __restrict__ colind = p.colind;
        const int cp0 = cp * NP;   // the thread's first column pair
        // a sweep takes the scalars and the record values of the thread's column group (the NP
        // pairs of a thread lie in one group)
        const int grp = sweep_mode(MODE) ? cp0 / p.sw_gpairs : 0;
        const int cpg = cp0 - grp * (sweep_mode(MODE) ? p.sw_gpairs : 0);   // first pair within the group
        const size_t grow = (size_t)grp * (size_t)n;                        // the group's first row in the stacks
        const StepScalars<PREC> S0 = sweep_mode(MODE) ? StepScalars<PREC>::group(p, grp)
                                                      : StepScalars<PREC>(p, cp0, stop_mode(MODE) && MB == MODE_ACCUM);
        const StepScalars<PREC> S1 = sweep_mode(MODE) ? S0 : StepScalars<PREC>(p, cp0 + NP - 1, stop_mode(MODE) && MB == MODE_ACCUM);
        const Raw* __restrict__ gvals = vals + (sweep_mode(MODE) ? (size_t)grp * (size_t)p.sw_vstride : 0);
        const unsigned goff = sweep_mode(MODE) ? (unsigned)grp * (unsigned)q.gsz : 0u;   // the group's part of a stage
        const unsigned cpoff = (unsigned)(cpg * sizeof(WP)) + goff;
        const unsigned own_off = (unsigned)(rlane + TMA_HALO) * (unsigned)q.rowbytes + cpoff;
        const unsigned aux_off = (unsigned)q.off_aux + (unsigned)rlane * (unsigned)q.auxbytes +
                                 (unsigned)(cpg * (MB == MODE_ACCUM ? sizeof(PP) : sizeof(WP))) + goff;
        int s = 0, ph = 0;
        int gbase = 0;   // (the gradient contraction: the lane group that takes the tile's first entry)
        int r = (int)blockIdx.x * R + rlane;
        WP* wo = wout + (grow + (size_t)r) * ldq + cpg;   // this thread's W_{j+1} and P pairs, advanced per tile
        PP* po_ptr = pblk + (grow + (size_t)r) * ldpq + cpg;
        const size_t wstep = (size_t)rstep * ldq, pstep = (size_t)rstep * ldpq;
        for (int i = 0; i < my; ++i) {
            // every lane waits (acquiring the stage's copies); the warp gives up together
            const bool ok = mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)ph, q.spin_budget);
            if (!__all_sync(0xffffffffu, ok)) {
                dead = true;
                if ((tid & 31) == 0) atomicCAS(q.error, 0, TMA_ERR_FULL);
                break;
            }
            const unsigned char* st = smem + s * q.stage_bytes;
            if (active && r < n) {
                const int* srp = reinterpret_cast<const int*>(st + q.off_desc);
                const unsigned char* recb = st + q.off_desc + q.hdr_bytes;
                const RecT* rec = reinterpret_cast<const RecT*>(recb);
                const int k0 = srp[rlane], k1 = srp[rlane + 1];
                const int g = srp[R + 2];
                WP wr[NP], vr[NP] = {};
                PP po[NP] = {};
                ld_pairs<NP>(wr, st + own_off);
                if constexpr (MB == MODE_DOT || MB == MODE_ADJ) ld_pairs<NP>(vr, st + aux_off);
                if constexpr (MB == MODE_ACCUM) {
                    if (!p.first) {
#pragma unroll
                        for (int qq = 0; qq < NP; ++qq) po[qq] = reinterpret_cast<const PP*>(st + aux_off)[qq];
                    }
                }
                RowAcc A[NP];
                const int kend = min(k1, g);
                const unsigned char* stc = st + cpoff;
                if constexpr (sweep_mode(MODE)) {
                    // multi-value records: the operand offset, then one value per active group
                    const unsigned char* rv = recb + sweep_rec_head(PREC) + grp * (int)sizeof(Raw);
#pragma unroll 4
                    for (int k = k0; k < kend; ++k) {
                        const int off = *reinterpret_cast<const int*>(recb + k * q.recbytes);
                        const auto ex = expand(*reinterpret_cast<const Raw*>(rv + k * q.recbytes));
                        WP x[NP];
                        ld_pairs<NP>(x, stc + off);
#pragma unroll
                        for (int qq = 0; qq < NP; ++qq) row_mac<PREC>(A[qq], ex, x[qq]);
                    }
                } else {
#pragma unroll 4
                    for (int k = k0; k < kend; ++k) {
                        const RecT rk = rec[k];
                        const auto ex = expand(rk.a);
                        WP x[NP];
                        ld_pairs<NP>(x, stc + rk.off);
#pragma unroll
                        for (int qq = 0; qq < NP; ++qq) row_mac<PREC>(A[qq], ex, x[qq]);
                    }
                }
                if (k1 > g) {   // beyond the records: direct loads, eight in flight, added in entry order
                    const int z0 = srp[R + 1];
                    int k = max(k0, g);
                    for (; k + 8 <= k1; k += 8) {
                        WP x[8][NP];
                        Raw v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            v[u] = gvals[z0 + k + u];
                            ld_pairs<NP>(x[u], win + (grow + (size_t)colind[z0 + k + u]) * ldq + cpg);
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const auto ex = expand(v[u]);
#pragma unroll
                            for (int qq = 0; qq < NP; ++qq) row_mac<PREC>(A[qq], ex, x[u][qq]);
                        }
                    }
                    for (; k < k1; ++k) {
                        WP x[NP];
                        ld_pairs<NP>(x, win + (grow + (size_t)colind[z0 + k]) * ldq + cpg);
                        const auto ex = expand(gvals[z0 + k]);
#pragma unroll
                        for (int qq = 0; qq < NP; ++qq) row_mac<PREC>(A[qq], ex, x[qq]);
                    }
                }
                WP wn[NP];
                PP pn[NP];
#pragma unroll
                for (int qq = 0; qq < NP; ++qq)
                    row_epilogue<PREC, MODE>(p, qq == 0 ? S0 : S1, A[qq], wr[qq], vr[qq], po[qq], &wn[qq], &pn[qq], T[qq]);
                st_pairs<NP>(wo, wn);
                if constexpr (MB == MODE_ACCUM) {
#pragma unroll
                    for (int qq = 0; qq < NP; ++qq) po_ptr[qq] = pn[qq];
                }
            }
            if constexpr (grad_mode(MODE)) {
                // the gradient contraction of the tile's entries: entry e = (rw, c) adds
                // gscale <Lambda_{j+1}[c], W_j[rw]> to grad[e] (the transposed entry's term, in the
                // tile's entry order: neighbouring entries update neighbouring words, and the old
                // value is loaded before the dot product), Lambda_{j+1}[c] from its record's
                // operand row (past the records: global memory), W_j[rw] from the staged rows.
                // An entry takes gsp adjacent lanes (lane u of the group: the column pairs
                // congruent to u mod gsp, from a start that differs between neighbouring entries,
                // so that they meet other bank groups), and the entries go round the CTA's lane
                // groups from where the previous tile's left off, so that every warp takes its
                // share.
                const int* srp = reinterpret_cast<const int*>(st + q.off_desc);
                const RecT* rec = reinterpret_cast<const RecT*>(st + q.off_desc + q.hdr_bytes);
                const int r0t = (int)(blockIdx.x + (long long)i * gridDim.x) * R;
                const int nr = min(R, n - r0t);
                const int z0 = srp[R + 1], gcap = srp[R + 2];
                int ktot = srp[nr];
                if (ktot < 0 || (long long)ktot > (long long)nr * n || gcap < 0 || gcap > q.ecap) {   // (a header that cannot be)
                    if (tid == 0) atomicCAS(q.error, 0, TMA_ERR_DESC);
                    ktot = 0;
                }
                const int sp = q.gsp;
                const int nslot = cthreads / sp;
                const int sub = tid & (sp - 1);
                const unsigned gmask = ((1u << sp) - 1u) << ((tid & 31) & ~(sp - 1));
                const int npairs = (p.b + 1) / 2;
                int k = tid / sp - gbase;
                if (k < 0) k += nslot;
                for (; k < ktot; k += nslot) {
                    int lo = 0;   // the entry's row: srp[lo] <= k < srp[lo + 1] (16-byte records carry it)
                    if (PREC != LL_PREC_F32_MIXED && k < gcap) {
                        lo = rec_row(rec[k]);
                    } else {
                        int hi = nr;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (srp[mid] <= k) lo = mid; else hi = mid;
                        }
                    }
                    const WP* wrow = reinterpret_cast<const WP*>(st + q.off_wj + lo * q.rowbytes);
                    const WP* lrow = k < gcap ? reinterpret_cast<const WP*>(st + rec[k].off)
                                              : win + (size_t)colind[z0 + k] * ldq;
                    const int rot = (k * sp) % npairs;
                    const double gold = sub == 0 ? p.grad[z0 + k] : 0.0;
                    // two independent accumulators (alternate pairs of the lane's share)
                    f2x sh[2] = {0ull, 0ull}, sl[2] = {0ull, 0ull};
                    double a[4] = {0.0, 0.0, 0.0, 0.0};
                    auto mac = [&](int u, int qr) {
                        int qq = qr + rot;
                        if (qq >= npairs) qq -= npairs;
                        const WP lv = lrow[qq];
                        const WP wv = wrow[qq];
                        if constexpr (PREC == LL_PREC_F64) {
                            a[2 * u] = fma(lv.x, wv.x, a[2 * u]);
                            a[2 * u + 1] = fma(lv.y, wv.y, a[2 * u + 1]);
                        } else if constexpr (PREC == LL_PREC_DF64) {
                            df2_mac_pp(sh[u], sl[u], lv.x, lv.y, f2_sub(0ull, lv.x), wv.x, wv.y);
                        } else {
                            df2_mac_f(sh[u], sl[u], lv, 0ull, f2_sub(0ull, lv), wv);   // exact FP32 products
                        }
                    };
                    int qr = sub;
#pragma unroll 2
                    for (; qr + sp < npairs; qr += 2 * sp) {
                        mac(0, qr);
                        mac(1, qr + sp);
                    }
                    if (qr < npairs) mac(0, qr);
                    double dot;
                    if constexpr (PREC == LL_PREC_F64) {
                        dot = (a[0] + a[1]) + (a[2] + a[3]);
                        for (int o = 1; o < sp; o <<= 1) dot += __shfl_xor_sync(gmask, dot, o);
                    } else {
                        float h = 0.f, lo2 = 0.f;
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            float h0, h1, l0, l1;
                            f2_unpack(sh[u], h0, h1);
                            f2_unpack(sl[u], l0, l1);
                            df_mac(h, lo2, h0, l0, 1.f, 0.f);
                            df_mac(h, lo2, h1, l1, 1.f, 0.f);
                        }
                        for (int o = 1; o < sp; o <<= 1) {
                            const float ph = __shfl_xor_sync(gmask, h, o), pl = __shfl_xor_sync(gmask, lo2, o);
                            df_mac(h, lo2, ph, pl, 1.f, 0.f);
                        }
                        dot = (double)h + (double)lo2;
                    }
                    if (sub == 0) p.grad[z0 + k] = gold + p.gscale * dot;
                }
                gbase += ktot % nslot;
                if (gbase >= nslot) gbase -= nslot;
            }
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(smem_u32(&empty[s]));
            r += rstep;
            wo += wstep;
            po_ptr += pstep;
            if (++s == NST) {
                s = 0;
                ph ^= 1;
            }
        }
    }
    const int any_dead = __syncthreads_or(dead ? 1 : 0);
    if constexpr (MB == MODE_DOT || stop_mode(MODE)) {
        if (!any_dead) trace_reduce<PREC, MODE, NP>(p, T, reinterpret_cast<double*>(smem), tp, R, &s_last);
    }
}

// ------------------------------------------------------------------------------------------ host

namespace {

template <int PREC, int MODE, int NP>
int occupancy_tma(int threads, size_t smem) {
    cudaFuncSetAttribute(k_leja_tma<PREC, MODE, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leja_tma<PREC, MODE, NP>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

template <int PREC, int MODE, int NP>
cudaError_t launch_tma_typed(const TmaLaunch& L, const CUtensorMap& g, const CUtensorMap& o, const CUtensorMap& a,
                             const StepParams& p, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_leja_tma<PREC, MODE, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_leja_tma<PREC, MODE, NP><<<L.grid, L.threads, L.smem, s>>>(g, o, a, p, L.q);
    return cudaGetLastError();
}

}  // namespace

bool plan_step_tma(int precision, int mode, int n, int64_t nnz, int64_t nfar, int64_t nrun, int maxrow, int b,
                   int threads_target, int ctas_per_sm, StepParams& p, TmaLaunch& L, int sm_count, int np) {
    L = TmaLaunch{};
    if (n <= 0 || b <= 0 || !encode_fn()) return false;
    // two column pairs per thread: the block's pairs must come in twos (ldw a multiple of 4), since a
    // thread reads and writes both of its pairs (the last thread's second pair would otherwise lie
    // past the row: in the last row, past the block). FP32-mixed (one 16-byte access for both
    // pairs) and DF64 (two pairs share each entry record and give two independent double-float
    // chains); F64 only in the sweep modes, whose blocks of several groups would leave few rows per
    // tile.
    if (np != 1 && np != 2) return false;
    if (np == 2 && (p.ldw % 4 != 0 || (base_mode(mode) == MODE_ACCUM && p.ldp % 4 != 0))) return false;
    if (np == 2 && precision == LL_PREC_F64 && !sweep_mode(mode)) return false;
    if (grad_mode(mode) && (np != 1 || base_mode(mode) != MODE_ADJ || !p.wj || !p.grad)) return false;
    // a sweep's blocks are stacks of ngrp groups of n rows of one group width (ldw = 2 sw_gpairs),
    // b the columns of the groups together
    const int ngrp = sweep_mode(mode) ? (p.sw_gpairs > 0 ? (b / 2) / p.sw_gpairs : 0) : 1;
    if (sweep_mode(mode) && (p.sw_gpairs < 1 || b % 2 != 0 || (b / 2) % p.sw_gpairs != 0 || p.sw_gpairs % np != 0 ||
                             p.ldw != 2 * p.sw_gpairs || (long long)ngrp * n >= (1LL << 31)))
        return false;
    L.np = np;
    if (ctas_per_sm < 1 || ctas_per_sm > 2) ctas_per_sm = 1;
    const int ew = (int)elem_size(w_type_of(precision));
    const long long ld = p.ldw;
    if (ld > 256 || (ld * ew) % 16 != 0) return false;
    int auxbytes = 0;
    if (base_mode(mode) == MODE_DOT || base_mode(mode) == MODE_ADJ) {
        if (p.ldv != p.ldw) return false;
        auxbytes = (int)(ld * ew);
    } else if (base_mode(mode) == MODE_ACCUM) {
        if (p.ldp > 256 || (p.ldp * 8) % 16 != 0 || (sweep_mode(mode) && p.ldp != p.ldw)) return false;
        auxbytes = (int)(p.ldp * 8);
    }
    if (threads_target <= 0 || threads_target > 512) threads_target = 512 / ctas_per_sm;
    const int tp = (b + 2 * np - 1) / (2 * np);
    int R = threads_target / tp;
    if (R < 1) R = 1;
    if (R > 256 - 2 * TMA_HALO) R = 256 - 2 * TMA_HALO;   // window box rows <= 256
    if (R + 2 * TMA_HALO > n) R = n - 2 * TMA_HALO;        // a box no taller than the matrix
    if (R < 1 || R * tp > 512) return false;
    TmaParams& q = L.q;
    q.rowbytes = (int)(ld * ew);
    q.auxbytes = auxbytes;
    q.hub_rows = p.hub_bytes > 0 && !sweep_mode(mode) ? (int)std::min<long long>(n, p.hub_bytes / q.rowbytes) : 0;
    // the gradient contraction: the tile's W_j rows staged beside the operand rows; the entries'
    // dot products split over gsp lanes, about as many lanes per tile as the tile has threads
    q.wjbytes = grad_mode(mode) ? q.rowbytes : 0;
    q.gsp = 1;
    if (grad_mode(mode)) {
        if ((reinterpret_cast<uintptr_t>(p.wj) & 15) != 0) return false;
        const double lanes = (double)tp * (double)n / (double)(nnz > 0 ? nnz : 1);
        q.gsp = lanes >= 4.0 ? 4 : (lanes >= 2.0 ? 2 : 1);
    }
    q.slot = (int)a128((size_t)4 * q.rowbytes);
    // sweep records: the offset (padded to the value size), then the values of the b / (2 sw_gpairs)
    // groups
    q.recbytes = sweep_mode(mode) ? sweep_rec_head(precision) + ((b / 2) / p.sw_gpairs) * raw_size(precision)
                                  : (int)rec_size(precision);
    const double avg = (double)nnz / (double)n;
    const double avgfar = nfar >= 0 && nfar <= nnz ? (double)nfar / (double)n : avg;
    const double avgrun = nrun > 0 && nrun <= nfar && nfar <= nnz ? (double)nrun / (double)n : 0.0;
    // tile capacity slack over the mean: more for irregular row lengths (power-law graphs), where
    // tiles above the mean by far are common
    const double slack = maxrow > 4.0 * avg + 16.0 ? 2.0 : 1.25;
    const size_t budget = (ctas_per_sm == 2 ? 112 : 224) * 1024 - 1024;
    // Producer warps: two keep up with the double-float consumers; the FP32 consumers are fast
    // enough that a third producer pays (Matérn 1024², FP32: forward 39.7 -> 35.3 ms; DF64 2%
    // slower with three). A producer waits for the release of tile i - nst only after the release
    // of its previous wait target i - nprod - nst, so with nprod <= nst the stage's empty barrier
    // is never more than one phase behind and the parity wait is unambiguous.
    const int np_cap = precision == LL_PREC_F32_MIXED ? TMA_MAX_PROD : 2;
    // layout for R rows per tile; returns the stage count that fits
    auto layout = [&](int Rt) {
        tma_stage_layout(q, Rt, avg, avgfar, slack, avgrun);
        // a sweep's stage: one group part (window, V or P rows, gathered rows) per group, then the
        // shared descriptor
        q.ngrp = ngrp;
        q.gsz = 0;
        if (sweep_mode(mode)) {
            q.gsz = (int)a128((size_t)q.off_desc);
            q.off_desc = ngrp * q.gsz;
            q.stage_bytes = (int)a128((size_t)q.off_desc + (size_t)q.desc_stride);
        }
        const size_t ring_total = (size_t)np_cap * TMA_GRING * q.gcol_stride;
        const int nst = budget > ring_total ? (int)((budget - ring_total) / q.stage_bytes) : 0;
        q.nst = nst > TMA_MAX_STAGES ? TMA_MAX_STAGES : nst;
        return q.nst;
    };
    // the most rows per tile that keep three stages (two at the least) in shared memory; the
    // reverse step with the gradient contraction takes the most rows that keep two (its staged
    // W_j rows would cut config 3's tiles from 17 to 12 rows at three stages, and its latency-bound
    // contraction gains more from the warps than from the third stage: 83.4 -> 74.8 ms per DF64
    // backward)
    int Rbest = 0;
    for (int Rt = R; Rt >= 1; Rt = Rt > 4 ? Rt * 3 / 4 : Rt - 1) {
        const int nst = layout(Rt);
        if (nst >= (grad_mode(mode) ? 2 : 3)) { Rbest = Rt; break; }
        if (nst >= 2 && Rbest == 0) Rbest = Rt;
    }
    if (Rbest == 0) return false;
    R = Rbest;
    layout(R);
    if (q.nst < 2) return false;
    const int nprod = np_cap < q.nst ? np_cap : q.nst;
    q.nprod = nprod;
    q.ring_base = q.nst * q.stage_bytes;
    L.smem = (size_t)q.ring_base + (size_t)nprod * TMA_GRING * q.gcol_stride;
    L.threads = ((R * tp + 31) / 32) * 32 + 32 * nprod;   // consumer warps and the producer warps
    if (L.smem < (size_t)L.threads * 2 * np * sizeof(double)) L.smem = (size_t)L.threads * 2 * np * sizeof(double);
    L.smem += 128;
    p.tp = tp;
    p.rl = R;
    p.rpt = 1;
    p.b = b;
    p.n = n;
    p.num_tiles = (n + R - 1) / R;
    L.desc_bytes = (size_t)p.num_tiles * q.desc_stride;
    L.gcol_bytes = (size_t)p.num_tiles * q.gcol_stride;
    L.meta_bytes = (size_t)p.num_tiles * sizeof(int4);
    int per_sm = 0;
    switch ((np - 1) * 3 * NUM_MODES + precision * NUM_MODES + mode) {
#define OCC(N_, P_, M_) case (N_ - 1) * 3 * NUM_MODES + P_ * NUM_MODES + M_: per_sm = occupancy_tma<P_, M_, N_>(L.threads, L.smem); break;
#define OCC4(N_, P_) OCC(N_, P_, MODE_PLAIN) OCC(N_, P_, MODE_ACCUM) OCC(N_, P_, MODE_DOT) OCC(N_, P_, MODE_ADJ) \
    OCC(N_, P_, MODE_ACCUM_STOP) OCC(N_, P_, MODE_DOT_STOP) OCC(N_, P_, MODE_ACCUM_SWEEP) OCC(N_, P_, MODE_DOT_SWEEP)
#define OCCSW(N_, P_) OCC(N_, P_, MODE_ACCUM_SWEEP) OCC(N_, P_, MODE_DOT_SWEEP)
        OCC4(1, LL_PREC_F64) OCC4(1, LL_PREC_DF64) OCC4(1, LL_PREC_F32_MIXED) OCC4(2, LL_PREC_F32_MIXED)
        OCC(1, LL_PREC_F64, MODE_ADJ_GRAD) OCC(1, LL_PREC_DF64, MODE_ADJ_GRAD) OCC(1, LL_PREC_F32_MIXED, MODE_ADJ_GRAD)
        OCC4(2, LL_PREC_DF64) OCCSW(2, LL_PREC_F64)
#undef OCCSW
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

cudaError_t launch_tma_describe(int precision, const TmaLaunch& L, const StepParams& p, cudaStream_t s) {
    const int warps_per_cta = 8;
    int grid = (p.num_tiles + warps_per_cta - 1) / warps_per_cta;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) return cudaSuccess;
    // a sweep's records carry the values of its b / (2 sw_gpairs) groups
    const int ngv = p.sw_gpairs > 0 ? (p.b / 2) / p.sw_gpairs : 0;
    switch (precision) {
        case LL_PREC_F64:
            k_tma_describe<LL_PREC_F64><<<grid, 32 * warps_per_cta, 0, s>>>(p.rowptr, p.colind, static_cast<const double*>(p.vals),
                                                                        p.n, p.num_tiles, L.q, L.q.desc_w, L.q.gcol_w, L.q.meta_w,
                                                                        ngv, p.sw_vstride);
            break;
        case LL_PREC_DF64:
            k_tma_describe<LL_PREC_DF64><<<grid, 32 * warps_per_cta, 0, s>>>(p.rowptr, p.colind, static_cast<const float2*>(p.vals),
                                                                         p.n, p.num_tiles, L.q, L.q.desc_w, L.q.gcol_w, L.q.meta_w,
                                                                         ngv, p.sw_vstride);
            break;
        default:
            k_tma_describe<LL_PREC_F32_MIXED><<<grid, 32 * warps_per_cta, 0, s>>>(p.rowptr, p.colind, static_cast<const float*>(p.vals),
                                                                              p.n, p.num_tiles, L.q, L.q.desc_w, L.q.gcol_w, L.q.meta_w,
                                                                              ngv, p.sw_vstride);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_step_tma(int precision, int mode, const TmaLaunch& L, const StepParams& p, cudaStream_t s) {
    if (p.num_tiles <= 0) return cudaSuccess;
    const int ew = (int)elem_size(w_type_of(precision));
    // rows of the maps: a sweep's blocks stack its groups (group g's row r is row g n + r)
    const int rows = (sweep_mode(mode) ? L.q.ngrp : 1) * p.n;
    CUtensorMap g{}, w{}, a{};
    if (!encode_rows(&g, p.win, ew, p.ldw, rows, 1) || !encode_rows(&w, p.win, ew, p.ldw, rows, L.q.R + 2 * TMA_HALO))
        return cudaErrorInvalidValue;
    bool aux_ok = true;
    if (base_mode(mode) == MODE_DOT || base_mode(mode) == MODE_ADJ) aux_ok = encode_rows(&a, p.v, ew, p.ldv, rows, L.q.R);
    else if (base_mode(mode) == MODE_ACCUM && !p.first) aux_ok = encode_rows(&a, p.p, 8, p.ldp, rows, L.q.R);
    else a = w;
    if (!aux_ok) return cudaErrorInvalidValue;
    switch ((L.np - 1) * 3 * NUM_MODES + precision * NUM_MODES + mode) {
#define LCH(N_, P_, M_) case (N_ - 1) * 3 * NUM_MODES + P_ * NUM_MODES + M_: return launch_tma_typed<P_, M_, N_>(L, g, w, a, p, s);
#define LCH4(N_, P_) LCH(N_, P_, MODE_PLAIN) LCH(N_, P_, MODE_ACCUM) LCH(N_, P_, MODE_DOT) LCH(N_, P_, MODE_ADJ) \
    LCH(N_, P_, MODE_ACCUM_STOP) LCH(N_, P_, MODE_DOT_STOP) LCH(N_, P_, MODE_ACCUM_SWEEP) LCH(N_, P_, MODE_DOT_SWEEP)
#define LCHSW(N_, P_) LCH(N_, P_, MODE_ACCUM_SWEEP) LCH(N_, P_, MODE_DOT_SWEEP)
        LCH4(1, LL_PREC_F64) LCH4(1, LL_PREC_DF64) LCH4(1, LL_PREC_F32_MIXED) LCH4(2, LL_PREC_F32_MIXED)
        LCH(1, LL_PREC_F64, MODE_ADJ_GRAD) LCH(1, LL_PREC_DF64, MODE_ADJ_GRAD) LCH(1, LL_PREC_F32_MIXED, MODE_ADJ_GRAD)
        LCH4(2, LL_PREC_DF64) LCHSW(2, LL_PREC_F64)
#undef LCHSW
#undef LCH4
#undef LCH
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ll
