// Batched Léja passes fed by TMA: many independent matrices, all their Léja steps (Algorithm 2,
// Eq. 4), in one persistent launch per pass, over the tile pipeline of the single-matrix TMA step.
//
// Work items are (step j, matrix i, row tile t), numbered step-major over the matrices still
// active at step j (sorted by degree, descending, so they are a prefix). A CTA has these roles:
//  * the producer warp takes item numbers from a global ticket, BT_TAKE at a time, one batch
//    ahead: BT_TAKE lanes decode a batch from tables held in shared memory and start the loads of each
//    item's step scalars, pointers, tile counts and arrival counter; one batch later the batch is
//    written into a ring of taken items and the copies of its gather-column lists start. To issue
//    an item, the producer makes sure every tile of step j - 1 of matrix i has finished (known
//    when the item was taken, else a bounded wait), waits for a free stage, and issues the item's
//    copies: descriptor, operand windows, V/P rows and the gathered rows of W_j of matrix i,
//    through that matrix's own tensor maps;
//  * the consumer warps compute the item's rows with the per-row arithmetic of the single-matrix
//    kernels and store W_{j+1} (and P). In pass 2 each thread keeps its trace terms over a run of
//    tiles (consecutive items of one batch with the same step and matrix), then writes them to
//    one of BT_NRB buffers, and after writing those of a run each warp sums its share of column
//    pairs of the previous run's buffer over the rows (so no warp waits for all the others to
//    finish a run); the run's sums are the partials of its last tile (its other tiles get zero),
//    and the per-tile partials of every step are reduced per matrix after the pass;
//  * the freeing warp waits for each stage's consumers, frees the stage for the producer and
//    queues the finished tile's matrix;
//  * the releasing warp publishes the queued tiles' completion: one release fence for all the
//    tiles queued so far (so the stores of W_{j+1} and P are visible before it), then one add per
//    run of tiles of the same matrix to its arrival counter. The fence latency stays off the
//    consumers, the producer and the stage recycling.
// Every dependency of an item has a smaller ticket; consumers wait only on copies (and on one
// another's earlier trace buffers), the freeing warp only on consumers (and queue room), the
// releasing warp only on the queue, so the smallest unfinished item can always proceed and the
// launch cannot deadlock whatever the residency. W_j and P of step j - 1 were written by other
// CTAs with generic stores; after the acquire of the arrival counter a proxy fence orders them
// before this CTA's TMA reads. Every wait is bounded (clock64); when one runs out the CTA records
// the error, hands the consumers an end marker, waits (bounded) for its copies in flight and
// returns, and the host reports LL_ERR_TIMEOUT.
#include "common.cuh"
#include "kernels.cuh"
#include "step_common.cuh"
#include "tma_common.cuh"

namespace ll {

namespace {

constexpr int BT_SIGQ = 64;          // finished tiles queued from the freeing warp to the releasing warp
static_assert((BT_IRING & (BT_IRING - 1)) == 0 && BT_IRING % BT_TAKE == 0 && BT_TAKE <= 32, "take-ahead ring");

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_relaxed_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ unsigned int ld_acquire_cta(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(unsigned int* p, unsigned int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
// decodes ticket g into (step, matrix, tile) from the tables; x = -1 past the last item
__device__ __forceinline__ int3 bt_decode(const int* t_off, const int* t_act, const int* t_pre, int max_m, int total, int g) {
    if (g >= total) return make_int3(-1, 0, 0);
    int lo = 0, hi = max_m - 1;
    while (lo < hi) {   // last step whose first item is <= g
        const int mid = (lo + hi + 1) >> 1;
        if (t_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int local = g - t_off[lo];
    int a = 0, b = t_act[lo] - 1;   // last active matrix whose first tile is <= local
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (t_pre[mid] <= local) a = mid; else b = mid - 1;
    }
    return make_int3(lo, a, local - t_pre[a]);
}

__device__ __forceinline__ void copy_item(BItem* dst, const BItem* src, int lane) {
    if (lane < (int)(sizeof(BItem) / 4)) reinterpret_cast<int*>(dst)[lane] = reinterpret_cast<const int*>(src)[lane];
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(m) : "memory");
}

__device__ __forceinline__ f2x shfl_down_f2(f2x v, int off) {
    return __shfl_down_sync(0xffffffffu, v, off);
}

}  // namespace

template <int PREC, int MODE>
__global__ void __launch_bounds__(BT_MAX_THREADS, 1) k_leja_tma_batched(const BatchTmaParams bp, const int off_red, const int off_tab) {
    using WP = typename PairT<PREC>::W;
    using PP = typename PairT<PREC>::P;
    using Raw = typename PairT<PREC>::Raw;
    using RecT = Rec<PREC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[TMA_MAX_STAGES];
    __shared__ __align__(8) unsigned long long empty[TMA_MAX_STAGES];
    __shared__ __align__(8) unsigned long long freeb[TMA_MAX_STAGES];
    __shared__ __align__(8) unsigned long long gbar[BT_IRING];
    __shared__ __align__(8) unsigned long long rfull[BT_NRB];    // pass 2: trace terms written (every consumer warp)
    __shared__ __align__(8) unsigned long long rempty[BT_NRB];   // pass 2: trace terms reduced (every consumer warp)
    __shared__ __align__(16) BItem ring[BT_IRING];
    __shared__ __align__(16) BItem sitem[TMA_MAX_STAGES];
    __shared__ int sigq[BT_SIGQ];            // matrices of freed tiles, in item order
    __shared__ unsigned int q_head, q_tail;  // tiles queued (freeing warp) and published (releasing warp)
    __shared__ void* rpart[BT_NRB];          // pass 2: where the reduced terms go
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);

    const TmaParams& q = bp.q;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int NST = q.nst;
    const int R = q.R;
    const int cthreads = (int)blockDim.x - 96;   // consumer threads; then the producer, freeing and releasing warps
    const int cwarps = cthreads >> 5;
    const long long budget = bp.spin_budget;
    int* tab = reinterpret_cast<int*>(smem + off_tab);
    const int ntab = bt_table_ints(bp.max_m, bp.count);
    for (int x = tid; x < ntab; x += blockDim.x) tab[x] = bp.tables[x];
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), cwarps);
            mbar_init(smem_u32(&freeb[s]), 1);
        }
        for (int s = 0; s < BT_IRING; ++s) mbar_init(smem_u32(&gbar[s]), 1);
        for (int x = 0; x < BT_NRB; ++x) {
            mbar_init(smem_u32(&rfull[x]), cwarps);
            mbar_init(smem_u32(&rempty[x]), cwarps);
        }
        q_head = 0u;
        q_tail = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    if (warp == cwarps) {
        // ------------------------------------------------------------------ producer warp
        const int* t_off = tab;
        const int* t_act = t_off + bp.max_m + 1;
        const int* t_pre = t_act + bp.max_m + 1;
        const int* t_coef = t_pre + bp.count + 1;
        unsigned char* gring = smem + q.ring_base;
        int taken = 0, k = 0;
        bool ended = false, dead = false;
        int ci = -1, cj = 0;   // lane 0: the matrix whose finished steps were last read, and their count
        // Items are taken in batches of BT_TAKE tickets, in two phases one batch apart so that the
        // issue path waits for no global load: fetch() decodes a batch (lane l < BT_TAKE: ticket
        // g + l) and starts the loads of its step scalars, pointers, tile counts and arrival
        // counter into registers (and the ticket increment of the batch after it); put() writes
        // the fetched batch into the ring, starts the copies of its gather-column lists and, with
        // one acquire fence for the batch, turns the arrival counts it read into dependencies
        // known to be met.
        unsigned int g_next = 0;   // lane 0: first ticket of the batch after the fetched one
        int err_seen = 0;          // lane 0: the error flag as last read
        int fj = -1, fi = 0, ft = 0, fgt = 0, fn = 0, fT = 0;
        bool flast = true;   // the last item of its run (same matrix and step) within the batch
        int4 fmt = make_int4(0, 0, 0, 0);
        double fbeta = 0.0, fd0 = 0.0, fdn = 0.0;
        float2 fbd = make_float2(0.f, 0.f), fd0d = fbd, fdnd = fbd;
        const void* fwin = nullptr;
        void* fwout = nullptr;
        void* faux = nullptr;
        const int32_t* fcol = nullptr;
        const void* fvals = nullptr;
        unsigned long long farr = 0;
        auto fetch = [&]() {
            unsigned int g0 = 0;
            if (lane == 0) {
                const bool stop = ended || err_seen;
                g0 = stop ? (unsigned int)bp.total_items : g_next;
                if (!stop) g_next = atomicAdd(bp.ticket, (unsigned int)BT_TAKE);
                err_seen = *((volatile int*)bp.error);
            }
            g0 = __shfl_sync(0xffffffffu, g0, 0);
            if (lane < BT_TAKE) {
                const unsigned int g = g0 + (unsigned int)lane;
                const int3 d = bt_decode(t_off, t_act, t_pre, bp.max_m, bp.total_items,
                                         g >= (unsigned int)bp.total_items ? bp.total_items : (int)g);
                fj = d.x;
                fi = d.y;
                ft = d.z;
                if (d.x >= 0) {
                    const BatchTmaMat* M = bp.mats + d.y;
                    fgt = t_pre[d.y] + d.z;
                    fmt = bp.meta[fgt];
                    const double* cf = bp.coef + t_coef[d.y];
                    const float2* cfd = bp.coef_df + t_coef[d.y];
                    fbeta = cf[2 * d.x];
                    fd0 = cf[1];
                    fdn = cf[2 * (d.x + 1) + 1];
                    fbd = cfd[2 * d.x];
                    fd0d = cfd[1];
                    fdnd = cfd[2 * (d.x + 1) + 1];
                    const int buf = d.x == 0 ? 0 : ((d.x & 1) ? 1 : 2);
                    fwin = M->w[buf];
                    fwout = M->w[(d.x & 1) ? 2 : 1];
                    faux = MODE == MODE_ACCUM ? M->p : static_cast<void*>(M->partials);
                    fcol = M->colind;
                    fvals = M->vals;
                    fn = M->n;
                    fT = M->T;
                    if (d.x > 0) farr = ld_relaxed_u64(&bp.arrived[d.y]);
                    prefetch_map(&M->win[buf]);
                    prefetch_map(&M->gat[buf]);
                    if (MODE == MODE_DOT || d.x > 0) prefetch_map(&M->aux);
                }
            }
            // runs of consecutive tickets with the same (step, matrix) inside a batch share one
            // trace reduction (tickets are step-major, then matrix, then tile; batches start at
            // multiples of BT_TAKE, so the runs do not depend on which CTA takes a batch)
            const int nj = __shfl_down_sync(0xffffffffu, fj, 1), ni = __shfl_down_sync(0xffffffffu, fi, 1);
            flast = lane >= BT_TAKE - 1 || nj != fj || ni != fi;
        };
        auto put = [&]() {
            bool none = false, acq = false;
            if (lane < BT_TAKE) {
                const int slot = (taken + lane) & (BT_IRING - 1);
                BItem& it = ring[slot];   // filled in place
                it.j = fj;
                it.i = fi;
                it.t = ft;
                const uint32_t bar = smem_u32(&gbar[slot]);
                if (fj >= 0) {
                    it.beta = fbeta;
                    it.d0 = fd0;
                    it.dn = fdn;
                    it.beta_df = fbd;
                    it.d0_df = fd0d;
                    it.dn_df = fdnd;
                    it.win = fwin;
                    it.wout = fwout;
                    it.aux = faux;
                    it.colind = fcol;
                    it.vals = fvals;
                    it.n = fn;
                    it.T = fT;
                    it.gt = fgt;
                    it.nrec = fmt.x;
                    it.ng = fmt.y;
                    it.nw = fmt.z;
                    // the dependency (every tile of step j - 1 finished) was already met when read
                    // bit 0: the dependency (every tile of step j - 1 finished) was already met when
                    // read; bit 1: the item ends its run
                    const int met = (fj == 0 || farr >= (unsigned long long)fj * (unsigned long long)fT) ? 1 : 0;
                    it.dep = met | (flast ? 2 : 0);
                    acq = fj > 0 && met;
                    // the extra windows' start rows, then the gathered columns
                    const uint32_t bytes = (fmt.y > 0 || fmt.z > 0) ? (uint32_t)(TMA_MAX_WIN + ((fmt.y + 3) & ~3)) * 4u : 0u;
                    if (bytes) {
                        mbar_arrive_expect_tx(bar, bytes);
                        bulk_copy(smem_u32(gring + slot * q.gcol_stride), bp.gcol + (size_t)fgt * (q.gcol_stride >> 2), bytes, bar);
                    } else {
                        mbar_arrive(bar);
                    }
                } else {
                    it.dep = 1;
                    none = true;
                    mbar_arrive(bar);
                }
            }
            ended = __any_sync(0xffffffffu, none) || ended;
            // acquire pattern: the relaxed reads of the arrival counters, then a fence (every lane
            // that read one); after the warp barrier, the proxy fence of every lane orders the
            // other CTAs' generic stores before this warp's TMA reads
            const bool any_acq = __any_sync(0xffffffffu, acq);
            if (any_acq) fence_acq_rel_gpu();
            __syncwarp();   // the ring entries are read by every lane
            if (any_acq) fence_proxy_async();
            taken += BT_TAKE;
        };
        if (lane == 0) g_next = atomicAdd(bp.ticket, (unsigned int)BT_TAKE);
        for (int x = 0; x < BT_IRING / BT_TAKE; ++x) {
            fetch();
            put();
        }
        fetch();
        for (;; ++k) {
            if (taken - k <= BT_IRING - BT_TAKE) {
                put();
                fetch();
            }
            const int slot = k & (BT_IRING - 1);
            // every lane reads the gather-column list: every lane waits for its copy
            bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(smem_u32(&gbar[slot]), (uint32_t)((k / BT_IRING) & 1), budget));
            const int j = ring[slot].j, i = ring[slot].i;
            // a dependency not yet met when the item was taken: wait (bounded) until step j - 1
            // of matrix i finished (arrival count j * T), then order the other CTAs' generic
            // stores of W_j and P before this warp's TMA reads of them (the cache ci, cj lives in
            // lane 0: its decision is the warp's)
            const bool wait_dep = __shfl_sync(0xffffffffu, (ok && j > 0 && !(ring[slot].dep & 1) && !(i == ci && j <= cj)) ? 1 : 0, 0) != 0;
            if (wait_dep && lane == 0) {
                const unsigned long long T = (unsigned long long)ring[slot].T;
                const long long t0 = clock64();
                for (;;) {
                    const unsigned long long v = ld_acquire_u64(&bp.arrived[i]);
                    if (v >= (unsigned long long)j * T) {
                        ci = i;
                        cj = (int)(v / T);
                        break;
                    }
                    if (*((volatile int*)bp.error) || clock64() - t0 > budget) {
                        ok = false;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (wait_dep) {
                __syncwarp();
                fence_proxy_async();
            }
            const int s = k % NST;
            if (ok && lane == 0 && k >= NST) ok = mbar_wait_bounded(smem_u32(&freeb[s]), (uint32_t)(((k / NST) & 1) ^ 1), budget);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                dead = true;
                if (lane == 0) atomicExch(bp.error, 1);
                break;
            }
            // publish the item to the consumers and the freeing warp
            copy_item(&sitem[s], &ring[slot], lane);
            __syncwarp();
            const uint32_t bar = smem_u32(&full[s]);
            if (j < 0) {   // no more items: the end marker
                if (lane == 0) mbar_arrive(bar);
                break;
            }
            const BatchTmaMat* M = bp.mats + i;
            const int t = ring[slot].t, gt = ring[slot].gt, ng = ring[slot].ng, nw = ring[slot].nw;
            const int buf = j == 0 ? 0 : ((j & 1) ? 1 : 2);
            const bool has_aux = (MODE == MODE_DOT) || (MODE == MODE_ACCUM && j > 0);
            const int ngr = (ng + 3) >> 2;
            unsigned char* st = smem + s * q.stage_bytes;
            if (lane == 0) {
                const uint32_t dbytes16 = ((uint32_t)q.hdr_bytes + (uint32_t)ring[slot].nrec * (uint32_t)q.recbytes + 15u) & ~15u;
                const uint32_t bytes = dbytes16 + (uint32_t)ngr * 4u * (uint32_t)q.rowbytes +
                                       (uint32_t)(1 + nw) * (uint32_t)(R + 2 * TMA_HALO) * (uint32_t)q.rowbytes +
                                       (has_aux ? (uint32_t)R * (uint32_t)q.auxbytes : 0u) +
                                       ((q.inject == LL_INJECT_STALL && k == 0 && blockIdx.x == 0) ? 16u : 0u);
                mbar_arrive_expect_tx(bar, bytes);
                bulk_copy(smem_u32(st + q.off_desc), bp.desc + (size_t)gt * q.desc_stride, dbytes16, bar);
                tma_load_rows(smem_u32(st), &M->win[buf], t * R - TMA_HALO, bar);
                if (has_aux) tma_load_rows(smem_u32(st + q.off_aux), &M->aux, t * R, bar);
            }
            const int* gcs = reinterpret_cast<const int*>(gring + slot * q.gcol_stride);
            // extra windows (runs of far columns) in the first gather slots, then the gathers
            if (lane < nw) tma_load_rows(smem_u32(st + q.off_gat + lane * q.wslots * q.slot), &M->win[buf], gcs[lane], bar);
            const int gs0 = nw * q.wslots;
            for (int gi = lane; gi < ngr; gi += 32) {
                const int4 c4 = *reinterpret_cast<const int4*>(gcs + TMA_MAX_WIN + 4 * gi);
                tma_gather4(smem_u32(st + q.off_gat + (gs0 + gi) * q.slot), &M->gat[buf], c4.x, c4.y, c4.z, c4.w, bar);
            }
            __syncwarp();
        }
        bool marked = false;
        if (dead) {
            // hand the consumers an end marker once the stage is free (bounded), so that they stop
            // after the items already issued
            const int s = k % NST;
            bool ok = true;
            if (lane == 0 && k >= NST) ok = mbar_wait_bounded(smem_u32(&freeb[s]), (uint32_t)(((k / NST) & 1) ^ 1), budget);
            marked = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (marked && lane == 0) {
                sitem[s].j = -1;
                mbar_arrive(smem_u32(&full[s]));
            }
        }
        // wait (bounded) for the copies still in flight so that none lands in shared memory after
        // the CTA exits: after a failure, the stages the consumers may not have waited for (the
        // last nst issued items; with an end marker in place, the stage it took was freed, so its
        // previous item is complete); always, the gather-column lists taken ahead and not issued
        if (lane == 0) {
            const long long drain = budget > TMA_DRAIN_MIN ? budget : TMA_DRAIN_MIN;
            if (dead)
                for (int kk = (k > NST ? k - NST : 0) + (marked && k >= NST ? 1 : 0); kk < k; ++kk)
                    mbar_wait_bounded(smem_u32(&full[kk % NST]), (uint32_t)((kk / NST) & 1), drain);
            for (int pos = k; pos < taken; ++pos)
                mbar_wait_bounded(smem_u32(&gbar[pos & (BT_IRING - 1)]), (uint32_t)((pos / BT_IRING) & 1), drain);
        }
    } else if (warp == cwarps + 1) {
        // ------------------------------------------------------------------ freeing warp (lane 0)
        if (lane == 0) {
            unsigned int head = 0;
            bool ok = true;
            for (int k = 0;; ++k) {
                const int s = k % NST;
                const uint32_t par = (uint32_t)((k / NST) & 1);
                // the item is published (full), then its consumers are done with it (empty)
                ok = mbar_wait_bounded(smem_u32(&full[s]), par, budget);
                const int j = sitem[s].j, i = sitem[s].i;
                if (ok && j < 0) break;
                if (ok) ok = mbar_wait_bounded(smem_u32(&empty[s]), par, budget);
                if (ok) {
                    const long long t0 = clock64();
                    while (head - ld_acquire_cta(&q_tail) >= (unsigned int)BT_SIGQ) {
                        if (clock64() - t0 > budget) {
                            ok = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                if (!ok) break;
                mbar_arrive(smem_u32(&freeb[s]));
                sigq[head % BT_SIGQ] = i;
                st_release_cta(&q_head, ++head);
            }
            if (!ok) atomicExch(bp.error, 1);
            // the end marker, when there is room (else the releasing warp's wait runs out)
            if (head - ld_acquire_cta(&q_tail) < (unsigned int)BT_SIGQ) {
                sigq[head % BT_SIGQ] = -1;
                st_release_cta(&q_head, ++head);
            }
        }
    } else if (warp == cwarps + 2) {
        // ------------------------------------------------------------------ releasing warp (lane 0)
        if (lane == 0) {
            unsigned int tail = 0;
            for (bool done = false; !done;) {
                unsigned int head;
                const long long t0 = clock64();
                while ((head = ld_acquire_cta(&q_head)) == tail) {
                    if (clock64() - t0 > budget) {
                        atomicExch(bp.error, 1);
                        done = true;
                        break;
                    }
                    __nanosleep(32);
                }
                if (done) break;
                // the consumers' stores of the queued tiles (W_{j+1}, P) happen before the adds:
                // one fence for all of them
                fence_acq_rel_gpu();
                int cur = -1;
                unsigned long long cnt = 0;
                for (; tail != head; ++tail) {
                    const int i = sigq[tail % BT_SIGQ];
                    if (i < 0) {
                        done = true;
                        break;
                    }
                    if (i != cur) {
                        if (cnt) red_relaxed_add(&bp.arrived[cur], cnt);
                        cur = i;
                        cnt = 0;
                    }
                    ++cnt;
                }
                if (cnt) red_relaxed_add(&bp.arrived[cur], cnt);
                st_release_cta(&q_tail, tail);
            }
        }
    } else if (warp < cwarps) {
        // ------------------------------------------------------------------ consumer warps
        const int b = bp.b;
        const int tp = (b + 1) / 2;
        const int rlane = tid / tp;
        const int cp = tid - rlane * tp;
        const bool active = rlane < R;
        const long long ldq = bp.ldw >> 1;
        const long long ldpq = bp.ldp >> 1;
        const unsigned cpoff = (unsigned)(cp * sizeof(WP));
        const unsigned own_off = (unsigned)(rlane + TMA_HALO) * (unsigned)q.rowbytes + cpoff;
        const unsigned aux_off = (unsigned)q.off_aux + (unsigned)rlane * (unsigned)q.auxbytes +
                                 (unsigned)(cp * (MODE == MODE_ACCUM ? sizeof(PP) : sizeof(WP)));
        double* red = reinterpret_cast<double*>(smem + off_red);   // BT_NRB buffers of cthreads x 16 bytes
        int nreduce = 0;   // trace-term hand-overs so far
        // This warp's share of reduction x: column pairs warp, warp + cwarps, ...; lane l sums rows
        // l, l + 32, ... in order, then a shuffle tree (fixed order) gives lane 0 the column sums.
        // It waits until every consumer warp has written reduction x (they do so one reduction
        // earlier in their own sequence, so the wait is short and cannot close a cycle).
        auto reduce_share = [&](int x) {
            const int rb = x % BT_NRB;
            const bool okw = mbar_wait_bounded(smem_u32(&rfull[rb]), (uint32_t)((x / BT_NRB) & 1), budget);
            if (__any_sync(0xffffffffu, !okw) && lane == 0) atomicExch(bp.error, 1);
            const double* rbuf = red + (size_t)rb * 2 * cthreads;
            void* part = rpart[rb];
            for (int c2 = warp; c2 < tp; c2 += cwarps) {
                if constexpr (PREC == LL_PREC_F64) {
                    double a0 = 0.0, a1 = 0.0;
                    for (int l = lane; l < R; l += 32) {
                        a0 += rbuf[2 * (l * tp + c2)];
                        a1 += rbuf[2 * (l * tp + c2) + 1];
                    }
                    for (int off = 16; off > 0; off >>= 1) {
                        a0 += __shfl_down_sync(0xffffffffu, a0, off);
                        a1 += __shfl_down_sync(0xffffffffu, a1, off);
                    }
                    if (lane == 0) {
                        double* pd = static_cast<double*>(part);
                        pd[2 * c2] = a0;
                        if (2 * c2 + 1 < b) pd[2 * c2 + 1] = a1;
                    }
                } else {
                    const ulonglong2* rd = reinterpret_cast<const ulonglong2*>(rbuf);
                    f2x ah = 0ull, al = 0ull;
                    for (int l = lane; l < R; l += 32) {
                        const ulonglong2 v = rd[l * tp + c2];
                        df2_add(ah, al, v.x, v.y);
                    }
                    for (int off = 16; off > 0; off >>= 1) {
                        const f2x oh = shfl_down_f2(ah, off), ol = shfl_down_f2(al, off);
                        df2_add(ah, al, oh, ol);
                    }
                    if (lane == 0) {
                        float h0, h1, l0, l1;
                        f2_unpack(ah, h0, h1);
                        f2_unpack(al, l0, l1);
                        float2* pf = static_cast<float2*>(part);
                        pf[2 * c2] = make_float2(h0, l0);
                        if (2 * c2 + 1 < b) pf[2 * c2 + 1] = make_float2(h1, l1);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&rempty[rb]));
        };
        TracePart TP;   // pass 2: this thread's trace terms of the current run
        for (int k = 0;; ++k) {
            const int s = k % NST;
            // a warp-wide vote (a consumer-wide one would couple the warps every tile): a warp whose
            // wait ran out leaves; the others' waits run out in turn (every wait is bounded)
            const bool ok = mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((k / NST) & 1), budget);
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0) atomicExch(bp.error, 1);
                break;
            }
            const int j = sitem[s].j;
            if (j < 0) break;
            const int t = sitem[s].t, n = sitem[s].n, T = sitem[s].T;
            const int r = t * R + rlane;
            const unsigned char* st = smem + s * q.stage_bytes;
            StepParams p{};
            p.first = (j == 0);
            p.beta = sitem[s].beta;
            p.d0 = sitem[s].d0;
            p.dn = sitem[s].dn;
            p.beta_df = sitem[s].beta_df;
            p.d0_df = sitem[s].d0_df;
            p.dn_df = sitem[s].dn_df;
            const StepScalars<PREC> S(p, cp);
            if (active && r < n) {
                const WP* __restrict__ win = static_cast<const WP*>(sitem[s].win);
                WP* wout = static_cast<WP*>(sitem[s].wout);
                PP* pblk = static_cast<PP*>(sitem[s].aux);
                const int* srp = reinterpret_cast<const int*>(st + q.off_desc);
                const RecT* rec = reinterpret_cast<const RecT*>(st + q.off_desc + q.hdr_bytes);
                const int k0 = srp[rlane], k1 = srp[rlane + 1];
                const int g = srp[R + 2];
                const WP wr = *reinterpret_cast<const WP*>(st + own_off);
                WP vr{};
                PP po{};
                if constexpr (MODE == MODE_DOT) vr = *reinterpret_cast<const WP*>(st + aux_off);
                if constexpr (MODE == MODE_ACCUM) {
                    if (j > 0) po = *reinterpret_cast<const PP*>(st + aux_off);
                }
                RowAcc A;
                const int kend = min(k1, g);
                const unsigned char* stc = st + cpoff;
#pragma unroll 4
                for (int kk = k0; kk < kend; ++kk) {
                    const RecT rk = rec[kk];
                    row_mac<PREC>(A, expand(rk.a), *reinterpret_cast<const WP*>(stc + rk.off));
                }
                if (k1 > g) {   // beyond the records: direct loads through L2 (W_j was written during the launch)
                    const int z0 = srp[R + 1];
                    const int32_t* colind = sitem[s].colind;
                    const Raw* vals = static_cast<const Raw*>(sitem[s].vals);
                    for (int kk = max(k0, g); kk < k1; ++kk) {
                        WP x;
                        const WP* src = win + (size_t)colind[z0 + kk] * ldq + cp;
                        if constexpr (sizeof(WP) == 16) x = __ldcg(src);
                        else x = __ldcg(reinterpret_cast<const unsigned long long*>(src));
                        row_mac<PREC>(A, expand(vals[z0 + kk]), x);
                    }
                }
                row_epilogue<PREC, MODE>(p, S, A, wr, vr, po, wout + (size_t)r * ldq + cp, pblk + (size_t)r * ldpq + cp, TP);
            }
            if constexpr (MODE == MODE_DOT) {
                // At the end of a run, write the run's per-thread trace terms (slot j + 1: the
                // step's W_{j+1} traces; slot 0: the W_0 traces) to the next of BT_NRB buffers,
                // then sum this warp's share of the reduction before it; the run's sums go to the
                // partials of its last tile. The other tiles of the run get zero partials, so the
                // per-tile sum in tile order stays fixed.
                const int nred = j == 0 ? 2 : 1;
                const bool run_end = (sitem[s].dep & 2) != 0;
                if (!run_end && warp == 0) {
                    for (int qq = 0; qq < nred; ++qq) {
                        const int slot = qq ? 0 : j + 1;
                        for (int c = lane; c < b; c += 32) {
                            if constexpr (PREC == LL_PREC_F64)
                                static_cast<double*>(sitem[s].aux)[((size_t)slot * T + t) * b + c] = 0.0;
                            else
                                static_cast<float2*>(sitem[s].aux)[((size_t)slot * T + t) * b + c] = make_float2(0.f, 0.f);
                        }
                    }
                }
                for (int qq = 0; run_end && qq < nred; ++qq, ++nreduce) {
                    const int slot = qq ? 0 : j + 1;
                    const int rb = nreduce % BT_NRB;
                    const bool okr = nreduce < BT_NRB ||
                                     mbar_wait_bounded(smem_u32(&rempty[rb]), (uint32_t)(((nreduce / BT_NRB) - 1) & 1), budget);
                    if (__any_sync(0xffffffffu, !okr) && lane == 0) atomicExch(bp.error, 1);
                    double* rbuf = red + (size_t)rb * 2 * cthreads;
                    if constexpr (PREC == LL_PREC_F64) {
                        rbuf[2 * tid] = qq ? TP.t0d[0] : TP.td[0];
                        rbuf[2 * tid + 1] = qq ? TP.t0d[1] : TP.td[1];
                        if (tid == 0) rpart[rb] = static_cast<double*>(sitem[s].aux) + ((size_t)slot * T + t) * b;
                    } else {
                        reinterpret_cast<ulonglong2*>(rbuf)[tid] = qq ? make_ulonglong2(TP.t0h2, TP.t0l2) : make_ulonglong2(TP.th2, TP.tl2);
                        if (tid == 0) rpart[rb] = static_cast<float2*>(sitem[s].aux) + ((size_t)slot * T + t) * b;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&rfull[rb]));
                    if (nreduce > 0) reduce_share(nreduce - 1);
                }
                if (run_end) TP = TracePart{};
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
        }
        if constexpr (MODE == MODE_DOT) {
            if (nreduce > 0) reduce_share(nreduce - 1);   // the last tile's terms
        }
    }
    __syncthreads();
}


// dots[j][c] = sum_t partials[j][t][c] (tiles in order, in FP64) of every matrix (blockIdx.y), step
// slot and column; one thread per (slot, column). DF: the partials are double-float pairs.
template <bool DF>
__global__ void k_batched_dots(const BatchTmaMat* mats, int b) {
    const BatchTmaMat& M = mats[blockIdx.y];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (M.m + 1) * b) return;
    const int slot = idx / b, c = idx - slot * b;
    const size_t base = (size_t)slot * M.T * b + c;
    double s = 0.0;
    if constexpr (DF) {
        const float2* part = reinterpret_cast<const float2*>(M.partials) + base;
        for (int t = 0; t < M.T; ++t) {
            const float2 v = part[(size_t)t * b];
            s += (double)v.x + (double)v.y;
        }
    } else {
        const double* part = M.partials + base;
        for (int t = 0; t < M.T; ++t) s += part[(size_t)t * b];
    }
    M.dots[(size_t)slot * b + c] = s;
}

namespace {

template <int PREC, int MODE>
cudaError_t launch_bt_typed(const BatchTmaParams& bp, const BatchTmaLaunch& L, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_leja_tma_batched<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_leja_tma_batched<PREC, MODE><<<L.grid, L.threads, L.smem, s>>>(bp, (int)L.off_red, (int)L.off_tab);
    return cudaGetLastError();
}

template <int PREC, int MODE>
int occupancy_bt(int threads, size_t smem) {
    if (cudaFuncSetAttribute(k_leja_tma_batched<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leja_tma_batched<PREC, MODE>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

}  // namespace

bool plan_batched_tma(int precision, int mode, int n_min, double avg_nnz, double avg_far, int b, long long ldw,
                      long long ldp, int max_m, int count, int sm_count, BatchTmaLaunch& L, int threads_target) {
    L = BatchTmaLaunch{};
    if (n_min <= 0 || b <= 0 || max_m < 1 || count < 1 || !encode_fn()) return false;
    if (mode != MODE_ACCUM && mode != MODE_DOT) return false;
    const int ew = (int)elem_size(w_type_of(precision));
    if (ldw > 256 || (ldw * ew) % 16 != 0) return false;
    TmaParams& q = L.q;
    q.rowbytes = (int)(ldw * ew);
    if (mode == MODE_ACCUM) {
        if (ldp > 256 || (ldp * 8) % 16 != 0) return false;
        q.auxbytes = (int)(ldp * 8);
    } else {
        q.auxbytes = q.rowbytes;
    }
    q.wjbytes = 0;
    q.gsp = 1;
    q.slot = (int)a128((size_t)4 * q.rowbytes);
    q.recbytes = (int)rec_size(precision);
    const int tp = (b + 1) / 2;
    if (threads_target < 32 || threads_target > 512) threads_target = 512;
    int R = threads_target / tp;
    if (R < 1) R = 1;
    if (R > 256 - 2 * TMA_HALO) R = 256 - 2 * TMA_HALO;   // window box rows <= 256
    if (R + 2 * TMA_HALO > n_min) R = n_min - 2 * TMA_HALO;  // a box no taller than the smallest matrix
    if (R < 1) return false;
    const double avgfar = avg_far >= 0.0 && avg_far <= avg_nnz ? avg_far : avg_nnz;
    const size_t tab_bytes = a16((size_t)bt_table_ints(max_m, count) * 4);
    const size_t budget = 220 * 1024;   // dynamic shared memory (the static part holds the barriers, items and queue)
    auto fit = [&](int Rt) {
        tma_stage_layout(q, Rt, avg_nnz, avgfar, 1.25);
        const size_t ct = (size_t)((Rt * tp + 31) / 32) * 32;
        const size_t extra = a128((size_t)BT_IRING * q.gcol_stride) + (mode == MODE_DOT ? BT_NRB * ct * 16 : 0) + tab_bytes + 128;
        const int nst = budget > extra ? (int)((budget - extra) / q.stage_bytes) : 0;
        q.nst = nst > TMA_MAX_STAGES ? TMA_MAX_STAGES : nst;
        return q.nst;
    };
    // the most rows per tile that keep three stages (two at the least)
    int Rbest = 0;
    for (int Rt = R; Rt >= 1; Rt = Rt > 4 ? Rt * 3 / 4 : Rt - 1) {
        const int nst = fit(Rt);
        if (nst >= 3) { Rbest = Rt; break; }
        if (nst >= 2 && Rbest == 0) Rbest = Rt;
    }
    if (Rbest == 0) return false;
    fit(Rbest);
    if (q.nst < 2) return false;
    q.nprod = 1;
    q.ring_base = q.nst * q.stage_bytes;
    const int cthreads = ((Rbest * tp + 31) / 32) * 32;
    L.threads = cthreads + 96;
    L.off_red = a128((size_t)q.ring_base + (size_t)BT_IRING * q.gcol_stride);
    L.off_tab = L.off_red + (mode == MODE_DOT ? (size_t)BT_NRB * cthreads * 16 : 0);
    L.smem = L.off_tab + tab_bytes + 128;
    if (L.threads > BT_MAX_THREADS) return false;
    int per_sm = 0;
    switch (precision * NUM_MODES + mode) {
        case LL_PREC_F64 * NUM_MODES + MODE_ACCUM: per_sm = occupancy_bt<LL_PREC_F64, MODE_ACCUM>(L.threads, L.smem); break;
        case LL_PREC_F64 * NUM_MODES + MODE_DOT: per_sm = occupancy_bt<LL_PREC_F64, MODE_DOT>(L.threads, L.smem); break;
        case LL_PREC_DF64 * NUM_MODES + MODE_ACCUM: per_sm = occupancy_bt<LL_PREC_DF64, MODE_ACCUM>(L.threads, L.smem); break;
        case LL_PREC_DF64 * NUM_MODES + MODE_DOT: per_sm = occupancy_bt<LL_PREC_DF64, MODE_DOT>(L.threads, L.smem); break;
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_ACCUM: per_sm = occupancy_bt<LL_PREC_F32_MIXED, MODE_ACCUM>(L.threads, L.smem); break;
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_DOT: per_sm = occupancy_bt<LL_PREC_F32_MIXED, MODE_DOT>(L.threads, L.smem); break;
        default: break;
    }
    if (per_sm < 1) return false;
    L.grid = sm_count;
    return true;
}

cudaError_t launch_batched_tma(int precision, int mode, const BatchTmaParams& bp, const BatchTmaLaunch& L, cudaStream_t s) {
    switch (precision * NUM_MODES + mode) {
        case LL_PREC_F64 * NUM_MODES + MODE_ACCUM: return launch_bt_typed<LL_PREC_F64, MODE_ACCUM>(bp, L, s);
        case LL_PREC_F64 * NUM_MODES + MODE_DOT: return launch_bt_typed<LL_PREC_F64, MODE_DOT>(bp, L, s);
        case LL_PREC_DF64 * NUM_MODES + MODE_ACCUM: return launch_bt_typed<LL_PREC_DF64, MODE_ACCUM>(bp, L, s);
        case LL_PREC_DF64 * NUM_MODES + MODE_DOT: return launch_bt_typed<LL_PREC_DF64, MODE_DOT>(bp, L, s);
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_ACCUM: return launch_bt_typed<LL_PREC_F32_MIXED, MODE_ACCUM>(bp, L, s);
        case LL_PREC_F32_MIXED * NUM_MODES + MODE_DOT: return launch_bt_typed<LL_PREC_F32_MIXED, MODE_DOT>(bp, L, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batched_dots(int precision, const BatchTmaMat* mats, int count, int b, int max_span, cudaStream_t s) {
    if (max_span <= 0 || count <= 0) return cudaSuccess;
    const int threads = 128;
    const dim3 grid((unsigned)((max_span + threads - 1) / threads), (unsigned)count);
    if (precision == LL_PREC_F64) k_batched_dots<false><<<grid, threads, 0, s>>>(mats, b);
    else k_batched_dots<true><<<grid, threads, 0, s>>>(mats, b);
    return cudaGetLastError();
}

}  // namespace ll
