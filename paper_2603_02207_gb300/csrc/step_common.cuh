// Per-row arithmetic of one Léja step (Algorithm 2 loop body), shared by the two step kernels
// (register-gather and TMA-gather) so that both produce the same W_{j+1}, P and trace terms.
//
// A thread owns a pair of adjacent columns (2cp, 2cp+1) of a row. It accumulates
// sum_k a_k W_j[c_k, pair] over the row's entries (row_mac), then applies the epilogue: the shift
// beta_j W_j[r, pair], the store of W_{j+1}, and the P-axpy (pass 1), the trace terms (pass 2) or
// the adjoint's U term. Double-float blocks are stored in column pairs (hi, hi, lo, lo), so the
// 16-byte pair feeds the f32x2 instructions directly.
#pragma once

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

// running row sum of one column pair
struct RowAcc {
    double a0 = 0.0, a1 = 0.0;   // F64
    f2x ah = 0ull, al = 0ull;    // DF64 (hi, lo pairs); F32 uses ah
};

template <int PREC>
__device__ __forceinline__ void row_mac(RowAcc& A, const typename ExT<PREC>::T& v, const typename PairT<PREC>::W& x) {
    if constexpr (PREC == LL_PREC_F64) {
        A.a0 = fma(v, x.x, A.a0);
        A.a1 = fma(v, x.y, A.a1);
    } else if constexpr (PREC == LL_PREC_DF64) {
        df2_mac(A.ah, A.al, v.ah2, v.al2, v.nah2, x.x, x.y);
    } else {
        A.ah = f2_fma(v, x, A.ah);
    }
}

// trace partials of the thread's two columns (double-float; FP64 in the F64 mode)
struct TracePart {
    f2x th2 = 0ull, tl2 = 0ull, t0h2 = 0ull, t0l2 = 0ull;
    double td[2] = {0.0, 0.0}, t0d[2] = {0.0, 0.0};
    f2x nh2 = 0ull, nl2 = 0ull;    // STOP modes: ||W_{j+1} col||^2 partials
    double nd[2] = {0.0, 0.0};
};

// per-step scalars broadcast to both lanes, and the adjoint's per-column coefficients
template <int PREC>
struct StepScalars {
    f2x bh2, bl2, nbh2, beta2, dnh2, dnl2, ndnh2, d0h2, d0l2, nd0h2;
    double cadj0, cadj1;
    f2x ch2, cl2, nch2, cf2;
    double dn0, dn1;   // d_{j+1} per column (zero in retired columns under the stopping rule)
    double betad, d0d;   // beta_j and d_0 (FP64)
    __device__ __forceinline__ StepScalars() {}
    // the scalars of column group g of a sweep (beta_{g,j}, d_{g,j+1}, d_{g,0}; no stopping rule)
    __device__ __forceinline__ static StepScalars group(const StepParams& p, int g) {
        StepScalars S;
        const float2* q = p.sw_scal_df + g * SWEEP_SCALARS;
        const double* qd = p.sw_scal + g * SWEEP_SCALARS;
        S.betad = qd[0];
        S.dn0 = S.dn1 = qd[1];
        S.d0d = qd[2];
        S.bh2 = f2_pack(q[0].x, q[0].x);
        S.bl2 = f2_pack(q[0].y, q[0].y);
        S.nbh2 = f2_pack(-q[0].x, -q[0].x);
        S.beta2 = S.bh2;
        S.dnh2 = f2_pack(q[1].x, q[1].x);
        S.dnl2 = f2_pack(q[1].y, q[1].y);
        S.ndnh2 = f2_pack(-q[1].x, -q[1].x);
        S.d0h2 = f2_pack(q[2].x, q[2].x);
        S.d0l2 = f2_pack(q[2].y, q[2].y);
        S.nd0h2 = f2_pack(-q[2].x, -q[2].x);
        S.cadj0 = S.cadj1 = 0.0;
        S.ch2 = S.cl2 = S.nch2 = S.cf2 = 0ull;
        return S;
    }
    // masked = true: d_{j+1} applies only to the columns with live[col] set
    __device__ __forceinline__ StepScalars(const StepParams& p, int cp, bool masked = false) {
        betad = p.beta;
        d0d = p.d0;
        bh2 = f2_pack(p.beta_df.x, p.beta_df.x);
        bl2 = f2_pack(p.beta_df.y, p.beta_df.y);
        nbh2 = f2_pack(-p.beta_df.x, -p.beta_df.x);
        beta2 = f2_pack(p.beta_df.x, p.beta_df.x);   // the leading float of beta_j: (float)beta_j
        const bool l0 = !masked || p.live[2 * cp] != 0, l1 = !masked || p.live[2 * cp + 1] != 0;
        dn0 = l0 ? p.dn : 0.0;
        dn1 = l1 ? p.dn : 0.0;
        dnh2 = f2_pack(l0 ? p.dn_df.x : 0.f, l1 ? p.dn_df.x : 0.f);
        dnl2 = f2_pack(l0 ? p.dn_df.y : 0.f, l1 ? p.dn_df.y : 0.f);
        ndnh2 = f2_pack(l0 ? -p.dn_df.x : 0.f, l1 ? -p.dn_df.x : 0.f);
        d0h2 = f2_pack(p.d0_df.x, p.d0_df.x);
        d0l2 = f2_pack(p.d0_df.y, p.d0_df.y);
        nd0h2 = f2_pack(-p.d0_df.x, -p.d0_df.x);
        const bool q0 = 2 * cp < p.adj_split, q1 = 2 * cp + 1 < p.adj_split;
        cadj0 = q0 ? p.adj_q : p.adj_g;
        cadj1 = q1 ? p.adj_q : p.adj_g;
        const float2 cdf0 = q0 ? p.adj_q_df : p.adj_g_df, cdf1 = q1 ? p.adj_q_df : p.adj_g_df;
        ch2 = f2_pack(cdf0.x, cdf1.x);
        cl2 = f2_pack(cdf0.y, cdf1.y);
        nch2 = f2_pack(-cdf0.x, -cdf1.x);
        cf2 = f2_pack(cdf0.x, cdf1.x);
    }
};

// Epilogue of one row: W_{j+1} = acc + beta_j W_j[r] (+ coef U[r] in the adjoint), stored to
// *wout; pass 1: *pout = (first ? d_0 W_j[r] : po) + d_{j+1} W_{j+1}; pass 2: trace terms
// V[r] . W_{j+1}[r] (and V[r] . W_j[r] on the first step).
template <int PREC, int MODE>
__device__ __forceinline__ void row_epilogue(const StepParams& p, const StepScalars<PREC>& S, RowAcc& A,
                                             const typename PairT<PREC>::W& wr, const typename PairT<PREC>::W& vr,
                                             const typename PairT<PREC>::P& po, typename PairT<PREC>::W* wout,
                                             typename PairT<PREC>::P* pout, TracePart& T) {
    const f2x zero2 = 0ull;
    constexpr int MB = base_mode(MODE);
    constexpr bool STOP = stop_mode(MODE);
    if constexpr (PREC == LL_PREC_F64) {
        double w0 = fma(S.betad, wr.x, A.a0), w1 = fma(S.betad, wr.y, A.a1);
        if constexpr (MB == MODE_ADJ) {
            w0 = fma(S.cadj0, vr.x, w0);
            w1 = fma(S.cadj1, vr.y, w1);
        }
        *wout = make_double2(w0, w1);
        if constexpr (MB == MODE_ACCUM) {
            const double b0 = p.first ? S.d0d * wr.x : po.x, b1 = p.first ? S.d0d * wr.y : po.y;
            *pout = make_double2(fma(S.dn0, w0, b0), fma(S.dn1, w1, b1));
        }
        if constexpr (MB == MODE_DOT) {
            T.td[0] = fma(vr.x, w0, T.td[0]);
            T.td[1] = fma(vr.y, w1, T.td[1]);
            if (p.first) { T.t0d[0] = fma(vr.x, wr.x, T.t0d[0]); T.t0d[1] = fma(vr.y, wr.y, T.t0d[1]); }
        }
        if constexpr (STOP) {
            T.nd[0] = fma(w0, w0, T.nd[0]);
            T.nd[1] = fma(w1, w1, T.nd[1]);
        }
    } else if constexpr (PREC == LL_PREC_DF64) {
        df2_mac(A.ah, A.al, S.bh2, S.bl2, S.nbh2, wr.x, wr.y);
        if constexpr (MB == MODE_ADJ) df2_mac_pp(A.ah, A.al, S.ch2, S.cl2, S.nch2, vr.x, vr.y);
        f2x wh, wl;
        df2_norm(A.ah, A.al, wh, wl);
        *wout = make_ulonglong2(wh, wl);
        if constexpr (STOP) df2_mac_pp(T.nh2, T.nl2, wh, wl, f2_sub(zero2, wh), wh, wl);
        if constexpr (MB == MODE_ACCUM) {
            f2x ph = zero2, pl = zero2;
            if (p.first) df2_mac(ph, pl, S.d0h2, S.d0l2, S.nd0h2, wr.x, wr.y);
            else { ph = po.x; pl = po.y; }
            df2_mac(ph, pl, S.dnh2, S.dnl2, S.ndnh2, wh, wl);
            f2x oh, ol;
            df2_norm(ph, pl, oh, ol);
            *pout = make_ulonglong2(oh, ol);
        }
        if constexpr (MB == MODE_DOT) {
            const f2x nvh = f2_sub(zero2, vr.x);
            df2_mac_pp(T.th2, T.tl2, vr.x, vr.y, nvh, wh, wl);
            if (p.first) df2_mac_pp(T.t0h2, T.t0l2, vr.x, vr.y, nvh, wr.x, wr.y);
        }
    } else {  // LL_PREC_F32_MIXED
        f2x wn = f2_fma(S.beta2, wr, A.ah);
        if constexpr (MB == MODE_ADJ) wn = f2_fma(S.cf2, vr, wn);
        *wout = wn;
        if constexpr (STOP) df2_mac_f(T.nh2, T.nl2, wn, zero2, f2_sub(zero2, wn), wn);
        if constexpr (MB == MODE_ACCUM) {
            f2x ph = zero2, pl = zero2;
            if (p.first) df2_mac_f(ph, pl, S.d0h2, S.d0l2, S.nd0h2, wr);
            else { ph = po.x; pl = po.y; }
            df2_mac_f(ph, pl, S.dnh2, S.dnl2, S.ndnh2, wn);
            f2x oh, ol;
            df2_norm(ph, pl, oh, ol);
            *pout = make_ulonglong2(oh, ol);
        }
        if constexpr (MB == MODE_DOT) {
            // exact FP32 products v * w accumulated in double-float
            const f2x nv = f2_sub(zero2, vr);
            df2_mac_f(T.th2, T.tl2, vr, zero2, nv, wn);
            if (p.first) df2_mac_f(T.t0h2, T.t0l2, vr, zero2, nv, wr);
        }
    }
}

// Block reduction of the per-column partials in row-lane order, then the last CTA sums the
// per-CTA partials in CTA order (both orders fixed: the result is deterministic). Quantities:
// 0 = V . W_{j+1} and 1 = V . W_0 (first step) in the DOT modes, 2 = ||W_{j+1}||^2 in the STOP
// modes, where the last CTA then applies Algorithm 2's test |d_{j+1}| ||W_{j+1}|| > tol to every
// live column. A thread holds NP consecutive column pairs (T[0..NP-1]): thread (row lane l,
// column group g) of `tp` groups per row owns columns 2 NP g .. 2 NP g + 2 NP - 1. `red` must hold
// 2 NP * blockDim.x doubles; every thread of the CTA calls this.
template <int PREC, int MODE, int NP = 1>
__device__ __forceinline__ void trace_reduce(const StepParams& p, TracePart* T, double* red, int tp, int rows,
                                             bool* s_last) {
    constexpr int MB = base_mode(MODE);
    constexpr bool STOP = stop_mode(MODE);
    constexpr int CW = 2 * NP;   // columns per thread
    const int tid = threadIdx.x;
    if constexpr (PREC != LL_PREC_F64) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float h0, h1, l0, l1;
            if constexpr (MB == MODE_DOT) {
                f2_unpack(T[q].th2, h0, h1);
                f2_unpack(T[q].tl2, l0, l1);
                T[q].td[0] = (double)h0 + (double)l0;
                T[q].td[1] = (double)h1 + (double)l1;
                f2_unpack(T[q].t0h2, h0, h1);
                f2_unpack(T[q].t0l2, l0, l1);
                T[q].t0d[0] = (double)h0 + (double)l0;
                T[q].t0d[1] = (double)h1 + (double)l1;
            }
            if constexpr (STOP) {
                f2_unpack(T[q].nh2, h0, h1);
                f2_unpack(T[q].nl2, l0, l1);
                T[q].nd[0] = (double)h0 + (double)l0;
                T[q].nd[1] = (double)h1 + (double)l1;
            }
        }
    }
    const int b = p.b;
    for (int qn = 0; qn < 3; ++qn) {
        if (qn < 2 && MB != MODE_DOT) continue;
        if (qn == 1 && !p.first) continue;
        if (qn == 2 && !STOP) continue;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            red[CW * tid + 2 * q] = qn == 0 ? T[q].td[0] : (qn == 1 ? T[q].t0d[0] : T[q].nd[0]);
            red[CW * tid + 2 * q + 1] = qn == 0 ? T[q].td[1] : (qn == 1 ? T[q].t0d[1] : T[q].nd[1]);
        }
        __syncthreads();
        for (int c = tid; c < b; c += blockDim.x) {
            const int pc = c / CW, e = c - pc * CW;
            double s = 0.0;
            for (int l = 0; l < rows; ++l) s += red[CW * (l * tp + pc) + e];
            p.partials[((size_t)qn * gridDim.x + blockIdx.x) * b + c] = s;
        }
        __syncthreads();
    }
    __threadfence();
    if (tid == 0) *s_last = (atomicAdd(p.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (*s_last) {
        __threadfence();
        if constexpr (MB == MODE_DOT) {
            const int nred = p.first ? 2 : 1;
            for (int c = tid; c < nred * b; c += blockDim.x) {
                const int q = c / b, cc = c - q * b;
                double s = 0.0;
                for (int g = 0; g < (int)gridDim.x; ++g) s += __ldcg(&p.partials[((size_t)q * gridDim.x + g) * b + cc]);
                if (q == 0) p.dots_next[cc] = s; else p.dots_first[cc] = s;
            }
        }
        if constexpr (STOP) {
            int any = 0;
            for (int c = tid; c < b; c += blockDim.x) {
                double s = 0.0;
                for (int g = 0; g < (int)gridDim.x; ++g) s += __ldcg(&p.partials[((size_t)2 * gridDim.x + g) * b + c]);
                int l = p.live[c];
                if (l && !(fabs(p.dn) * sqrt(s) > p.tol)) {
                    p.live[c] = 0;
                    p.stop_deg[c] = p.jnext;
                    l = 0;
                }
                any |= l;
            }
            any = __syncthreads_or(any);
            if (tid == 0 && !any) *p.done = 1;
        }
        if (tid == 0) *p.ticket = 0u;
    }
}

}  // namespace ll
