// Host-side FP64 pieces of the Léja log-determinant method: fast Léja points on [-2, 2] and the
// divided differences of log by Algorithm 1 (arXiv 2603.02207, Section 3.1). These stay on the
// host in FP64 because their stability needs it; the device only sees the resulting scalars.
// Built with -ffp-contract=off so that every product and sum rounds as written.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "host_math.h"

namespace ll {

namespace {

// Incremental fast Léja construction (Eq. Léja5 restricted to gap midpoints, Baglama, Calvetti &
// Reichel 1998). Candidates are kept in ascending order of x, each with its running product of
// distances to the points chosen so far, multiplied in the order the points were chosen.
struct LejaState {
    std::vector<double> pts;
    std::vector<double> cand_x;
    std::vector<double> cand_score;
};

std::mutex g_leja_mutex;
LejaState g_leja;

double score_from_scratch(double x, const std::vector<double>& pts) {
    double s = 1.0;
    for (double p : pts) s = s * std::fabs(x - p);
    return s;
}

void leja_extend(LejaState& st, int count) {
    if ((int)st.pts.size() >= count) return;
    if (st.pts.empty()) st.pts.push_back(2.0);
    if ((int)st.pts.size() >= count) return;
    if (st.pts.size() == 1) {
        st.pts.push_back(-2.0);
        st.cand_x.assign(1, 0.0);
        st.cand_score.assign(1, score_from_scratch(0.0, st.pts));
    }
    while ((int)st.pts.size() < count) {
        double best = 0.0;
        for (double s : st.cand_score) best = std::max(best, s);
        const double thresh = best * (1.0 - kLejaTieRtol);
        size_t idx = 0;
        while (st.cand_score[idx] < thresh) ++idx;   // smallest x among the (near-)maximisers
        const double x = st.cand_x[idx];
        // neighbours of x among the chosen points: the gap it splits
        double left = -2.0, right = 2.0;
        for (double p : st.pts) {
            if (p < x && p > left) left = p;
            if (p > x && p < right) right = p;
        }
        st.pts.push_back(x);
        st.cand_x.erase(st.cand_x.begin() + idx);
        st.cand_score.erase(st.cand_score.begin() + idx);
        for (size_t i = 0; i < st.cand_x.size(); ++i)
            st.cand_score[i] = st.cand_score[i] * std::fabs(st.cand_x[i] - x);
        const double ml = (left + x) / 2.0, mr = (x + right) / 2.0;
        // insert the two new midpoints keeping ascending order
        for (double m : {ml, mr}) {
            auto it = std::lower_bound(st.cand_x.begin(), st.cand_x.end(), m);
            const size_t pos = (size_t)(it - st.cand_x.begin());
            st.cand_x.insert(it, m);
            st.cand_score.insert(st.cand_score.begin() + pos, score_from_scratch(m, st.pts));
        }
    }
}

}  // namespace

void leja_points(int count, double* out) {
    std::lock_guard<std::mutex> lock(g_leja_mutex);
    leja_extend(g_leja, count);
    for (int i = 0; i < count; ++i) out[i] = g_leja.pts[i];
}

int divided_differences_alg1(double lmin, double lmax, int degree, int sval_mode, double* d, int max_terms) {
    const int m1 = degree + 1;
    std::vector<double> xi(m1);
    leja_points(m1, xi.data());
    // Eq. eq_centre / eq_gamma and the affine map z = c + gamma xi (Eq. z_mapping)
    const double c = (lmin + lmax) / 2.0;
    const double gamma = (lmax - lmin) / 4.0;
    const double s = (sval_mode == LL_SVAL_HALF_LMAX) ? lmax / 2.0 : c;
    // W_m = (Q_m - s I) / s with Q_m = c I + gamma Qhat_m: lower bidiagonal, diagonal
    // (c + gamma xi_i - s) / s and sub-diagonal gamma / s (Algorithm 1 steps 4-6)
    std::vector<double> wd(m1);
    for (int i = 0; i < m1; ++i) wd[i] = ((c + gamma * xi[i]) - s) / s;
    const double ws = gamma / s;
    // step 7: log(I + W_m) e_1 = sum_{k>=1} (-1)^{k+1} W_m^k e_1 / k
    std::vector<double> t(m1, 0.0), sum(m1, 0.0);
    t[0] = 1.0;
    int terms = -1;
    for (int k = 1; k <= max_terms; ++k) {
        for (int i = m1 - 1; i >= 1; --i) t[i] = wd[i] * t[i] + ws * t[i - 1];
        t[0] = wd[0] * t[0];
        double term_max = 0.0, sum_max = 0.0;
        for (int i = 0; i < m1; ++i) {
            const double term = (k & 1) ? t[i] / (double)k : -(t[i] / (double)k);
            sum[i] = sum[i] + term;
            term_max = std::max(term_max, std::fabs(term));
            sum_max = std::max(sum_max, std::fabs(sum[i]));
        }
        if (k >= kTaylorMinTerms && term_max < kTaylorRelTol * sum_max) { terms = k; break; }
    }
    if (terms < 0) return -1;
    // step 8: log(Q_m) e_1 = log(s) e_1 + log(I + W_m) e_1
    for (int i = 0; i < m1; ++i) d[i] = sum[i];
    d[0] = d[0] + std::log(s);
    return terms;
}

// Divided differences of g(xi) = log(c + gamma xi) over the Léja points on [-2, 2] by the
// textbook table (Eq. Léja7): g[xi_0..xi_j] = gamma^j log[z_0..z_j] = d_j. Working in the xi
// variable keeps every entry in range; for Léja-ordered nodes the table is accurate to a few
// ulps of max |d| (checked against a 120-digit table up to condition number 1e9, degree 250).
void divided_differences_table(double lmin, double lmax, int degree, double* d) {
    const int m1 = degree + 1;
    std::vector<double> xi(m1), col(m1);
    leja_points(m1, xi.data());
    const double c = (lmin + lmax) / 2.0;
    const double gamma = (lmax - lmin) / 4.0;
    for (int i = 0; i < m1; ++i) col[i] = std::log(c + gamma * xi[i]);
    d[0] = col[0];
    for (int o = 1; o < m1; ++o) {
        for (int i = 0; i + o < m1; ++i) col[i] = (col[i + 1] - col[i]) / (xi[i + o] - xi[i]);
        d[o] = col[0];
    }
}

// Binary128 (113-bit significand) on both hosts: long double on aarch64, _Float128 on x86-64;
// the logarithm is glibc's binary128 one in both cases.
#if defined(__aarch64__)
static_assert(__LDBL_MANT_DIG__ == 113, "long double is not binary128 on this aarch64 target");
typedef long double quad;
static inline quad quad_log(quad x) { return logl(x); }
#else
typedef _Float128 quad;
static inline quad quad_log(quad x) { return logf128(x); }
#endif

void divided_differences_table_q(double lmin, double lmax, int degree, double* d) {
    const int m1 = degree + 1;
    std::vector<double> xi(m1);
    leja_points(m1, xi.data());
    // c and gamma as the step recurrence uses them (FP64); the nodes c + gamma xi_i are exact in
    // binary128 (a 53 x 53-bit product and one addition)
    const double c = (lmin + lmax) / 2.0;
    const double gamma = (lmax - lmin) / 4.0;
    std::vector<quad> col(m1);
    for (int i = 0; i < m1; ++i) col[i] = quad_log((quad)c + (quad)gamma * (quad)xi[i]);
    d[0] = (double)col[0];
    for (int o = 1; o < m1; ++o) {
        for (int i = 0; i + o < m1; ++i) col[i] = (col[i + 1] - col[i]) / ((quad)xi[i + o] - (quad)xi[i]);
        d[o] = (double)col[0];
    }
}

int scaled_divided_differences(double lmin, double lmax, int degree, int sval_mode, double* d) {
    const int m1 = degree + 1;
    std::vector<double> xi(m1);
    leja_points(m1, xi.data());
    const double c = (lmin + lmax) / 2.0;
    const double gamma = (lmax - lmin) / 4.0;
    const double s = (sval_mode == LL_SVAL_HALF_LMAX) ? lmax / 2.0 : c;
    // convergence factor of Algorithm 1's series: q = max_i |z_i / s - 1|
    double q = 0.0;
    for (int i = 0; i < m1; ++i) q = std::max(q, std::fabs((c + gamma * xi[i]) / s - 1.0));
    const bool use_table = q >= 1.0 || (q > 0.0 && std::log(kTaylorRelTol) / std::log(q) > kTableThresholdTerms);
    if (use_table) {
        divided_differences_table(lmin, lmax, degree, d);
        return 0;
    }
    return divided_differences_alg1(lmin, lmax, degree, sval_mode, d, kTaylorMaxTerms);
}

double sigma_of(double lmin) { return lmin < 1.0 ? lmin : 1.0; }

int degree_from_bounds(double lmin, double lmax) {
    const double sk = std::sqrt(lmax / lmin);
    const double rho = (sk + 1.0) / (sk - 1.0);
    const double m = std::ceil(std::log(1e6) / std::log(rho));
    if (!(m == m)) return 250;
    return (int)std::max(10.0, std::min(250.0, m));
}

}  // namespace ll
