// Host-side FP64 method pieces (see host_math.cpp).
#pragma once
#include "leja.h"

namespace ll {

constexpr double kLejaTieRtol = 1e-10;      // relative tie tolerance of the fast Léja argmax
constexpr double kTaylorRelTol = 1e-18;     // Algorithm 1 series stop: term < tol * sum (max-norms)
constexpr int kTaylorMinTerms = 10;
constexpr int kTaylorMaxTerms = 5000000;
constexpr double kTableThresholdTerms = 1e6;   // predicted series length beyond which the table is used

// First `count` fast Léja points on [-2, 2] (cached, thread-safe).
void leja_points(int count, double* out);
// Algorithm 1 on [lmin, lmax]: d[0..degree]; returns the number of Taylor terms, -1 if the
// series did not converge within max_terms.
int divided_differences_alg1(double lmin, double lmax, int degree, int sval_mode, double* d, int max_terms);
// The xi-variable divided-difference table of log(c + gamma xi) (Eq. Léja7): d[0..degree].
void divided_differences_table(double lmin, double lmax, int degree, double* d);
// The same table in binary128 arithmetic, rounded to FP64 at the end: the table's cancellation
// costs no digit of the FP64 coefficients at the degrees and conditionings the library takes.
void divided_differences_table_q(double lmin, double lmax, int degree, double* d);
// Algorithm 1 when its series would converge within kTableThresholdTerms terms, else the table.
// Returns the Taylor terms used (0 = table), -1 if Algorithm 1 did not converge.
int scaled_divided_differences(double lmin, double lmax, int degree, int sval_mode, double* d);
// Section 4: sigma = lmin if lmin < 1 else 1.
double sigma_of(double lmin);
// Proposition 3.1 degree rule: clamp(ceil(ln 1e6 / ln rho), 10, 250).
int degree_from_bounds(double lmin, double lmax);

}  // namespace ll
