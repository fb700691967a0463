// psl1_soe.h -- parameters and host routine of the fast (sum-of-exponentials)
// history of the uniform L1 scheme (see psl1_soe.cu).
#pragma once

namespace psl1 {

constexpr int SOE_NLOC = 16;        // exact local window: weights b(x), x < SOE_NLOC
constexpr double SOE_EPS = 1e-12;   // sets the largest exponent (tau1 = log(1/eps)/nloc)
constexpr int SOE_GJ = 10;          // Gauss-Jacobi nodes on [0, 1/X]
constexpr int SOE_GL = 14;          // Gauss-Legendre nodes per segment in log tau
constexpr int SOE_MAXL = 128;       // most exponentials of one instance

// Exponents s (> 0) and weights w (> 0) with b(x) ~ sum_i w_i exp(-s_i x) for
// nloc <= x <= X; returns their number (0 for alpha = 1: no history), or -1.
int soe_nodes(double alpha, int nloc, int X, double eps, int maxn, double* s, double* w);

}  // namespace psl1
