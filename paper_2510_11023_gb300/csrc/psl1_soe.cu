// psl1_soe.cu -- exponents and weights of the fast (sum-of-exponentials)
// history of the uniform L1 scheme (host code).
//
// The paper names a fast evaluation of the nonlocal memory term as future work
// (Conclusion, item (i)) without a construction.  The one used here writes the
// L1 weight as a Laplace-type integral,
//   b(x) = (x+1)^{1-a} - x^{1-a} = c int_0^inf tau^{a-2} (1 - e^{-tau}) e^{-x tau} dtau,
//   c = (1-a)/Gamma(a)        (from s^{-a} = Gamma(a)^{-1} int tau^{a-1} e^{-s tau}),
// and discretises it on [0, tau0], tau0 = 1/X, by Gauss-Jacobi quadrature with
// the weight tau^{a-1} (SOE_GJ nodes) and on [tau0, tau1] by composite
// Gauss-Legendre quadrature in y = log tau (SOE_GL nodes on each of
// ceil((y1 - y0)/2) equal segments, y1 = log(log(1/eps)/nloc) + 0.3), so that
//   b(x) ~ sum_i w_i exp(-s_i x)    for nloc <= x <= X
// to about 5e-15 relative (eps = 1e-12, 0.2 <= a < 1, X <= 8192).
//
// Both rules come from the Jacobi matrix of their weight's three-term
// recurrence: the nodes are its eigenvalues, found one by one by bisection on
// the Sturm-sequence count, and the weights are the Christoffel numbers
// mu0 / sum_k p_k(t)^2 of the orthonormal polynomials.
#include <cmath>
#include <vector>

#include "psl1_soe.h"

namespace psl1 {

namespace {

// Jacobi matrix of the weight (1-t)^ja (1+t)^jb on (-1,1): diagonal d, off-diagonal e (e[0] unused)
void jacobi_matrix(int n, double ja, double jb, std::vector<double>& d, std::vector<double>& e)
{
    d.assign(n, 0.0);
    e.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double s = 2.0 * k + ja + jb;
        d[k] = (k == 0) ? (jb - ja) / (ja + jb + 2.0) : (jb * jb - ja * ja) / (s * (s + 2.0));
        if (k > 0)
            e[k] = std::sqrt(4.0 * k * (k + ja) * (k + jb) * (k + ja + jb) / (s * s * (s + 1.0) * (s - 1.0)));
    }
}

// number of eigenvalues of the tridiagonal (d, e) below x (Sturm sequence)
int count_below(const std::vector<double>& d, const std::vector<double>& e, double x)
{
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        q = (d[i] - x) - (i ? e[i] * e[i] / q : 0.0);
        if (q == 0.0) q = -1e-300;   // x is an eigenvalue of the leading block: count it below
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Gauss rule of the Jacobi weight with total mass mu0: nodes ascending on (-1,1)
void gauss_rule(int n, double ja, double jb, double mu0, double* t, double* w)
{
    std::vector<double> d, e;
    jacobi_matrix(n, ja, jb, d, e);
    for (int k = 0; k < n; ++k) {
        double lo = -1.0, hi = 1.0;   // every node lies inside (-1, 1)
        for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (count_below(d, e, mid) > k)
                hi = mid;
            else
                lo = mid;
        }
        const double x = 0.5 * (lo + hi);
        // orthonormal polynomials (up to the common factor mu0^{-1/2}) at x
        double pm = 0.0, p = 1.0, sum = 1.0;
        for (int j = 0; j + 1 < n; ++j) {
            const double pn = ((x - d[j]) * p - (j ? e[j] * pm : 0.0)) / e[j + 1];
            pm = p;
            p = pn;
            sum += p * p;
        }
        t[k] = x;
        w[k] = mu0 / sum;
    }
}

}  // namespace

int soe_nodes(double alpha, int nloc, int X, double eps, int maxn, double* s, double* w)
{
    if (!(alpha > 0.0) || nloc < 1 || X < 1 || !(eps > 0.0 && eps < 1.0)) return -1;
    if (alpha >= 1.0) return 0;   // no history: every weight b(x), x >= 1, is zero
    const double c = (1.0 - alpha) / std::tgamma(alpha);
    const double tau0 = 1.0 / X;
    const double y0 = std::log(tau0), y1 = std::log(std::log(1.0 / eps) / nloc) + 0.3;
    int nseg = (int)std::ceil((y1 - y0) / 2.0);
    if (nseg < 1) nseg = 1;
    const int L = SOE_GJ + nseg * SOE_GL;
    if (L > maxn) return -1;
    double t[SOE_GJ > SOE_GL ? SOE_GJ : SOE_GL], wt[SOE_GJ > SOE_GL ? SOE_GJ : SOE_GL];
    // [0, tau0]: tau = tau0 (1+t)/2, tau^{a-1} dtau = (tau0/2)^a (1+t)^{a-1} dt,
    // integrand (1 - e^{-tau}) / tau against the Jacobi weight (1+t)^{a-1} (mass 2^a / a)
    gauss_rule(SOE_GJ, 0.0, alpha - 1.0, std::pow(2.0, alpha) / alpha, t, wt);
    const double sc = c * std::pow(0.5 * tau0, alpha);
    for (int i = 0; i < SOE_GJ; ++i) {
        const double tau = 0.5 * tau0 * (1.0 + t[i]);
        s[i] = tau;
        w[i] = sc * wt[i] * (-std::expm1(-tau)) / tau;
    }
    // [y0, y1]: integrand c e^{(a-1) y} (1 - e^{-e^y}) e^{-x e^y} dy, Legendre rule per segment
    gauss_rule(SOE_GL, 0.0, 0.0, 2.0, t, wt);
    const double h = (y1 - y0) / nseg;
    for (int g = 0; g < nseg; ++g)
        for (int i = 0; i < SOE_GL; ++i) {
            const double y = y0 + h * (g + 0.5 * (1.0 + t[i]));
            const double tau = std::exp(y);
            const int k = SOE_GJ + g * SOE_GL + i;
            s[k] = tau;
            w[k] = c * 0.5 * h * wt[i] * std::exp((alpha - 1.0) * y) * (-std::expm1(-tau));
        }
    return L;
}

}  // namespace psl1
