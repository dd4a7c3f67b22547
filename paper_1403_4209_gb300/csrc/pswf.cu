// Zeroth-order prolate spheroidal function psi_0(c, x), |x| <= 1 (taper of thesis Sec. 2.3.3,
// chosen in Sec. 4.2.1), as an even Legendre series.
//
// psi_0 is the eigenfunction with the smallest eigenvalue chi of the prolate operator
//   L f = -d/dx[(1 - x^2) f'] + c^2 x^2 f.
// On orthonormal Legendre functions Pb_k = sqrt(k + 1/2) P_k, L is tridiagonal in steps of 2:
//   <Pb_k, L Pb_k>     = k(k+1) + c^2 (2k^2 + 2k - 1) / ((2k - 1)(2k + 3))
//   <Pb_{k+2}, L Pb_k> = c^2 (k+1)(k+2) / ((2k + 3) sqrt((2k + 1)(2k + 5)))
// (from x^2 P_k = a P_{k+2} + b P_k + c' P_{k-2}).  psi_0 is even, so only k = 0, 2, 4, ...
// enter.  The smallest eigenvalue is bracketed by Sturm-sequence bisection and its
// eigenvector found by inverse iteration with a shift just below it (the shifted matrix is
// then positive definite, so the tridiagonal elimination needs no pivoting).  The series is
// scaled so that psi_0(0) = 1.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace wg {

static int sturm_count_below(const std::vector<double>& d, const std::vector<double>& e, double x)
{
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (size_t i = 1; i < d.size(); ++i) {
        double qq = (q == 0.0) ? 1e-300 : q;
        q = d[i] - x - e[i - 1] * e[i - 1] / qq;
        if (q < 0) ++cnt;
    }
    return cnt;
}

std::vector<double> pswf_coefficients(double c)
{
    const int n = static_cast<int>(c) + 40;
    std::vector<double> d(n), e(n - 1);
    const double c2 = c * c;
    for (int m = 0; m < n; ++m) {
        const double k = 2.0 * m;
        d[m] = k * (k + 1) + c2 * (2 * k * k + 2 * k - 1) / ((2 * k - 1) * (2 * k + 3));
        if (m + 1 < n)
            e[m] = c2 * (k + 1) * (k + 2) / ((2 * k + 3) * std::sqrt((2 * k + 1) * (2 * k + 5)));
    }
    // Gershgorin interval
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0) + (i + 1 < n ? std::fabs(e[i]) : 0);
        lo = std::fmin(lo, d[i] - r);
        hi = std::fmax(hi, d[i] + r);
    }
    // smallest eigenvalue: largest x with no eigenvalue below it
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count_below(d, e, mid) == 0) lo = mid; else hi = mid;
    }
    const double lam = lo;
    const double shift = lam - 1e-9 * std::fmax(1.0, std::fabs(lam));
    // inverse iteration: solve (T - shift I) y = x by tridiagonal elimination
    std::vector<double> y(n, 1.0), cp(n), dp(n);
    for (int it = 0; it < 6; ++it) {
        double b0 = d[0] - shift;
        cp[0] = (n > 1 ? e[0] : 0) / b0;
        dp[0] = y[0] / b0;
        for (int i = 1; i < n; ++i) {
            double den = (d[i] - shift) - e[i - 1] * cp[i - 1];
            cp[i] = (i + 1 < n ? e[i] : 0) / den;
            dp[i] = (y[i] - e[i - 1] * dp[i - 1]) / den;
        }
        y[n - 1] = dp[n - 1];
        for (int i = n - 2; i >= 0; --i) y[i] = dp[i] - cp[i] * y[i + 1];
        double nrm = 0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (double& v : y) v /= nrm;
    }
    // coefficients on plain Legendre polynomials of even degree, scaled to psi_0(0) = 1
    std::vector<double> a(n);
    double p0 = 1.0, at0 = 0.0;   // P_{2m}(0) = (-1)^m (2m-1)!! / (2m)!!
    for (int m = 0; m < n; ++m) {
        if (m > 0) p0 *= -(2.0 * m - 1) / (2.0 * m);
        a[m] = y[m] * std::sqrt(2.0 * m + 0.5);
        at0 += a[m] * p0;
    }
    for (double& v : a) v /= at0;
    return a;
}

double pswf_eval_host(const std::vector<double>& a, double x)
{
    double pm1 = 1.0, p = x, s = a[0];
    const int deg = 2 * static_cast<int>(a.size()) - 2;
    for (int j = 1; j < deg; ++j) {
        double pn = ((2.0 * j + 1) * x * p - j * pm1) / (j + 1);
        pm1 = p;
        p = pn;
        if ((j + 1) % 2 == 0) s += a[(j + 1) / 2] * p;
    }
    return s;
}

}  // namespace wg
