// host_math.h -- host-side quadrature and polynomial helpers of the table setup (FP64):
// Gauss-Legendre rules on [0, 1], the collapsed triangle rule, Chebyshev nodes and polynomials,
// and the Lagrange polynomials of an interval on its transformed Chebyshev nodes (Section 3.1).
#pragma once

#include <cmath>
#include <vector>

namespace pfmm {
namespace hostm {

constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre nodes and weights on [0, 1] (Newton iteration on P_n)
inline void gauss01(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p1 = 1.0, p2 = 0.0;
        for (int k = 1; k <= n; ++k) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
    }
}

// collapsed (Duffy) rule on {0 <= s2 <= s1 <= 1}: s1 = u, s2 = u v, weight w_u w_v u
inline std::vector<double> collapsed_rule(int n)
{
    std::vector<double> x, w, r(3 * (size_t)n * n);
    gauss01(n, x, w);
    int q = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j, ++q) {
            r[q] = x[i];
            r[n * n + q] = x[i] * x[j];
            r[2 * n * n + q] = w[i] * w[j] * x[i];
        }
    return r;
}

inline double cheb_node(int k, int m) { return std::cos((2.0 * k + 1.0) * kPi / (2.0 * m + 2.0)); }

inline double cheb_T(int k, double x)
{
    double t0 = 1.0, t1 = x;
    if (k == 0) return 1.0;
    for (int i = 2; i <= k; ++i) {
        double t2 = 2.0 * x * t1 - t0;
        t0 = t1;
        t1 = t2;
    }
    return t1;
}

inline double lagrange(int b, int m, double lo, double hi, double t)
{
    double c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo), xb = c + hw * cheb_node(b, m), v = 1.0;
    for (int k = 0; k <= m; ++k)
        if (k != b) {
            double xk = c + hw * cheb_node(k, m);
            v *= (t - xk) / (xb - xk);
        }
    return v;
}

}  // namespace hostm
}  // namespace pfmm
