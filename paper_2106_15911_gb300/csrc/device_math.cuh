// device_math.cuh -- time-integrated heat kernels and Chebyshev helpers for the GPU kernels.
//
// Section 2, Eq. heat_kernel: G(r, s) = (4 pi alpha s)^(-3/2) exp(-r^2 / (4 alpha s)) for s > 0.
// The Galerkin entries of V_h integrate G over a target step and a source step; with uniform
// steps h and offset d = k - j they are second differences of the second time antiderivative
//   G2(r, s) = [(s + r^2/(2 alpha)) erfc(u) - r sqrt(s/(pi alpha)) e^{-u^2}] / (4 pi alpha r),
//   u = r / (2 sqrt(alpha s)),
// V_d(r) = G2((d+1)h) - 2 G2(d h) + G2((d-1)h)   (G2 = 0 for s <= 0).
// For d >= 1 the part of G2 linear in s cancels; when u is small we evaluate the bounded form
//   G2t = G2 - s/(4 pi alpha r)
//       = r erfc(u)/(8 pi alpha^2) - sqrt(s) (erf(u)/u)/(8 pi alpha^1.5) - sqrt(s) e^{-u^2}/(4 pi^1.5 alpha^1.5),
// and for large u the plain form (whose terms then carry no common linear part).
// The double layer alpha dG/dn_y = (x - y).n_y G / (2 s) integrates to (x - y).n_y * DL2 with
//   DL2 = [(s/r^2 - 1/(2 alpha)) erfc(u) + sqrt(s/(pi alpha)) e^{-u^2} / r] / (4 pi r),
//   DL2t = DL2 - s/(4 pi r^3) = -[u phi2(u)/2 + erfc(u)] / (8 pi alpha r),
//   phi2(u) = (erf(u) - 2u e^{-u^2}/sqrt(pi)) / u^3.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace pfmm {
namespace dev {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;

__device__ __forceinline__ double d_erf(double x) { return erf(x); }
__device__ __forceinline__ float d_erf(float x) { return erff(x); }
__device__ __forceinline__ double d_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float d_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }

// erf(u) and erfc(u), each from the function that is accurate for it
template <typename R>
__device__ __forceinline__ void erf_pair(R u, R &ef, R &efc)
{
    if (u < R(0.5)) {
        ef = d_erf(u);
        efc = R(1) - ef;
    } else {
        efc = d_erfc(u);
        ef = R(1) - efc;
    }
}

// erf(u)/u (Maclaurin series below 0.05)
template <typename R>
__device__ __forceinline__ R erf_over_u(R u, R ef)
{
    if (u < R(0.05)) {
        R u2 = u * u;
        R s = R(1) + u2 * (R(-1.0 / 3.0) + u2 * (R(1.0 / 10.0) + u2 * (R(-1.0 / 42.0) + u2 * R(1.0 / 216.0))));
        return R(2.0 / kSqrtPi) * s;
    }
    return ef / u;
}

// phi2(u) = (erf(u) - 2u e^{-u^2}/sqrt(pi)) / u^3; series (2/sqrt(pi)) sum_{n>=1} (-1)^{n+1} 2n u^{2n-2} / (n! (2n+1))
template <typename R>
__device__ __forceinline__ R phi2(R u, R ef, R ex)
{
    if (u < R(0.5)) {
        R u2 = u * u, acc = R(0);
        // Horner from n = 12 down to n = 1
        double fact[13] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320, 362880, 3628800, 39916800, 479001600};
#pragma unroll
        for (int n = 12; n >= 1; --n) {
            double c = (2.0 * n) / (fact[n] * (2.0 * n + 1.0));
            acc = acc * u2 + R((n % 2) ? c : -c);
        }
        return R(2.0 / kSqrtPi) * acc;
    }
    return (ef - R(2.0 / kSqrtPi) * u * ex) / (u * u * u);
}

// Single-layer time integrals for d = 0 .. nd-1 at distance r (nd <= 8).  r must be > 0 when
// d = 0 is requested; for d >= 1 r = 0 is allowed.
template <typename R>
__device__ __forceinline__ void time_V_all(R r, R h, R alpha, int nd, R *out)
{
    R g2[9], g2t[9];
    g2[0] = R(0);
    g2t[0] = R(0);
    const R a32 = alpha * d_sqrt(alpha);
    const R c_lin = R(1) / (R(4 * kPi) * alpha);
    for (int k = 1; k <= nd; ++k) {
        R s = R(k) * h;
        R ss = d_sqrt(s);
        R u = r / (R(2) * d_sqrt(alpha) * ss);
        R ef, efc;
        erf_pair(u, ef, efc);
        R ex = d_exp(-u * u);
        g2t[k] = r * efc / (R(8 * kPi) * alpha * alpha) - ss * erf_over_u(u, ef) / (R(8 * kPi) * a32) -
                 ss * ex / (R(4 * kPi * kSqrtPi) * a32);
        g2[k] = (r > R(0)) ? ((s + r * r / (R(2) * alpha)) * efc - r * ss / d_sqrt(R(kPi) * alpha) * ex) * c_lin / r
                           : R(0);
    }
    out[0] = g2[1];
    for (int d = 1; d < nd; ++d) {
        R u = r / (R(2) * d_sqrt(alpha * R(d + 1) * h));
        out[d] = (u < R(1)) ? (g2t[d + 1] - g2t[d] - g2t[d] + g2t[d - 1]) : (g2[d + 1] - g2[d] - g2[d] + g2[d - 1]);
    }
}

// G2 and its bounded form G2t (above) at one time difference s (both 0 for s <= 0)
__device__ __forceinline__ void g2_and_g2t(double r, double s, double alpha, double &g2, double &g2t)
{
    if (!(s > 0.0)) {
        g2 = g2t = 0.0;
        return;
    }
    const double ss = sqrt(s), a32 = alpha * sqrt(alpha), u = r / (2.0 * sqrt(alpha) * ss);
    double ef, efc;
    erf_pair(u, ef, efc);
    const double ex = exp(-u * u);
    g2t = r * efc / (8.0 * kPi * alpha * alpha) - ss * erf_over_u(u, ef) / (8.0 * kPi * a32) -
          ss * ex / (4.0 * kPi * kSqrtPi * a32);
    g2 = r > 0.0 ? ((s + r * r / (2.0 * alpha)) * efc - r * ss / sqrt(kPi * alpha) * ex) / (4.0 * kPi * alpha * r) : 0.0;
}

// Single-layer entry factor for a target step (tk0, tk1] and a source step (tj0, tj1] of any
// lengths (general time steps): the second difference of G2 over the four time differences;
// 0 for a later source step, G2(tk1 - tk0) alone for the same step (r > 0 then).  As for uniform
// steps the bounded form is taken when u at the largest difference is below 1 (the linear parts
// cancel when the source step precedes the target step).
__device__ __forceinline__ double time_V_steps(double r, double tk0, double tk1, double tj0, double tj1,
                                               double alpha)
{
    if (tj0 >= tk1) return 0.0;
    double g[4], gt[4];
    if (tj0 == tk0 && tj1 == tk1) {
        g2_and_g2t(r, tk1 - tk0, alpha, g[0], gt[0]);
        return g[0];
    }
    const double s[4] = {tk1 - tj0, tk1 - tj1, tk0 - tj0, tk0 - tj1};
    for (int i = 0; i < 4; ++i) g2_and_g2t(r, s[i], alpha, g[i], gt[i]);
    const double u = r / (2.0 * sqrt(alpha * s[0]));
    return u < 1.0 ? (gt[0] - gt[1]) - (gt[2] - gt[3]) : (g[0] - g[1]) - (g[2] - g[3]);
}

// Double-layer time factors for d = 0 .. nd-1 (multiply by (x - y).n_y); 0 at r = 0.
template <typename R>
__device__ __forceinline__ void time_K_all(R r, R h, R alpha, int nd, R *out)
{
    if (!(r > R(0))) {
        for (int d = 0; d < nd; ++d) out[d] = R(0);
        return;
    }
    R dl[9], dlt[9];
    dl[0] = R(0);
    dlt[0] = R(0);
    for (int k = 1; k <= nd; ++k) {
        R s = R(k) * h;
        R u = r / (R(2) * d_sqrt(alpha * s));
        R ef, efc;
        erf_pair(u, ef, efc);
        R ex = d_exp(-u * u);
        dl[k] = ((s / (r * r) - R(1) / (R(2) * alpha)) * efc + d_sqrt(s / (R(kPi) * alpha)) * ex / r) / (R(4 * kPi) * r);
        dlt[k] = -(R(0.5) * u * phi2(u, ef, ex) + efc) / (R(8 * kPi) * alpha * r);
    }
    out[0] = dl[1];
    for (int d = 1; d < nd; ++d) {
        R u = r / (R(2) * d_sqrt(alpha * R(d + 1) * h));
        out[d] = (u < R(1)) ? (dlt[d + 1] - dlt[d] - dlt[d] + dlt[d - 1]) : (dl[d + 1] - dl[d] - dl[d] + dl[d - 1]);
    }
}

// Chebyshev polynomials T_0..T_m at x (three-term recurrence)
template <typename R>
__device__ __forceinline__ void cheb_all(R x, int m, R *T)
{
    T[0] = R(1);
    if (m >= 1) T[1] = x;
    for (int k = 2; k <= m; ++k) T[k] = R(2) * x * T[k - 1] - T[k - 2];
}

// derivatives T_k'(x) = k U_{k-1}(x)
template <typename R>
__device__ __forceinline__ void cheb_deriv_all(R x, int m, R *dT)
{
    R u0 = R(1), u1 = R(2) * x;
    dT[0] = R(0);
    if (m >= 1) dT[1] = R(1);
    for (int k = 2; k <= m; ++k) {
        dT[k] = R(k) * u1;
        R u2 = R(2) * x * u1 - u0;
        u0 = u1;
        u1 = u2;
    }
}

}  // namespace dev
}  // namespace pfmm
