/*
 * pfmm_oracle.c -- CPU FP64 oracle for the space-time heat BEM operators and the pFMM matvec.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load it.  It shares no code, header, table or helper with the library
 * under paper_2106_15911_gb300/; it is plain, slow, loop-by-loop C written from the paper
 * (arXiv 2106.15911):
 *
 *   Section 2            heat kernel (Eq. heat_kernel), Galerkin matrices V_h, K_h, M_h
 *   Section 3.1          Chebyshev / Lagrange expansion (Eq. kernel_approx, exp_coeffs_3d/1d)
 *   Section 3.2, Alg. 1  4D box cluster tree, padding
 *   Section 3.3          nearfield and interaction lists (Eq. 03:ILtemp, 03:Iarea,
 *                        def_st_nearfield, def_st_interaction_list)
 *   Section 3.4, Alg. 2  S2M, M2M, M2L, L2L, L2T and nearfield evaluation
 *
 * Readings where the paper is silent (its nearfield quadrature is in a reference that is not
 * reproduced):
 *   - time integrals are closed-form second antiderivatives of the heat kernel in the time
 *     difference (derived from Eq. heat_kernel, pinned against adaptive quadrature);
 *   - spatial integrals: a collapsed (Duffy) Gauss-Legendre n_r x n_r rule per triangle for
 *     regular pairs; the Sauter-Schwab regularising transformations with n_s Gauss points per
 *     direction for identical / edge-adjacent / vertex-adjacent pairs at time offsets d = 0, 1.
 *
 * Parity unpinned: the absolute accuracy of that nearfield rule relative to the paper's
 * (unavailable) semi-analytic scheme; it is pinned only by self-convergence and by closed-form
 * Laplace single/double-layer potentials of a flat triangle.
 *
 * Uniform time steps t_j = j*h only.  Every length is in the units of the input mesh.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAXL 32
#define OR_MAXQ 64

/* ======================================================================================
 * 1. Heat kernel and its time integrals (Section 2, Eq. heat_kernel)
 *
 *   G(r, s)  = (4 pi alpha s)^(-3/2) exp(-r^2 / (4 alpha s)),  s > 0;   0 for s <= 0
 *   G1(r, s) = int_0^s G(r, q) dq = erfc(u) / (4 pi alpha r),  u = r / (2 sqrt(alpha s))
 *   G2(r, s) = int_0^s G1(r, q) dq
 *            = [(s + r^2/(2 alpha)) erfc(u) - r sqrt(s/(pi alpha)) exp(-u^2)] / (4 pi alpha r)
 *   The Galerkin time integral over steps k and j (1-based, uniform h) of G(r, t - tau) is
 *   G2(t_k - t_{j-1}) - G2(t_k - t_j) - G2(t_{k-1} - t_{j-1}) + G2(t_{k-1} - t_j).
 *   For k > j the parts of G2 linear in s cancel, so G2 may be replaced by
 *   G2t = G2 - s/(4 pi alpha r), which stays finite as r -> 0.
 *
 *   Double layer: alpha dG/dn_y(x - y, s) = (x - y).n_y * G(r, s) / (2 s); its two time
 *   integrals are (x - y).n_y * DL2(r, s) with DL2 = -(alpha / r) dG2/dr:
 *   DL2(r, s) = [(s/r^2 - 1/(2 alpha)) erfc(u) + sqrt(s/(pi alpha)) exp(-u^2) / r] / (4 pi r)
 *   and, again for k > j, DL2t = DL2 - s/(4 pi r^3).
 * ====================================================================================== */

double orc_G(double r, double s, double alpha)
{
    if (s <= 0.0) return 0.0;
    return pow(4.0 * OR_PI * alpha * s, -1.5) * exp(-r * r / (4.0 * alpha * s));
}

/* erf(u)/u, by its Maclaurin series for small u */
static double or_erf_over_u(double u)
{
    if (u < 0.05) {
        double u2 = u * u;
        /* 2/sqrt(pi) * sum_n (-1)^n u^{2n} / (n! (2n+1)) */
        double s = 1.0 - u2 / 3.0 + u2 * u2 / 10.0 - u2 * u2 * u2 / 42.0 + u2 * u2 * u2 * u2 / 216.0;
        return 2.0 / sqrt(OR_PI) * s;
    }
    return erf(u) / u;
}

/* (erf(u) - 2u/sqrt(pi) exp(-u^2)) / u^3, by its series for small u */
static double or_phi2(double u)
{
    if (u < 0.2) {
        double u2 = u * u, term = 0.0, p = 1.0, fact = 1.0;
        for (int n = 1; n <= 10; ++n) {
            fact *= n;
            double c = (double)(2 * n) / (fact * (double)(2 * n + 1));
            term += ((n % 2) ? c : -c) * p;
            p *= u2;
        }
        return 2.0 / sqrt(OR_PI) * term;
    }
    return (erf(u) - 2.0 * u / sqrt(OR_PI) * exp(-u * u)) / (u * u * u);
}

double orc_G1(double r, double s, double alpha)
{
    if (s <= 0.0) return 0.0;
    return erfc(r / (2.0 * sqrt(alpha * s))) / (4.0 * OR_PI * alpha * r);
}

double orc_G2(double r, double s, double alpha)
{
    if (s <= 0.0) return 0.0;
    double u = r / (2.0 * sqrt(alpha * s));
    return ((s + r * r / (2.0 * alpha)) * erfc(u) - r * sqrt(s / (OR_PI * alpha)) * exp(-u * u)) /
           (4.0 * OR_PI * alpha * r);
}

double orc_G2t(double r, double s, double alpha)
{
    if (s <= 0.0) return 0.0;
    double u = r / (2.0 * sqrt(alpha * s));
    double a32 = alpha * sqrt(alpha);
    return r * erfc(u) / (8.0 * OR_PI * alpha * alpha) - sqrt(s) * or_erf_over_u(u) / (8.0 * OR_PI * a32) -
           sqrt(s) * exp(-u * u) / (4.0 * OR_PI * sqrt(OR_PI) * a32);
}

double orc_DL2(double r, double s, double alpha)
{
    if (s <= 0.0) return 0.0;
    double u = r / (2.0 * sqrt(alpha * s));
    return ((s / (r * r) - 1.0 / (2.0 * alpha)) * erfc(u) + sqrt(s / (OR_PI * alpha)) * exp(-u * u) / r) /
           (4.0 * OR_PI * r);
}

double orc_DL2t(double r, double s, double alpha)
{
    if (s <= 0.0 || r <= 0.0) return 0.0;
    double u = r / (2.0 * sqrt(alpha * s));
    return -(0.5 * u * or_phi2(u) + erfc(u)) / (8.0 * OR_PI * alpha * r);
}

/* Time-integrated single-layer kernel for target step k and source step j (1-based) of a
 * uniform grid with step h; d = k - j. */
double orc_time_V(double r, int d, double h, double alpha)
{
    if (d < 0) return 0.0;
    if (d == 0) return orc_G2(r, h, alpha); /* the other three differences are <= 0 */
    double s1 = (d + 1) * h, s2 = d * h, s3 = d * h, s4 = (d - 1) * h;
    double u = r / (2.0 * sqrt(alpha * s1));
    if (u < 1.0)
        return orc_G2t(r, s1, alpha) - orc_G2t(r, s2, alpha) - orc_G2t(r, s3, alpha) + orc_G2t(r, s4, alpha);
    return orc_G2(r, s1, alpha) - orc_G2(r, s2, alpha) - orc_G2(r, s3, alpha) + orc_G2(r, s4, alpha);
}

/* Time-integrated double-layer factor: the entry integrand is (x - y).n_y * orc_time_K. */
double orc_time_K(double r, int d, double h, double alpha)
{
    if (d < 0) return 0.0;
    if (d == 0) return orc_DL2(r, h, alpha);
    double s1 = (d + 1) * h, s2 = d * h, s3 = d * h, s4 = (d - 1) * h;
    double u = r / (2.0 * sqrt(alpha * s1));
    if (u < 1.0)
        return orc_DL2t(r, s1, alpha) - orc_DL2t(r, s2, alpha) - orc_DL2t(r, s3, alpha) + orc_DL2t(r, s4, alpha);
    return orc_DL2(r, s1, alpha) - orc_DL2(r, s2, alpha) - orc_DL2(r, s3, alpha) + orc_DL2(r, s4, alpha);
}

/* ======================================================================================
 * 2. Quadrature: Gauss-Legendre on [0,1]; collapsed rule on the reference triangle
 *    T = {(s1, s2): 0 <= s2 <= s1 <= 1}, mapped to a triangle (P0, P1, P2) by
 *    chi(s) = P0 + s1 (P1 - P0) + s2 (P2 - P1)   (barycentric (1 - s1, s1 - s2, s2)).
 * ====================================================================================== */

int orc_gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1 || n > OR_MAXQ) return -1;
    for (int i = 0; i < n; ++i) {
        /* Newton iteration on the Legendre polynomial P_n on [-1, 1] */
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp); /* = (2/((1-z^2) P'^2)) / 2 */
    }
    return 0;
}

typedef struct { int n; double s1[OR_MAXQ * OR_MAXQ], s2[OR_MAXQ * OR_MAXQ], w[OR_MAXQ * OR_MAXQ]; } or_trirule;

/* collapsed rule: s1 = u, s2 = u v, weight w_u w_v u; sum of weights = 1/2 = |T| */
static void or_make_trirule(int n, or_trirule *R)
{
    double x[OR_MAXQ], w[OR_MAXQ];
    orc_gauss_legendre01(n, x, w);
    R->n = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            R->s1[R->n] = x[i];
            R->s2[R->n] = x[i] * x[j];
            R->w[R->n] = w[i] * w[j] * x[i];
            R->n++;
        }
}

static void or_chi(const double *P0, const double *P1, const double *P2, double s1, double s2, double *out)
{
    for (int c = 0; c < 3; ++c) out[c] = P0[c] + s1 * (P1[c] - P0[c]) + s2 * (P2[c] - P1[c]);
}

static double or_tri_area(const double *P0, const double *P1, const double *P2)
{
    double a[3], b[3];
    for (int c = 0; c < 3; ++c) { a[c] = P1[c] - P0[c]; b[c] = P2[c] - P0[c]; }
    double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

static void or_tri_normal(const double *P0, const double *P1, const double *P2, double *n)
{
    double a[3], b[3];
    for (int c = 0; c < 3; ++c) { a[c] = P1[c] - P0[c]; b[c] = P2[c] - P0[c]; }
    n[0] = a[1] * b[2] - a[2] * b[1];
    n[1] = a[2] * b[0] - a[0] * b[2];
    n[2] = a[0] * b[1] - a[1] * b[0];
    double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= l; n[1] /= l; n[2] /= l;
}

/* ======================================================================================
 * 3. Element-pair integrals.  An integrand returns ncomp values at a point pair (x, y);
 *    bary_y are the barycentric coordinates of y with respect to the source triangle's
 *    ORIGINAL vertex order (needed for the p1 trial functions of K_h).
 * ====================================================================================== */

enum { ORK_V = 0, ORK_K = 1, ORK_LAPSL = 2, ORK_LAPDL = 3, ORK_POLY = 4, ORK_VSTEPS = 5 };

typedef struct {
    int kind;
    int d0, nd;        /* time offsets d0 .. d0 + nd - 1 (kinds V, K); step pairs (kind VSTEPS) */
    double h, alpha;
    double ny[3];      /* outward unit normal of the source triangle */
    double poly[4];    /* coefficients of the smooth test kernel */
    const double *tb;  /* kind VSTEPS: [nd][4] target step (t0, t1] and source step (t0, t1] */
} or_kernel;

double orc_time_V_steps(double r, double tk0, double tk1, double tj0, double tj1, double alpha);

static int or_ncomp(const or_kernel *k)
{
    switch (k->kind) {
    case ORK_V: return k->nd;
    case ORK_VSTEPS: return k->nd;
    case ORK_K: return 3 * k->nd;
    default: return 1;
    }
}

static void or_eval(const or_kernel *k, const double *x, const double *y, const double *by, double *out)
{
    double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    switch (k->kind) {
    case ORK_V:
        for (int i = 0; i < k->nd; ++i) out[i] = orc_time_V(r, k->d0 + i, k->h, k->alpha);
        break;
    case ORK_K: {
        double dn = dx * k->ny[0] + dy * k->ny[1] + dz * k->ny[2];
        for (int i = 0; i < k->nd; ++i) {
            double v = (r > 0.0) ? dn * orc_time_K(r, k->d0 + i, k->h, k->alpha) : 0.0;
            out[3 * i + 0] = v * by[0];
            out[3 * i + 1] = v * by[1];
            out[3 * i + 2] = v * by[2];
        }
        break;
    }
    case ORK_VSTEPS:
        for (int i = 0; i < k->nd; ++i)
            out[i] = orc_time_V_steps(r, k->tb[4 * i], k->tb[4 * i + 1], k->tb[4 * i + 2], k->tb[4 * i + 3], k->alpha);
        break;
    case ORK_LAPSL: out[0] = 1.0 / (4.0 * OR_PI * r); break;
    case ORK_LAPDL: {
        double dn = dx * k->ny[0] + dy * k->ny[1] + dz * k->ny[2];
        out[0] = dn / (4.0 * OR_PI * r * r * r);
        break;
    }
    default: /* smooth test kernel: a polynomial in x and y plus a Gaussian of |x - y| */
        out[0] = k->poly[0] + k->poly[1] * x[0] * y[1] + k->poly[2] * x[2] * x[2] * y[0] * y[1] +
                 k->poly[3] * exp(-r * r);
        break;
    }
}

/* regular pair: product of collapsed rules on both triangles */
static void or_pair_regular(const double *X[3], const double *Y[3], const or_kernel *k, int n, double *acc)
{
    or_trirule *R = (or_trirule *)malloc(sizeof(or_trirule));
    or_make_trirule(n, R);
    int nc = or_ncomp(k);
    double Jx = 2.0 * or_tri_area(X[0], X[1], X[2]), Jy = 2.0 * or_tri_area(Y[0], Y[1], Y[2]);
    double val[3 * 64];
    for (int c = 0; c < nc; ++c) acc[c] = 0.0;
    for (int i = 0; i < R->n; ++i) {
        double x[3];
        or_chi(X[0], X[1], X[2], R->s1[i], R->s2[i], x);
        for (int j = 0; j < R->n; ++j) {
            double y[3], by[3] = {1.0 - R->s1[j], R->s1[j] - R->s2[j], R->s2[j]};
            or_chi(Y[0], Y[1], Y[2], R->s1[j], R->s2[j], y);
            or_eval(k, x, y, by, val);
            double wt = R->w[i] * R->w[j] * Jx * Jy;
            for (int c = 0; c < nc; ++c) acc[c] += wt * val[c];
        }
    }
    free(R);
}

/* Sauter-Schwab regularising transformations (Sauter & Schwab, Boundary Element Methods,
 * Sec. 5.2) on [0,1]^4 with coordinates (xi, e1, e2, e3).  cls = 3: identical triangles,
 * 2: common edge P0-P1 in both parametrisations, 1: common vertex P0 in both.
 * perm_y maps the local (permuted) vertex slots of Y back to its original slots. */
static void or_pair_ss(int cls, const double *X[3], const double *Y[3], const int *perm_y, const or_kernel *k, int n,
                       double *acc)
{
    double gx[OR_MAXQ], gw[OR_MAXQ];
    orc_gauss_legendre01(n, gx, gw);
    int nc = or_ncomp(k);
    double Jx = 2.0 * or_tri_area(X[0], X[1], X[2]), Jy = 2.0 * or_tri_area(Y[0], Y[1], Y[2]);
    double val[3 * 64];
    for (int c = 0; c < nc; ++c) acc[c] = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c)
                for (int d = 0; d < n; ++d) {
                    double xi = gx[a], e1 = gx[b], e2 = gx[c], e3 = gx[d];
                    double w4 = gw[a] * gw[b] * gw[c] * gw[d];
                    double pts[6][4], jac[6];
                    int np = 0;
                    if (cls == 3) {
                        double j = xi * xi * xi * e1 * e1 * e2;
                        double A[6][4] = {
                            {xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1)},
                            {xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2)},
                            {xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
                            {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3)},
                            {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2)},
                            {xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)}};
                        for (int q = 0; q < 6; ++q) {
                            memcpy(pts[q], A[q], sizeof(A[q]));
                            jac[q] = j;
                        }
                        np = 6;
                    } else if (cls == 2) {
                        double j0 = xi * xi * xi * e1 * e1, j1 = j0 * e2;
                        double A[5][4] = {
                            {xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
                            {xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)},
                            {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3},
                            {xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1},
                            {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2}};
                        for (int q = 0; q < 5; ++q) {
                            memcpy(pts[q], A[q], sizeof(A[q]));
                            jac[q] = q == 0 ? j0 : j1;
                        }
                        np = 5;
                    } else {
                        double j = xi * xi * xi * e2;
                        double A[2][4] = {{xi, xi * e1, xi * e2, xi * e2 * e3}, {xi * e2, xi * e2 * e3, xi, xi * e1}};
                        for (int q = 0; q < 2; ++q) {
                            memcpy(pts[q], A[q], sizeof(A[q]));
                            jac[q] = j;
                        }
                        np = 2;
                    }
                    for (int q = 0; q < np; ++q) {
                        double x[3], y[3], byl[3], by[3];
                        or_chi(X[0], X[1], X[2], pts[q][0], pts[q][1], x);
                        or_chi(Y[0], Y[1], Y[2], pts[q][2], pts[q][3], y);
                        byl[0] = 1.0 - pts[q][2];
                        byl[1] = pts[q][2] - pts[q][3];
                        byl[2] = pts[q][3];
                        for (int v = 0; v < 3; ++v) by[perm_y[v]] = byl[v];
                        or_eval(k, x, y, by, val);
                        double wt = w4 * jac[q] * Jx * Jy;
                        for (int cc = 0; cc < nc; ++cc) acc[cc] += wt * val[cc];
                    }
                }
}

/* number of shared vertex ids of two triangles */
static int or_shared(const int *tx, const int *ty)
{
    int s = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += (tx[i] == ty[j]);
    return s;
}

/* Set up the Sauter-Schwab vertex orders of X and Y for a singular pair.
 * On return PX/PY are the vertex positions in the order required by or_pair_ss and perm_y
 * maps the permuted slots of Y to its original slots. */
static int or_ss_order(const double *V, const int *tx, const int *ty, const double *PX[3], const double *PY[3],
                       int *perm_y)
{
    int cls = or_shared(tx, ty);
    int ox[3] = {0, 1, 2}, oy[3] = {0, 1, 2};
    if (cls == 3) {
        for (int i = 0; i < 3; ++i) {
            ox[i] = i;
            for (int j = 0; j < 3; ++j)
                if (ty[j] == tx[i]) oy[i] = j;
        }
    } else if (cls == 2) {
        int n = 0;
        for (int i = 0; i < 3 && n < 2; ++i)
            for (int j = 0; j < 3; ++j)
                if (tx[i] == ty[j]) { ox[n] = i; oy[n] = j; n++; }
        ox[2] = 3 - ox[0] - ox[1];
        oy[2] = 3 - oy[0] - oy[1];
    } else if (cls == 1) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (tx[i] == ty[j]) { ox[0] = i; oy[0] = j; }
        ox[1] = (ox[0] + 1) % 3; ox[2] = (ox[0] + 2) % 3;
        oy[1] = (oy[0] + 1) % 3; oy[2] = (oy[0] + 2) % 3;
    } else {
        return 0;
    }
    for (int i = 0; i < 3; ++i) {
        PX[i] = V + 3 * tx[ox[i]];
        PY[i] = V + 3 * ty[oy[i]];
        perm_y[i] = oy[i];
    }
    return cls;
}

/* All entries of a triangle pair for time offsets d0 .. d0+nd-1 (kind V: nd values, kind K:
 * 3 nd values, one per source vertex in original order).  Singular classes use Sauter-Schwab
 * at d in {0, 1}; everything else uses the regular product rule. */
static void or_pair_entries(const double *V, const int *tx, const int *ty, int kind, int d0, int nd, double h,
                            double alpha, int n_r, int n_s, double *out)
{
    const double *X[3] = {V + 3 * tx[0], V + 3 * tx[1], V + 3 * tx[2]};
    const double *Y[3] = {V + 3 * ty[0], V + 3 * ty[1], V + 3 * ty[2]};
    or_kernel k;
    memset(&k, 0, sizeof(k));
    k.kind = kind;
    k.h = h;
    k.alpha = alpha;
    or_tri_normal(Y[0], Y[1], Y[2], k.ny);
    int per = kind == ORK_K ? 3 : 1;
    int cls = or_shared(tx, ty);
    for (int i = 0; i < nd; ++i) {
        int d = d0 + i;
        double acc[3];
        k.d0 = d;
        k.nd = 1;
        if (cls > 0 && d <= 1) {
            const double *PX[3], *PY[3];
            int perm[3];
            or_ss_order(V, tx, ty, PX, PY, perm);
            or_pair_ss(cls, PX, PY, perm, &k, n_s, acc);
        } else {
            or_pair_regular(X, Y, &k, n_r, acc);
        }
        for (int c = 0; c < per; ++c) out[i * per + c] = acc[c];
    }
}

/* Exposed for the quadrature pins: integrate kernel `kind` over a triangle pair given by
 * explicit coordinates.  cls < 0 selects the class from the shared vertex ids in tx/ty.
 * use_ss = 0 forces the regular rule.  Returns ncomp values in out. */
int orc_pair_integral(const double *V, const int *tx, const int *ty, int kind, int d, double h, double alpha,
                      const double *poly, int n, int use_ss, double *out)
{
    const double *X[3] = {V + 3 * tx[0], V + 3 * tx[1], V + 3 * tx[2]};
    const double *Y[3] = {V + 3 * ty[0], V + 3 * ty[1], V + 3 * ty[2]};
    or_kernel k;
    memset(&k, 0, sizeof(k));
    k.kind = kind;
    k.h = h;
    k.alpha = alpha;
    k.d0 = d;
    k.nd = 1;
    if (poly) memcpy(k.poly, poly, sizeof(k.poly));
    or_tri_normal(Y[0], Y[1], Y[2], k.ny);
    int cls = or_shared(tx, ty);
    if (use_ss && cls > 0) {
        const double *PX[3], *PY[3];
        int perm[3];
        or_ss_order(V, tx, ty, PX, PY, perm);
        or_pair_ss(cls, PX, PY, perm, &k, n, out);
    } else {
        or_pair_regular(X, Y, &k, n, out);
    }
    return or_ncomp(&k);
}

/* ======================================================================================
 * 4. Dense Galerkin blocks (Section 2).  For uniform steps V_h is block lower triangular
 *    (causality) and block Toeplitz: its (k, j) block depends on d = k - j only.
 *    out_V[d][x][y]  = V[(k, x), (k - d, y)]          (d = d0 .. d0+nd-1)
 *    out_K[d][x][i]  = K[(k, x), (k - d, i)]          (node columns, p1 in space)
 *    out_M[x][i]     = M[(k, x), (k, i)] = h |gamma_x| / 3 for i a vertex of gamma_x
 * ====================================================================================== */

int orc_assemble_V(int nv, const double *V, int nt, const int *T, double h, double alpha, int d0, int nd, int n_r,
                   int n_s, double *out, int nthreads)
{
    (void)nv;
    if (nd > 64) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int x = 0; x < nt; ++x) {
        double e[64];
        for (int y = 0; y < nt; ++y) {
            or_pair_entries(V, T + 3 * x, T + 3 * y, ORK_V, d0, nd, h, alpha, n_r, n_s, e);
            for (int i = 0; i < nd; ++i) out[((size_t)i * nt + x) * nt + y] = e[i];
        }
    }
    return 0;
}

/* The rows of the listed target triangles only: out_V[d][i][y] = V[(k, rows[i]), (k - d, y)],
 * d = d0 .. d0+nd-1 (same entries as orc_assemble_V, for a sample of rows). */
int orc_assemble_V_rows(int nv, const double *V, int nt, const int *T, double h, double alpha, int d0, int nd,
                        int n_r, int n_s, const int *rows, int nrows, double *out, int nthreads)
{
    (void)nv;
    if (nd > 64) return -1;
    for (int i = 0; i < nrows; ++i)
        if (rows[i] < 0 || rows[i] >= nt) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for collapse(2) schedule(dynamic, 64)
#endif
    for (int i = 0; i < nrows; ++i) {
        for (int y = 0; y < nt; ++y) {
            double e[64];
            or_pair_entries(V, T + 3 * rows[i], T + 3 * y, ORK_V, d0, nd, h, alpha, n_r, n_s, e);
            for (int j = 0; j < nd; ++j) out[((size_t)j * nrows + i) * nt + y] = e[j];
        }
    }
    return 0;
}

int orc_assemble_K(int nv, const double *V, int nt, const int *T, double h, double alpha, int d0, int nd, int n_r,
                   int n_s, double *out, int nthreads)
{
    if (nd > 64) return -1;
    memset(out, 0, sizeof(double) * (size_t)nd * nt * nv);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int x = 0; x < nt; ++x) {
        double e[3 * 64];
        for (int y = 0; y < nt; ++y) {
            or_pair_entries(V, T + 3 * x, T + 3 * y, ORK_K, d0, nd, h, alpha, n_r, n_s, e);
            for (int i = 0; i < nd; ++i)
                for (int v = 0; v < 3; ++v) out[((size_t)i * nt + x) * nv + T[3 * y + v]] += e[3 * i + v];
        }
    }
    return 0;
}

int orc_assemble_M(int nv, const double *V, int nt, const int *T, double h, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)nt * nv);
    for (int x = 0; x < nt; ++x) {
        const int *t = T + 3 * x;
        double a = or_tri_area(V + 3 * t[0], V + 3 * t[1], V + 3 * t[2]);
        for (int v = 0; v < 3; ++v) out[(size_t)x * nv + t[v]] += h * a / 3.0;
    }
    return 0;
}

/* ======================================================================================
 * 5. Expansion ingredients (Section 3.1)
 * ====================================================================================== */

/* Chebyshev nodes of order m+1 on [-1,1]: roots of T_{m+1}, indexed 0..m */
static double or_cheb_node(int k, int m) { return cos((2.0 * k + 1.0) * OR_PI / (2.0 * m + 2.0)); }

/* T_k(x) = cos(k arccos x), evaluated by the three-term recurrence (valid for any x) */
static double or_cheb_T(int k, double x)
{
    if (k == 0) return 1.0;
    double t0 = 1.0, t1 = x;
    for (int i = 2; i <= k; ++i) {
        double t2 = 2.0 * x * t1 - t0;
        t0 = t1;
        t1 = t2;
    }
    return t1;
}

/* T_k'(x) = k U_{k-1}(x) */
static double or_cheb_dT(int k, double x)
{
    if (k == 0) return 0.0;
    double u0 = 1.0, u1 = 2.0 * x;
    if (k == 1) return 1.0;
    for (int i = 2; i <= k - 1; ++i) {
        double u2 = 2.0 * x * u1 - u0;
        u0 = u1;
        u1 = u2;
    }
    return k * u1;
}

/* Lagrange polynomial L_{I,b}(t) of the interval I = (lo, hi] on the transformed Chebyshev nodes */
static double or_lagrange(int b, int m, double lo, double hi, double t)
{
    double c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo), xb = c + hw * or_cheb_node(b, m), v = 1.0;
    for (int k = 0; k <= m; ++k)
        if (k != b) {
            double xk = c + hw * or_cheb_node(k, m);
            v *= (t - xk) / (xb - xk);
        }
    return v;
}

static double or_lam(int k) { return k == 0 ? 1.0 : 2.0; }

/* 1D expansion coefficient E_{k,l}(r, d) of Eq. exp_coeffs_1d */
static double or_E1(int k, int l, double r, double dab, int mx)
{
    double s = 0.0;
    for (int n = 0; n <= mx; ++n)
        for (int m = 0; m <= mx; ++m) {
            double xn = or_cheb_node(n, mx), xm = or_cheb_node(m, mx), z = r + xn - xm;
            s += exp(-z * z / dab) * or_cheb_T(l, xn) * or_cheb_T(k, xm);
        }
    return or_lam(k) * or_lam(l) / ((mx + 1.0) * (mx + 1.0)) * s;
}

/* ======================================================================================
 * 6. The 4D box cluster tree (Section 3.2, Alg. 1) for a tensor mesh with uniform steps.
 *    Readings: root = the cube around the vertices' bounding box (centre = box midpoint,
 *    half-size = largest half extent); a space-time element belongs to the box that holds its
 *    centre, half-open (a, b] per direction (clamped at the root's faces); temporal leaves hold
 *    leaf_steps steps (uniform depth p); the level-l -> l+1 refinement is temporal when
 *    hx_l^2 <= c_st * 4 alpha * ht_{l+1} (Eq. rel_h_t_h_x, unpadded hx) or when no box of level
 *    l holds more than leaf_tris triangles, otherwise space-time; padding per level is the
 *    largest overshoot of a triangle over its (unpadded) box, made monotone in the level.
 * ====================================================================================== */

typedef struct {
    int nv, nt;
    const double *V;
    const int *T;
    double Tend;
    int Et;
    double alpha;
    int m_t, m_x;
    double c_st;
    int n_tr;
    double eps_tr;
    int leaf_steps, leaf_tris;
    int n_r, n_s;
} orc_problem;

typedef struct {
    int p;                 /* leaf level */
    int lx[OR_MAXL];       /* spatial refinements of level l */
    double H, corner[3];   /* root cube: (corner, corner + 2H] */
    double pad[OR_MAXL];
    int nbox[OR_MAXL];     /* non-empty spatial boxes of level l */
    int *bgrid[OR_MAXL];   /* [nbox][3] grid multi-indices, lexicographic */
    int *lookup[OR_MAXL];  /* [G^3] -> box index or -1 */
    int *tbox[OR_MAXL];    /* [nt] box index of each triangle */
    int ntr_far[OR_MAXL];  /* interaction-area radius for M2L at level l */
    int ntr_near;          /* interaction-area radius of the leaf nearfield */
} or_tree;

static int or_cell(double z, double corner, double w, int G)
{
    double s = (z - corner) / w;
    int i = (int)ceil(s) - 1;
    if (i < 0) i = 0;
    if (i > G - 1) i = G - 1;
    return i;
}

static int or_ntr(const orc_problem *P, double hx, double pad, double dmax, int G)
{
    if (P->n_tr >= 0) return P->n_tr;
    for (int n = 1; n < G; ++n) {
        double s = n * 2.0 * hx - 2.0 * pad;
        if (s < 0) s = 0;
        if (exp(-s * s / (4.0 * P->alpha * dmax)) <= P->eps_tr) return n;
    }
    return G > 1 ? G - 1 : 0;
}

static void or_tree_free(or_tree *t)
{
    for (int l = 0; l <= t->p; ++l) {
        free(t->bgrid[l]);
        free(t->lookup[l]);
        free(t->tbox[l]);
    }
}

static int or_tree_build(const orc_problem *P, or_tree *t)
{
    memset(t, 0, sizeof(*t));
    if (P->Et % P->leaf_steps) return -1;
    int nleaf = P->Et / P->leaf_steps, p = 0;
    while ((1 << p) < nleaf) p++;
    if ((1 << p) != nleaf || p >= OR_MAXL) return -1;
    t->p = p;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < P->nv; ++i)
        for (int c = 0; c < 3; ++c) {
            if (P->V[3 * i + c] < lo[c]) lo[c] = P->V[3 * i + c];
            if (P->V[3 * i + c] > hi[c]) hi[c] = P->V[3 * i + c];
        }
    t->H = 0.0;
    for (int c = 0; c < 3; ++c)
        if (0.5 * (hi[c] - lo[c]) > t->H) t->H = 0.5 * (hi[c] - lo[c]);
    for (int c = 0; c < 3; ++c) t->corner[c] = 0.5 * (lo[c] + hi[c]) - t->H;

    double *cent = (double *)malloc(sizeof(double) * 3 * P->nt);
    for (int x = 0; x < P->nt; ++x)
        for (int c = 0; c < 3; ++c)
            cent[3 * x + c] = ((P->V[3 * P->T[3 * x] + c] + P->V[3 * P->T[3 * x + 1] + c]) + P->V[3 * P->T[3 * x + 2] + c]) / 3.0;

    /* initial spatial refinements so that the root satisfies Eq. rel_h_t_h_x (Alg. 1, line 1) */
    int lx0 = 0;
    while (1) {
        double hx = t->H / (double)(1 << lx0);
        if (hx * hx <= P->c_st * 4.0 * P->alpha * (P->Tend / 2.0) || lx0 > 20) break;
        lx0++;
    }
    t->lx[0] = lx0;
    for (int l = 0; l <= p; ++l) {
        if (l > 0) {
            double ht = P->Tend / (double)(1 << (l + 1)); /* half-size of the children's intervals */
            double hx = t->H / (double)(1 << t->lx[l - 1]);
            int maxcnt = 0;
            {
                int G = 1 << t->lx[l - 1];
                int *cnt = (int *)calloc((size_t)G * G * G, sizeof(int));
                for (int x = 0; x < P->nt; ++x) {
                    double w = 2.0 * t->H / G;
                    int i = or_cell(cent[3 * x], t->corner[0], w, G), j = or_cell(cent[3 * x + 1], t->corner[1], w, G),
                        k = or_cell(cent[3 * x + 2], t->corner[2], w, G);
                    int c = ++cnt[((size_t)i * G + j) * G + k];
                    if (c > maxcnt) maxcnt = c;
                }
                free(cnt);
            }
            if (hx * hx <= P->c_st * 4.0 * P->alpha * ht || maxcnt <= P->leaf_tris)
                t->lx[l] = t->lx[l - 1];
            else
                t->lx[l] = t->lx[l - 1] + 1;
        }
        int G = 1 << t->lx[l];
        double w = 2.0 * t->H / G;
        t->lookup[l] = (int *)malloc(sizeof(int) * (size_t)G * G * G);
        for (size_t i = 0; i < (size_t)G * G * G; ++i) t->lookup[l][i] = -1;
        int *cell = (int *)malloc(sizeof(int) * 3 * P->nt);
        for (int x = 0; x < P->nt; ++x) {
            for (int c = 0; c < 3; ++c) cell[3 * x + c] = or_cell(cent[3 * x + c], t->corner[c], w, G);
            t->lookup[l][((size_t)cell[3 * x] * G + cell[3 * x + 1]) * G + cell[3 * x + 2]] = 0;
        }
        int nb = 0;
        for (size_t i = 0; i < (size_t)G * G * G; ++i)
            if (t->lookup[l][i] == 0) t->lookup[l][i] = nb++;
        t->nbox[l] = nb;
        t->bgrid[l] = (int *)malloc(sizeof(int) * 3 * (nb > 0 ? nb : 1));
        for (int i = 0; i < G; ++i)
            for (int j = 0; j < G; ++j)
                for (int k = 0; k < G; ++k) {
                    int b = t->lookup[l][((size_t)i * G + j) * G + k];
                    if (b >= 0) { t->bgrid[l][3 * b] = i; t->bgrid[l][3 * b + 1] = j; t->bgrid[l][3 * b + 2] = k; }
                }
        t->tbox[l] = (int *)malloc(sizeof(int) * P->nt);
        for (int x = 0; x < P->nt; ++x)
            t->tbox[l][x] = t->lookup[l][((size_t)cell[3 * x] * G + cell[3 * x + 1]) * G + cell[3 * x + 2]];
        /* overshoot of the triangles over their unpadded boxes */
        double ov = 0.0;
        for (int x = 0; x < P->nt; ++x)
            for (int v = 0; v < 3; ++v)
                for (int c = 0; c < 3; ++c) {
                    double z = P->V[3 * P->T[3 * x + v] + c];
                    double blo = t->corner[c] + cell[3 * x + c] * w, bhi = blo + w;
                    if (blo - z > ov) ov = blo - z;
                    if (z - bhi > ov) ov = z - bhi;
                }
        t->pad[l] = ov;
        free(cell);
    }
    for (int l = p - 1; l >= 0; --l)
        if (t->pad[l + 1] > t->pad[l]) t->pad[l] = t->pad[l + 1];
    for (int l = 0; l <= p; ++l) {
        int G = 1 << t->lx[l];
        double hx = t->H / G;
        double ht = P->Tend / (double)(1 << (l + 1));
        t->ntr_far[l] = or_ntr(P, hx, t->pad[l], 8.0 * ht, G);
    }
    {
        int G = 1 << t->lx[p];
        double hx = t->H / G, hstep = P->Tend / P->Et;
        t->ntr_near = or_ntr(P, hx, t->pad[p], 2.0 * P->leaf_steps * hstep, G);
    }
    free(cent);
    return 0;
}

/* grid distance (Eq. 03:Iarea) */
static int or_gdist(const int *a, const int *b)
{
    int d = 0;
    for (int c = 0; c < 3; ++c) {
        int e = abs(a[c] - b[c]);
        if (e > d) d = e;
    }
    return d;
}

/* temporal interaction list of interval k (Eq. 03:ILtemp); returns count, fills js */
static int or_interaction_list(int k, int *js)
{
    if (k < 2) return 0;
    if (k % 2 == 0) { js[0] = k - 2; return 1; }
    js[0] = k - 3;
    js[1] = k - 2;
    return 2;
}

/* temporal nearfield of interval k at the (uniform) leaf level (Eq. 03:ILtemp); the term
 * N(parent) /\ leaves is empty because all leaves sit on the same level */
static int or_nearfield_list(int k, int *js)
{
    if (k == 0) { js[0] = 0; return 1; }
    js[0] = k - 1;
    js[1] = k;
    return 2;
}

/* exposed for the tree pins: per level lx, nbox, pad, ntr_far; plus p and ntr_near */
int orc_tree_info(const orc_problem *P, int *p_out, int *lx, int *nbox, double *pad, int *ntr_far, int *ntr_near,
                  double *root /*[4]: corner xyz, H*/)
{
    or_tree t;
    if (or_tree_build(P, &t)) return -1;
    *p_out = t.p;
    for (int l = 0; l <= t.p; ++l) {
        lx[l] = t.lx[l];
        nbox[l] = t.nbox[l];
        pad[l] = t.pad[l];
        ntr_far[l] = t.ntr_far[l];
    }
    *ntr_near = t.ntr_near;
    root[0] = t.corner[0]; root[1] = t.corner[1]; root[2] = t.corner[2]; root[3] = t.H;
    or_tree_free(&t);
    return 0;
}

/* ======================================================================================
 * 7. The space-time FMM (Section 3.4, Alg. 2) for f = V_h w (op 0) or f = K_h g (op 1).
 *    parts: bit 0 = nearfield, bit 1 = farfield.  targets: list of triangles whose rows
 *    (all time steps) are computed, or NULL for all.  f is [Et][nt]; rows not computed
 *    are set to zero.
 * ====================================================================================== */

typedef struct {
    int nk;
    int (*k)[3];
    int *lookup; /* [(m+1)^3] -> index or -1 */
} or_mi;

static void or_mi_make(int m, or_mi *mi)
{
    int n = 0;
    mi->lookup = (int *)malloc(sizeof(int) * (m + 1) * (m + 1) * (m + 1));
    for (int i = 0; i < (m + 1) * (m + 1) * (m + 1); ++i) mi->lookup[i] = -1;
    for (int a = 0; a <= m; ++a)
        for (int b = 0; a + b <= m; ++b)
            for (int c = 0; a + b + c <= m; ++c) n++;
    mi->k = malloc(sizeof(int[3]) * n);
    n = 0;
    for (int a = 0; a <= m; ++a)
        for (int b = 0; a + b <= m; ++b)
            for (int c = 0; a + b + c <= m; ++c) {
                mi->k[n][0] = a; mi->k[n][1] = b; mi->k[n][2] = c;
                mi->lookup[(a * (m + 1) + b) * (m + 1) + c] = n;
                n++;
            }
    mi->nk = n;
}

typedef struct {
    const orc_problem *P;
    or_tree t;
    or_mi mi;
    int na;
    double h;
} or_fmm;

/* spatial box of level l with grid index g: padded centre and half-size */
static void or_box_geom(const or_fmm *F, int l, const int *g, double *cen, double *hp)
{
    int G = 1 << F->t.lx[l];
    double hx = F->t.H / G;
    for (int c = 0; c < 3; ++c) cen[c] = F->t.corner[c] + (2.0 * g[c] + 1.0) * hx;
    *hp = hx + F->t.pad[l];
}

/* q^(t)_{ac,ap}(I_c, I_p) = L_{I_p,ap}(xi_{I_c,ac}), I_c the lower (c = 0) or upper half of I_p */
static double or_qt(int c, int ac, int ap, int m)
{
    double lo = -1.0, hi = 1.0;
    double clo = c == 0 ? -1.0 : 0.0, chi = c == 0 ? 0.0 : 1.0;
    double xc = 0.5 * (clo + chi) + 0.5 * (chi - clo) * or_cheb_node(ac, m);
    return or_lagrange(ap, m, lo, hi, xc);
}

/* q^(x)_{kap,nu}(X_c, X_p) in one direction for child/parent padded intervals */
static double or_qx(int kap, int nu, double cc, double hc, double cp, double hp, int m)
{
    double s = 0.0;
    for (int n = 0; n <= m; ++n) {
        double xn = or_cheb_node(n, m), z = cc + hc * xn;
        s += or_cheb_T(nu, (z - cp) / hp) * or_cheb_T(kap, xn);
    }
    return or_lam(kap) / (m + 1.0) * s;
}

/* spatial integral of T_{Y,kappa} over a triangle (or of alpha n.grad T_{Y,kappa} phi_v) */
static void or_space_moments(const or_fmm *F, int x, const double *cen, double hp, int op, double *out /* nk or 3 nk */)
{
    const orc_problem *P = F->P;
    const int *t = P->T + 3 * x;
    const double *A = P->V + 3 * t[0], *B = P->V + 3 * t[1], *C = P->V + 3 * t[2];
    or_trirule *R = (or_trirule *)malloc(sizeof(or_trirule));
    or_make_trirule(P->m_x / 2 + 2, R);
    double J = 2.0 * or_tri_area(A, B, C), n[3];
    or_tri_normal(A, B, C, n);
    int nk = F->mi.nk;
    for (int i = 0; i < (op ? 3 * nk : nk); ++i) out[i] = 0.0;
    for (int q = 0; q < R->n; ++q) {
        double y[3], yh[3];
        or_chi(A, B, C, R->s1[q], R->s2[q], y);
        for (int c = 0; c < 3; ++c) yh[c] = (y[c] - cen[c]) / hp;
        double by[3] = {1.0 - R->s1[q], R->s1[q] - R->s2[q], R->s2[q]};
        for (int i = 0; i < nk; ++i) {
            const int *k = F->mi.k[i];
            double T0 = or_cheb_T(k[0], yh[0]), T1 = or_cheb_T(k[1], yh[1]), T2 = or_cheb_T(k[2], yh[2]);
            if (!op) {
                out[i] += R->w[q] * J * T0 * T1 * T2;
            } else {
                double g0 = or_cheb_dT(k[0], yh[0]) * T1 * T2 / hp, g1 = T0 * or_cheb_dT(k[1], yh[1]) * T2 / hp,
                       g2 = T0 * T1 * or_cheb_dT(k[2], yh[2]) / hp;
                double dn = P->alpha * (n[0] * g0 + n[1] * g1 + n[2] * g2);
                for (int v = 0; v < 3; ++v) out[3 * i + v] += R->w[q] * J * dn * by[v];
            }
        }
    }
    free(R);
}

/* int over step (lo, lo+h] of L_{J,a}, J = (jlo, jhi], by Gauss-Legendre (exact) */
static double or_time_moment(int a, int m, double jlo, double jhi, double lo, double h)
{
    double gx[OR_MAXQ], gw[OR_MAXQ];
    int n = m + 1;
    orc_gauss_legendre01(n, gx, gw);
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += gw[i] * h * or_lagrange(a, m, jlo, jhi, lo + h * gx[i]);
    return s;
}

#define OR_MU(F, l, k, b, a, i) (((((size_t)(k) * (F)->t.nbox[l] + (b)) * (F)->na + (a)) * (F)->mi.nk) + (i))

int orc_pfmm_apply(const orc_problem *P, int op, const double *xin, double *f, const int *targets, int ntargets,
                   int parts, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    or_fmm F;
    F.P = P;
    if (or_tree_build(P, &F.t)) return -1;
    or_mi_make(P->m_x, &F.mi);
    F.na = P->m_t + 1;
    F.h = P->Tend / P->Et;
    const int p = F.t.p, na = F.na, nk = F.mi.nk, mt = P->m_t, mx = P->m_x, nt = P->nt, Et = P->Et;
    const int ncol = op ? P->nv : nt;
    memset(f, 0, sizeof(double) * (size_t)Et * nt);

    unsigned char *is_tgt = (unsigned char *)calloc(nt, 1);
    if (targets && ntargets >= 0)
        for (int i = 0; i < ntargets; ++i) is_tgt[targets[i]] = 1;
    else
        memset(is_tgt, 1, nt);
    /* target boxes per level: boxes holding a target triangle */
    unsigned char *tbx[OR_MAXL];
    for (int l = 0; l <= p; ++l) {
        tbx[l] = (unsigned char *)calloc(F.t.nbox[l] > 0 ? F.t.nbox[l] : 1, 1);
        for (int x = 0; x < nt; ++x)
            if (is_tgt[x]) tbx[l][F.t.tbox[l][x]] = 1;
    }

    if (parts & 2) {
        double *mu[OR_MAXL] = {0}, *lam[OR_MAXL] = {0};
        for (int l = 2; l <= p; ++l) {
            size_t n = (size_t)(1 << l) * F.t.nbox[l] * na * nk;
            mu[l] = (double *)calloc(n, sizeof(double));
            lam[l] = (double *)calloc(n, sizeof(double));
        }
        if (p >= 2) {
            /* --- S2M at the leaves (Eq. s2m) --- */
            const int ls = P->leaf_steps;
            double *smom = (double *)malloc(sizeof(double) * (size_t)nt * nk * (op ? 3 : 1));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
            for (int x = 0; x < nt; ++x) {
                int b = F.t.tbox[p][x];
                double cen[3], hp;
                or_box_geom(&F, p, F.t.bgrid[p] + 3 * b, cen, &hp);
                or_space_moments(&F, x, cen, hp, op, smom + (size_t)x * nk * (op ? 3 : 1));
            }
            double *tmom = (double *)malloc(sizeof(double) * ls * na); /* identical for all leaves */
            for (int s = 0; s < ls; ++s)
                for (int a = 0; a < na; ++a) tmom[s * na + a] = or_time_moment(a, mt, 0.0, ls * F.h, s * F.h, F.h);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int k = 0; k < (1 << p); ++k)
                for (int x = 0; x < nt; ++x) {
                    int b = F.t.tbox[p][x];
                    for (int s = 0; s < ls; ++s) {
                        int jt = k * ls + s;
                        for (int a = 0; a < na; ++a)
                            for (int i = 0; i < nk; ++i) {
                                double v;
                                if (!op) {
                                    v = xin[(size_t)jt * ncol + x] * smom[(size_t)x * nk + i];
                                } else {
                                    v = 0.0;
                                    for (int q = 0; q < 3; ++q)
                                        v += xin[(size_t)jt * ncol + P->T[3 * x + q]] * smom[((size_t)x * nk + i) * 3 + q];
                                }
                                mu[p][OR_MU(&F, p, k, b, a, i)] += tmom[s * na + a] * v;
                            }
                    }
                }
            free(tmom);
            free(smom);

            /* --- M2M for levels p-1 .. 2 (Eq. temp_m2m, st_m2m) --- */
            for (int l = p - 1; l >= 2; --l) {
                int st = F.t.lx[l + 1] != F.t.lx[l];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
                for (int bp = 0; bp < F.t.nbox[l]; ++bp) {
                    const int *gp = F.t.bgrid[l] + 3 * bp;
                    double cp[3], hp;
                    or_box_geom(&F, l, gp, cp, &hp);
                    for (int bc = 0; bc < F.t.nbox[l + 1]; ++bc) {
                        const int *gc = F.t.bgrid[l + 1] + 3 * bc;
                        int child = st ? ((gc[0] >> 1) == gp[0] && (gc[1] >> 1) == gp[1] && (gc[2] >> 1) == gp[2])
                                       : (gc[0] == gp[0] && gc[1] == gp[1] && gc[2] == gp[2]);
                        if (!child) continue;
                        double cc[3], hc;
                        or_box_geom(&F, l + 1, gc, cc, &hc);
                        /* 1D factors q^(x)_{kap_j, nu_j}(X_c,j, X_p,j) of this child, per direction */
                        double q1[3][OR_MAXQ][OR_MAXQ];
                        if (st)
                            for (int d = 0; d < 3; ++d)
                                for (int a1 = 0; a1 <= mx; ++a1)
                                    for (int n1 = 0; n1 <= mx; ++n1) q1[d][a1][n1] = or_qx(a1, n1, cc[d], hc, cp[d], hp, mx);
                        for (int kp = 0; kp < (1 << l); ++kp)
                            for (int c = 0; c < 2; ++c) {
                                int kc = 2 * kp + c;
                                for (int ap = 0; ap < na; ++ap)
                                    for (int ac = 0; ac < na; ++ac) {
                                        double qt = or_qt(c, ac, ap, mt);
                                        for (int iv = 0; iv < nk; ++iv) {
                                            const int *nu = F.mi.k[iv];
                                            if (!st) {
                                                mu[l][OR_MU(&F, l, kp, bp, ap, iv)] += qt * mu[l + 1][OR_MU(&F, l + 1, kc, bc, ac, iv)];
                                                continue;
                                            }
                                            double acc = 0.0; /* sum over kappa <= nu (componentwise) */
                                            for (int k0 = 0; k0 <= nu[0]; ++k0)
                                                for (int k1 = 0; k1 <= nu[1]; ++k1)
                                                    for (int k2 = 0; k2 <= nu[2]; ++k2) {
                                                        int ik = F.mi.lookup[(k0 * (mx + 1) + k1) * (mx + 1) + k2];
                                                        acc += q1[0][k0][nu[0]] * q1[1][k1][nu[1]] * q1[2][k2][nu[2]] *
                                                               mu[l + 1][OR_MU(&F, l + 1, kc, bc, ac, ik)];
                                                    }
                                            mu[l][OR_MU(&F, l, kp, bp, ap, iv)] += qt * acc;
                                        }
                                    }
                            }
                    }
                }
            }

            /* --- M2L for all levels >= 2 (Eq. m2l with Eq. exp_coeffs_3d / exp_coeffs_1d) --- */
            for (int l = 2; l <= p; ++l) {
                int G = 1 << F.t.lx[l];
                double hx = F.t.H / G, hp = hx + F.t.pad[l];
                double L = P->Tend / (double)(1 << l), ht = 0.5 * L;
                int no = 2 * G - 1, m1 = mx + 1;
                /* 1D coefficients for every (Delta in {2,3}, a, b, grid offset) of this level */
                double *E1 = (double *)malloc(sizeof(double) * 2 * na * na * no * m1 * m1);
                double *pref = (double *)malloc(sizeof(double) * 2 * na * na);
                for (int D = 2; D <= 3; ++D)
                    for (int a = 0; a < na; ++a)
                        for (int b = 0; b < na; ++b) {
                            /* xi_{I,b} - xi_{J,a} with J = I - D intervals */
                            double dt = D * L + ht * (or_cheb_node(b, mt) - or_cheb_node(a, mt));
                            double dab = 4.0 * P->alpha * dt / (hp * hp);
                            pref[((D - 2) * na + a) * na + b] = pow(4.0 * OR_PI * P->alpha * dt, -1.5);
                            for (int o = 0; o < no; ++o) {
                                double r = 2.0 * hx * (o - (G - 1)) / hp;
                                for (int kk = 0; kk <= mx; ++kk)
                                    for (int ll = 0; ll + kk <= mx; ++ll)
                                        E1[(((((size_t)(D - 2) * na + a) * na + b) * no + o) * m1 + kk) * m1 + ll] =
                                            or_E1(kk, ll, r, dab, mx);
                            }
                        }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
#endif
                for (int k = 0; k < (1 << l); ++k)
                    for (int bt = 0; bt < F.t.nbox[l]; ++bt) {
                        if (!tbx[l][bt]) continue;
                        int js[2], nj = or_interaction_list(k, js);
                        const int *gt = F.t.bgrid[l] + 3 * bt;
                        for (int jj = 0; jj < nj; ++jj) {
                            int D = k - js[jj];
                            for (int bs = 0; bs < F.t.nbox[l]; ++bs) {
                                const int *gs = F.t.bgrid[l] + 3 * bs;
                                if (or_gdist(gt, gs) > F.t.ntr_far[l]) continue;
                                int o[3] = {gt[0] - gs[0] + G - 1, gt[1] - gs[1] + G - 1, gt[2] - gs[2] + G - 1};
                                for (int b = 0; b < na; ++b)
                                    for (int iv = 0; iv < nk; ++iv) {
                                        const int *nu = F.mi.k[iv];
                                        double acc = 0.0;
                                        for (int a = 0; a < na; ++a) {
                                            double pf = pref[((D - 2) * na + a) * na + b];
                                            size_t e0 = ((((size_t)(D - 2) * na + a) * na + b) * no);
                                            for (int ik = 0; ik < nk; ++ik) {
                                                const int *ka = F.mi.k[ik];
                                                if (ka[0] + ka[1] + ka[2] + nu[0] + nu[1] + nu[2] > mx) continue;
                                                double E = pf;
                                                for (int d = 0; d < 3; ++d) E *= E1[((e0 + o[d]) * m1 + ka[d]) * m1 + nu[d]];
                                                acc += E * mu[l][OR_MU(&F, l, js[jj], bs, a, ik)];
                                            }
                                        }
                                        lam[l][OR_MU(&F, l, k, bt, b, iv)] += acc;
                                    }
                            }
                        }
                    }
                free(E1);
                free(pref);
            }

            /* --- L2L for levels 3 .. p (transposes of the M2M operations) --- */
            for (int l = 3; l <= p; ++l) {
                int st = F.t.lx[l] != F.t.lx[l - 1];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
                for (int bc = 0; bc < F.t.nbox[l]; ++bc) {
                    if (!tbx[l][bc]) continue;
                    const int *gc = F.t.bgrid[l] + 3 * bc;
                    int gpi[3] = {st ? gc[0] >> 1 : gc[0], st ? gc[1] >> 1 : gc[1], st ? gc[2] >> 1 : gc[2]};
                    int G = 1 << F.t.lx[l - 1];
                    int bp = F.t.lookup[l - 1][((size_t)gpi[0] * G + gpi[1]) * G + gpi[2]];
                    double cc[3], hc, cp[3], hp;
                    or_box_geom(&F, l, gc, cc, &hc);
                    or_box_geom(&F, l - 1, gpi, cp, &hp);
                    double q1[3][OR_MAXQ][OR_MAXQ];
                    if (st)
                        for (int d = 0; d < 3; ++d)
                            for (int a1 = 0; a1 <= mx; ++a1)
                                for (int n1 = 0; n1 <= mx; ++n1) q1[d][a1][n1] = or_qx(a1, n1, cc[d], hc, cp[d], hp, mx);
                    for (int kc = 0; kc < (1 << l); ++kc) {
                        int kp = kc / 2, c = kc % 2;
                        for (int bcI = 0; bcI < na; ++bcI)
                            for (int ik = 0; ik < nk; ++ik) {
                                const int *ka = F.mi.k[ik];
                                double acc = 0.0;
                                for (int bpI = 0; bpI < na; ++bpI) {
                                    double qt = or_qt(c, bcI, bpI, mt);
                                    if (!st) {
                                        acc += qt * lam[l - 1][OR_MU(&F, l - 1, kp, bp, bpI, ik)];
                                        continue;
                                    }
                                    /* sum over nu >= kappa (componentwise) with |nu| <= m_x */
                                    for (int n0 = ka[0]; n0 <= mx; ++n0)
                                        for (int n1 = ka[1]; n0 + n1 <= mx; ++n1)
                                            for (int n2 = ka[2]; n0 + n1 + n2 <= mx; ++n2) {
                                                int iv = F.mi.lookup[(n0 * (mx + 1) + n1) * (mx + 1) + n2];
                                                acc += qt * q1[0][ka[0]][n0] * q1[1][ka[1]][n1] * q1[2][ka[2]][n2] *
                                                       lam[l - 1][OR_MU(&F, l - 1, kp, bp, bpI, iv)];
                                            }
                                }
                                lam[l][OR_MU(&F, l, kc, bc, bcI, ik)] += acc;
                            }
                    }
                }
            }

            /* --- L2T at the leaves (Eq. l2t) --- */
            {
                double *tmom = (double *)malloc(sizeof(double) * ls * na);
                for (int s = 0; s < ls; ++s)
                    for (int b = 0; b < na; ++b) tmom[s * na + b] = or_time_moment(b, mt, 0.0, ls * F.h, s * F.h, F.h);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
                for (int x = 0; x < nt; ++x) {
                    if (!is_tgt[x]) continue;
                    int b = F.t.tbox[p][x];
                    double cen[3], hp, *sm = (double *)malloc(sizeof(double) * nk);
                    or_box_geom(&F, p, F.t.bgrid[p] + 3 * b, cen, &hp);
                    or_space_moments(&F, x, cen, hp, 0, sm);
                    for (int k = 0; k < (1 << p); ++k)
                        for (int s = 0; s < ls; ++s) {
                            double acc = 0.0;
                            for (int bb = 0; bb < na; ++bb)
                                for (int i = 0; i < nk; ++i)
                                    acc += lam[p][OR_MU(&F, p, k, b, bb, i)] * tmom[s * na + bb] * sm[i];
                            f[(size_t)(k * ls + s) * nt + x] += acc;
                        }
                    free(sm);
                }
                free(tmom);
            }
        }
        for (int l = 2; l <= p; ++l) { free(mu[l]); free(lam[l]); }
    }

    if (parts & 1) {
        /* --- nearfield (Eq. eval_sl_nf_block) with entries from Section 2 --- */
        const int ls = P->leaf_steps, G = 1 << F.t.lx[p];
        const int dmaxn = 2 * ls; /* largest step offset inside N(I) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int x = 0; x < nt; ++x) {
            if (!is_tgt[x]) continue;
            int bx = F.t.tbox[p][x];
            const int *gx = F.t.bgrid[p] + 3 * bx;
            double *ent = (double *)malloc(sizeof(double) * 3 * dmaxn);
            for (int y = 0; y < nt; ++y) {
                int by = F.t.tbox[p][y];
                if (or_gdist(gx, F.t.bgrid[p] + 3 * by) > F.t.ntr_near) continue;
                or_pair_entries(P->V, P->T + 3 * x, P->T + 3 * y, op ? ORK_K : ORK_V, 0, dmaxn, F.h, P->alpha, P->n_r,
                                P->n_s, ent);
                for (int kt = 0; kt < Et; ++kt) {
                    int i = kt / ls, js[2], nj = or_nearfield_list(i, js);
                    double acc = 0.0;
                    for (int jj = 0; jj < nj; ++jj)
                        for (int s = 0; s < ls; ++s) {
                            int jt = js[jj] * ls + s, d = kt - jt;
                            if (d < 0) continue;
                            if (!op)
                                acc += ent[d] * xin[(size_t)jt * ncol + y];
                            else
                                for (int v = 0; v < 3; ++v) acc += ent[3 * d + v] * xin[(size_t)jt * ncol + P->T[3 * y + v]];
                        }
                    f[(size_t)kt * nt + x] += acc;
                }
            }
            free(ent);
        }
        (void)G;
    }

    for (int l = 0; l <= p; ++l) free(tbx[l]);
    free(is_tgt);
    free(F.mi.k);
    free(F.mi.lookup);
    or_tree_free(&F.t);
    return 0;
}

/* Exposed for the expansion pins: the 1D coefficient of Eq. exp_coeffs_1d and the
 * interpolation coefficients q^(t), q^(x). */
double orc_E1(int k, int l, double r, double dab, int mx) { return or_E1(k, l, r, dab, mx); }
double orc_qt(int c, int ac, int ap, int m) { return or_qt(c, ac, ap, m); }
double orc_qx(int kap, int nu, double cc, double hc, double cp, double hp, int m) { return or_qx(kap, nu, cc, hc, cp, hp, m); }
double orc_lagrange(int b, int m, double lo, double hi, double t) { return or_lagrange(b, m, lo, hi, t); }
double orc_cheb_node(int k, int m) { return or_cheb_node(k, m); }
int orc_sizeof_problem(void) { return (int)sizeof(orc_problem); }
int orc_interaction_list(int k, int *js) { return or_interaction_list(k, js); }
int orc_nearfield_list(int k, int *js) { return or_nearfield_list(k, js); }

/* Exposed for the S2M / L2T moment pins (Eq. s2m, l2t): the spatial moments of triangle x about
 * the padded box (cen, hp) -- op 0: int_x T_{Y,kappa}; op 1: int_x alpha n.grad T_{Y,kappa} phi_v,
 * three per multi-index -- in the oracle's multi-index order (kappa_1 slowest); returns their
 * count n_kappa.  And the time moment int_(lo, lo+h] L_{J,a} of the interval J = (jlo, jhi]. */
int orc_space_moments(const orc_problem *P, int x, const double *cen, double hp, int op, double *out)
{
    or_fmm F;
    memset(&F, 0, sizeof F);
    F.P = P;
    or_mi_make(P->m_x, &F.mi);
    or_space_moments(&F, x, cen, hp, op, out);
    const int nk = F.mi.nk;
    free(F.mi.k);
    free(F.mi.lookup);
    return nk;
}
double orc_time_moment(int a, int m, double jlo, double jhi, double lo, double h)
{
    return or_time_moment(a, m, jlo, jhi, lo, h);
}

/* ======================================================================================
 * 9. Representation formula (Section 2): for (x, t) in Omega x (0, T)
 *      u(x, t) = (V~ w)(x, t) - (W u)(x, t),
 *    V~ w = int_0^t int_Gamma G(x - y, t - tau) w(y, tau),
 *    W u  = int_0^t int_Gamma alpha dG/dn_y(x - y, t - tau) u(y, tau),
 *    with the discrete data of Eq. 02:linear:system: w_h piecewise constant on the space-time
 *    elements, u = g_h piecewise constant in time and piecewise linear (nodal) in space.
 *    Time: over step j the integrals of G(r, t - tau) and of G(r, t - tau) / (2 (t - tau)) are
 *    differences of the first antiderivatives in s = t - tau,
 *      G1(r, s) = int_0^s G(r, q) dq = erfc(u) / (4 pi alpha r),
 *      H1(r, s) = int_0^s G(r, q) / (2 q) dq = [erfc(u) + 2 u exp(-u^2) / sqrt(pi)] / (4 pi r^3),
 *    u = r / (2 sqrt(alpha s)), taken as 0 for s <= 0 (causality); the double-layer integrand is
 *    (x - y).n_y G / (2 s).  Space: the collapsed Gauss rule with n_r x n_r points per triangle
 *    (the points must not lie on Gamma).
 * ====================================================================================== */

double orc_H1(double r, double s, double alpha)
{
    if (s <= 0.0) return 0.0;
    double u = r / (2.0 * sqrt(alpha * s));
    return (erfc(u) + 2.0 * u * exp(-u * u) / sqrt(OR_PI)) / (4.0 * OR_PI * r * r * r);
}

/* u[p] for the points pts[p] = (x, y, z, t), p < np; w: [Et][nt], g: [Et][nv] or NULL (single-layer
 * potential only) */
int orc_repr_eval(const orc_problem *P, const double *w, const double *g, const double *pts, int np, double *u,
                  int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    or_trirule *R = (or_trirule *)malloc(sizeof(or_trirule));
    if (!R) return -1;
    or_make_trirule(P->n_r, R);
    const double h = P->Tend / P->Et, alpha = P->alpha;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int p = 0; p < np; ++p) {
        const double *x = pts + 4 * p, t = pts[4 * p + 3];
        double acc = 0.0;
        for (int tr = 0; tr < P->nt; ++tr) {
            const int *tv = P->T + 3 * tr;
            const double *P0 = P->V + 3 * tv[0], *P1 = P->V + 3 * tv[1], *P2 = P->V + 3 * tv[2];
            const double jac = 2.0 * or_tri_area(P0, P1, P2);
            double n[3];
            or_tri_normal(P0, P1, P2, n);
            for (int q = 0; q < R->n; ++q) {
                double y[3];
                or_chi(P0, P1, P2, R->s1[q], R->s2[q], y);
                const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
                const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
                const double phi[3] = {1.0 - R->s1[q], R->s1[q] - R->s2[q], R->s2[q]};
                for (int j = 1; j <= P->Et; ++j) {
                    const double s0 = t - (j - 1) * h, s1 = t - j * h;  /* tau = t_{j-1}, t_j */
                    if (s0 <= 0.0) break;
                    const double dG = orc_G1(r, s0, alpha) - orc_G1(r, s1, alpha);
                    double v = w[(size_t)(j - 1) * P->nt + tr] * dG;
                    if (g) {
                        const double dH = orc_H1(r, s0, alpha) - orc_H1(r, s1, alpha);
                        double gy = 0.0;
                        for (int c = 0; c < 3; ++c) gy += g[(size_t)(j - 1) * P->nv + tv[c]] * phi[c];
                        v -= dn * dH * gy;
                    }
                    acc += R->w[q] * jac * v;
                }
            }
        }
        u[p] = acc;
    }
    free(R);
    return 0;
}

/* ======================================================================================
 * 10. General time steps t_0 = 0 < t_1 < ... < t_Et = T (Section 3.2 with Alg. 1 in full,
 *     Section 3.3, Alg. 2; the adaptive direction of Section 6).  Single layer V_h only.
 *     Step j is (t_j, t_{j+1}] (0-based).  No Toeplitz structure: every target / source step
 *     pair is integrated on its own.
 *     Readings (where Section 3.2 leaves the rule open):
 *      - levels: level 0 holds the cells of the grid 2^lx0 (the root refined in space until it
 *        satisfies Eq. rel_h_t_h_x, as for uniform steps) with the interval (0, T]; the refinement
 *        of level l into level l+1 is temporal iff hx_l^2 <= c_st 4 alpha T / 2^(l+2) (the nominal
 *        half-size h_t^(l+1) of Alg. 1), the same for every box of the level;
 *      - RefineCluster: a box Z = X x I is refined iff it holds at least n_max elements, unless
 *        an element is oversized (the early stop of Section 3.2): I holds a single step, a step
 *        of I is longer than the nominal interval length T / 2^l of the level, or a triangle of
 *        X extends over more than the box width 2 hx_l in some direction;
 *      - the temporal split of (t_a, t_b] is at the step t_s (a < s < b) nearest to
 *        (t_a + t_b) / 2, the smaller s on a tie; children without elements are not added;
 *      - padding per level as for uniform steps; the interaction-area radii of level l from the
 *        longest interval L_l of the level (separation 4 L_l for M2L, 2 L_l for the nearfield).
 * ====================================================================================== */

/* int over the target step (tk0, tk1] and the source step (tj0, tj1] of the heat kernel (Section
 * 2): the second difference of G2 at the four time differences, 0 for a later source step; the
 * bounded form G2t for small u as for uniform steps (the parts linear in s cancel when the source
 * step precedes the target step; the same step keeps G2 alone). */
double orc_time_V_steps(double r, double tk0, double tk1, double tj0, double tj1, double alpha)
{
    if (tj0 >= tk1) return 0.0;
    if (tj0 == tk0 && tj1 == tk1) return orc_G2(r, tk1 - tk0, alpha);
    const double s1 = tk1 - tj0, s2 = tk1 - tj1, s3 = tk0 - tj0, s4 = tk0 - tj1;
    const double u = r / (2.0 * sqrt(alpha * s1));
    if (u < 1.0)
        return orc_G2t(r, s1, alpha) - orc_G2t(r, s2, alpha) - orc_G2t(r, s3, alpha) + orc_G2t(r, s4, alpha);
    return orc_G2(r, s1, alpha) - orc_G2(r, s2, alpha) - orc_G2(r, s3, alpha) + orc_G2(r, s4, alpha);
}

/* V_h entries of the triangle pair (x, y) for n step pairs pr[i] = (k, j): out[i] = V[(k,x),(j,y)].
 * Touching triangles use the Sauter-Schwab rule when the source step is the target step or the
 * one before it (the time integral is singular in r there), the regular rule otherwise. */
static void og_pair_steps(const orc_problem *P, const double *ts, int x, int y, const int (*pr)[2], int n,
                          double *out)
{
    const int *tx = P->T + 3 * x, *ty = P->T + 3 * y;
    const double *X[3] = {P->V + 3 * tx[0], P->V + 3 * tx[1], P->V + 3 * tx[2]};
    const double *Y[3] = {P->V + 3 * ty[0], P->V + 3 * ty[1], P->V + 3 * ty[2]};
    const int cls = or_shared(tx, ty);
    double tb[4 * 64], acc[64];
    int sel[64];
    for (int pass = 0; pass < 2; ++pass) { /* pass 0: regular pairs, pass 1: Sauter-Schwab pairs */
        int m = 0;
        for (int i = 0; i <= n; ++i) {
            if (i < n) {
                const int k = pr[i][0], j = pr[i][1];
                const int ss = cls > 0 && k - j <= 1;
                if (j > k) { out[i] = 0.0; continue; }
                if (ss != pass) continue;
                tb[4 * m] = ts[k];
                tb[4 * m + 1] = ts[k + 1];
                tb[4 * m + 2] = ts[j];
                tb[4 * m + 3] = ts[j + 1];
                sel[m++] = i;
            }
            if (m == 64 || (i == n && m > 0)) {
                or_kernel kr;
                memset(&kr, 0, sizeof(kr));
                kr.kind = ORK_VSTEPS;
                kr.nd = m;
                kr.alpha = P->alpha;
                kr.tb = tb;
                if (pass) {
                    const double *PX[3], *PY[3];
                    int perm[3];
                    or_ss_order(P->V, tx, ty, PX, PY, perm);
                    or_pair_ss(cls, PX, PY, perm, &kr, P->n_s, acc);
                } else {
                    or_pair_regular(X, Y, &kr, P->n_r, acc);
                }
                for (int q = 0; q < m; ++q) out[sel[q]] = acc[q];
                m = 0;
            }
        }
    }
}

typedef struct {
    int nlev;
    int lx[OR_MAXL], st[OR_MAXL];   /* st[l]: level l -> l+1 is a space-time refinement */
    double H, corner[3], pad[OR_MAXL];
    int ntr_far[OR_MAXL], ntr_near[OR_MAXL];
    int nb[OR_MAXL];
    int *cell[OR_MAXL];             /* [nb][3] grid multi-index of the spatial part */
    int *kk[OR_MAXL];               /* [nb] index k of the temporal part I_k^(l) */
    int *leaf[OR_MAXL];             /* [nb] */
    int *par[OR_MAXL];              /* [nb] parent box (-1 at level 0) */
    int *ia[OR_MAXL], *ib[OR_MAXL]; /* [2^l] steps [ia, ib) of interval k, -1 when absent */
    int *cstart[OR_MAXL];           /* [G^3 + 1] triangles of each cell: ctri[cstart[c] .. cstart[c+1]) */
    int *ctri[OR_MAXL];
    long long *key[OR_MAXL];        /* [nb] sorted k G^3 + cell */
    int *kbox[OR_MAXL];             /* [nb] the box of key[i] */
} og_tree;

static int og_G(const og_tree *t, int l) { return 1 << t->lx[l]; }
static int og_lin(const int *c, int G) { return (c[0] * G + c[1]) * G + c[2]; }

static void og_tree_free(og_tree *t)
{
    for (int l = 0; l < OR_MAXL; ++l) {
        free(t->cell[l]); free(t->kk[l]); free(t->leaf[l]); free(t->par[l]);
        free(t->ia[l]); free(t->ib[l]); free(t->cstart[l]); free(t->ctri[l]);
        free(t->key[l]); free(t->kbox[l]);
    }
    memset(t, 0, sizeof(*t));
}

static int og_find(const og_tree *t, int l, int k, const int *c)
{
    const int G = og_G(t, l);
    for (int d = 0; d < 3; ++d)
        if (c[d] < 0 || c[d] >= G) return -1;
    const long long q = (long long)k * G * G * G + og_lin(c, G);
    int lo = 0, hi = t->nb[l] - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) / 2;
        if (t->key[l][mid] == q) return t->kbox[l][mid];
        if (t->key[l][mid] < q) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

typedef struct { long long k; int b; } og_kb;
static int og_kb_cmp(const void *a, const void *b)
{
    const long long x = ((const og_kb *)a)->k, y = ((const og_kb *)b)->k;
    return x < y ? -1 : x > y;
}

/* cells of the triangles at level l (CSR by cell) */
static void og_cells(const orc_problem *P, const double *cent, og_tree *t, int l)
{
    const int G = og_G(t, l), nc = G * G * G;
    const double w = 2.0 * t->H / G;
    t->cstart[l] = (int *)calloc((size_t)nc + 1, sizeof(int));
    t->ctri[l] = (int *)malloc(sizeof(int) * (P->nt > 0 ? P->nt : 1));
    int *lin = (int *)malloc(sizeof(int) * P->nt);
    for (int x = 0; x < P->nt; ++x) {
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = or_cell(cent[3 * x + d], t->corner[d], w, G);
        lin[x] = og_lin(c, G);
        t->cstart[l][lin[x] + 1]++;
    }
    for (int c = 0; c < nc; ++c) t->cstart[l][c + 1] += t->cstart[l][c];
    int *fill = (int *)malloc(sizeof(int) * nc);
    memcpy(fill, t->cstart[l], sizeof(int) * nc);
    for (int x = 0; x < P->nt; ++x) t->ctri[l][fill[lin[x]]++] = x;
    free(fill);
    free(lin);
}

static int og_tree_build(const orc_problem *P, const double *ts, int n_max, og_tree *t)
{
    memset(t, 0, sizeof(*t));
    const int nt = P->nt, E = P->Et;
    if (nt < 1 || E < 1 || n_max < 1) return -1;
    for (int j = 0; j < E; ++j)
        if (!(ts[j + 1] > ts[j])) return -1;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < P->nv; ++i)
        for (int c = 0; c < 3; ++c) {
            if (P->V[3 * i + c] < lo[c]) lo[c] = P->V[3 * i + c];
            if (P->V[3 * i + c] > hi[c]) hi[c] = P->V[3 * i + c];
        }
    for (int c = 0; c < 3; ++c)
        if (0.5 * (hi[c] - lo[c]) > t->H) t->H = 0.5 * (hi[c] - lo[c]);
    for (int c = 0; c < 3; ++c) t->corner[c] = 0.5 * (lo[c] + hi[c]) - t->H;
    double *cent = (double *)malloc(sizeof(double) * 3 * nt), *ext = (double *)malloc(sizeof(double) * nt);
    for (int x = 0; x < nt; ++x) {
        ext[x] = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double a = P->V[3 * P->T[3 * x] + c], b = P->V[3 * P->T[3 * x + 1] + c], d = P->V[3 * P->T[3 * x + 2] + c];
            cent[3 * x + c] = ((a + b) + d) / 3.0;
            const double mx_ = fmax(a, fmax(b, d)), mn = fmin(a, fmin(b, d));
            if (mx_ - mn > ext[x]) ext[x] = mx_ - mn;
        }
    }
    const double T = ts[E];
    int lx0 = 0;
    while (1) {
        const double hx = t->H / (double)(1 << lx0);
        if (hx * hx <= P->c_st * 4.0 * P->alpha * (T / 2.0) || lx0 > 20) break;
        lx0++;
    }
    /* level 0: every non-empty cell with the interval (0, T] */
    t->lx[0] = lx0;
    og_cells(P, cent, t, 0);
    {
        const int G = og_G(t, 0), nc = G * G * G;
        int nb = 0;
        for (int c = 0; c < nc; ++c) nb += t->cstart[0][c + 1] > t->cstart[0][c];
        t->nb[0] = nb;
        t->cell[0] = (int *)malloc(sizeof(int) * 3 * nb);
        t->kk[0] = (int *)calloc(nb, sizeof(int));
        t->par[0] = (int *)malloc(sizeof(int) * nb);
        nb = 0;
        for (int c = 0; c < nc; ++c)
            if (t->cstart[0][c + 1] > t->cstart[0][c]) {
                t->cell[0][3 * nb] = c / (G * G);
                t->cell[0][3 * nb + 1] = (c / G) % G;
                t->cell[0][3 * nb + 2] = c % G;
                t->par[0][nb++] = -1;
            }
        t->ia[0] = (int *)malloc(sizeof(int));
        t->ib[0] = (int *)malloc(sizeof(int));
        t->ia[0][0] = 0;
        t->ib[0][0] = E;
    }
    int l = 0, rc = 0;
    while (1) {
        const int G = og_G(t, l), nb = t->nb[l];
        const double hx = t->H / G;
        t->leaf[l] = (int *)malloc(sizeof(int) * (nb > 0 ? nb : 1));
        int nref = 0;
        for (int b = 0; b < nb; ++b) {
            const int *c = t->cell[l] + 3 * b, k = t->kk[l][b], a = t->ia[l][k], e = t->ib[l][k];
            const int cl = og_lin(c, G), ntri = t->cstart[l][cl + 1] - t->cstart[l][cl];
            double maxstep = 0.0, maxext = 0.0;
            for (int j = a; j < e; ++j)
                if (ts[j + 1] - ts[j] > maxstep) maxstep = ts[j + 1] - ts[j];
            for (int q = t->cstart[l][cl]; q < t->cstart[l][cl + 1]; ++q)
                if (ext[t->ctri[l][q]] > maxext) maxext = ext[t->ctri[l][q]];
            const int refine = (long long)ntri * (e - a) >= n_max && e - a >= 2 && maxstep <= T / (double)(1 << l) &&
                               maxext <= 2.0 * hx;
            t->leaf[l][b] = !refine;
            nref += refine;
        }
        if (nref == 0) break;
        if (l + 1 >= OR_MAXL) { rc = -1; break; }
        const double ht1 = T / (double)(1 << (l + 2));
        t->st[l] = !(hx * hx <= P->c_st * 4.0 * P->alpha * ht1);
        t->lx[l + 1] = t->lx[l] + t->st[l];
        og_cells(P, cent, t, l + 1);
        const int G1 = og_G(t, l + 1), n1 = 1 << (l + 1);
        t->ia[l + 1] = (int *)malloc(sizeof(int) * n1);
        t->ib[l + 1] = (int *)malloc(sizeof(int) * n1);
        for (int k = 0; k < n1; ++k) t->ia[l + 1][k] = t->ib[l + 1][k] = -1;
        int cap = 16 * nref + 16, nb1 = 0;
        t->cell[l + 1] = (int *)malloc(sizeof(int) * 3 * cap);
        t->kk[l + 1] = (int *)malloc(sizeof(int) * cap);
        t->par[l + 1] = (int *)malloc(sizeof(int) * cap);
        for (int b = 0; b < nb; ++b) {
            if (t->leaf[l][b]) continue;
            const int *c = t->cell[l] + 3 * b, k = t->kk[l][b], a = t->ia[l][k], e = t->ib[l][k];
            /* split at the step nearest the centre (smaller index on a tie) */
            const double mid = 0.5 * (ts[a] + ts[e]);
            int s = a + 1;
            for (int q = a + 2; q < e; ++q)
                if (fabs(ts[q] - mid) < fabs(ts[s] - mid)) s = q;
            t->ia[l + 1][2 * k] = a;
            t->ib[l + 1][2 * k] = s;
            t->ia[l + 1][2 * k + 1] = s;
            t->ib[l + 1][2 * k + 1] = e;
            for (int ci = 0; ci < 2; ++ci)
                for (int o = 0; o < (t->st[l] ? 8 : 1); ++o) {
                    int cc[3];
                    for (int d = 0; d < 3; ++d) cc[d] = t->st[l] ? 2 * c[d] + ((o >> (2 - d)) & 1) : c[d];
                    const int cl = og_lin(cc, G1);
                    if (t->cstart[l + 1][cl + 1] == t->cstart[l + 1][cl]) continue;
                    memcpy(t->cell[l + 1] + 3 * nb1, cc, sizeof(cc));
                    t->kk[l + 1][nb1] = 2 * k + ci;
                    t->par[l + 1][nb1++] = b;
                }
        }
        t->nb[l + 1] = nb1;
        l++;
    }
    t->nlev = l + 1;
    /* padding: largest overshoot of a triangle over its unpadded cell, monotone in the level */
    for (int q = 0; q < t->nlev; ++q) {
        const int G = og_G(t, q);
        const double w = 2.0 * t->H / G;
        double ov = 0.0;
        for (int x = 0; x < nt; ++x) {
            int c[3];
            for (int d = 0; d < 3; ++d) c[d] = or_cell(cent[3 * x + d], t->corner[d], w, G);
            for (int v = 0; v < 3; ++v)
                for (int d = 0; d < 3; ++d) {
                    const double z = P->V[3 * P->T[3 * x + v] + d], blo = t->corner[d] + c[d] * w, bhi = blo + w;
                    if (blo - z > ov) ov = blo - z;
                    if (z - bhi > ov) ov = z - bhi;
                }
        }
        t->pad[q] = ov;
    }
    for (int q = t->nlev - 2; q >= 0; --q)
        if (t->pad[q + 1] > t->pad[q]) t->pad[q] = t->pad[q + 1];
    for (int q = 0; q < t->nlev; ++q) {
        const int G = og_G(t, q);
        double L = 0.0;
        for (int k = 0; k < (1 << q); ++k)
            if (t->ia[q][k] >= 0 && ts[t->ib[q][k]] - ts[t->ia[q][k]] > L) L = ts[t->ib[q][k]] - ts[t->ia[q][k]];
        t->ntr_far[q] = or_ntr(P, t->H / G, t->pad[q], 4.0 * L, G);
        t->ntr_near[q] = or_ntr(P, t->H / G, t->pad[q], 2.0 * L, G);
        og_kb *kb = (og_kb *)malloc(sizeof(og_kb) * (t->nb[q] > 0 ? t->nb[q] : 1));
        for (int b = 0; b < t->nb[q]; ++b) {
            kb[b].k = (long long)t->kk[q][b] * G * G * G + og_lin(t->cell[q] + 3 * b, G);
            kb[b].b = b;
        }
        qsort(kb, t->nb[q], sizeof(og_kb), og_kb_cmp);
        t->key[q] = (long long *)malloc(sizeof(long long) * (t->nb[q] > 0 ? t->nb[q] : 1));
        t->kbox[q] = (int *)malloc(sizeof(int) * (t->nb[q] > 0 ? t->nb[q] : 1));
        for (int b = 0; b < t->nb[q]; ++b) {
            t->key[q][b] = kb[b].k;
            t->kbox[q][b] = kb[b].b;
        }
        free(kb);
    }
    free(cent);
    free(ext);
    if (rc) og_tree_free(t);
    return rc;
}

/* the same-level nearfield of box b of level l (Eq. def_st_nearfield, first set): boxes Y x J of
 * level l with J in {I_{k-1}, I_k} and Y in the interaction area of X; returns their count */
static int og_near_same(const og_tree *t, int l, int b, int *out, int cap)
{
    const int *c = t->cell[l] + 3 * b, k = t->kk[l][b], r = t->ntr_near[l], G = og_G(t, l);
    int n = 0, lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = c[d] - r < 0 ? 0 : c[d] - r;
        hi[d] = c[d] + r > G - 1 ? G - 1 : c[d] + r;
    }
    for (int j = k - 1; j <= k; ++j) {
        if (j < 0) continue;
        for (int a0 = lo[0]; a0 <= hi[0]; ++a0)
            for (int a1 = lo[1]; a1 <= hi[1]; ++a1)
                for (int a2 = lo[2]; a2 <= hi[2]; ++a2) {
                    const int cc[3] = {a0, a1, a2};
                    const int s = og_find(t, l, j, cc);
                    if (s >= 0 && n < cap) out[n++] = s;
                }
    }
    return n;
}

/* an upper bound of the nearfield list length of any leaf */
static int og_nf_cap(const og_tree *t)
{
    int c = 0;
    for (int l = 0; l < t->nlev; ++l) c += 2 * og_G(t, l) * og_G(t, l) * og_G(t, l);
    return c;
}

/* the nearfield N(Z) of a leaf box (Eq. def_st_nearfield): its same-level nearfield and the
 * leaves in the same-level nearfields of all its ancestors (N(parent(Z)) /\ L_Sigma, recursively);
 * entries (level, box); returns the count */
static int og_nearfield(const og_tree *t, int l, int b, int (*out)[2], int cap)
{
    const int tcap = og_nf_cap(t);
    int *tmp = (int *)malloc(sizeof(int) * tcap), n = 0;
    int m = og_near_same(t, l, b, tmp, tcap);
    for (int i = 0; i < m && n < cap; ++i) { out[n][0] = l; out[n][1] = tmp[i]; n++; }
    for (int q = l - 1, a = t->par[l][b]; q >= 0 && a >= 0; a = t->par[q][a], --q) {
        m = og_near_same(t, q, a, tmp, tcap);
        for (int i = 0; i < m && n < cap; ++i)
            if (t->leaf[q][tmp[i]]) { out[n][0] = q; out[n][1] = tmp[i]; n++; }
    }
    free(tmp);
    return n;
}

/* the interaction list I(Z) of box b of level l >= 2 (Eq. def_st_interaction_list) */
static int og_interaction(const og_tree *t, int l, int b, int *out, int cap)
{
    const int *c = t->cell[l] + 3 * b, k = t->kk[l][b], r = t->ntr_far[l], G = og_G(t, l);
    int js[2], nj = or_interaction_list(k, js), n = 0, lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = c[d] - r < 0 ? 0 : c[d] - r;
        hi[d] = c[d] + r > G - 1 ? G - 1 : c[d] + r;
    }
    for (int q = 0; q < nj; ++q)
        for (int a0 = lo[0]; a0 <= hi[0]; ++a0)
            for (int a1 = lo[1]; a1 <= hi[1]; ++a1)
                for (int a2 = lo[2]; a2 <= hi[2]; ++a2) {
                    const int cc[3] = {a0, a1, a2};
                    const int s = og_find(t, l, js[q], cc);
                    if (s >= 0 && n < cap) out[n++] = s;
                }
    return n;
}

/* spatial part of box b of level l: padded centre and half-size */
static void og_box_geom(const og_tree *t, int l, int b, double *cen, double *hp)
{
    const int G = og_G(t, l);
    const double hx = t->H / G;
    for (int c = 0; c < 3; ++c) cen[c] = t->corner[c] + (2.0 * t->cell[l][3 * b + c] + 1.0) * hx;
    *hp = hx + t->pad[l];
}

/* tree summary for the pins and the GPU comparison: nlev; per level l: lx, boxes, leaves,
 * intervals present, ntr_far, ntr_near, st (levels [0, OR_MAXL)); boxes_out (optional, cap
 * entries of 6 ints: level, cell x y z, k, leaf) */
int orc_gen_tree_info(const orc_problem *P, const double *ts, int n_max, int *nlev, int *lx, int *nbox, int *nleaf,
                      int *nint, int *ntr_far, int *ntr_near, int *st, double *pad, int *boxes_out, int cap)
{
    og_tree t;
    if (og_tree_build(P, ts, n_max, &t)) return -1;
    *nlev = t.nlev;
    int w = 0;
    for (int l = 0; l < t.nlev; ++l) {
        lx[l] = t.lx[l];
        nbox[l] = t.nb[l];
        nleaf[l] = 0;
        for (int b = 0; b < t.nb[l]; ++b) {
            nleaf[l] += t.leaf[l][b];
            if (boxes_out && w < cap) {
                int *o = boxes_out + 6 * w++;
                o[0] = l; o[1] = t.cell[l][3 * b]; o[2] = t.cell[l][3 * b + 1]; o[3] = t.cell[l][3 * b + 2];
                o[4] = t.kk[l][b]; o[5] = t.leaf[l][b];
            }
        }
        nint[l] = 0;
        for (int k = 0; k < (1 << l); ++k) nint[l] += t.ia[l][k] >= 0;
        ntr_far[l] = t.ntr_far[l];
        ntr_near[l] = t.ntr_near[l];
        st[l] = t.st[l];
        pad[l] = t.pad[l];
    }
    og_tree_free(&t);
    return 0;
}

/* interval bounds of interval k of level l: [ia, ib) steps, or -1 when absent (for the pins) */
int orc_gen_interval(const orc_problem *P, const double *ts, int n_max, int l, int k, int *ia, int *ib)
{
    og_tree t;
    if (og_tree_build(P, ts, n_max, &t)) return -1;
    *ia = *ib = -1;
    if (l < t.nlev && k >= 0 && k < (1 << l)) {
        *ia = t.ia[l][k];
        *ib = t.ib[l][k];
    }
    og_tree_free(&t);
    return 0;
}

/* How often the FMM partition of Alg. 2 covers every element pair: cover[e][e'] for target
 * element e = k nt + x and source element e' = j nt + y, over the nearfield blocks of the leaves
 * (causal pairs j <= k only: the other entries of a block vanish) and the admissible blocks of
 * all M2L pairs (their pairs are all causal).  For tiny problems: (Et nt)^2 ints. */
int orc_gen_coverage(const orc_problem *P, const double *ts, int n_max, int *cover)
{
    og_tree t;
    if (og_tree_build(P, ts, n_max, &t)) return -1;
    const int nt = P->nt;
    const size_t ne = (size_t)P->Et * nt;
    memset(cover, 0, sizeof(int) * ne * ne);
    const int cap = og_nf_cap(&t);
    int (*nf)[2] = (int(*)[2])malloc(sizeof(int) * 2 * (size_t)cap);
    int *il = (int *)malloc(sizeof(int) * (size_t)cap);
    for (int l = 0; l < t.nlev; ++l) {
        const int G = og_G(&t, l);
        for (int b = 0; b < t.nb[l]; ++b) {
            const int ct = og_lin(t.cell[l] + 3 * b, G), kt = t.kk[l][b];
            /* nearfield of a leaf */
            int nn = t.leaf[l][b] ? og_nearfield(&t, l, b, nf, cap) : 0;
            for (int q = 0; q < nn; ++q) {
                const int ls = nf[q][0], s = nf[q][1], Gs = og_G(&t, ls), cs = og_lin(t.cell[ls] + 3 * s, Gs);
                const int ks = t.kk[ls][s];
                for (int i = t.cstart[l][ct]; i < t.cstart[l][ct + 1]; ++i)
                    for (int k = t.ia[l][kt]; k < t.ib[l][kt]; ++k)
                        for (int i2 = t.cstart[ls][cs]; i2 < t.cstart[ls][cs + 1]; ++i2)
                            for (int j = t.ia[ls][ks]; j < t.ib[ls][ks] && j <= k; ++j)
                                cover[((size_t)k * nt + t.ctri[l][i]) * ne + (size_t)j * nt + t.ctri[ls][i2]]++;
            }
            /* admissible blocks */
            const int ni = l >= 2 ? og_interaction(&t, l, b, il, cap) : 0;
            for (int q = 0; q < ni; ++q) {
                const int s = il[q], cs = og_lin(t.cell[l] + 3 * s, G), ks = t.kk[l][s];
                for (int i = t.cstart[l][ct]; i < t.cstart[l][ct + 1]; ++i)
                    for (int k = t.ia[l][kt]; k < t.ib[l][kt]; ++k)
                        for (int i2 = t.cstart[l][cs]; i2 < t.cstart[l][cs + 1]; ++i2)
                            for (int j = t.ia[l][ks]; j < t.ib[l][ks]; ++j)
                                cover[((size_t)k * nt + t.ctri[l][i]) * ne + (size_t)j * nt + t.ctri[l][i2]]++;
            }
        }
    }
    free(nf);
    free(il);
    og_tree_free(&t);
    return 0;
}

/* f = V_h w by the pFMM (Alg. 2) on the general tree; w, f: [Et][nt].  parts: bit 0 nearfield,
 * bit 1 far field; targets: triangles whose rows are computed (NULL: all), the other rows are 0. */
int orc_gen_pfmm_apply(const orc_problem *P, const double *ts, int n_max, const double *w, double *f,
                       const int *targets, int ntargets, int parts, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    og_tree t;
    if (og_tree_build(P, ts, n_max, &t)) return -1;
    or_fmm F;
    memset(&F, 0, sizeof(F));
    F.P = P;
    or_mi_make(P->m_x, &F.mi);
    const int na = P->m_t + 1, nk = F.mi.nk, mt = P->m_t, mx = P->m_x, nt = P->nt, L = t.nlev;
    memset(f, 0, sizeof(double) * (size_t)P->Et * nt);
    unsigned char *is_tgt = (unsigned char *)calloc(nt, 1);
    if (targets && ntargets >= 0)
        for (int i = 0; i < ntargets; ++i) is_tgt[targets[i]] = 1;
    else
        memset(is_tgt, 1, nt);

    if ((parts & 2) && L >= 3) {
        double *mu[OR_MAXL] = {0}, *lam[OR_MAXL] = {0};
        for (int l = 0; l < L; ++l) {
            mu[l] = (double *)calloc((size_t)t.nb[l] * na * nk + 1, sizeof(double));
            lam[l] = (double *)calloc((size_t)t.nb[l] * na * nk + 1, sizeof(double));
        }
        /* S2M at every leaf of a level >= 2 (Eq. s2m); leaves above level 2 have no far field */
        for (int l = 2; l < L; ++l) {
            const int G = og_G(&t, l);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int b = 0; b < t.nb[l]; ++b) {
                if (!t.leaf[l][b]) continue;
                const int cl = og_lin(t.cell[l] + 3 * b, G), k = t.kk[l][b], a0 = t.ia[l][k], a1 = t.ib[l][k];
                double cen[3], hp, *sm = (double *)malloc(sizeof(double) * nk), tm[OR_MAXQ];
                og_box_geom(&t, l, b, cen, &hp);
                double *m = mu[l] + (size_t)b * na * nk;
                for (int q = t.cstart[l][cl]; q < t.cstart[l][cl + 1]; ++q) {
                    const int x = t.ctri[l][q];
                    or_space_moments(&F, x, cen, hp, 0, sm);
                    for (int j = a0; j < a1; ++j) {
                        for (int a = 0; a < na; ++a) tm[a] = or_time_moment(a, mt, ts[a0], ts[a1], ts[j], ts[j + 1] - ts[j]);
                        const double wv = w[(size_t)j * nt + x];
                        for (int a = 0; a < na; ++a)
                            for (int i = 0; i < nk; ++i) m[a * nk + i] += wv * tm[a] * sm[i];
                    }
                }
                free(sm);
            }
        }
        /* M2M (Eq. temp_m2m, st_m2m): parents of levels L-2 .. 2 */
        for (int l = L - 2; l >= 2; --l) {
            for (int bc = 0; bc < t.nb[l + 1]; ++bc) { /* serial: children of one parent add into it */
                const int bp = t.par[l + 1][bc], kc = t.kk[l + 1][bc], kp = t.kk[l][bp];
                double cc[3], hc, cp[3], hp, q1[3][OR_MAXQ][OR_MAXQ], qt[OR_MAXQ][OR_MAXQ];
                og_box_geom(&t, l + 1, bc, cc, &hc);
                og_box_geom(&t, l, bp, cp, &hp);
                const double clo = ts[t.ia[l + 1][kc]], chi = ts[t.ib[l + 1][kc]];
                for (int ac = 0; ac < na; ++ac) {
                    const double xi = 0.5 * (clo + chi) + 0.5 * (chi - clo) * or_cheb_node(ac, mt);
                    for (int ap = 0; ap < na; ++ap) qt[ac][ap] = or_lagrange(ap, mt, ts[t.ia[l][kp]], ts[t.ib[l][kp]], xi);
                }
                if (t.st[l])
                    for (int d = 0; d < 3; ++d)
                        for (int a1 = 0; a1 <= mx; ++a1)
                            for (int n1 = 0; n1 <= mx; ++n1) q1[d][a1][n1] = or_qx(a1, n1, cc[d], hc, cp[d], hp, mx);
                const double *mc = mu[l + 1] + (size_t)bc * na * nk;
                double *mp = mu[l] + (size_t)bp * na * nk;
                for (int ap = 0; ap < na; ++ap)
                    for (int ac = 0; ac < na; ++ac)
                        for (int iv = 0; iv < nk; ++iv) {
                            const int *nu = F.mi.k[iv];
                            double acc = 0.0;
                            if (!t.st[l]) {
                                acc = mc[ac * nk + iv];
                            } else {
                                for (int k0 = 0; k0 <= nu[0]; ++k0)
                                    for (int k1 = 0; k1 <= nu[1]; ++k1)
                                        for (int k2 = 0; k2 <= nu[2]; ++k2) {
                                            const int ik = F.mi.lookup[(k0 * (mx + 1) + k1) * (mx + 1) + k2];
                                            acc += q1[0][k0][nu[0]] * q1[1][k1][nu[1]] * q1[2][k2][nu[2]] * mc[ac * nk + ik];
                                        }
                            }
                            mp[ap * nk + iv] += qt[ac][ap] * acc;
                        }
            }
        }
        /* M2L (Eq. m2l with Eq. exp_coeffs_3d / exp_coeffs_1d) at every level >= 2 */
        for (int l = 2; l < L; ++l) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int bt = 0; bt < t.nb[l]; ++bt) {
                const int cap = og_nf_cap(&t);
                int *il = (int *)malloc(sizeof(int) * (size_t)cap);
                const int ni = og_interaction(&t, l, bt, il, cap), kt = t.kk[l][bt];
                double ct[3], hpx, *E1 = (double *)malloc(sizeof(double) * 3 * OR_MAXQ * OR_MAXQ);
                og_box_geom(&t, l, bt, ct, &hpx);
                const double tlo = ts[t.ia[l][kt]], thi = ts[t.ib[l][kt]];
                double *lt = lam[l] + (size_t)bt * na * nk;
                for (int q = 0; q < ni; ++q) {
                    const int bs = il[q], ks = t.kk[l][bs];
                    double cs[3], hs;
                    og_box_geom(&t, l, bs, cs, &hs);
                    const double slo = ts[t.ia[l][ks]], shi = ts[t.ib[l][ks]];
                    const double *ms = mu[l] + (size_t)bs * na * nk;
                    for (int a = 0; a < na; ++a)
                        for (int b = 0; b < na; ++b) {
                            /* xi_{I,b} - xi_{J,a} */
                            const double dt = (0.5 * (tlo + thi) + 0.5 * (thi - tlo) * or_cheb_node(b, mt)) -
                                              (0.5 * (slo + shi) + 0.5 * (shi - slo) * or_cheb_node(a, mt));
                            const double dab = 4.0 * P->alpha * dt / (hpx * hpx), pf = pow(4.0 * OR_PI * P->alpha * dt, -1.5);
                            for (int d = 0; d < 3; ++d)
                                for (int kk = 0; kk <= mx; ++kk)
                                    for (int ll = 0; ll + kk <= mx; ++ll)
                                        E1[(d * OR_MAXQ + kk) * OR_MAXQ + ll] = or_E1(kk, ll, (ct[d] - cs[d]) / hpx, dab, mx);
                            for (int iv = 0; iv < nk; ++iv) {
                                const int *nu = F.mi.k[iv];
                                double acc = 0.0;
                                for (int ik = 0; ik < nk; ++ik) {
                                    const int *ka = F.mi.k[ik];
                                    if (ka[0] + ka[1] + ka[2] + nu[0] + nu[1] + nu[2] > mx) continue;
                                    double E = pf;
                                    for (int d = 0; d < 3; ++d) E *= E1[(d * OR_MAXQ + ka[d]) * OR_MAXQ + nu[d]];
                                    acc += E * ms[a * nk + ik];
                                }
                                lt[b * nk + iv] += acc;
                            }
                        }
                }
                free(E1);
                free(il);
            }
        }
        /* L2L (transposed M2M) for levels 3 .. L-1 */
        for (int l = 3; l < L; ++l) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int bc = 0; bc < t.nb[l]; ++bc) {
                const int bp = t.par[l][bc], kc = t.kk[l][bc], kp = t.kk[l - 1][bp];
                double cc[3], hc, cp[3], hp, q1[3][OR_MAXQ][OR_MAXQ], qt[OR_MAXQ][OR_MAXQ];
                og_box_geom(&t, l, bc, cc, &hc);
                og_box_geom(&t, l - 1, bp, cp, &hp);
                const double clo = ts[t.ia[l][kc]], chi = ts[t.ib[l][kc]];
                for (int bcI = 0; bcI < na; ++bcI) {
                    const double xi = 0.5 * (clo + chi) + 0.5 * (chi - clo) * or_cheb_node(bcI, mt);
                    for (int bpI = 0; bpI < na; ++bpI)
                        qt[bcI][bpI] = or_lagrange(bpI, mt, ts[t.ia[l - 1][kp]], ts[t.ib[l - 1][kp]], xi);
                }
                if (t.st[l - 1])
                    for (int d = 0; d < 3; ++d)
                        for (int a1 = 0; a1 <= mx; ++a1)
                            for (int n1 = 0; n1 <= mx; ++n1) q1[d][a1][n1] = or_qx(a1, n1, cc[d], hc, cp[d], hp, mx);
                const double *lp = lam[l - 1] + (size_t)bp * na * nk;
                double *lc = lam[l] + (size_t)bc * na * nk;
                for (int bcI = 0; bcI < na; ++bcI)
                    for (int ik = 0; ik < nk; ++ik) {
                        const int *ka = F.mi.k[ik];
                        double acc = 0.0;
                        for (int bpI = 0; bpI < na; ++bpI) {
                            if (!t.st[l - 1]) {
                                acc += qt[bcI][bpI] * lp[bpI * nk + ik];
                                continue;
                            }
                            for (int n0 = ka[0]; n0 <= mx; ++n0)
                                for (int n1 = ka[1]; n0 + n1 <= mx; ++n1)
                                    for (int n2 = ka[2]; n0 + n1 + n2 <= mx; ++n2) {
                                        const int iv = F.mi.lookup[(n0 * (mx + 1) + n1) * (mx + 1) + n2];
                                        acc += qt[bcI][bpI] * q1[0][ka[0]][n0] * q1[1][ka[1]][n1] * q1[2][ka[2]][n2] *
                                               lp[bpI * nk + iv];
                                    }
                        }
                        lc[bcI * nk + ik] += acc;
                    }
            }
        }
        /* L2T at every leaf of a level >= 2 (Eq. l2t) */
        for (int l = 2; l < L; ++l) {
            const int G = og_G(&t, l);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int b = 0; b < t.nb[l]; ++b) {
                if (!t.leaf[l][b]) continue;
                const int cl = og_lin(t.cell[l] + 3 * b, G), k = t.kk[l][b], a0 = t.ia[l][k], a1 = t.ib[l][k];
                double cen[3], hp, *sm = (double *)malloc(sizeof(double) * nk), tm[OR_MAXQ];
                og_box_geom(&t, l, b, cen, &hp);
                const double *lb = lam[l] + (size_t)b * na * nk;
                for (int q = t.cstart[l][cl]; q < t.cstart[l][cl + 1]; ++q) {
                    const int x = t.ctri[l][q];
                    if (!is_tgt[x]) continue;
                    or_space_moments(&F, x, cen, hp, 0, sm);
                    for (int kt = a0; kt < a1; ++kt) {
                        for (int bb = 0; bb < na; ++bb) tm[bb] = or_time_moment(bb, mt, ts[a0], ts[a1], ts[kt], ts[kt + 1] - ts[kt]);
                        double acc = 0.0;
                        for (int bb = 0; bb < na; ++bb)
                            for (int i = 0; i < nk; ++i) acc += lb[bb * nk + i] * tm[bb] * sm[i];
                        f[(size_t)kt * nt + x] += acc;
                    }
                }
                free(sm);
            }
        }
        for (int l = 0; l < L; ++l) { free(mu[l]); free(lam[l]); }
    }

    if (parts & 1) {
        /* nearfield of every leaf (Eq. eval_sl_nf_block over N(Z) of Eq. def_st_nearfield) */
        for (int l = 0; l < L; ++l) {
            const int G = og_G(&t, l);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
            for (int b = 0; b < t.nb[l]; ++b) {
                if (!t.leaf[l][b]) continue;
                const int cap = og_nf_cap(&t);
                int (*nf)[2] = (int(*)[2])malloc(sizeof(int) * 2 * (size_t)cap);
                const int nn = og_nearfield(&t, l, b, nf, cap);
                const int cl = og_lin(t.cell[l] + 3 * b, G), kt = t.kk[l][b];
                const int k0 = t.ia[l][kt], k1 = t.ib[l][kt];
                int (*pr)[2] = (int(*)[2])malloc(sizeof(int) * 2 * (size_t)P->Et * P->Et);
                double *ent = (double *)malloc(sizeof(double) * (size_t)P->Et * P->Et);
                for (int q = t.cstart[l][cl]; q < t.cstart[l][cl + 1]; ++q) {
                    const int x = t.ctri[l][q];
                    if (!is_tgt[x]) continue;
                    for (int s = 0; s < nn; ++s) {
                        const int ls = nf[s][0], bs = nf[s][1], cs = og_lin(t.cell[ls] + 3 * bs, og_G(&t, ls));
                        const int ks = t.kk[ls][bs], j0 = t.ia[ls][ks], j1 = t.ib[ls][ks];
                        int np = 0;
                        for (int k = k0; k < k1; ++k)
                            for (int j = j0; j < j1 && j <= k; ++j) { pr[np][0] = k; pr[np][1] = j; np++; }
                        if (!np) continue;
                        for (int q2 = t.cstart[ls][cs]; q2 < t.cstart[ls][cs + 1]; ++q2) {
                            const int y = t.ctri[ls][q2];
                            og_pair_steps(P, ts, x, y, (const int(*)[2])pr, np, ent);
                            for (int i = 0; i < np; ++i) f[(size_t)pr[i][0] * nt + x] += ent[i] * w[(size_t)pr[i][1] * nt + y];
                        }
                    }
                }
                free(pr);
                free(ent);
                free(nf);
            }
        }
    }
    free(is_tgt);
    free(F.mi.k);
    free(F.mi.lookup);
    og_tree_free(&t);
    return 0;
}

/* The dense Galerkin product of Section 2 on the listed target rows: f[k][x] = sum over all
 * source steps j <= k and all triangles y of V[(k,x),(j,y)] w[j][y] (no FMM, no truncation). */
int orc_gen_dense_apply(const orc_problem *P, const double *ts, const double *w, const int *targets, int ntargets,
                        double *f, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    const int nt = P->nt, E = P->Et;
    memset(f, 0, sizeof(double) * (size_t)E * nt);
    int (*pr)[2] = (int(*)[2])malloc(sizeof(int) * 2 * (size_t)E * (E + 1) / 2);
    int np = 0;
    for (int k = 0; k < E; ++k)
        for (int j = 0; j <= k; ++j) { pr[np][0] = k; pr[np][1] = j; np++; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < ntargets; ++i) {
        const int x = targets[i];
        double *ent = (double *)malloc(sizeof(double) * np);
        for (int y = 0; y < nt; ++y) {
            og_pair_steps(P, ts, x, y, (const int(*)[2])pr, np, ent);
            for (int q = 0; q < np; ++q) f[(size_t)pr[q][0] * nt + x] += ent[q] * w[(size_t)pr[q][1] * nt + y];
        }
        free(ent);
    }
    free(pr);
    return 0;
}
