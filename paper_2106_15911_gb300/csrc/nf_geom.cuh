// nf_geom.cuh -- triangle geometry and the regular-pair quadrature shared by the stored and the
// on-the-fly nearfield kernels: vertex loads, Jacobians, outward normals, shared-vertex counts,
// and the collapsed Gauss rule over a pair of triangles for all step offsets.
#pragma once

#include "device_math.cuh"
#include "kernels.h"

namespace pfmm {

__device__ __forceinline__ void load_tri(const double *verts, const int *tri, int x, double P[3][3])
{
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c) P[v][c] = verts[3 * tri[3 * x + v] + c];
}

__device__ __forceinline__ double tri_jac(const double P[3][3], double n[3])
{
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) { e1[c] = P[1][c] - P[0][c]; e2[c] = P[2][c] - P[1][c]; }
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double J = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    n[0] = cr[0] / J; n[1] = cr[1] / J; n[2] = cr[2] / J;
    return J;
}

__device__ __forceinline__ double tri_normal_orig(const double P[3][3], double n[3])
{
    // outward normal from the stored vertex order: (P1 - P0) x (P2 - P0)
    double a[3], b[3];
    for (int c = 0; c < 3; ++c) { a[c] = P[1][c] - P[0][c]; b[c] = P[2][c] - P[0][c]; }
    n[0] = a[1] * b[2] - a[2] * b[1];
    n[1] = a[2] * b[0] - a[0] * b[2];
    n[2] = a[0] * b[1] - a[1] * b[0];
    double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= l; n[1] /= l; n[2] /= l;
    return l;
}

__device__ __forceinline__ int shared_count(const int *tri, int x, int y)
{
    int s = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += tri[3 * x + i] == tri[3 * y + j];
    return s;
}

// The Sauter-Schwab regularising substitutions (Sauter & Schwab, Boundary Element Methods,
// Sec. 5.2) at the point (xi, e1, e2, e3) of [0,1]^4: the pairs (s1, s2) on x's and (t1, t2) on
// y's reference triangle, pts[u] = {s1, s2, t1, t2}, with their Jacobians; cls 3 identical, 2
// common edge, 1 common vertex (vertices in the rule's local order).  Returns the count.
__device__ __forceinline__ int ss_points(int cls, double xi, double e1, double e2, double e3, double pts[6][4],
                                         double jac[6])
{
    if (cls == 3) {
        const double j = xi * xi * xi * e1 * e1 * e2;
        const double A_[6][4] = {{xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1)},
                                 {xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2)},
                                 {xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
                                 {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3)},
                                 {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2)},
                                 {xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)}};
        for (int u = 0; u < 6; ++u) {
            for (int c = 0; c < 4; ++c) pts[u][c] = A_[u][c];
            jac[u] = j;
        }
        return 6;
    }
    if (cls == 2) {
        const double j0 = xi * xi * xi * e1 * e1, j1 = j0 * e2;
        const double A_[5][4] = {{xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
                                 {xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)},
                                 {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3},
                                 {xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1},
                                 {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2}};
        for (int u = 0; u < 5; ++u) {
            for (int c = 0; c < 4; ++c) pts[u][c] = A_[u][c];
            jac[u] = u == 0 ? j0 : j1;
        }
        return 5;
    }
    const double j = xi * xi * xi * e2;
    const double A_[2][4] = {{xi, xi * e1, xi * e2, xi * e2 * e3}, {xi * e2, xi * e2 * e3, xi, xi * e1}};
    for (int u = 0; u < 2; ++u) {
        for (int c = 0; c < 4; ++c) pts[u][c] = A_[u][c];
        jac[u] = j;
    }
    return 2;
}

// Regular quadrature of the pair (x, y) (internal triangles) for the step offsets d0 .. nd-1 of
// Eq. eval_sl_nf_block: acc[d] (V) or acc[3 d + v] (K, v: y's vertices in mesh order) are
// accumulated (the caller zeroes them).  Touching pairs start at d0 = 2: their d = 0, 1 entries
// come from the Sauter-Schwab rule.  Returns d0.
template <typename R, bool KOP>
__device__ __forceinline__ int nf_regular_pair(const NfQuadArgs &a, int x, int y, R *acc)
{
    double PX[3][3], PY[3][3], nx[3], ny[3];
    load_tri(a.verts, a.tri, x, PX);
    load_tri(a.verts, a.tri, y, PY);
    double Jx = tri_jac(PX, nx), Jy = tri_jac(PY, ny);
    tri_normal_orig(PY, ny);
    const int nd = a.nd;
    int d0 = shared_count(a.tri, x, y) > 0 ? 2 : 0;  // d = 0, 1 of touching pairs: singular rule
    const int nq = a.nq_reg;
    const R h = R(a.h), alpha = R(a.alpha);
    for (int i = 0; i < nq; ++i) {
        double s1 = a.rule_reg[i], s2 = a.rule_reg[nq + i], wi = a.rule_reg[2 * nq + i];
        double xp[3];
        for (int c = 0; c < 3; ++c) xp[c] = PX[0][c] + s1 * (PX[1][c] - PX[0][c]) + s2 * (PX[2][c] - PX[1][c]);
        for (int j = 0; j < nq; ++j) {
            double t1 = a.rule_reg[j], t2 = a.rule_reg[nq + j], wj = a.rule_reg[2 * nq + j];
            double yp[3], dx[3];
            for (int c = 0; c < 3; ++c) {
                yp[c] = PY[0][c] + t1 * (PY[1][c] - PY[0][c]) + t2 * (PY[2][c] - PY[1][c]);
                dx[c] = xp[c] - yp[c];
            }
            double r = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
            R wt = R(wi * wj * Jx * Jy);
            R vals[8];
            if (!KOP) {
                dev::time_V_all<R>(R(r), h, alpha, nd, vals);
                for (int d = d0; d < nd; ++d) acc[d] += wt * vals[d];
            } else {
                dev::time_K_all<R>(R(r), h, alpha, nd, vals);
                R dn = R(dx[0] * ny[0] + dx[1] * ny[1] + dx[2] * ny[2]);
                R by[3] = {R(1.0 - t1), R(t1 - t2), R(t2)};
                for (int d = d0; d < nd; ++d) {
                    R v = wt * dn * vals[d];
                    acc[3 * d + 0] += v * by[0];
                    acc[3 * d + 1] += v * by[1];
                    acc[3 * d + 2] += v * by[2];
                }
            }
        }
    }
    return d0;
}

}  // namespace pfmm
