// k_setup.cu -- one-time device work of pfmm_build_trees: expansion tables and the nearfield
// quadrature of V_h and K_h.
//
// Tables (Section 3.1, 3.4):
//   Sx[x][kappa]    = int_{gamma_x} T_{Y,kappa}(y) ds_y           (S2M / L2T space part, Eq. s2m, l2t)
//   SK[x][v][kappa] = int_{gamma_x} alpha n_x . grad T_{Y,kappa}(y) phi_v(y) ds_y
//                     (double-layer moments: the normal derivative falls on the expansion of
//                      the source variable, Section 3 "slight modifications")
//   E1[D][a][b][o][k][l] = E_{k,l}(r_o, d_ab) of Eq. exp_coeffs_1d for the interval gap D in {2,3}
//                          and grid offset o of one level; pref[D][a][b] = (4 pi alpha dt_ab)^{-3/2}
// Nearfield (Eq. eval_sl_nf_block with the entries of Section 2): collapsed Gauss-Legendre
// n_r x n_r per triangle for regular pairs; Sauter-Schwab (Sauter & Schwab, Boundary Element
// Methods, Sec. 5.2) with n_s points per direction for triangles sharing a vertex at d = 0, 1.
#include <cstdio>

#include "device_math.cuh"
#include "kernels.h"
#include "nf_geom.cuh"

namespace pfmm {

using namespace dev;

// ------------------------------------------------------------------------------------------
// Sx, SK: thread per (triangle, kappa)
__global__ void k_space_tables(const double *__restrict__ verts, const int *__restrict__ tri, const int *__restrict__ tri_leaf,
                               const int *__restrict__ leaf_grid, double c0, double c1, double c2, double hx, double hxp,
                               int nt, int mx, int nk, const int *__restrict__ kidx, const double *__restrict__ rule,
                               int nq, double alpha, double *__restrict__ Sx, double *__restrict__ SK)
{
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nt * nk) return;
    int x = gid / nk, ik = gid % nk;
    int k0 = kidx[3 * ik], k1 = kidx[3 * ik + 1], k2 = kidx[3 * ik + 2];
    const int *t = tri + 3 * x;
    double P[3][3];
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c) P[v][c] = verts[3 * t[v] + c];
    double e1[3], e2[3], cr[3];
    for (int c = 0; c < 3; ++c) { e1[c] = P[1][c] - P[0][c]; e2[c] = P[2][c] - P[1][c]; }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double J = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double n[3] = {cr[0] / J, cr[1] / J, cr[2] / J};
    const int *g = leaf_grid + 3 * tri_leaf[x];
    double cen[3] = {c0 + (2.0 * g[0] + 1.0) * hx, c1 + (2.0 * g[1] + 1.0) * hx, c2 + (2.0 * g[2] + 1.0) * hx};
    double s = 0.0, sk[3] = {0.0, 0.0, 0.0};
    double T[3][kMaxMx + 1], dT[3][kMaxMx + 1];
    for (int q = 0; q < nq; ++q) {
        double s1 = rule[q], s2 = rule[nq + q], w = rule[2 * nq + q] * J;
        double yh[3];
        for (int c = 0; c < 3; ++c) yh[c] = (P[0][c] + s1 * e1[c] + s2 * e2[c] - cen[c]) / hxp;
        for (int c = 0; c < 3; ++c) {
            cheb_all(yh[c], mx, T[c]);
            cheb_deriv_all(yh[c], mx, dT[c]);
        }
        double tv = T[0][k0] * T[1][k1] * T[2][k2];
        s += w * tv;
        double gr[3] = {dT[0][k0] * T[1][k1] * T[2][k2] / hxp, T[0][k0] * dT[1][k1] * T[2][k2] / hxp,
                        T[0][k0] * T[1][k1] * dT[2][k2] / hxp};
        double dn = alpha * (n[0] * gr[0] + n[1] * gr[1] + n[2] * gr[2]);
        double by[3] = {1.0 - s1, s1 - s2, s2};
        for (int v = 0; v < 3; ++v) sk[v] += w * dn * by[v];
    }
    Sx[(size_t)x * nk + ik] = s;
    for (int v = 0; v < 3; ++v) SK[((size_t)x * 3 + v) * nk + ik] = sk[v];
}

void launch_space_tables(const SetupArgs &a, cudaStream_t st)
{
    int n = a.nt * a.nk;
    k_space_tables<<<(n + 127) / 128, 128, 0, st>>>(a.verts, a.tri, a.tri_leaf, a.leaf_grid, a.corner[0], a.corner[1],
                                                    a.corner[2], a.hx_leaf, a.hxp_leaf, a.nt, a.mx, a.nk, a.kidx,
                                                    a.rule_tab, a.nq_tab, a.alpha, a.Sx, a.SK);
}

// ------------------------------------------------------------------------------------------
// E1 tables of one level: thread per (D, a, b, o, k, l)
__global__ void k_e1_table(int na, int mt, int mx, int G, double hx, double hxp, double ht, double alpha,
                           double *__restrict__ E1, double *__restrict__ pref)
{
    const int m1 = mx + 1, no = 2 * G - 1;
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    int total = 2 * na * na * no * m1 * m1;
    if (gid >= total) return;
    int l = gid % m1, r_ = gid / m1;
    int k = r_ % m1;
    r_ /= m1;
    int o = r_ % no;
    r_ /= no;
    int b = r_ % na;
    r_ /= na;
    int a = r_ % na;
    int D = r_ / na + 2;
    double L = 2.0 * ht;
    double xb = cos((2.0 * b + 1.0) * kPi / (2.0 * mt + 2.0)), xa = cos((2.0 * a + 1.0) * kPi / (2.0 * mt + 2.0));
    double dt = D * L + ht * (xb - xa);  // xi_{I,b} - xi_{J,a}, J = I - D intervals
    double dab = 4.0 * alpha * dt / (hxp * hxp);
    if (o == 0 && k == 0 && l == 0) pref[((D - 2) * na + a) * na + b] = pow(4.0 * kPi * alpha * dt, -1.5);
    double val = 0.0;
    if (k + l <= mx) {
        double r = 2.0 * hx * (o - (G - 1)) / hxp;
        double s = 0.0;
        for (int n = 0; n <= mx; ++n) {
            double xn = cos((2.0 * n + 1.0) * kPi / (2.0 * mx + 2.0));
            double Tl = cos(l * acos(xn));
            for (int mm = 0; mm <= mx; ++mm) {
                double xm = cos((2.0 * mm + 1.0) * kPi / (2.0 * mx + 2.0));
                double z = r + xn - xm;
                s += exp(-z * z / dab) * Tl * cos(k * acos(xm));
            }
        }
        double lam = (k == 0 ? 1.0 : 2.0) * (l == 0 ? 1.0 : 2.0);
        val = lam / ((mx + 1.0) * (mx + 1.0)) * s;
    }
    E1[gid] = val;
}

void launch_e1_table(int na, int mt, int mx, int G, double hx, double hxp, double ht, double alpha, double *E1,
                     double *pref, cudaStream_t st)
{
    int m1 = mx + 1, no = 2 * G - 1;
    int total = 2 * na * na * no * m1 * m1;
    k_e1_table<<<(total + 127) / 128, 128, 0, st>>>(na, mt, mx, G, hx, hxp, ht, alpha, E1, pref);
}

// ------------------------------------------------------------------------------------------
// Regular nearfield quadrature.  Thread per (row, column) of one panel.
template <typename R, typename S, bool KOP>
__global__ void __launch_bounds__(256) k_nf_regular(NfQuadArgs a, int panel_rows0, int nrows, int rows_pad,
                                                      int cols_pad, const int *__restrict__ cols, S *__restrict__ A,
                                                      const int *__restrict__ kmap_p, int colsK_pad, int ncols)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y * blockDim.y + threadIdx.y;
    if (row >= nrows || col >= ncols) return;
    int y = cols[col];
    if (y < 0) return;
    int x = panel_rows0 + row;
    R acc[3 * 8];
#pragma unroll
    for (int i = 0; i < 3 * 8; ++i) acc[i] = R(0);
    const int d0 = nf_regular_pair<R, KOP>(a, x, y, acc);
    const int nd = a.nd;
    if (!KOP) {
        for (int d = d0; d < nd; ++d) A[((size_t)d * rows_pad + row) * cols_pad + col] = S(acc[d]);
    } else {
        for (int v = 0; v < 3; ++v) {
            int kc = kmap_p[a.tri[3 * y + v]];
            for (int d = d0; d < nd; ++d) atomicAdd(&A[((size_t)d * rows_pad + row) * colsK_pad + kc], S(acc[3 * d + v]));
        }
    }
}

template <typename R, typename S>
void launch_nf_regular_T(const NfQuadArgs &a, const PanelGPU &P, S *AV, S *AK, cudaStream_t st)
{
    dim3 blk(32, 8);
    dim3 grd((P.ncolV + 31) / 32, (P.nrows + 7) / 8);
    k_nf_regular<R, S, false><<<grd, blk, 0, st>>>(a, P.row0, P.nrows, P.rows_pad, P.colsV_pad, a.colV + P.colV_at,
                                                     AV + P.offV, nullptr, 0, P.ncolV);
    k_nf_regular<R, S, true><<<grd, blk, 0, st>>>(a, P.row0, P.nrows, P.rows_pad, P.colsV_pad, a.colV + P.colV_at,
                                                    AK + P.offK, a.kmap + (size_t)P.index * a.nv, P.colsK_pad, P.ncolV);
}

void launch_nf_regular(const NfQuadArgs &a, const PanelGPU &P, void *AV, void *AK, bool mixed, cudaStream_t st)
{
    if (mixed)
        launch_nf_regular_T<float, float>(a, P, (float *)AV, (float *)AK, st);
    else
        launch_nf_regular_T<double, double>(a, P, (double *)AV, (double *)AK, st);
}

// ------------------------------------------------------------------------------------------
// Sauter-Schwab quadrature of touching pairs at d = 0, 1: one warp per pair, FP64.
// Output: into the stored panels (AV, AK), or, when cV is given (on-the-fly nearfield), compactly
// per pair: cV[pair][d], cK[pair][d][v] (v: the source triangle's vertices in mesh order).
template <typename S>
__global__ void __launch_bounds__(128) k_nf_singular(NfQuadArgs a, const int *__restrict__ sing /*[n][12]*/, int nsing,
                                                       const PanelGPU *__restrict__ panels, S *__restrict__ AV,
                                                       S *__restrict__ AK, double *__restrict__ cV,
                                                       double *__restrict__ cK)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nsing) return;
    const int *sp = sing + 12 * warp;
    int x = sp[0], y = sp[1], panel = sp[2], row = sp[3], colV = sp[4], code = sp[5];
    int cls = code & 3;
    int ox[3] = {(code >> 2) & 3, (code >> 4) & 3, (code >> 6) & 3};
    int oy[3] = {(code >> 8) & 3, (code >> 10) & 3, (code >> 12) & 3};
    double PXo[3][3], PYo[3][3], PX[3][3], PY[3][3], ny[3], nx[3];
    load_tri(a.verts, a.tri, x, PXo);
    load_tri(a.verts, a.tri, y, PYo);
    tri_normal_orig(PYo, ny);
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c) {
            PX[v][c] = PXo[ox[v]][c];
            PY[v][c] = PYo[oy[v]][c];
        }
    double Jx = tri_jac(PX, nx), Jy = tri_jac(PY, nx);
    const int n = a.nq_sing;
    const double *gx = a.gl_sing, *gw = a.gl_sing + n;
    double accV[2] = {0, 0}, accK[2][3] = {{0, 0, 0}, {0, 0, 0}};
    const int n4 = n * n * n * n;
    for (int q = lane; q < n4; q += 32) {
        int i0 = q / (n * n * n), i1 = (q / (n * n)) % n, i2 = (q / n) % n, i3 = q % n;
        double xi = gx[i0], e1 = gx[i1], e2 = gx[i2], e3 = gx[i3];
        double w4 = gw[i0] * gw[i1] * gw[i2] * gw[i3];
        double pts[6][4], jac[6];
        const int np = ss_points(cls, xi, e1, e2, e3, pts, jac);
        for (int u = 0; u < np; ++u) {
            double xp[3], yp[3], dx[3];
            for (int c = 0; c < 3; ++c) {
                xp[c] = PX[0][c] + pts[u][0] * (PX[1][c] - PX[0][c]) + pts[u][1] * (PX[2][c] - PX[1][c]);
                yp[c] = PY[0][c] + pts[u][2] * (PY[1][c] - PY[0][c]) + pts[u][3] * (PY[2][c] - PY[1][c]);
                dx[c] = xp[c] - yp[c];
            }
            double r = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
            double wt = w4 * jac[u] * Jx * Jy;
            double vv[2], kk[2];
            time_V_all<double>(r, a.h, a.alpha, 2, vv);
            time_K_all<double>(r, a.h, a.alpha, 2, kk);
            accV[0] += wt * vv[0];
            accV[1] += wt * vv[1];
            double dn = dx[0] * ny[0] + dx[1] * ny[1] + dx[2] * ny[2];
            double byl[3] = {1.0 - pts[u][2], pts[u][2] - pts[u][3], pts[u][3]}, by[3];
            for (int v = 0; v < 3; ++v) by[oy[v]] = byl[v];
            for (int d = 0; d < 2; ++d)
                for (int v = 0; v < 3; ++v) accK[d][v] += wt * dn * kk[d] * by[v];
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        for (int d = 0; d < 2; ++d) {
            accV[d] += __shfl_xor_sync(0xffffffffu, accV[d], off);
            for (int v = 0; v < 3; ++v) accK[d][v] += __shfl_xor_sync(0xffffffffu, accK[d][v], off);
        }
    }
    if (lane == 0 && cV) {
        for (int d = 0; d < 2; ++d) {
            cV[2 * (size_t)warp + d] = d < a.nd ? accV[d] : 0.0;
            for (int v = 0; v < 3; ++v) cK[6 * (size_t)warp + 3 * d + v] = d < a.nd ? accK[d][v] : 0.0;
        }
    } else if (lane == 0) {
        const PanelGPU &P = panels[panel];
        for (int d = 0; d < 2 && d < a.nd; ++d) {
            AV[P.offV + ((size_t)d * P.rows_pad + row) * P.colsV_pad + colV] = S(accV[d]);
            for (int v = 0; v < 3; ++v)
                atomicAdd(&AK[P.offK + ((size_t)d * P.rows_pad + row) * P.colsK_pad + sp[6 + v]], S(accK[d][v]));
        }
    }
}

void launch_nf_singular(const NfQuadArgs &a, const int *sing, int nsing, const PanelGPU *panels, void *AV, void *AK,
                        bool mixed, cudaStream_t st, double *cV, double *cK)
{
    if (nsing == 0) return;
    int blocks = (nsing * 32 + 127) / 128;
    if (mixed)
        k_nf_singular<float><<<blocks, 128, 0, st>>>(a, sing, nsing, panels, (float *)AV, (float *)AK, cV, cK);
    else
        k_nf_singular<double><<<blocks, 128, 0, st>>>(a, sing, nsing, panels, (double *)AV, (double *)AK, cV, cK);
}

}  // namespace pfmm
