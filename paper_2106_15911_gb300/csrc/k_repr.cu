// k_repr.cu -- the representation formula of Section 2 at interior space-time points:
//   u(x, t) = (V~ w)(x, t) - (W g)(x, t),
//   V~ w = int_0^t int_Gamma G(x - y, t - tau) w(y, tau),  W g = int_0^t int_Gamma alpha dG/dn_y g,
// for the discrete data of the boundary integral equation (w piecewise constant on the space-time
// elements, g piecewise constant in time and nodal in space).  Over step j the time integrals are
// differences of first antiderivatives in s = t - tau:
//   int G(r, s) ds       -> G1(r, s) = erfc(u) / (4 pi alpha r),
//   int G(r, s) / (2 s)  -> H1(r, s) = [erfc(u) + 2 u e^{-u^2} / sqrt(pi)] / (4 pi r^3),
// u = r / (2 sqrt(alpha s)), 0 for s <= 0 (causality); the double-layer integrand is
// (x - y).n_y G / (2 s).  Space: the handle's collapsed Gauss rule on every triangle.  One CTA per
// (point, rhs): threads stride over (triangle, quadrature point) pairs, each runs the step loop
// with one new G1 / H1 evaluation per step (the upper limit of step j is the lower one of step
// j + 1), and the CTA sums its threads in a fixed tree order (deterministic).  FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>

#include "kernels.h"

namespace pfmm {

namespace {

constexpr double kPiR = 3.14159265358979323846;

__device__ __forceinline__ void g1h1(double r, double s, double alpha, double &g1, double &h1)
{
    if (s <= 0.0) {
        g1 = h1 = 0.0;
        return;
    }
    const double u = r / (2.0 * sqrt(alpha * s)), ec = erfc(u);
    g1 = ec / (4.0 * kPiR * alpha * r);
    h1 = (ec + 2.0 * u * exp(-u * u) / sqrt(kPiR)) / (4.0 * kPiR * r * r * r);
}

}  // namespace

__global__ void __launch_bounds__(256) k_repr(const double *__restrict__ verts, const int *__restrict__ tri, int nt,
                                                int nv, const double *__restrict__ rule, int nq,
                                                const double *__restrict__ w, const double *__restrict__ g,
                                                const double *__restrict__ pts, int np, int Et, double h, double alpha,
                                                double *__restrict__ u)
{
    __shared__ double red[256];
    const int p = blockIdx.x, rhs = blockIdx.y;
    const double x0 = pts[4 * p], x1 = pts[4 * p + 1], x2 = pts[4 * p + 2], t = pts[4 * p + 3];
    const double *wr = w + (size_t)rhs * Et * nt;
    const double *gr = g ? g + (size_t)rhs * Et * nv : nullptr;
    const int jmax = t > 0.0 ? min(Et, (int)ceil(t / h)) : 0;  // steps with t_{j-1} < t
    double acc = 0.0;
    for (int e = threadIdx.x; e < nt * nq; e += blockDim.x) {
        const int tr = e / nq, q = e - tr * nq;
        const int v0 = tri[3 * tr], v1 = tri[3 * tr + 1], v2 = tri[3 * tr + 2];
        const double *P0 = verts + 3 * v0, *P1 = verts + 3 * v1, *P2 = verts + 3 * v2;
        const double a0 = P1[0] - P0[0], a1 = P1[1] - P0[1], a2 = P1[2] - P0[2];
        const double b0 = P2[0] - P0[0], b1 = P2[1] - P0[1], b2 = P2[2] - P0[2];
        double n0 = a1 * b2 - a2 * b1, n1 = a2 * b0 - a0 * b2, n2 = a0 * b1 - a1 * b0;
        const double jac = sqrt(n0 * n0 + n1 * n1 + n2 * n2);  // 2 |gamma|
        n0 /= jac;
        n1 /= jac;
        n2 /= jac;
        const double s1 = rule[q], s2 = rule[nq + q], wq = rule[2 * nq + q] * jac;
        // y = P0 + s1 (P1 - P0) + s2 (P2 - P1): barycentric weights 1 - s1, s1 - s2, s2
        const double y0 = P0[0] + s1 * a0 + s2 * (P2[0] - P1[0]);
        const double y1 = P0[1] + s1 * a1 + s2 * (P2[1] - P1[1]);
        const double y2 = P0[2] + s1 * a2 + s2 * (P2[2] - P1[2]);
        const double d0 = x0 - y0, d1 = x1 - y1, d2 = x2 - y2;
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2), dn = d0 * n0 + d1 * n1 + d2 * n2;
        const double f0 = 1.0 - s1, f1 = s1 - s2, f2 = s2;
        double gA, hA;  // antiderivatives at the step's lower limit tau = t_{j-1}
        g1h1(r, t, alpha, gA, hA);
        double sum = 0.0;
        for (int j = 1; j <= jmax; ++j) {
            double gB, hB;  // at tau = t_j
            g1h1(r, t - j * h, alpha, gB, hB);
            double v = wr[(size_t)(j - 1) * nt + tr] * (gA - gB);
            if (gr) {
                const double *gj = gr + (size_t)(j - 1) * nv;
                v -= dn * (hA - hB) * (gj[v0] * f0 + gj[v1] * f1 + gj[v2] * f2);
            }
            sum += v;
            gA = gB;
            hA = hB;
        }
        acc += wq * sum;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) u[(size_t)rhs * np + p] = red[0];
}

void launch_repr(const double *verts, const int *tri, int nt, int nv, const double *rule, int nq, const double *w,
                 const double *g, const double *pts, int np, int nrhs, int Et, double h, double alpha, double *u,
                 cudaStream_t st)
{
    if (np > 0) k_repr<<<dim3((unsigned)np, (unsigned)nrhs), 256, 0, st>>>(verts, tri, nt, nv, rule, nq, w, g, pts, np,
                                                                            Et, h, alpha, u);
}

}  // namespace pfmm
