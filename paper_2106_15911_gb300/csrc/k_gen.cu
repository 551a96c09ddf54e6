// k_gen.cu -- kernels of the space-time FMM for general time steps (Alg. 2 on the general tree of
// Alg. 1; single layer V_h, FP64):
//   nearfield entries  Eq. eval_sl_nf_block with the entries of Section 2 for arbitrary target and
//                      source steps (collapsed Gauss rule for regular pairs, Sauter-Schwab for
//                      touching triangles on the same or the previous step);
//   nearfield apply    one CTA per leaf box over the blocks of its nearfield N(Z) (Eq.
//                      def_st_nearfield), each target element written once (no atomics);
//   S2M                Eq. s2m at every leaf of a level >= 2;
//   M2M / L2L          Eq. temp_m2m / st_m2m and their transposes with q^(t) of the actual
//                      (unequal) intervals: M2M as one CTA per child (its contribution) plus a
//                      per-parent sum in child order, L2L as one CTA per child;
//   M2L                Eq. m2l with Eq. exp_coeffs_3d in double-FP32: one CTA per target box, its
//                      warps taking (source, a) tasks over the interaction list; E as prefactor x
//                      three 1D factors tabulated per interval pair (the time nodes of unequal
//                      intervals differ pair by pair);
//   L2T                Eq. l2t at every leaf of a level >= 2.
// Every kernel is a plain grid over the boxes of one phase; phases that depend on coarser or finer
// levels are launched level by level.  Moments are staged in shared memory as dense cubes and the
// tensor-product factors are applied one direction at a time.
#include "df64.cuh"
#include "device_math.cuh"
#include "gtree.h"
#include "nf_geom.cuh"
#include "pfmm_internal.h"

namespace pfmm {

using namespace dev;

namespace {

constexpr int kGenRhs = 8;  // right-hand sides per pass of the nearfield apply

__device__ __forceinline__ void load_tri_v(const double *verts, const int *tv, double P[3][3])
{
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c) P[v][c] = verts[3 * tv[v] + c];
}

// regular pair (x, y): collapsed Gauss rule on both triangles
__device__ double gen_regular(const GenQuad &q, int x, int y, double tk0, double tk1, double tj0, double tj1)
{
    double PX[3][3], PY[3][3], n[3];
    load_tri_v(q.verts, q.tri + 3 * x, PX);
    load_tri_v(q.verts, q.tri + 3 * y, PY);
    const double Jx = tri_jac(PX, n), Jy = tri_jac(PY, n);
    const int nq = q.nq_reg;
    double acc = 0.0;
    for (int i = 0; i < nq; ++i) {
        const double s1 = q.rule_reg[i], s2 = q.rule_reg[nq + i], wi = q.rule_reg[2 * nq + i];
        double xp[3];
        for (int c = 0; c < 3; ++c) xp[c] = PX[0][c] + s1 * (PX[1][c] - PX[0][c]) + s2 * (PX[2][c] - PX[1][c]);
        for (int j = 0; j < nq; ++j) {
            const double t1 = q.rule_reg[j], t2 = q.rule_reg[nq + j], wj = q.rule_reg[2 * nq + j];
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double d = xp[c] - (PY[0][c] + t1 * (PY[1][c] - PY[0][c]) + t2 * (PY[2][c] - PY[1][c]));
                d2 += d * d;
            }
            acc += wi * wj * time_V_steps(sqrt(d2), tk0, tk1, tj0, tj1, q.alpha);
        }
    }
    return acc * Jx * Jy;
}

// touching pair (x, y) with Sauter-Schwab class and vertex order `code` (see ss_code)
__device__ double gen_singular(const GenQuad &q, int x, int y, int code, double tk0, double tk1, double tj0,
                               double tj1)
{
    const int cls = code & 3;
    const int ox[3] = {(code >> 2) & 3, (code >> 4) & 3, (code >> 6) & 3};
    const int oy[3] = {(code >> 8) & 3, (code >> 10) & 3, (code >> 12) & 3};
    double PXo[3][3], PYo[3][3], PX[3][3], PY[3][3], n[3];
    load_tri_v(q.verts, q.tri + 3 * x, PXo);
    load_tri_v(q.verts, q.tri + 3 * y, PYo);
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c) {
            PX[v][c] = PXo[ox[v]][c];
            PY[v][c] = PYo[oy[v]][c];
        }
    const double Jx = tri_jac(PX, n), Jy = tri_jac(PY, n);
    const int ns = q.nq_sing;
    const double *gx = q.gl_sing, *gw = q.gl_sing + ns;
    double acc = 0.0;
    for (int i0 = 0; i0 < ns; ++i0)
        for (int i1 = 0; i1 < ns; ++i1)
            for (int i2 = 0; i2 < ns; ++i2)
                for (int i3 = 0; i3 < ns; ++i3) {
                    double pts[6][4], jac[6];
                    const int np = ss_points(cls, gx[i0], gx[i1], gx[i2], gx[i3], pts, jac);
                    const double w4 = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    for (int u = 0; u < np; ++u) {
                        double d2 = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            const double xp = PX[0][c] + pts[u][0] * (PX[1][c] - PX[0][c]) + pts[u][1] * (PX[2][c] - PX[1][c]);
                            const double yp = PY[0][c] + pts[u][2] * (PY[1][c] - PY[0][c]) + pts[u][3] * (PY[2][c] - PY[1][c]);
                            d2 += (xp - yp) * (xp - yp);
                        }
                        acc += w4 * jac[u] * time_V_steps(sqrt(d2), tk0, tk1, tj0, tj1, q.alpha);
                    }
                }
    return acc * Jx * Jy;
}

// index of (rhs r, box b, time index a, multi-index i) in mu / lam
__device__ __forceinline__ size_t gidx(const GenDev &g, int r, int b, int a, int i)
{
    return (((size_t)r * g.nbox + b) * g.na + a) * g.nk + i;
}

}  // namespace

// one CTA per nearfield block, thread per entry [jj][y][kk][x]
__global__ void __launch_bounds__(128) k_gen_nf_entries(GenQuad q, const GBox *__restrict__ box,
                                                          const GNear *__restrict__ blocks, double *__restrict__ A)
{
    const GNear B = blocks[blockIdx.x];
    const GBox T = box[B.tgt], S = box[B.src];
    const int ntx = T.t1 - T.t0, nkt = T.a1 - T.a0, nys = S.t1 - S.t0, nks = S.a1 - S.a0;
    const int64_t n = (int64_t)ntx * nkt * nys * nks;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int x = (int)(e % ntx), kk = (int)((e / ntx) % nkt), y = (int)((e / ((int64_t)ntx * nkt)) % nys);
        const int jj = (int)(e / ((int64_t)ntx * nkt * nys));
        const int k = T.a0 + kk, j = S.a0 + jj, xi = T.t0 + x, yi = S.t0 + y;
        double v = 0.0;
        if (j <= k) {
            const double tk0 = q.ts[k], tk1 = q.ts[k + 1], tj0 = q.ts[j], tj1 = q.ts[j + 1];
            const int code = ss_code(q.tri + 3 * xi, q.tri + 3 * yi);
            v = (code && k - j <= 1) ? gen_singular(q, xi, yi, code, tk0, tk1, tj0, tj1)
                                     : gen_regular(q, xi, yi, tk0, tk1, tj0, tj1);
        }
        A[B.off + e] = v;
    }
}

void launch_gen_nf_entries(const GenQuad &q, const GBox *box, const GNear *blocks, int nblocks, double *A,
                           cudaStream_t st)
{
    if (nblocks > 0) k_gen_nf_entries<<<nblocks, 128, 0, st>>>(q, box, blocks, A);
}

// E1[p][a][b][o][kappa][nu] of Eq. exp_coeffs_1d and pref[p][a][b] = (4 pi alpha dt)^{-3/2} for the
// interval pairs p of one level: dt = xi_{I,b} - xi_{J,a} from dts[p][a][b]; thread per entry
__global__ void k_gen_e1(int npairs, const double *__restrict__ dts, int na, int mx, int G, double hx, double hxp,
                         double alpha, double *__restrict__ E1, double *__restrict__ pref)
{
    const int m1 = mx + 1, no = 2 * G - 1;
    const int64_t total = (int64_t)npairs * na * na * no * m1 * m1;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int nu = (int)(gid % m1), ka = (int)((gid / m1) % m1), o = (int)((gid / (m1 * m1)) % no);
    const int64_t pab = gid / ((int64_t)m1 * m1 * no);  // (p, a, b)
    const double dt = dts[pab];
    if (o == 0 && ka == 0 && nu == 0) pref[pab] = pow(4.0 * kPi * alpha * dt, -1.5);
    double val = 0.0;
    if (ka + nu <= mx) {
        const double r = 2.0 * hx * (o - (G - 1)) / hxp, dab = 4.0 * alpha * dt / (hxp * hxp);
        double s = 0.0;
        for (int n = 0; n <= mx; ++n) {
            const double xn = cos((2.0 * n + 1.0) * kPi / (2.0 * mx + 2.0)), Tn = cos(nu * acos(xn));
            for (int m = 0; m <= mx; ++m) {
                const double xm = cos((2.0 * m + 1.0) * kPi / (2.0 * mx + 2.0)), z = r + xn - xm;
                s += exp(-z * z / dab) * Tn * cos(ka * acos(xm));
            }
        }
        val = (ka == 0 ? 1.0 : 2.0) * (nu == 0 ? 1.0 : 2.0) / ((mx + 1.0) * (mx + 1.0)) * s;
    }
    E1[gid] = val;
}

void launch_gen_e1(int npairs, const double *dts, int na, int mx, int G, double hx, double hxp, double alpha,
                   double *E1, double *pref, cudaStream_t st)
{
    const int64_t total = (int64_t)npairs * na * na * (2 * G - 1) * (mx + 1) * (mx + 1);
    if (total > 0)
        k_gen_e1<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(npairs, dts, na, mx, G, hx, hxp, alpha, E1, pref);
}

// w_int[row][i] = w[row][perm[i]], f[row][perm[i]] = f_int[row][i]
__global__ void k_gen_permute_in(const double *__restrict__ w, double *__restrict__ w_int, const int *__restrict__ perm,
                                 int nt, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w_int[i] = w[i - i % nt + perm[i % nt]];
}
__global__ void k_gen_permute_out(const double *__restrict__ f_int, double *__restrict__ f, const int *__restrict__ perm,
                                  int nt, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i - i % nt + perm[i % nt]] = f_int[i];
}
void launch_gen_permute_in(const double *w, double *w_int, const int *perm, int nt, int rows, cudaStream_t st)
{
    const int64_t n = (int64_t)nt * rows;
    if (n > 0) k_gen_permute_in<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, w_int, perm, nt, n);
}
void launch_gen_permute_out(const double *f_int, double *f, const int *perm, int nt, int rows, cudaStream_t st)
{
    const int64_t n = (int64_t)nt * rows;
    if (n > 0) k_gen_permute_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f_int, f, perm, nt, n);
}

// f_int[r][k][x] = sum over the blocks of the leaf of A[jj][y][kk][x] w_int[r][j][y] (entries with
// j > k are stored as zeros).  The target elements e = kk ntx + x of the leaf go 32 at a time to the
// lanes; the 8 warps of the CTA take every 8th source column (jj, y) of the leaf's blocks (the
// column's 32 entries are one coalesced load) and their partial sums are added in warp order.
constexpr int kGenNfWarps = 8;
template <int R>
__global__ void __launch_bounds__(32 * kGenNfWarps) k_gen_nf_apply(const GBox *__restrict__ box,
                                                                    const int *__restrict__ leaves,
                                                                    const int *__restrict__ nptr,
                                                                    const GNear *__restrict__ blocks,
                                                                    const double *__restrict__ A,
                                                                    const double *__restrict__ w_int,
                                                                    double *__restrict__ f_int, int nt, int Et, int r0)
{
    __shared__ double red[kGenNfWarps][R][32];
    const int b = leaves[blockIdx.x];
    const GBox T = box[b];
    const int ntx = T.t1 - T.t0, ne = ntx * (T.a1 - T.a0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t per_rhs = (size_t)Et * nt;
    for (int e0 = 0; e0 < ne; e0 += 32) {
        const int e = e0 + lane;
        const bool valid = e < ne;
        double acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.0;
        for (int q = nptr[b]; q < nptr[b + 1]; ++q) {
            const GNear B = blocks[q];
            const GBox S = box[B.src];
            const int nys = S.t1 - S.t0, ncol = nys * (S.a1 - S.a0);
            const double *Ab = A + B.off + (valid ? e : 0);
            const double *w0 = w_int + (size_t)r0 * per_rhs + (size_t)S.a0 * nt + S.t0;
            int jj = warp / nys, y = warp - jj * nys;  // column c = jj nys + y, advanced by kGenNfWarps
#pragma unroll 4
            for (int c = warp; c < ncol; c += kGenNfWarps) {
                const double a = valid ? Ab[(size_t)c * ne] : 0.0;
                const double *wj = w0 + (size_t)jj * nt + y;
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fma(a, wj[(size_t)r * per_rhs], acc[r]);
                y += kGenNfWarps;
                while (y >= nys) {
                    y -= nys;
                    ++jj;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) red[warp][r][lane] = acc[r];
        __syncthreads();
        if (warp == 0 && valid) {
            const int kk = e / ntx, x = e - kk * ntx;
            for (int r = 0; r < R; ++r) {
                double s = 0.0;
                for (int w = 0; w < kGenNfWarps; ++w) s += red[w][r][lane];
                f_int[(size_t)(r0 + r) * per_rhs + (size_t)(T.a0 + kk) * nt + T.t0 + x] = s;
            }
        }
        __syncthreads();
    }
}

void launch_gen_nf_apply(const GBox *box, const int *leaves, int nleaves, const int *nptr, const GNear *blocks,
                         const double *A, const double *w_int, double *f_int, int nt, int Et, int nrhs,
                         cudaStream_t st)
{
    if (nleaves <= 0) return;
    const dim3 grid(nleaves), blk(32 * kGenNfWarps);
    for (int r0 = 0; r0 < nrhs;) {
        const int n = nrhs - r0;
        if (n >= 4) {
            k_gen_nf_apply<4><<<grid, blk, 0, st>>>(box, leaves, nptr, blocks, A, w_int, f_int, nt, Et, r0);
            r0 += 4;
        } else if (n >= 2) {
            k_gen_nf_apply<2><<<grid, blk, 0, st>>>(box, leaves, nptr, blocks, A, w_int, f_int, nt, Et, r0);
            r0 += 2;
        } else {
            k_gen_nf_apply<1><<<grid, blk, 0, st>>>(box, leaves, nptr, blocks, A, w_int, f_int, nt, Et, r0);
            r0 += 1;
        }
    }
}

// mu[r][b][a][kappa] = sum_j St[l][j][a] sum_x Sx[slot][x][kappa] w_int[r][j][x]  (Eq. s2m)
__global__ void __launch_bounds__(128) k_gen_s2m(GenDev g, const int *__restrict__ leaves,
                                                   const double *__restrict__ w_int)
{
    const int b = leaves[blockIdx.x];
    const GBox B = g.box[b];
    const double *Sx = g.Sx + (size_t)B.sx * g.nt * g.nk, *St = g.St + (size_t)B.level * g.Et * g.na;
    const size_t per_rhs = (size_t)g.Et * g.nt;
    for (int r = 0; r < g.nrhs; ++r)
        for (int ik = threadIdx.x; ik < g.nk; ik += blockDim.x) {
            double acc[kMaxNa];
            for (int a = 0; a < g.na; ++a) acc[a] = 0.0;
            for (int j = B.a0; j < B.a1; ++j) {
                const double *w = w_int + r * per_rhs + (size_t)j * g.nt;
                double Q = 0.0;
                for (int x = B.t0; x < B.t1; ++x) Q += Sx[(size_t)x * g.nk + ik] * w[x];
                for (int a = 0; a < g.na; ++a) acc[a] += St[(size_t)j * g.na + a] * Q;
            }
            for (int a = 0; a < g.na; ++a) g.mu[gidx(g, r, b, a, ik)] = acc[a];
        }
}

void launch_gen_s2m(const GenDev &g, const int *leaves, int n, const double *w_int, cudaStream_t st)
{
    if (n > 0) k_gen_s2m<<<n, 128, 0, st>>>(g, leaves, w_int);
}

// M2M in two launches per level, deterministic: each child Z_c writes its contribution
//   contrib(Z_c)[ap][nu] = sum_ac q^(t)_{ac,ap} (sum_{kappa <= nu} q^(x)_{kappa,nu} mu(Z_c)[ac][kappa])
// (Eq. st_m2m; Eq. temp_m2m when refined in time only: kappa = nu), one CTA per child with its moments
// staged as dense cubes [ac][m1^3] and the 1D factors applied one direction at a time; then every
// parent adds its children's contributions in child order.
constexpr int kGenPassThreads = 256;
__global__ void __launch_bounds__(kGenPassThreads) k_gen_m2m_child(GenDev g, const int *__restrict__ children,
                                                                    double *__restrict__ contrib)
{
    extern __shared__ double sm[];
    const int na = g.na, nk = g.nk, m1 = g.mx + 1, m3 = m1 * m1 * m1;
    double *sc = sm;  // [na][m1^3]
    const int c = children[blockIdx.x];
    const GBox C = g.box[c];
    const int st = g.lvst[C.level];
    const double *q1 = g.q1 + (size_t)C.level * 2 * m1 * m1;
    const double *qa = q1 + (size_t)(C.bits & 1) * m1 * m1, *qb = q1 + (size_t)((C.bits >> 1) & 1) * m1 * m1,
                 *qc = q1 + (size_t)((C.bits >> 2) & 1) * m1 * m1;
    const double *qtc = g.qt + (size_t)c * na * na;
    for (int r = 0; r < g.nrhs; ++r) {
        __syncthreads();
        for (int i = threadIdx.x; i < na * nk; i += blockDim.x) {
            const int a = i / nk, ik = i - a * nk;
            sc[a * m3 + (g.kidx[3 * ik] * m1 + g.kidx[3 * ik + 1]) * m1 + g.kidx[3 * ik + 2]] =
                g.mu[gidx(g, r, c, 0, 0) + i];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < na * nk; t += blockDim.x) {
            const int ap = t / nk, iv = t - ap * nk;
            const int n0 = g.kidx[3 * iv], n1 = g.kidx[3 * iv + 1], n2 = g.kidx[3 * iv + 2];
            double sum = 0.0;
            for (int ac = 0; ac < na; ++ac) {
                const double *cube = sc + ac * m3;
                double v;
                if (!st) {
                    v = cube[(n0 * m1 + n1) * m1 + n2];
                } else {
                    v = 0.0;
                    for (int k0 = 0; k0 <= n0; ++k0) {
                        double v1 = 0.0;
                        for (int k1 = 0; k1 <= n1; ++k1) {
                            const double *row = cube + (k0 * m1 + k1) * m1;
                            double v2 = 0.0;
                            for (int k2 = 0; k2 <= n2; ++k2) v2 += qc[k2 * m1 + n2] * row[k2];
                            v1 += qb[k1 * m1 + n1] * v2;
                        }
                        v += qa[k0 * m1 + n0] * v1;
                    }
                }
                sum += qtc[ac * na + ap] * v;
            }
            contrib[gidx(g, r, c, 0, 0) + t] = sum;
        }
    }
}

__global__ void k_gen_m2m_sum(GenDev g, const int *__restrict__ parents, const double *__restrict__ contrib)
{
    const int bp = parents[blockIdx.x];
    const GBox P = g.box[bp];
    for (int r = 0; r < g.nrhs; ++r)
        for (int t = threadIdx.x; t < g.na * g.nk; t += blockDim.x) {
            double s = 0.0;
            for (int c = P.c0; c < P.c1; ++c) s += contrib[gidx(g, r, c, 0, 0) + t];
            g.mu[gidx(g, r, bp, 0, 0) + t] = s;
        }
}

size_t gen_pass_smem(int na, int mx) { return sizeof(double) * (size_t)na * (mx + 1) * (mx + 1) * (mx + 1); }

void launch_gen_m2m(const GenDev &g, const int *parents, int n, const int *children, int nc, double *contrib,
                    cudaStream_t st)
{
    if (n <= 0 || nc <= 0) return;
    const size_t smem = gen_pass_smem(g.na, g.mx);
    cudaFuncSetAttribute(k_gen_m2m_child, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gen_m2m_child<<<nc, kGenPassThreads, smem, st>>>(g, children, contrib);
    k_gen_m2m_sum<<<n, 128, 0, st>>>(g, parents, contrib);
}

// lam(Z)[b][nu] = sum over I(Z) of sum_a pref[a][b] sum_{|kappa + nu| <= m_x} prod_d E1_d mu(Z_s)[a][kappa]
// (Eq. m2l with Eq. exp_coeffs_3d; E1 of the pair's intervals, offsets of the cells per direction),
// in double-FP32 (pairs of floats, about 48 significant bits: the FP32 pipe issues such operations
// several times faster than GB300's FP64 pipe) from tables converted once (Edf, prefdf, mudf).
// One CTA per target box, 8 warps working independently: a warp takes the tasks (source, a) in
// turn, stages the source's moment cube mu(Z_s)[a] and the 1D factor slices of all b in its own
// shared memory, and its lanes sum for nu = lane, lane + 32, ... over the simplex |kappa| <= m_x -
// |nu| one direction at a time; the warps' partial sums are added in warp order at the end.
constexpr int kGenM2lWarps = 8;
constexpr int kGenM2lSlots = 64;  // items (b, nu) per lane: na nk <= 2048 (checked at creation)

// item t of the (b, nu) list in degree-major order: all (b, nu) with |nu| = 0, then |nu| = 1, ...
// (so the 32 lanes of a slot mostly share |nu| and run loops of one length)
__device__ __forceinline__ void m2l_item(int t, int na, int &b, int &iv)
{
    int sdeg = 0;
    while (true) {
        const int grp = (sdeg + 1) * (sdeg + 2) / 2;  // multi-indices of degree sdeg
        if (t < na * grp) {
            b = t / grp;
            iv = sdeg * (sdeg + 1) * (sdeg + 2) / 6 + t % grp;  // its place in the degree-graded order
            return;
        }
        t -= na * grp;
        ++sdeg;
    }
}

__global__ void __launch_bounds__(32 * kGenM2lWarps) k_gen_m2l(GenDev g, const int *__restrict__ targets,
                                                                const int *__restrict__ mptr,
                                                                const GPair *__restrict__ pairs,
                                                                const df64 *__restrict__ Edf,
                                                                const int64_t *__restrict__ e1off,
                                                                const df64 *__restrict__ prefdf,
                                                                const df64 *__restrict__ mudf)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int na = g.na, nk = g.nk, m1 = g.mx + 1, mm = m1 * m1, m3 = mm * m1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_warp = m3 + 3 * na * mm;  // cube + slices of all b
    df64 *cube = (df64 *)smraw + (size_t)warp * per_warp, *sE = cube + m3;  // sE [b][d][m1][m1]
    const int bt = targets[blockIdx.x];
    const GBox T = g.box[bt];
    const int G = g.lvG[T.level], no = 2 * G - 1;
    const int nsrc = mptr[bt + 1] - mptr[bt];
    const int nitem = na * nk, nslot = (nitem + 31) / 32;
    for (int r = 0; r < g.nrhs; ++r) {
        df64 acc[kGenM2lSlots];
        for (int sl = 0; sl < nslot; ++sl) acc[sl] = df64(0);
        for (int task = warp; task < nsrc * na; task += kGenM2lWarps) {
            const int q = mptr[bt] + task / na, a = task % na;
            const GPair pr = pairs[q];
            const GBox S = g.box[pr.src];
            const int o[3] = {T.cell[0] - S.cell[0] + G - 1, T.cell[1] - S.cell[1] + G - 1, T.cell[2] - S.cell[2] + G - 1};
            __syncwarp();
            const df64 *ms = mudf + gidx(g, r, pr.src, a, 0);
            for (int ik = lane; ik < nk; ik += 32)
                cube[(g.kidx[3 * ik] * m1 + g.kidx[3 * ik + 1]) * m1 + g.kidx[3 * ik + 2]] = ms[ik];
            const df64 *Ep = Edf + e1off[pr.e];
            for (int b = 0; b < na; ++b)
                for (int d = 0; d < 3; ++d) {
                    const df64 *src = Ep + ((size_t)(a * na + b) * no + o[d]) * mm;
                    df64 *dst = sE + (size_t)(b * 3 + d) * mm;
                    for (int kv = lane; kv < mm; kv += 32) dst[kv] = src[kv];
                }
            __syncwarp();
            const df64 *pf = prefdf + (size_t)pr.e * na * na + a * na;
            for (int sl = 0; sl < nslot; ++sl) {
                const int t = lane + 32 * sl;
                if (t >= nitem) break;
                int b, iv;
                m2l_item(t, na, b, iv);
                const int n0 = g.kidx[3 * iv], n1 = g.kidx[3 * iv + 1], n2 = g.kidx[3 * iv + 2];
                const int dd = g.mx - (n0 + n1 + n2);
                const df64 *E0 = sE + (size_t)(b * 3) * mm, *Ea = E0 + mm, *Eb = Ea + mm;
                df64 v0(0);
                for (int k0 = 0; k0 <= dd; ++k0) {
                    df64 v1(0);
                    for (int k1 = 0; k1 <= dd - k0; ++k1) {
                        const df64 *row = cube + (k0 * m1 + k1) * m1;
                        df64 v2(0);
                        for (int k2 = 0; k2 <= dd - k0 - k1; ++k2) mac(v2, Eb[k2 * m1 + n2], row[k2]);
                        mac(v1, Ea[k1 * m1 + n1], v2);
                    }
                    mac(v0, E0[k0 * m1 + n0], v1);
                }
                mac(acc[sl], pf[b], v0);
            }
        }
        // the warps' partial sums, added in warp order (the staging area is reused)
        __syncthreads();
        df64 *red = (df64 *)smraw;  // [warps][items]
        for (int sl = 0; sl < nslot; ++sl) {
            const int t = lane + 32 * sl;
            if (t < nitem) red[(size_t)warp * nitem + t] = acc[sl];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nitem; t += blockDim.x) {
            df64 sum = red[t];
            for (int w = 1; w < kGenM2lWarps; ++w) sum += red[(size_t)w * nitem + t];
            int b, iv;
            m2l_item(t, na, b, iv);
            g.lam[gidx(g, r, bt, b, iv)] = as_double(sum);
        }
        __syncthreads();
    }
}

// double -> double-FP32 copies of the M2L operands
__global__ void k_gen_to_df64(const double *__restrict__ x, df64 *__restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = df64(x[i]);
}

void launch_gen_to_df64(const double *x, void *y, int64_t n, cudaStream_t st)
{
    if (n > 0) k_gen_to_df64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, (df64 *)y, n);
}

size_t gen_m2l_smem(int na, int nk, int mx)
{
    const size_t m1 = mx + 1, stage = (size_t)kGenM2lWarps * (m1 * m1 * m1 + 3 * (size_t)na * m1 * m1),
                 red = (size_t)kGenM2lWarps * na * nk;
    return sizeof(df64) * (stage > red ? stage : red);
}

void launch_gen_m2l(const GenDev &g, const int *targets, int n, const int *mptr, const GPair *pairs,
                    const void *Edf, const int64_t *e1off, const void *prefdf, const void *mudf, cudaStream_t st)
{
    if (n <= 0) return;
    const size_t smem = gen_m2l_smem(g.na, g.nk, g.mx);
    cudaFuncSetAttribute(k_gen_m2l, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gen_m2l<<<n, 32 * kGenM2lWarps, smem, st>>>(g, targets, mptr, pairs, (const df64 *)Edf, e1off,
                                                   (const df64 *)prefdf, (const df64 *)mudf);
}

// lam(Z_c)[bc][kappa] += sum_bp q^(t)_{bc,bp} sum_{nu >= kappa, |nu| <= m_x} q^(x)_{kappa,nu} lam(Z_p)[bp][nu]
// (the transposes of Eq. temp_m2m / st_m2m).  One CTA per child; the parent's local contributions
// are staged as dense cubes and summed one direction at a time.
__global__ void __launch_bounds__(kGenPassThreads) k_gen_l2l(GenDev g, const int *__restrict__ children)
{
    extern __shared__ double sm[];
    const int na = g.na, nk = g.nk, m1 = g.mx + 1, m3 = m1 * m1 * m1;
    double *sp = sm;  // [na][m1^3]
    const int bc = children[blockIdx.x];
    const GBox C = g.box[bc];
    const int st = g.lvst[C.level], bp = C.par;
    const double *q1 = g.q1 + (size_t)C.level * 2 * m1 * m1;
    const double *qa = q1 + (size_t)(C.bits & 1) * m1 * m1, *qb = q1 + (size_t)((C.bits >> 1) & 1) * m1 * m1,
                 *qc = q1 + (size_t)((C.bits >> 2) & 1) * m1 * m1;
    const double *qtc = g.qt + (size_t)bc * na * na;
    for (int r = 0; r < g.nrhs; ++r) {
        __syncthreads();
        for (int i = threadIdx.x; i < na * nk; i += blockDim.x) {
            const int a = i / nk, ik = i - a * nk;
            sp[a * m3 + (g.kidx[3 * ik] * m1 + g.kidx[3 * ik + 1]) * m1 + g.kidx[3 * ik + 2]] =
                g.lam[gidx(g, r, bp, 0, 0) + i];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < na * nk; t += blockDim.x) {
            const int bcI = t / nk, ik = t - bcI * nk;
            const int k0 = g.kidx[3 * ik], k1 = g.kidx[3 * ik + 1], k2 = g.kidx[3 * ik + 2];
            double acc = 0.0;
            for (int bpI = 0; bpI < na; ++bpI) {
                const double *cube = sp + bpI * m3;
                double v;
                if (!st) {
                    v = cube[(k0 * m1 + k1) * m1 + k2];
                } else {
                    v = 0.0;
                    for (int n0 = k0; n0 <= g.mx; ++n0) {
                        double v1 = 0.0;
                        for (int n1 = k1; n0 + n1 <= g.mx; ++n1) {
                            const double *row = cube + (n0 * m1 + n1) * m1;
                            double v2 = 0.0;
                            for (int n2 = k2; n0 + n1 + n2 <= g.mx; ++n2) v2 += qc[k2 * m1 + n2] * row[n2];
                            v1 += qb[k1 * m1 + n1] * v2;
                        }
                        v += qa[k0 * m1 + n0] * v1;
                    }
                }
                acc += qtc[bcI * na + bpI] * v;
            }
            g.lam[gidx(g, r, bc, bcI, ik)] += acc;
        }
    }
}

void launch_gen_l2l(const GenDev &g, const int *children, int n, cudaStream_t st)
{
    if (n <= 0) return;
    const size_t smem = gen_pass_smem(g.na, g.mx);
    cudaFuncSetAttribute(k_gen_l2l, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gen_l2l<<<n, kGenPassThreads, smem, st>>>(g, children);
}

// f_int[r][k][x] += sum_b St[l][k][b] sum_nu lam(Z)[b][nu] Sx[slot][x][nu]  (Eq. l2t)
__global__ void __launch_bounds__(128) k_gen_l2t(GenDev g, const int *__restrict__ leaves, double *__restrict__ f_int)
{
    const int b = leaves[blockIdx.x];
    const GBox B = g.box[b];
    const double *Sx = g.Sx + (size_t)B.sx * g.nt * g.nk, *St = g.St + (size_t)B.level * g.Et * g.na;
    const size_t per_rhs = (size_t)g.Et * g.nt;
    for (int r = 0; r < g.nrhs; ++r)
        for (int x = B.t0 + threadIdx.x; x < B.t1; x += blockDim.x) {
            double P[kMaxNa];
            for (int bb = 0; bb < g.na; ++bb) {
                double s = 0.0;
                for (int iv = 0; iv < g.nk; ++iv) s += g.lam[gidx(g, r, b, bb, iv)] * Sx[(size_t)x * g.nk + iv];
                P[bb] = s;
            }
            for (int k = B.a0; k < B.a1; ++k) {
                double v = 0.0;
                for (int bb = 0; bb < g.na; ++bb) v += St[(size_t)k * g.na + bb] * P[bb];
                f_int[r * per_rhs + (size_t)k * g.nt + x] += v;
            }
        }
}

void launch_gen_l2t(const GenDev &g, const int *leaves, int n, double *f_int, cudaStream_t st)
{
    if (n > 0) k_gen_l2t<<<n, 128, 0, st>>>(g, leaves, f_int);
}

}  // namespace pfmm
