// k_apply.cu -- the per-matvec kernels of Alg. 2 (Section 3.4).
//
// Layouts (per right-hand side r):
//   w_int[r][t][i]        input in internal triangle order (triangles grouped by leaf box)
//   g[r][t][node]         double-layer input in the caller's node order
//   f_int[r][t][i]        FP64 output in internal order
//   mu_l[r][k][b][a][i]   moments of level l: interval k, spatial box b, time node a, graded
//                         multi-index i (all kappa with |kappa| <= q come first)
//   lam_l                 local contributions, same layout
// R is the arithmetic type of the FMM passes: float in mixed mode, df64 (double-FP32, about 48
// significant bits on the FP32 pipe) in FP64 mode, or double when native FP64 passes are asked for;
// outputs accumulate in FP64.  The stored nearfield blocks are float (mixed) or double (FP64).
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>
#include <cstdio>

#include "df64.cuh"
#include "device_math.cuh"
#include "kernels.h"

namespace pfmm {

// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_permute_in(const double *__restrict__ w, T *__restrict__ wi, const int *__restrict__ perm, int nt,
                             size_t total)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    size_t rt = gid / nt;
    int i = (int)(gid - rt * nt);
    wi[gid] = T(w[rt * nt + perm[i]]);
}

void launch_permute_in(const double *w, void *w_int, bool to_float, int nrhs, const ApplyGeo &g, cudaStream_t st)
{
    size_t total = (size_t)nrhs * g.Et * g.nt;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (to_float)
        k_permute_in<float><<<blocks, 256, 0, st>>>(w, (float *)w_int, g.perm, g.nt, total);
    else
        k_permute_in<double><<<blocks, 256, 0, st>>>(w, (double *)w_int, g.perm, g.nt, total);
}

__global__ void k_permute_out(const double *__restrict__ fi, double *__restrict__ f, const int *__restrict__ perm, int nt,
                              size_t total)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    size_t rt = gid / nt;
    int i = (int)(gid - rt * nt);
    f[rt * nt + perm[i]] = fi[gid];
}

void launch_permute_out(const double *f_int, double *f, int nrhs, const ApplyGeo &g, cudaStream_t st)
{
    size_t total = (size_t)nrhs * g.Et * g.nt;
    k_permute_out<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(f_int, f, g.perm, g.nt, total);
}

__global__ void k_cast(const double *__restrict__ x, float *__restrict__ y, size_t n)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < n) y[gid] = (float)x[gid];
}

void launch_cast_to_float(const double *x, float *y, size_t n, cudaStream_t st)
{
    k_cast<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
}

__global__ void k_to_df64(double *__restrict__ x, size_t n)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < n) {
        const df64 v(x[gid]);
        reinterpret_cast<float2 *>(x)[gid] = make_float2(v.hi, v.lo);
    }
}

void launch_to_df64(double *x, size_t n, cudaStream_t st)
{
    if (n) k_to_df64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n);
}

// ------------------------------------------------------------------------------------------
// Nearfield apply (Alg. 2, last loop; Eq. eval_sl_nf_block) with the block-Toeplitz structure
// of uniform steps: for target step t = k*ls + s of leaf interval k the temporal nearfield
// N(I_k) = {I_{k-1}, I_k} contributes the step offsets d = 0 .. ls + s, so
//   f[t][rows of X] = sum_{d=0}^{ls+s} A_d[X] x[t - d][cols of X].
// One CTA computes a 64 x 64 tile (64 rows of a panel x 64 steps of one phase s) over all d
// and all columns, so every output element is written exactly once.
template <typename S>
__global__ void __launch_bounds__(256) k_nf_apply(const S *__restrict__ A, const int *__restrict__ colidx,
                                                    const int *__restrict__ tiles, const PanelGPU *__restrict__ panels,
                                                    const S *__restrict__ x, int ncolg, int Et, int ls, int nint,
                                                    double *__restrict__ f, int nt, int kop, int ndmax,
                                                    NfHalfSplit hs)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    constexpr bool kFloat = sizeof(S) == 4;
    __shared__ S As[BK][BM + 1];
    __shared__ S Ws[BK][BN + 1];
    const int tid = threadIdx.x;
    const int rg = tid & 15, cg = tid >> 4;
    const PanelGPU P = panels[tiles[2 * blockIdx.x]];
    const int r0 = tiles[2 * blockIdx.x + 1];
    const int s = blockIdx.y % ls, ib = blockIdx.y / ls;
    const int rhs = blockIdx.z;
    const S *xr = x + (size_t)rhs * Et * ncolg;
    const int *cols = colidx + (kop ? P.colK_at : P.colV_at);
    const int ncp = kop ? P.colsK_pad : P.colsV_pad;
    const bool half = hs.hi != nullptr;  // FP32 only
    const size_t off = kop ? P.offK : P.offV;
    const __half *Hh = reinterpret_cast<const __half *>(hs.hi), *Hl = reinterpret_cast<const __half *>(hs.lo);
    S acc[4][4];
    double accd[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = S(0);
            accd[i][j] = 0.0;
        }
    const int nd = min(ls + s + 1, ndmax);
    int ktiles = 0;
    for (int d = 0; d < nd; ++d) {
        const size_t dbase = off + ((size_t)d * P.rows_pad + r0) * ncp;
        const size_t rbase = off / ncp + (size_t)d * P.rows_pad + r0;  // global row (FP16 parts)
        for (int k0 = 0; k0 < ncp; k0 += BK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int e = tid + 256 * q;
                int i = e >> 4, j = e & 15;
                if (half) {
                    const size_t ia = nf_tiled_index(rbase + i, k0 + j, ncp >> 6);
                    As[j][i] = S((__half2float(Hh[ia]) + __half2float(Hl[ia])) * hs.inv_scale);
                } else {
                    As[j][i] = A[dbase + (size_t)i * ncp + k0 + j];
                }
                int c = e >> 4;
                int t = ((ib * BN + c) * ls + s);
                int col = cols[k0 + j];
                S v = S(0);
                if (col >= 0 && ib * BN + c < nint && t - d >= 0) v = xr[(size_t)(t - d) * ncolg + col];
                Ws[j][c] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < BK; ++j) {
                S a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = As[j][rg + 16 * q];
                    b[q] = Ws[j][cg + 16 * q];
                }
#pragma unroll
                for (int qi = 0; qi < 4; ++qi)
#pragma unroll
                    for (int qj = 0; qj < 4; ++qj) acc[qi][qj] += a[qi] * b[qj];
            }
            __syncthreads();
            if (kFloat && ++ktiles == 32) {  // FP32 partial sums over 512 columns, then FP64
                ktiles = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        accd[i][j] += (double)acc[i][j];
                        acc[i][j] = S(0);
                    }
            }
        }
    }
#pragma unroll
    for (int qj = 0; qj < 4; ++qj) {
        int iv = ib * BN + cg + 16 * qj;
        if (iv >= nint) continue;
        int t = iv * ls + s;
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
            int row = r0 + rg + 16 * qi;
            if (row < P.nrows) f[((size_t)rhs * Et + t) * nt + P.row0 + row] = accd[qi][qj] + (double)acc[qi][qj];
        }
    }
}

void launch_nf_apply(bool mixed, bool kop, const void *A, const int *colidx, const int *tiles, int ntiles,
                     const PanelGPU *panels, const void *x, int ncolg, int nrhs, const ApplyGeo &g, double *f_int,
                     cudaStream_t st, int ndmax, const NfHalfSplit *hs)
{
    int nint = g.Et / g.ls;
    dim3 grd(ntiles, g.ls * ((nint + 63) / 64), nrhs);
    if (mixed)
        k_nf_apply<float><<<grd, 256, 0, st>>>((const float *)A, colidx, tiles, panels, (const float *)x, ncolg, g.Et,
                                               g.ls, nint, f_int, g.nt, kop ? 1 : 0, ndmax, hs ? *hs : NfHalfSplit{});
    else
        k_nf_apply<double><<<grd, 256, 0, st>>>((const double *)A, colidx, tiles, panels, (const double *)x, ncolg,
                                                g.Et, g.ls, nint, f_int, g.nt, kop ? 1 : 0, ndmax, NfHalfSplit{});
}

// ------------------------------------------------------------------------------------------
// S2M at the leaves (Eq. s2m): mu[k][X][a][i] = sum_s St[s][a] sum_{x in X} x[k ls + s][x] Sx[x][i]
// (double layer: sum over the triangle's three nodes with SK).  CTA per (leaf box, interval
// chunk, rhs).
constexpr int kTSB = 32;   // steps per S2M / L2T block
constexpr int kTSP = kTSB + 4;  // padded row of kTSB steps (16-byte aligned rows)

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void lds4(const float *p, float (&w)[4])
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
}
__device__ __forceinline__ void lds4(const double *p, double (&w)[4])
{
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    w[0] = a.x;
    w[1] = a.y;
    w[2] = b.x;
    w[3] = b.y;
}
constexpr int kS2MCK = 6;  // moment groups of 32 per thread: a CTA covers a chunk of 192 moments
constexpr int kS2MChunk = 32 * kS2MCK;

template <typename R, typename XT, bool KOP>
__global__ void __launch_bounds__(256) k_s2m(const XT *__restrict__ xin, int ncolg, const int *__restrict__ tri,
                                               const R *__restrict__ Stab, const R *__restrict__ St, R *__restrict__ mu,
                                               const int *__restrict__ leaf_start, int nk, int na, int ls, int Et,
                                               int nint, int nbox, int nchk)
{
    // register-blocked: a CTA covers one leaf box, kTSB steps, one chunk of at most 192 moments
    // (grid z = rhs x chunk) and one rhs; thread (tg = warp, kg = lane) accumulates steps
    // 4 tg .. 4 tg + 3 for the moments i0 + kg + 32 c of the chunk
    extern __shared__ unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);
    constexpr int XCH = KOP ? 16 : 32, PER = KOP ? 3 : 1, KC = XCH * PER;
    const int X = blockIdx.x, rhs = blockIdx.z / nchk, i0 = (blockIdx.z % nchk) * kS2MChunk;
    const int nkc = min(nk - i0, kS2MChunk);
    const int ipb = kTSB / ls;
    const int k0 = blockIdx.y * ipb, kend = min(nint, k0 + ipb), nts = (kend - k0) * ls, t0 = k0 * ls;
    const int x0 = leaf_start[X], x1 = leaf_start[X + 1];
    R *Ws = sm;              // [kTSB][KC]
    R *Ss = sm + kTSB * KC;  // [KC][nkc]
    const XT *xr = xin + (size_t)rhs * Et * ncolg;
    const int kg = threadIdx.x & 31, tg = threadIdx.x >> 5, ck = (nkc + 31) / 32;
    R acc[4][kS2MCK];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kS2MCK; ++c) acc[r][c] = R(0);
    for (int xb = x0; xb < x1; xb += XCH) {
        const int nx = min(XCH, x1 - xb);
        __syncthreads();
        for (int e = threadIdx.x; e < kTSB * KC; e += blockDim.x) {
            const int ts = e / KC, j = e % KC, xi = j / PER, v = j % PER;
            R val = R(0);
            if (ts < nts && xi < nx) {
                const int col = KOP ? tri[3 * (xb + xi) + v] : xb + xi;
                val = R(xr[(size_t)(t0 + ts) * ncolg + col]);
            }
            Ws[e] = val;
        }
        for (int e = threadIdx.x; e < KC * nkc; e += blockDim.x) {
            const int j = e / nkc;
            Ss[e] = (j / PER < nx) ? Stab[(size_t)(xb * PER + j) * nk + i0 + (e % nkc)] : R(0);
        }
        __syncthreads();
        for (int j = 0; j < KC; ++j) {
            R w[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) w[r] = Ws[(tg * 4 + r) * KC + j];
#pragma unroll
            for (int c = 0; c < kS2MCK; ++c) {
                const int i = kg + 32 * c;
                if (c < ck && i < nkc) {
                    const R sv = Ss[j * nkc + i];
#pragma unroll
                    for (int r = 0; r < 4; ++r) mac(acc[r][c], w[r], sv);
                }
            }
        }
    }
    __syncthreads();
    R *Ps = sm;  // [kTSB][nkc]
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kS2MCK; ++c) {
            const int i = kg + 32 * c;
            if (c < ck && i < nkc) Ps[(tg * 4 + r) * nkc + i] = acc[r][c];
        }
    __syncthreads();
    const int nmo = (kend - k0) * na * nkc;
    for (int o = threadIdx.x; o < nmo; o += blockDim.x) {
        int kk = o / (na * nkc), a = (o / nkc) % na, i = o % nkc;
        R v = R(0);
        for (int s = 0; s < ls; ++s) v += St[s * na + a] * Ps[((kk * ls) + s) * nkc + i];
        mu[((((size_t)rhs * nint + k0 + kk) * nbox + X) * na + a) * nk + i0 + i] = v;
    }
}

// Balanced S2M in two stages (leaf boxes hold from a few to several hundred triangles):
// stage 1, CTA per (64-row tile of a leaf box, kTSB steps, rhs): the spatial moments of the
// tile's triangles, P[tile][t][i] = sum_{x in tile} x[t][x] Sx[x][i], same register blocking as
// k_s2m; stage 2, thread per moment: mu[k][X][a][i] = sum_s St[s][a] sum_{tiles of X} P[tile][k ls + s][i]
// in tile order (deterministic).
template <typename R, typename XT, bool KOP>
__global__ void __launch_bounds__(256) k_s2m_tile(const XT *__restrict__ xin, int ncolg, const int *__restrict__ tri,
                                                    const R *__restrict__ Stab, R *__restrict__ part,
                                                    const int *__restrict__ tiles, int ntiles,
                                                    const int *__restrict__ leaf_start, int nk, int Et, int nchk)
{
    extern __shared__ __align__(16) unsigned char s2m_raw[];
    R *sm = reinterpret_cast<R *>(s2m_raw);
    constexpr int XCH = KOP ? 16 : 32, PER = KOP ? 3 : 1, KC = XCH * PER;
    const int tile = blockIdx.x, rhs = blockIdx.z / nchk, i0 = (blockIdx.z % nchk) * kS2MChunk;
    const int nkc = min(nk - i0, kS2MChunk);
    const int X = tiles[2 * tile];
    const int x0 = leaf_start[X] + tiles[2 * tile + 1], x1 = min(x0 + 64, leaf_start[X + 1]);
    const int t0 = blockIdx.y * kTSB, nts = min(kTSB, Et - t0);
    R *Ws = sm;              // [KC][kTSP]: a thread's four steps are one vector load
    R *Ss = sm + KC * kTSP;  // [KC][nkc]
    const XT *xr = xin + (size_t)rhs * Et * ncolg;
    const int kg = threadIdx.x & 31, tg = threadIdx.x >> 5, ck = (nkc + 31) / 32;
    R acc[4][kS2MCK];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kS2MCK; ++c) acc[r][c] = R(0);
    for (int xb = x0; xb < x1; xb += XCH) {
        const int nx = min(XCH, x1 - xb);
        __syncthreads();
        for (int e = threadIdx.x; e < kTSB * KC; e += blockDim.x) {
            const int ts = e / KC, j = e % KC, xi = j / PER, v = j % PER;
            R val = R(0);
            if (ts < nts && xi < nx) {
                const int col = KOP ? tri[3 * (xb + xi) + v] : xb + xi;
                val = R(xr[(size_t)(t0 + ts) * ncolg + col]);
            }
            Ws[j * kTSP + ts] = val;
        }
        for (int e = threadIdx.x; e < KC * nkc; e += blockDim.x) {
            const int j = e / nkc;
            Ss[e] = (j / PER < nx) ? Stab[(size_t)(xb * PER + j) * nk + i0 + (e % nkc)] : R(0);
        }
        __syncthreads();
        for (int j = 0; j < KC; ++j) {
            R w[4];
            lds4(Ws + j * kTSP + tg * 4, w);
#pragma unroll
            for (int c = 0; c < kS2MCK; ++c) {
                const int i = kg + 32 * c;
                if (c < ck && i < nkc) {
                    const R sv = Ss[j * nkc + i];
#pragma unroll
                    for (int r = 0; r < 4; ++r) mac(acc[r][c], w[r], sv);
                }
            }
        }
    }
    R *pt = part + (((size_t)rhs * ntiles + tile) * Et + t0) * nk;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int ts = tg * 4 + r;
        if (ts >= nts) continue;
#pragma unroll
        for (int c = 0; c < kS2MCK; ++c) {
            const int i = kg + 32 * c;
            if (c < ck && i < nkc) pt[(size_t)ts * nk + i0 + i] = acc[r][c];
        }
    }
}

// stage 2: thread per (rhs, interval k) [grid x] and (box X, moment i) [grid y, x threads]; each
// partial is read once and weighted for every time node a (registers)
template <typename R>
__global__ void k_s2m_time(const R *__restrict__ part, const R *__restrict__ St, R *__restrict__ mu,
                           const int *__restrict__ box_tiles, int ntiles, int nk, int na, int ls, int Et, int nint,
                           int nbox)
{
    const int xi = blockIdx.y * blockDim.x + threadIdx.x;
    if (xi >= nbox * nk) return;
    const int X = xi / nk, i = xi - X * nk;
    const int k = blockIdx.x % nint, rhs = blockIdx.x / nint;
    R v[kMaxNa];
#pragma unroll
    for (int a = 0; a < kMaxNa; ++a) v[a] = R(0);
    for (int tl = box_tiles[X]; tl < box_tiles[X + 1]; ++tl) {
        const R *pt = part + (((size_t)rhs * ntiles + tl) * Et + (size_t)k * ls) * nk + i;
        for (int s = 0; s < ls; ++s) {
            const R pv = pt[(size_t)s * nk];
#pragma unroll
            for (int a = 0; a < kMaxNa; ++a)
                if (a < na) mac(v[a], St[s * na + a], pv);
        }
    }
    R *mo = mu + ((((size_t)rhs * nint + k) * nbox + X) * na) * nk + i;
#pragma unroll
    for (int a = 0; a < kMaxNa; ++a)
        if (a < na) mo[(size_t)a * nk] = v[a];
}

// L2T's temporal factor for every (step, leaf box): Q[rhs][t][X][nu] = sum_b St[s][b] lam[k][X][b][nu],
// t = k ls + s; thread per (rhs, k) [grid x] and (X, nu)
template <typename R>
__global__ void k_l2t_time(const R *__restrict__ lam, const R *__restrict__ St, R *__restrict__ Q, int nk, int na,
                           int ls, int Et, int nint, int nbox)
{
    const int xi = blockIdx.y * blockDim.x + threadIdx.x;
    if (xi >= nbox * nk) return;
    const int X = xi / nk, i = xi - X * nk;
    const int k = blockIdx.x % nint, rhs = blockIdx.x / nint;
    R lv[kMaxNa];
    const R *lp = lam + ((((size_t)rhs * nint + k) * nbox + X) * na) * nk + i;
#pragma unroll
    for (int b = 0; b < kMaxNa; ++b) lv[b] = b < na ? lp[(size_t)b * nk] : R(0);
    for (int s = 0; s < ls; ++s) {
        R v = R(0);
#pragma unroll
        for (int b = 0; b < kMaxNa; ++b)
            if (b < na) mac(v, St[s * na + b], lv[b]);
        Q[(((size_t)rhs * Et + (size_t)k * ls + s) * nbox + X) * nk + i] = v;
    }
}

void launch_s2m(int prec, bool kop, const void *x, int ncolg, const void *Stab, const void *St, void *mu_leaf, int nrhs,
                const ApplyGeo &g, cudaStream_t st, void *ws, size_t ws_elems)
{
    const size_t es = prec == 1 ? 4 : 8;
    const int nint = g.Et / g.ls;
    dispatch_prec(prec, [&](auto tag) {
        using R = decltype(tag);
        // input in the arithmetic type, or FP64 converted on load for the double-FP32 passes
        using XT = typename std::conditional<std::is_same<R, df64>::value, double, R>::type;
        const int nchk = (g.nk + kS2MChunk - 1) / kS2MChunk, nkc = std::min(g.nk, kS2MChunk);
        if (ws && g.tiles && (size_t)nrhs * g.ntiles * g.Et * g.nk <= ws_elems) {
            const int KC = kop ? 48 : 32;
            const size_t smem = ((size_t)KC * kTSP + (size_t)KC * nkc) * es;
            const dim3 grd(g.ntiles, (g.Et + kTSB - 1) / kTSB, nrhs * nchk);
            const dim3 g2((unsigned)(nrhs * nint), (unsigned)((g.nbox_leaf * g.nk + 255) / 256));
            auto kt = kop ? k_s2m_tile<R, XT, true> : k_s2m_tile<R, XT, false>;
            cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kt<<<grd, 256, smem, st>>>((const XT *)x, ncolg, g.tri, (const R *)Stab, (R *)ws, g.tiles, g.ntiles,
                                       g.leaf_start, g.nk, g.Et, nchk);
            k_s2m_time<R><<<g2, 256, 0, st>>>((const R *)ws, (const R *)St, (R *)mu_leaf, g.box_tiles, g.ntiles, g.nk,
                                              g.na, g.ls, g.Et, nint, g.nbox_leaf);
            return;
        }
        const int ipb = kTSB / g.ls;
        const int KC = kop ? 48 : 32;
        const size_t sm1 = (size_t)kTSB * KC + (size_t)KC * nkc, sm2 = (size_t)kTSB * nkc;
        const size_t smem = (sm1 > sm2 ? sm1 : sm2) * es;
        const dim3 grd(g.nbox_leaf, (nint + ipb - 1) / ipb, nrhs * nchk);
        auto kb = kop ? k_s2m<R, XT, true> : k_s2m<R, XT, false>;
        cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kb<<<grd, 256, smem, st>>>((const XT *)x, ncolg, g.tri, (const R *)Stab, (const R *)St, (R *)mu_leaf,
                                   g.leaf_start, g.nk, g.na, g.ls, g.Et, nint, g.nbox_leaf, nchk);
    });
}

// ------------------------------------------------------------------------------------------
// M2M from level l+1 to level l (Eq. temp_m2m, st_m2m): thread per parent moment.
template <typename R>
__global__ void k_m2m(const R *__restrict__ mu_c, R *__restrict__ mu_p, const int *__restrict__ ch_ptr,
                      const int *__restrict__ ch_idx, const int *__restrict__ oct_c, const R *__restrict__ q1,
                      const R *__restrict__ qt, const int *__restrict__ kidx, const int *__restrict__ kinv, int st, int na,
                      int nk, int mx, int nint_p, int nbox_p, int nbox_c, int nrhs)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nrhs * nint_p * nbox_p * na * nk;
    if (gid >= total) return;
    int iv = gid % nk;
    size_t r_ = gid / nk;
    int ap = r_ % na;
    r_ /= na;
    int bp = r_ % nbox_p;
    r_ /= nbox_p;
    int kp = r_ % nint_p;
    int rhs = (int)(r_ / nint_p);
    const int m1 = mx + 1;
    int n0 = kidx[3 * iv], n1 = kidx[3 * iv + 1], n2 = kidx[3 * iv + 2];
    R acc = R(0);
    for (int e = ch_ptr[bp]; e < ch_ptr[bp + 1]; ++e) {
        int bc = ch_idx[e], oc = oct_c[bc];
        const R *qa = q1 + (oc & 1) * m1 * m1, *qb = q1 + ((oc >> 1) & 1) * m1 * m1, *qc = q1 + ((oc >> 2) & 1) * m1 * m1;
        for (int c = 0; c < 2; ++c) {
            int kc = 2 * kp + c;
            const R *mc = mu_c + (((size_t)rhs * 2 * nint_p + kc) * nbox_c + bc) * na * nk;
            for (int ac = 0; ac < na; ++ac) {
                R qtv = qt[(c * na + ac) * na + ap];
                const R *m = mc + ac * nk;
                if (!st) {
                    acc += qtv * m[iv];
                } else {
                    R s = R(0);
                    for (int k0 = 0; k0 <= n0; ++k0)
                        for (int k1 = 0; k1 <= n1; ++k1)
                            for (int k2 = 0; k2 <= n2; ++k2)
                                s += qa[k0 * m1 + n0] * qb[k1 * m1 + n1] * qc[k2 * m1 + n2] *
                                     m[kinv[(k0 * m1 + k1) * m1 + k2]];
                    acc += qtv * s;
                }
            }
        }
    }
    mu_p[gid] = acc;
}

// Space-time M2M (Eq. st_m2m) with one CTA per parent (interval kp, box bp, rhs): the temporal
// contraction of each child's moments is staged in shared memory,
//   tmp_c[ap][kap] = sum_{c, ac} q^(t)_c[ac][ap] mu[2 kp + c][child][ac][kap],
// then mu_p[ap][nu] = sum_children sum_{kap <= nu} q^(x)_{kap,nu}(child) tmp_c[ap][kap].
template <typename R>
__global__ void __launch_bounds__(256) k_m2m_st(const R *__restrict__ mu_c, R *__restrict__ mu_p,
                                                  const int *__restrict__ ch_ptr, const int *__restrict__ ch_idx,
                                                  const int *__restrict__ oct_c, const R *__restrict__ q1,
                                                  const R *__restrict__ qt, const int *__restrict__ kidx,
                                                  const int *__restrict__ kinv, int na, int nk, int mx, int nint_p,
                                                  int nbox_p, int nbox_c)
{
    extern __shared__ unsigned char smem_raw[];
    const int m1 = mx + 1;
    R *tmp = reinterpret_cast<R *>(smem_raw);  // [8][nk]: children's contracted moments for node ap
    R *part = tmp + 8 * nk;                    // [8][nk]: partial sums over children, per thread group
    R *qs = part + 8 * nk;                     // [2][m1][m1]
    int *kin = reinterpret_cast<int *>(qs + 2 * m1 * m1);
    // one CTA per (kp, bp, ap): the outputs of one parent time node
    const int ap = blockIdx.x % na, pb = blockIdx.x / na;
    const int kp = pb / nbox_p, bp = pb % nbox_p, rhs = blockIdx.y;
    const int c0 = ch_ptr[bp], nch = ch_ptr[bp + 1] - c0;
    for (int i = threadIdx.x; i < 2 * m1 * m1; i += blockDim.x) qs[i] = q1[i];
    for (int i = threadIdx.x; i < m1 * m1 * m1; i += blockDim.x) kin[i] = kinv[i];
    for (int i = threadIdx.x; i < nch * nk; i += blockDim.x) {
        int e = i / nk, ik = i % nk, bc = ch_idx[c0 + e];
        R v = R(0);
        for (int c = 0; c < 2; ++c) {
            const R *m = mu_c + (((size_t)rhs * 2 * nint_p + 2 * kp + c) * nbox_c + bc) * na * nk + ik;
            for (int ac = 0; ac < na; ++ac) v += qt[(c * na + ac) * na + ap] * m[(size_t)ac * nk];
        }
        tmp[i] = v;
    }
    __syncthreads();
    // output iv: `per` threads take every per-th child; their partial sums are added in a fixed
    // order afterwards (deterministic)
    const int per = max(1, min((int)blockDim.x / nk, 8));
    for (int o = threadIdx.x; o < nk * per; o += blockDim.x) {
        const int iv = o % nk, g = o / nk;
        const int n0 = kidx[3 * iv], n1 = kidx[3 * iv + 1], n2 = kidx[3 * iv + 2];
        R acc = R(0);
        for (int e = g; e < nch; e += per) {
            const int oc = oct_c[ch_idx[c0 + e]];
            const R *qa = qs + (oc & 1) * m1 * m1, *qb = qs + ((oc >> 1) & 1) * m1 * m1, *qc = qs + ((oc >> 2) & 1) * m1 * m1;
            const R *tp = tmp + e * nk;
            for (int k0 = 0; k0 <= n0; ++k0)
                for (int k1 = 0; k1 <= n1; ++k1) {
                    const R q01 = qa[k0 * m1 + n0] * qb[k1 * m1 + n1];
                    for (int k2 = 0; k2 <= n2; ++k2) acc += q01 * qc[k2 * m1 + n2] * tp[kin[(k0 * m1 + k1) * m1 + k2]];
                }
        }
        part[g * nk + iv] = acc;
    }
    __syncthreads();
    R *out = mu_p + (((size_t)rhs * nint_p + kp) * nbox_p + bp) * na * nk + (size_t)ap * nk;
    for (int iv = threadIdx.x; iv < nk; iv += blockDim.x) {
        R sum = R(0);
        for (int g = 0; g < per; ++g) sum += part[g * nk + iv];
        out[iv] = sum;
    }
}

// Space-time L2L (transpose of Eq. st_m2m) with one CTA per (parent (kp, bp), child box, rhs):
//   tmp[bp_][kap] = sum_{nu >= kap, |nu| <= m_x} q^(x)_{kap,nu}(child) lam_p[bp_][nu],
//   lam_c[2 kp + c][child][bc][kap] += sum_{bp_} q^(t)_c[bc][bp_] tmp[bp_][kap].
template <typename R>
__global__ void __launch_bounds__(256) k_l2l_st(const R *__restrict__ lam_p, R *__restrict__ lam_c,
                                                  const int *__restrict__ ch_ptr, const int *__restrict__ ch_idx,
                                                  const int *__restrict__ oct_c, const R *__restrict__ q1,
                                                  const R *__restrict__ qt, const int *__restrict__ kidx,
                                                  const int *__restrict__ kinv, int na, int nk, int mx, int nint_p,
                                                  int nbox_p, int nbox_c)
{
    extern __shared__ unsigned char smem_raw[];
    const int m1 = mx + 1;
    R *lp = reinterpret_cast<R *>(smem_raw);  // [na][nk]
    R *tmp = lp + na * nk;                    // [na][nk]
    R *qs = tmp + na * nk;                    // [2][m1][m1]
    int *kin = reinterpret_cast<int *>(qs + 2 * m1 * m1);
    const int e = blockIdx.x % 8, pb = blockIdx.x / 8;
    const int kp = pb / nbox_p, bp = pb % nbox_p, rhs = blockIdx.y;
    const int c0 = ch_ptr[bp], nch = ch_ptr[bp + 1] - c0;
    if (e >= nch) return;  // the parent has fewer children
    for (int i = threadIdx.x; i < 2 * m1 * m1; i += blockDim.x) qs[i] = q1[i];
    for (int i = threadIdx.x; i < m1 * m1 * m1; i += blockDim.x) kin[i] = kinv[i];
    const R *src = lam_p + (((size_t)rhs * nint_p + kp) * nbox_p + bp) * na * nk;
    for (int i = threadIdx.x; i < na * nk; i += blockDim.x) lp[i] = src[i];
    {
        const int bc = ch_idx[c0 + e], oc = oct_c[bc];
        const R *qa = qs + (oc & 1) * m1 * m1, *qb = qs + ((oc >> 1) & 1) * m1 * m1, *qc = qs + ((oc >> 2) & 1) * m1 * m1;
        __syncthreads();
        for (int o = threadIdx.x; o < na * nk; o += blockDim.x) {
            const int bpI = o / nk, ik = o % nk;
            const int k0 = kidx[3 * ik], k1 = kidx[3 * ik + 1], k2 = kidx[3 * ik + 2];
            const R *l = lp + bpI * nk;
            R s = R(0);
            for (int n0 = k0; n0 <= mx; ++n0)
                for (int n1 = k1; n0 + n1 <= mx; ++n1) {
                    const R q01 = qa[k0 * m1 + n0] * qb[k1 * m1 + n1];
                    for (int n2 = k2; n0 + n1 + n2 <= mx; ++n2) s += q01 * qc[k2 * m1 + n2] * l[kin[(n0 * m1 + n1) * m1 + n2]];
                }
            tmp[o] = s;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < 2 * na * nk; o += blockDim.x) {
            const int c = o / (na * nk), bcI = (o / nk) % na, ik = o % nk;
            R v = R(0);
            for (int bpI = 0; bpI < na; ++bpI) v += qt[(c * na + bcI) * na + bpI] * tmp[bpI * nk + ik];
            lam_c[((((size_t)rhs * 2 * nint_p + 2 * kp + c) * nbox_c + bc) * na + bcI) * nk + ik] += v;
        }
    }
}

void launch_m2m(int prec, const DevLevel &par, const DevLevel &ch, int l, const void *qt, void *mu, int nrhs,
                const ApplyGeo &g, int64_t mu_stride, cudaStream_t st)
{
    (void)l;
    (void)mu_stride;
    const size_t total = (size_t)nrhs * par.nint * par.nbox * g.na * g.nk;
    const unsigned blocks = (unsigned)((total + 127) / 128);
    const size_t es = prec == 1 ? 4 : 8;
    char *base = (char *)mu;
    const int m1 = g.mx + 1;
    dispatch_prec(prec, [&](auto tag) {
        using R = decltype(tag);
        const R *mc = (const R *)(base + ch.mom_off * es * nrhs);
        R *mp = (R *)(base + par.mom_off * es * nrhs);
        if (ch.st) {
            const size_t smem = es * ((size_t)16 * g.nk + 2 * m1 * m1) + 4 * (size_t)m1 * m1 * m1;
            const dim3 grd(par.nint * par.nbox * g.na, nrhs);
            cudaFuncSetAttribute(k_m2m_st<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_m2m_st<R><<<grd, 256, smem, st>>>(mc, mp, par.ch_ptr, par.ch_idx, ch.octant, (const R *)ch.qx,
                                                (const R *)qt, g.kidx, g.kinv, g.na, g.nk, g.mx, par.nint, par.nbox,
                                                ch.nbox);
            return;
        }
        k_m2m<R><<<blocks, 128, 0, st>>>(mc, mp, par.ch_ptr, par.ch_idx, ch.octant, (const R *)ch.qx, (const R *)qt,
                                         g.kidx, g.kinv, ch.st, g.na, g.nk, g.mx, par.nint, par.nbox, ch.nbox, nrhs);
    });
}

// ------------------------------------------------------------------------------------------
// M2L at level l (Eq. m2l with Eq. exp_coeffs_3d), applied one direction at a time.
//
// For a target interval k, a source interval J in I(k) (Eq. 03:ILtemp: I_{k-2} for even k,
// I_{k-3}, I_{k-2} for odd k) and time nodes (a, b), the coefficients factor as
// pref_ab * E^x[o_1]_{kap_1 nu_1} E^y[o_2]_{kap_2 nu_2} E^z[o_3]_{kap_3 nu_3}, where o = X - Y is
// the grid offset of target and source box.  The interaction area (Eq. 03:Iarea) is the cube
// |o_j| <= n_tr, so the sum over source boxes is a separable convolution over the box grid
// (empty cells carry zero moments).  The truncation |kappa + nu| <= m_x is kept exactly with
// a cumulative degree budget B:
//   T1[nu1,k2,k3][B](X1,Y2,Y3) = sum_{Y1} sum_{k1 <= B - nu1 - k2 - k3} E^x[X1-Y1]_{k1 nu1} mu[k1,k2,k3](Y)
//   T2[nu1,nu2,k3][B](X1,X2,Y3) = sum_{Y2} sum_{k2 <= B - nu1 - nu2 - k3} E^y[X2-Y2]_{k2 nu2}
//                                 T1[nu1,k2,k3][B - nu2](X1,Y2,Y3)
//   lam[b][nu](X) = sum_{J,a} pref_ab sum_{Y3} sum_{k3 <= m - |nu|} E^z[X3-Y3]_{k3 nu3}
//                   T2[nu1,nu2,k3][m - nu3](X1,X2,Y3)
// Triples (t0,t1,t2) with t0+t1+t2 <= m use the graded enumeration of the multi-indices;
// eoff[t] is the offset of the budget range B = |t| .. m of triple t (C(m+4,4) entries).
struct M2LArgs {
    int G, ntr, na, nk, mx, ne, nint, nbox;
    const int *cellbox;                   // [G^3] -> box or -1
    const int *boxcell;                   // [nbox] -> cell
    const int *pk, *pJ;                   // problem pairs (target k, source J) of this chunk
    int npair;
    const int *kidx, *kinv, *eoff;
};

template <typename R>
__global__ void k_m2l_s1(M2LArgs A, const R *__restrict__ mu, const R *__restrict__ E1, R *__restrict__ T1, int nrhs)
{
    const int G = A.G, G3 = G * G * G, m1 = A.mx + 1, no = 2 * G - 1, na = A.na;
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nrhs * A.npair * na * na * G3 * A.nk;
    if (gid >= total) return;
    int t = gid % A.nk;
    size_t r_ = gid / A.nk;
    int cell = r_ % G3;
    r_ /= G3;
    int b = r_ % na;
    r_ /= na;
    int a = r_ % na;
    r_ /= na;
    int pr = r_ % A.npair;
    int rhs = (int)(r_ / A.npair);
    const int k = A.pk[pr], J = A.pJ[pr], D = k - J;
    const int X1 = cell / (G * G), Y2 = (cell / G) % G, Y3 = cell % G;
    const int nu1 = A.kidx[3 * t], k2 = A.kidx[3 * t + 1], k3 = A.kidx[3 * t + 2];
    const int s0 = nu1 + k2 + k3;
    const R *E = E1 + (size_t)(((D - 2) * na + a) * na + b) * no * m1 * m1;
    const R *mJ = mu + ((size_t)rhs * A.nint + J) * A.nbox * na * A.nk;
    const int y_lo = max(0, X1 - A.ntr), y_hi = min(G - 1, X1 + A.ntr);
    R *out = T1 + ((((size_t)rhs * A.npair + pr) * na + a) * na + b) * (size_t)G3 * A.ne + (size_t)cell * A.ne + A.eoff[t];
    R acc = R(0);
    for (int B = s0; B <= A.mx; ++B) {
        const int k1 = B - s0;
        const int im = A.kinv[(k1 * m1 + k2) * m1 + k3];
        for (int Y1 = y_lo; Y1 <= y_hi; ++Y1) {
            int box = A.cellbox[(Y1 * G + Y2) * G + Y3];
            if (box < 0) continue;
            mac(acc, E[((X1 - Y1 + G - 1) * m1 + k1) * m1 + nu1], mJ[((size_t)box * na + a) * A.nk + im]);
        }
        out[B - s0] = acc;
    }
}

template <typename R>
__global__ void k_m2l_s2(M2LArgs A, const R *__restrict__ E1, const R *__restrict__ T1, R *__restrict__ T2, int nrhs)
{
    const int G = A.G, G3 = G * G * G, m1 = A.mx + 1, no = 2 * G - 1, na = A.na;
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nrhs * A.npair * na * na * G3 * A.nk;
    if (gid >= total) return;
    int t = gid % A.nk;
    size_t r_ = gid / A.nk;
    int cell = r_ % G3;
    size_t P = r_ / G3;  // ((rhs * npair + pr) * na + a) * na + b
    int b = P % na, a = (P / na) % na, pr = (P / (na * na)) % A.npair;
    const int D = A.pk[pr] - A.pJ[pr];
    const int X1 = cell / (G * G), X2 = (cell / G) % G, Y3 = cell % G;
    const int nu1 = A.kidx[3 * t], nu2 = A.kidx[3 * t + 1], k3 = A.kidx[3 * t + 2];
    const int s0 = nu1 + nu2 + k3;
    const R *E = E1 + (size_t)(((D - 2) * na + a) * na + b) * no * m1 * m1;
    const R *Tin = T1 + P * (size_t)G3 * A.ne;
    R *out = T2 + P * (size_t)G3 * A.ne + (size_t)cell * A.ne + A.eoff[t];
    const int y_lo = max(0, X2 - A.ntr), y_hi = min(G - 1, X2 + A.ntr);
    for (int Bp = s0; Bp <= A.mx; ++Bp) {
        R acc = R(0);
        for (int Y2 = y_lo; Y2 <= y_hi; ++Y2) {
            const R *Ey = E + (size_t)(X2 - Y2 + G - 1) * m1 * m1;
            const R *Tc = Tin + (size_t)((X1 * G + Y2) * G + Y3) * A.ne;
            for (int k2 = 0; k2 <= Bp - s0; ++k2) {
                int t1 = A.kinv[(nu1 * m1 + k2) * m1 + k3];
                mac(acc, Ey[k2 * m1 + nu2], Tc[A.eoff[t1] + (Bp - nu2 - nu1 - k2 - k3)]);
            }
        }
        out[Bp - s0] = acc;
    }
}

template <typename R>
__global__ void k_m2l_s3(M2LArgs A, const R *__restrict__ E1, const R *__restrict__ pref, const R *__restrict__ T2,
                         R *__restrict__ lam, const int *__restrict__ kptr, int p0, int k_lo, int k_hi, int nrhs)
{
    const int G = A.G, G3 = G * G * G, m1 = A.mx + 1, no = 2 * G - 1, na = A.na;
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nk_ = k_hi - k_lo;
    size_t total = (size_t)nrhs * nk_ * A.nbox * na * A.nk;
    if (gid >= total) return;
    int iv = gid % A.nk;
    size_t r_ = gid / A.nk;
    int b = r_ % na;
    r_ /= na;
    int box = r_ % A.nbox;
    r_ /= A.nbox;
    int k = k_lo + (int)(r_ % nk_);
    int rhs = (int)(r_ / nk_);
    const int cell = A.boxcell[box];
    const int X1 = cell / (G * G), X2 = (cell / G) % G, X3 = cell % G;
    const int nu1 = A.kidx[3 * iv], nu2 = A.kidx[3 * iv + 1], nu3 = A.kidx[3 * iv + 2];
    const int smax = A.mx - nu1 - nu2 - nu3;
    const int y_lo = max(0, X3 - A.ntr), y_hi = min(G - 1, X3 + A.ntr);
    R val = R(0);
    for (int pr = kptr[k] - p0; pr < kptr[k + 1] - p0; ++pr) {
        const int D = k - A.pJ[pr];
        for (int a = 0; a < na; ++a) {
            const size_t P = (((size_t)rhs * A.npair + pr) * na + a) * na + b;
            const R *E = E1 + (size_t)(((D - 2) * na + a) * na + b) * no * m1 * m1;
            const R *Tin = T2 + P * (size_t)G3 * A.ne;
            R s = R(0);
            for (int Y3 = y_lo; Y3 <= y_hi; ++Y3) {
                const R *Ez = E + (size_t)(X3 - Y3 + G - 1) * m1 * m1;
                const R *Tc = Tin + (size_t)((X1 * G + X2) * G + Y3) * A.ne;
                for (int k3 = 0; k3 <= smax; ++k3) {
                    int t2 = A.kinv[(nu1 * m1 + nu2) * m1 + k3];
                    mac(s, Ez[k3 * m1 + nu3], Tc[A.eoff[t2] + (A.mx - nu3 - nu1 - nu2 - k3)]);
                }
            }
            val += pref[((D - 2) * na + a) * na + b] * s;
        }
    }
    lam[((((size_t)rhs * A.nint + k) * A.nbox + box) * na + b) * A.nk + iv] = val;
}

// Fused M2L for grids of at most 4^3 cells: one CTA per (target interval k, time node b, rhs)
// keeps the source moments of all cells, the intermediates T1, T2 of all cells and the target
// locals in shared memory.  The grid is padded to FG^3 cells (FG = 4, or 2 for levels with G <= 2,
// whose CTAs then need an eighth of the shared memory and work).  A unit of passes 1 and 2 is a
// multi-index triple, one budget chain (pass 1: the whole prefix chain; pass 2: one budget value)
// and two grid coordinates, with the FG cells of the third in registers; an item of pass 3 is a
// target multi-index and two target coordinates, whose FG locals stay in registers over all
// terms.  Each step does FG^2 FMAs from FG loads of moments or intermediates and 7 coefficient
// loads.  Units and items are short chains dealt round-robin over the CTA, so the passes end
// together.  Coefficients beyond the
// interaction radius are zeroed once per (J, a), which applies Eq. 03:Iarea without branches.
// Same arithmetic as the three-pass kernels (cells with G < 4 are padded with empty cells).
// Split mode (levels with too few intervals to fill the GPU): one CTA per (k, b, source term)
// with source term = (J, a) of the interaction list; each term's locals go to its own slice of a
// workspace and k_m2l_sum_terms adds the slices in a fixed order (deterministic).
constexpr int FGMax = 4;  // padded grid extent per direction: 4, or 2 for the coarse levels (G <= 2)

// C(n, 4), 0 for n < 4: the budget rows of all triples with |t| <= n - 4 (slice offsets of T2)
__host__ __device__ inline int binom4(int n) { return n < 4 ? 0 : n * (n - 1) * (n - 2) * (n - 3) / 24; }

constexpr int kM2LThreads = 384;
// split mode below this many (interval, node, rhs) CTAs per SM: eight.  At two resident CTAs per
// SM and work per CTA that differs by 2x between even and odd intervals, fewer than four waves
// lose much of the last one; one-term CTAs are uniform and many
constexpr int kM2LSplitCtasPerSm = 8;

template <typename R, int FG, bool SL>
__global__ void __launch_bounds__(kM2LThreads, FG == 2 ? 2 : (sizeof(R) == 4 && !SL ? 2 : 1)) k_m2l_fused(M2LArgs A, const R *__restrict__ mu,
                                                                const R *__restrict__ E1, const R *__restrict__ pref,
                                                                R *__restrict__ lam, int nrhs, int split,
                                                                R *__restrict__ part)
{
    extern __shared__ unsigned char smem_raw[];
    constexpr int C3 = FG * FG * FG, CS = C3 + 1;  // cell rows are padded by one (bank spread)
    const int G = A.G, nk = A.nk, ne = A.ne, mx = A.mx, m1 = mx + 1, na = A.na, esz = m1 * m1;
    // SL (sliced): T2 is formed and consumed one value of nu1 at a time, so U needs only nk rows
    // (the largest slice, nu1 = 0, has C(m_x+3, 3) = nk budget entries); the shared memory of
    // degrees whose full T2 would not fit
    const int nu_rows = SL ? nk : max(ne, nk);
    R *T1s = reinterpret_cast<R *>(smem_raw);  // [ne][CS]  cells (X1, Y2, Y3)
    R *U = T1s + ne * CS;                      // [nu_rows][CS]  moments [nk][CS] in pass 1, then T2 (X1, X2, Y3)
    R *Es = U + nu_rows * CS;                  // [7][m1][m1] offsets -3..3, zero outside the radius
    int *kid = reinterpret_cast<int *>(Es + 7 * esz);
    int *kin = kid + nk;
    int *eof = kin + m1 * m1 * m1;
    int *cbx = eof + nk;                       // [C3] padded cell -> box or -1
    int *eofs = cbx + C3;                      // SL: offset of a triple's budget range within its nu1 slice
    int *rs = eofs + nk;                       // [ne] pass-2 rows: triple | budget index << 16, per slice
    const int nterm = split ? 2 * na : 1;  // source terms per CTA group: (J index, a)
    const int kb = blockIdx.x / nterm, term = blockIdx.x % nterm;
    const int k = kb / na, b = kb % na, rhs = blockIdx.y;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
        kid[i] = A.kidx[3 * i] | (A.kidx[3 * i + 1] << 8) | (A.kidx[3 * i + 2] << 16);
        eof[i] = A.eoff[i];
    }
    for (int i = threadIdx.x; i < m1 * m1 * m1; i += blockDim.x) kin[i] = A.kinv[i];
    for (int i = threadIdx.x; i < C3; i += blockDim.x) {
        int x = i / (FG * FG), y = (i / FG) % FG, z = i % FG;
        cbx[i] = (x < G && y < G && z < G) ? A.cellbox[(x * G + y) * G + z] : -1;
    }
    if (SL && threadIdx.x == 0) {
        int off[kMaxMx + 1];
        for (int v = 0; v <= mx; ++v) off[v] = 0;
        for (int t = 0; t < nk; ++t) {
            const int n1 = A.kidx[3 * t], s0 = n1 + A.kidx[3 * t + 1] + A.kidx[3 * t + 2];
            eofs[t] = off[n1];
            off[n1] += mx - s0 + 1;
        }
    }
    __syncthreads();
    // rows of T2 (triple t, budget index j = B' - |t|) in the order pass 2 writes them: T1's order,
    // or slice by slice (slice nu1 = v holds C(m_x - v + 3, 3) rows, after C(m_x + 4, 4) -
    // C(m_x - v + 4, 4) rows of the slices before it)
    for (int t = threadIdx.x; t < nk; t += blockDim.x) {
        const int tk = kid[t], n1 = tk & 255, s0 = n1 + ((tk >> 8) & 255) + (tk >> 16);
        const int base = SL ? ne - binom4(mx - n1 + 4) + eofs[t] : eof[t];
        for (int j = 0; j <= mx - s0; ++j) rs[base + j] = t | (j << 16);
    }
    // target locals of this thread's pass-3 items (nu, X1, X2), cells X3, kept in registers
    constexpr int Q3 = 2 * FG;  // items per thread: nk * FG <= 2 * blockDim.x
    const int nit3 = nk * FG * FG;
    R lamr[Q3][FG];
#pragma unroll
    for (int q = 0; q < Q3; ++q)
#pragma unroll
        for (int z = 0; z < FG; ++z) lamr[q][z] = R(0);
    int js[2], nj = 0;
    if (k >= 2) {
        if (k % 2 == 0) { js[0] = k - 2; nj = 1; }
        else { js[0] = k - 3; js[1] = k - 2; nj = 2; }
    }
    const int no = 2 * G - 1, nitems = nk * FG;
    const int j_lo = split ? term / na : 0, j_hi = split ? j_lo + 1 : nj;
    const int a_lo = split ? term % na : 0, a_hi = split ? a_lo + 1 : na;
    if (split && j_lo >= nj) return;  // this (k) has fewer source intervals
    for (int jj = j_lo; jj < j_hi; ++jj) {
        const int J = js[jj], D = k - J;
        for (int a = a_lo; a < a_hi; ++a) {
            __syncthreads();
            const R *mJ = mu + ((size_t)rhs * A.nint + J) * A.nbox * na * nk;
            for (int i = threadIdx.x; i < nk * C3; i += blockDim.x) {  // consecutive threads: consecutive kappa
                int c = i / nk, ik = i % nk, box = cbx[c];
                U[ik * CS + c] = box >= 0 ? mJ[((size_t)box * na + a) * nk + ik] : R(0);
            }
            const R *Eab = E1 + (size_t)(((D - 2) * na + a) * na + b) * no * esz;
            for (int i = threadIdx.x; i < 7 * esz; i += blockDim.x) {
                int o = i / esz - 3;  // offset X - Y
                Es[i] = (o >= -(G - 1) && o <= G - 1 && (o < 0 ? -o : o) <= A.ntr) ? Eab[(o + G - 1) * esz + i % esz]
                                                                                      : R(0);
            }
            const R coef = pref[((D - 2) * na + a) * na + b];
            __syncthreads();
            // pass 1 (direction x): unit = (triple (nu1, k2, k3), Y2, Y3); registers: cells X1.  The
            // budget loop over B is a prefix sum (T1 holds the cumulative budget), so a unit is a
            // sequential chain of 1 .. m_x + 1 steps; units are spread over all threads
            for (int u = threadIdx.x; u < nitems * FG; u += blockDim.x) {
                const int z = u % FG, Y2 = (u / FG) % FG, t = u / (FG * FG), tk = kid[t];
                const int nu1 = tk & 255, k2 = (tk >> 8) & 255, k3 = tk >> 16, s0 = nu1 + k2 + k3;
                R acc[FG];
#pragma unroll
                for (int x = 0; x < FG; ++x) acc[x] = R(0);
                for (int B = s0; B <= mx; ++B) {
                    const int k1 = B - s0;
                    const R *mrow = U + kin[(k1 * m1 + k2) * m1 + k3] * CS + Y2 * FG + z;
                    R e[7];
#pragma unroll
                    for (int o = 0; o < 7; ++o) e[o] = Es[o * esz + k1 * m1 + nu1];
#pragma unroll
                    for (int Y1 = 0; Y1 < FG; ++Y1) {
                        const R mv = mrow[Y1 * FG * FG];
#pragma unroll
                        for (int X1 = 0; X1 < FG; ++X1) acc[X1] += e[X1 - Y1 + 3] * mv;
                    }
                    R *out = T1s + (eof[t] + k1) * CS + Y2 * FG + z;
#pragma unroll
                    for (int X1 = 0; X1 < FG; ++X1) out[X1 * FG * FG] = acc[X1];
                }
            }
            __syncthreads();
            for (int sl = 0; sl < (SL ? m1 : 1); ++sl) {
            if (SL && sl > 0) __syncthreads();  // the previous slice's pass 3 is done with U
            // pass 2 (direction y): unit = (row (triple (nu1, nu2, k3), budget B'), X1, Y3); registers:
            // cells X2; T2 -> U.  One budget value per unit keeps the chains short (at most m_x + 1
            // steps) and spreads a slice's rows over all threads
            const int r0 = SL ? ne - binom4(mx - sl + 4) : 0;
            const int r1 = SL ? ne - binom4(mx - sl + 3) : ne;
            for (int u = r0 * FG * FG + threadIdx.x; u < r1 * FG * FG; u += blockDim.x) {
                const int z = u % FG, X1 = (u / FG) % FG, rw = rs[u / (FG * FG)];
                const int t = rw & 0xffff, j = rw >> 16, tk = kid[t];
                const int nu1 = tk & 255, nu2 = (tk >> 8) & 255, k3 = tk >> 16;
                R acc[FG];
#pragma unroll
                for (int y = 0; y < FG; ++y) acc[y] = R(0);
                for (int k2 = 0; k2 <= j; ++k2) {
                    const int row = eof[kin[(nu1 * m1 + k2) * m1 + k3]] + (j - k2);
                    const R *trow = T1s + row * CS + X1 * FG * FG + z;
                    R e[7];
#pragma unroll
                    for (int o = 0; o < 7; ++o) e[o] = Es[o * esz + k2 * m1 + nu2];
#pragma unroll
                    for (int Y2 = 0; Y2 < FG; ++Y2) {
                        const R tv = trow[Y2 * FG];
#pragma unroll
                        for (int X2 = 0; X2 < FG; ++X2) acc[X2] += e[X2 - Y2 + 3] * tv;
                    }
                }
                R *out = U + (u / (FG * FG) - r0) * CS + X1 * FG * FG + z;
#pragma unroll
                for (int X2 = 0; X2 < FG; ++X2) out[X2 * FG] = acc[X2];
            }
            __syncthreads();
            // pass 3 (direction z): item = (nu, X1, X2), fixed per thread; registers: cells X3
#pragma unroll
            for (int q = 0; q < Q3; ++q) {
                const int it = threadIdx.x + q * blockDim.x;
                if (it >= nit3) break;
                const int iv = it / (FG * FG), X1 = (it / FG) % FG, X2 = it % FG, tk = kid[iv];
                const int nu1 = tk & 255, nu2 = (tk >> 8) & 255, nu3 = tk >> 16, smax = mx - nu1 - nu2 - nu3;
                if (SL && nu1 != sl) continue;
                R acc[FG];
#pragma unroll
                for (int z = 0; z < FG; ++z) acc[z] = R(0);
                for (int k3 = 0; k3 <= smax; ++k3) {
                    const int t2 = kin[(nu1 * m1 + nu2) * m1 + k3];
                    const int row = (SL ? eofs[t2] : eof[t2]) + (mx - nu3 - nu1 - nu2 - k3);
                    const R *trow = U + row * CS + X1 * FG * FG + X2 * FG;
                    R e[7];
#pragma unroll
                    for (int o = 0; o < 7; ++o) e[o] = Es[o * esz + k3 * m1 + nu3];
                    R tv[FG];
#pragma unroll
                    for (int Y3 = 0; Y3 < FG; ++Y3) tv[Y3] = trow[Y3];
#pragma unroll
                    for (int X3 = 0; X3 < FG; ++X3)
#pragma unroll
                        for (int Y3 = 0; Y3 < FG; ++Y3) acc[X3] += e[X3 - Y3 + 3] * tv[Y3];
                }
#pragma unroll
                for (int X3 = 0; X3 < FG; ++X3) lamr[q][X3] += coef * acc[X3];
            }
            }  // slices
        }
    }
    // write the locals of the non-empty target boxes (intervals 0 and 1 get zeros); split mode:
    // this term's slice of the workspace
    R *lk = (split ? part + (size_t)term * nrhs * A.nint * A.nbox * na * nk : lam) +
            ((size_t)rhs * A.nint + k) * A.nbox * na * nk;
#pragma unroll
    for (int q = 0; q < Q3; ++q) {
        const int it = threadIdx.x + q * blockDim.x;
        if (it >= nit3) break;
        const int iv = it / (FG * FG), X1 = (it / FG) % FG, X2 = it % FG;
        if (X1 >= G || X2 >= G) continue;
#pragma unroll
        for (int X3 = 0; X3 < FG; ++X3) {
            if (X3 >= G) continue;
            const int box = A.cellbox[(X1 * G + X2) * G + X3];
            if (box >= 0) lk[((size_t)box * na + b) * nk + iv] = lamr[q][X3];
        }
    }
}

// lam = sum of the term slices in term order; interval k has nj(k) * na terms (nj = 0 for k < 2,
// 1 for even k, 2 for odd k): the slices of the other terms are never written and are not read
template <typename R>
__global__ void k_m2l_sum_terms(const R *__restrict__ part, int na, size_t n, size_t per_k, int nint,
                                R *__restrict__ lam)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = (int)((i / per_k) % nint);
    const int nterm = k < 2 ? 0 : (k % 2 == 0 ? na : 2 * na);
    R s = R(0);
    for (int t = 0; t < nterm; ++t) s += part[(size_t)t * n + i];
    lam[i] = s;
}

// M2L for grids of 5^3 .. 8^3 cells (FP32), one CTA per (target interval k, time node b, target
// x-slab X1, rhs) over all source terms (J, a) of the interaction list.  The three directional
// passes of k_m2l_fused restricted to one X1: pass 1 streams the source x-slabs Y1 within the
// interaction radius through shared memory (the moments of one slab, cells (Y2, Y3)) and adds
// their budget chains into T1(X1, Y2, Y3); pass 2 (registers: X2) and pass 3 (registers: X3)
// need only this slab of T1 and T2.  The locals of the slab's cells (X2, X3) accumulate in
// shared memory over the terms, so each is written once (no partials).  Same arithmetic as the
// three-pass kernels; cells beyond G are empty.
constexpr int SG = 8;  // padded grid extent per direction
constexpr int kM2LSlabThreads = 512;

// asynchronous global -> shared copy of one element of B = 4 or 8 bytes (zero fill when !valid),
// its commit and wait
template <int B>
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "n"(B), "r"(valid ? B : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename R>
__global__ void __launch_bounds__(kM2LSlabThreads, 1) k_m2l_slab(M2LArgs A, const R *__restrict__ mu,
                                                                  const R *__restrict__ E1, const R *__restrict__ pref,
                                                                  R *__restrict__ lam)
{
    extern __shared__ __align__(16) unsigned char slab_raw[];
    constexpr int SC = SG * SG, SCS = SC + 1, NO = 2 * SG - 1;
    const int G = A.G, nk = A.nk, ne = A.ne, mx = A.mx, m1 = mx + 1, na = A.na, esz = m1 * m1;
    R *Ms = reinterpret_cast<R *>(slab_raw);  // [nk][SCS]  moments of one source slab Y1, cells (Y2, Y3)
    R *Ms2 = Ms + nk * SCS;                    // [nk][SCS]  the next source slab (double buffer)
    R *T1s = Ms2 + nk * SCS;                   // [ne][SCS]  cells (Y2, Y3) at X1
    R *T2s = T1s + ne * SCS;                   // [ne][SCS]  cells (X2, Y3) at X1
    R *Ls = T2s + ne * SCS;                    // [nk][SCS]  locals, cells (X2, X3) at X1
    R *Es = Ls + nk * SCS;                     // [NO][m1][m1] offsets -(SG-1)..SG-1, zero outside the radius
    int *kid = reinterpret_cast<int *>(Es + NO * esz);
    int *kin = kid + nk;
    int *eof = kin + m1 * m1 * m1;
    int *cbx = eof + nk;  // [SG^3] padded cell -> box or -1
    const int X1 = blockIdx.x % G, kb = blockIdx.x / G;
    const int k = kb / na, b = kb % na, rhs = blockIdx.y;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
        kid[i] = A.kidx[3 * i] | (A.kidx[3 * i + 1] << 8) | (A.kidx[3 * i + 2] << 16);
        eof[i] = A.eoff[i];
    }
    for (int i = threadIdx.x; i < m1 * m1 * m1; i += blockDim.x) kin[i] = A.kinv[i];
    for (int i = threadIdx.x; i < SG * SC; i += blockDim.x) {
        const int x = i / SC, y = (i / SG) % SG, z = i % SG;
        cbx[i] = (x < G && y < G && z < G) ? A.cellbox[(x * G + y) * G + z] : -1;
    }
    for (int i = threadIdx.x; i < nk * SCS; i += blockDim.x) Ls[i] = R(0);
    int js[2], nj = 0;
    if (k >= 2) {
        if (k % 2 == 0) { js[0] = k - 2; nj = 1; }
        else { js[0] = k - 3; js[1] = k - 2; nj = 2; }
    }
    const int no = 2 * G - 1;
    const int y_lo = max(0, X1 - A.ntr), y_hi = min(G - 1, X1 + A.ntr);
    for (int jj = 0; jj < nj; ++jj) {
        const int J = js[jj], D = k - J;
        const R *mJ = mu + ((size_t)rhs * A.nint + J) * A.nbox * na * nk;
        for (int a = 0; a < na; ++a) {
            __syncthreads();  // the previous term's passes are done with Es, T1s, T2s
            const R *Eab = E1 + (size_t)(((D - 2) * na + a) * na + b) * no * esz;
            for (int i = threadIdx.x; i < NO * esz; i += blockDim.x) {
                const int o = i / esz - (SG - 1);  // offset X - Y
                Es[i] = (o >= -(G - 1) && o <= G - 1 && (o < 0 ? -o : o) <= A.ntr) ? Eab[(o + G - 1) * esz + i % esz]
                                                                                      : R(0);
            }
            for (int i = threadIdx.x; i < ne * SCS; i += blockDim.x) T1s[i] = R(0);
            const R coef = pref[((D - 2) * na + a) * na + b];
            // pass 1 (direction x): unit = (triple (nu1, k2, k3), cell (Y2, Y3)); per source slab Y1
            // the budget chain over B is added into T1 (the cumulative budget).  The moments of slab
            // Y1 + 1 are copied asynchronously into the other buffer while slab Y1 is used
            auto load_slab = [&](int Y1, R *dst) {  // consecutive threads: consecutive kappa
                for (int i = threadIdx.x; i < nk * SC; i += blockDim.x) {
                    const int c = i / nk, ik = i % nk, box = cbx[Y1 * SC + c];
                    cp_async_elem<sizeof(R)>(dst + ik * SCS + c, box >= 0 ? mJ + ((size_t)box * na + a) * nk + ik : mJ,
                                             box >= 0);
                }
                cp_async_commit();
            };
            load_slab(y_lo, Ms);
            for (int Y1 = y_lo; Y1 <= y_hi; ++Y1) {
                R *Mc = ((Y1 - y_lo) & 1) ? Ms2 : Ms;
                if (Y1 < y_hi) {
                    load_slab(Y1 + 1, ((Y1 - y_lo) & 1) ? Ms : Ms2);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();  // slab Y1 in place for every thread; Es and T1s ready
                const R *Eo = Es + (X1 - Y1 + SG - 1) * esz;
                for (int u = threadIdx.x; u < nk * SC; u += blockDim.x) {
                    const int c = u % SC, t = u / SC, tk = kid[t];
                    const int nu1 = tk & 255, k2 = (tk >> 8) & 255, k3 = tk >> 16, s0 = nu1 + k2 + k3;
                    R acc = R(0);
                    for (int B = s0; B <= mx; ++B) {
                        const int k1 = B - s0;
                        acc += Eo[k1 * m1 + nu1] * Mc[kin[(k1 * m1 + k2) * m1 + k3] * SCS + c];
                        T1s[(eof[t] + k1) * SCS + c] += acc;
                    }
                }
                __syncthreads();  // done with Mc before its refill two slabs later
            }
            // pass 2 (direction y): unit = (triple (nu1, nu2, k3), Y3); registers: cells X2
            for (int u = threadIdx.x; u < nk * SG; u += blockDim.x) {
                const int Y3 = u % SG, t = u / SG, tk = kid[t];
                const int nu1 = tk & 255, nu2 = (tk >> 8) & 255, k3 = tk >> 16, s0 = nu1 + nu2 + k3;
                for (int Bp = s0; Bp <= mx; ++Bp) {
                    R acc[SG];
#pragma unroll
                    for (int x = 0; x < SG; ++x) acc[x] = R(0);
                    for (int k2 = 0; k2 <= Bp - s0; ++k2) {
                        const int row = eof[kin[(nu1 * m1 + k2) * m1 + k3]] + (Bp - nu2 - nu1 - k2 - k3);
                        const R *trow = T1s + row * SCS + Y3;
                        R e[NO];
#pragma unroll
                        for (int o = 0; o < NO; ++o) e[o] = Es[o * esz + k2 * m1 + nu2];
#pragma unroll
                        for (int Y2 = 0; Y2 < SG; ++Y2) {
                            const R tv = trow[Y2 * SG];
#pragma unroll
                            for (int X2 = 0; X2 < SG; ++X2) acc[X2] += e[X2 - Y2 + SG - 1] * tv;
                        }
                    }
                    R *out = T2s + (eof[t] + Bp - s0) * SCS + Y3;
#pragma unroll
                    for (int X2 = 0; X2 < SG; ++X2) out[X2 * SG] = acc[X2];
                }
            }
            __syncthreads();
            // pass 3 (direction z): item = (nu, X2); registers: cells X3; locals += coef * sum
            for (int it = threadIdx.x; it < nk * SG; it += blockDim.x) {
                const int X2 = it % SG, iv = it / SG, tk = kid[iv];
                const int nu1 = tk & 255, nu2 = (tk >> 8) & 255, nu3 = tk >> 16, smax = mx - nu1 - nu2 - nu3;
                R acc[SG];
#pragma unroll
                for (int x = 0; x < SG; ++x) acc[x] = R(0);
                for (int k3 = 0; k3 <= smax; ++k3) {
                    const int row = eof[kin[(nu1 * m1 + nu2) * m1 + k3]] + (mx - nu3 - nu1 - nu2 - k3);
                    const R *trow = T2s + row * SCS + X2 * SG;
                    R e[NO];
#pragma unroll
                    for (int o = 0; o < NO; ++o) e[o] = Es[o * esz + k3 * m1 + nu3];
#pragma unroll
                    for (int Y3 = 0; Y3 < SG; ++Y3) {
                        const R tv = trow[Y3];
#pragma unroll
                        for (int X3 = 0; X3 < SG; ++X3) acc[X3] += e[X3 - Y3 + SG - 1] * tv;
                    }
                }
                R *lrow = Ls + iv * SCS + X2 * SG;
#pragma unroll
                for (int X3 = 0; X3 < SG; ++X3) lrow[X3] += coef * acc[X3];
            }
        }
    }
    __syncthreads();
    // the locals of the non-empty target boxes of this slab (intervals 0 and 1: zeros)
    R *lk = lam + ((size_t)rhs * A.nint + k) * A.nbox * na * nk;
    for (int i = threadIdx.x; i < nk * SC; i += blockDim.x) {
        const int c = i / nk, iv = i % nk, X2 = c / SG, X3 = c % SG;
        if (X2 >= G || X3 >= G) continue;
        const int box = cbx[X1 * SC + c];
        if (box >= 0) lk[((size_t)box * na + b) * nk + iv] = Ls[iv * SCS + c];
    }
}

size_t m2l_slab_smem(int nk, int ne, int mx, size_t es)
{
    const int SCS = SG * SG + 1, m1 = mx + 1;
    return es * ((size_t)(3 * nk + 2 * ne) * SCS + (size_t)(2 * SG - 1) * m1 * m1) +
           4 * ((size_t)2 * nk + (size_t)m1 * m1 * m1 + SG * SG * SG);
}

// padded grid extent of the fused kernel for a G^3 grid
int m2l_fused_fg(int G) { return G <= 2 ? 2 : FGMax; }

size_t m2l_fused_smem(int G, int nk, int ne, int mx, size_t es, bool sliced)
{
    const int FG = m2l_fused_fg(G), CS = FG * FG * FG + 1, m1 = mx + 1;
    const size_t urows = sliced ? (size_t)nk : (size_t)std::max(ne, nk);
    return es * (((size_t)ne + urows) * CS + (size_t)7 * m1 * m1) +
           4 * ((size_t)3 * nk + (size_t)m1 * m1 * m1 + FG * FG * FG + ne);
}

// Which M2L kernel a level takes (prec: 0 FP64, 1 FP32, 2 double-FP32): the fused kernel for FP32
// grids of at most 4^3 cells whose intermediates fit its shared memory (m_x <= 7; double-FP32:
// m_x <= 6 at one CTA per SM), the slab kernel
// for FP32 grids of 5^3 .. 8^3 cells with m_x <= 6 (its per-thread arrays and shared memory are
// sized for that), else the three separable passes through the global workspace (the 8-byte
// formats, larger grids or degrees).  FP32 degrees whose full T2 does not fit the fused kernel
// (m_x = 8) take its sliced form (T2 one nu1 value at a time).
int m2l_engine(int prec, int G, int nk, int ne, int mx)
{
    // double-FP32: the fused kernel at one CTA per SM when its 8-byte intermediates fit the
    // 227 KB of shared memory a CTA may hold (m_x <= 6)
    const int FG = m2l_fused_fg(G);
    if (prec == 2 && G <= FG && m2l_fused_smem(G, nk, ne, mx, 8, false) <= 227 * 1024 && nk * FG <= 2 * kM2LThreads)
        return kM2LFused;
    if (prec != 1) return kM2LThreePass;
    if (G <= FG && m2l_fused_smem(G, nk, ne, mx, 4, false) <= 200 * 1024 && nk * FG <= 2 * kM2LThreads)
        return kM2LFused;
    if (G <= FG && m2l_fused_smem(G, nk, ne, mx, 4, true) <= 227 * 1024 && nk * FG <= 2 * kM2LThreads)
        return kM2LFusedSliced;
    if (G > FGMax && G <= SG && mx <= 6 && m2l_slab_smem(nk, ne, mx, 4) <= 220 * 1024 && nk <= 256) return kM2LSlab;
    return kM2LThreePass;
}

int m2l_engine_for(int prec, int G, int nk, int ne, int mx, int force)
{
    const int def = m2l_engine(prec, G, nk, ne, mx);
    const int FG = m2l_fused_fg(G);
    const size_t es = prec == 1 ? 4 : 8, cap = prec == 1 ? 200 * 1024 : 227 * 1024;
    const bool fits_fused = prec != 0 && G <= FG && nk * FG <= 2 * kM2LThreads;
    switch (force) {
    case 1:  // PFMM_M2L_THREE_PASS
        return kM2LThreePass;
    case 2:  // PFMM_M2L_FUSED
        return fits_fused && m2l_fused_smem(G, nk, ne, mx, es, false) <= cap ? kM2LFused : def;
    case 4:  // PFMM_M2L_FUSED_SLICED
        return fits_fused && m2l_fused_smem(G, nk, ne, mx, es, true) <= 227 * 1024 ? kM2LFusedSliced : def;
    default:
        return def;
    }
}

// Runs the three passes over chunks of target intervals so that the intermediates fit the
// workspace (ws_elems elements of R for each of T1 and T2).
int launch_m2l(int prec, const DevLevel &L, int l, const void *mu, void *lam, int nrhs, const ApplyGeo &g,
               void *T1, void *T2, size_t ws_elems, cudaStream_t st)
{
    (void)l;
    const size_t es = prec == 1 ? 4 : 8;
    const int G3 = L.G * L.G * L.G, na = g.na;
    const int engine = m2l_engine_for(prec, L.G, g.nk, g.ne, g.mx, g.m2l_force);
    const char *mb = (const char *)mu + L.mom_off * es * nrhs;
    char *lb = (char *)lam + L.mom_off * es * nrhs;
    int rc = 0;
    dispatch_prec(prec, [&](auto tag) {
        using R = decltype(tag);
        if (engine == kM2LFused || engine == kM2LFusedSliced) {
            const bool sl = engine == kM2LFusedSliced;
            const size_t fsm = m2l_fused_smem(L.G, g.nk, g.ne, g.mx, es, sl);
            M2LArgs A{L.G, L.ntr, na, g.nk, g.mx, g.ne, L.nint, L.nbox, L.cellbox, L.boxcell, L.pk, L.pJ, 0,
                      g.kidx, g.kinv, g.eoff};
            // few (interval, node) CTAs: one CTA per source term as well, when the terms' partial
            // locals fit the workspace
            const size_t per_k = (size_t)L.nbox * na * g.nk, nlev = (size_t)nrhs * L.nint * per_k;
            const int nterm = 2 * na;
            const int64_t split_ctas = (int64_t)kM2LSplitCtasPerSm * (g.nsm > 0 ? g.nsm : 152);
            const int split = ((int64_t)L.nint * na * nrhs < split_ctas && (size_t)nterm * nlev <= ws_elems) ? 1 : 0;
            const dim3 grd(L.nint * na * (split ? nterm : 1), nrhs);
            auto kf = m2l_fused_fg(L.G) == 2 ? (sl ? k_m2l_fused<R, 2, true> : k_m2l_fused<R, 2, false>)
                                             : (sl ? k_m2l_fused<R, FGMax, true> : k_m2l_fused<R, FGMax, false>);
            cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
            kf<<<grd, kM2LThreads, fsm, st>>>(A, (const R *)mb, (const R *)L.E1, (const R *)L.pref, (R *)lb, nrhs,
                                              split, (R *)T1);
            if (split)
                k_m2l_sum_terms<R><<<(unsigned)((nlev + 255) / 256), 256, 0, st>>>((const R *)T1, na, nlev, per_k,
                                                                                  L.nint, (R *)lb);
            return;
        }
        if (engine == kM2LSlab) {
            const size_t ssm = m2l_slab_smem(g.nk, g.ne, g.mx, es);
            M2LArgs A{L.G, L.ntr, na, g.nk, g.mx, g.ne, L.nint, L.nbox, L.cellbox, L.boxcell, L.pk, L.pJ, 0,
                      g.kidx, g.kinv, g.eoff};
            cudaFuncSetAttribute(k_m2l_slab<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
            k_m2l_slab<R><<<dim3((unsigned)(L.nint * na * L.G), nrhs), kM2LSlabThreads, ssm, st>>>(
                A, (const R *)mb, (const R *)L.E1, (const R *)L.pref, (R *)lb);
            return;
        }
        const size_t per_pair = (size_t)nrhs * na * na * G3 * g.ne;
        // intervals 0 and 1 have no interaction list: their locals start at zero
        for (int r = 0; r < nrhs; ++r)
            cudaMemsetAsync(lb + es * (size_t)r * L.nint * L.nbox * na * g.nk, 0,
                            es * (size_t)L.nbox * na * g.nk * std::min(2, L.nint), st);
        int k = 2;
        while (k < L.nint) {
            // largest chunk [k, k1) whose problem pairs fit the workspace
            int k1 = k, p0 = L.kptr_host[k];
            while (k1 < L.nint && (size_t)(L.kptr_host[k1 + 1] - p0) * per_pair <= ws_elems) k1++;
            if (k1 == k) {  // a single interval does not fit: workspace too small
                rc = -1;
                return;
            }
            const int npair = L.kptr_host[k1] - p0;
            M2LArgs A{L.G, L.ntr, na, g.nk, g.mx, g.ne, L.nint, L.nbox, L.cellbox, L.boxcell, L.pk + p0, L.pJ + p0,
                      npair, g.kidx, g.kinv, g.eoff};
            const size_t n12 = (size_t)nrhs * npair * na * na * G3 * g.nk;
            const unsigned b12 = (unsigned)((n12 + 127) / 128);
            const size_t n3 = (size_t)nrhs * (k1 - k) * L.nbox * na * g.nk;
            const unsigned b3 = (unsigned)((n3 + 127) / 128);
            k_m2l_s1<R><<<b12, 128, 0, st>>>(A, (const R *)mb, (const R *)L.E1, (R *)T1, nrhs);
            k_m2l_s2<R><<<b12, 128, 0, st>>>(A, (const R *)L.E1, (const R *)T1, (R *)T2, nrhs);
            k_m2l_s3<R><<<b3, 128, 0, st>>>(A, (const R *)L.E1, (const R *)L.pref, (const R *)T2, (R *)lb, L.kptr, p0, k,
                                            k1, nrhs);
            k = k1;
        }
    });
    return rc;
}

// ------------------------------------------------------------------------------------------
// L2L from level l-1 to level l (transposes of Eq. temp_m2m, st_m2m): thread per child local.
template <typename R>
__global__ void k_l2l(const R *__restrict__ lam_p, R *__restrict__ lam_c, const int *__restrict__ parent,
                      const int *__restrict__ oct_c, const R *__restrict__ q1, const R *__restrict__ qt,
                      const int *__restrict__ kidx, const int *__restrict__ kinv, int st, int na, int nk, int mx,
                      int nint_c, int nbox_c, int nbox_p, int nrhs)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nrhs * nint_c * nbox_c * na * nk;
    if (gid >= total) return;
    int ik = gid % nk;
    size_t r_ = gid / nk;
    int bcI = r_ % na;
    r_ /= na;
    int bc = r_ % nbox_c;
    r_ /= nbox_c;
    int kc = r_ % nint_c;
    int rhs = (int)(r_ / nint_c);
    const int m1 = mx + 1;
    int kp = kc >> 1, c = kc & 1, bp = parent[bc], oc = oct_c[bc];
    const R *qa = q1 + (oc & 1) * m1 * m1, *qb = q1 + ((oc >> 1) & 1) * m1 * m1, *qc = q1 + ((oc >> 2) & 1) * m1 * m1;
    int k0 = kidx[3 * ik], k1 = kidx[3 * ik + 1], k2 = kidx[3 * ik + 2];
    const R *lp = lam_p + (((size_t)rhs * (nint_c >> 1) + kp) * nbox_p + bp) * na * nk;
    R acc = R(0);
    for (int bpI = 0; bpI < na; ++bpI) {
        R qtv = qt[(c * na + bcI) * na + bpI];
        const R *l = lp + bpI * nk;
        if (!st) {
            acc += qtv * l[ik];
        } else {
            R s = R(0);
            for (int n0 = k0; n0 <= mx; ++n0)
                for (int n1 = k1; n0 + n1 <= mx; ++n1)
                    for (int n2 = k2; n0 + n1 + n2 <= mx; ++n2)
                        s += qa[k0 * m1 + n0] * qb[k1 * m1 + n1] * qc[k2 * m1 + n2] * l[kinv[(n0 * m1 + n1) * m1 + n2]];
            acc += qtv * s;
        }
    }
    lam_c[gid] += acc;
}

void launch_l2l(int prec, const DevLevel &par, const DevLevel &ch, int l, const void *qt, void *lam, int nrhs,
                const ApplyGeo &g, int64_t mu_stride, cudaStream_t st)
{
    (void)l;
    (void)mu_stride;
    const size_t total = (size_t)nrhs * ch.nint * ch.nbox * g.na * g.nk;
    const unsigned blocks = (unsigned)((total + 127) / 128);
    const size_t es = prec == 1 ? 4 : 8;
    char *base = (char *)lam;
    const int m1 = g.mx + 1;
    dispatch_prec(prec, [&](auto tag) {
        using R = decltype(tag);
        const R *lp = (const R *)(base + par.mom_off * es * nrhs);
        R *lc = (R *)(base + ch.mom_off * es * nrhs);
        if (ch.st) {
            const size_t smem = es * ((size_t)2 * g.na * g.nk + 2 * m1 * m1) + 4 * (size_t)m1 * m1 * m1;
            const dim3 grd(par.nint * par.nbox * 8, nrhs);  // one CTA per (parent, child slot); empty slots exit
            k_l2l_st<R><<<grd, 256, smem, st>>>(lp, lc, par.ch_ptr, par.ch_idx, ch.octant, (const R *)ch.qx,
                                                (const R *)qt, g.kidx, g.kinv, g.na, g.nk, g.mx, par.nint, par.nbox,
                                                ch.nbox);
            return;
        }
        k_l2l<R><<<blocks, 128, 0, st>>>(lp, lc, ch.parent, ch.octant, (const R *)ch.qx, (const R *)qt, g.kidx,
                                         g.kinv, ch.st, g.na, g.nk, g.mx, ch.nint, ch.nbox, par.nbox, nrhs);
    });
}

// ------------------------------------------------------------------------------------------
// L2T at the leaves (Eq. l2t): f[k ls + s][x] += sum_b St[s][b] sum_nu lam[k][X][b][nu] Sx[x][nu].
template <typename R>
__global__ void __launch_bounds__(256) k_l2t(const R *__restrict__ lam, const R *__restrict__ Sx, const R *__restrict__ St,
                                               double *__restrict__ f, const int *__restrict__ leaf_start, int nk, int na,
                                               int ls, int Et, int nint, int nbox, int nt, const int *__restrict__ tiles,
                                               const R *__restrict__ Qg, int i0, int nkc)
{
    // the multi-indices nu = i0 .. i0 + nkc - 1 (one launch per chunk when n_kappa is large; the
    // launches add into f one after the other)
    // a CTA covers one 64-row tile of a leaf box (tiles: (box, first row); without a tile list, the
    // whole box), kTSB steps and one rhs: Q[ts][nu] = sum_b St[s][b] lam[k][X][b][nu] in shared
    // memory, then thread (tg = warp, xl = lane) forms steps 4 tg .. 4 tg + 3 for the triangles xl
    // and xl + 32 of each 64-triangle chunk
    extern __shared__ __align__(16) unsigned char l2t_raw[];
    R *Qs = reinterpret_cast<R *>(l2t_raw);  // [nkc][kTSP]: a thread's four steps are one vector load
    constexpr int XCH = 64, SP = XCH + 1;      // Sx chunk stored transposed, rows padded
    R *Ss = Qs + kTSP * nkc;                   // [nkc][SP]
    const int X = tiles ? tiles[2 * blockIdx.x] : blockIdx.x, rhs = blockIdx.z;
    const int ipb = kTSB / ls;
    const int k0 = blockIdx.y * ipb, kend = min(nint, k0 + ipb), nts = (kend - k0) * ls, t0 = k0 * ls;
    const int x0 = leaf_start[X] + (tiles ? tiles[2 * blockIdx.x + 1] : 0);
    const int x1 = tiles ? min(x0 + 64, leaf_start[X + 1]) : leaf_start[X + 1];
    for (int o = threadIdx.x; o < kTSB * nkc; o += blockDim.x) {
        const int ts = o / nkc, i = o % nkc;
        R v = R(0);
        if (ts < nts) {
            if (Qg) {  // precomputed by k_l2t_time
                v = Qg[(((size_t)rhs * Et + t0 + ts) * nbox + X) * nk + i0 + i];
            } else {
                const int kk = ts / ls, s = ts % ls;
                const R *lp = lam + ((((size_t)rhs * nint + k0 + kk) * nbox + X) * na) * nk + i0 + i;
                for (int b = 0; b < na; ++b) v += St[s * na + b] * lp[(size_t)b * nk];
            }
        }
        Qs[i * kTSP + ts] = v;
    }
    const int xl = threadIdx.x & 31, tg = threadIdx.x >> 5;
    for (int xb = x0; xb < x1; xb += XCH) {
        const int nx = min(XCH, x1 - xb);
        __syncthreads();
        for (int e = threadIdx.x; e < XCH * nkc; e += blockDim.x) {  // coalesced reads along nu
            const int xi = e / nkc, i = e % nkc;
            Ss[i * SP + xi] = xi < nx ? Sx[(size_t)(xb + xi) * nk + i0 + i] : R(0);
        }
        __syncthreads();
        R acc[4][2];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = R(0);
        for (int i = 0; i < nkc; ++i) {
            const R s0 = Ss[i * SP + xl], s1 = Ss[i * SP + xl + 32];
            R q[4];
            lds4(Qs + i * kTSP + tg * 4, q);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                mac(acc[r][0], q[r], s0);
                mac(acc[r][1], q[r], s1);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int ts = tg * 4 + r;
            if (ts >= nts) continue;
            double *fr = f + ((size_t)rhs * Et + t0 + ts) * nt + xb;
            if (xl < nx) fr[xl] += as_double(acc[r][0]);
            if (xl + 32 < nx) fr[xl + 32] += as_double(acc[r][1]);
        }
    }
}

void launch_l2t(int prec, const void *lam_leaf, const void *Sx, const void *St, double *f_int, int nrhs,
                const ApplyGeo &g, int64_t mu_stride, cudaStream_t st, void *ws, size_t ws_elems)
{
    (void)mu_stride;
    const int nint = g.Et / g.ls;
    // temporal factor once per (step, box) in the workspace when it fits (else per CTA)
    const bool qg = ws && (size_t)nrhs * g.Et * g.nbox_leaf * g.nk <= ws_elems;
    const dim3 gq((unsigned)(nrhs * nint), (unsigned)((g.nbox_leaf * g.nk + 255) / 256));
    const int ipb = kTSB / g.ls;
    const size_t es = prec == 1 ? 4 : 8;
    constexpr int kL2TChunk = 256;  // multi-indices per launch: the shared memory of a CTA bounds it
    const int nkc_max = std::min(g.nk, kL2TChunk);
    const size_t smem = ((size_t)kTSP * nkc_max + (size_t)nkc_max * 65) * es;
    // one CTA per 64-row tile (balanced over leaf boxes of different sizes)
    const dim3 grd(g.tiles ? g.ntiles : g.nbox_leaf, (nint + ipb - 1) / ipb, nrhs);
    dispatch_prec(prec, [&](auto tag) {
        using R = decltype(tag);
        if (qg)
            k_l2t_time<R><<<gq, 256, 0, st>>>((const R *)lam_leaf, (const R *)St, (R *)ws, g.nk, g.na, g.ls, g.Et, nint,
                                              g.nbox_leaf);
        cudaFuncSetAttribute(k_l2t<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        for (int i0 = 0; i0 < g.nk; i0 += kL2TChunk)
            k_l2t<R><<<grd, 256, smem, st>>>((const R *)lam_leaf, (const R *)Sx, (const R *)St, f_int, g.leaf_start,
                                             g.nk, g.na, g.ls, g.Et, nint, g.nbox_leaf, g.nt, g.tiles,
                                             qg ? (const R *)ws : nullptr, i0, std::min(kL2TChunk, g.nk - i0));
    });
}

// ------------------------------------------------------------------------------------------
// f = M_h g: f[t][x] = h |gamma_x| / 3 * sum of g[t] over the vertices of gamma_x (Section 2).
__global__ void k_apply_M(const double *__restrict__ g, double *__restrict__ f, const int *__restrict__ tri,
                          const double *__restrict__ area, int nt, int nv, size_t total, double h)
{
    size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    size_t rt = gid / nt;
    int x = (int)(gid - rt * nt);
    const double *gr = g + rt * nv;
    f[gid] = h * area[x] / 3.0 * (gr[tri[3 * x]] + gr[tri[3 * x + 1]] + gr[tri[3 * x + 2]]);
}

void launch_apply_M(const double *g_in, double *f, const int *tri_user, const double *area, int nrhs, int nt, int nv,
                    int Et, double h, cudaStream_t st)
{
    size_t total = (size_t)nrhs * Et * nt;
    k_apply_M<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g_in, f, tri_user, area, nt, nv, total, h);
}

}  // namespace pfmm
