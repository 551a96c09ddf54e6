// k_nf_otf.cu -- on-the-fly nearfield (Eq. eval_sl_nf_block, Alg. 2 last loop) without stored
// panels: the quadrature of a tile of the nearfield blocks is fused into its apply.
//
// Persistent CTAs over 64-row tiles of the target leaf boxes.  For every chunk of CH source
// triangles of the tile's interaction area:
//   phase 1: A_d[row][col] (d = 0 .. nd-1; K: three node columns per source triangle) by the same
//            regular collapsed-Gauss rule as the stored path (nf_regular_pair), plus the
//            Sauter-Schwab values of touching pairs at d = 0, 1 from a compact per-pair list
//            computed once at build time; held in shared memory only;
//   phase 2: f[t][row] += sum_d sum_col A_d[row][col] x[t - d][col] for every step t (d < ls + t mod
//            ls + 1, t - d >= 0) and right-hand side, in time blocks of 64 steps, the chunk's
//            partial sums (arithmetic type) added to the FP64 output rows the CTA owns.
// The quadrature is paid once per apply; only the compact singular list is stored.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"
#include "nf_geom.cuh"

namespace pfmm {

namespace {

constexpr int OT_R = 64;    // rows per tile
constexpr int OT_TB = 64;   // steps per time block
constexpr int OT_NDMAX = 8; // step offsets (2 leaf_steps) the kernel supports

template <typename R, bool KOP>
__global__ void __launch_bounds__(256) k_nf_otf(OtfArgs a, int CH, int WP)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nd = a.q.nd;
    const int CK = KOP ? 3 * CH : CH;        // shared-memory columns per chunk
    R *As = reinterpret_cast<R *>(sm_raw);   // [nd][CK][OT_R]
    R *Ws = As + (size_t)nd * CK * OT_R;     // [CK][WP]: steps tb0 - (nd - 1) ..
    const int tid = threadIdx.x, rg = tid & 15, cg = tid >> 4;
    const R *x = reinterpret_cast<const R *>(a.x);
    for (int item = blockIdx.x; item < a.ntiles; item += gridDim.x) {
        const PanelGPU P = a.panels[a.tiles[2 * item]];
        const int r0 = a.tiles[2 * item + 1];
        const int nrow = min(OT_R, P.nrows - r0);
        const int *cols = a.q.colV + P.colV_at;
        for (int c0 = 0; c0 < P.ncolV; c0 += CH) {
            const int nc = min(CH, P.ncolV - c0);
            __syncthreads();  // the previous chunk's phase 2 is done with As and Ws
            // ---- phase 1: quadrature of the chunk
            for (int e = tid; e < OT_R * CH; e += blockDim.x) {
                const int r = e % OT_R, c = e / OT_R;
                R acc[3 * OT_NDMAX];
#pragma unroll
                for (int q = 0; q < 3 * OT_NDMAX; ++q) acc[q] = R(0);
                const int y = (r < nrow && c < nc) ? cols[c0 + c] : -1;
                if (y >= 0) nf_regular_pair<R, KOP>(a.q, P.row0 + r0 + r, y, acc);
                for (int d = 0; d < nd; ++d) {
                    if (KOP) {
                        for (int v = 0; v < 3; ++v) As[((size_t)d * CK + 3 * c + v) * OT_R + r] = acc[3 * d + v];
                    } else {
                        As[((size_t)d * CK + c) * OT_R + r] = acc[d];
                    }
                }
            }
            __syncthreads();
            // touching pairs of this tile whose source lies in the chunk (distinct entries)
            for (int s = a.tile_sing[item] + tid; s < a.tile_sing[item + 1]; s += blockDim.x) {
                const int *sp = a.sing + 12 * (size_t)s;
                const int r = sp[3] - r0, c = sp[4] - c0;
                if (c < 0 || c >= nc) continue;
                for (int d = 0; d < 2 && d < nd; ++d) {
                    if (KOP) {
                        for (int v = 0; v < 3; ++v)
                            As[((size_t)d * CK + 3 * c + v) * OT_R + r] += R(a.singK[6 * (size_t)s + 3 * d + v]);
                    } else {
                        As[((size_t)d * CK + c) * OT_R + r] += R(a.singV[2 * (size_t)s + d]);
                    }
                }
            }
            const int cka = KOP ? 3 * nc : nc;  // active shared-memory columns
            // ---- phase 2: apply to every step and right-hand side
            for (int rhs = 0; rhs < a.nrhs; ++rhs) {
                const R *xr = x + (size_t)rhs * a.Et * a.ncolg;
                for (int tb0 = 0; tb0 < a.Et; tb0 += OT_TB) {
                    __syncthreads();  // As complete / Ws free
                    const int wt = OT_TB + nd - 1;
                    for (int e = tid; e < cka * wt; e += blockDim.x) {
                        const int cc = e / wt, tt = e % wt;
                        const int t = tb0 - (nd - 1) + tt;
                        R v = R(0);
                        if (t >= 0 && t < a.Et) {
                            const int c = KOP ? cc / 3 : cc;
                            const int y = cols[c0 + c];
                            if (y >= 0) {
                                const int col = KOP ? a.q.tri[3 * y + cc % 3] : y;
                                v = xr[(size_t)t * a.ncolg + col];
                            }
                        }
                        Ws[(size_t)cc * WP + tt] = v;
                    }
                    __syncthreads();
                    R acc[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = R(0);
                    int dcnt[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = tb0 + cg + 16 * j;
                        dcnt[j] = min(a.ls + t % a.ls + 1, a.ndmax);
                    }
                    for (int d = 0; d < nd; ++d) {
                        R msk[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) msk[j] = d < dcnt[j] ? R(1) : R(0);
                        const R *Ad = As + (size_t)d * CK * OT_R;
                        const int woff = cg + (nd - 1) - d;
                        for (int cc = 0; cc < cka; ++cc) {
                            R av[4], bv[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) av[i] = Ad[(size_t)cc * OT_R + rg + 16 * i];
#pragma unroll
                            for (int j = 0; j < 4; ++j) bv[j] = Ws[(size_t)cc * WP + woff + 16 * j] * msk[j];
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = tb0 + cg + 16 * j;
                        if (t >= a.Et) continue;
                        double *fr = a.f + ((size_t)rhs * a.Et + t) * a.nt + P.row0 + r0;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int r = rg + 16 * i;
                            if (r < nrow) fr[r] += (double)acc[i][j];
                        }
                    }
                }
            }
        }
    }
}

template <typename R, bool KOP>
void launch_T(const OtfArgs &a, int nsm, cudaStream_t st)
{
    const int nd = a.q.nd, es = (int)sizeof(R);
    const int per_col = nd * OT_R * es * (KOP ? 3 : 1);
    int CH = (150 * 1024 / per_col) / 16 * 16;
    CH = std::max(16, std::min(CH, 128));
    const int CK = KOP ? 3 * CH : CH;
    const int WP = (OT_TB + nd - 1 + 3) / 4 * 4;
    const size_t smem = ((size_t)nd * CK * OT_R + (size_t)CK * WP) * es;
    cudaFuncSetAttribute(k_nf_otf<R, KOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = std::min(a.ntiles, nsm);
    if (grid > 0) k_nf_otf<R, KOP><<<grid, 256, smem, st>>>(a, CH, WP);
}

}  // namespace

void launch_nf_otf(bool mixed, bool kop, const OtfArgs &a, int nsm, cudaStream_t st)
{
    if (mixed) {
        if (kop) launch_T<float, true>(a, nsm, st);
        else launch_T<float, false>(a, nsm, st);
    } else {
        if (kop) launch_T<double, true>(a, nsm, st);
        else launch_T<double, false>(a, nsm, st);
    }
}

}  // namespace pfmm
