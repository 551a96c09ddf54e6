// kernels.h -- launch interfaces between the host orchestration (capi.cpp) and the CUDA files.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pfmm_internal.h"

namespace pfmm {

struct PanelGPU {  // device copy of Panel
    int index, row0, nrows, rows_pad;
    int ncolV, colsV_pad, ncolK, colsK_pad;
    long long offV, offK;
    int colV_at, colK_at;
};

struct SetupArgs {
    const double *verts;   // [nv][3]
    const int *tri;        // [nt][3] internal order
    const int *tri_leaf;   // [nt]
    const int *leaf_grid;  // [nbox_p][3]
    double corner[3], hx_leaf, hxp_leaf, alpha;
    int nt, mx, nk;
    const int *kidx;       // [nk][3] graded multi-indices
    const double *rule_tab;// collapsed rule s1[nq], s2[nq], w[nq] (exact for degree m_x)
    int nq_tab;
    double *Sx, *SK;       // [nt][nk], [nt][3][nk]
};

struct NfQuadArgs {
    const double *verts;
    const int *tri;        // internal order
    int nv, nd;            // nd = 2 leaf_steps step offsets
    double h, alpha;
    const double *rule_reg;// collapsed rule s1, s2, w (n_r^2 points)
    int nq_reg;
    const double *gl_sing; // Gauss-Legendre on [0,1]: x[n], w[n]
    int nq_sing;
    const int *colV;       // all panels' V columns
    const int *kmap;       // [npanel][nv]
};

void launch_space_tables(const SetupArgs &a, cudaStream_t st);
void launch_e1_table(int na, int mt, int mx, int G, double hx, double hxp, double ht, double alpha, double *E1,
                     double *pref, cudaStream_t st);
void launch_nf_regular(const NfQuadArgs &a, const PanelGPU &P, void *AV, void *AK, bool mixed, cudaStream_t st);
void launch_nf_singular(const NfQuadArgs &a, const int *sing, int nsing, const PanelGPU *panels, void *AV, void *AK,
                        bool mixed, cudaStream_t st, double *cV = nullptr, double *cK = nullptr);

// on-the-fly nearfield (quadrature fused into the apply, no stored panels)
struct OtfArgs {
    NfQuadArgs q;              // geometry, time step, regular rule
    const PanelGPU *panels;
    const int *tiles;          // [ntiles][2] (panel, first row) of 64-row tiles
    int ntiles;
    const int *tile_sing;      // [ntiles + 1] ranges of the singular list per tile
    const int *sing;           // [n][12] singular pairs (x, y, panel, row, colV, code, ...)
    const double *singV;       // [n][2] Sauter-Schwab values, d = 0, 1
    const double *singK;       // [n][2][3]
    const void *x;             // V: permuted input [rhs][Et][nt]; K: nodal input [rhs][Et][nv] (arithmetic type)
    int ncolg, Et, ls, nrhs, ndmax;
    double *f;                 // [rhs][Et][nt] internal rows, accumulated (+=)
    int nt;
};
// f += nearfield(x) with the panels recomputed tile by tile; kop: double layer (node columns)
void launch_nf_otf(bool mixed, bool kop, const OtfArgs &a, int nsm, cudaStream_t st);

// ---- apply ------------------------------------------------------------------------------
struct ApplyGeo {
    int nt, nv, Et, ls, nd, na, nk, mx, p;
    const int *perm;       // [nt] internal -> caller triangle
    const int *tri;        // [nt][3] internal order
    const int *leaf_start; // [nbox_p + 1]
    int nbox_leaf;
    const int *kidx;       // [nk][3] graded
    const int *kinv;       // [(m+1)^3] -> graded index
    int ne;                // C(m_x+4, 4): budget-indexed entries of the separable M2L intermediates
    const int *eoff;       // [nk] offset of the budget range of each triple
    const int *tiles;      // [ntiles][2] (leaf box, first row) of the 64-row tiles of every leaf box
    int ntiles;
    const int *box_tiles;  // [nbox_p + 1] first tile of each leaf box (tiles are box-major)
    int nsm;               // streaming multiprocessors of the device (grid sizing)
    int m2l_force;         // M2L engine asked for by the batch autotuner (PFMM_M2L_* code, 0: none)
};

// prec of the FMM launchers: 0 FP64, 1 FP32 (mixed mode), 2 double-FP32 (FP64 mode); every
// moment, local and table buffer holds 8-byte elements in modes 0 and 2, 4-byte ones in mode 1
void launch_permute_in(const double *w, void *w_int, bool to_float, int nrhs, const ApplyGeo &g, cudaStream_t st);
void launch_permute_out(const double *f_int, double *f, int nrhs, const ApplyGeo &g, cudaStream_t st);
void launch_cast_to_float(const double *x, float *y, size_t n, cudaStream_t st);
// rewrite n FP64 values in place as double-FP32 pairs (hi, lo) of the same 8 bytes
void launch_to_df64(double *x, size_t n, cudaStream_t st);
// FP32 panels held only as the tensor-core engine's FP16 parts: A = (hi + lo) * inv_scale
struct NfHalfSplit {
    const uint16_t *hi = nullptr, *lo = nullptr;  // FP16 bit patterns in 64 x 64 blocks (nf_tiled_index)
    float inv_scale = 1.f;                        // 2^-E of the split's scale (exact)
};
// Position of element (R, c) of the FP16 parts.  R is the global panel row (panel element offset /
// columns + d * rows_pad + r: every panel's step block starts at a multiple of 64 rows) and c the
// column of a layout with 64 * nkb columns; the parts are stored as contiguous 64-row x 64-column
// blocks (8 KB, 128-byte rows), block (R / 64, c / 64) at index (R / 64) * nkb + c / 64, so a
// tensor-core tile half is one contiguous copy.
__host__ __device__ inline size_t nf_tiled_index(size_t R, int c, int nkb)
{
    return (((R >> 6) * (size_t)nkb + (size_t)(c >> 6)) << 12) + ((R & 63) << 6) + (size_t)(c & 63);
}
void launch_nf_apply(bool mixed, bool kop, const void *A, const int *colidx, const int *tiles, int ntiles,
                     const PanelGPU *panels, const void *x, int ncolg, int nrhs, const ApplyGeo &g, double *f_int,
                     cudaStream_t st, int ndmax = 1 << 30,  // ndmax: only offsets d < ndmax
                     const NfHalfSplit *hs = nullptr);      // FP32 only: blocks from the FP16 parts, A unused
// ws: scratch of ws_elems elements of the arithmetic type for the per-tile partial moments (the
// M2L workspace, idle at this point); too small: one CTA per whole leaf box instead
void launch_s2m(int prec, bool kop, const void *x, int ncolg, const void *Stab /*Sx or SK*/, const void *St,
                void *mu_leaf, int nrhs, const ApplyGeo &g, cudaStream_t st, void *ws = nullptr, size_t ws_elems = 0);
void launch_m2m(int prec, const DevLevel &par, const DevLevel &ch, int l, const void *qt, void *mu, int nrhs,
                const ApplyGeo &g, int64_t mu_stride, cudaStream_t st);
int launch_m2l(int prec, const DevLevel &L, int l, const void *mu, void *lam, int nrhs, const ApplyGeo &g,
               void *T1, void *T2, size_t ws_elems, cudaStream_t st);
// M2L kernel of a level with a G^3 grid (launch_m2l's choice): only kM2LThreePass uses T1 / T2
enum { kM2LThreePass = 0, kM2LFused = 1, kM2LSlab = 2, kM2LFusedSliced = 3 };
int m2l_engine(int prec, int G, int nk, int ne, int mx);
// the engine of a level when an autotuner asks for `force` (a PFMM_M2L_* code; 0: none): the forced
// engine where it can run that level, else m2l_engine's choice
int m2l_engine_for(int prec, int G, int nk, int ne, int mx, int force);
void launch_l2l(int prec, const DevLevel &par, const DevLevel &ch, int l, const void *qt, void *lam, int nrhs,
                const ApplyGeo &g, int64_t mu_stride, cudaStream_t st);
// ws: scratch (ws_elems elements of the arithmetic type) for the temporal factor of every (step,
// leaf box), the M2L workspace idle at this point; too small: computed per CTA
void launch_l2t(int prec, const void *lam_leaf, const void *Sx, const void *St, double *f_int, int nrhs,
                const ApplyGeo &g, int64_t mu_stride, cudaStream_t st, void *ws = nullptr, size_t ws_elems = 0);
void launch_apply_M(const double *g_in, double *f, const int *tri_user, const double *area, int nrhs, int nt, int nv,
                    int Et, double h, cudaStream_t st);
// representation formula u[rhs][p] = V~ w - W g at the points pts [np][4] = (x, y, z, t)
// (caller's triangle and node order; g may be null: single-layer potential only)
void launch_repr(const double *verts, const int *tri, int nt, int nv, const double *rule, int nq, const double *w,
                 const double *g, const double *pts, int np, int nrhs, int Et, double h, double alpha, double *u,
                 cudaStream_t st);

}  // namespace pfmm
