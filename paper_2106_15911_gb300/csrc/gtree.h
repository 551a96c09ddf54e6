// gtree.h -- the space-time FMM for general (non-uniform) time steps: device descriptors of the
// general box cluster tree (Alg. 1 in full: early leaves, splits at the step nearest an
// interval's centre, the oversized-element stop) and the launch interface of its kernels
// (k_gen.cu).  Single layer V_h, FP64.  No Toeplitz structure: every nearfield block holds the
// entries of all its (target step, source step) pairs.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pfmm {

// one box Z = X x I of the general tree (global ids: the levels concatenated)
struct GBox {
    int t0, t1;    // internal triangles of X: [t0, t1)
    int a0, a1;    // time steps of I: [a0, a1) (step j is (t_j, t_{j+1}])
    int level, k;  // level and index k of I = I_k^(level)
    int cell[3];   // grid cell of X on its level
    int c0, c1;    // children [c0, c1) (global ids); c0 == c1 for a leaf
    int par;       // parent (global id), -1 on level 0
    int bits;      // bit d set: X lies in the upper half of its parent's cell in direction d
    int sx;        // slot of the spatial moment table of its level (leaves of levels >= 2), else -1
};

// a nearfield block (Eq. eval_sl_nf_block): the leaf target box against one box of N(Z); its
// entries are stored [source step][source triangle][target step][target triangle] from `off`
struct GNear {
    int tgt, src;
    int64_t off;
};

// an M2L source of a target box and the table of its interval pair (E1 and prefactors)
struct GPair {
    int src, e;
};

// shared arguments of the far-field kernels
struct GenDev {
    const GBox *box;
    int nbox;           // boxes of all levels
    int nt, Et, nrhs;   // triangles, steps, right-hand sides of the call
    int na, nk, mx;     // m_t + 1, multi-indices |kappa| <= m_x, m_x
    const int *kidx;    // [nk][3]
    const int *kinv;    // [(m_x+1)^3] -> multi-index or -1
    const int *lvG;     // [levels] grid cells per direction
    const int *lvst;    // [levels] level l was reached from level l-1 by a space-time refinement
    const double *Sx;   // [slots][nt][nk] spatial moments int_gamma_x T_{X,kappa} (Eq. s2m, l2t)
    const double *St;   // [levels][Et][na] int over step j of L_{I,a}, I the level's interval holding j
    const double *qt;   // [boxes][na][na] q^(t)_{ac,ap} of a box against its parent (Eq. temp_m2m)
    const double *q1;   // [levels][2][m1][m1] q^(x) of a level's boxes into their parents, per half
    double *mu, *lam;   // [nrhs][boxes][na][nk] moments and local contributions
};

struct GenQuad {            // nearfield quadrature of the general-step entries
    const double *verts;    // [nv][3]
    const int *tri;         // [nt][3] internal order
    const double *ts;       // [Et + 1] step times
    double alpha;
    const double *rule_reg; // collapsed rule s1[nq], s2[nq], w[nq]
    int nq_reg;
    const double *gl_sing;  // Gauss-Legendre on [0,1]: x[n], w[n]
    int nq_sing;
};

void launch_gen_nf_entries(const GenQuad &q, const GBox *box, const GNear *blocks, int nblocks, double *A,
                           cudaStream_t st);
void launch_gen_e1(int npairs, const double *dts, int na, int mx, int G, double hx, double hxp, double alpha,
                   double *E1, double *pref, cudaStream_t st);
void launch_gen_permute_in(const double *w, double *w_int, const int *perm, int nt, int rows, cudaStream_t st);
void launch_gen_permute_out(const double *f_int, double *f, const int *perm, int nt, int rows, cudaStream_t st);
void launch_gen_nf_apply(const GBox *box, const int *leaves, int nleaves, const int *nptr, const GNear *blocks,
                         const double *A, const double *w_int, double *f_int, int nt, int Et, int nrhs,
                         cudaStream_t st);
void launch_gen_s2m(const GenDev &g, const int *leaves, int n, const double *w_int, cudaStream_t st);
// M2M of the parents of one level: the children (all boxes of the next level) write their
// contributions into contrib ([nrhs][boxes][na][nk]), the parents add them in child order
void launch_gen_m2m(const GenDev &g, const int *parents, int n, const int *children, int nc, double *contrib,
                    cudaStream_t st);
// M2L of all target boxes in double-FP32: Edf, prefdf, mudf are double-FP32 copies (pairs of
// floats) of the E1 tables, the prefactors and the moments
void launch_gen_m2l(const GenDev &g, const int *targets, int n, const int *mptr, const GPair *pairs,
                    const void *Edf, const int64_t *e1off, const void *prefdf, const void *mudf, cudaStream_t st);
// y = x as double-FP32 pairs (8 bytes per value)
void launch_gen_to_df64(const double *x, void *y, int64_t n, cudaStream_t st);
// dynamic shared memory of the M2L kernel (the create call refuses parameters beyond 227 KB)
size_t gen_m2l_smem(int na, int nk, int mx);
void launch_gen_l2l(const GenDev &g, const int *children, int n, cudaStream_t st);
void launch_gen_l2t(const GenDev &g, const int *leaves, int n, double *f_int, cudaStream_t st);

}  // namespace pfmm
