// pfmm_internal.h -- host-side structures of the GB300 pFMM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pfmm.h"

namespace pfmm {

constexpr int kMaxLevels = 30;
constexpr int kMaxMx = 12;
constexpr int kMaxNa = 12;
constexpr int kRowTile = 64;  // nearfield panel rows are padded to this
constexpr int kColTile = 32;  // nearfield panel columns are padded to this
// columns of panels that index the whole mesh (the tensor-core engine's one column space) are
// padded to 64: one 128-byte swizzle row of FP16 per K block
constexpr int kTcColTile = 64;

// ---------------------------------------------------------------------------------------------
// Host description of one level of the box cluster tree (Section 3.2, Alg. 1).  Every level
// holds all 2^l temporal intervals (uniform steps, uniform-depth temporal tree) times the
// non-empty cells of a uniform 2^lx grid (the spatial parts are uniform per level).
struct Level {
    int lx = 0, G = 1;         // spatial refinements, grid cells per direction
    double hx = 0, pad = 0;    // unpadded spatial half-size, uniform padding
    double hxp = 0;            // padded half-size hx + pad
    double ht = 0;             // temporal half-size of the intervals
    int nint = 1;              // 2^l intervals
    int nbox = 0;              // non-empty spatial boxes
    std::vector<int> grid;     // [nbox][3] cell multi-indices (Morton order)
    std::vector<int> parent;   // [nbox] parent box at level l-1
    std::vector<int> octant;   // [nbox] position in the parent (bit c set: upper half in dir c)
    bool st = false;           // reached from level l-1 by a space-time refinement
    int ntr = 0;               // interaction-area radius for M2L at this level
    std::vector<int> m2l_ptr;  // CSR over target boxes: source boxes in the interaction area
    std::vector<int> m2l_src;
    std::vector<int> m2l_off;  // packed (ox + G-1) | (oy + G-1) << 8 | (oz + G-1) << 16
    std::vector<int> ch_ptr;   // CSR over boxes: children at level l+1
    std::vector<int> ch_idx;
};

// One nearfield row panel: the rows of a target leaf box X against the columns of all leaf
// boxes in its interaction area (Eq. def_st_nearfield at the leaves).
struct Panel {
    int row0 = 0, nrows = 0, rows_pad = 0;  // internal triangle range of X
    int ncolV = 0, colsV_pad = 0;           // source triangles (V columns)
    int ncolK = 0, colsK_pad = 0;           // source nodes (K columns)
    int64_t offV = 0, offK = 0;             // element offsets of the panel data (per d: rows_pad*cols_pad)
    int colV_at = 0, colK_at = 0;           // offsets into the column index arrays
};

struct SingularPair {  // identical / edge / vertex-adjacent pair handled by Sauter-Schwab
    int x, y;          // internal triangles
    int panel, row;    // panel of x and row within it
    int colV;          // column of y in the panel's V columns
    int colK[3];       // columns of y's nodes in the panel's K columns
    int code;          // class (1..3) | ox0 << 2 | ox1 << 4 | ox2 << 6 | oy0 << 8 | oy1 << 10 | oy2 << 12
};

struct Tree {
    int p = 0;
    double H = 0, corner[3] = {0, 0, 0};
    std::vector<Level> lv;
    std::vector<int> perm;        // internal slot -> caller triangle
    std::vector<int> leaf_start;  // [nbox_p + 1]
    std::vector<int> tri_leaf;    // internal triangle -> leaf box
    int ntr_near = 0;
    std::vector<Panel> panels;
    std::vector<int> colV;        // concatenated V column lists (internal triangles, -1 pad)
    std::vector<int> colK;        // concatenated K column lists (nodes, -1 pad)
    std::vector<int> kmap;        // [npanel][N_v] node -> K column of the panel or -1
    std::vector<SingularPair> sing;
    bool dense_cols = false;      // panels index all triangles / nodes (holes: -1 in colV)
    int64_t sizeV = 0, sizeK = 0; // panel elements per operator (all d)
    int n_m2l_pairs = 0;
};

int build_tree(const pfmm_mesh &m, const pfmm_params &prm, Tree &t, std::string &err);

// Sauter-Schwab class and vertex order of a triangle pair (vertex ids tx, ty): 0 when the
// triangles share no vertex, else shared | ox[0..2] << 2, 4, 6 | oy[0..2] << 8, 10, 12 (the
// rule's local vertex order: shared vertices first, in matching order)
__host__ __device__ inline int ss_code(const int *tx, const int *ty)
{
    int shared = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) shared += tx[i] == ty[j];
    int ox[3] = {0, 1, 2}, oy[3] = {0, 1, 2};
    if (shared == 3) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (ty[j] == tx[i]) oy[i] = j;
    } else if (shared == 2) {
        int n = 0;
        for (int i = 0; i < 3 && n < 2; ++i)
            for (int j = 0; j < 3; ++j)
                if (tx[i] == ty[j]) { ox[n] = i; oy[n] = j; n++; }
        ox[2] = 3 - ox[0] - ox[1];
        oy[2] = 3 - oy[0] - oy[1];
    } else if (shared == 1) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (tx[i] == ty[j]) { ox[0] = i; oy[0] = j; }
        ox[1] = (ox[0] + 1) % 3; ox[2] = (ox[0] + 2) % 3;
        oy[1] = (oy[0] + 1) % 3; oy[2] = (oy[0] + 2) % 3;
    } else {
        return 0;
    }
    return shared | (ox[0] << 2) | (ox[1] << 4) | (ox[2] << 6) | (oy[0] << 8) | (oy[1] << 10) | (oy[2] << 12);
}

// ---------------------------------------------------------------------------------------------
// Device-side descriptors.
struct DevLevel {
    int G, nint, nbox, st;
    double hxp;
    int *grid;       // [nbox*3]
    int *parent;     // [nbox]
    int *octant;     // [nbox]
    int *m2l_ptr, *m2l_src, *m2l_off;
    int *ch_ptr, *ch_idx;
    void *E1;        // [2][na][na][2G-1][m1][m1]  (R)
    void *pref;      // [2][na][na]                (R)
    void *qx;        // [2 bits][m1][m1] q^(x) from this level's boxes into their parents (R)
    int64_t mom_off; // element offset of this level's moments in the moment buffer (per rhs)
    int ntr;         // interaction-area radius (Eq. 03:Iarea)
    int *cellbox;    // [G^3] -> box or -1
    int *boxcell;    // [nbox] -> cell
    int *pk, *pJ;    // M2L interval pairs (target k, source J in I(k)) for k = 2 .. nint-1
    int *kptr;       // [nint+1] pairs of target k: [kptr[k], kptr[k+1])
    std::vector<int> kptr_host;
};

}  // namespace pfmm
