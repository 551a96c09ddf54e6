// tree.cpp -- box cluster tree, lists and nearfield layout on the host.
//
// Section 3.2 (Alg. 1) for a tensor mesh with uniform steps, read as follows:
//  * root: the cube around the vertices' bounding box (centre = box midpoint, half-size = the
//    largest half extent); if it violates Eq. rel_h_t_h_x it is refined in space first (the
//    remark after Alg. 1);
//  * an element belongs to the box holding its centre ((v0 + v1) + v2) / 3, half-open (a, b]
//    per direction, clamped at the root's faces;
//  * temporal leaves hold leaf_steps steps, so every level l holds all 2^l intervals;
//  * the refinement l -> l+1 is temporal when hx_l^2 <= c_st 4 alpha ht_{l+1} (unpadded hx,
//    Eq. rel_h_t_h_x) or when no box of level l holds more than leaf_tris triangles, and
//    space-time otherwise; the split is uniform (all boxes of a level have the same size);
//  * padding: per level the largest overshoot of a triangle over its unpadded box, made
//    monotone (pad_l >= pad_{l+1}) as the paper requires.
// Section 3.3: interaction areas (Eq. 03:Iarea) with the radius n_tr, or, when n_tr < 0, the
// smallest radius beyond which exp(-s^2 / (4 alpha delta_max)) <= eps_tr for the separation s
// of the excluded boxes (delta_max = 4 interval lengths for M2L, 2 leaf intervals for the
// nearfield).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <map>
#include <set>

#include "pfmm_internal.h"

namespace pfmm {

static int cell_of(double z, double corner, double w, int G)
{
    double s = (z - corner) / w;
    int i = (int)std::ceil(s) - 1;
    if (i < 0) i = 0;
    if (i > G - 1) i = G - 1;
    return i;
}

static uint64_t morton3(int i, int j, int k)
{
    uint64_t c = 0;
    for (int b = 0; b < 20; ++b) {
        c |= (uint64_t)((i >> b) & 1) << (3 * b + 2);
        c |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
        c |= (uint64_t)((k >> b) & 1) << (3 * b + 0);
    }
    return c;
}

static int radius(const pfmm_params &prm, double alpha, double hx, double pad, double dmax, int G)
{
    if (prm.n_tr >= 0) return prm.n_tr;
    for (int n = 1; n < G; ++n) {
        double s = n * 2.0 * hx - 2.0 * pad;
        if (s < 0) s = 0;
        if (std::exp(-s * s / (4.0 * alpha * dmax)) <= prm.eps_tr) return n;
    }
    return G > 1 ? G - 1 : 0;
}

static int gdist(const int *a, const int *b)
{
    int d = 0;
    for (int c = 0; c < 3; ++c) d = std::max(d, std::abs(a[c] - b[c]));
    return d;
}

int build_tree(const pfmm_mesh &m, const pfmm_params &prm, Tree &t, std::string &err)
{
    const int nv = m.n_vertices, nt = m.n_triangles, Et = m.n_steps;
    if (nv < 3 || nt < 1 || Et < 1 || !(m.T > 0) || !(m.alpha > 0) || !m.vertices || !m.triangles) {
        err = "invalid mesh (sizes, T, alpha or NULL arrays)";
        return PFMM_ERR_INVALID_ARG;
    }
    if (prm.m_t < 0 || prm.m_t >= kMaxNa || prm.m_x < 0 || prm.m_x > kMaxMx || prm.leaf_steps < 1 ||
        !(prm.c_st > 0) || prm.quad_regular < 1 || prm.quad_regular > 16 || prm.quad_singular < 1 ||
        prm.quad_singular > 16) {
        err = "invalid parameters (m_t, m_x, leaf_steps, c_st or quadrature orders)";
        return PFMM_ERR_INVALID_ARG;
    }
    if (Et % prm.leaf_steps) {
        err = "n_steps must be a multiple of leaf_steps";
        return PFMM_ERR_INVALID_ARG;
    }
    int nleaf = Et / prm.leaf_steps, p = 0;
    while ((1 << p) < nleaf) p++;
    if ((1 << p) != nleaf || p >= kMaxLevels) {
        err = "n_steps / leaf_steps must be a power of two";
        return PFMM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(m.vertices[i])) {
            err = "non-finite vertex coordinate";
            return PFMM_ERR_NONFINITE;
        }
    for (int i = 0; i < 3 * nt; ++i)
        if (m.triangles[i] < 0 || m.triangles[i] >= nv) {
            err = "triangle vertex index out of range";
            return PFMM_ERR_INVALID_ARG;
        }
    t.p = p;
    const double *V = m.vertices;
    const int *T = m.triangles;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], V[3 * i + c]);
            hi[c] = std::max(hi[c], V[3 * i + c]);
        }
    t.H = 0;
    for (int c = 0; c < 3; ++c) t.H = std::max(t.H, 0.5 * (hi[c] - lo[c]));
    if (!(t.H > 0)) {
        err = "degenerate mesh extent";
        return PFMM_ERR_INVALID_ARG;
    }
    for (int c = 0; c < 3; ++c) t.corner[c] = 0.5 * (lo[c] + hi[c]) - t.H;
    std::vector<double> cen(3 * (size_t)nt);
    for (int x = 0; x < nt; ++x)
        for (int c = 0; c < 3; ++c)
            cen[3 * x + c] = ((V[3 * T[3 * x] + c] + V[3 * T[3 * x + 1] + c]) + V[3 * T[3 * x + 2] + c]) / 3.0;

    int lx0 = 0;
    while (true) {
        double hx = t.H / (double)(1 << lx0);
        if (hx * hx <= prm.c_st * 4.0 * m.alpha * (m.T / 2.0) || lx0 > 20) break;
        lx0++;
    }
    t.lv.assign(p + 1, Level());
    std::vector<std::vector<int>> tbox(p + 1, std::vector<int>(nt));
    std::vector<std::vector<int>> lookup(p + 1);
    for (int l = 0; l <= p; ++l) {
        Level &L = t.lv[l];
        if (l == 0) {
            L.lx = lx0;
        } else {
            const Level &P = t.lv[l - 1];
            double ht = m.T / (double)(1 << (l + 1));
            double hx = t.H / (double)(1 << P.lx);
            std::vector<int> cnt(P.nbox, 0);
            int maxcnt = 0;
            for (int x = 0; x < nt; ++x) maxcnt = std::max(maxcnt, ++cnt[tbox[l - 1][x]]);
            bool temporal = hx * hx <= prm.c_st * 4.0 * m.alpha * ht || maxcnt <= prm.leaf_tris;
            L.lx = temporal ? P.lx : P.lx + 1;
            if (L.lx > 20) {
                err = "spatial refinement too deep";
                return PFMM_ERR_UNSUPPORTED;
            }
        }
        L.G = 1 << L.lx;
        L.nint = 1 << l;
        L.hx = t.H / L.G;
        L.ht = m.T / (double)(1 << (l + 1));
        double w = 2.0 * t.H / L.G;
        std::vector<int> cell(3 * (size_t)nt);
        std::map<uint64_t, std::array<int, 3>> occ;
        for (int x = 0; x < nt; ++x) {
            for (int c = 0; c < 3; ++c) cell[3 * x + c] = cell_of(cen[3 * x + c], t.corner[c], w, L.G);
            occ[morton3(cell[3 * x], cell[3 * x + 1], cell[3 * x + 2])] = {cell[3 * x], cell[3 * x + 1], cell[3 * x + 2]};
        }
        L.nbox = (int)occ.size();
        L.grid.resize(3 * (size_t)L.nbox);
        lookup[l].assign((size_t)L.G * L.G * L.G, -1);
        int b = 0;
        for (auto &kv : occ) {
            for (int c = 0; c < 3; ++c) L.grid[3 * b + c] = kv.second[c];
            lookup[l][((size_t)kv.second[0] * L.G + kv.second[1]) * L.G + kv.second[2]] = b;
            b++;
        }
        double ov = 0.0;
        for (int x = 0; x < nt; ++x) {
            tbox[l][x] = lookup[l][((size_t)cell[3 * x] * L.G + cell[3 * x + 1]) * L.G + cell[3 * x + 2]];
            for (int v = 0; v < 3; ++v)
                for (int c = 0; c < 3; ++c) {
                    double z = V[3 * T[3 * x + v] + c];
                    double blo = t.corner[c] + cell[3 * x + c] * w, bhi = blo + w;
                    ov = std::max(ov, std::max(blo - z, z - bhi));
                }
        }
        L.pad = ov;
    }
    for (int l = p - 1; l >= 0; --l) t.lv[l].pad = std::max(t.lv[l].pad, t.lv[l + 1].pad);
    for (int l = 0; l <= p; ++l) {
        Level &L = t.lv[l];
        L.hxp = L.hx + L.pad;
        L.ntr = radius(prm, m.alpha, L.hx, L.pad, 8.0 * L.ht, L.G);
        if (l > 0) {
            const Level &P = t.lv[l - 1];
            L.st = L.lx != P.lx;
            L.parent.resize(L.nbox);
            L.octant.resize(L.nbox);
            for (int b = 0; b < L.nbox; ++b) {
                int g[3], o = 0;
                for (int c = 0; c < 3; ++c) {
                    g[c] = L.st ? L.grid[3 * b + c] >> 1 : L.grid[3 * b + c];
                    if (L.st && (L.grid[3 * b + c] & 1)) o |= 1 << c;
                }
                L.parent[b] = lookup[l - 1][((size_t)g[0] * P.G + g[1]) * P.G + g[2]];
                L.octant[b] = o;
            }
        }
    }
    for (int l = 0; l < p; ++l) {
        Level &L = t.lv[l];
        const Level &C = t.lv[l + 1];
        L.ch_ptr.assign(L.nbox + 1, 0);
        for (int b = 0; b < C.nbox; ++b) L.ch_ptr[C.parent[b] + 1]++;
        for (int b = 0; b < L.nbox; ++b) L.ch_ptr[b + 1] += L.ch_ptr[b];
        L.ch_idx.resize(C.nbox);
        std::vector<int> fill(L.ch_ptr.begin(), L.ch_ptr.end() - 1);
        for (int b = 0; b < C.nbox; ++b) L.ch_idx[fill[C.parent[b]]++] = b;
    }
    t.n_m2l_pairs = 0;
    for (int l = 2; l <= p; ++l) {
        Level &L = t.lv[l];
        L.m2l_ptr.assign(L.nbox + 1, 0);
        for (int bt = 0; bt < L.nbox; ++bt) {
            for (int bs = 0; bs < L.nbox; ++bs) {
                const int *gt = &L.grid[3 * bt], *gs = &L.grid[3 * bs];
                if (gdist(gt, gs) > L.ntr) continue;
                L.m2l_src.push_back(bs);
                L.m2l_off.push_back((gt[0] - gs[0] + L.G - 1) | ((gt[1] - gs[1] + L.G - 1) << 8) |
                                    ((gt[2] - gs[2] + L.G - 1) << 16));
            }
            L.m2l_ptr[bt + 1] = (int)L.m2l_src.size();
        }
        int nsrc_int = 0;
        for (int k = 0; k < L.nint; ++k) nsrc_int += k < 2 ? 0 : (k % 2 ? 2 : 1);
        t.n_m2l_pairs += nsrc_int * (int)L.m2l_src.size();
    }
    {
        const Level &Lp = t.lv[p];
        double hstep = m.T / Et;
        t.ntr_near = radius(prm, m.alpha, Lp.hx, Lp.pad, 2.0 * prm.leaf_steps * hstep, Lp.G);
    }

    // internal triangle order: by leaf box (Morton order of the boxes), then caller order
    const Level &Lp = t.lv[p];
    t.perm.resize(nt);
    for (int x = 0; x < nt; ++x) t.perm[x] = x;
    std::stable_sort(t.perm.begin(), t.perm.end(), [&](int a, int b) { return tbox[p][a] < tbox[p][b]; });
    std::vector<int> iperm(nt);
    for (int i = 0; i < nt; ++i) iperm[t.perm[i]] = i;
    t.leaf_start.assign(Lp.nbox + 1, 0);
    t.tri_leaf.resize(nt);
    for (int i = 0; i < nt; ++i) {
        t.tri_leaf[i] = tbox[p][t.perm[i]];
        t.leaf_start[t.tri_leaf[i] + 1]++;
    }
    for (int b = 0; b < Lp.nbox; ++b) t.leaf_start[b + 1] += t.leaf_start[b];

    // nearfield panels (one per target leaf box)
    const int npan = Lp.nbox;
    t.panels.resize(npan);
    t.kmap.assign((size_t)npan * nv, -1);
    t.colV.clear();
    t.colK.clear();
    const int ND = 2 * prm.leaf_steps;  // step offsets inside the temporal nearfield
    int64_t offV = 0, offK = 0;
    std::vector<std::vector<int>> srcboxes(npan);
    int64_t covered = 0;
    for (int X = 0; X < npan; ++X) {
        for (int Y = 0; Y < npan; ++Y)
            if (gdist(&Lp.grid[3 * X], &Lp.grid[3 * Y]) <= t.ntr_near) {
                srcboxes[X].push_back(Y);
                covered += t.leaf_start[Y + 1] - t.leaf_start[Y];
            }
    }
    // Dense-column layout when the interaction areas cover most of the mesh: every panel
    // indexes all triangles (column = internal index, -1 where the source is not near) and all
    // nodes, so the panels share one column space (tensor-core engine) at a small cost in zeros.
    t.dense_cols = covered >= (int64_t)(0.75 * (double)npan * (double)nt);
    for (int X = 0; X < npan; ++X) {
        Panel &P = t.panels[X];
        P.row0 = t.leaf_start[X];
        P.nrows = t.leaf_start[X + 1] - t.leaf_start[X];
        P.rows_pad = (P.nrows + kRowTile - 1) / kRowTile * kRowTile;
        if (t.dense_cols) {
            std::vector<char> near(npan, 0);
            for (int Y : srcboxes[X]) near[Y] = 1;
            P.colV_at = (int)t.colV.size();
            for (int i = 0; i < nt; ++i) t.colV.push_back(near[t.tri_leaf[i]] ? i : -1);
            P.ncolV = nt;
            P.colsV_pad = (nt + kTcColTile - 1) / kTcColTile * kTcColTile;
            while ((int)t.colV.size() < P.colV_at + P.colsV_pad) t.colV.push_back(-1);
            P.colK_at = (int)t.colK.size();
            for (int nd = 0; nd < nv; ++nd) {
                t.kmap[(size_t)X * nv + nd] = nd;
                t.colK.push_back(nd);
            }
            P.ncolK = nv;
            P.colsK_pad = (nv + kTcColTile - 1) / kTcColTile * kTcColTile;
            while ((int)t.colK.size() < P.colK_at + P.colsK_pad) t.colK.push_back(-1);
            P.offV = offV;
            P.offK = offK;
            offV += (int64_t)ND * P.rows_pad * P.colsV_pad;
            offK += (int64_t)ND * P.rows_pad * P.colsK_pad;
            continue;
        }
        P.colV_at = (int)t.colV.size();
        std::set<int> nodes;
        for (int Y : srcboxes[X])
            for (int i = t.leaf_start[Y]; i < t.leaf_start[Y + 1]; ++i) {
                t.colV.push_back(i);
                for (int v = 0; v < 3; ++v) nodes.insert(T[3 * t.perm[i] + v]);
            }
        P.ncolV = (int)t.colV.size() - P.colV_at;
        const int tv = P.ncolV == nt ? kTcColTile : kColTile;
        P.colsV_pad = (P.ncolV + tv - 1) / tv * tv;
        while ((int)t.colV.size() < P.colV_at + P.colsV_pad) t.colV.push_back(-1);
        P.colK_at = (int)t.colK.size();
        for (int nd : nodes) {
            t.kmap[(size_t)X * nv + nd] = (int)t.colK.size() - P.colK_at;
            t.colK.push_back(nd);
        }
        P.ncolK = (int)nodes.size();
        const int tk = P.ncolK == nv ? kTcColTile : kColTile;
        P.colsK_pad = (P.ncolK + tk - 1) / tk * tk;
        while ((int)t.colK.size() < P.colK_at + P.colsK_pad) t.colK.push_back(-1);
        P.offV = offV;
        P.offK = offK;
        offV += (int64_t)ND * P.rows_pad * P.colsV_pad;
        offK += (int64_t)ND * P.rows_pad * P.colsK_pad;
    }
    t.sizeV = offV;
    t.sizeK = offK;

    // singular pairs: triangles sharing at least one vertex (Sauter-Schwab classes)
    std::vector<std::vector<int>> star(nv);
    for (int i = 0; i < nt; ++i)
        for (int v = 0; v < 3; ++v) star[T[3 * t.perm[i] + v]].push_back(i);
    t.sing.clear();
    for (int x = 0; x < nt; ++x) {
        std::set<int> cand;
        const int *tx = &T[3 * t.perm[x]];
        for (int v = 0; v < 3; ++v)
            for (int y : star[tx[v]]) cand.insert(y);
        int X = t.tri_leaf[x];
        const Panel &P = t.panels[X];
        for (int y : cand) {
            int Y = t.tri_leaf[y];
            if (gdist(&Lp.grid[3 * X], &Lp.grid[3 * Y]) > t.ntr_near) continue;
            const int *ty = &T[3 * t.perm[y]];
            const int code = ss_code(tx, ty);
            if (!code) continue;
            SingularPair s;
            s.x = x;
            s.y = y;
            s.panel = X;
            s.row = x - P.row0;
            int colv = -1, acc = 0;
            if (t.dense_cols) {
                colv = y;
            } else {
                for (int Yb : srcboxes[X]) {
                    if (Yb == Y) { colv = acc + (y - t.leaf_start[Y]); break; }
                    acc += t.leaf_start[Yb + 1] - t.leaf_start[Yb];
                }
            }
            s.colV = colv;
            for (int v = 0; v < 3; ++v) s.colK[v] = t.kmap[(size_t)X * nv + ty[v]];
            s.code = code;
            t.sing.push_back(s);
        }
    }
    return PFMM_OK;
}

}  // namespace pfmm
