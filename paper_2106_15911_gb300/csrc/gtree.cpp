// gtree.cpp -- the space-time FMM for general (non-uniform) time steps t_0 = 0 < t_1 < ... < t_Et = T:
// the box cluster tree of Alg. 1 in full, the nearfield and interaction lists of Section 3.3, the
// expansion tables, the stored nearfield and the C ABI (pfmm_gen_*).  Single layer V_h, FP64.
//
// Readings of Section 3.2 (the same as for the oracle of this method):
//  * level 0 holds the non-empty cells of the grid 2^lx0 (the root refined in space until it
//    satisfies Eq. rel_h_t_h_x) with the interval (0, T];
//  * the refinement of level l into level l+1 is temporal iff hx_l^2 <= c_st 4 alpha T / 2^(l+2)
//    (the nominal half-size h_t^(l+1) of Alg. 1), for every box of the level alike;
//  * RefineCluster: a box Z = X x I is refined iff it holds at least n_max elements, unless an
//    element is oversized: I holds a single step, a step of I is longer than the nominal interval
//    length T / 2^l, or a triangle of X extends over more than the cell width 2 hx_l;
//  * the temporal split of (t_a, t_b] is at the step t_s (a < s < b) nearest (t_a + t_b) / 2, the
//    smaller s on a tie; children without elements are not created;
//  * padding per level: the largest overshoot of a triangle over its unpadded cell, monotone in
//    the level; interaction-area radii from the longest interval L_l of the level (separation
//    4 L_l for M2L, 2 L_l for the nearfield) unless n_tr >= 0 is given.
// Lists (Eq. def_st_nearfield, def_st_interaction_list): the nearfield of a leaf is its
// same-level nearfield {Y x J: J in {I_{k-1}, I_k}, Y in I_A(X)} plus the leaves in the same-level
// nearfields of all its ancestors (N(parent(Z)) /\ L_Sigma, recursively); the interaction list of
// a box of level >= 2 is {Y x J: J in I(I) (Eq. 03:ILtemp), Y in I_A(X)}; boxes that do not exist
// are skipped.
// Internal triangle order: Morton order of the cells of the finest level, so the triangles of
// any cell of any level form one contiguous range.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "gtree.h"
#include "host_math.h"
#include "kernels.h"
#include "pfmm_internal.h"

using namespace pfmm;

namespace pfmm {
int set_error(int code, const std::string &msg);  // records the message for pfmm_last_error (capi.cpp)
}

namespace {

struct GenLevel {
    int lx = 0, G = 1, st_next = 0;  // st_next: level l -> l+1 is a space-time refinement
    double hx = 0, pad = 0, hxp = 0;
    int ntr_far = 0, ntr_near = 0;
    std::vector<int> cell, kk, leaf, par;  // per box (cell: 3 ints)
    std::vector<int> c0, nch;               // first child (index on level l+1) and child count
    std::vector<int> ia, ib;                // per interval k < 2^l: steps [ia, ib) or -1
    std::unordered_map<int64_t, int> lookup;
    int64_t key(int k, const int *c) const { return (((int64_t)k * G + c[0]) * G + c[1]) * G + c[2]; }
    int find(int k, const int *c) const
    {
        for (int d = 0; d < 3; ++d)
            if (c[d] < 0 || c[d] >= G) return -1;
        auto it = lookup.find(key(k, c));
        return it == lookup.end() ? -1 : it->second;
    }
};

int cell_of(double z, double corner, double w, int G)
{
    int i = (int)std::ceil((z - corner) / w) - 1;
    return i < 0 ? 0 : (i > G - 1 ? G - 1 : i);
}

int radius(int n_tr, double eps_tr, double alpha, double hx, double pad, double dmax, int G)
{
    if (n_tr >= 0) return n_tr;
    for (int n = 1; n < G; ++n) {
        double s = n * 2.0 * hx - 2.0 * pad;
        if (s < 0) s = 0;
        if (std::exp(-s * s / (4.0 * alpha * dmax)) <= eps_tr) return n;
    }
    return G > 1 ? G - 1 : 0;
}

uint64_t morton(const int *c)
{
    uint64_t m = 0;
    for (int b = 0; b < 21; ++b)
        for (int d = 0; d < 3; ++d) m |= (uint64_t)((c[d] >> b) & 1) << (3 * b + 2 - d);
    return m;
}

int fail(int code, const std::string &msg) { return pfmm::set_error(code, msg); }

}  // namespace

struct pfmm_gen {
    int nv = 0, nt = 0, Et = 0;
    double alpha = 0;
    pfmm_params prm{};
    int n_max = 0, nlev = 0, na = 0, nk = 0, mx = 0;
    std::vector<GenLevel> lv;
    std::vector<int> lvoff;  // first global box id of each level
    int nbox = 0;
    std::vector<GBox> boxes;
    std::vector<int> leaves_all, leaves_far, m2l_targets;
    std::vector<std::vector<int>> parents_lv, all_lv;  // non-leaf boxes / all boxes of each level (global ids)
    int64_t n_m2l_pairs = 0, n_blocks = 0, nf_entries = 0;
    // device
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;
    GBox *d_box = nullptr;
    int *d_perm = nullptr, *d_tri = nullptr, *d_kidx = nullptr, *d_kinv = nullptr, *d_lvG = nullptr, *d_lvst = nullptr;
    double *d_Sx = nullptr, *d_St = nullptr, *d_qt = nullptr, *d_q1 = nullptr;
    int *d_leaves_all = nullptr, *d_leaves_far = nullptr, *d_m2l_targets = nullptr, *d_mptr = nullptr;
    GPair *d_pairs = nullptr;
    double *d_E1 = nullptr, *d_pref = nullptr;
    void *d_E1df = nullptr, *d_prefdf = nullptr;  // double-FP32 copies for the M2L kernel
    int64_t *d_e1off = nullptr;
    int *d_nptr = nullptr;
    GNear *d_blocks = nullptr;
    double *d_A = nullptr;
    std::vector<int *> d_parents_lv, d_all_lv;
    int ws_nrhs = 0;
    double *d_wint = nullptr, *d_fint = nullptr, *d_mu = nullptr, *d_lam = nullptr, *d_contrib = nullptr;

    ~pfmm_gen()
    {
        for (void *p : allocs) cudaFree(p);
    }
    template <typename T_>
    int alloc(T_ **p, size_t n)
    {
        void *q = nullptr;
        const size_t bytes = std::max<size_t>(n * sizeof(T_), 16);
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? PFMM_ERR_OOM : PFMM_ERR_CUDA,
                        "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
        }
        allocs.push_back(q);
        dev_bytes += (int64_t)bytes;
        *p = (T_ *)q;
        return PFMM_OK;
    }
    template <typename T_>
    int upload(T_ **p, const std::vector<T_> &v, cudaStream_t st)
    {
        int rc = alloc(p, v.size());
        if (rc) return rc;
        if (!v.empty() && cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T_), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(PFMM_ERR_CUDA, "host to device copy failed");
        return PFMM_OK;
    }
};

namespace {

// ---- Alg. 1 -----------------------------------------------------------------------------------
int build_levels(pfmm_gen *h, const pfmm_mesh &m, const double *ts, std::vector<int> &perm, double corner[3],
                 double &H)
{
    const int nt = m.n_triangles, E = m.n_steps;
    const double *V = m.vertices;
    const int *Tr = m.triangles;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < m.n_vertices; ++i)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], V[3 * i + c]);
            hi[c] = std::max(hi[c], V[3 * i + c]);
        }
    H = 0;
    for (int c = 0; c < 3; ++c) H = std::max(H, 0.5 * (hi[c] - lo[c]));
    if (!(H > 0)) return fail(PFMM_ERR_INVALID_ARG, "degenerate mesh extent");
    for (int c = 0; c < 3; ++c) corner[c] = 0.5 * (lo[c] + hi[c]) - H;
    std::vector<double> cen(3 * (size_t)nt), ext(nt);
    for (int x = 0; x < nt; ++x) {
        ext[x] = 0;
        for (int c = 0; c < 3; ++c) {
            const double a = V[3 * Tr[3 * x] + c], b = V[3 * Tr[3 * x + 1] + c], d = V[3 * Tr[3 * x + 2] + c];
            cen[3 * x + c] = ((a + b) + d) / 3.0;
            ext[x] = std::max(ext[x], std::max(a, std::max(b, d)) - std::min(a, std::min(b, d)));
        }
    }
    const double T = ts[E], alpha = m.alpha, c_st = h->prm.c_st;
    int lx0 = 0;
    while (true) {
        const double hx = H / (double)(1 << lx0);
        if (hx * hx <= c_st * 4.0 * alpha * (T / 2.0) || lx0 > 20) break;
        lx0++;
    }
    auto cells_of = [&](int lx, std::vector<int> &c3) {
        const int G = 1 << lx;
        const double w = 2.0 * H / G;
        c3.resize(3 * (size_t)nt);
        for (int x = 0; x < nt; ++x)
            for (int d = 0; d < 3; ++d) c3[3 * x + d] = cell_of(cen[3 * x + d], corner[d], w, G);
    };
    auto lin = [](const int *c, int G) { return ((int64_t)c[0] * G + c[1]) * G + c[2]; };
    std::vector<GenLevel> &lv = h->lv;
    lv.assign(1, GenLevel());
    lv[0].lx = lx0;
    lv[0].G = 1 << lx0;
    lv[0].ia = {0};
    lv[0].ib = {E};
    std::vector<int> c3;
    cells_of(lx0, c3);
    {
        std::vector<int64_t> ls;
        for (int x = 0; x < nt; ++x) ls.push_back(lin(&c3[3 * x], lv[0].G));
        std::sort(ls.begin(), ls.end());
        ls.erase(std::unique(ls.begin(), ls.end()), ls.end());
        const int G = lv[0].G;
        for (int64_t q : ls) {
            lv[0].cell.insert(lv[0].cell.end(), {(int)(q / ((int64_t)G * G)), (int)((q / G) % G), (int)(q % G)});
            lv[0].kk.push_back(0);
            lv[0].par.push_back(-1);
        }
    }
    for (int l = 0;; ++l) {
        GenLevel &L = lv[l];
        L.G = 1 << L.lx;
        L.hx = H / L.G;
        cells_of(L.lx, c3);
        std::unordered_map<int64_t, std::pair<int, double>> cinfo;  // cell -> (triangles, largest extent)
        for (int x = 0; x < nt; ++x) {
            auto &ci = cinfo[lin(&c3[3 * x], L.G)];
            ci.first++;
            ci.second = std::max(ci.second, ext[x]);
        }
        const int nb = (int)L.kk.size();
        L.leaf.assign(nb, 1);
        L.c0.assign(nb, 0);
        L.nch.assign(nb, 0);
        int nref = 0;
        for (int b = 0; b < nb; ++b) {
            const int k = L.kk[b], a = L.ia[k], e = L.ib[k];
            const auto &ci = cinfo[lin(&L.cell[3 * b], L.G)];
            double maxstep = 0;
            for (int j = a; j < e; ++j) maxstep = std::max(maxstep, ts[j + 1] - ts[j]);
            const bool refine = (int64_t)ci.first * (e - a) >= h->n_max && e - a >= 2 &&
                                maxstep <= T / (double)(1 << l) && ci.second <= 2.0 * L.hx;
            L.leaf[b] = !refine;
            nref += refine;
        }
        if (nref == 0) break;
        if (l + 1 >= 30) return fail(PFMM_ERR_UNSUPPORTED, "general tree deeper than 30 levels");
        L.st_next = !(L.hx * L.hx <= c_st * 4.0 * alpha * (T / (double)(1 << (l + 2))));
        lv.push_back(GenLevel());  // invalidates L
        GenLevel &L0 = lv[l], &N = lv[l + 1];
        N.lx = L0.lx + L0.st_next;
        N.G = 1 << N.lx;
        std::vector<int> c3n;
        cells_of(N.lx, c3n);
        std::unordered_map<int64_t, int> ncount;
        for (int x = 0; x < nt; ++x) ncount[lin(&c3n[3 * x], N.G)]++;
        N.ia.assign((size_t)1 << (l + 1), -1);
        N.ib.assign((size_t)1 << (l + 1), -1);
        for (int b = 0; b < nb; ++b) {
            if (L0.leaf[b]) continue;
            const int k = L0.kk[b], a = L0.ia[k], e = L0.ib[k];
            const double mid = 0.5 * (ts[a] + ts[e]);
            int s = a + 1;
            for (int q = a + 2; q < e; ++q)
                if (std::fabs(ts[q] - mid) < std::fabs(ts[s] - mid)) s = q;
            N.ia[2 * k] = a;
            N.ib[2 * k] = s;
            N.ia[2 * k + 1] = s;
            N.ib[2 * k + 1] = e;
            L0.c0[b] = (int)N.kk.size();
            for (int ci = 0; ci < 2; ++ci)
                for (int o = 0; o < (L0.st_next ? 8 : 1); ++o) {
                    int cc[3];
                    for (int d = 0; d < 3; ++d) cc[d] = L0.st_next ? 2 * L0.cell[3 * b + d] + ((o >> (2 - d)) & 1) : L0.cell[3 * b + d];
                    if (!ncount.count(lin(cc, N.G))) continue;
                    N.cell.insert(N.cell.end(), cc, cc + 3);
                    N.kk.push_back(2 * k + ci);
                    N.par.push_back(b);
                }
            L0.nch[b] = (int)N.kk.size() - L0.c0[b];
        }
    }
    h->nlev = (int)lv.size();
    // padding, radii, lookups
    for (int l = 0; l < h->nlev; ++l) {
        GenLevel &L = lv[l];
        cells_of(L.lx, c3);
        const double w = 2.0 * H / L.G;
        double ov = 0;
        for (int x = 0; x < nt; ++x)
            for (int v = 0; v < 3; ++v)
                for (int d = 0; d < 3; ++d) {
                    const double z = V[3 * Tr[3 * x + v] + d], blo = corner[d] + c3[3 * x + d] * w;
                    ov = std::max(ov, std::max(blo - z, z - (blo + w)));
                }
        L.pad = ov;
    }
    for (int l = h->nlev - 2; l >= 0; --l) lv[l].pad = std::max(lv[l].pad, lv[l + 1].pad);
    for (int l = 0; l < h->nlev; ++l) {
        GenLevel &L = lv[l];
        L.hxp = L.hx + L.pad;
        double Lmax = 0;
        for (size_t k = 0; k < L.ia.size(); ++k)
            if (L.ia[k] >= 0) Lmax = std::max(Lmax, ts[L.ib[k]] - ts[L.ia[k]]);
        L.ntr_far = radius(h->prm.n_tr, h->prm.eps_tr, alpha, L.hx, L.pad, 4.0 * Lmax, L.G);
        L.ntr_near = radius(h->prm.n_tr, h->prm.eps_tr, alpha, L.hx, L.pad, 2.0 * Lmax, L.G);
        for (size_t b = 0; b < L.kk.size(); ++b) L.lookup[L.key(L.kk[b], &L.cell[3 * b])] = (int)b;
    }
    // internal order: Morton order of the finest cells
    cells_of(lv.back().lx, c3);
    perm.resize(nt);
    std::vector<std::pair<uint64_t, int>> key(nt);
    for (int x = 0; x < nt; ++x) key[x] = {morton(&c3[3 * x]), x};
    std::sort(key.begin(), key.end());
    for (int i = 0; i < nt; ++i) perm[i] = key[i].second;
    return PFMM_OK;
}

// the same-level nearfield of box b of level l (first set of Eq. def_st_nearfield)
void near_same(const GenLevel &L, int b, std::vector<int> &out)
{
    out.clear();
    const int *c = &L.cell[3 * b], k = L.kk[b], r = L.ntr_near;
    for (int j = k - 1; j <= k; ++j) {
        if (j < 0) continue;
        for (int a0 = std::max(0, c[0] - r); a0 <= std::min(L.G - 1, c[0] + r); ++a0)
            for (int a1 = std::max(0, c[1] - r); a1 <= std::min(L.G - 1, c[1] + r); ++a1)
                for (int a2 = std::max(0, c[2] - r); a2 <= std::min(L.G - 1, c[2] + r); ++a2) {
                    const int cc[3] = {a0, a1, a2};
                    const int s = L.find(j, cc);
                    if (s >= 0) out.push_back(s);
                }
    }
}

int build_impl(pfmm_gen *h, const pfmm_mesh &m, const double *ts_host, cudaStream_t st)
{
    int rc;
    const int nt = m.n_triangles, E = m.n_steps;
    std::vector<int> perm;
    double corner[3], H;
    if ((rc = build_levels(h, m, ts_host, perm, corner, H))) return rc;
    std::vector<GenLevel> &lv = h->lv;
    const int L = h->nlev;
    // ---- boxes with global ids
    h->lvoff.assign(L + 1, 0);
    for (int l = 0; l < L; ++l) h->lvoff[l + 1] = h->lvoff[l] + (int)lv[l].kk.size();
    h->nbox = h->lvoff[L];
    std::vector<int> slot_of(L, -1);
    int nslot = 0;
    for (int l = 2; l < L; ++l)
        if (std::count(lv[l].leaf.begin(), lv[l].leaf.end(), 1) > 0) slot_of[l] = nslot++;
    auto centroid = [&](int x, int d) {
        const int *tv = m.triangles + 3 * x;
        return ((m.vertices[3 * tv[0] + d] + m.vertices[3 * tv[1] + d]) + m.vertices[3 * tv[2] + d]) / 3.0;
    };
    // triangle ranges of the cells of each level in the internal order
    h->boxes.resize(h->nbox);
    h->parents_lv.assign(L, {});
    h->all_lv.assign(L, {});
    for (int l = 0; l < L; ++l) {
        const GenLevel &Lv = lv[l];
        const double w = 2.0 * H / Lv.G;
        std::unordered_map<int64_t, std::pair<int, int>> range;  // cell -> [first, last]
        for (int i = 0; i < nt; ++i) {
            int c[3];
            for (int d = 0; d < 3; ++d) c[d] = cell_of(centroid(perm[i], d), corner[d], w, Lv.G);
            const int64_t q = ((int64_t)c[0] * Lv.G + c[1]) * Lv.G + c[2];
            auto it = range.find(q);
            if (it == range.end()) {
                range[q] = {i, i};
            } else {
                if (it->second.second != i - 1) return fail(PFMM_ERR_CUDA, "internal error: cell triangles not contiguous");
                it->second.second = i;
            }
        }
        for (size_t b = 0; b < Lv.kk.size(); ++b) {
            GBox &B = h->boxes[h->lvoff[l] + b];
            const int *c = &Lv.cell[3 * b];
            const auto &rg = range.at(((int64_t)c[0] * Lv.G + c[1]) * Lv.G + c[2]);
            B.t0 = rg.first;
            B.t1 = rg.second + 1;
            B.a0 = Lv.ia[Lv.kk[b]];
            B.a1 = Lv.ib[Lv.kk[b]];
            B.level = l;
            B.k = Lv.kk[b];
            for (int d = 0; d < 3; ++d) B.cell[d] = c[d];
            B.c0 = Lv.leaf[b] ? 0 : h->lvoff[l + 1] + Lv.c0[b];
            B.c1 = Lv.leaf[b] ? 0 : B.c0 + Lv.nch[b];
            B.par = l ? h->lvoff[l - 1] + Lv.par[b] : -1;
            B.bits = 0;
            if (l && lv[l - 1].st_next) {
                const int *pc = &lv[l - 1].cell[3 * Lv.par[b]];
                for (int d = 0; d < 3; ++d) B.bits |= (c[d] - 2 * pc[d]) << d;
            }
            B.sx = slot_of[l];
            const int g = h->lvoff[l] + (int)b;
            h->all_lv[l].push_back(g);
            if (!Lv.leaf[b]) h->parents_lv[l].push_back(g);
            if (Lv.leaf[b]) {
                h->leaves_all.push_back(g);
                if (l >= 2) h->leaves_far.push_back(g);
            }
        }
    }
    // ---- interaction lists (M2L) and their interval pairs
    const int na = h->na = h->prm.m_t + 1, mx = h->mx = h->prm.m_x, m1 = mx + 1;
    std::vector<int> mptr(h->nbox + 1, 0);
    std::vector<GPair> pairs;
    std::vector<double> dts;   // [pairs][na][na]: xi_{I,b} - xi_{J,a}
    std::vector<int> e_level;  // level of each interval pair
    std::map<std::tuple<int, int, int>, int> epair;
    auto node = [&](int l, int k, int a) {
        const double lo_ = ts_host[lv[l].ia[k]], hi_ = ts_host[lv[l].ib[k]];
        return 0.5 * (lo_ + hi_) + 0.5 * (hi_ - lo_) * hostm::cheb_node(a, h->prm.m_t);
    };
    for (int l = 0; l < L; ++l) {
        const GenLevel &Lv = lv[l];
        for (size_t b = 0; b < Lv.kk.size(); ++b) {
            const int g = h->lvoff[l] + (int)b;
            mptr[g + 1] = mptr[g];
            if (l < 2) continue;
            const int k = Lv.kk[b], *c = &Lv.cell[3 * b], r = Lv.ntr_far;
            int js[2], nj = 0;
            if (k >= 2) {
                if (k % 2 == 0) {
                    js[nj++] = k - 2;
                } else {
                    js[nj++] = k - 3;
                    js[nj++] = k - 2;
                }
            }
            for (int q = 0; q < nj; ++q) {
                const int j = js[q];
                if (j < 0 || Lv.ia[j] < 0) continue;
                int eid = -1;
                for (int a0 = std::max(0, c[0] - r); a0 <= std::min(Lv.G - 1, c[0] + r); ++a0)
                    for (int a1 = std::max(0, c[1] - r); a1 <= std::min(Lv.G - 1, c[1] + r); ++a1)
                        for (int a2 = std::max(0, c[2] - r); a2 <= std::min(Lv.G - 1, c[2] + r); ++a2) {
                            const int cc[3] = {a0, a1, a2};
                            const int s = Lv.find(j, cc);
                            if (s < 0) continue;
                            if (eid < 0) {
                                const auto key = std::make_tuple(l, k, j);
                                auto it = epair.find(key);
                                if (it == epair.end()) {
                                    eid = (int)e_level.size();
                                    epair[key] = eid;
                                    e_level.push_back(l);
                                    for (int a = 0; a < na; ++a)
                                        for (int bb = 0; bb < na; ++bb) dts.push_back(node(l, k, bb) - node(l, j, a));
                                } else {
                                    eid = it->second;
                                }
                            }
                            pairs.push_back({h->lvoff[l] + s, eid});
                            mptr[g + 1]++;
                        }
            }
            if (mptr[g + 1] > mptr[g]) h->m2l_targets.push_back(g);
        }
    }
    h->n_m2l_pairs = (int64_t)pairs.size();
    // ---- nearfield blocks of the leaves
    std::vector<int> nptr(h->nbox + 1, 0);
    std::vector<GNear> blocks;
    int64_t off = 0;
    std::vector<int> tmp;
    for (int l = 0; l < L; ++l) {
        const GenLevel &Lv = lv[l];
        for (size_t b = 0; b < Lv.kk.size(); ++b) {
            const int g = h->lvoff[l] + (int)b;
            nptr[g + 1] = nptr[g];
            if (!Lv.leaf[b]) continue;
            std::vector<int> src;
            near_same(Lv, (int)b, tmp);
            for (int s : tmp) src.push_back(h->lvoff[l] + s);
            for (int q = l - 1, a = Lv.par[b]; q >= 0 && a >= 0; a = lv[q].par[a], --q) {
                near_same(lv[q], a, tmp);
                for (int s : tmp)
                    if (lv[q].leaf[s]) src.push_back(h->lvoff[q] + s);
            }
            const GBox &T = h->boxes[g];
            for (int s : src) {
                const GBox &S = h->boxes[s];
                blocks.push_back({g, s, off});
                off += (int64_t)(T.t1 - T.t0) * (T.a1 - T.a0) * (S.t1 - S.t0) * (S.a1 - S.a0);
                nptr[g + 1]++;
            }
        }
    }
    h->n_blocks = (int64_t)blocks.size();
    h->nf_entries = off;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(PFMM_ERR_CUDA, "cudaMemGetInfo failed");
    if ((double)off * 8.0 > 0.6 * (double)fr)
        return fail(PFMM_ERR_OOM, "general-step nearfield needs " + std::to_string(off * 8) + " bytes (" +
                                      std::to_string(fr) + " free)");
    // ---- device copies of the tree and lists
    std::vector<int> tri_int(3 * (size_t)nt), lvG(L), lvst(L, 0);
    for (int i = 0; i < nt; ++i)
        for (int v = 0; v < 3; ++v) tri_int[3 * i + v] = m.triangles[3 * perm[i] + v];
    for (int l = 0; l < L; ++l) {
        lvG[l] = lv[l].G;
        lvst[l] = l ? lv[l - 1].st_next : 0;
    }
    // multi-indices |kappa| <= m_x graded by total degree: those with |kappa| <= d are a prefix of
    // C(d + 3, 3) entries (the M2L kernel sums over such prefixes)
    std::vector<int> kidx, kinv((size_t)m1 * m1 * m1, -1);
    for (int deg = 0; deg <= mx; ++deg)
        for (int a = deg; a >= 0; --a)
            for (int b = deg - a; b >= 0; --b) {
                const int c = deg - a - b;
                kinv[((size_t)a * m1 + b) * m1 + c] = (int)kidx.size() / 3;
                kidx.insert(kidx.end(), {a, b, c});
            }
    h->nk = (int)kidx.size() / 3;
    std::vector<double> verts(m.vertices, m.vertices + 3 * (size_t)m.n_vertices), tsv(ts_host, ts_host + E + 1);
    double *d_verts = nullptr, *d_ts = nullptr;
    if ((rc = h->upload(&h->d_box, h->boxes, st)) || (rc = h->upload(&h->d_perm, perm, st)) ||
        (rc = h->upload(&h->d_tri, tri_int, st)) || (rc = h->upload(&d_verts, verts, st)) ||
        (rc = h->upload(&d_ts, tsv, st)) || (rc = h->upload(&h->d_kidx, kidx, st)) ||
        (rc = h->upload(&h->d_kinv, kinv, st)) || (rc = h->upload(&h->d_lvG, lvG, st)) ||
        (rc = h->upload(&h->d_lvst, lvst, st)) || (rc = h->upload(&h->d_leaves_all, h->leaves_all, st)) ||
        (rc = h->upload(&h->d_leaves_far, h->leaves_far, st)) ||
        (rc = h->upload(&h->d_m2l_targets, h->m2l_targets, st)) || (rc = h->upload(&h->d_mptr, mptr, st)) ||
        (rc = h->upload(&h->d_pairs, pairs, st)) || (rc = h->upload(&h->d_nptr, nptr, st)) ||
        (rc = h->upload(&h->d_blocks, blocks, st)))
        return rc;
    h->d_parents_lv.assign(L, nullptr);
    h->d_all_lv.assign(L, nullptr);
    for (int l = 0; l < L; ++l)
        if ((rc = h->upload(&h->d_parents_lv[l], h->parents_lv[l], st)) ||
            (rc = h->upload(&h->d_all_lv[l], h->all_lv[l], st)))
            return rc;
    // ---- time tables: St[l][j][a] = int over step j of L_{I,a} (I the level-l interval holding j),
    // q^(t) of every box against its parent (Eq. temp_m2m); Gauss-Legendre with m_t + 1 points (exact)
    std::vector<double> gx, gw;
    hostm::gauss01(na, gx, gw);
    std::vector<double> St((size_t)L * E * na, 0.0), qt((size_t)h->nbox * na * na, 0.0);
    for (int l = 0; l < L; ++l)
        for (size_t k = 0; k < lv[l].ia.size(); ++k) {
            const int a0 = lv[l].ia[k], a1 = lv[l].ib[k];
            if (a0 < 0) continue;
            for (int j = a0; j < a1; ++j)
                for (int a = 0; a < na; ++a) {
                    double v = 0;
                    const double hj = ts_host[j + 1] - ts_host[j];
                    for (int i = 0; i < na; ++i)
                        v += gw[i] * hj * hostm::lagrange(a, h->prm.m_t, ts_host[a0], ts_host[a1], ts_host[j] + hj * gx[i]);
                    St[((size_t)l * E + j) * na + a] = v;
                }
        }
    for (int g = 0; g < h->nbox; ++g) {
        const GBox &B = h->boxes[g];
        if (B.par < 0) continue;
        const GBox &P = h->boxes[B.par];
        for (int ac = 0; ac < na; ++ac)
            for (int ap = 0; ap < na; ++ap)
                qt[((size_t)g * na + ac) * na + ap] =
                    hostm::lagrange(ap, h->prm.m_t, ts_host[P.a0], ts_host[P.a1], node(B.level, B.k, ac));
    }
    // q^(x) of each level's boxes into their parents after a space-time refinement (Eq. st_m2m)
    std::vector<double> q1((size_t)L * 2 * m1 * m1, 0.0);
    for (int l = 1; l < L; ++l) {
        if (!lvst[l]) continue;
        for (int bit = 0; bit < 2; ++bit) {
            const double dc = (2.0 * bit - 1.0) * lv[l].hx;  // child centre - parent centre
            for (int ka = 0; ka <= mx; ++ka)
                for (int nu = 0; nu <= mx; ++nu) {
                    double s = 0;
                    for (int n = 0; n <= mx; ++n) {
                        const double xn = hostm::cheb_node(n, mx);
                        s += hostm::cheb_T(nu, (dc + lv[l].hxp * xn) / lv[l - 1].hxp) * hostm::cheb_T(ka, xn);
                    }
                    q1[(((size_t)l * 2 + bit) * m1 + ka) * m1 + nu] = (ka == 0 ? 1.0 : 2.0) / (mx + 1.0) * s;
                }
        }
    }
    if ((rc = h->upload(&h->d_St, St, st)) || (rc = h->upload(&h->d_qt, qt, st)) || (rc = h->upload(&h->d_q1, q1, st)))
        return rc;
    // ---- spatial moments of the leaf levels: Sx[slot][x][kappa] w.r.t. the cell of x on that level
    {
        std::vector<double> rule = hostm::collapsed_rule(mx / 2 + 2);
        double *d_rule = nullptr, *d_SK = nullptr;
        int *d_ident = nullptr, *d_cells = nullptr;
        std::vector<int> ident(nt);
        for (int i = 0; i < nt; ++i) ident[i] = i;
        if ((rc = h->upload(&d_rule, rule, st)) || (rc = h->upload(&d_ident, ident, st)) ||
            (rc = h->alloc(&d_cells, 3 * (size_t)nt)) ||
            (rc = h->alloc(&h->d_Sx, (size_t)std::max(nslot, 1) * nt * h->nk)) ||
            (rc = h->alloc(&d_SK, (size_t)nt * 3 * h->nk)))
            return rc;
        for (int l = 0; l < L; ++l) {
            if (slot_of[l] < 0) continue;
            std::vector<int> cells(3 * (size_t)nt);
            const double w = 2.0 * H / lv[l].G;
            for (int i = 0; i < nt; ++i)
                for (int d = 0; d < 3; ++d) cells[3 * i + d] = cell_of(centroid(perm[i], d), corner[d], w, lv[l].G);
            if (cudaMemcpyAsync(d_cells, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return fail(PFMM_ERR_CUDA, "host to device copy failed");
            SetupArgs a{};
            a.verts = d_verts;
            a.tri = h->d_tri;
            a.tri_leaf = d_ident;
            a.leaf_grid = d_cells;
            for (int c = 0; c < 3; ++c) a.corner[c] = corner[c];
            a.hx_leaf = lv[l].hx;
            a.hxp_leaf = lv[l].hxp;
            a.alpha = m.alpha;
            a.nt = nt;
            a.mx = mx;
            a.nk = h->nk;
            a.kidx = h->d_kidx;
            a.rule_tab = d_rule;
            a.nq_tab = (mx / 2 + 2) * (mx / 2 + 2);
            a.Sx = h->d_Sx + (size_t)slot_of[l] * nt * h->nk;
            a.SK = d_SK;
            launch_space_tables(a, st);
            // the cell array is rewritten for the next level: finish this one first
            if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
                return fail(PFMM_ERR_CUDA, "spatial moment tables failed");
        }
    }
    // ---- E1 tables of the interval pairs (Eq. exp_coeffs_1d), level by level
    {
        const int npairs = (int)e_level.size();
        std::vector<int64_t> e1off(npairs + 1, 0);
        for (int e = 0; e < npairs; ++e)
            e1off[e + 1] = e1off[e] + (int64_t)na * na * (2 * lv[e_level[e]].G - 1) * m1 * m1;
        double *d_dts = nullptr;
        if ((rc = h->alloc(&h->d_E1, (size_t)std::max<int64_t>(e1off[npairs], 1))) ||
            (rc = h->alloc(&h->d_pref, (size_t)std::max(npairs, 1) * na * na)) || (rc = h->upload(&h->d_e1off, e1off, st)) ||
            (rc = h->upload(&d_dts, dts, st)))
            return rc;
        for (int e0 = 0; e0 < npairs;) {
            int e1 = e0;
            while (e1 < npairs && e_level[e1] == e_level[e0]) ++e1;
            const GenLevel &Lv = lv[e_level[e0]];
            launch_gen_e1(e1 - e0, d_dts + (size_t)e0 * na * na, na, mx, Lv.G, Lv.hx, Lv.hxp, m.alpha,
                          h->d_E1 + e1off[e0], h->d_pref + (size_t)e0 * na * na, st);
            e0 = e1;
        }
        double *e1df = nullptr, *prefdf = nullptr;  // 8 bytes per value either way
        if ((rc = h->alloc(&e1df, (size_t)std::max<int64_t>(e1off[npairs], 1))) ||
            (rc = h->alloc(&prefdf, (size_t)std::max(npairs, 1) * na * na)))
            return rc;
        launch_gen_to_df64(h->d_E1, e1df, e1off[npairs], st);
        launch_gen_to_df64(h->d_pref, prefdf, (int64_t)npairs * na * na, st);
        h->d_E1df = e1df;
        h->d_prefdf = prefdf;
    }
    // ---- the nearfield entries (Eq. eval_sl_nf_block with the entries of Section 2)
    {
        std::vector<double> rreg = hostm::collapsed_rule(h->prm.quad_regular), gsx, gsw;
        hostm::gauss01(h->prm.quad_singular, gsx, gsw);
        gsx.insert(gsx.end(), gsw.begin(), gsw.end());
        double *d_rreg = nullptr, *d_gls = nullptr;
        if ((rc = h->upload(&d_rreg, rreg, st)) || (rc = h->upload(&d_gls, gsx, st)) ||
            (rc = h->alloc(&h->d_A, (size_t)std::max<int64_t>(off, 1))))
            return rc;
        GenQuad q{};
        q.verts = d_verts;
        q.tri = h->d_tri;
        q.ts = d_ts;
        q.alpha = m.alpha;
        q.rule_reg = d_rreg;
        q.nq_reg = h->prm.quad_regular * h->prm.quad_regular;
        q.gl_sing = d_gls;
        q.nq_sing = h->prm.quad_singular;
        launch_gen_nf_entries(q, h->d_box, h->d_blocks, (int)blocks.size(), h->d_A, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(PFMM_ERR_CUDA, "general-step set-up kernels failed");
    return PFMM_OK;
}

int ensure_ws(pfmm_gen *h, int nrhs)
{
    if (nrhs <= h->ws_nrhs) return PFMM_OK;
    int rc;
    const size_t n = (size_t)nrhs * h->Et * h->nt, nm = (size_t)nrhs * h->nbox * h->na * h->nk;
    if ((rc = h->alloc(&h->d_wint, n)) || (rc = h->alloc(&h->d_fint, n)) || (rc = h->alloc(&h->d_mu, nm)) ||
        (rc = h->alloc(&h->d_lam, nm)) || (rc = h->alloc(&h->d_contrib, nm)))
        return rc;
    h->ws_nrhs = nrhs;
    return PFMM_OK;
}

}  // namespace

extern "C" {

int pfmm_gen_create(const pfmm_mesh *mesh, const double *t_steps, const pfmm_params *params, int32_t n_max,
                    void *stream, pfmm_gen **out)
{
    if (!mesh || !t_steps || !params || !out || n_max < 1)
        return fail(PFMM_ERR_INVALID_ARG, "invalid pfmm_gen_create arguments");
    *out = nullptr;
    const pfmm_mesh &m = *mesh;
    const pfmm_params &p = *params;
    if (m.n_vertices < 3 || m.n_triangles < 1 || m.n_steps < 1 || !m.vertices || !m.triangles || !(m.alpha > 0))
        return fail(PFMM_ERR_INVALID_ARG, "invalid mesh");
    if (p.m_t < 0 || p.m_t >= kMaxNa || p.m_x < 0 || p.m_x > kMaxMx || !(p.c_st > 0) || p.quad_regular < 1 ||
        p.quad_regular > 16 || p.quad_singular < 1 || p.quad_singular > 16)
        return fail(PFMM_ERR_INVALID_ARG, "invalid parameters (m_t, m_x, c_st or quadrature orders)");
    if (p.precision != PFMM_FP64) return fail(PFMM_ERR_UNSUPPORTED, "general time steps: FP64 only");
    {
        const int m1 = p.m_x + 1, nk = m1 * (m1 + 1) * (m1 + 2) / 6;
        if (gen_m2l_smem(p.m_t + 1, nk, p.m_x) > 227 * 1024 || (p.m_t + 1) * nk > 2048)
            return fail(PFMM_ERR_UNSUPPORTED, "general time steps: m_t and m_x too large for the M2L kernel (shared memory, or (m_t + 1) x multi-indices > 2048)");
    }
    if (t_steps[0] != 0.0) return fail(PFMM_ERR_INVALID_ARG, "t_steps[0] must be 0");
    for (int j = 0; j < m.n_steps; ++j)
        if (!(t_steps[j + 1] > t_steps[j]) || !std::isfinite(t_steps[j + 1]))
            return fail(PFMM_ERR_INVALID_ARG, "t_steps must increase strictly and be finite");
    if (std::fabs(t_steps[m.n_steps] - m.T) > 1e-12 * std::fabs(m.T))
        return fail(PFMM_ERR_INVALID_ARG, "t_steps[n_steps] must equal mesh->T");
    for (int i = 0; i < 3 * m.n_vertices; ++i)
        if (!std::isfinite(m.vertices[i])) return fail(PFMM_ERR_NONFINITE, "non-finite vertex coordinate");
    for (int i = 0; i < 3 * m.n_triangles; ++i)
        if (m.triangles[i] < 0 || m.triangles[i] >= m.n_vertices)
            return fail(PFMM_ERR_INVALID_ARG, "triangle vertex index out of range");
    pfmm_gen *h = new (std::nothrow) pfmm_gen();
    if (!h) return fail(PFMM_ERR_OOM, "host allocation failed");
    h->nv = m.n_vertices;
    h->nt = m.n_triangles;
    h->Et = m.n_steps;
    h->alpha = m.alpha;
    h->prm = p;
    h->n_max = n_max;
    int rc;
    try {
        rc = build_impl(h, m, t_steps, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        rc = fail(PFMM_ERR_OOM, "host allocation failed");
    } catch (const std::exception &e) {
        rc = fail(PFMM_ERR_INVALID_ARG, std::string("general tree build: ") + e.what());
    }
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return PFMM_OK;
}

int pfmm_gen_apply_V(pfmm_gen *h, const double *w, double *f, int32_t nrhs, int32_t parts, void *stream)
{
    if (!h || !w || !f || nrhs < 1 || parts < 1 || parts > 3) return fail(PFMM_ERR_INVALID_ARG, "invalid apply arguments");
    int rc;
    if ((rc = ensure_ws(h, nrhs))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int rows = nrhs * h->Et;
    launch_gen_permute_in(w, h->d_wint, h->d_perm, h->nt, rows, st);
    if (parts & PFMM_PART_NEAR)
        launch_gen_nf_apply(h->d_box, h->d_leaves_all, (int)h->leaves_all.size(), h->d_nptr, h->d_blocks, h->d_A,
                            h->d_wint, h->d_fint, h->nt, h->Et, nrhs, st);
    else if (cudaMemsetAsync(h->d_fint, 0, sizeof(double) * rows * (size_t)h->nt, st) != cudaSuccess)
        return fail(PFMM_ERR_CUDA, "cudaMemsetAsync failed");
    if ((parts & PFMM_PART_FAR) && h->nlev >= 3) {
        GenDev g{};
        g.box = h->d_box;
        g.nbox = h->nbox;
        g.nt = h->nt;
        g.Et = h->Et;
        g.nrhs = nrhs;
        g.na = h->na;
        g.nk = h->nk;
        g.mx = h->mx;
        g.kidx = h->d_kidx;
        g.kinv = h->d_kinv;
        g.lvG = h->d_lvG;
        g.lvst = h->d_lvst;
        g.Sx = h->d_Sx;
        g.St = h->d_St;
        g.qt = h->d_qt;
        g.q1 = h->d_q1;
        g.mu = h->d_mu;
        g.lam = h->d_lam;
        launch_gen_s2m(g, h->d_leaves_far, (int)h->leaves_far.size(), h->d_wint, st);
        for (int l = h->nlev - 2; l >= 2; --l)
            launch_gen_m2m(g, h->d_parents_lv[l], (int)h->parents_lv[l].size(), h->d_all_lv[l + 1],
                           (int)h->all_lv[l + 1].size(), h->d_contrib, st);
        if (cudaMemsetAsync(h->d_lam, 0, sizeof(double) * (size_t)nrhs * h->nbox * h->na * h->nk, st) != cudaSuccess)
            return fail(PFMM_ERR_CUDA, "cudaMemsetAsync failed");
        // the moments as double-FP32 pairs (into the M2M contribution buffer, free by now)
        launch_gen_to_df64(h->d_mu, h->d_contrib, (int64_t)nrhs * h->nbox * h->na * h->nk, st);
        launch_gen_m2l(g, h->d_m2l_targets, (int)h->m2l_targets.size(), h->d_mptr, h->d_pairs, h->d_E1df, h->d_e1off,
                       h->d_prefdf, h->d_contrib, st);
        for (int l = 3; l < h->nlev; ++l) launch_gen_l2l(g, h->d_all_lv[l], (int)h->all_lv[l].size(), st);
        launch_gen_l2t(g, h->d_leaves_far, (int)h->leaves_far.size(), h->d_fint, st);
    }
    launch_gen_permute_out(h->d_fint, f, h->d_perm, h->nt, rows, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, std::string("general-step apply: ") + cudaGetErrorString(e));
    return PFMM_OK;
}

int pfmm_gen_get_info(const pfmm_gen *h, pfmm_gen_info *info)
{
    if (!h || !info) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->nlev = h->nlev;
    for (int l = 0; l < h->nlev && l < 32; ++l) {
        const GenLevel &L = h->lv[l];
        info->lx[l] = L.lx;
        info->nbox[l] = (int32_t)L.kk.size();
        info->nleaf[l] = (int32_t)std::count(L.leaf.begin(), L.leaf.end(), 1);
        info->nint[l] = (int32_t)std::count_if(L.ia.begin(), L.ia.end(), [](int a) { return a >= 0; });
        info->ntr_far[l] = L.ntr_far;
        info->ntr_near[l] = L.ntr_near;
        info->st[l] = L.st_next;
        info->pad[l] = L.pad;
    }
    info->n_m2l_pairs = h->n_m2l_pairs;
    info->n_near_blocks = h->n_blocks;
    info->nearfield_entries = h->nf_entries;
    info->device_bytes = h->dev_bytes;
    return PFMM_OK;
}

int pfmm_gen_boxes(const pfmm_gen *h, int32_t *rows, int64_t cap, int64_t *count)
{
    if (!h || !count || cap < 0 || (cap > 0 && !rows)) return fail(PFMM_ERR_INVALID_ARG, "invalid pfmm_gen_boxes arguments");
    *count = h->nbox;
    for (int64_t g = 0; g < h->nbox && g < cap; ++g) {
        const GBox &B = h->boxes[g];
        const GenLevel &L = h->lv[B.level];
        const int b = (int)(g - h->lvoff[B.level]);
        int32_t *o = rows + 8 * g;
        o[0] = B.level;
        o[1] = B.cell[0];
        o[2] = B.cell[1];
        o[3] = B.cell[2];
        o[4] = B.k;
        o[5] = L.leaf[b];
        o[6] = B.a0;
        o[7] = B.a1;
    }
    return PFMM_OK;
}

void pfmm_gen_destroy(pfmm_gen *h) { delete h; }

}  // extern "C"
