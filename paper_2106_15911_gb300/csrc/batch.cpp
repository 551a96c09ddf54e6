// batch.cpp -- many independent problems per call: a batch of handles applied through one
// captured CUDA graph (one branch per problem on a pool of streams, joined at the end), and an
// autotuner for the expansion degree and the nearfield engine.
//
// Degree selection (a priori): the spatial expansion of Section 3.1 truncates the Chebyshev
// expansion of exp(-(r + x - y)^2 / d) (Eq. exp_coeffs_1d) at total degree m_x.  For every level
// with M2L the smallest d_ab = 4 alpha dt_min / h~x^2 (dt_min = separation of interval nodes at
// gap 2) is the hardest case; the estimate for m_x is the largest dropped coefficient
// |E_{k,l}(r, d_min)| with k + l in {m_x + 1, m_x + 2} and r in {0, 2} (coincident and
// neighbouring boxes), relative to |E_{0,0}(0, d_min)|.  The smallest m_x in
// [m_lo, m_hi] whose estimate is below tol is taken.
// Engine selection (measured with CUDA events): for each problem the tensor-core and CUDA-core
// nearfield applies (where the panels allow the tensor cores) and the M2L kernel forms (fused,
// sliced fused, three global passes, where each can run the problem's levels) are timed after a
// warm-up, and the fastest of each is kept.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "handle.h"
#include "kernels.h"

namespace {

using pfmm::set_error;

constexpr double kPi = 3.14159265358979323846;

double cheb_node(int k, int m) { return std::cos((2.0 * k + 1.0) * kPi / (2.0 * m + 2.0)); }

// E_{k,l}(r, d) of Eq. exp_coeffs_1d
double e1(int k, int l, double r, double d, int m)
{
    double s = 0.0;
    for (int n = 0; n <= m; ++n)
        for (int q = 0; q <= m; ++q) {
            double xn = cheb_node(n, m), xq = cheb_node(q, m), z = r + xn - xq;
            s += std::exp(-z * z / d) * std::cos(l * std::acos(xn)) * std::cos(k * std::acos(xq));
        }
    return (k ? 2.0 : 1.0) * (l ? 2.0 : 1.0) / ((m + 1.0) * (m + 1.0)) * s;
}

}  // namespace

struct pfmm_batch {
    std::vector<pfmm_handle *> h;
    std::vector<cudaStream_t> pool;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const double *> last_w;
    std::vector<double *> last_f;
    std::vector<int> last_n;
    ~pfmm_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto s : pool) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
        if (fork) cudaEventDestroy(fork);
        for (auto e : join) cudaEventDestroy(e);
        for (auto x : h) pfmm_destroy(x);
    }
};

extern "C" {

int pfmm_autotune_params(const pfmm_mesh *mesh, const pfmm_params *base, double tol, int32_t m_lo, int32_t m_hi,
                         pfmm_params *out)
{
    if (!mesh || !base || !out || !(tol > 0) || m_lo < 0 || m_hi < m_lo || m_hi > pfmm::kMaxMx)
        return set_error(PFMM_ERR_INVALID_ARG, "invalid autotune arguments");
    pfmm::Tree t;
    std::string err;
    int rc = pfmm::build_tree(*mesh, *base, t, err);
    if (rc) return set_error(rc, err);
    double dmin = 1e300;
    for (int l = 2; l <= t.p; ++l) {
        const pfmm::Level &L = t.lv[l];
        const double dt = 4.0 * L.ht - 2.0 * L.ht * cheb_node(0, base->m_t);  // gap-2 intervals, extreme nodes
        dmin = std::min(dmin, 4.0 * mesh->alpha * dt / (L.hxp * L.hxp));
    }
    *out = *base;
    if (dmin == 1e300) {  // no M2L level: the degree does not matter
        out->m_x = m_lo;
        return PFMM_OK;
    }
    for (int m = m_lo; m <= m_hi; ++m) {
        // first two dropped diagonals (the odd one vanishes for coincident boxes by symmetry), for
        // coincident (r = 0) and face-neighbouring (r = 2) boxes
        const double e00 = std::fabs(e1(0, 0, 0.0, dmin, m + 3));
        double worst = 0.0;
        for (double r : {0.0, 2.0})
            for (int s = m + 1; s <= m + 2; ++s)
                for (int k = 0; k <= s; ++k) worst = std::max(worst, std::fabs(e1(k, s - k, r, dmin, m + 3)));
        out->m_x = m;
        if (worst <= tol * e00) return PFMM_OK;
    }
    out->m_x = m_hi;
    return PFMM_OK;
}

int pfmm_build_trees_batched(int32_t n, const pfmm_mesh *meshes, const pfmm_params *params, int32_t tune_engines,
                             void *stream, pfmm_batch **out)
{
    if (n < 1 || !meshes || !params || !out) return set_error(PFMM_ERR_INVALID_ARG, "invalid batch arguments");
    *out = nullptr;
    pfmm_batch *B = new pfmm_batch();
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        pfmm_handle *h = nullptr;
        int rc = pfmm_build_trees(&meshes[i], &params[i], stream, &h);
        if (rc) {
            delete B;
            return rc;
        }
        B->h.push_back(h);
    }
    const int S = std::min(n, 16);
    B->pool.resize(S);
    for (int i = 0; i < S; ++i) cudaStreamCreateWithFlags(&B->pool[i], cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    B->join.resize(n);
    for (auto &e : B->join) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (tune_engines) {
        // per problem, timed with CUDA events on the build stream after a warm-up: the nearfield
        // engine (tensor cores or CUDA cores) on the nearfield part, then the M2L kernel form
        // (the per-level default, the fused kernel, its sliced form, the three global passes) on
        // the far field; the fastest of each is kept
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        int rc_t = PFMM_OK;
        for (pfmm_handle *h : B->h) {
            double *x = nullptr, *f = nullptr;
            size_t nn = (size_t)h->Et * h->nt;
            if (cudaMalloc(&x, nn * sizeof(double)) != cudaSuccess || cudaMalloc(&f, nn * sizeof(double)) != cudaSuccess) {
                cudaFree(x);
                rc_t = set_error(PFMM_ERR_OOM, "autotune buffers");
                break;
            }
            cudaMemsetAsync(x, 0, nn * sizeof(double), st);
            auto timed = [&](int parts, float &ms) {
                int rc = pfmm_apply_parts(h, 0, x, f, 1, parts, stream);  // warm-up
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3 && !rc; ++r) rc = pfmm_apply_parts(h, 0, x, f, 1, parts, stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                return rc;
            };
            float best = 1e30f, ms = 0.f;
            if (h->tcV) {
                bool cc = false;
                for (int eng = 0; eng < 2 && !rc_t; ++eng) {
                    h->nf_cuda_cores = eng == 1;
                    if ((rc_t = timed(PFMM_PART_NEAR, ms))) break;
                    if (ms < best) {
                        best = ms;
                        cc = eng == 1;
                    }
                }
                h->nf_cuda_cores = cc;
            }
            const int cands[4] = {0, PFMM_M2L_FUSED, PFMM_M2L_FUSED_SLICED, PFMM_M2L_THREE_PASS};
            int best_c = 0;
            best = 1e30f;
            for (int c : cands) {
                if (rc_t || h->p < 2) break;
                // skip a candidate that runs the same kernels as one already timed
                bool differs = c == 0;
                for (int l = 2; l <= h->p && !differs; ++l)
                    differs = pfmm::m2l_engine_for(h->fprec, h->dl[l].G, h->nk, h->ne, h->mx, c) !=
                              pfmm::m2l_engine(h->fprec, h->dl[l].G, h->nk, h->ne, h->mx);
                if (!differs) continue;
                h->m2l_force = c;
                if ((rc_t = timed(PFMM_PART_FAR, ms))) break;
                if (ms < best) {
                    best = ms;
                    best_c = c;
                }
            }
            h->m2l_force = best_c;
            cudaFree(x);
            cudaFree(f);
            if (rc_t) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc_t) {
            delete B;
            return rc_t;
        }
    }
    *out = B;
    return PFMM_OK;
}

int pfmm_batch_handle(pfmm_batch *b, int32_t i, pfmm_handle **h)
{
    if (!b || !h || i < 0 || i >= (int)b->h.size()) return set_error(PFMM_ERR_INVALID_ARG, "invalid batch index");
    *h = b->h[i];
    return PFMM_OK;
}

int pfmm_apply_V_batched(pfmm_batch *b, const double *const *w, double *const *f, const int32_t *nrhs, void *stream)
{
    if (!b || !w || !f || !nrhs) return set_error(PFMM_ERR_INVALID_ARG, "invalid batched apply arguments");
    const int n = (int)b->h.size();
    bool same = (int)b->last_w.size() == n && b->exec;
    for (int i = 0; i < n; ++i) {
        if (!w[i] || !f[i] || nrhs[i] < 1) return set_error(PFMM_ERR_INVALID_ARG, "invalid batched apply arguments");
        if (same && (b->last_w[i] != w[i] || b->last_f[i] != f[i] || b->last_n[i] != nrhs[i])) same = false;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!same) {
        // workspaces must exist before the capture (no allocation inside a graph)
        for (int i = 0; i < n; ++i) {
            int rc = pfmm::ensure_ws(b->h[i], nrhs[i]);
            if (rc) return rc;
            b->h[i]->prof = false;
        }
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        cudaEventRecord(b->fork, b->cap);
        int rc_all = PFMM_OK;
        for (int i = 0; i < n; ++i) {
            cudaStream_t s = b->pool[i % b->pool.size()];
            cudaStreamWaitEvent(s, b->fork, 0);
            int rc = pfmm_apply_V(b->h[i], w[i], f[i], nrhs[i], s);
            if (rc && !rc_all) rc_all = rc;
            cudaEventRecord(b->join[i], s);
            cudaStreamWaitEvent(b->cap, b->join[i], 0);
        }
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (rc_all) return rc_all;
        if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        b->last_w.assign(w, w + n);
        b->last_f.assign(f, f + n);
        b->last_n.assign(nrhs, nrhs + n);
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return PFMM_OK;
}

int32_t pfmm_batch_size(const pfmm_batch *b) { return b ? (int32_t)b->h.size() : 0; }

int pfmm_batch_set_streams(pfmm_batch *b, int32_t nstreams)
{
    if (!b || nstreams < 1 || nstreams > 64) return set_error(PFMM_ERR_INVALID_ARG, "stream count must be 1..64");
    for (auto s : b->pool) cudaStreamDestroy(s);
    b->pool.assign(std::min<int>(nstreams, (int)b->h.size()), nullptr);
    for (auto &s : b->pool)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(PFMM_ERR_CUDA, "stream creation failed");
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->last_w.clear();  // the next apply captures again
    return PFMM_OK;
}

void pfmm_batch_destroy(pfmm_batch *b) { delete b; }

}  // extern "C"
