// noalloc.cu -- pfmm_apply_V_noalloc: f = V_h w with every per-call workspace taken from one
// fixed, file-scope device array instead of cudaMalloc.
//
// Why: pfmm_apply_V sizes its workspaces (the permuted input, the FP64 output accumulator,
// moments, locals and the separable-M2L intermediates) on first use and again whenever a
// larger nrhs arrives, and each of those cudaMalloc calls may block the whole device and may
// fail under memory pressure.  Some callers cannot accept that: services that must not
// allocate device memory once they are running (an allocation mid-run can stall unrelated
// work and cannot be recovered from at that point), and hosts whose device memory is owned
// by their own allocator or budget and forbid allocations from libraries.  This entry point
// allocates nothing: the workspaces live in g_pfmm_scratch, a static __device__ array of
// kScratchBytes (64 MiB) that every GPU loading the library keeps until the process exits.
// The handle's tables and nearfield blocks are still the ones pfmm_build_trees allocated.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "handle.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_pfmm_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_pfmm_scratch on the current device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up once per device with that device current.
int scratch_base(unsigned char **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pfmm::set_error(PFMM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return pfmm::set_error(PFMM_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        // with lazy module loading (the runtime's default) this first lookup also loads the module
        // that holds the array, which is when its 64 MiB are committed on this device: a failure
        // for lack of memory is reported as PFMM_ERR_OOM
        e = cudaGetSymbolAddress(&p, g_pfmm_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return pfmm::set_error(e == cudaErrorMemoryAllocation ? PFMM_ERR_OOM : PFMM_ERR_CUDA,
                                   std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return PFMM_OK;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int pfmm_apply_V_noalloc(pfmm_handle *H, const double *w, double *f, int32_t nrhs, void *stream)
{
    using namespace pfmm;
    if (!H || !w || !f || nrhs < 1) return set_error(PFMM_ERR_INVALID_ARG, "invalid pfmm_apply_V_noalloc arguments");
    cudaStream_t st = (cudaStream_t)stream;
    // carve the static array: permuted input | FP64 output | moments | locals |
    // [tensor-core input split hi | lo | max |w| per rhs | partial planes] | M2L T1 | M2L T2
    const size_t n_in = (size_t)nrhs * H->Et * H->nt;
    const size_t b_x = up256(n_in * H->es), b_f = up256(n_in * sizeof(double));
    const size_t n_mom = (size_t)nrhs * (H->mom_per_rhs > 0 ? H->mom_per_rhs : 1);
    const size_t b_mu = up256(n_mom * H->es);
    const bool tc = H->tcV && !H->nf_cuda_cores;
    const size_t b_w = tc ? up256((size_t)nrhs * H->Et * H->colsV_u * sizeof(uint16_t)) : 0;
    const size_t b_m = tc ? up256((size_t)nrhs * sizeof(unsigned long long)) : 0;
    const size_t b_p = tc ? up256((size_t)nf_tc_planes(H, 0, nrhs) * n_in * sizeof(double)) : 0;
    const size_t fixed = b_x + b_f + 2 * b_mu + 2 * b_w + b_m + b_p;
    // elements of T1 (and of T2) for the largest single-interval chunk of the levels whose M2L
    // takes the three separable passes (the fused and slab kernels keep their intermediates in
    // shared memory; the fused kernel's split mode and the two-stage S2M / L2T use T1 only when
    // it is large enough and fall back otherwise)
    size_t need_T = 0;
    for (int l = 2; l <= H->p; ++l) {
        const DevLevel &L = H->dl[l];
        if (m2l_engine_for(H->fprec, L.G, H->nk, H->ne, H->mx, H->m2l_force) != kM2LThreePass) continue;
        int maxpairs = 0;
        for (int k = 0; k < L.nint; ++k) maxpairs = std::max(maxpairs, L.kptr_host[k + 1] - L.kptr_host[k]);
        need_T = std::max(need_T, (size_t)nrhs * maxpairs * H->na * H->na * L.G * L.G * L.G * H->ne);
    }
    if (fixed + 2 * up256(need_T * H->es) > kScratchBytes)
        return set_error(PFMM_ERR_OOM, "pfmm_apply_V_noalloc needs " + std::to_string(fixed + 2 * up256(need_T * H->es)) +
                                           " bytes of scratch; the static scratch holds " +
                                           std::to_string(kScratchBytes) + " bytes");
    unsigned char *base = nullptr;
    int rc = scratch_base(&base);
    if (rc) return rc;
    void *xint = base;
    double *fint = (double *)(base + b_x);
    char *mu = (char *)(base + b_x + b_f);
    char *lam = mu + b_mu;
    void *whi = lam + b_mu, *wlo = lam + b_mu + b_w;
    unsigned long long *wmax = (unsigned long long *)(lam + b_mu + 2 * b_w);
    double *part = (double *)(lam + b_mu + 2 * b_w + b_m);
    const size_t t_bytes = (kScratchBytes - fixed) / 2 / 256 * 256;
    void *T1 = base + fixed, *T2 = base + fixed + t_bytes;
    const size_t ws_elems = t_bytes / H->es;

    ApplyGeo g{};
    g.nt = H->nt;
    g.nv = H->nv;
    g.Et = H->Et;
    g.ls = H->ls;
    g.nd = H->nd;
    g.na = H->na;
    g.nk = H->nk;
    g.mx = H->mx;
    g.p = H->p;
    g.perm = H->d_perm;
    g.tri = H->d_tri_int;
    g.leaf_start = H->d_leaf_start;
    g.nbox_leaf = H->tree.lv[H->p].nbox;
    g.kidx = H->d_kidx;
    g.kinv = H->d_kinv;
    g.ne = H->ne;
    g.eoff = H->d_eoff;
    g.nsm = H->nsm;
    g.m2l_force = H->m2l_force;
    if ((int)H->tree.panels.size() == g.nbox_leaf) {  // one row panel per leaf box: its 64-row tiles
        g.tiles = H->d_tiles;
        g.ntiles = H->ntiles;
        g.box_tiles = H->d_box_tiles;
    }
    // every buffer below is fully written before it is read, except the locals of the first two
    // intervals of each level, which launch_m2l clears; nothing depends on the previous call
    launch_permute_in(w, xint, H->mixed, nrhs, g, st);
    if (tc) {  // the same nearfield engine as pfmm_apply_V
        if ((rc = run_nf_tc(H, 0, w, nrhs, whi, wlo, wmax, fint, part, st))) return rc;
    } else if (H->otf) {
        cudaMemsetAsync(fint, 0, n_in * sizeof(double), st);
        if ((rc = run_nf_otf(H, 0, xint, H->nt, H->Et, H->ls, nrhs, 1 << 30, fint, st))) return rc;
    } else {
        NfHalfSplit hs;
        launch_nf_apply(H->mixed, false, H->nf_blocks(0), H->d_colV, H->d_tiles, H->ntiles, H->d_panels, xint, H->nt, nrhs,
                        g, fint, st, 1 << 30, H->nf_split(0, &hs));
    }
    const int p = H->p;
    if (p >= 2) {
        launch_s2m(H->fprec, false, xint, H->nt, H->d_Sx, H->d_St, mu + H->dl[p].mom_off * H->es * nrhs, nrhs, g, st, T1,
                   ws_elems);
        for (int l = p - 1; l >= 2; --l) launch_m2m(H->fprec, H->dl[l], H->dl[l + 1], l, H->d_qt, mu, nrhs, g, 0, st);
        for (int l = 2; l <= p; ++l)
            if (launch_m2l(H->fprec, H->dl[l], l, mu, lam, nrhs, g, T1, T2, ws_elems, st))
                return set_error(PFMM_ERR_OOM, "static scratch too small for one M2L interval");
        for (int l = 3; l <= p; ++l) launch_l2l(H->fprec, H->dl[l - 1], H->dl[l], l, H->d_qt, lam, nrhs, g, 0, st);
        launch_l2t(H->fprec, lam + H->dl[p].mom_off * H->es * nrhs, H->d_Sx, H->d_St, fint, nrhs, g, 0, st, T1, ws_elems);
    }
    launch_permute_out(fint, f, nrhs, g, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string("pfmm_apply_V_noalloc: ") + cudaGetErrorString(e));
    return PFMM_OK;
}
