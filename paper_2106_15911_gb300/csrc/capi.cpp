// capi.cpp -- the C ABI of include/pfmm.h: handle life cycle, one-time set-up and the apply
// sequence of Alg. 2 (Section 3.4) on the caller's CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "host_math.h"
#include "kernels.h"
#include "nf_tc.h"
#include "nf_crt.h"
#include "pfmm_internal.h"

using namespace pfmm;

namespace pfmm {
int set_error(int code, const std::string &msg);
}

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? PFMM_ERR_OOM : PFMM_ERR_CUDA,                \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

}  // namespace

int pfmm::set_error(int code, const std::string &msg) { return fail(code, msg); }

namespace {

using hostm::cheb_node;
using hostm::cheb_T;
using hostm::collapsed_rule;
using hostm::gauss01;
using hostm::lagrange;

}  // namespace

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// FP16 tensor map, 128-byte swizzle, zero fill out of bounds; dims innermost first
int encode_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
               const uint32_t *box)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(PFMM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t d[5], s[4];
    cuuint32_t b[5], e[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i > 0) s[i - 1] = strides_bytes[i - 1];
    }
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, rank, const_cast<void *>(base), d, s, b, e,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PFMM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return PFMM_OK;
}

template <typename T_>
int upload(pfmm_handle *H, T_ **dst, const std::vector<T_> &src, cudaStream_t st)
{
    int rc = H->alloc(dst, src.size());
    if (rc) return rc;
    if (!src.empty()) CK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T_), cudaMemcpyHostToDevice, st));
    return PFMM_OK;
}

// upload a host FP64 table in the arithmetic type of the handle's FMM passes (FP32, FP64, or
// double-FP32 pairs converted in place)
int upload_R(pfmm_handle *H, void **dst, const std::vector<double> &src, cudaStream_t st)
{
    if (!H->mixed) {
        int rc = upload(H, (double **)dst, src, st);
        if (!rc && H->fprec == 2) launch_to_df64((double *)*dst, src.size(), st);
        return rc;
    }
    std::vector<float> f(src.begin(), src.end());
    return upload(H, (float **)dst, f, st);
}

// convert a device FP64 table to the handle's type (in place of a new buffer)
int device_to_R(pfmm_handle *H, void **dst, double *src, size_t n, cudaStream_t st)
{
    if (!H->mixed) {
        if (H->fprec == 2) launch_to_df64(src, n, st);
        *dst = src;
        return PFMM_OK;
    }
    float *f = nullptr;
    int rc = H->alloc(&f, n);
    if (rc) return rc;
    launch_cast_to_float(src, f, n, st);
    *dst = f;
    return PFMM_OK;
}

int ensure_workspace(pfmm_handle *H, int nrhs)
{
    if (nrhs <= H->ws_nrhs) return PFMM_OK;
    H->release(H->d_xint);
    H->release(H->d_gf);
    H->release(H->d_mu);
    H->release(H->d_lam);
    H->release(H->d_fint);
    H->d_xint = H->d_gf = H->d_mu = H->d_lam = nullptr;
    H->d_fint = nullptr;
    H->ws_nrhs = 0;
    size_t n_in = (size_t)nrhs * H->Et * H->nt, n_g = (size_t)nrhs * H->Et * H->nv;
    int rc;
    if ((rc = H->alloc((char **)&H->d_xint, n_in * H->es, 1))) return rc;
    if (H->mixed && (rc = H->alloc((float **)&H->d_gf, n_g))) return rc;
    if ((rc = H->alloc(&H->d_fint, n_in))) return rc;
    size_t nm = (size_t)nrhs * std::max<int64_t>(H->mom_per_rhs, 1);
    if ((rc = H->alloc((char **)&H->d_mu, nm * H->es, 1))) return rc;
    if ((rc = H->alloc((char **)&H->d_lam, nm * H->es, 1))) return rc;
    // separable M2L intermediates: a whole level at once when it fits in 2 x 256 MB, else chunks
    H->release(H->d_T1);
    H->release(H->d_T2);
    H->d_T1 = H->d_T2 = nullptr;
    size_t need = (size_t)nrhs * std::max<int64_t>(H->m2l_ws_need, 1);
    size_t cap = (size_t)(256u << 20) / H->es;
    size_t min_chunk = (size_t)nrhs * 2 * H->na * H->na * H->ne * 64;  // at least two pairs of a 4^3 grid
    H->ws_m2l = std::max(std::min(need, cap), min_chunk);
    if ((rc = H->alloc((char **)&H->d_T1, H->ws_m2l * H->es, 1))) return rc;
    if ((rc = H->alloc((char **)&H->d_T2, H->ws_m2l * H->es, 1))) return rc;
    H->release(H->d_Whi);
    H->release(H->d_Wlo);
    H->release(H->d_wmax);
    H->release(H->d_nfpart);
    H->d_Whi = H->d_Wlo = nullptr;
    H->d_wmax = nullptr;
    H->d_nfpart = nullptr;
    if (H->tcV || H->tcK) {
        H->w_elems = (size_t)nrhs * H->Et * std::max(H->colsV_u, H->colsK_u);
        const int planes = std::max(H->tcV ? pfmm::nf_tc_planes(H, 0, nrhs) : 1, H->tcK ? pfmm::nf_tc_planes(H, 1, nrhs) : 1);
        if ((rc = H->alloc(&H->d_Whi, H->w_elems)) || (rc = H->alloc(&H->d_Wlo, H->w_elems)) ||
            (rc = H->alloc(&H->d_wmax, (size_t)nrhs)) || (rc = H->alloc(&H->d_nfpart, (size_t)planes * n_in)))
            return rc;
    }
    H->release(H->d_Wres);
    H->release(H->d_res8);
    H->d_Wres = nullptr;
    H->d_res8 = nullptr;
    if (H->crtV || H->crtK) {
        const size_t nw = (size_t)kCrtModuli * nrhs * H->Et * std::max(H->colsV_u, H->colsK_u);
        if ((rc = H->alloc(&H->d_Wres, nw)) || (rc = H->alloc(&H->d_res8, (size_t)kCrtModuli * n_in)) ||
            (!H->d_wmax && (rc = H->alloc(&H->d_wmax, (size_t)nrhs))))
            return rc;
    }
    H->ws_nrhs = nrhs;
    return PFMM_OK;
}

void prof_collect(pfmm_handle *H, int upto_pending)
{
    while (H->ev_pending > upto_pending) {
        int idx = (H->ev_head - H->ev_pending + (int)H->evs.size()) % (int)H->evs.size();
        EvSet &e = H->evs[idx];
        cudaEventSynchronize(e.ev[8]);
        for (int i = 0; i < 8; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e.ev[i], e.ev[i + 1]);
            H->acc_ms[i] += ms;
        }
        if (e.nf) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e.ev[9], e.ev[10]);
            H->acc_nf_ms += ms;
            H->n_nf++;
            e.nf = false;
        }
        H->n_prof++;
        H->ev_pending--;
    }
}

}  // namespace

int pfmm::ensure_ws(pfmm_handle *H, int nrhs) { return ensure_workspace(H, nrhs); }

// Tensor-core nearfield of op (0: V, 1: K) into fint (zeroed here): splits the FP64 input into
// scaled FP16 hi/lo parts in whi/wlo ([nrhs][E_t][cols] each; per-rhs scale from max |x| in
// wmax), encodes their TMA views and launches.
int pfmm::nf_tc_planes(const pfmm_handle *H, int op, int nrhs)
{
    const int cols = op == 0 ? H->colsV_u : H->colsK_u, nint = H->Et / 2;
    return nf_tc_ksplit(nrhs * H->ntiles128 * ((nint + 127) / 128), cols / 64, H->nsm);
}

int pfmm::run_nf_tc(pfmm_handle *H, int op, const double *x, int nrhs, void *whi, void *wlo,
                    unsigned long long *wmax, double *fint, double *part, cudaStream_t st)
{
    int rc;
    const int cols = op == 0 ? H->colsV_u : H->colsK_u;
    launch_split_input(x, op == 0 ? H->d_perm : nullptr, op == 0 ? H->nt : H->nv, cols, nrhs, H->Et, whi, wlo, wmax,
                       st);
    const int nint = H->Et / 2;
    uint64_t dims[4] = {(uint64_t)cols, 2, (uint64_t)nint, (uint64_t)nrhs};
    uint64_t str[3] = {(uint64_t)cols * 2, (uint64_t)cols * 4, (uint64_t)cols * 4 * nint};
    uint32_t box[4] = {64, 1, 128, 1};
    CUtensorMap mWhi, mWlo;
    if ((rc = encode_map(&mWhi, whi, 4, dims, str, box)) || (rc = encode_map(&mWlo, wlo, 4, dims, str, box))) return rc;
    NfTcParams P{};
    P.panels = H->d_panels;
    P.tiles = H->d_tiles128;
    P.ntiles = H->ntiles128;
    P.nib = (nint + 127) / 128;
    P.nkb = cols / 64;
    const int tiles = nrhs * P.ntiles * P.nib;
    // split K into a few chunks for SM balance (each chunk accumulates 32-stage sub-chunks into its
    // own FP64 partial plane; the planes are summed in order afterwards)
    const int ks = nf_tc_ksplit(tiles, P.nkb, H->nsm);
    P.ksplit = ks;
    P.nitems = tiles * ks;
    P.cols_pad = cols;
    P.kop = op;
    P.nint = nint;
    P.Et = H->Et;
    P.nt = H->nt;
    P.a_exp = op == 0 ? H->a_expV : H->a_expK;
    P.wmax = wmax;
    P.part = part;
    P.nrhs = nrhs;
    P.err = H->d_err;
    if (H->cur_ev) cudaEventRecord(H->cur_ev->ev[9], st);
    if (launch_nf_apply_tc(op == 0 ? H->mapAVhi : H->mapAKhi, op == 0 ? H->mapAVlo : H->mapAKlo, mWhi, mWlo, P, H->nsm,
                           st))
        return fail(PFMM_ERR_CUDA, std::string("tensor-core nearfield launch: ") + cudaGetErrorString(cudaGetLastError()));
    if (H->cur_ev) {
        cudaEventRecord(H->cur_ev->ev[10], st);
        H->cur_ev->nf = true;
    }
    launch_nf_tc_reduce(part, ks, (size_t)nrhs * H->Et * H->nt, fint, st);
    return PFMM_OK;
}

// FP64 exact nearfield: residues of x, the residue products on the tensor cores, their FP64
// combination into fint (every element written)
int pfmm::run_nf_crt(pfmm_handle *H, int op, const double *x, int nrhs, double *fint, cudaStream_t st)
{
    int rc;
    const int cols = op == 0 ? H->colsV_u : H->colsK_u, b = op == 0 ? H->crt_bV : H->crt_bK;
    launch_crt_split_input(x, op == 0 ? H->d_perm : nullptr, op == 0 ? H->nt : H->nv, cols, nrhs, H->Et, b, H->d_Wres,
                           H->d_wmax, st);
    const int nint = H->Et / 2;
    uint64_t dims[5] = {(uint64_t)cols, 2, (uint64_t)nint, (uint64_t)nrhs, (uint64_t)kCrtModuli};
    uint64_t str[4] = {(uint64_t)cols * 2, (uint64_t)cols * 4, (uint64_t)cols * 4 * nint,
                       (uint64_t)cols * 4 * nint * nrhs};
    uint32_t box[5] = {64, 1, 128, 1, 1};
    CUtensorMap mW;
    if ((rc = encode_map(&mW, H->d_Wres, 5, dims, str, box))) return rc;
    NfCrtParams P{};
    P.panels = H->d_panels;
    P.tiles = H->d_tiles128;
    P.ntiles = H->ntiles128;
    P.nib = (nint + 127) / 128;
    P.nkb = cols / 64;
    P.nrhs = nrhs;
    P.nitems = (kCrtModuli / 2) * nrhs * P.ntiles * P.nib;
    P.cols_pad = cols;
    P.kop = op;
    P.nint = nint;
    P.Et = H->Et;
    P.nt = H->nt;
    P.res = H->d_res8;
    P.err = H->d_err;
    if (H->cur_ev) cudaEventRecord(H->cur_ev->ev[9], st);
    if (launch_nf_apply_crt(op == 0 ? H->mapAVres : H->mapAKres, mW, P, H->nsm, st, H->crt_form))
        return fail(PFMM_ERR_CUDA, std::string("FP64 tensor-core nearfield launch: ") +
                                       cudaGetErrorString(cudaGetLastError()));
    if (H->cur_ev) {
        cudaEventRecord(H->cur_ev->ev[10], st);
        H->cur_ev->nf = true;
    }
    launch_crt_combine(H->d_res8, nrhs, H->Et, H->nt, op == 0 ? H->d_rexpV : H->d_rexpK, H->d_wmax, b, fint, st);
    return PFMM_OK;
}

int pfmm::run_nf_otf(pfmm_handle *H, int op, const void *xin, int ncolg, int Et, int ls, int nrhs, int ndmax,
                     double *fint, cudaStream_t st)
{
    OtfArgs a{};
    a.q = H->quad;
    a.panels = H->d_panels;
    a.tiles = H->d_tiles;
    a.ntiles = H->ntiles;
    a.tile_sing = H->d_tile_sing;
    a.sing = H->d_sing;
    a.singV = H->d_singV;
    a.singK = H->d_singK;
    a.x = xin;
    a.ncolg = ncolg;
    a.Et = Et;
    a.ls = ls;
    a.nrhs = nrhs;
    a.ndmax = ndmax;
    a.f = fint;
    a.nt = H->nt;
    launch_nf_otf(H->mixed, op == 1, a, H->nsm, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, std::string("on-the-fly nearfield: ") + cudaGetErrorString(e));
    return PFMM_OK;
}

// f_b = A_0 x_b for ns independent slices b (user triangle order, [ns][E_x] FP64): the stored
// nearfield block of offset d = 0 (same time step, neighbouring leaf boxes), applied with each
// slice taken as its own step.  xint: ns E_x elements of the arithmetic type, fint: ns E_x doubles.
int pfmm::apply_same_step(pfmm_handle *H, const double *x, double *f, int ns, void *xint, double *fint, cudaStream_t st)
{
    ApplyGeo g{};
    g.nt = H->nt;
    g.nv = H->nv;
    g.Et = ns;
    g.ls = 1;
    g.perm = H->d_perm;
    g.nsm = H->nsm;
    g.m2l_force = H->m2l_force;
    launch_permute_in(x, xint, H->mixed, 1, g, st);
    if (H->otf) {
        cudaMemsetAsync(fint, 0, sizeof(double) * ns * (size_t)H->nt, st);
        int rc = pfmm::run_nf_otf(H, 0, xint, H->nt, ns, 1, 1, 1, fint, st);
        if (rc) return rc;
    } else {
        NfHalfSplit hs;
        launch_nf_apply(H->mixed, false, H->nf_blocks(0), H->d_colV, H->d_tiles, H->ntiles, H->d_panels, xint, H->nt, 1, g,
                        fint, st, 1, H->nf_split(0, &hs));
    }
    launch_permute_out(fint, f, 1, g, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, std::string("same-step apply: ") + cudaGetErrorString(e));
    return PFMM_OK;
}

extern "C" {

const char *pfmm_last_error(void) { return g_err.c_str(); }

int pfmm_default_params(pfmm_params *p)
{
    if (!p) return fail(PFMM_ERR_INVALID_ARG, "params is NULL");
    p->m_t = 4;
    p->m_x = 4;
    p->c_st = 1.0;
    p->n_tr = -1;
    p->eps_tr = 1e-12;
    p->leaf_steps = 2;
    p->leaf_tris = 16;
    p->precision = PFMM_FP64;
    p->nearfield = PFMM_NEARFIELD_STORED;
    p->quad_regular = 3;
    p->quad_singular = 6;
    p->nf_engine = PFMM_NF_AUTO;
    p->fp64_native = 0;
    p->nf_form = 0;
    return PFMM_OK;
}

// The faster of the two forms of the FP64 tensor-core nearfield (one row tile and two moduli per
// work item, or two row tiles sharing each input stage), timed with CUDA events on this handle's
// V product of a zero input (the work does not depend on the values).
static int tune_crt_form(pfmm_handle *H, cudaStream_t st)
{
    int rc = ensure_workspace(H, 1);
    if (rc) return rc;
    double *x = nullptr;
    if ((rc = H->alloc(&x, (size_t)H->Et * H->nt))) return rc;
    CK(cudaMemsetAsync(x, 0, sizeof(double) * H->Et * H->nt, st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // one warm-up run of each form, then the forms alternate and each keeps its fastest of four
    // runs (alternating and taking minima keeps clock ramps and other users' work from deciding)
    float best_ms[2] = {1e30f, 1e30f};
    for (int form = 1; form <= 2 && !rc; ++form) {
        H->crt_form = form;
        rc = pfmm::run_nf_crt(H, 0, x, 1, H->d_fint, st);
    }
    for (int rep = 0; rep < 4 && !rc; ++rep)
        for (int form = 1; form <= 2 && !rc; ++form) {
            H->crt_form = form;
            cudaEventRecord(e0, st);
            rc = pfmm::run_nf_crt(H, 0, x, 1, H->d_fint, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms[form - 1] = std::min(best_ms[form - 1], ms);
        }
    if (!rc) {
        H->crt_form_ms[0] = best_ms[0];
        H->crt_form_ms[1] = best_ms[1];
        H->crt_best_form = best_ms[1] < best_ms[0] ? 2 : 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    H->crt_form = H->crt_best_form;
    H->release(x);
    if (rc) return rc;
    CK(cudaGetLastError());
    return PFMM_OK;
}

// FP64 mode on panels that span all columns: per-row exponents and the residues of the scaled,
// rounded panels for the exact tensor-core nearfield.  Skipped (CUDA-core FP64 engine kept) when
// the residues (32 bytes per stored element) would not leave room on the device.
static int build_crt(pfmm_handle *H, const Tree &t, bool fullV, bool fullK, cudaStream_t st)
{
    using namespace pfmm;
    if (crt_upload_constants(st)) return fail(PFMM_ERR_CUDA, "CRT constants upload failed");
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const size_t need = (fullV ? (size_t)t.sizeV : 0) * 2 * kCrtModuli + (fullK ? (size_t)t.sizeK : 0) * 2 * kCrtModuli;
    if (need > free_b / 10 * 7) return PFMM_OK;
    const int nd = H->nd, npanel = (int)t.panels.size();
    unsigned long long *rowmax = nullptr;
    int rc;
    if ((rc = H->alloc(&rowmax, (size_t)H->nt))) return rc;
    for (int op = 0; op < 2; ++op) {
        if (!(op == 0 ? fullV : fullK)) continue;
        const int cols = op == 0 ? t.panels[0].colsV_pad : t.panels[0].colsK_pad;
        const size_t n = op == 0 ? (size_t)t.sizeV : (size_t)t.sizeK;
        const int b = crt_bits(4ll * cols);
        int *rexp = nullptr, *rexpR = nullptr;
        uint16_t *res = nullptr;
        if ((rc = H->alloc(&rexp, (size_t)H->nt)) || (rc = H->alloc(&rexpR, n / cols)) ||
            (rc = H->alloc(&res, n * kCrtModuli)))
            return rc;
        const double *A = (const double *)(op == 0 ? H->d_AV : H->d_AK);
        launch_crt_row_exps(A, H->d_panels, npanel, op, nd, cols, b, rowmax, H->nt, rexp, rexpR, st);
        launch_crt_split_panel(A, rexpR, n, cols, res, st);
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        H->release(rexpR);
        // [modulus][block][64 rows][64 columns]
        uint64_t dims[4] = {64, 64, (uint64_t)(n / 4096), (uint64_t)kCrtModuli}, str[3] = {128, 8192, (n / 4096) * 8192};
        uint32_t box[4] = {64, 64, 1, 1};
        if (op == 0) {
            H->colsV_u = cols;
            H->crt_bV = b;
            H->d_AVres = res;
            H->d_rexpV = rexp;
            if ((rc = encode_map(&H->mapAVres, res, 4, dims, str, box))) return rc;
            H->crtV = true;
        } else {
            H->colsK_u = cols;
            H->crt_bK = b;
            H->d_AKres = res;
            H->d_rexpK = rexp;
            if ((rc = encode_map(&H->mapAKres, res, 4, dims, str, box))) return rc;
            H->crtK = true;
        }
    }
    H->release(rowmax);
    return PFMM_OK;
}

static int build_impl(const pfmm_mesh *mesh, const pfmm_params *prm, cudaStream_t st, pfmm_handle *H)
{
    H->nv = mesh->n_vertices;
    H->nt = mesh->n_triangles;
    H->Et = mesh->n_steps;
    H->T = mesh->T;
    H->alpha = mesh->alpha;
    H->h = mesh->T / mesh->n_steps;
    H->prm = *prm;
    if (prm->precision != PFMM_FP64 && prm->precision != PFMM_MIXED)
        return fail(PFMM_ERR_INVALID_ARG, "precision must be PFMM_FP64 or PFMM_MIXED");
    if (prm->nearfield != PFMM_NEARFIELD_STORED && prm->nearfield != PFMM_NEARFIELD_ONTHEFLY)
        return fail(PFMM_ERR_INVALID_ARG, "unknown nearfield mode");
    if (prm->nearfield == PFMM_NEARFIELD_ONTHEFLY && 2 * prm->leaf_steps > 8)
        return fail(PFMM_ERR_UNSUPPORTED, "the on-the-fly nearfield supports leaf_steps <= 4");
    H->mixed = prm->precision == PFMM_MIXED;
    H->es = H->mixed ? 4 : 8;
    H->fprec = H->mixed ? 1 : (prm->fp64_native ? 0 : 2);
    std::string err;
    int rc = build_tree(*mesh, *prm, H->tree, err);
    if (rc) return fail(rc, err);
    Tree &t = H->tree;
    H->ls = prm->leaf_steps;
    H->nd = 2 * H->ls;
    if (H->nd > 8) return fail(PFMM_ERR_UNSUPPORTED, "leaf_steps > 4 is not supported");
    H->na = prm->m_t + 1;
    H->mx = prm->m_x;
    H->p = t.p;
    const int mx = H->mx, m1 = mx + 1, na = H->na;
    // graded multi-indices: all kappa with |kappa| = s, for s = 0 .. m_x
    std::vector<int> kidx, kinv((size_t)m1 * m1 * m1, -1);
    for (int s = 0; s <= mx; ++s)
        for (int a = s; a >= 0; --a)
            for (int b = s - a; b >= 0; --b) {
                int c = s - a - b;
                kinv[((size_t)a * m1 + b) * m1 + c] = (int)kidx.size() / 3;
                kidx.push_back(a);
                kidx.push_back(b);
                kidx.push_back(c);
            }
    H->nk = (int)kidx.size() / 3;
    std::vector<int> eoff(H->nk);
    H->ne = 0;
    for (int t_ = 0; t_ < H->nk; ++t_) {
        eoff[t_] = H->ne;
        H->ne += mx - (kidx[3 * t_] + kidx[3 * t_ + 1] + kidx[3 * t_ + 2]) + 1;
    }
    if (H->ls * H->nk > 2048) return fail(PFMM_ERR_UNSUPPORTED, "leaf_steps * C(m_x+3,3) > 2048");
    if (H->na * H->nk > 4096) return fail(PFMM_ERR_UNSUPPORTED, "(m_t+1) * C(m_x+3,3) > 4096");

    // ---- geometry in internal order
    const int nt = H->nt, nv = H->nv, p = t.p;
    std::vector<double> verts(mesh->vertices, mesh->vertices + 3 * (size_t)nv);
    std::vector<int> tri_user(mesh->triangles, mesh->triangles + 3 * (size_t)nt), tri_int(3 * (size_t)nt);
    std::vector<double> area(nt);
    for (int i = 0; i < nt; ++i)
        for (int v = 0; v < 3; ++v) tri_int[3 * i + v] = tri_user[3 * t.perm[i] + v];
    for (int x = 0; x < nt; ++x) {
        const double *A = &verts[3 * tri_user[3 * x]], *B = &verts[3 * tri_user[3 * x + 1]], *C = &verts[3 * tri_user[3 * x + 2]];
        double a[3], b[3];
        for (int c = 0; c < 3; ++c) { a[c] = B[c] - A[c]; b[c] = C[c] - A[c]; }
        double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
        area[x] = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    if ((rc = upload(H, &H->d_verts, verts, st)) || (rc = upload(H, &H->d_tri_int, tri_int, st)) ||
        (rc = upload(H, &H->d_tri_user, tri_user, st)) || (rc = upload(H, &H->d_area, area, st)) ||
        (rc = upload(H, &H->d_perm, t.perm, st)) || (rc = upload(H, &H->d_tri_leaf, t.tri_leaf, st)) ||
        (rc = upload(H, &H->d_leaf_start, t.leaf_start, st)) || (rc = upload(H, &H->d_leaf_grid, t.lv[p].grid, st)) ||
        (rc = upload(H, &H->d_kidx, kidx, st)) || (rc = upload(H, &H->d_kinv, kinv, st)) ||
        (rc = upload(H, &H->d_eoff, eoff, st)))
        return rc;

    // ---- S2M / L2T tables (Eq. s2m, l2t)
    {
        std::vector<double> rule = collapsed_rule(mx / 2 + 2);
        double *rule_d = nullptr, *Sx = nullptr, *SK = nullptr;
        if ((rc = upload(H, &rule_d, rule, st)) || (rc = H->alloc(&Sx, (size_t)nt * H->nk)) ||
            (rc = H->alloc(&SK, (size_t)nt * 3 * H->nk)))
            return rc;
        SetupArgs a{};
        a.verts = H->d_verts;
        a.tri = H->d_tri_int;
        a.tri_leaf = H->d_tri_leaf;
        a.leaf_grid = H->d_leaf_grid;
        for (int c = 0; c < 3; ++c) a.corner[c] = t.corner[c];
        a.hx_leaf = t.lv[p].hx;
        a.hxp_leaf = t.lv[p].hxp;
        a.alpha = H->alpha;
        a.nt = nt;
        a.mx = mx;
        a.nk = H->nk;
        a.kidx = H->d_kidx;
        a.rule_tab = rule_d;
        a.nq_tab = (mx / 2 + 2) * (mx / 2 + 2);
        a.Sx = Sx;
        a.SK = SK;
        launch_space_tables(a, st);
        CK(cudaGetLastError());
        if ((rc = device_to_R(H, &H->d_Sx, Sx, (size_t)nt * H->nk, st)) ||
            (rc = device_to_R(H, &H->d_SK, SK, (size_t)nt * 3 * H->nk, st)))
            return rc;
        // St[s][a] = int over step s of a leaf interval of L_{J,a} (exact Gauss-Legendre)
        std::vector<double> gx, gw, St((size_t)H->ls * na), qt(2 * (size_t)na * na);
        gauss01(na, gx, gw);
        double Lleaf = H->ls * H->h;
        for (int s = 0; s < H->ls; ++s)
            for (int aa = 0; aa < na; ++aa) {
                double v = 0.0;
                for (int i = 0; i < na; ++i) v += gw[i] * H->h * lagrange(aa, prm->m_t, 0.0, Lleaf, (s + gx[i]) * H->h);
                St[s * na + aa] = v;
            }
        // q^(t)[c][ac][ap] = L_{I_p,ap}(xi_{I_c,ac})  (Eq. temp_m2m)
        for (int c = 0; c < 2; ++c)
            for (int ac = 0; ac < na; ++ac)
                for (int ap = 0; ap < na; ++ap) {
                    double clo = c == 0 ? -1.0 : 0.0, chi = c == 0 ? 0.0 : 1.0;
                    double xc = 0.5 * (clo + chi) + 0.5 * (chi - clo) * cheb_node(ac, prm->m_t);
                    qt[(c * na + ac) * na + ap] = lagrange(ap, prm->m_t, -1.0, 1.0, xc);
                }
        if ((rc = upload_R(H, &H->d_St, St, st)) || (rc = upload_R(H, &H->d_qt, qt, st))) return rc;
    }

    // ---- levels: lists, q^(x) (Eq. st_m2m) and E tables (Eq. exp_coeffs_3d / 1d)
    H->dl.assign(p + 1, DevLevel{});
    H->mom_per_rhs = 0;
    for (int l = 0; l <= p; ++l) {
        const Level &L = t.lv[l];
        DevLevel &D = H->dl[l];
        D.G = L.G;
        D.nint = L.nint;
        D.nbox = L.nbox;
        D.st = L.st ? 1 : 0;
        D.hxp = L.hxp;
        D.mom_off = H->mom_per_rhs;
        if (l >= 2) H->mom_per_rhs += (int64_t)L.nint * L.nbox * na * H->nk;
        if ((rc = upload(H, &D.grid, L.grid, st))) return rc;
        if (l > 0 && ((rc = upload(H, &D.parent, L.parent, st)) || (rc = upload(H, &D.octant, L.octant, st)))) return rc;
        if (l < p && ((rc = upload(H, &D.ch_ptr, L.ch_ptr, st)) || (rc = upload(H, &D.ch_idx, L.ch_idx, st)))) return rc;
        if (l >= 2 && ((rc = upload(H, &D.m2l_ptr, L.m2l_ptr, st)) || (rc = upload(H, &D.m2l_src, L.m2l_src, st)) ||
                       (rc = upload(H, &D.m2l_off, L.m2l_off, st))))
            return rc;
        if (l > 0 && L.st) {
            // q^(x)_{kap,nu}(X_c, X_p) per direction for a child in the lower (bit 0) or upper half
            const Level &P = t.lv[l - 1];
            std::vector<double> q1(2 * (size_t)m1 * m1);
            for (int bit = 0; bit < 2; ++bit) {
                double dc = (2.0 * bit - 1.0) * L.hx;  // child centre - parent centre
                for (int ka = 0; ka <= mx; ++ka)
                    for (int nu = 0; nu <= mx; ++nu) {
                        double s = 0.0;
                        for (int n = 0; n <= mx; ++n) {
                            double xn = cheb_node(n, mx);
                            s += cheb_T(nu, (dc + L.hxp * xn) / P.hxp) * cheb_T(ka, xn);
                        }
                        q1[(bit * m1 + ka) * m1 + nu] = (ka == 0 ? 1.0 : 2.0) / (mx + 1.0) * s;
                    }
            }
            if ((rc = upload_R(H, &D.qx, q1, st))) return rc;
        }
        if (l >= 2) {
            // separable M2L: dense cell map and the interval pairs of Eq. 03:ILtemp
            std::vector<int> cellbox((size_t)L.G * L.G * L.G, -1), boxcell(L.nbox), pk, pJ;
            for (int b = 0; b < L.nbox; ++b) {
                int c = (L.grid[3 * b] * L.G + L.grid[3 * b + 1]) * L.G + L.grid[3 * b + 2];
                cellbox[c] = b;
                boxcell[b] = c;
            }
            D.kptr_host.assign(L.nint + 1, 0);
            for (int k = 0; k < L.nint; ++k) {
                if (k >= 2) {
                    if (k % 2 == 0) { pk.push_back(k); pJ.push_back(k - 2); }
                    else { pk.push_back(k); pJ.push_back(k - 3); pk.push_back(k); pJ.push_back(k - 2); }
                }
                D.kptr_host[k + 1] = (int)pk.size();
            }
            D.ntr = std::min(L.ntr, L.G - 1);
            if ((rc = upload(H, &D.cellbox, cellbox, st)) || (rc = upload(H, &D.boxcell, boxcell, st)) ||
                (rc = upload(H, &D.pk, pk, st)) || (rc = upload(H, &D.pJ, pJ, st)) ||
                (rc = upload(H, &D.kptr, D.kptr_host, st)))
                return rc;
            H->m2l_ws_need = std::max<int64_t>(H->m2l_ws_need, (int64_t)pk.size() * na * na * L.G * L.G * L.G * H->ne);
            size_t ne = 2 * (size_t)na * na * (2 * L.G - 1) * m1 * m1;
            double *E1 = nullptr, *pref = nullptr;
            if ((rc = H->alloc(&E1, ne)) || (rc = H->alloc(&pref, 2 * (size_t)na * na))) return rc;
            launch_e1_table(na, prm->m_t, mx, L.G, L.hx, L.hxp, L.ht, H->alpha, E1, pref, st);
            CK(cudaGetLastError());
            if ((rc = device_to_R(H, &D.E1, E1, ne, st)) || (rc = device_to_R(H, &D.pref, pref, 2 * (size_t)na * na, st)))
                return rc;
        }
    }

    // ---- nearfield blocks (Eq. eval_sl_nf_block)
    {
        std::vector<PanelGPU> pg(t.panels.size());
        std::vector<int> tiles, box_tiles(t.panels.size() + 1, 0);  // panel i = leaf box i
        for (size_t i = 0; i < t.panels.size(); ++i) {
            const Panel &P = t.panels[i];
            box_tiles[i] = (int)tiles.size() / 2;
            pg[i] = PanelGPU{(int)i, P.row0, P.nrows, P.rows_pad, P.ncolV, P.colsV_pad, P.ncolK, P.colsK_pad,
                             (long long)P.offV, (long long)P.offK, P.colV_at, P.colK_at};
            for (int r0 = 0; r0 < P.nrows; r0 += kRowTile) {
                tiles.push_back((int)i);
                tiles.push_back(r0);
            }
        }
        H->ntiles = (int)tiles.size() / 2;
        box_tiles[t.panels.size()] = H->ntiles;
        std::vector<int> sing(12 * t.sing.size(), 0);
        for (size_t i = 0; i < t.sing.size(); ++i) {
            const SingularPair &s = t.sing[i];
            int *o = &sing[12 * i];
            o[0] = s.x; o[1] = s.y; o[2] = s.panel; o[3] = s.row; o[4] = s.colV; o[5] = s.code;
            o[6] = s.colK[0]; o[7] = s.colK[1]; o[8] = s.colK[2];
        }
        int *d_sing = nullptr;
        H->otf = prm->nearfield == PFMM_NEARFIELD_ONTHEFLY;
        if ((rc = upload(H, &H->d_panels, pg, st)) || (rc = upload(H, &H->d_tiles, tiles, st)) ||
            (rc = upload(H, &H->d_box_tiles, box_tiles, st)) ||
            (rc = upload(H, &H->d_colV, t.colV, st)) || (rc = upload(H, &d_sing, sing, st)))
            return rc;
        if (!H->otf) {
            if ((rc = upload(H, &H->d_colK, t.colK, st)) || (rc = upload(H, &H->d_kmap, t.kmap, st))) return rc;
            if ((rc = H->alloc((char **)&H->d_AV, (size_t)t.sizeV * H->es, 1)) ||
                (rc = H->alloc((char **)&H->d_AK, (size_t)t.sizeK * H->es, 1)))
                return rc;
            CK(cudaMemsetAsync(H->d_AV, 0, (size_t)t.sizeV * H->es, st));
            CK(cudaMemsetAsync(H->d_AK, 0, (size_t)t.sizeK * H->es, st));
        } else {
            // singular pairs grouped by 64-row tile (the list is ordered by panel, then row)
            std::vector<int> tile_base(t.panels.size() + 1, 0), tsing(H->ntiles + 1, 0);
            for (size_t i = 0; i < t.panels.size(); ++i)
                tile_base[i + 1] = tile_base[i] + (t.panels[i].nrows + kRowTile - 1) / kRowTile;
            for (size_t i = 0; i < t.sing.size(); ++i) {
                const SingularPair &sp = t.sing[i];
                const int tile = tile_base[sp.panel] + sp.row / kRowTile;
                if (i > 0) {
                    const SingularPair &q = t.sing[i - 1];
                    if (tile < tile_base[q.panel] + q.row / kRowTile)
                        return fail(PFMM_ERR_UNSUPPORTED, "singular pairs are not ordered by tile");
                }
                tsing[tile + 1]++;
            }
            for (int i = 0; i < H->ntiles; ++i) tsing[i + 1] += tsing[i];
            if ((rc = upload(H, &H->d_tile_sing, tsing, st)) ||
                (rc = H->alloc(&H->d_singV, 2 * std::max<size_t>(t.sing.size(), 1))) ||
                (rc = H->alloc(&H->d_singK, 6 * std::max<size_t>(t.sing.size(), 1))))
                return rc;
            H->d_sing = d_sing;
            H->otf_bytes = (int64_t)t.sing.size() * (12 * 4 + 8 * 8) + (int64_t)(H->ntiles + 1) * 4;
        }
        std::vector<double> rreg = collapsed_rule(prm->quad_regular), gx, gw;
        gauss01(prm->quad_singular, gx, gw);
        std::vector<double> gls(gx);
        gls.insert(gls.end(), gw.begin(), gw.end());
        double *d_rreg = nullptr, *d_gls = nullptr;
        if ((rc = upload(H, &d_rreg, rreg, st)) || (rc = upload(H, &d_gls, gls, st))) return rc;
        H->d_rule_reg = d_rreg;
        H->nq_reg = prm->quad_regular * prm->quad_regular;
        NfQuadArgs a{};
        a.verts = H->d_verts;
        a.tri = H->d_tri_int;
        a.nv = nv;
        a.nd = H->nd;
        a.h = H->h;
        a.alpha = H->alpha;
        a.rule_reg = d_rreg;
        a.nq_reg = prm->quad_regular * prm->quad_regular;
        a.gl_sing = d_gls;
        a.nq_sing = prm->quad_singular;
        a.colV = H->d_colV;
        a.kmap = H->d_kmap;
        if (H->otf) {
            H->quad = a;
            launch_nf_singular(a, d_sing, (int)t.sing.size(), H->d_panels, nullptr, nullptr, H->mixed, st, H->d_singV,
                               H->d_singK);
        } else {
            for (size_t i = 0; i < t.panels.size(); ++i) {
                launch_nf_regular(a, pg[i], H->d_AV, H->d_AK, H->mixed, st);
                CK(cudaGetLastError());
            }
            launch_nf_singular(a, d_sing, (int)t.sing.size(), H->d_panels, H->d_AV, H->d_AK, H->mixed, st);
        }
        CK(cudaGetLastError());

        // tensor-core nearfield: mixed mode, two steps per leaf, every panel spans all columns
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&H->nsm, cudaDevAttrMultiProcessorCount, dev));
        int cc_major = 0, cc_minor = 0;
        CK(cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev));
        CK(cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
        // tensor cores for the stored panels when every panel spans all columns: the FP16 split
        // (mixed mode) or the exact residue arithmetic (FP64 mode)
        bool eligible = !H->otf && H->ls == 2 && prm->nf_engine == PFMM_NF_AUTO && cc_major == 10 && encode_fn() &&
                        (H->mixed || !prm->fp64_native);
        bool fullV = eligible, fullK = eligible;
        for (const Panel &P : t.panels) {
            fullV = fullV && P.ncolV == nt && P.colsV_pad == t.panels[0].colsV_pad;
            fullK = fullK && P.ncolK == nv && P.colsK_pad == t.panels[0].colsK_pad;
        }
        // every panel's column k is triangle (node) k or a hole: one column space for all panels
        for (const Panel &P : t.panels) {
            for (int k = 0; fullV && k < nt; ++k) fullV = t.colV[P.colV_at + k] == k || t.colV[P.colV_at + k] == -1;
            for (int k = 0; fullK && k < nv; ++k) fullK = t.colK[P.colK_at + k] == k;
        }
        CK(cudaMalloc((void **)&H->d_err, sizeof(int)));
        H->allocs.push_back(H->d_err);
        CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), st));
        if (fullV || fullK) {
            std::vector<int> t128;
            for (size_t i = 0; i < t.panels.size(); ++i)
                for (int r0 = 0; r0 < t.panels[i].nrows; r0 += 128) {
                    t128.push_back((int)i);
                    t128.push_back(r0);
                }
            H->ntiles128 = (int)t128.size() / 2;
            if ((rc = upload(H, &H->d_tiles128, t128, st))) return rc;
        }
        if (!H->mixed && (fullV || fullK)) {
            if ((rc = build_crt(H, t, fullV, fullK, st))) return rc;
            fullV = fullK = false;
        }
        if (fullV) {
            H->colsV_u = t.panels[0].colsV_pad;
            size_t n = (size_t)t.sizeV;
            if ((rc = H->alloc(&H->d_AVhi, n)) || (rc = H->alloc(&H->d_AVlo, n))) return rc;
            H->a_expV = panel_scale_exp((const float *)H->d_AV, n, (unsigned *)H->d_err, st);
            if (H->a_expV == INT32_MIN) return fail(PFMM_ERR_CUDA, "panel scale");
            CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), st));
            launch_split_panel((const float *)H->d_AV, H->d_AVhi, H->d_AVlo, n, H->colsV_u, H->a_expV, st);
            CK(cudaStreamSynchronize(st));
            H->release(H->d_AV);  // hi + lo represent it; the CUDA-core path reads their sum
            H->d_AV = nullptr;
            // [block][64 rows][64 columns] view of the 64 x 64 blocks (n is a multiple of 4096)
            uint64_t dims[3] = {64, 64, (uint64_t)(n / 4096)}, str[2] = {128, 8192};
            uint32_t box[3] = {64, 64, 1};
            if ((rc = encode_map(&H->mapAVhi, H->d_AVhi, 3, dims, str, box)) ||
                (rc = encode_map(&H->mapAVlo, H->d_AVlo, 3, dims, str, box)))
                return rc;
            H->tcV = true;
        }
        if (fullK) {
            H->colsK_u = t.panels[0].colsK_pad;
            size_t n = (size_t)t.sizeK;
            if ((rc = H->alloc(&H->d_AKhi, n)) || (rc = H->alloc(&H->d_AKlo, n))) return rc;
            H->a_expK = panel_scale_exp((const float *)H->d_AK, n, (unsigned *)H->d_err, st);
            if (H->a_expK == INT32_MIN) return fail(PFMM_ERR_CUDA, "panel scale");
            CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), st));
            launch_split_panel((const float *)H->d_AK, H->d_AKhi, H->d_AKlo, n, H->colsK_u, H->a_expK, st);
            CK(cudaStreamSynchronize(st));
            H->release(H->d_AK);
            H->d_AK = nullptr;
            uint64_t dims[3] = {64, 64, (uint64_t)(n / 4096)}, str[2] = {128, 8192};
            uint32_t box[3] = {64, 64, 1};
            if ((rc = encode_map(&H->mapAKhi, H->d_AKhi, 3, dims, str, box)) ||
                (rc = encode_map(&H->mapAKlo, H->d_AKlo, 3, dims, str, box)))
                return rc;
            H->tcK = true;
        }
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(st));
    if (H->crtV && (prm->nf_form == 1 || prm->nf_form == 2)) H->crt_form = prm->nf_form;
    else if (H->crtV && (rc = tune_crt_form(H, st))) return rc;
    return PFMM_OK;
}

int pfmm_build_trees(const pfmm_mesh *mesh, const pfmm_params *params, void *stream, pfmm_handle **out)
{
    if (!mesh || !params || !out) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    pfmm_handle *H = new (std::nothrow) pfmm_handle();
    if (!H) return fail(PFMM_ERR_OOM, "host allocation failed");
    int rc;
    try {
        rc = build_impl(mesh, params, (cudaStream_t)stream, H);
    } catch (const std::bad_alloc &) {
        rc = fail(PFMM_ERR_OOM, "host allocation failed");
    } catch (...) {
        rc = fail(PFMM_ERR_CUDA, "unexpected exception during build");
    }
    if (rc) {
        delete H;
        return rc;
    }
    *out = H;
    return PFMM_OK;
}

static int apply_impl(pfmm_handle *H, int op, const double *x, double *f, int nrhs, int parts, cudaStream_t st)
{
    if (!H || !x || !f || nrhs < 1 || (op != 0 && op != 1) || parts < 1 || parts > 3)
        return fail(PFMM_ERR_INVALID_ARG, "invalid apply arguments");
    int rc = ensure_workspace(H, nrhs);
    if (rc) return rc;
    const Tree &t = H->tree;
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
    g.nbox_leaf = t.lv[H->p].nbox;
    g.kidx = H->d_kidx;
    g.kinv = H->d_kinv;
    g.ne = H->ne;
    g.eoff = H->d_eoff;
    g.nsm = H->nsm;
    g.m2l_force = H->m2l_force;
    if ((int)t.panels.size() == g.nbox_leaf) {  // one row panel per leaf box: its 64-row tiles
        g.tiles = H->d_tiles;
        g.ntiles = H->ntiles;
        g.box_tiles = H->d_box_tiles;
    }
    EvSet *ev = nullptr;
    if (H->prof) {
        if (H->evs.empty()) {
            H->evs.resize(256);
            for (auto &e : H->evs)
                for (int i = 0; i < 11; ++i) CK(cudaEventCreate(&e.ev[i]));
        }
        if (H->ev_pending == (int)H->evs.size()) prof_collect(H, H->ev_pending - 1);
        ev = &H->evs[H->ev_head];
        ev->nf = false;
        H->ev_head = (H->ev_head + 1) % (int)H->evs.size();
        H->ev_pending++;
    }
    H->cur_ev = ev;
    struct CurEvReset {
        pfmm_handle *H;
        ~CurEvReset() { H->cur_ev = nullptr; }
    } cur_ev_reset{H};
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev->ev[i], st);
    };
    mark(0);
    const void *xin;  // input in the arithmetic type, and its column count
    int ncolg;
    if (op == 0) {
        launch_permute_in(x, H->d_xint, H->mixed, nrhs, g, st);
        xin = H->d_xint;
        ncolg = H->nt;
    } else if (H->mixed) {
        launch_cast_to_float(x, (float *)H->d_gf, (size_t)nrhs * H->Et * H->nv, st);
        xin = H->d_gf;
        ncolg = H->nv;
    } else {
        xin = x;
        ncolg = H->nv;
    }
    mark(1);
    const bool tc = (parts & PFMM_PART_NEAR) && (op == 0 ? H->tcV : H->tcK) && !H->nf_cuda_cores;
    const bool crt = (parts & PFMM_PART_NEAR) && (op == 0 ? H->crtV : H->crtK) && !H->nf_cuda_cores;
    if (tc) {
        if ((rc = pfmm::run_nf_tc(H, op, x, nrhs, H->d_Whi, H->d_Wlo, H->d_wmax, H->d_fint, H->d_nfpart, st)))
            return rc;
    } else if (crt) {
        if ((rc = pfmm::run_nf_crt(H, op, x, nrhs, H->d_fint, st))) return rc;
    } else if ((parts & PFMM_PART_NEAR) && H->otf) {
        CK(cudaMemsetAsync(H->d_fint, 0, sizeof(double) * nrhs * (size_t)H->Et * H->nt, st));
        if ((rc = pfmm::run_nf_otf(H, op, xin, ncolg, H->Et, H->ls, nrhs, 1 << 30, H->d_fint, st))) return rc;
    } else if (parts & PFMM_PART_NEAR) {
        NfHalfSplit hs;
        launch_nf_apply(H->mixed, op == 1, H->nf_blocks(op), op == 0 ? H->d_colV : H->d_colK, H->d_tiles, H->ntiles,
                        H->d_panels, xin, ncolg, nrhs, g, H->d_fint, st, 1 << 30, H->nf_split(op, &hs));
    } else {
        CK(cudaMemsetAsync(H->d_fint, 0, sizeof(double) * nrhs * (size_t)H->Et * H->nt, st));
    }
    mark(2);
    const int p = H->p;
    bool far = (parts & PFMM_PART_FAR) && p >= 2;
    char *mu = (char *)H->d_mu, *lam = (char *)H->d_lam;
    if (far) {
        launch_s2m(H->fprec, op == 1, xin, ncolg, op == 0 ? H->d_Sx : H->d_SK, H->d_St,
                   mu + H->dl[p].mom_off * H->es * nrhs, nrhs, g, st, H->d_T1, H->ws_m2l);
    }
    mark(3);
    if (far)
        for (int l = p - 1; l >= 2; --l) launch_m2m(H->fprec, H->dl[l], H->dl[l + 1], l, H->d_qt, mu, nrhs, g, 0, st);
    mark(4);
    if (far)
        for (int l = 2; l <= p; ++l)
            if (launch_m2l(H->fprec, H->dl[l], l, mu, lam, nrhs, g, H->d_T1, H->d_T2, H->ws_m2l, st))
                return fail(PFMM_ERR_OOM, "M2L workspace too small for one interval");
    mark(5);
    if (far)
        for (int l = 3; l <= p; ++l) launch_l2l(H->fprec, H->dl[l - 1], H->dl[l], l, H->d_qt, lam, nrhs, g, 0, st);
    mark(6);
    if (far)
        launch_l2t(H->fprec, lam + H->dl[p].mom_off * H->es * nrhs, H->d_Sx, H->d_St, H->d_fint, nrhs, g, 0, st, H->d_T1,
                   H->ws_m2l);
    mark(7);
    launch_permute_out(H->d_fint, f, nrhs, g, st);
    mark(8);
    CK(cudaGetLastError());
    return PFMM_OK;
}

int pfmm_apply_parts(pfmm_handle *h, int32_t op, const double *x, double *f, int32_t nrhs, int32_t parts, void *stream)
{
    return apply_impl(h, op, x, f, nrhs, parts, (cudaStream_t)stream);
}

int pfmm_count_apply_kernels(pfmm_handle *h, int32_t op, const double *x, double *f, int32_t nrhs, int32_t parts,
                             int64_t *kernels)
{
    if (!h || !x || !f || !kernels || nrhs < 1 || (op != 0 && op != 1) || parts < 1 || parts > 3)
        return fail(PFMM_ERR_INVALID_ARG, "invalid pfmm_count_apply_kernels arguments");
    *kernels = 0;
    int rc = ensure_workspace(h, nrhs);  // no allocation may happen inside the capture
    if (rc) return rc;
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const bool prof = h->prof;
    h->prof = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        rc = apply_impl(h, op, x, f, nrhs, parts, cs);
        e = cudaStreamEndCapture(cs, &graph);
    }
    h->prof = prof;
    size_t n = 0;
    if (e == cudaSuccess && !rc && graph) e = cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && !rc && n) e = cudaGraphGetNodes(graph, nodes.data(), &n);
    int64_t k = 0;
    for (size_t i = 0; e == cudaSuccess && !rc && i < n; ++i) {
        cudaGraphNodeType t;
        if ((e = cudaGraphNodeGetType(nodes[i], &t)) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, std::string("apply capture: ") + cudaGetErrorString(e));
    *kernels = k;
    return PFMM_OK;
}

int pfmm_apply_V(pfmm_handle *h, const double *w, double *f, int32_t nrhs, void *stream)
{
    return apply_impl(h, 0, w, f, nrhs, PFMM_PART_ALL, (cudaStream_t)stream);
}

int pfmm_apply_K(pfmm_handle *h, const double *g, double *f, int32_t nrhs, void *stream)
{
    return apply_impl(h, 1, g, f, nrhs, PFMM_PART_ALL, (cudaStream_t)stream);
}

int pfmm_apply_M(pfmm_handle *h, const double *g, double *f, int32_t nrhs, void *stream)
{
    if (!h || !g || !f || nrhs < 1) return fail(PFMM_ERR_INVALID_ARG, "invalid apply_M arguments");
    launch_apply_M(g, f, h->d_tri_user, h->d_area, nrhs, h->nt, h->nv, h->Et, h->h, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return PFMM_OK;
}

int pfmm_set_profiling(pfmm_handle *h, int32_t on)
{
    if (!h) return fail(PFMM_ERR_INVALID_ARG, "handle is NULL");
    h->prof = on != 0;
    return PFMM_OK;
}

int pfmm_phase_times(pfmm_handle *h, double *ms8, int32_t *n_applies)
{
    if (!h || !ms8) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
    prof_collect(h, 0);
    for (int i = 0; i < 8; ++i) {
        ms8[i] = h->acc_ms[i];
        h->acc_ms[i] = 0;
    }
    if (n_applies) *n_applies = h->n_prof;
    h->n_prof = 0;
    return PFMM_OK;
}

int pfmm_nf_kernel_time(pfmm_handle *h, double *ms, int32_t *n_launches)
{
    if (!h || !ms) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
    prof_collect(h, 0);
    *ms = h->acc_nf_ms;
    if (n_launches) *n_launches = h->n_nf;
    h->acc_nf_ms = 0;
    h->n_nf = 0;
    return PFMM_OK;
}

int pfmm_eval_repr(pfmm_handle *h, const double *w, const double *g, const double *points, int32_t npoints,
                   double *u, int32_t nrhs, void *stream)
{
    if (!h || !w || !points || !u || npoints < 0 || nrhs < 1)
        return fail(PFMM_ERR_INVALID_ARG, "invalid pfmm_eval_repr arguments");
    if (!h->d_rule_reg) return fail(PFMM_ERR_UNSUPPORTED, "handle has no quadrature rule");
    launch_repr(h->d_verts, h->d_tri_user, h->nt, h->nv, h->d_rule_reg, h->nq_reg, w, g, points, npoints, nrhs, h->Et,
                h->h, h->alpha, u, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return PFMM_OK;
}

int pfmm_get_info(const pfmm_handle *h, pfmm_info *info)
{
    if (!h || !info) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    const Tree &t = h->tree;
    info->p = t.p;
    for (int l = 0; l <= t.p && l < 32; ++l) {
        info->lx[l] = t.lv[l].lx;
        info->nbox[l] = t.lv[l].nbox;
        info->pad[l] = t.lv[l].pad;
    }
    info->n_m2l_pairs = t.n_m2l_pairs;
    // stored blocks: the arithmetic-type panels, or their two FP32 parts once split for tcgen05
    info->nearfield_bytes = h->otf ? h->otf_bytes
                                   : t.sizeV * (h->tcV ? 4 : (int64_t)h->es) + t.sizeK * (h->tcK ? 4 : (int64_t)h->es);
    info->device_bytes = h->dev_bytes;
    info->nf_tensor_cores = (h->tcV || h->crtV ? 1 : 0) | (h->tcK || h->crtK ? 2 : 0);
    info->nf_form = h->crtV || h->crtK ? h->crt_form : 0;
    info->nf_form_ms[0] = h->crt_form_ms[0];
    info->nf_form_ms[1] = h->crt_form_ms[1];
    if (h->crtV || h->crtK)
        info->nearfield_bytes += (h->crtV ? t.sizeV : 0) * 2 * pfmm::kCrtModuli + (h->crtK ? t.sizeK : 0) * 2 * pfmm::kCrtModuli;
    info->nearfield_v_elements = t.sizeV;
    info->nf_dense_columns = t.dense_cols ? 1 : 0;
    // separable M2L work per level: pass 1 over cells (X1, Y2, Y3) and the budget chains of every
    // triple (ne entries), pass 2 over cells (X1, X2, Y3) and C(m_x+5, 5) (budget, k2) pairs, pass 3
    // over the non-empty target boxes and ne (nu, k3) pairs; each sums over the R cells of one
    // direction within the interaction radius (R averaged over the target coordinate)
    double c5 = 1.0;
    for (int i = 1; i <= 5; ++i) c5 = c5 * (h->mx + i) / i;
    for (int l = 2; l <= h->p && l < (int)h->dl.size(); ++l) {
        const pfmm::DevLevel &L = h->dl[l];
        double R = 0.0;
        for (int X = 0; X < L.G; ++X) R += std::min(L.G - 1, X + L.ntr) - std::max(0, X - L.ntr) + 1;
        R /= L.G;
        const double pairs = L.kptr_host.empty() ? 0.0 : (double)L.kptr_host[L.nint], na2 = (double)h->na * h->na;
        const double G3 = (double)L.G * L.G * L.G;
        info->m2l_flops += 2.0 * pairs * na2 * R * (G3 * h->ne + G3 * c5 + (double)L.nbox * h->ne);
    }
    for (int l = 2; l <= h->p && l < 32 && l < (int)h->dl.size(); ++l) {
        const int e = pfmm::m2l_engine_for(h->fprec, h->dl[l].G, h->nk, h->ne, h->mx, h->m2l_force);
        info->m2l_engine[l] = e == pfmm::kM2LFused ? PFMM_M2L_FUSED
                              : e == pfmm::kM2LFusedSliced ? PFMM_M2L_FUSED_SLICED
                              : (e == pfmm::kM2LSlab ? PFMM_M2L_SLAB : PFMM_M2L_THREE_PASS);
    }
    return PFMM_OK;
}

int pfmm_check(pfmm_handle *h)
{
    if (!h) return fail(PFMM_ERR_INVALID_ARG, "handle is NULL");
    CK(cudaDeviceSynchronize());
    int e = 0;
    if (h->d_err) {
        CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemset(h->d_err, 0, sizeof(int)));
    }
    if (e) return fail(PFMM_ERR_TIMEOUT, "a bounded wait in the tensor-core nearfield kernel gave up (code " +
                                             std::to_string(e) + ")");
    return PFMM_OK;
}

void pfmm_destroy(pfmm_handle *h)
{
    if (!h) return;
    delete h;  // cudaFree waits for outstanding work on the buffers
}

}  // extern "C"
