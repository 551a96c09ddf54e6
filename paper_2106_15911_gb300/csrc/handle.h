// handle.h -- definition of the opaque pfmm_handle (shared by the C ABI translation units).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"
#include "pfmm_internal.h"

namespace pfmm {
// records an error message for pfmm_last_error() and returns the code
int set_error(int code, const std::string &msg);
}  // namespace pfmm

struct pfmm_handle;
namespace pfmm {
// tensor-core nearfield of op (0: V, 1: K) into fint; whi/wlo: [nrhs][E_t][cols] FP32 workspaces
// whi, wlo: FP16 input parts ([nrhs][E_t][cols] each); wmax: nrhs words of scratch
// part: FP64 partial planes, nf_tc_planes(H, op, nrhs) x nrhs x E_t x E_x doubles
int run_nf_tc(pfmm_handle *H, int op, const double *x, int nrhs, void *whi, void *wlo, unsigned long long *wmax,
              double *fint, double *part, cudaStream_t st);
// K-chunk partial planes of the tensor-core nearfield of op for nrhs right-hand sides
int nf_tc_planes(const pfmm_handle *H, int op, int nrhs);
// FP64 mode: exact residue-arithmetic nearfield of op on the tensor cores into fint (overwritten)
int run_nf_crt(pfmm_handle *H, int op, const double *x, int nrhs, double *fint, cudaStream_t st);
// size the per-call workspaces of a handle for nrhs right-hand sides (may allocate)
int ensure_ws(pfmm_handle *H, int nrhs);
// the on-the-fly nearfield of op into fint (+=): arguments of launch_nf_otf for this handle
int run_nf_otf(pfmm_handle *H, int op, const void *xin, int ncolg, int Et, int ls, int nrhs, int ndmax, double *fint,
               cudaStream_t st);
// f_b = A_0 x_b (same-step nearfield block) for ns slices [ns][E_x] in user order; xint holds
// ns E_x elements of the arithmetic type, fint ns E_x doubles
int apply_same_step(pfmm_handle *H, const double *x, double *f, int ns, void *xint, double *fint, cudaStream_t st);
// triangles and time steps a learned preconditioner was built for
void mpnn_dims(const pfmm_mpnn *net, int *nt, int *Et);
}  // namespace pfmm

struct EvSet {
    cudaEvent_t ev[11];  // 0..8: phase boundaries; 9, 10: around the nearfield product kernel
    bool nf = false;     // 9 and 10 were recorded
};

struct pfmm_handle {
    int nv = 0, nt = 0, Et = 0;
    double T = 0, alpha = 0, h = 0;
    pfmm_params prm{};
    pfmm::Tree tree;
    bool mixed = false;
    int fprec = 0;  // arithmetic of the FMM passes: 0 FP64, 1 FP32 (mixed), 2 double-FP32 (FP64 mode)
    int ls = 2, nd = 4, na = 0, nk = 0, mx = 0, p = 0;
    size_t es = 8;  // bytes of R
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;

    double *d_verts = nullptr, *d_area = nullptr;
    double *d_rule_reg = nullptr;  // collapsed Gauss rule of the regular quadrature: s1[nq], s2[nq], w[nq]
    int nq_reg = 0;
    int *d_tri_int = nullptr, *d_tri_user = nullptr, *d_perm = nullptr, *d_tri_leaf = nullptr, *d_leaf_start = nullptr,
        *d_leaf_grid = nullptr, *d_kidx = nullptr, *d_kinv = nullptr;
    void *d_Sx = nullptr, *d_SK = nullptr, *d_St = nullptr, *d_qt = nullptr;
    std::vector<pfmm::DevLevel> dl;
    void *d_AV = nullptr, *d_AK = nullptr;
    int *d_colV = nullptr, *d_colK = nullptr, *d_kmap = nullptr, *d_tiles = nullptr;
    int *d_box_tiles = nullptr;  // [leaf boxes + 1] first 64-row tile of each leaf box
    pfmm::PanelGPU *d_panels = nullptr;
    int ntiles = 0;
    int64_t mom_per_rhs = 0;
    // on-the-fly nearfield: no stored blocks, the compact singular values and the quadrature setup
    bool otf = false;
    pfmm::NfQuadArgs quad{};
    int *d_sing = nullptr, *d_tile_sing = nullptr;
    double *d_singV = nullptr, *d_singK = nullptr;
    int64_t otf_bytes = 0;

    int ne = 0;              // C(m_x+4,4) entries of the separable M2L intermediates per cell
    int *d_eoff = nullptr;   // [nk] offsets of the budget ranges
    int64_t m2l_ws_need = 0; // elements of T1 (and of T2) for a whole level, per rhs

    int ws_nrhs = 0;
    size_t ws_m2l = 0;
    void *d_T1 = nullptr, *d_T2 = nullptr;
    void *d_xint = nullptr, *d_gf = nullptr, *d_mu = nullptr, *d_lam = nullptr;
    double *d_fint = nullptr;

    // tensor-core nearfield (mixed mode, untruncated panels of equal width, 2 steps per leaf)
    bool tcV = false, tcK = false;
    bool nf_cuda_cores = false;     // engine override chosen by the batch autotuner
    int m2l_force = 0;              // M2L engine chosen by the batch autotuner (PFMM_M2L_* code, 0: per-level default)
    uint16_t *d_AVhi = nullptr, *d_AVlo = nullptr, *d_AKhi = nullptr, *d_AKlo = nullptr;  // FP16 parts
    int a_expV = 0, a_expK = 0;     // scale exponents of the panels' FP16 split
    CUtensorMap mapAVhi{}, mapAVlo{}, mapAKhi{}, mapAKlo{};
    int colsV_u = 0, colsK_u = 0;  // common padded column count of the panels
    int *d_tiles128 = nullptr;
    int ntiles128 = 0, nsm = 0;
    int *d_err = nullptr;           // bounded-wait error word of the device kernels
    // FP64 mode, exact residue-arithmetic nearfield on the tensor cores (k_nf_crt.cu)
    bool crtV = false, crtK = false;
    int crt_bV = 0, crt_bK = 0;                       // fixed-point bits of the operands
    int crt_form = 1, crt_best_form = 1;              // kernel form (1: two moduli, 2: two row tiles per item)
    double crt_form_ms[2] = {0, 0};                   // build-time timing of the two forms
    uint16_t *d_AVres = nullptr, *d_AKres = nullptr;  // FP16 residues [16][panel elements]
    int *d_rexpV = nullptr, *d_rexpK = nullptr;       // row scale exponents by triangle
    CUtensorMap mapAVres{}, mapAKres{};
    uint16_t *d_Wres = nullptr;                       // input residues [16][nrhs][E_t][cols]
    unsigned char *d_res8 = nullptr;                  // output residues [16][nrhs][E_t][E_x]
    uint16_t *d_Whi = nullptr, *d_Wlo = nullptr;  // FP16 input parts
    unsigned long long *d_wmax = nullptr;          // [ws_nrhs] max |input| per rhs (FP64 bits)
    double *d_nfpart = nullptr;                    // partial planes of the tensor-core nearfield
    size_t w_elems = 0;

    bool prof = false;
    std::vector<EvSet> evs;
    int ev_head = 0, ev_pending = 0;
    double acc_ms[8] = {0};
    int n_prof = 0;
    EvSet *cur_ev = nullptr;  // events of the apply in progress (profiling on)
    double acc_nf_ms = 0;     // nearfield product kernel alone
    int n_nf = 0;

    // stored nearfield blocks of op for the CUDA-core engine: the FP32/FP64 panels, or null once
    // only the tensor-core split exists (nf_split then describes it)
    const void *nf_blocks(int op) const { return op == 0 ? d_AV : d_AK; }
    pfmm::NfHalfSplit split_desc(int op) const
    {
        pfmm::NfHalfSplit s;
        s.hi = op == 0 ? d_AVhi : d_AKhi;
        s.lo = op == 0 ? d_AVlo : d_AKlo;
        s.inv_scale = std::ldexp(1.0f, -(op == 0 ? a_expV : a_expK));
        return s;
    }
    // the split to read in place of the panels, or null while the panels exist
    const pfmm::NfHalfSplit *nf_split(int op, pfmm::NfHalfSplit *buf) const
    {
        if (nf_blocks(op)) return nullptr;
        *buf = split_desc(op);
        return buf;
    }

    ~pfmm_handle()
    {
        for (void *p : allocs) cudaFree(p);
        for (auto &e : evs)
            for (int i = 0; i < 11; ++i) cudaEventDestroy(e.ev[i]);
    }

    template <typename T_>
    int alloc(T_ **p, size_t n_elems, size_t elem = sizeof(T_))
    {
        void *q = nullptr;
        size_t bytes = std::max<size_t>(n_elems * elem, 16);
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return pfmm::set_error(e == cudaErrorMemoryAllocation ? PFMM_ERR_OOM : PFMM_ERR_CUDA,
                        "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
        }
        allocs.push_back(q);
        dev_bytes += (int64_t)bytes;
        *p = (T_ *)q;
        return PFMM_OK;
    }

    void release(void *p)
    {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) {
            cudaFree(p);
            allocs.erase(it);
        }
    }
};

