// nf_tc.h -- launch interface of the tensor-core nearfield apply (k_nf_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace pfmm {

constexpr int kScaleExpMax = 100;  // bound on |E| of the power-of-two scales

// Scale exponents E of the FP16 split for a largest magnitude m: 2^E m lies in [2^14, 2^15); 0 for
// m = 0, infinite or NaN; clamped to +-kScaleExpMax (subnormal maxima get the bound).
// From the FP32 bits of m (panels): m = 1.f * 2^(b - 127) with biased exponent b, E = 141 - b.
__host__ __device__ inline int f32_scale_exp(unsigned bits)
{
    bits &= 0x7fffffffu;
    const int b = (int)(bits >> 23);
    if (bits == 0u || b == 255) return 0;
    const int E = 141 - b;
    return E > kScaleExpMax ? kScaleExpMax : (E < -kScaleExpMax ? -kScaleExpMax : E);
}
// From the FP64 bits of m (input): m = 1.f * 2^(b - 1023), E = 1037 - b.
__host__ __device__ inline int f64_scale_exp(unsigned long long bits)
{
    bits &= 0x7fffffffffffffffull;
    const int b = (int)(bits >> 52);
    if (bits == 0ull || b == 2047) return 0;
    const int E = 1037 - b;
    return E > kScaleExpMax ? kScaleExpMax : (E < -kScaleExpMax ? -kScaleExpMax : E);
}

struct NfTcParams {
    const PanelGPU *panels;
    const int *tiles;   // [ntiles][2] (panel, first row) with 128-row tiles
    int ntiles, nib, ksplit, nkb, nitems, cols_pad, kop;
    int nint, Et, nt;
    int a_exp;              // scale exponent of the panels' FP16 split
    const unsigned long long *wmax;  // [nrhs] FP64 bits of max |W| per rhs (scale of the input split)
    double *part;       // FP64 partial planes [ksplit][nrhs][Et][nt] (internal order), every element written
    int nrhs;
    int *err;           // set non-zero when a bounded wait gave up
};

// per-rhs max |x| of x [nrhs][per_rhs] FP64 into wmax (FP64 bits, accumulated with atomicMax: zero it first)
void launch_absmax_input(const double *x, size_t per_rhs, int nrhs, unsigned grid_x, unsigned long long *wmax,
                         cudaStream_t st);
size_t nf_tc_smem_bytes();
// K chunks (partial planes) of the tensor-core nearfield for `tiles` output tiles of nkb column
// blocks: 1 .. 8 (at most the tile's 32-stage sub-chunks), chosen so the work items fill the
// rounds of the persistent grid of nsm CTAs best
int nf_tc_ksplit(int tiles, int nkb, int nsm);
// f[i] = sum_kc part[kc][i] (n elements per plane, plane order)
void launch_nf_tc_reduce(const double *part, int ks, size_t n, double *f, cudaStream_t st);
int launch_nf_apply_tc(const CUtensorMap &Ahi, const CUtensorMap &Alo, const CUtensorMap &Whi, const CUtensorMap &Wlo,
                       const NfTcParams &P, int nsm, cudaStream_t st);
// scale exponent of n stored FP32 panel values (synchronises st; scratch: one device word);
// INT32_MIN on a CUDA error
int panel_scale_exp(const float *A, size_t n, unsigned *scratch, cudaStream_t st);
// hi/lo FP16 parts ([n] each, 64 x 64 blocks of nf_tiled_index) of 2^a_exp A (row-major, ncp
// columns, a multiple of 64)
void launch_split_panel(const float *A, void *hi, void *lo, size_t n, int ncp, int a_exp, cudaStream_t st);
// per-rhs max |x| into wmax[nrhs], then the hi/lo FP16 parts [nrhs][Et][ncol_pad] of the scaled,
// permuted (V) or padded (K) input
void launch_split_input(const double *x, const int *perm, int ncol, int ncol_pad, int nrhs, int Et, void *hi,
                        void *lo, unsigned long long *wmax, cudaStream_t st);

}  // namespace pfmm
