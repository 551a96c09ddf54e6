// nf_crt.h -- launch interface of the FP64-accurate tensor-core nearfield (k_nf_crt.cu): the
// block-Toeplitz product computed exactly modulo 16 primes on tcgen05 and combined by the Chinese
// remainder theorem.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace pfmm {

constexpr int kCrtModuli = 16;

struct NfCrtParams {
    const PanelGPU *panels;
    const int *tiles;      // [ntiles][2] (panel, first row) with 128-row tiles
    int ntiles, nib, nkb, nitems, cols_pad, kop;
    int nint, Et, nt, nrhs;
    unsigned char *res;    // out: residues [modulus][rhs][Et][nt] in [0, p)
    int *err;              // set non-zero when a bounded wait gave up
};

// moduli tables into constant memory of the current device (once per device); 0 or -1
int crt_upload_constants(cudaStream_t st);
// fixed-point bits b of both operands for a reduction over k_total terms: 2 k_total 2^(2b) < M
int crt_bits(long long k_total);
// per-row exponents of the stored FP64 panels (largest |A| of the row over d and columns in
// [2^(b-1), 2^b) after scaling): rowexp_tri[nt] by triangle, rowexp_R by global panel row
void launch_crt_row_exps(const double *A, const PanelGPU *panels, int npanel, int kop, int nd, int ncp, int b,
                         unsigned long long *rowmax, int nt, int *rowexp_tri, int *rowexp_R, cudaStream_t st);
// residues [kCrtModuli][n] (FP16, 64 x 64 blocks of nf_tiled_index) of the scaled, rounded panels
void launch_crt_split_panel(const double *A, const int *rowexp_R, size_t n, int ncp, void *res, cudaStream_t st);
// per-rhs max |x| into wmax, residues [kCrtModuli][nrhs][Et][ncol_pad] of the scaled, rounded,
// permuted (V) or padded (K) input
void launch_crt_split_input(const double *x, const int *perm, int ncol, int ncol_pad, int nrhs, int Et, int b,
                            void *res, unsigned long long *wmax, cudaStream_t st);
// f[rhs][t][row] (overwritten) from the residues of the exact products
void launch_crt_combine(const unsigned char *res, int nrhs, int Et, int nt, const int *rowexp,
                        const unsigned long long *wmax, int b, double *f, cudaStream_t st);
size_t nf_crt_smem_bytes();
// form 1: one row tile and two moduli per CTA work item; form 2: two row tiles sharing each W
// stage, one modulus per item (P.nitems is recomputed for it)
int launch_nf_apply_crt(const CUtensorMap &A, const CUtensorMap &W, const NfCrtParams &P, int nsm, cudaStream_t st,
                        int form);

}  // namespace pfmm
