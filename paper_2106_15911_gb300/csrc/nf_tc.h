// nf_tc.h -- launch interface of the tensor-core nearfield apply (k_nf_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace pfmm {

struct NfTcParams {
    const PanelGPU *panels;
    const int *tiles;   // [ntiles][2] (panel, first row) with 128-row tiles
    int ntiles, nib, ksplit, nkb, nitems, cols_pad, kop;
    int nint, Et, nt;
    double *f;          // FP64 output [rhs][Et][nt] (internal order), accumulated with atomics
    int *err;           // set non-zero when a bounded wait gave up
};

size_t nf_tc_smem_bytes();
int launch_nf_apply_tc(const CUtensorMap &Ahi, const CUtensorMap &Alo, const CUtensorMap &Whi, const CUtensorMap &Wlo,
                       const NfTcParams &P, int nsm, cudaStream_t st);
void launch_split_panel(const float *A, float *hi, float *lo, size_t n, cudaStream_t st);
void launch_split_input(const double *x, const int *perm, int ncol, int ncol_pad, int nrhs, int Et, float *hi,
                        float *lo, cudaStream_t st);

}  // namespace pfmm
