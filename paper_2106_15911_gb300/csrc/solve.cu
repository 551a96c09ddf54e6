// solve.cu -- pfmm_solve: the space-time system V_h w = b of Section 2 (Eq. 02:linear:system)
// solved at once with restarted flexible GMRES (the paper solves the whole system with GMRES,
// Section 3 and Section 5), all vectors FP64 on the device.
//
//   b = (1/2 M_h + K_h) g   (direct formulation, Section 2)   or   b = M_h g   (indirect)
//   FGMRES(m): right-preconditioned, Arnoldi with classical Gram-Schmidt applied twice,
//              Givens rotations on the host, x0 = 0 (Saad 1993).  The preconditioner slot is the
//              identity.
//   GMRES-IR:  when opts->refine is an FP64 handle of the same problem, the outer loop computes
//              r = b - V_h x with it in FP64 and the inner FGMRES runs with the (mixed-precision)
//              handle h to opts->inner_tol, then x += d (Carson & Higham 2017, 2018).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "handle.h"
#include "kernels.h"

namespace {

using pfmm::set_error;

#define SCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kDotBlocks = 304, kDotThreads = 256;

// partial dot products of w with the columns V[0..nvec) (stride ldv): grid (kDotBlocks, nvec)
__global__ void k_dots(const double *__restrict__ V, size_t ldv, const double *__restrict__ w, size_t n,
                       double *__restrict__ part)
{
    __shared__ double red[kDotThreads / 32];
    const double *v = V + (size_t)blockIdx.y * ldv;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s += v[i] * w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_reduce_parts(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(size_t)blockIdx.x * nb + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[blockIdx.x] = s;
    }
}

// w -= sum_j V[j] h[j]   (h on the device)
__global__ void k_sub_combo(const double *__restrict__ V, size_t ldv, int nvec, const double *__restrict__ h,
                            double *__restrict__ w, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s += V[(size_t)j * ldv + i] * h[j];
    w[i] -= s;
}

// y += sum_j Z[j] c[j]   (c on the device)
__global__ void k_add_combo(const double *__restrict__ Z, size_t ldz, int nvec, const double *__restrict__ c,
                            double *__restrict__ y, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s += Z[(size_t)j * ldz + i] * c[j];
    y[i] += s;
}

__global__ void k_axpby(double a, const double *__restrict__ x, double b, double *__restrict__ y, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_scale_to(double a, const double *__restrict__ x, double *__restrict__ y, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

__global__ void k_finite(const double *__restrict__ x, size_t n, int *__restrict__ bad)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) *bad = 1;
}

unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

struct Ws {
    double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *d = nullptr, *part = nullptr, *hv = nullptr;
    int *bad = nullptr;
    std::vector<void *> mem;
    ~Ws()
    {
        for (void *p : mem) cudaFree(p);
    }
    int get(double **p, size_t n)
    {
        cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(double));
        if (e != cudaSuccess) return set_error(PFMM_ERR_OOM, "solver workspace allocation failed");
        mem.push_back(*p);
        return PFMM_OK;
    }
};

// dots[0..nvec) = V[0..nvec)^T w  (synchronises the stream, result on the host)
int dots(Ws &W, const double *V, size_t ldv, int nvec, const double *w, size_t n, double *host, cudaStream_t st)
{
    k_dots<<<dim3(kDotBlocks, nvec), kDotThreads, 0, st>>>(V, ldv, w, n, W.part);
    k_reduce_parts<<<nvec, 256, 0, st>>>(W.part, kDotBlocks, W.hv);
    SCK(cudaMemcpyAsync(host, W.hv, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    return PFMM_OK;
}

// one right-hand side: FGMRES(m) on op(h) for V x = b, x updated in place (x0 as given).
// Returns PFMM_OK when ||b - V x|| <= tol_abs, PFMM_ERR_NOT_CONVERGED when max_it was reached.
int fgmres(pfmm_handle *h, const double *b, double *x, double tol_abs, int restart, int max_it, int *iters, Ws &W,
           size_t n, cudaStream_t st, double *res_out)
{
    const size_t ld = n;
    std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), gv(restart + 1), hh(restart + 2),
        y(restart);
    int total = 0;
    double beta = 0.0;
    while (true) {
        // r = b - V x
        int rc = pfmm_apply_V(h, x, W.w, 1, st);
        if (rc) return rc;
        k_axpby<<<nblk(n), 256, 0, st>>>(1.0, b, -1.0, W.w, n);
        double d2;
        if ((rc = dots(W, W.w, ld, 1, W.w, n, &d2, st))) return rc;
        beta = std::sqrt(d2);
        *res_out = beta;
        if (!(beta > tol_abs) || total >= max_it) break;
        k_scale_to<<<nblk(n), 256, 0, st>>>(1.0 / beta, W.w, W.V, n);
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int j = 0;
        for (; j < restart && total < max_it; ++j, ++total) {
            // z_j = P(v_j): identity preconditioner; w = V_h z_j
            SCK(cudaMemcpyAsync(W.Z + (size_t)j * ld, W.V + (size_t)j * ld, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            if ((rc = pfmm_apply_V(h, W.Z + (size_t)j * ld, W.w, 1, st))) return rc;
            // classical Gram-Schmidt, twice
            for (int i = 0; i <= j; ++i) H[(size_t)i * restart + j] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                if ((rc = dots(W, W.V, ld, j + 1, W.w, n, hh.data(), st))) return rc;
                SCK(cudaMemcpyAsync(W.hv, hh.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
                k_sub_combo<<<nblk(n), 256, 0, st>>>(W.V, ld, j + 1, W.hv, W.w, n);
                for (int i = 0; i <= j; ++i) H[(size_t)i * restart + j] += hh[i];
            }
            double nw2;
            if ((rc = dots(W, W.w, ld, 1, W.w, n, &nw2, st))) return rc;
            const double hn = std::sqrt(nw2);
            H[(size_t)(j + 1) * restart + j] = hn;
            if (hn > 0.0) k_scale_to<<<nblk(n), 256, 0, st>>>(1.0 / hn, W.w, W.V + (size_t)(j + 1) * ld, n);
            // Givens rotations
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * restart + j], c = H[(size_t)(i + 1) * restart + j];
                H[(size_t)i * restart + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * restart + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)j * restart + j], c = H[(size_t)(j + 1) * restart + j];
            double den = std::hypot(a, c);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? c / den : 0.0;
            H[(size_t)j * restart + j] = den;
            H[(size_t)(j + 1) * restart + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            if (std::fabs(gv[j + 1]) <= tol_abs || hn == 0.0) {
                ++j;
                ++total;
                break;
            }
        }
        // y = R^{-1} g, x += Z y
        for (int i = j - 1; i >= 0; --i) {
            double s = gv[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * restart + k] * y[k];
            y[i] = s / H[(size_t)i * restart + i];
        }
        SCK(cudaMemcpyAsync(W.hv, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
        k_add_combo<<<nblk(n), 256, 0, st>>>(W.Z, ld, j, W.hv, x, n);
        SCK(cudaGetLastError());
    }
    *iters += total;
    return beta <= tol_abs ? PFMM_OK : PFMM_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" int pfmm_solve(pfmm_handle *h, int32_t formulation, const double *g, double *x, int32_t nrhs,
                          const pfmm_solve_opts *opts_in, pfmm_solve_info *info, void *stream)
{
    if (!h || !g || !x || nrhs < 1 || (formulation != PFMM_DIRECT && formulation != PFMM_INDIRECT))
        return set_error(PFMM_ERR_INVALID_ARG, "invalid pfmm_solve arguments");
    pfmm_solve_opts o;
    pfmm_default_solve_opts(&o);
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0) || o.restart < 1 || o.restart > 500 || o.max_it < 1)
        return set_error(PFMM_ERR_INVALID_ARG, "invalid solver options");
    pfmm_handle *h64 = o.refine;
    if (h64 && (h64->nt != h->nt || h64->Et != h->Et || h64->nv != h->nv))
        return set_error(PFMM_ERR_INVALID_ARG, "refinement handle describes a different problem");
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const size_t n = (size_t)h->Et * h->nt, ng = (size_t)h->Et * h->nv;
    Ws W;
    int rc;
    if ((rc = W.get(&W.V, (size_t)(o.restart + 1) * n)) || (rc = W.get(&W.Z, (size_t)o.restart * n)) ||
        (rc = W.get(&W.w, n)) || (rc = W.get(&W.r, n)) || (rc = W.get(&W.d, n)) ||
        (rc = W.get(&W.part, (size_t)kDotBlocks * (o.restart + 2))) || (rc = W.get(&W.hv, (size_t)o.restart + 2)))
        return rc;
    SCK(cudaMalloc((void **)&W.bad, sizeof(int)));
    W.mem.push_back(W.bad);
    double *b = nullptr;
    if ((rc = W.get(&b, n))) return rc;
    int iters = 0, outer = 0;
    double worst = 0.0;
    int status = PFMM_OK;
    for (int r = 0; r < nrhs; ++r) {
        const double *gr = g + (size_t)r * ng;
        double *xr = x + (size_t)r * n;
        SCK(cudaMemsetAsync(W.bad, 0, sizeof(int), st));
        k_finite<<<nblk(ng), 256, 0, st>>>(gr, ng, W.bad);
        int bad = 0;
        SCK(cudaMemcpyAsync(&bad, W.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        if (bad) return set_error(PFMM_ERR_NONFINITE, "the datum g holds NaN or Inf");
        // right-hand side (Eq. 02:linear:system), with the FP64 handle when refining
        pfmm_handle *hb = h64 ? h64 : h;
        if ((rc = pfmm_apply_M(hb, gr, b, 1, st))) return rc;
        if (formulation == PFMM_DIRECT) {
            if ((rc = pfmm_apply_K(hb, gr, W.r, 1, st))) return rc;
            k_axpby<<<nblk(n), 256, 0, st>>>(1.0, W.r, 0.5, b, n);
        }
        double bn2;
        if ((rc = dots(W, b, n, 1, b, n, &bn2, st))) return rc;
        const double bn = std::sqrt(bn2);
        SCK(cudaMemsetAsync(xr, 0, n * sizeof(double), st));
        double res = bn;
        if (bn == 0.0) continue;
        if (!h64) {
            int s = fgmres(h, b, xr, o.tol * bn, o.restart, o.max_it, &iters, W, n, st, &res);
            if (s == PFMM_ERR_NOT_CONVERGED) status = s;
            else if (s) return s;
        } else {
            // GMRES-IR: FP64 residual with h64, inner solve with h
            for (int it = 0;; ++it) {
                if ((rc = pfmm_apply_V(h64, xr, W.r, 1, st))) return rc;
                k_axpby<<<nblk(n), 256, 0, st>>>(1.0, b, -1.0, W.r, n);
                double rn2;
                if ((rc = dots(W, W.r, n, 1, W.r, n, &rn2, st))) return rc;
                res = std::sqrt(rn2);
                if (res <= o.tol * bn) break;
                if (it >= o.max_outer || iters >= o.max_it) {
                    status = PFMM_ERR_NOT_CONVERGED;
                    break;
                }
                ++outer;
                SCK(cudaMemsetAsync(W.d, 0, n * sizeof(double), st));
                double ires = res;
                int s = fgmres(h, W.r, W.d, o.inner_tol * res, o.restart, o.max_it - iters, &iters, W, n, st, &ires);
                if (s && s != PFMM_ERR_NOT_CONVERGED) return s;
                k_axpby<<<nblk(n), 256, 0, st>>>(1.0, W.d, 1.0, xr, n);
            }
        }
        worst = std::max(worst, res / bn);
    }
    SCK(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = iters;
        info->outer = outer;
        info->rel_res = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status) set_error(status, "the solver reached max_it / max_outer before the tolerance");
    return status;
}

extern "C" int pfmm_default_solve_opts(pfmm_solve_opts *o)
{
    if (!o) return set_error(PFMM_ERR_INVALID_ARG, "opts is NULL");
    o->tol = 1e-8;
    o->restart = 50;
    o->max_it = 1000;
    o->refine = nullptr;
    o->inner_tol = 1e-4;
    o->max_outer = 20;
    return PFMM_OK;
}
