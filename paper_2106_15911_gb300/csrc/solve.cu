// solve.cu -- pfmm_solve: the space-time system V_h w = b of Section 2 (Eq. 02:linear:system)
// solved at once with restarted flexible GMRES (the paper solves the whole system with GMRES,
// Section 3 and Section 5), all vectors FP64 on the device.
//
//   b = (1/2 M_h + K_h) g   (direct formulation, Section 2)   or   b = M_h g   (indirect)
//   FGMRES(m): right-preconditioned, Arnoldi with classical Gram-Schmidt applied twice,
//              Givens rotations on the host, x0 = 0 (Saad 1993).  The preconditioner is the
//              identity or a learned network z = P(v) (mpnn.cu); P is dropped for the rest of
//              the solve when it yields a non-finite direction or a cycle that cuts the residual
//              by less than 10 %, so plain FGMRES is the fallback.
//   Recording: at every rec_every-th Arnoldi step j of a cycle, x_j = x + Z_j y_j and
//              r_j = V_{j+1} (beta e_1 - Hbar_j y_j) (the Arnoldi relation, no extra matvec) are
//              stored; once the right-hand side is solved the stored iterates become errors
//              x - x_j.
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
    double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *d = nullptr, *part = nullptr, *hv = nullptr,
           *cy = nullptr;
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

struct Rec {
    double *R = nullptr, *E = nullptr;
    int cap = 0, every = 5, count = 0;
    bool basis = false;      // record the Arnoldi vectors v_j instead of (r_j, e_j)
    double floor_abs = 0.0;  // record only while the residual norm is above this
};

struct Prec {
    pfmm_mpnn *net = nullptr;
    bool on = false;
    int dropped = 0;
};

// one right-hand side: FGMRES(m) on op(h) for V x = b, x updated in place (x0 as given).
// Returns PFMM_OK when ||b - V x|| <= tol_abs, PFMM_ERR_NOT_CONVERGED when max_it was reached.
int fgmres(pfmm_handle *h, Prec &P, Rec *rec, const double *b, double *x, double tol_abs, int restart, int max_it,
           int *iters, Ws &W, size_t n, cudaStream_t st, double *res_out)
{
    const size_t ld = n;
    std::vector<double> H((size_t)(restart + 1) * restart), Hraw((size_t)(restart + 1) * restart), cs(restart),
        sn(restart), gv(restart + 1), hh(restart + 2), y(restart), c(restart + 1);
    int total = 0;
    double beta = 0.0, beta_prev = HUGE_VAL;
    // y = R_j^{-1} g_j from the rotated Hessenberg rows 0 .. j-1
    auto solve_r = [&](int j) {
        for (int i = j - 1; i >= 0; --i) {
            double s = gv[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * restart + k] * y[k];
            y[i] = s / H[(size_t)i * restart + i];
        }
    };
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
        if (P.on && beta > 0.9 * beta_prev) {  // the last preconditioned cycle stagnated
            P.on = false;
            ++P.dropped;
        }
        beta_prev = beta;
        k_scale_to<<<nblk(n), 256, 0, st>>>(1.0 / beta, W.w, W.V, n);
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int j = 0;
        while (j < restart && total < max_it) {
            if (rec && rec->basis && rec->count < rec->cap && j % rec->every == 0) {
                SCK(cudaMemcpyAsync(rec->R + (size_t)rec->count * n, W.V + (size_t)j * ld, n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
                ++rec->count;
            } else if (rec && !rec->basis && rec->count < rec->cap && j % rec->every == 0 &&
                       std::fabs(gv[j]) > rec->floor_abs) {
                // x_j and r_j of the current cycle into the next slot
                double *Rs = rec->R + (size_t)rec->count * n, *Es = rec->E ? rec->E + (size_t)rec->count * n : nullptr;
                if (Es) SCK(cudaMemcpyAsync(Es, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
                if (j == 0) {
                    k_scale_to<<<nblk(n), 256, 0, st>>>(beta, W.V, Rs, n);
                } else {
                    solve_r(j);
                    for (int i = 0; i <= j; ++i) {
                        double s = i == 0 ? beta : 0.0;
                        for (int k = 0; k < j; ++k) s -= Hraw[(size_t)i * restart + k] * y[k];
                        c[i] = s;
                    }
                    SCK(cudaMemcpyAsync(W.cy, c.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
                    SCK(cudaMemcpyAsync(W.cy + restart + 1, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
                    SCK(cudaMemsetAsync(Rs, 0, n * sizeof(double), st));
                    k_add_combo<<<nblk(n), 256, 0, st>>>(W.V, ld, j + 1, W.cy, Rs, n);
                    if (Es) k_add_combo<<<nblk(n), 256, 0, st>>>(W.Z, ld, j, W.cy + restart + 1, Es, n);
                    SCK(cudaStreamSynchronize(st));  // c and y are reused by the next record
                }
                ++rec->count;
            }
            // z_j = P(v_j); w = V_h z_j
            double *zj = W.Z + (size_t)j * ld;
            if (P.on) {
                if ((rc = pfmm_mpnn_apply(P.net, W.V + (size_t)j * ld, zj, 1, st))) return rc;
            } else {
                SCK(cudaMemcpyAsync(zj, W.V + (size_t)j * ld, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
            if ((rc = pfmm_apply_V(h, zj, W.w, 1, st))) return rc;
            // classical Gram-Schmidt, twice
            for (int i = 0; i <= j; ++i) H[(size_t)i * restart + j] = 0.0;
            bool finite = true;
            for (int pass = 0; pass < 2 && finite; ++pass) {
                if ((rc = dots(W, W.V, ld, j + 1, W.w, n, hh.data(), st))) return rc;
                for (int i = 0; i <= j; ++i) finite = finite && std::isfinite(hh[i]);
                if (!finite) break;
                SCK(cudaMemcpyAsync(W.hv, hh.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
                k_sub_combo<<<nblk(n), 256, 0, st>>>(W.V, ld, j + 1, W.hv, W.w, n);
                for (int i = 0; i <= j; ++i) H[(size_t)i * restart + j] += hh[i];
            }
            double nw2 = 0.0;
            if (finite && (rc = dots(W, W.w, ld, 1, W.w, n, &nw2, st))) return rc;
            if (!finite || !std::isfinite(nw2)) {
                if (!P.on) return set_error(PFMM_ERR_NONFINITE, "non-finite Krylov vector (operator output)");
                P.on = false;  // the network gave a non-finite direction: redo this step without it
                ++P.dropped;
                continue;
            }
            const double hn = std::sqrt(nw2);
            H[(size_t)(j + 1) * restart + j] = hn;
            for (int i = 0; i <= j + 1; ++i) Hraw[(size_t)i * restart + j] = H[(size_t)i * restart + j];
            if (hn > 0.0) k_scale_to<<<nblk(n), 256, 0, st>>>(1.0 / hn, W.w, W.V + (size_t)(j + 1) * ld, n);
            // Givens rotations
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * restart + j], cc = H[(size_t)(i + 1) * restart + j];
                H[(size_t)i * restart + j] = cs[i] * a + sn[i] * cc;
                H[(size_t)(i + 1) * restart + j] = -sn[i] * a + cs[i] * cc;
            }
            double a = H[(size_t)j * restart + j], cc = H[(size_t)(j + 1) * restart + j];
            double den = std::hypot(a, cc);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? cc / den : 0.0;
            H[(size_t)j * restart + j] = den;
            H[(size_t)(j + 1) * restart + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            ++j;
            ++total;
            if (std::fabs(gv[j]) <= tol_abs || hn == 0.0) break;
        }
        // y = R^{-1} g, x += Z y
        solve_r(j);
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
    if (o.rec_cap < 0 || (o.rec_cap > 0 && (!o.rec_r || h64 || o.rec_every < 1)))
        return set_error(PFMM_ERR_INVALID_ARG, "recording needs rec_r, rec_every >= 1 and no refine handle");
    if (o.precond) {
        int pnt = 0, pEt = 0;
        pfmm::mpnn_dims(o.precond, &pnt, &pEt);
        if (pnt != h->nt || pEt != h->Et) return set_error(PFMM_ERR_INVALID_ARG, "the preconditioner is for another mesh");
    }
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const size_t n = (size_t)h->Et * h->nt, ng = (size_t)h->Et * h->nv;
    Prec P;
    P.net = o.precond;
    P.on = o.precond != nullptr;
    Rec rec;
    rec.R = o.rec_r;
    rec.E = o.rec_e;
    rec.cap = o.rec_cap;
    rec.every = o.rec_every;
    rec.basis = o.rec_basis != 0;
    if (rec.basis) rec.E = nullptr;
    Rec *recp = o.rec_cap > 0 ? &rec : nullptr;
    Ws W;
    int rc;
    if ((rc = W.get(&W.V, (size_t)(o.restart + 1) * n)) || (rc = W.get(&W.Z, (size_t)o.restart * n)) ||
        (rc = W.get(&W.w, n)) || (rc = W.get(&W.r, n)) || (rc = W.get(&W.d, n)) ||
        (rc = W.get(&W.part, (size_t)kDotBlocks * (o.restart + 2))) || (rc = W.get(&W.hv, (size_t)o.restart + 2)) ||
        (rc = W.get(&W.cy, 2 * (size_t)o.restart + 2)))
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
            const int first = rec.count;
            rec.floor_abs = 100.0 * o.tol * bn;
            int s = fgmres(h, P, recp, b, xr, o.tol * bn, o.restart, o.max_it, &iters, W, n, st, &res);
            if (s == PFMM_ERR_NOT_CONVERGED) status = s;
            else if (s) return s;
            for (int k = first; rec.E && k < rec.count; ++k)  // stored iterates -> errors x - x_k
                k_axpby<<<nblk(n), 256, 0, st>>>(1.0, xr, -1.0, rec.E + (size_t)k * n, n);
        } else {
            // GMRES-IR: FP64 residual with h64, inner solve with h
            for (int it = 0;; ++it) {
                if (it == 0) {  // x = 0: the residual is b itself
                    SCK(cudaMemcpyAsync(W.r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
                } else {
                    if ((rc = pfmm_apply_V(h64, xr, W.r, 1, st))) return rc;
                    k_axpby<<<nblk(n), 256, 0, st>>>(1.0, b, -1.0, W.r, n);
                }
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
                int s = fgmres(h, P, nullptr, W.r, W.d, o.inner_tol * res, o.restart, o.max_it - iters, &iters, W, n,
                               st, &ires);
                if (s && s != PFMM_ERR_NOT_CONVERGED) return s;
                k_axpby<<<nblk(n), 256, 0, st>>>(1.0, W.d, 1.0, xr, n);
            }
        }
        worst = std::max(worst, res / bn);
    }
    SCK(cudaStreamSynchronize(st));
    if (o.precond && (rc = pfmm_mpnn_check(o.precond))) return rc;
    if (info) {
        info->iterations = iters;
        info->outer = outer;
        info->rel_res = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->recorded = rec.count;
        info->precond_off = P.dropped;
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
    o->precond = nullptr;
    o->rec_r = nullptr;
    o->rec_e = nullptr;
    o->rec_cap = 0;
    o->rec_every = 5;
    o->rec_basis = 0;
    return PFMM_OK;
}
