// mpnn.cu -- a learned flexible right preconditioner for FGMRES: a message-passing network over
// the edge adjacency of the surface triangles, applied to every time slice of a Krylov vector.
// The paper's solver is plain GMRES; the network is an addition, and FGMRES with the exact pFMM
// operator still judges every residual, so the answer never depends on it.
//
// For a slice v (the E_x values of time step t of a vector), s = RMS(v) + 1e-30, and the
// geometry/step features f_i = (|gamma_i| / mean area, n_i (3 components), (t + 1/2) / E_t):
//   e_i     = SiLU(W_g^T f_i + b_g)                                   5 -> W, geometry embedding
//   h^0_i   = (v_i / s) e_i
//   h^{l+1} = h^l + W_s^T h^l + W_n^T mean_{j in N(i)} h^l_j            l = 0 .. L-1
//   z_i     = c s (w_o . h^L_i)
// N(i): the triangles sharing an edge with triangle i; c: a fixed output scale (estimated from
// the first training batch, or set by the caller).  The map v -> z is linear (s cancels) with
// coefficients that depend nonlinearly on the geometry: FGMRES needs a consistent preconditioner,
// and an input-dependent (nonlinear) map loses the gain of an approximate inverse even at a few
// per cent of inconsistency.
// Parameters: FP32 master copy (Adam), BF16 copy for the passes.  For widths 32 and 64 the
// layers run on the tensor cores (tcgen05.mma kind::f16, BF16 weights, layer input split into
// BF16 hi + lo parts so that the product is FP32-accurate, FP32 accumulation in TMEM); the
// rest, and the backward pass, are FP32 on the CUDA cores.  Parameter vector, in this order
// (matrices input-major, M[k][o]):
//   W_g [5][W], b_g [W],  per layer { W_s [W][W], W_n [W][W] },  w_o [W]
// Training on a batch of S residual slices r_b (recorded from FGMRES runs), in one of two forms:
//   same-step form (a pFMM handle given): the correction the network should produce for r_b is
//     c_b = A_0^{-1} r_b (A_0: the same-step block of V_h, the time-block-diagonal part), measured
//     in the residual norm, which needs no c_b:
//       loss = (1/S) sum_b ||A_0 z(r_b) - r_b||^2 / (||r_b||^2 + 1e-30)
//     Its gradient applies A_0 in place of A_0^T: the Galerkin block of the symmetric heat kernel
//     is symmetric up to the quadrature error of the singular rules.
//   error form (no handle): regression on the recorded errors e_b (V_h e = r),
//       loss = (1/S) sum_b ||z(r_b) - e_b||^2 / (||e_b||^2 + 1e-30)
// minimised by Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected, cosine-decayed step size).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <random>
#include <string>
#include <utility>
#include <vector>

#include "handle.h"
#include "tc_ptx.cuh"

namespace {

using pfmm::set_error;

constexpr int NG = 5;      // geometry / step features
constexpr int XS = 8;      // row stride of the stored inputs (v / s, the 5 features, padding)
constexpr int RT = 64;     // rows per CTA of the dense layer kernels
constexpr int RW = 32;     // rows per tile of the weight-gradient kernels
constexpr int NTH = 256;   // threads per CTA of the dense kernels
constexpr int64_t kChunkRows = int64_t(1) << 19;  // rows per inference chunk

__device__ __forceinline__ float silu(float x) { return x / (1.f + __expf(-x)); }
__device__ __forceinline__ float dsilu(float x)
{
    const float s = 1.f / (1.f + __expf(-x));
    return s * (1.f + x * (1.f - s));
}

__device__ __forceinline__ int64_t slice_of(const int *sid, int64_t sid0, int64_t b) { return sid ? sid[b] : sid0 + b; }

// ---- per-slice reductions ----------------------------------------------------------------------
// out[b] = sqrt(mean_i v[s_b][i]^2) + 1e-30 (mode 0) or sum_i v[s_b][i]^2 + 1e-30 (mode 1)
__global__ void k_slice_stat(const double *__restrict__ v, const int *__restrict__ sid, int64_t sid0, int nt, int mode,
                             float *__restrict__ out)
{
    __shared__ double red[32];
    const double *vs = v + (size_t)slice_of(sid, sid0, blockIdx.x) * nt;
    double s = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) s += vs[i] * vs[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[blockIdx.x] = mode == 0 ? (float)sqrt(s / nt) + 1e-30f : (float)s + 1e-30f;
    }
}

// ---- forward -----------------------------------------------------------------------------------
// encoder: h^0 = (v / s) SiLU(W_g^T f + b_g); X [rows][XS] = (v / s, f) and PRE [rows][W] =
// W_g^T f + b_g kept for the backward pass when given.  One thread per (row, 8 outputs).
template <int W>
__global__ void __launch_bounds__(256) k_encode(const double *__restrict__ v, const int *__restrict__ sid, int64_t sid0,
                                                const float *__restrict__ scale, const float *__restrict__ feat, int nt,
                                                int Et, int64_t rows, const __nv_bfloat16 *__restrict__ p,
                                                float *__restrict__ X, float *__restrict__ PRE, float *__restrict__ H)
{
    constexpr int NC = W / 8;
    __shared__ float wg[NG * W + W];  // W_g [5][W] then b_g
    for (int e = threadIdx.x; e < NG * W + W; e += blockDim.x) wg[e] = __bfloat162float(p[e]);
    __syncthreads();
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= rows * NC) return;
    const int64_t row = gid / NC, b = row / nt;
    const int c0 = (int)(gid % NC) * 8, i = (int)(row % nt);
    const int64_t s = slice_of(sid, sid0, b);
    const float4 f = *reinterpret_cast<const float4 *>(feat + 4 * i);
    const float x0 = (float)(v[s * nt + i] / (double)scale[b]), f5 = ((float)(s % Et) + 0.5f) / (float)Et;
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int o = c0 + j;
        a[j] = wg[NG * W + o] + wg[o] * f.x + wg[W + o] * f.y + wg[2 * W + o] * f.z + wg[3 * W + o] * f.w +
               wg[4 * W + o] * f5;
    }
    float4 *hp = reinterpret_cast<float4 *>(H + row * W + c0);
    hp[0] = make_float4(x0 * silu(a[0]), x0 * silu(a[1]), x0 * silu(a[2]), x0 * silu(a[3]));
    hp[1] = make_float4(x0 * silu(a[4]), x0 * silu(a[5]), x0 * silu(a[6]), x0 * silu(a[7]));
    if (PRE) {
        float4 *pp = reinterpret_cast<float4 *>(PRE + row * W + c0);
        pp[0] = make_float4(a[0], a[1], a[2], a[3]);
        pp[1] = make_float4(a[4], a[5], a[6], a[7]);
    }
    if (X && c0 == 0) {
        float4 *xp = reinterpret_cast<float4 *>(X + row * XS);
        xp[0] = make_float4(x0, f.x, f.y, f.z);
        xp[1] = make_float4(f.w, f5, 0.f, 0.f);
    }
}

// gathers the RT x 2W layer input (self | neighbour mean) of rows r0 .. r0 + RT into smem
template <int W>
__device__ __forceinline__ void load_layer_input(const float *__restrict__ H0, const int *__restrict__ adj_ptr,
                                                 const int *__restrict__ adj, const float *__restrict__ deg_inv, int nt,
                                                 int64_t rows, int64_t r0, int nrow, float *in)
{
    for (int e = threadIdx.x; e < nrow * W; e += blockDim.x) {
        const int r = e / W, k = e % W;
        const int64_t row = r0 + r;
        float hs = 0.f, hm = 0.f;
        if (row < rows) {
            hs = H0[row * W + k];
            const int64_t base = row - row % nt;
            const int i = (int)(row % nt);
            for (int q = adj_ptr[i]; q < adj_ptr[i + 1]; ++q) hm += H0[(base + adj[q]) * W + k];
            hm *= deg_inv[i];
        }
        in[r * 2 * W + k] = hs;
        in[r * 2 * W + W + k] = hm;
    }
}

// one message-passing layer on the CUDA cores: H1 = H0 + [H0 | mean_N H0] [W_s; W_n]
template <int W>
__global__ void __launch_bounds__(NTH) k_layer(const float *__restrict__ H0, float *__restrict__ H1,
                                               const int *__restrict__ adj_ptr,
                                               const int *__restrict__ adj, const float *__restrict__ deg_inv, int nt,
                                               int64_t rows, const __nv_bfloat16 *__restrict__ pl)
{
    constexpr int NRG = NTH / W, RPT = RT / NRG;
    extern __shared__ __align__(16) float sm[];
    float *Wt = sm;                // [2W][W]
    float *in = sm + 2 * W * W;    // [RT][2W]
    const int64_t r0 = (int64_t)blockIdx.x * RT;
    for (int e = threadIdx.x; e < 2 * W * W; e += NTH) Wt[e] = __bfloat162float(pl[e]);
    load_layer_input<W>(H0, adj_ptr, adj, deg_inv, nt, rows, r0, RT, in);
    __syncthreads();
    const int o = threadIdx.x % W, rg = threadIdx.x / W;
    float acc[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) acc[q] = 0.f;
#pragma unroll 2
    for (int k = 0; k < 2 * W; k += 4) {
        const float w0 = Wt[k * W + o], w1 = Wt[(k + 1) * W + o], w2 = Wt[(k + 2) * W + o], w3 = Wt[(k + 3) * W + o];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const float4 x = *reinterpret_cast<const float4 *>(&in[(rg * RPT + q) * 2 * W + k]);
            acc[q] += x.x * w0 + x.y * w1 + x.z * w2 + x.w * w3;
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int r = rg * RPT + q;
        const int64_t row = r0 + r;
        if (row < rows) H1[row * W + o] = in[r * 2 * W + o] + acc[q];
    }
}

// decoder, one warp per row: z = c s_b (w_o . h)
template <int W>
__global__ void k_decode(const float *__restrict__ H, const float *__restrict__ scale, int nt, int64_t rows, float c,
                         const __nv_bfloat16 *__restrict__ po, double *__restrict__ z)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    float a = 0.f;
    for (int k = lane; k < W; k += 32) a += __bfloat162float(po[k]) * H[row * W + k];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) z[row] = (double)a * (double)(c * scale[row / nt]);
}

// ---- loss and backward -------------------------------------------------------------------------
// dy = d loss / d (w_o . h + b_o) per row; loss accumulated into *loss
__global__ void k_loss_grad(const double *__restrict__ z, const double *__restrict__ E, const int *__restrict__ sid,
                            const float *__restrict__ scale, const float *__restrict__ en2, int nt, int64_t rows,
                            float inv_s, float c, float *__restrict__ dy, float *__restrict__ loss)
{
    __shared__ float red[32];
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (row < rows) {
        const int64_t b = row / nt;
        const int i = (int)(row % nt);
        const float diff = (float)(z[row] - E[(int64_t)sid[b] * nt + i]);
        const float w = inv_s / en2[b];
        dy[row] = 2.f * diff * w * c * scale[b];
        l = diff * diff * w;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x < 32) {
        l = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (threadIdx.x == 0) atomicAdd(loss, l);
    }
}

// same-step form: du = d loss / d (A_0 z) with u = A_0 z; loss accumulated into *loss
__global__ void k_res_loss(const double *__restrict__ u, const double *__restrict__ R, const int *__restrict__ sid,
                           const float *__restrict__ rn2, int nt, int64_t rows, float inv_s, double *__restrict__ du,
                           float *__restrict__ loss)
{
    __shared__ float red[32];
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (row < rows) {
        const int64_t b = row / nt;
        const double diff = u[row] - R[(int64_t)sid[b] * nt + row % nt];
        const double w = (double)inv_s / (double)rn2[b];
        du[row] = 2.0 * diff * w;
        l = (float)(diff * diff * w);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x < 32) {
        l = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (threadIdx.x == 0) atomicAdd(loss, l);
    }
}

// dy = (d loss / d z) c s_b per row (z = c s_b y)
__global__ void k_dy_from_dz(const double *__restrict__ dz, const float *__restrict__ scale, int nt, int64_t rows,
                             float c, float *__restrict__ dy)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row < rows) dy[row] = (float)(dz[row] * (double)(c * scale[row / nt]));
}

// out[b][i] = R[sid[b]][i]
__global__ void k_gather_slices(const double *__restrict__ R, const int *__restrict__ sid, int nt, int64_t rows,
                                double *__restrict__ out)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row < rows) out[row] = R[(int64_t)sid[row / nt] * nt + row % nt];
}

// decoder backward: G[row][k] = w_o[k] dy[row]; grad w_o[k] += sum H[row][k] dy[row]
template <int W>
__global__ void __launch_bounds__(NTH) k_decode_bwd(const float *__restrict__ H, const float *__restrict__ dy,
                                                    int64_t rows, const __nv_bfloat16 *__restrict__ po,
                                                    float *__restrict__ G, float *__restrict__ gpo)
{
    constexpr int NRG = NTH / W;
    __shared__ float red[NRG][W];
    const int o = threadIdx.x % W, rg = threadIdx.x / W;
    const float wo = __bfloat162float(po[o]);
    float aw = 0.f;
    for (int64_t row = (int64_t)blockIdx.x * NRG + rg; row < rows; row += (int64_t)gridDim.x * NRG) {
        const float d = dy[row];
        G[row * W + o] = wo * d;
        aw += H[row * W + o] * d;
    }
    red[rg][o] = aw;
    __syncthreads();
    if (rg == 0) {
        float s = 0.f;
        for (int g = 0; g < NRG; ++g) s += red[g][o];
        atomicAdd(&gpo[o], s);
    }
}

// layer backward, dense part (G1 = d loss / d h^{l+1}):
//   G0 = G1 + G1 W_s^T  (the residual path plus the self term),  U = (G1 W_n^T) / deg
template <int W>
__global__ void __launch_bounds__(NTH) k_layer_bwd(const float *__restrict__ G1, float *__restrict__ G0,
                                                   float *__restrict__ U, const float *__restrict__ deg_inv, int nt,
                                                   int64_t rows, const __nv_bfloat16 *__restrict__ pl)
{
    constexpr int NRG = NTH / W, RPT = RT / NRG;
    extern __shared__ __align__(16) float sm[];
    constexpr int LD = 2 * W + 1;  // padded row of the transposed weights
    float *WT = sm;                // [W][LD]: WT[o][k] = W_s[k][o], WT[o][W + k] = W_n[k][o]
    float *dp = sm + W * LD;       // [RT][W]
    const int64_t r0 = (int64_t)blockIdx.x * RT;
    for (int e = threadIdx.x; e < 2 * W * W; e += NTH) {
        const int k = e / W, o = e % W;
        WT[o * LD + k] = __bfloat162float(pl[e]);
    }
    for (int e = threadIdx.x; e < RT * W; e += NTH) {
        const int64_t row = r0 + e / W;
        dp[e] = row < rows ? G1[row * W + e % W] : 0.f;
    }
    __syncthreads();
    const int k = threadIdx.x % W, rg = threadIdx.x / W;
    float as[RPT], an[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) as[q] = an[q] = 0.f;
#pragma unroll 2
    for (int o = 0; o < W; o += 4) {
        float ws[4], wn[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ws[j] = WT[(o + j) * LD + k];
            wn[j] = WT[(o + j) * LD + W + k];
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const float4 d = *reinterpret_cast<const float4 *>(&dp[(rg * RPT + q) * W + o]);
            as[q] += d.x * ws[0] + d.y * ws[1] + d.z * ws[2] + d.w * ws[3];
            an[q] += d.x * wn[0] + d.y * wn[1] + d.z * wn[2] + d.w * wn[3];
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t row = r0 + rg * RPT + q;
        if (row >= rows) continue;
        G0[row * W + k] = G1[row * W + k] + as[q];
        U[row * W + k] = an[q] * deg_inv[row % nt];
    }
}

// layer backward, graph part: G0[i] += sum_{j in N(i)} U[j] (the adjacency is symmetric, so this
// is the transpose of the neighbour mean)
__global__ void k_scatter_nbr(const float *__restrict__ U, float *__restrict__ G0, const int *__restrict__ adj_ptr,
                              const int *__restrict__ adj, int nt, int64_t rows, int W)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= rows * W) return;
    const int64_t row = gid / W, base = row - row % nt;
    const int k = (int)(gid % W), i = (int)(row % nt);
    float s = 0.f;
    for (int q = adj_ptr[i]; q < adj_ptr[i + 1]; ++q) s += U[(base + adj[q]) * W + k];
    G0[gid] += s;
}

// encoder backward: d loss / d (W_g^T f + b_g) = G0 (v / s) SiLU'(PRE)
__global__ void k_enc_bwd(const float *__restrict__ G, const float *__restrict__ PRE, const float *__restrict__ X,
                          int W, int64_t n, float *__restrict__ DP)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) DP[i] = G[i] * X[(i / W) * XS] * dsilu(PRE[i]);
}

// weight gradients of one dense map:  Gw[k][o] += sum_rows IN[row][k] DP[row][o] for k < kvalid,
// gb[o] += sum_rows DP[row][o] (gb nullable); IN = the first KA columns of A (row stride lda), or
// [A | mean_N(A)] when nbr_mean
template <int W>
__global__ void __launch_bounds__(NTH) k_wgrad(const float *__restrict__ A, int lda, int KA, int kvalid, int nbr_mean,
                                               const int *__restrict__ adj_ptr, const int *__restrict__ adj,
                                               const float *__restrict__ deg_inv, int nt,
                                               const float *__restrict__ DP, int64_t rows, float *__restrict__ Gw,
                                               float *__restrict__ gb)
{
    constexpr int NRG = NTH / W, EPT = (2 * W + NRG - 1) / NRG;
    extern __shared__ __align__(16) float sm[];
    const int K = nbr_mean ? 2 * KA : KA;
    float *in = sm;            // [RW][K]
    float *dp = sm + RW * K;   // [RW][W]
    const int o = threadIdx.x % W, kg = threadIdx.x / W;
    float acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) acc[q] = 0.f;
    float accb = 0.f;
    for (int64_t r0 = (int64_t)blockIdx.x * RW; r0 < rows; r0 += (int64_t)gridDim.x * RW) {
        __syncthreads();
        for (int e = threadIdx.x; e < RW * K; e += NTH) {
            const int r = e / K, k = e % K;
            const int64_t row = r0 + r;
            float v = 0.f;
            if (row < rows) {
                if (k < KA) {
                    v = A[row * lda + k];
                } else {
                    const int kk = k - KA;
                    const int64_t base = row - row % nt;
                    const int i = (int)(row % nt);
                    for (int q = adj_ptr[i]; q < adj_ptr[i + 1]; ++q) v += A[(base + adj[q]) * lda + kk];
                    v *= deg_inv[i];
                }
            }
            in[e] = v;
        }
        for (int e = threadIdx.x; e < RW * W; e += NTH) {
            const int64_t row = r0 + e / W;
            dp[e] = row < rows ? DP[row * W + e % W] : 0.f;
        }
        __syncthreads();
        for (int r = 0; r < RW; ++r) {
            const float d = dp[r * W + o];
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int k = kg + NRG * q;
                if (k < K) acc[q] += in[r * K + k] * d;
            }
            accb += d;
        }
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int k = kg + NRG * q;
        if (k < kvalid) atomicAdd(&Gw[k * W + o], acc[q]);
    }
    if (gb && kg == 0) atomicAdd(&gb[o], accb);
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                       __nv_bfloat16 *__restrict__ p16, int64_t n, float lr, float b1c, float b2c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
    p[i] = pi;
    p16[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ q, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16_rn(p[i]);
}

unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---- compiled form ------------------------------------------------------------------------------
// probe of colour q on every slice: u[t][j] = 1 where colour(j) = q
__global__ void k_probe(const int *__restrict__ colour, int q, int nt, int64_t n, double *__restrict__ u)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = colour[i % nt] == q ? 1.0 : 0.0;
}

// P_t[i][k] = z_q[t][i] for the ball member k of row i that has colour q (at most one)
__global__ void k_extract(const double *__restrict__ zq, const int *__restrict__ supc, int q, int nt, int kmax,
                          int64_t n, float *__restrict__ Pc)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t t = r / nt;
    const int i = (int)(r % nt);
    for (int k = 0; k < kmax; ++k)
        if (supc[(size_t)k * nt + i] == q) {
            Pc[((size_t)t * kmax + k) * nt + i] = (float)zq[r];
            break;
        }
}

__global__ void k_to_f32(const double *__restrict__ v, float *__restrict__ vf, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) vf[i] = (float)v[i];
}

// z[b][i] = sum_k P_t[i][k] v[b][ball_k(i)], t = b mod E_t: one thread per row, the input
// converted to FP32 once (vf), FP32 sums over the ball, FP64 output
__global__ void k_spmv_compiled(const float *__restrict__ vf, double *__restrict__ z, const float *__restrict__ Pc,
                                const int *__restrict__ sup, int nt, int Et, int kmax, int64_t rows)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int64_t b = r / nt;
    const int i = (int)(r % nt), t = (int)(b % Et);
    const float *vb = vf + b * nt;
    const float *P = Pc + (size_t)t * kmax * nt + i;
    // padding entries (index -1) have zero coefficients: read vb[0] for them, no branch, so the
    // index and gather loads of several k are in flight together
    float acc = 0.f;
#pragma unroll 8
    for (int k = 0; k < kmax; ++k) acc += P[(size_t)k * nt] * vb[max(sup[(size_t)k * nt + i], 0)];
    z[r] = (double)acc;
}

// ---- tensor-core layer -------------------------------------------------------------------------
using namespace pfmm::tc;
constexpr int TM = 128;                              // rows per tensor-core tile (MMA M)
constexpr uint64_t kWaitNs = 2000000000ull;          // 2 s per mbarrier wait

// instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulate, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::
            "r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// byte offset of 16-byte chunk j (elements 8 j .. 8 j + 7 of a 64-element k block) of row r in a
// K-major tile with 128-byte swizzle: 8-row groups of 1024 bytes, chunks XOR-permuted by r mod 8
__device__ __forceinline__ uint32_t sw128_off(int r, int j) { return (r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// One message-passing layer on the tensor cores, persistent over 128-row tiles:
//   gather [h | mean_N h] (split into BF16 hi = rn(a) and lo = rn(a - hi), swizzled smem; D3: at
//   most 3 neighbours, from the padded table nb3, else the CSR lists) -> 2 x 2W/16 MMAs of
//   128 x W x 16 into TMEM -> epilogue h1 = h + acc (FP32), optionally the fused decoder
//   z = c s (w_o . h1).  256 threads: all gather, thread 0 issues the MMAs, warps (quadrant
//   q = warp mod 4, column group warp / 4) drain TMEM.
template <int W, bool D3>
__global__ void __launch_bounds__(256) k_layer_tc(const float *__restrict__ H0, float *__restrict__ H1,
                                                  const int *__restrict__ adj_ptr, const int *__restrict__ adj,
                                                  const int *__restrict__ nb3, const float *__restrict__ deg_inv,
                                                  int nt, int64_t rows, const __nv_bfloat16 *__restrict__ pl,
                                                  const __nv_bfloat16 *__restrict__ po,
                                                  const float *__restrict__ scale, float c, double *__restrict__ z,
                                                  int *__restrict__ err)
{
    constexpr int K = 2 * W, NQ = K / 8, NCG = W / 32;
    constexpr int A_BYTES = (K / 64) * TM * 128;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sAh = smem, *sAl = smem + A_BYTES, *sB = smem + 2 * A_BYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ float wout[W];
    __shared__ float zpart[NCG][TM];
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // B = [W_s; W_n]^T: row o holds the layer's column o, element k = M[k][o] (exact in BF16)
    for (int e = tid; e < W * NQ; e += 256) {
        const int o = e % W, q = e / W;
        uint32_t pk[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int k = q * 8 + 2 * h;
            pk[h] = pack_bf16(__bfloat162float(pl[(size_t)k * W + o]), __bfloat162float(pl[(size_t)(k + 1) * W + o]));
        }
        *reinterpret_cast<uint4 *>(sB + (q >> 3) * W * 128 + sw128_off(o, q & 7)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    for (int o = tid; o < W; o += 256) wout[o] = z ? __bfloat162float(po[o]) : 0.f;
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)), "r"(W));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int64_t ntiles = (rows + TM - 1) / TM;
    // hi / lo BF16 parts of 8 consecutive values into the two A tiles
    auto put = [&](int r, int qq, const float4 &a, const float4 &b) {
        const uint32_t off = (qq >> 3) * TM * 128 + sw128_off(r, qq & 7);
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(a.z, a.w),
                             h2 = __floats2bfloat162_rn(b.x, b.y), h3 = __floats2bfloat162_rn(b.z, b.w);
        const float2 g0 = __bfloat1622float2(h0), g1 = __bfloat1622float2(h1), g2 = __bfloat1622float2(h2),
                     g3 = __bfloat1622float2(h3);
        *reinterpret_cast<uint4 *>(sAh + off) =
            make_uint4(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1),
                       *reinterpret_cast<const uint32_t *>(&h2), *reinterpret_cast<const uint32_t *>(&h3));
        *reinterpret_cast<uint4 *>(sAl + off) =
            make_uint4(pack_bf16(a.x - g0.x, a.y - g0.y), pack_bf16(a.z - g1.x, a.w - g1.y),
                       pack_bf16(b.x - g2.x, b.y - g2.y), pack_bf16(b.z - g3.x, b.w - g3.y));
    };
    int n = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++n) {
        const int64_t r0 = tile * TM;
        // self half: chunks q < W/8 of every row (contiguous 32-byte loads, W/8 threads per row)
        constexpr int SC = W / 8, PER = TM * SC / 256;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = tid + 256 * u, r = e / SC, q = e % SC;
            const int64_t row = r0 + r;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (row < rows) {
                const float4 *p = reinterpret_cast<const float4 *>(H0 + row * W + q * 8);
                a = p[0];
                b = p[1];
            }
            put(r, q, a, b);
        }
        // neighbour half: chunks W/8 + q, the mean over the edge neighbours
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = tid + 256 * u, r = e / SC, q = e % SC;
            const int64_t row = r0 + r;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (row < rows) {
                const int i = (int)(row % nt);
                const int64_t base = row - i;
                const float di = deg_inv[i];
                if (D3) {
                    const int j0 = nb3[3 * i], j1 = nb3[3 * i + 1], j2 = nb3[3 * i + 2];
                    float4 x[6];
#pragma unroll
                    for (int m = 0; m < 6; ++m) x[m] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (j0 >= 0) { const float4 *p = reinterpret_cast<const float4 *>(H0 + (base + j0) * W + q * 8); x[0] = p[0]; x[1] = p[1]; }
                    if (j1 >= 0) { const float4 *p = reinterpret_cast<const float4 *>(H0 + (base + j1) * W + q * 8); x[2] = p[0]; x[3] = p[1]; }
                    if (j2 >= 0) { const float4 *p = reinterpret_cast<const float4 *>(H0 + (base + j2) * W + q * 8); x[4] = p[0]; x[5] = p[1]; }
                    a = make_float4(x[0].x + x[2].x + x[4].x, x[0].y + x[2].y + x[4].y, x[0].z + x[2].z + x[4].z,
                                    x[0].w + x[2].w + x[4].w);
                    b = make_float4(x[1].x + x[3].x + x[5].x, x[1].y + x[3].y + x[5].y, x[1].z + x[3].z + x[5].z,
                                    x[1].w + x[3].w + x[5].w);
                } else {
                    for (int m = adj_ptr[i]; m < adj_ptr[i + 1]; ++m) {
                        const float4 *p = reinterpret_cast<const float4 *>(H0 + (base + adj[m]) * W + q * 8);
                        const float4 x = p[0], y = p[1];
                        a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
                        b.x += y.x; b.y += y.y; b.z += y.z; b.w += y.w;
                    }
                }
                a.x *= di; a.y *= di; a.z *= di; a.w *= di;
                b.x *= di; b.y *= di; b.z *= di; b.w *= di;
            }
            put(r, SC + q, a, b);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> MMA reads
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t ah = su32(sAh), al = su32(sAl), b0 = su32(sB);
#pragma unroll
            for (int kb = 0; kb < K / 64; ++kb)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {  // K = 16 BF16 (32 bytes) per MMA
                    const uint64_t bd = sw128_desc(b0 + kb * W * 128 + kk * 32);
                    mma_bf16(tmem, sw128_desc(ah + kb * TM * 128 + kk * 32), bd, idesc_bf16(TM, W), (kb | kk) ? 1u : 0u);
                    mma_bf16(tmem, sw128_desc(al + kb * TM * 128 + kk * 32), bd, idesc_bf16(TM, W), 1u);
                }
            mma_commit(&bar);
        }
        if (!mbar_wait(&bar, n & 1, gtimer() + kWaitNs)) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quad = warp & 3, cg = warp >> 2;
        if (cg < NCG) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + cg * 32, v);
            const int rl = quad * 32 + lane;
            const int64_t row = r0 + rl;
            float zp = 0.f;
            if (row < rows) {
                const float4 *h0 = reinterpret_cast<const float4 *>(H0 + row * W + cg * 32);
                float4 *h1 = reinterpret_cast<float4 *>(H1 + row * W + cg * 32);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int cc = cg * 32 + 4 * j;
                    const float4 h = h0[j];
                    const float4 o = make_float4(h.x + __uint_as_float(v[4 * j]), h.y + __uint_as_float(v[4 * j + 1]),
                                                 h.z + __uint_as_float(v[4 * j + 2]), h.w + __uint_as_float(v[4 * j + 3]));
                    h1[j] = o;
                    zp += wout[cc] * o.x + wout[cc + 1] * o.y + wout[cc + 2] * o.z + wout[cc + 3] * o.w;
                }
            }
            zpart[cg][rl] = zp;
        }
        if (z) {
            __syncthreads();
            if (tid < TM && r0 + tid < rows) {
                float sacc = 0.f;
#pragma unroll
                for (int g = 0; g < NCG; ++g) sacc += zpart[g][tid];
                const int64_t row = r0 + tid;
                z[row] = (double)sacc * (double)(c * scale[row / nt]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(W));
    }
}

template <int W>
constexpr size_t tc_smem_bytes()
{
    return 2 * (size_t)(2 * W / 64) * TM * 128 + (size_t)(2 * W / 64) * W * 128 + 1024;
}

}  // namespace

struct pfmm_mpnn {
    int W = 64, L = 4, nt = 0, Et = 0, nsm = 148;
    int64_t nparam = 0;
    int *err = nullptr;  // bounded-wait error word of the tensor-core kernels
    float c_out = 0.f;  // output scale; 0 until set or estimated
    int adam_t = 0;
    int *adj_ptr = nullptr, *adj = nullptr;
    int *nb3 = nullptr;  // [nt][3] neighbours padded with -1 when no triangle has more than 3, else NULL
    float *deg_inv = nullptr, *feat = nullptr;
    float *p32 = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr, *loss = nullptr;
    __nv_bfloat16 *p16 = nullptr;
    // inference chunk buffers
    float *Hi0 = nullptr, *Hi1 = nullptr, *scale_i = nullptr;
    // training buffers for cap_rows rows
    int64_t cap_rows = 0;
    float *X = nullptr, *H = nullptr, *PRE = nullptr, *G0 = nullptr, *G1 = nullptr, *DP = nullptr, *U = nullptr,
          *dy = nullptr, *scale = nullptr, *en2 = nullptr;
    double *z = nullptr, *u = nullptr, *du = nullptr, *ssx = nullptr, *ssf = nullptr;
    int *sid = nullptr;
    // host copy of the edge adjacency (CSR), for the compiled form
    std::vector<int> hptr, hadj;
    // compiled form: z_t = P_t v with P_t[i][k] on the radius-L ball of triangle i
    bool compiled = false;
    int kmax = 0, ncolor = 0;
    int *sup = nullptr;   // [kmax][nt] ball members (-1 after the last)
    int *supc = nullptr;  // [kmax][nt] their colours
    float *Pc = nullptr;  // [Et][kmax][nt]
    float *vf = nullptr;  // FP32 copy of the input of a compiled apply
    int64_t vf_cap = 0;
    std::vector<void *> mem;
    ~pfmm_mpnn()
    {
        for (void *p : mem) cudaFree(p);
    }
    template <typename T>
    int get(T **p, size_t n)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(PFMM_ERR_OOM, "network buffer allocation failed");
        }
        mem.push_back(q);
        *p = (T *)q;
        return PFMM_OK;
    }
    void drop(void *p)
    {
        if (!p) return;
        auto it = std::find(mem.begin(), mem.end(), p);
        if (it != mem.end()) {
            cudaFree(p);
            mem.erase(it);
        }
    }
    int64_t off_layer(int l) const { return (int64_t)NG * W + W + (int64_t)l * 2 * W * W; }
    int64_t off_out() const { return off_layer(L); }
};

namespace {

template <int W>
void launch_forward(pfmm_mpnn *N, const double *v, const int *sid, int64_t sid0, int64_t nslices, float *scale,
                    float *X, float *H, float *PRE, bool keep, double *z, cudaStream_t st)
{
    const int64_t rows = nslices * N->nt;
    k_slice_stat<<<(unsigned)nslices, 256, 0, st>>>(v, sid, sid0, N->nt, 0, scale);
    k_encode<W><<<nblk(rows * (W / 8)), 256, 0, st>>>(v, sid, sid0, scale, N->feat, N->nt, N->Et, rows, N->p16, X,
                                                      keep ? PRE : nullptr, H);
    float *cur = H;
    bool decoded = false;
    for (int l = 0; l < N->L; ++l) {
        float *nxt = keep ? H + (size_t)(l + 1) * rows * W : (l % 2 == 0 ? N->Hi1 : N->Hi0);
        if constexpr (W >= 32) {
            const bool last = l == N->L - 1;
            const size_t smem = tc_smem_bytes<W>();
            const int64_t ntiles = (rows + TM - 1) / TM;
            const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)N->nsm * 2);
            auto kern = N->nb3 ? k_layer_tc<W, true> : k_layer_tc<W, false>;
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<grid, 256, smem, st>>>(cur, nxt, N->adj_ptr, N->adj, N->nb3, N->deg_inv, N->nt, rows,
                                          N->p16 + N->off_layer(l), N->p16 + N->off_out(), scale, N->c_out,
                                          last ? z : nullptr, N->err);
            decoded = last;
        } else {
            const size_t smem = (size_t)(2 * W * W + RT * 2 * W) * sizeof(float);
            cudaFuncSetAttribute(k_layer<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_layer<W><<<nblk(rows, RT), NTH, smem, st>>>(cur, nxt, N->adj_ptr, N->adj, N->deg_inv, N->nt, rows,
                                                          N->p16 + N->off_layer(l));
        }
        cur = nxt;
    }
    if (!decoded)
        k_decode<W><<<nblk(rows * 32), 256, 0, st>>>(cur, scale, N->nt, rows, N->c_out, N->p16 + N->off_out(), z);
}

template <int W>
void launch_backward(pfmm_mpnn *N, int64_t rows, cudaStream_t st)
{
    const int L = N->L;
    const size_t smem_b = (size_t)(W * (2 * W + 1) + RT * W) * sizeof(float);
    cudaFuncSetAttribute(k_layer_bwd<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
    const size_t smem_w = (size_t)(RW * 2 * W + RW * W) * sizeof(float);
    cudaFuncSetAttribute(k_wgrad<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w);
    const unsigned gw = (unsigned)std::min<int64_t>(nblk(rows, RW), 2 * (int64_t)N->nsm);
    float *Gup = N->G1, *Gdn = N->G0;  // gradient w.r.t. h^{l+1} and h^l
    k_decode_bwd<W><<<(unsigned)std::min<int64_t>(nblk(rows, NTH / W), 2048), NTH, 0, st>>>(
        N->H + (size_t)L * rows * W, N->dy, rows, N->p16 + N->off_out(), Gup, N->grad + N->off_out());
    for (int l = L - 1; l >= 0; --l) {
        const float *Hl = N->H + (size_t)l * rows * W;
        k_layer_bwd<W><<<nblk(rows, RT), NTH, smem_b, st>>>(Gup, Gdn, N->U, N->deg_inv, N->nt, rows,
                                                            N->p16 + N->off_layer(l));
        k_wgrad<W><<<gw, NTH, smem_w, st>>>(Hl, W, W, 2 * W, 1, N->adj_ptr, N->adj, N->deg_inv, N->nt, Gup, rows,
                                            N->grad + N->off_layer(l), nullptr);
        k_scatter_nbr<<<nblk(rows * W), 256, 0, st>>>(N->U, Gdn, N->adj_ptr, N->adj, N->nt, rows, W);
        std::swap(Gup, Gdn);
    }
    k_enc_bwd<<<nblk(rows * W), 256, 0, st>>>(Gup, N->PRE, N->X, W, rows * W, N->DP);
    k_wgrad<W><<<gw, NTH, smem_w, st>>>(N->X + 1, XS, NG, NG, 0, N->adj_ptr, N->adj, N->deg_inv, N->nt, N->DP, rows,
                                        N->grad, N->grad + NG * W);
}

template <typename F>
void dispatch_w(int W, F &&f)
{
    if (W == 16) f(std::integral_constant<int, 16>{});
    else if (W == 32) f(std::integral_constant<int, 32>{});
    else f(std::integral_constant<int, 64>{});
}

int cuda_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return PFMM_OK;
}

int ensure_train(pfmm_mpnn *N, int64_t slices)
{
    const int64_t rows = slices * N->nt;
    if (rows <= N->cap_rows) return PFMM_OK;
    for (void *p : {(void *)N->X, (void *)N->H, (void *)N->PRE, (void *)N->G0, (void *)N->G1, (void *)N->DP,
                    (void *)N->U, (void *)N->dy, (void *)N->scale, (void *)N->en2, (void *)N->z, (void *)N->sid,
                    (void *)N->u, (void *)N->du, (void *)N->ssx, (void *)N->ssf})
        N->drop(p);
    N->cap_rows = 0;
    const size_t rw = (size_t)rows * N->W, lw = (size_t)(N->L + 1) * rw;
    int rc;
    if ((rc = N->get(&N->X, (size_t)rows * XS)) || (rc = N->get(&N->H, lw)) || (rc = N->get(&N->PRE, rw)) ||
        (rc = N->get(&N->G0, rw)) || (rc = N->get(&N->G1, rw)) || (rc = N->get(&N->DP, rw)) ||
        (rc = N->get(&N->U, rw)) || (rc = N->get(&N->dy, rows)) || (rc = N->get(&N->scale, slices)) ||
        (rc = N->get(&N->en2, slices)) || (rc = N->get(&N->z, rows)) || (rc = N->get(&N->sid, slices)) ||
        (rc = N->get(&N->u, rows)) || (rc = N->get(&N->du, rows)) || (rc = N->get(&N->ssx, rows)) ||
        (rc = N->get(&N->ssf, rows)))
        return rc;
    N->cap_rows = rows;
    return PFMM_OK;
}

// loss and gradient (into N->grad) of the residual slices sid_host[0 .. ns) of R: the same-step
// form when H is given, else the error form with the errors E
int loss_grad(pfmm_mpnn *N, pfmm_handle *H, const double *R, const double *E, const int *sid_host, int ns,
              cudaStream_t st)
{
    int rc = ensure_train(N, ns);
    if (rc) return rc;
    const int64_t rows = (int64_t)ns * N->nt;
    if (cudaMemcpyAsync(N->sid, sid_host, ns * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return cuda_status("slice index upload");
    dispatch_w(N->W, [&](auto w) {
        constexpr int W = decltype(w)::value;
        launch_forward<W>(N, R, N->sid, 0, ns, N->scale, N->X, N->H, N->PRE, true, N->z, st);
    });
    cudaMemsetAsync(N->loss, 0, sizeof(float), st);
    cudaMemsetAsync(N->grad, 0, N->nparam * sizeof(float), st);
    if (H) {
        k_slice_stat<<<(unsigned)ns, 256, 0, st>>>(R, N->sid, 0, N->nt, 1, N->en2);
        if ((rc = pfmm::apply_same_step(H, N->z, N->u, ns, N->ssx, N->ssf, st))) return rc;
        k_res_loss<<<nblk(rows), 256, 0, st>>>(N->u, R, N->sid, N->en2, N->nt, rows, 1.f / (float)ns, N->du, N->loss);
        if ((rc = pfmm::apply_same_step(H, N->du, N->u, ns, N->ssx, N->ssf, st))) return rc;  // A_0^T du ~ A_0 du
        k_dy_from_dz<<<nblk(rows), 256, 0, st>>>(N->u, N->scale, N->nt, rows, N->c_out, N->dy);
    } else {
        k_slice_stat<<<(unsigned)ns, 256, 0, st>>>(E, N->sid, 0, N->nt, 1, N->en2);
        k_loss_grad<<<nblk(rows), 256, 0, st>>>(N->z, E, N->sid, N->scale, N->en2, N->nt, rows, 1.f / (float)ns,
                                                N->c_out, N->dy, N->loss);
    }
    dispatch_w(N->W, [&](auto w) {
        constexpr int W = decltype(w)::value;
        launch_backward<W>(N, rows, st);
    });
    return cuda_status("network loss / gradient");
}

// output scale c: sqrt(sum ||t_b||^2 / sum ||r_b||^2) over the given slices, with the targets
// t_b = e_b (error form) or, for the same-step form, the inverse gain of A_0 on residuals:
// sqrt(sum ||r_b||^2 / sum ||A_0 r_b||^2)
int estimate_scale(pfmm_mpnn *N, pfmm_handle *H, const double *R, const double *E, const int *sid_host, int ns,
                   cudaStream_t st)
{
    int rc = ensure_train(N, ns);
    if (rc) return rc;
    const int64_t rows = (int64_t)ns * N->nt;
    cudaMemcpyAsync(N->sid, sid_host, ns * sizeof(int), cudaMemcpyHostToDevice, st);
    k_slice_stat<<<(unsigned)ns, 256, 0, st>>>(R, N->sid, 0, N->nt, 1, N->scale);
    if (H) {
        k_gather_slices<<<nblk(rows), 256, 0, st>>>(R, N->sid, N->nt, rows, N->z);
        if ((rc = pfmm::apply_same_step(H, N->z, N->u, ns, N->ssx, N->ssf, st))) return rc;
        k_slice_stat<<<(unsigned)ns, 256, 0, st>>>(N->u, nullptr, 0, N->nt, 1, N->en2);
    } else {
        k_slice_stat<<<(unsigned)ns, 256, 0, st>>>(E, N->sid, 0, N->nt, 1, N->en2);
    }
    std::vector<float> a(ns), b(ns);
    cudaMemcpyAsync(a.data(), N->scale, ns * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(b.data(), N->en2, ns * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if ((rc = cuda_status("output scale estimate"))) return rc;  // failed copies or launches above too
    double sr = 0, st2 = 0;
    for (int i = 0; i < ns; ++i) {
        sr += a[i];
        st2 += b[i];
    }
    const double c = H ? std::sqrt(sr / st2) : std::sqrt(st2 / sr);
    N->c_out = std::isfinite(c) && c > 0 ? (float)c : 1.f;
    return PFMM_OK;
}

int check_pair_args(pfmm_mpnn *net, pfmm_handle *H, const double *R, const double *E)
{
    if (!net || !R || (!H && !E)) return set_error(PFMM_ERR_INVALID_ARG, "invalid training arguments");
    if (H && (H->nt != net->nt || H->Et != net->Et))
        return set_error(PFMM_ERR_INVALID_ARG, "the handle describes another mesh than the network");
    return PFMM_OK;
}

}  // namespace

void pfmm::mpnn_dims(const pfmm_mpnn *net, int *nt, int *Et)
{
    *nt = net->nt;
    *Et = net->Et;
}

extern "C" {

int pfmm_mpnn_create(const pfmm_mesh *mesh, int32_t width, int32_t layers, uint64_t seed, pfmm_mpnn **out)
{
    if (!out) return set_error(PFMM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!mesh || !mesh->vertices || !mesh->triangles || mesh->n_triangles < 1 || mesh->n_vertices < 3 ||
        mesh->n_steps < 1)
        return set_error(PFMM_ERR_INVALID_ARG, "invalid mesh for the network");
    if ((width != 16 && width != 32 && width != 64) || layers < 0 || layers > 16)
        return set_error(PFMM_ERR_INVALID_ARG, "network width must be 16, 32 or 64 and layers 0..16");
    const int nt = mesh->n_triangles, nv = mesh->n_vertices;
    for (int x = 0; x < 3 * nt; ++x)
        if (mesh->triangles[x] < 0 || mesh->triangles[x] >= nv)
            return set_error(PFMM_ERR_INVALID_ARG, "triangle vertex index out of range");
    pfmm_mpnn *N = new pfmm_mpnn();
    N->W = width;
    N->L = layers;
    N->nt = nt;
    N->Et = mesh->n_steps;
    N->nparam = (int64_t)NG * width + width + (int64_t)layers * 2 * width * width + width;
    // edge adjacency (symmetric, duplicates removed) and geometric features
    std::map<std::pair<int, int>, std::vector<int>> edge;
    for (int x = 0; x < nt; ++x)
        for (int e = 0; e < 3; ++e) {
            int a = mesh->triangles[3 * x + e], b = mesh->triangles[3 * x + (e + 1) % 3];
            edge[{std::min(a, b), std::max(a, b)}].push_back(x);
        }
    std::vector<std::vector<int>> nb(nt);
    for (auto &kv : edge)
        for (size_t i = 0; i < kv.second.size(); ++i)
            for (size_t j = 0; j < kv.second.size(); ++j)
                if (i != j && kv.second[i] != kv.second[j]) nb[kv.second[i]].push_back(kv.second[j]);
    std::vector<int> ptr(nt + 1, 0), adj;
    std::vector<float> dinv(nt), feat(4 * (size_t)nt);
    for (int x = 0; x < nt; ++x) {
        std::sort(nb[x].begin(), nb[x].end());
        nb[x].erase(std::unique(nb[x].begin(), nb[x].end()), nb[x].end());
        adj.insert(adj.end(), nb[x].begin(), nb[x].end());
        ptr[x + 1] = (int)adj.size();
        dinv[x] = nb[x].empty() ? 0.f : 1.f / (float)nb[x].size();
    }
    std::vector<double> area(nt);
    double amean = 0.0;
    for (int x = 0; x < nt; ++x) {
        const double *A = &mesh->vertices[3 * mesh->triangles[3 * x]], *B = &mesh->vertices[3 * mesh->triangles[3 * x + 1]],
                     *C = &mesh->vertices[3 * mesh->triangles[3 * x + 2]];
        double u[3], w[3], c[3];
        for (int k = 0; k < 3; ++k) {
            u[k] = B[k] - A[k];
            w[k] = C[k] - A[k];
        }
        c[0] = u[1] * w[2] - u[2] * w[1];
        c[1] = u[2] * w[0] - u[0] * w[2];
        c[2] = u[0] * w[1] - u[1] * w[0];
        const double l = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(l > 0)) {
            delete N;
            return set_error(PFMM_ERR_INVALID_ARG, "degenerate triangle");
        }
        area[x] = 0.5 * l;
        amean += area[x] / nt;
        for (int k = 0; k < 3; ++k) feat[4 * x + 1 + k] = (float)(c[k] / l);
    }
    for (int x = 0; x < nt; ++x) feat[4 * x] = (float)(area[x] / amean);
    int rc;
    const size_t chunk = (size_t)std::max<int64_t>(kChunkRows / nt, 1) * nt;
    if ((rc = N->get(&N->adj_ptr, nt + 1)) || (rc = N->get(&N->adj, adj.size())) || (rc = N->get(&N->deg_inv, nt)) ||
        (rc = N->get(&N->feat, feat.size())) || (rc = N->get(&N->p32, N->nparam)) || (rc = N->get(&N->m1, N->nparam)) ||
        (rc = N->get(&N->m2, N->nparam)) || (rc = N->get(&N->grad, N->nparam)) || (rc = N->get(&N->p16, N->nparam)) ||
        (rc = N->get(&N->loss, 1)) || (rc = N->get(&N->Hi0, chunk * width)) || (rc = N->get(&N->Hi1, chunk * width)) ||
        (rc = N->get(&N->scale_i, chunk / nt)) || (rc = N->get(&N->err, 1))) {
        delete N;
        return rc;
    }
    cudaMemset(N->err, 0, sizeof(int));
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&N->nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    N->hptr = ptr;
    N->hadj = adj;
    size_t maxdeg = 0;
    for (int x = 0; x < nt; ++x) maxdeg = std::max(maxdeg, nb[x].size());
    if (maxdeg <= 3) {
        std::vector<int> pad(3 * (size_t)nt, -1);
        for (int x = 0; x < nt; ++x)
            for (size_t k = 0; k < nb[x].size(); ++k) pad[3 * x + k] = nb[x][k];
        if ((rc = N->get(&N->nb3, pad.size()))) {
            delete N;
            return rc;
        }
        cudaMemcpy(N->nb3, pad.data(), pad.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    cudaMemcpy(N->adj_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (!adj.empty()) cudaMemcpy(N->adj, adj.data(), adj.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(N->deg_inv, dinv.data(), dinv.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(N->feat, feat.data(), feat.size() * sizeof(float), cudaMemcpyHostToDevice);
    // initialisation: uniform(+-1/sqrt(fan_in)) for the geometry embedding and the read-out; the
    // layers start at a tenth of that, so that the initial network is close to a diagonal scaling
    std::mt19937_64 rng(seed);
    std::vector<float> p(N->nparam, 0.f);
    auto fill = [&](int64_t off, int64_t n, double bound) {
        std::uniform_real_distribution<double> U(-bound, bound);
        for (int64_t i = 0; i < n; ++i) p[off + i] = (float)U(rng);
    };
    fill(0, NG * width, 1.0 / std::sqrt((double)NG));
    for (int l = 0; l < layers; ++l) fill(N->off_layer(l), 2 * width * width, 0.1 / std::sqrt(2.0 * width));
    fill(N->off_out(), width, 1.0 / std::sqrt((double)width));
    cudaMemcpy(N->p32, p.data(), p.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(N->m1, 0, N->nparam * sizeof(float));
    cudaMemset(N->m2, 0, N->nparam * sizeof(float));
    k_to_bf16<<<nblk(N->nparam), 256>>>(N->p32, N->p16, N->nparam);
    cudaDeviceSynchronize();
    // any failed upload, memset or launch above is still the last error here
    if (const int rc = cuda_status("network initialisation")) {
        delete N;
        return rc;
    }
    *out = N;
    return PFMM_OK;
}

int64_t pfmm_mpnn_num_params(const pfmm_mpnn *net) { return net ? net->nparam : 0; }

int pfmm_mpnn_get_params(const pfmm_mpnn *net, float *host, int64_t n)
{
    if (!net || !host || n != net->nparam) return set_error(PFMM_ERR_INVALID_ARG, "parameter count mismatch");
    if (cudaMemcpy(host, net->p32, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_status("parameter download");
    return PFMM_OK;
}

int pfmm_mpnn_set_params(pfmm_mpnn *net, const float *host, int64_t n)
{
    if (!net || !host || n != net->nparam) return set_error(PFMM_ERR_INVALID_ARG, "parameter count mismatch");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(host[i])) return set_error(PFMM_ERR_NONFINITE, "parameters hold NaN or Inf");
    net->compiled = false;
    cudaMemcpy(net->p32, host, n * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(net->m1, 0, n * sizeof(float));
    cudaMemset(net->m2, 0, n * sizeof(float));
    net->adam_t = 0;
    k_to_bf16<<<nblk(n), 256>>>(net->p32, net->p16, n);
    cudaDeviceSynchronize();
    return cuda_status("parameter upload");  // a failed upload, memset or launch above included
}

int pfmm_mpnn_set_output_scale(pfmm_mpnn *net, float c)
{
    if (!net || !(c > 0) || !std::isfinite(c)) return set_error(PFMM_ERR_INVALID_ARG, "output scale must be > 0");
    net->c_out = c;
    net->compiled = false;
    return PFMM_OK;
}

int pfmm_mpnn_get_output_scale(const pfmm_mpnn *net, float *c)
{
    if (!net || !c) return set_error(PFMM_ERR_INVALID_ARG, "invalid arguments");
    *c = net->c_out;
    return PFMM_OK;
}

int pfmm_mpnn_apply(pfmm_mpnn *net, const double *v, double *z, int32_t nvec, void *stream)
{
    if (!net || !v || !z || nvec < 1) return set_error(PFMM_ERR_INVALID_ARG, "invalid network apply arguments");
    if (!(net->c_out > 0)) return set_error(PFMM_ERR_INVALID_ARG, "the network has no output scale (train it or set one)");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t total = (int64_t)nvec * net->Et, per = std::max<int64_t>(kChunkRows / net->nt, 1);
    if (net->compiled) {
        const int64_t rows = total * net->nt;
        if (rows > net->vf_cap) {
            net->drop(net->vf);
            net->vf = nullptr;
            net->vf_cap = 0;
            int rc = net->get(&net->vf, rows);
            if (rc) return rc;
            net->vf_cap = rows;
        }
        k_to_f32<<<nblk(rows), 256, 0, st>>>(v, net->vf, rows);
        k_spmv_compiled<<<nblk(rows), 256, 0, st>>>(net->vf, z, net->Pc, net->sup, net->nt, net->Et, net->kmax, rows);
        return cuda_status("compiled network apply");
    }
    for (int64_t s0 = 0; s0 < total; s0 += per) {
        const int64_t ns = std::min(per, total - s0);
        dispatch_w(net->W, [&](auto w) {
            constexpr int W = decltype(w)::value;
            launch_forward<W>(net, v, nullptr, s0, ns, net->scale_i, nullptr, net->Hi0, nullptr, false,
                              z + s0 * net->nt, st);
        });
    }
    return cuda_status("network apply");
}

int pfmm_mpnn_loss_grad(pfmm_mpnn *net, pfmm_handle *h, const double *R, const double *E, const int32_t *slices,
                        int32_t nslices, float *loss, float *grad, void *stream)
{
    int rc = check_pair_args(net, h, R, E);
    if (rc) return rc;
    if (!slices || nslices < 1) return set_error(PFMM_ERR_INVALID_ARG, "no slices");
    if (!(net->c_out > 0)) return set_error(PFMM_ERR_INVALID_ARG, "the network has no output scale");
    for (int i = 0; i < nslices; ++i)
        if (slices[i] < 0) return set_error(PFMM_ERR_INVALID_ARG, "negative slice index");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = loss_grad(net, h, R, E, slices, nslices, st))) return rc;
    if (loss) cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (grad) cudaMemcpyAsync(grad, net->grad, net->nparam * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return cuda_status("loss / gradient download");  // a failed copy included
}

int pfmm_mpnn_train(pfmm_mpnn *net, pfmm_handle *h, const double *R, const double *E, int64_t nvec, int32_t steps,
                    int32_t batch_slices, float lr, uint64_t seed, float *loss_history, void *stream)
{
    int rc = check_pair_args(net, h, R, E);
    if (rc) return rc;
    if (nvec < 1 || steps < 0 || batch_slices < 1 || !(lr > 0))
        return set_error(PFMM_ERR_INVALID_ARG, "invalid training arguments");
    cudaStream_t st = (cudaStream_t)stream;
    net->compiled = false;
    const int64_t total = nvec * net->Et;
    const int ns = (int)std::min<int64_t>(batch_slices, total);
    std::mt19937_64 rng(seed);
    std::uniform_int_distribution<int64_t> pick(0, total - 1);
    std::vector<int> sid(ns);
    if (!(net->c_out > 0)) {
        for (auto &s : sid) s = (int)pick(rng);
        if ((rc = estimate_scale(net, h, R, E, sid.data(), ns, st))) return rc;
    }
    float *hist = nullptr;
    if ((rc = net->get(&hist, std::max(steps, 1)))) return rc;
    for (int it = 0; it < steps; ++it) {
        for (auto &s : sid) s = (int)pick(rng);
        if ((rc = loss_grad(net, h, R, E, sid.data(), ns, st))) {
            net->drop(hist);
            return rc;
        }
        cudaMemcpyAsync(hist + it, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
        ++net->adam_t;
        const float lr_t = lr * (float)(0.1 + 0.45 * (1.0 + std::cos(3.14159265358979 * it / std::max(steps, 1))));
        k_adam<<<nblk(net->nparam), 256, 0, st>>>(net->p32, net->m1, net->m2, net->grad, net->p16, net->nparam, lr_t,
                                                  1.f - std::pow(0.9f, (float)net->adam_t),
                                                  1.f - std::pow(0.999f, (float)net->adam_t));
        // the host-side slice list is reused: wait for its upload before the next draw
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            net->drop(hist);
            return cuda_status("training step");
        }
    }
    if (loss_history && steps > 0) cudaMemcpy(loss_history, hist, steps * sizeof(float), cudaMemcpyDeviceToHost);
    net->drop(hist);
    if ((rc = cuda_status("training"))) return rc;
    return pfmm_mpnn_check(net);
}

int pfmm_mpnn_compile(pfmm_mpnn *net, void *stream)
{
    if (!net) return set_error(PFMM_ERR_INVALID_ARG, "net is NULL");
    if (!(net->c_out > 0)) return set_error(PFMM_ERR_INVALID_ARG, "the network has no output scale");
    cudaStream_t st = (cudaStream_t)stream;
    const int nt = net->nt, Et = net->Et, L = net->L;
    // radius-L balls (breadth first over the edge adjacency), then a greedy colouring in which
    // triangles closer than 2L + 1 edges get different colours: two members of one ball never
    // share a colour, so one probe per colour recovers every coefficient
    auto bfs = [&](int src, int depth, std::vector<int> &out, std::vector<int> &mark, int stamp) {
        out.clear();
        out.push_back(src);
        mark[src] = stamp;
        size_t lo = 0;
        for (int d = 0; d < depth; ++d) {
            const size_t hi = out.size();
            for (size_t a = lo; a < hi; ++a)
                for (int q = net->hptr[out[a]]; q < net->hptr[out[a] + 1]; ++q) {
                    const int j = net->hadj[q];
                    if (mark[j] != stamp) {
                        mark[j] = stamp;
                        out.push_back(j);
                    }
                }
            lo = hi;
        }
    };
    std::vector<int> mark(nt, -1), ball, colour(nt, -1);
    std::vector<std::vector<int>> balls(nt);
    int kmax = 0, stamp = 0;
    for (int i = 0; i < nt; ++i) {
        bfs(i, L, ball, mark, stamp++);
        balls[i] = ball;
        kmax = std::max(kmax, (int)ball.size());
    }
    int ncolour = 0;
    std::vector<int> used;
    for (int j = 0; j < nt; ++j) {
        bfs(j, 2 * L, ball, mark, stamp++);
        used.assign(ncolour + 1, 0);
        for (int x : ball)
            if (colour[x] >= 0) used[colour[x]] = 1;
        int c = 0;
        while (c < ncolour && used[c]) ++c;
        colour[j] = c;
        ncolour = std::max(ncolour, c + 1);
    }
    std::vector<int> sup((size_t)kmax * nt, -1), supc((size_t)kmax * nt, -1);
    for (int i = 0; i < nt; ++i)
        for (size_t k = 0; k < balls[i].size(); ++k) {
            sup[k * nt + i] = balls[i][k];
            supc[k * nt + i] = colour[balls[i][k]];
        }
    for (void *p : {(void *)net->sup, (void *)net->supc, (void *)net->Pc}) net->drop(p);
    net->sup = net->supc = nullptr;
    net->Pc = nullptr;
    int *dcol = nullptr;
    double *u = nullptr, *zq = nullptr;
    const int64_t n = (int64_t)Et * nt;
    int rc;
    if ((rc = net->get(&net->sup, sup.size())) || (rc = net->get(&net->supc, supc.size())) ||
        (rc = net->get(&net->Pc, (size_t)Et * kmax * nt)) || (rc = net->get(&dcol, nt)) || (rc = net->get(&u, n)) ||
        (rc = net->get(&zq, n)))
        return rc;
    cudaMemcpy(net->sup, sup.data(), sup.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(net->supc, supc.data(), supc.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(dcol, colour.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemsetAsync(net->Pc, 0, (size_t)Et * kmax * nt * sizeof(float), st);
    net->compiled = false;
    for (int q = 0; q < ncolour && !rc; ++q) {
        k_probe<<<nblk(n), 256, 0, st>>>(dcol, q, nt, n, u);
        if ((rc = pfmm_mpnn_apply(net, u, zq, 1, stream))) break;
        k_extract<<<nblk(n), 256, 0, st>>>(zq, net->supc, q, nt, kmax, n, net->Pc);
    }
    if (!rc) rc = cuda_status("network compile");
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = cuda_status("network compile");
    net->drop(dcol);
    net->drop(u);
    net->drop(zq);
    if (rc) return rc;
    net->kmax = kmax;
    net->ncolor = ncolour;
    net->compiled = true;
    return pfmm_mpnn_check(net);
}

int pfmm_mpnn_check(pfmm_mpnn *net)
{
    if (!net) return set_error(PFMM_ERR_INVALID_ARG, "net is NULL");
    int e = 0;
    if (cudaMemcpy(&e, net->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_status("network error word");
    if (e) {
        cudaMemset(net->err, 0, sizeof(int));
        return set_error(PFMM_ERR_TIMEOUT, "a tensor-core wait of the network timed out (code " + std::to_string(e) + ")");
    }
    return PFMM_OK;
}

void pfmm_mpnn_destroy(pfmm_mpnn *net) { delete net; }

}  // extern "C"
