// k_nf_tc.cu -- nearfield apply (Alg. 2, last loop; Eq. eval_sl_nf_block) on the sm_103a
// tensor cores: tcgen05.mma (kind::f16, FP16 operands) with TMA-staged operands and TMEM
// accumulators.
//
// The block-Toeplitz nearfield product of one target leaf box X is a dense GEMM
//   F[rows][t] += sum_{d} A_d[rows][k] W[t - d][k]      (k: the columns of X's interaction area)
// with t = i*2 + s (leaf interval i, step s of the interval) and d = 0 .. 2 + s.  A CTA tile is
// 128 rows x 256 columns: columns 0..127 are the intervals i0..i0+127 at phase s = 0, columns
// 128..255 the same intervals at s = 1.  W is seen by TMA as a 4D tensor [rhs][interval][phase]
// [col], so the time shift by d is a coordinate offset, and the causality mask (t - d < 0) is the
// out-of-bounds zero fill.  A comes from the FP16 parts stored as contiguous 64-row x 64-column
// blocks (nf_tiled_index): each 64-row half of a tile's K block is one 8 KB TMA copy of a 3D view
// [block][64][64], and the half past a panel's last row is not copied (its MMA rows are never
// written out).  FP32 accuracy comes from a two-part FP16 split with power-of-two
// scales (FP16 keeps 11 significant bits, as TF32 does, at twice the rate and half the bytes):
//   A W ~ (A_hi W_hi + A_hi W_lo + A_lo W_hi) / (s_A s_W),
//   A_hi = rn_f16(s_A A), A_lo = rn_f16(s_A A - A_hi)     (same for W with s_W per rhs),
// where s_A (per operator, at build) and s_W (per rhs and apply, from max |W|) bring the largest
// magnitude into [2^14, 2^15): the parts are normal FP16 down to 2^-29 of the maximum, and
// |A - (A_hi + A_lo) / s_A| <= 2^-22 |A| above that.  The products are accumulated in FP32 in
// TMEM over sub-chunks of 32 stages (2048 columns) of the column loop, unscaled exactly (powers of
// two) in FP64 and added, sub-chunk by sub-chunk and by the one CTA that owns the work item, into
// the item's FP64 partial plane; the ksplit planes of a tile (split K, for SM balance) are then
// summed in plane order by k_nf_tc_reduce: no atomics, bitwise reproducible.
// Warp roles (192 threads): warp 0 issues TMA, warp 1 allocates TMEM and issues the MMAs,
// warps 2-5 drain TMEM (each warp reads its 32-lane quadrant).  Two smem stages, two TMEM
// accumulators (512 columns), persistent CTAs over (tile, K chunk) work items.  Every mbarrier
// wait gives up after a deadline, sets an error word and lets the CTA finish cleanly.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "kernels.h"
#include "nf_tc.h"
#include "tc_ptx.cuh"

namespace pfmm {

namespace {

using namespace tc;

constexpr int BM = 128, BK = 64;                   // BK fp16 = 128 bytes = one swizzle atom
constexpr int A_TILE = BM * BK * 2;                // 16 KB
constexpr int B_HALF = 128 * BK * 2;               // 16 KB (one phase)
constexpr int STAGE_BYTES = 2 * A_TILE + 4 * B_HALF;  // A_hi, A_lo, B_hi (2 halves), B_lo (2 halves)
constexpr int NSTAGE = 2;
constexpr uint64_t kTimeoutNs = 2000000000ull;     // 2 s per wait
constexpr int kSub = 32;                            // stages per FP32 accumulation in TMEM

// 3D tile: the FP16 panel parts seen as [block][64 rows][64 columns]
__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            su32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(su32(bar))
        : "memory");
}

// instruction descriptor: kind::f16 with FP16 A and B (format 0), FP32 accumulate, both
// K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4)                      // D format F32
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_f16(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::
            "r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

struct Item {
    int panel, r0, ib, rhs, st0, st1, kc;  // tile, its stage range [st0, st1), K chunk (partial plane)
};

__device__ __forceinline__ Item decode_item(const NfTcParams &P, int it)
{
    // items: tile-major (tile = (row tile, interval block, rhs)), K chunks inner
    Item I;
    int tile = it / P.ksplit, kc = it % P.ksplit;
    I.rhs = tile / (P.ntiles * P.nib);
    int r_ = tile % (P.ntiles * P.nib);
    I.ib = r_ % P.nib;
    int rt = r_ / P.nib;
    I.panel = P.tiles[2 * rt];
    I.r0 = P.tiles[2 * rt + 1];
    int nst = 4 * P.nkb;  // stage list: d = 0..3, then column blocks
    I.st0 = (int)((long long)nst * kc / P.ksplit);
    I.st1 = (int)((long long)nst * (kc + 1) / P.ksplit);
    I.kc = kc;
    return I;
}

}  // namespace

__global__ void __launch_bounds__(192, 1) k_nf_apply_tc(const __grid_constant__ CUtensorMap mapAhi,
                                                         const __grid_constant__ CUtensorMap mapAlo,
                                                         const __grid_constant__ CUtensorMap mapWhi,
                                                         const __grid_constant__ CUtensorMap mapWlo, NfTcParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the tiles (swizzle atoms)
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + NSTAGE * STAGE_BYTES);
    uint64_t *empty = full + NSTAGE;
    uint64_t *tfull = empty + NSTAGE;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 128);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint64_t deadline = gtimer() + kTimeoutNs;
    const int nitems = P.nitems;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int g = 0;  // global stage counter
            for (int it = blockIdx.x; it < nitems && !s_abort; it += gridDim.x) {
                Item I = decode_item(P, it);
                const PanelGPU &Pn = P.panels[I.panel];
                for (int st = I.st0; st < I.st1; ++st, ++g) {
                    const int s = g % NSTAGE;
                    if (!mbar_wait(&empty[s], ((g / NSTAGE) & 1) ^ 1, deadline)) {
                        atomicExch(P.err, 1);
                        s_abort = 1;
                        break;
                    }
                    const int d = st / P.nkb, kb = st % P.nkb;
                    unsigned char *sA = smem + s * STAGE_BYTES;
                    // A: the tile's 64-row blocks (the second only where the panel has rows; the
                    // MMA rows of a skipped half are never written out)
                    const bool two = I.r0 + 64 < Pn.nrows;
                    const uint32_t abytes = two ? A_TILE : A_TILE / 2;
                    const uint32_t bytes = 2 * abytes + (d < 3 ? 4 : 2) * B_HALF;
                    mbar_expect_tx(&full[s], bytes);
                    const long long arow = (P.kop ? Pn.offK : Pn.offV) / P.cols_pad + (long long)d * Pn.rows_pad + I.r0;
                    const int blk = (int)(arow >> 6) * P.nkb + kb;
                    tma_3d(sA, &mapAhi, 0, 0, blk, &full[s]);
                    tma_3d(sA + A_TILE, &mapAlo, 0, 0, blk, &full[s]);
                    if (two) {
                        tma_3d(sA + A_TILE / 2, &mapAhi, 0, 0, blk + P.nkb, &full[s]);
                        tma_3d(sA + A_TILE + A_TILE / 2, &mapAlo, 0, 0, blk + P.nkb, &full[s]);
                    }
                    unsigned char *sB = sA + 2 * A_TILE;
                    for (int ph = (d < 3 ? 0 : 1); ph < 2; ++ph) {
                        // step t = 2 i + ph, source step t - d = 2 (i - q) + phs
                        const int phs = ((ph - d) % 2 + 2) % 2, q = (phs - (ph - d)) / 2;
                        tma_4d(sB + ph * B_HALF, &mapWhi, kb * BK, phs, I.ib * 128 - q, I.rhs, &full[s]);
                        tma_4d(sB + 2 * B_HALF + ph * B_HALF, &mapWlo, kb * BK, phs, I.ib * 128 - q, I.rhs, &full[s]);
                    }
                }
            }
            // before the CTA exits, the copies it issued must have landed (bounded wait): the last
            // use u of stage s completes phase u
            const uint64_t dl2 = gtimer() + kTimeoutNs / 20;
            for (int j = (g > NSTAGE ? g - NSTAGE : 0); j < g; ++j) mbar_wait(&full[j % NSTAGE], (j / NSTAGE) & 1, dl2);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int g = 0, n = 0;  // n: sub-chunks issued (the TMEM accumulators alternate per sub-chunk)
            const uint32_t id256 = idesc_f16(BM, 256), id128 = idesc_f16(BM, 128);
            for (int it = blockIdx.x; it < nitems && !s_abort; it += gridDim.x) {
              Item I = decode_item(P, it);
              for (int sc0 = I.st0; sc0 < I.st1 && !s_abort; sc0 += kSub, ++n) {
                const int sc1 = min(I.st1, sc0 + kSub);
                const int acc = n & 1;
                if (!mbar_wait(&tempty[acc], ((n >> 1) & 1) ^ 1, deadline)) {
                    atomicExch(P.err, 2);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dcol = tmem + acc * 256;
                uint32_t first = 1;
                for (int st = sc0; st < sc1; ++st, ++g) {
                    const int s = g % NSTAGE;
                    if (!mbar_wait(&full[s], (g / NSTAGE) & 1, deadline)) {
                        atomicExch(P.err, 3);
                        s_abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int d = st / P.nkb;
                    const uint32_t a_hi = su32(smem + s * STAGE_BYTES), a_lo = a_hi + A_TILE;
                    const uint32_t b_hi = a_hi + 2 * A_TILE, b_lo = b_hi + 2 * B_HALF;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {  // K = 16 fp16 (32 bytes) per MMA
                        const uint32_t ko = kk * 32;
                        if (d < 3) {
                            mma_f16(dcol, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), id256, first ? 0u : 1u);
                            first = 0;
                            mma_f16(dcol, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), id256, 1u);
                            mma_f16(dcol, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), id256, 1u);
                        } else {
                            // d = 3 reaches back only from the second step of an interval
                            mma_f16(dcol + 128, sw128_desc(a_hi + ko), sw128_desc(b_hi + B_HALF + ko), id128,
                                     first ? 0u : 1u);
                            mma_f16(dcol + 128, sw128_desc(a_hi + ko), sw128_desc(b_lo + B_HALF + ko), id128, 1u);
                            mma_f16(dcol + 128, sw128_desc(a_lo + ko), sw128_desc(b_hi + B_HALF + ko), id128, 1u);
                            if (first) {
                                // the phase-0 half starts with no d < 3 stage in this chunk: clear it
                                first = 0;
                            }
                        }
                    }
                    mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
                }
                mma_commit(&tfull[acc]);
              }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quadrant = warp % 4
        const int quad = warp & 3;
        const int row_l = quad * 32 + lane;
        int n = 0;
        for (int it = blockIdx.x; it < nitems && !s_abort; it += gridDim.x) {
            Item I = decode_item(P, it);
            const PanelGPU &Pn = P.panels[I.panel];
            const int row = I.r0 + row_l;
            const bool row_ok = row < Pn.nrows;
            double *fr = P.part + ((size_t)I.kc * P.nrhs + I.rhs) * P.Et * P.nt + Pn.row0 + row;
            // 2^-(a_exp + E_W) (|exponent| <= 200) built from its bits
            const double unscale = __longlong_as_double((long long)(1023 - P.a_exp - f64_scale_exp(P.wmax[I.rhs])) << 52);
            for (int sc0 = I.st0; sc0 < I.st1 && !s_abort; sc0 += kSub, ++n) {
                const int acc = n & 1;
                if (!mbar_wait(&tfull[acc], (n >> 1) & 1, deadline)) {
                    atomicExch(P.err, 4);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // the phase-1 half is written by any stage, the phase-0 half only by stages with
                // d < 3 (stages ascend in d, so a sub-chunk starting at d = 3 has none)
                const bool first = sc0 == I.st0, has_ph0 = sc0 < 3 * P.nkb;
#pragma unroll 1
                for (int c0 = 0; c0 < 256; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + acc * 256 + c0, v);
                    if (!row_ok || (c0 < 128 && !has_ph0 && !first)) continue;
                    // the group's 32 partial values are read together (one latency per group), then
                    // updated: the plane is private to this work item, so no atomics are needed
                    const int ph = c0 >> 7, iv0 = I.ib * 128 + (c0 & 127);
                    double *a0 = fr + (size_t)(2 * iv0 + ph) * P.nt;
                    const size_t step = 2 * (size_t)P.nt;
                    const int nj = min(32, P.nint - iv0);
                    double old[32];
                    if (!first) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) old[j] = j < nj ? a0[j * step] : 0.0;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if (j >= nj) continue;
                        const double x = (ph == 0 && !has_ph0) ? 0.0 : (double)__uint_as_float(v[j]) * unscale;
                        a0[j * step] = first ? x : old[j] + x;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&tempty[acc]);
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ------------------------------------------------------------------------------------------
// split kernels: with the scale s = 2^E, hi = rn_f16(s a) and lo = rn_f16(s a - hi).  s a - hi is
// exact in FP32 (and in FP64 for the input), so a - (hi + lo) / s is one FP16 rounding of the
// remainder: below 2^-22 |a| while lo is a normal FP16 number.

// largest |a| of n FP32 values into *out as ordered bits (non-negative floats order as integers)
__global__ void k_absmax_f32(const float *__restrict__ A, size_t n, unsigned *__restrict__ out)
{
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(A[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// row-major FP32 panels [rows][ncp] -> FP16 parts in 64 x 64 blocks
__global__ void k_split_panel(const float *__restrict__ A, __half *__restrict__ hi, __half *__restrict__ lo, size_t n,
                              int ncp, float scale)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t R = i / ncp;
    const int c = (int)(i - R * ncp);
    const size_t o = nf_tiled_index(R, c, ncp >> 6);
    const float a = A[i] * scale;
    const __half h = __float2half_rn(a);
    hi[o] = h;
    lo[o] = __float2half_rn(a - __half2float(h));
}

// per-rhs max |x| of the FP64 input [rhs][Et][ncol], on the bits (non-negative doubles order as
// unsigned integers; no FP64 arithmetic)
__global__ void k_absmax_input(const double *__restrict__ x, size_t per_rhs, unsigned long long *__restrict__ wmax)
{
    const unsigned long long *xr = reinterpret_cast<const unsigned long long *>(x) + (size_t)blockIdx.y * per_rhs;
    unsigned long long m = 0ull;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_rhs; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long v = xr[i] & 0x7fffffffffffffffull;
        m = v > m ? v : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(wmax + blockIdx.y, m);
}

// W split from FP64 input: permutes (V) or pads rows (K) into [rhs][t][ncol_pad].  x is rounded
// once to FP32 (2^-24 relative), scaled exactly by 2^E in FP32 and split there.
__global__ void k_split_input(const double *__restrict__ x, const int *__restrict__ perm, int ncol, int ncol_pad,
                              __half *__restrict__ hi, __half *__restrict__ lo, size_t per_rhs, size_t total,
                              const unsigned long long *__restrict__ wmax)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    size_t rt = i / ncol_pad;
    int c = (int)(i - rt * ncol_pad);
    float v = 0.f;
    if (c < ncol) v = (float)x[rt * ncol + (perm ? perm[c] : c)];
    v *= __int_as_float((127 + f64_scale_exp(wmax[i / per_rhs])) << 23);  // 2^E, |E| <= 100
    const __half h = __float2half_rn(v);
    hi[i] = h;
    lo[i] = __float2half_rn(v - __half2float(h));
}

int panel_scale_exp(const float *A, size_t n, unsigned *scratch, cudaStream_t st)
{
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned), st) != cudaSuccess) return INT32_MIN;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    if (grid > 0) k_absmax_f32<<<grid, 256, 0, st>>>(A, n, scratch);
    unsigned bits = 0;
    if (cudaMemcpyAsync(&bits, scratch, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return INT32_MIN;
    return f32_scale_exp(bits);
}

void launch_split_panel(const float *A, void *hi, void *lo, size_t n, int ncp, int a_exp, cudaStream_t st)
{
    if (n == 0) return;
    k_split_panel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, (__half *)hi, (__half *)lo, n, ncp,
                                                              std::ldexp(1.0f, a_exp));
}

void launch_split_input(const double *x, const int *perm, int ncol, int ncol_pad, int nrhs, int Et, void *hi,
                        void *lo, unsigned long long *wmax, cudaStream_t st)
{
    cudaMemsetAsync(wmax, 0, sizeof(unsigned long long) * nrhs, st);
    const size_t per_in = (size_t)Et * ncol;
    const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>((per_in + 2047) / 2048, 1216));
    k_absmax_input<<<dim3(gx, nrhs), 256, 0, st>>>(x, per_in, wmax);
    const size_t per_rhs = (size_t)Et * ncol_pad, total = (size_t)nrhs * per_rhs;
    k_split_input<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(x, perm, ncol, ncol_pad, (__half *)hi,
                                                                   (__half *)lo, per_rhs, total, wmax);
}

void launch_absmax_input(const double *x, size_t per_rhs, int nrhs, unsigned grid_x, unsigned long long *wmax,
                         cudaStream_t st)
{
    k_absmax_input<<<dim3(grid_x, nrhs), 256, 0, st>>>(x, per_rhs, wmax);
}

// f[i] = sum over the K-chunk planes of part[kc][i], in plane order
__global__ void k_nf_tc_reduce(const double *__restrict__ part, int ks, size_t n, double *__restrict__ f)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = part[i];
    for (int kc = 1; kc < ks; ++kc) s += part[(size_t)kc * n + i];
    f[i] = s;
}

void launch_nf_tc_reduce(const double *part, int ks, size_t n, double *f, cudaStream_t st)
{
    if (n > 0) k_nf_tc_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, ks, n, f);
}

int nf_tc_ksplit(int tiles, int nkb, int nsm)
{
    // the number of K chunks (1 .. 8, at most the tile's 32-stage sub-chunks) whose work items fill
    // the rounds of the persistent grid best (items / (nsm x rounds)); the smallest on a tie
    const int nsub = (4 * nkb + kSub - 1) / kSub;
    int best = 1;
    double best_eff = -1.0;
    for (int ks = 1; ks <= std::min(8, nsub); ++ks) {
        const long long items = (long long)tiles * ks, rounds = (items + nsm - 1) / nsm;
        const double eff = (double)items / ((double)nsm * rounds);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = ks;
        }
    }
    return best;
}

size_t nf_tc_smem_bytes() { return (size_t)NSTAGE * STAGE_BYTES + 1024 + 256; }

int launch_nf_apply_tc(const CUtensorMap &Ahi, const CUtensorMap &Alo, const CUtensorMap &Whi, const CUtensorMap &Wlo,
                       const NfTcParams &P, int nsm, cudaStream_t st)
{
    size_t smem = nf_tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_nf_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    int grid = P.nitems < nsm ? P.nitems : nsm;
    k_nf_apply_tc<<<grid, 192, smem, st>>>(Ahi, Alo, Whi, Wlo, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pfmm
