// k_nf_crt.cu -- FP64-accurate nearfield apply (Alg. 2, last loop; Eq. eval_sl_nf_block) on
// the sm_103a tensor cores, by exact integer arithmetic in residues (a multi-modular form of the
// Ozaki error-free splitting scheme for matrix products: Ozaki, Ogita, Oishi, Rump, Numerical
// Algorithms 59 (2012); here with the Chinese remainder theorem instead of digit slices, as in
// Ozaki, Uchino, Imamura, "Ozaki Scheme II", 2024).
//
// GB300 executes FP64 FMAs at about 1 TFLOP/s but FP16 tensor-core products at about 2 PFLOP/s.
// The block-Toeplitz nearfield product F[r][t] = sum_d sum_k A_d[r][k] W[t-d][k] is therefore
// computed exactly in integers and rounded to FP64 once:
//   * every row r of the stored FP64 blocks is scaled by 2^e_r (largest |A_d[r][k]| over d, k in
//     [2^(b-1), 2^b)) and rounded to the integer A'; the input by 2^s per rhs to W' (|W'| <= 2^b),
//     b chosen so that the exact integer product X = sum A' W' satisfies 2 |X| < M;
//   * X is computed modulo 16 primes p_i < 256 (M = prod p_i ~ 2^123): the residues of A' and W'
//     in [-(p-1)/2, (p-1)/2] are exact FP16 numbers, their products are below 2^14, and a tcgen05
//     kind::f16 MMA chain accumulates them in FP32 exactly (integers below 2^24) over chunks of
//     1024 columns; after each chunk the epilogue reduces the accumulator modulo p in place
//     (tcgen05.ld / .st), so the next chunk adds onto a small residue;
//   * the 16 residues of X are combined by Garner's mixed-radix algorithm (balanced digits, exact
//     FP32 arithmetic), X is assembled exactly in 128-bit integers and X 2^-(e_r + s) is rounded
//     to FP64 (relative error ~2^-52).
// The only rounding before the final FP64 result is that of A and W to b-bit fixed point per row /
// per rhs (b = 52..53): the product is as accurate as an FP64 dot product of the same terms.
//
// Tiles as in the FP16-split kernel: 128 rows x 256 columns (128 leaf intervals x 2 steps), W a
// TMA tensor [modulus][rhs][interval][phase][column] so the time shift d is a coordinate offset
// and causality the zero fill.  A work item is (moduli pair, row tile, interval block, rhs): the
// two moduli alternate chunk by chunk between two TMEM accumulators (2 x 256 columns), so the MMA
// of one overlaps the epilogue's reduction of the other.  Warp roles (192 threads): warp 0 TMA,
// warp 1 TMEM allocation and MMA issue, warps 2-5 epilogue (one 32-lane TMEM quadrant each).
// Four 48 KB smem stages.  Every mbarrier wait is bounded (error word, clean exit).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "kernels.h"
#include "nf_crt.h"
#include "nf_tc.h"
#include "tc_ptx.cuh"

namespace pfmm {

namespace {

using namespace tc;

__constant__ int c_p[kCrtModuli];              // the moduli
__constant__ float c_invp[kCrtModuli];         // 1 / p (FP32)
__constant__ float c_pf[kCrtModuli];           // the moduli (FP32)
__constant__ float c_pow11[kCrtModuli][5];     // 2^(11 k) mod p_i (FP32), k = 0 .. 4
__constant__ float c_pjmodpif[kCrtModuli][kCrtModuli];  // (p_0 ... p_{j-1}) mod p_i, j < i (FP32)
__constant__ float c_invPif[kCrtModuli];       // (p_0 ... p_{i-1})^-1 mod p_i (FP32)

constexpr int BM = 128, BK = 64;
constexpr int A_TILE = BM * BK * 2;      // 16 KB
constexpr int B_HALF = 128 * BK * 2;     // 16 KB per phase
constexpr int STAGE_BYTES = A_TILE + 2 * B_HALF;  // 48 KB
constexpr int NSTAGE = 4;
constexpr int CHUNK = 16;                // stages per exact FP32 accumulation chunk (1024 columns)
constexpr uint64_t kTimeoutNs = 2000000000ull;

__device__ __forceinline__ void tma_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_5d(void *dst, const CUtensorMap *map, int x, int y, int z, int w, int v,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(v), "r"(su32(bar))
        : "memory");
}

// kind::f16, FP16 A and B, FP32 accumulate, K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::
            "r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

struct CItem {
    int panel, r0, ib, rhs, m0;  // row tile, interval block, rhs, first modulus of the pair
};

__device__ __forceinline__ CItem decode_citem(const NfCrtParams &P, int it)
{
    // pair-major: consecutive CTAs share the moduli (their W residues stay in L2)
    const int ntile = P.ntiles * P.nib * P.nrhs;
    CItem I;
    I.m0 = 2 * (it / ntile);
    int tile = it % ntile;
    I.rhs = tile / (P.ntiles * P.nib);
    int r_ = tile % (P.ntiles * P.nib);
    I.ib = r_ % P.nib;
    int rt = r_ / P.nib;
    I.panel = P.tiles[2 * rt];
    I.r0 = P.tiles[2 * rt + 1];
    return I;
}

// x mod p into [-(p-1)/2 - p, (p-1)/2 + p] for an integer-valued |x| < 2^24 (exact): the FP32
// quotient may be one off near a half-integer, which leaves a congruent value within 1.5 p
__device__ __forceinline__ float mod_small(float x, float p, float invp)
{
    const float q = rintf(x * invp);
    return fmaf(-q, p, x);
}

}  // namespace

__global__ void __launch_bounds__(192, 1) k_nf_apply_crt(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapW, NfCrtParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
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
    uint64_t deadline = gtimer() + kTimeoutNs;  // renewed per chunk: each wait is bounded by 2 s
    const int nst = 4 * P.nkb;                   // stages per modulus: d = 0..3 x column blocks
    const int nch = (nst + CHUNK - 1) / CHUNK;   // exact accumulation chunks

    if (warp == 0) {
        // ---------------- TMA producer: (chunk, slot, stage) in the MMA's order
        if (lane == 0) {
            int g = 0;
            for (int it = blockIdx.x; it < P.nitems && !s_abort; it += gridDim.x) {
                const CItem I = decode_citem(P, it);
                const PanelGPU &Pn = P.panels[I.panel];
                const bool two = I.r0 + 64 < Pn.nrows;
                const long long rbase = (P.kop ? Pn.offK : Pn.offV) / P.cols_pad + I.r0;
                for (int ch = 0; ch < nch && !s_abort; ++ch)
                    for (int slot = 0; slot < 2 && !s_abort; ++slot) {
                        deadline = gtimer() + kTimeoutNs;
                        const int m = I.m0 + slot;
                        const int st1 = min(nst, (ch + 1) * CHUNK);
                        for (int st = ch * CHUNK; st < st1; ++st, ++g) {
                            const int s = g % NSTAGE;
                            if (!mbar_wait(&empty[s], ((g / NSTAGE) & 1) ^ 1, deadline)) {
                                atomicExch(P.err, 11);
                                s_abort = 1;
                                break;
                            }
                            const int d = st / P.nkb, kb = st % P.nkb;
                            unsigned char *sA = smem + s * STAGE_BYTES;
                            const uint32_t abytes = two ? A_TILE : A_TILE / 2;
                            mbar_expect_tx(&full[s], abytes + (d < 3 ? 2 : 1) * B_HALF);
                            const int blk = (int)((rbase + (long long)d * Pn.rows_pad) >> 6) * P.nkb + kb;
                            tma_4d(sA, &mapA, 0, 0, blk, m, &full[s]);
                            if (two) tma_4d(sA + A_TILE / 2, &mapA, 0, 0, blk + P.nkb, m, &full[s]);
                            unsigned char *sB = sA + A_TILE;
                            for (int ph = (d < 3 ? 0 : 1); ph < 2; ++ph) {
                                const int phs = ((ph - d) % 2 + 2) % 2, q = (phs - (ph - d)) / 2;
                                tma_5d(sB + ph * B_HALF, &mapW, kb * BK, phs, I.ib * 128 - q, I.rhs, m, &full[s]);
                            }
                        }
                    }
            }
            const uint64_t dl2 = gtimer() + kTimeoutNs / 20;
            for (int j = (g > NSTAGE ? g - NSTAGE : 0); j < g; ++j) mbar_wait(&full[j % NSTAGE], (j / NSTAGE) & 1, dl2);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int g = 0, u = 0;  // u: accumulator uses (both slots advance together)
            const uint32_t id256 = idesc_f16(BM, 256), id128 = idesc_f16(BM, 128);
            for (int it = blockIdx.x; it < P.nitems && !s_abort; it += gridDim.x) {
                for (int ch = 0; ch < nch && !s_abort; ++ch, ++u)
                    for (int slot = 0; slot < 2 && !s_abort; ++slot) {
                        deadline = gtimer() + kTimeoutNs;
                        if (!mbar_wait(&tempty[slot], (u & 1) ^ 1, deadline)) {
                            atomicExch(P.err, 12);
                            s_abort = 1;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t dcol = tmem + slot * 256;
                        const int st1 = min(nst, (ch + 1) * CHUNK);
                        for (int st = ch * CHUNK; st < st1; ++st, ++g) {
                            const int s = g % NSTAGE;
                            if (!mbar_wait(&full[s], (g / NSTAGE) & 1, deadline)) {
                                atomicExch(P.err, 13);
                                s_abort = 1;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const int d = st / P.nkb;
                            const uint32_t a0 = su32(smem + s * STAGE_BYTES), b0 = a0 + A_TILE;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint32_t ko = kk * 32;
                                // the item's first MMA starts from zero (d = 0 covers both phases)
                                const uint32_t accf = (ch == 0 && st == 0 && kk == 0) ? 0u : 1u;
                                if (d < 3)
                                    mma_f16(dcol, sw128_desc(a0 + ko), sw128_desc(b0 + ko), id256, accf);
                                else
                                    mma_f16(dcol + 128, sw128_desc(a0 + ko), sw128_desc(b0 + B_HALF + ko), id128, 1u);
                            }
                            mma_commit(&empty[s]);
                        }
                        mma_commit(&tfull[slot]);
                    }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quadrant = warp % 4
        const int quad = warp & 3;
        const int row_l = quad * 32 + lane;
        int u = 0;
        for (int it = blockIdx.x; it < P.nitems && !s_abort; it += gridDim.x) {
            const CItem I = decode_citem(P, it);
            const PanelGPU &Pn = P.panels[I.panel];
            const int row = I.r0 + row_l;
            const bool row_ok = row < Pn.nrows;
            for (int ch = 0; ch < nch && !s_abort; ++ch, ++u)
                for (int slot = 0; slot < 2 && !s_abort; ++slot) {
                    deadline = gtimer() + kTimeoutNs;
                    if (!mbar_wait(&tfull[slot], u & 1, deadline)) {
                        atomicExch(P.err, 14);
                        s_abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int m = I.m0 + slot;
                    const float p = (float)c_p[m], invp = c_invp[m];
                    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + slot * 256;
                    const bool last = ch == nch - 1;
                    unsigned char *out = P.res + ((size_t)m * P.nrhs + I.rhs) * P.Et * (size_t)P.nt + Pn.row0 + row;
#pragma unroll 1
                    for (int c0 = 0; c0 < 256; c0 += 32) {
                        uint32_t v[32];
                        tmem_ld32(tbase + c0, v);
                        if (!last) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(mod_small(__uint_as_float(v[j]), p, invp));
                            tmem_st32(tbase + c0, v);
                        } else if (row_ok) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int c = c0 + j, ph = c >> 7, iv = I.ib * 128 + (c & 127);
                                float r = mod_small(__uint_as_float(v[j]), p, invp);
                                r = r < 0.f ? r + p : r;
                                r = r < 0.f ? r + p : r;
                                r = r >= p ? r - p : r;
                                if (iv < P.nint) out[(size_t)(2 * iv + ph) * P.nt] = (unsigned char)(int)r;
                            }
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&tempty[slot]);
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
// Two row tiles per CTA: the W stage (32 KB) feeds the MMAs of two 128-row tiles, so every byte
// brought from L2 / HBM serves twice the tensor work of the form above.  A work item is (modulus,
// pair of row tiles, interval block, rhs); the two tiles' accumulators take all 512 TMEM columns,
// so the epilogue's reduction after each 1024-column chunk pauses the MMAs (about 900 of 16000
// cycles).  Warps: 0 TMA, 1 MMA, 2..9 epilogue (warp w serves tile (w - 2) / 4 and TMEM lane
// quadrant w % 4).  Three 64 KB stages.
constexpr int STAGE2 = 2 * A_TILE + 2 * B_HALF;  // 64 KB
constexpr int NSTAGE2 = 3;
constexpr int kCrt2Threads = 320;

struct CItem2 {
    int m, rhs, ib;
    int panel[2], r0[2];
    bool has1;
};

__device__ __forceinline__ CItem2 decode_citem2(const NfCrtParams &P, int it)
{
    const int ntp = (P.ntiles + 1) / 2, per_m = ntp * P.nib * P.nrhs;
    CItem2 I;
    I.m = it / per_m;  // modulus-major: consecutive CTAs share the modulus (its W residues stay in L2)
    int r_ = it % per_m;
    I.rhs = r_ / (ntp * P.nib);
    r_ %= ntp * P.nib;
    I.ib = r_ % P.nib;
    const int tp = r_ / P.nib;
    const int t0 = 2 * tp, t1 = 2 * tp + 1;
    I.panel[0] = P.tiles[2 * t0];
    I.r0[0] = P.tiles[2 * t0 + 1];
    I.has1 = t1 < P.ntiles;
    I.panel[1] = I.has1 ? P.tiles[2 * t1] : I.panel[0];
    I.r0[1] = I.has1 ? P.tiles[2 * t1 + 1] : I.r0[0];
    return I;
}

__global__ void __launch_bounds__(kCrt2Threads, 1) k_nf_apply_crt2(const __grid_constant__ CUtensorMap mapA,
                                                                   const __grid_constant__ CUtensorMap mapW,
                                                                   NfCrtParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + NSTAGE2 * STAGE2);
    uint64_t *empty = full + NSTAGE2;
    uint64_t *tfull = empty + NSTAGE2;
    uint64_t *tempty = tfull + 1;
    uint32_t *tmem_slot = (uint32_t *)(tempty + 1);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE2; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, 256);
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
    uint64_t deadline = gtimer() + kTimeoutNs;  // renewed per chunk: each wait is bounded by 2 s
    const int nst = 4 * P.nkb;
    const int nch = (nst + CHUNK - 1) / CHUNK;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int g = 0;
            for (int it = blockIdx.x; it < P.nitems && !s_abort; it += gridDim.x) {
                const CItem2 I = decode_citem2(P, it);
                bool two[2];
                long long rbase[2];
                int rpad[2];
                for (int q = 0; q < 2; ++q) {
                    const PanelGPU &Pn = P.panels[I.panel[q]];
                    two[q] = I.r0[q] + 64 < Pn.nrows;
                    rbase[q] = (P.kop ? Pn.offK : Pn.offV) / P.cols_pad + I.r0[q];
                    rpad[q] = Pn.rows_pad;
                }
                for (int ch = 0; ch < nch && !s_abort; ++ch) {
                    deadline = gtimer() + kTimeoutNs;
                    const int st1 = min(nst, (ch + 1) * CHUNK);
                    for (int st = ch * CHUNK; st < st1; ++st, ++g) {
                        const int s = g % NSTAGE2;
                        if (!mbar_wait(&empty[s], ((g / NSTAGE2) & 1) ^ 1, deadline)) {
                            atomicExch(P.err, 21);
                            s_abort = 1;
                            break;
                        }
                        const int d = st / P.nkb, kb = st % P.nkb;
                        unsigned char *sA = smem + s * STAGE2;
                        uint32_t bytes = (d < 3 ? 2 : 1) * B_HALF;
                        for (int q = 0; q < (I.has1 ? 2 : 1); ++q) bytes += two[q] ? A_TILE : A_TILE / 2;
                        mbar_expect_tx(&full[s], bytes);
                        for (int q = 0; q < (I.has1 ? 2 : 1); ++q) {
                            const int blk = (int)((rbase[q] + (long long)d * rpad[q]) >> 6) * P.nkb + kb;
                            tma_4d(sA + q * A_TILE, &mapA, 0, 0, blk, I.m, &full[s]);
                            if (two[q]) tma_4d(sA + q * A_TILE + A_TILE / 2, &mapA, 0, 0, blk + P.nkb, I.m, &full[s]);
                        }
                        unsigned char *sB = sA + 2 * A_TILE;
                        for (int ph = (d < 3 ? 0 : 1); ph < 2; ++ph) {
                            const int phs = ((ph - d) % 2 + 2) % 2, q = (phs - (ph - d)) / 2;
                            tma_5d(sB + ph * B_HALF, &mapW, kb * BK, phs, I.ib * 128 - q, I.rhs, I.m, &full[s]);
                        }
                    }
                }
            }
            const uint64_t dl2 = gtimer() + kTimeoutNs / 20;
            for (int j = (g > NSTAGE2 ? g - NSTAGE2 : 0); j < g; ++j)
                mbar_wait(&full[j % NSTAGE2], (j / NSTAGE2) & 1, dl2);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int g = 0, u = 0;
            const uint32_t id256 = idesc_f16(BM, 256), id128 = idesc_f16(BM, 128);
            for (int it = blockIdx.x; it < P.nitems && !s_abort; it += gridDim.x) {
                const CItem2 I = decode_citem2(P, it);
                for (int ch = 0; ch < nch && !s_abort; ++ch, ++u) {
                    deadline = gtimer() + kTimeoutNs;
                    if (!mbar_wait(tempty, (u & 1) ^ 1, deadline)) {
                        atomicExch(P.err, 22);
                        s_abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int st1 = min(nst, (ch + 1) * CHUNK);
                    for (int st = ch * CHUNK; st < st1; ++st, ++g) {
                        const int s = g % NSTAGE2;
                        if (!mbar_wait(&full[s], (g / NSTAGE2) & 1, deadline)) {
                            atomicExch(P.err, 23);
                            s_abort = 1;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const int d = st / P.nkb;
                        const uint32_t a0 = su32(smem + s * STAGE2), b0 = a0 + 2 * A_TILE;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint32_t ko = kk * 32;
                            const uint32_t accf = (ch == 0 && st == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                if (q == 1 && !I.has1) break;
                                const uint32_t aq = a0 + q * A_TILE + ko, dq = tmem + q * 256;
                                if (d < 3)
                                    mma_f16(dq, sw128_desc(aq), sw128_desc(b0 + ko), id256, accf);
                                else
                                    mma_f16(dq + 128, sw128_desc(aq), sw128_desc(b0 + B_HALF + ko), id128, 1u);
                            }
                        }
                        mma_commit(&empty[s]);
                    }
                    mma_commit(tfull);
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9; tile (warp - 2) / 4, TMEM lane quadrant warp % 4
        const int quad = warp & 3, tq = (warp - 2) >> 2;
        const int row_l = quad * 32 + lane;
        int u = 0;
        for (int it = blockIdx.x; it < P.nitems && !s_abort; it += gridDim.x) {
            const CItem2 I = decode_citem2(P, it);
            const bool active = tq == 0 || I.has1;
            const PanelGPU &Pn = P.panels[I.panel[tq]];
            const int row = I.r0[tq] + row_l;
            const bool row_ok = active && row < Pn.nrows;
            const float p = (float)c_p[I.m], invp = c_invp[I.m];
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + tq * 256;
            unsigned char *out = P.res + ((size_t)I.m * P.nrhs + I.rhs) * P.Et * (size_t)P.nt + Pn.row0 + row;
            for (int ch = 0; ch < nch && !s_abort; ++ch, ++u) {
                deadline = gtimer() + kTimeoutNs;
                if (!mbar_wait(tfull, u & 1, deadline)) {
                    atomicExch(P.err, 24);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const bool last = ch == nch - 1;
                if (active) {
#pragma unroll 1
                    for (int c0 = 0; c0 < 256; c0 += 32) {
                        uint32_t v[32];
                        tmem_ld32(tbase + c0, v);
                        if (!last) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(mod_small(__uint_as_float(v[j]), p, invp));
                            tmem_st32(tbase + c0, v);
                        } else if (row_ok) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int c = c0 + j, ph = c >> 7, iv = I.ib * 128 + (c & 127);
                                float r = mod_small(__uint_as_float(v[j]), p, invp);
                                r = r < 0.f ? r + p : r;
                                r = r < 0.f ? r + p : r;
                                r = r >= p ? r - p : r;
                                if (iv < P.nint) out[(size_t)(2 * iv + ph) * P.nt] = (unsigned char)(int)r;
                            }
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(tempty);
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
// scaling and residues

// largest |A| of every target row over the step offsets and columns of its panel, as FP64 bits
// (non-negative doubles order as unsigned integers), into rowmax[row0 + r]
__global__ void k_row_absmax(const double *__restrict__ A, const PanelGPU *__restrict__ panels, int npanel, int kop,
                             int nd, unsigned long long *__restrict__ rowmax)
{
    const PanelGPU &Pn = panels[blockIdx.y];
    const int cols = kop ? Pn.colsK_pad : Pn.colsV_pad;
    const long long off = kop ? Pn.offK : Pn.offV;
    for (int r = blockIdx.x; r < Pn.nrows; r += gridDim.x) {
        unsigned long long m = 0ull;
        for (int d = 0; d < nd; ++d) {
            const unsigned long long *a =
                reinterpret_cast<const unsigned long long *>(A + off + ((size_t)d * Pn.rows_pad + r) * cols);
            for (int c = threadIdx.x; c < cols; c += blockDim.x) {
                const unsigned long long v = a[c] & 0x7fffffffffffffffull;
                m = v > m ? v : m;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
            m = v > m ? v : m;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(rowmax + Pn.row0 + r, m);
    }
}

// exponent e with 2^e m in [2^(b-1), 2^b) for the FP64 bits of m (0 for m = 0 or non-finite)
__host__ __device__ inline int crt_scale_exp(unsigned long long bits, int b)
{
    bits &= 0x7fffffffffffffffull;
    const int be = (int)(bits >> 52);
    if (bits == 0ull || be == 2047) return 0;
    const int E = (be == 0) ? -1074 + 63 - __builtin_clzll(bits) : be - 1023;  // m in [2^E, 2^(E+1))
    return b - 1 - E;
}

__device__ __forceinline__ double pow2(int e)
{
    // 2^e for -1022 <= e <= 1023 from its bits; beyond: two steps
    if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(1023 + e) << 52);
    return ldexp(1.0, e);
}

// balanced residue of an integer-valued x (|x| < 2^22) modulo p, in [-(p-1)/2, (p-1)/2]: the
// FP32 quotient of mod_small is off by at most one, so one correction each way suffices
__device__ __forceinline__ float mod_balanced(float x, float p, float invp)
{
    float t = mod_small(x, p, invp);
    const float hp = 0.5f * (p - 1.f);
    t = t > hp ? t - p : t;
    return t < -hp ? t + p : t;
}

// balanced residues of the integer a (|a| < 2^55) modulo the 16 primes, exactly in FP32: |a| is
// cut into five 11-bit digits a_k and sum_k a_k (2^(11 k) mod p) < 5 * 2^11 * 2^8 < 2^22 is reduced
// once; the residue of -a is minus that of a
__device__ __forceinline__ void residues16(long long a, float (&r)[kCrtModuli])
{
    const bool neg = a < 0;
    const unsigned long long u = neg ? 0ull - (unsigned long long)a : (unsigned long long)a;
    float dg[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) dg[k] = (float)(unsigned)((u >> (11 * k)) & 0x7ffull);
#pragma unroll
    for (int m = 0; m < kCrtModuli; ++m) {
        float x = dg[0];
#pragma unroll
        for (int k = 1; k < 5; ++k) x = fmaf(dg[k], c_pow11[m][k], x);
        const float t = mod_balanced(x, c_pf[m], c_invp[m]);
        r[m] = neg ? -t : t;
    }
}

// FP64 panels -> residues of A' = rint(2^e_R A) for every modulus, [modulus][n] in the 64 x 64
// block layout of nf_tiled_index (row R of the concatenated panels has exponent rowexp_R[R])
__global__ void k_crt_split_panel(const double *__restrict__ A, const int *__restrict__ rowexp_R, size_t n, int ncp,
                                  __half *__restrict__ res)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t R = i / ncp;
    const int c = (int)(i - R * ncp);
    const size_t o = nf_tiled_index(R, c, ncp >> 6);
    float r[kCrtModuli];
    residues16(__double2ll_rn(A[i] * pow2(rowexp_R[R])), r);
#pragma unroll
    for (int m = 0; m < kCrtModuli; ++m) res[(size_t)m * n + o] = __float2half_rn(r[m]);
}

// per-row exponents of global panel rows: rowexp_R[R] = e of the row's triangle
__global__ void k_row_exps(const PanelGPU *__restrict__ panels, int npanel, int kop, int nd, int ncp, int b,
                           const unsigned long long *__restrict__ rowmax, int *__restrict__ rowexp_tri,
                           int *__restrict__ rowexp_R)
{
    const PanelGPU &Pn = panels[blockIdx.x];
    const long long R0 = (kop ? Pn.offK : Pn.offV) / ncp;
    for (int i = threadIdx.x; i < nd * Pn.rows_pad; i += blockDim.x) {
        const int r = i % Pn.rows_pad;
        const int e = r < Pn.nrows ? crt_scale_exp(rowmax[Pn.row0 + r], b) : 0;
        rowexp_R[R0 + i] = e;
        if (i < Pn.nrows) rowexp_tri[Pn.row0 + r] = e;
    }
}

// input: per-rhs scale 2^s (|W'| <= 2^b), W' = rint(2^s x) permuted (V) or padded (K) into
// [rhs][t][ncol_pad], residues [modulus][rhs][t][ncol_pad]
__global__ void k_crt_split_input(const double *__restrict__ x, const int *__restrict__ perm, int ncol, int ncol_pad,
                                  size_t per_rhs, size_t total, const unsigned long long *__restrict__ wmax, int b,
                                  __half *__restrict__ res)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t rt = i / ncol_pad;
    const int c = (int)(i - rt * ncol_pad);
    long long wi = 0;
    if (c < ncol) {
        const double v = x[rt * ncol + (perm ? perm[c] : c)];
        wi = __double2ll_rn(v * pow2(crt_scale_exp(wmax[i / per_rhs], b)));
    }
    float r[kCrtModuli];
    residues16(wi, r);
#pragma unroll
    for (int m = 0; m < kCrtModuli; ++m) res[(size_t)m * total + i] = __float2half_rn(r[m]);
}

// f[rhs][t][row] = X 2^-(e_row + s_rhs), X from its residues by Garner's algorithm: the balanced
// mixed-radix digits v_j = (r_j - sum_{k<j} v_k P_k) P_j^-1 mod p_j (P_j = p_0 ... p_{j-1}) in exact
// FP32 arithmetic (every intermediate is an integer below 2^20), then X = sum_j v_j P_j by Horner's
// rule in 128-bit integers (|X| < M / 2 < 2^123, exact) and one conversion to FP64
__global__ void k_crt_combine(const unsigned char *__restrict__ res, size_t per_mod, size_t per_rhs, int nt,
                              const int *__restrict__ rowexp, const unsigned long long *__restrict__ wmax, int b,
                              double *__restrict__ f)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per_mod) return;
    float acc[kCrtModuli], v[kCrtModuli];
#pragma unroll
    for (int k = 0; k < kCrtModuli; ++k) acc[k] = 0.f;
#pragma unroll
    for (int j = 0; j < kCrtModuli; ++j) {
        const float p = c_pf[j], invp = c_invp[j];
        const float t = mod_small((float)res[(size_t)j * per_mod + i] - acc[j], p, invp);
        v[j] = mod_balanced(t * c_invPif[j], p, invp);
#pragma unroll
        for (int k = j + 1; k < kCrtModuli; ++k) acc[k] = fmaf(v[j], c_pjmodpif[j][k], acc[k]);
    }
    __int128 X = (__int128)(int)v[kCrtModuli - 1];
#pragma unroll
    for (int j = kCrtModuli - 2; j >= 0; --j) X = X * (__int128)c_p[j] + (__int128)(int)v[j];
    // |X| = hi 2^64 + lo: both parts non-negative, so the two roundings cannot cancel
    const bool neg = X < 0;
    const unsigned __int128 U = neg ? (unsigned __int128)0 - (unsigned __int128)X : (unsigned __int128)X;
    const unsigned long long hi = (unsigned long long)(U >> 64), lo = (unsigned long long)U;
    const double ax = hi ? fma((double)hi, 18446744073709551616.0, (double)lo) : (double)lo;
    const double x = neg ? -ax : ax;
    const int row = (int)(i % nt);
    const int e = rowexp[row] + crt_scale_exp(wmax[i / per_rhs], b);
    f[i] = x * pow2(-e);
}

// ------------------------------------------------------------------------------------------
// host side

static int g_moduli[kCrtModuli] = {251, 241, 239, 233, 229, 227, 223, 211, 199, 197, 193, 191, 181, 179, 173, 167};

static long long modinv(long long a, long long p)
{
    long long t = 0, nt = 1, r = p, nr = ((a % p) + p) % p;
    while (nr) {
        long long q = r / nr, tmp = t - q * nt;
        t = nt;
        nt = tmp;
        tmp = r - q * nr;
        r = nr;
        nr = tmp;
    }
    return t < 0 ? t + p : t;
}

int crt_upload_constants(cudaStream_t st)
{
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    if (done[dev]) return 0;
    float invp[kCrtModuli], pf[kCrtModuli], pow11[kCrtModuli][5];
    float pj[kCrtModuli][kCrtModuli] = {{0.f}}, invPi[kCrtModuli];
    for (int i = 0; i < kCrtModuli; ++i) {
        pf[i] = (float)g_moduli[i];
        invp[i] = 1.0f / (float)g_moduli[i];
        long long q = 1;  // p_0 ... p_{j-1} mod p_i, for j = 0 .. i
        for (int j = 0; j < i; ++j) {
            pj[j][i] = (float)q;
            q = q * g_moduli[j] % g_moduli[i];
        }
        invPi[i] = (float)modinv(q, g_moduli[i]);
        long long w = 1;  // 2^(11 k) mod p_i
        for (int k = 0; k < 5; ++k) {
            pow11[i][k] = (float)w;
            w = (w << 11) % g_moduli[i];
        }
    }
    if (cudaMemcpyToSymbolAsync(c_p, g_moduli, sizeof(g_moduli), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_pf, pf, sizeof(pf), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_invp, invp, sizeof(invp), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_pow11, pow11, sizeof(pow11), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_pjmodpif, pj, sizeof(pj), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_invPif, invPi, sizeof(invPi), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return -1;
    done[dev] = true;
    return 0;
}

int crt_bits(long long k_total)
{
    double l2m = 0.0;
    for (int i = 0; i < kCrtModuli; ++i) l2m += std::log2((double)g_moduli[i]);
    int lk = 0;
    while ((1ll << lk) < k_total) ++lk;
    const int b = (int)std::floor((l2m - 1.0 - lk) / 2.0);
    return std::min(b, 53);
}

void launch_crt_row_exps(const double *A, const PanelGPU *panels, int npanel, int kop, int nd, int ncp, int b,
                         unsigned long long *rowmax, int nt, int *rowexp_tri, int *rowexp_R, cudaStream_t st)
{
    cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * nt, st);
    k_row_absmax<<<dim3(64, npanel), 256, 0, st>>>(A, panels, npanel, kop, nd, rowmax);
    k_row_exps<<<npanel, 256, 0, st>>>(panels, npanel, kop, nd, ncp, b, rowmax, rowexp_tri, rowexp_R);
}

void launch_crt_split_panel(const double *A, const int *rowexp_R, size_t n, int ncp, void *res, cudaStream_t st)
{
    if (n == 0) return;
    k_crt_split_panel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, rowexp_R, n, ncp, (__half *)res);
}

void launch_crt_split_input(const double *x, const int *perm, int ncol, int ncol_pad, int nrhs, int Et, int b,
                            void *res, unsigned long long *wmax, cudaStream_t st)
{
    cudaMemsetAsync(wmax, 0, sizeof(unsigned long long) * nrhs, st);
    const size_t per_in = (size_t)Et * ncol;
    const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>((per_in + 2047) / 2048, 1216));
    launch_absmax_input(x, per_in, nrhs, gx, wmax, st);
    const size_t per_rhs = (size_t)Et * ncol_pad, total = (size_t)nrhs * per_rhs;
    k_crt_split_input<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(x, perm, ncol, ncol_pad, per_rhs, total, wmax,
                                                                       b, (__half *)res);
}

void launch_crt_combine(const unsigned char *res, int nrhs, int Et, int nt, const int *rowexp,
                        const unsigned long long *wmax, int b, double *f, cudaStream_t st)
{
    const size_t per_rhs = (size_t)Et * nt, per_mod = (size_t)nrhs * per_rhs;
    k_crt_combine<<<(unsigned)((per_mod + 255) / 256), 256, 0, st>>>(res, per_mod, per_rhs, nt, rowexp, wmax, b, f);
}

size_t nf_crt_smem_bytes() { return (size_t)NSTAGE * STAGE_BYTES + 1024 + 256; }

int launch_nf_apply_crt(const CUtensorMap &A, const CUtensorMap &W, const NfCrtParams &P, int nsm, cudaStream_t st,
                        int form)
{
    if (form == 2) {  // two row tiles per CTA, one modulus per item
        NfCrtParams Q = P;
        Q.nitems = kCrtModuli * ((P.ntiles + 1) / 2) * P.nib * P.nrhs;
        const size_t smem = (size_t)NSTAGE2 * STAGE2 + 1024 + 256;
        cudaError_t e = cudaFuncSetAttribute(k_nf_apply_crt2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return -1;
        const int grid = Q.nitems < nsm ? Q.nitems : nsm;
        k_nf_apply_crt2<<<grid, kCrt2Threads, smem, st>>>(A, W, Q);
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    const size_t smem = nf_crt_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_nf_apply_crt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -1;
    const int grid = P.nitems < nsm ? P.nitems : nsm;
    k_nf_apply_crt<<<grid, 192, smem, st>>>(A, W, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace pfmm
