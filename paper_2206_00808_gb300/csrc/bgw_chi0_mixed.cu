// Mixed-precision contraction of chi0 on tcgen05 tensor cores (sm_103a).
//
// chi0_j[g][g'] += sum_p w_pj conj(M_p[g]) M_p[g']   (the polarizability
// formula of arXiv:2206.00808 Sec. II on the imaginary axis; M complex64,
// w FP64).  In real form with the interleaved rows x_{2g} = Re M_g,
// x_{2g+1} = Im M_g:
//   D_j[r][r'] = sum_p w_pj x_r(p) x_r'(p),
//   Re chi = D[2g][2g'] + D[2g+1][2g'+1],  Im chi = D[2g][2g'+1] - D[2g+1][2g'].
// D_j is a GEMM with K = pairs: A = X (shared by every frequency) and
// B_j = w_j X.  Each operand is split into BF16 hi + lo (x ~ hi + lo to
// ~2^-17 relative) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi runs on tcgen05
// kind::f16 with FP32 accumulation in tensor memory.  Each 64-pair K block
// loads the four tiles once and issues all three products.  Two TF32 forms
// use the same kernels on kind::tf32: three products of TF32 hi + lo
// (x ~ hi + lo to ~2^-22; 32-pair K blocks, half the BF16 MMA rate), or the
// single product hi.hi (~2^-11 per operand).  The accumulator
// truncates on every add, so the large hi.hi products rotate over three TMEM
// accumulators that are drained into FP32 registers (round to nearest) every
// kSub K blocks, and the two small cross products go to a fourth: no
// accumulator takes more than 4 kSub large adds, and the small terms are not
// rounded against the large sum.  At each work item's end the sums are
// folded from 2x2 real blocks into complex chi and added to the FP64
// accumulator (the FP64 reduction across k blocks).
//
// Kernels:
//   k5_split   M -> X planes [1 + nfreq][hi, lo] (hi only for one product),
//              each stored as tiles [R/128][Kp/Kb][128 rows][Kb pairs] of
//              128-byte rows (Kb = 64 BF16 or 32 TF32; K-major inside a tile,
//              zero padded to R = 128-multiple rows, Kp = 64-multiple pairs):
//              one 16 KB TMA box is one contiguous piece of memory, so the
//              split writes and the GEMM loads whole DRAM pages
//   k5_gemm    persistent, one CTA per SM walking the work items (lower
//              128x128 tile of D, frequency) of every q-point of a group: TMA
//              loads (128B swizzle) into a ring of 192 KB (3 stages of four
//              tiles, or 6 of two for one product), one thread issues
//              tcgen05.mma, four warps drain TMEM and fold each finished tile
//              into a complex FP32 tile in shared memory, two warps add that
//              tile to chi in FP64.
// Every mbarrier wait gives up after about 2 s (with an iteration backstop);
// on expiry the kernel records an error code in *err, waits (bounded) for its
// own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "bgw_mixed.h"
#include "bgw_tc_common.cuh"

namespace bgw {
namespace {

using namespace tc;

constexpr int kTileM = 128;           // rows of D per CTA (A rows)
constexpr int kTileN = 128;           // columns of D per CTA (B rows)
constexpr int kRowBytes = 128;        // one swizzled operand row (K-major)
constexpr int kTileBytes = kTileM * kRowBytes;                   // 16 KB per operand tile
constexpr int kPadK = 64;             // pair padding of the planes (both formats)
constexpr int kAccCols = 4 * kTileN;                             // 3 hi.hi + 1 cross accumulator
constexpr int kMaxGroup = 48;                                    // q-points per grouped launch
constexpr int kErrFull = 1, kErrEmpty = 2, kErrAccum = 3, kErrDrain = 4;

// Operand format F (the kMixed* values): element size, pairs per 128-byte
// row, hi/lo planes per operand, ring depth and the MMA instruction
// descriptor (D = F32, A = B = BF16 or TF32, both K-major, M = N = 128).
template <int F>
struct Fmt {
    static constexpr bool tf32 = F != kMixedBF16x3;
    static constexpr bool three = F != kMixedTF32;
    static constexpr int esize = tf32 ? 4 : 2;
    static constexpr int blockK = kRowBytes / esize;
    static constexpr int halves = three ? 2 : 1;
    static constexpr int stageBytes = 2 * halves * kTileBytes;
    static constexpr int stages = three ? 3 : 6;
    static constexpr uint32_t ab = tf32 ? 2u : 1u;
    static constexpr uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                                      ((uint32_t)(kTileM >> 4) << 24);
};

// ------------------------------------------------------------ split kernel --
// operand 0: A = X; operand 1 + j: B_j = w_j X.  Output [operand][hi|lo] of
// tiles [R/128][Kp/Kb][128][Kb].
// One CTA per (32 complex G = 64 real rows) x (64 pairs) block writes every
// plane of that block: M is read once, the weights are converted to FP32
// once per pair, and each thread stores 16 consecutive pairs of one row
// (two 16-byte stores per plane and half).  Rows 2*ng..R-1 and pairs
// P..Kp-1 are written as zeros.
constexpr int kSplitG = 32;
constexpr int kSplitP = 64;
constexpr int kSplitRow = kSplitG + 1;                  // padded shared row (floats)

__host__ __device__ constexpr size_t split_smem_floats(int nfreq) {
    return (size_t)2 * kSplitP * kSplitRow + 16 + (size_t)nfreq * kSplitP;
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) {
    return *reinterpret_cast<uint32_t *>(&v);
}

// Nearest TF32 value (10 stored mantissa bits), ties away from zero: add half
// a unit of the 13 dropped bits to the magnitude, then clear them (a carry
// into the exponent is the correct rounding up).
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <int F>
__global__ void __launch_bounds__(256)
k5_split(const float2 *__restrict__ M, int P, int ng, const double *__restrict__ w, int nfreq, int R,
         int Kp, uint8_t *__restrict__ X) {
    using T = Fmt<F>;
    extern __shared__ float split_sm[];
    float *re = split_sm;                                // [kSplitP][kSplitRow]
    float *im = re + kSplitP * kSplitRow + 16;           // offset by 16 banks from re
    float *wt = im + kSplitP * kSplitRow;                // [nfreq][kSplitP]
    // blockIdx.x runs along the pairs, so CTAs resident together write
    // neighbouring 128-byte pieces of the same rows (whole DRAM pages)
    const int p0 = blockIdx.x * kSplitP, g0 = blockIdx.y * kSplitG;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    // one FP64 -> FP32 conversion per pair and frequency (the FP64 unit is slow on this part)
    for (int i = threadIdx.x; i < nfreq * kSplitP; i += 256) {
        const int j = i / kSplitP, p = p0 + i % kSplitP;
        wt[i] = p < P ? (float)w[(long)j * P + p] : 0.f;
    }
    for (int i = ty; i < kSplitP; i += 8) {
        const int p = p0 + i, g = g0 + tx;
        float2 v = make_float2(0.f, 0.f);
        if (p < P && g < ng) v = M[(long)p * ng + g];
        re[i * kSplitRow + tx] = v.x;
        im[i * kSplitRow + tx] = v.y;
    }
    __syncthreads();
    // four threads per row (16 pairs each): a warp stores 8 whole rows of the
    // tile, 1 KB of contiguous memory
    const int r = threadIdx.x / 4;                       // local real row: G = g0 + r/2, Re/Im = r&1
    const int pq = (threadIdx.x % 4) * 16;               // first of this thread's 16 pairs
    const int row = 2 * g0 + r;
    const float *src = ((r & 1) ? im : re) + (r >> 1);
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = src[(pq + i) * kSplitRow];
    const long planeBytes = (long)R * Kp * T::esize;
    const long kblocks = Kp / T::blockK;                 // K blocks per row tile
    const int pc = p0 + pq;                              // this thread's first pair
    uint8_t *base = X + ((((long)(row / 128) * kblocks + pc / T::blockK) * 128 + row % 128) * T::blockK +
                         pc % T::blockK) * T::esize;
    constexpr int kWords = 16 * T::esize / 4;            // 16 pairs in 32-bit words
    for (int op = 0; op <= nfreq; ++op) {
        const float *wp = wt + (op - 1) * kSplitP + pq;
        uint32_t h[kWords], l[kWords];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            float a = x[i], b = x[i + 1];
            if (op > 0) {
                a *= wp[i];
                b *= wp[i + 1];
            }
            if constexpr (T::tf32) {
                const float ha = tf32_round(a), hb = tf32_round(b);
                h[i] = __float_as_uint(ha);
                h[i + 1] = __float_as_uint(hb);
                l[i] = __float_as_uint(tf32_round(a - ha));
                l[i + 1] = __float_as_uint(tf32_round(b - hb));
            } else {
                const __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
                const float2 hf = __bfloat1622float2(hh);
                h[i / 2] = bf2_bits(hh);
                l[i / 2] = bf2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
            }
        }
        uint4 *ho = reinterpret_cast<uint4 *>(base + (long)op * T::halves * planeBytes);
#pragma unroll
        for (int v = 0; v < kWords / 4; ++v) ho[v] = make_uint4(h[4 * v], h[4 * v + 1], h[4 * v + 2], h[4 * v + 3]);
        if constexpr (T::three) {
            uint4 *lo = reinterpret_cast<uint4 *>(base + ((long)op * 2 + 1) * planeBytes);
#pragma unroll
            for (int v = 0; v < kWords / 4; ++v)
                lo[v] = make_uint4(l[4 * v], l[4 * v + 1], l[4 * v + 2], l[4 * v + 3]);
        }
    }
}

// One 128-row tile (k-block kb, row tile rt, plane) of the tiled operand
// layout: coordinates {0, 0, kb, rt, plane} of the 5-D map.
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap *map, uint32_t bar, int kb,
                                              int rt, int plane) {
    const int zero = 0;
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(zero), "r"(kb), "r"(rt), "r"(plane)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 B, 8-row swizzle atoms 1024 B apart (SBO), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// D (+)= A B^T for one 32-byte K step: kind::f16 (BF16) or kind::tf32.
template <int F>
__device__ __forceinline__ void mma_step(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    if constexpr (Fmt<F>::tf32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(Fmt<F>::idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(Fmt<F>::idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void lower_tile(int t, int &bi, int &bj) {
    int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    bi = i;
    bj = t - i * (i + 1) / 2;
}

// --------------------------------------------------------------- GEMM --
// Persistent grouped kernel: the work items of every q-point of a group
// (lower 128x128 tiles x frequencies, tile-major so the CTAs of one wave
// share A tiles in L2) are dealt round-robin to one CTA per SM.
// Warp roles: warps 0-3 drain tensor memory (warp w owns TMEM lanes
// 32w..32w+31 = tile rows), warp 4 allocates TMEM and issues the TMA loads,
// warp 5 issues the MMAs, warps 6-7 add finished tiles to the FP64
// accumulator.  The hi.hi products of each run of kSub K blocks go to one of
// three TMEM slots in turn; when a run completes, warps 0-3 add that slot
// into FP32 registers (round to nearest) and hand it back, so no TMEM
// accumulator takes more than 4*kSub truncating adds of the large products
// whatever K is.  The two cross products go to a fourth slot, read once per
// item; the next item's MMAs start once it has been read.  Warps 0-3 then
// fold the 2x2 real blocks into a complex FP32 tile in shared memory and go
// back to draining slots, while warps 6-7 add that tile into chi in FP64 (the
// slow FP64 pipe stays off the path that frees the slots).  Barrier phases
// run on across items.
constexpr int kSub = 8;
constexpr int kSlots = 3;
constexpr int kGemmWarps = 8;
constexpr int kFoldRow = kTileN / 2 + 1;                          // padded row of the complex tile
constexpr int kFoldBytes = kTileM / 2 * kFoldRow * 8;             // 64 x 65 complex FP32

struct GroupParams {
    CUtensorMap map[kMaxGroup];   // operand planes of each q-point
    double2 *acc[kMaxGroup];      // FP64 accumulator [nfreq][ng][ng]
    int kp[kMaxGroup];            // padded pair count (multiple of kPadK)
    int ng[kMaxGroup];
    int first[kMaxGroup + 1];     // first work item of each q-point
    int nq, nfreq;
    int drop_first_load;          // test hook: block 0 never issues its first stage
};

struct Item {
    int q, ti, tj, j, nkb;
};

__device__ __forceinline__ Item decode(const GroupParams &gp, int item, int blockK) {
    Item it;
    int q = 0;
    while (q + 1 < gp.nq && gp.first[q + 1] <= item) ++q;
    // frequency-major within a q-point: the CTAs working at the same time
    // cover whole lower triangles of one or two frequencies, so they share
    // the A tiles (every frequency) and each B_j tile (every row below it)
    // while they stream K together, and most operand reads hit L2
    const int local = item - gp.first[q];
    const int ntiles = (gp.first[q + 1] - gp.first[q]) / gp.nfreq;
    lower_tile(local % ntiles, it.ti, it.tj);
    it.q = q;
    it.j = local / ntiles;
    it.nkb = gp.kp[q] / blockK;
    return it;
}

template <int F>
__global__ void __launch_bounds__(kGemmWarps * 32, 1)
k5_gemm(const __grid_constant__ GroupParams gp, int *__restrict__ err) {
    using T = Fmt<F>;
    constexpr int kStages = T::stages, kStageBytes = T::stageBytes;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages];
    __shared__ __align__(8) uint64_t empty_bar[kStages];
    __shared__ __align__(8) uint64_t slot_full[kSlots];
    __shared__ __align__(8) uint64_t slot_free[kSlots];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ __align__(8) uint64_t tmem_free;
    __shared__ __align__(8) uint64_t fold_full;   // warps 0-3 wrote the complex tile
    __shared__ __align__(8) uint64_t fold_free;   // warps 6-7 added it to chi
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int total = gp.first[gp.nq];

    // 1024-byte aligned stage ring, then the complex FP32 tile [64][kFoldRow]
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t ring = (raw + 1023u) & ~1023u;
    float2 *ftile = reinterpret_cast<float2 *>(smem_raw + (ring - raw) + kStages * kStageBytes);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(smem_u32(&slot_full[s]), 1);
            mbar_init(smem_u32(&slot_free[s]), 128);
        }
        mbar_init(smem_u32(&accum_bar), 1);
        mbar_init(smem_u32(&tmem_free), 128);
        mbar_init(smem_u32(&fold_full), 128);
        mbar_init(smem_u32(&fold_free), 64);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kAccCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        if (lane == 0) {
            // TMA producer; planes: 0 A_hi, 1 A_lo, 2 + 2j B_j hi, 3 + 2j B_j lo
            // (one product: 0 A, 1 + j B_j)
            long pit = 0, issued_from = 0, dropped = -1;
            for (int item = blockIdx.x; item < total; item += gridDim.x) {
                const Item w = decode(gp, item, T::blockK);
                const CUtensorMap *map = &gp.map[w.q];
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
                const int bhi = T::halves * (1 + w.j), blo = bhi + 1;
                for (int it = 0; it < w.nkb; ++it, ++pit) {
                    const int s = (int)(pit % kStages);
                    if (!mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((pit / kStages) & 1) ^ 1))) {
                        atomicExch(err, kErrEmpty);
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                    if (*(volatile int *)&abort_flag) break;
                    if (gp.drop_first_load && blockIdx.x == 0 && pit == 0) {   // test hook
                        dropped = pit;
                        continue;
                    }
                    const uint32_t st0 = ring + s * kStageBytes;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    if constexpr (T::three) {
                        tma_load_tile(st0, map, fb, it, w.ti, 0);
                        tma_load_tile(st0 + kTileBytes, map, fb, it, w.ti, 1);
                        tma_load_tile(st0 + 2 * kTileBytes, map, fb, it, w.tj, bhi);
                        tma_load_tile(st0 + 3 * kTileBytes, map, fb, it, w.tj, blo);
                    } else {
                        tma_load_tile(st0, map, fb, it, w.ti, 0);
                        tma_load_tile(st0 + kTileBytes, map, fb, it, w.tj, bhi);
                    }
                }
                if (*(volatile int *)&abort_flag) break;
            }
            // every issued load must land before the CTA can exit
            issued_from = pit > kStages ? pit - kStages : 0;
            for (long q = issued_from; q < pit; ++q) {
                if (q == dropped) continue;
                if (!mbar_wait(smem_u32(&full_bar[q % kStages]), (uint32_t)((q / kStages) & 1))) {
                    atomicExch(err, kErrDrain);
                    break;
                }
            }
        }
        __syncwarp();
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t acc_x = tmem + (uint32_t)(kSlots * kTileN);
            long pit = 0, gsub = 0;
            int nitem = 0;
            bool stop = false;
            for (int item = blockIdx.x; item < total && !stop; item += gridDim.x, ++nitem) {
                const Item w = decode(gp, item, T::blockK);
                if (nitem > 0 && !mbar_wait(smem_u32(&tmem_free), (uint32_t)((nitem - 1) & 1))) {
                    atomicExch(err, kErrAccum);
                    atomicExch(&abort_flag, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                int slot = 0;
                for (int it = 0; it < w.nkb; ++it, ++pit) {
                    const bool first_in_sub = (it % kSub) == 0;
                    if (first_in_sub) {
                        slot = (int)(gsub % kSlots);
                        if (!mbar_wait(smem_u32(&slot_free[slot]), (uint32_t)(((gsub / kSlots) & 1) ^ 1))) {
                            atomicExch(err, kErrAccum);
                            atomicExch(&abort_flag, 1);
                            stop = true;
                            break;
                        }
                    }
                    const int s = (int)(pit % kStages);
                    if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((pit / kStages) & 1))) {
                        atomicExch(err, kErrFull);
                        atomicExch(&abort_flag, 1);
                        stop = true;
                        break;
                    }
                    if (*(volatile int *)&abort_flag) {
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st0 = ring + s * kStageBytes;
                    const uint32_t acc_hh = tmem + (uint32_t)(slot * kTileN);
                    if constexpr (T::three) {
                        const uint64_t ahi = smem_desc(st0), alo = smem_desc(st0 + kTileBytes);
                        const uint64_t bhd = smem_desc(st0 + 2 * kTileBytes), bld = smem_desc(st0 + 3 * kTileBytes);
#pragma unroll
                        for (int k = 0; k < kRowBytes / 32; ++k) {
                            // advance 32 bytes along K inside the swizzled row (16 BF16 or 8 TF32)
                            const uint64_t o = (uint64_t)(2 * k);
                            mma_step<F>(acc_hh, ahi + o, bhd + o, (first_in_sub && k == 0) ? 0u : 1u);
                            mma_step<F>(acc_x, ahi + o, bld + o, (it == 0 && k == 0) ? 0u : 1u);
                            mma_step<F>(acc_x, alo + o, bhd + o, 1u);
                        }
                    } else {
                        const uint64_t ad = smem_desc(st0), bd = smem_desc(st0 + kTileBytes);
#pragma unroll
                        for (int k = 0; k < kRowBytes / 32; ++k) {
                            const uint64_t o = (uint64_t)(2 * k);
                            mma_step<F>(acc_hh, ad + o, bd + o, (first_in_sub && k == 0) ? 0u : 1u);
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[s]));
                    if ((it % kSub) == kSub - 1 || it == w.nkb - 1) {
                        mma_commit(smem_u32(&slot_full[slot]));
                        ++gsub;
                    }
                }
                mma_commit(smem_u32(&accum_bar));
            }
        }
        __syncwarp();
    } else if (warp >= 6) {
        // warps 6-7: add each finished complex tile to chi in FP64 (a warp
        // takes 32 consecutive columns of a row: whole 512-byte segments)
        const int tid = threadIdx.x - 6 * 32;
        int nitem = 0;
        for (int item = blockIdx.x; item < total; item += gridDim.x, ++nitem) {
            const Item w = decode(gp, item, T::blockK);
            bool ok = mbar_wait(smem_u32(&fold_full), (uint32_t)(nitem & 1));
            if (!ok && lane == 0) atomicExch(err, kErrAccum);
            ok = __all_sync(0xffffffffu, ok && !*(volatile int *)&abort_flag);
            if (!ok) {
                atomicExch(&abort_flag, 1);
                break;
            }
            const int ng = gp.ng[w.q];
            double2 *acc = gp.acc[w.q] + (long)w.j * ng * ng;
            const int g0 = w.ti * (kTileM / 2), h0 = w.tj * (kTileN / 2);
            for (int i = tid; i < (kTileM / 2) * (kTileN / 2); i += 64) {
                const int gl = i / (kTileN / 2), hl = i % (kTileN / 2);
                const int g = g0 + gl, h = h0 + hl;
                if (g < ng && h < ng) {
                    const float2 v = ftile[gl * kFoldRow + hl];
                    double2 *o = acc + (long)g * ng + h;
                    double2 t = *o;
                    t.x += (double)v.x;
                    t.y += (double)v.y;
                    *o = t;
                }
            }
            mbar_arrive(smem_u32(&fold_free));
        }
    } else {
        // warps 0-3: promote finished hi.hi slots into FP32 registers, then
        // fold the 2x2 real blocks into the complex FP32 tile
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        long gsub = 0;
        int nitem = 0;
        for (int item = blockIdx.x; item < total; item += gridDim.x, ++nitem) {
            const Item w = decode(gp, item, T::blockK);
            const int nsub = (w.nkb + kSub - 1) / kSub;
            float racc[kTileN];
#pragma unroll
            for (int i = 0; i < kTileN; ++i) racc[i] = 0.f;
            bool ok = true;
            for (int sub = 0; sub < nsub; ++sub, ++gsub) {
                const int slot = (int)(gsub % kSlots);
                bool got = mbar_wait(smem_u32(&slot_full[slot]), (uint32_t)((gsub / kSlots) & 1));
                got = __all_sync(0xffffffffu, got && !*(volatile int *)&abort_flag);
                if (!got) {
                    if (lane == 0) atomicExch(err, kErrAccum);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int c0 = 0; c0 < kTileN; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(lane_base + (uint32_t)(slot * kTileN + c0), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) racc[c0 + i] += __uint_as_float(v[i]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(smem_u32(&slot_free[slot]));
            }
            if (ok) {
                ok = mbar_wait(smem_u32(&accum_bar), (uint32_t)(nitem & 1));
                if (!ok && lane == 0) atomicExch(err, kErrAccum);
                ok = __all_sync(0xffffffffu, ok && !*(volatile int *)&abort_flag);   // warp-uniform
            }
            if (!ok) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if constexpr (T::three) {
#pragma unroll
                for (int c0 = 0; c0 < kTileN; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(lane_base + (uint32_t)(kSlots * kTileN + c0), v);   // cross terms
#pragma unroll
                    for (int i = 0; i < 32; ++i) racc[c0 + i] += __uint_as_float(v[i]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&tmem_free));   // the MMAs of the next item may start
            // the previous item's tile must have been added to chi
            if (nitem > 0) {
                bool fr = mbar_wait(smem_u32(&fold_free), (uint32_t)((nitem - 1) & 1));
                if (!fr && lane == 0) atomicExch(err, kErrAccum);
                fr = __all_sync(0xffffffffu, fr && !*(volatile int *)&abort_flag);
                if (!fr) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
            }
            const int r = 32 * warp + lane;            // tile row
            const bool even = (r & 1) == 0;
            float2 *frow = ftile + (r >> 1) * kFoldRow;
#pragma unroll
            for (int c0 = 0; c0 < kTileN; c0 += 32) {
                float other[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) other[i] = __shfl_xor_sync(0xffffffffu, racc[c0 + i], 1);
                // rows 2g (re-row) and 2g+1 (im-row) now sit in both lanes of the pair;
                // the even lane writes column pairs 0..7 of this chunk, the odd lane 8..15
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int cc = 2 * q;
                    const float d00 = even ? racc[c0 + cc] : other[cc];           // D[2g][2g']
                    const float d01 = even ? racc[c0 + cc + 1] : other[cc + 1];   // D[2g][2g'+1]
                    const float d10 = even ? other[cc] : racc[c0 + cc];           // D[2g+1][2g']
                    const float d11 = even ? other[cc + 1] : racc[c0 + cc + 1];   // D[2g+1][2g'+1]
                    if ((q < 8) == even) frow[(c0 + cc) >> 1] = make_float2(d00 + d11, d01 - d10);
                }
            }
            mbar_arrive(smem_u32(&fold_full));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAccCols)
                     : "memory");
    }
}

// ---------------------------------------------------------- tensor map --
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() { return tc::tensor_map_encoder(&g_encode); }

long round_up(long x, long m) { return (x + m - 1) / m * m; }

}  // namespace

static bool known_format(int fmt) { return fmt == kMixedBF16x3 || fmt == kMixedTF32x3 || fmt == kMixedTF32; }

static int elem_size(int fmt) { return fmt == kMixedBF16x3 ? 2 : 4; }

static int halves(int fmt) { return fmt == kMixedTF32 ? 1 : 2; }

size_t mixed_workspace_bytes(long P, int ng, int nfreq, int fmt) {
    const long R = round_up(2L * ng, kTileM);
    const long Kp = round_up(P, kPadK);
    return (size_t)(1 + nfreq) * halves(fmt) * R * Kp * elem_size(fmt) + 256;
}

namespace {

template <int F>
cudaError_t split_launch(const void *M, int P, int ng, const double *w, int nfreq, void *ws, cudaStream_t st) {
    const long R = round_up(2L * ng, kTileM);
    const long Kp = round_up(P, kPadK);
    // R is a multiple of 128 (64 real rows per block) and Kp of 64
    dim3 sgrid((unsigned)(Kp / kSplitP), (unsigned)(R / (2 * kSplitG)));
    const size_t smem = sizeof(float) * split_smem_floats(nfreq);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k5_split<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k5_split<F><<<sgrid, 256, smem, st>>>(static_cast<const float2 *>(M), P, ng, w, nfreq, (int)R, (int)Kp,
                                          static_cast<uint8_t *>(ws));
    return cudaGetLastError();
}

template <int F>
cudaError_t gemm_launch(const GroupParams &gp, int items, int sm_count, cudaStream_t st, int *err) {
    const int smem = Fmt<F>::stages * Fmt<F>::stageBytes + 1024 + kFoldBytes;
    cudaError_t e = cudaFuncSetAttribute(k5_gemm<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = items < sm_count ? items : sm_count;
    k5_gemm<F><<<grid, kGemmWarps * 32, smem, st>>>(gp, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mixed_split(const void *M, int P, int ng, const double *w, int nfreq, void *ws, int fmt,
                        cudaStream_t st) {
    if (!known_format(fmt)) return cudaErrorInvalidValue;
    if (P == 0) return cudaSuccess;
    switch (fmt) {
        case kMixedTF32x3: return split_launch<kMixedTF32x3>(M, P, ng, w, nfreq, ws, st);
        case kMixedTF32: return split_launch<kMixedTF32>(M, P, ng, w, nfreq, ws, st);
        default: return split_launch<kMixedBF16x3>(M, P, ng, w, nfreq, ws, st);
    }
}

int mixed_max_group() { return kMaxGroup; }

cudaError_t mixed_gemm(const MixedQ *qs, int nq, int nfreq, int fmt, int sm_count, cudaStream_t st, int *err,
                       int drop_first_load) {
    if (nq < 1 || nq > kMaxGroup || !known_format(fmt)) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    const int es = elem_size(fmt), blockK = kRowBytes / es;
    GroupParams gp;
    memset(&gp, 0, sizeof gp);
    gp.nq = nq;
    gp.nfreq = nfreq;
    gp.drop_first_load = drop_first_load;
    int items = 0;
    for (int i = 0; i < nq; ++i) {
        gp.first[i] = items;
        const long R = round_up(2L * qs[i].ng, kTileM);
        const long Kp = round_up(qs[i].P, kPadK);
        const int nt = (int)(R / kTileM);
        if (qs[i].P > 0) items += nt * (nt + 1) / 2 * nfreq;
        gp.kp[i] = (int)Kp;
        gp.ng[i] = qs[i].ng;
        gp.acc[i] = static_cast<double2 *>(qs[i].acc);
        // tiled planes [plane][R/128][Kp/Kb][128][Kb]: a box is one whole tile
        const int planes = halves(fmt) * (1 + nfreq);
        const cuuint64_t tile = (cuuint64_t)kTileBytes;
        const cuuint64_t nkb = (cuuint64_t)(Kp / blockK);
        const cuuint64_t dims[5] = {(cuuint64_t)blockK, (cuuint64_t)kTileM, nkb, (cuuint64_t)(R / kTileM),
                                    (cuuint64_t)planes};
        const cuuint64_t strides[4] = {(cuuint64_t)kRowBytes, tile, tile * nkb, tile * nkb * (cuuint64_t)(R / kTileM)};
        const cuuint32_t box[5] = {(cuuint32_t)blockK, kTileM, 1, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        CUresult cr = g_encode(&gp.map[i], es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               5, qs[i].ws, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    gp.first[nq] = items;
    if (items == 0) return cudaSuccess;
    switch (fmt) {
        case kMixedTF32x3: return gemm_launch<kMixedTF32x3>(gp, items, sm_count, st, err);
        case kMixedTF32: return gemm_launch<kMixedTF32>(gp, items, sm_count, st, err);
        default: return gemm_launch<kMixedBF16x3>(gp, items, sm_count, st, err);
    }
}

}  // namespace bgw
