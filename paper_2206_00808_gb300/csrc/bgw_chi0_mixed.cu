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
// loads the four tiles once and issues all three products.  The accumulator
// truncates on every add, so the large hi.hi products go to three TMEM
// accumulators (one per third of K) and the two small cross products to a
// fourth: no accumulator takes more than a third of the large adds, and the
// small terms are not rounded against the large sum.  The epilogue adds the
// four, folds the 2x2 blocks into complex chi and adds them to the FP64
// accumulator (the FP64 reduction across k blocks).
//
// Kernels:
//   k5_split   M -> X planes [1 + nfreq][hi, lo], each stored as tiles
//              [R/128][Kp/64][128 rows][64 pairs] BF16 (K-major inside a tile,
//              zero padded to R = 128-multiple rows, Kp = 64-multiple pairs):
//              one 16 KB TMA box is one contiguous piece of memory, so the
//              split writes and the GEMM loads whole DRAM pages
//   k5_gemm    one CTA per (lower 128x128 tile of D, frequency): TMA loads
//              (128B swizzle) into a 3-stage ring of 64 KB, one thread issues
//              tcgen05.mma, all four warps drain TMEM and update chi in FP64.
// Every mbarrier wait has an iteration limit; on expiry the kernel records
// an error code in *err, waits (bounded) for its own copies in flight,
// frees its tensor memory and returns.
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
constexpr int kBlockK = 64;           // BF16 elements per 128-byte swizzled row
constexpr int kStages = 3;
constexpr int kTileBytes = kTileM * kBlockK * 2;                 // 16 KB per operand tile
constexpr int kStageBytes = 4 * kTileBytes;                      // A_hi, A_lo, B_hi, B_lo
constexpr int kAccCols = 4 * kTileN;                             // 3 hi.hi + 1 cross accumulator
constexpr int kMaxGroup = 48;                                    // q-points per grouped launch
constexpr int kErrFull = 1, kErrEmpty = 2, kErrAccum = 3, kErrDrain = 4;

// ------------------------------------------------------------ split kernel --
// plane 0: A = X; plane 1 + j: B_j = w_j X.  Output [plane][hi|lo] of tiles
// [R/128][Kp/64][128][64].
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

__global__ void __launch_bounds__(256)
k5_split(const float2 *__restrict__ M, int P, int ng, const double *__restrict__ w, int nfreq, int R,
         int Kp, __nv_bfloat16 *__restrict__ X) {
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
    const long planeElems = (long)R * Kp;
    const long kblocks = Kp / kSplitP;                   // 64-pair blocks per row tile
    __nv_bfloat16 *base = X + (((long)(row / 128) * kblocks + p0 / kSplitP) * 128 + row % 128) * kSplitP + pq;
    for (int plane = 0; plane <= nfreq; ++plane) {
        const float *wp = wt + (plane - 1) * kSplitP + pq;
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            float a = x[i], b = x[i + 1];
            if (plane > 0) {
                a *= wp[i];
                b *= wp[i + 1];
            }
            const __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
            const float2 hf = __bfloat1622float2(hh);
            h[i / 2] = bf2_bits(hh);
            l[i / 2] = bf2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
        }
        uint4 *ho = reinterpret_cast<uint4 *>(base + (long)plane * 2 * planeElems);
        uint4 *lo = reinterpret_cast<uint4 *>(base + ((long)plane * 2 + 1) * planeElems);
        ho[0] = make_uint4(h[0], h[1], h[2], h[3]);
        ho[1] = make_uint4(h[4], h[5], h[6], h[7]);
        lo[0] = make_uint4(l[0], l[1], l[2], l[3]);
        lo[1] = make_uint4(l[4], l[5], l[6], l[7]);
    }
}

// One 128 x 64 tile (k-block kb, row tile rt, plane) of the tiled operand
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

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
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
// warp 5 issues the MMAs.  The hi.hi products of each run of kSub K blocks go
// to one of three TMEM slots in turn; when a run completes, warps 0-3 add
// that slot into FP32 registers (round to nearest) and hand it back, so no
// TMEM accumulator takes more than 4*kSub truncating adds of the large
// products whatever K is.  The two cross products go to a fourth slot, read
// once per item; the next item's MMAs start once it has been read.  Barrier
// phases run on across items.
constexpr int kSub = 8;
constexpr int kSlots = 3;
constexpr int kGemmWarps = 6;

struct GroupParams {
    CUtensorMap map[kMaxGroup];   // operand planes of each q-point
    double2 *acc[kMaxGroup];      // FP64 accumulator [nfreq][ng][ng]
    int kp[kMaxGroup];            // padded pair count (multiple of kBlockK)
    int ng[kMaxGroup];
    int first[kMaxGroup + 1];     // first work item of each q-point
    int nq, nfreq;
    int drop_first_load;          // test hook: block 0 never issues its first stage
};

struct Item {
    int q, ti, tj, j, nkb;
};

__device__ __forceinline__ Item decode(const GroupParams &gp, int item) {
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
    it.nkb = gp.kp[q] / kBlockK;
    return it;
}

__global__ void __launch_bounds__(kGemmWarps * 32, 1)
k5_gemm(const __grid_constant__ GroupParams gp, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages];
    __shared__ __align__(8) uint64_t empty_bar[kStages];
    __shared__ __align__(8) uint64_t slot_full[kSlots];
    __shared__ __align__(8) uint64_t slot_free[kSlots];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ __align__(8) uint64_t tmem_free;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int total = gp.first[gp.nq];

    // 1024-byte aligned stage ring
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t ring = (raw + 1023u) & ~1023u;

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
            long pit = 0, issued_from = 0, dropped = -1;
            for (int item = blockIdx.x; item < total; item += gridDim.x) {
                const Item w = decode(gp, item);
                const CUtensorMap *map = &gp.map[w.q];
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
                const int bhi = 2 + 2 * w.j, blo = 3 + 2 * w.j;
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
                    tma_load_tile(st0, map, fb, it, w.ti, 0);
                    tma_load_tile(st0 + kTileBytes, map, fb, it, w.ti, 1);
                    tma_load_tile(st0 + 2 * kTileBytes, map, fb, it, w.tj, bhi);
                    tma_load_tile(st0 + 3 * kTileBytes, map, fb, it, w.tj, blo);
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
                const Item w = decode(gp, item);
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
                    const uint64_t ahi = smem_desc(st0), alo = smem_desc(st0 + kTileBytes);
                    const uint64_t bhd = smem_desc(st0 + 2 * kTileBytes), bld = smem_desc(st0 + 3 * kTileBytes);
                    const uint32_t acc_hh = tmem + (uint32_t)(slot * kTileN);
#pragma unroll
                    for (int k = 0; k < kBlockK / 16; ++k) {
                        // advance 16 BF16 = 32 bytes along K inside the swizzled row
                        const uint64_t o = (uint64_t)(2 * k);
                        mma_bf16(acc_hh, ahi + o, bhd + o, (first_in_sub && k == 0) ? 0u : 1u);
                        mma_bf16(acc_x, ahi + o, bld + o, (it == 0 && k == 0) ? 0u : 1u);
                        mma_bf16(acc_x, alo + o, bhd + o, 1u);
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
    } else {
        // warps 0-3: promote finished hi.hi slots into FP32 registers, then
        // fold the tile into complex chi and add it in FP64
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        long gsub = 0;
        int nitem = 0;
        for (int item = blockIdx.x; item < total; item += gridDim.x, ++nitem) {
            const Item w = decode(gp, item);
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
#pragma unroll
            for (int c0 = 0; c0 < kTileN; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(lane_base + (uint32_t)(kSlots * kTileN + c0), v);   // cross terms
#pragma unroll
                for (int i = 0; i < 32; ++i) racc[c0 + i] += __uint_as_float(v[i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&tmem_free));   // the MMAs of the next item may start
            const int ng = gp.ng[w.q];
            double2 *acc = gp.acc[w.q];
            const int a_row = w.ti * kTileM, b_row = w.tj * kTileN;
            const int r = 32 * warp + lane;            // tile row
            const int g = (a_row + r) >> 1;            // complex row
            const bool even = (r & 1) == 0;
#pragma unroll
            for (int c0 = 0; c0 < kTileN; c0 += 32) {
                float other[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) other[i] = __shfl_xor_sync(0xffffffffu, racc[c0 + i], 1);
                // rows 2g (re-row) and 2g+1 (im-row) now sit in both lanes of the pair;
                // the even lane writes column pairs 0..7 of this chunk, the odd lane 8..15.
                if (g < ng) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int cc = 2 * q;
                        const float d00 = even ? racc[c0 + cc] : other[cc];           // D[2g][2g']
                        const float d01 = even ? racc[c0 + cc + 1] : other[cc + 1];   // D[2g][2g'+1]
                        const float d10 = even ? other[cc] : racc[c0 + cc];           // D[2g+1][2g']
                        const float d11 = even ? other[cc + 1] : racc[c0 + cc + 1];   // D[2g+1][2g'+1]
                        const int gp2 = (b_row + c0 + cc) >> 1;
                        if ((q < 8) == even && gp2 < ng) {
                            double2 *o = acc + ((long)w.j * ng + g) * ng + gp2;
                            double2 t = *o;
                            t.x += (double)d00 + (double)d11;
                            t.y += (double)d01 - (double)d10;
                            *o = t;
                        }
                    }
                }
            }
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

size_t mixed_workspace_bytes(long P, int ng, int nfreq) {
    const long R = round_up(2L * ng, kTileM);
    const long Kp = round_up(P, kBlockK);
    return (size_t)(1 + nfreq) * 2 * R * Kp * sizeof(__nv_bfloat16) + 256;
}

cudaError_t mixed_split(const void *M, int P, int ng, const double *w, int nfreq, void *ws,
                        cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    const long R = round_up(2L * ng, kTileM);
    const long Kp = round_up(P, kBlockK);
    // R is a multiple of 128 (64 real rows per block) and Kp of 64
    dim3 sgrid((unsigned)(Kp / kSplitP), (unsigned)(R / (2 * kSplitG)));
    const size_t smem = sizeof(float) * split_smem_floats(nfreq);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k5_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k5_split<<<sgrid, 256, smem, st>>>(static_cast<const float2 *>(M), P, ng, w, nfreq, (int)R, (int)Kp,
                                       static_cast<__nv_bfloat16 *>(ws));
    return cudaGetLastError();
}

int mixed_max_group() { return kMaxGroup; }

cudaError_t mixed_gemm(const MixedQ *qs, int nq, int nfreq, int sm_count, cudaStream_t st, int *err,
                       int drop_first_load) {
    if (nq < 1 || nq > kMaxGroup) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    GroupParams gp;
    memset(&gp, 0, sizeof gp);
    gp.nq = nq;
    gp.nfreq = nfreq;
    gp.drop_first_load = drop_first_load;
    int items = 0;
    for (int i = 0; i < nq; ++i) {
        gp.first[i] = items;
        const long R = round_up(2L * qs[i].ng, kTileM);
        const long Kp = round_up(qs[i].P, kBlockK);
        const int nt = (int)(R / kTileM);
        if (qs[i].P > 0) items += nt * (nt + 1) / 2 * nfreq;
        gp.kp[i] = (int)Kp;
        gp.ng[i] = qs[i].ng;
        gp.acc[i] = static_cast<double2 *>(qs[i].acc);
        // tiled planes [plane][R/128][Kp/64][128][64]: a box is one whole tile
        const int planes = 2 * (1 + nfreq);
        const cuuint64_t tile = (cuuint64_t)kTileM * kBlockK * 2;
        const cuuint64_t dims[5] = {(cuuint64_t)kBlockK, (cuuint64_t)kTileM, (cuuint64_t)(Kp / kBlockK),
                                    (cuuint64_t)(R / kTileM), (cuuint64_t)planes};
        const cuuint64_t strides[4] = {(cuuint64_t)kBlockK * 2, tile, tile * (cuuint64_t)(Kp / kBlockK),
                                       tile * (cuuint64_t)(Kp / kBlockK) * (cuuint64_t)(R / kTileM)};
        const cuuint32_t box[5] = {kBlockK, kTileM, 1, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        CUresult cr = g_encode(&gp.map[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, qs[i].ws, dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    gp.first[nq] = items;
    if (items == 0) return cudaSuccess;
    const int smem = kStages * kStageBytes + 1024;
    e = cudaFuncSetAttribute(k5_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = items < sm_count ? items : sm_count;
    k5_gemm<<<grid, kGemmWarps * 32, smem, st>>>(gp, err);
    return cudaGetLastError();
}

}  // namespace bgw
