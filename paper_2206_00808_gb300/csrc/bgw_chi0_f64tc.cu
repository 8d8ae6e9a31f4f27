// FP64-accurate contraction of chi0 on tcgen05 tensor cores (sm_103a).
//
// chi0_j[g][g'] += sum_p w_pj conj(M_p[g]) M_p[g']  (the P formula of
// arXiv:2206.00808 Sec. II on the imaginary axis, w_pj = 2D/(D^2 + w_j^2) <= 0).
// With s_pj = sqrt(-w_pj) and the interleaved rows
//   Y_j[2g][p] = s_pj Re M_p[g],  Y_j[2g+1][p] = s_pj Im M_p[g],
// D_j = -Y_j Y_j^T and Re chi = D[2g][2g'] + D[2g+1][2g'+1],
// Im chi = D[2g][2g'+1] - D[2g+1][2g'].
//
// FP64 accuracy from BF16 products: each row r of Y_j gets an exponent e with
// |Y[r][p]| <= 2^(e-1) for every pair, and Y 2^(40-e) rounded to an integer N
// (|N| <= 2^39) is cut into signed base-256 digits d_0..d_4 in [-128, 128]:
//   Y = 2^(e-8) sum_t S_t + O(2^(e-41)),   S_t = d_t 2^(-8t)  (exact in BF16).
// Then Y Y^T = 2^(e_r + e_r' - 16) sum_{t,u} S_t S_u^T, and the 15 products
// with t + u <= 4 are kept (the rest are ~2^-40 of the result).  The products
// of one order t + u are integers in units of 2^(-8(t+u)); over 224 pairs the
// sums of orders 0, 1 and 2 stay below 2^24 units (1, 2 and 3 products of at
// most 128^2 per pair), so an FP32 accumulator holds them exactly whatever its
// rounding.  Orders 3 and 4 share a fourth accumulator, whose rounding is
// ~2^-48 of the result.  Every 224 pairs the epilogue moves the three exact
// sums into int32 registers (in their own units) and the fourth into FP32, and
// it folds them into the FP64 accumulator of chi every 128 such steps and at
// the end of each work item.
//
// Kernels:
//   k5z_rowmax  per frequency and row, max_p |Y| in FP32 (an upper bound
//               with margin), merged across blocks by atomicMax on float bits
//   k5z_split   Y in FP64, N by the 1.5 * 2^52 rounding constant, the digits
//               by integer shifts; the five planes per frequency stored as
//               tiles [R/128][Kp/32][128 rows][32 pairs] of BF16 (64-byte rows)
//   k5z_gemm    persistent, one CTA per SM over (lower 128 x 64 tile of D,
//               frequency) items: warp 8 issues TMA loads (64-byte swizzle; the
//               ten digit tiles of a 32-pair block form one 60 KB stage of a
//               3-stage ring), warp 9 issues the 30 MMAs per block
//               (M = 128, N = 64, K = 16) into one of two sets of four TMEM
//               accumulators, warps 0-7 promote and fold.
// Every mbarrier wait is bounded; on expiry the kernel records an error code,
// waits (bounded) for its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <climits>
#include <cstdint>
#include <cstring>

#include "bgw_f64tc.h"
#include "bgw_tc_common.cuh"

namespace bgw {
namespace {

using namespace tc;

constexpr int kM = 128;                       // rows of D per item (A rows)
constexpr int kN = 64;                        // columns of D per item (B rows)
constexpr int kKB = 32;                       // pairs per K block: one 64-byte row of BF16
constexpr int kSl = 5;                        // base-256 digits per value
constexpr int kStg = 3;
constexpr int kTileA = kM * kKB * 2;          // 8 KB
constexpr int kTileB = kN * kKB * 2;          // 4 KB
constexpr int kStage = kSl * (kTileA + kTileB);   // 60 KB
constexpr int kSub = 7;                       // K blocks per promotion (224 pairs)
constexpr int kFlush = 128;                   // promotions between FP64 folds
constexpr int kAcc = 4;                       // orders 0, 1, 2 and 3-4
constexpr int kCols = 2 * kAcc * kN;          // two sets: 512 TMEM columns
constexpr int kThreads = 10 * 32;             // warps 0-7 epilogue, 8 TMA, 9 MMA
constexpr int kErrFull = 1, kErrEmpty = 2, kErrAccum = 3, kErrDrain = 4;
constexpr int kErrSign = F64TC_ERR_SIGN;      // a pair weight > 0 (see f64tc_contract)

// ---------------------------------------------------------- row maxima --
constexpr int kRmP = 256, kRmG = 32, kRmF = 16;

__global__ void __launch_bounds__(256)
k5z_rowmax(const double2 *__restrict__ M, int P, int ng, const double *__restrict__ w, int nfreq, int R,
           unsigned *__restrict__ rmax, int *__restrict__ err) {
    __shared__ float sv[kRmF][kRmP];
    __shared__ float red[8][kRmF][2][kRmG];
    const int p0 = blockIdx.x * kRmP, g0 = blockIdx.y * kRmG;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = g0 + lane;
    for (int j0 = 0; j0 < nfreq; j0 += kRmF) {
        const int nj = min(kRmF, nfreq - j0);
        __syncthreads();
        for (int i = threadIdx.x; i < kRmF * kRmP; i += 256) {
            const int j = i / kRmP, pp = i % kRmP, p = p0 + pp;
            float s = 0.f;
            if (j < nj && p < P) {
                const double wv = w[(long)(j0 + j) * P + p];
                s = wv < 0.0 ? sqrtf((float)(-wv)) : 0.f;
                if (wv > 0.0) atomicExch(err, kErrSign);
            }
            sv[j][pp] = s;
        }
        __syncthreads();
        float mr[kRmF], mi[kRmF];
#pragma unroll
        for (int j = 0; j < kRmF; ++j) mr[j] = mi[j] = 0.f;
        for (int pp = warp; pp < kRmP && p0 + pp < P; pp += 8) {
            float ar = 0.f, ai = 0.f;
            if (g < ng) {
                const double2 m = M[(long)(p0 + pp) * ng + g];
                ar = fabsf((float)m.x);
                ai = fabsf((float)m.y);
            }
#pragma unroll
            for (int j = 0; j < kRmF; ++j) {
                mr[j] = fmaxf(mr[j], sv[j][pp] * ar);
                mi[j] = fmaxf(mi[j], sv[j][pp] * ai);
            }
        }
#pragma unroll
        for (int j = 0; j < kRmF; ++j) {
            red[warp][j][0][lane] = mr[j];
            red[warp][j][1][lane] = mi[j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kRmF * 2 * kRmG; i += 256) {
            const int j = i / (2 * kRmG), c = (i / kRmG) % 2, l = i % kRmG;
            float m = 0.f;
            for (int q = 0; q < 8; ++q) m = fmaxf(m, red[q][j][c][l]);
            const int gg = g0 + l;
            if (j < nj && gg < ng && m > 0.f) atomicMax(&rmax[(long)(j0 + j) * R + 2 * gg + c], __float_as_uint(m));
        }
    }
}

// ------------------------------------------------------------ digits --
constexpr int kSpG = 32;   // complex G per block (64 real rows)
constexpr int kSpP = 32;   // pairs per block (one K block)

// Exponent of a row from its maximum |Y| (float bits; 0 for an all-zero row):
// the smallest e with 2^(e-1) >= max (1 + 2^-20), the margin covering the
// FP32 rounding of the bound.
__device__ __forceinline__ int row_exponent(unsigned mb) {
    if (mb == 0u) return 0;
    const float mm = __fmul_ru(__uint_as_float(mb), 1.0f + 0x1p-20f);
    int k;
    frexpf(mm, &k);   // mm = f 2^k, f in [1/2, 1): mm < 2^k
    return k + 1;
}

// Signed base-256 digits of N = rint(y sc), |N| <= 2^39 (1 + 2^-20):
// N = d0 2^32 + d1 2^24 + d2 2^16 + d3 2^8 + d4, every |d_t| <= 128.
__device__ __forceinline__ void digits(double y, double sc, int (&d)[kSl]) {
    const double magic = 6755399441055744.0;   // 1.5 * 2^52: fma rounds y sc to an integer
    long long n = __double_as_longlong(fma(y, sc, magic)) - __double_as_longlong(magic);
    d[0] = (int)((n + (1LL << 31)) >> 32);
    n -= (long long)d[0] << 32;
    d[1] = (int)((n + (1LL << 23)) >> 24);
    n -= (long long)d[1] << 24;
    d[2] = (int)((n + (1LL << 15)) >> 16);
    n -= (long long)d[2] << 16;
    d[3] = (int)((n + (1LL << 7)) >> 8);
    n -= (long long)d[3] << 8;
    d[4] = (int)n;
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }

// One block: 64 real rows (32 complex G) x 32 pairs, every frequency.  Each
// thread takes one row and 8 pairs: per frequency and digit one 16-byte store.
__global__ void __launch_bounds__(256)
k5z_split(const double2 *__restrict__ M, int P, int ng, const double *__restrict__ w, int nfreq, int R, int Kp,
          const unsigned *__restrict__ rmax, int *__restrict__ rexp, __nv_bfloat16 *__restrict__ X) {
    __shared__ double2 sm[kSpP][kSpG + 1];
    __shared__ double ss[kSpP];
    const int p0 = blockIdx.x * kSpP, g0 = blockIdx.y * kSpG;
    for (int i = threadIdx.x; i < kSpP * kSpG; i += 256) {
        const int pp = i / kSpG, gg = i % kSpG;
        const int p = p0 + pp, g = g0 + gg;
        sm[pp][gg] = (p < P && g < ng) ? M[(long)p * ng + g] : make_double2(0.0, 0.0);
    }
    const int r = threadIdx.x / 4;              // local real row
    const int pq = (threadIdx.x % 4) * 8;       // first of this thread's 8 pairs
    const int row = 2 * g0 + r;
    const long kblocks = Kp / kKB;
    const long planeElems = (long)R * Kp;
    __nv_bfloat16 *base = X + (((long)(row / kM) * kblocks + p0 / kKB) * kM + row % kM) * kKB + pq;
    const float dscale[kSl] = {1.0f, 0x1p-8f, 0x1p-16f, 0x1p-24f, 0x1p-32f};
    for (int j = 0; j < nfreq; ++j) {
        __syncthreads();
        if (threadIdx.x < kSpP) {
            const int p = p0 + threadIdx.x;
            const double wv = p < P ? w[(long)j * P + p] : 0.0;
            ss[threadIdx.x] = wv < 0.0 ? sqrt(-wv) : 0.0;
        }
        __syncthreads();
        const int e = row_exponent(rmax[(long)j * R + row]);
        if (blockIdx.x == 0 && (threadIdx.x % 4) == 0) rexp[(long)j * R + row] = e;
        const double sc = __longlong_as_double((long long)(1023 + 40 - e) << 52);   // 2^(40-e)
        uint32_t h[kSl][4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            const double2 ma = sm[pq + i][r >> 1], mb = sm[pq + i + 1][r >> 1];
            int da[kSl], db[kSl];
            digits(ss[pq + i] * ((r & 1) ? ma.y : ma.x), sc, da);
            digits(ss[pq + i + 1] * ((r & 1) ? mb.y : mb.x), sc, db);
#pragma unroll
            for (int t = 0; t < kSl; ++t)
                h[t][i / 2] = bf2_bits(__floats2bfloat162_rn((float)da[t] * dscale[t], (float)db[t] * dscale[t]));
        }
#pragma unroll
        for (int t = 0; t < kSl; ++t)
            *reinterpret_cast<uint4 *>(base + ((long)j * kSl + t) * planeElems) =
                make_uint4(h[t][0], h[t][1], h[t][2], h[t][3]);
    }
}

// ---------------------------------------------------------------- GEMM --
// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 B, 8-row swizzle atoms 512 B apart (SBO), version 1.
__device__ __forceinline__ uint64_t desc64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)4 << 61;             // 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_z(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// 64 rows x 32 pairs (4 KB) at coordinates {0, row, kb, rt, plane} of the
// 5-D map of the digit planes.
__device__ __forceinline__ void tma_rows(uint32_t dst, const CUtensorMap *map, uint32_t bar, int row, int kb,
                                         int rt, int plane) {
    const int zero = 0;
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(zero), "r"(row), "r"(kb), "r"(rt), "r"(plane)
        : "memory");
}

struct ZParams {
    CUtensorMap map;        // digit planes [nfreq * 5][R/128][Kp/32][128][32]
    double2 *acc;           // FP64 accumulator [nfreq][ng][ng]
    const int *rexp;        // row exponents [nfreq][R]
    int ng, R, nt, nkb, items;
};

// Work item -> (row tile ti of 128, column block tj of 64, frequency j):
// frequency-major, then the lower tiles tj <= 2 ti + 1 row by row.
__device__ __forceinline__ void decode(const ZParams &zp, int item, int &ti, int &tj, int &j) {
    const int per = zp.nt * (zp.nt + 1);
    j = item / per;
    const int t = item % per;
    int i = (int)((sqrt(4.0 * t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) <= t) ++i;
    while (i * (i + 1) > t) --i;
    ti = i;
    tj = t - i * (i + 1);
}

__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Fold the running sums of one tile row (32 columns of this thread) into
// the complex FP64 accumulator and clear them.
__device__ __forceinline__ void fold(const ZParams &zp, int j, int grow, int gcol0, int (&a0)[32], int (&a1)[32],
                                     int (&a2)[32], float (&a3)[32], int lane) {
    const int er = zp.rexp[(long)j * zp.R + grow];
    const int g = grow >> 1;
    const bool even = (grow & 1) == 0;
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 8) {
        double d[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ec = zp.rexp[(long)j * zp.R + gcol0 + c0 + i];
            const long long n = ((long long)a0[c0 + i] << 16) + ((long long)a1[c0 + i] << 8) + (long long)a2[c0 + i];
            const double v = fma((double)n, 0x1p-16, (double)a3[c0 + i]);
            d[i] = -v * pow2(er + ec - 16);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = __shfl_xor_sync(0xffffffffu, d[i], 1);
        // rows 2g (even lane) and 2g+1 (odd lane): the even lane writes the
        // first two complex columns of these eight real ones, the odd lane the
        // last two
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            if ((qq < 2) != even) continue;
            const double d00 = even ? d[2 * qq] : o[2 * qq];           // D[2g][2g']
            const double d01 = even ? d[2 * qq + 1] : o[2 * qq + 1];   // D[2g][2g'+1]
            const double d10 = even ? o[2 * qq] : d[2 * qq];           // D[2g+1][2g']
            const double d11 = even ? o[2 * qq + 1] : d[2 * qq + 1];   // D[2g+1][2g'+1]
            const int gp = (gcol0 + c0 + 2 * qq) >> 1;
            if (g < zp.ng && gp < zp.ng) {
                double2 *out = zp.acc + ((long)j * zp.ng + g) * zp.ng + gp;
                double2 t = *out;
                t.x += d00 + d11;
                t.y += d01 - d10;
                *out = t;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        a0[i] = a1[i] = a2[i] = 0;
        a3[i] = 0.f;
    }
    (void)lane;
}

__global__ void __launch_bounds__(kThreads, 1) k5z_gemm(const __grid_constant__ ZParams zp, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStg];
    __shared__ __align__(8) uint64_t empty_bar[kStg];
    __shared__ __align__(8) uint64_t set_full[2];
    __shared__ __align__(8) uint64_t set_free[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t ring = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStg; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&set_full[s]), 1);
            mbar_init(smem_u32(&set_free[s]), 256);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 8) {
        if (lane == 0) {
            // TMA producer: per 32-pair block the five A digit tiles (two
            // 64-row loads each) and the five B digit tiles of the frequency
            long pit = 0;
            for (int item = blockIdx.x; item < zp.items; item += gridDim.x) {
                int ti, tj, j;
                decode(zp, item, ti, tj, j);
                const CUtensorMap *map = &zp.map;
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
                for (int kb = 0; kb < zp.nkb; ++kb, ++pit) {
                    const int s = (int)(pit % kStg);
                    if (!mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((pit / kStg) & 1) ^ 1))) {
                        atomicExch(err, kErrEmpty);
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                    if (*(volatile int *)&abort_flag) break;
                    const uint32_t st0 = ring + s * kStage;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect_tx(fb, kStage);
                    for (int t = 0; t < kSl; ++t) {
                        const int plane = j * kSl + t;
                        tma_rows(st0 + t * kTileA, map, fb, 0, kb, ti, plane);
                        tma_rows(st0 + t * kTileA + kTileA / 2, map, fb, 64, kb, ti, plane);
                        tma_rows(st0 + kSl * kTileA + t * kTileB, map, fb, (tj & 1) * 64, kb, tj >> 1, plane);
                    }
                }
                if (*(volatile int *)&abort_flag) break;
            }
            // every issued load must land before the CTA can exit
            for (long q = pit > kStg ? pit - kStg : 0; q < pit; ++q) {
                if (!mbar_wait(smem_u32(&full_bar[q % kStg]), (uint32_t)((q / kStg) & 1))) {
                    atomicExch(err, kErrDrain);
                    break;
                }
            }
        }
        __syncwarp();
    } else if (warp == 9) {
        if (lane == 0) {
            // MMA issuer: 15 digit products per 16-pair step, orders 0, 1, 2
            // and 3-4 into the four accumulators of the current set
            long pit = 0, gsub = 0;
            bool stop = false;
            for (int item = blockIdx.x; item < zp.items && !stop; item += gridDim.x) {
                int ti, tj, j;
                decode(zp, item, ti, tj, j);
                int set = 0;
                for (int kb = 0; kb < zp.nkb; ++kb, ++pit) {
                    const bool first = (kb % kSub) == 0;
                    if (first) {
                        set = (int)(gsub & 1);
                        if (!mbar_wait(smem_u32(&set_free[set]), (uint32_t)(((gsub >> 1) & 1) ^ 1))) {
                            atomicExch(err, kErrAccum);
                            atomicExch(&abort_flag, 1);
                            stop = true;
                            break;
                        }
                    }
                    const int s = (int)(pit % kStg);
                    if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((pit / kStg) & 1))) {
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
                    const uint32_t st0 = ring + s * kStage;
                    const uint32_t accb = tmem + (uint32_t)(set * kAcc * kN);
#pragma unroll
                    for (int k = 0; k < kKB / 16; ++k) {
                        const uint64_t o = (uint64_t)(2 * k);   // 16 BF16 = 32 bytes along K
#pragma unroll
                        for (int t = 0; t < kSl; ++t) {
                            const uint64_t ad = desc64(st0 + t * kTileA) + o;
#pragma unroll
                            for (int u = 0; u + t < kSl; ++u) {
                                const int lev = (t + u) < 3 ? (t + u) : 3;
                                const uint64_t bd = desc64(st0 + kSl * kTileA + u * kTileB) + o;
                                const bool start = first && k == 0 && t == 0 && u <= 3;
                                mma_z(accb + (uint32_t)(lev * kN), ad, bd, start ? 0u : 1u);
                            }
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[s]));
                    if ((kb % kSub) == kSub - 1 || kb == zp.nkb - 1) {
                        mma_commit(smem_u32(&set_full[set]));
                        ++gsub;
                    }
                }
            }
        }
        __syncwarp();
    } else {
        // warps 0-7: warp w reads TMEM lanes 32 (w & 3).. (tile rows) and
        // columns 32 (w >> 2).. of each accumulator
        const int quarter = warp & 3, half = warp >> 2;
        const int r = 32 * quarter + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * half);
        int a0[32], a1[32], a2[32];
        float a3[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            a0[i] = a1[i] = a2[i] = 0;
            a3[i] = 0.f;
        }
        long gsub = 0;
        for (int item = blockIdx.x; item < zp.items; item += gridDim.x) {
            int ti, tj, j;
            decode(zp, item, ti, tj, j);
            const int nsub = (zp.nkb + kSub - 1) / kSub;
            const int grow = ti * kM + r, gcol0 = tj * kN + 32 * half;
            bool ok = true;
            for (int sub = 0; sub < nsub; ++sub, ++gsub) {
                const int set = (int)(gsub & 1);
                bool got = mbar_wait(smem_u32(&set_full[set]), (uint32_t)((gsub >> 1) & 1));
                got = __all_sync(0xffffffffu, got && !*(volatile int *)&abort_flag);
                if (!got) {
                    if (lane == 0) atomicExch(err, kErrAccum);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = lane_base + (uint32_t)(set * kAcc * kN);
                uint32_t v[32];
                tmem_ld32(sb, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) a0[i] += __float2int_rn(__uint_as_float(v[i]));
                tmem_ld32(sb + kN, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) a1[i] += __float2int_rn(__uint_as_float(v[i]) * 256.0f);
                tmem_ld32(sb + 2 * kN, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) a2[i] += __float2int_rn(__uint_as_float(v[i]) * 65536.0f);
                tmem_ld32(sb + 3 * kN, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) a3[i] += __uint_as_float(v[i]);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(smem_u32(&set_free[set]));
                if ((sub + 1) % kFlush == 0 || sub == nsub - 1) fold(zp, j, grow, gcol0, a0, a1, a2, a3, lane);
            }
            if (!ok) {
                atomicExch(&abort_flag, 1);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

long round_up(long x, long m) { return (x + m - 1) / m * m; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;

}  // namespace

size_t f64tc_workspace_bytes(long P, int ng, int nfreq) {
    const long R = round_up(2L * ng, kM);
    const long Kp = round_up(P, kKB);
    return align256((size_t)nfreq * kSl * R * Kp * sizeof(__nv_bfloat16)) + 2 * align256(sizeof(int) * (size_t)nfreq * R);
}

cudaError_t f64tc_contract(const void *M, int P, int ng, const double *w, int nfreq, void *acc, void *ws,
                           int sm_count, cudaStream_t st, int *err) {
    if (P == 0) return cudaSuccess;
    cudaError_t e = tc::tensor_map_encoder(&g_enc);
    if (e != cudaSuccess) return e;
    const long R = round_up(2L * ng, kM);
    const long Kp = round_up(P, kKB);
    const size_t planes = align256((size_t)nfreq * kSl * R * Kp * sizeof(__nv_bfloat16));
    __nv_bfloat16 *X = static_cast<__nv_bfloat16 *>(ws);
    unsigned *rmax = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + planes);
    int *rexp = reinterpret_cast<int *>(static_cast<char *>(ws) + planes + align256(sizeof(int) * (size_t)nfreq * R));
    e = cudaMemsetAsync(rmax, 0, sizeof(unsigned) * (size_t)nfreq * R, st);
    if (e != cudaSuccess) return e;
    const double2 *Md = static_cast<const double2 *>(M);
    dim3 g1((unsigned)((P + kRmP - 1) / kRmP), (unsigned)((ng + kRmG - 1) / kRmG));
    k5z_rowmax<<<g1, 256, 0, st>>>(Md, P, ng, w, nfreq, (int)R, rmax, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)(Kp / kSpP), (unsigned)(R / (2 * kSpG)));
    k5z_split<<<g2, 256, 0, st>>>(Md, P, ng, w, nfreq, (int)R, (int)Kp, rmax, rexp, X);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    ZParams zp;
    memset(&zp, 0, sizeof zp);
    const cuuint64_t tile = (cuuint64_t)kM * kKB * 2;
    const cuuint64_t dims[5] = {(cuuint64_t)kKB, (cuuint64_t)kM, (cuuint64_t)(Kp / kKB), (cuuint64_t)(R / kM),
                                (cuuint64_t)nfreq * kSl};
    const cuuint64_t strides[4] = {(cuuint64_t)kKB * 2, tile, tile * (cuuint64_t)(Kp / kKB),
                                   tile * (cuuint64_t)(Kp / kKB) * (cuuint64_t)(R / kM)};
    const cuuint32_t box[5] = {kKB, 64, 1, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult cr = g_enc(&zp.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, X, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    zp.acc = static_cast<double2 *>(acc);
    zp.rexp = rexp;
    zp.ng = ng;
    zp.R = (int)R;
    zp.nt = (int)(R / kM);
    zp.nkb = (int)(Kp / kKB);
    zp.items = nfreq * zp.nt * (zp.nt + 1);
    const int smem = kStg * kStage + 1024;
    e = cudaFuncSetAttribute(k5z_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = zp.items < sm_count ? zp.items : sm_count;
    k5z_gemm<<<grid, kThreads, smem, st>>>(zp, err);
    return cudaGetLastError();
}

}  // namespace bgw
