// FP64 pair weights, Hermitian rank-P update and finalisation of chi0
// (the polarizability formula of arXiv:2206.00808 Sec. II on the imaginary
// axis, omega -> i omega, eta -> 0; no spin-degeneracy factor).
//
// chi0_j[g][g'] = (1/N_k) sum_p w_pj conj(M_p[g]) M_p[g'], w_pj = 2D_p/(D_p^2 + omega_j^2).
// GB300 issues FP64 at a small fraction of its FP32 rate, so these kernels
// are bound by the FP64 pipe: what matters is the FP64 operation count per
// useful multiply-add and keeping every SM busy to the end (the pair range
// is split so the blocks fill several waves; the partial sums are reduced in
// a fixed order, so results are reproducible).
#include <algorithm>
#include <cmath>

#include "bgw_bounds.cuh"
#include "bgw_internal.h"

namespace bgw {
namespace {

// w[j][kl*P + v*nc + c] for the kn k-points k0..k0+kn-1 of one q-point;
// kmap[k] is the grid index k' of k + q.
__global__ void k3_pair_weights(const double *__restrict__ energy, int nb, int nv, int nc,
                                const int *__restrict__ kmap, int k0, int kn,
                                const double *__restrict__ freq, int nfreq, double *__restrict__ w) {
    const long P = (long)nv * nc;
    const long PT = P * kn;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= PT * nfreq) return;
    const long pt = t % PT;
    const int j = (int)(t / PT);
    const int kl = (int)(pt / P);
    const long p = pt % P;
    const int k = k0 + kl;
    const int kq = kmap[k];
    if (!BGW_IN_BOUNDS(kq >= 0, kBoundsKMap)) {
        w[t] = 0.0;
        return;
    }
    const double ev = energy[(long)k * nb + p / nc];
    const double ec = energy[(long)kq * nb + nv + p % nc];
    const double d = ev - ec;
    const double f = freq[j];
    w[t] = 2.0 * d / (d * d + f * f);
}

constexpr int kTB = 32;   // chi0 tile edge (complex entries)
constexpr int kPK = 16;   // pairs staged per step
constexpr int kHerkThreads = 256;   // 16 x 16 threads, 2 x 2 outputs each
constexpr int kMaxW = 5;  // frequencies per block (more spill at two blocks per SM)

// Tile index t -> (bi, bj) with bi >= bj, row-major over the lower triangle.
__device__ __forceinline__ void lower_tile(int t, int &bi, int &bj) {
    int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    bi = i;
    bj = t - i * (i + 1) / 2;
}

// Partial sums part[s][j][g][g'] = sum_{p in range s} w[j][p] conj(M[p][g]) M[p][g']
// for one 32x32 tile of the lower block triangle, pair range s and
// frequencies j0..j0+NW-1.  The product conj(M_g) M_g' is formed once per
// pair and weighted for every frequency (4 + 2 NW FP64 operations per entry
// and pair instead of 4 NW).
template <int NW>
__global__ void __launch_bounds__(kHerkThreads, 2)
k4_herk_f64(const double2 *__restrict__ M, int P, int ng, const double *__restrict__ w, int nfreq,
            int prange, double2 *__restrict__ part) {
    __shared__ double2 sa[kPK][kTB];
    __shared__ double2 sb[kPK][kTB];
    __shared__ double sw[NW][kPK];
    int bi, bj;
    lower_tile(blockIdx.x, bi, bj);
    const int s = blockIdx.y;
    const int j0 = blockIdx.z * NW;
    const int nw = min(NW, nfreq - j0);
    const int p_begin = s * prange, p_end = min(P, p_begin + prange);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int g0 = bi * kTB, h0 = bj * kTB;

    double re[NW][2][2], im[NW][2][2];
#pragma unroll
    for (int j = 0; j < NW; ++j)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) re[j][r][c] = im[j][r][c] = 0.0;

    for (int p0 = p_begin; p0 < p_end; p0 += kPK) {
        for (int e = threadIdx.x; e < kPK * kTB; e += kHerkThreads) {
            const int pp = e / kTB, i = e % kTB;
            const long p = p0 + pp;
            double2 va = make_double2(0.0, 0.0), vb = va;
            if (p < p_end) {
                if (g0 + i < ng) va = M[p * ng + g0 + i];
                if (h0 + i < ng) vb = M[p * ng + h0 + i];
            }
            sa[pp][i] = va;
            sb[pp][i] = vb;
        }
        if (threadIdx.x < NW * kPK) {
            const int j = threadIdx.x / kPK, pp = threadIdx.x % kPK;
            sw[j][pp] = (j < nw && p0 + pp < p_end) ? w[(long)(j0 + j) * P + p0 + pp] : 0.0;
        }
        __syncthreads();
#pragma unroll 2
        for (int pp = 0; pp < kPK; ++pp) {
            const double2 a0 = sa[pp][ty * 2], a1 = sa[pp][ty * 2 + 1];
            const double2 b0 = sb[pp][tx * 2], b1 = sb[pp][tx * 2 + 1];
            double pr[2][2], pi[2][2];
            // conj(a) * b
            pr[0][0] = fma(a0.x, b0.x, a0.y * b0.y);
            pi[0][0] = fma(a0.x, b0.y, -a0.y * b0.x);
            pr[0][1] = fma(a0.x, b1.x, a0.y * b1.y);
            pi[0][1] = fma(a0.x, b1.y, -a0.y * b1.x);
            pr[1][0] = fma(a1.x, b0.x, a1.y * b0.y);
            pi[1][0] = fma(a1.x, b0.y, -a1.y * b0.x);
            pr[1][1] = fma(a1.x, b1.x, a1.y * b1.y);
            pi[1][1] = fma(a1.x, b1.y, -a1.y * b1.x);
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                const double wj = sw[j][pp];
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        re[j][r][c] = fma(wj, pr[r][c], re[j][r][c]);
                        im[j][r][c] = fma(wj, pi[r][c], im[j][r][c]);
                    }
            }
        }
        __syncthreads();
    }
    const long nn = (long)ng * ng;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        if (j >= nw) break;
        double2 *pj = part + ((long)s * nfreq + j0 + j) * nn;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int g = g0 + ty * 2 + r;
            if (g >= ng) continue;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int h = h0 + tx * 2 + c;
                if (h < ng) pj[(long)g * ng + h] = make_double2(re[j][r][c], im[j][r][c]);
            }
        }
    }
}

// acc[j][g][g'] += sum_{s < S} part[s][j][g][g'] in order of s, on the lower
// block triangle (the entries the partial kernel wrote).
__global__ void k4_reduce(const double2 *__restrict__ part, int S, int ng, int nfreq,
                          double2 *__restrict__ acc) {
    const long nn = (long)ng * ng;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nn * nfreq) return;
    const int g = (int)((t % nn) / ng), h = (int)(t % ng);
    if (g / kTB < h / kTB) return;
    double2 v = acc[t];
    for (int s = 0; s < S; ++s) {
        const double2 q = part[(long)s * nn * nfreq + t];
        v.x += q.x;
        v.y += q.y;
    }
    acc[t] = v;
}

__global__ void k7_finalize(const double2 *__restrict__ acc, int ng, long total, double scale,
                            double2 *__restrict__ out) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const long nn = (long)ng * ng;
    const long j = t / nn;
    const int g = (int)((t % nn) / ng), h = (int)(t % ng);
    double2 v;
    if (g == h) {
        v = acc[j * nn + (long)g * ng + h];
        v.y = 0.0;   // the diagonal of a Hermitian matrix is real
    } else if (g > h) {
        v = acc[j * nn + (long)g * ng + h];
    } else {
        v = acc[j * nn + (long)h * ng + g];
        v.y = -v.y;
    }
    out[t] = make_double2(v.x * scale, v.y * scale);
}

}  // namespace

cudaError_t pair_weights(const double *energy, int nb, int nv, int nc, const int *kmap, int k0,
                         int kn, const double *freq, int nfreq, double *w, cudaStream_t st) {
    const long n = (long)nv * nc * kn * nfreq;
    if (n == 0) return cudaSuccess;
    k3_pair_weights<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(energy, nb, nv, nc, kmap, k0, kn,
                                                                 freq, nfreq, w);
    return cudaGetLastError();
}

int herk_f64_splits(int P, int ng, int nfreq, int sm_count) {
    const int nb = (ng + kTB - 1) / kTB;
    const int tiles = nb * (nb + 1) / 2;
    const int nwc = (nfreq + kMaxW - 1) / kMaxW;
    const int target = 4 * 2 * sm_count;   // four waves of two blocks per SM
    int S = (target + tiles * nwc - 1) / (tiles * nwc);
    S = std::max(1, std::min(S, (P + 63) / 64));
    return S;
}

size_t herk_f64_workspace_bytes(int P, int ng, int nfreq, int sm_count) {
    return sizeof(double2) * (size_t)herk_f64_splits(P, ng, nfreq, sm_count) * nfreq * ng * ng;
}

cudaError_t herk_f64(const void *M, int P, int ng, const double *w, int nfreq, void *acc, void *ws,
                     int sm_count, cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    const int nb = (ng + kTB - 1) / kTB;
    const int S = herk_f64_splits(P, ng, nfreq, sm_count);
    const int prange = (((P + S - 1) / S) + kPK - 1) / kPK * kPK;
    // frequencies per block: all of them up to kMaxW, else chunks of kMaxW
    const int NWr = std::min(nfreq, kMaxW);
    dim3 grid(nb * (nb + 1) / 2, S, (nfreq + NWr - 1) / NWr);
    const double2 *Mp = static_cast<const double2 *>(M);
    double2 *part = static_cast<double2 *>(ws);
    switch (NWr) {
        case 1: k4_herk_f64<1><<<grid, kHerkThreads, 0, st>>>(Mp, P, ng, w, nfreq, prange, part); break;
        case 2: k4_herk_f64<2><<<grid, kHerkThreads, 0, st>>>(Mp, P, ng, w, nfreq, prange, part); break;
        case 3: k4_herk_f64<3><<<grid, kHerkThreads, 0, st>>>(Mp, P, ng, w, nfreq, prange, part); break;
        case 4: k4_herk_f64<4><<<grid, kHerkThreads, 0, st>>>(Mp, P, ng, w, nfreq, prange, part); break;
        default: k4_herk_f64<5><<<grid, kHerkThreads, 0, st>>>(Mp, P, ng, w, nfreq, prange, part); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long total = (long)nfreq * ng * ng;
    k4_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, S, ng, nfreq,
                                                               static_cast<double2 *>(acc));
    return cudaGetLastError();
}

cudaError_t bounds_take_chi0(unsigned *word) { return bgw_bounds_take(word); }

cudaError_t chi0_finalize(const void *acc, int ng, int nfreq, double scale, void *out,
                          cudaStream_t st) {
    const long total = (long)nfreq * ng * ng;
    k7_finalize<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        static_cast<const double2 *>(acc), ng, total, scale, static_cast<double2 *>(out));
    return cudaGetLastError();
}

}  // namespace bgw
