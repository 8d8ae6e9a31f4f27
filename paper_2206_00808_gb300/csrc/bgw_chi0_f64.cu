// FP64 pair weights, Hermitian rank-P update and finalisation of chi0
// (the polarizability formula of arXiv:2206.00808 Sec. II on the imaginary
// axis, omega -> i omega, eta -> 0; no spin-degeneracy factor).
//
// chi0_j[g][g'] = (1/N_k) sum_p w_pj conj(M_p[g]) M_p[g'], w_pj = 2D_p/(D_p^2 + omega_j^2).
// GB300 issues FP64 at a small fraction of its FP32 rate, so these kernels
// are bound by the FP64 pipe: the tiling only has to keep it busy (a few
// warps per SM with 16 independent complex accumulators each) and every
// operand comes from shared memory or L2.
#include <cmath>

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
    const double ev = energy[(long)k * nb + p / nc];
    const double ec = energy[(long)kmap[k] * nb + nv + p % nc];
    const double d = ev - ec;
    const double f = freq[j];
    w[t] = 2.0 * d / (d * d + f * f);
}

constexpr int kTB = 32;   // chi0 tile edge (complex entries)
constexpr int kPK = 16;   // pairs staged per step
constexpr int kHerkThreads = 64;

// Tile index t -> (bi, bj) with bi >= bj, row-major over the lower triangle.
__device__ __forceinline__ void lower_tile(int t, int &bi, int &bj) {
    int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    bi = i;
    bj = t - i * (i + 1) / 2;
}

// acc[j][g][g'] += sum_p w[j][p] conj(M[p][g]) M[p][g'] for one 32x32 tile of
// the lower block triangle and one frequency j.  Each (tile, j) belongs to
// exactly one block, so the read-modify-write of acc needs no atomics and the
// order of the sum over p is fixed.
__global__ void __launch_bounds__(kHerkThreads)
k4_herk_f64(const double2 *__restrict__ M, int P, int ng, const double *__restrict__ w,
            double2 *__restrict__ acc) {
    __shared__ double2 sa[kPK][kTB];
    __shared__ double2 sb[kPK][kTB];
    __shared__ double sw[kPK];
    int bi, bj;
    lower_tile(blockIdx.x, bi, bj);
    const int j = blockIdx.y;
    const double *wj = w + (long)j * P;
    const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;
    const int g0 = bi * kTB, h0 = bj * kTB;

    double re[4][4], im[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) re[r][c] = im[r][c] = 0.0;

    for (int p0 = 0; p0 < P; p0 += kPK) {
        for (int e = threadIdx.x; e < kPK * kTB; e += kHerkThreads) {
            const int pp = e / kTB, i = e % kTB;
            const long p = p0 + pp;
            double2 va = make_double2(0.0, 0.0), vb = va;
            if (p < P) {
                if (g0 + i < ng) va = M[p * ng + g0 + i];
                if (h0 + i < ng) vb = M[p * ng + h0 + i];
            }
            sa[pp][i] = va;
            sb[pp][i] = vb;
        }
        if (threadIdx.x < kPK) sw[threadIdx.x] = (p0 + threadIdx.x < P) ? wj[p0 + threadIdx.x] : 0.0;
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < kPK; ++pp) {
            const double wp = sw[pp];
            double2 a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = sa[pp][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double2 v = sb[pp][tx * 4 + c];
                b[c] = make_double2(v.x * wp, v.y * wp);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // conj(a) * (w b)
                    re[r][c] = fma(a[r].x, b[c].x, fma(a[r].y, b[c].y, re[r][c]));
                    im[r][c] = fma(a[r].x, b[c].y, fma(-a[r].y, b[c].x, im[r][c]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int g = g0 + ty * 4 + r;
        if (g >= ng) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int h = h0 + tx * 4 + c;
            if (h >= ng) continue;
            double2 *o = acc + ((long)j * ng + g) * ng + h;
            double2 v = *o;
            v.x += re[r][c];
            v.y += im[r][c];
            *o = v;
        }
    }
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

cudaError_t herk_f64(const void *M, int P, int ng, const double *w, int nfreq, void *acc,
                     cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    const int nb = (ng + kTB - 1) / kTB;
    dim3 grid(nb * (nb + 1) / 2, nfreq);
    k4_herk_f64<<<grid, kHerkThreads, 0, st>>>(static_cast<const double2 *>(M), P, ng, w,
                                               static_cast<double2 *>(acc));
    return cudaGetLastError();
}

cudaError_t chi0_finalize(const void *acc, int ng, int nfreq, double scale, void *out,
                          cudaStream_t st) {
    const long total = (long)nfreq * ng * ng;
    k7_finalize<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        static_cast<const double2 *>(acc), ng, total, scale, static_cast<double2 *>(out));
    return cudaGetLastError();
}

}  // namespace bgw
