// FP64 complex products for the steps after chi0 that contract matrix
// elements with an interaction (arXiv:2206.00808, Sec. II): the static
// screened-exchange and Coulomb-hole terms of the self-energy (the
// M* M eps^-1 v sums of Eqs. sigma_sx and sigma_coh) and the exchange and
// direct BSE kernels (the K^X and K^D integrals, both traces of spin-summed
// matrix elements).  All of them are products of an M block with a diagonal
// or dense interaction matrix; they run on the FP64 pipe.
//
//   k9_zgemm   C(m, n) = beta C(m, n) + alpha sum_k opA(m, k) w_k opB(k, n) with
//              arbitrary element strides, optional conjugation of either
//              operand and an optional real weight per k; 32 x 32 tiles of C,
//              16 k per shared-memory stage, 2 x 2 outputs per thread
//   k9_rowdot  s[p] = Re sum_g conj(M[p][g]) Y[p][g] and t[p] = sum_g v_g |M[p][g]|^2
//   k9_sum     per-band sums of those over the other band index, in order
//   k9_perm    K[(v c)][(v' c')] = T[(c c')][(v v')]
#include <cuda_runtime.h>

#include "bgw_internal.h"

namespace bgw {
namespace {

constexpr int kT = 32;
constexpr int kK = 16;

template <bool CA, bool CB>
__global__ void __launch_bounds__(256)
k9_zgemm(int M, int N, int K, const double2 *__restrict__ A, long sam, long sak, const double2 *__restrict__ B,
         long sbk, long sbn, const double *__restrict__ wk, double2 *__restrict__ C, long scm, long scn,
         double ar, double ai, int beta) {
    __shared__ double2 sa[kK][kT];
    __shared__ double2 sb[kK][kT];
    const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double re[2][2] = {{0, 0}, {0, 0}}, im[2][2] = {{0, 0}, {0, 0}};
    for (int k0 = 0; k0 < K; k0 += kK) {
        for (int e = threadIdx.x; e < kK * kT; e += 256) {
            const int kk = e / kT, i = e % kT;
            const int k = k0 + kk;
            double2 a = make_double2(0.0, 0.0), b = a;
            if (k < K) {
                if (m0 + i < M) {
                    a = A[(long)(m0 + i) * sam + (long)k * sak];
                    if (CA) a.y = -a.y;
                    if (wk) {
                        const double w = wk[k];
                        a.x *= w;
                        a.y *= w;
                    }
                }
                if (n0 + i < N) {
                    b = B[(long)k * sbk + (long)(n0 + i) * sbn];
                    if (CB) b.y = -b.y;
                }
            }
            sa[kk][i] = a;
            sb[kk][i] = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kK; ++kk) {
            const double2 a0 = sa[kk][ty * 2], a1 = sa[kk][ty * 2 + 1];
            const double2 b0 = sb[kk][tx * 2], b1 = sb[kk][tx * 2 + 1];
            const double2 a[2] = {a0, a1}, b[2] = {b0, b1};
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    re[r][c] = fma(a[r].x, b[c].x, fma(-a[r].y, b[c].y, re[r][c]));
                    im[r][c] = fma(a[r].x, b[c].y, fma(a[r].y, b[c].x, im[r][c]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int m = m0 + ty * 2 + r;
        if (m >= M) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int n = n0 + tx * 2 + c;
            if (n >= N) continue;
            double2 *o = C + (long)m * scm + (long)n * scn;
            double2 v = make_double2(ar * re[r][c] - ai * im[r][c], ar * im[r][c] + ai * re[r][c]);
            if (beta) {
                const double2 old = *o;
                v.x += old.x;
                v.y += old.y;
            }
            *o = v;
        }
    }
}

// One warp per row p: s[p] = Re sum_g conj(M[p][g]) Y[p][g]; t[p] = sum_g v_g |M[p][g]|^2
// (t only when v is given).
__global__ void k9_rowdot(const double2 *__restrict__ M, const double2 *__restrict__ Y, const double *__restrict__ v,
                          long P, int ng, double *__restrict__ s, double *__restrict__ t) {
    const long p = (long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (p >= P) return;
    double a = 0.0, b = 0.0;
    for (int g = lane; g < ng; g += 32) {
        const double2 m = M[p * ng + g], y = Y[p * ng + g];
        a = fma(m.x, y.x, fma(m.y, y.y, a));
        if (v) b = fma(v[g], fma(m.x, m.x, m.y * m.y), b);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        s[p] = a;
        if (t) t[p] = b;
    }
}

// out[n] = sum_{i < n_first} x[i * nn + n] (rows of band i in order)
__global__ void k9_sum(const double *__restrict__ x, int n_first, int nn, double *__restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    double a = 0.0;
    for (int i = 0; i < n_first; ++i) a += x[(long)i * nn + n];
    out[n] = a;
}

__global__ void k9_perm(const double2 *__restrict__ T, int nv, int nc, double2 *__restrict__ K) {
    const long P = (long)nv * nc;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * P) return;
    const long row = t / P, col = t % P;
    const int v = (int)(row / nc), c = (int)(row % nc), v2 = (int)(col / nc), c2 = (int)(col % nc);
    K[t] = T[((long)c * nc + c2) * ((long)nv * nv) + (long)v * nv + v2];
}

}  // namespace

cudaError_t zgemm_f64(int M, int N, int K, const void *A, long sam, long sak, bool conjA, const void *B, long sbk,
                      long sbn, bool conjB, const double *wk, void *C, long scm, long scn, double alpha_re,
                      double alpha_im, bool accumulate, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + kT - 1) / kT), (unsigned)((M + kT - 1) / kT));
    const double2 *a = static_cast<const double2 *>(A);
    const double2 *b = static_cast<const double2 *>(B);
    double2 *c = static_cast<double2 *>(C);
    const int beta = accumulate ? 1 : 0;
    if (conjA && conjB)
        k9_zgemm<true, true><<<grid, 256, 0, st>>>(M, N, K, a, sam, sak, b, sbk, sbn, wk, c, scm, scn, alpha_re,
                                                   alpha_im, beta);
    else if (conjA)
        k9_zgemm<true, false><<<grid, 256, 0, st>>>(M, N, K, a, sam, sak, b, sbk, sbn, wk, c, scm, scn, alpha_re,
                                                    alpha_im, beta);
    else if (conjB)
        k9_zgemm<false, true><<<grid, 256, 0, st>>>(M, N, K, a, sam, sak, b, sbk, sbn, wk, c, scm, scn, alpha_re,
                                                    alpha_im, beta);
    else
        k9_zgemm<false, false><<<grid, 256, 0, st>>>(M, N, K, a, sam, sak, b, sbk, sbn, wk, c, scm, scn, alpha_re,
                                                     alpha_im, beta);
    return cudaGetLastError();
}

cudaError_t rowdot_f64(const void *M, const void *Y, const double *v, long P, int ng, double *s, double *t,
                       cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    k9_rowdot<<<(unsigned)((P + 7) / 8), 256, 0, st>>>(static_cast<const double2 *>(M),
                                                       static_cast<const double2 *>(Y), v, P, ng, s, t);
    return cudaGetLastError();
}

cudaError_t band_sum_f64(const double *x, int n_first, int nn, double *out, cudaStream_t st) {
    if (nn <= 0) return cudaSuccess;
    k9_sum<<<(unsigned)((nn + 127) / 128), 128, 0, st>>>(x, n_first, nn, out);
    return cudaGetLastError();
}

cudaError_t bse_permute_f64(const void *T, int nv, int nc, void *K, cudaStream_t st) {
    const long n = (long)nv * nc * nv * nc;
    if (n == 0) return cudaSuccess;
    k9_perm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(static_cast<const double2 *>(T), nv, nc,
                                                         static_cast<double2 *>(K));
    return cudaGetLastError();
}

}  // namespace bgw
