// Dielectric matrix inverse and screened interaction on the GPU (FP64).
//
// arXiv:2206.00808, Sec. II, the two equations before the P formula:
//     eps_GG'(q, w) = delta_GG' - v(q+G) P_GG'(q, w),    W_GG' = eps^-1_GG' v(q+G').
// With s_G = sqrt(v(q+G)) the symmetrised matrix
//     eps~ = S^-1 eps S = I - S P S        (S = diag(s))
// is Hermitian, and positive definite because P = chi0 is negative
// semidefinite on the imaginary axis (every pair weight 2D/(D^2+w^2) < 0).
// Then eps^-1 = S eps~^-1 S^-1 and W = eps^-1 S^2 = S eps~^-1 S.
//
// eps~ is inverted in place by blocked Gauss-Jordan elimination without
// pivoting (valid for Hermitian positive definite matrices: every pivot block
// is a Schur complement of one and is itself positive definite).  For the
// block K of kb <= 32 indices and the rest R, one step is
//     P = A_KK^-1,  A_RR -= A_RK P A_KR,  A_KR <- P A_KR,  A_RK <- -A_RK P,  A_KK <- P
// (the block form of the scalar in-place Gauss-Jordan step); after every block
// has been taken the array holds the inverse.  Each step is four launches:
// k6_diag (one CTA per matrix inverts the kb x kb block in shared memory),
// k6_panels (P A_KR and A_RK P into a workspace), k6_update (the rank-kb
// update of all (r, c) outside K, tiled 32 x 32 in shared memory: this is
// where the 8 n^3 flops per matrix go, on the FP64 pipe), k6_writeback.
// All matrices of a call (one per frequency) go through each launch together.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/bgw_chi.h"

namespace {

constexpr int kB = 32;           // Gauss-Jordan block
constexpr int kTile = 32;        // update tile (rows and columns): many CTAs per panel step
constexpr int kErrPivot = 1;

struct Z {
    double x, y;
};
__device__ __forceinline__ Z zmul(Z a, Z b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ Z zfma(Z a, Z b, Z c) {   // a * b + c
    return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}

// A = I - S chi S in place; chi: [nf][n][n] complex128.
__global__ void k6_build(double2 *__restrict__ A, const double *__restrict__ s, int n) {
    const long j = blockIdx.z;
    const int r = blockIdx.y;
    double2 *row = A + (j * n + r) * (long)n;
    const double sr = s[r];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double2 v = row[c];
        const double f = -sr * s[c];
        v.x *= f;
        v.y *= f;
        if (c == r) v.x += 1.0;
        row[c] = v;
    }
}

// Invert the kb x kb block at (k0, k0) of every matrix in place (unblocked
// Gauss-Jordan, no pivoting).  One CTA per matrix.
__global__ void __launch_bounds__(256) k6_diag(double2 *__restrict__ A, int n, int k0, int kb, int *err) {
    __shared__ Z a[kB][kB + 1];
    __shared__ Z prow[kB];
    __shared__ Z pcol[kB];
    const long j = blockIdx.x;
    double2 *M = A + j * (long)n * n;
    for (int i = threadIdx.x; i < kb * kb; i += blockDim.x) {
        const int r = i / kb, c = i % kb;
        const double2 v = M[(long)(k0 + r) * n + k0 + c];
        a[r][c] = {v.x, v.y};
    }
    __syncthreads();
    for (int k = 0; k < kb; ++k) {
        const Z p = a[k][k];
        const double den = p.x * p.x + p.y * p.y;
        if (!(p.x > 0.0) || !isfinite(den)) {            // not positive definite (uniform branch)
            if (threadIdx.x == 0) atomicExch(err, kErrPivot);
            return;
        }
        const Z pinv = {p.x / den, -p.y / den};
        // old column k and scaled row k
        for (int i = threadIdx.x; i < kb; i += blockDim.x) {
            pcol[i] = a[i][k];
            prow[i] = (i == k) ? pinv : zmul(a[k][i], pinv);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kb * kb; i += blockDim.x) {
            const int r = i / kb, c = i % kb;
            Z v;
            if (r == k) {
                v = prow[c];
            } else if (c == k) {                          // -a_rk / p
                const Z f = pcol[r];
                v = {-(f.x * pinv.x - f.y * pinv.y), -(f.x * pinv.y + f.y * pinv.x)};
            } else {                                      // a_rc - a_rk (a_kc / p)
                const Z f = pcol[r], g = prow[c];
                v = a[r][c];
                v.x -= f.x * g.x - f.y * g.y;
                v.y -= f.x * g.y + f.y * g.x;
            }
            a[r][c] = v;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kb * kb; i += blockDim.x) {
        const int r = i / kb, c = i % kb;
        M[(long)(k0 + r) * n + k0 + c] = make_double2(a[r][c].x, a[r][c].y);
    }
}

// T[j][i][c] = sum_k P[i][k] A[k0+k][c]   (row panel, every column c)
// U[j][r][i] = sum_k A[r][k0+k] P[k][i]   (column panel, every row r)
// with P = A_KK already inverted in place.  Each thread computes kPanelI
// consecutive i for one column (or row) x.  grid (ceil(n/128), kB/kPanelI,
// 2 nf): z even for T, odd for U.
constexpr int kPanelI = 8;

__global__ void __launch_bounds__(128) k6_panels(const double2 *__restrict__ A, int n, int k0, int kb,
                                                 double2 *__restrict__ T, double2 *__restrict__ U) {
    __shared__ Z P[kB][kB + 1];
    const long j = blockIdx.z >> 1;
    const bool row_panel = (blockIdx.z & 1) == 0;
    const double2 *M = A + j * (long)n * n;
    for (int i = threadIdx.x; i < kb * kb; i += blockDim.x) {
        const double2 v = M[(long)(k0 + i / kb) * n + k0 + i % kb];
        P[i / kb][i % kb] = {v.x, v.y};
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int i0 = blockIdx.y * kPanelI;
    if (x >= n || i0 >= kb) return;
    Z acc[kPanelI];
#pragma unroll
    for (int i = 0; i < kPanelI; ++i) acc[i] = {0.0, 0.0};
    if (row_panel) {                                      // column c = x of P A_K.
        for (int k = 0; k < kb; ++k) {
            const double2 v = M[(long)(k0 + k) * n + x];
            const Z b = {v.x, v.y};
#pragma unroll
            for (int i = 0; i < kPanelI; ++i)
                if (i0 + i < kb) acc[i] = zfma(P[i0 + i][k], b, acc[i]);
        }
        double2 *t = T + j * (long)kB * n + x;
#pragma unroll
        for (int i = 0; i < kPanelI; ++i)
            if (i0 + i < kb) t[(long)(i0 + i) * n] = make_double2(acc[i].x, acc[i].y);
    } else {                                              // row r = x of A_.K P
        const double2 *row = M + (long)x * n + k0;
        for (int k = 0; k < kb; ++k) {
            const double2 v = row[k];
            const Z a = {v.x, v.y};
#pragma unroll
            for (int i = 0; i < kPanelI; ++i)
                if (i0 + i < kb) acc[i] = zfma(a, P[k][i0 + i], acc[i]);
        }
        double2 *u = U + (j * (long)n + x) * kB + i0;
#pragma unroll
        for (int i = 0; i < kPanelI; ++i)
            if (i0 + i < kb) u[i] = make_double2(acc[i].x, acc[i].y);
    }
}

// A[r][c] -= sum_k A[r][k0+k] T[k][c] for r, c outside [k0, k0+kb).
// One CTA per 32 x 32 tile (rows r0.., columns c0..) of one matrix; 256
// threads, each a 2 x 2 block of complex outputs (small tiles keep every SM
// busy at N_G of a few hundred); outputs in the K rows or K columns are
// computed and dropped.
constexpr int kLRow = kB + 1, kRRow = kTile + 1;
constexpr size_t kUpdateSmem = sizeof(Z) * ((size_t)kTile * kLRow + (size_t)kB * kRRow);

__global__ void __launch_bounds__(256) k6_update(double2 *__restrict__ A, int n, int k0, int kb,
                                                 const double2 *__restrict__ T) {
    extern __shared__ Z upd_sm[];
    Z (*L)[kLRow] = reinterpret_cast<Z (*)[kLRow]>(upd_sm);                       // A[r0 + i][k0 + k]
    Z (*R)[kRRow] = reinterpret_cast<Z (*)[kRRow]>(upd_sm + (size_t)kTile * kLRow);   // T[k][c0 + i]
    const long j = blockIdx.z;
    const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
    double2 *M = A + j * (long)n * n;
    const double2 *Tj = T + j * (long)kB * n;
    for (int i = threadIdx.x; i < kTile * kB; i += blockDim.x) {
        const int r = i / kB, k = i % kB;
        Z v = {0.0, 0.0};
        if (r0 + r < n && k < kb) {
            const double2 w = M[(long)(r0 + r) * n + k0 + k];
            v = {w.x, w.y};
        }
        L[r][k] = v;
    }
    for (int i = threadIdx.x; i < kB * kTile; i += blockDim.x) {
        const int k = i / kTile, c = i % kTile;
        Z v = {0.0, 0.0};
        if (c0 + c < n && k < kb) {
            const double2 w = Tj[(long)k * n + c0 + c];
            v = {w.x, w.y};
        }
        R[k][c] = v;
    }
    __syncthreads();
    constexpr int RA = kTile / 16;                              // outputs per thread per axis
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;   // rows tr + 16a, columns tc + 16b
    Z acc[RA][RA];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RA; ++b) acc[a][b] = {0.0, 0.0};
    for (int k = 0; k < kb; ++k) {
        Z l[RA], r[RA];
#pragma unroll
        for (int a = 0; a < RA; ++a) l[a] = L[tr + 16 * a][k];
#pragma unroll
        for (int b = 0; b < RA; ++b) r[b] = R[k][tc + 16 * b];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RA; ++b) acc[a][b] = zfma(l[a], r[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < RA; ++a) {
        const int r = r0 + tr + 16 * a;
        if (r >= n || (r >= k0 && r < k0 + kb)) continue;
#pragma unroll
        for (int b = 0; b < RA; ++b) {
            const int c = c0 + tc + 16 * b;
            if (c >= n || (c >= k0 && c < k0 + kb)) continue;
            double2 *o = M + (long)r * n + c;
            double2 v = *o;
            v.x -= acc[a][b].x;
            v.y -= acc[a][b].y;
            *o = v;
        }
    }
}

// A_KR <- T (columns outside K), A_RK <- -U (rows outside K).
__global__ void k6_writeback(double2 *__restrict__ A, int n, int k0, int kb, const double2 *__restrict__ T,
                             const double2 *__restrict__ U) {
    const long j = blockIdx.z;
    double2 *M = A + j * (long)n * n;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n || (x >= k0 && x < k0 + kb)) return;
    const double2 *t = T + j * (long)kB * n + x;
    for (int i = 0; i < kb; ++i) M[(long)(k0 + i) * n + x] = t[(long)i * n];
    const double2 *u = U + (j * (long)n + x) * kB;
    for (int i = 0; i < kb; ++i) {
        const double2 v = u[i];
        M[(long)x * n + k0 + i] = make_double2(-v.x, -v.y);
    }
}

// W = S eps~^-1 S (mode 1) or eps^-1 = S eps~^-1 S^-1 (mode 2).
__global__ void k6_scale(double2 *__restrict__ A, const double *__restrict__ s, int n, int inverse_cols) {
    const long j = blockIdx.z;
    const int r = blockIdx.y;
    double2 *row = A + (j * n + r) * (long)n;
    const double sr = s[r];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double2 v = row[c];
        const double f = inverse_cols ? sr / s[c] : sr * s[c];
        v.x *= f;
        v.y *= f;
        row[c] = v;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

void bgw_set_global_error(const std::string &msg);

extern "C" size_t bgw_epsinv_workspace_bytes(int ng, int nfreq) {
    if (ng < 1 || nfreq < 1) return 0;
    return 2 * align256(sizeof(double2) * (size_t)nfreq * kB * ng) + align256(sizeof(double) * ng) + 256;
}

extern "C" bgw_status bgw_coulomb_sqrt(const double *avec, const double *q, int ng, const int *gvec, double *s) {
    if (!avec || !q || !gvec || !s || ng < 1) {
        bgw_set_global_error("coulomb_sqrt: null pointer or ng < 1");
        return BGW_E_ARG;
    }
    const double kPi = 3.14159265358979323846;
    const double kE2 = 27.211386245988;     // e^2 in eV bohr (1 Hartree bohr)
    const double *a0 = avec, *a1 = avec + 3, *a2 = avec + 6;
    // reciprocal rows b_i = 2 pi (a_j x a_k) / det, (i, j, k) cyclic
    const double *pa[3][2] = {{a1, a2}, {a2, a0}, {a0, a1}};
    double b[3][3];
    const double det = a0[0] * (a1[1] * a2[2] - a1[2] * a2[1]) - a0[1] * (a1[0] * a2[2] - a1[2] * a2[0]) +
                       a0[2] * (a1[0] * a2[1] - a1[1] * a2[0]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
        bgw_set_global_error("coulomb_sqrt: singular cell");
        return BGW_E_ARG;
    }
    for (int i = 0; i < 3; ++i) {
        const double *u = pa[i][0], *w = pa[i][1];
        b[i][0] = 2 * kPi * (u[1] * w[2] - u[2] * w[1]) / det;
        b[i][1] = 2 * kPi * (u[2] * w[0] - u[0] * w[2]) / det;
        b[i][2] = 2 * kPi * (u[0] * w[1] - u[1] * w[0]) / det;
    }
    const double omega = std::fabs(det);
    for (int g = 0; g < ng; ++g) {
        double k[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i)
            for (int x = 0; x < 3; ++x) k[x] += (q[i] + gvec[3 * g + i]) * b[i][x];
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        s[g] = k2 > 1e-24 ? std::sqrt(4 * kPi * kE2 / (omega * k2)) : 0.0;
    }
    return BGW_OK;
}

extern "C" bgw_status bgw_epsinv(int ng, int nfreq, const double *s, void *chi, int mode, void *work,
                                 size_t work_bytes, void *stream) {
    auto fail = [](bgw_status st, const std::string &m) {
        bgw_set_global_error(m);
        return st;
    };
    if (ng < 1 || nfreq < 1 || !s || !chi) return fail(BGW_E_ARG, "epsinv: ng, nfreq >= 1 and s, chi required");
    if (mode < 0 || mode > 2) return fail(BGW_E_ARG, "epsinv: mode must be 0 (eps~^-1), 1 (W) or 2 (eps^-1)");
    if (nfreq > 32767 || ng > 65535) return fail(BGW_E_ARG, "epsinv: ng <= 65535 and nfreq <= 32767 required");
    for (int g = 0; g < ng; ++g) {
        if (!(s[g] >= 0.0) || !std::isfinite(s[g])) return fail(BGW_E_ARG, "epsinv: s must be finite and >= 0");
        if (mode == 2 && s[g] == 0.0) return fail(BGW_E_ARG, "epsinv: mode 2 needs s > 0 (q + G = 0 in the sphere)");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t need = bgw_epsinv_workspace_bytes(ng, nfreq);
    void *own = nullptr;
    cudaError_t e = cudaSuccess;
    if (!work) {
        e = cudaMalloc(&own, need);
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? BGW_E_NOMEM : BGW_E_CUDA,
                        std::string("epsinv: workspace: ") + cudaGetErrorString(e));
        work = own;
    } else if (work_bytes < need) {
        return fail(BGW_E_ARG, "epsinv: workspace of " + std::to_string(work_bytes) + " bytes, " +
                                   std::to_string(need) + " needed");
    }
    char *w = static_cast<char *>(work);
    double2 *T = reinterpret_cast<double2 *>(w);
    double2 *U = reinterpret_cast<double2 *>(w + align256(sizeof(double2) * (size_t)nfreq * kB * ng));
    double *sd = reinterpret_cast<double *>(w + 2 * align256(sizeof(double2) * (size_t)nfreq * kB * ng));
    int *err = reinterpret_cast<int *>(reinterpret_cast<char *>(sd) + align256(sizeof(double) * ng));
    double2 *A = static_cast<double2 *>(chi);
    e = cudaMemcpyAsync(sd, s, sizeof(double) * ng, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    const unsigned rowblocks = (unsigned)((ng + 255) / 256);
    if (e == cudaSuccess) {
        k6_build<<<dim3(rowblocks, ng, nfreq), 256, 0, st>>>(A, sd, ng);
        e = cudaGetLastError();
    }
    const unsigned tiles = (unsigned)((ng + kTile - 1) / kTile);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k6_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdateSmem);
    for (int k0 = 0; k0 < ng && e == cudaSuccess; k0 += kB) {
        const int kb = ng - k0 < kB ? ng - k0 : kB;
        k6_diag<<<nfreq, 256, 0, st>>>(A, ng, k0, kb, err);
        k6_panels<<<dim3((ng + 127) / 128, kB / kPanelI, 2 * nfreq), 128, 0, st>>>(A, ng, k0, kb, T, U);
        k6_update<<<dim3(tiles, tiles, nfreq), 256, kUpdateSmem, st>>>(A, ng, k0, kb, T);
        k6_writeback<<<dim3((ng + 127) / 128, 1, nfreq), 128, 0, st>>>(A, ng, k0, kb, T, U);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mode > 0) {
        k6_scale<<<dim3(rowblocks, ng, nfreq), 256, 0, st>>>(A, sd, ng, mode == 2);
        e = cudaGetLastError();
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (own) cudaFree(own);
    if (e != cudaSuccess) return fail(BGW_E_CUDA, std::string("epsinv: ") + cudaGetErrorString(e));
    if (flag) return fail(BGW_E_ARG, "epsinv: a pivot is not positive: I - S chi S is not positive definite "
                                     "(chi0 must be Hermitian negative semidefinite); the output is invalid");
    return BGW_OK;
}
