// Real-space grids and matrix elements (the FFT route of Eq. matrix_el,
// arXiv:2206.00808 Sec. II), one template for FP64 and FP32.
//
// Included once per precision by bgw_grid_f64.cu / bgw_grid_f32.cu with
// BGW_REAL and BGW_SUFFIX defined.
//
// Both 3-D transforms are done one axis at a time (one line per thread up to
// N = 40; eight lanes per line through shared memory for cubic 48 and 64;
// four lanes per line with warp shuffles for non-cubic boxes of those
// lengths), with pruning on the side where most of the box is empty:
//   sphere -> grid (inverse, u(r) = sum_h c(h) e^{+2 pi i h.r/N}): only the
//     lines that meet the sphere's bounding cube are transformed along x,
//     then along y, then along z (cube w0*w1*w2 -> n0*w1*w2 -> n0*n1*w2 -> n0*n1*n2);
//   pair density -> M (forward, e^{-2 pi i f.r/N}): z first on all n0*n1
//     lines, keeping the w2 needed outputs, then y keeping w1, then x keeping
//     w0, then a gather of the dielectric sphere from the kept cube.
// A cube that starts at box index s (not 0) is placed by rotating memory
// indices, not by phase factors: cube entry j sits at box position
// (s + j) mod N, so the inverse transform loads register f from cube slot
// (f - s) mod N and the forward transform stores output f to slot
// (f - s) mod N (see rot<N>).  Register indices stay compile-time.
#pragma once
#include <cuda_pipeline.h>

#include <cmath>
#include <cstring>

#include "bgw_bounds.cuh"
#include "bgw_fft.cuh"
#include "bgw_internal.h"
#include "bgw_tc_common.cuh"

namespace bgw {

namespace BGW_SUFFIX {

using T = BGW_REAL;
using C = cpx<T>;

constexpr int kLineThreads = 128;

// ---------------------------------------------------------------- tables --
static cudaError_t upload_tables() {
    double2 t64[kTwTotal];
    float2 t32[kTwTotal];
    for (int i = 0; i < kNumFftLens; ++i) {
        const int n = kFftLens[i];
        const int off = tw_offset(n);
        for (int j = 0; j < n; ++j) {
            // exp(-2 pi i j / n); exact values where the angle is a multiple of pi/4
            const double ang = -2.0 * 3.14159265358979323846264338327950288 * (double)j / (double)n;
            double c = std::cos(ang), s = std::sin(ang);
            if ((8 * j) % n == 0) {
                const int o = (8 * j) / n;   // multiple of pi/4
                const double r = 0.70710678118654752440084436210484904;
                const double cs[8] = {1, r, 0, -r, -1, -r, 0, r};
                const double sn[8] = {0, -r, -1, -r, 0, r, 1, r};
                c = cs[o];
                s = sn[o];
            }
            t64[off + j] = make_double2(c, s);
            t32[off + j] = make_float2((float)c, (float)s);
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tw64, t64, sizeof(double2) * kTwTotal);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_tw32, t32, sizeof(float2) * kTwTotal);
}

// Cube origins.  A pruned input that starts at box index s (entries j = 0..w-1
// at positions (s + j) mod N) is placed by reading slot (f - s) mod N into
// register f; a pruned output that starts at s is written by sending register
// f to slot (f - s) mod N.  Register indices stay compile-time; only the
// memory index is rotated.  ns = N - s, in [1, N].
template <int N>
__device__ __forceinline__ int rot(int f, int ns) {
    const int j = f + ns;
    return j >= N ? j - N : j;
}

// Kept outputs of a forward line whose cube starts at s: f = (s + j) mod N,
// j < w.  WIN: every such f lies within kWin of 0, so only those 2 kWin + 1
// registers are stored and the compiler drops the butterflies that feed no
// kept output.
constexpr int kWin = 8;

template <int N, bool WIN>
__device__ __forceinline__ void store_kept(const C (&a)[N], C *o, int stride, int ns, int w) {
    if constexpr (WIN) {
#pragma unroll
        for (int i = 0; i < 2 * kWin + 1; ++i) {
            const int f = i <= kWin ? i : N - (2 * kWin + 1) + i;
            const int j = rot<N>(f, ns);
            if (j < w) o[j * stride] = a[f];
        }
    } else {
#pragma unroll
        for (int f = 0; f < N; ++f) {
            const int j = rot<N>(f, ns);
            if (j < w) o[j * stride] = a[f];
        }
    }
}


// ------------------------------------------------------ sphere -> grid --
// Pass x: one thread per (band component b, y', z') line of the cube.
template <int N>
__global__ void __launch_bounds__(kLineThreads)
k1_xpass(const double2 *__restrict__ coeff, int ngw, long B, const int *__restrict__ cube_map,
         int w0, int w1, int w2, int s0, C *__restrict__ S) {
    const long yzs = (long)w1 * w2;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * yzs) return;
    const long yz = t % yzs;
    const long b = t / yzs;
    const int ns = N - s0;
    C a[N];
#pragma unroll
    for (int f = 0; f < N; ++f) {
        const int j = rot<N>(f, ns);
        C v = {T(0), T(0)};
        if (j < w0) {
            const int idx = __ldg(cube_map + j * yzs + yz);
            if (idx >= 0 && BGW_IN_BOUNDS(idx < ngw, kBoundsCubeMap)) {
                const double2 c = __ldg(coeff + b * ngw + idx);
                v = {(T)c.x, (T)c.y};
            }
        }
        a[f] = v;
    }
    fft_line<T, +1, N>(a);
    C *out = S + b * N * yzs + yz;
#pragma unroll
    for (int x = 0; x < N; ++x) out[x * yzs] = a[x];
}

// Pass y: one thread per (b, x, z') line; input rows y' < w1 of S.
template <int N>
__global__ void __launch_bounds__(kLineThreads)
k1_ypass(const C *__restrict__ S, long nbx, int w1, int w2, int s1, C *__restrict__ R) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nbx * w2) return;
    const long z = t % w2;
    const long bx = t / w2;
    const int ns = N - s1;
    C a[N];
#pragma unroll
    for (int f = 0; f < N; ++f) {
        const int j = rot<N>(f, ns);
        a[f] = (j < w1) ? S[(bx * w1 + j) * w2 + z] : C{T(0), T(0)};
    }
    fft_line<T, +1, N>(a);
#pragma unroll
    for (int y = 0; y < N; ++y) R[(bx * N + y) * w2 + z] = a[y];
}

// Pass z: one thread per (b, x, y) line; writes full grid lines.
template <int N>
__global__ void __launch_bounds__(kLineThreads)
k1_zpass(const C *__restrict__ R, long nbxy, int w2, int s2, C *__restrict__ U) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nbxy) return;
    const int ns = N - s2;
    C a[N];
#pragma unroll
    for (int f = 0; f < N; ++f) {
        const int j = rot<N>(f, ns);
        a[f] = (j < w2) ? R[t * w2 + j] : C{T(0), T(0)};
    }
    fft_line<T, +1, N>(a);
#pragma unroll
    for (int z = 0; z < N; ++z) U[t * N + z] = a[z];
}

// ------------------------------------------------ pair density -> M --
// Pass z: one thread per (pair p, x, y): rho(z) = sum_alpha conj(u_v) u_c,
// forward transform along z, keep outputs s2 .. s2+w2-1.
template <int N, bool WIN>
__global__ void __launch_bounds__(kLineThreads)
k2_zpass(const C *__restrict__ Uv, const C *__restrict__ Uc, int nc, long P, long plane, int w2,
         int s2, C *__restrict__ A) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * plane) return;
    const long xy = t % plane;
    // pairs run conduction-major, so each conduction grid is read by all the
    // batch's valence bands while it is in L2; A keeps the pair order v * nc + c
    const long po = t / plane, nvb = P / nc;
    const long c = po / nvb, v = po % nvb;
    const long p = v * nc + c;
    const long vol = plane * N;
    const C *v0 = Uv + (2 * v) * vol + xy * N;
    const C *c0 = Uc + (2 * c) * vol + xy * N;
    C a[N];
#pragma unroll
    for (int z = 0; z < N; ++z)
        a[z] = rho2(v0[z], c0[z], v0[vol + z], c0[vol + z]);
    fft_line<T, -1, N>(a);
    store_kept<N, WIN>(a, A + (p * plane + xy) * w2, 1, N - s2, w2);
}

// Pass y: one thread per (p, x, j2); keep outputs s1 .. s1+w1-1.
template <int N, bool WIN>
__global__ void __launch_bounds__(kLineThreads)
k2_ypass(const C *__restrict__ A, long npx, int w1, int w2, int s1, C *__restrict__ Bs) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npx * w2) return;
    const long jz = t % w2;
    const long px = t / w2;
    C a[N];
#pragma unroll
    for (int y = 0; y < N; ++y) a[y] = A[(px * N + y) * w2 + jz];
    fft_line<T, -1, N>(a);
    store_kept<N, WIN>(a, Bs + px * w1 * w2 + jz, w2, N - s1, w1);
}

// Pass x + gather: one block per PP pairs (so that the w1*w2 x lines of
// all of them fill the block); each pair's kept w0*w1*w2 cube goes to shared
// memory, then M[p][g] = cube[gmap[g]] / N^3.
constexpr int kGatherThreads = 256;

template <int N, bool WIN>
__global__ void __launch_bounds__(kGatherThreads)
k2_xpass_gather(const C *__restrict__ Bs, long P, int PP, int w0, int w1, int w2, int s0,
                const int *__restrict__ gmap, int ng, T scale, C *__restrict__ M, long ldm) {
    extern __shared__ unsigned char smem_raw[];
    C *cube = reinterpret_cast<C *>(smem_raw);          // [PP][w0][w1][w2]
    const long p0 = (long)blockIdx.x * PP;
    const int np = (int)(P - p0 < PP ? P - p0 : PP);
    const int lines = w1 * w2, csz = w0 * lines;
    const int ns = N - s0;
    for (int l = threadIdx.x; l < np * lines; l += kGatherThreads) {
        const int pp = l / lines, ll = l % lines;
        const C *bi = Bs + ((p0 + pp) * N) * lines + ll;
        C a[N];
#pragma unroll
        for (int x = 0; x < N; ++x) a[x] = bi[x * lines];
        fft_line<T, -1, N>(a);
        store_kept<N, WIN>(a, cube + pp * csz + ll, lines, ns, w0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np * ng; i += kGatherThreads) {
        const int pp = i / ng, g = i % ng;
        const int cell = __ldg(gmap + g);
        const C v = BGW_IN_BOUNDS(cell >= 0 && cell < csz, kBoundsGatherMap) ? cube[pp * csz + cell] : C{T(0), T(0)};
        M[(p0 + pp) * ldm + g] = C{v.x * scale, v.y * scale};
    }
}

// Pairs per CTA of k2_xpass_gather: enough x lines to fill its threads,
// within 96 KB of kept cubes.
static int gather_pairs(const Axes &a, long P) {
    const int lines = a.w[1] * a.w[2];
    const size_t csz = sizeof(C) * (size_t)a.w[0] * lines;
    int pp = kGatherThreads / lines;
    if (pp < 1) pp = 1;
    if (pp > 8) pp = 8;
    while (pp > 1 && (size_t)pp * csz > (size_t)96 * 1024) --pp;
    if (pp > P) pp = (int)(P > 0 ? P : 1);
    return pp;
}

// Pass x + scatter: one thread per (pair, line); every kept output goes to
// M[p][imap[cell]] when that cell holds a G-vector (large kept cubes).
template <int N>
__global__ void __launch_bounds__(kLineThreads)
k2_xpass_scatter(const C *__restrict__ Bs, long P, int w0, int w1, int w2, int s0,
                 const int *__restrict__ imap, T scale, C *__restrict__ M, long ldm) {
    const long lines = (long)w1 * w2;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * lines) return;
    const long l = t % lines, p = t / lines;
    C a[N];
#pragma unroll
    for (int x = 0; x < N; ++x) a[x] = Bs[(p * N + x) * lines + l];
    fft_line<T, -1, N>(a);
    const int ns = N - s0;
#pragma unroll
    for (int f = 0; f < N; ++f) {
        const int j = rot<N>(f, ns);
        if (j < w0) {
            const int g = __ldg(imap + j * lines + l);
            if (g >= 0 && BGW_IN_BOUNDS(g < ldm, kBoundsScatterMap)) M[p * ldm + g] = C{a[f].x * scale, a[f].y * scale};
        }
    }
}

// -------------------- four lanes per line (non-cubic boxes, N >= 48) --
// Long lines do not fit one thread's registers; four lanes share each line
// (fft_line_coop4).  Whole quads of lanes stay alive through the shuffles:
// a quad past the end works on line 0 and stores nothing.
constexpr int kCoopMinN = 48;

template <int N>
__global__ void __launch_bounds__(kLineThreads)
k2_zpass_c4(const C *__restrict__ Uv, const C *__restrict__ Uc, int nc, long P, long plane, int w2,
            int s2, C *__restrict__ A) {
    constexpr int M = N / 4, Q = M / 4;
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = (int)(tid & 3);
    long line = tid >> 2;
    const bool valid = line < P * plane;
    if (!valid) line = 0;
    const long xy = line % plane;
    const long po = line / plane, nvb = P / nc;       // conduction-major, as k2_zpass
    const long c = po / nvb, v = po % nvb;
    const long p = v * nc + c;
    const long vol = plane * N;
    const C *v0 = Uv + (2 * v) * vol + xy * N;
    const C *c0 = Uc + (2 * c) * vol + xy * N;
    C a[M], out[4][Q];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int z = 4 * m + t;
        a[m] = rho2(v0[z], c0[z], v0[vol + z], c0[vol + z]);
    }
    fft_line_coop4<T, -1, N>(a, t, out);
    if (!valid) return;
    const int ns = N - s2;
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int jj = rot<N>(t * Q + j + M * k1, ns);
            if (jj < w2) A[(p * plane + xy) * w2 + jj] = out[k1][j];
        }
}

// Threads of the eight-lane kernels below: 32 groups of eight lanes.
constexpr int kOctThreads = 256;

// Pair density + z and y forward passes of one (pair, x-plane) per CTA for
// the eight-lane lengths (48, 64): group y of eight lanes forms the pair
// density of z line y from the grids (both spin components) and transforms
// it (fft_line_oct); the kept w2 outputs go to shared Zs[N][w2p]; then group
// jz transforms y line jz of Zs and writes the kept w1 outputs to
// Bs[p][x][w1][w2].  The z-pass output never leaves the SM.  Each group has
// its own 8 x 9 exchange block after Zs.  Lane t handles z = 8m + t on the
// way in and the outputs f = t + (N/8) k1 on the way out.  A warp whose four
// groups all lie past the last line skips the iteration (the lanes of a warp
// synchronise inside the transform).  Three CTAs per SM (80 registers) hide
// the latency of the grid loads.  grid (P, n0).
template <int N>
__global__ void __launch_bounds__(kOctThreads, 3)
k2_zy_oct(const C *__restrict__ Uv, const C *__restrict__ Uc, int nc, int w1, int w2, int s1, int s2,
          C *__restrict__ Bs) {
    extern __shared__ unsigned char zy_sm[];
    constexpr int M = N / 8, G = kOctThreads / 8;      // groups per CTA
    const int w2p = w2 | 1;
    C *Zs = reinterpret_cast<C *>(zy_sm);
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7;
    C *ex = Zs + ((N * w2p + 1) & ~1) + grp * kOctBlock;
    const int warp_first_grp = (threadIdx.x >> 5) * 4;
    C tw[M];
    oct_twiddles<T, -1, N>(t, tw);
    const long p = blockIdx.x;
    const int x = blockIdx.y, n0 = gridDim.y;
    const long v = p / nc, c = p % nc;
    const long plane = (long)N * N, vol = (long)n0 * plane;
    const C *pv = Uv + (2 * v) * vol + x * plane;
    const C *pc = Uc + (2 * c) * vol + x * plane;
    const int ns2 = N - s2, ns1 = N - s1;
    for (int y0 = 0; y0 < N; y0 += G) {
        if (y0 + warp_first_grp >= N) break;            // warp-uniform
        const int y = y0 + grp;
        const bool valid = y < N;
        const long row = (long)(valid ? y : 0) * N;
        C a[M], out[8];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const long o = row + 8 * m + t;
            a[m] = rho2(pv[o], pc[o], pv[vol + o], pc[vol + o]);
        }
        fft_line_oct<T, -1, N>(a, t, ex, tw, out);
        if (valid && t < M) {
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) {
                const int jj = rot<N>(t + M * k1, ns2);
                if (jj < w2) Zs[y * w2p + jj] = out[k1];
            }
        }
    }
    __syncthreads();
    for (int base = 0; base < w2; base += G) {
        if (base + warp_first_grp >= w2) break;          // warp-uniform
        const int jz = base + grp;
        const bool valid = jz < w2;
        const int jc = valid ? jz : 0;
        C a[M], out[8];
#pragma unroll
        for (int m = 0; m < M; ++m) a[m] = Zs[(8 * m + t) * w2p + jc];
        fft_line_oct<T, -1, N>(a, t, ex, tw, out);
        if (valid && t < M) {
            C *bo = Bs + ((p * n0 + x) * w1) * w2 + jz;
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) {
                const int jj = rot<N>(t + M * k1, ns1);
                if (jj < w1) bo[jj * w2] = out[k1];
            }
        }
    }
}

// Last forward pass with eight lanes per line: Bs[p][x][w1][w2] -> M through
// the inverse map (cube cell -> G index or -1).  One group per (pair, y'z'
// line); 32 groups per CTA.
template <int N>
__global__ void __launch_bounds__(kOctThreads)
k2_xpass_scatter_oct(const C *__restrict__ Bs, long P, int w0, int w1, int w2, int s0,
                     const int *__restrict__ imap, T scale, C *__restrict__ Mo, long ldm) {
    __shared__ C exs[(kOctThreads / 8) * kOctBlock];
    constexpr int M = N / 8;
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7;
    C *ex = exs + grp * kOctBlock;
    C tw[M];
    oct_twiddles<T, -1, N>(t, tw);
    const long lines = (long)w1 * w2;
    long line = (long)blockIdx.x * (kOctThreads / 8) + grp;
    const bool valid = line < P * lines;
    if (!valid) line = 0;
    const long l = line % lines, p = line / lines;
    C a[M], out[8];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = Bs[(p * N + 8 * m + t) * lines + l];
    fft_line_oct<T, -1, N>(a, t, ex, tw, out);
    if (!valid || t >= M) return;
    const int ns = N - s0;
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        const int jj = rot<N>(t + M * k1, ns);
        if (jj < w0) {
            const int g = __ldg(imap + jj * lines + l);
            if (g >= 0 && BGW_IN_BOUNDS(g < ldm, kBoundsScatterMap)) Mo[p * ldm + g] = C{out[k1].x * scale, out[k1].y * scale};
        }
    }
}

// Sphere -> grid for the eight-lane lengths (48, 64): x lines of the cube
// (gathered through the cube map) into S[b][n0][w1][w2], then one CTA per
// (band component, x-plane) for the y lines (into shared Ys[N][w2p]) and the
// z lines (written to the grid).  grid of k1_xpass_oct: groups of eight.
template <int N>
__global__ void __launch_bounds__(kOctThreads)
k1_xpass_oct(const double2 *__restrict__ coeff, int ngw, long B, const int *__restrict__ cube_map, int w0,
             int w1, int w2, int s0, C *__restrict__ S) {
    __shared__ C exs[(kOctThreads / 8) * kOctBlock];
    constexpr int M = N / 8;
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7;
    C *ex = exs + grp * kOctBlock;
    C tw[M];
    oct_twiddles<T, +1, N>(t, tw);
    const long yzs = (long)w1 * w2;
    long line = (long)blockIdx.x * (kOctThreads / 8) + grp;
    const bool valid = line < B * yzs;
    if (!valid) line = 0;
    const long yz = line % yzs, b = line / yzs;
    const int ns = N - s0;
    C a[M], out[8];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int j = rot<N>(8 * m + t, ns);
        C v = {T(0), T(0)};
        if (j < w0) {
            const int idx = __ldg(cube_map + j * yzs + yz);
            if (idx >= 0 && BGW_IN_BOUNDS(idx < ngw, kBoundsCubeMap)) {
                const double2 c = __ldg(coeff + b * ngw + idx);
                v = {(T)c.x, (T)c.y};
            }
        }
        a[m] = v;
    }
    fft_line_oct<T, +1, N>(a, t, ex, tw, out);
    if (!valid || t >= M) return;
    C *o = S + b * N * yzs + yz;
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) o[(t + M * k1) * yzs] = out[k1];
}

template <int N>
__global__ void __launch_bounds__(kOctThreads, 2)
k1_yz_oct(const C *__restrict__ S, int w1, int w2, int s1, int s2, C *__restrict__ U) {
    extern __shared__ unsigned char yz_sm[];
    constexpr int M = N / 8, G = kOctThreads / 8;
    const int w2p = w2 | 1;
    C *Ys = reinterpret_cast<C *>(yz_sm);
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7;
    C *ex = Ys + ((N * w2p + 1) & ~1) + grp * kOctBlock;
    const int warp_first_grp = (threadIdx.x >> 5) * 4;
    C tw[M];
    oct_twiddles<T, +1, N>(t, tw);
    const long b = blockIdx.x;
    const int x = blockIdx.y, n0 = gridDim.y;
    const C *si = S + ((b * n0 + x) * w1) * (long)w2;
    const int ns1 = N - s1, ns2 = N - s2;
    for (int base = 0; base < w2; base += G) {
        if (base + warp_first_grp >= w2) break;          // warp-uniform
        const int jz = base + grp;
        const bool valid = jz < w2;
        const int jc = valid ? jz : 0;
        C a[M], out[8];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int j = rot<N>(8 * m + t, ns1);
            a[m] = (j < w1) ? si[j * w2 + jc] : C{T(0), T(0)};
        }
        fft_line_oct<T, +1, N>(a, t, ex, tw, out);
        if (valid && t < M) {
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) Ys[(t + M * k1) * w2p + jz] = out[k1];
        }
    }
    __syncthreads();
    C *uo = U + (b * n0 + x) * (long)N * N;
    for (int y0 = 0; y0 < N; y0 += G) {
        if (y0 + warp_first_grp >= N) break;             // warp-uniform
        const int y = y0 + grp;
        const bool valid = y < N;
        const int yc = valid ? y : 0;
        C a[M], out[8];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int j = rot<N>(8 * m + t, ns2);
            a[m] = (j < w2) ? Ys[yc * w2p + j] : C{T(0), T(0)};
        }
        fft_line_oct<T, +1, N>(a, t, ex, tw, out);
        if (valid && t < M) {
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) uo[(long)y * N + t + M * k1] = out[k1];
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kLineThreads)
k2_ypass_c4(const C *__restrict__ A, long npx, int w1, int w2, int s1, C *__restrict__ Bs) {
    constexpr int M = N / 4, Q = M / 4;
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = (int)(tid & 3);
    long line = tid >> 2;
    const bool valid = line < npx * w2;
    if (!valid) line = 0;
    const long jz = line % w2, px = line / w2;
    C a[M], out[4][Q];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = A[(px * N + 4 * m + t) * w2 + jz];
    fft_line_coop4<T, -1, N>(a, t, out);
    if (!valid) return;
    const int ns = N - s1;
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int jj = rot<N>(t * Q + j + M * k1, ns);
            if (jj < w1) Bs[(px * w1 + jj) * w2 + jz] = out[k1][j];
        }
}

template <int N>
__global__ void __launch_bounds__(kLineThreads)
k2_xpass_scatter_c4(const C *__restrict__ Bs, long P, int w0, int w1, int w2, int s0,
                    const int *__restrict__ imap, T scale, C *__restrict__ M, long ldm) {
    constexpr int MM = N / 4, Q = MM / 4;
    const long lines = (long)w1 * w2;
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = (int)(tid & 3);
    long line = tid >> 2;
    const bool valid = line < P * lines;
    if (!valid) line = 0;
    const long l = line % lines, p = line / lines;
    C a[MM], out[4][Q];
#pragma unroll
    for (int m = 0; m < MM; ++m) a[m] = Bs[(p * N + 4 * m + t) * lines + l];
    fft_line_coop4<T, -1, N>(a, t, out);
    if (!valid) return;
    const int ns = N - s0;
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int jj = rot<N>(t * Q + j + MM * k1, ns);
            if (jj < w0) {
                const int g = __ldg(imap + jj * lines + l);
                if (g >= 0 && BGW_IN_BOUNDS(g < ldm, kBoundsScatterMap))
                    M[p * ldm + g] = C{out[k1][j].x * scale, out[k1][j].y * scale};
            }
        }
}

// ------------------------------------------ sphere -> grid, one kernel --
// Whole inverse transform of one band component per CTA, for boxes whose
// x-transformed cube fits in shared memory.  The band's coefficients are read
// once, coalesced, and scattered into the sphere's bounding cube in shared
// memory (inv[i] = cube cell of coefficient i); x lines of the cube go to
// X[N][w1][w2]; then, KP x-planes at a time, y lines go to Y[KP][N][w2p]
// (over the dead cube) and z lines are written to the grid.  No
// intermediate array leaves the SM.
constexpr int kFusedThreads = 256;

// kCube = false (FP32, on request): no shared cube; the x lines gather their
// coefficients from global memory through the cube map (cmap), which frees
// the cube's shared memory for a third CTA per SM.
// The transform of one band component: coefficients cb[ngw] -> grid out[N^3].
template <int N, bool kCube>
__device__ __forceinline__ void k1_fused_body(const double2 *__restrict__ cb, int ngw, const int *__restrict__ inv,
                                              const int *__restrict__ cmap, int w0, int w1, int w2, int s0,
                                              int s1, int s2, int KP, C *__restrict__ out,
                                              unsigned char *smem_raw) {
    C *X = reinterpret_cast<C *>(smem_raw);
    const int yzs = w1 * w2;
    const int w2p = w2 | 1;                    // odd row stride: conflict-free z-line reads
    C *cube = X + (long)N * yzs;               // [w0][w1][w2], later Y[KP][N][w2p]
    C *Y = cube;
    if constexpr (kCube) {
        const int ncube = w0 * yzs;
        for (int i = threadIdx.x; i < ncube; i += kFusedThreads) cube[i] = C{T(0), T(0)};
        __syncthreads();
        for (int i = threadIdx.x; i < ngw; i += kFusedThreads) {
            const double2 c = __ldg(cb + i);
            const int cell = __ldg(inv + i);
            if (BGW_IN_BOUNDS(cell >= 0 && cell < ncube, kBoundsInverseMap)) cube[cell] = C{(T)c.x, (T)c.y};
        }
        __syncthreads();
    }
    const int ns0 = N - s0, ns1 = N - s1, ns2 = N - s2;
    for (int l = threadIdx.x; l < yzs; l += kFusedThreads) {
        C a[N];
#pragma unroll
        for (int f = 0; f < N; ++f) {
            const int j = rot<N>(f, ns0);
            if constexpr (kCube) {
                a[f] = (j < w0) ? cube[j * yzs + l] : C{T(0), T(0)};
            } else {
                C v = {T(0), T(0)};
                if (j < w0) {
                    const int idx = __ldg(cmap + j * yzs + l);
                    if (idx >= 0 && BGW_IN_BOUNDS(idx < ngw, kBoundsCubeMap)) {
                        const double2 c = __ldg(cb + idx);
                        v = {(T)c.x, (T)c.y};
                    }
                }
                a[f] = v;
            }
        }
        fft_line<T, +1, N>(a);
#pragma unroll
        for (int x = 0; x < N; ++x) X[x * yzs + l] = a[x];
    }
    __syncthreads();
    for (int x0 = 0; x0 < N; x0 += KP) {
        const int kp = min(KP, N - x0);
        for (int l = threadIdx.x; l < kp * w2; l += kFusedThreads) {
            const int xl = l / w2, z = l % w2;
            const C *xi = X + (x0 + xl) * yzs + z;
            C a[N];
#pragma unroll
            for (int f = 0; f < N; ++f) {
                const int j = rot<N>(f, ns1);
                a[f] = (j < w1) ? xi[j * w2] : C{T(0), T(0)};
            }
            fft_line<T, +1, N>(a);
            C *yo = Y + xl * N * w2p + z;
#pragma unroll
            for (int y = 0; y < N; ++y) yo[y * w2p] = a[y];
        }
        __syncthreads();
        for (int l = threadIdx.x; l < kp * N; l += kFusedThreads) {
            const int xl = l / N, y = l % N;
            const C *yi = Y + (xl * N + y) * w2p;
            C a[N];
#pragma unroll
            for (int f = 0; f < N; ++f) {
                const int j = rot<N>(f, ns2);
                a[f] = (j < w2) ? yi[j] : C{T(0), T(0)};
            }
            fft_line<T, +1, N>(a);
            C *o = out + ((long)(x0 + xl) * N + y) * N;
            if constexpr (sizeof(T) == 4 && N % 2 == 0) {
#pragma unroll
                for (int z = 0; z < N; z += 2)
                    *reinterpret_cast<float4 *>(o + z) = make_float4(a[z].x, a[z].y, a[z + 1].x, a[z + 1].y);
            } else {
#pragma unroll
                for (int z = 0; z < N; ++z) o[z] = a[z];
            }
        }
        __syncthreads();
    }
}

template <int N, bool kCube>
__global__ void __launch_bounds__(kFusedThreads, sizeof(T) == 4 ? (kCube ? 2 : 3) : 1)
k1_fused(const double2 *__restrict__ coeff, int ngw, const int *__restrict__ inv,
         const int *__restrict__ cmap, int w0, int w1, int w2, int s0, int s1, int s2, int KP,
         C *__restrict__ U) {
    extern __shared__ unsigned char smem_raw[];
    const long b = blockIdx.x;
    k1_fused_body<N, kCube>(coeff + b * ngw, ngw, inv, cmap, w0, w1, w2, s0, s1, s2, KP,
                            U + b * (long)N * N * N, smem_raw);
}

// Several k-points in one launch (deferred uploads): CTA x = (job, band
// component), so the launch has no wave tail per k-point.
constexpr int kK1BatchMax = 64;
struct K1BatchJob {
    const double2 *coeff;
    const int *inv;
    C *U;
    int ngw, w0, w1, w2, s0, s1, s2, KP;
};
struct K1Batch {
    int njobs, B;
    K1BatchJob job[kK1BatchMax];
};

template <int N>
__global__ void __launch_bounds__(kFusedThreads, sizeof(T) == 4 ? 2 : 1)
k1_fused_batch(const __grid_constant__ K1Batch jb) {
    extern __shared__ unsigned char smem_raw[];
    const int j = blockIdx.x / jb.B;
    const long b = blockIdx.x % jb.B;
    const K1BatchJob &e = jb.job[j];
    k1_fused_body<N, true>(e.coeff + b * e.ngw, e.ngw, e.inv, nullptr, e.w0, e.w1, e.w2, e.s0, e.s1, e.s2, e.KP,
                           e.U + b * (long)N * N * N, smem_raw);
}

// Shared bytes of k1_fused with KP planes per chunk (Y reuses the cube).
static size_t fused_smem(const Axes &a, int KP, bool cube_in_smem = true) {
    const size_t cube = cube_in_smem ? (size_t)a.w[0] * a.w[1] * a.w[2] : 0;
    const size_t y = (size_t)KP * a.n[1] * (a.w[2] | 1);
    return sizeof(C) * ((size_t)a.n[0] * a.w[1] * a.w[2] + (cube > y ? cube : y));
}
// The cube-less variant: three CTAs per SM.
static constexpr size_t kFusedSmem3 = 72 * 1024;
// Automatic choice: two CTAs per SM; on request (path 2) up to one per SM.
static constexpr size_t kFusedSmemAuto = 110 * 1024;
static constexpr size_t kFusedSmemMax = 200 * 1024;

// Planes per chunk for k1_fused: the fewest chunks of equal size that fit
// in `limit` bytes (0: the box does not fit; use the pass kernels).
static int fused_planes(const Axes &a, size_t limit) {
    if (a.n[0] != a.n[1] || a.n[1] != a.n[2] || a.n[0] >= kCoopMinN) return 0;
    const int n = a.n[0];
    for (int chunks = 1; chunks <= n; ++chunks) {
        const int KP = (n + chunks - 1) / chunks;
        if (fused_smem(a, KP) <= limit) return KP;
    }
    return 0;
}

// ----------------------------------------- plane-fused passes (FP32) --
// Band planes staged through shared memory with batched loads (kStageU in
// flight per thread); every line is then read from a padded shared row.
// Used when the box has n1 == n2.
constexpr int kPlaneThreads = 256;
constexpr int kStageU = 8;

// Shared row length of a staged plane: one complex of padding for odd N, two
// for even N (keeps rows 16-byte aligned for paired FP32 accesses).
template <int N>
__host__ __device__ constexpr int plane_row() { return N % 2 == 0 ? N + 2 : N + 1; }

// Pair density + z pass + y pass for one x-plane and a tile of tv x tc pairs.
// Shared: planes[(tv+tc)][2][N][N+1], then Z[tv*tc][N][w2].
template <int N, int MINB, int THREADS, bool WIN = false>
__global__ void __launch_bounds__(THREADS, MINB)
k2_zy_plane(const C *__restrict__ Uv, const C *__restrict__ Uc, int nv, int nc, int TV, int TC,
            int w1, int w2, int s1, int s2, C *__restrict__ Bs) {
    extern __shared__ unsigned char smem_raw[];
    C *planes = reinterpret_cast<C *>(smem_raw);
    const int x = blockIdx.x;
    const int v0 = blockIdx.y * TV, c0 = blockIdx.z * TC;
    const int tv = min(TV, nv - v0), tc = min(TC, nc - c0);
    const int n0 = gridDim.x;
    constexpr int RS = plane_row<N>();         // padded row
    constexpr int PS = N * RS;                  // one spin component of a plane
    constexpr int NN = N * N;
    constexpr bool kVec = sizeof(T) == 4 && N % 2 == 0;   // two complex per 16-byte access
    C *Z = planes + (long)(TV + TC) * 2 * PS;
    const long vol = (long)n0 * NN;
    // 1. stage the x-plane of every band of the tile (both spin components)
    constexpr int VW = kVec ? 2 : 1;            // complex values per access
    const int total = (tv + tc) * 2 * NN / VW;
    for (int base = threadIdx.x; base < total; base += THREADS * kStageU) {
        C tmp[kStageU][VW];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int i = base + u * THREADS;
            if (i < total) {
                const int ba = (i * VW) / NN, yz = (i * VW) % NN;     // ba = band * 2 + alpha
                const int b = ba >> 1, a = ba & 1;
                const C *src = (b < tv) ? Uv + ((long)(v0 + b) * 2 + a) * vol
                                        : Uc + ((long)(c0 + b - tv) * 2 + a) * vol;
                if constexpr (kVec) {
                    const float4 q = *reinterpret_cast<const float4 *>(src + (long)x * NN + yz);
                    tmp[u][0] = C{q.x, q.y};
                    tmp[u][VW - 1] = C{q.z, q.w};
                } else {
                    tmp[u][0] = src[(long)x * NN + yz];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int i = base + u * THREADS;
            if (i < total) {
                const int ba = (i * VW) / NN, yz = (i * VW) % NN;
                C *dst = planes + ba * PS + (yz / N) * RS + (yz % N);
                if constexpr (kVec) {
                    *reinterpret_cast<float4 *>(dst) =
                        make_float4(tmp[u][0].x, tmp[u][0].y, tmp[u][VW - 1].x, tmp[u][VW - 1].y);
                } else {
                    dst[0] = tmp[u][0];
                }
            }
        }
    }
    __syncthreads();
    // 2. z lines: rho(z) = sum_alpha conj(u_v) u_c, forward FFT, keep w2 outputs
    const int npair = tv * tc;
    const int ns2 = N - s2, ns1 = N - s1;
    for (int l = threadIdx.x; l < npair * N; l += THREADS) {
        const int pr = l / N, y = l % N;
        const int v = pr / tc, c = pr % tc;
        const C *pv = planes + (v * 2) * PS + y * RS;
        const C *pc = planes + ((tv + c) * 2) * PS + y * RS;
        C a[N];
        if constexpr (kVec) {
            const float4 *v4 = reinterpret_cast<const float4 *>(pv);
            const float4 *c4 = reinterpret_cast<const float4 *>(pc);
            constexpr int P4 = PS / 2;
#pragma unroll
            for (int z = 0; z < N / 2; ++z) {
                const float4 va = v4[z], vb = v4[P4 + z], ca = c4[z], cb = c4[P4 + z];
                a[2 * z] = rho2(C{va.x, va.y}, C{ca.x, ca.y}, C{vb.x, vb.y}, C{cb.x, cb.y});
                a[2 * z + 1] = rho2(C{va.z, va.w}, C{ca.z, ca.w}, C{vb.z, vb.w}, C{cb.z, cb.w});
            }
        } else {
#pragma unroll
            for (int z = 0; z < N; ++z) a[z] = rho2(pv[z], pc[z], pv[PS + z], pc[PS + z]);
        }
        fft_line<T, -1, N>(a);
        store_kept<N, WIN>(a, Z + ((long)pr * N + y) * w2, 1, ns2, w2);
    }
    __syncthreads();
    // 3. y lines over the kept z outputs; keep w1 outputs -> Bs[p][x][jy][jz]
    for (int l = threadIdx.x; l < npair * w2; l += THREADS) {
        const int pr = l / w2, jz = l % w2;
        const int v = pr / tc, c = pr % tc;
        const C *zi = Z + (long)pr * N * w2 + jz;
        C a[N];
#pragma unroll
        for (int y = 0; y < N; ++y) a[y] = zi[y * w2];
        fft_line<T, -1, N>(a);
        const long p = (long)(v0 + v) * nc + (c0 + c);
        store_kept<N, WIN>(a, Bs + ((p * n0 + x) * w1) * w2 + jz, w2, ns1, w1);
    }
}

// Streamed form of the pair density + z + y passes (FP32, even N <= 32): one
// CTA per (x-plane, group of up to SV valence bands, range of conduction
// bands).  The valence x-planes stay in shared memory for the whole item; the
// conduction x-planes come in groups of SC bands through two buffers, filled
// by TMA on 32^3 boxes (one thread, an mbarrier per buffer) and by cp.async
// from the z-line threads otherwise.  Each phase k, after which the CTA
// synchronises once:
//   threads 0..kZThreads-1  z lines of group k (pair density, FFT, kept outputs
//                           into Z[k & 1]),
//   the other threads       y lines of group k - 1 (from Z[(k - 1) & 1] to Bs),
//   copies                  of group k + 1 into the buffer group k - 1 used,
// so copies, z lines and y lines of consecutive groups run together.
// Shared: V[SV][2][N][RS], Cb[2][SC][2][N][RS], Z[2][SV*SC][N][W] with RS the
// padded row N + 2 (dense and swizzled with TMA) and W = kZW (w2 with TMA).
constexpr int kZThreads = 256, kYThreads = 128, kStreamThreads = kZThreads + kYThreads;
constexpr int kZW = 17;   // largest kept z width the Z buffers hold

// Default valence and conduction group sizes per box length: as many z
// lines (SV * SC * N) as z threads, or nearly (32^3 TMA launches may take
// 2 x 4 instead, see mtxel_batch).
template <int N>
struct StreamTile {
    static constexpr int V = N == 24 ? 5 : 4;
    static constexpr int C = N >= 24 ? 2 : (N >= 18 ? 3 : 4);
};

// TMA staging (N = 32): a plane component is two boxes of N rows x kTmaHalf
// values (128 bytes) in the 128-byte swizzle, 16-byte chunk c of row r at
// chunk c ^ (r & 7); 1024-byte aligned, so one more KB is requested.
constexpr int kTmaHalf = 16;
constexpr int kErrCopy = 5;   // a plane copy of the streamed kernel did not land in time

// Shared memory of the streamed kernel with SV x SC band groups: the valence
// planes, two conduction buffers and two Z buffers (kept width w2 with TMA,
// kZW otherwise).
template <int N, int SV, int SC, bool TMA>
__host__ __device__ constexpr size_t stream_smem(int w2) {
    return sizeof(cpx<float>) * ((size_t)(SV + 2 * SC) * 2 * N * (TMA ? N : plane_row<N>()) +
                                 (size_t)2 * SV * SC * N * (TMA ? w2 : kZW)) +
           (TMA ? 1024 : 0);
}

template <int N, int SV, int SC, bool WIN, bool TMA>
__global__ void __launch_bounds__(kStreamThreads, 1)
k2_zy_stream(const C *__restrict__ Uv, const C *__restrict__ Uc, int nv, int nc, int CC, int w1, int w2, int s1,
             int s2, C *__restrict__ Bs, const __grid_constant__ CUtensorMap map_v,
             const __grid_constant__ CUtensorMap map_c, int *__restrict__ err, int drop_first_copy) {
    constexpr int kStreamV = SV, kStreamC = SC;
    static_assert(N % 2 == 0 && kStreamV * kStreamC * N <= kZThreads, "one z line per z thread");
    static_assert(!TMA || (N == 2 * kTmaHalf && sizeof(T) == 4), "TMA staging: N = 32, FP32");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_v, bar_c[2];
    constexpr int RS = TMA ? N : plane_row<N>();   // row of a staged plane (dense and swizzled with TMA)
    constexpr int PS = N * RS;                   // one spin component of a plane
    constexpr int NN = N * N;
    constexpr int CH = NN / 2;                   // 16-byte chunks per plane component
    const int ZS = kStreamV * kStreamC * N * (TMA ? w2 : kZW);   // as the host sized them
    unsigned char *sbase = smem_raw;
    if constexpr (TMA) sbase += (1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u;
    C *V = reinterpret_cast<C *>(sbase);
    C *Cb0 = V + kStreamV * 2 * PS;
    C *Z0 = Cb0 + 2 * kStreamC * 2 * PS;
    const int x = blockIdx.x, n0 = gridDim.x;
    const int v0 = blockIdx.y * kStreamV, cbeg = blockIdx.z * CC;
    const int tv = min(kStreamV, nv - v0), cend = min(nc, cbeg + CC);
    const long vol = (long)n0 * NN;
    const int ns1 = N - s1, ns2 = N - s2;
    // copies of band planes (both spin components of x-plane x) into rows of
    // RS by threads [t0, t0 + nt): all threads for the prologue, the z-line
    // threads in the phases (the y lines are the longer role)
    auto copy_planes = [&](C *dst, const C *src, long band0, int nb, int t0, int nt) {
        const int total = nb * 2 * CH;
        for (int i = threadIdx.x - t0; i < total; i += nt) {
            const int ba = i / CH, ch = i % CH;           // ba = band * 2 + alpha
            const int yz = 2 * ch;
            const C *g = src + ((band0 + (ba >> 1)) * 2 + (ba & 1)) * vol + (long)x * NN + yz;
            C *d = dst + ba * PS + (yz / N) * RS + (yz % N);
            __pipeline_memcpy_async(d, g, 16);
        }
    };
    // TMA: nb band planes (both spin components, two boxes each) issued by one
    // thread onto one mbarrier; every thread waits (bounded) for them
    auto tma_planes = [&](C *dst, const CUtensorMap *map, int band0, int nb, uint64_t *bar) {
        if (threadIdx.x != 0) return;
        const uint32_t b = tc::smem_u32(bar);
        tc::fence_proxy_async_smem();            // the buffer's last readers passed a barrier
        tc::mbar_expect_tx(b, (uint32_t)(nb * 2 * NN * sizeof(C)));
        for (int ba = 0; ba < 2 * nb; ++ba)
            for (int h = 0; h < 2; ++h)
                tc::tma_load_4d(tc::smem_u32(dst + ba * PS + h * (N * kTmaHalf)), map, b, h * 2 * kTmaHalf, 0, x,
                                2 * band0 + ba);
    };
    auto wait_planes = [&](uint64_t *bar, uint32_t parity) {
        if (!tc::mbar_wait(tc::smem_u32(bar), parity) && err) atomicExch(err, kErrCopy);
    };
    const int ng = (cend - cbeg + kStreamC - 1) / kStreamC;
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            tc::mbar_init(tc::smem_u32(&bar_v), 1);
            tc::mbar_init(tc::smem_u32(&bar_c[0]), 1);
            tc::mbar_init(tc::smem_u32(&bar_c[1]), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        // test hook: the first CTA never issues its valence planes, so its
        // bounded wait expires and records kErrCopy
        if (!(drop_first_copy && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0))
            tma_planes(V, &map_v, v0, tv, &bar_v);
        if (ng > 0) tma_planes(Cb0, &map_c, cbeg, min(kStreamC, cend - cbeg), &bar_c[0]);
        wait_planes(&bar_v, 0);
        if (ng > 0) wait_planes(&bar_c[0], 0);
    } else {
        copy_planes(V, Uv, v0, tv, 0, kStreamThreads);
        if (ng > 0) copy_planes(Cb0, Uc, cbeg, min(kStreamC, cend - cbeg), 0, kStreamThreads);
        __pipeline_commit();
        __pipeline_wait_prior(0);
    }
    __syncthreads();
    for (int k = 0; k <= ng; ++k) {
        if (k + 1 < ng) {
            const int c1 = cbeg + (k + 1) * kStreamC;
            if constexpr (TMA)
                tma_planes(Cb0 + ((k + 1) & 1) * (kStreamC * 2 * PS), &map_c, c1, min(kStreamC, cend - c1),
                           &bar_c[(k + 1) & 1]);
            else if (threadIdx.x < kZThreads)
                copy_planes(Cb0 + ((k + 1) & 1) * (kStreamC * 2 * PS), Uc, c1, min(kStreamC, cend - c1), 0,
                            kZThreads);
        }
        if constexpr (!TMA) __pipeline_commit();
        if (threadIdx.x < kZThreads) {
            // z line (pair, y) of group k, pair = v * tc + c
            const int tc = k < ng ? min(kStreamC, cend - (cbeg + k * kStreamC)) : 0;
            const int l = threadIdx.x;
            if (l < tv * tc * N) {
                const int pr = l / N, y = l % N;
                const int v = pr / tc, c = pr % tc;
                const C *cur = Cb0 + (k & 1) * (kStreamC * 2 * PS);
                const float4 *v4 = reinterpret_cast<const float4 *>(V + (v * 2) * PS + y * RS);
                const float4 *c4 = reinterpret_cast<const float4 *>(cur + (c * 2) * PS + y * RS);
                constexpr int P4 = PS / 2;
                C a[N];
#pragma unroll
                for (int z = 0; z < N / 2; ++z) {
                    // float4 index of values 2z, 2z+1 of row y (swizzled boxes with TMA)
                    int q = z;
                    if constexpr (TMA)
                        q = (z / 8) * (N * kTmaHalf / 2) - y * (RS / 2) + y * (kTmaHalf / 2) + ((z % 8) ^ (y & 7));
                    const float4 va = v4[q], vb = v4[P4 + q], ca = c4[q], cb = c4[P4 + q];
                    a[2 * z] = rho2(C{va.x, va.y}, C{ca.x, ca.y}, C{vb.x, vb.y}, C{cb.x, cb.y});
                    a[2 * z + 1] = rho2(C{va.z, va.w}, C{ca.z, ca.w}, C{vb.z, vb.w}, C{cb.z, cb.w});
                }
                fft_line<T, -1, N>(a);
                store_kept<N, WIN>(a, Z0 + (k & 1) * ZS + ((long)pr * N + y) * w2, 1, ns2, w2);
            }
        } else if (k >= 1) {
            // y lines of group k - 1; keep w1 outputs -> Bs[p][x][jy][jz]
            const int c0 = cbeg + (k - 1) * kStreamC;
            const int tc = min(kStreamC, cend - c0);
            const C *Z = Z0 + ((k - 1) & 1) * ZS;
            for (int t = threadIdx.x - kZThreads; t < tv * tc * w2; t += kYThreads) {
                const int q = t / w2, jz = t % w2;
                const int v = q / tc, c = q % tc;
                const C *zi = Z + (long)q * N * w2 + jz;
                C b[N];
#pragma unroll
                for (int yy = 0; yy < N; ++yy) b[yy] = zi[yy * w2];
                fft_line<T, -1, N>(b);
                const long p = (long)(v0 + v) * nc + (c0 + c);
                store_kept<N, WIN>(b, Bs + ((p * n0 + x) * w1) * w2 + jz, w2, ns1, w1);
            }
        }
        if constexpr (TMA) {
            if (k + 1 < ng) wait_planes(&bar_c[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1));
        } else {
            __pipeline_wait_prior(0);    // group k + 1 has landed
        }
        __syncthreads();                 // Z[k & 1] written, Z[(k - 1) & 1] and Cb[k & 1] read
    }
}

// Sphere -> grid y and z passes for one x-plane of TB band components:
// S[b][x][w1][w2] -> U[b][x][N][N].  Shared: in[TB][w1][w2], P[TB][N][w2+1],
// out[TB][N][N+1].
template <int N>
__global__ void __launch_bounds__(kPlaneThreads, 2)
k1_yz_plane(const C *__restrict__ S, long B, int TB, int w1, int w2, int s1, int s2,
            C *__restrict__ U) {
    extern __shared__ unsigned char smem_raw[];
    C *in = reinterpret_cast<C *>(smem_raw);
    const int x = blockIdx.x, n0 = gridDim.x;
    const long b0 = (long)blockIdx.y * TB;
    const int tb = (int)min((long)TB, B - b0);
    const int PW = w2 + 1;
    C *P = in + (long)TB * w1 * w2;
    C *out = P + (long)TB * N * PW;
    const int wsz = w1 * w2;
    const int total = tb * wsz;
    for (int base = threadIdx.x; base < total; base += kPlaneThreads * kStageU) {
        C tmp[kStageU];
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int i = base + u * kPlaneThreads;
            if (i < total) tmp[u] = S[((b0 + i / wsz) * n0 + x) * wsz + i % wsz];
        }
#pragma unroll
        for (int u = 0; u < kStageU; ++u) {
            const int i = base + u * kPlaneThreads;
            if (i < total) in[i] = tmp[u];
        }
    }
    __syncthreads();
    const int ns1 = N - s1, ns2 = N - s2;
    for (int l = threadIdx.x; l < tb * w2; l += kPlaneThreads) {
        const int b = l / w2, z = l % w2;
        C a[N];
#pragma unroll
        for (int f = 0; f < N; ++f) {
            const int j = rot<N>(f, ns1);
            a[f] = (j < w1) ? in[(b * w1 + j) * w2 + z] : C{T(0), T(0)};
        }
        fft_line<T, +1, N>(a);
#pragma unroll
        for (int y = 0; y < N; ++y) P[(b * N + y) * PW + z] = a[y];
    }
    __syncthreads();
    for (int l = threadIdx.x; l < tb * N; l += kPlaneThreads) {
        const int b = l / N, y = l % N;
        C a[N];
#pragma unroll
        for (int f = 0; f < N; ++f) {
            const int j = rot<N>(f, ns2);
            a[f] = (j < w2) ? P[(b * N + y) * PW + j] : C{T(0), T(0)};
        }
        fft_line<T, +1, N>(a);
        C *o = out + ((long)b * N + y) * (N + 1);
#pragma unroll
        for (int z = 0; z < N; ++z) o[z] = a[z];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tb * N * N; i += kPlaneThreads) {
        const int b = i / (N * N), r = i % (N * N);
        U[((b0 + b) * n0 + x) * N * N + r] = out[((long)b * N + r / N) * (N + 1) + (r % N)];
    }
}

// -------------------------------------------------------------- launch --
static inline unsigned blocks_for(long n) { return (unsigned)((n + kLineThreads - 1) / kLineThreads); }

#define BGW_FOR_EACH_LEN(n, ...)                                                        \
    switch (n) {                                                                         \
        case 16: { constexpr int N = 16; __VA_ARGS__; } break;                                  \
        case 18: { constexpr int N = 18; __VA_ARGS__; } break;                                  \
        case 20: { constexpr int N = 20; __VA_ARGS__; } break;                                  \
        case 24: { constexpr int N = 24; __VA_ARGS__; } break;                                  \
        case 27: { constexpr int N = 27; __VA_ARGS__; } break;                                  \
        case 30: { constexpr int N = 30; __VA_ARGS__; } break;                                  \
        case 32: { constexpr int N = 32; __VA_ARGS__; } break;                                  \
        case 36: { constexpr int N = 36; __VA_ARGS__; } break;                                  \
        case 40: { constexpr int N = 40; __VA_ARGS__; } break;                                  \
        case 48: { constexpr int N = 48; __VA_ARGS__; } break;                                  \
        case 64: { constexpr int N = 64; __VA_ARGS__; } break;                                  \
        default: return cudaErrorInvalidValue;                                           \
    }

static constexpr size_t kPlaneSmemMax = 110 * 1024;   // two blocks per SM
static constexpr size_t kPlaneSmemLarge = 200 * 1024;  // one block per SM (large boxes)

static bool use_plane_kernels(const Axes &a) {
    return sizeof(T) == 4 && a.n[1] == a.n[2] && a.n[1] < kCoopMinN;
}

static bool use_coop(const Axes &a) {
    return a.n[0] >= kCoopMinN && a.n[1] >= kCoopMinN && a.n[2] >= kCoopMinN && a.n[0] % 16 == 0 &&
           a.n[1] % 16 == 0 && a.n[2] % 16 == 0;
}

// The eight-lane kernels: cubic boxes of the four-lane lengths (48, 64).
static bool use_oct(const Axes &a) { return a.n[0] == a.n[1] && a.n[1] == a.n[2] && a.n[0] <= 64; }
// Cubic boxes the eight-lane kernels can take at all (N = 8M, 4 <= M <= 8);
// automatically chosen only for the four-lane lengths, on request for 32, 40.
static bool oct_len(const Axes &a) {
    const int n = a.n[0];
    return a.n[1] == n && a.n[2] == n && (n == 32 || n == 40 || n == 48 || n == 64);
}

static inline unsigned quads_for(long lines) { return (unsigned)((4 * lines + kLineThreads - 1) / kLineThreads); }

#define BGW_FOR_EACH_OCT_LEN(n, ...)                                                  \
    switch (n) {                                                                      \
        case 32: { constexpr int N = 32; __VA_ARGS__; } break;                        \
        case 40: { constexpr int N = 40; __VA_ARGS__; } break;                        \
        case 48: { constexpr int N = 48; __VA_ARGS__; } break;                        \
        case 64: { constexpr int N = 64; __VA_ARGS__; } break;                        \
        default: return cudaErrorInvalidValue;                                        \
    }

#define BGW_FOR_EACH_COOP_LEN(n, ...)                                                 \
    switch (n) {                                                                      \
        case 48: { constexpr int N = 48; __VA_ARGS__; } break;                        \
        case 64: { constexpr int N = 64; __VA_ARGS__; } break;                        \
        default: return cudaErrorInvalidValue;                                        \
    }

static cudaError_t wfn_to_grid(const double *coeff, int ngw, int B, const int *cube_map,
                               const Axes &a, void *S, void *R, void *U, cudaStream_t st, int path) {
    const long nb = B;
    C *Sp = static_cast<C *>(S), *Rp = static_cast<C *>(R), *Up = static_cast<C *>(U);
    const double2 *cf = reinterpret_cast<const double2 *>(coeff);
    const int *inv = cube_map + (long)a.w[0] * a.w[1] * a.w[2];
    bool oct = oct_len(a) && (path == 3 || (use_coop(a) && use_oct(a)));
    if (path == 4 && sizeof(T) == 4 && a.n[0] == a.n[1] && a.n[1] == a.n[2] && a.n[0] < kCoopMinN) {
        // cube-less one-kernel transform, three CTAs per SM, where it fits
        int KP = 0;
        for (int chunks = 1; chunks <= a.n[0] && !KP; ++chunks) {
            const int kp = (a.n[0] + chunks - 1) / chunks;
            if (fused_smem(a, kp, false) <= kFusedSmem3) KP = kp;
        }
        if (KP) {
            const size_t smem = fused_smem(a, KP, false);
            cudaError_t e = cudaSuccess;
            BGW_FOR_EACH_LEN(a.n[0], {
                if constexpr (N < kCoopMinN) {
                    if (smem > 48 * 1024) {
                        e = cudaFuncSetAttribute(k1_fused<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
                        if (e != cudaSuccess) return e;
                    }
                    k1_fused<N, false><<<(unsigned)nb, kFusedThreads, smem, st>>>(
                        cf, ngw, inv, cube_map, a.w[0], a.w[1], a.w[2], a.s[0], a.s[1], a.s[2], KP, Up);
                }
            });
            return cudaGetLastError();
        }
    }
    const int KP = (path == 1 || oct) ? 0 : fused_planes(a, path == 2 ? kFusedSmemMax : kFusedSmemAuto);
    // automatic choice for cubic FP32 boxes of 32 and 40 whose x-transformed
    // cube does not fit the one-kernel transform: the eight-lane kernels
    // (GaSb-like 32^3: 48.8 -> 41.4 ms per q-point against the one-lane passes)
    if (path == 0 && !KP && sizeof(T) == 4 && oct_len(a)) oct = true;
    if (KP) {
        const size_t smem = fused_smem(a, KP);
        cudaError_t e = cudaSuccess;
        BGW_FOR_EACH_LEN(a.n[0], {
            if constexpr (N < kCoopMinN) {
                if (smem > 48 * 1024) {
                    e = cudaFuncSetAttribute(k1_fused<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
                    if (e != cudaSuccess) return e;
                }
                k1_fused<N, true><<<(unsigned)nb, kFusedThreads, smem, st>>>(
                    cf, ngw, inv, cube_map, a.w[0], a.w[1], a.w[2], a.s[0], a.s[1], a.s[2], KP, Up);
            }
        });
        return cudaGetLastError();
    }
    if (oct) {
        const long groups = nb * a.w[1] * a.w[2];
        BGW_FOR_EACH_OCT_LEN(a.n[0], (k1_xpass_oct<N><<<(unsigned)((groups + 31) / 32), kOctThreads, 0, st>>>(
                                         cf, ngw, nb, cube_map, a.w[0], a.w[1], a.w[2], a.s[0], Sp)));
        const size_t ys = sizeof(C) * ((((size_t)a.n[1] * (a.w[2] | 1)) + 1) / 2 * 2 +
                                       (size_t)(kOctThreads / 8) * kOctBlock);
        cudaError_t e = cudaSuccess;
        BGW_FOR_EACH_OCT_LEN(a.n[1], {
            if (ys > 48 * 1024) {
                e = cudaFuncSetAttribute(k1_yz_oct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ys);
                if (e != cudaSuccess) return e;
            }
            k1_yz_oct<N><<<dim3((unsigned)nb, (unsigned)a.n[0]), kOctThreads, ys, st>>>(Sp, a.w[1], a.w[2], a.s[1],
                                                                                          a.s[2], Up);
        });
        return cudaGetLastError();
    }
    {
        const long lines = nb * a.w[1] * a.w[2];
        BGW_FOR_EACH_LEN(a.n[0], (k1_xpass<N><<<blocks_for(lines), kLineThreads, 0, st>>>(
                                     cf, ngw, nb, cube_map, a.w[0], a.w[1], a.w[2], a.s[0], Sp)));
    }
    if (use_plane_kernels(a)) {
        const int n = a.n[1];
        auto yz_smem = [&](int tb) {
            return sizeof(C) * ((size_t)tb * a.w[1] * a.w[2] + (size_t)tb * n * (a.w[2] + 1) +
                                (size_t)tb * n * (n + 1));
        };
        // band components per CTA: as many as fit two CTAs per SM (fills the
        // 256 threads with w2 y lines and N z lines per component)
        int TB = 16;
        while (TB > 1 && yz_smem(TB) > kPlaneSmemMax) --TB;
        const size_t smem = yz_smem(TB);
        if (smem <= kPlaneSmemLarge) {
            dim3 grid((unsigned)a.n[0], (unsigned)((nb + TB - 1) / TB));
            cudaError_t e = cudaSuccess;
            BGW_FOR_EACH_LEN(n, {
                if (smem > 48 * 1024) {
                    e = cudaFuncSetAttribute(k1_yz_plane<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
                    if (e != cudaSuccess) return e;
                }
                k1_yz_plane<N><<<grid, kPlaneThreads, smem, st>>>(Sp, nb, TB, a.w[1], a.w[2], a.s[1],
                                                                 a.s[2], Up);
            });
            return cudaGetLastError();
        }
    }
    {
        const long nbx = nb * a.n[0];
        BGW_FOR_EACH_LEN(a.n[1], (k1_ypass<N><<<blocks_for(nbx * a.w[2]), kLineThreads, 0, st>>>(
                                     Sp, nbx, a.w[1], a.w[2], a.s[1], Rp)));
    }
    {
        const long nbxy = nb * a.n[0] * a.n[1];
        BGW_FOR_EACH_LEN(a.n[2], (k1_zpass<N><<<blocks_for(nbxy), kLineThreads, 0, st>>>(
                                     Rp, nbxy, a.w[2], a.s[2], Up)));
    }
    return cudaGetLastError();
}

// K1 of several k-points in launches of up to kK1BatchMax: only when every
// job takes the shared-cube one-kernel transform of the automatic path with
// the same box (else *batched = false and nothing is launched; the caller
// runs them one by one).  Same body, planes per chunk and launch bounds as
// k1_fused<N, true>, so the grids are the ones wfn_to_grid writes.
static cudaError_t wfn_to_grid_batch(const K1Job *jobs, int n, int B, cudaStream_t st, bool *batched) {
    *batched = false;
    if (n < 1) return cudaSuccess;
    const int N0 = jobs[0].a.n[0];
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        const Axes &a = jobs[i].a;
        if (a.n[0] != N0 || (oct_len(a) && use_coop(a) && use_oct(a))) return cudaSuccess;
        const int KP = fused_planes(a, kFusedSmemAuto);
        if (!KP) return cudaSuccess;
        const size_t sm = fused_smem(a, KP);
        smem = sm > smem ? sm : smem;
    }
    cudaError_t e = cudaSuccess;
    for (int i0 = 0; i0 < n; i0 += kK1BatchMax) {
        K1Batch jb;
        jb.njobs = n - i0 < kK1BatchMax ? n - i0 : kK1BatchMax;
        jb.B = B;
        for (int i = 0; i < jb.njobs; ++i) {
            const K1Job &j = jobs[i0 + i];
            K1BatchJob &d = jb.job[i];
            d.coeff = reinterpret_cast<const double2 *>(j.coeff);
            d.inv = j.cube_map + (long)j.a.w[0] * j.a.w[1] * j.a.w[2];
            d.U = static_cast<C *>(j.U);
            d.ngw = j.ngw;
            d.w0 = j.a.w[0];
            d.w1 = j.a.w[1];
            d.w2 = j.a.w[2];
            d.s0 = j.a.s[0];
            d.s1 = j.a.s[1];
            d.s2 = j.a.s[2];
            d.KP = fused_planes(j.a, kFusedSmemAuto);
        }
        BGW_FOR_EACH_LEN(N0, {
            if constexpr (N < kCoopMinN) {
                if (smem > 48 * 1024) {
                    e = cudaFuncSetAttribute(k1_fused_batch<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
                    if (e != cudaSuccess) return e;
                }
                k1_fused_batch<N><<<(unsigned)(jb.njobs * B), kFusedThreads, smem, st>>>(jb);
            }
        });
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    *batched = true;
    return cudaSuccess;
}

// Pair tiles (TV valence x TC conduction) of the plane kernel that fit
// kPlaneSmemMax, best first: least staged data per pair, then most pairs.
static size_t plane_smem(int tv, int tc, int n, int w2) {
    const int rs = n % 2 == 0 ? n + 2 : n + 1;
    return sizeof(C) * ((size_t)(tv + tc) * 2 * n * rs + (size_t)tv * tc * n * w2);
}

// Three CTAs per SM (80 registers per thread, no spills up to N = 30) for
// tiles whose shared memory allows it; tiles above kPlaneSmemMax run one CTA
// of 512 threads per SM.
static constexpr size_t kPlaneSmem3 = 72 * 1024;
static bool plane_three_per_sm(const Axes &a, size_t smem) { return a.n[1] <= 30 && smem <= kPlaneSmem3; }
static constexpr int kPlaneThreadsLarge = 512;

static int plane_tile_list(int nv, int nc, const Axes &a, int *TV, int *TC, int max) {
    if (!use_plane_kernels(a)) return 0;
    struct Cand { double cost; int tv, tc; };
    // three ranked lists: tiles for two CTAs per SM (the default first),
    // smaller tiles that allow three, and large tiles for one CTA of 512
    // threads
    Cand best[3][64];
    int nbest[3] = {0, 0, 0};
    for (int tv = 1; tv <= nv && tv <= 16; ++tv)
        for (int tc = 1; tc <= nc && tc <= 16; ++tc) {
            const size_t sm = plane_smem(tv, tc, a.n[1], a.w[2]);
            if (sm > kPlaneSmemLarge) continue;
            const int cls = sm > kPlaneSmemMax ? 2 : plane_three_per_sm(a, sm) ? 1 : 0;
            Cand *b = best[cls];
            const Cand c{(double)(tv + tc) / (tv * tc) - 1e-3 * tv * tc, tv, tc};
            int pos = nbest[cls] < 64 ? nbest[cls]++ : 63;
            if (pos == 63 && c.cost >= b[63].cost) continue;
            b[pos] = c;
            while (pos > 0 && b[pos].cost < b[pos - 1].cost) {
                const Cand t = b[pos];
                b[pos] = b[pos - 1];
                b[pos - 1] = t;
                --pos;
            }
        }
    int n = 0;
    for (int i = 0; n < max && (i < nbest[0] || i < nbest[1] || i < nbest[2]); ++i)
        for (int cls = 0; cls < 3 && n < max; ++cls)
            if (i < nbest[cls]) {
                TV[n] = best[cls][i].tv;
                TC[n] = best[cls][i].tc;
                ++n;
            }
    return n;
}

// The x pass of the one-lane-per-line paths: gather through shared memory
// when the kept cube is small, else scatter through the inverse map.
// Whether every kept output along axis ax lies within kWin of 0.
static bool kept_in_window(const Axes &a, int ax) {
    for (int j = 0; j < a.w[ax]; ++j) {
        const int f = (a.s[ax] + j) % a.n[ax];
        if (f > kWin && f < a.n[ax] - kWin) return false;
    }
    return true;
}

static cudaError_t xpass(const C *Bp, long P, const Axes &a, const int *gmap, int ng, C *Mp, long ldm,
                         cudaStream_t st) {
    const size_t smem = sizeof(C) * (size_t)a.w[0] * a.w[1] * a.w[2];
    const T scale = (T)(1.0 / ((double)a.n[0] * a.n[1] * a.n[2]));
    cudaError_t e = cudaSuccess;
    if (mtxel_scatter_mode(a, sizeof(C))) {
        const long lines = (long)a.w[1] * a.w[2];
        BGW_FOR_EACH_LEN(a.n[0], (k2_xpass_scatter<N><<<blocks_for(P * lines), kLineThreads, 0, st>>>(
                                     Bp, P, a.w[0], a.w[1], a.w[2], a.s[0], gmap + ng, scale, Mp, ldm)));
        return cudaGetLastError();
    }
    BGW_FOR_EACH_LEN(a.n[0], {
        const int PP = gather_pairs(a, P);
        auto kern = k2_xpass_gather<N, false>;
        if constexpr (N > 2 * kWin + 1)
            if (kept_in_window(a, 0)) kern = k2_xpass_gather<N, true>;
        if (smem * PP > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem * PP));
            if (e != cudaSuccess) return e;
        }
        kern<<<(unsigned)((P + PP - 1) / PP), kGatherThreads, smem * PP, st>>>(
            Bp, P, PP, a.w[0], a.w[1], a.w[2], a.s[0], gmap, ng, scale, Mp, ldm);
    });
    return cudaGetLastError();
}

// The streamed z + y kernel applies to FP32 boxes of the plane kernels with an
// even N <= 32 whose kept z outputs of 16 pairs fit in one conduction buffer.
#define BGW_FOR_EACH_STREAM_LEN(n, ...)                                                \
    switch (n) {                                                                       \
        case 16: { constexpr int N = 16; __VA_ARGS__; } break;                         \
        case 18: { constexpr int N = 18; __VA_ARGS__; } break;                         \
        case 20: { constexpr int N = 20; __VA_ARGS__; } break;                         \
        case 24: { constexpr int N = 24; __VA_ARGS__; } break;                         \
        case 30: { constexpr int N = 30; __VA_ARGS__; } break;                         \
        case 32: { constexpr int N = 32; __VA_ARGS__; } break;                         \
        default: return cudaErrorInvalidValue;                                         \
    }


static bool use_stream(const Axes &a) {
    const int n = a.n[1];
    if (!use_plane_kernels(a) || n % 2 != 0 || n > 32 || n == 28 || n == 26 || n == 22) return false;
    return a.w[2] <= kZW;
}

// Marks around one x-pass launch group for the profiling hook.
struct XMark {
    const XPassHook *h;
    XMark(const XPassHook *hook, int zy_kernels) : h(hook) {
        if (h) h->fn(h->ctx, 1, zy_kernels);
    }
    ~XMark() {
        if (h) h->fn(h->ctx, 0, 1);
    }
};

// Tensor maps of the valence (nvb bands from uv) and conduction (nc bands
// from uc) grids for the TMA form of the streamed kernel: 4-D, innermost the
// 2 N floats of a z row, then y, x and band component; one box is half a row
// (kTmaHalf values, 128 bytes) by all N rows, 128-byte swizzle.
static cudaError_t stream_maps(const C *uv, int nvb, const C *uc, int nc, const Axes &a, CUtensorMap *mv,
                               CUtensorMap *mc) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    cudaError_t e = tc::tensor_map_encoder(&enc);
    if (e != cudaSuccess) return e;
    auto one = [&](const C *base, int nb, CUtensorMap *m) -> cudaError_t {
        const cuuint64_t row = (cuuint64_t)a.n[2] * sizeof(C);
        const cuuint64_t dims[4] = {(cuuint64_t)2 * a.n[2], (cuuint64_t)a.n[1], (cuuint64_t)a.n[0], (cuuint64_t)2 * nb};
        const cuuint64_t strides[3] = {row, row * a.n[1], row * a.n[1] * a.n[0]};
        const cuuint32_t box[4] = {2 * kTmaHalf, (cuuint32_t)a.n[1], 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<C *>(base), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
    };
    e = one(uv, nvb, mv);
    if (e == cudaSuccess) e = one(uc, nc, mc);
    return e;
}

static cudaError_t mtxel_batch(const C *uv, const C *uc, int nv, int nc, const Axes &a,
                               const int *gmap, int ng, C *Ap, C *Bp, C *Mp, long ldm,
                               cudaStream_t st, int tv_req, int tc_req, int lanes, int zy,
                               const XPassHook *hook, int *err, int drop) {
    const long P = (long)nv * nc;
    if (oct_len(a) && (lanes == 8 || (lanes == 0 && use_coop(a) && use_oct(a)))) {
        // eight lanes per line: fused z+y, then the x pass
        const size_t zs = sizeof(C) * ((((size_t)a.n[1] * (a.w[2] | 1)) + 1) / 2 * 2 +
                                       (size_t)(kOctThreads / 8) * kOctBlock);
        cudaError_t e = cudaSuccess;
        BGW_FOR_EACH_OCT_LEN(a.n[2], {
            if (zs > 48 * 1024) {
                e = cudaFuncSetAttribute(k2_zy_oct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zs);
                if (e != cudaSuccess) return e;
            }
            k2_zy_oct<N><<<dim3((unsigned)P, (unsigned)a.n[0]), kOctThreads, zs, st>>>(
                uv, uc, nc, a.w[1], a.w[2], a.s[1], a.s[2], Bp);
        });
        const long lines = (long)a.w[1] * a.w[2];
        const T scale = (T)(1.0 / ((double)a.n[0] * a.n[1] * a.n[2]));
        XMark xm(hook, 1);
        if (mtxel_scatter_mode(a, sizeof(C))) {
            const long groups = P * lines;
            BGW_FOR_EACH_OCT_LEN(a.n[0], (k2_xpass_scatter_oct<N><<<(unsigned)((groups + 31) / 32), kOctThreads,
                                                                     0, st>>>(Bp, P, a.w[0], a.w[1], a.w[2], a.s[0],
                                                                              gmap + ng, scale, Mp, ldm)));
            return cudaGetLastError();
        }
        const size_t smem = sizeof(C) * (size_t)a.w[0] * a.w[1] * a.w[2];
        BGW_FOR_EACH_LEN(a.n[0], {
            const int PP = gather_pairs(a, P);
            auto kern = k2_xpass_gather<N, false>;
            if constexpr (N > 2 * kWin + 1)
                if (kept_in_window(a, 0)) kern = k2_xpass_gather<N, true>;
            if (smem * PP > 48 * 1024) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem * PP));
                if (e != cudaSuccess) return e;
            }
            kern<<<(unsigned)((P + PP - 1) / PP), kGatherThreads, smem * PP, st>>>(
                Bp, P, PP, a.w[0], a.w[1], a.w[2], a.s[0], gmap, ng, scale, Mp, ldm);
        });
        return cudaGetLastError();
    }
    if ((zy == 2 || (zy == 0 && tv_req <= 0)) && use_stream(a)) {
        // streamed pair density + z + y: conduction ranges sized for about four
        // waves of one CTA per SM
        static int sms = 0;
        if (sms == 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
                sms = 148;
        }
        cudaError_t e = cudaSuccess;
        const bool win = kept_in_window(a, 1) && kept_in_window(a, 2);
        CUtensorMap mv, mc;
        memset(&mv, 0, sizeof mv);
        memset(&mc, 0, sizeof mc);
        auto launch = [&](auto kern, int SV, int SC, size_t ss) -> cudaError_t {
            const int nvg = (nv + SV - 1) / SV;
            const long want = 4L * sms;
            const long per = (long)a.n[0] * nvg;
            const int chunks = (int)((want + per - 1) / per);
            int CC = (nc + chunks - 1) / chunks;
            CC = (CC + SC - 1) / SC * SC;
            if (CC < SC) CC = SC;
            dim3 grid((unsigned)a.n[0], (unsigned)nvg, (unsigned)((nc + CC - 1) / CC));
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
            if (r != cudaSuccess) return r;
            kern<<<grid, kStreamThreads, ss, st>>>(uv, uc, nv, nc, CC, a.w[1], a.w[2], a.s[1], a.s[2], Bp, mv, mc,
                                                   err, drop);
            return cudaSuccess;
        };
        BGW_FOR_EACH_STREAM_LEN(a.n[1], {
            constexpr bool kTma = N == 2 * kTmaHalf && sizeof(T) == 4;   // 32^3 boxes: planes by TMA
            constexpr int V0 = StreamTile<N>::V, C0 = StreamTile<N>::C;
            if constexpr (kTma) {
                e = stream_maps(uv, nv, uc, nc, a, &mv, &mc);
                if (e != cudaSuccess) return e;
                // 2 x 4 band groups where they need fewer phases than 4 x 2 (a
                // valence count that is not a multiple of 4) and fit
                const long ph0 = (long)((nv + V0 - 1) / V0) * ((nc + C0 - 1) / C0);
                const long ph1 = (long)((nv + 1) / 2) * ((nc + 3) / 4);
                const size_t ss1 = stream_smem<N, 2, 4, true>(a.w[2]);
                if (ph1 < ph0 && ss1 + 256 <= (size_t)227 * 1024) {
                    e = win ? launch(k2_zy_stream<N, 2, 4, true, true>, 2, 4, ss1)
                            : launch(k2_zy_stream<N, 2, 4, false, true>, 2, 4, ss1);
                    break;
                }
            }
            const size_t ss = stream_smem<N, V0, C0, kTma>(a.w[2]);
            auto kern = k2_zy_stream<N, V0, C0, false, kTma>;
            if constexpr (N > 2 * kWin + 1)
                if (win) kern = k2_zy_stream<N, V0, C0, true, kTma>;
            e = launch(kern, V0, C0, ss);
        });
        if (e != cudaSuccess) return e;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        XMark xm(hook, 1);
        return xpass(Bp, P, a, gmap, ng, Mp, ldm, st);
    }
    int TV = 0, TC = 0;
    if (use_plane_kernels(a)) {
        if (tv_req > 0 && tc_req > 0 && plane_smem(tv_req, tc_req, a.n[1], a.w[2]) <= kPlaneSmemLarge) {
            TV = tv_req < nv ? tv_req : nv;
            TC = tc_req < nc ? tc_req : nc;
        } else {
            plane_tile_list(nv, nc, a, &TV, &TC, 1);
        }
    }
    const size_t psmem = TV > 0 ? plane_smem(TV, TC, a.n[1], a.w[2]) : 0;
    if (use_coop(a)) {                                  // non-cubic boxes of the four-lane lengths
        const long plane = (long)a.n[0] * a.n[1];
        BGW_FOR_EACH_COOP_LEN(a.n[2], (k2_zpass_c4<N><<<quads_for(P * plane), kLineThreads, 0, st>>>(
                                          uv, uc, nc, P, plane, a.w[2], a.s[2], Ap)));
        const long npx = P * a.n[0];
        BGW_FOR_EACH_COOP_LEN(a.n[1], (k2_ypass_c4<N><<<quads_for(npx * a.w[2]), kLineThreads, 0, st>>>(
                                          Ap, npx, a.w[1], a.w[2], a.s[1], Bp)));
        const long lines = (long)a.w[1] * a.w[2];
        const T scale = (T)(1.0 / ((double)a.n[0] * a.n[1] * a.n[2]));
        XMark xm(hook, 2);
        BGW_FOR_EACH_COOP_LEN(a.n[0], (k2_xpass_scatter_c4<N><<<quads_for(P * lines), kLineThreads, 0, st>>>(
                                          Bp, P, a.w[0], a.w[1], a.w[2], a.s[0], gmap + ng, scale, Mp, ldm)));
        return cudaGetLastError();
    }
    if (TV > 0) {
        dim3 grid((unsigned)a.n[0], (unsigned)((nv + TV - 1) / TV), (unsigned)((nc + TC - 1) / TC));
        cudaError_t e = cudaSuccess;
        const bool three = plane_three_per_sm(a, psmem);
        const bool large = psmem > kPlaneSmemMax;
        const bool win = kept_in_window(a, 1) && kept_in_window(a, 2);
        BGW_FOR_EACH_LEN(a.n[1], {
            auto kern = k2_zy_plane<N, 2, kPlaneThreads>;
            if constexpr (N <= 30)
                if (three) kern = k2_zy_plane<N, 3, kPlaneThreads>;
            if (large) kern = k2_zy_plane<N, 1, kPlaneThreadsLarge>;
            if constexpr (N > 2 * kWin + 1 && sizeof(T) == 4) {   // the plane kernels run in FP32 only
                if (win) {
                    kern = k2_zy_plane<N, 2, kPlaneThreads, true>;
                    if constexpr (N <= 30)
                        if (three) kern = k2_zy_plane<N, 3, kPlaneThreads, true>;
                    if (large) kern = k2_zy_plane<N, 1, kPlaneThreadsLarge, true>;
                }
            }
            if (psmem > 48 * 1024) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
                if (e != cudaSuccess) return e;
            }
            kern<<<grid, large ? kPlaneThreadsLarge : kPlaneThreads, psmem, st>>>(
                uv, uc, nv, nc, TV, TC, a.w[1], a.w[2], a.s[1], a.s[2], Bp);
        });
    } else {
        const long plane = (long)a.n[0] * a.n[1];
        const bool wz = kept_in_window(a, 2), wy = kept_in_window(a, 1);
        BGW_FOR_EACH_LEN(a.n[2], {
            auto kern = k2_zpass<N, false>;
            if constexpr (N > 2 * kWin + 1)
                if (wz) kern = k2_zpass<N, true>;
            kern<<<blocks_for(P * plane), kLineThreads, 0, st>>>(uv, uc, nc, P, plane, a.w[2], a.s[2], Ap);
        });
        const long npx = P * a.n[0];
        BGW_FOR_EACH_LEN(a.n[1], {
            auto kern = k2_ypass<N, false>;
            if constexpr (N > 2 * kWin + 1)
                if (wy) kern = k2_ypass<N, true>;
            kern<<<blocks_for(npx * a.w[2]), kLineThreads, 0, st>>>(Ap, npx, a.w[1], a.w[2], a.s[1], Bp);
        });
    }
    XMark xm(hook, TV > 0 ? 1 : 2);
    return xpass(Bp, P, a, gmap, ng, Mp, ldm, st);
}

static cudaError_t mtxel(const void *Uv, const void *Uc, int nv, int nc, const Axes &a,
                         const int *gmap, int ng, void *A, void *Bs, void *M, long ldm,
                         cudaStream_t st, int tv_req, int tc_req, int lanes, int zy, const XPassHook *hook,
                         int *err, int drop) {
    if ((long)nv * nc == 0) return cudaSuccess;
    const C *uv = static_cast<const C *>(Uv), *uc = static_cast<const C *>(Uc);
    C *Ap = static_cast<C *>(A), *Bp = static_cast<C *>(Bs), *Mp = static_cast<C *>(M);
    const long vol = (long)a.n[0] * a.n[1] * a.n[2];
    const int VB = mtxel_v_batch(nv, nc, a, sizeof(C));
    for (int vb0 = 0; vb0 < nv; vb0 += VB) {
        const int nvb = nv - vb0 < VB ? nv - vb0 : VB;
        cudaError_t e = mtxel_batch(uv + (long)vb0 * 2 * vol, uc, nvb, nc, a, gmap, ng, Ap, Bp,
                                    Mp + (long)vb0 * nc * ldm, ldm, st, tv_req, tc_req, lanes, zy, hook, err, drop);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

#undef BGW_FOR_EACH_LEN
#undef BGW_FOR_EACH_COOP_LEN
#undef BGW_FOR_EACH_OCT_LEN
#undef BGW_FOR_EACH_STREAM_LEN

}  // namespace BGW_SUFFIX
}  // namespace bgw
