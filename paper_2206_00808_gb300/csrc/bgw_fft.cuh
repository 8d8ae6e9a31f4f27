// Mixed-radix FFT of one line per thread in registers (with four- and
// eight-lane variants for long lines, below), for the short box
// lengths of plane-wave codes (products of 2, 3 and 5 up to 64).
//
// The transform of Eq. (matrix_el) of arXiv:2206.00808 is a 3-D DFT; it is
// done here one axis at a time, each line held in the registers of one
// thread.  Lengths are compile-time, so every index below is a constant and
// the arrays stay in registers.
//
// Decomposition (Cooley-Tukey, decimation in time): N = R * M with
// n = R*n2 + n1 and k = k1 + M*k2,
//   X[k1 + M k2] = sum_{n1} w_R^{n1 k2} [ w_N^{n1 k1} (sum_{n2} x[R n2 + n1] w_M^{n2 k1}) ],
// i.e. R sub-transforms of length M, a twiddle, then M transforms of length R.
// w_N = exp(S * 2 pi i / N): S = -1 forward (e^{-iG.r}), S = +1 inverse.
//
// Twiddles are exp(-2 pi i j / N) for every supported N, computed on the
// host in double precision (std::cos / std::sin) and kept in constant memory
// (one table per translation unit; bgw_fft_upload_tables fills it).
#pragma once
#include <cuda_runtime.h>

namespace bgw {

template <typename T> struct cpx { T x, y; };

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
// conj(a) * b
template <typename T>
__device__ __forceinline__ cpx<T> cconjmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
// conj(a0) b0 + conj(a1) b1 (the spinor trace of a pair density) as one
// multiply-add chain per component: 8 operations instead of 10.
template <typename T>
__device__ __forceinline__ cpx<T> rho2(cpx<T> a0, cpx<T> b0, cpx<T> a1, cpx<T> b1) {
    T re = a0.x * b0.x;
    re = fma(a0.y, b0.y, re);
    re = fma(a1.x, b1.x, re);
    re = fma(a1.y, b1.y, re);
    T im = a0.x * b0.y;
    im = fma(-a0.y, b0.x, im);
    im = fma(a1.x, b1.y, im);
    im = fma(-a1.y, b1.x, im);
    return {re, im};
}

// ----------------------------------------------------------- twiddle tables --
constexpr int kFftLens[] = {16, 18, 20, 24, 27, 30, 32, 36, 40, 48, 64};
constexpr int kNumFftLens = sizeof(kFftLens) / sizeof(int);

__host__ __device__ constexpr int tw_offset(int n) {
    // running sum of the lengths listed in kFftLens before n
    return n == 16 ? 0 : n == 18 ? 16 : n == 20 ? 34 : n == 24 ? 54 : n == 27 ? 78
         : n == 30 ? 105 : n == 32 ? 135 : n == 36 ? 167 : n == 40 ? 203 : n == 48 ? 243
         : n == 64 ? 291 : -1;
}
constexpr int kTwTotal = tw_offset(64) + 64;

__host__ __device__ constexpr bool fft_len_supported(int n) { return tw_offset(n) >= 0; }

// Forward roots w^j = exp(-2 pi i j / N); j-th entry of length N at tw_offset(N).
static __constant__ double2 c_tw64[kTwTotal];
static __constant__ float2 c_tw32[kTwTotal];

template <typename T> struct Tw;
template <> struct Tw<double> {
    static __device__ __forceinline__ cpx<double> at(int i) {
        double2 v = c_tw64[i];
        return {v.x, v.y};
    }
};
template <> struct Tw<float> {
    static __device__ __forceinline__ cpx<float> at(int i) {
        float2 v = c_tw32[i];
        return {v.x, v.y};
    }
};

// exp(-2 pi i j / NTOP) with runtime j in [0, NTOP) (warp-uniform j is cheap).
template <typename T, int NTOP>
__device__ __forceinline__ cpx<T> root_fwd(int j) {
    return Tw<T>::at(tw_offset(NTOP) + j);
}
// exp(+2 pi i j / NTOP)
template <typename T, int NTOP>
__device__ __forceinline__ cpx<T> root_inv(int j) {
    cpx<T> w = Tw<T>::at(tw_offset(NTOP) + j);
    return {w.x, -w.y};
}

// Multiply by w_N^E (w_N = exp(S 2 pi i / N)) with E a compile-time exponent;
// the table of the top-level length NTOP serves every sub-length N | NTOP.
template <typename T, int S, int N, int NTOP, int E>
__device__ __forceinline__ cpx<T> twiddle(cpx<T> a) {
    constexpr int e = E % N;
    if constexpr (e == 0) {
        return a;
    } else if constexpr (2 * e == N) {
        return {-a.x, -a.y};
    } else if constexpr (4 * e == N) {        // w = S i
        return {-(T)S * a.y, (T)S * a.x};
    } else if constexpr (4 * e == 3 * N) {    // w = -S i
        return {(T)S * a.y, -(T)S * a.x};
    } else {
        cpx<T> w = Tw<T>::at(tw_offset(NTOP) + e * (NTOP / N));
        if constexpr (S > 0) w.y = -w.y;
        return cmul(a, w);
    }
}

__host__ __device__ constexpr int first_radix(int n) {
    return (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : n;
}

// Length-R DFT in place, R in {2, 3, 4, 5}.
template <typename T, int S, int R, int NTOP>
__device__ __forceinline__ void dft_small(cpx<T> (&a)[R]) {
    if constexpr (R == 2) {
        cpx<T> t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    } else if constexpr (R == 4) {
        cpx<T> t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        cpx<T> t2 = cadd(a[1], a[3]), d = csub(a[1], a[3]);
        cpx<T> t3 = {-(T)S * d.y, (T)S * d.x};   // (a1 - a3) * (S i)
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    } else if constexpr (R == 3) {
        // w_3 = -1/2 + S i sqrt(3)/2
        constexpr T h = (T)0.86602540378443864676372317075293618;
        cpx<T> t1 = cadd(a[1], a[2]), t2 = csub(a[1], a[2]);
        cpx<T> m = {a[0].x - (T)0.5 * t1.x, a[0].y - (T)0.5 * t1.y};
        cpx<T> r = {-(T)S * h * t2.y, (T)S * h * t2.x};   // S i (sqrt3/2) t2
        a[0] = cadd(a[0], t1);
        a[1] = cadd(m, r);
        a[2] = csub(m, r);
    } else {
        static_assert(R == 5, "radix");
        cpx<T> x[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) x[k] = a[k];
        // direct 5-point sum with table roots (w_5^j = w_NTOP^{j NTOP/5})
        a[0] = cadd(cadd(cadd(x[0], x[1]), cadd(x[2], x[3])), x[4]);
#pragma unroll
        for (int k = 1; k < 5; ++k) {
            cpx<T> s = x[0];
#pragma unroll
            for (int n = 1; n < 5; ++n) {
                const int e = (n * k) % 5;
                cpx<T> w = Tw<T>::at(tw_offset(NTOP) + e * (NTOP / 5));
                if (S > 0) w.y = -w.y;
                s = cadd(s, cmul(x[n], w));
            }
            a[k] = s;
        }
    }
}

template <typename T, int S, int N, int NTOP>
struct Fft {
    static constexpr int R = first_radix(N);
    static constexpr int M = N / R;

    // sub[n1][k1] *= w_N^{n1 k1}, unrolled at compile time over (n1, k1).
    template <int N1, int K1>
    __device__ __forceinline__ static void stage_twiddle(cpx<T> (&sub)[R][M]) {
        if constexpr (N1 < R) {
            if constexpr (K1 < M) {
                sub[N1][K1] = twiddle<T, S, N, NTOP, N1 * K1>(sub[N1][K1]);
                stage_twiddle<N1, K1 + 1>(sub);
            } else {
                stage_twiddle<N1 + 1, 0>(sub);
            }
        }
    }

    __device__ __forceinline__ static void run(cpx<T> (&a)[N]) {
        if constexpr (M == 1) {
            dft_small<T, S, R, NTOP>(a);
        } else {
            cpx<T> sub[R][M];
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1)
#pragma unroll
                for (int n2 = 0; n2 < M; ++n2) sub[n1][n2] = a[R * n2 + n1];
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) Fft<T, S, M, NTOP>::run(sub[n1]);
            stage_twiddle<1, 0>(sub);
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                cpx<T> t[R];
#pragma unroll
                for (int n1 = 0; n1 < R; ++n1) t[n1] = sub[n1][k1];
                dft_small<T, S, R, NTOP>(t);
#pragma unroll
                for (int k2 = 0; k2 < R; ++k2) a[k1 + M * k2] = t[k2];
            }
        }
    }
};

// Forward (S = -1) or inverse (S = +1) unnormalised DFT of length N.
template <typename T, int S, int N>
__device__ __forceinline__ void fft_line(cpx<T> (&a)[N]) {
    static_assert(fft_len_supported(N), "unsupported FFT length");
    Fft<T, S, N, N>::run(a);
}

// ------------------------------------------- four lanes per line (N >= 32) --
// Lanes t = 0..3 of an aligned group of four transform one line of length
// N = 4M together (Cooley-Tukey with the stride-4 split):
//   lane t enters with a[m] = x[4m + t], m < M;
//   Y_t[k2] = sum_m x[4m + t] w_M^{m k2}           (M-point DFT in registers)
//   Y_t[k2] *= w_N^{t k2}                          (twiddle)
//   X[k2 + M k1] = sum_t' Y_t'[k2] w_4^{t' k1}    (4-point DFT across lanes)
// and leaves with out[k1][j] = X[t Q + j + M k1], Q = M/4, j < Q.
// Values are picked with selects on t and exchanged with __shfl_xor, so no
// register array is indexed at run time.
template <typename T>
__device__ __forceinline__ cpx<T> sel4(int i, cpx<T> v0, cpx<T> v1, cpx<T> v2, cpx<T> v3) {
    cpx<T> r = v0;
    r = (i == 1) ? v1 : r;
    r = (i == 2) ? v2 : r;
    r = (i == 3) ? v3 : r;
    return r;
}

template <typename T>
__device__ __forceinline__ cpx<T> shfl_xor_c(cpx<T> v, int d) {
    return {__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d)};
}

template <typename T, int S, int N>
__device__ __forceinline__ void fft_line_coop4(cpx<T> (&a)[N / 4], int t, cpx<T> (&out)[4][N / 16]) {
    static_assert(fft_len_supported(N) && N % 16 == 0, "four-lane FFT needs N a multiple of 16");
    constexpr int M = N / 4;
    constexpr int Q = M / 4;
    Fft<T, S, M, N>::run(a);
    // twiddle w_N^{t k2}: pick among the warp-uniform roots of exponents k2, 2k2, 3k2
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) {
        cpx<T> w1 = Tw<T>::at(tw_offset(N) + (k2 % N));
        cpx<T> w2 = Tw<T>::at(tw_offset(N) + ((2 * k2) % N));
        cpx<T> w3 = Tw<T>::at(tw_offset(N) + ((3 * k2) % N));
        if (S > 0) {
            w1.y = -w1.y;
            w2.y = -w2.y;
            w3.y = -w3.y;
        }
        const cpx<T> w = sel4<T>(t, cpx<T>{T(1), T(0)}, w1, w2, w3);
        a[k2] = cmul(a[k2], w);
    }
    // lane t gathers Y_t'[t Q + j] from every lane t'
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        cpx<T> y[4];
        // own value
        y[0] = sel4<T>(t, a[j], a[Q + j], a[2 * Q + j], a[3 * Q + j]);
#pragma unroll
        for (int d = 1; d < 4; ++d) {
            // send the entry of the partner's block, receive the partner's entry of ours
            const int pb = t ^ d;
            const cpx<T> send = sel4<T>(pb, a[j], a[Q + j], a[2 * Q + j], a[3 * Q + j]);
            y[d] = shfl_xor_c(send, d);
        }
        // y[d] came from lane t ^ d: order by source lane
        cpx<T> z[4];
#pragma unroll
        for (int tp = 0; tp < 4; ++tp) {
            const int d = t ^ tp;
            z[tp] = sel4<T>(d, y[0], y[1], y[2], y[3]);
        }
        dft_small<T, S, 4, N>(z);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) out[k1][j] = z[k1];
    }
}

// ---------------------------------------------- eight lanes per line (N = 8M) --
// Lanes t = 0..7 of an aligned group of eight transform one line of length
// N = 8M (M = 6 or 8) together, exchanging through shared memory:
//   lane t enters with a[m] = x[8m + t], m < M;
//   Y_t[k2] = sum_m x[8m + t] w_M^{m k2}            (M-point DFT in registers)
//   Y_t[k2] *= w_N^{t k2}                           (lane twiddles, tw[k2])
//   ex[k2][t] = Y_t[k2]                             (8 x 9 padded shared block)
//   lane k2 < M: X[k2 + M k1] = sum_t Y_t[k2] w_8^{t k1}   (8-point DFT)
// and leaves with out[k1] = X[t + M k1] (meaningful for t < M).  The row pad
// of 9 keeps both the column writes and the row reads free of bank conflicts
// for two groups per half-warp when groups sit 72 entries apart.  Every lane
// of the warp must call this together (it synchronises the warp).
constexpr int kOctRow = 9;
constexpr int kOctBlock = 8 * kOctRow;

// tw[k2] = w_N^{S t k2} for this lane (computed once per kernel).
template <typename T, int S, int N>
__device__ __forceinline__ void oct_twiddles(int t, cpx<T> (&tw)[N / 8]) {
#pragma unroll
    for (int k2 = 0; k2 < N / 8; ++k2) {
        cpx<T> w = Tw<T>::at(tw_offset(N) + (t * k2) % N);
        if (S > 0) w.y = -w.y;
        tw[k2] = w;
    }
}

template <typename T, int S, int N>
__device__ __forceinline__ void fft_line_oct(cpx<T> (&a)[N / 8], int t, cpx<T> *ex,
                                             const cpx<T> (&tw)[N / 8], cpx<T> (&out)[8]) {
    static_assert(fft_len_supported(N) && N % 8 == 0 && N / 8 <= 8, "eight-lane FFT: N = 8M, M <= 8");
    constexpr int M = N / 8;
    Fft<T, S, M, N>::run(a);
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) a[k2] = cmul(a[k2], tw[k2]);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) ex[k2 * kOctRow + t] = a[k2];
    __syncwarp();
    const int r = t < M ? t : 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = ex[r * kOctRow + i];
    __syncwarp();
    Fft<T, S, 8, N>::run(out);
}

}  // namespace bgw
