// Internal launchers shared by the C-ABI layer (bgw_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#ifdef BGW_BOUNDS
#define BGW_BOUNDS_BUILD (BGW_BOUNDS != 0)
#else
#define BGW_BOUNDS_BUILD false
#endif

namespace bgw {

// Extents of a pruned transform along the three box axes.
struct Axes {
    int n[3];   // FFT box N1, N2, N3
    int w[3];   // kept (or occupied) width along each axis, 1 <= w <= n
    int s[3];   // start index along each axis (mod n), 0 <= s < n
};

// ---- bgw_grid_f64.cu / bgw_grid_f32.cu (T = double / float) -------------
// Twiddle tables into this translation unit's constant memory (per device).
cudaError_t grid_tables_init_f64();
cudaError_t grid_tables_init_f32();

// Sphere -> real space for B = 2*nb band components of one k:
//   u_b(r) = sum_{h in sphere} c_b(h) e^{+2 pi i h.r / N}
// coeff: complex128 [B][ngw]; cube_map: [w0][w1][w2] -> coefficient index or
// -1 (cube origin at Miller index s, i.e. a.s = sphere minimum), followed by
// the inverse map [ngw] -> cube cell; S: [B][n0][w1][w2], R: [B][n0][n1][w2]
// scratch of T-complex; U: [B][n0][n1][n2] T-complex.  path: 0 automatic,
// 1 the per-axis pass kernels, 2 the one-kernel transform where it fits,
// 3 the eight-lane kernels where the box is cubic with N = 32, 40, 48 or 64,
// 4 the one-kernel transform without the shared cube (FP32, three CTAs/SM).
cudaError_t wfn_to_grid_f64(const double *coeff, int ngw, int B, const int *cube_map,
                            const Axes &a, void *S, void *R, void *U, cudaStream_t st, int path = 0);
cudaError_t wfn_to_grid_f32(const double *coeff, int ngw, int B, const int *cube_map,
                            const Axes &a, void *S, void *R, void *U, cudaStream_t st, int path = 0);

// One k-point's sphere -> grid job for the batched launcher.
struct K1Job {
    const double *coeff;      // complex128 [B][ngw] (device)
    int ngw;
    const int *cube_map;      // cube map followed by the inverse map (device)
    Axes a;
    void *U;                  // grid slot [B][n0][n1][n2]
};
// K1 of n k-points in as few launches as possible, when every job takes the
// shared-cube one-kernel transform with one box length; *batched = false and
// nothing launched otherwise.
cudaError_t wfn_to_grid_batch_f64(const K1Job *jobs, int n, int B, cudaStream_t st, bool *batched);
cudaError_t wfn_to_grid_batch_f32(const K1Job *jobs, int n, int B, cudaStream_t st, bool *batched);

// Pair density, pruned forward FFT and gather for P = nv*nc pairs of one k:
//   M[v*nc+c][g] = N^-3 sum_r sum_alpha conj(u_v,alpha(r)) u_c,alpha(r) e^{-2 pi i f_g.r/N}
// with f_g the output frequency of G-vector g (G + G0).  Uv: [nv][2][N^3],
// Uc: [nc][2][N^3] (T-complex); a.s = first kept frequency per axis,
// a.w = kept widths; gmap[g] = j0*w1*w2 + j1*w2 + j2 (position in the kept
// cube); A: [P][n0][n1][w2], Bs: [P][n0][w1][w2] scratch; M row stride ldm.
// tv, tc: pair tile of the plane-fused FP32 kernel (0 = choose automatically).
// lanes: 0 automatic; 8 eight lanes per line wherever the box is cubic with
// N = 32, 40, 48 or 64 (automatic choice uses them for 48 and 64 only).
// Pairs are processed in batches of mtxel_v_batch(...) valence bands x nc, so
// A and Bs need room for that many pairs only.
// zy (FP32): 0 automatic (the streamed z + y kernel where it applies, unless a
// pair tile tv x tc is given), 1 the plane kernel with the pair tile tv x tc,
// 2 streamed where it applies.
// hook (profiling, may be NULL): fn(ctx, 1, n) just before each x-pass launch
// group (n = kernels launched since the previous mark) and fn(ctx, 0, n)
// right after it.  err (may be NULL): device int that a bounded wait of the
// streamed FP32 kernel's TMA staging sets to 5 when it gives up.  drop
// (tests only): the first CTA of that kernel skips one plane copy, so that
// wait expires.
struct XPassHook {
    void (*fn)(void *ctx, int begin, int kernels);
    void *ctx;
};
cudaError_t mtxel_f64(const void *Uv, const void *Uc, int nv, int nc, const Axes &a,
                      const int *gmap, int ng, void *A, void *Bs, void *M, long ldm,
                      cudaStream_t st, int tv = 0, int tc = 0, int lanes = 0, int zy = 0,
                      const XPassHook *hook = nullptr, int *err = nullptr, int drop = 0);
cudaError_t mtxel_f32(const void *Uv, const void *Uc, int nv, int nc, const Axes &a,
                      const int *gmap, int ng, void *A, void *Bs, void *M, long ldm,
                      cudaStream_t st, int tv = 0, int tc = 0, int lanes = 0, int zy = 0,
                      const XPassHook *hook = nullptr, int *err = nullptr, int drop = 0);
// The last forward pass gathers the kept w0*w1*w2 cube through shared memory
// when it is small; a larger cube is written straight to M through an
// inverse map (cube cell -> G index or -1) stored in the map buffer right
// after the ng-entry gather map.
inline bool mtxel_scatter_mode(const Axes &a, size_t csize) {
    const bool long_lines = a.n[0] >= 48 && a.n[1] >= 48 && a.n[2] >= 48 && a.n[0] % 16 == 0 &&
                            a.n[1] % 16 == 0 && a.n[2] % 16 == 0;   // four-lane FFT kernels
    return long_lines || (size_t)a.w[0] * a.w[1] * a.w[2] * csize > (size_t)64 * 1024;
}

// Whether the matrix-element kernels keep the z-pass output in the global
// scratch A: every path but the fused z+y eight-lane kernel (cubic boxes of
// N = 48 or 64), which keeps it in shared memory.
inline bool mtxel_uses_a(const Axes &a) {
    const bool four_lane = a.n[0] >= 48 && a.n[1] >= 48 && a.n[2] >= 48 && a.n[0] % 16 == 0 &&
                           a.n[1] % 16 == 0 && a.n[2] % 16 == 0;
    const bool cubic = a.n[0] == a.n[1] && a.n[1] == a.n[2];
    return !(four_lane && cubic && a.n[0] <= 64);
}

// Whether wfn_to_grid may need the y-pass scratch R: only the one-line-per-
// thread pass kernels use it (FP64 boxes that the one-kernel transform does
// not take, and non-square FP32 boxes); the eight-lane kernels (cubic 48 and
// 64) and the FP32 square-plane kernels keep it on chip.
inline bool wfn_uses_r(const Axes &a, size_t csize) {
    if (!mtxel_uses_a(a)) return false;
    const bool fp32_square = csize == 8 && a.n[1] == a.n[2] && a.n[0] < 48 && a.n[1] < 48;
    return !fp32_square;
}

// Valence bands per batch of the matrix-element kernels: their scratch
// (A, where used, + Bs per pair) stays under 1 GiB.  When the bands need more
// than one batch, a batch is a whole number of the streamed FP32 kernel's
// valence groups (5 bands at N = 24, else 4), so no batch but the last ends
// in a short group (18 bands ran as 17 + 1: groups 4,4,4,4,1 and 1).
inline int mtxel_v_batch(int nv, int nc, const Axes &a, size_t csize) {
    const size_t per_pair =
        csize * ((mtxel_uses_a(a) ? (size_t)a.n[0] * a.n[1] * a.w[2] : 0) + (size_t)a.n[0] * a.w[1] * a.w[2]);
    const size_t cap = (size_t)1 << 30;
    size_t vb = cap / (per_pair * (size_t)(nc > 0 ? nc : 1) + 1);
    if (vb < 1) vb = 1;
    if (vb >= (size_t)nv) return nv;
    const size_t group = a.n[1] == 24 ? 5 : 4;
    if (vb >= group) vb -= vb % group;
    return (int)vb;
}

// Candidate pair tiles (tv, tc) of the plane-fused FP32 kernel for this shape,
// best first by the staging heuristic; returns how many were written.
int plane_tile_candidates(int nv, int nc, const Axes &a, int *tv, int *tc, int max);

// ---- bgw_chi0_f64.cu ------------------------------------------------------
// w[j][kl*P + v*nc + c] = 2D/(D^2 + freq_j^2), D = e[k][v] - e[k'][nv + c],
// k = k0 + kl, k' = kmap[k], P = nv*nc (the bracket of the polarizability at
// w -> i w, eta -> 0) for kl < kn.  energy: [nk][nb].
cudaError_t pair_weights(const double *energy, int nb, int nv, int nc, const int *kmap, int k0,
                         int kn, const double *freq, int nfreq, double *w, cudaStream_t st);

// acc[j][g][g'] += sum_p w[j][p] conj(M[p][g]) M[p][g'] on the lower block
// triangle (FP64 throughout).  M: complex128 [P][ng].  ws: workspace of
// herk_f64_workspace_bytes for the partial sums of the split pair range.
size_t herk_f64_workspace_bytes(int P, int ng, int nfreq, int sm_count);
cudaError_t herk_f64(const void *M, int P, int ng, const double *w, int nfreq, void *acc, void *ws,
                     int sm_count, cudaStream_t st);

// out[j][g][g'] = scale * (g >= g' ? acc[j][g][g'] : conj(acc[j][g'][g])).
cudaError_t chi0_finalize(const void *acc, int ng, int nfreq, double scale, void *out,
                          cudaStream_t st);

// ---- bounds-checking build (bgw_bounds.cuh) ------------------------------
// Each translation unit's index-check status word, read and cleared; always
// 0 in the default build.
cudaError_t bounds_take_grid_f64(unsigned *word);
cudaError_t bounds_take_grid_f32(unsigned *word);
cudaError_t bounds_take_chi0(unsigned *word);
constexpr bool kBoundsBuild = BGW_BOUNDS_BUILD;

// ---- bgw_zgemm.cu (FP64, for the self-energy and BSE kernel steps) -------
// C(m, n) = [C(m, n) if accumulate] + alpha sum_k opA(m, k) wk[k] opB(k, n),
// opA(m, k) = A[m*sam + k*sak] (conjugated if conjA), opB(k, n) = B[k*sbk +
// n*sbn] (conjugated if conjB), C(m, n) at C[m*scm + n*scn]; complex128
// throughout, wk (device, may be null) a real weight per k.
cudaError_t zgemm_f64(int M, int N, int K, const void *A, long sam, long sak, bool conjA, const void *B, long sbk,
                      long sbn, bool conjB, const double *wk, void *C, long scm, long scn, double alpha_re,
                      double alpha_im, bool accumulate, cudaStream_t st);
// s[p] = Re sum_g conj(M[p][g]) Y[p][g]; t[p] = sum_g v[g] |M[p][g]|^2 (when v
// and t are given); M, Y complex128 [P][ng].
cudaError_t rowdot_f64(const void *M, const void *Y, const double *v, long P, int ng, double *s, double *t,
                       cudaStream_t st);
// out[n] = sum_{i < n_first} x[i*nn + n], summed in order of i.
cudaError_t band_sum_f64(const double *x, int n_first, int nn, double *out, cudaStream_t st);
// K[(v*nc + c)][(v'*nc + c')] = T[(c*nc + c')][(v*nv + v')], complex128.
cudaError_t bse_permute_f64(const void *T, int nv, int nc, void *K, cudaStream_t st);

}  // namespace bgw
