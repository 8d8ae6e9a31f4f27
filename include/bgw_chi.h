/*
 * bgw_chi.h -- C ABI of libbgwchi.so: the spinor RPA polarizability
 * chi0_GG'(q, i w) on one GB300 (sm_103a).
 *
 * Method (arXiv:2206.00808, Sec. II):
 *   Spinor states psi_nk = sum_alpha phi_nk,alpha |alpha>, normalised over
 *   both components together; plane-wave coefficients c_nk,alpha(G) on a
 *   wavefunction G-sphere at each k (Sec. II; plane-wave form, Sec. III.A).
 *   Matrix element, Eq. (matrix_el): multiply the real-space wavefunctions of a
 *   common spin component, Fourier transform the product, sum over alpha:
 *       M_vc(k,q,G) = N^-3 sum_r sum_alpha u*_{v,k,alpha}(r) u_{c,k+q,alpha}(r) e^{-iG.r}.
 *   Polarizability (the P_GG'(q,w) formula of Sec. II) on the imaginary axis,
 *   w -> i w, eta -> 0, no spin-degeneracy factor:
 *       chi0_GG'(q,iw) = (1/N_k) sum_k sum_v sum_c w_vc(iw) conj(M_vc(G)) M_vc(G'),
 *       w_vc(iw) = 2 D / (D^2 + w^2),  D = e_{v,k} - e_{c,k+q}   (eV, chi0 in 1/eV).
 *   Occupied bands sit at k, empty bands at k+q; the paper's own arrangement
 *   (occupied at k+q, e^{+i(q+G)r}) is the same matrix at -q with G -> -G.
 *   k + q is reduced to a grid point k' with k + q = k' + G0 (G0 integer);
 *   c_{k+q}(G) = c_{k'}(G + G0).
 *
 * Conventions
 *   - Complex numbers are interleaved (re, im) pairs: complex128 = 2 doubles,
 *     complex64 = 2 floats.  Arrays are C row-major, last index fastest.
 *   - G-vectors are Miller triples (int32[3]) in the reciprocal basis; k and q
 *     are in crystal coordinates.  Only the FFT box, the Miller spheres and
 *     the k list enter: the cell itself is not needed.
 *   - Supported FFT lengths per axis: 16, 18, 20, 24, 27, 30, 32, 36, 40, 48, 64
 *     (products of 2, 3 and 5 up to 64).
 *
 * Ownership and streams
 *   - The caller owns every pointer it passes.  The context owns its device
 *     buffers (real-space grids, scratch, accumulators) and frees them in
 *     bgw_destroy.
 *   - All device work is queued on the stream given to bgw_create (NULL = the
 *     legacy default stream) and is asynchronous unless a function says
 *     otherwise.  Host input buffers are read by copies queued on that stream:
 *     keep them alive and unchanged until the stream has passed this work (a
 *     blocking bgw_chi0_finalize, or a stream synchronize).
 *   - A context is not thread-safe: use one context per host thread.
 *
 * Errors
 *   - Negative status: the call was rejected or failed; no accumulated state
 *     changed, except BGW_E_CUDA (the device state is then unknown; destroy
 *     the context).
 *   - Positive status: a warning; the result is defined.
 *   - bgw_last_error(ctx) returns a message for the last call on ctx;
 *     bgw_last_error(NULL) for a failed bgw_create.
 */
#ifndef BGW_CHI_H
#define BGW_CHI_H

#include <stddef.h>

#if defined(__GNUC__)
#define BGW_API __attribute__((visibility("default")))
#else
#define BGW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bgw_ctx_s *bgw_ctx;

typedef enum {
    BGW_OK = 0,
    BGW_E_ARG = -1,      /* invalid argument (null pointer, range, shape) */
    BGW_E_STATE = -2,    /* call out of order (e.g. k not uploaded, q-set mismatch) */
    BGW_E_CUDA = -3,     /* a CUDA call failed; see bgw_last_error */
    BGW_E_NOMEM = -4,    /* a device allocation failed; context unchanged */
    BGW_E_GRID = -5,     /* a wavefunction sphere does not fit the FFT box */
    BGW_E_TIMEOUT = -6,  /* a device-side wait gave up (bounded spin) */
    BGW_W_ALIAS = 1      /* the box is smaller than the alias-free size for this
                            (q, k): the result is the cyclic (box) M, exactly
                            what the FFT route computes */
} bgw_status;

typedef enum {
    BGW_FP64 = 0,          /* FP64 grids, FFTs and M; the contraction to FP64
                              accuracy on tensor cores (exact BF16 digit
                              slices) or, by option, on the FP64 pipe */
    BGW_MIXED_BF16X3 = 1,  /* FP32 grids/FFTs, complex64 M, contraction as
                              split-BF16 (3 products) on tensor cores with FP32
                              accumulation per k, FP64 weights and FP64
                              reduction across k */
    BGW_MIXED_TF32X3 = 2,  /* as BGW_MIXED_BF16X3 with split-TF32 operands
                              (hi + lo to ~2^-22; 3 products, tcgen05
                              kind::tf32 at half the BF16 rate): the same
                              FP32 accumulation, twice the operand bytes */
    BGW_MIXED_TF32 = 3     /* as BGW_MIXED_BF16X3 with ONE TF32 product
                              (operands rounded to 11 significant bits):
                              ~4e-5 relative error in chi0 (3e-4 in its
                              off-diagonal part), above the 2e-5 bar of the
                              mixed forms; for estimates only */
} bgw_precision;

/* One momentum transfer with its dielectric G-sphere (the G, G' of chi0). */
typedef struct {
    double q[3];        /* crystal coordinates; k + q must land on the k list */
    int ng;             /* number of G-vectors, >= 1 */
    const int *gvec;    /* host, [ng][3] Miller indices, no duplicates */
    int nc;             /* conduction bands used for this q, 1..nc_max */
} bgw_q;

/* Library version string (static storage). */
BGW_API const char *bgw_version(void);

/*
 * Create a context for one k list and band layout.
 *   fft[3]  : FFT box N1, N2, N3 (each a supported length)
 *   nk      : number of k-points (the N_k of the 1/N_k factor)
 *   kcrys   : host, [nk][3] crystal coordinates
 *   nv      : occupied bands per k (bands 0..nv-1 of each upload)
 *   nc_max  : empty bands held per k (bands nv..nv+nc_max-1)
 *   prec    : BGW_FP64, BGW_MIXED_BF16X3, BGW_MIXED_TF32X3 or BGW_MIXED_TF32
 *   stream  : cudaStream_t to queue all work on (NULL = default stream)
 * The real-space grids, nk * (nv+nc_max) * 2 * N1*N2*N3 complex values
 * (complex128 for FP64, complex64 for mixed; fewer with BGW_OPT_GRID_SLOTS),
 * are allocated on the current device at the first bgw_wfn_upload.
 * Errors: BGW_E_ARG, BGW_E_NOMEM, BGW_E_CUDA.
 */
BGW_API bgw_status bgw_create(bgw_ctx *out, const int fft[3], int nk, const double *kcrys,
                      int nv, int nc_max, bgw_precision prec, void *stream);

/*
 * Load the spinor wavefunctions of k-point ik and transform them to the
 * real-space grid (scatter of the G-sphere into the box, inverse 3-D FFT per
 * band and spin component; Sec. II Eq. matrix_el needs u_nk,alpha(r)).
 *   ngw       : sphere size N_w(ik) >= 1
 *   gvec      : HOST, [ngw][3] Miller indices of the sphere, no duplicates
 *   coeff     : [nv+nc_max][2][ngw] complex128, band-major then spin
 *   energy_eV : [nv+nc_max] band energies (float64)
 *   on_device : 0 = coeff and energy_eV are host pointers (copied on the
 *               stream); 1 = they are device pointers on this device
 * The transform is queued before the call returns unless BGW_OPT_DEFER_K1
 * defers it to the next call that reads grids, and a host copy runs on a
 * second stream with BGW_OPT_COPY_AHEAD (see the options for what either
 * asks of the caller's buffers).
 * Errors: BGW_E_ARG (range, duplicate G), BGW_E_GRID (sphere wider than the
 * box on some axis), BGW_E_NOMEM, BGW_E_CUDA.
 */
BGW_API bgw_status bgw_wfn_upload(bgw_ctx ctx, int ik, int ngw, const int *gvec,
                          const double *coeff, const double *energy_eV, int on_device);

/*
 * Matrix elements M_vc(k,q,G) (Eq. matrix_el) for valence bands v0..v0+nv-1
 * at k = kcrys[ik] and conduction bands c0..c0+nc-1 at k+q, on q->gvec.
 *   M_dev : caller-owned DEVICE buffer [nv][nc][q->ng], complex128 for a
 *           BGW_FP64 context, complex64 for a mixed one
 * The k-point ik and its partner k' must have been uploaded.
 * Returns BGW_W_ALIAS (and the cyclic result) when the box is too small to be
 * alias-free for this pair of spheres.  Asynchronous.
 */
BGW_API bgw_status bgw_mtxel_spinor(bgw_ctx ctx, const bgw_q *q, int ik, int v0, int nv,
                            int c0, int nc, void *M_dev);

/* Discard all chi0 accumulators (the next accumulate starts a new sum). */
BGW_API bgw_status bgw_chi0_reset(bgw_ctx ctx);

/*
 * Add the contribution of k-points k_begin..k_end-1 to chi0 for each of the
 * nq q-points at the nfreq imaginary frequencies freq_eV[j] >= 0 (the P
 * formula, Sec. II).  Repeated calls with the same q-set and frequencies
 * accumulate (k-chunking); a different q-set or frequency list after a call
 * is BGW_E_STATE until bgw_chi0_reset.  The sum over k runs in index order
 * and the result does not depend on how k is split over calls as long as the
 * split points are multiples of BGW_OPT_KCHUNK.  Every k in the range and its
 * k+q partner must have been uploaded.  Asynchronous.
 */
BGW_API bgw_status bgw_chi0_accumulate(bgw_ctx ctx, int nq, const bgw_q *qs, int nfreq,
                               const double *freq_eV, int k_begin, int k_end);

/*
 * Write chi0 for q-point iq (an index into the q-set of the accumulate calls)
 * to chi0: complex128 [nfreq][ng][ng], row G, column G' fastest, scaled by
 * 1/N_k and Hermitian by construction.
 *   on_device : 1 = chi0 is a device pointer (asynchronous);
 *               0 = chi0 is a host pointer (blocks until written).
 * The accumulators are kept (call bgw_chi0_reset to start over).  A host
 * finalize also reads the context's device error word: BGW_E_TIMEOUT if a
 * bounded device-side wait gave up since the last such read (the result is
 * invalid; the context stays usable), BGW_E_ARG if the FP64 tensor-core
 * contraction met a positive pair weight.
 */
BGW_API bgw_status bgw_chi0_finalize(bgw_ctx ctx, int iq, void *chi0, int on_device);

/*
 * Progress, checkpoint and resume of a running sum.  The k sum of the
 * polarizability (the 1/N_k sum over k of Sec. II's P formula) is linear, so
 * the state between two k-blocks is the FP64 accumulators alone; the paper
 * has no counterpart of these calls (they serve long runs that must survive
 * a restart).
 *
 * bgw_chi0_progress: k_counts[nk] (host, caller-owned) receives, for every
 *   k, how many accumulate calls since the q-set was installed (first
 *   accumulate after a reset, or a resume) summed that k.  Calls captured in
 *   a graph count once, at capture; replays are not counted.
 *   BGW_E_STATE without a running sum.
 * bgw_chi0_checkpoint_bytes: *bytes = size of a checkpoint of the running
 *   sum (56-byte header, 4 bytes per k padded to 16, then per q-point 16 + 16 N_w N_G^2).
 * bgw_chi0_checkpoint: writes the running sum into the host buffer buf
 *   (caller-owned, `bytes` long): header (format tag, version, precision, a
 *   64-bit FNV-1a hash of the box, k list, band layout, precision, q-set and
 *   frequencies), the k counts, then each q-point's FP64 accumulators as
 *   complex128 [N_w][N_G][N_G] (lower block triangle meaningful).  Waits for
 *   the context stream.  BGW_E_TIMEOUT if a device-side wait of the mixed
 *   or FP64 tensor-core contraction or of the TMA-staged FP32 matrix-element
 *   kernel gave up (the sum is invalid); BGW_E_STATE during graph
 *   capture or without a running sum; BGW_E_ARG if buf is too small.
 * bgw_chi0_resume: starts a running sum from a checkpoint: the q-set and
 *   frequencies (as for accumulate) must be those the checkpoint was taken
 *   with, on a context created with the same box, k list, bands and
 *   precision (BGW_E_STATE otherwise).  Replaces any running sum; the k
 *   counts are restored; later accumulate calls add to it.  Returns when the
 *   buffer has been read.  Resuming and accumulating the remaining k-blocks
 *   with the same k-chunk gives bitwise the same chi0 as one uninterrupted
 *   run over the same blocks.
 */
BGW_API bgw_status bgw_chi0_progress(bgw_ctx ctx, int *k_counts);
BGW_API bgw_status bgw_chi0_checkpoint_bytes(bgw_ctx ctx, size_t *bytes);
BGW_API bgw_status bgw_chi0_checkpoint(bgw_ctx ctx, void *buf, size_t bytes);
BGW_API bgw_status bgw_chi0_resume(bgw_ctx ctx, int nq, const bgw_q *qs, int nfreq, const double *freq_eV,
                                   const void *buf, size_t bytes);

/*
 * Dielectric matrix inverse and screened interaction (the step after chi0:
 * Sec. II, the two equations before the P formula,
 *     eps_GG' = delta_GG' - v(q+G) P_GG',    W_GG' = eps^-1_GG' v(q+G')).
 * The P formula prints no 1/Omega; here it is carried by the bare Coulomb
 * interaction v(q+G) = 4 pi e^2 / (Omega |q+G|^2) (e^2 = 27.211386245988
 * eV bohr), so that with chi0 from bgw_chi0_finalize (eV^-1) v chi0 is
 * dimensionless and W is in eV.
 *
 * bgw_coulomb_sqrt: s[g] = sqrt(v(q + G_g)) in eV^1/2 for the Miller vectors
 *   gvec[g][3] of the sphere, cell rows avec[3][3] (bohr, row i = a_i), q in
 *   crystal coordinates; s = 0 where q + G = 0.  Host computation.
 *   BGW_E_ARG for null pointers, ng < 1 or a singular cell.
 * bgw_epsinv_workspace_bytes: device workspace bgw_epsinv needs.
 * bgw_epsinv: for each of the nfreq matrices chi[j] (device, complex128
 *   [nfreq][ng][ng], row G, column G'; overwritten) forms the Hermitian
 *   eps~ = I - S chi S (S = diag(s), s on the host) and inverts it in FP64 on
 *   the GPU (blocked Gauss-Jordan without pivoting: eps~ is positive definite
 *   when chi is Hermitian negative semidefinite, as chi0 on the imaginary axis
 *   is).  Output per mode: 0 eps~^-1; 1 W = S eps~^-1 S (eV); 2 the paper's
 *   eps^-1 = S eps~^-1 S^-1 (needs every s > 0).  work: device workspace of
 *   work_bytes >= bgw_epsinv_workspace_bytes(ng, nfreq) bytes, or NULL (the
 *   call then allocates and frees it).  Runs on `stream` and waits for it.
 *   BGW_E_ARG for bad sizes, s < 0 or non-finite, or when a pivot is not
 *   positive (the input is not negative semidefinite; the output is then
 *   invalid); BGW_E_NOMEM / BGW_E_CUDA on allocation or CUDA failure.
 *   Errors are reported by bgw_last_error(NULL).  The paper has no
 *   counterpart of the symmetrised form; it is the standard way to make the
 *   inversion Hermitian positive definite.
 */
BGW_API bgw_status bgw_coulomb_sqrt(const double *avec, const double *q, int ng, const int *gvec, double *s);
BGW_API size_t bgw_epsinv_workspace_bytes(int ng, int nfreq);
BGW_API bgw_status bgw_epsinv(int ng, int nfreq, const double *s, void *chi, int mode, void *work,
                              size_t work_bytes, void *stream);

/*
 * Spinor symmetry unfolding (Sec. "Spinor wavefunctions and symmetries": the
 * unfolding relation c_{n,k}(G) -> c~_{n,Rk}(R^-1 G) e^{-i G.tau}, the 2 x 2
 * SU(2) spin rotation, and the axis/angle extraction by Markley's version of
 * Shepperd's quaternion algorithm).  Lets a caller that stores states in the
 * irreducible wedge build the states at symmetry-equivalent k-points on the
 * GPU and upload them (bgw_wfn_upload with on_device = 1).
 *
 * bgw_symmetry_su2: for the operation rot_lat[3][3] (integers, row-major,
 *   acting on crystal coordinates of r: r' = R_lat r + tau) of the cell
 *   avec[3][3] (rows a_i, bohr): U[8] = row-major complex [2][2] (re, im)
 *   of cos(theta/2) I - i sin(theta/2) n.sigma, the spin rotation whose
 *   adjoint action turns spin vectors with the Cartesian rotation
 *   A R_lat A^-1 (its proper part -R for det = -1); axis_angle[4] = (n_x,
 *   n_y, n_z, theta), theta in [0, 2 pi].  Either output may be NULL.  Host
 *   only.  BGW_E_ARG if R_lat is not unimodular or not a rotation of this
 *   cell (R^T R != I to 1e-8).
 * bgw_unfold_spinor: coefficients at Rk from those at k.  gvec_in[ngw][3]
 *   (host) is the Miller list of the sphere at k; gvec_out[ngw][3] (host,
 *   caller-owned) receives h'_i = R_lat^-T h_i, the sphere at Rk in the same
 *   order.  c_in (device, complex128 [nb][2][ngw]) is read and c_out (device,
 *   same shape, must not alias c_in) written on `stream`:
 *       c_out[n][a][i] = e^{-2 pi i h'_i . tau} sum_b U[a][b] c_in[n][b][i],
 *   tau[3] in crystal coordinates; the common phase e^{-i Rk.tau} of all
 *   bands is dropped.  When Rk differs from the stored grid point k' by a
 *   reciprocal vector G0 (Rk = k' + G0), the caller adds G0 to gvec_out
 *   before uploading at k'.  gvec_out is written before the call returns;
 *   c_out when the stream reaches the call.  Uses a stream-ordered device
 *   allocation of 12 ngw bytes (the Miller list; the phases are formed on the
 *   device).  BGW_E_ARG on bad arguments, as for
 *   bgw_symmetry_su2, or aliasing; errors via bgw_last_error(NULL).
 */
BGW_API bgw_status bgw_symmetry_su2(const double *avec, const int *rot_lat, double *U, double *axis_angle);
BGW_API bgw_status bgw_unfold_spinor(const double *avec, const int *rot_lat, const double *tau, int nb, int ngw,
                                     const int *gvec_in, int *gvec_out, const void *c_in, void *c_out,
                                     void *stream);

/*
 * CUDA-graph capture of a sequence of calls on this context (for repeated
 * identical steps, e.g. serving the same workload).  bgw_graph_begin starts
 * capturing the context stream (which must not be the legacy default
 * stream); the calls that follow queue their device work into the graph
 * instead of running it; bgw_graph_end instantiates it (replacing any
 * earlier graph); bgw_graph_launch replays it on the stream.  A replay
 * repeats exactly the captured device work with the same buffers and
 * arguments; host-side state is what the captured calls left.  Captured
 * calls must be capture-safe: device-resident inputs (on_device = 1 or
 * pinned host buffers), a device finalize, spheres and q-sets already seen
 * (no new host-to-device metadata copies) and scratch already sized by an
 * identical uncaptured sequence; otherwise the call or bgw_graph_end fails
 * with BGW_E_CUDA and the context can be used uncaptured again.
 */
BGW_API bgw_status bgw_graph_begin(bgw_ctx ctx);
BGW_API bgw_status bgw_graph_end(bgw_ctx ctx);
BGW_API bgw_status bgw_graph_launch(bgw_ctx ctx);

/*
 * Tuning options (per context; they change speed, not the mathematics):
 *   BGW_OPT_KCHUNK       k-points contracted per launch (1..256, default 1).
 *                        The result is bitwise independent of how a k range is
 *                        split over accumulate calls when every split point is
 *                        a multiple of the k-chunk.
 *   BGW_OPT_PAIR_TILE_V  valence x conduction pair tile of the FP32 matrix-
 *   BGW_OPT_PAIR_TILE_C  element kernel (0 = automatic, else 1..16).
 *   BGW_OPT_GRID_SLOTS   real-space grids kept on the device: 0 (default) =
 *                        every k, built at upload; n < nk = k-point
 *                        streaming: uploads keep only the coefficients on the
 *                        device and accumulate builds the grids of the k-points
 *                        it needs into n slots (least recently used first),
 *                        for workloads whose grids exceed device memory.  Set
 *                        before the first upload.  In this mode a device
 *                        upload (on_device = 1) keeps a reference to the
 *                        caller's coefficient buffer instead of a copy: keep it
 *                        alive and unchanged until the k-point is uploaded
 *                        again or the context is destroyed.
 *   BGW_OPT_K1_PATH      kernels of the sphere -> real-space transform of
 *                        bgw_wfn_upload: 0 automatic (default: the one-kernel
 *                        transform where it fits, else eight lanes per line on
 *                        cubic boxes of 32, 40 (FP32), 48 and 64, else one
 *                        kernel per axis), 1 one kernel
 *                        per axis, 2 one kernel for the whole transform of a
 *                        band component where the box fits in shared memory
 *                        (else as 1), 3 eight lanes per FFT line where the box
 *                        is cubic with N = 32, 40, 48 or 64 (else automatic),
 *                        4 (FP32 cubic boxes below 48) one kernel per band
 *                        component without the shared cube, three per SM,
 *                        where it fits (else automatic).  All give the same
 *                        grids up to rounding.
 *   BGW_OPT_MTXEL_LANES  FFT lanes per line of the matrix-element kernels:
 *                        0 automatic (default: eight for cubic 48 and 64 boxes,
 *                        one elsewhere), 1 one, 8 eight where the box is cubic
 *                        with N = 32, 40, 48 or 64.  Same results up to
 *                        rounding.
 *   BGW_OPT_MTXEL_ZY     pair density + z and y passes of the FP32 matrix-
 *                        element kernels on boxes with N2 = N3 <= 40: 0
 *                        automatic (default: the streamed kernel where it
 *                        applies, even N2 <= 32, unless a pair tile is set),
 *                        1 the plane kernel with the
 *                        pair tile of BGW_OPT_PAIR_TILE_V/C (or the autotuner's),
 *                        2 the streamed kernel where it applies: a CTA keeps
 *                        a group of valence x-planes (4, or 2 where that needs
 *                        fewer passes; 5 at N = 24) in shared memory and streams
 *                        the conduction x-planes in groups (2, or 4), copying
 *                        the next group (by TMA on 32^3 boxes) while the current
 *                        one is transformed.  Same results up to rounding.
 *   BGW_OPT_DEFER_K1     0 (default): bgw_wfn_upload builds the k-point's
 *                        real-space grid before it returns (on the stream).
 *                        1: the build is deferred to the next call that reads
 *                        grids (bgw_mtxel_spinor, bgw_chi0_accumulate,
 *                        bgw_autotune) or to bgw_graph_begin, and the grids of
 *                        all deferred k-points are built together, in one
 *                        launch per 64 k-points where the box and path allow.
 *                        A device upload (on_device = 1) then keeps a reference
 *                        to the caller's coefficient buffer until that build:
 *                        keep it alive and unchanged until then; a host upload
 *                        is kept in a device copy per k-point.  No effect with
 *                        k-point streaming (BGW_OPT_GRID_SLOTS), whose grids
 *                        are built on demand already.  Same grids, bitwise.
 *   BGW_OPT_COPY_AHEAD   0 (default): a host upload (on_device = 0) copies
 *                        the coefficients on the context stream, after the
 *                        work queued there before it.  1: the copy runs on
 *                        one of four copy streams of the context (k-point ik
 *                        on stream ik mod 4, so several copy engines share the
 *                        transfer) into a device buffer of the k-point's own,
 *                        so the copies of later k-points overlap the
 *                        transforms of earlier ones; work queued
 *                        on the context stream after the call still waits for
 *                        the copy.  The host buffer must hold its data when
 *                        the call is made (the copy is not ordered after
 *                        earlier work on the context stream) and stay
 *                        unchanged until the context stream has passed the
 *                        call.  Costs one device copy of every k-point's
 *                        coefficients.  Not used during a graph capture nor
 *                        with k-point streaming.  Same grids, bitwise.
 *                        Replays through bgw_graph_launch are ordered before
 *                        later copy-ahead copies; a graph the caller captures
 *                        from the context stream itself is not tracked, so
 *                        synchronise its replays before the next upload.
 *   BGW_OPT_OVERLAP      mixed precision only.  0 (default): every step of an
 *                        accumulate runs on the context stream.  1: the
 *                        weights, operand split and contraction of each block
 *                        of matrix elements run on a second, high-priority
 *                        stream of the context while the matrix elements of
 *                        the next block are computed on the context stream
 *                        (the blocks alternate between two M buffers: twice
 *                        the M scratch).  The launches still sum into each
 *                        accumulator in the same order, so the result is
 *                        bitwise the same; work queued on the context stream
 *                        after the call waits for all of it.  Not changeable
 *                        during a graph capture.
 *   BGW_OPT_FP64_CONTRACTION  FP64 contexts only.  0 (default): the pair sum
 *                        runs on tcgen05 tensor cores from exact BF16 digit
 *                        slices (per row a power-of-two exponent, five signed
 *                        base-256 digits, the 15 products of total order <= 4
 *                        with exact integer sums; about 2e-11 relative error,
 *                        inside the FP64 path's 1e-10).  1: the FP64 FMA kernel
 *                        (FP64 pipe only, rounding of plain FP64 sums).  Not
 *                        changeable during a graph capture.
 *   BGW_OPT_TEST_FAIL_ALLOC for failure-handling tests only: when n > 0, the
 *                        n-th device allocation made by the library from now on
 *                        (by any context of the process) fails as if the device
 *                        were out of memory, so the call needing it returns
 *                        BGW_E_NOMEM; 0 switches it off.  The environment
 *                        variable BGW_FAULT=oom@n, read by bgw_create, does the
 *                        same.
 *   BGW_OPT_TEST_DROP_LOAD  for failure-handling tests only: 1, the next mixed
 *                        contractions lose one operand load on purpose, so the
 *                        kernel's bounded waits (about 2 s) expire, it frees its
 *                        resources and records an error that a host finalize
 *                        reports as BGW_E_TIMEOUT; 2, the same for the streamed
 *                        z + y kernel of FP32 32^3 boxes (whose planes arrive by
 *                        TMA): its first CTA skips one plane copy.  No fault,
 *                        trap or hang.
 */
enum { BGW_OPT_KCHUNK = 1, BGW_OPT_PAIR_TILE_V = 2, BGW_OPT_PAIR_TILE_C = 3, BGW_OPT_GRID_SLOTS = 4,
       BGW_OPT_TEST_DROP_LOAD = 5, BGW_OPT_TEST_FAIL_ALLOC = 6, BGW_OPT_K1_PATH = 7,
       BGW_OPT_MTXEL_LANES = 8, BGW_OPT_DEFER_K1 = 9, BGW_OPT_COPY_AHEAD = 10,
       BGW_OPT_OVERLAP = 11, BGW_OPT_FP64_CONTRACTION = 12, BGW_OPT_MTXEL_ZY = 13 };
BGW_API bgw_status bgw_set_option(bgw_ctx ctx, int option, long value);
BGW_API bgw_status bgw_get_option(bgw_ctx ctx, int option, long *value);

/*
 * Autotuner: times the candidate matrix-element kernels (mixed precision:
 * the streamed z + y kernel and the plane kernel's best pair tiles) and then
 * the k-chunks on k-points k_begin..k_end-1 of the given q-set and frequencies
 * (CUDA events on the context stream, one warm-up and the median of three
 * timed runs each) and sets the fastest (BGW_OPT_KCHUNK, BGW_OPT_PAIR_TILE_V/C,
 * BGW_OPT_MTXEL_ZY).
 * The running chi0 sums are not touched.  Chunks whose M block and split
 * operands would exceed 2 GiB are not tried.  cache_path (may
 * be NULL): a text file of "key|kchunk tile_v tile_c zy" lines; a hit skips
 * the timing, a miss appends the result.  Blocks until done.
 */
BGW_API bgw_status bgw_autotune(bgw_ctx ctx, int nq, const bgw_q *qs, int nfreq,
                                const double *freq_eV, int k_begin, int k_end,
                                const char *cache_path);

/*
 * Stage timing with CUDA events recorded on the context stream around each
 * launch group.  Stages: 0 sphere->grid (bgw_wfn_upload), 1 matrix elements:
 * pair density with the z and y passes, 2 pair weights, 3 contraction,
 * 4 finalize, 5 operand split (mixed path), 6 matrix elements: x pass with
 * the dielectric-sphere gather.
 *   bgw_profile(ctx, 1) clears the totals and starts recording; 0 stops.
 *   bgw_profile_read(ctx, ms, calls, kernels, n) fills the first n stages:
 *   device milliseconds, launch groups and kernels launched since the last
 *   bgw_profile(ctx, 1).  It blocks until the stream is idle.
 */
BGW_API bgw_status bgw_profile(bgw_ctx ctx, int enable);
BGW_API bgw_status bgw_profile_read(bgw_ctx ctx, double *ms, long *calls, long *kernels, int n);

/*
 * Matrix elements without any allocation (the paper has no counterpart; this
 * is a deployment variant of bgw_mtxel_spinor).
 *
 * For callers that cannot allocate device memory when they need matrix
 * elements: code whose memory pool or arena already owns the device memory,
 * plug-ins whose host forbids cudaMalloc/cudaFree after start-up (both
 * synchronise the whole device and may fail late), and loops that must not
 * block in an allocator.  It needs no context: the caller passes the
 * real-space grids and the output, and the call computes
 *     M[v][c][g] = N^-3 sum_r sum_alpha conj(Uv[v][alpha](r)) Uc[c][alpha](r) e^{-i(G_g+G0).r}
 * in FP64 with the same kernels as bgw_mtxel_spinor.
 *   fft[3] : FFT box (supported lengths as above)
 *   Uv     : DEVICE complex128 [nv][2][N1*N2*N3], u_{v,k,alpha}(r) with
 *            u(r) = sum_h c(h) e^{+2 pi i h.r/N} (unnormalised)
 *   Uc     : DEVICE complex128 [nc][2][N1*N2*N3], the bands at k' = k+q-G0,
 *            unshifted (the call applies G0)
 *   G0[3]  : host, umklapp vector with k + q = k' + G0
 *   ng, gvec : host, [ng][3] dielectric sphere, 1 <= ng <= 65536
 *   M_dev  : DEVICE complex128 [nv][nc][ng]
 *   stream : cudaStream_t (NULL = default stream); asynchronous
 * Scratch: one static device array of BGW_NOALLOC_SCRATCH_BYTES inside the
 * library, reserved on every GPU that loads it until the process exits.  The
 * call runs in blocks of whole valence bands sized to fit it; only a call
 * where one valence band with all nc conduction bands needs more (about
 * nc*N1*N2*(w3 + w2*w3/N2)*16 bytes, w the sphere's extent per axis) is
 * rejected with BGW_E_ARG; split the conduction range then.  Every call
 * shares the array and fully rewrites what it reads, so nothing needs
 * clearing, but calls that overlap on the GPU (different streams or host
 * threads racing on one device) corrupt each other: serialise them.
 * Uv, Uc and M_dev must be device (or managed) memory of the current device
 * (checked with cudaPointerGetAttributes; BGW_E_ARG otherwise); their sizes
 * cannot be checked here, so the shapes above are the caller's promise.
 * The sphere map is copied from a static pageable host array, so the call
 * waits for earlier work on `stream` before it returns, and it is rejected
 * with BGW_E_ARG while `stream` is being captured (a captured copy would read
 * that array at replay time).  The first call on a device sets up that
 * device (FFT tables and the array's device address); make it before any
 * stream capture.  Errors go to bgw_last_error(NULL), which keeps one
 * message per host thread.
 */
#define BGW_NOALLOC_SCRATCH_BYTES (64u << 20)
BGW_API bgw_status bgw_mtxel_spinor_noalloc(const int fft[3], const void *Uv, const void *Uc,
                                            int nv, int nc, const int G0[3], int ng,
                                            const int *gvec, void *M_dev, void *stream);

/*
 * Matrix elements of any two band ranges (Eq. matrix_el with free band
 * indices): M[n][m][g] = M_{n0+n, m0+m}(k, q, G_g) for bands n0..n0+nn-1 at
 * k = kcrys[ik] and m0..m0+nm-1 at k+q, band indices counted over the whole
 * upload (0..nv+nc_max-1: occupied then empty).  This is what the self-energy
 * and the BSE kernel need beyond the polarizability's occupied-empty pairs:
 * the paper's M_{n''n}(k, -q, -G) of Eqs. sigma_sx and sigma_coh equals
 * M_{n''n}(k', q, G) here with k' = k - q (first band at k - q, second at
 * k), and the spin-traced M of the BSE kernel section is the same element.
 *   q      : q->q and its sphere q->gvec (q->nc is not used)
 *   M_dev  : caller-owned DEVICE buffer [nn][nm][q->ng], complex128 (FP64
 *            context) or complex64 (mixed)
 * The k-point ik and its partner must have been uploaded.  BGW_W_ALIAS as for
 * bgw_mtxel_spinor.  Asynchronous.
 */
BGW_API bgw_status bgw_mtxel_bands(bgw_ctx ctx, const bgw_q *q, int ik, int n0, int nn, int m0, int nm,
                                   void *M_dev);

/*
 * Screened-exchange and Coulomb-hole diagonal elements of the self-energy,
 * Eqs. sigma_sx and sigma_coh, in the static limit (COHSEX: the screened
 * interaction at zero frequency, W_GG'(q) = eps^-1_GG'(q, 0) v(q+G'); the
 * frequency integral of the Coulomb-hole term then reduces to half the
 * induced interaction W - v summed over every band n'').  The contribution of
 * one q-point to bands n0..n0+nn-1 at k = kcrys[ik] is ADDED to sx[] and
 * coh[] (host, caller-owned, eV):
 *   sx[n]  += -(1/N_k) sum_{n'' occupied} sum_{G,G'} conj(M_{n''n}(G)) W_GG' M_{n''n}(G')
 *   coh[n] += (1/2)(1/N_k) sum_{n'' all bands} sum_{G,G'} conj(M_{n''n}(G)) (W_GG' - delta_GG' v(q+G)) M_{n''n}(G')
 * with M_{n''n}(G) = M_{n''n}(k - q, q, G) (bgw_mtxel_bands at the k-point
 * k - q, which must be on the k list and uploaded, as must k).  Occupied
 * bands are 0..nv-1; "all bands" are the nv + nc_max bands of the upload.
 * Summing the calls over every q of the k-grid gives the Brillouin-zone
 * average (the 1/N_k; the paper prints the q sum without it).
 *   W_dev : DEVICE complex128 [q->ng][q->ng], row G, column G' (eV), e.g.
 *           bgw_epsinv mode 1 applied to the static chi0 of this q
 *   vq    : host [q->ng], v(q+G) in eV (the square of bgw_coulomb_sqrt)
 * Needs a BGW_FP64 context; uses context-owned scratch of about
 * 32 (nv+nc_max) nn q->ng bytes.  Waits for the stream (the sums are read
 * back); not capturable (BGW_E_STATE during a capture).
 */
BGW_API bgw_status bgw_sigma_cohsex(bgw_ctx ctx, const bgw_q *q, int ik, int n0, int nn, const void *W_dev,
                                    const double *vq, double *sx, double *coh);

/*
 * One (k_i, k_j) block of the exchange and direct BSE kernels in the
 * Tamm-Dancoff approximation (the K^X and K^D integrals of the BSE section),
 * for valence bands v0..v0+nv-1 and conduction bands c0..c0+nc-1 (counted
 * within the occupied and the empty bands) at both k-points; rows are (v c)
 * at k_i = kcrys[ik], columns (v' c') at k_j = kcrys[jk], index v*nc + c:
 *   KX[(v c)][(v' c')] =  (1/N_k) sum_G v(G) M_vc(k_i, 0, G) conj(M_v'c'(k_j, 0, G))
 *   KD[(v c)][(v' c')] = -(1/N_k) sum_{G,G'} conj(M_cc'(k_i, q, G)) W_GG'(q) M_vv'(k_i, q, G')
 * with q = k_j - k_i, M as in bgw_mtxel_bands (spin traced) and W the static
 * screened interaction of q.  The printed kernels carry -i and +i from the
 * time integration; the factor i that turns them into energies gives the
 * usual repulsive exchange and attractive direct terms above.
 *   q0, v0_coul : the exchange sphere at q = 0 (q0->q a reciprocal lattice
 *                 vector) and v(G) there, host [q0->ng] eV (0 where G = 0:
 *                 the long-range term is left out, as bgw_coulomb_sqrt does)
 *   qd, W_dev   : q = k_j - k_i (mod a reciprocal vector) with its sphere, and
 *                 DEVICE complex128 W [qd->ng][qd->ng] (eV)
 *   KX_dev, KD_dev : caller-owned DEVICE complex128 [nv*nc][nv*nc]; either
 *                 may be NULL to skip that kernel
 * Needs a BGW_FP64 context with both k-points uploaded; context-owned
 * scratch.  Asynchronous (the host v0_coul is read before the call returns).
 */
BGW_API bgw_status bgw_bse_kernel(bgw_ctx ctx, int ik, int jk, const bgw_q *q0, const double *v0_coul,
                                  const bgw_q *qd, const void *W_dev, int v0, int nv, int c0, int nc,
                                  void *KX_dev, void *KD_dev);

/*
 * Index checks (a development aid; the paper has no counterpart).  The
 * library built with -DBGW_BOUNDS=1 (libbgwchi_bounds.so) tests every index
 * its kernels read from a device map against the range it must lie in: the
 * cube, inverse, gather and scatter maps of the FFT passes and the k + q map
 * of the pair weights.  An index out of range skips that access and sets bit
 * `site` in a device status word (0 cube map, 1 inverse map, 2 gather map,
 * 3 scatter map, 4 k + q map); nothing traps.  bgw_bounds_check waits for the
 * device, returns the OR of the words in *word and clears them.  In the
 * default build it returns BGW_E_STATE with *word = 0.  Errors go to
 * bgw_last_error(NULL).
 */
BGW_API bgw_status bgw_bounds_check(unsigned *word);

/* Release every device buffer of the context (synchronizes its stream). */
BGW_API void bgw_destroy(bgw_ctx ctx);

/* Message of the last failing call on ctx (NULL ctx: the last failed create or
   context-free call of the calling host thread). */
BGW_API const char *bgw_last_error(bgw_ctx ctx);

#ifdef __cplusplus
}
#endif
#endif /* BGW_CHI_H */
