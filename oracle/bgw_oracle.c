/*
 * CPU FP64 oracle for the spinor RPA polarizability chi0_GG'(q, i omega).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this file's library.  It shares no
 * code, header, table or helper with the CUDA path; it is plain C99 with
 * OpenMP, no FFT and no BLAS, written to be checked against the paper by eye.
 *
 * What it computes (arXiv:2206.00808, Sec. II):
 *
 *  Matrix element, Eq. (matrix_el) and the M_nn' definition above it.  With
 *  the band at k written as v and the band at k+q as c, and plane-wave
 *  coefficients u_{n,k,alpha}(r) = sum_h c_{n,k,alpha}(h) e^{2 pi i h.r/N}
 *  (Sec. III.A, the plane-wave form of a Bloch function), the FFT route
 *      M_vc(k,q,G) = N^-3 sum_r sum_alpha u*_{v,k,alpha}(r) u_{c,k+q,alpha}(r) e^{-2 pi i G.r/N}
 *  is identical, for every box, to the cyclic convolution in G-space
 *      M_vc(k,q,G) = sum_alpha sum_{h1 in sphere(k)} conj(c_{v,k,alpha}(h1)) C_{c,k+q,alpha}[(h1+G) mod N]
 *  where C is the coefficient array of the band at k+q scattered (additively)
 *  onto the N1 x N2 x N3 box.  This oracle evaluates the second form directly.
 *  The band at k+q is stored at the grid point k' = k + q - G0 (Bloch
 *  periodicity, c_{k+q}(h) = c_{k'}(h + G0)), so a coefficient of k' at Miller
 *  index m lands at box index (m - G0) mod N.
 *
 *  Polarizability, the unnumbered P_GG'(q, omega) formula of Sec. II,
 *  evaluated on the imaginary axis (omega -> i omega, eta -> 0):
 *      chi0_GG'(q, i w) = (1/N_k) sum_k sum_v sum_c w_vc(i w) conj(M_vc(G)) M_vc(G')
 *      w_vc(i w) = 1/(D - i w) + 1/(D + i w) = 2 D / (D^2 + w^2),  D = e_{v,k} - e_{c,k+q}
 *  in eV^-1, with no spin-degeneracy factor: spinor bands carry both spin
 *  components, and the sum over alpha inside M is the only spin sum
 *  (Sec. II, the paragraph after Eq. matrix_el).
 *
 * Summation order is fixed (k outer in the caller, then v, c), and the
 * parallel loops split only independent output entries, so the result does
 * not depend on the thread count.
 *
 *  Dielectric matrix and screened interaction (Sec. II, the two equations
 *  before the P formula): eps = delta - v(q+G) P, W = eps^-1 v(q+G'), with
 *  eps^-1 by a plain LU (oracle_coulomb, oracle_epsinv at the end of this
 *  file).
 *
 * Parity status: every function here is pinned by the CPU tests (brute-force
 * real-space sums, numpy.fft, closed forms and invariants); none is unpinned.
 */
#include <stdlib.h>
#include <string.h>

static long wrap_index(long h, long n)
{
    long r = h % n;
    return r < 0 ? r + n : r;
}

static long box_index(const int *box, long h0, long h1, long h2)
{
    return (wrap_index(h0, box[0]) * box[1] + wrap_index(h1, box[1])) * box[2]
           + wrap_index(h2, box[2]);
}

/*
 * Matrix elements for one k: M[v][c][g] (interleaved complex128).
 *   box      : N1, N2, N3
 *   gv, cv   : sphere at k (ngw_v Miller triples) and valence coefficients
 *              [nv][2][ngw_v] interleaved complex128
 *   gc, cc   : sphere at k' and conduction coefficients [nc][2][ngw_c]
 *   G0       : umklapp vector, k + q = k' + G0
 *   geps     : dielectric sphere, ng Miller triples
 * Returns 0, or -1 if a scratch allocation failed.
 */
int oracle_mtxel(const int *box,
                 int ngw_v, const int *gv, int nv, const double *cv,
                 int ngw_c, const int *gc, int nc, const double *cc,
                 const int *G0, int ng, const int *geps, double *M)
{
    const long nbox = (long)box[0] * box[1] * box[2];
    int failed = 0;

#pragma omp parallel
    {
        double *cbox = (double *)malloc(sizeof(double) * 2 * 2 * nbox);
        if (!cbox) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < nc; ++c) {
            if (!cbox) continue;
            /* C_{c,k+q,alpha} on the box: coefficient of k' at m sits at m - G0. */
            memset(cbox, 0, sizeof(double) * 2 * 2 * nbox);
            for (int a = 0; a < 2; ++a) {
                const double *src = cc + 2 * ((long)(c * 2 + a) * ngw_c);
                double *dst = cbox + 2 * (long)a * nbox;
                for (int i = 0; i < ngw_c; ++i) {
                    long idx = box_index(box, (long)gc[3 * i] - G0[0],
                                         (long)gc[3 * i + 1] - G0[1],
                                         (long)gc[3 * i + 2] - G0[2]);
                    dst[2 * idx] += src[2 * i];
                    dst[2 * idx + 1] += src[2 * i + 1];
                }
            }
            for (int v = 0; v < nv; ++v) {
                for (int g = 0; g < ng; ++g) {
                    double re = 0.0, im = 0.0;
                    for (int a = 0; a < 2; ++a) {
                        const double *vv = cv + 2 * ((long)(v * 2 + a) * ngw_v);
                        const double *cb = cbox + 2 * (long)a * nbox;
                        for (int i = 0; i < ngw_v; ++i) {
                            long idx = box_index(box, (long)gv[3 * i] + geps[3 * g],
                                                 (long)gv[3 * i + 1] + geps[3 * g + 1],
                                                 (long)gv[3 * i + 2] + geps[3 * g + 2]);
                            /* conj(a) * b */
                            double ar = vv[2 * i], ai = vv[2 * i + 1];
                            double br = cb[2 * idx], bi = cb[2 * idx + 1];
                            re += ar * br + ai * bi;
                            im += ar * bi - ai * br;
                        }
                    }
                    double *out = M + 2 * (((long)v * nc + c) * ng + g);
                    out[0] = re;
                    out[1] = im;
                }
            }
        }
        free(cbox);
    }
    return failed ? -1 : 0;
}

/*
 * Weight of one pair on the imaginary axis: the bracket of the P formula with
 * omega -> i w and eta -> 0, 1/(D - i w) + 1/(D + i w) = 2 D / (D^2 + w^2).
 */
double oracle_weight(double e_v, double e_c, double w)
{
    double d = e_v - e_c;
    return 2.0 * d / (d * d + w * w);
}

/*
 * chi[j][G][G'] += sum_{v,c} w_vc(i w_j) conj(M[v][c][G]) M[v][c][G'] for one k,
 * all G, G' (the full matrix, no symmetry used).  e_v: [nv] energies at k,
 * e_c: [nc] energies at k+q, freq: [nfreq] eV.  The 1/N_k factor is applied by
 * oracle_scale once all k are in.
 */
void oracle_chi0_accumulate(int nv, int nc, int ng, const double *M,
                            const double *e_v, const double *e_c,
                            int nfreq, const double *freq, double *chi)
{
    for (int j = 0; j < nfreq; ++j) {
        double *cj = chi + 2 * (long)j * ng * ng;
#pragma omp parallel for schedule(static)
        for (int g = 0; g < ng; ++g) {
            for (int v = 0; v < nv; ++v) {
                for (int c = 0; c < nc; ++c) {
                    double w = oracle_weight(e_v[v], e_c[c], freq[j]);
                    const double *mp = M + 2 * (((long)v * nc + c) * ng);
                    double ar = mp[2 * g], ai = mp[2 * g + 1];
                    double *row = cj + 2 * (long)g * ng;
                    for (int h = 0; h < ng; ++h) {
                        double br = mp[2 * h], bi = mp[2 * h + 1];
                        row[2 * h] += w * (ar * br + ai * bi);
                        row[2 * h + 1] += w * (ar * bi - ai * br);
                    }
                }
            }
        }
    }
}

/* x[i] *= s for n doubles (applies the 1/N_k of the P formula). */
void oracle_scale(long n, double s, double *x)
{
    for (long i = 0; i < n; ++i) x[i] *= s;
}

/*
 * ---------------------------------------------------------------------------
 * Dielectric matrix, its inverse and the screened interaction (Sec. II, the
 * two equations before the P formula):
 *      eps_GG'(q, w) = delta_GG' - v(q+G) P_GG'(q, w)
 *      W_GG'(q, w)   = eps^-1_GG'(q, w) v(q+G')
 * with the bare Coulomb interaction v(q+G) = 4 pi e^2 / (Omega |q+G|^2).
 * The P formula as printed has no 1/Omega; it is carried here by v, so that
 * with chi0 in eV^-1 and e^2 = 1 Hartree bohr = 27.211386245988 eV bohr the
 * product v chi0 is dimensionless and W is in eV.  v = 0 where q + G = 0 (the
 * head at q = 0 is not defined by these equations; eps is then the identity
 * in that row).
 * ---------------------------------------------------------------------------
 */
#define ORACLE_E2_EV_BOHR 27.211386245988
#define ORACLE_PI 3.14159265358979323846

/*
 * v[g] = 4 pi e^2 / (Omega |(q + h_g) B|^2) in eV for the Miller vectors
 * gvec[g] = h_g, with avec the rows a_1, a_2, a_3 (bohr), B = 2 pi A^-T and
 * Omega = |det A|.
 */
void oracle_coulomb(const double *avec, const double *q, int ng, const int *gvec, double *v)
{
    const double *a0 = avec, *a1 = avec + 3, *a2 = avec + 6;
    /* b_i = 2 pi (a_j x a_k) / (a_0 . (a_1 x a_2)) */
    double c12[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
    double c20[3] = {a2[1] * a0[2] - a2[2] * a0[1], a2[2] * a0[0] - a2[0] * a0[2], a2[0] * a0[1] - a2[1] * a0[0]};
    double c01[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]};
    double det = a0[0] * c12[0] + a0[1] * c12[1] + a0[2] * c12[2];
    double omega = det < 0 ? -det : det;
    double b[3][3];
    for (int x = 0; x < 3; ++x) {
        b[0][x] = 2.0 * ORACLE_PI * c12[x] / det;
        b[1][x] = 2.0 * ORACLE_PI * c20[x] / det;
        b[2][x] = 2.0 * ORACLE_PI * c01[x] / det;
    }
    for (int g = 0; g < ng; ++g) {
        double k[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            double c = q[i] + gvec[3 * g + i];
            for (int x = 0; x < 3; ++x) k[x] += c * b[i][x];
        }
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        v[g] = k2 > 1e-24 ? 4.0 * ORACLE_PI * ORACLE_E2_EV_BOHR / (omega * k2) : 0.0;
    }
}

/*
 * For each frequency j: eps = I - diag(v) chi[j] (as printed), eps^-1 by LU
 * with partial pivoting (Doolittle, column by column of the identity), and
 * W = eps^-1 diag(v).  chi, epsinv, W: complex128 [nfreq][ng][ng] row-major
 * (G row, G' column).  Returns -1 on a zero pivot or allocation failure.
 */
int oracle_epsinv(int ng, int nfreq, const double *chi, const double *v, double *epsinv, double *W)
{
    long n = ng;
    double *a = (double *)malloc(sizeof(double) * 2 * n * n);
    int *piv = (int *)malloc(sizeof(int) * n);
    if (!a || !piv) {
        free(a);
        free(piv);
        return -1;
    }
    int failed = 0;
    for (int j = 0; j < nfreq && !failed; ++j) {
        const double *cj = chi + 2 * (long)j * n * n;
        double *ej = epsinv + 2 * (long)j * n * n;
        double *wj = W + 2 * (long)j * n * n;
        /* eps = delta - v(q+G) P */
        for (long r = 0; r < n; ++r)
            for (long c = 0; c < n; ++c) {
                a[2 * (r * n + c)] = (r == c ? 1.0 : 0.0) - v[r] * cj[2 * (r * n + c)];
                a[2 * (r * n + c) + 1] = -v[r] * cj[2 * (r * n + c) + 1];
            }
        /* LU with partial pivoting: P a = L U, L unit lower, stored in place */
        for (long k = 0; k < n; ++k) {
            long p = k;
            double best = -1.0;
            for (long r = k; r < n; ++r) {
                double m = a[2 * (r * n + k)] * a[2 * (r * n + k)] + a[2 * (r * n + k) + 1] * a[2 * (r * n + k) + 1];
                if (m > best) {
                    best = m;
                    p = r;
                }
            }
            piv[k] = (int)p;
            if (best <= 0.0) {
                failed = 1;
                break;
            }
            if (p != k)
                for (long c = 0; c < 2 * n; ++c) {
                    double t = a[2 * k * n + c];
                    a[2 * k * n + c] = a[2 * p * n + c];
                    a[2 * p * n + c] = t;
                }
            double pr = a[2 * (k * n + k)], pi = a[2 * (k * n + k) + 1];
            double den = pr * pr + pi * pi;
            for (long r = k + 1; r < n; ++r) {
                double xr = a[2 * (r * n + k)], xi = a[2 * (r * n + k) + 1];
                double lr = (xr * pr + xi * pi) / den, li = (xi * pr - xr * pi) / den;   /* x / pivot */
                a[2 * (r * n + k)] = lr;
                a[2 * (r * n + k) + 1] = li;
                for (long c = k + 1; c < n; ++c) {
                    double ur = a[2 * (k * n + c)], ui = a[2 * (k * n + c) + 1];
                    a[2 * (r * n + c)] -= lr * ur - li * ui;
                    a[2 * (r * n + c) + 1] -= lr * ui + li * ur;
                }
            }
        }
        if (failed) break;
        /* columns of eps^-1: solve L U x = P e_c */
#pragma omp parallel for schedule(static)
        for (long c = 0; c < n; ++c) {
            double *x = (double *)malloc(sizeof(double) * 2 * n);
            if (!x) {
#pragma omp atomic write
                failed = 1;
                continue;
            }
            for (long r = 0; r < n; ++r) x[2 * r] = x[2 * r + 1] = 0.0;
            /* permuted unit vector: apply the row swaps in order */
            double *e = (double *)calloc(2 * n, sizeof(double));
            if (!e) {
                free(x);
#pragma omp atomic write
                failed = 1;
                continue;
            }
            e[2 * c] = 1.0;
            for (long k = 0; k < n; ++k) {
                long p = piv[k];
                if (p != k) {
                    double t0 = e[2 * k], t1 = e[2 * k + 1];
                    e[2 * k] = e[2 * p];
                    e[2 * k + 1] = e[2 * p + 1];
                    e[2 * p] = t0;
                    e[2 * p + 1] = t1;
                }
            }
            /* forward: L y = e */
            for (long r = 0; r < n; ++r) {
                double sr = e[2 * r], si = e[2 * r + 1];
                for (long k = 0; k < r; ++k) {
                    double lr = a[2 * (r * n + k)], li = a[2 * (r * n + k) + 1];
                    sr -= lr * x[2 * k] - li * x[2 * k + 1];
                    si -= lr * x[2 * k + 1] + li * x[2 * k];
                }
                x[2 * r] = sr;
                x[2 * r + 1] = si;
            }
            /* backward: U x = y */
            for (long r = n - 1; r >= 0; --r) {
                double sr = x[2 * r], si = x[2 * r + 1];
                for (long k = r + 1; k < n; ++k) {
                    double ur = a[2 * (r * n + k)], ui = a[2 * (r * n + k) + 1];
                    sr -= ur * x[2 * k] - ui * x[2 * k + 1];
                    si -= ur * x[2 * k + 1] + ui * x[2 * k];
                }
                double pr = a[2 * (r * n + r)], pi = a[2 * (r * n + r) + 1];
                double den = pr * pr + pi * pi;
                x[2 * r] = (sr * pr + si * pi) / den;
                x[2 * r + 1] = (si * pr - sr * pi) / den;
            }
            for (long r = 0; r < n; ++r) {
                ej[2 * (r * n + c)] = x[2 * r];
                ej[2 * (r * n + c) + 1] = x[2 * r + 1];
            }
            free(e);
            free(x);
        }
        /* W = eps^-1 v(q+G') */
        for (long r = 0; r < n; ++r)
            for (long c = 0; c < n; ++c) {
                wj[2 * (r * n + c)] = ej[2 * (r * n + c)] * v[c];
                wj[2 * (r * n + c) + 1] = ej[2 * (r * n + c) + 1] * v[c];
            }
    }
    free(a);
    free(piv);
    return failed ? -1 : 0;
}

/*
 * ---------------------------------------------------------------------------
 * Self-energy terms (Sec. II, Eqs. sigma_sx and sigma_coh) in the static
 * limit, and the BSE kernels (the K^X and K^D integrals of the BSE section).
 * Both are sums of spin-traced matrix elements, computed by oracle_mtxel with
 * free band ranges, against an interaction matrix.
 * ---------------------------------------------------------------------------
 */

/*
 * out[p] = Re sum_G sum_G' conj(M[p][G]) A[G][G'] M[p][G'] for np rows M[p]
 * of ng complex values and a complex ng x ng matrix A (row G, column G').
 * For a Hermitian A the sum is real; its real part is returned.
 */
void oracle_quad(long np, int ng, const double *M, const double *A, double *out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < np; ++p) {
        const double *m = M + 2 * p * ng;
        double sr = 0.0;
        for (int g = 0; g < ng; ++g) {
            /* y = sum_G' A[g][G'] M[G'] */
            double yr = 0.0, yi = 0.0;
            const double *row = A + 2 * (long)g * ng;
            for (int h = 0; h < ng; ++h) {
                yr += row[2 * h] * m[2 * h] - row[2 * h + 1] * m[2 * h + 1];
                yi += row[2 * h] * m[2 * h + 1] + row[2 * h + 1] * m[2 * h];
            }
            /* conj(M[g]) y, real part */
            sr += m[2 * g] * yr + m[2 * g + 1] * yi;
        }
        out[p] = sr;
    }
}

/*
 * Exchange kernel block:
 *   K[(v c)][(v' c')] = scale sum_G v[G] Mi[v][c][G] conj(Mj[v'][c'][G])
 * Mi, Mj: [nv][nc][ng] complex (M_vc at k_i and at k_j, q = 0), v: [ng].
 */
void oracle_bse_exchange(int nv, int nc, int ng, const double *Mi, const double *Mj, const double *v,
                         double scale, double *K)
{
    const long P = (long)nv * nc;
#pragma omp parallel for schedule(static)
    for (long I = 0; I < P; ++I) {
        const double *a = Mi + 2 * I * ng;
        for (long J = 0; J < P; ++J) {
            const double *b = Mj + 2 * J * ng;
            double sr = 0.0, si = 0.0;
            for (int g = 0; g < ng; ++g) {
                /* a * conj(b) */
                sr += v[g] * (a[2 * g] * b[2 * g] + a[2 * g + 1] * b[2 * g + 1]);
                si += v[g] * (a[2 * g + 1] * b[2 * g] - a[2 * g] * b[2 * g + 1]);
            }
            K[2 * (I * P + J)] = scale * sr;
            K[2 * (I * P + J) + 1] = scale * si;
        }
    }
}

/*
 * Direct kernel block:
 *   K[(v c)][(v' c')] = -scale sum_G sum_G' conj(Mcc[c][c'][G]) W[G][G'] Mvv[v][v'][G']
 * Mcc: [nc][nc][ng] (M_cc' with c at k_i, c' at k_j), Mvv: [nv][nv][ng],
 * W: [ng][ng] complex.
 */
void oracle_bse_direct(int nv, int nc, int ng, const double *Mcc, const double *Mvv, const double *W,
                       double scale, double *K)
{
    const long P = (long)nv * nc;
#pragma omp parallel for schedule(static)
    for (long I = 0; I < P; ++I) {
        const int v = (int)(I / nc), c = (int)(I % nc);
        for (long J = 0; J < P; ++J) {
            const int v2 = (int)(J / nc), c2 = (int)(J % nc);
            const double *a = Mcc + 2 * (((long)c * nc + c2) * ng);
            const double *b = Mvv + 2 * (((long)v * nv + v2) * ng);
            double sr = 0.0, si = 0.0;
            for (int g = 0; g < ng; ++g) {
                double yr = 0.0, yi = 0.0;   /* sum_G' W[g][G'] b[G'] */
                const double *row = W + 2 * (long)g * ng;
                for (int h = 0; h < ng; ++h) {
                    yr += row[2 * h] * b[2 * h] - row[2 * h + 1] * b[2 * h + 1];
                    yi += row[2 * h] * b[2 * h + 1] + row[2 * h + 1] * b[2 * h];
                }
                /* conj(a[g]) y */
                sr += a[2 * g] * yr + a[2 * g + 1] * yi;
                si += a[2 * g] * yi - a[2 * g + 1] * yr;
            }
            K[2 * (I * P + J)] = -scale * sr;
            K[2 * (I * P + J) + 1] = -scale * si;
        }
    }
}
