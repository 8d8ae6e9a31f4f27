"""CPU FP64 oracle for the spinor polarizability (TEST INFRASTRUCTURE ONLY).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path (the CUDA library and
its binding) never does.  The arithmetic lives in `bgw_oracle.c` (plain C,
FP64, direct G-space convolution, no FFT); this module compiles it with gcc,
loads it with ctypes and walks k in a fixed order.

What the functions follow (arXiv:2206.00808, Sec. II):
  * `mtxel`      -- M_vc(k,q,G), Eq. (matrix_el) as a cyclic convolution;
  * `weight`     -- the P-formula bracket at omega -> i omega, eta -> 0;
  * `chi0`       -- the P formula: (1/N_k) sum_k sum_v sum_c w conj(M) M,
                    no spin-degeneracy factor;
  * `umklapp`    -- k + q = k' + G0 with k' on the grid (Bloch periodicity;
                    the paper is silent on it);
  * `coulomb`    -- v(q+G) = 4 pi e^2 / (Omega |q+G|^2) in eV;
  * `epsinv`     -- eps = delta - v(q+G) P and W = eps^-1 v(q+G') (the two
                    equations before the P formula), eps^-1 by a plain LU;
  * `sigma_cohsex` -- the screened-exchange and Coulomb-hole diagonal
                    elements, Eqs. sigma_sx and sigma_coh, with the static W;
  * `bse_kernel` -- the exchange and direct BSE kernel blocks (the K^X and
                    K^D integrals of the BSE section, spin traced).
All are pinned by tests/test_oracle_pins.py; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile bgw_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_mtxel.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P,
                                         ctypes.c_int, P, ctypes.c_int, P, P,
                                         ctypes.c_int, P, P]
            lib.oracle_mtxel.restype = ctypes.c_int
            lib.oracle_weight.argtypes = [ctypes.c_double] * 3
            lib.oracle_weight.restype = ctypes.c_double
            lib.oracle_chi0_accumulate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                                   P, P, ctypes.c_int, P, P]
            lib.oracle_chi0_accumulate.restype = None
            lib.oracle_scale.argtypes = [ctypes.c_long, ctypes.c_double, P]
            lib.oracle_scale.restype = None
            lib.oracle_coulomb.argtypes = [P, P, ctypes.c_int, P, P]
            lib.oracle_coulomb.restype = None
            lib.oracle_epsinv.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P]
            lib.oracle_epsinv.restype = ctypes.c_int
            lib.oracle_quad.argtypes = [ctypes.c_long, ctypes.c_int, P, P, P]
            lib.oracle_quad.restype = None
            lib.oracle_bse_exchange.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P,
                                                ctypes.c_double, P]
            lib.oracle_bse_exchange.restype = None
            lib.oracle_bse_direct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P,
                                              ctypes.c_double, P]
            lib.oracle_bse_direct.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mtxel(box, gv, cv, gc, cc, G0, geps) -> np.ndarray:
    """M[v][c][g] (complex128) for valence coefficients cv [nv][2][ngw_v] on
    sphere gv at k and conduction coefficients cc [nc][2][ngw_c] on sphere gc
    at k' = k + q - G0; geps is the dielectric sphere (ng, 3)."""
    lib = _load()
    box, gv, gc, G0, geps = _i32(box), _i32(gv), _i32(gc), _i32(G0), _i32(geps)
    cv, cc = _c128(cv), _c128(cc)
    nv, nc, ng = cv.shape[0], cc.shape[0], geps.shape[0]
    M = np.zeros((nv, nc, ng), dtype=np.complex128)
    rc = lib.oracle_mtxel(_ptr(box), gv.shape[0], _ptr(gv), nv, _ptr(cv),
                          gc.shape[0], _ptr(gc), nc, _ptr(cc), _ptr(G0), ng, _ptr(geps), _ptr(M))
    if rc != 0:
        raise MemoryError("oracle_mtxel: scratch allocation failed")
    return M


def weight(e_v: float, e_c: float, w: float) -> float:
    """2 D / (D^2 + w^2), D = e_v - e_c (eV^-1)."""
    return _load().oracle_weight(float(e_v), float(e_c), float(w))


def chi0_accumulate(M, e_v, e_c, freq, chi) -> None:
    """chi[j] += sum_{v,c} w_vc(i w_j) conj(M[v,c,:])^T M[v,c,:] (in place)."""
    lib = _load()
    M, e_v, e_c, freq = _c128(M), _f64(e_v), _f64(e_c), _f64(freq)
    assert chi.dtype == np.complex128 and chi.flags.c_contiguous
    nv, nc, ng = M.shape
    assert chi.shape == (len(freq), ng, ng)
    lib.oracle_chi0_accumulate(nv, nc, ng, _ptr(M), _ptr(e_v), _ptr(e_c), len(freq),
                               _ptr(freq), _ptr(chi))


def umklapp(kcrys: np.ndarray, ik: int, q) -> tuple[int, np.ndarray]:
    """(k', G0) with kcrys[ik] + q = kcrys[k'] + G0, G0 integer."""
    target = np.asarray(kcrys[ik], float) + np.asarray(q, float)
    for kp in range(len(kcrys)):
        d = target - kcrys[kp]
        if np.all(np.abs(d - np.round(d)) < 1e-8):
            return kp, np.round(d).astype(np.int32)
    raise ValueError(f"k + q is not on the k-grid (k index {ik}, q = {q})")


def chi0(problem, iq: int = 0, k_indices=None, nc=None, g_indices=None,
         contraction: str = "loop") -> np.ndarray:
    """chi0[j][G][G'] (complex128, eV^-1) of a synthetic Problem for q-point iq.

    Sums k over `k_indices` (default: every k, in index order) and always
    divides by the full N_k, so a subset gives that subset's share of the sum.
    g_indices: only the G-vectors geps[g_indices] (rows and columns of that
    block of chi0; each M(G) is an independent convolution sum).
    contraction: "loop" (the C triple loop) or "matmul" (the same sum as the
    library product A^H diag(w_j) A with A = M as a pairs x G matrix, for the
    large cases; pinned against the loop on the CPU).
    """
    lib = _load()
    q, geps, ncq = problem.qs[iq]
    if nc is not None:
        ncq = nc
    if g_indices is not None:
        geps = np.asarray(geps)[np.asarray(g_indices)]
    nv = problem.nv
    ng = len(geps)
    freq = _f64(problem.freq)
    chi = np.zeros((len(freq), ng, ng), dtype=np.complex128)
    ks = range(problem.nk) if k_indices is None else k_indices
    for ik in ks:
        kp, G0 = umklapp(problem.kcrys, ik, q)
        M = mtxel(problem.box, problem.gvec[ik], problem.coeff[ik][:nv],
                  problem.gvec[kp], problem.coeff[kp][nv:nv + ncq], G0, geps)
        e_v, e_c = problem.energy[ik][:nv], problem.energy[kp][nv:nv + ncq]
        if contraction == "loop":
            chi0_accumulate(M, e_v, e_c, freq, chi)
        else:
            A = M.reshape(nv * ncq, ng)
            w = np.array([[weight(a, b, f) for a in e_v for b in e_c] for f in freq])
            for j in range(len(freq)):
                chi[j] += (A.conj().T * w[j][None, :]) @ A
    flat = chi.reshape(-1).view(np.float64)
    lib.oracle_scale(flat.size, 1.0 / problem.nk, _ptr(flat))
    return chi


def coulomb(avec, q, gvec) -> np.ndarray:
    """v(q+G) = 4 pi e^2 / (Omega |q+G|^2) in eV for Miller vectors gvec
    (ng, 3), cell rows avec (bohr); 0 where q + G = 0."""
    lib = _load()
    a, qq, g = _f64(np.asarray(avec).reshape(9)), _f64(q), _i32(gvec)
    v = np.zeros(len(g), dtype=np.float64)
    lib.oracle_coulomb(_ptr(a), _ptr(qq), len(g), _ptr(g), _ptr(v))
    return v


def epsinv(chi, v) -> tuple[np.ndarray, np.ndarray]:
    """(eps^-1, W) per frequency for chi [nfreq][ng][ng] (eV^-1) and v [ng] (eV):
    eps = delta - v(q+G) chi, W = eps^-1 v(q+G')."""
    lib = _load()
    chi = _c128(chi)
    if chi.ndim == 2:
        chi = chi[None]
    nf, ng, _ = chi.shape
    vv = _f64(v)
    e = np.zeros_like(chi)
    w = np.zeros_like(chi)
    if lib.oracle_epsinv(ng, nf, _ptr(chi), _ptr(vv), _ptr(e), _ptr(w)) != 0:
        raise ArithmeticError("oracle_epsinv: singular matrix or allocation failure")
    return e, w


def quad(M, A) -> np.ndarray:
    """Re sum_GG' conj(M[p][G]) A[G][G'] M[p][G'] for every row p of M (np, ng)."""
    lib = _load()
    M, A = _c128(M), _c128(A)
    np_, ng = M.shape
    out = np.zeros(np_, dtype=np.float64)
    lib.oracle_quad(np_, ng, _ptr(M), _ptr(A), _ptr(out))
    return out


def k_minus_q(kcrys, ik, q) -> int:
    """Grid index j with kcrys[j] + q = kcrys[ik] + G0 (G0 integer)."""
    for j in range(len(kcrys)):
        kp, _ = umklapp_or_none(kcrys, j, q)
        if kp == ik:
            return j
    raise ValueError(f"k - q is not on the k-grid (k index {ik}, q = {q})")


def umklapp_or_none(kcrys, ik, q):
    try:
        return umklapp(kcrys, ik, q)
    except ValueError:
        return None, None


def sigma_cohsex(problem, ik, q, geps, W, vq, n0, nn):
    """(sx, coh) [nn] in eV: one q-point's share of the static screened-exchange
    and Coulomb-hole diagonal elements (Eqs. sigma_sx, sigma_coh with
    W = eps^-1(q, 0) v(q+G')) for bands n0..n0+nn-1 at k = kcrys[ik]:
        sx[n]  = -(1/N_k) sum_{n'' occupied} conj(M)^T W M
        coh[n] = (1/2)(1/N_k) sum_{n'' all} conj(M)^T (W - diag v) M
    with M = M_{n''n}(k - q, q, G): band n'' at k - q, band n at k (the
    paper's M_{n''n}(k, -q, -G))."""
    jk = k_minus_q(problem.kcrys, ik, q)
    kp, G0 = umklapp(problem.kcrys, jk, q)
    nb = problem.nbands
    M = mtxel(problem.box, problem.gvec[jk], problem.coeff[jk], problem.gvec[kp],
              problem.coeff[kp][n0:n0 + nn], G0, geps)            # [nb][nn][ng]
    ng = len(geps)
    sw = quad(M.reshape(nb * nn, ng), W).reshape(nb, nn)
    sv = quad(M.reshape(nb * nn, ng), np.diag(np.asarray(vq, np.float64)).astype(np.complex128)).reshape(nb, nn)
    sx = np.zeros(nn)
    coh = np.zeros(nn)
    for n in range(nn):
        for m in range(nb):
            if m < problem.nv:
                sx[n] -= sw[m, n] / problem.nk
            coh[n] += 0.5 * (sw[m, n] - sv[m, n]) / problem.nk
    return sx, coh


def bse_kernel(problem, ik, jk, geps0, v0, qd, gepsd, W, vb, cb):
    """(KX, KD) [(v c)][(v' c')] in eV for bands vb = (v0, nv) of the occupied
    and cb = (c0, nc) of the empty bands at k_i = kcrys[ik] (rows) and
    k_j = kcrys[jk] (columns), q = k_j - k_i = qd:
        KX = (1/N_k) sum_G v(G) M_vc(k_i, 0, G) conj(M_v'c'(k_j, 0, G))
        KD = -(1/N_k) sum_GG' conj(M_cc'(k_i, q, G)) W_GG' M_vv'(k_i, q, G')
    (the K^X and K^D integrals of the BSE section times the factor i of the
    time integration)."""
    p = problem
    (va, nv), (ca, nc) = vb, cb
    ca += p.nv
    box = p.box
    zero = np.zeros(3, np.int32)
    Mi = mtxel(box, p.gvec[ik], p.coeff[ik][va:va + nv], p.gvec[ik], p.coeff[ik][ca:ca + nc], zero, geps0)
    Mj = mtxel(box, p.gvec[jk], p.coeff[jk][va:va + nv], p.gvec[jk], p.coeff[jk][ca:ca + nc], zero, geps0)
    lib = _load()
    P = nv * nc
    KX = np.zeros((P, P), dtype=np.complex128)
    lib.oracle_bse_exchange(nv, nc, len(geps0), _ptr(Mi), _ptr(Mj), _ptr(_f64(v0)), 1.0 / p.nk, _ptr(KX))
    kp, G0 = umklapp(p.kcrys, ik, qd)
    assert kp == jk, "k_i + q must land on k_j"
    Mcc = mtxel(box, p.gvec[ik], p.coeff[ik][ca:ca + nc], p.gvec[jk], p.coeff[jk][ca:ca + nc], G0, gepsd)
    Mvv = mtxel(box, p.gvec[ik], p.coeff[ik][va:va + nv], p.gvec[jk], p.coeff[jk][va:va + nv], G0, gepsd)
    KD = np.zeros((P, P), dtype=np.complex128)
    lib.oracle_bse_direct(nv, nc, len(gepsd), _ptr(Mcc), _ptr(Mvv), _ptr(_c128(W)), 1.0 / p.nk, _ptr(KD))
    return KX, KD
