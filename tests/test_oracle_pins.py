"""Pins for the CPU FP64 oracle: it is checked here against things other than
itself -- brute-force real-space sums, numpy's FFT, closed forms, a golden
fixture derived by hand and invariants of the paper's formulas (Sec. II of
arXiv:2206.00808: the P_GG'(q, w) formula and Eq. matrix_el).  No GPU needed.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers --

def random_spinors(rng, ngw, nb):
    z = rng.standard_normal((2 * ngw, nb)) + 1j * rng.standard_normal((2 * ngw, nb))
    q, _ = np.linalg.qr(z)
    return np.ascontiguousarray(q.T.reshape(nb, 2, ngw))


def random_miller_set(rng, lo, hi, n):
    pts = np.array([(a, b, c) for a in range(lo, hi + 1) for b in range(lo, hi + 1)
                    for c in range(lo, hi + 1)], dtype=np.int32)
    idx = rng.choice(len(pts), size=n, replace=False)
    return pts[np.sort(idx)]


def realspace_u(box, gvec, coeff, shift=(0, 0, 0)):
    """u_alpha(r) = sum_h c_alpha(h) exp(2 pi i (h - shift).r / N) by direct sums
    (the plane-wave form of Sec. III.A, shifted for the k+q umklapp)."""
    N = np.asarray(box)
    r = np.stack(np.meshgrid(*[np.arange(n) for n in box], indexing="ij"), -1).reshape(-1, 3)
    h = np.asarray(gvec, float) - np.asarray(shift, float)
    phase = np.exp(2j * np.pi * (r / N) @ h.T)          # (Nr, ngw)
    return np.einsum("rg,nag->nar", phase, coeff)           # [nb][2][Nr]


def realspace_M(box, uv, uc, geps):
    """M_vc(G) = N^-3 sum_r sum_alpha conj(u_v) u_c exp(-2 pi i G.r/N) by direct sums."""
    N = np.asarray(box)
    r = np.stack(np.meshgrid(*[np.arange(n) for n in box], indexing="ij"), -1).reshape(-1, 3)
    phase = np.exp(-2j * np.pi * (r / N) @ np.asarray(geps, float).T)   # (Nr, ng)
    rho = np.einsum("var,car->vcr", uv.conj(), uc)
    return rho @ phase / np.prod(N)


def tiny_problem(rng, box=(5, 6, 4), kgrid=(2, 1, 1), nv=2, nc=3, ngw=9, ng=7,
                 q=(0.5, 0.0, 0.0), freq=(0.0, 3.0), coeff_fn=None, energy_fn=None):
    kc = syn.kgrid_points(kgrid)
    gvec = [random_miller_set(rng, -1, 1, ngw) for _ in kc]
    coeff = [random_spinors(rng, ngw, nv + nc) if coeff_fn is None else coeff_fn(ik, gvec[ik])
             for ik in range(len(kc))]
    energy = [np.concatenate([np.sort(rng.uniform(-5, 0, nv)), np.sort(rng.uniform(1, 9, nc))])
              if energy_fn is None else energy_fn(ik) for ik in range(len(kc))]
    geps = random_miller_set(rng, -1, 1, ng)
    return syn.Problem("tiny", np.eye(3) * 8.0, tuple(box), tuple(kgrid), kc, nv, nc, gvec,
                       coeff, energy, [(np.asarray(q, float), geps, nc)], np.asarray(freq, float))


def bruteforce_chi0_paper_convention(p, q, geps):
    """The paper's own arrangement of the P formula, by real-space sums:
    occupied band n at k+q, empty band n' at k,
      M_nn'(k,q,G) = sum_alpha <n,k+q,alpha| e^{i(q+G).r} |n',k,alpha>
                   = N^-3 sum_r sum_alpha conj(u_{n,k+q}) u_{n',k} e^{+iG.r},
      P_GG' = (1/N_k) sum conj(M(G)) M(G') [1/(D - i w) + 1/(D + i w)],
      D = e_{n,k+q} - e_{n',k}."""
    ng = len(geps)
    P = np.zeros((len(p.freq), ng, ng), dtype=np.complex128)
    for ik in range(p.nk):
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)      # k+q = k' + G0
        u_occ = realspace_u(p.box, p.gvec[kp], p.coeff[kp][:p.nv], shift=G0)
        u_emp = realspace_u(p.box, p.gvec[ik], p.coeff[ik][p.nv:])
        M = realspace_M(p.box, u_occ, u_emp, -np.asarray(geps))   # e^{+iG.r}
        for j, w in enumerate(p.freq):
            for n in range(p.nv):
                for m in range(p.nc):
                    d = p.energy[kp][n] - p.energy[ik][p.nv + m]
                    wt = (1.0 / (d - 1j * w) + 1.0 / (d + 1j * w))
                    P[j] += wt * np.outer(M[n, m].conj(), M[n, m])
    return P / p.nk


# --------------------------------------------------------------- mtxel pins --

@pytest.mark.parametrize("G0", [(0, 0, 0), (1, 0, -1), (-1, 2, 0)])
def test_mtxel_matches_realspace_bruteforce(G0):
    """Eq. matrix_el by direct real-space sums equals the oracle's G-space
    convolution, including an umklapp shift and spheres that wrap the box."""
    rng = np.random.default_rng(11)
    box = (5, 6, 4)
    gv = random_miller_set(rng, -2, 2, 30)       # wider than the 4-box: wraps
    gc = random_miller_set(rng, -2, 2, 25)
    cv = random_spinors(rng, 30, 3)
    cc = random_spinors(rng, 25, 4)
    geps = random_miller_set(rng, -2, 2, 11)
    M = oracle.mtxel(box, gv, cv, gc, cc, G0, geps)
    uv = realspace_u(box, gv, cv)
    uc = realspace_u(box, gc, cc, shift=G0)
    ref = realspace_M(box, uv, uc, geps)
    assert np.abs(M - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())


def test_mtxel_matches_numpy_fft():
    """The FFT route of Eq. matrix_el through numpy.fft on a realistic sphere."""
    p = syn.make_problem("si18_qx")
    q, geps, nc = p.qs[0]
    ik = 4                                   # k = (1/2,0,0): k + q wraps
    kp, G0 = oracle.umklapp(p.kcrys, ik, q)
    nv = p.nv
    M = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:nv], p.gvec[kp], p.coeff[kp][nv:nv + 4],
                     G0, geps)
    N = np.array(p.box)
    n3 = np.prod(N)

    def to_box(g, c, shift):
        b = np.zeros((c.shape[0], 2) + p.box, dtype=np.complex128)
        idx = np.mod(np.asarray(g) - shift, N)
        np.add.at(b, (slice(None), slice(None), idx[:, 0], idx[:, 1], idx[:, 2]), c)
        return np.fft.ifftn(b, axes=(2, 3, 4)) * n3         # e^{+i h r}, unnormalised

    uv = to_box(p.gvec[ik], p.coeff[ik][:nv], np.zeros(3, int))
    uc = to_box(p.gvec[kp], p.coeff[kp][nv:nv + 4], G0)
    rho = np.einsum("vaxyz,caxyz->vcxyz", uv.conj(), uc)
    F = np.fft.fftn(rho, axes=(2, 3, 4)) / n3
    gi = np.mod(geps, N)
    ref = F[:, :, gi[:, 0], gi[:, 1], gi[:, 2]]
    assert tuple(G0) != (0, 0, 0)            # this k exercises the umklapp
    assert np.abs(M - ref).max() < 1e-13


def test_orthonormality_q0_head():
    """M_nm(q=0, G=0) = delta_nm for orthonormal spinors (unit norm over both
    components, Sec. II)."""
    p = syn.make_problem("si16_q0")
    c = p.coeff[2]
    M = oracle.mtxel(p.box, p.gvec[2], c, p.gvec[2], c, (0, 0, 0), [[0, 0, 0]])
    assert np.abs(M[:, :, 0] - np.eye(len(c))).max() < 1e-13


def test_plane_wave_mtxel_closed_form():
    """Single plane waves: M(G) = 1 iff spins agree and h_c - G0 = h_v + G (mod N)."""
    box = (6, 6, 6)
    gv = np.array([[0, 0, 0], [1, -1, 2], [2, 2, -2]], dtype=np.int32)
    gc = np.array([[1, 0, 0], [0, 1, 0], [-2, 1, 1]], dtype=np.int32)
    cv = syn.plane_wave_bands(gv, [(0, 0), (1, 1), (2, 0)])
    cc = syn.plane_wave_bands(gc, [(0, 0), (1, 1), (2, 0), (0, 1)])
    G0 = np.array([1, 0, -1])
    geps = np.array([(a, b, c) for a in range(-3, 3) for b in range(-3, 3) for c in range(-3, 3)],
                    dtype=np.int32)
    M = oracle.mtxel(box, gv, cv, gc, cc, G0, geps)
    vpick = [(0, 0), (1, 1), (2, 0)]
    cpick = [(0, 0), (1, 1), (2, 0), (0, 1)]
    exp = np.zeros_like(M)
    for v, (iv, av) in enumerate(vpick):
        for c, (ic, ac) in enumerate(cpick):
            if av != ac:
                continue
            target = np.mod(gc[ic] - G0 - gv[iv], 6)
            for g, G in enumerate(geps):
                if np.all(np.mod(G, 6) == target):
                    exp[v, c, g] = 1.0
    assert np.array_equal(M, exp)
    assert np.abs(M).sum() > 0


# ---------------------------------------------------------------- chi0 pins --

def test_weight_is_the_papers_bracket():
    """w = 1/(D - i w) + 1/(D + i w) (the bracket of the P formula at
    omega -> i omega, eta -> 0) is real and equals the oracle's weight."""
    for ev, ec, w in [(-1.0, 3.0, 0.0), (-7.5, 1.25, 2.0), (-0.1, 29.0, 40.0)]:
        d = ev - ec
        z = 1.0 / (d - 1j * w) + 1.0 / (d + 1j * w)
        assert abs(z.imag) < 1e-15
        assert abs(oracle.weight(ev, ec, w) - z.real) <= 1e-15 * abs(z.real)


def test_golden_plane_wave_chi0():
    """Hand-derived closed form (tests/golden/plane_wave_chi0.txt)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "plane_wave_chi0.txt"))
    g = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    coeff = np.zeros((5, 2, 3), dtype=np.complex128)
    coeff[0, 0, 0] = 1      # v0 = |000, up>
    coeff[1, 1, 0] = 1      # v1 = |000, down>
    coeff[2, 0, 1] = 1      # c0 = |100, up>
    coeff[3, 1, 1] = 1      # c1 = |100, down>
    coeff[4, 0, 2] = 1      # c2 = |010, up>
    energy = np.array([-1.0, -2.0, 3.0, 1.0, 2.0])
    geps = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0]], dtype=np.int32)
    freq = np.array(sorted(set(rows[:, 0])))
    p = syn.Problem("pw", np.eye(3) * 8.0, (4, 4, 4), (1, 1, 1), np.zeros((1, 3)), 2, 3,
                    [g], [coeff], [energy], [(np.zeros(3), geps, 3)], freq)
    chi = oracle.chi0(p)
    exp = np.zeros_like(chi)
    for w, r, c, re, im in rows:
        exp[list(freq).index(w), int(r), int(c)] = re + 1j * im
    assert np.abs(chi - exp).max() < 1e-15


def test_chi0_matches_bruteforce_in_papers_convention():
    """Whole chi0 against an independent real-space brute force written in the
    paper's own arrangement (occupied at k+q, empty at k, e^{+i(q+G)r}):
    P_GG'(q) = chi0_{-G,-G'}(-q) on the same data.  This pins M, the umklapp,
    the weights, the 1/N_k and the absence of a spin factor together."""
    rng = np.random.default_rng(5)
    p = tiny_problem(rng, kgrid=(2, 1, 1), q=(0.5, 0.0, 0.0), freq=(0.0, 2.5))
    q, geps, _ = p.qs[0]
    P = bruteforce_chi0_paper_convention(p, q, geps)
    p.qs = [(-q, -geps, p.nc)]
    chi = oracle.chi0(p)
    assert np.abs(chi - P).max() < 1e-14 * np.abs(P).max()
    assert np.abs(P).max() > 1e-3


def test_spinless_times_spin_gives_factor_two():
    """Spinors phi x |up>, phi x |down> from spinless phi reproduce twice the
    spinless chi0 (the P formula with the doubled band set, Sec. II)."""
    rng = np.random.default_rng(7)
    nv, nc = 3, 4
    kc = syn.kgrid_points((2, 1, 1))
    gvec = [random_miller_set(rng, -2, 2, 40) for _ in kc]
    phis, ens = [], []
    for ik in range(2):
        z = rng.standard_normal((40, nv + nc)) + 1j * rng.standard_normal((40, nv + nc))
        phis.append(np.linalg.qr(z)[0].T)
        ens.append(np.concatenate([np.sort(rng.uniform(-5, 0, nv)), np.sort(rng.uniform(1, 9, nc))]))
    geps = random_miller_set(rng, -1, 1, 9)
    q = np.array([0.5, 0, 0])
    freq = np.array([0.0, 4.0])
    up = [np.stack([ph, np.zeros_like(ph)], 1) for ph in phis]      # spinless as |up> only
    p1 = syn.Problem("s", np.eye(3) * 8, (6, 6, 6), (2, 1, 1), kc, nv, nc, gvec, up, ens,
                     [(q, geps, nc)], freq)
    chi_spinless = oracle.chi0(p1)
    sp = [syn.spinless_to_spinor(ph) for ph in phis]
    en2 = [np.repeat(e, 2) for e in ens]
    p2 = syn.Problem("s2", np.eye(3) * 8, (6, 6, 6), (2, 1, 1), kc, 2 * nv, 2 * nc, gvec, sp, en2,
                     [(q, geps, 2 * nc)], freq)
    chi_spinor = oracle.chi0(p2)
    assert np.abs(chi_spinor - 2 * chi_spinless).max() < 1e-14 * np.abs(chi_spinless).max()


def test_global_spin_rotation_invariance():
    """A fixed SU(2)/U(2) rotation of (up, down) in every band leaves M and
    chi0 unchanged (the trace over alpha in M; the SU(2) action of Sec. IV)."""
    p = syn.make_problem("si18_qx")
    chi = oracle.chi0(p, k_indices=[0, 5])
    th, ph, xi = 0.7, 1.9, -0.4
    u = np.array([[np.cos(th) * np.exp(1j * ph), np.sin(th) * np.exp(1j * xi)],
                  [-np.sin(th) * np.exp(-1j * xi), np.cos(th) * np.exp(-1j * ph)]])
    p.coeff = [syn.rotate_spin(c, u) for c in p.coeff]
    chi_r = oracle.chi0(p, k_indices=[0, 5])
    assert np.abs(chi_r - chi).max() < 1e-13 * np.abs(chi).max()


def test_band_unitary_invariance_with_degenerate_energies():
    """With all valence (conduction) energies at each k equal, any unitary
    mixing of the valence (conduction) bands leaves chi0 unchanged."""
    rng = np.random.default_rng(3)
    nv, nc = 3, 4
    p = tiny_problem(rng, nv=nv, nc=nc, ngw=20, energy_fn=lambda ik: np.array([-2.0] * 3 + [5.0] * 4))
    chi = oracle.chi0(p)
    for ik in range(p.nk):
        uv = np.linalg.qr(rng.standard_normal((nv, nv)) + 1j * rng.standard_normal((nv, nv)))[0]
        uc = np.linalg.qr(rng.standard_normal((nc, nc)) + 1j * rng.standard_normal((nc, nc)))[0]
        c = p.coeff[ik].copy()
        c[:nv] = np.einsum("mn,nag->mag", uv, c[:nv])
        c[nv:] = np.einsum("mn,nag->mag", uc, c[nv:])
        p.coeff[ik] = c
    chi_r = oracle.chi0(p)
    assert np.abs(chi_r - chi).max() < 1e-13 * np.abs(chi).max()


@pytest.fixture(scope="module")
def si18_multi_freq():
    p = syn.make_problem("si18_qx")
    p.freq = np.array([0.0, 1.5, 6.0, 40.0, 1.0e4])
    return p, oracle.chi0(p)


def test_hermitian_and_negative_semidefinite(si18_multi_freq):
    """chi0(i w) is Hermitian and <= 0 for every w, since every weight < 0."""
    _, chi = si18_multi_freq
    for cj in chi:
        scale = np.abs(cj).max()
        assert np.abs(cj - cj.conj().T).max() < 1e-15 * scale * 10
        ev = np.linalg.eigvalsh(0.5 * (cj + cj.conj().T))
        assert ev.max() < 1e-13 * scale
        assert ev.min() < -1e-3 * scale


def test_loewner_monotone_in_imaginary_frequency(si18_multi_freq):
    """chi0(i w2) - chi0(i w1) is positive semidefinite for w2 > w1."""
    _, chi = si18_multi_freq
    for j in range(len(chi) - 1):
        d = chi[j + 1] - chi[j]
        ev = np.linalg.eigvalsh(0.5 * (d + d.conj().T))
        assert ev.min() > -1e-13 * np.abs(chi[j]).max()


def test_large_frequency_asymptote(si18_multi_freq):
    """w -> infinity: chi0 -> (2/w^2)(1/N_k) sum D conj(M) M."""
    p, chi = si18_multi_freq
    q, geps, nc = p.qs[0]
    ng = len(geps)
    big = p.freq[-1]
    lim = np.zeros((ng, ng), dtype=np.complex128)
    for ik in range(p.nk):
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        M = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:p.nv], p.gvec[kp],
                         p.coeff[kp][p.nv:], G0, geps)
        D = p.energy[ik][:p.nv, None] - p.energy[kp][None, p.nv:]
        lim += np.einsum("vc,vcg,vch->gh", D, M.conj(), M)
    lim *= 2.0 / big ** 2 / p.nk
    rel = np.abs(chi[-1] - lim).max() / np.abs(lim).max()
    assert rel < 1e-5          # the next term is O((D/w)^2) ~ (30/1e4)^2


def test_completeness_closed_form():
    """With every band of the box at k' (a full unitary over 2 N^3 spinor
    plane waves): sum_n conj(M_vn(G)) M_vn(G') = sum_alpha sum_h c_v(h)
    conj(c_v((h + G - G') mod N))."""
    rng = np.random.default_rng(9)
    box = (3, 3, 2)
    full = np.array([(a, b, c) for a in range(3) for b in range(3) for c in range(2)], dtype=np.int32)
    nfull = 2 * len(full)
    U = np.linalg.qr(rng.standard_normal((nfull, nfull)) + 1j * rng.standard_normal((nfull, nfull)))[0]
    cc = np.ascontiguousarray(U.T.reshape(nfull, 2, len(full)))
    cv = random_spinors(rng, len(full), 2)
    geps = random_miller_set(rng, -1, 1, 6)
    M = oracle.mtxel(box, full, cv, full, cc, (0, 0, 0), geps)
    # D = e_v - e_c = 2 at w = 0 makes every weight 2D/D^2 = 1.
    S = np.zeros((1, len(geps), len(geps)), dtype=np.complex128)
    oracle.chi0_accumulate(M[:1], [0.0], np.full(nfull, -2.0), [0.0], S)
    N = np.array(box)
    cvbox = np.zeros((2,) + box, dtype=np.complex128)
    cvbox[:, full[:, 0], full[:, 1], full[:, 2]] = cv[0]
    exp = np.zeros((len(geps), len(geps)), dtype=np.complex128)
    for a, G in enumerate(geps):
        for b, Gp in enumerate(geps):
            sh = np.mod(full + G - Gp, N)
            exp[a, b] = np.sum(cvbox[:, full[:, 0], full[:, 1], full[:, 2]]
                               * cvbox[:, sh[:, 0], sh[:, 1], sh[:, 2]].conj())
    assert np.abs(S[0] - exp).max() < 1e-13


def test_q0_head_vanishes():
    """At q = 0, M_vc(G=0) = 0 for v != c, so the head chi0_00 is 0."""
    p = syn.make_problem("si16_q0")
    chi = oracle.chi0(p)
    geps = p.qs[0][1]
    i0 = int(np.where((geps == 0).all(1))[0][0])
    assert abs(chi[0, i0, i0]) < 1e-14 * np.abs(chi).max()
    assert abs(chi[0, i0]).max() < 1e-14 * np.abs(chi).max()


# ---------------------------------------------------------------------------
# Dielectric matrix, eps^-1 and W (Sec. II: eps = delta - v(q+G) P,
# W = eps^-1 v(q+G')), v(q+G) = 4 pi e^2 / (Omega |q+G|^2) in eV.
E2 = 27.211386245988   # e^2 in eV bohr


def test_coulomb_simple_cubic_closed_form():
    a = 2.0                                   # bohr; B = (2 pi / a) I = pi I, Omega = 8
    q = [0.5, 0.0, 0.0]
    g = np.array([[0, 0, 0], [1, 0, 0], [-1, 2, 0], [0, 0, 3]])
    k2 = np.pi ** 2 * np.array([0.25, 2.25, 0.25 + 4.0, 0.25 + 9.0])
    want = 4 * np.pi * E2 / (8.0 * k2)
    assert np.allclose(oracle.coulomb(a * np.eye(3), q, g), want, rtol=1e-14)


def test_coulomb_fcc_against_independent_reciprocal_and_head():
    from paper_2206_00808_gb300 import synthetic as syn
    a = 10.26
    avec = syn.fcc_cell(a)
    omega = a ** 3 / 4                        # FCC primitive cell volume
    B = 2 * np.pi * np.linalg.inv(np.asarray(avec)).T
    rng = np.random.default_rng(3)
    g = rng.integers(-4, 5, (40, 3))
    q = np.array([0.25, -0.125, 0.0])
    k = (q + g) @ B
    want = 4 * np.pi * E2 / (omega * (k * k).sum(1))
    assert np.allclose(oracle.coulomb(avec, q, g), want, rtol=1e-13)
    # q + G = 0: v is defined as 0 there
    assert oracle.coulomb(avec, [0, 0, 0], [[0, 0, 0], [1, 0, 0]])[0] == 0.0


def _nsd_chi(rng, n, nf, rank=None):
    chis = []
    for _ in range(nf):
        X = rng.normal(size=(n, rank or n)) + 1j * rng.normal(size=(n, rank or n))
        chis.append(-(X @ X.conj().T) * 0.05)
    return np.array(chis)


def test_epsinv_is_the_inverse_of_eps_and_w_is_hermitian():
    rng = np.random.default_rng(5)
    n = 23
    chi = _nsd_chi(rng, n, 3)
    v = rng.uniform(0.2, 3.0, n)
    e, w = oracle.epsinv(chi, v)
    for j in range(3):
        eps = np.eye(n) - v[:, None] * chi[j]
        assert np.abs(e[j] @ eps - np.eye(n)).max() < 1e-12
        assert np.abs(eps @ e[j] - np.eye(n)).max() < 1e-12
        assert np.abs(w[j] - w[j].conj().T).max() < 1e-12 * np.abs(w[j]).max()
        # eps is similar to I + (PSD), so its eigenvalues are real and >= 1
        ev = np.linalg.eigvals(eps)
        assert np.abs(ev.imag).max() < 1e-10 and ev.real.min() > 1 - 1e-12


def test_epsinv_diagonal_closed_form():
    n = 6
    d = -np.linspace(0.1, 2.0, n)
    v = np.linspace(0.5, 1.5, n)
    e, w = oracle.epsinv(np.diag(d).astype(complex)[None], v)
    assert np.allclose(np.diag(e[0]), 1 / (1 - v * d), rtol=1e-15)
    assert np.allclose(np.diag(w[0]), v / (1 - v * d), rtol=1e-15)
    assert np.abs(e[0] - np.diag(np.diag(e[0]))).max() == 0.0


def test_w_rank_one_sherman_morrison():
    """chi = -u u^H: eps = I + diag(v) u u^H, so
    W = eps^-1 V = V - (V u)(V u)^H / (1 + u^H V u)."""
    rng = np.random.default_rng(11)
    n = 9
    u = rng.normal(size=n) + 1j * rng.normal(size=n)
    v = rng.uniform(0.1, 2.0, n)
    chi = -np.outer(u, u.conj())[None]
    _, w = oracle.epsinv(chi, v)
    vu = v * u
    want = np.diag(v) - np.outer(vu, vu.conj()) / (1 + (u.conj() * v * u).sum().real)
    assert np.abs(w[0] - want).max() < 1e-13 * np.abs(want).max()


def test_epsinv_head_row_is_identity_when_v_is_zero():
    rng = np.random.default_rng(2)
    n = 5
    chi = _nsd_chi(rng, n, 1)
    v = rng.uniform(0.5, 1.0, n)
    v[0] = 0.0
    e, w = oracle.epsinv(chi, v)
    assert np.allclose(e[0][0], np.eye(n)[0], atol=1e-15)
    assert np.abs(w[0][:, 0]).max() == 0.0


# ------------------------------------------- large-case forms of the oracle --

def test_matmul_contraction_equals_the_loop_and_bruteforce():
    """The library-product form of the chi0 sum (used for the full-size
    parity cases) equals the plain loop, and both the real-space brute force."""
    rng = np.random.default_rng(11)
    p = tiny_problem(rng, nv=3, nc=4, freq=(0.0, 2.5, 9.0))
    loop = oracle.chi0(p)
    mm = oracle.chi0(p, contraction="matmul")
    assert np.linalg.norm(mm - loop) <= 1e-13 * np.linalg.norm(loop)
    # brute force of one k-point's share: real-space M, the bracket in complex form
    ik = 1
    kp, G0 = oracle.umklapp(p.kcrys, ik, p.qs[0][0])
    uv = realspace_u(p.box, p.gvec[ik], p.coeff[ik][:p.nv])
    uc = realspace_u(p.box, p.gvec[kp], p.coeff[kp][p.nv:], shift=G0)
    M = realspace_M(p.box, uv, uc, p.qs[0][1]).reshape(-1, len(p.qs[0][1]))
    d = (p.energy[ik][:p.nv, None] - p.energy[kp][None, p.nv:]).reshape(-1)
    share = oracle.chi0(p, k_indices=[ik], contraction="matmul")
    for j, f in enumerate(p.freq):
        w = (1.0 / (d - 1j * f) + 1.0 / (d + 1j * f)).real
        want = (M.conj().T * w) @ M / p.nk
        assert np.abs(share[j] - want).max() <= 1e-13 * np.abs(want).max()


def test_g_subset_is_the_block_of_the_full_chi0():
    """chi0 over a subset of the dielectric sphere is exactly that block of the
    full chi0 (every M(G) is its own convolution sum)."""
    p = syn.make_problem("si18_qx", nv=2, nc=3, nfreq=2)
    full = oracle.chi0(p)
    S = [0, 3, 40, 99, 136]
    sub = oracle.chi0(p, g_indices=S)
    assert np.array_equal(sub, full[:, S][:, :, S])
