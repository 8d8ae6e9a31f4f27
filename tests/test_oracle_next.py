"""Pins for the oracle's self-energy (static screened exchange and Coulomb
hole, Eqs. sigma_sx and sigma_coh of arXiv:2206.00808 Sec. II) and BSE
kernel blocks (the K^X and K^D integrals of the BSE section): closed forms
from completeness and single plane waves, the spinless (x) |up>,|down>
structure the paper points out, and real-space brute force.  No GPU needed.
"""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn
from test_oracle_pins import random_miller_set, random_spinors, realspace_M, realspace_u, tiny_problem


def random_hermitian(rng, n):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (a + a.conj().T)


def spinless_problem(rng, nvs, ncs, ngw=10, ng=7, box=(5, 6, 4)):
    """Spinors phi (x) |up>, phi (x) |down> of random orthonormal spinless
    orbitals phi (bands 2i, 2i+1), on a two-point k-grid with q = (1/2,0,0)."""
    phis = {}

    def coeff(ik, gv):
        z = rng.standard_normal((len(gv), nvs + ncs)) + 1j * rng.standard_normal((len(gv), nvs + ncs))
        phi = np.linalg.qr(z)[0].T
        phis[ik] = phi
        return syn.spinless_to_spinor(phi)

    p = tiny_problem(rng, box=box, nv=2 * nvs, nc=2 * ncs, ngw=ngw, ng=ng, coeff_fn=coeff)
    return p, phis


# -------------------------------------------------------------- self-energy --

def test_sigma_of_spinor_pairs_is_the_spinless_sigma():
    """phi (x) |alpha> pairs with phi'' (x) |beta> only for alpha = beta, so
    each spin partner of a spinless band gets exactly the spinless self-energy
    (no factor 2, unlike chi0): screened exchange over the nvs occupied
    spinless bands, Coulomb hole over all of them."""
    rng = np.random.default_rng(21)
    nvs, ncs = 2, 3
    p, phi = spinless_problem(rng, nvs, ncs)
    q, geps, _ = p.qs[0]
    ng = len(geps)
    W = random_hermitian(rng, ng)
    v = rng.uniform(0.5, 2.0, ng)
    ik = 0
    sx, coh = oracle.sigma_cohsex(p, ik, q, geps, W, v, 0, p.nbands)
    # spinless brute force in real space: band n'' at k - q (index 1), n at k
    jk = 1
    kp, G0 = oracle.umklapp(p.kcrys, jk, q)
    assert kp == ik
    u_kq = realspace_u(p.box, p.gvec[jk], phi[jk][:, None, :])
    u_k = realspace_u(p.box, p.gvec[ik], phi[ik][:, None, :], shift=G0)
    M = realspace_M(p.box, u_kq, u_k, geps)                    # [n''][n][G]
    Wv = W - np.diag(v)
    for n in range(nvs + ncs):
        sx0 = -sum(M[m, n].conj() @ W @ M[m, n] for m in range(nvs)).real / p.nk
        coh0 = 0.5 * sum(M[m, n].conj() @ Wv @ M[m, n] for m in range(nvs + ncs)).real / p.nk
        for s in (0, 1):
            assert abs(sx[2 * n + s] - sx0) <= 1e-12 * max(1.0, abs(sx0))
            assert abs(coh[2 * n + s] - coh0) <= 1e-12 * max(1.0, abs(coh0))


def complete_problem(rng, nv):
    """Every spinor plane wave of a 3x3x2 box at both k-points (a full
    unitary over the 36 components), nv of the 36 bands occupied."""
    box = (3, 3, 2)
    full = np.array([(a, b, c) for a in range(3) for b in range(3) for c in range(2)], dtype=np.int32)
    nfull = 2 * len(full)

    def coeff(ik, gv):
        U = np.linalg.qr(rng.standard_normal((nfull, nfull)) + 1j * rng.standard_normal((nfull, nfull)))[0]
        return np.ascontiguousarray(U.T.reshape(nfull, 2, len(full)))

    p = tiny_problem(rng, box=box, nv=nv, nc=nfull - nv, ngw=len(full), ng=6, coeff_fn=coeff)
    p.gvec = [full.copy() for _ in p.gvec]
    p.coeff = [coeff(ik, full) for ik in range(p.nk)]
    return p, full


def test_bare_exchange_with_every_band_occupied_is_minus_the_coulomb_sum():
    """With W = v and a complete occupied set at k - q, completeness gives
    sum_n'' |M_n''n(G)|^2 = 1 for a normalised band n, so
    Sigma^SX = -(1/N_k) sum_G v(q+G) and Sigma^COH = 0."""
    rng = np.random.default_rng(5)
    p, _ = complete_problem(rng, nv=36)
    q, geps, _ = p.qs[0]
    v = rng.uniform(0.2, 3.0, len(geps))
    sx, coh = oracle.sigma_cohsex(p, 0, q, geps, np.diag(v).astype(complex), v, 0, 5)
    assert np.allclose(sx, -v.sum() / p.nk, rtol=0, atol=1e-12)
    assert np.allclose(coh, 0.0, atol=1e-13)


def test_coulomb_hole_completeness_closed_form():
    """Every band n'' at k - q summed: sum_n'' conj(M(G)) M(G') =
    sum_alpha sum_h conj(C_n(h)) C_n(h + G' - G) on the box, so
    Sigma^COH_n = (1/2N_k) sum_GG' (W - v)_GG' sum_alpha sum_h conj(C_n(h)) C_n((h + G' - G) mod N),
    where C_n is band n at k placed on the box (shifted by the umklapp G0)."""
    rng = np.random.default_rng(8)
    p, full = complete_problem(rng, nv=10)
    q, geps, _ = p.qs[0]
    ng = len(geps)
    W = random_hermitian(rng, ng)
    v = rng.uniform(0.2, 3.0, ng)
    ik = 0
    sx, coh = oracle.sigma_cohsex(p, ik, q, geps, W, v, 0, 4)
    jk = oracle.k_minus_q(p.kcrys, ik, q)
    _, G0 = oracle.umklapp(p.kcrys, jk, q)
    N = np.array(p.box)
    for n in range(4):
        C = np.zeros((2,) + p.box, dtype=np.complex128)
        idx = np.mod(full - G0, N)
        C[:, idx[:, 0], idx[:, 1], idx[:, 2]] = p.coeff[ik][n]
        S = np.zeros((ng, ng), dtype=complex)
        for a, G in enumerate(geps):
            for b, Gp in enumerate(geps):
                sh = np.mod(full + Gp - G, N)
                S[a, b] = np.sum(C[:, full[:, 0], full[:, 1], full[:, 2]].conj() * C[:, sh[:, 0], sh[:, 1], sh[:, 2]])
        want = 0.5 * np.sum((W - np.diag(v)) * S).real / p.nk
        assert abs(coh[n] - want) <= 1e-12


# --------------------------------------------------------------- BSE kernel --

def plane_wave_problem(box, picks_v, picks_c, q=(0.5, 0.0, 0.0)):
    """Two k-points whose bands are single spinor plane waves: picks are
    (Miller index, spin) lists for the occupied and the empty bands."""
    hs = sorted({h for h, _ in picks_v + picks_c})
    gv = np.array(hs, dtype=np.int32)
    pos = {h: i for i, h in enumerate(hs)}
    coeff = syn.plane_wave_bands(gv, [(pos[h], a) for h, a in picks_v + picks_c])
    kc = syn.kgrid_points((2, 1, 1))
    nv, nc = len(picks_v), len(picks_c)
    return syn.Problem("pw", np.eye(3) * 8.0, tuple(box), (2, 1, 1), kc, nv, nc, [gv, gv.copy()],
                       [coeff, coeff.copy()], [np.zeros(nv + nc)] * 2, [(np.asarray(q), gv, nc)],
                       np.zeros(1))


def test_bse_kernels_of_plane_waves():
    """Single plane waves h with spin alpha: M_ab(G) = delta(alpha_a, alpha_b)
    [h_a + G = h_b - G0 mod N], so
      K^X[(vc)][(v'c')] = (1/N_k) sum_G v_G [G = h_c - h_v][G = h_c' - h_v'] d(a_v,a_c) d(a_v',a_c')
      K^D[(vc)][(v'c')] = -(1/N_k) W[G1][G2] d(a_c,a_c') d(a_v,a_v')
    with G1 = h_c' - G0 - h_c and G2 = h_v' - G0 - h_v when both lie in the sphere."""
    box = (6, 6, 6)
    pv = [((0, 0, 0), 0), ((1, 0, 0), 1), ((0, 1, 0), 0)]
    pc = [((1, 1, 0), 0), ((0, 0, 1), 1), ((2, 0, 0), 0), ((1, 0, 1), 1)]
    p = plane_wave_problem(box, pv, pc)
    rng = np.random.default_rng(2)
    geps = np.array([(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)], dtype=np.int32)
    ng = len(geps)
    v0 = rng.uniform(0.1, 2.0, ng)
    W = random_hermitian(rng, ng)
    qd = (0.5, 0.0, 0.0)
    KX, KD = oracle.bse_kernel(p, 0, 1, geps, v0, qd, geps, W, (0, 3), (0, 4))
    _, G0 = oracle.umklapp(p.kcrys, 0, qd)
    N = np.array(box)
    gidx = {tuple(np.mod(g, N)): i for i, g in enumerate(geps)}
    nk = p.nk
    for i, (hv, av) in enumerate(pv):
        for j, (hc, ac) in enumerate(pc):
            for i2, (hv2, av2) in enumerate(pv):
                for j2, (hc2, ac2) in enumerate(pc):
                    I, J = i * 4 + j, i2 * 4 + j2
                    x = 0.0
                    if av == ac and av2 == ac2:
                        g1 = gidx.get(tuple(np.mod(np.subtract(hc, hv), N)))
                        g2 = gidx.get(tuple(np.mod(np.subtract(hc2, hv2), N)))
                        if g1 is not None and g1 == g2:
                            x = v0[g1] / nk
                    assert abs(KX[I, J] - x) < 1e-14
                    d = 0.0
                    if ac == ac2 and av == av2:
                        g1 = gidx.get(tuple(np.mod(np.subtract(hc2, hc) - G0, N)))
                        g2 = gidx.get(tuple(np.mod(np.subtract(hv2, hv) - G0, N)))
                        if g1 is not None and g2 is not None:
                            d = -W[g1, g2] / nk
                    assert abs(KD[I, J] - d) < 1e-14


def test_bse_kernels_of_spinor_pairs_have_the_spin_block_structure():
    """Spinors phi (x) |alpha>: M_ab carries delta(alpha_a, alpha_b), so
    K^X[(v s_v, c s_c)][(v' s_v', c' s_c')] = d(s_v,s_c) d(s_v',s_c') K^X_0 and
    K^D[...] = d(s_c,s_c') d(s_v,s_v') K^D_0, with K_0 the kernel of the
    spinless orbitals (computed as spin-up spinors alone)."""
    rng = np.random.default_rng(17)
    nvs, ncs = 2, 2
    p, phi = spinless_problem(rng, nvs, ncs)
    q, geps, _ = p.qs[0]
    ng = len(geps)
    v0 = rng.uniform(0.1, 2.0, ng)
    W = random_hermitian(rng, ng)
    KX, KD = oracle.bse_kernel(p, 0, 1, geps, v0, q, geps, W, (0, 2 * nvs), (0, 2 * ncs))
    # spin-up only: bands phi_i (x) |up>
    import copy
    up = copy.copy(p)
    up.nv, up.nc = nvs, ncs
    up.coeff = [np.concatenate([c[0:2 * nvs:2], c[2 * nvs::2]]) for c in p.coeff]
    KX0, KD0 = oracle.bse_kernel(up, 0, 1, geps, v0, q, geps, W, (0, nvs), (0, ncs))
    assert np.abs(KX0).max() > 1e-3 and np.abs(KD0).max() > 1e-3
    nc2 = 2 * ncs
    for v in range(2 * nvs):
        for c in range(nc2):
            for v2 in range(2 * nvs):
                for c2 in range(nc2):
                    I, J = v * nc2 + c, v2 * nc2 + c2
                    I0, J0 = (v // 2) * ncs + c // 2, (v2 // 2) * ncs + c2 // 2
                    sx = (v % 2 == c % 2) and (v2 % 2 == c2 % 2)
                    sd = (c % 2 == c2 % 2) and (v % 2 == v2 % 2)
                    assert abs(KX[I, J] - (KX0[I0, J0] if sx else 0.0)) < 1e-13
                    assert abs(KD[I, J] - (KD0[I0, J0] if sd else 0.0)) < 1e-13


def test_bse_kernels_match_realspace_bruteforce():
    """Every matrix element by direct real-space sums (u(r) from the plane-wave
    form, the spin trace, the Fourier sum over the box), then the two
    contractions."""
    rng = np.random.default_rng(4)
    p = tiny_problem(rng, nv=2, nc=3)
    q, geps, _ = p.qs[0]
    ng = len(geps)
    v0 = rng.uniform(0.1, 2.0, ng)
    W = random_hermitian(rng, ng)
    KX, KD = oracle.bse_kernel(p, 0, 1, geps, v0, q, geps, W, (0, 2), (0, 3))
    kp, G0 = oracle.umklapp(p.kcrys, 0, q)
    u = {ik: realspace_u(p.box, p.gvec[ik], p.coeff[ik]) for ik in (0, 1)}
    u1s = realspace_u(p.box, p.gvec[1], p.coeff[1], shift=G0)
    Mi = realspace_M(p.box, u[0][:2], u[0][2:], geps).reshape(6, ng)
    Mj = realspace_M(p.box, u[1][:2], u[1][2:], geps).reshape(6, ng)
    kx = (Mi * v0) @ Mj.conj().T / p.nk
    Mcc = realspace_M(p.box, u[0][2:], u1s[2:], geps)       # [c][c'][G]
    Mvv = realspace_M(p.box, u[0][:2], u1s[:2], geps)       # [v][v'][G]
    kd = np.zeros_like(KD)
    for v in range(2):
        for c in range(3):
            for v2 in range(2):
                for c2 in range(3):
                    kd[v * 3 + c, v2 * 3 + c2] = -(Mcc[c, c2].conj() @ W @ Mvv[v, v2]) / p.nk
    assert np.abs(KX - kx).max() <= 1e-13 * np.abs(kx).max()
    assert np.abs(KD - kd).max() <= 1e-13 * np.abs(kd).max()
    # the exchange kernel over both k-points is Hermitian: the (k_i, k_i)
    # blocks are, and the (k_j, k_i) block is the adjoint of (k_i, k_j)
    z = np.zeros(3)
    KX00 = oracle.bse_kernel(p, 0, 0, geps, v0, z, geps, W, (0, 2), (0, 3))[0]
    KX10 = oracle.bse_kernel(p, 1, 0, geps, v0, q, geps, W, (0, 2), (0, 3))[0]
    assert np.abs(KX00 - KX00.conj().T).max() <= 1e-15 * np.abs(KX00).max()
    assert np.abs(KX10 - KX.conj().T).max() <= 1e-15 * np.abs(KX).max()
