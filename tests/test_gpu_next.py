"""GPU parity of the steps after chi0 that reuse the matrix elements, through
the C-ABI against the CPU FP64 oracle: matrix elements of any two band ranges
(bgw_mtxel_bands), the static screened-exchange and Coulomb-hole diagonal
elements of the self-energy (bgw_sigma_cohsex; Eqs. sigma_sx and sigma_coh of
arXiv:2206.00808 Sec. II) and the exchange and direct BSE kernel blocks
(bgw_bse_kernel; the K^X and K^D integrals of the BSE section).
Bars: M within 1e-12 (FP64) / 5e-6 (mixed) of max|M| elementwise; the
self-energy and kernel entries within 1e-12 of their largest magnitude."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_M = {"fp64": 1e-12, "mixed": 5e-6}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def si18():
    return syn.make_problem("si18_qx", nv=6, nc=10, ng=89)


def random_hermitian(rng, n):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (a + a.conj().T)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("ik, n0, nn, m0, nm", [
    (0, 0, 6, 0, 6),        # occupied x occupied (the BSE direct kernel's M_vv')
    (4, 6, 10, 6, 10),      # empty x empty at an umklapp k (M_cc')
    (4, 2, 9, 0, 16),       # a range across the gap x every band (the self-energy's n'')
    (0, 0, 16, 5, 3),
])
def test_mtxel_bands_matches_oracle(gpu_lib, torch_cuda, si18, prec, ik, n0, nn, m0, nm):
    torch = torch_cuda
    p = si18
    q, geps, _ = p.qs[0]
    ctx = gpu_lib.Chi0Context(p, prec)
    ctx.upload()
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    M = torch.zeros((nn, nm, len(geps)), dtype=dt, device="cuda")
    gpu_lib.bgw_mtxel_bands(ctx.ctx, q, geps, ik, n0, nn, m0, nm, M)
    kp, G0 = oracle.umklapp(p.kcrys, ik, q)
    ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][n0:n0 + nn], p.gvec[kp], p.coeff[kp][m0:m0 + nm], G0, geps)
    ctx.close()
    assert np.abs(M.cpu().numpy() - ref).max() <= TOL_M[prec] * np.abs(ref).max()


def physical_w(p, q, geps):
    """Static W = eps^-1 v(q+G') of the oracle's chi0 at this q (eV)."""
    import copy
    sub = copy.copy(p)
    sub.qs = [(np.asarray(q, float), geps, p.nc)]
    sub.freq = np.zeros(1)
    chi = oracle.chi0(sub)
    v = oracle.coulomb(p.avec, q, geps)
    _, W = oracle.epsinv(chi, v)
    return W[0], v


@pytest.mark.parametrize("which", ["random", "physical"])
@pytest.mark.parametrize("ik", [0, 4])
def test_sigma_cohsex_matches_oracle(gpu_lib, torch_cuda, si18, which, ik):
    torch = torch_cuda
    p = si18
    q, geps, _ = p.qs[0]
    ng = len(geps)
    if which == "random":
        rng = np.random.default_rng(ik + 3)
        W = random_hermitian(rng, ng)
        v = rng.uniform(0.1, 3.0, ng)
    else:
        W, v = physical_w(p, q, geps)
    n0, nn = 3, 7          # across the gap
    sx_ref, coh_ref = oracle.sigma_cohsex(p, ik, q, geps, W, v, n0, nn)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    sx = np.full(nn, 0.25)          # the call adds to what is there
    coh = np.full(nn, -0.5)
    gpu_lib.bgw_sigma_cohsex(ctx.ctx, q, geps, ik, n0, nn, Wd, v, sx, coh)
    ctx.close()
    scale = max(np.abs(sx_ref).max(), np.abs(coh_ref).max())
    assert np.abs(sx - 0.25 - sx_ref).max() <= 1e-12 * scale
    assert np.abs(coh + 0.5 - coh_ref).max() <= 1e-12 * scale
    if which == "physical":
        assert (sx_ref < 0).all()           # W = eps^-1 v is positive semidefinite here


@pytest.mark.parametrize("ik, jk, qd", [(0, 4, (0.5, 0, 0)), (4, 0, (0.5, 0, 0)), (1, 1, (0, 0, 0))])
def test_bse_kernel_matches_oracle(gpu_lib, torch_cuda, si18, ik, jk, qd):
    """(4, 0): k_i + q = k_j + (1, 0, 0), the umklapp case."""
    torch = torch_cuda
    p = si18
    bvec = syn.reciprocal(p.avec)
    z = np.zeros(3)
    geps0 = syn.eps_sphere(bvec, z, 59)
    v0 = oracle.coulomb(p.avec, z, geps0)
    qd = np.asarray(qd, float)
    gepsd = syn.eps_sphere(bvec, qd, 65)
    rng = np.random.default_rng(ik * 8 + jk)
    W = random_hermitian(rng, len(gepsd))
    vb, cb = (1, 4), (2, 5)
    KXr, KDr = oracle.bse_kernel(p, ik, jk, geps0, v0, qd, gepsd, W, vb, cb)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    P = vb[1] * cb[1]
    KX = torch.zeros((P, P), dtype=torch.complex128, device="cuda")
    KD = torch.zeros((P, P), dtype=torch.complex128, device="cuda")
    Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    gpu_lib.bgw_bse_kernel(ctx.ctx, ik, jk, z, geps0, v0, qd, gepsd, Wd, vb[0], vb[1], cb[0], cb[1], KX, KD)
    ctx.close()
    assert np.abs(KX.cpu().numpy() - KXr).max() <= 1e-12 * np.abs(KXr).max()
    assert np.abs(KD.cpu().numpy() - KDr).max() <= 1e-12 * np.abs(KDr).max()
    if ik == jk:
        kx = KX.cpu().numpy()
        assert np.abs(kx - kx.conj().T).max() <= 1e-13 * np.abs(kx).max()
