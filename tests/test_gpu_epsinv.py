"""GPU dielectric-matrix inverse and screened interaction (FP64) against the
oracle's plain-LU inversion of the paper's unsymmetrised eps = 1 - v P:
W, eps^-1 and the symmetrised eps~^-1, on chi0 of the small workloads and on
synthetic negative semidefinite matrices with ragged block counts."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def gpu_modes(B, chi, s):
    import torch
    out = {}
    for mode in ("W", "epsinv", "epsinv_sym"):
        t = torch.from_numpy(np.ascontiguousarray(chi)).cuda()
        B.bgw_epsinv(t, s, mode)
        torch.cuda.synchronize()
        out[mode] = t.cpu().numpy()
    return out


@pytest.mark.parametrize("name,overrides", [("si18_qx", {}), ("si18_qx", {"ng": 59, "nc": 13, "nfreq": 3}),
                                            ("si16_q0", {"q": (0.5, 0.5, 0.0)})])
def test_epsinv_of_chi0_matches_oracle(gpu_lib, name, overrides):
    p = syn.make_problem(name, **overrides)
    q, geps, _ = p.qs[0]
    chi = oracle.chi0(p)
    v = oracle.coulomb(p.avec, q, geps)
    e_ref, w_ref = oracle.epsinv(chi, v)
    s = gpu_lib.bgw_coulomb_sqrt(p.avec, q, geps)
    got = gpu_modes(gpu_lib, chi, s)
    assert rel(got["W"], w_ref) <= TOL
    assert rel(got["epsinv"], e_ref) <= TOL
    sv = np.sqrt(v)
    assert rel(got["epsinv_sym"], e_ref * sv[None, :] / sv[:, None]) <= TOL


@pytest.mark.parametrize("n,nf", [(1, 1), (20, 2), (32, 1), (33, 2), (350, 3)])
def test_epsinv_synthetic_sizes(gpu_lib, n, nf):
    rng = np.random.default_rng(n)
    chis = []
    for _ in range(nf):
        X = rng.normal(size=(n, n + 3)) + 1j * rng.normal(size=(n, n + 3))
        chis.append(-(X @ X.conj().T) / n)
    chi = np.array(chis)
    v = rng.uniform(0.05, 5.0, n)
    e_ref, w_ref = oracle.epsinv(chi, v)
    got = gpu_modes(gpu_lib, chi, np.sqrt(v))
    assert rel(got["W"], w_ref) <= TOL
    assert rel(got["epsinv"], e_ref) <= TOL


def test_epsinv_head_zero_and_explicit_workspace(gpu_lib):
    import torch
    B = gpu_lib
    p = syn.make_problem("si16_q0")                     # q = 0: q + G = 0 for G = 0
    q, geps, _ = p.qs[0]
    chi = oracle.chi0(p)
    s = B.bgw_coulomb_sqrt(p.avec, q, geps)
    assert s[np.all(geps == 0, axis=1)][0] == 0.0
    _, w_ref = oracle.epsinv(chi, s ** 2)
    t = torch.from_numpy(chi.copy()).cuda()
    ws = torch.empty(B.bgw_epsinv_workspace_bytes(len(geps), chi.shape[0]), dtype=torch.uint8, device="cuda")
    B.bgw_epsinv(t, s, "W", work=ws)
    torch.cuda.synchronize()
    assert rel(t.cpu().numpy(), w_ref) <= TOL
    with pytest.raises(B.BgwError) as e:                # eps^-1 needs s > 0 everywhere
        B.bgw_epsinv(torch.from_numpy(chi.copy()).cuda(), s, "epsinv")
    assert e.value.status == B.BGW_E_ARG


def test_epsinv_rejects_indefinite_input(gpu_lib):
    import torch
    B = gpu_lib
    n = 40
    chi = np.diag(np.linspace(0.5, 2.0, n)).astype(np.complex128)[None]   # positive: eps~ indefinite
    t = torch.from_numpy(chi).cuda()
    with pytest.raises(B.BgwError) as e:
        B.bgw_epsinv(t, np.full(n, 1.0), "W")
    assert e.value.status == B.BGW_E_ARG
    # the library stays usable
    good = -np.eye(n, dtype=np.complex128)[None]
    t = torch.from_numpy(good).cuda()
    B.bgw_epsinv(t, np.full(n, 1.0), "W")
    assert np.allclose(t.cpu().numpy()[0], np.eye(n) / 2, atol=1e-15)
