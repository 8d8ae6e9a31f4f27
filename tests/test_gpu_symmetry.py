"""Spinor symmetry unfolding on the GPU: element-by-element parity with the
oracle for several operations and fractional translations, and an
end-to-end check: chi0 at q = 0 computed by the library from the unfolded
states of every k equals the oracle chi0 of the original states with its
G-vectors rotated and the phases e^{i (G' - G'').tau} applied."""
import numpy as np
import pytest

import oracle
from oracle import symmetry as sym
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def lattice_op(avec, index):
    A = np.asarray(avec).T
    return np.rint(np.linalg.inv(A) @ sym.cubic_operations()[index] @ A).astype(np.int32)


@pytest.mark.parametrize("index,tau", [(0, (0, 0, 0)), (5, (0.25, 0.25, 0.25)), (13, (0.5, 0.0, 0.25)),
                                       (40, (0.125, 0.375, 0.0))])
def test_unfold_matches_oracle(gpu_lib, index, tau):
    import torch
    p = syn.make_problem("si18_qx")
    R_lat = lattice_op(p.avec, index)
    c = p.coeff[3]
    ref, gref = sym.unfold(c, p.gvec[3], p.avec, R_lat, tau)
    cin = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    cout = torch.empty_like(cin)
    g2 = gpu_lib.bgw_unfold_spinor(p.avec, R_lat, tau, p.gvec[3], cin, cout)
    torch.cuda.synchronize()
    assert np.array_equal(g2, gref)
    assert np.abs(cout.cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max() * 10


def test_chi0_from_unfolded_states(gpu_lib):
    import copy

    import torch
    B = gpu_lib
    p = syn.make_problem("si16_q0")                          # q = 0, 2x2x2 grid, closed N_G shell
    q, geps, nc = p.qs[0]
    R_lat = lattice_op(p.avec, 13)
    tau = np.array([0.25, 0.25, 0.25])
    M = np.rint(np.linalg.inv(R_lat.astype(float)).T).astype(np.int64)   # Miller / k transform
    u = copy.copy(p)
    u.coeff, u.gvec, u.energy = list(p.coeff), list(p.gvec), list(p.energy)
    for j in range(p.nk):
        k2 = M @ p.kcrys[j]
        i = next(i for i in range(p.nk) if np.allclose((k2 - p.kcrys[i]) - np.rint(k2 - p.kcrys[i]), 0))
        G0 = np.rint(k2 - p.kcrys[i]).astype(np.int32)
        cin = torch.from_numpy(np.ascontiguousarray(p.coeff[j])).cuda()
        cout = torch.empty_like(cin)
        g2 = B.bgw_unfold_spinor(p.avec, R_lat, tau, p.gvec[j], cin, cout)
        torch.cuda.synchronize()
        u.coeff[i] = cout.cpu().numpy()
        u.gvec[i] = g2 + G0                                  # the state at Rk = k_i + G0, stored at k_i
        u.energy[i] = p.energy[j]
    ctx = B.Chi0Context(u, "fp64")
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    ref = oracle.chi0(p)
    # chi0'(G', G'') = e^{2 pi i (h' - h'').tau} chi0(R^-1 G', R^-1 G'')
    inv = {tuple(g): n for n, g in enumerate(np.asarray(geps))}
    Minv = np.rint(np.linalg.inv(M.astype(float))).astype(np.int64)
    perm = np.array([inv[tuple(Minv @ g)] for g in np.asarray(geps, np.int64)])
    ph = np.exp(2j * np.pi * (np.asarray(geps) @ tau))
    want = ph[None, :, None] * ref[:, perm][:, :, perm] * ph.conj()[None, None, :]
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
