"""Large boxes: cubic 48^3 and 64^3 use the eight-lanes-per-line FFT
kernels, non-cubic boxes of those lengths the four-lane ones (and the
one-line-per-thread sphere-to-grid passes): parity with the oracle in both
precisions."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("box", [(48, 48, 48), (64, 64, 64), (48, 64, 64)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_box_chi0_matches_oracle(gpu_lib, box, prec):
    p = syn.make_problem("si18_qx", box=box, ng=89, nv=4, nc=9, nfreq=2)
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, prec)
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, ref) <= (1e-10 if prec == "fp64" else 2e-5)


def test_large_box_mtxel_elementwise(gpu_lib):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx", box=(64, 64, 64), ng=137, nv=3, nc=5, nfreq=1)
    q, geps, nc = p.qs[0]
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    for ik in (0, 4):
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        M = torch.zeros((p.nv, nc, len(geps)), dtype=torch.complex128, device="cuda")
        gpu_lib.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, 0, p.nv, 0, nc, M)
        ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:p.nv], p.gvec[kp],
                           p.coeff[kp][p.nv:p.nv + nc], G0, geps)
        assert np.abs(M.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.close()
