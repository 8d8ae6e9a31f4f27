"""Both sphere -> real-space kernel paths (one kernel per axis, and one
kernel for the whole transform of a band component) give matrix elements
that match the oracle, FP64 and FP32, with and without the umklapp shift."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 5e-6)])
@pytest.mark.parametrize("name,overrides", [("si18_qx", {}), ("si16_q0", {"box": (20, 20, 20)})])
def test_k1_paths_match_oracle(gpu_lib, path, precision, tol, name, overrides):
    import torch
    B = gpu_lib
    p = syn.make_problem(name, **overrides)
    q, geps, nc = p.qs[0]
    ctx = B.Chi0Context(p, precision)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_K1_PATH, path)
    ctx.upload()
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    for ik in (0, p.nk - 1):
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        M = torch.zeros((p.nv, nc, len(geps)), dtype=dt, device="cuda")
        B.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, 0, p.nv, 0, nc, M)
        ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:p.nv], p.gvec[kp],
                           p.coeff[kp][p.nv:p.nv + nc], G0, geps)
        assert np.abs(M.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    ctx.close()
