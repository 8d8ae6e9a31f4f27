"""Every kernel path of the sphere -> real-space transform and of the matrix
elements (one kernel per axis, one kernel per band component, eight lanes per
FFT line) gives matrix elements that match the oracle, FP64 and FP32, with and
without the umklapp shift, on boxes each path takes (or falls back from)."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k1_path,lanes", [(1, 1), (2, 0), (3, 8), (4, 0)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 5e-6)])
@pytest.mark.parametrize("name,overrides", [("si18_qx", {}), ("si16_q0", {"box": (20, 20, 20)}),
                                            ("si18_qx", {"box": (32, 32, 32)}),
                                            ("si18_qx", {"box": (40, 40, 40), "nv": 4, "nc": 7})])
def test_k1_and_mtxel_paths_match_oracle(gpu_lib, k1_path, lanes, precision, tol, name, overrides):
    import torch
    B = gpu_lib
    p = syn.make_problem(name, **overrides)
    q, geps, nc = p.qs[0]
    ctx = B.Chi0Context(p, precision)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_K1_PATH, k1_path)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_MTXEL_LANES, lanes)
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_chi0_with_eight_lanes_at_32_matches_oracle(gpu_lib, precision, tol):
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=(32, 32, 32), ng=89, nv=4, nc=9, nfreq=2)
    ref = oracle.chi0(p)
    ctx = B.Chi0Context(p, precision)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_K1_PATH, 3)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_MTXEL_LANES, 8)
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
