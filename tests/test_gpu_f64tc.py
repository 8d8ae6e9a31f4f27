"""The FP64 path's contraction on tcgen05 tensor cores (exact BF16 digit
slices of sqrt(-w) (Re M, Im M), the default) against the CPU FP64 oracle
and against the FP64 FMA kernel (BGW_OPT_FP64_CONTRACTION = 1): chi0 within
1e-10 relative Frobenius, overall and per frequency, on a launch long enough
to fold its integer sums into FP64 mid-item (more than 128 x 224 pairs)."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def run(gpu_lib, p, dfma, kchunk=1, chunks=None):
    ctx = gpu_lib.Chi0Context(p, "fp64")
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_FP64_CONTRACTION, 1 if dfma else 0)
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_KCHUNK, kchunk)
    ctx.upload()
    for k0, k1 in (chunks or [(0, p.nk)]):
        ctx.accumulate(k0, k1)
    out = ctx.finalize()
    ctx.close()
    return out


@pytest.mark.parametrize("name, over", [("si16_q0", {}), ("si18_qx", dict(nfreq=3, ng=59, nc=13))])
def test_tensor_core_fp64_matches_oracle(gpu_lib, name, over):
    p = syn.make_problem(name, **over)
    ref = oracle.chi0(p)
    got = run(gpu_lib, p, dfma=False, kchunk=4)
    assert rel_fro(got, ref) <= TOL
    for j in range(len(p.freq)):
        assert rel_fro(got[j], ref[j]) <= TOL
    assert np.array_equal(got, run(gpu_lib, p, dfma=False, kchunk=4))     # deterministic


def test_long_launch_against_fma_kernel_and_sampled_oracle(gpu_lib):
    """8 k x 16 x 400 pairs in one launch: 229 promotions of 224 pairs, so the
    int32 sums are folded into FP64 after 128 of them and again at the end."""
    p = syn.make_problem("si18_qx", nv=16, nc=400, ng=137, nfreq=2)
    tc = run(gpu_lib, p, dfma=False, kchunk=8)
    fma = run(gpu_lib, p, dfma=True, kchunk=8)
    assert rel_fro(tc, fma) <= TOL
    S = np.array([0, 1, 17, 60, 99, 136])
    ref = oracle.chi0(p, g_indices=S)
    blk = tc[:, S][:, :, S]
    assert rel_fro(blk, ref) <= TOL


def test_positive_weight_is_reported_not_dropped(gpu_lib):
    """An occupied band above an empty one gives a positive pair weight: the
    digit form cannot take it, finalize says so; the FMA kernel sums it."""
    p = syn.make_problem("si18_qx", nv=2, nc=3, ng=27)
    p.energy = [e.copy() for e in p.energy]
    p.energy[4][1] = 7.0        # valence band 1 at k = 4 above conduction band 0 (5.8 eV) of its k + q
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    ctx.accumulate()
    with pytest.raises(gpu_lib.BgwError) as e:
        ctx.finalize()
    assert e.value.status == gpu_lib.BGW_E_ARG and "positive" in str(e.value)
    ctx.close()
    got = run(gpu_lib, p, dfma=True)
    assert rel_fro(got, ref) <= TOL
