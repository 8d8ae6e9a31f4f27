"""Tuning options and the autotuner change speed, not results: k-chunked
contraction and explicit pair tiles against the oracle and against the
default settings."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5}


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.fixture(scope="module")
def case():
    p = syn.make_problem("si18_qx", nfreq=2)
    return p, oracle.chi0(p)


def run(gpu_lib, p, prec, opts=(), chunks=None):
    ctx = gpu_lib.Chi0Context(p, prec)
    for o, v in opts:
        gpu_lib.bgw_set_option(ctx.ctx, o, v)
    ctx.upload()
    for k0, k1 in (chunks or [(0, p.nk)]):
        ctx.accumulate(k0, k1)
    out = ctx.finalize()
    ctx.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kchunk", [2, 3, 8])
def test_kchunk_matches_oracle(gpu_lib, case, prec, kchunk):
    p, ref = case
    got = run(gpu_lib, p, prec, [(gpu_lib.BGW_OPT_KCHUNK, kchunk)])
    assert rel_fro(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_kchunk_aligned_splits_are_bitwise_identical(gpu_lib, case, prec):
    p, _ = case
    opt = [(gpu_lib.BGW_OPT_KCHUNK, 2)]
    one = run(gpu_lib, p, prec, opt)
    split = run(gpu_lib, p, prec, opt, chunks=[(0, 2), (2, 6), (6, 8)])
    assert np.array_equal(one, split)


@pytest.mark.parametrize("tile", [(1, 1), (2, 3), (8, 2), (2, 2), (8, 8)])
def test_pair_tiles_give_identical_results(gpu_lib, case, tile):
    p, _ = case
    auto = run(gpu_lib, p, "mixed", [(gpu_lib.BGW_OPT_MTXEL_ZY, 1)])      # plane kernel, automatic tile
    got = run(gpu_lib, p, "mixed", [(gpu_lib.BGW_OPT_PAIR_TILE_V, tile[0]),
                                    (gpu_lib.BGW_OPT_PAIR_TILE_C, tile[1])])
    assert np.array_equal(got, auto)


def test_autotune_keeps_results_and_uses_cache(gpu_lib, case, tmp_path):
    p, ref = case
    cache = str(tmp_path / "tune.txt")
    for prec in ("fp64", "mixed"):
        ctx = gpu_lib.Chi0Context(p, prec)
        ctx.upload()
        ctx.accumulate(0, 3)                     # a running sum the autotuner must not touch
        choice = ctx.autotune(cache_path=cache)
        assert choice["kchunk"] >= 1 and choice["mtxel_zy"] in (0, 1, 2)
        ctx.accumulate(3, 8)                     # the sum continues with the tuned settings
        got = ctx.finalize()
        ctx.close()
        assert rel_fro(got, ref) <= TOL[prec]
        # a second context reads the cached choice
        ctx2 = gpu_lib.Chi0Context(p, prec)
        ctx2.upload()
        assert ctx2.autotune(cache_path=cache) == choice
        ctx2.close()
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 2 and all("|" in l for l in lines)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_profile_splits_the_matrix_element_stages(gpu_lib, prec):
    """bgw_profile times the pair density + z + y kernels (stage 1) apart from
    the x pass with the sphere gather (stage 6): both non-empty, one x-pass
    kernel per launch group and at least one group per k-point."""
    p = syn.make_problem("si18_qx")
    ctx = gpu_lib.Chi0Context(p, prec)
    ctx.upload()
    ctx.accumulate()
    ctx.reset()
    gpu_lib.bgw_profile(ctx.ctx, True)
    ctx.accumulate()
    prof = gpu_lib.bgw_profile_read(ctx.ctx)
    gpu_lib.bgw_profile(ctx.ctx, False)
    ctx.close()
    zy, x = prof["mtxel"], prof["mtxel_x"]
    assert zy[0] > 0 and x[0] > 0
    assert x[2] == x[1] >= p.nk
    assert zy[2] >= zy[1] >= p.nk
