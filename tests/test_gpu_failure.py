"""Failure detection without a GPU fault: a mixed contraction that loses one
operand load on purpose (test hook) lets its bounded device waits expire;
the kernel unwinds, frees its tensor memory and records an error, the host
finalize reports BGW_E_TIMEOUT, and the same context then computes a
correct result."""
import time

import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_dropped_load_reports_timeout_and_context_recovers(gpu_lib):
    p = syn.make_problem("si18_qx")
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, "mixed")
    ctx.upload()
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_TEST_DROP_LOAD, 1)
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_KCHUNK, p.nk)   # one contraction launch
    ctx.accumulate()
    t0 = time.time()
    with pytest.raises(gpu_lib.BgwError) as e:
        ctx.finalize()
    assert e.value.status == gpu_lib.BGW_E_TIMEOUT
    assert time.time() - t0 < 60
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_TEST_DROP_LOAD, 0)
    ctx.reset()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5


def test_dropped_plane_copy_of_the_zy_kernel_reports_timeout(gpu_lib):
    """The streamed z + y kernel of a 32^3 box receives its band planes by TMA
    onto mbarriers; with the test hook its first CTA never issues one copy, the
    bounded wait gives up (~2 s), the host finalize reports BGW_E_TIMEOUT and
    the same context then computes a correct result."""
    p = syn.make_problem("si18_qx", box=(32, 32, 32), nv=5, nc=13, ng=181, nfreq=2)
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, "mixed")
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_MTXEL_ZY, 2)
    ctx.upload()
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_TEST_DROP_LOAD, 2)
    ctx.accumulate(0, 1)
    t0 = time.time()
    with pytest.raises(gpu_lib.BgwError) as e:
        ctx.finalize()
    assert e.value.status == gpu_lib.BGW_E_TIMEOUT
    assert time.time() - t0 < 60
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_TEST_DROP_LOAD, 0)
    ctx.reset()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-5


def test_drop_load_option_range(gpu_lib):
    p = syn.make_problem("si18_qx")
    ctx = gpu_lib.Chi0Context(p, "mixed")
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_TEST_DROP_LOAD, 3)
    assert e.value.status == gpu_lib.BGW_E_ARG
    ctx.close()
