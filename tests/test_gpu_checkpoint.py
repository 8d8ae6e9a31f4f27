"""Checkpoint / resume of a running sum and allocation-failure injection.

Resume + the remaining k-blocks equals one uninterrupted run over the same
blocks bitwise (the k sum is linear and each block adds into the FP64
accumulators in a fixed order); a checkpoint of another problem or a cut
buffer is refused; an injected out-of-memory makes the call that needed the
allocation return BGW_E_NOMEM and the context keeps working."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_equals_one_shot_bitwise(gpu_lib, precision):
    B = gpu_lib
    p = syn.make_problem("si18_qx")
    split = 4
    one = B.Chi0Context(p, precision)
    B.bgw_set_option(one.ctx, B.BGW_OPT_KCHUNK, 2)
    one.upload()
    one.accumulate(0, split)
    one.accumulate(split, p.nk)
    ref = one.finalize()
    one.close()

    first = B.Chi0Context(p, precision)
    B.bgw_set_option(first.ctx, B.BGW_OPT_KCHUNK, 2)
    first.upload()
    first.accumulate(0, split)
    ck = B.bgw_chi0_checkpoint(first.ctx)
    assert list(B.bgw_chi0_progress(first.ctx, p.nk)) == [1] * split + [0] * (p.nk - split)
    first.close()

    second = B.Chi0Context(p, precision)
    B.bgw_set_option(second.ctx, B.BGW_OPT_KCHUNK, 2)
    second.upload()
    B.bgw_chi0_resume(second.ctx, second.qlist(), p.freq, ck)
    assert list(B.bgw_chi0_progress(second.ctx, p.nk)) == [1] * split + [0] * (p.nk - split)
    second.accumulate(split, p.nk)
    got = second.finalize()
    assert list(B.bgw_chi0_progress(second.ctx, p.nk)) == [1] * p.nk
    second.close()
    assert np.array_equal(got, ref)
    if precision == "fp64":
        o = oracle.chi0(p)
        assert np.linalg.norm(got - o) <= 1e-10 * np.linalg.norm(o)


def test_resume_refuses_other_problem_and_cut_buffer(gpu_lib):
    B = gpu_lib
    p = syn.make_problem("si18_qx")
    ctx = B.Chi0Context(p, "fp64")
    ctx.upload()
    ctx.accumulate(0, 2)
    ck = B.bgw_chi0_checkpoint(ctx.ctx)
    with pytest.raises(B.BgwError) as e:
        B.bgw_chi0_resume(ctx.ctx, ctx.qlist(), p.freq + 1.0, ck)      # other frequencies
    assert e.value.status == B.BGW_E_STATE
    with pytest.raises(B.BgwError) as e:
        B.bgw_chi0_resume(ctx.ctx, ctx.qlist(), p.freq, ck[:len(ck) // 2])
    assert e.value.status == B.BGW_E_ARG
    with pytest.raises(B.BgwError) as e:
        B.bgw_chi0_resume(ctx.ctx, ctx.qlist(), p.freq, b"x" * len(ck))
    assert e.value.status == B.BGW_E_ARG
    ctx.close()


def test_injected_out_of_memory_is_reported_and_recoverable(gpu_lib):
    B = gpu_lib
    p = syn.make_problem("si16_q0")
    ctx = B.Chi0Context(p, "fp64")
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_TEST_FAIL_ALLOC, 1)       # the next allocation fails
    with pytest.raises(B.BgwError) as e:
        ctx.upload(ks=[0])
    assert e.value.status == B.BGW_E_NOMEM
    assert B.bgw_get_option(ctx.ctx, B.BGW_OPT_TEST_FAIL_ALLOC) == 0
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    ref = oracle.chi0(p)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
