"""Overlapped mixed contraction (BGW_OPT_OVERLAP): weights, operand split
and contraction of each block of matrix elements run on a second stream
while the next block's matrix elements are computed, the blocks alternating
between two M buffers.  The launches sum into every accumulator in the same
order, so chi0 must be bitwise the plain path's: for one q and for a ragged
multi-q batch, over k-chunks that give many blocks (each buffer reused
several times), across accumulate calls, inside a captured graph, and for
the autotuner."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _run(B, p, kchunk, overlap, stream=None, splits=None):
    ctx = B.Chi0Context(p, "mixed", stream)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_KCHUNK, kchunk)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, overlap)
    ctx.upload()
    bounds = splits or [0, p.nk]
    for a, b in zip(bounds[:-1], bounds[1:]):
        ctx.accumulate(a, b)
    out = [ctx.finalize(iq) for iq in range(len(p.qs))]
    ctx.close()
    return out


@pytest.mark.parametrize("kchunk", [1, 2, 3])
def test_overlap_is_bitwise_the_plain_path(gpu_lib, kchunk):
    p = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=3)
    ref = oracle.chi0(p)
    plain = _run(gpu_lib, p, kchunk, 0)
    over = _run(gpu_lib, p, kchunk, 1)
    assert np.array_equal(plain[0], over[0])
    assert np.linalg.norm(over[0] - ref) <= 2e-5 * np.linalg.norm(ref)


def test_overlap_over_split_accumulate_calls(gpu_lib):
    p = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=2)
    plain = _run(gpu_lib, p, 2, 0)
    over = _run(gpu_lib, p, 2, 1, splits=[0, 2, 6, 8])
    assert np.array_equal(plain[0], over[0])


def test_overlap_ragged_batch(gpu_lib):
    p = syn.make_batched_problem(config_id=7, a=10.26, box=(18, 18, 18), ecut_wfn=28.1,
                                 kgrid=(2, 2, 2), nv=8, nq=5, ng_range=(20, 150),
                                 nc_range=(5, 24), nfreq=3, precision="mixed")
    plain = _run(gpu_lib, p, 1, 0)
    over = _run(gpu_lib, p, 1, 1)
    for a, b in zip(plain, over):
        assert np.array_equal(a, b)


def test_overlap_in_a_captured_graph(gpu_lib):
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=(24, 24, 24), nv=4, nc=6, nfreq=2)
    ng = len(p.qs[0][1])
    plain = _run(B, p, 2, 0)[0]
    s = torch.cuda.Stream()
    out = torch.zeros((len(p.freq), ng, ng), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ctx = B.Chi0Context(p, "mixed", s)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_KCHUNK, 2)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, 1)

    def step():
        ctx.reset()
        ctx.accumulate()
        B.bgw_chi0_finalize(ctx.ctx, 0, out)

    ctx.upload()
    step()
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), plain)
    out.zero_()
    torch.cuda.synchronize()
    B.bgw_graph_begin(ctx.ctx)
    step()
    with pytest.raises(B.BgwError):
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, 0)     # fixed while capturing
    B.bgw_graph_end(ctx.ctx)
    for _ in range(2):
        B.bgw_graph_launch(ctx.ctx)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy(), plain)
    ctx.close()


def test_overlap_with_autotune(gpu_lib):
    p = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, "mixed")
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_OVERLAP, 1)
    ctx.upload()
    ctx.autotune(0, 4)
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) <= 2e-5 * np.linalg.norm(ref)
