"""CUDA-graph capture through the C-ABI: a captured step replays to the same
bits as the eager step; a call that would allocate during capture fails
cleanly and leaves the context usable."""
import numpy as np
import pytest

from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_is_bitwise_equal_to_eager(gpu_lib, prec):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx", nfreq=2)
    ng = len(p.qs[0][1])
    s = torch.cuda.Stream()
    dev = [(torch.from_numpy(np.ascontiguousarray(p.coeff[k])).cuda(),
            torch.from_numpy(np.ascontiguousarray(p.energy[k])).cuda()) for k in range(p.nk)]
    out = torch.zeros((len(p.freq), ng, ng), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ctx = gpu_lib.Chi0Context(p, prec, s)
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_KCHUNK, 4)

    def step():
        ctx.reset()
        ctx.upload(device_inputs=dev)
        ctx.accumulate()
        gpu_lib.bgw_chi0_finalize(ctx.ctx, 0, out)

    step()
    s.synchronize()
    eager = out.cpu().numpy()
    out.zero_()
    torch.cuda.synchronize()
    gpu_lib.bgw_graph_begin(ctx.ctx)
    step()
    gpu_lib.bgw_graph_end(ctx.ctx)
    s.synchronize()
    assert not out.cpu().numpy().any()          # capture ran nothing
    for _ in range(2):
        gpu_lib.bgw_graph_launch(ctx.ctx)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy(), eager)
    ctx.close()


def test_allocation_during_capture_fails_cleanly(gpu_lib):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si16_q0")
    s = torch.cuda.Stream()
    ctx = gpu_lib.Chi0Context(p, "fp64", s)
    gpu_lib.bgw_graph_begin(ctx.ctx)
    with pytest.raises(gpu_lib.BgwError) as e:
        ctx.upload(ks=[0])                       # first upload must allocate scratch
    assert "graph capture" in str(e.value)
    try:
        gpu_lib.bgw_graph_end(ctx.ctx)
    except gpu_lib.BgwError:
        pass
    ctx.upload()                                 # the context works uncaptured again
    ctx.accumulate()
    got = ctx.finalize()
    assert np.isfinite(got).all() and np.abs(got).max() > 0
    ctx.close()
