"""Deferred sphere -> real-space transforms (BGW_OPT_DEFER_K1): the grids the
batched build writes are the ones an eager upload writes, bit for bit, on
boxes where the batched launch applies (cubic, one kernel per band component)
and where it falls back to one transform per k-point; uploads re-made before
the build, host and device inputs, more than one launch's worth of k-points,
graph capture and k-point streaming all keep chi0 equal to the oracle's;
copy-ahead host uploads (a second stream, per-k buffers) give the same grids
and stay correct across steps and graph replays."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _mtxel_all(B, ctx, p, dt):
    import torch
    q, geps, nc = p.qs[0]
    out = []
    for ik in range(p.nk):
        M = torch.zeros((p.nv, nc, len(geps)), dtype=dt, device="cuda")
        B.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, 0, p.nv, 0, nc, M)
        out.append(M.cpu())
    return out


def _device_inputs(p):
    import torch
    return [(torch.from_numpy(np.ascontiguousarray(p.coeff[ik])).cuda(),
             torch.from_numpy(np.ascontiguousarray(p.energy[ik])).cuda()) for ik in range(p.nk)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("box", [(18, 18, 18), (24, 24, 24), (32, 32, 32), (48, 48, 48), (18, 20, 24)])
@pytest.mark.parametrize("on_device", [False, True])
def test_deferred_grids_equal_eager_bitwise(gpu_lib, precision, box, on_device):
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=box, nv=4, nc=6)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    dev = _device_inputs(p) if on_device else None
    got = {}
    for defer in (0, 1):
        ctx = B.Chi0Context(p, precision)
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, defer)
        ctx.upload(device_inputs=dev)
        got[defer] = _mtxel_all(B, ctx, p, dt)
        ctx.close()
    for a, b in zip(got[0], got[1]):
        assert torch.equal(a, b)


def test_reupload_before_build_takes_the_last_coefficients(gpu_lib):
    """A k uploaded twice before the build gets the second coefficients."""
    B = gpu_lib
    p = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    ctx = B.Chi0Context(p, "fp64")
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, 1)
    rng = np.random.default_rng(3)
    for ik in range(p.nk):
        shape = p.coeff[ik].shape
        wrong = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        B.bgw_wfn_upload(ctx.ctx, ik, p.gvec[ik], np.ascontiguousarray(wrong), p.energy[ik])
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_more_than_one_launch_of_k_points(gpu_lib):
    """75 k-points: two batched launches (64 + 11), bitwise the eager grids."""
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", kgrid=(5, 5, 3), q=(0.2, 0, 0), nv=2, nc=3, ecut_wfn=12.0, ng=27)
    got = {}
    for defer in (0, 1):
        ctx = B.Chi0Context(p, "mixed")
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, defer)
        ctx.upload()
        got[defer] = _mtxel_all(B, ctx, p, torch.complex64)
        ctx.close()
    for a, b in zip(got[0], got[1]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_deferred_uploads_inside_a_captured_graph(gpu_lib, precision, tol):
    """Device uploads and the accumulate captured in one graph: the batched
    build runs inside it on every replay, which gives the eager step's bits."""
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=(24, 24, 24), nv=4, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    ng = len(p.qs[0][1])
    dev = _device_inputs(p)
    s = torch.cuda.Stream()
    out = torch.zeros((len(p.freq), ng, ng), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ctx = B.Chi0Context(p, precision, s)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, 1)

    def step():
        ctx.reset()
        ctx.upload(device_inputs=dev)
        ctx.accumulate()
        B.bgw_chi0_finalize(ctx.ctx, 0, out)

    step()
    s.synchronize()
    eager = out.cpu().numpy()
    assert np.linalg.norm(eager - ref) <= tol * np.linalg.norm(ref)
    out.zero_()
    torch.cuda.synchronize()
    B.bgw_graph_begin(ctx.ctx)
    step()
    B.bgw_graph_end(ctx.ctx)
    s.synchronize()
    assert not out.cpu().numpy().any()          # capture ran nothing
    for _ in range(2):
        B.bgw_graph_launch(ctx.ctx)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy(), eager)
    ctx.close()


def test_defer_is_inert_with_k_point_streaming(gpu_lib):
    B = gpu_lib
    p = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    ctx = B.Chi0Context(p, "fp64")
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_GRID_SLOTS, 3)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, 1)
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def _pinned_inputs(p, coeff=None):
    import torch
    coeff = p.coeff if coeff is None else coeff
    return [(torch.from_numpy(np.ascontiguousarray(coeff[ik])).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(p.energy[ik])).pin_memory()) for ik in range(p.nk)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
@pytest.mark.parametrize("defer", [0, 1])
def test_copy_ahead_host_uploads_over_two_steps(gpu_lib, precision, tol, defer):
    """Copy-ahead host uploads (BGW_OPT_COPY_AHEAD): a step on other
    coefficients, then a step on the problem's; the second reuses every
    k's device buffer after the first step's transforms read it."""
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=(24, 24, 24), nv=4, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    rng = np.random.default_rng(11)
    other = [rng.normal(size=c.shape) + 1j * rng.normal(size=c.shape) for c in p.coeff]
    s = torch.cuda.Stream()
    ctx = B.Chi0Context(p, precision, s)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_COPY_AHEAD, 1)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, defer)
    first, second = _pinned_inputs(p, other), _pinned_inputs(p)
    ctx.upload(device_inputs=first)
    ctx.accumulate()
    ctx.reset()
    ctx.upload(device_inputs=second)
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_copy_ahead_grids_equal_stream_ordered_copies(gpu_lib):
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=(20, 20, 20), nv=4, nc=6)
    pin = _pinned_inputs(p)
    got = {}
    for ahead in (0, 1):
        ctx = B.Chi0Context(p, "fp64")
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_COPY_AHEAD, ahead)
        ctx.upload(device_inputs=pin)
        got[ahead] = _mtxel_all(B, ctx, p, torch.complex128)
        ctx.close()
    for a, b in zip(got[0], got[1]):
        assert torch.equal(a, b)


def test_copy_ahead_after_graph_replays(gpu_lib):
    """Host uploads captured in a graph use the stream-ordered copy; a
    copy-ahead upload after the replays waits for them, and a later replay
    still gives the eager bits."""
    import torch
    B = gpu_lib
    p = syn.make_problem("si18_qx", box=(24, 24, 24), nv=4, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    ng = len(p.qs[0][1])
    pin = _pinned_inputs(p)
    s = torch.cuda.Stream()
    out = torch.zeros((len(p.freq), ng, ng), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ctx = B.Chi0Context(p, "mixed", s)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_COPY_AHEAD, 1)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, 1)

    def step():
        ctx.reset()
        ctx.upload(device_inputs=pin)
        ctx.accumulate()
        B.bgw_chi0_finalize(ctx.ctx, 0, out)

    step()
    s.synchronize()
    eager = out.cpu().numpy()
    assert np.linalg.norm(eager - ref) <= 2e-5 * np.linalg.norm(ref)
    B.bgw_graph_begin(ctx.ctx)
    step()
    B.bgw_graph_end(ctx.ctx)
    B.bgw_graph_launch(ctx.ctx)
    step()                                          # copy-ahead again, after the replay
    B.bgw_graph_launch(ctx.ctx)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), eager)
    ctx.close()


def test_option_values(gpu_lib):
    B = gpu_lib
    p = syn.make_problem("si16_q0", nv=2, nc=2)
    ctx = B.Chi0Context(p, "fp64")
    for opt in (B.BGW_OPT_DEFER_K1, B.BGW_OPT_COPY_AHEAD):
        assert B.bgw_get_option(ctx.ctx, opt) == 0
        B.bgw_set_option(ctx.ctx, opt, 1)
        assert B.bgw_get_option(ctx.ctx, opt) == 1
        for bad in (-1, 2):
            with pytest.raises(B.BgwError):
                B.bgw_set_option(ctx.ctx, opt, bad)
        assert B.bgw_get_option(ctx.ctx, opt) == 1
    ctx.close()
