"""k-point streaming (real-space grids rebuilt into a few device slots) gives
the same bits as keeping every grid resident; the scatter form of the last
FFT pass (wide dielectric spheres) matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def run(gpu_lib, p, prec, slots=0, kchunk=1, device_inputs=None):
    ctx = gpu_lib.Chi0Context(p, prec)
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_GRID_SLOTS, slots)
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_KCHUNK, kchunk)
    ctx.upload(device_inputs=device_inputs)
    ctx.accumulate()
    out = ctx.finalize()
    assert gpu_lib.bgw_get_option(ctx.ctx, gpu_lib.BGW_OPT_GRID_SLOTS) == (slots or p.nk)
    ctx.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("slots, kchunk", [(2, 1), (3, 4)])
def test_streaming_is_bitwise_equal_to_resident(gpu_lib, prec, slots, kchunk):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx", nfreq=2)
    resident = run(gpu_lib, p, prec, 0, kchunk)
    dev = [(torch.from_numpy(np.ascontiguousarray(p.coeff[k])).cuda(),
            torch.from_numpy(np.ascontiguousarray(p.energy[k])).cuda()) for k in range(p.nk)]
    streamed_dev = run(gpu_lib, p, prec, slots, kchunk, device_inputs=dev)
    streamed_host = run(gpu_lib, p, prec, slots, kchunk)
    assert np.array_equal(streamed_dev, resident)
    assert np.array_equal(streamed_host, resident)


def test_grid_slots_fixed_after_first_upload(gpu_lib):
    p = syn.make_problem("si16_q0")
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload(ks=[0])
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_GRID_SLOTS, 2)
    assert e.value.status == gpu_lib.BGW_E_STATE
    ctx.close()


@pytest.mark.parametrize("prec, box, ng", [("fp64", (18, 18, 18), 2000), ("mixed", (24, 24, 24), 3000)])
def test_wide_dielectric_sphere_scatter_path(gpu_lib, prec, box, ng):
    """A kept cube above 64 KB is written through the inverse map."""
    p = syn.make_problem("si18_qx", box=box, ng=ng, nv=3, nc=6, nfreq=2)
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, prec)
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, ref) <= (1e-10 if prec == "fp64" else 2e-5)
