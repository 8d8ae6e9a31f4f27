"""The allocation-free matrix-element entry point (bgw_mtxel_spinor_noalloc)
against the context-based bgw_mtxel_spinor, through the C-ABI.

It exists for callers that cannot allocate device memory when they need
matrix elements (a pool that owns the device memory, a host application that
forbids cudaMalloc/cudaFree after start-up, loops that must not block in an
allocator); its scratch is one static device array inside the library.
This file is collected last on purpose: it must pass alone in a fresh
process and after every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_M_FP64 = 1e-12


def grids(torch, p, ik, bands):
    """u_{n,k,alpha}(r) = sum_h c(h) e^{+2 pi i h.r/N} on the box (numpy FFT),
    as a device complex128 tensor [nb][2][N^3]."""
    N = np.array(p.box)
    c = p.coeff[ik][bands]
    box = np.zeros((len(c), 2) + p.box, dtype=np.complex128)
    idx = np.mod(p.gvec[ik], N)
    box[:, :, idx[:, 0], idx[:, 1], idx[:, 2]] = c
    u = np.fft.ifftn(box, axes=(2, 3, 4)) * np.prod(N)
    return torch.from_numpy(np.ascontiguousarray(u.reshape(len(c), 2, -1))).cuda()


def compare_with_context(gpu_lib, torch, p, iks):
    """Two (or more) calls in a row of the allocation-free entry point against
    bgw_mtxel_spinor of a context on the same k-points."""
    q, geps, nc = p.qs[0]
    ng = len(geps)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    for ik in iks:
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        ref = torch.zeros((p.nv, nc, ng), dtype=torch.complex128, device="cuda")
        gpu_lib.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, 0, p.nv, 0, nc, ref)
        Uv = grids(torch, p, ik, slice(0, p.nv))
        Uc = grids(torch, p, kp, slice(p.nv, p.nv + nc))
        M = torch.full((p.nv, nc, ng), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        st = gpu_lib.bgw_mtxel_spinor_noalloc(p.box, Uv, Uc, p.nv, nc, G0, geps, M)
        assert st == gpu_lib.BGW_OK
        torch.cuda.synchronize()
        got, want = M.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= TOL_M_FP64 * np.abs(want).max()
    ctx.close()


def test_noalloc_matches_context_mtxel_on_two_calls(gpu_lib):
    torch = pytest.importorskip("torch")
    # an umklapp k first, then a plain one
    compare_with_context(gpu_lib, torch, syn.make_problem("si18_qx"), (4, 0))


@pytest.mark.parametrize("box", [(48, 48, 48), (48, 64, 64)])
def test_noalloc_large_boxes(gpu_lib, box):
    """48^3: the eight-lane kernels with the scatter through the inverse map
    and no z-pass scratch; 48x64x64: the four-lane kernels of non-cubic boxes."""
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx", box=box, ng=137, nv=3, nc=5, nfreq=1)
    compare_with_context(gpu_lib, torch, p, (4, 0))


def test_noalloc_runs_in_valence_blocks(gpu_lib):
    """8 x 200 pairs need about 77 MiB of kernel scratch on the 18^3 box, more
    than the static array: the call runs in blocks of valence bands."""
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx", nc=200)
    compare_with_context(gpu_lib, torch, p, (4, 0))


def test_noalloc_rejects_calls_beyond_its_scratch(gpu_lib):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx")
    geps = p.qs[0][1]
    nbox = int(np.prod(p.box))
    nc = 1400        # one valence band with 1400 conduction bands: about 67 MiB of scratch
    Uv = torch.zeros((1, 2, nbox), dtype=torch.complex128, device="cuda")
    Uc = torch.zeros((nc, 2, nbox), dtype=torch.complex128, device="cuda")
    M = torch.zeros((1, nc, len(geps)), dtype=torch.complex128, device="cuda")
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_mtxel_spinor_noalloc(p.box, Uv, Uc, 1, nc, (0, 0, 0), geps, M)
    assert e.value.status == gpu_lib.BGW_E_ARG and "maximum" in str(e.value)


def test_noalloc_binding_checks_shapes(gpu_lib):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx")
    geps = p.qs[0][1]
    small = torch.zeros(2, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        gpu_lib.bgw_mtxel_spinor_noalloc(p.box, small, small, 2, 3, (0, 0, 0), geps, small)
