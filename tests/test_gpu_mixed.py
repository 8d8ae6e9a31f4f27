"""GPU parity of the mixed-precision path (FP32 grids and matrix elements,
split-BF16 tensor-core contraction with FP64 weights and FP64 reduction over
k) against the CPU FP64 oracle.  Bars: M within 5e-6 of max|M| elementwise;
chi0 within 2e-5 relative Frobenius, overall and per frequency.  The TF32
forms of the contraction: three products (BGW_MIXED_TF32X3) to the same 2e-5;
one product (BGW_MIXED_TF32) to 1e-3, twice the unit roundoff 2^-11 of an
operand rounded to 11 significant bits (each term x_r (w x_r') carries two
such roundings; cancellation between terms is not counted)."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_M_FP32 = 5e-6
TOL_CHI_MIXED = 2e-5
TOL_CHI = {"mixed": TOL_CHI_MIXED, "tf32x3": TOL_CHI_MIXED, "tf32": 2 * 2.0 ** -11}


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def run(gpu_lib, p, chunks=None, prec="mixed"):
    ctx = gpu_lib.Chi0Context(p, prec)
    ctx.upload()
    st = [ctx.accumulate(k0, k1) for k0, k1 in (chunks or [(0, p.nk)])]
    out = ctx.finalize()
    ctx.close()
    return out, st


def test_mtxel_fp32_matches_oracle(gpu_lib):
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx")
    q, geps, nc = p.qs[0]
    ctx = gpu_lib.Chi0Context(p, "mixed")
    ctx.upload()
    for ik in (0, 4):
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        M = torch.zeros((p.nv, nc, len(geps)), dtype=torch.complex64, device="cuda")
        gpu_lib.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, 0, p.nv, 0, nc, M)
        ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:p.nv], p.gvec[kp],
                           p.coeff[kp][p.nv:p.nv + nc], G0, geps)
        assert np.abs(M.cpu().numpy() - ref).max() <= TOL_M_FP32 * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("name", ["si16_q0", "si18_qx"])
def test_chi0_mixed_matches_oracle(gpu_lib, name):
    p = syn.make_problem(name)
    ref = oracle.chi0(p)
    got, _ = run(gpu_lib, p)
    assert rel_fro(got, ref) <= TOL_CHI_MIXED
    for j in range(len(p.freq)):
        assert rel_fro(got[j], ref[j]) <= TOL_CHI_MIXED


def test_chi0_mixed_ragged_multi_frequency(gpu_lib):
    """ng = 59 (2*ng = 118 rows: one partial 128-row tile), 13 conduction bands
    (104 pairs: a partial 64-pair block), 3 frequencies."""
    p = syn.make_problem("si18_qx", ng=59, nc=13, nfreq=3)
    ref = oracle.chi0(p)
    got, _ = run(gpu_lib, p)
    assert rel_fro(got, ref) <= TOL_CHI_MIXED


def test_chi0_mixed_several_row_tiles(gpu_lib):
    """ng = 200: 400 real rows -> 4 row tiles, 10 lower tiles."""
    p = syn.make_problem("si18_qx", ng=200, nfreq=2)
    ref = oracle.chi0(p)
    got, _ = run(gpu_lib, p)
    assert rel_fro(got, ref) <= TOL_CHI_MIXED


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
@pytest.mark.parametrize("shape", [
    {},                                   # si18_qx defaults
    {"ng": 59, "nc": 13, "nfreq": 3},     # one partial row tile, a partial pair block
    {"ng": 200, "nfreq": 2},              # 4 row tiles, 10 lower tiles
])
def test_chi0_tf32_contraction_matches_oracle(gpu_lib, prec, shape):
    p = syn.make_problem("si18_qx", **shape)
    ref = oracle.chi0(p)
    got, _ = run(gpu_lib, p, prec=prec)
    err = rel_fro(got, ref)
    assert err <= TOL_CHI[prec]
    for j in range(len(p.freq)):
        assert rel_fro(got[j], ref[j]) <= TOL_CHI[prec]
    if prec == "tf32":
        assert err > 1e-7          # the single product is visibly coarser than the split forms


def test_chi0_tf32x3_k_chunking_is_bitwise_identical(gpu_lib):
    p = syn.make_problem("si18_qx")
    one, _ = run(gpu_lib, p, prec="tf32x3")
    chunked, _ = run(gpu_lib, p, chunks=[(0, 3), (3, 8)], prec="tf32x3")
    assert np.array_equal(one, chunked)


def test_chi0_mixed_k_chunking_is_bitwise_identical(gpu_lib):
    p = syn.make_problem("si18_qx")
    one, _ = run(gpu_lib, p)
    chunked, _ = run(gpu_lib, p, chunks=[(0, 5), (5, 8)])
    assert np.array_equal(one, chunked)


def test_chi0_mixed_si24_k_subset(gpu_lib):
    p = syn.make_problem("si24")
    ks = [0, 12]
    ref = oracle.chi0(p, k_indices=ks)
    ctx = gpu_lib.Chi0Context(p, "mixed")
    ctx.upload()
    for k in ks:
        ctx.accumulate(k, k + 1)
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, ref) <= TOL_CHI_MIXED


@pytest.mark.parametrize("zy", [1, 2])
@pytest.mark.parametrize("over", [{}, dict(box=(24, 24, 24), nv=9, nc=30, ng=113, nfreq=2),
                                  dict(box=(32, 32, 32), nv=5, nc=13, ng=181, nfreq=2),
                                  dict(box=(20, 20, 20), nv=6, nc=7, ng=89, nfreq=1),
                                  dict(box=(16, 16, 16), nv=3, nc=9, ng=59, nfreq=1)])
def test_both_zy_kernels_match_oracle(gpu_lib, zy, over):
    """The FP32 pair density + z + y passes as the plane kernel (pair tiles)
    and as the streamed kernel (resident valence planes, conduction planes in
    double-buffered groups; ragged last groups here) against the oracle."""
    p = syn.make_problem("si18_qx", **over)
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, "mixed")
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_MTXEL_ZY, zy)
    ctx.upload()
    ctx.accumulate()
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, ref) <= TOL_CHI_MIXED



@pytest.mark.parametrize("shift", [(0, 0, 0), (0, 0, 7), (0, 7, 0)])
def test_streamed_zy_kernel_off_centre_sphere(gpu_lib, shift):
    """M of the streamed z + y kernel on a 32^3 box (TMA staging) element by
    element against the oracle for a G set shifted off centre: (0, 0, 0)
    keeps every output within 8 of zero (the pruned store window), the other
    two put kept z or y outputs outside it (the full store loop)."""
    torch = pytest.importorskip("torch")
    p = syn.make_problem("si18_qx", box=(32, 32, 32), nv=5, nc=9, ng=181, nfreq=1)
    q, geps, _ = p.qs[0]
    g = np.ascontiguousarray(geps + np.asarray(shift, dtype=geps.dtype))
    nc = 9
    ctx = gpu_lib.Chi0Context(p, "mixed")
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_MTXEL_ZY, 2)
    ctx.upload()
    for ik in (0, 4):
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        M = torch.zeros((p.nv, nc, len(g)), dtype=torch.complex64, device="cuda")
        gpu_lib.bgw_mtxel_spinor(ctx.ctx, q, g, ik, 0, p.nv, 0, nc, M)
        ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:p.nv], p.gvec[kp],
                           p.coeff[kp][p.nv:p.nv + nc], G0, g)
        assert np.abs(M.cpu().numpy() - ref).max() <= TOL_M_FP32 * np.abs(ref).max()
    ctx.close()
