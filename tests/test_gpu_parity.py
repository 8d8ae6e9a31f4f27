"""GPU parity: the CUDA path through the C-ABI against the CPU FP64 oracle on
the same seeded inputs.  Bars: M elementwise within 1e-12 of max|M| and chi0
within 1e-10 relative Frobenius (FP64 path)."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_M_FP64 = 1e-12
TOL_CHI_FP64 = 1e-10


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def problems():
    return {name: syn.make_problem(name) for name in ["si16_q0", "si18_qx"]}


@pytest.fixture(scope="module")
def oracle_chi(problems):
    return {name: oracle.chi0(p) for name, p in problems.items()}


def run_chi0(gpu_lib, p, precision="fp64", chunks=None):
    ctx = gpu_lib.Chi0Context(p, precision)
    ctx.upload()
    for k0, k1 in (chunks or [(0, p.nk)]):
        ctx.accumulate(k0, k1)
    out = ctx.finalize()
    ctx.close()
    return out


# ------------------------------------------------------------------- mtxel --

@pytest.mark.parametrize("name, iks", [("si16_q0", [0, 5]), ("si18_qx", [0, 4, 7])])
def test_mtxel_fp64_matches_oracle(gpu_lib, torch_cuda, problems, name, iks):
    torch = torch_cuda
    p = problems[name]
    q, geps, nc = p.qs[0]
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    for ik in iks:
        kp, G0 = oracle.umklapp(p.kcrys, ik, q)
        M = torch.zeros((p.nv, nc, len(geps)), dtype=torch.complex128, device="cuda")
        st = gpu_lib.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, 0, p.nv, 0, nc, M)
        assert st == gpu_lib.BGW_OK
        ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][:p.nv], p.gvec[kp],
                           p.coeff[kp][p.nv:p.nv + nc], G0, geps)
        got = M.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL_M_FP64 * np.abs(ref).max()
    ctx.close()


def test_mtxel_band_subranges(gpu_lib, torch_cuda, problems):
    torch = torch_cuda
    p = problems["si18_qx"]
    q, geps, nc = p.qs[0]
    ik = 4
    kp, G0 = oracle.umklapp(p.kcrys, ik, q)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    v0, nv, c0, ncs = 3, 2, 5, 7
    M = torch.zeros((nv, ncs, len(geps)), dtype=torch.complex128, device="cuda")
    gpu_lib.bgw_mtxel_spinor(ctx.ctx, q, geps, ik, v0, nv, c0, ncs, M)
    ref = oracle.mtxel(p.box, p.gvec[ik], p.coeff[ik][v0:v0 + nv], p.gvec[kp],
                       p.coeff[kp][p.nv + c0:p.nv + c0 + ncs], G0, geps)
    assert np.abs(M.cpu().numpy() - ref).max() <= TOL_M_FP64 * np.abs(ref).max()
    ctx.close()


def test_mtxel_orthonormality_on_gpu(gpu_lib, torch_cuda, problems):
    """q = 0, G = 0: M_vc = <v|c> = 0 for the orthonormal synthetic bands."""
    torch = torch_cuda
    p = problems["si16_q0"]
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    M = torch.zeros((p.nv, p.nc, 1), dtype=torch.complex128, device="cuda")
    gpu_lib.bgw_mtxel_spinor(ctx.ctx, (0, 0, 0), np.zeros((1, 3)), 3, 0, p.nv, 0, p.nc, M)
    assert np.abs(M.cpu().numpy()).max() < 1e-13
    ctx.close()


# -------------------------------------------------------------------- chi0 --

@pytest.mark.parametrize("name", ["si16_q0", "si18_qx"])
def test_chi0_fp64_matches_oracle(gpu_lib, problems, oracle_chi, name):
    p = problems[name]
    got = run_chi0(gpu_lib, p)
    ref = oracle_chi[name]
    assert rel_fro(got, ref) <= TOL_CHI_FP64
    for j in range(len(p.freq)):
        assert rel_fro(got[j], ref[j]) <= TOL_CHI_FP64
    assert np.array_equal(got[0], got[0].conj().T)


def test_chi0_k_chunking_is_bitwise_identical(gpu_lib, problems):
    p = problems["si18_qx"]
    one = run_chi0(gpu_lib, p)
    chunked = run_chi0(gpu_lib, p, chunks=[(0, 3), (3, 4), (4, 8)])
    assert np.array_equal(one, chunked)


def test_chi0_multi_frequency_and_ragged_sphere(gpu_lib):
    """Several frequencies, an eps sphere that is not a multiple of the tile
    (ng = 59) and an odd conduction count."""
    p = syn.make_problem("si18_qx", ng=59, nc=13, nfreq=3)
    ref = oracle.chi0(p)
    got = run_chi0(gpu_lib, p)
    assert rel_fro(got, ref) <= TOL_CHI_FP64


def test_chi0_degenerate_sizes(gpu_lib):
    """One G-vector, one valence and one conduction band."""
    p = syn.make_problem("si18_qx", ng=1, nv=1, nc=1)
    ref = oracle.chi0(p)
    got = run_chi0(gpu_lib, p)
    assert rel_fro(got, ref) <= TOL_CHI_FP64


def test_device_resident_inputs_match_host_inputs(gpu_lib, torch_cuda, problems):
    torch = torch_cuda
    p = problems["si16_q0"]
    host = run_chi0(gpu_lib, p)
    dev = [(torch.from_numpy(np.ascontiguousarray(p.coeff[ik])).cuda(),
            torch.from_numpy(np.ascontiguousarray(p.energy[ik])).cuda()) for ik in range(p.nk)]
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload(device_inputs=dev)
    ctx.accumulate()
    out = torch.zeros((len(p.freq),) + (len(p.qs[0][1]),) * 2, dtype=torch.complex128, device="cuda")
    gpu_lib.bgw_chi0_finalize(ctx.ctx, 0, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)
    ctx.close()


def test_aliased_box_warns_and_matches_cyclic_oracle(gpu_lib):
    """A 400-vector eps sphere (extent -5..5) with wavefunction spheres of
    extent -6..6 and an umklapp needs a box of at least 19; on a 16-box the
    library warns and returns the cyclic (box) result, which the oracle
    defines too."""
    p = syn.make_problem("si18_qx", box=(16, 16, 16), ng=400)
    ref = oracle.chi0(p)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    assert ctx.accumulate() == gpu_lib.BGW_W_ALIAS
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, ref) <= TOL_CHI_FP64


def test_errors_leave_state_usable(gpu_lib, problems):
    p = problems["si16_q0"]
    ctx = gpu_lib.Chi0Context(p, "fp64")
    # nothing uploaded yet
    with pytest.raises(gpu_lib.BgwError) as e:
        ctx.accumulate()
    assert e.value.status == gpu_lib.BGW_E_STATE
    # a sphere wider than the box
    wide = np.array([[-9, 0, 0], [9, 0, 0]], dtype=np.int32)
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_wfn_upload(ctx.ctx, 0, wide, np.zeros((p.nbands, 2, 2), complex), p.energy[0])
    assert e.value.status == gpu_lib.BGW_E_GRID
    # duplicate G
    dup = np.array([[1, 0, 0], [1, 0, 0]], dtype=np.int32)
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_wfn_upload(ctx.ctx, 0, dup, np.zeros((p.nbands, 2, 2), complex), p.energy[0])
    assert e.value.status == gpu_lib.BGW_E_ARG
    ctx.upload()
    # q off the k-grid
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_chi0_accumulate(ctx.ctx, [((0.3, 0, 0), p.qs[0][1], p.nc)], p.freq, 0, p.nk)
    assert e.value.status == gpu_lib.BGW_E_ARG
    ctx.accumulate(0, 4)
    # a different q-set mid-sum
    with pytest.raises(gpu_lib.BgwError) as e:
        gpu_lib.bgw_chi0_accumulate(ctx.ctx, [((0, 0, 0), p.qs[0][1][:5], p.nc)], p.freq, 4, 8)
    assert e.value.status == gpu_lib.BGW_E_STATE
    ctx.accumulate(4, 8)
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, oracle.chi0(p)) <= TOL_CHI_FP64


def test_empty_k_range_gives_zero(gpu_lib, problems):
    p = problems["si16_q0"]
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    ctx.accumulate(3, 3)
    got = ctx.finalize()
    ctx.close()
    assert not got.any()


# ------------------------------------------------- Si-like 24^3 workload --

@pytest.fixture(scope="module")
def si24():
    return syn.make_problem("si24")


def test_chi0_si24_k_subset_matches_oracle(gpu_lib, si24):
    """The 24^3 / N_G = 350 / N_c = 200 / 5-frequency workload on 3 k-points
    (one with an umklapp), oracle over the same k."""
    p = si24
    ks = [0, 12, 48]
    ref = oracle.chi0(p, k_indices=ks)
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    for k in ks:
        ctx.accumulate(k, k + 1)
    got = ctx.finalize()
    ctx.close()
    assert rel_fro(got, ref) <= TOL_CHI_FP64


def test_chi0_si24_full_sampled_entries(gpu_lib, si24):
    """Full 64-k workload as the benchmark runs it; the oracle computes the
    entries of 6 sampled G (all k) one sub-sphere at a time."""
    p = si24
    q, geps, nc = p.qs[0]
    got = run_chi0(gpu_lib, p)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(geps), 6, replace=False))
    sub = syn.Problem(p.name, p.avec, p.box, p.kgrid, p.kcrys, p.nv, p.nc, p.gvec, p.coeff,
                      p.energy, [(q, geps[pick], nc)], p.freq)
    ref = oracle.chi0(sub)
    g = got[:, pick][:, :, pick]
    assert rel_fro(g, ref) <= TOL_CHI_FP64
    for j in range(len(p.freq)):
        cj = got[j]
        assert np.array_equal(cj, cj.conj().T)
        ev = np.linalg.eigvalsh(cj)
        assert ev.max() <= 1e-12 * np.abs(ev).max()
