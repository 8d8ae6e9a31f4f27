"""Host-side pieces of bench.py that set the reported figures: the FLOP and
least-bytes models scale with the workload as their definitions say, and the
roofline denominators fall back when no measured peaks are on disk."""
import numpy as np

import bench
from paper_2206_00808_gb300 import synthetic as syn


def test_byte_model_counts_each_grid_and_coefficient_once():
    p = syn.make_problem("si18_qx", nv=4, nc=6)
    vol = float(np.prod(p.box))
    for csize in (8, 16):
        bm = bench.byte_model(p, csize)
        coeff = sum(p.nbands * 2 * len(g) * 16 for g in p.gvec)
        assert bm["wfn_to_grid"] == coeff + p.nk * p.nbands * 2 * vol * csize
        _, geps, nc = p.qs[0]
        assert bm["mtxel"] == p.nk * (p.nv + nc) * 2 * vol * csize          # grids read by the z + y kernel
        assert bm["mtxel_x"] == p.nk * p.nv * nc * len(geps) * csize        # M written by the x pass


def test_flop_model_scales_with_pairs_and_frequencies():
    p = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=1)
    q = syn.make_problem("si18_qx", nv=4, nc=6, nfreq=3)
    a, b = bench.flop_model(p), bench.flop_model(q)
    assert np.isclose(b["contraction"], 3 * a["contraction"])
    assert np.isclose(b["mtxel"], a["mtxel"]) and np.isclose(b["wfn_to_grid"], a["wfn_to_grid"])
    assert np.isclose(a["total"], a["wfn_to_grid"] + a["mtxel"] + a["mtxel_x"] + a["contraction"])
    # x lines: w_y w_z per pair against N^2 + N w_y lines of the z + y kernel
    n = p.box[0]
    w = p.qs[0][1].max(0) - p.qs[0][1].min(0) + 1
    fft = 5 * n * np.log2(n)
    pairs = p.nk * p.nv * p.qs[0][2]
    assert np.isclose(a["mtxel_x"], pairs * fft * w[1] * w[2])
    assert np.isclose(a["mtxel"], pairs * (fft * (n * n + n * w[1]) + 16 * n ** 3))
    ng = len(p.qs[0][1])
    assert np.isclose(a["contraction"], 8.0 * p.nk * p.nv * p.qs[0][2] * ng * (ng + 1) / 2)


def test_measured_hbm_rate_is_positive():
    assert bench.measured_hbm_gbs() > 1000.0


def test_umklapp_and_partner_bookkeeping():
    p = syn.make_problem("gasb32", coeff_on=None)
    umk = bench.umklapp_ks(p)
    # k1 = 5/6 (indices 180..215) is where k + q = k' + (1, 0, 0) on the 6x6x6 grid
    assert umk == list(range(180, 216))
    assert bench.with_partners(p, [0, 3, 180]) == [0, 3, 36, 39, 180]
    assert bench.k_runs([0, 1, 2, 3, 180, 181, 183]) == [(0, 4), (180, 182), (183, 184)]


def test_error_stats_of_a_known_perturbation():
    rng = np.random.default_rng(3)
    ref = rng.standard_normal((2, 4, 4)) + 1j * rng.standard_normal((2, 4, 4))
    got = ref.copy()
    got[1, 0, 1] += 1e-3
    e = bench.error_stats(got, ref)
    assert e["rel_fro_per_freq"][0] == 0.0
    assert np.isclose(e["rel_fro_per_freq"][1], 1e-3 / np.linalg.norm(ref[1]))
    assert np.isclose(e["max_entry_err_rel_to_max"], 1e-3 / np.abs(ref).max())
    assert e["offdiag_rel_fro_max"] > 0 and np.isclose(e["rel_fro"], 1e-3 / np.linalg.norm(ref))


def test_oracle_sample_sizes():
    p = syn.make_problem("gasb32", coeff_on=None)
    assert 1 <= bench.sample_nc(p) < p.nc
    assert bench.sample_nc(syn.make_problem("si18_qx")) == 24


def test_zy_kernel_names_follow_the_library_rule():
    g = syn.make_problem("gasb32", coeff_on=None)
    assert bench.zy_kernel_name(g, "mixed", 0) == "k2_zy_stream"
    assert bench.zy_kernel_name(g, "mixed", 1) == "k2_zy_plane"
    assert bench.zy_kernel_name(g, "fp64", 2).startswith("k2_zpass")
    b = syn.make_bi2se3_problem(kgrid=(1, 1, 1), nv=2, nc=2, nfreq=1, device=None)
    assert bench.zy_kernel_name(b, "mixed", 2) == "k2_zy_oct"


def test_captured_traffic_lookup_and_operand_bytes():
    """roofline.traffic comes only from a capture of the same launch shape
    with an unchanged kernel source; the operand bytes of one GaSb-like
    contraction launch (k-chunk 2) are 34 planes x 1664 rows x 14,400 pairs x
    2 B."""
    nbytes, why = bench.captured_traffic("k5_gemm", "gasb32", "mixed", 4)
    assert nbytes is None and "no ncu capture" in why
    nbytes, why = bench.captured_traffic("k5_gemm", "si24", "mixed", 2)
    assert nbytes is None
    p = syn.make_problem("gasb32", coeff_on=None)
    assert bench.gemm_operand_bytes(p, 2) == 34 * 1664 * 14400 * 2
    saved = dict(bench.CAPTURED_TRAFFIC)
    try:
        key = ("k5_gemm", "gasb32", "mixed", 2)
        path, _, b = bench.CAPTURED_TRAFFIC[key]
        bench.CAPTURED_TRAFFIC[key] = (path, "0" * 16, b)          # a source edited since the capture
        nbytes, why = bench.captured_traffic(*key)
        assert nbytes is None and "changed since the capture" in why
    finally:
        bench.CAPTURED_TRAFFIC.clear()
        bench.CAPTURED_TRAFFIC.update(saved)
