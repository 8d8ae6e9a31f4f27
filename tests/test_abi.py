"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; argument checks that run before any CUDA call reject bad input.
No GPU is used here."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_00808_gb300 import build
    build.build()
    from paper_2206_00808_gb300 import binding
    return binding


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"BGW_API\s+[\w\s\*]+?\b(bgw_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["bgw_wfn_upload", "bgw_mtxel_spinor", "bgw_chi0_accumulate", "bgw_chi0_finalize",
              "bgw_create", "bgw_destroy", "bgw_last_error"]:
        assert n in names


def test_precision_enum_matches_binding(lib):
    """The four precisions of the boundary and their values, as the header
    declares them and the binding passes them."""
    import os
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "bgw_chi.h")).read()
    body = text[text.index("typedef enum {\n    BGW_FP64"):]
    body = body[:body.index("} bgw_precision;")]
    vals = {n: int(v) for n, v in re.findall(r"\b(BGW_\w+)\s*=\s*(\d+)", body)}
    assert vals == {"BGW_FP64": 0, "BGW_MIXED_BF16X3": 1, "BGW_MIXED_TF32X3": 2, "BGW_MIXED_TF32": 3}
    assert lib.PRECISIONS == {"fp64": 0, "mixed": 1, "tf32x3": 2, "tf32": 3}


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in declared_symbols():
        assert hasattr(so, n), n
    assert set(lib.EXPORTED) == declared_symbols()


def test_version_string(lib):
    assert "sm_103a" in lib.bgw_version()


@pytest.mark.parametrize("fft, msg", [((16, 17, 16), "not supported"), ((0, 16, 16), "not supported")])
def test_create_rejects_unsupported_box(lib, fft, msg):
    with pytest.raises(lib.BgwError) as e:
        lib.bgw_create(fft, np.zeros((1, 3)), 1, 1, "fp64")
    assert e.value.status == lib.BGW_E_ARG and msg in str(e.value)


def test_create_rejects_bad_counts_and_precision(lib):
    with pytest.raises(lib.BgwError) as e:
        lib.bgw_create((16, 16, 16), np.zeros((1, 3)), 0, 1, "fp64")
    assert e.value.status == lib.BGW_E_ARG
    with pytest.raises(lib.BgwError) as e:
        lib.bgw_create((16, 16, 16), np.zeros((1, 3)), 2, 2, 7)
    assert e.value.status == lib.BGW_E_ARG
    with pytest.raises(lib.BgwError) as e:
        lib.bgw_create((16, 16, 16), np.array([[np.nan, 0, 0]]), 2, 2, "fp64")
    assert e.value.status == lib.BGW_E_ARG


def test_null_context_calls_are_rejected(lib):
    import ctypes
    so = lib._lib
    assert so.bgw_chi0_reset(None) == lib.BGW_E_ARG
    assert so.bgw_chi0_finalize(None, 0, None, 0) == lib.BGW_E_ARG
    so.bgw_destroy(None)


def test_coulomb_sqrt_host_matches_oracle():
    """bgw_coulomb_sqrt is a host computation: checked here without a GPU."""
    import oracle
    from paper_2206_00808_gb300 import binding as B
    from paper_2206_00808_gb300 import synthetic as syn
    p = syn.make_problem("si18_qx")
    q, geps, _ = p.qs[0]
    s = B.bgw_coulomb_sqrt(p.avec, q, geps)
    v = oracle.coulomb(p.avec, q, geps)
    assert np.allclose(s ** 2, v, rtol=1e-13, atol=0)


def test_epsinv_argument_errors_without_gpu():
    from paper_2206_00808_gb300 import binding as B
    rc = B._lib.bgw_epsinv(0, 1, None, None, 1, None, 0, None)
    assert rc == B.BGW_E_ARG
    s = np.array([-1.0])
    rc = B._lib.bgw_epsinv(1, 1, B._host_ptr(s), B.ctypes.c_void_p(16), 1, None, 0, None)
    assert rc == B.BGW_E_ARG
    assert b"finite" in B._lib.bgw_last_error(None)


def test_symmetry_su2_host_matches_oracle_for_fcc_operations():
    """bgw_symmetry_su2 is a host computation: every operation of the FCC
    lattice (48, improper ones through their proper part) against the oracle."""
    from oracle import symmetry as sym
    from paper_2206_00808_gb300 import binding as B
    from paper_2206_00808_gb300 import synthetic as syn
    avec = syn.fcc_cell(10.26)
    A = avec.T
    for R in sym.cubic_operations():
        R_lat = np.rint(np.linalg.inv(A) @ R @ A).astype(np.int32)
        U, n, theta = B.bgw_symmetry_su2(avec, R_lat)
        assert np.abs(U - sym.spin_matrix(avec, R_lat)).max() < 1e-13
        P = -R if np.linalg.det(R) < 0 else R
        assert np.abs(sym.axis_angle_matrix(n, theta) - P).max() < 1e-13


def test_symmetry_rejects_non_rotations():
    from paper_2206_00808_gb300 import binding as B
    from paper_2206_00808_gb300 import synthetic as syn
    avec = syn.fcc_cell(10.26)
    with pytest.raises(B.BgwError):
        B.bgw_symmetry_su2(avec, np.array([[2, 0, 0], [0, 1, 0], [0, 0, 1]]))   # not unimodular
    with pytest.raises(B.BgwError):
        B.bgw_symmetry_su2(avec, np.array([[1, 1, 0], [0, 1, 0], [0, 0, 1]]))   # shear: not a rotation


def test_default_build_has_no_index_checks():
    from paper_2206_00808_gb300 import binding as B
    st, word = B.bgw_bounds_check()
    assert st == B.BGW_E_STATE and word == 0
    assert "BGW_BOUNDS" in B.bgw_last_error(None)
