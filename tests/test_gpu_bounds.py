"""The index-checking build (libbgwchi_bounds.so, -DBGW_BOUNDS=1): the small
parity cases run through every sphere-to-grid and matrix-element path in a
child process that loads that library, and the device status word of the
index checks stays clear while chi0 still matches the CPU FP64 oracle.  No
out-of-range input is given: the checks are for catching kernel index bugs,
and they record instead of trapping."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (workload, overrides, precision, options): the default paths, each K1 path
# option, the eight-lane kernels with the scatter (48^3) and the non-cubic
# four-lane ones
CASES = [
    ("si16_q0", {}, "fp64", {}),
    ("si18_qx", {}, "fp64", {"K1_PATH": 1}),
    ("si18_qx", {}, "mixed", {}),
    ("si18_qx", {}, "mixed", {"DEFER_K1": 1}),
    ("si18_qx", {}, "mixed", {"K1_PATH": 4}),
    ("si18_qx", dict(box=(48, 48, 48), ng=89, nv=4, nc=9, nfreq=2), "fp64", {}),
    ("si18_qx", dict(box=(48, 48, 48), ng=89, nv=4, nc=9, nfreq=2), "mixed", {"K1_PATH": 3}),
    ("si18_qx", dict(box=(48, 64, 64), ng=89, nv=4, nc=9, nfreq=2), "mixed", {}),
]


def child():
    import numpy as np
    import oracle
    from paper_2206_00808_gb300 import binding as B
    from paper_2206_00808_gb300 import synthetic as syn
    assert B.LIB_PATH.endswith("libbgwchi_bounds.so")
    out = []
    st, word = B.bgw_bounds_check()          # clear
    for name, over, prec, opts in CASES:
        p = syn.make_problem(name, **over)
        ref = oracle.chi0(p)
        ctx = B.Chi0Context(p, prec)
        for k, v in opts.items():
            B.bgw_set_option(ctx.ctx, getattr(B, "BGW_OPT_" + k), v)
        ctx.upload()
        ctx.accumulate()
        got = ctx.finalize()
        ctx.close()
        st, word = B.bgw_bounds_check()
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        out.append({"case": f"{name} {over} {prec} {opts}", "status": st, "word": word, "err": err,
                    "tol": 1e-10 if prec == "fp64" else 2e-5})
    print("RESULT " + json.dumps(out))


def test_index_checks_stay_clear_on_every_path(gpu_lib):
    env = dict(os.environ, BGW_LIBRARY="bounds")
    code = f"import sys; sys.path[:0] = [{ROOT!r}, {HERE!r}]; import test_gpu_bounds as t; t.child()"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    for res in json.loads(line[len("RESULT "):]):
        assert res["status"] == 0, res
        assert res["word"] == 0, res
        assert res["err"] <= res["tol"], res
