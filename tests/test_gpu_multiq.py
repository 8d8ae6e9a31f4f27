"""Several q-points of ragged sizes in one accumulate call (the batched
form): every q's chi0 against the oracle, for both precisions; the mixed
path contracts all q-points of a k-chunk in one persistent grouped launch."""
import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5}


def rel_fro(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.fixture(scope="module")
def ragged():
    p = syn.make_batched_problem(config_id=7, a=10.26, box=(18, 18, 18), ecut_wfn=28.1,
                                 kgrid=(2, 2, 2), nv=8, nq=5, ng_range=(20, 150),
                                 nc_range=(5, 24), nfreq=3, precision="mixed")
    refs = [oracle.chi0(p, iq=iq) for iq in range(len(p.qs))]
    return p, refs


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kchunk", [1, 3])
def test_ragged_q_batch_matches_oracle(gpu_lib, ragged, prec, kchunk):
    p, refs = ragged
    assert len({len(g) for _, g, _ in p.qs}) > 1 and len({nc for _, _, nc in p.qs}) > 1
    ctx = gpu_lib.Chi0Context(p, prec)
    gpu_lib.bgw_set_option(ctx.ctx, gpu_lib.BGW_OPT_KCHUNK, kchunk)
    ctx.upload()
    ctx.accumulate()
    for iq, ref in enumerate(refs):
        got = ctx.finalize(iq)
        assert rel_fro(got, ref) <= TOL[prec], (iq, rel_fro(got, ref))
    ctx.close()


def test_batched_and_single_q_agree(gpu_lib, ragged):
    """A q-point contracted inside a group gives the same bits as alone."""
    p, _ = ragged
    ctx = gpu_lib.Chi0Context(p, "mixed")
    ctx.upload()
    ctx.accumulate()
    grouped = ctx.finalize(2)
    ctx.close()
    single = syn.Problem(p.name, p.avec, p.box, p.kgrid, p.kcrys, p.nv, p.nc, p.gvec, p.coeff,
                         p.energy, [p.qs[2]], p.freq)
    ctx = gpu_lib.Chi0Context(single, "mixed")
    ctx.upload()
    ctx.accumulate()
    alone = ctx.finalize(0)
    ctx.close()
    assert np.array_equal(grouped, alone)
