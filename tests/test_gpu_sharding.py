"""k-split polarizability on the GPU: the partials of two k-blocks (computed
one after the other on this GPU) sum to the one-shot chi0, and
sharding.chi0_k_split runs its NCCL all-reduce in a one-rank process group."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2206_00808_gb300 import sharding
from paper_2206_00808_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_k_block_partials_sum_to_full(gpu_lib):
    p = syn.make_problem("si18_qx")
    ctx = gpu_lib.Chi0Context(p, "fp64")
    ctx.upload()
    full = np.zeros((len(p.freq), len(p.qs[0][1]), len(p.qs[0][1])), np.complex128)
    world = 3
    for r in range(world):
        k0, k1 = sharding.k_block(p.nk, world, r)
        ctx.reset()
        ctx.accumulate(k0, k1)
        full += ctx.finalize()
    ctx.reset()
    ctx.accumulate()
    one = ctx.finalize()
    ctx.close()
    assert np.abs(full - one).max() <= 1e-12 * np.abs(one).max()
    ref = oracle.chi0(p)
    assert np.linalg.norm(full - ref) <= 1e-10 * np.linalg.norm(ref)


def test_chi0_k_split_single_rank_nccl(gpu_lib):
    import torch
    import torch.distributed as dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        p = syn.make_problem("si16_q0")
        stream = torch.cuda.Stream()
        ctx = gpu_lib.Chi0Context(p, "fp64", stream)
        ctx.upload()
        got = sharding.chi0_k_split(ctx, ctx.qlist(), p.freq, p.nk, 1, 0)
        torch.cuda.synchronize()
        ctx.close()
    finally:
        dist.destroy_process_group()
    ref = oracle.chi0(p)
    assert np.linalg.norm(got.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
