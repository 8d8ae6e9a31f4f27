"""Division of the polarizability over ranks: the k-block and q-share rules
(host logic), and the k-split sum of FP64 partials over two gloo ranks on the
CPU, with the oracle standing in for each rank's GPU work."""
import os
import socket

import numpy as np
import pytest

from paper_2206_00808_gb300 import sharding


@pytest.mark.parametrize("nk,world", [(0, 1), (1, 1), (5, 2), (64, 3), (7, 8), (216, 8)])
def test_k_blocks_cover_once_and_balance(nk, world):
    blocks = [sharding.k_block(nk, world, r) for r in range(world)]
    seen = [k for k0, k1 in blocks for k in range(k0, k1)]
    assert seen == list(range(nk))                       # contiguous, in order, each once
    sizes = [k1 - k0 for k0, k1 in blocks]
    assert max(sizes) - min(sizes) <= 1


def test_k_block_rejects_bad_rank():
    with pytest.raises(ValueError):
        sharding.k_block(10, 2, 2)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_q_share_partitions_and_balances(world):
    rng = np.random.default_rng(7)
    ng = rng.integers(700, 901, 40)
    nc = rng.integers(300, 501, 40)
    costs = [sharding.q_cost(int(g), int(c), 18, 216) for g, c in zip(ng, nc)]
    shares = [sharding.q_share(costs, world, r) for r in range(world)]
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(40))
    loads = [sum(costs[i] for i in s) for s in shares]
    # LPT bound: no rank exceeds the mean by more than the largest single job
    assert max(loads) <= sum(costs) / world + max(costs) + 1e-6


def test_q_share_equal_costs_round_robin():
    assert sharding.q_share([1.0] * 5, 2, 0) == [0, 2, 4]
    assert sharding.q_share([1.0] * 5, 2, 1) == [1, 3]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _k_split_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2206_00808_gb300 import synthetic as syn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = syn.make_problem("si16_q0", nv=4, nc=8)
        k0, k1 = sharding.k_block(p.nk, world, rank)
        part = oracle.chi0(p, 0, k_indices=range(k0, k1))   # this rank's share, 1/N_k applied
        t = torch.from_numpy(part).contiguous()
        sharding.allreduce_chi0(t)
        np.save(os.path.join(out_dir, f"chi_{rank}.npy"), t.numpy())
    finally:
        dist.destroy_process_group()


def test_k_split_allreduce_gloo_two_ranks(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2206_00808_gb300 import synthetic as syn
    oracle.build()
    world = 2
    mp.start_processes(_k_split_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    full = oracle.chi0(syn.make_problem("si16_q0", nv=4, nc=8), 0)
    for r in range(world):
        got = np.load(tmp_path / f"chi_{r}.npy")
        # the two partials sum in one fixed pairing: agreement to FP64 rounding
        assert np.abs(got - full).max() <= 1e-13 * np.abs(full).max()
