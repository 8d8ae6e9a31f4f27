"""Work division of the polarizability over several ranks (one GPU each).

The sum that defines chi0_GG'(q, i w) (Sec. II, the P formula) runs over
k-points and band pairs, separately for every q-point, so it splits two ways:

* across q-points: every q is an independent problem; ranks take disjoint
  shares of the q list and exchange nothing (`q_share`);
* within one q-point: ranks take disjoint contiguous k-blocks, each
  accumulates its share of the k sum (finalize already applies the full
  1/N_k), and one element-wise sum of the FP64 partials over ranks gives chi0
  (`k_block`, `allreduce_chi0`).

This module only decides who does what and sums the partials; the
polarizability itself is computed by the CUDA library on each rank.  The
collective is torch.distributed's all-reduce (NCCL for device tensors, gloo
for host tensors).
"""
from __future__ import annotations

from typing import Sequence


def k_block(nk: int, world: int, rank: int) -> tuple[int, int]:
    """[k_begin, k_end) of this rank: contiguous blocks whose sizes differ by
    at most one, in rank order, covering 0..nk-1 exactly once."""
    if world < 1 or not 0 <= rank < world or nk < 0:
        raise ValueError(f"k_block: bad nk={nk}, world={world}, rank={rank}")
    base, extra = divmod(nk, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def q_cost(ng: int, nc: int, nv: int, nk: int) -> float:
    """Relative cost of one q-point: the contraction's Hermitian work,
    N_k N_v N_c N_G (N_G + 1) / 2, which dominates at the sizes of interest."""
    return float(nk) * nv * nc * ng * (ng + 1) / 2


def q_share(costs: Sequence[float], world: int, rank: int) -> list[int]:
    """Indices of the q-points this rank computes.

    Longest-processing-time assignment: q-points in decreasing cost (ties by
    index) each go to the rank with the least total so far (ties to the lower
    rank).  Every rank evaluates the same deterministic rule, so the shares
    are disjoint and cover every q without any exchange.  Returned in
    increasing index order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"q_share: bad world={world}, rank={rank}")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        load[r] += float(costs[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def allreduce_chi0(chi, group=None):
    """Sum a rank's partial chi0 over all ranks, in place, and return it.

    chi: a complex128 (or complex64) torch tensor, on the device for NCCL or
    on the host for gloo; every rank passes the same shape.  The sum is taken
    on the real view (re, im interleaved), which is exactly the complex sum."""
    import torch
    import torch.distributed as dist
    if not chi.is_complex():
        raise TypeError("allreduce_chi0: expected a complex tensor")
    if not chi.is_contiguous():
        raise ValueError("allreduce_chi0: tensor must be contiguous")
    dist.all_reduce(torch.view_as_real(chi), op=dist.ReduceOp.SUM, group=group)
    return chi


def chi0_k_split(ctx, qlist, freq, nk: int, world: int, rank: int, iq: int = 0, group=None):
    """chi0 of q-point `iq` with the k sum split over ranks.

    ctx is this rank's Chi0Context (binding.Chi0Context) with every k-point
    it needs already uploaded.  Each rank accumulates its k_block, finalizes
    to a device tensor (scaled by the full 1/N_k) and the partials are summed
    over ranks; every rank returns the full chi0 [N_w][N_G][N_G]."""
    import torch
    from . import binding as B
    k0, k1 = k_block(nk, world, rank)
    B.bgw_chi0_reset(ctx.ctx)
    if k1 > k0:
        B.bgw_chi0_accumulate(ctx.ctx, qlist, freq, k0, k1)
        ng = len(qlist[iq][1])
        out = torch.empty((len(freq), ng, ng), dtype=torch.complex128, device="cuda")
        B.bgw_chi0_finalize(ctx.ctx, iq, out)
        if getattr(ctx, "stream", None) is not None:       # finalize ran on the context's stream
            torch.cuda.current_stream().wait_stream(ctx.stream)
    else:
        ng = len(qlist[iq][1])
        out = torch.zeros((len(freq), ng, ng), dtype=torch.complex128, device="cuda")
    return allreduce_chi0(out, group)
