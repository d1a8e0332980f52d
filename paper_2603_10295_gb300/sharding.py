"""q sharding across ranks (one process per GPU).

The interpolation is independent per q (the paper's images need no exchange
inside the q loop), so each rank takes a contiguous block of the q list; the
forward pass needs no collective.  The backward pass sums the per-rank L and
dL/dg(Re,Rp) with one all-reduce (NCCL on GPUs, gloo on CPU tensors).
"""
from __future__ import annotations


def q_shard(nq: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of this rank's q block; blocks differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or nq < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(nq, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def step_q_indices(nq: int, nsteps: int, q_batch: int, rank: int, world: int):
    """Indices into a list of nq q points for this rank's nsteps batches of q_batch points.

    The ranks take consecutive blocks of the list extended cyclically, so that every rank has
    the same amount of work (weak scaling) and, while world * nsteps * q_batch <= nq, no q
    point is processed twice."""
    import numpy as np
    if nq < 1 or nsteps < 0 or q_batch < 1:
        raise ValueError("bad step request")
    start, _ = q_shard(world * nsteps * q_batch, rank, world)
    return (np.arange(nsteps * q_batch) + start) % nq


def allreduce_loss_and_grad(L, grad, group=None):
    """Sums a rank-local scalar L and gradient tensor over all ranks (in place for grad)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor([float(L)], dtype=torch.float64, device=grad.device)
    dist.all_reduce(t, group=group)
    if torch.is_complex(grad):
        dist.all_reduce(torch.view_as_real(grad), group=group)
    else:
        dist.all_reduce(grad, group=group)
    return float(t.item()), grad
