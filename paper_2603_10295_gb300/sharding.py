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
