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


# ---------------------------------------------------------------------------------------------
# Rp partition of g(Re,Rp) (the paper's pools): for a g(Re,Rp) that does not fit one GPU, each
# rank holds a contiguous block of the Rp vectors (eph_create_rp_slice), forms the partial Eq. 9
# sum over its block (eph_g1_partial), and one all-reduce of G1 per q batch gives every rank the
# whole G1, from which it runs the rest of the path for its own k points (eph_interp_q_g1).
# ---------------------------------------------------------------------------------------------
def rp_slice(np_total: int, rank: int, world: int) -> tuple[int, int]:
    """(rp_begin, rp_count) of this rank's block of the Rp list; every block holds >= 1 vector."""
    if np_total < world:
        raise ValueError(f"{np_total} Rp vectors cannot be split over {world} ranks")
    a, b = q_shard(np_total, rank, world)
    return a, b - a


def allreduce_g1(G1, group=None):
    """Sums the ranks' partial G1 tensors in place (complex tensors as their real views)."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(torch.view_as_real(G1) if torch.is_complex(G1) else G1, group=group)
    return G1


def interp_q_rp_partitioned(ctx, nq, qpts, G1, eps_kq=None, omega=None, g=None, group=None):
    """One q batch on an Rp-partitioned g(Re,Rp): partial Eq. 9 on this rank's slice, all-reduce
    of G1 over `group`, then the k stage from the summed G1.  `ctx` is a device-pointer
    binding.Context on torch's current stream (so the collective is ordered after the partial
    sum); G1 is a caller tensor [nq][nm][ne][nb][nb] complex128 on the same device."""
    ctx.eph_g1_partial(nq, qpts, G1)
    allreduce_g1(G1, group)
    ctx.eph_interp_q_g1(nq, qpts, G1, eps_kq, omega, g)
