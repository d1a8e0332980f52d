"""Multi-rank host logic on CPU (gloo, world size 2): q sharding covers every q
once, and the all-reduced per-rank loss and gradient equal the single-process
ones.  The per-rank work is done by the CPU oracle here (no GPU on this host);
on GPUs each rank calls eph_interp_backward on its shard instead."""
import os
import socket

import numpy as np
import pytest

from paper_2603_10295_gb300.sharding import q_shard, step_q_indices


@pytest.mark.parametrize("nq,world", [(1, 1), (7, 2), (256, 3), (5, 8), (0, 2)])
def test_q_shard_partitions(nq, world):
    seen = []
    for r in range(world):
        a, b = q_shard(nq, r, world)
        assert 0 <= a <= b <= nq
        seen.extend(range(a, b))
    assert seen == list(range(nq))
    sizes = [q_shard(nq, r, world)[1] - q_shard(nq, r, world)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_bench_step_indices_disjoint_equal_work(world):
    # the bench's per-rank q points: equal counts, and disjoint while the list is long enough
    nq, nsteps, qb = 1000, 13, 4
    blocks = [step_q_indices(nq, nsteps, qb, r, world) for r in range(world)]
    assert all(len(b) == nsteps * qb for b in blocks)
    allq = np.concatenate(blocks)
    assert np.array_equal(np.sort(allq), np.arange(world * nsteps * qb))
    # a longer run wraps around the list; every rank still gets nsteps * qb valid indices
    wrap = [step_q_indices(7, nsteps, qb, r, world) for r in range(world)]
    assert all(len(b) == nsteps * qb and b.min() >= 0 and b.max() < 7 for b in wrap)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2603_10295_gb300 import synth
    from paper_2603_10295_gb300.sharding import allreduce_loss_and_grad, q_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.make_workload("si_tiny", nb=3, nk=10, nq=5)
    eps_k, _ = oracle.electron_eigen(oracle.hamiltonian_k(wl.kpts, wl.Re, wl.we, wl.H_Re))
    w, _ = oracle.fermi_weights(eps_k, 1)
    a, b = q_shard(len(wl.qpts), rank, world)
    L, grad = oracle.loss_and_grad(wl, wl.kpts, wl.qpts[a:b], w, 1e-6)
    L, g = allreduce_loss_and_grad(L, torch.from_numpy(grad))
    if rank == 0:
        np.save(os.path.join(out_dir, "grad.npy"), g.numpy())
        np.save(os.path.join(out_dir, "L.npy"), np.array([L]))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_sum_equals_single_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    from paper_2603_10295_gb300 import synth
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    wl = synth.make_workload("si_tiny", nb=3, nk=10, nq=5)
    eps_k, _ = oracle.electron_eigen(oracle.hamiltonian_k(wl.kpts, wl.Re, wl.we, wl.H_Re))
    w, _ = oracle.fermi_weights(eps_k, 1)
    L_ref, g_ref = oracle.loss_and_grad(wl, wl.kpts, wl.qpts, w, 1e-6)
    L = float(np.load(tmp_path / "L.npy")[0])
    g = np.load(tmp_path / "grad.npy")
    assert abs(L - L_ref) <= 1e-12 * abs(L_ref)
    assert np.abs(g - g_ref).max() <= 1e-12 * np.abs(g_ref).max()


@pytest.mark.parametrize("np_total,world", [(27, 2), (216, 3), (15, 8), (8, 8)])
def test_rp_slices_cover_the_list(np_total, world):
    from paper_2603_10295_gb300.sharding import rp_slice
    blocks = [rp_slice(np_total, r, world) for r in range(world)]
    covered = [i for b, c in blocks for i in range(b, b + c)]
    assert covered == list(range(np_total)) and min(c for _, c in blocks) >= 1
    with pytest.raises(ValueError):
        rp_slice(world - 1, 0, world)


class _OracleSliceContext:
    """Stands in for a device context on CPU ranks: eph_g1_partial is the oracle's Eq. 9 over
    the rank's Rp block; eph_interp_q_g1 records the G1 it is given."""

    def __init__(self, wl, begin, count):
        self.wl, self.b, self.c = wl, begin, count
        self.seen = None

    def eph_g1_partial(self, nq, qpts, G1):
        import torch

        import oracle
        part = oracle.g_rp_to_q(qpts[:nq], self.wl.Rp[self.b:self.b + self.c], self.wl.wp[self.b:self.b + self.c],
                                self.wl.g_ReRp[self.b:self.b + self.c])
        G1.copy_(torch.from_numpy(part.reshape(G1.shape)))

    def eph_interp_q_g1(self, nq, qpts, G1, eps_kq, omega, g):
        self.seen = G1.clone()


def _rp_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2603_10295_gb300 import synth
    from paper_2603_10295_gb300.sharding import interp_q_rp_partitioned, rp_slice
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.make_workload("si_tiny", nb=3, nk=4, nq=5)
    b, c = rp_slice(wl.np_, rank, world)
    ctx = _OracleSliceContext(wl, b, c)
    G1 = torch.empty((5, wl.nm, wl.ne, wl.nb, wl.nb), dtype=torch.complex128)
    interp_q_rp_partitioned(ctx, 5, wl.qpts, G1)
    np.save(os.path.join(out_dir, f"g1_{rank}.npy"), ctx.seen.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_rp_partition_sums_to_eq9(tmp_path, world):
    # every rank ends with the whole Eq. 9 result although it holds only its Rp block of g(Re,Rp)
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    from paper_2603_10295_gb300 import synth
    mp.spawn(_rp_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    wl = synth.make_workload("si_tiny", nb=3, nk=4, nq=5)
    ref = oracle.g_rp_to_q(wl.qpts, wl.Rp, wl.wp, wl.g_ReRp)
    for r in range(world):
        got = np.load(tmp_path / f"g1_{r}.npy").reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
