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
