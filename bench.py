#!/usr/bin/env python
"""Throughput of e-ph Wannier interpolation on GB300: g(k,q) elements per second.

Workload (default): the silicon-shaped full configuration -- Nb=8 Wannier
functions, Na=2 atoms (Nm=6), Re = Rp = the 216 vectors of a 6x6x6 centred fcc
box, a 40x40x40 uniform k grid (64,000 k) and 1,000 random q points, synthetic
seeded inputs (paper_2603_10295_gb300.synth).  One step = one q batch (q_batch
q points against all 64,000 k): phases, D(q) and its eigensolve, the Rp->q
contraction (Eq. 9), the mode rotation, the Re->k contraction fused with H(k+q)
(Eq. 10), the batched H(k+q) eigensolves and the band rotation, with g written
to device memory.  The k-side preparation (H(k) eigensolves, once per job) is
timed separately and its share for the processed q points is added.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp64|mixed]
    python bench.py --impl reference     # the FP64 CPU oracle on the host cores

Multi-GPU (torchrun): weak scaling, each rank takes its own q points; NCCL is
used only for the barrier and the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "e-ph g(k,q) elements/s, 1 GB300: split-precision vs FP64 form at stated rel. error"
UNIT = "g elements/s"
# FP64 pipe of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (unit counts and max clock)
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel from one ncu capture of a one-q launch, scaled to the bench launch by the units
# processed (profiles/k_zgemm_si_full_fp64.md).  Keyed by (kernel, workload, q batch).
TRAFFIC = {("k_zgemm", "si_full", 4): 4 * (225.011712e6 + 404.513024e6),
           ("k_zgemm", "si_full", 1): 225.011712e6 + 404.513024e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libeph", choices=["libeph", "reference"])
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="si_full")
    ap.add_argument("--q-batch", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-k", type=int, default=16000)
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def flops_per_pair(nb, nm, ne, np_, nk):
    """Algorithmic FP64 work per (k,q) pair, in flops (8 per complex multiply-add)."""
    nb2 = nb * nb
    cmac = (nb2 * ne          # H(k+q) Fourier sum
            + nm * nb2 * ne   # Re->k contraction (Eq. 10)
            + 2 * nb2 * nb * nm   # band rotation
            + (nm * nb2 * ne * np_ + nm * nm * nb2 * ne) / nk)   # Eq. 9 and the mode rotation, per k
    return 8.0 * cmac


def cpu_baseline(wl, nk_sample, steps=1):
    """The FP64 oracle on the host cores on a bounded sample: 1 q x nk_sample k."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(1)
    ks = np.sort(rng.choice(len(wl.kpts), size=min(nk_sample, len(wl.kpts)), replace=False))
    kp = wl.kpts[ks]
    qp = wl.qpts[:1]
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.interpolate(wl, kp, qp)
        times.append(time.perf_counter() - t0)
    units = len(ks) * 1 * wl.nm * wl.nb * wl.nb
    t = statistics.median(times)
    return {"value": units / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{wl.name}: 1 q x {len(ks)} random k of the grid (numpy FP64, BLAS threads = all cores)",
            "seconds": t}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2603_10295_gb300 import synth
    wl = synth.make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_baseline(wl, args.cpu_sample_k)
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        r = cpu_baseline(wl, args.cpu_sample_k)
        units += r["value"] * r["seconds"]
    el = time.perf_counter() - t0
    value = units / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": describe(wl, args), "form": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: 1 q x {args.cpu_sample_k} random k of {wl.name}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def describe(wl, args):
    nk = len(wl.kpts)
    grid = "x".join(map(str, wl.kgrid)) if wl.kgrid else str(nk)
    return (f"{wl.name}: Nb={wl.nb} Na={wl.na} Nm={wl.nm} Ne=Np={wl.ne}, k grid {grid} ({nk} k) x "
            f"{len(wl.qpts)} random q; one step = {args.q_batch} q x {nk} k")


# ----------------------------------------------------------------------------- libeph arm
def run_libeph(args):
    import numpy as np
    import torch

    from paper_2603_10295_gb300 import binding, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = synth.make_workload(args.workload)
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    QB = args.q_batch
    st = torch.cuda.current_stream()
    ctx = binding.Context.from_workload(wl, form=args.form, device_ptrs=True, q_batch=QB, stream=st)
    # this rank's q points: (warmup + steps) batches, disjoint across ranks, cycling the q list
    nsteps = args.warmup + args.steps
    qidx = (np.arange(nsteps * QB) + rank * nsteps * QB) % len(wl.qpts)
    q_dev = torch.from_numpy(np.ascontiguousarray(wl.qpts[qidx])).to(dev)
    k_dev = torch.from_numpy(wl.kpts).to(dev)
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    gdt = torch.complex128 if args.form == "fp64" else torch.complex64
    eps_kq = torch.empty(QB, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(QB, nm, dtype=torch.float64, device=dev)
    g = torch.empty(QB, nk, nm, nb, nb, dtype=gdt, device=dev)

    # k-side preparation, once per job
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    ctx.eph_set_k(nk, k_dev, eps_k)
    e1.record(st)
    torch.cuda.synchronize()
    setk_ms = e0.elapsed_time(e1)

    def step(i):
        ctx.eph_interp_q(QB, q_dev[i * QB:(i + 1) * QB], eps_kq, om, g)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_reset()
    launches0 = ctx.launches()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0.record(st)
    for i in range(args.warmup, nsteps):
        step(i)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    el_ms = e0.elapsed_time(e1)
    launches = ctx.launches() - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([el_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        el_ms = float(t.item())
    units_rank = args.steps * QB * nk * nm * nb * nb
    # share of the once-per-job k preparation for the q points processed here
    setk_share_ms = setk_ms * (args.steps * QB) / len(wl.qpts)
    value = world * units_rank / ((el_ms + setk_share_ms) * 1e-3)

    # roofline: the dominant kernel is the fused Re->k / H(k+q) FP64 contraction (stage ft_k)
    ft_ms, ft_n = prof["ft_k"]
    NW = nb * nb * (1 + nm)
    flop_launch = 8.0 * QB * nk * NW * wl.ne          # one launch covers the q batch x all k
    achieved = flop_launch / (ft_ms / max(ft_n, 1) * 1e-3) if ft_n else None
    roof = {"bound": "alu", "kernel": "k_zgemm (Re->k contraction fused with H(k+q), FP64 DFMA)",
            "achieved": achieved / 1e12 if achieved else None, "peak": FP64_PEAK_FLOPS / 1e12,
            "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_FLOPS) if achieved else None,
            "traffic": TRAFFIC.get(("k_zgemm", args.workload, QB)),
            "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 unit count, max clock)"}
    stage_ms = {k: round(v[0] / args.steps, 3) for k, v in prof.items()}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "tf32x3/f32",
                "data": "synthetic",
                "config": {"workload": describe(wl, args), "form": args.form, "q_batch": QB,
                           "l2": "inputs larger than L2: g(Re,Rp) 287 MB, P_k 221 MB resident; "
                                 f"g out {g.numel() * g.element_size() / 1e9:.2f} GB per step",
                           "k_setup_ms": setk_ms, "k_setup_share_ms": setk_share_ms,
                           "stage_ms_per_step": stage_ms},
                "roofline": roof, "gpu_launches": launches, "clocks": clk}
    del g, eps_kq, om
    ctx.close()
    torch.cuda.empty_cache()

    # end to end through the public C-ABI with HOST buffers (pinned), copies inside the timed region
    if rank == 0 and not args.no_e2e:
        hctx = binding.Context.from_workload(wl, form=args.form, device_ptrs=False, q_batch=QB)
        kp_h = torch.from_numpy(wl.kpts).pin_memory()
        epsk_h = torch.empty(nk, nb, dtype=torch.float64).pin_memory()
        q_h = torch.from_numpy(np.ascontiguousarray(wl.qpts[qidx])).pin_memory()
        g_h = torch.empty(QB, nk, nm, nb, nb, dtype=gdt).pin_memory()
        ekq_h = torch.empty(QB, nk, nb, dtype=torch.float64).pin_memory()
        om_h = torch.empty(QB, nm, dtype=torch.float64).pin_memory()
        t0 = time.perf_counter()
        hctx.eph_set_k(nk, kp_h, epsk_h)
        t_setk = time.perf_counter() - t0
        for i in range(args.warmup):
            hctx.eph_interp_q(QB, q_h[i * QB:(i + 1) * QB], ekq_h, om_h, g_h)
        t0 = time.perf_counter()
        for i in range(args.warmup, nsteps):
            hctx.eph_interp_q(QB, q_h[i * QB:(i + 1) * QB], ekq_h, om_h, g_h)
        t_e2e = time.perf_counter() - t0
        hctx.close()
        e2e_units = args.steps * QB * nk * nm * nb * nb
        line["e2e"] = {"value": e2e_units / (t_e2e + t_setk * (args.steps * QB) / len(wl.qpts)), "unit": UNIT,
                       "h2d_bytes_per_step": QB * 3 * 8,
                       "d2h_bytes_per_step": g_h.numel() * g_h.element_size() + ekq_h.numel() * 8 + om_h.numel() * 8}
        del g_h
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample_k)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_libeph(args)


if __name__ == "__main__":
    sys.exit(main())
