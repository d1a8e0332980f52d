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
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one bench launch (q batch 4
# x 64000 k), from an ncu capture of that launch; profiles/k_zgemm_si_full_fp64.md,
# profiles/k_tc_fixed_gemm_si_full.md, profiles/k_jacobi_split_si_full.md.
# Keyed by (kernel, workload, q batch).
# Per-matrix work of the batched 8x8 H(k+q) eigensolve, keyed by (nb, form): (kernel, warp
# instructions issued, FP64 flops = 2 DFMA + DMUL + DADD thread instructions) per kernel of one eig
# call, from one ncu capture of the 55,296-matrix launches (bench.py --capture si-fp64-grid /
# si-mixed-grid; profiles/k_jacobi_split_si_full.md)
EIG_COUNTS = {(8, "fp64"): [("k_jacobi_f32<8>", 161562742 / 55296, 0.0),
                            ("k_jacobi_mixed<8>", 205258752 / 55296, (2 * 185794560 + 884736 + 69451776) / 55296)],
              (8, "mixed"): [("k_jacobi_f32<8>", 161562742 / 55296, 0.0),
                             ("k_jacobi_mixed<8>", 147654144 / 55296, (2 * 884736 + 442368 + 11059200) / 55296)]}
# instruction issue of GB300: 152 SMs x 4 schedulers x one warp instruction per clock x 2.07 GHz,
# which equals the FP64 unit peak in flop/s (152 SMs x 2 DFMA x 2 flop per clock): a kernel's floor
# in issue slots is max(warp instructions, FP64 flops)
ISSUE_PEAK = 152 * 4 * 2.07e9
# dram__bytes_read.sum + dram__bytes_write.sum of one launch at one step = 4 q x 64,000 k
TRAFFIC = {("k_tc_fixed_gemm", "si_full", 4): 185421824.0 + 731285504.0,
           ("k_zgemm", "si_full", 4): 242432512.0 + 1777470464.0,
           ("k_band_rotate", "si_full", 4): 2097285888.0 + 1534482688.0,
           # the 16,000-k capture (bench.py --capture si-fp64-list) scaled to the 64,000-k launch: the
           # phase digits and Y, which dominate, grow with the k rows (B digits, 22 MB, do not)
           ("k_tc_zgemm64", "si_full", 4): 4.0 * (137323520.0 + 412080128.0)}
# DRAM bytes per unit (pair or matrix) of the current kernels from the 24^3-grid captures
# (bench.py --capture si-fp64-grid / si-mixed-grid, 55,296 pairs per launch), scaled to a launch
# by its units: these kernels stream their inputs once, so traffic grows in proportion
TRAFFIC_PER_UNIT = {  # one eig call: k_jacobi_f32 + k_jacobi_mixed (A is read by both)
                    ("k_jacobi", "si_full", 4, "fp64"): (56677888.0 + 2453248.0 + 85100800.0 + 15118848.0) / 55296,
                    ("k_jacobi", "si_full", 4, "mixed"): (56679424.0 + 2064128.0 + 85020928.0 + 14424064.0) / 55296,
                    ("k_band_tc_small64", "si_full", 4, "grid"): (424918528.0 + 287893248.0) / 55296,
                    ("k_band_tc_small", "si_full", 4, "grid"): (424756224.0 + 136090112.0) / 55296}


def gpu_local_cpus(gpu_index):
    """CPUs of the NUMA node the GPU hangs off (sysfs, via the GPU's PCI bus id), or None.  Pinned
    host buffers first touched from those CPUs sit in the memory next to the GPU's link, so that
    device->host copies do not cross to the other CPU's memory."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(gpu_index)],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/numa_node"
        node = int(open(path).read().strip())
        if node < 0:
            return None, None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            if not part:
                continue
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return (cpus or None), node
    except (OSError, ValueError, subprocess.SubprocessError):
        return None, None


def fp64_peak_probe(dev):
    """Measured FP64 rates of this GPU: a DFMA loop (four independent FMA chains per element,
    compiled at run time by torch's jiterator, 4,096 flop per element over 2^24 elements) and
    cuBLAS DGEMM (torch.matmul, float64 8192^3); best of 5 each, CUDA events.  The rooflines'
    FP64 denominator stays the unit count x max clock; these numbers are printed beside it."""
    import torch
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def best(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        return min(t) * 1e-3

    try:
        from torch.cuda.jiterator import _create_jit_fn
        code = """
template <typename T> T dfma_chains(T x, T y) {
  T a0 = x, a1 = y, a2 = x + y, a3 = x - y;
  for (int i = 0; i < 512; ++i) {
    a0 = fma(a0, y, x); a1 = fma(a1, y, x); a2 = fma(a2, y, x); a3 = fma(a3, y, x);
  }
  return a0 + a1 + a2 + a3;
}"""
        fn = _create_jit_fn(code)
        x = torch.rand(1 << 24, dtype=torch.float64, device=dev)
        y = torch.full_like(x, 0.999)
        t = best(lambda: fn(x, y))
        out["dfma_loop_tflops"] = 4096.0 * x.numel() / t / 1e12
        del x, y
    except Exception as exc:  # noqa: BLE001 - a probe that cannot compile is reported, not fatal
        out["dfma_loop_error"] = str(exc).splitlines()[0][:200]
    a = torch.rand(8192, 8192, dtype=torch.float64, device=dev)
    b = torch.rand(8192, 8192, dtype=torch.float64, device=dev)
    t = best(lambda: torch.matmul(a, b), reps=3)
    out["dgemm_tflops"] = 2.0 * 8192 ** 3 / t / 1e12
    out["unit_count_tflops"] = FP64_PEAK_FLOPS / 1e12
    out["how"] = ("DFMA loop: jiterator elementwise kernel, 4 x 512 dependent FMA chains per element, 2^24 "
                  "elements; DGEMM: torch.matmul float64 8192^3; best of 5 / 3, CUDA events")
    del a, b
    torch.cuda.empty_cache()
    return out


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
    ap.add_argument("--fp64-only", action="store_true", help="skip the mixed-form measurement")
    ap.add_argument("--no-backward", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-linewidths", action="store_true", help="skip the fused linewidth measurement")
    ap.add_argument("--no-other", action="store_true", help="skip the MoS2- and stanene-shaped forward lines")
    ap.add_argument("--capture", default=None, choices=sorted(CAPTURES),
                    help="run one small untimed case for an ncu capture and exit (no JSON line)")
    ap.add_argument("--graph-full", action="store_true",
                    help="time only the batching workload with the stanene context's q batches as written "
                         "(1400 q, mixed form; minutes per replay) and print its JSON object")
    ap.add_argument("--k-path", default="grid", choices=["grid", "list"],
                    help="FP64 form: sum-factorised Re->k on the workload's uniform k grid, or the dense "
                         "Re->k GEMM on the k list")
    return ap.parse_args()


# ----------------------------------------------------------------------------- ncu capture cases
# name -> (workload, its overrides, form, q points per call, calls, kind).  Each sets the k list
# (kind "list": eph_set_k; "grid": eph_set_k_grid on the workload's grid) and makes `calls`
# eph_interp_q calls on device buffers, untimed; kind "backward" makes `calls` eph_interp_backward
# calls on the grid instead.  These are the programs the small-case profiles were taken from: a
# 120-band, 180-mode case small enough for a full-section capture of the band-rotation
# tensor-core product, the bench's stanene mixed leg, a silicon-shaped grid (Ne = 216) for the
# mixed and FP64 forms' band rotation (tensor cores; "-ff" / "-dfma": the CUDA-core kernels), and
# the MoS2-shaped differentiation workload on 8 q.
CAPTURES = {
    "stanene-band-tc": ("stanene", dict(nk=16, nq=2, box=(range(0, 1), range(-1, 2), range(0, 1))), "mixed", 1, 2,
                        "list"),
    "stanene-mixed": ("stanene", dict(nk=512, nq=8), "mixed", 4, 2, "list"),
    "si-mixed-grid": ("si_full", dict(nq=8), "mixed", 4, 2, "grid24"),
    "si-mixed-grid-ff": ("si_full", dict(nq=8), "mixed", 4, 2, "grid24", dict(band_alu=True)),
    "si-fp64-grid": ("si_full", dict(nq=8), "fp64", 4, 2, "grid24"),
    "si-fp64-grid-dfma": ("si_full", dict(nq=8), "fp64", 4, 2, "grid24", dict(band_alu=True)),
    "mos2-diff-backward": ("mos2_diff", dict(nq=8), "fp64", 4, 1, "backward"),
    # FP64 form on a k list of 16,000 random k with the silicon Re set: the tensor-core Re->k GEMM
    "si-fp64-list": ("si_full", dict(nk=16000, nq=8), "fp64", 4, 2, "list"),
}


def run_capture(args):
    import numpy as np
    import torch

    from paper_2603_10295_gb300 import binding, synth
    name, over, form, QB, calls, kind, *extra = CAPTURES[args.capture]
    extra = extra[0] if extra else {}
    dev = torch.device("cuda:0")
    wl = synth.make_workload(name, **over)
    if kind == "grid24":   # a 24^3 grid of the silicon-shaped workload: 13,824 k
        wl.kgrid = (24, 24, 24)
        wl.kpts = synth.uniform_grid(24, 24, 24)
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    ctx = binding.Context.from_workload(wl, form=form, device_ptrs=True, stream=torch.cuda.current_stream(),
                                        q_batch=QB, **extra)
    if kind == "list":
        ctx.eph_set_k(nk, torch.from_numpy(wl.kpts).to(dev))
    else:
        ctx.eph_set_k_grid(*wl.kgrid, None, None)
    q_d = torch.from_numpy(wl.qpts).to(dev)
    if kind == "backward":
        w = torch.from_numpy(np.full((nk, nb), 0.5)).to(dev)
        L = torch.zeros(1, dtype=torch.float64, device=dev)
        grad = torch.empty(wl.g_ReRp.shape, dtype=torch.complex128, device=dev)
        for i in range(calls):
            ctx.eph_interp_backward(nk, None, len(wl.qpts), q_d, w, 1e-6, L, grad)
    else:
        gdt = torch.complex128 if form == "fp64" else torch.complex64
        e = torch.empty(QB, nk, nb, dtype=torch.float64, device=dev)
        o = torch.empty(QB, nm, dtype=torch.float64, device=dev)
        g = torch.empty(QB, nk, nm, nb, nb, dtype=gdt, device=dev)
        for i in range(calls):
            ctx.eph_interp_q(QB, q_d[i * QB:(i + 1) * QB], e, o, g)
    torch.cuda.synchronize()
    print(f"capture {args.capture}: {wl.name} Nb={nb} Nm={nm} Ne={wl.ne}, {nk} k, {calls} call(s), "
          f"{ctx.launches()} kernel launches", flush=True)
    ctx.close()
    return 0


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


def cpu_baseline_config(wl, nq_full, nk_small, nk_large):
    """The FP64 oracle on a workload's full configuration, timed on samples and extrapolated.

    One q point at two random k subsets (nk_small, nk_large) gives the per-q time as a line in Nk:
    the k-independent part (the Rp->q sum of Eq. 9, D(q) and its eigensolve) plus a per-k part
    (H(k), H(k+q), their eigensolves, the Re->k sum and the band rotation).  The full grid's per-q
    time follows from that line; the configuration's time is Nq times it (the cost is linear in Nq
    apart from the k-only H(k) work, which the oracle repeats per q and this leaves in)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(1)
    perm = rng.permutation(len(wl.kpts))
    ts = []
    for n in (nk_small, nk_large):
        ks = np.sort(perm[:n])
        t0 = time.perf_counter()
        oracle.interpolate(wl, wl.kpts[ks], wl.qpts[:1])
        ts.append(time.perf_counter() - t0)
    per_k = max((ts[1] - ts[0]) / (nk_large - nk_small), 0.0)
    per_q0 = max(ts[0] - per_k * nk_small, 0.0)
    nk = len(wl.kpts)
    per_q = per_q0 + per_k * nk
    units = nk * wl.nm * wl.nb * wl.nb
    return {"value": units / per_q, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 q x {nk_small} and 1 q x {nk_large} random k of {nk} (numpy FP64, BLAS threads = "
                      f"all cores); per-q time fitted as a + b Nk, extrapolated to {nk} k and {nq_full} q",
            "seconds_sampled": sum(ts), "s_per_q_k_independent": per_q0, "s_per_k": per_k,
            "s_per_q_extrapolated": per_q, "s_full_config_extrapolated": per_q * nq_full}


def cpu_baseline_adjoint(wl, nq_full, w_nk, omega_min):
    """The FP64 oracle's loss and gradient (forward plus the reverse chain) on the full k grid for
    one and for two q points; per-q time = the difference, extrapolated linearly to nq_full q."""
    import oracle
    ts = []
    for nq in (1, 2):
        t0 = time.perf_counter()
        oracle.loss_and_grad(wl, wl.kpts, wl.qpts[:nq], w_nk, omega_min)
        ts.append(time.perf_counter() - t0)
    per_q = max(ts[1] - ts[0], 0.0)
    fixed = max(ts[0] - per_q, 0.0)
    el = len(wl.kpts) * wl.nm * wl.nb * wl.nb
    full = fixed + per_q * nq_full
    return {"value": el * nq_full / full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle.loss_and_grad on all {len(wl.kpts)} k for 1 and 2 q (numpy FP64); per-q time = "
                      f"their difference, extrapolated to {nq_full} q",
            "seconds_sampled": sum(ts), "s_per_q": per_q, "s_full_config_extrapolated": full}


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
BF16_PEAK_TFLOPS = None  # read from MEASURED_PEAKS.json when present


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def time_form(wl, form, args, q_dev, k_dev, rank, world, local, dev, QB, use_grid=False):
    """Times args.steps q batches of one form on the device (inputs resident in HBM).

    The timed steps run through an asynchronous context (no host synchronisation between calls,
    as a pipelined caller would run it); the per-stage breakdown comes from the same steps
    repeated through a synchronous context with CUDA-event profiling."""
    import torch

    from paper_2603_10295_gb300 import binding
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    # an explicit stream: the library enqueues on it and the timing events bracket its work
    # (torch's legacy default stream would leave the library on a stream of its own)
    st = torch.cuda.Stream()
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    gdt = torch.complex128 if form == "fp64" else torch.complex64
    eps_kq = torch.empty(QB, nk, nb, dtype=torch.float64, device=dev)
    om = torch.empty(QB, nm, dtype=torch.float64, device=dev)
    g = torch.empty(QB, nk, nm, nb, nb, dtype=gdt, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nsteps = args.warmup + args.steps

    def context(asyn):
        c = binding.Context.from_workload(wl, form=form, device_ptrs=True, q_batch=QB, stream=st, async_mode=asyn)
        torch.cuda.synchronize()
        e0.record(st)
        if use_grid:
            c.eph_set_k_grid(*wl.kgrid, None, eps_k)
        else:
            c.eph_set_k(nk, k_dev, eps_k)
        e1.record(st)
        torch.cuda.synchronize()
        c.eph_sync()
        return c, e0.elapsed_time(e1)

    ctx, setk_ms = context(True)

    def step(c, i):
        c.eph_interp_q(QB, q_dev[i * QB:(i + 1) * QB], eps_kq, om, g)

    for i in range(args.warmup):
        step(ctx, i)
    ctx.eph_sync()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0.record(st)
    for i in range(args.warmup, nsteps):
        step(ctx, i)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.eph_sync()  # device status flags of the timed calls
    el_ms = e0.elapsed_time(e1)
    launches = ctx.launches() - launches0
    ctx.close()
    # stage breakdown: the same steps, synchronous calls with CUDA-event profiling
    pctx, _ = context(False)
    step(pctx, 0)
    pctx.profile(True)
    pctx.profile_reset()
    for i in range(args.warmup, nsteps):
        step(pctx, i)
    prof = pctx.profile_read()
    pctx.profile(False)
    pctx.close()
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([el_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        el_ms = float(t.item())
    units_rank = args.steps * QB * nk * nm * nb * nb
    setk_share_ms = setk_ms * (args.steps * QB) / len(wl.qpts)
    out = dict(value=world * units_rank / ((el_ms + setk_share_ms) * 1e-3), ms_per_step=el_ms / args.steps,
               setk_ms=setk_ms, setk_share_ms=setk_share_ms, launches=launches, prof=prof, clocks=clk,
               g_bytes=g.numel() * g.element_size(), form=form)
    del g, eps_kq, om
    torch.cuda.empty_cache()
    return out


def time_backward(args, cpu=True):
    """eph_interp_backward on the differentiation workload (mos2_diff: 48x48 k grid x 256 q, FP64):
    the library call on the resident grid (forward Re->k sum and its adjoint sum-factorised), its
    stage breakdown, the same call on the points as a plain k list (dense GEMMs), and one
    optimisation step through torch.autograd (EphLoss forward + backward on device tensors)."""
    import numpy as np
    import torch

    from paper_2603_10295_gb300 import binding, synth
    from paper_2603_10295_gb300.autograd import EphLoss
    wl = synth.make_workload("mos2_diff")
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream()
    nk, nq, nb, nm = len(wl.kpts), len(wl.qpts), wl.nb, wl.nm
    k_d = torch.from_numpy(wl.kpts).to(dev)
    q_d = torch.from_numpy(wl.qpts).to(dev)
    e_d = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    ctx = binding.Context.from_workload(wl, device_ptrs=True, stream=st)
    ctx.eph_set_k_grid(*wl.kgrid, None, e_d)
    # Fermi weights at 300 K around the median of band 3 (1-based) over the k grid
    e = e_d.cpu().numpy()
    mu = float(np.median(e[:, 2]))
    w_np = 1.0 / (np.exp((e - mu) / 0.025852) + 1.0)
    w_d = torch.from_numpy(w_np).to(dev)
    L = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.empty(wl.g_ReRp.shape, dtype=torch.complex128, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()                                   # warm-up
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_grid = timed(lambda: ctx.eph_interp_backward(nk, None, nq, q_d, w_d, 1e-6, L, grad), 3)
    ctx.profile(True)
    ctx.profile_reset()
    ctx.eph_interp_backward(nk, None, nq, q_d, w_d, 1e-6, L, grad)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    lctx = binding.Context.from_workload(wl, device_ptrs=True, stream=st)
    ms_list = timed(lambda: lctx.eph_interp_backward(nk, k_d, nq, q_d, w_d, 1e-6, L, grad), 1)
    lctx.close()
    # one optimisation step through torch.autograd (the model's cached device context)
    gW = torch.from_numpy(wl.g_ReRp.copy()).to(dev).requires_grad_(True)

    def step():
        gW.grad = None
        EphLoss.apply(gW, wl, None, q_d, w_d, 1e-6).backward()

    ms_autograd = timed(step, 3)
    el = nk * nq * nm * nb * nb
    # the band stage of the backward call: per (q batch, k tile) two launches of the FP64-accuracy
    # tensor-core rotation k_band_tc_small64, g = V_{k+q}^H G3 V_k with the loss terms in its
    # epilogue (2 c g over G3, L per pair), then V_{k+q} (2 c g) V_k^H over the same rows.  Against
    # HBM: per pair G3 in and 2 c g out, 2 c g in and G3bar out (complex128 rows of Nm Nb^2), V_{k+q}
    # per pair and V_k per tile in each launch
    band_ms, band_n = prof.get("band", (0.0, 0))
    pairs = float(nk) * nq
    ppt = max(1, min(4, 128 // (((nm * nb + 31) // 32) * 32)))
    per_pair = 4 * 16.0 * nm * nb * nb + 2 * (16.0 * nb * nb + 16.0 * nb * nb / ppt) + 8.0 * nb
    ach = per_pair * pairs / (band_ms * 1e-3) if band_ms else None
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    roof = {"bound": "hbm",
            "kernel": "k_band_tc_small64 (tcgen05 kind::f16, six-digit operands, FP64 accuracy): the rotation with the "
                      "loss terms, then its adjoint (V conjugate-transposed) in place",
            "achieved": ach / 1e9 if ach else None, "peak": peak, "unit": "GB/s",
            "frac": ach / 1e9 / peak if (ach and peak) else None,
            "launches": band_n, "ms_per_launch": band_ms / max(band_n, 1),
            "algorithmic_bytes_per_pair": per_pair, "pairs_per_launch_pair": pairs / max(band_n // 2, 1),
            "cmac_per_pair": 4 * nb ** 3 * nm,
            "fp64_equivalent_tflops": 8.0 * 4 * nb ** 3 * nm * pairs / (band_ms * 1e-3) / 1e12 if band_ms else None,
            "share_of_call": band_ms / ms_grid if ms_grid else None,
            "note": "issue-bound on the integer digit arithmetic like the forward rotation "
                    "(profiles/k_band_tc_small64_si_fp64_grid24.md); the FP64 CUDA-core adjoint (band_alu) took "
                    "206.7 ms per call, 43 % of the FP64 peak",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs, measured" if peak else "unavailable"}
    return {"workload": "mos2_diff: Nb=11 Nm=9 Ne=Np=144, 48x48 k grid x 256 q, FP64 adjoint (forward recomputed)",
            "ms_per_call": ms_grid, "g_elements_per_s": el / (ms_grid * 1e-3), "k_path": "grid (kpts NULL)",
            "stage_ms_per_call": {k: round(v[0], 3) for k, v in prof.items() if v[0] > 0},
            "roofline": roof,
            "k_list": {"ms_per_call": ms_list, "g_elements_per_s": el / (ms_list * 1e-3)},
            "autograd_step": {"what": "EphLoss.apply + backward() on CUDA tensors: eph_set_gw (device copy of "
                                      "g(Re,Rp)), eph_interp_backward on the grid, grad scaling",
                              "ms_per_step": ms_autograd, "host_round_trips": 0},
            "parity": "vs FP64 CPU adjoint <= 1e-12, central differences <= 1e-6 (tests/test_gpu_adjoint.py)",
            # the same loss and gradient by the FP64 oracle on the host cores (same weights)
            "cpu_baseline": cpu_baseline_adjoint(wl, nq, w_np, 1e-6) if cpu else None}


def time_linewidths(wl, args, q_dev, k_dev, dev, QB, use_grid=False):
    """eph_linewidths (FP64 consumer of g) over the same q points the timed steps cover."""
    import torch

    from paper_2603_10295_gb300 import binding
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    st = torch.cuda.current_stream()
    ctx = binding.Context.from_workload(wl, device_ptrs=True, q_batch=QB, stream=st)
    eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    if use_grid:
        ctx.eph_set_k_grid(*wl.kgrid, None, eps_k)
    else:
        ctx.eph_set_k(nk, k_dev, eps_k)
    gamma = torch.empty(nk, nb, dtype=torch.float64, device=dev)
    nq = args.steps * QB
    qs = q_dev[args.warmup * QB:args.warmup * QB + nq]
    ctx.eph_linewidths(QB, q_dev[:QB], None, 0.025852, 0.0, 0.05, 1e-6, gamma)   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    ctx.eph_linewidths(nq, qs, None, 0.025852, 0.0, 0.05, 1e-6, gamma)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    return {"what": f"electron linewidths (imaginary Fan-Migdal self-energy, 300 K, Gaussian 0.05 eV) over "
                    f"{nq} q x {nk} k; g formed over the G3 rows of the k-tile workspace by the FP64-accuracy "
                    "tensor-core rotation and reduced there by k_linewidth_terms, never returned",
            "ms_per_step": ms / args.steps, "g_elements_per_s": nq * nk * nm * nb * nb / (ms * 1e-3),
            "parity": "vs oracle.linewidths <= 1e-10 per k (tests/test_gpu_linewidths.py)"}


def time_workload(name, args, dev, legs, warmup, steps, cpu_k=None):
    """Forward throughput on another of the paper-shaped workloads (device buffers, CUDA events).
    legs: (form, uniform-grid path, q points per call); cpu_k: the two k sample sizes of the
    oracle's timing on the same workload (None: no CPU baseline)."""
    import torch

    from paper_2603_10295_gb300 import binding, synth
    wl = synth.make_workload(name)
    nk, nb, nm = len(wl.kpts), wl.nb, wl.nm
    out = {"workload": describe(wl, argparse.Namespace(q_batch=legs[0][2]))}
    for form, grid, QB in legs:
        q_dev = torch.from_numpy(wl.qpts[:(warmup + steps) * QB].copy()).to(dev)
        st = torch.cuda.current_stream()
        ctx = binding.Context.from_workload(wl, form=form, device_ptrs=True, q_batch=QB, stream=st)
        if grid:
            ctx.eph_set_k_grid(*wl.kgrid, None, None)
        else:
            ctx.eph_set_k(nk, torch.from_numpy(wl.kpts).to(dev), None)
        gdt = torch.complex128 if form == "fp64" else torch.complex64
        e = torch.empty(QB, nk, nb, dtype=torch.float64, device=dev)
        o = torch.empty(QB, nm, dtype=torch.float64, device=dev)
        g = torch.empty(QB, nk, nm, nb, nb, dtype=gdt, device=dev)
        for i in range(warmup):
            ctx.eph_interp_q(QB, q_dev[i * QB:(i + 1) * QB], e, o, g)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_reset()
        e0.record(st)
        for i in range(warmup, warmup + steps):
            ctx.eph_interp_q(QB, q_dev[i * QB:(i + 1) * QB], e, o, g)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = ctx.profile_read()
        key = form + ("_grid" if grid else "_list")
        out[key] = {"value": QB * nk * nm * nb * nb / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "q_per_step": QB,
                    "stage_ms_per_step": {k: round(v[0] / steps, 3) for k, v in prof.items() if v[0] > 0}}
        del g, e, o
        ctx.close()
        torch.cuda.empty_cache()
    if cpu_k is not None:
        out["cpu_baseline"] = cpu_baseline_config(wl, synth.CONFIGS[name]["q"][1], *cpu_k)
    return out


# the batching workload: stanene-shaped (full shapes, 512 k) with uneven q batches in one CUDA graph
# with a silicon-shaped (Nb=8) and a MoS2-shaped (Nb=11) context.  The silicon- and MoS2-shaped
# contexts take the batch sizes as written (1400 q); the stanene context the first batches of
# the list, scaled so that a replay stays ~10 s (one stanene q costs ~0.17 s mixed, ~2.1 s FP64).
GRAPH_STANENE = {"mixed": ([17, 40, 11], 4), "fp64": ([1, 2], 1)}


def time_batched_graph(form, dev, replays=3, full=False):
    """One captured graph over three materials (GraphBatcher), autotuned tiles; total g el/s over
    the replays and each material's share (its calls timed eagerly, one after the other)."""
    import torch

    from paper_2603_10295_gb300 import synth
    from paper_2603_10295_gb300.batching import graph_of_materials
    batches = list(synth.STANENE_Q_BATCHES)
    si = synth.make_workload("si_tiny", nk=1024, nq=sum(batches))
    mo = synth.make_workload("mos2_diff", nq=sum(batches))
    st = synth.make_workload("stanene")
    sb, sch = (batches, 4) if full else GRAPH_STANENE[form]
    specs = [(si, batches, 16, False), (mo, batches, 16, True), (st, sb, sch, False)]
    gb, mats = graph_of_materials(specs, form, dev, autotune=True)
    gb.replay()                     # warm replay (the capture's eager pass ran before it)
    gb.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(gb.stream)
    for _ in range(replays):
        gb.replay()
    e1.record(gb.stream)
    gb.check()
    ms = e0.elapsed_time(e1) / replays
    # each material's calls alone, eagerly (the per-material share of the work)
    eager = []
    for m in mats:
        with torch.cuda.stream(gb.stream):
            e0.record(gb.stream)
            for ctx, q, e, o, g in gb.items:
                if ctx is m.ctx:
                    ctx.eph_interp_q(q.shape[0], q, e, o, g)
            e1.record(gb.stream)
        gb.check()
        eager.append(e0.elapsed_time(e1))
    total_el = sum(m.g_elements() for m in mats)
    out = {"value": total_el / (ms * 1e-3), "unit": UNIT, "ms_per_replay": ms, "replays": replays,
           "graph_launches_per_replay": 1, "library_calls_per_replay": len(gb.items),
           "eager_sum_ms": sum(eager), "materials": []}
    for m, t in zip(mats, eager):
        out["materials"].append({"workload": m.wl.name, "nb": m.wl.nb, "nm": m.wl.nm, "ne": m.wl.ne, "nk": m.nk,
                                 "k_path": "grid" if m.grid else "list", "q_batches": m.batches,
                                 "q_per_call": m.chunk, "autotuned_q_batch_k_tile": list(m.tuned),
                                 "g_elements": m.g_elements(), "eager_ms": t, "time_share": t / sum(eager),
                                 "g_el_per_s_eager": m.g_elements() / (t * 1e-3)})
        m.ctx.close()
    del gb, mats
    torch.cuda.empty_cache()
    return out


def time_multi_material(dev, replays=5):
    """Three FP64 materials with uneven q batches (Si-shaped Nb=8, MoS2-shaped Nb=11 on a 12x12
    grid, a 3-band one-atom Si box), few k points each so that one (q batch, k tile) of one material
    fills well under one wave of the SMs: one CUDA graph of separate eph_interp_q calls against one
    graph of a single eph_interp_q_multi call, whose band rotations run as one persistent launch
    per round over every material's pairs."""
    import torch

    from paper_2603_10295_gb300 import binding, synth
    from paper_2603_10295_gb300.batching import GraphBatcher
    mo = synth.make_workload("mos2_diff", nq=40)
    mo.kgrid, mo.kpts = (12, 12, 1), synth.uniform_grid(12, 12, 1)
    mats = [(synth.make_workload("si_tiny", nk=256, nq=40), 17, False), (mo, 11, True),
            (synth.make_workload("si_tiny", nb=3, na=1, nk=128, nq=40), 25, False)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for mode in ("separate", "multi"):
        gb = GraphBatcher(dev)
        ctxs, qs, bufs = [], [], []
        for wl, nq, grid in mats:
            c = binding.Context.from_workload(wl, device_ptrs=True, async_mode=True, stream=gb.stream, q_batch=4)
            with torch.cuda.stream(gb.stream):
                if grid:
                    c.eph_set_k_grid(*wl.kgrid, None, None)
                else:
                    c.eph_set_k(len(wl.kpts), torch.from_numpy(wl.kpts).to(dev))
            nk, nb, nm = c.nk, wl.nb, wl.nm
            q = torch.from_numpy(wl.qpts[:nq].copy()).to(dev)
            b = (torch.empty(nq, nk, nb, dtype=torch.float64, device=dev),
                 torch.empty(nq, nm, dtype=torch.float64, device=dev),
                 torch.empty(nq, nk, nm, nb, nb, dtype=torch.complex128, device=dev))
            ctxs.append(c)
            qs.append(q)
            bufs.append(b)
            if mode == "separate":
                gb.add(c, q, *b)
        if mode == "multi":
            gb.add_multi(ctxs, qs, [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs])
        gb.capture()
        gb.replay()
        gb.check()
        torch.cuda.synchronize()
        e0.record(gb.stream)
        for _ in range(replays):
            gb.replay()
        e1.record(gb.stream)
        gb.check()
        ms = e0.elapsed_time(e1) / replays
        el = sum(nq * c.nk * wl.nm * wl.nb * wl.nb for (wl, nq, _), c in zip(mats, ctxs))
        launches = sum(c.launches() for c in ctxs)
        out[mode] = {"ms_per_replay": ms, "value": el / (ms * 1e-3), "unit": UNIT,
                     "kernel_launches_total": launches}
        for c in ctxs:
            c.close()
        del gb, bufs
        torch.cuda.empty_cache()
    out["materials"] = [{"workload": wl.name, "nb": wl.nb, "nm": wl.nm, "q": nq, "k_path": "grid" if g else "list"}
                        for wl, nq, g in mats]
    out["multi_over_separate"] = out["separate"]["ms_per_replay"] / out["multi"]["ms_per_replay"]
    return out


def run_libeph(args):
    import numpy as np
    import torch

    from paper_2603_10295_gb300 import binding, synth
    from paper_2603_10295_gb300.sharding import step_q_indices

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = synth.make_workload(args.workload)
    nk, nb, nm, ne = len(wl.kpts), wl.nb, wl.nm, wl.ne
    QB = args.q_batch
    # this rank's q points: a contiguous block of the (cyclically extended) q list
    nsteps = args.warmup + args.steps
    qidx = step_q_indices(len(wl.qpts), nsteps, QB, rank, world)
    q_dev = torch.from_numpy(np.ascontiguousarray(wl.qpts[qidx])).to(dev)
    k_dev = torch.from_numpy(wl.kpts).to(dev)

    use_grid = args.k_path == "grid" and wl.kgrid is not None
    # (form, grid) legs: the headline first, the mixed form on the same path, then the
    # dense-GEMM k-list path of both forms
    legs = [("fp64", use_grid)]
    if args.form == "mixed":
        legs = [("mixed", use_grid)]
    elif not args.fp64_only:
        legs.append(("mixed", use_grid))
        if use_grid:
            legs += [("fp64", False), ("mixed", False)]
    res = {(f, gr): time_form(wl, f, args, q_dev, k_dev, rank, world, local, dev, QB, use_grid=gr) for f, gr in legs}
    head = res[legs[0]]
    forms = [legs[0][0]]
    peaks = measured_peaks()

    def roof_axis(r):
        # axis-1 transform of the product-grid path (k_axis_dft, the per-k part; the axis-3 and
        # axis-2 transforms run per q batch in stage "mode"): on the symmetric slots of half-width
        # M, an output pair (j, N-j) takes 4M FMA and 4 additions = 4M + 2 flop per output
        ft_ms, ft_n = r["prof"]["ft_k"]
        M = int(np.abs(wl.Re[:, 0]).max())
        NW = nb * nb * (1 + nm)
        outs = float(args.steps) * QB * nk * NW / max(ft_n, 1)
        t = ft_ms / max(ft_n, 1) * 1e-3
        ach = (4 * M + 2) * outs / t
        # the slot columns read once (16 B), the outputs written once: 16 B each, except the mixed
        # form's G3 columns (all but the first Nb^2 of each row), written as complex64
        mixed_out = r.get("form") == "mixed"
        out_bytes = (16.0 * nb * nb + (8.0 if mixed_out else 16.0) * nm * nb * nb) / NW
        algo = outs * (out_bytes + 16.0 * (2 * M + 1) / float(wl.kgrid[0]))
        if r.get("form") == "mixed" or 2 * M + 1 <= 9:
            # the double-float kernel (k_axis_dft_df, FP32 pipe): its floor is the HBM traffic
            peak = peaks.get("hbm_gbs")
            gbs = algo / t / 1e9
            return {"bound": "hbm",
                    "kernel": "k_axis_dft_df (axis 1 of the sum-factorised Re->k contraction, double-float on the "
                              "FP32 pipe)",
                    "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak if peak else None,
                    "algorithmic_bytes": algo, "outputs_per_launch": outs,
                    "fp64_equivalent_tflops": ach / 1e12, "flop_per_output": 4 * M + 2,
                    "note": "algorithmic bytes: the slot columns read once (16 B), the outputs written once (16 B; "
                            "the mixed form's G3 columns 8 B, complex64 for the band rotation); the FP64 kernel "
                            "k_axis_dft ran this stage at 75 % of the FP64 peak",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs, measured" if peak else "unavailable"}
        return {"bound": "alu", "kernel": "k_axis_dft (axis 1 of the sum-factorised Re->k contraction)",
                "achieved": ach / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_FLOPS, "flop_per_output": 4 * M + 2, "outputs_per_launch": outs,
                "algorithmic_bytes": algo}

    def roof_hkq(r):
        # H(k+q) on the tensor cores: 15 bf16 digit products per K step (5 x 5 digits, levels <= 4);
        # stage ft_k of the mixed k-list path also holds the float-pair -> complex128 conversion
        ft_ms, ft_n = r["prof"]["ft_k"]
        kpd = ((2 * ne + 63) // 64) * 64
        nrh = 2 * nb * nb
        mpad = ((nk + 127) // 128) * 128
        npad = ((nrh + 127) // 128) * 128
        issued = 15 * 2.0 * mpad * npad * kpd * QB
        t = ft_ms / max(args.steps, 1) * 1e-3
        peak = peaks.get("bf16_tflops")
        useful = 8.0 * nk * nb * nb * ne * QB
        return {"bound": "tensor", "kernel": "k_tc_hkq_gemm (tcgen05 kind::f16, 5 x 5 BF16 digits) + conversion",
                "achieved": useful / t / 1e12 if t else None, "peak": peak, "unit": "TFLOP/s",
                "frac": (useful / t / 1e12 / peak) if (t and peak) else None,
                "achieved_issued": issued / t / 1e12 if t else None,
                "frac_issued": (issued / t / 1e12 / peak) if (t and peak) else None, "ms_per_step": ft_ms / args.steps,
                "useful_tflops": useful / t / 1e12 if t else None}

    def roof_band(r):
        if nb <= 16 and nm * nb <= 128:  # the default FP64 rotation: six-digit tensor-core products
            return roof_band_tc(r, 16.0, fp64=True)
        bd_ms, bd_n = r["prof"]["band"]
        cmac = 2.0 * nb ** 3 * nm * QB * nk          # V_kq^H G3 V_k per (q,k) pair
        t = bd_ms / max(args.steps, 1) * 1e-3
        ach = 8.0 * cmac / t                         # the method's work: 8 flop per complex multiply-add
        issued = 6.0 * cmac / t                      # three-multiplication form: 3 FMA per CMAC
        pairs = float(QB) * nk
        return {"bound": "alu", "kernel": "k_band_rotate (FP64, three-multiplication products)",
                "achieved": ach / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_FLOPS, "flop_per_cmac": 8,
                "frac_issued": issued / FP64_PEAK_FLOPS, "issued_flop_per_cmac": 6,
                "note": "frac counts 8 flop per complex multiply-add of 2 Nb^3 Nm per pair; the kernel issues "
                        "3 DFMA (6 flop) per one in the three-multiplication form, hence frac > frac_issued",
                "traffic": TRAFFIC.get(("k_band_rotate", args.workload, QB)),
                # G3 rows, V_k and V_{k+q} read, g written (complex128)
                "algorithmic_bytes": 16.0 * (pairs * (nm * nb * nb + nb * nb + nb * nb) + pairs * nm * nb * nb),
                "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 unit count, max clock)"}

    def roof_eig(r, form="fp64"):
        # each kernel of the eigensolve is bounded by its warp instructions at one per scheduler and
        # clock or by its FP64 flops at the FP64 unit peak, whichever is larger (both in issue
        # slots, the two peaks being equal); the kernels run one after the other, so their floors add
        eg_ms, eg_n = r["prof"]["eig"]
        ks = EIG_COUNTS.get((nb, form))
        t = eg_ms / max(eg_n, 1) * 1e-3
        mats = float(args.steps) * QB * nk / max(eg_n, 1)
        npd = nb + (nb & 1)
        out = {"bound": "alu",
               "kernel": "k_jacobi_f32<%d> (FP32 Jacobi sweeps) + k_jacobi_mixed<%d> (Ogita-Aishima refinement: "
                         "one double-float step on the FP32 pipe%s)"
                         % (npd, npd, ", one FP64 step" if form == "fp64" else ""),
               "achieved": None, "peak": ISSUE_PEAK / 1e12, "unit": "T issue slots/s", "frac": None,
               "matrices_per_call": mats,
               "traffic": (TRAFFIC_PER_UNIT.get(("k_jacobi", args.workload, QB, form), 0.0) * mats) or None,
               "algorithmic_bytes": mats * (nb * nb * 16 + nb * nb * 16 + nb * 8),
               "peak_source": "152 SMs x 4 schedulers x 1 warp instruction/clk x 2.07 GHz (= the FP64 unit "
                              "peak in flop/s)"}
        if not (ks and t):
            return out
        slots = sum(max(wi, f64) for _, wi, f64 in ks)
        out.update({"achieved": slots * mats / t / 1e12, "frac": slots * mats / ISSUE_PEAK / t,
                    "issue_slots_per_matrix": slots,
                    "per_kernel": [{"kernel": k, "warp_inst_per_matrix": wi, "fp64_flop_per_matrix": f64,
                                    "binding": "FP64 pipe" if f64 > wi else "instruction issue"}
                                   for k, wi, f64 in ks]})
        return out

    def roof_band_tc(r, g3_bytes, fp64=False, grid=False):
        # the fused tensor-core band rotation (k_band_tc_small, mixed; k_band_tc_small64, FP64 form)
        # against HBM: G3 rows in (complex128 from the FP64 grid transforms, complex64 from the
        # tensor-core contraction), V_{k+q} per pair and V_k per tile of pairs (two q at one k for
        # these shapes) in, g out (complex64 mixed, complex128 FP64)
        bd_ms, bd_n = r["prof"]["band"]
        pairs = float(args.steps) * QB * nk
        ppt = max(1, min(4, 128 // (((nm * nb + 31) // 32) * 32)))
        gbytes = 16.0 if fp64 else 8.0
        per_pair = g3_bytes * nm * nb * nb + 16.0 * nb * nb + 16.0 * nb * nb / ppt + gbytes * nm * nb * nb
        t = bd_ms * 1e-3
        ach = per_pair * pairs / t if t else None
        peak = peaks.get("hbm_gbs")
        # traffic per pair from the 24^3 captures: the FP64 kernel on the grid path; the mixed kernel's
        # capture read complex128 G3, which its grid path no longer does (complex64 from axis 1)
        key = ("k_band_tc_small64" if fp64 else "k_band_tc_small", args.workload, QB,
               "grid" if (g3_bytes == 16.0 and not grid) else ("grid_c64" if grid else "list"))
        tr = TRAFFIC_PER_UNIT.get(key)
        return {"bound": "hbm",
                "kernel": "k_band_tc_small64 (tcgen05 kind::f16, six-digit operands, exact level sums, FP64 accuracy, "
                          "no FP64 instruction)" if fp64 else
                          "k_band_tc_small (tcgen05 kind::f16, four-digit fixed-point BF16 operands)",
                "achieved": ach / 1e9 if ach else None, "peak": peak, "unit": "GB/s",
                "frac": (ach / 1e9 / peak) if (ach and peak) else None,
                "algorithmic_bytes_per_pair": per_pair, "pairs_per_launch": pairs / max(bd_n, 1),
                "traffic": tr * pairs / max(bd_n, 1) if tr else None,
                "cmac_per_pair": 2 * nb ** 3 * nm,
                "note": ("issue-bound on integer digit arithmetic (ncu: 48 % issue, ALU pipe 49 %, tensor pipe 8 %); "
                         "profiles/k_band_tc_small64_si_fp64_grid24.md" if fp64 else
                         "issue-bound on the digit arithmetic (ncu: 63 % issue, tensor pipe 9 %, DRAM 26 %); "
                         "profiles/k_band_tc_small_si_mixed_grid24.md")
                + "; traffic = DRAM bytes per pair of the 24^3 capture x pairs per launch",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs, measured" if peak else "unavailable"}

    def dominant_roofline(r):
        st = {k: v[0] for k, v in r["prof"].items()}
        top = max(("ft_k", "eig", "band"), key=lambda s: st.get(s, 0.0))
        if top == "eig":
            return roof_eig(r)
        if top == "band":
            return roof_band(r)
        return roof_fp64(r)

    def roof_fp64(r):
        ft_ms, ft_n = r["prof"]["ft_k"]
        NW = nb * nb * (1 + nm)
        # the timed steps cover steps x QB q points x all k; each launch one (q batch, k tile)
        cmac_launch = float(args.steps) * QB * nk * NW * ne / max(ft_n, 1)
        t = ft_ms / max(ft_n, 1) * 1e-3 if ft_n else None
        nkt = -(-nk // max(ft_n // max(args.steps, 1), 1))
        # P_k tile read, W_q read, Y = [H(k+q) | G3] written once (complex128)
        algo_bytes = 16.0 * (nkt * ne + QB * ne * NW + QB * nkt * NW)
        # the method's work: 8 flop per complex multiply-add; the kernel (3M) issues 3 DFMA = 6 flop
        ach = 8.0 * cmac_launch / t if t else None
        issued = 6.0 * cmac_launch / t if t else None
        if 2 * ne <= 512 and nb <= 16 and nm <= 16:
            # the tensor-core form (k_tc_zgemm64): 34 bf16 digit products per K step on the real
            # embedding (M = k tile, N = 2 NW per q, K = 2 Ne padded to 32); digits read once, Y
            # written once in complex128
            kp = ((2 * ne + 31) // 32) * 32
            iss = 34 * 2.0 * nkt * 2 * NW * kp * QB
            peak = peaks.get("bf16_tflops")
            useful = ach / 1e12 if ach else None
            return {"bound": "tensor",
                    "kernel": "k_tc_zgemm64 (Re->k contraction fused with H(k+q) at FP64 accuracy: tcgen05 kind::f16, "
                              "seven base-128 digits per operand, exact level sums, integer-assembled doubles)",
                    "achieved": useful, "peak": peak, "unit": "TFLOP/s",
                    "frac": useful / peak if (useful and peak) else None, "flop_per_cmac": 8,
                    "achieved_issued": iss / t / 1e12 if t else None,
                    "frac_issued": iss / t / 1e12 / peak if (t and peak) else None,
                    "note": "frac: the complex contraction at 8 flop per complex multiply-add; frac_issued: the 34 "
                            "digit products per K step the kernel issues; the FP64 DFMA GEMM (option gemm_alu) ran "
                            "this stage at 94 % of the FP64 peak in 123 ms per step",
                    "algorithmic_bytes": 2.0 * 7 * (nkt * kp + QB * 2 * NW * kp) + 16.0 * QB * nkt * NW,
                    "traffic": TRAFFIC.get(("k_tc_zgemm64", args.workload, QB)),
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), measured" if peak else "unavailable"}
        return {"bound": "alu", "kernel": "k_zgemm (Re->k contraction fused with H(k+q), FP64 DFMA, 3M)",
                "achieved": ach / 1e12 if ach else None, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": (ach / FP64_PEAK_FLOPS) if ach else None, "flop_per_cmac": 8,
                "frac_issued": (issued / FP64_PEAK_FLOPS) if issued else None, "issued_flop_per_cmac": 6,
                "traffic": TRAFFIC.get(("k_zgemm", args.workload, QB)), "algorithmic_bytes": algo_bytes,
                "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 unit count, max clock)"}

    def roof_tc(r):
        tc_ms, tc_n = r["prof"]["tc"]
        kpd = ((2 * ne + 63) // 64) * 64
        nr = 2 * nm * nb * nb
        tiles = max(tc_n // max(args.steps, 1), 1)      # k tiles per q batch
        mpad = ((-(-nk // tiles) + 127) // 128) * 128
        npad = ((nr + 127) // 128) * 128
        issued = 9 * 2.0 * mpad * npad * kpd * QB     # nine bf16 digit products per K step
        useful = 8.0 * nk * nm * nb * nb * ne * QB / tiles     # complex Re->k contraction, 8 flop per CMAC
        t = tc_ms / max(tc_n, 1) * 1e-3 if tc_n else None
        # A digits (3) and B digits (4) in bf16 read once, the FP32 product written once
        algo_bytes = 2.0 * (3 * mpad * kpd + 4 * QB * npad * kpd) + 4.0 * QB * min(mpad, nk) * nr
        peak = peaks.get("bf16_tflops")
        return {"bound": "tensor", "kernel": "k_tc_fixed_gemm (tcgen05 kind::f16, fixed-point BF16 digits)",
                "achieved": useful / t / 1e12 if t else None, "peak": peak, "unit": "TFLOP/s",
                "frac": (useful / t / 1e12 / peak) if (t and peak) else None,
                "achieved_issued": issued / t / 1e12 if t else None,
                "frac_issued": (issued / t / 1e12 / peak) if (t and peak) else None,
                "note": "frac: the complex Re->k contraction at 8 flop per complex multiply-add; frac_issued: the "
                        "nine bf16 digit products the kernel issues per K step on the real embedding",
                "useful_tflops": useful / t / 1e12 if t else None, "ms_per_launch": tc_ms / max(tc_n, 1),
                "traffic": TRAFFIC.get(("k_tc_fixed_gemm", args.workload, QB)), "algorithmic_bytes": algo_bytes,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), measured" if peak else "unavailable"}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if forms[0] == "fp64" else "bf16-digits/f32",
                "data": "synthetic",
                "config": {"workload": describe(wl, args), "form": forms[0], "q_batch": QB,
                           "k_path": ("uniform grid %dx%dx%d, sum-factorised Re->k (eph_set_k_grid)" % wl.kgrid)
                           if legs[0][1] else "k list, dense Re->k GEMM (eph_set_k)",
                           "l2": "inputs larger than L2: g(Re,Rp) 287 MB, P_k 221 MB resident; "
                                 f"g out {head['g_bytes'] / 1e9:.2f} GB per step",
                           "k_setup_ms": head["setk_ms"], "k_setup_share_ms": head["setk_share_ms"],
                           "stage_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in head["prof"].items()},
                           "parity": "FP64 form vs FP64 CPU oracle: max rel err <= 1e-12 (eps, omega, |g|^2 "
                                     "subspace sums); tests/test_gpu_parity.py"},
                "roofline": dominant_roofline(head) if forms[0] == "fp64" else roof_tc(head),
                "gpu_launches": head["launches"], "clocks": head["clocks"]}
        if forms[0] == "fp64":
            line["stage_rooflines"] = {"band": roof_band(head), "eig": roof_eig(head)}
            if legs[0][1]:
                line["stage_rooflines"]["ft_k"] = roof_axis(head)
        if ("mixed", use_grid) in res and forms[0] == "fp64":
            m = res[("mixed", use_grid)]
            line["mixed"] = {"value": m["value"], "unit": UNIT, "ms_per_step": m["ms_per_step"],
                             "k_path": line["config"]["k_path"],
                             "gain_vs_fp64": m["value"] / head["value"],
                             "dtype": "double-float (FP32 pipe) Re->k axis transforms and eigensolve refinement, "
                                      "tensor-core (bf16 digit) band rotation and Eq. 9, c64 g" if use_grid
                                      else "bf16 digits / f32 accumulate",
                             "rel_err_bar": "<= 1e-6 on |g|^2 subspace sums (tests/test_gpu_mixed.py, "
                                            "tests/test_gpu_grid.py); eps, omega <= 1e-10",
                             "stage_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in m["prof"].items()},
                             "gpu_launches": m["launches"], "clocks": m["clocks"]}
            mst = {k: v[0] for k, v in m["prof"].items()}
            if use_grid:
                sr = {"eig": roof_eig(m, "mixed"), "ft_k": roof_axis(m), "band": roof_band_tc(m, 8.0, grid=True)}
                line["mixed"]["roofline"] = sr[max(("eig", "ft_k", "band"), key=lambda k: mst.get(k, 0.0))]
                line["mixed"]["stage_rooflines"] = sr
            else:
                line["mixed"]["roofline_tensor_kernel"] = roof_tc(m)
        if use_grid and ("fp64", False) in res:
            fl, ml = res[("fp64", False)], res[("mixed", False)]
            line["k_list"] = {
                "what": "the same k points as a plain k list: dense Re->k GEMM (FP64) or tcgen05 (mixed)",
                "fp64": {"value": fl["value"], "unit": UNIT, "ms_per_step": fl["ms_per_step"],
                         "stage_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in fl["prof"].items()},
                         "roofline": roof_fp64(fl), "gpu_launches": fl["launches"], "clocks": fl["clocks"]},
                "mixed": {"value": ml["value"], "unit": UNIT, "ms_per_step": ml["ms_per_step"],
                          "gain_vs_fp64": ml["value"] / fl["value"], "dtype": "bf16 digits / f32 accumulate",
                          "rel_err_bar": "<= 1e-6 on |g|^2 subspace sums (measured 4.1e-7 si_full); eps_kq <= 1e-10 "
                                         "(measured 2.1e-11)",
                          "stage_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in ml["prof"].items()},
                          "roofline_tensor_kernel": roof_tc(ml), "roofline_hkq_kernel": roof_hkq(ml),
                          "roofline_band_kernel": roof_band_tc(ml, 8.0),
                          "gpu_launches": ml["launches"], "clocks": ml["clocks"]}}

    # end to end through the public C-ABI with HOST buffers (pinned), copies inside the timed region
    def e2e(form, grid=False):
        # through the C-ABI with pinned host buffers.  The FP64 flow (and the mixed form on the grid
        # path) runs in async mode: a step's g is copied to the host while the next step computes,
        # into one of two alternating output sets; eph_sync at the end of the timed region waits for
        # every copy.  The tensor-core k-list path of the mixed form runs synchronously.
        gdt = torch.complex128 if form == "fp64" else torch.complex64
        asyn = form == "fp64" or grid
        # host thread and pinned buffers on the GPU's own NUMA node (restored after the leg)
        cpus, node = gpu_local_cpus(local)
        old_aff = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
        if cpus and old_aff is not None:
            try:
                os.sched_setaffinity(0, cpus & old_aff or cpus)
            except OSError:
                node = None
        hctx = binding.Context.from_workload(wl, form=form, device_ptrs=False, q_batch=QB, async_mode=asyn)
        kp_h = torch.from_numpy(wl.kpts).pin_memory()
        epsk_h = torch.empty(nk, nb, dtype=torch.float64).pin_memory()
        q_h = torch.from_numpy(np.ascontiguousarray(wl.qpts[qidx])).pin_memory()
        outs = [(torch.empty(QB, nk, nb, dtype=torch.float64).pin_memory(),
                 torch.empty(QB, nm, dtype=torch.float64).pin_memory(),
                 torch.empty(QB, nk, nm, nb, nb, dtype=gdt).pin_memory()) for _ in range(2 if asyn else 1)]
        t0 = time.perf_counter()
        if grid:
            hctx.eph_set_k_grid(*wl.kgrid, None, epsk_h)
        else:
            hctx.eph_set_k(nk, kp_h, epsk_h)
        hctx.eph_sync()
        t_setk = time.perf_counter() - t0
        for i in range(args.warmup):
            hctx.eph_interp_q(QB, q_h[i * QB:(i + 1) * QB], *outs[i % len(outs)])
        hctx.eph_sync()
        # three timed passes over the same K steps, the median reported: the copies share the
        # host's memory and link with other tenants, and single passes of the same code have
        # ranged over 1.6x
        passes = []
        for _ in range(3):
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
                torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(args.warmup, nsteps):
                hctx.eph_interp_q(QB, q_h[i * QB:(i + 1) * QB], *outs[i % len(outs)])
            hctx.eph_sync()
            passes.append(time.perf_counter() - t0)
        t_e2e = sorted(passes)[1]
        hctx.close()
        if cpus and old_aff is not None:
            try:
                os.sched_setaffinity(0, old_aff)
            except OSError:
                pass
        if world > 1:  # whole job: every rank's units over the slowest rank's time
            t = torch.tensor([t_e2e, t_setk], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e, t_setk = (float(x) for x in t.tolist())
        ekq_h, om_h, g_h = outs[0]
        e2e_units = world * args.steps * QB * nk * nm * nb * nb
        out = {"value": e2e_units / (t_e2e + t_setk * (args.steps * QB) / len(wl.qpts)), "unit": UNIT,
               "h2d_bytes_per_step": QB * 3 * 8,
               "d2h_bytes_per_step": g_h.numel() * g_h.element_size() + ekq_h.numel() * 8 + om_h.numel() * 8,
               "ms_per_step": 1e3 * t_e2e / args.steps, "k_setup_ms": 1e3 * t_setk,
               "host_numa_node": node, "d2h_gbs_effective": (g_h.numel() * g_h.element_size() + ekq_h.numel() * 8)
               * args.steps / t_e2e / 1e9,
               "timing": "median of 3 timed passes of the K steps",
               "ms_per_step_passes": [1e3 * x / args.steps for x in passes]}
        del g_h
        return out

    # every rank runs the end-to-end leg (the whole job's rate); the other workloads, linewidths,
    # adjoint and CPU baseline are single-GPU extras, run at N=1 only
    if not args.no_e2e:
        e2e_head = e2e(forms[0], grid=legs[0][1])
        e2e_mixed = e2e("mixed", grid=use_grid) if ("mixed", use_grid) in res and forms[0] == "fp64" else None
        if rank == 0:
            line["e2e"] = e2e_head
            if e2e_mixed is not None:
                line["mixed"]["e2e"] = e2e_mixed
    single = rank == 0 and world == 1
    # oracle k samples (small, large) per workload for the per-configuration CPU baselines
    cpu_k = {"mos2": (1000, 4000), "stanene": (2, 6)} if not args.no_cpu_baseline else {"mos2": None, "stanene": None}
    if single and not args.no_other:
        # the MoS2-shaped (200x200 grid, Nb=11, Nm=9) and stanene-shaped (Nb=120, Nm=180) workloads
        line["other_workloads"] = {
            "mos2": time_workload("mos2", args, dev, [("fp64", True, QB), ("mixed", True, QB), ("mixed", False, QB)], 2, 5,
                                  cpu_k=cpu_k["mos2"]),
            # FP64: one q per call keeps the Re->k GEMM's k tiles whole waves of 152 rows; the mixed
            # form batches 4 q so that their dynamical-matrix eigensolves run side by side
            "stanene": time_workload("stanene", args, dev, [("fp64", False, 1), ("mixed", False, 4)], 2, 3,
                                     cpu_k=cpu_k["stanene"])}
        line["other_workloads"]["batched_graph"] = {
            "what": "one CUDA graph: stanene-shaped (Nb=120, Nm=180, Ne=Np=15, 512 k) + si_tiny-shaped "
                    "(Nb=8, 1024 k) + MoS2-shaped (Nb=11, 48x48 k grid) contexts, uneven q batches "
                    f"{list(synth.STANENE_Q_BATCHES)} (stanene: the first batches, scaled: "
                    f"mixed {GRAPH_STANENE['mixed'][0]}, FP64 {GRAPH_STANENE['fp64'][0]}), eph_autotune's "
                    "(q_batch, k_tile) per context, g through a per-material ring buffer",
            "parity": "sampled (k,q) of every material after a replay vs the oracle "
                      "(tests/test_gpu_config5_graph.py)",
            "mixed": time_batched_graph("mixed", dev), "fp64": time_batched_graph("fp64", dev)}
        line["other_workloads"]["multi_material_persistent"] = time_multi_material(dev)
    if single and not args.no_linewidths:
        line["linewidths"] = time_linewidths(wl, args, q_dev, k_dev, dev, QB, use_grid=legs[0][1])
    if single and not args.no_backward:
        line["backward"] = time_backward(args, cpu=not args.no_cpu_baseline)
    if single:
        line["fp64_peak_probe"] = fp64_peak_probe(dev)
    if single and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample_k)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.capture:
        return run_capture(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.graph_full:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"batched_graph_full": time_batched_graph("mixed", torch.device("cuda", 0),
                                                                   replays=max(1, args.steps), full=True)}))
        return 0
    return run_libeph(args)


if __name__ == "__main__":
    sys.exit(main())
