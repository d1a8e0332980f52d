"""Several materials with uneven q batches in one captured CUDA graph.

Each material is an eph context created with ``async_mode=True``,
``device_ptrs=True`` and the batcher's stream; its q batches are device
tensors.  ``capture()`` reserves every context's workspace (so the captured
calls allocate nothing), runs the sequence once eagerly, then records it into
one CUDA graph; ``replay()`` launches the whole multi-material work list with a
single graph launch.  New inputs are passed by copying into the captured q
buffers.  ``check()`` reads each context's device status (eph_sync).
The kernels are the library's; this module only orders the calls.
"""
from __future__ import annotations

import torch


class GraphBatcher:
    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.stream = torch.cuda.Stream(device=self.device)
        self.items = []      # (ctx, q_dev, eps_kq, omega, g)
        self.graph = None

    def add(self, ctx, q_dev, eps_kq=None, omega=None, g=None):
        if not (ctx.device_ptrs and getattr(ctx, "async_mode", False)):
            raise ValueError("contexts in a graph batch need device_ptrs=True and async_mode=True")
        self.items.append((ctx, q_dev, eps_kq, omega, g))

    def _run_all(self):
        for ctx, q, e, o, g in self.items:
            ctx.eph_interp_q(q.shape[0], q, e, o, g)

    def capture(self):
        for ctx in {id(i[0]): i[0] for i in self.items}.values():
            nq_max = max(q.shape[0] for c, q, *_ in self.items if c is ctx)
            ctx.eph_reserve(nq_max)
        with torch.cuda.stream(self.stream):
            self._run_all()              # eager pass: primes function attributes and tensor maps
        self.stream.synchronize()
        self.check()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
            self._run_all()
        return self

    def replay(self):
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def check(self):
        self.stream.synchronize()
        for ctx in {id(i[0]): i[0] for i in self.items}.values():
            ctx.eph_sync()
