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
        self.multi = []      # (ctxs, [q_dev], [eps_kq], [omega], [g]): one eph_interp_q_multi call each
        self.graph = None

    def add(self, ctx, q_dev, eps_kq=None, omega=None, g=None):
        if not (ctx.device_ptrs and getattr(ctx, "async_mode", False)):
            raise ValueError("contexts in a graph batch need device_ptrs=True and async_mode=True")
        self.items.append((ctx, q_dev, eps_kq, omega, g))

    def add_batch(self, ctx, q_dev, eps_kq, omega, g_ring, chunk):
        """An uneven q batch of any size, as calls of at most `chunk` q points: eps_kq [nq][nk][nb]
        and omega [nq][nm] receive every q point; g goes through `g_ring` [chunk][nk][nm][nb][nb],
        which each call overwrites (a batch's whole g -- 10.6 GB per q at the stanene shapes in
        complex64 -- is consumed tile by tile, never held), so after a replay it holds the g of the
        batch's last call.  Returns the number of calls added."""
        nq = q_dev.shape[0]
        calls = 0
        for a in range(0, nq, chunk):
            b = min(nq, a + chunk)
            self.add(ctx, q_dev[a:b], None if eps_kq is None else eps_kq[a:b], None if omega is None else omega[a:b],
                     None if g_ring is None else g_ring[:b - a])
            calls += 1
        return calls

    def add_multi(self, ctxs, qs, eps_kq=None, omega=None, g=None):
        """One eph_interp_q_multi call over several contexts (FP64 form, nb, nm <= 16): their band
        rotations run as one persistent launch per round over the pairs of every context."""
        for ctx in ctxs:
            if not (ctx.device_ptrs and getattr(ctx, "async_mode", False)):
                raise ValueError("contexts in a graph batch need device_ptrs=True and async_mode=True")
        n = len(ctxs)
        self.multi.append((list(ctxs), list(qs), list(eps_kq or [None] * n), list(omega or [None] * n),
                           list(g or [None] * n)))

    def contexts(self):
        out = {id(i[0]): i[0] for i in self.items}
        for cs, *_ in self.multi:
            out.update({id(c): c for c in cs})
        return list(out.values())

    def _run_all(self):
        from .binding import interp_q_multi
        for ctx, q, e, o, g in self.items:
            ctx.eph_interp_q(q.shape[0], q, e, o, g)
        for cs, qs, es, os_, gs in self.multi:
            interp_q_multi(cs, [q.shape[0] for q in qs], qs, es, os_, gs)

    def capture(self):
        for ctx in self.contexts():
            nq_max = max([q.shape[0] for c, q, *_ in self.items if c is ctx] +
                         [q.shape[0] for cs, qs, *_ in self.multi for c, q in zip(cs, qs) if c is ctx])
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
        for ctx in self.contexts():
            ctx.eph_sync()


class Material:
    """One material of a multi-material graph: its context, q points, outputs and batches."""

    def __init__(self, wl, batches, grid, ctx, q_dev, eps_k, eps_kq, omega, g_ring, chunk, tuned):
        self.wl, self.batches, self.grid, self.ctx = wl, list(batches), grid, ctx
        self.q_dev, self.eps_k, self.eps_kq, self.omega, self.g_ring = q_dev, eps_k, eps_kq, omega, g_ring
        self.chunk, self.tuned = chunk, tuned
        self.calls = 0

    @property
    def nq(self):
        return sum(self.batches)

    @property
    def nk(self):
        return self.eps_k.shape[0]

    def g_elements(self):
        return self.nq * self.nk * self.wl.nm * self.wl.nb * self.wl.nb

    def last_call_q(self):
        """Indices (into this material's q list) of the q points whose g the ring holds."""
        last = self.batches[-1]
        start = self.nq - last + ((last - 1) // self.chunk) * self.chunk
        return list(range(start, self.nq))


def graph_of_materials(specs, form, device, autotune=True):
    """Several materials in one captured CUDA graph (the library's calls, in order).

    specs: [(workload, q batch sizes, chunk, use the uniform k grid)]; each material takes the
    first sum(batches) q points of its workload, and every batch runs as calls of at most `chunk`
    q points whose g goes through one ring buffer per material.  With autotune, eph_autotune picks
    (q_batch, k_tile) and the kernel variants (band_alu, gemm_alu) for a call of `chunk` q points on
    a synchronous context first (the choice is cached per problem shape), and the graph's context
    uses that choice.
    Returns (GraphBatcher, [Material]) with the graph captured."""
    from .binding import Context
    dev = torch.device(device)
    gb = GraphBatcher(dev)
    mats = []
    for wl, batches, chunk, grid in specs:
        nq, nk, nb, nm = sum(batches), len(wl.kpts), wl.nb, wl.nm
        q_dev = torch.from_numpy(wl.qpts[:nq].copy()).to(dev)
        k_dev = torch.from_numpy(wl.kpts).to(dev)
        tuned = (0, 0)
        variants = {}
        if autotune:
            tctx = Context.from_workload(wl, form=form, device_ptrs=True, stream=torch.cuda.current_stream(dev))
            if grid:
                tctx.eph_set_k_grid(*wl.kgrid, None, None)
            else:
                tctx.eph_set_k(nk, k_dev, None)
            tuned = tctx.eph_autotune(min(chunk, nq), q_dev[:min(chunk, nq)])
            t = tctx.tuning()
            variants = {"band_alu": bool(t["band_alu"]), "gemm_alu": bool(t["gemm_alu"])}
            tctx.close()
            torch.cuda.empty_cache()
        ctx = Context.from_workload(wl, form=form, device_ptrs=True, async_mode=True, stream=gb.stream,
                                    q_batch=tuned[0], k_tile=tuned[1], **variants)
        eps_k = torch.empty(nk, nb, dtype=torch.float64, device=dev)
        with torch.cuda.stream(gb.stream):
            if grid:
                ctx.eph_set_k_grid(*wl.kgrid, None, eps_k)
            else:
                ctx.eph_set_k(nk, k_dev, eps_k)
        gb.stream.synchronize()
        ctx.eph_sync()
        gdt = torch.complex128 if form == "fp64" else torch.complex64
        eps_kq = torch.empty(nq, nk, nb, dtype=torch.float64, device=dev)
        omega = torch.empty(nq, nm, dtype=torch.float64, device=dev)
        g_ring = torch.empty(min(chunk, nq), nk, nm, nb, nb, dtype=gdt, device=dev)
        m = Material(wl, batches, grid, ctx, q_dev, eps_k, eps_kq, omega, g_ring, chunk, tuned)
        q0 = 0
        for nqb in batches:
            m.calls += gb.add_batch(ctx, q_dev[q0:q0 + nqb], eps_kq[q0:q0 + nqb], omega[q0:q0 + nqb], g_ring, chunk)
            q0 += nqb
        mats.append(m)
    gb.capture()
    return gb, mats
