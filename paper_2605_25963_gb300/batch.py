"""Batched runs: many (energy, source, history count) instances in one persistent
launch, captured in a CUDA graph, with an autotuned launch shape.

The device side is the plan of libgadep (``gadep_plan_*``): one work counter over
the flattened history range of all instances feeds every warp, so instances with
uneven history counts share the GPU without per-instance launch tails.  This
module captures the plan's launch (tally clearing + kernel) once and replays it,
and picks block size, histories per warp fetch and blocks per SM by timing
candidates on a scaled-down copy of the batch.
"""
from __future__ import annotations

import itertools
import time

from . import api


class GraphBatch:
    """A plan whose launch is captured in a CUDA graph and replayed."""

    def __init__(self, bvh, mats, items, opts_kw=None, grad=False):
        import torch
        self.torch = torch
        self.items = list(items)
        self.opts = api.make_opts(**(opts_kw or {}))
        self.plan = api.Plan(bvh, mats, api.make_instances(self.items), self.opts, grad=grad)
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.plan.launch(stream=s.cuda_stream)        # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(self.graph):
            self.plan.launch()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()

    def results(self, want_spectra=True):
        self.torch.cuda.synchronize()
        return self.plan.results(want_spectra=want_spectra)


def _scaled(items, total):
    n = sum(it[2] for it in items)
    f = min(1.0, total / max(n, 1))
    return [(E, s, max(1, int(c * f)), i, sc) for E, s, c, i, sc in items]


def autotune(bvh, mats, items, grad=False, sample_histories=4_000_000, candidates=None, repeats=2):
    """Time each launch shape on a scaled copy of the batch; return (best opts, table)."""
    import torch
    cands = candidates or [dict(block=b, chunk=c, blocks_per_sm=0)
                           for b, c in itertools.product((128, 256), (64, 256, 1024))]
    sample = api.make_instances(_scaled(items, sample_histories))
    table = []
    for kw in cands:
        plan = api.Plan(bvh, mats, sample, api.make_opts(**kw), grad=grad)
        plan.launch()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.launch()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        table.append((kw, best))
        del plan
    kw, _ = min(table, key=lambda x: x[1])
    return kw, table


def time_plain(bvh, mats, items, opts_kw=None, grad=False):
    """Per-instance launches (one plan each, created before timing); seconds."""
    import torch
    plans = [api.Plan(bvh, mats, api.make_instances([it]), api.make_opts(**(opts_kw or {})), grad=grad)
             for it in items]
    for p in plans[:2]:
        p.launch()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for p in plans:
        p.launch()
    b.record()
    torch.cuda.synchronize()
    del t0
    return a.elapsed_time(b) / 1e3, plans
