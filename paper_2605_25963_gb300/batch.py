"""Batched runs: many (energy, source, history count) instances in one launch.

The device side is a libgadep plan (``gadep_plan_*``): one work counter over the
flattened history range of all instances feeds every warp, so instances with
uneven history counts share the GPU without per-instance launch tails.  Two
forms exist: the persistent megakernel (one kernel launch) and the wavefront
kernels (photon slots in device memory, iterations of spawn / sort / trace /
physics / gen / ctrl repeated by a device-side WHILE node of a CUDA graph).
Both launch without host synchronisation, so ``GraphBatch`` captures either in
a CUDA graph and replays it.  ``autotune`` times both forms and the
megakernel's launch shapes on a scaled-down copy of the batch and keeps the
fastest.
"""
from __future__ import annotations

import itertools

from . import api

MEGA, WAVEFRONT = 1, 2


class GraphBatch:
    """A plan (either form) whose launch is captured in a CUDA graph and replayed."""

    def __init__(self, bvh, mats, items, opts_kw=None, grad=False):
        import torch
        self.torch = torch
        kw = dict(opts_kw or {})
        self.items = list(items)
        self.opts = api.make_opts(**kw)
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


def default_candidates():
    """Megakernel launch shapes, and the wavefront form with the slot count sized
    from the run (0) or fixed.  The slot count trades the trace kernel, which
    prefers every photon in flight at once (fuller, better sorted queues), against
    the physics kernel, whose random 64-byte slot records stay in L2 when there
    are fewer of them (batched workload: physics 299 ms at 2^25 slots, 204 ms at
    2^22; the whole plan fastest at 2^22)."""
    cands = [dict(variant=MEGA, block=b, chunk=c, blocks_per_sm=0)
             for b, c in itertools.product((128, 256), (64, 256, 1024))]
    cands += [dict(variant=WAVEFRONT, wf_slots=s) for s in (0, 1 << 21, 1 << 22, 1 << 23)]
    return cands


def _time_plan(plan, repeats):
    import torch
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
    return best


def autotune(bvh, mats, items, grad=False, sample_histories=100_000_000, candidates=None, repeats=2,
             opts_kw=None):
    """Time each launch form / shape on a scaled copy of the batch; return (best opts, table).

    opts_kw: the caller's own options (e_model, e_cut_keV, seed, ...), kept in every
    candidate; the returned options include them."""
    base = dict(opts_kw or {})
    cands = [dict(base, **kw) for kw in (candidates or default_candidates())]
    sample = api.make_instances(_scaled(items, sample_histories))
    table = []
    for kw in cands:
        plan = api.Plan(bvh, mats, sample, api.make_opts(**kw), grad=grad)
        table.append((kw, _time_plan(plan, repeats)))
        del plan
    kw, _ = min(table, key=lambda x: x[1])
    return kw, table


def time_plain(bvh, mats, items, opts_kw=None, grad=False, keep_results=False):
    """Per-instance runs, one plan each, in turn; seconds of device time summed over
    the launches (plan creation is outside the timed spans).  Returns (seconds,
    [results per instance] if keep_results)."""
    import torch
    total = 0.0
    out = []
    warm = api.Plan(bvh, mats, api.make_instances([items[0]]), api.make_opts(**(opts_kw or {})), grad=grad)
    warm.launch()
    torch.cuda.synchronize()
    del warm
    for it in items:
        p = api.Plan(bvh, mats, api.make_instances([it]), api.make_opts(**(opts_kw or {})), grad=grad)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        p.launch()
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b) / 1e3
        if keep_results:
            out.append(p.results(want_spectra=False))
        del p
    return total, out
