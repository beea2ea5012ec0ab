"""Benchmark: photon histories/s on one GB300 (and N GPUs, one process each).

Workload (default "coax"): p-type coaxial HPGe in an Al endcap with a Cu holder,
128 segments per circle (~1.4e4 triangles), isotropic point source 25 mm above
the endcap, energies 59.5 / 122 / 662 / 1332 keV, 1e8 histories each, pair
production on, closed-form synthetic cross sections, Philox seed 1.  One step =
the four transport launches (one per energy) with the tally reduction; the mesh,
BVH and plans are built once before timing (like model weights).  Between timed
steps a 512 MB buffer is written to flush L2.  The K timed steps run as the API
runs them (each plan launch one CUDA graph, the wavefront iterations driven by its
device-side WHILE node); a second pass over the same K steps, with the iterations
issued by the host and a CUDA event pair around every kernel, gives the per-kernel
times, the roofline of the dominant kernel and the launch count.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gadep|reference]

With N > 1 (torchrun), every rank transports its own history-id range (weak
scaling); the time is the max over ranks.  --impl reference times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2605_25963_gb300 import workloads as W  # noqa: E402

METRIC = "photon histories/s on 1 GB300, FEPE within 3σ of oracle; batched/grad vs plain"
UNIT = "histories/s"
# FP32 operations per traversal unit (counted from the kernel's arithmetic):
# child box test = 6 slab FMAs (2 FLOP) + 6 min/max -> 18 (a 4-wide node visit
# tests its 2..4 children); triangle test = 9 vertex translations + 6 shear FMAs
# (12) + 6 mul + 3 sub (edge functions) + 2 add (det) + 3 mul + 2 FMA (T, 5) + 1 div
# + 2 compares -> ~45.
FLOP_PER_BOX = 18.0
FLOP_PER_TRI = 45.0
SM_COUNT = 152
FP32_LANES_PER_SM = 128
NODE_BYTES, TRI_BYTES = 64, 48        # 4-wide BVH node (quantised child boxes); three float4 vertices
L2_FLUSH_BYTES = 512 << 20


def workload_config(name, n_hist):
    if name == "coax":
        return dict(det=W.COAX_P, src=W.COAX_POINT_25, energies=W.COAX_ENERGIES, n_hist=n_hist or W.COAX_HISTORIES,
                    desc="coax_p: p-type coaxial HPGe (R 30.5 L 62, bore 5x48, 0.7 mm dead layer, 0.3 um contact, "
                         "Al endcap, Cu holder), 128 segments (13824 triangles), point source 25 mm, "
                         "59.5/122/662/1332 keV")
    if name == "table4":
        return dict(det=W.DET2, src=W.TABLE4_SOURCE, energies=W.TABLE4_ENERGIES, n_hist=n_hist or 100_000_000,
                    desc="table4: detector #2 of Table 1 (crystal 68.1 x 63.3, hole 10.1 x 50.2, 0.7 mm / 0.3 um "
                         "dead layers) in the coax housing, N_theta 32, N_phi 10, point source 250 mm above "
                         "the window, the 13 Table 3 energies 59.54-1408.02 keV",
                    paper_s={"1e7": 11.96, "1e8": 66.08})
    if name == "stress":
        return dict(det=W.STRESS_DET, src=W.STRESS_SOURCE, energies=W.STRESS_ENERGIES,
                    n_hist=n_hist or W.STRESS_HISTORIES,
                    desc="stress: coax at 1024 segments with a 2 x 1 mm contact groove and a Cu flange with 16 "
                         "bolt holes (1,501,300 triangles), water-prism volume source, 8 energies 59.5-1836 keV")
    if name == "bare":
        return dict(det=W.BARE_CYLINDER, src=W.BARE_POINT_100, energies=(662.0,), n_hist=n_hist or 1_000_000,
                    desc="bare Ge cylinder R 30 L 60, 48 segments (192 triangles), point source 100 mm, 662 keV")
    raise SystemExit("unknown workload %r" % name)


def kernel_hash():
    h = hashlib.sha256()
    for f in ("transport.cu", "wavefront.cu", "transport_common.cuh", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_2605_25963_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, kind, queries_per_launch):
    """DRAM bytes per launch of kernel `kind`: the committed per-query figure
    (ncu on a small case of the workload, a few launches of that kernel alone,
    divided by the queries those launches served) times the queries of an average
    launch here; None when the kernels changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    per_query = e.get("dram_bytes_per_query", {}).get(kind)
    return None if per_query is None else per_query * queries_per_launch


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        loaded = [s for s, _, _ in rows if s > 0.5 * rows[0][1]] or [s for s, _, _ in rows]
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": max(m for _, m, _ in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(cfg, budget_s=15.0, threads=None):
    """The FP64 oracle as it stands on the host cores, on a bounded sample."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    om = O.Mesh.build(O.Det(**cfg["det"].as_dict()))
    ot = O.Tables.build(W.MATERIAL_CODES)
    s = cfg["src"]
    osrc = O.Source(kind=s.kind, pos=s.pos, dir=s.dir, radius=s.radius, height=s.height, n_sides=s.n_sides)
    probe = 20_000
    t0 = time.perf_counter()
    for E in cfg["energies"]:
        O.transport(om, ot, osrc, E, probe, n_threads=threads)
    rate = probe * len(cfg["energies"]) / (time.perf_counter() - t0)
    n = int(max(probe, min(cfg["n_hist"], rate * budget_s / len(cfg["energies"]))))
    t0 = time.perf_counter()
    for E in cfg["energies"]:
        O.transport(om, ot, osrc, E, n, n_threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n * len(cfg["energies"]) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d histories per energy x %d energies of the same workload (history ids 0..%d), "
                      "%.1f s" % (n, len(cfg["energies"]), n - 1, dt)}


def measure_forms(dev, scale=1.0):
    """Batched and gradient forms against the plain per-instance kernel, same
    histories (hence the same FEPE sigma) on the same GPU.

    batched: bare-cylinder detector with a water prism, 40 energies x 3 sources,
    log-uniform 1e6-5e7 histories per instance (1.5e9 in all): 120 per-instance
    runs (each in the form AUTO picks) vs one batched run in the autotuned form
    (the megakernel replayed from a CUDA graph, or the wavefront kernels).
    gradient: coax detector + water prism volume source, 4 energies x 5e7
    histories: plain runs vs the score-accumulating kernels (dFEPE/ds for 4
    density groups); also against central finite differences (1 + 2 x 4 runs).
    stress: the gradient geometry at 1024 segments with a contact groove and a
    bolted flange (~1e6 triangles), 8 energies x 1.25e8 histories: per-instance
    runs vs one batched plan, plain and with gradients.
    electrons: the coax workload's 4 energies x 2.5e7 histories with charged
    particles tracked in the continuous-slowing-down approximation (e_model 1)
    vs deposited at the interaction point; the FEPE of both.
    """
    import torch
    from paper_2605_25963_gb300 import api, batch
    out = {}
    mats = api.Materials.default()
    # ---- batched ----
    m3 = api.detmesh_build(W.BATCH_DET)
    b3 = api.gadep_bvh_build(m3, dev)
    items = [(E, W.BATCH_SOURCES[s], max(1, int(n * scale)), i, [1, 1, 1, sm])
             for i, (E, s, n, sm) in enumerate(W.batch_instances())]
    total = sum(it[2] for it in items)
    t_plain, _ = batch.time_plain(b3, mats, items)
    kw, table = batch.autotune(b3, mats, items)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g = batch.GraphBatch(b3, mats, items, kw)
    g.replay()
    torch.cuda.synchronize()
    a.record()
    g.replay()
    e.record()
    torch.cuda.synchronize()
    res, _, _, _ = g.results(want_spectra=False)
    how = ("wavefront" if kw.get("variant") == batch.WAVEFRONT else "megakernel") + " plan replayed from a CUDA graph"
    t_batch = a.elapsed_time(e) / 1e3
    out["batched"] = {"instances": len(items), "histories": total, "plain_s": t_plain, "batched_s": t_batch,
                      "plain_hist_per_s": total / t_plain, "batched_hist_per_s": total / t_batch,
                      "batched_vs_plain": t_plain / t_batch, "autotuned": kw, "batched_form": how,
                      "autotune_ms": [[k, round(v, 3)] for k, v in table],
                      "fepe_first": res[0]["fepe"], "n_err": sum(r["n_err"] for r in res)}
    del g
    # the same comparison end to end through the public calls a user makes, host
    # buffers: 120 gadep_run calls (each stages its tables and instance, runs and
    # reads its spectrum back) against one gadep_run_batch call with the autotuned
    # options; wall-clock seconds after one warm-up call of each
    ob = api.make_opts(**kw)
    api.gadep_run(b3, mats, items[0][1], items[0][0], items[0][2], instance=items[0][3],
                  opts=api.make_opts(group_scale=items[0][4]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for E, src, n, iid, sc in items:
        api.gadep_run(b3, mats, src, E, n, instance=iid, opts=api.make_opts(group_scale=sc))
    torch.cuda.synchronize()
    e2e_plain = time.perf_counter() - t0
    inst3 = api.make_instances(items)
    api.gadep_run_batch(b3, mats, inst3, ob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.gadep_run_batch(b3, mats, inst3, ob)
    torch.cuda.synchronize()
    e2e_batch = time.perf_counter() - t0
    out["batched"]["e2e"] = {"plain_s": e2e_plain, "batched_s": e2e_batch, "batched_vs_plain": e2e_plain / e2e_batch,
                             "note": "wall clock: 120 gadep_run calls vs one gadep_run_batch call, host buffers"}
    # ---- gradient ----
    m4 = api.detmesh_build(W.GRAD_DET)
    b4 = api.gadep_bvh_build(m4, dev)
    n4 = max(1, int(W.GRAD_HISTORIES * scale))
    items4 = [(E, W.GRAD_SOURCE, n4, i, [1, 1, 1, 1]) for i, E in enumerate(W.GRAD_ENERGIES)]
    t_p, _ = batch.time_plain(b4, mats, items4)
    t_g, gres = batch.time_plain(b4, mats, items4, opts_kw=dict(n_group=4), grad=True, keep_results=True)
    grads = []
    for res, _, d, ds in gres:
        grads.append({"fepe": res[0]["fepe"], "dfepe": [float(x) for x in d[0]],
                      "dsigma": [float(x) for x in ds[0]]})
    out["gradient"] = {"histories": n4 * len(items4), "plain_s": t_p, "grad_s": t_g,
                       "grad_vs_plain": t_p / t_g, "grad_vs_central_fd": (1 + 2 * 4) * t_p / t_g,
                       "per_energy": dict(zip([str(E) for E in W.GRAD_ENERGIES], grads))}
    # ---- electrons: CSDA tracks vs local deposition, same histories ----
    m6 = api.detmesh_build(W.COAX_P)
    b6 = api.gadep_bvh_build(m6, dev)
    n6 = max(1, int(25_000_000 * scale))
    times6, fepe6 = {}, {}
    for em in (0, 1):
        o6 = api.make_opts(e_model=em)
        api.gadep_run(b6, mats, W.COAX_POINT_25, W.COAX_ENERGIES[0], n6, opts=o6)      # warm-up
        plans = [api.Plan(b6, mats, api.make_instances([(E, W.COAX_POINT_25, n6, i, [])]), o6)
                 for i, E in enumerate(W.COAX_ENERGIES)]
        torch.cuda.synchronize()
        a6, e6 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a6.record()
        for p6 in plans:
            p6.launch()
        e6.record()
        torch.cuda.synchronize()
        times6[em] = a6.elapsed_time(e6) / 1e3
        fepe6[em] = [p6.results(want_spectra=False)[0][0]["fepe"] for p6 in plans]
        del plans
    h6 = n6 * len(W.COAX_ENERGIES)
    out["electrons"] = {"histories": h6, "local_hist_per_s": h6 / times6[0], "csda_hist_per_s": h6 / times6[1],
                        "csda_vs_local": times6[0] / times6[1],
                        "fepe_local": fepe6[0], "fepe_csda": fepe6[1]}
    # ---- stress: ~1e6-triangle mesh, 8 energies, batched and with gradients ----
    t0 = time.perf_counter()
    m5 = api.detmesh_build(W.STRESS_DET)
    t_mesh5 = time.perf_counter() - t0
    t0 = time.perf_counter()
    b5 = api.gadep_bvh_build(m5, dev)
    t_bvh5 = time.perf_counter() - t0
    n5 = max(1, int(W.STRESS_HISTORIES * scale))
    items5 = [(E, W.STRESS_SOURCE, n5, i, [1, 1, 1, 1]) for i, E in enumerate(W.STRESS_ENERGIES)]
    total5 = n5 * len(items5)
    t_p5, _ = batch.time_plain(b5, mats, items5)

    def one_plan(grad):
        p = api.Plan(b5, mats, api.make_instances(items5), api.make_opts(n_group=4 if grad else 0), grad=grad)
        p.launch()                                   # warm-up (slot buffers, caches)
        torch.cuda.synchronize()
        a5, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a5.record()
        p.launch()
        e5.record()
        torch.cuda.synchronize()
        return a5.elapsed_time(e5) / 1e3, p.results(want_spectra=False)

    t_b5, (rb5, _, _, _) = one_plan(False)
    t_g5, (rg5, _, dg5, _) = one_plan(True)
    roof5 = stress_roofline(b5, mats, items5, dev)
    out["stress"] = {"triangles": int(b5.stats()["n_tri"]), "mesh_build_s": round(t_mesh5, 3),
                     "bvh_build_s": round(t_bvh5, 3), "instances": len(items5), "histories": total5,
                     "plain_hist_per_s": total5 / t_p5, "batched_hist_per_s": total5 / t_b5,
                     "batched_grad_hist_per_s": total5 / t_g5, "batched_vs_plain": t_p5 / t_b5,
                     "batched_grad_vs_plain": t_p5 / t_g5,
                     "fepe": [r["fepe"] for r in rg5], "dfepe_first": [float(x) for x in dg5[0]],
                     "n_err": sum(r["n_err"] for r in rb5) + sum(r["n_err"] for r in rg5),
                     "bvh": b5.stats()["opts"], "bvh_mb": round((b5.stats()["node_bytes"] + b5.stats()["tri_bytes"]) / 1e6, 1),
                     "roofline": roof5}
    del b5, m5
    # ---- Table 4 shape (detector #2, 13 energies, source 250 mm) and the mesh-density sweep ----
    out["table4"] = table4_form(dev, scale)
    cfg_c = workload_config("coax", 0)
    out["mesh_sweep"] = {"coax": mesh_sweep(cfg_c, dev, max(1, int(10_000_000 * scale)), api.make_opts()),
                         "table4": mesh_sweep(workload_config("table4", 0), dev, max(1, int(10_000_000 * scale)),
                                              api.make_opts()),
                         "histories_per_energy": max(1, int(10_000_000 * scale))}
    return out


def stress_roofline(bvh, mats, items, dev):
    """Roofline of the trace kernel on the stress workload: the one batched plan
    timed again with a CUDA event pair around every kernel (host-issued
    iterations), the traversal work counted by the instrumented kernels on the
    same histories, and the algorithmic FLOPs and node/triangle bytes per second
    against the derived FP32 peak and the measured L2 and HBM peaks."""
    from paper_2605_25963_gb300 import api
    p = api.Plan(bvh, mats, api.make_instances(items), api.make_opts())
    p.launch()
    p.set_timing(True)
    p.kernel_stats(reset=True)
    p.launch()
    st = p.kernel_stats(reset=True)
    res, _, _, _ = p.results(want_spectra=False)
    del p
    _, nodes, tris, _, boxes = api.gadep_count_work(bvh, mats, api.make_instances(items), api.make_opts())
    segs = sum(r["n_segments"] for r in res)
    queries = segs - sum(r["n_culled"] for r in res)
    nl, ms = st.get("trace", (0, 0.0))
    if not nl:
        return None
    flops = FLOP_PER_BOX * boxes + FLOP_PER_TRI * tris
    bytes_ = NODE_BYTES * nodes + TRI_BYTES * tris
    sm_max = measured_peaks().get("sm_max_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (ms / 1e3) / 1e12
    hbm = measured_peaks().get("hbm_gbs")
    return {"bound": "alu", "kernel": "trace", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": recorded_traffic("stress", "trace", queries / nl),
            "launches": nl, "avg_launch_ms": ms / nl, "flop_per_launch": flops / nl,
            "node_tri_bytes_gbs": bytes_ / (ms / 1e3) / 1e9, "hbm_peak_gbs": hbm,
            "per_query": {"nodes": nodes / max(queries, 1), "boxes": boxes / max(queries, 1),
                          "tris": tris / max(queries, 1)},
            "kernels_ms": {k: round(v, 2) for k, (n, v) in st.items() if n},
            "queries": queries,
            "note": "stress BVH (clipped references) exceeds L2: node and triangle bytes per second of the trace "
                    "kernel are served partly from HBM"}


def table4_form(dev, scale=1.0):
    """The Table 4 shape workload: detector #2 of Table 1, point source 250 mm on
    the axis, the 13 Table 3 energies, at 1e7 and 1e8 histories per energy (one
    step each, device time after a warm-up step), beside the paper's RTX 4090
    times for coupled photon-electron transport (context only)."""
    import torch
    from paper_2605_25963_gb300 import api
    cfg = workload_config("table4", 0)
    mats = api.Materials.default()
    m = api.detmesh_build(cfg["det"])
    b = api.gadep_bvh_build(m, dev)
    out = {"triangles": int(b.stats()["n_tri"]), "energies": len(cfg["energies"])}
    for n in (10_000_000, 100_000_000):
        nn = max(1, int(n * scale))
        plans = [api.Plan(b, mats, api.make_instances([(E, cfg["src"], nn, i, [])]), api.make_opts())
                 for i, E in enumerate(cfg["energies"])]
        for p in plans:
            p.launch()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for p in plans:
            p.launch()
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        fe = [p.results(want_spectra=False)[0][0]["fepe"] for p in plans]
        out["%.0e" % n] = {"histories_per_energy": nn, "ms_all_energies": round(ms, 2),
                           "hist_per_s": nn * len(plans) / (ms / 1e3),
                           "paper_rtx4090_s": cfg["paper_s"]["1e7" if n == 10_000_000 else "1e8"],
                           "fepe": fe, "form": "AUTO (per energy)"}
        del plans
    return out


def mesh_sweep(cfg, dev, n, opts):
    """Mesh-density sensitivity (Sec. 3.3): the workload's detector discretised at
    N_theta x N_phi from 32 x 10 to 1024 x 40, same histories; device time of one
    step per mesh after one warm-up step."""
    import dataclasses
    import torch
    from paper_2605_25963_gb300 import api
    mats = api.Materials.default()
    out = []
    for nt, nph in ((32, 10), (64, 20), (128, 10), (256, 20), (512, 20), (1024, 40)):
        det = dataclasses.replace(cfg["det"], n_theta=nt, n_phi=nph)
        m = api.detmesh_build(det)
        b = api.gadep_bvh_build(m, dev)
        plans = [api.Plan(b, mats, api.make_instances([(E, cfg["src"], n, i, [])]), opts)
                 for i, E in enumerate(cfg["energies"])]
        for p in plans:
            p.launch()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for p in plans:
            p.launch()
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        st = b.stats()
        out.append({"n_theta": nt, "n_phi": nph, "triangles": int(st["n_tri"]),
                    "bvh_mb": round((st["node_bytes"] + st["tri_bytes"]) / 1e6, 2), "ms_per_step": round(ms, 2),
                    "hist_per_s": n * len(plans) / (ms / 1e3)})
        del plans, b, m
    return out


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(cfg, budget_s=max(5.0, 20.0 / max(1, args.steps + args.warmup)))
    per_step = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": per_step, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "n_hist_per_energy": cfg["n_hist"], "seed": 1,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": cb, "e2e": {"value": per_step, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1, help="GPUs, one process each (launch with torchrun when > 1)")
    ap.add_argument("--steps", type=int, default=5, help="timed steps")
    ap.add_argument("--warmup", type=int, default=3, help="untimed warm-up steps")
    ap.add_argument("--impl", default="gadep", choices=["gadep", "reference"],
                    help="gadep: the CUDA path; reference: the FP64 CPU oracle on a bounded sample")
    ap.add_argument("--workload", default="coax", choices=["coax", "bare", "table4", "stress"],
                    help="coax: the headline (4 energies x 1e8); bare: Ge cylinder; table4: detector #2, "
                         "13 energies at 250 mm; stress: ~1e6-triangle mesh with a volume source")
    ap.add_argument("--hist", type=int, default=0, help="histories per energy (default: the workload's)")
    ap.add_argument("--block", type=int, default=0, help="threads per block (0: the library default)")
    ap.add_argument("--chunk", type=int, default=0, help="histories a warp takes from the work counter at once (0: the library default)")
    ap.add_argument("--variant", default="auto", choices=["auto", "mega", "wavefront"],
                    help="transport form (auto: by the histories expected to reach the scene)")
    ap.add_argument("--e-model", type=int, default=0, choices=[0, 1],
                    help="charged particles: 0 deposit at the interaction point, 1 CSDA tracks")
    ap.add_argument("--bvh", default="", help="BVH build options, e.g. split_alpha=0,max_leaf=3 "
                                             "(max_leaf, c_trav, c_tri, split_alpha, max_dup, clip_ratio, clip_pieces)")
    ap.add_argument("--wf-slots", type=int, default=0, help="wavefront photon slots (0: sized from the run)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip timing the oracle on the host cores")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run through gadep_run with host buffers")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / gradient comparison")
    ap.add_argument("--forms-scale", type=float, default=1.0, help="history-count scale of the form runs")
    ap.add_argument("--queue-log", action="store_true",
                    help="add the trace queue size of every wavefront iteration of the instrumented pass "
                         "(per plan) to the line, to turn ncu counters of single launches into per-query figures")
    ap.add_argument("--mesh-sweep", action="store_true",
                    help="also time the workload's detector at N_theta x N_phi from 32 x 10 to 1024 x 40")
    args = ap.parse_args()
    cfg = workload_config(args.workload, args.hist)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return

    import torch
    from paper_2605_25963_gb300 import api
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    dev = torch.cuda.current_device()

    bvh_kw = {}
    for item in filter(None, args.bvh.split(",")):
        k, v = item.split("=")
        bvh_kw[k.strip()] = int(v) if k.strip() in ("max_leaf", "clip_pieces") else float(v)
    t0 = time.perf_counter()
    mesh = api.detmesh_build(cfg["det"])
    t_mesh = time.perf_counter() - t0
    t0 = time.perf_counter()
    bvh = api.gadep_bvh_build(mesh, dev, **bvh_kw)
    t_bvh = time.perf_counter() - t0
    mats = api.Materials.default()
    n = cfg["n_hist"]
    from paper_2605_25963_gb300 import dist as shard
    offset = shard.history_offset(rank, n)   # disjoint history ids per rank
    opts = api.make_opts(history_offset=offset, block=args.block, chunk=args.chunk,
                         variant={"auto": 0, "mega": 1, "wavefront": 2}[args.variant], wf_slots=args.wf_slots,
                         e_model=args.e_model)
    plans = [api.Plan(bvh, mats, api.make_instances([(E, cfg["src"], n, i, [])]), opts)
             for i, E in enumerate(cfg["energies"])]
    stream = torch.cuda.current_stream()
    spectra = [torch.zeros(opts.n_bins, dtype=torch.int32, device="cuda") for _ in plans]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(events=None):
        for i, (p, s) in enumerate(zip(plans, spectra)):
            if events is not None:
                events[i][0].record(stream)
            p.launch(spectra=s)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()

    def timed_steps():
        """K steps, one CUDA event pair per plan launch on the launching stream (the
        L2 flush before each step outside them); total device ms."""
        ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plans]
            step(ev)
            torch.cuda.synchronize()
            ms.append(ev[0][0].elapsed_time(ev[-1][1]))
        return float(sum(ms))

    sampler = ClockSampler(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    # (A) the timed steps as a caller runs them: each plan launch is one CUDA graph
    # whose WHILE node drives the wavefront iterations on the device
    total_ms = timed_steps()
    # (B) the same steps again, instrumented: iterations issued by the host with a
    # CUDA event pair around every kernel, for the per-kernel times and launch counts
    for p in plans:
        p.set_timing(True)
        p.kernel_stats(reset=True)
    torch.cuda.synchronize()
    instrumented_ms = timed_steps()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    hist_per_step = n * len(plans) * world
    value = hist_per_step * args.steps / (total_ms / 1e3)

    # results of the last step (FEPE per energy); with several ranks the tallies and
    # spectra of every rank's history range are summed (after the timed region)
    fepe = []
    for p in plans:
        res, spec, _, _ = p.results(want_spectra=dist is not None, raise_device_errors=False)
        f = {"E_keV": None, "fepe": res[0]["fepe"], "sigma": res[0]["sigma"], "n_err": res[0]["n_err"],
             "dev_err": res[0]["dev_err"], "segments": res[0]["n_segments"], "culled": res[0]["n_culled"]}
        if dist is not None:
            tot, _, f_all, s_all = shard.reduce_tallies(res[0], spec[0])
            f["all_ranks"] = {"n_hist": tot["n_hist"], "n_fep": tot["n_fep"], "fepe": f_all, "sigma": s_all}
        fepe.append(f)
    for f, E in zip(fepe, cfg["energies"]):
        f["E_keV"] = E

    qlog = [p.queue_sizes() for p in plans] if args.queue_log else None
    # algorithmic work of one step (instrumented copy of the kernel, untimed)
    nodes = tris = relocated = boxes = 0
    for i, E in enumerate(cfg["energies"]):
        _, nv, nt, nr, nb = api.gadep_count_work(bvh, mats, api.make_instances([(E, cfg["src"], n, i, [])]), opts)
        nodes += nv
        tris += nt
        relocated += nr
        boxes += nb
    flops_per_step = FLOP_PER_BOX * boxes + FLOP_PER_TRI * tris
    # launches and device time per kernel kind over the timed steps
    kstats = {}
    for p in plans:
        for k, (nl, ms) in p.kernel_stats(reset=True).items():
            a = kstats.setdefault(k, [0, 0.0])
            a[0] += nl
            a[1] += ms
        p.set_timing(False)
    ktot = sum(ms for _, ms in kstats.values()) or 1.0
    kernels = {k: {"launches": nl, "ms_per_step": ms / args.steps, "share": ms / ktot}
               for k, (nl, ms) in kstats.items() if nl}
    # the traversal (all node and triangle work) runs in the megakernel or in the trace kernel
    dom = "trace" if kstats.get("trace", (0, 0.0))[0] else "mega"
    dom_launches, dom_ms = kstats[dom]
    achieved_tflops = flops_per_step * args.steps / (dom_ms / 1e3) / 1e12
    sm_max = (clocks or {}).get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    # the library's own microbenchmarks (after the timed region): FP32 FMA and L2 read peaks
    fp32_meas, l2_meas = api.measure_peaks(dev)
    peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    segs = sum(f["segments"] for f in fepe)
    # nearest-hit queries: every segment but the one of a history that ends at birth
    # (born in the world aimed away from the scene box), which is counted without a query
    queries = segs - sum(f["culled"] for f in fepe)
    # algorithmic node and triangle bytes of the traversal (64 B per node visit, 48 B per
    # triangle test), served by L1 and L2, per second of the dominant kernel
    l1l2_gbs = (NODE_BYTES * nodes + TRI_BYTES * tris) * args.steps / (dom_ms / 1e3) / 1e9
    # the timed plans hold the mesh's cached wavefront buffers; release them so the
    # public-API calls below find the cache free, as a caller's successive runs do
    n_plans, shape = len(plans), plans[0].shape()
    del plans
    torch.cuda.synchronize()

    # end to end through the public API with host buffers (tables and instance
    # uploaded, spectrum and tallies read back, every call)
    e2e = None
    if not args.no_e2e:
        xs_bytes = 3 * 1000 * 16            # staged tables of Ge, Al, Cu
        n_region = len(mesh.arrays()[3]) + 1
        h2d = n_plans * (xs_bytes + 16 * n_region + 96 + 8)   # tables, regions, instance, prefix
        # spectrum, the tally copies (256 stripes of 224 bytes for one instance), work counters
        d2h = n_plans * (opts.n_bins * 4 + 256 * 224 + 32)
        api.gadep_run(bvh, mats, cfg["src"], cfg["energies"][0], n, instance=0, opts=opts)   # warm-up
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            for i, E in enumerate(cfg["energies"]):
                api.gadep_run(bvh, mats, cfg["src"], E, n, instance=i, opts=opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": hist_per_step * max(1, args.steps) / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    forms = None
    if not args.no_forms and world == 1:
        forms = measure_forms(dev, args.forms_scale)
    sweep = mesh_sweep(cfg, dev, n, opts) if args.mesh_sweep and world == 1 else None

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(cfg)

    if rank == 0:
        g, blk, smem = shape
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["desc"], "n_hist_per_energy": n, "energies_keV": list(cfg["energies"]),
                       "seed": 1, "triangles": bvh.stats()["n_tri"], "grid": g, "block": blk,
                       "smem_bytes": smem, "l2": "flushed between steps (512 MB write)",
                       "timing": "device time of the K steps as the API runs them (one CUDA graph per plan "
                                 "launch, iterations driven by its WHILE node); kernels, roofline and "
                                 "gpu_launches from a second, instrumented pass over the same K steps "
                                 "(host-issued iterations, CUDA events around every kernel)",
                       "instrumented_ms_per_step": instrumented_ms / args.steps,
                       "e_model": args.e_model,
                       "paper_rtx4090_s_all_energies": cfg.get("paper_s"),
                       "mesh_build_s": round(t_mesh, 4), "bvh_build_s": round(t_bvh, 4),
                       "bvh": bvh.stats()["opts"]},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved_tflops, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved_tflops / peak_tflops,
                         "traffic": recorded_traffic(args.workload, dom,
                                                     queries * args.steps / max(dom_launches, 1)),
                         "launches": dom_launches, "avg_launch_ms": dom_ms / max(dom_launches, 1),
                         "flop_per_launch": flops_per_step * args.steps / max(dom_launches, 1),
                         "peak_note": "FP32 non-tensor: %d SMs x %d lanes x 2 x %.0f MHz (derived)" % (
                             SM_COUNT, FP32_LANES_PER_SM, sm_max),
                         "microbenchmarks": {"fp32_tflops": fp32_meas, "l2_read_gbs": l2_meas,
                                             "frac_of_measured_fp32": achieved_tflops / fp32_meas,
                                             "l1l2_bytes_gbs": l1l2_gbs,
                                             "frac_of_measured_l2": l1l2_gbs / l2_meas if l2_meas else None,
                                             "note": "library microbenchmarks: independent FMA chains on every "
                                                     "SM; 64 MB re-read from L2"},
                         "per_query": {"nodes": nodes / max(queries, 1), "boxes": boxes / max(queries, 1),
                                       "tris": tris / max(queries, 1),
                                       "relocated": relocated / max(queries, 1)},
                         "queries_per_step": queries, "segments_per_step": segs},
            "cpu_baseline": cb,
            "e2e": e2e,
            "gpu_launches": sum(nl for nl, _ in kstats.values()),
            "kernels": kernels,
            "clocks": clocks,
            "hits_only": {"value": sum(n - f["culled"] for f in fepe) * world * args.steps / (total_ms / 1e3),
                          "unit": UNIT, "note": "histories whose first ray reaches the scene box"},
            "fepe": fepe,
            "forms": forms,
        }
        if sweep is not None:
            line["mesh_sweep"] = sweep
        if qlog is not None:
            line["queue_sizes"] = qlog
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
