"""The benchmark's reference arm (the FP64 oracle on the host cores) against the
output contract: one JSON line from rank 0 with the metric, unit, value, the CPU
baseline it measured and an end-to-end entry; ranks other than 0 print nothing
and exit 0.  Runs on the CPU (bounded oracle sample, about five seconds)."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env):
    env = dict(os.environ, **extra_env)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "bare",
           "--steps", "3", "--warmup", "1"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line(orc):
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "histories/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 1 and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and d["data"] == "synthetic"


def test_reference_arm_other_ranks_do_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_gpu_arm_fails_loudly_without_a_gpu():
    """No CPU fallback: without a CUDA device the benchmark's GPU arm exits
    non-zero and prints no result line, and the API raises."""
    import torch
    if torch.cuda.is_available():
        return
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
    from paper_2605_25963_gb300 import api, capi
    from paper_2605_25963_gb300 import workloads as W
    m = api.detmesh_build(W.BARE_CYLINDER)
    try:
        api.gadep_bvh_build(m, 0)
    except capi.GadepError as e:
        assert "no CUDA device" in str(e)
    else:
        raise AssertionError("gadep_bvh_build on device 0 succeeded without a GPU")


def test_traffic_record_matches_the_kernels():
    """The DRAM-per-query record in profiles/traffic.json was taken on the transport
    kernels as they stand: its hash is the hash of their sources (the benchmark
    reports no traffic otherwise), and the benchmark scales each per-query figure
    by the queries of a launch."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = [argv[0]]
        spec.loader.exec_module(bench)
    finally:
        sys.argv = argv
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    h = bench.kernel_hash()
    for workload, kinds in (("coax", ("trace", "physics", "sort")), ("stress", ("trace",))):
        assert rec[workload]["kernel_hash"] == h, workload
        for kind in kinds:
            per_query = rec[workload]["dram_bytes_per_query"][kind]
            assert per_query > 0
            assert bench.recorded_traffic(workload, kind, 1000) == per_query * 1000
