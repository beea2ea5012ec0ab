"""Wavefront form of the transport: same histories, same tallies as the
persistent megakernel (the region update is idempotent at exact ties, so the two
agree history by history), and parity with the oracle through the traced
deposits."""
import numpy as np
import pytest

from paper_2605_25963_gb300 import api
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

WAVEFRONT = 2


@pytest.mark.parametrize("E", [59.5, 662.0, 1332.0])
def test_wavefront_equals_megakernel(orc, E):
    m = api.detmesh_build(W.COAX_P)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    n = 300_001
    tr_m = torch.empty(n, dtype=torch.float32, device="cuda")
    tr_w = torch.empty(n, dtype=torch.float32, device="cuda")
    rm, sm = api.gadep_run(b, mats, W.COAX_POINT_25, E, n, edep_trace=tr_m)
    rw, sw = api.gadep_run(b, mats, W.COAX_POINT_25, E, n, edep_trace=tr_w,
                           opts=api.make_opts(variant=WAVEFRONT, wf_slots=32768))
    assert rw["n_hist"] == n and rw["n_err"] == 0
    same = np.mean(tr_m.cpu().numpy() == tr_w.cpu().numpy())
    assert same >= 0.9999, same
    for k in ("n_fep", "n_zero", "n_over"):
        assert abs(rm[k] - rw[k]) <= 2, (k, rm[k], rw[k])
    assert np.abs(sm.astype(np.int64) - sw.astype(np.int64)).sum() <= 4
    assert rw["sum_dep_all"] + rw["sum_esc"] == pytest.approx(n * E, rel=1e-6)


def test_wavefront_batched_and_gradient():
    m = api.detmesh_build(W.GRAD_DET)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    items = [(E, W.GRAD_SOURCE, 60_000 + 1000 * i, i, [1, 1, 1, 1]) for i, E in enumerate((59.5, 122.0, 1332.0))]
    inst = api.make_instances(items)
    om = api.make_opts(n_group=4)
    ow = api.make_opts(n_group=4, variant=WAVEFRONT, wf_slots=16384)
    rm, sm, dm, _ = api.gadep_grad(b, mats, inst, om)
    rw, sw, dw, _ = api.gadep_grad(b, mats, inst, ow)
    for a, c in zip(rm, rw):
        assert a["n_hist"] == c["n_hist"]
        assert abs(a["n_fep"] - c["n_fep"]) <= 2
    assert np.allclose(dm, dw, rtol=1e-3, atol=1e-6)
    # the plain batched call through the wavefront form
    rb, sb = api.gadep_run_batch(b, mats, inst, api.make_opts(variant=WAVEFRONT, wf_slots=16384))
    assert [r["n_fep"] for r in rb] == [r["n_fep"] for r in rw]


def test_graph_loop_equals_host_loop():
    """The wavefront iterations driven by the graph's WHILE node (default) and by
    the host loop with per-kernel events (timing on) give the same histories."""
    m = api.detmesh_build(W.COAX_P)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    inst = api.make_instances([(662.0, W.COAX_POINT_25, 500_003, 0, []), (1332.0, W.COAX_POINT_25, 250_001, 1, [])])
    opts = api.make_opts(variant=WAVEFRONT, wf_slots=65536)
    p = api.Plan(b, mats, inst, opts)
    p.launch()
    rg, sg, _, _ = p.results()
    p.set_timing(True)
    p.launch()
    rh, sh, _, _ = p.results()
    stats = p.kernel_stats()
    p.set_timing(False)
    p.launch()                       # graph again, from the cached executable
    rg2, sg2, _, _ = p.results()
    for a, c, d in zip(rg, rh, rg2):
        for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_err", "n_segments", "n_interactions", "n_culled"):
            assert a[k] == c[k] == d[k], k
    assert np.array_equal(sg, sh) and np.array_equal(sg, sg2)
    assert stats["trace"][0] > 0 and stats["trace"][1] > 0.0
    # the queue log: one entry per iteration of the last launch, which served every
    # segment that needed a query (histories ended at birth need none); the host loop
    # may issue a few empty iterations past the end, so it launches at least as many
    q = p.queue_sizes()
    assert 0 < len(q) <= stats["trace"][0]
    assert sum(q) == sum(r["n_segments"] - r["n_culled"] for r in rg2)
    assert max(q) <= 65536


def test_smaller_slot_count_on_cached_buffers():
    """A run asking for fewer photon slots than the BVH's cached buffers hold keeps
    only those in flight (more iterations) and gives the same histories."""
    m = api.detmesh_build(W.COAX_P)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    inst = api.make_instances([(662.0, W.COAX_POINT_25, 800_000, 0, [])])
    big = api.Plan(b, mats, inst, api.make_opts(variant=WAVEFRONT, wf_slots=1 << 20))
    big.launch()
    rb, sb, _, _ = big.results()
    qb = big.queue_sizes()
    del big
    small = api.Plan(b, mats, inst, api.make_opts(variant=WAVEFRONT, wf_slots=1 << 14))
    small.launch()
    rs, ss, _, _ = small.results()
    qs = small.queue_sizes()
    assert max(qs) <= 1 << 14 < max(qb) and len(qs) > len(qb)
    for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_segments", "n_culled"):
        assert rb[0][k] == rs[0][k], k
    assert np.array_equal(sb, ss)


def test_graph_batch_captures_wavefront_plan():
    """A wavefront plan launched under stream capture (its WHILE node goes into the
    capturing graph) replays to the direct batched result."""
    from paper_2605_25963_gb300 import batch
    m = api.detmesh_build(W.BATCH_DET)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    items = []
    for i, (E, s, n, sm) in enumerate(W.batch_instances()[:7]):
        items.append((E, W.BATCH_SOURCES[s], int(n // 500) + 13 * i, i, [1, 1, 1, sm]))
    ref, ref_spec = api.gadep_run_batch(b, mats, api.make_instances(items), api.make_opts(variant=WAVEFRONT,
                                                                                              wf_slots=32768))
    g = batch.GraphBatch(b, mats, items, dict(variant=WAVEFRONT, wf_slots=32768))
    for _ in range(2):
        g.replay()
        res, spec, _, _ = g.results()
        for i in range(len(items)):
            for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_segments", "n_interactions"):
                assert res[i][k] == ref[i][k], (i, k)
        assert np.array_equal(spec, ref_spec)
