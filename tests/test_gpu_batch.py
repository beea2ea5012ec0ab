"""Batched runs on the GPU: CUDA-graph replay of a plan, autotuned launch shapes,
uneven instance sizes -- all bit-identical to the direct batched call."""
import numpy as np
import pytest

from paper_2605_25963_gb300 import api, batch
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _items(k=9, scale=2000):
    out = []
    for i, (E, s, n, sm) in enumerate(W.batch_instances()[:k]):
        out.append((E, W.BATCH_SOURCES[s], int(n // scale) + 17 * i, i, [1, 1, 1, sm]))
    return out


def test_graph_replay_equals_direct_batch():
    m = api.detmesh_build(W.BATCH_DET)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    items = _items()
    ref, ref_spec = api.gadep_run_batch(b, mats, api.make_instances(items))
    g = batch.GraphBatch(b, mats, items)
    for _ in range(3):
        g.replay()
        res, spec, _, _ = g.results()
        for i in range(len(items)):
            for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_segments", "n_interactions"):
                assert res[i][k] == ref[i][k]
        assert np.array_equal(spec, ref_spec)


def test_autotune_shapes_give_identical_results():
    m = api.detmesh_build(W.BATCH_DET)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    items = _items(k=6)
    kw, table = batch.autotune(b, mats, items, sample_histories=200_000, repeats=1)
    assert len(table) == len(batch.default_candidates()) and kw in [t[0] for t in table]
    base, base_spec = api.gadep_run_batch(b, mats, api.make_instances(items))
    for cand, _ in table:
        res, spec = api.gadep_run_batch(b, mats, api.make_instances(items), api.make_opts(**cand))
        assert [r["n_fep"] for r in res] == [r["n_fep"] for r in base]
        assert np.array_equal(spec, base_spec)


def test_autotune_keeps_caller_options():
    """The caller's options (here charged-particle tracks) go into every candidate,
    so the tuned batch computes what was asked for."""
    m = api.detmesh_build(W.BATCH_DET)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    items = _items(k=4)
    kw, table = batch.autotune(b, mats, items, sample_histories=100_000, repeats=1, opts_kw=dict(e_model=1))
    assert kw["e_model"] == 1 and all(c["e_model"] == 1 for c, _ in table)
    ref, _ = api.gadep_run_batch(b, mats, api.make_instances(items), api.make_opts(e_model=1))
    res, _ = api.gadep_run_batch(b, mats, api.make_instances(items), api.make_opts(**kw))
    assert [r["n_fep"] for r in res] == [r["n_fep"] for r in ref]
    assert [r["n_zero"] for r in res] == [r["n_zero"] for r in ref]
