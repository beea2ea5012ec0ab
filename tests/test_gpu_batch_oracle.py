"""The batched workload's geometry and sources against the FP64 oracle.

The batched workload runs a point, a disk and a volume (water prism) source on
one mesh: the bare Ge cylinder with the water prism on its top face, whose
density group is scaled to 0 for the point and disk instances (no matrix) and
to 1 for the volume source.  Each source is checked here against the oracle on
identical Philox streams, first as single runs large enough that AUTO takes the
wavefront form, then as instances of one batched plan (the form the benchmark
times), so that the batched path itself -- not only its agreement with
individual GPU runs -- is compared with the oracle.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2605_25963_gb300 import api
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

_cache = {}


@pytest.fixture(scope="module")
def mats():
    return api.Materials.default()


@pytest.fixture(scope="module")
def otab(orc):
    return orc.Tables.build(W.MATERIAL_CODES)


def scene(orc):
    if "b" not in _cache:
        m = api.detmesh_build(W.BATCH_DET)
        _cache["b"] = (m, api.gadep_bvh_build(m, 0), orc.Mesh.build(orc.Det(**W.BATCH_DET.as_dict())))
    return _cache["b"]


def osrc(orc, s):
    return orc.Source(kind=s.kind, pos=s.pos, dir=s.dir, radius=s.radius, height=s.height, n_sides=s.n_sides)


def chi2_two_sample(a, b, min_count=10):
    a, b = np.asarray(a, float), np.asarray(b, float)
    m = (a + b) >= min_count
    a, b = a[m], b[m]
    if len(a) < 2:
        return 1.0
    Na, Nb = a.sum(), b.sum()
    k1, k2 = math.sqrt(Nb / Na), math.sqrt(Na / Nb)
    return stats.chi2.sf(np.sum((k1 * a - k2 * b) ** 2 / (a + b)), len(a) - 1)


def scales_of(s):
    # dead layer, endcap, active Ge, source matrix: only the matrix changes
    return [1.0, 1.0, 1.0, 1.0 if s == 2 else 0.0]


@pytest.mark.parametrize("s", [0, 1, 2])
@pytest.mark.parametrize("E", [W.BATCH_ENERGIES[5], W.BATCH_ENERGIES[30]])
def test_batch_geometry_source_parity(orc, otab, mats, s, E):
    """One source of the batched workload, 400k histories (all born inside the
    scene box, so AUTO runs the wavefront form): per-history agreement, FEPE
    within 3 combined sigma, spectrum chi-square, energy bookkeeping."""
    m, b, om = scene(orc)
    src = W.BATCH_SOURCES[s]
    n = 400_000
    sc = scales_of(s)
    trace = torch.empty(n, dtype=torch.float32, device="cuda")
    r, spec = api.gadep_run(b, mats, src, E, n, instance=7, opts=api.make_opts(group_scale=sc), edep_trace=trace)
    ro = orc.transport(om, otab, osrc(orc, src), E, n, instance=7, want_edep=True, group_scale=tuple(sc))
    assert r["n_hist"] == n and r["n_err"] == 0 and r["dev_err"] == 0
    assert ro.tally["n_err"] == 0 and ro.tally["n_parity_mismatch"] == 0
    g = trace.cpu().numpy().astype(np.float64)
    same = np.abs(g - ro.edep) <= 1e-3 + 1e-6 * np.abs(ro.edep)
    assert same.mean() >= 0.999, same.mean()
    assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma), (r["fepe"], ro.fepe)
    assert chi2_two_sample(spec, ro.spectrum) > 0.01
    assert r["n_zero"] + r["n_over"] + spec.sum() == n
    assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(n * E, rel=1e-6)
    assert r["n_segments"] == pytest.approx(ro.tally["n_segments"], rel=2e-3)


def test_disk_source_births_and_parity_outside_a_matrix(orc, otab, mats):
    """The disk source on its own mesh (the bare cylinder, no prism), so that its
    births start in the world: per-history agreement and the full-energy-peak
    count against the oracle."""
    d = W.BARE_CYLINDER
    m = api.detmesh_build(d)
    b = api.gadep_bvh_build(m, 0)
    om = orc.Mesh.build(orc.Det(**d.as_dict()))
    src = W.BATCH_SOURCES[1]
    n = 300_000
    for E in (59.5, 1332.0):
        trace = torch.empty(n, dtype=torch.float32, device="cuda")
        r, spec = api.gadep_run(b, mats, src, E, n, edep_trace=trace)
        ro = orc.transport(om, otab, osrc(orc, src), E, n, want_edep=True)
        g = trace.cpu().numpy().astype(np.float64)
        assert np.mean(np.abs(g - ro.edep) <= 1e-3 + 1e-6 * np.abs(ro.edep)) >= 0.999
        assert abs(r["n_fep"] - ro.tally["n_fep"]) <= 3 + 0.002 * ro.tally["n_fep"]
        assert chi2_two_sample(spec, ro.spectrum) > 0.01
        # births outside the mesh whose first ray misses the scene box end at birth
        # on the GPU; on the oracle they are flights that meet no triangle
        assert 0 < r["n_culled"] <= ro.tally["n_first_none"]


def test_batched_plan_against_oracle(orc, otab, mats):
    """Six instances of the batched workload (three sources at two energies, uneven
    history counts, the workload's instance ids and matrix scales) in one
    gadep_run_batch launch, each against the oracle on the same streams: the
    full-energy-peak count to 0.2 % (the histories are the same ones), FEPE within
    3 combined sigma, spectrum chi-square.  Run with the AUTO choice and in each
    form forced."""
    m, b, om = scene(orc)
    items = []
    for k, (j, s) in enumerate([(3, 0), (3, 1), (3, 2), (33, 0), (33, 1), (33, 2)]):
        E = W.BATCH_ENERGIES[j]
        items.append((E, W.BATCH_SOURCES[s], 150_000 + 40_009 * k, 3 * j + s, scales_of(s)))
    inst = api.make_instances(items)
    expect = []
    for (E, src, n, iid, sc) in items:
        expect.append(orc.transport(om, otab, osrc(orc, src), E, n, instance=iid, group_scale=tuple(sc)))
    for variant in (0, 1, 2):
        res, spec = api.gadep_run_batch(b, mats, inst, api.make_opts(variant=variant))
        for i, ro in enumerate(expect):
            r = res[i]
            assert r["n_hist"] == items[i][2] and r["n_err"] == 0, (variant, i)
            assert abs(r["n_fep"] - ro.tally["n_fep"]) <= 3 + 0.002 * ro.tally["n_fep"], (variant, i)
            assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma), (variant, i)
            assert chi2_two_sample(spec[i], ro.spectrum) > 0.01, (variant, i)
