"""Stress geometry on the GPU: the coax with a back-face contact groove and a
bolted Cu flange, at 64 segments (oracle parity on whole runs) and at 1024
segments (~1e6 triangles: sampled histories and rays checked one by one against
the oracle's brute force, the two transport forms against each other, batched
gradients against individual runs)."""
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

MEGA, WAVEFRONT = 1, 2
_cache = {}


@pytest.fixture(scope="module")
def mats():
    return api.Materials.default()


@pytest.fixture(scope="module")
def otab(orc):
    return orc.Tables.build(W.MATERIAL_CODES)


def scene(orc, name):
    if name not in _cache:
        d = getattr(W, name)
        m = api.detmesh_build(d)
        _cache[name] = (m, api.gadep_bvh_build(m, 0), orc.Mesh.build(orc.Det(**d.as_dict())))
    return _cache[name]


def osrc(orc, s):
    return orc.Source(kind=s.kind, pos=s.pos, dir=s.dir, radius=s.radius, height=s.height, n_sides=s.n_sides)


def chi2_two_sample(a, b, min_count=10):
    a, b = np.asarray(a, float), np.asarray(b, float)
    m = (a + b) >= min_count
    a, b = a[m], b[m]
    Na, Nb = a.sum(), b.sum()
    k1, k2 = math.sqrt(Nb / Na), math.sqrt(Na / Nb)
    return stats.chi2.sf(np.sum((k1 * a - k2 * b) ** 2 / (a + b)), len(a) - 1)


@pytest.mark.parametrize("E", [W.STRESS_ENERGIES[0], W.STRESS_ENERGIES[4], W.STRESS_ENERGIES[7]])
def test_stress_small_parity(orc, otab, mats, E):
    m, b, om = scene(orc, "STRESS_SMALL")
    n = 100_000
    trace = torch.empty(n, dtype=torch.float32, device="cuda")
    r, spec = api.gadep_run(b, mats, W.STRESS_SOURCE, E, n, edep_trace=trace)
    ro = orc.transport(om, otab, osrc(orc, W.STRESS_SOURCE), E, n, want_edep=True)
    assert r["n_err"] == 0 and ro.tally["n_err"] == 0 and ro.tally["n_parity_mismatch"] == 0
    g = trace.cpu().numpy().astype(np.float64)
    same = np.abs(g - ro.edep[:n]) <= 1e-3 + 1e-6 * np.abs(ro.edep[:n])
    assert same.mean() >= 0.999, same.mean()
    assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma)
    assert chi2_two_sample(spec, ro.spectrum) > 0.01
    assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(n * E, rel=1e-6)


def test_stress_full_mesh_sampled_histories(orc, otab, mats):
    """~1e6 triangles: the first 5,000 histories of a GPU run at each of the eight
    stress energies, one by one, against the oracle's brute force over every
    triangle (same Philox streams).  40,000 histories in all, so a 0.1 % class of
    disagreement would show."""
    m, b, om = scene(orc, "STRESS_DET")
    assert b.stats()["n_tri"] >= 1_000_000 or len(m.arrays()[1]) >= 1_000_000
    n, n_check = 400_000, 5_000
    agree = []
    for E in W.STRESS_ENERGIES:
        trace = torch.empty(n, dtype=torch.float32, device="cuda")
        r, _ = api.gadep_run(b, mats, W.STRESS_SOURCE, E, n, edep_trace=trace)
        assert r["n_hist"] == n and r["n_err"] == 0 and r["dev_err"] == 0
        ro = orc.transport(om, otab, osrc(orc, W.STRESS_SOURCE), E, n_check, want_edep=True)
        assert ro.tally["n_err"] == 0 and ro.tally["n_parity_mismatch"] == 0
        g = trace.cpu().numpy()[:n_check].astype(np.float64)
        same = np.abs(g - ro.edep[:n_check]) <= 1e-3 + 1e-6 * np.abs(ro.edep[:n_check])
        agree.append(same.mean())
        assert same.mean() >= 0.997, (E, same.mean())
        assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(n * E, rel=1e-6)
    assert np.mean(agree) >= 0.999, agree


def test_stress_full_mesh_forms_agree(orc, mats):
    """Megakernel and wavefront give the same histories on the 1e6-triangle mesh."""
    m, b, _ = scene(orc, "STRESS_DET")
    n = 1_500_001
    E = W.STRESS_ENERGIES[5]
    tr_m = torch.empty(n, dtype=torch.float32, device="cuda")
    tr_w = torch.empty(n, dtype=torch.float32, device="cuda")
    rm, sm = api.gadep_run(b, mats, W.STRESS_SOURCE, E, n, edep_trace=tr_m, opts=api.make_opts(variant=MEGA))
    rw, sw = api.gadep_run(b, mats, W.STRESS_SOURCE, E, n, edep_trace=tr_w,
                           opts=api.make_opts(variant=WAVEFRONT, wf_slots=1 << 19))
    assert rm["n_err"] == rw["n_err"] == 0 and rm["n_hist"] == rw["n_hist"] == n
    assert np.mean(tr_m.cpu().numpy() == tr_w.cpu().numpy()) >= 0.9999
    for k in ("n_fep", "n_zero", "n_over"):
        assert abs(rm[k] - rw[k]) <= 3, (k, rm[k], rw[k])


def test_stress_full_mesh_nearest_hit(orc):
    """Sampled rays on the 1e6-triangle mesh: GPU distance and surface vs the
    oracle's FP64 brute force on the same binary32 vertices."""
    m, b, om64 = scene(orc, "STRESS_DET")
    X, T, S, sol = om64.arrays()
    X32 = X.astype(np.float32).astype(np.float64)
    om = orc.Mesh.from_arrays(X32, T, S, sol["material"], sol["active"], sol["group"], sol["parent"])
    gpu_solid = m.arrays()[2]
    rng = np.random.default_rng(5)
    n = 400
    o = np.column_stack([rng.uniform(-38, 38, n), rng.uniform(-38, 38, n), rng.uniform(-80, 10, n)])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3] = o
    rays[:, 4:7] = d
    rays[:, 7] = np.array([-1] * n, np.int32).view(np.float32)
    t, tri, ent = (x.cpu().numpy() for x in api.gadep_nearest_hit(b, torch.from_numpy(rays).cuda()))
    # 1e-5 relative where the hit is well conditioned.  Binary32 translation of the
    # vertices to the origin moves them by ~eps32 |v - o|: at grazing incidence that
    # adds ~eps32 (|o| + |v|) / |cos|, and on a sliver triangle (the endcap walls are
    # single 118 mm bands of 0.23 mm facets) it shifts the barycentrics by
    # ~eps32 L / h and t by ~eps32 L^2 / h, h = 2 A |cos| / L the projected width.
    eps32 = 2.0 ** -24
    agree = strict = 0
    for i in range(n):
        oo, dd = rays[i, 0:3].astype(np.float64), rays[i, 4:7].astype(np.float64)
        k, tt, ee = om.nearest_hit(oo, dd, 0.0, -1)
        if k < 0:
            assert tri[i] == -1
            agree += 1
            strict += 1
            continue
        v = X32[T[k]]
        nrm = np.cross(v[1] - v[0], v[2] - v[0])
        cosv = abs(np.dot(dd, nrm / np.linalg.norm(nrm)))
        L = np.linalg.norm(v - oo, axis=1).max()
        h = np.linalg.norm(nrm) * max(cosv, 1e-3) / L
        tol = (1e-5 * max(tt, 1.0) + 8 * eps32 * (np.abs(oo).max() + np.abs(v).max()) / max(cosv, 1e-3)
               + 2 * eps32 * L * L / h)
        assert abs(t[i] - tt) <= tol, (i, t[i], tt, cosv)
        strict += abs(t[i] - tt) <= 1e-5 * max(tt, 1.0)
        agree += tri[i] >= 0 and gpu_solid[tri[i]] == S[k] and ent[i] == ee
    assert strict / n >= 0.99 and agree / n >= 0.995, (strict / n, agree / n)


def test_stress_batched_gradient_equals_individual(orc, mats):
    """The eight stress energies in one batched gradient launch: tallies equal
    individual runs bit for bit, dFEPE matches each instance's own run.  Both in the
    same form (AUTO could pick the wavefront kernels for the batch and the
    megakernel for single runs; the two forms agree history by history only to
    rounding, not bit for bit)."""
    m, b, _ = scene(orc, "STRESS_DET")
    items = [(E, W.STRESS_SOURCE, 60_000 + 7919 * i, i, [1, 1, 1, 1]) for i, E in enumerate(W.STRESS_ENERGIES)]
    res, spec, dfe, dsg = api.gadep_grad(b, mats, api.make_instances(items), api.make_opts(n_group=4, variant=MEGA))
    for i, it in enumerate(items):
        r1, s1, d1, _ = api.gadep_grad(b, mats, api.make_instances([it]), api.make_opts(n_group=4, variant=MEGA))
        for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_segments", "n_interactions"):
            assert r1[0][k] == res[i][k], (i, k)
        assert np.array_equal(s1[0], spec[i])
        assert np.allclose(d1[0], dfe[i], rtol=1e-9, atol=1e-12)
        assert np.all(np.isfinite(dfe[i])) and np.all(dsg[i] >= 0)
