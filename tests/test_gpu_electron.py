"""Charged-particle tracks (e_model 1) on the GPU against the FP64 oracle.

The tracks draw no random numbers, so both sides follow the same photon
histories; a history whose charged particles all stop in the region they
start in deposits exactly as with local deposition.  Tracks that cross a
boundary deposit T - T' with T' from the FP32 range table on the GPU and from
the FP64 table and bisection in the oracle (relative difference ~1e-5 of T),
so the per-history comparison allows 0.05 keV + 1e-4 relative.
"""
import math

import numpy as np
import pytest

from paper_2605_25963_gb300 import api, capi
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_transport import chi2_two_sample, osrc, scene  # noqa: E402

MEGA, WAVEFRONT = 1, 2


@pytest.fixture(scope="module")
def mats():
    return api.Materials.default()


@pytest.fixture(scope="module")
def otab(orc):
    return orc.Tables.build(W.MATERIAL_CODES)


def run_both(orc, otab, mats, name, src, E, n, variant=MEGA, scales=()):
    m, b, om = scene(orc, name)
    trace = torch.empty(n, dtype=torch.float32, device="cuda")
    opts = api.make_opts(e_model=1, variant=variant, group_scale=list(scales) or None)
    r, spec = api.gadep_run(b, mats, src, E, n, opts=opts, edep_trace=trace)
    ro = orc.transport(om, otab, osrc(orc, src), E, n, want_edep=True, e_model=1, group_scale=scales)
    g = trace.cpu().numpy().astype(np.float64)
    same = np.abs(g - ro.edep) <= 0.05 + 1e-4 * np.abs(ro.edep)
    return r, spec, ro, same


@pytest.mark.parametrize("E", [122.0, 662.0, 1332.0])
def test_coax_tracks_parity(orc, otab, mats, E):
    n = 200_000
    r, spec, ro, same = run_both(orc, otab, mats, "COAX_P", W.COAX_POINT_25, E, n)
    assert r["n_err"] == 0 and ro.tally["n_err"] == 0
    assert same.mean() >= 0.999, same.mean()
    assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma)
    assert chi2_two_sample(spec, ro.spectrum) > 0.01
    assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(n * E, rel=1e-5)
    assert r["n_segments"] == pytest.approx(ro.tally["n_segments"], rel=2e-3)


def test_tracks_change_only_where_energy_lands(orc, otab, mats):
    """Same photon histories with and without tracks (the segment, interaction
    and history counts agree exactly); the full-energy peak loses the histories
    whose electrons leave the active volume.  The total active deposit may move
    either way: electrons set going in the dead layer carry energy inward."""
    m, b, _ = scene(orc, "COAX_P")
    n = 1_000_003
    r0, _ = api.gadep_run(b, mats, W.COAX_POINT_25, 1332.0, n, opts=api.make_opts(variant=MEGA))
    r1, _ = api.gadep_run(b, mats, W.COAX_POINT_25, 1332.0, n, opts=api.make_opts(variant=MEGA, e_model=1))
    for k in ("n_hist", "n_segments", "n_interactions", "n_culled"):
        assert r0[k] == r1[k], k
    assert r1["n_fep"] < r0["n_fep"]
    assert r1["sum_dep_active"] != r0["sum_dep_active"]
    for r in (r0, r1):
        assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(n * 1332.0, rel=1e-5)


def test_wavefront_equals_megakernel_with_tracks(mats, orc):
    m, b, _ = scene(orc, "COAX_P")
    n = 300_001
    tm = torch.empty(n, dtype=torch.float32, device="cuda")
    tw = torch.empty(n, dtype=torch.float32, device="cuda")
    rm, sm = api.gadep_run(b, mats, W.COAX_POINT_25, 1332.0, n, edep_trace=tm, opts=api.make_opts(variant=MEGA, e_model=1))
    rw, sw = api.gadep_run(b, mats, W.COAX_POINT_25, 1332.0, n, edep_trace=tw,
                           opts=api.make_opts(variant=WAVEFRONT, wf_slots=32768, e_model=1))
    assert rw["n_err"] == 0 and rw["n_hist"] == n
    # the wavefront form adds a track's deposits after the photon's segment when the
    # history goes on (etrack kernel), the megakernel at once: FP32 sums in another order
    assert np.mean(np.abs(tm.cpu().numpy() - tw.cpu().numpy()) <= 1e-3) >= 0.9999
    for k in ("n_fep", "n_zero", "n_over"):
        assert abs(rm[k] - rw[k]) <= 2, k
    assert rw["sum_dep_all"] + rw["sum_esc"] == pytest.approx(n * 1332.0, rel=1e-5)


def test_density_scale_and_volume_source_with_tracks(orc, otab, mats):
    # the water prism source on the coax: tracks start in water and in the
    # scaled dead layer (group 0) as well
    r, spec, ro, same = run_both(orc, otab, mats, "GRAD_DET", W.GRAD_SOURCE, 662.0, 100_000,
                                 scales=(1.6, 1.0, 1.0, 0.8))
    assert r["n_err"] == 0 and same.mean() >= 0.999, same.mean()
    assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma)


def test_track_argument_errors(orc, mats):
    m, b, _ = scene(orc, "COAX_P")
    bare = api.Materials(mats.mu)                       # no range tables
    with pytest.raises(capi.GadepError):
        api.gadep_run(b, bare, W.COAX_POINT_25, 662.0, 1000, opts=api.make_opts(e_model=1))
    with pytest.raises(capi.GadepError):
        api.gadep_run(b, mats, W.COAX_POINT_25, 662.0, 1000, opts=api.make_opts(e_model=2))
    inst = api.make_instances([(662.0, W.COAX_POINT_25, 1000, 0, [1, 1, 1, 1])])
    with pytest.raises(capi.GadepError):
        api.gadep_grad(b, mats, inst, api.make_opts(n_group=4, e_model=1))
    spec = torch.zeros(4096, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.GadepError):
        api.gadep_run_noalloc(b, mats, W.COAX_POINT_25, 662.0, 1000, spec, opts=api.make_opts(e_model=1))


def test_full_size_coax_tracks_against_oracle(orc, otab, mats):
    """Tracks at the bench's size and launch configuration (1e8 histories, AUTO
    form, the wavefront kernels here): against the oracle's e_model 1 at 1e7
    histories of the same streams, FEPE within 3 combined sigma, and the first
    1e5 histories one by one; a 1e7-history GPU run (the same histories as the
    oracle's) has the oracle's full-energy-peak count within 0.3 %."""
    m, b, om = scene(orc, "COAX_P")
    n, n_orc, n_trace = 100_000_000, 10_000_000, 100_000
    E = 1332.0
    trace = torch.empty(n_trace, dtype=torch.float32, device="cuda")
    r, spec = api.gadep_run(b, mats, W.COAX_POINT_25, E, n, edep_trace=trace, opts=api.make_opts(e_model=1))
    ro = orc.transport(om, otab, osrc(orc, W.COAX_POINT_25), E, n_orc, want_edep=True, e_model=1)
    assert r["n_err"] == 0 and ro.tally["n_err"] == 0
    assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma)
    r7, _ = api.gadep_run(b, mats, W.COAX_POINT_25, E, n_orc, opts=api.make_opts(e_model=1))
    assert abs(r7["n_fep"] - ro.tally["n_fep"]) <= 0.003 * ro.tally["n_fep"], (r7["n_fep"], ro.tally["n_fep"])
    g = trace.cpu().numpy().astype(np.float64)
    o = ro.edep[:n_trace]
    assert np.mean(np.abs(g - o) <= 0.05 + 1e-4 * np.abs(o)) >= 0.999
    assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(n * E, rel=1e-5)


def test_batched_tracks_equal_individual_runs(orc, mats):
    """Tracks in one batched launch (instances with their own density scales) give
    the tallies of the individual runs exactly."""
    m, b, _ = scene(orc, "BATCH_DET")
    items = []
    for i, (E, s, n, sm) in enumerate(W.batch_instances()[10:40:5]):
        items.append((E, W.BATCH_SOURCES[s], 20_000 + 991 * i, 5 * i + s, [1, 1, 1, sm]))
    res, spec = api.gadep_run_batch(b, mats, api.make_instances(items), api.make_opts(e_model=1, variant=MEGA))
    for i, (E, src, n, iid, sc) in enumerate(items):
        r, sp = api.gadep_run(b, mats, src, E, n, instance=iid,
                              opts=api.make_opts(e_model=1, group_scale=sc, variant=MEGA))
        for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_err", "n_segments", "n_interactions"):
            assert r[k] == res[i][k], (i, k)
        assert np.array_equal(sp, spec[i])


@pytest.mark.parametrize("E", [W.STRESS_ENERGIES[3], W.STRESS_ENERGIES[7]])
def test_stress_small_tracks_parity(orc, otab, mats, E):
    """Tracks through the groove, the bolted flange and the volume source."""
    r, spec, ro, same = run_both(orc, otab, mats, "STRESS_SMALL", W.STRESS_SOURCE, E, 100_000)
    assert r["n_err"] == 0 and ro.tally["n_err"] == 0
    assert same.mean() >= 0.999, same.mean()
    assert abs(r["fepe"] - ro.fepe) <= 3 * math.hypot(r["sigma"], ro.sigma)
    assert chi2_two_sample(spec, ro.spectrum) > 0.01
    assert r["sum_dep_all"] + r["sum_esc"] == pytest.approx(100_000 * E, rel=1e-5)
