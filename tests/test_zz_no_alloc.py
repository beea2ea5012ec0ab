"""gadep_run_noalloc: the run for callers that cannot let a library allocate
device memory (an application-owned device allocator holds the memory, or a
loop cannot take cudaFree's device synchronisation).

Its scratch lives in a fixed device array inside the library, so the check is
that two calls in a row -- the second reusing the array the first left behind --
give exactly what gadep_run gives for the same arguments.  This file is collected
last so a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2605_25963_gb300 import api, capi
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _same(a, b):
    for k in ("n_hist", "n_fep", "n_zero", "n_over", "n_err", "n_segments", "n_interactions", "n_culled", "dev_err"):
        assert a[k] == b[k], k
    assert a["fepe"] == b["fepe"] and a["sigma"] == b["sigma"]
    assert a["sum_dep_active"] == pytest.approx(b["sum_dep_active"], rel=1e-9)


@pytest.mark.parametrize("name,src,E,n", [
    ("COAX_P", W.COAX_POINT_25, 1332.0, 300_000),
    ("BARE_CYLINDER", W.BARE_POINT_100, 662.0, 200_003),
])
def test_noalloc_matches_gadep_run_twice(name, src, E, n):
    mesh = api.detmesh_build(getattr(W, name))
    bvh = api.gadep_bvh_build(mesh, 0)
    mats = api.Materials.default()
    opts = api.make_opts(seed=7)
    ref, ref_spec = api.gadep_run(bvh, mats, src, E, n, instance=3, opts=opts)
    spec = torch.full((opts.n_bins,), 12345, dtype=torch.int32, device="cuda")
    for _ in range(2):
        r = api.gadep_run_noalloc(bvh, mats, src, E, n, spec, instance=3, opts=opts)
        _same(r, ref)
        assert np.array_equal(spec.cpu().numpy().view(np.uint32), ref_spec)
        assert r["n_fep"] > 0


def test_noalloc_volume_source_and_limits():
    mesh = api.detmesh_build(W.GRAD_DET)
    bvh = api.gadep_bvh_build(mesh, 0)
    mats = api.Materials.default()
    opts = api.make_opts(group_scale=[1.0, 1.0, 1.0, 0.5])
    ref, ref_spec = api.gadep_run(bvh, mats, W.GRAD_SOURCE, 122.0, 100_000, opts=opts)
    spec = torch.zeros(opts.n_bins, dtype=torch.int32, device="cuda")
    r = api.gadep_run_noalloc(bvh, mats, W.GRAD_SOURCE, 122.0, 100_000, spec, opts=opts)
    _same(r, ref)
    assert np.array_equal(spec.cpu().numpy().view(np.uint32), ref_spec)
    # tables larger than the fixed scratch are refused with a clear error
    big = api.Materials(np.repeat(mats.mu, 5, axis=2))      # 4 used materials x 5000 points
    with pytest.raises(capi.GadepError) as e:
        api.gadep_run_noalloc(bvh, big, W.GRAD_SOURCE, 122.0, 1000, spec, opts=opts)
    assert e.value.status == capi.GADEP_E_INVAL and "12288" in str(e.value)


def test_noalloc_above_the_wavefront_threshold():
    """2e6 coax histories (about 5e5 reach the scene, so AUTO in gadep_run takes the
    wavefront form): the call runs the megakernel and equals gadep_run in that form
    exactly; against gadep_run's AUTO choice (the other form, equal to rounding)
    the tallies agree to a few histories.  The wavefront variant is refused."""
    mesh = api.detmesh_build(W.COAX_P)
    bvh = api.gadep_bvh_build(mesh, 0)
    mats = api.Materials.default()
    n = 2_000_000
    mega, mega_spec = api.gadep_run(bvh, mats, W.COAX_POINT_25, 662.0, n, opts=api.make_opts(variant=1))
    auto, _ = api.gadep_run(bvh, mats, W.COAX_POINT_25, 662.0, n)
    spec = torch.zeros(4096, dtype=torch.int32, device="cuda")
    r = api.gadep_run_noalloc(bvh, mats, W.COAX_POINT_25, 662.0, n, spec)
    _same(r, mega)
    assert np.array_equal(spec.cpu().numpy().view(np.uint32), mega_spec)
    assert r["n_culled"] > 0
    for k in ("n_fep", "n_zero", "n_over"):
        assert abs(r[k] - auto[k]) <= 5, (k, r[k], auto[k])
    with pytest.raises(capi.GadepError) as e:
        api.gadep_run_noalloc(bvh, mats, W.COAX_POINT_25, 662.0, 1000, spec, opts=api.make_opts(variant=2))
    assert e.value.status == capi.GADEP_E_INVAL
