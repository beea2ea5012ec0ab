"""Gradient-driven dead-layer characterisation on the GPU: "measured" FEPE
values come from the FP64 oracle at a hidden dead-layer density scale (an
independent seed, so their noise is independent of the GPU's histories); the
Gauss-Newton fit with the density-perturbation Jacobian must recover the hidden
scale within its own statistical error.  Also checks that the autograd
gradient of chi2 through FepeFn equals 2 sum_i r_i J_i / sigma_i."""
import math

import numpy as np
import pytest

from paper_2605_25963_gb300 import api, fit
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

HIDDEN = 1.4          # dead-layer density scale the "measurement" was taken at
ENERGIES = (59.5, 122.0, 662.0)


def test_dead_layer_scale_recovered(orc):
    m = api.detmesh_build(W.COAX_P)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    om = orc.Mesh.build(orc.Det(**W.COAX_P.as_dict()))
    tab = orc.Tables.build(W.MATERIAL_CODES)
    src = orc.Source(kind=W.COAX_POINT_25.kind, pos=W.COAX_POINT_25.pos, dir=W.COAX_POINT_25.dir)
    n_meas = 1_500_000
    targets, sigmas = [], []
    for i, E in enumerate(ENERGIES):
        ro = orc.transport(om, tab, src, E, n_meas, seed=7, instance=i, group_scale=(HIDDEN, 1.0, 1.0, 1.0))
        targets.append(ro.fepe)
        sigmas.append(ro.sigma)
    items = [(E, W.COAX_POINT_25, 4_000_000, i) for i, E in enumerate(ENERGIES)]
    s, sig, hist = fit.fit_density_scales(b, mats, items, targets, sigmas, free_groups=[0], s0=[1.0, 1.0, 1.0, 1.0])
    assert len(hist) <= 10
    assert abs(s[0] - HIDDEN) <= max(3.0 * sig[0], 0.01 * HIDDEN), (s[0], sig[0], hist[-1]["chi2"])
    assert hist[-1]["chi2"] < hist[0]["chi2"]


def test_autograd_gradient_of_chi2_matches_jacobian():
    from paper_2605_25963_gb300 import autograd
    m = api.detmesh_build(W.GRAD_DET)
    b = api.gadep_bvh_build(m, 0)
    mats = api.Materials.default()
    items = [(E, W.GRAD_SOURCE, 300_000, i, [1.0, 1.0, 1.0, 1.0]) for i, E in enumerate((59.5, 122.0))]
    scales = torch.tensor([1.1, 1.0, 1.0, 0.9], dtype=torch.float64, requires_grad=True)
    target = torch.tensor([0.002, 0.05], dtype=torch.float64)
    sig = torch.tensor([1e-4, 1e-3], dtype=torch.float64)
    f = autograd.fepe(scales, b, mats, items)
    chi2 = (((f - target) / sig) ** 2).sum()
    chi2.backward()
    inst = api.make_instances([(E, src, n, iid, [1.1, 1.0, 1.0, 0.9]) for E, src, n, iid, _ in items])
    res, _, d, _ = api.gadep_grad(b, mats, inst, api.make_opts(n_group=4))
    fv = np.array([r["fepe"] for r in res])
    expect = 2.0 * ((fv - target.numpy()) / sig.numpy() ** 2) @ d
    assert np.allclose(scales.grad.numpy(), expect, rtol=1e-9, atol=1e-6 * np.abs(expect).max())
    assert math.isclose(float(f.detach()[0]), fv[0], rel_tol=0, abs_tol=0)
