"""GPU density-perturbation gradient: against the oracle on identical streams,
the analytic slab identity, central finite differences with common random
numbers, and the autograd wrapper."""
import math

import numpy as np
import pytest

from paper_2605_25963_gb300 import api
from paper_2605_25963_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def mats():
    return api.Materials.default()


def test_grad_matches_oracle_volume_source(orc, mats):
    """Same histories: 2e5 per energy on both sides (identical streams, so the
    plain kernel's FEP count is the gradient kernel's), dFEPE/ds within 3 combined
    sigma of the oracle's."""
    d = W.GRAD_DET
    m = api.detmesh_build(d)
    b = api.gadep_bvh_build(m, 0)
    om = orc.Mesh.build(orc.Det(**d.as_dict()))
    ot = orc.Tables.build(W.MATERIAL_CODES)
    src = W.GRAD_SOURCE
    os_ = orc.Source(kind=src.kind, pos=src.pos, radius=src.radius, height=src.height, n_sides=src.n_sides)
    n = 200_000
    for E in (59.5, 662.0):
        inst = api.make_instances([(E, src, n, 0, [1, 1, 1, 1])])
        res, spec, g, gs = api.gadep_grad(b, mats, inst, api.make_opts(n_group=4))
        ro = orc.transport(om, ot, os_, E, n, group_scale=(1.0, 1.0, 1.0, 1.0))
        plain, _ = api.gadep_run(b, mats, src, E, n)
        assert res[0]["n_fep"] == plain["n_fep"]                 # same histories as the plain kernel
        for p in range(4):
            go, so = ro.dfepe(p), ro.dfepe_sigma(p)
            assert abs(g[0, p] - go) <= 3 * math.hypot(gs[0, p], so) + 1e-12, (E, p, g[0, p], go)


def test_grad_full_size_against_oracle(orc, mats):
    """The gradient workload at its full size on the GPU (4 energies x 5e7
    histories of the volume source, one gadep_grad launch) against the oracle at
    2e6 histories per energy: FEPE and dFEPE/ds of each of the four density groups
    within 3 combined sigma."""
    d = W.GRAD_DET
    m = api.detmesh_build(d)
    b = api.gadep_bvh_build(m, 0)
    om = orc.Mesh.build(orc.Det(**d.as_dict()))
    ot = orc.Tables.build(W.MATERIAL_CODES)
    src = W.GRAD_SOURCE
    os_ = orc.Source(kind=src.kind, pos=src.pos, radius=src.radius, height=src.height, n_sides=src.n_sides)
    items = [(E, src, W.GRAD_HISTORIES, i, [1, 1, 1, 1]) for i, E in enumerate(W.GRAD_ENERGIES)]
    res, _, g, gs = api.gadep_grad(b, mats, api.make_instances(items), api.make_opts(n_group=4))
    for i, E in enumerate(W.GRAD_ENERGIES):
        ro = orc.transport(om, ot, os_, E, 2_000_000, instance=i, group_scale=(1.0, 1.0, 1.0, 1.0))
        assert res[i]["n_err"] == 0 and ro.tally["n_err"] == 0
        assert abs(res[i]["fepe"] - ro.fepe) <= 3 * math.hypot(res[i]["sigma"], ro.sigma), (E,)
        for p in range(4):
            go, so = ro.dfepe(p), ro.dfepe_sigma(p)
            assert abs(g[i, p] - go) <= 3 * math.hypot(gs[i, p], so) + 1e-12, (E, p, g[i, p], go)


def test_slab_identity_and_finite_differences(mats):
    """Pencil beam through an Al slab onto a Ge absorber.  Boundary term of the
    density-perturbation score: dFEPE/ds_Al = -mu x FEPE, within 3 sigma.  Central
    finite differences (+-1 %, common random numbers) within 3 combined sigma,
    the finite difference's sigma taken from 40 batch means of the same histories."""
    x = 2.0
    xyz, tri, ts = W.box_mesh([(-50, -50, -x, 50, 50, 0.0), (-50, -50, -40, 50, 50, -x - 1.0)])
    m = api.detmesh_from_arrays(xyz, tri, ts, [W.MAT_AL, W.MAT_GE], [0, 1], [0, 1])
    b = api.gadep_bvh_build(m, 0)
    src = W.Source(kind=W.SRC_PENCIL, pos=(0, 0, 5.0), dir=(0, 0, -1.0))
    E, n = 122.0, 2_000_000
    res, _, g, gs = api.gadep_grad(b, mats, api.make_instances([(E, src, n, 0, [1, 1])]), api.make_opts(n_group=2))
    fepe = res[0]["fepe"]
    # mu_tot of Al at E from the library's own tables (linear in ln E)
    lnE = np.linspace(math.log(10), math.log(3000), 1000)
    mu_al = sum(np.interp(math.log(E), lnE, mats.mu[W.MAT_AL, c]) for c in range(3))
    expect = -mu_al * x * fepe
    assert abs(g[0, 0] - expect) <= 3 * gs[0, 0], (g[0, 0], expect, gs[0, 0])
    h, n_batch = 0.01, 40
    nb = n // n_batch
    fd_b = []
    for k in range(n_batch):
        fp, _ = api.gadep_run(b, mats, src, E, nb, opts=api.make_opts(group_scale=[1 + h, 1], history_offset=k * nb))
        fm, _ = api.gadep_run(b, mats, src, E, nb, opts=api.make_opts(group_scale=[1 - h, 1], history_offset=k * nb))
        fd_b.append((fp["fepe"] - fm["fepe"]) / (2 * h))
    fd = float(np.mean(fd_b))
    s_fd = float(np.std(fd_b, ddof=1) / math.sqrt(n_batch))
    assert s_fd > 0
    assert abs(fd - g[0, 0]) <= 3 * math.hypot(s_fd, gs[0, 0]), (fd, g[0, 0], s_fd, gs[0, 0])


def test_autograd_backward(mats):
    from paper_2605_25963_gb300.autograd import fepe
    m = api.detmesh_build(W.GRAD_DET)
    b = api.gadep_bvh_build(m, 0)
    items = [(E, W.GRAD_SOURCE, 100_000, i, [1, 1, 1, 1]) for i, E in enumerate((59.5, 122.0))]
    s = torch.ones(4, dtype=torch.float64, requires_grad=True)
    f = fepe(s, b, mats, items)
    w = torch.tensor([1.0, -2.0], dtype=torch.float64)
    (f * w).sum().backward()
    _, _, d, _ = api.gadep_grad(b, mats, api.make_instances(items), api.make_opts(n_group=4))
    assert np.allclose(s.grad.numpy(), w.numpy() @ d)
    s2 = torch.ones(4, dtype=torch.float64, requires_grad=True)
    f2 = fepe(s2, b, mats, items, fused=True)
    (f2 * w).sum().backward()
    assert np.allclose(s2.grad.numpy(), s.grad.numpy())
    assert torch.equal(f, f2)
