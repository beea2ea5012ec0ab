"""Host-side checks of libgadep (no GPU needed).

  * the library loads and exports every function include/gadep.h declares;
  * DetMesh surfaces equal the oracle's surfaces (vertex sets, triangle counts,
    per-solid volumes, Euler characteristics, nesting tree);
  * the library's attenuation tables equal the oracle's tables to 1 ulp;
  * BVH invariants on the host copy;
  * invalid inputs fail with status codes, broken meshes with GADEP_E_MESH.
"""
import ctypes as C
import os
import re

import numpy as np
from scipy.spatial import cKDTree
import pytest

from paper_2605_25963_gb300 import api, capi
from paper_2605_25963_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gadep.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_library_exports_every_declared_symbol():
    L = capi.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(capi.EXPORTS)
    assert L.gadep_abi_version() == 2


def det_pair(orc, d):
    return api.detmesh_build(d), orc.Mesh.build(orc.Det(**d.as_dict()))


@pytest.mark.parametrize("name", ["BARE_CYLINDER", "COAX_P", "COAX_N", "BATCH_DET", "GRAD_DET", "STRESS_SMALL",
                                  "STRESS_DET", "DET2"])
def test_detmesh_matches_oracle_surfaces(orc, name):
    d = getattr(W, name)
    m, o = det_pair(orc, d)
    X, T, S, solids = m.arrays()
    OX, OT, OS, osol = o.arrays()
    assert len(T) == len(OT) and len(solids) == o.n_solid
    for s in range(o.n_solid):
        v, e = m.solid_stats(s)
        assert v == pytest.approx(o.volume(s), rel=1e-6), s
        assert e == o.euler(s) == (-32 if (d.flange_h > 0 and s == W.STRESS_FLANGE_SOLID) else 2), s
        # the same vertex set per solid (FP32 storage vs FP64): as many vertices, and
        # each one's nearest counterpart on the other side within FP32 rounding
        a = X[np.unique(T[S == s])].astype(np.float64)
        b = OX[np.unique(OT[OS == s])]
        assert a.shape == b.shape, s
        for p, q in ((a, b), (b, a)):
            dist, _ = cKDTree(q).query(p)
            assert dist.max() <= 2e-4, (s, dist.max())
        assert (S == s).sum() == (OS == s).sum()
        assert solids[s]["material"] == osol["material"][s]
        assert solids[s]["active"] == osol["active"][s]
        assert solids[s]["group"] == osol["group"][s]
        assert solids[s]["parent"] == osol["parent"][s], (s, solids[s], osol["parent"][s])
    # outward normals: n = (v1 - v0) x (v2 - v0) has positive flux volume per solid
    for s in range(o.n_solid):
        assert m.solid_stats(s)[0] > 0


def test_detmesh_locate_matches_oracle(orc):
    m, o = det_pair(orc, W.GRAD_DET)
    rng = np.random.default_rng(7)
    pts = np.column_stack([rng.uniform(-45, 45, 400), rng.uniform(-45, 45, 400), rng.uniform(-130, 45, 400)])
    for p in pts:
        assert m.locate(p) == o.locate(p, (0.2672612, 0.5345225, 0.8017837)), p


@pytest.mark.parametrize("name", ["GRAD_DET", "STRESS_SMALL"])
def test_detmesh_locate_matches_oracle_near_surfaces(orc, name):
    """The host parity rule that localises birth points, against the oracle's,
    on both sides of 300 random triangles (0.003 and 0.2 mm along the normal,
    past every 1e-4 mm separation and the 0.01 mm source gap) and inside the
    0.3 um bore contact (1.5e-4 mm in from its side wall, midway to the bore
    vacuum's aligned facets).  Every solid and the world are reached."""
    d = getattr(W, name)
    m, o = det_pair(orc, d)
    xyz, tri, ts, _ = o.arrays()
    v = xyz[tri]
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    cen = v.mean(1)
    pick = np.random.default_rng(11).choice(len(tri), 300, replace=False)
    pts = [cen[pick] + s * nrm[pick] for s in (0.003, -0.003, 0.2, -0.2)]
    wall = np.where((ts == 5) & (np.abs(nrm[:, 2]) < 0.5))[0][::16]
    pts.append(cen[wall] - 1.5e-4 * nrm[wall])
    seen = set()
    for p in np.concatenate(pts):
        want = o.locate(tuple(p), (0.2672612, 0.5345225, 0.8017837))
        assert m.locate(p) == want, p
        seen.add(want)
    assert len(wall) > 0 and seen == set(range(-1, o.n_solid))


def test_electron_ranges_match_oracle(orc):
    """The library's CSDA range tables (Gauss-Legendre, FP32) against the oracle's
    independent ones (Simpson, FP64, pinned to ESTAR in test_oracle_electron)."""
    r = api.gadep_erange_build()
    t = orc.Tables.build(W.MATERIAL_CODES)
    T = np.exp(np.linspace(np.log(W.ERANGE_T_MIN), np.log(W.TABLE_E_MAX), W.ERANGE_N))
    assert r.shape == (5, W.ERANGE_N)
    assert np.all(np.isinf(r[0]))                         # vacuum slows nothing
    for m in range(1, 5):
        o = np.array([t.e_range(m, x) for x in T[::7]])
        assert np.allclose(r[m, ::7], o, rtol=1e-5, atol=0), m
        assert np.all(np.diff(r[m]) > 0)
    c = np.array([1], dtype=np.int32)
    out = np.zeros(4, dtype=np.float32)
    lib = capi.load()
    assert lib.gadep_erange_build(api._ptr(c, C.c_int32), 1, 1, 1.0, 10.0, api._ptr(out, C.c_float)) != 0
    assert lib.gadep_erange_build(api._ptr(c, C.c_int32), 1, 4, 10.0, 1.0, api._ptr(out, C.c_float)) != 0
    c[0] = 77
    assert lib.gadep_erange_build(api._ptr(c, C.c_int32), 1, 4, 1.0, 10.0, api._ptr(out, C.c_float)) != 0


def test_tables_match_oracle(orc):
    mu = api.gadep_xs_build()
    ref = orc.Tables.build(W.MATERIAL_CODES).array()
    assert mu.shape == ref.shape == (5, 3, 1000)
    a = mu.view(np.int32).astype(np.int64)
    b = ref.view(np.int32).astype(np.int64)
    assert np.max(np.abs(a - b)) <= 1          # at most one unit in the last place
    assert np.array_equal(mu[0], np.zeros_like(mu[0]))
    assert np.all(mu[:, 2, :][:, np.exp(np.linspace(np.log(10), np.log(3000), 1000)) <= 2 * 510.99895] == 0)


@pytest.mark.parametrize("name", ["BARE_CYLINDER", "COAX_P", "GRAD_DET"])
@pytest.mark.parametrize("spatial", [False, True])
def test_bvh_host_invariants(name, spatial):
    m = api.detmesh_build(getattr(W, name))
    b = api.gadep_bvh_build(m, device=-1, split_alpha=1e-5 if spatial else 0.0, max_dup=2.0)
    b.validate()
    st = b.stats()
    assert st["n_tri"] == len(m.arrays()[1])
    assert st["max_leaf_tris"] <= 4
    assert st["max_depth"] < 60
    # one tree over every triangle + one per region over its own and its children's
    # triangles: each triangle is in three trees (global, own region, parent region);
    # spatial splits add copies, within the budget of max_dup records per triangle
    assert st["node_bytes"] == 64 * st["n_nodes"] and st["tri_bytes"] == 48 * st["n_refs"]
    if spatial:
        assert 3 * st["n_tri"] <= st["n_refs"] <= 2 * 3 * st["n_tri"] + 64
    else:
        assert st["n_refs"] == 3 * st["n_tri"]
    # 4-wide nodes with 2..4 children (1 for a tree that is a single leaf): the
    # child slots, n_nodes - n_trees inner children plus the leaves, number between
    # 2 and 4 per node
    n_trees = 1 + st["n_region"]
    slots = st["n_nodes"] - n_trees + st["n_leaves"]
    assert 2 * st["n_nodes"] - n_trees <= slots <= 4 * st["n_nodes"]
    # the greedy collapse fills most slots of the large trees
    if name != "BARE_CYLINDER":
        assert slots >= 2.9 * st["n_nodes"], slots / st["n_nodes"]
    assert st["n_leaves"] >= st["n_refs"] / 4


@pytest.mark.parametrize("name", ["BARE_CYLINDER", "COAX_P", "STRESS_SMALL"])
def test_bvh_clipped_references(name):
    """Early split clipping: the centre-fan triangles of the flat end faces are
    stored as several references whose boxes fit their pieces; the tree still
    passes every invariant (each triangle covered by its leaf boxes, none twice in
    one leaf) and holds more records than triangles per tree."""
    m = api.detmesh_build(getattr(W, name))
    plain = api.gadep_bvh_build(m, device=-1).stats()
    b = api.gadep_bvh_build(m, device=-1, clip_ratio=6.0, clip_pieces=16)
    b.validate()
    st = b.stats()
    assert st["n_refs"] > plain["n_refs"]
    assert st["n_refs"] <= 16 * plain["n_refs"]
    assert st["opts"]["clip_ratio"] == 6.0


def test_bvh_options():
    m = api.detmesh_build(W.COAX_P)
    for kw in (dict(max_leaf=0), dict(max_leaf=8), dict(c_tri=0.0), dict(split_alpha=-1.0), dict(max_dup=0.5)):
        with pytest.raises(capi.GadepError):
            api.gadep_bvh_build(m, device=-1, **kw)
    with pytest.raises(TypeError):
        api.gadep_bvh_build(m, device=-1, leaf=2)
    b = api.gadep_bvh_build(m, device=-1, max_leaf=2, c_trav=0.5, split_alpha=0.0)
    b.validate()
    st = b.stats()
    assert st["max_leaf_tris"] <= 2 and st["opts"]["max_leaf"] == 2 and st["opts"]["c_trav"] == 0.5
    d = api.gadep_bvh_build(m, device=-1).stats()["opts"]
    # the options a tree reports are the ones it was built with: AUTO clipping
    # resolved to off for this small mesh
    assert d == {"max_leaf": 4, "c_trav": 1.5, "c_tri": 1.0, "split_alpha": 0.0, "max_dup": 2.0, "clip_ratio": 0.0,
                 "clip_pieces": 16}
    o = api.bvh_opts()
    assert o.clip_ratio < 0 and o.clip_pieces == 16
    for kw in (dict(clip_ratio=0.5), dict(clip_ratio=4.0, clip_pieces=0), dict(clip_ratio=4.0, clip_pieces=257)):
        with pytest.raises(capi.GadepError):
            api.gadep_bvh_build(m, device=-1, **kw)


def test_invalid_parameters_rejected():
    bad = W.Detector(**{**W.COAX_P.as_dict(), "n_theta": 2})
    with pytest.raises(capi.GadepError) as e:
        api.detmesh_build(bad)
    assert e.value.status == capi.GADEP_E_INVAL
    overlapping = W.Detector(**{**W.COAX_P.as_dict(), "D": (62.0, 40.0, 3.0, 0.7, 48.0, 5.0, 0.0003)})
    with pytest.raises(capi.GadepError) as e:
        api.detmesh_build(overlapping)
    assert e.value.status == capi.GADEP_E_INVAL
    with pytest.raises(capi.GadepError):
        api.detmesh_build(W.Detector(kind=7))
    with pytest.raises(capi.GadepError):
        api.gadep_xs_build(codes=(1, 99))


def test_broken_meshes_rejected():
    xyz, tri, ts = W.box_mesh([(0, 0, 0, 1, 1, 1)])
    ok = api.detmesh_from_arrays(xyz, tri, ts, [1], [1], [-1])
    assert ok.solid_stats(0)[0] == pytest.approx(1.0)
    # open surface: drop one triangle
    with pytest.raises(capi.GadepError) as e:
        api.detmesh_from_arrays(xyz, tri[:-1], ts[:-1], [1], [1], [-1])
    assert e.value.status == capi.GADEP_E_MESH
    # inward normals
    with pytest.raises(capi.GadepError) as e:
        api.detmesh_from_arrays(xyz, tri[:, ::-1], ts, [1], [1], [-1])
    assert e.value.status == capi.GADEP_E_MESH
    # one flipped triangle: inconsistent orientation
    t2 = tri.copy()
    t2[3] = t2[3][::-1]
    with pytest.raises(capi.GadepError) as e:
        api.detmesh_from_arrays(xyz, t2, ts, [1], [1], [-1])
    assert e.value.status == capi.GADEP_E_MESH
    # two intersecting boxes
    xyz2, tri2, ts2 = W.box_mesh([(0, 0, 0, 2, 2, 2), (1, 1, 1, 3, 3, 3)])
    with pytest.raises(capi.GadepError) as e:
        api.detmesh_from_arrays(xyz2, tri2, ts2, [1, 2], [1, 0], [-1, -1])
    assert e.value.status == capi.GADEP_E_MESH
    # nested boxes: nesting tree from the parity rule
    xyz3, tri3, ts3 = W.box_mesh([(0, 0, 0, 4, 4, 4), (1, 1, 1, 3, 3, 3), (10, 0, 0, 11, 1, 1)])
    m = api.detmesh_from_arrays(xyz3, tri3, ts3, [1, 2, 3], [0, 1, 0], [-1, -1, -1])
    assert [s["parent"] for s in m.arrays()[3]] == [-1, 0, -1]
    assert m.locate((2, 2, 2)) == 1 and m.locate((0.5, 2, 2)) == 0 and m.locate((5, 5, 5)) == -1


def test_transport_needs_device_copy():
    m = api.detmesh_build(W.BARE_CYLINDER)
    b = api.gadep_bvh_build(m, device=-1)
    mat = api.Materials.default()
    with pytest.raises(capi.GadepError) as e:
        api.gadep_run(b, mat, W.BARE_POINT_100, 662.0, 10)
    assert e.value.status == capi.GADEP_E_INVAL


def test_opts_defaults():
    o = api.make_opts()
    assert o.seed == 1 and o.n_bins == 4096 and o.step_cap == 10000
    assert abs(o.e_cut_keV - 10.0) < 1e-6 and abs(o.fep_delta_keV - 0.01) < 1e-9
    assert list(o.group_scale) == [1.0] * 8


STRUCTS = ("detmesh_params", "gadep_solid", "gadep_bvh_opts", "gadep_bvh_stats", "gadep_materials",
           "gadep_source", "gadep_opts", "gadep_result", "gadep_kernel_stats", "gadep_instance")


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors in capi.py have the sizes and field offsets the C compiler
    gives the structs of include/gadep.h (gcc, the host ABI the library is built with)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gadep.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(capi, name)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        name, key, val = line.split()
        got[(name, key)] = int(val)
    for name in STRUCTS:
        cls = getattr(capi, name)
        assert C.sizeof(cls) == got[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == got[(name, field)], (name, field)


def test_handles_release_once():
    """close() releases a handle once; a with-block closes it; later closes and
    collection do nothing."""
    with api.detmesh_build(W.BARE_CYLINDER) as m:
        assert m.handle
        b = api.gadep_bvh_build(m, -1)
        assert b.stats()["n_tri"] == 192
        b.close()
        assert b.handle is None
        b.close()
    assert m.handle is None
    m.close()
    del m, b
