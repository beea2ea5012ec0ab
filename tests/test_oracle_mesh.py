"""Pins of the oracle's detector surfaces (CPU only).

Closed forms: the exact volume of a faceted solid of revolution (sum of
similar-N-gon frusta over the profile), convergence to the smooth volume at
O(N^-2), Euler characteristic 2 per closed genus-0 solid, every directed edge
matched by exactly one opposite edge (closed and consistently oriented),
positive signed volume (outward normals), the vertex equations of Sec. 2.2.2,
and the parity rule at points whose region is known by construction.
"""
import math

import numpy as np
import pytest

from paper_2605_25963_gb300 import workloads as W


def det(orc, d: W.Detector):
    return orc.Mesh.build(orc.Det(**d.as_dict()))


def faceted_volume(profile, N):
    """Volume of a closed (rho, z) profile revolved with N-gon cross sections.

    Each profile segment sweeps a frustum of similar N-gons:
    (z_a - z_b) * (N/2) sin(2 pi / N) * (ra^2 + ra rb + rb^2) / 3, signed.
    """
    c = 0.5 * N * math.sin(2 * math.pi / N)
    v = 0.0
    for (ra, za), (rb, zb) in zip(profile[:-1], profile[1:]):
        v += (za - zb) * c * (ra * ra + ra * rb + rb * rb) / 3.0
    return v


def rounded_profile(R, rch, zf, zb, n_phi):
    pts = []
    if rch > 0:
        hemi = rch == R
        if not hemi:
            pts.append((0.0, zf))
        for j in range(n_phi, -1, -1):
            phi = 0.5 * math.pi * j / n_phi
            r = 0.0 if (hemi and j == n_phi) else (R - rch) + rch * math.cos(phi)
            pts.append((r, zf - rch * (1 - math.sin(phi))))
    else:
        pts += [(0.0, zf), (R, zf)]
    pts += [(R, zb), (0.0, zb)]
    return pts


def disk_rings(R, N):
    """Inner ring (radius, vertex count) of a flat end face whose outer ring has
    radius R and N vertices: spacing w = 4 arcs of the outer ring, vertices in
    proportion to the radius (at least 8), while the radius is at least w and the
    count falls."""
    w = 4.0 * (2.0 * math.pi * R / N)
    rings, prev, k = [], N, 1
    while k < 64:
        r = R - k * w
        m = max(8, int(math.floor(N * r / R + 0.5)))
        if r < w or m >= prev:
            break
        rings.append((r, m))
        prev, k = m, k + 1
    return rings


def profile_tris(profile, N):
    """Triangles of a revolved profile: 2N per band between rings, N per fan to
    an axis point off the ring's plane, and for a flat end face the bands
    between its rings (as many triangles as the two rings have vertices) plus
    the centre fan of the innermost ring."""
    n = 0
    for (ra, za), (rb, zb) in zip(profile[:-1], profile[1:]):
        if ra > 0 and rb > 0:
            n += 2 * N
        elif (ra > 0) != (rb > 0) and za == zb:
            counts = [N] + [m for _, m in disk_rings(max(ra, rb), N)]
            n += sum(a + b for a, b in zip(counts[:-1], counts[1:])) + counts[-1]
        elif (ra > 0) != (rb > 0):
            n += N
    return n


def test_bare_cylinder_counts_volume_topology(orc):
    m = det(orc, W.BARE_CYLINDER)
    assert (m.n_vert, m.n_tri, m.n_solid) == (98, 192, 1)
    N, R, H = 48, 30.0, 60.0
    assert m.volume(0) == pytest.approx(N / 2 * R * R * math.sin(2 * math.pi / N) * H, rel=1e-12)
    assert m.volume(0) == pytest.approx(169161.9, abs=0.1)
    deficit = 1 - m.volume(0) / (math.pi * R * R * H)
    assert deficit == pytest.approx((2 * math.pi / N) ** 2 / 6, rel=0.01)
    assert m.euler(0) == 2 and m.open_edges(0) == 0
    xyz, tri, ts, solids = m.arrays()
    # vertex equations: x = R cos(2 pi i / N), y = R sin(2 pi i / N) on the rings
    ring = xyz[np.isclose(np.hypot(xyz[:, 0], xyz[:, 1]), R)]
    ang = np.sort(np.mod(np.arctan2(ring[:, 1], ring[:, 0]), 2 * math.pi))
    i = np.round(ang / (2 * math.pi / N))
    assert np.allclose(ang, 2 * math.pi * i / N, atol=1e-14)
    assert solids["active"][0] == 1 and solids["material"][0] == W.MAT_GE


def test_volume_converges_second_order(orc):
    R, H = 30.0, 60.0
    errs = []
    for N in (16, 32, 64, 128):
        d = W.Detector(kind=W.DET_BARE_CYLINDER, D=(H, R, 0, 0, 0, 0, 0), n_theta=N)
        errs.append(abs(det(orc, d).volume(0) - math.pi * R * R * H))
    for a, b in zip(errs[:-1], errs[1:]):
        assert a / b == pytest.approx(4.0, rel=0.02)


def test_coax_solids(orc):
    d = W.COAX_P
    m = det(orc, d)
    assert m.n_solid == 7
    N, nphi = d.n_theta, d.n_phi
    ext, D = d.d, d.D
    zf = -(ext[1] + ext[4])
    zb = zf - D[0]
    sep = d.sep_delta
    profiles = {
        0: [(0, 0.0), (ext[0], 0.0), (ext[0], -ext[6]), (0, -ext[6])],
        1: [(0, -ext[1]), (ext[0] - ext[2], -ext[1]), (ext[0] - ext[2], -ext[6] + ext[8]),
            (0, -ext[6] + ext[8])],
        2: [(0, -ext[7] + ext[9]), (D[1] + ext[5], -ext[7] + ext[9]), (D[1] + ext[5], zf - 10.0),
            (D[1] + ext[5] + ext[3], zf - 10.0), (D[1] + ext[5] + ext[3], -ext[7]), (0, -ext[7])],
        3: rounded_profile(D[1], D[2], zf, zb, nphi),
        4: rounded_profile(D[1] - D[3], D[2] - D[3], zf - D[3], zb + sep, nphi),
        5: rounded_profile(D[5] + D[6], D[5] + D[6], zb + D[4] + D[6], zb + 2 * sep, nphi),
        6: rounded_profile(D[5], D[5], zb + D[4], zb + 3 * sep, nphi),
    }
    for s, prof in profiles.items():
        assert m.euler(s) == 2, s
        assert m.open_edges(s) == 0, s
        v = m.volume(s)
        assert v > 0, s
        assert v == pytest.approx(faceted_volume(prof, N), rel=1e-10), s
    # smooth-body limits: crystal volume vs the Pappus volume of the rounded profile
    R, rch, L = D[1], D[2], D[0]
    smooth = math.pi * R * R * L - (1 - math.pi / 4) * rch * rch * 2 * math.pi * (R - rch * (
        (10 - 3 * math.pi) / (12 - 3 * math.pi)))
    assert m.volume(3) == pytest.approx(smooth, rel=2e-3)
    # triangle budget of the revolved profiles, flat end faces as concentric rings
    assert m.n_tri == sum(profile_tris(prof, N) for prof in profiles.values())
    # each flat end face is the plane N-gon: its triangles cover exactly its area,
    # and its inner vertices sit on the rings of the stated rule
    xyz, tri, ts, solids = m.arrays()
    v = xyz[tri]
    area = 0.5 * np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    for s, prof in profiles.items():
        for (ra, za), (rb, zb) in zip(prof[:-1], prof[1:]):
            if (ra > 0) == (rb > 0) or za != zb:
                continue
            Rf = max(ra, rb)
            face = (ts == s) & np.all(np.abs(v[:, :, 2] - za) < 1e-9, axis=1)
            assert np.abs(area[face, 2]).sum() == pytest.approx(0.5 * N * Rf * Rf * math.sin(2 * math.pi / N),
                                                                rel=1e-10), (s, za)
            fv = xyz[np.unique(tri[face])]
            rad = np.hypot(fv[:, 0], fv[:, 1])
            for r, mcount in disk_rings(Rf, N):
                assert np.sum(np.abs(rad - r) < 1e-9) == mcount, (s, za, r)
            # no sliver: every triangle's box is within a small multiple of its area
            box = np.ptp(v[face][:, :, 0], axis=1) * np.ptp(v[face][:, :, 1], axis=1)
            if disk_rings(Rf, N):
                assert np.max(box / np.abs(area[face, 2])) < 40, (s, za)
    xyz, tri, ts, solids = m.arrays()
    assert list(solids["parent"]) == [-1, 0, 1, 1, 3, 4, 5]
    assert list(solids["material"]) == [W.MAT_AL, W.MAT_VACUUM, W.MAT_CU, W.MAT_GE, W.MAT_GE,
                                        W.MAT_GE, W.MAT_VACUUM]
    assert list(solids["active"]) == [0, 0, 0, 0, 1, 0, 0]
    # rounding vertices obey rho_j, z_j of Sec. 2.2.2 (crystal solid, j = 0..Nphi)
    cx = xyz[np.unique(tri[ts == 3])]
    for j in range(nphi + 1):
        phi = 0.5 * math.pi * j / nphi
        rho = (R - rch) + rch * math.cos(phi)
        z = zf - rch * (1 - math.sin(phi))
        # the outermost ring at height z_j (the front face's inner rings share z_N_phi)
        at = np.isclose(cx[:, 2], z, atol=1e-12)
        rad = np.hypot(cx[at, 0], cx[at, 1])
        sel = rad > rad.max() - 1e-9
        assert sel.sum() == N
        assert np.allclose(rad[sel], rho, atol=1e-12)


def test_parity_rule_locates_known_points(orc):
    m = det(orc, W.COAX_P)
    D = W.COAX_D_INT
    zf = -6.0
    zb = zf - D[0]
    cases = [
        ((0, 0, 10.0), -1),                 # above the endcap
        ((0, 0, -0.5), 0),                  # in the Al window
        ((0, 0, -3.0), 1),                  # vacuum gap
        ((0, 0, zf - 0.3), 3),              # front dead layer
        ((10.0, 0, -30.0), 4),              # active Ge
        ((0, 0, zb + 10.0), 6),             # bore vacuum
        ((5.00015, 0, zb + 20.0), 5),       # inside the 0.3 um bore contact
        ((31.4, 0, -50.0), 2),              # Cu holder wall
        ((37.5, 0, -60.0), 0),              # endcap side wall
        ((50.0, 0, -60.0), -1),
    ]
    dirs = [(0, 0, 1), (0.3, -0.5, 0.81), (-1, 0, 0), (0.1, 0.99, -0.05)]
    for p, want in cases:
        for dd in dirs:
            n = np.array(dd, dtype=float)
            n /= np.linalg.norm(n)
            assert m.locate(p, n) == want, (p, dd)


def test_bare_with_source_prism(orc):
    m = det(orc, W.BATCH_DET)
    assert m.n_solid == 2
    N = W.BATCH_DET.src_n_sides
    assert m.volume(1) == pytest.approx(N / 2 * 35.0 ** 2 * math.sin(2 * math.pi / N) * 40.0, rel=1e-12)
    assert m.euler(1) == 2 and m.open_edges(1) == 0
    assert m.locate((0, 0, 25.0), (0, 0, 1)) == 1
    assert m.locate((0, 0, -5.0), (1, 0, 0)) == 0


def test_box_mesh_input_generator(orc):
    xyz, tri, ts = W.box_mesh([(-1, -2, -3, 1, 2, 3)])
    m = orc.Mesh.from_arrays(xyz, tri, ts, [1], [1], [0], [-1])
    assert m.volume(0) == pytest.approx(48.0, rel=1e-14)
    assert m.euler(0) == 2 and m.open_edges(0) == 0


def groove_profile(R, rch, zf, zb, n_phi, g_in, g_out, depth):
    """rounded_profile with the back-face channel g_in < rho < g_out, depth deep."""
    pts = rounded_profile(R, rch, zf, zb, n_phi)[:-1]
    return pts + [(g_out, zb), (g_out, zb + depth), (g_in, zb + depth), (g_in, zb), (0.0, zb)]


@pytest.mark.parametrize("name", ["STRESS_SMALL", "STRESS_DET"])
def test_stress_groove_and_flange(orc, name):
    """The stress features against closed forms: the grooved crystal and active
    volume are revolved profiles (exact faceted volumes), the flange ring is an
    extruded polygon with holes -- volume h x (N-gon annulus - holes x M-gon),
    genus 17 (the ring's opening plus 16 bolt holes) so chi = 2 - 2 * 17 = -32."""
    d = getattr(W, name)
    m = det(orc, d)
    assert m.n_solid == 9
    N, nphi = d.n_theta, d.n_phi
    D, sep = d.D, d.sep_delta
    zf = -(d.d[1] + d.d[4])
    zb = zf - D[0]
    gi, go = d.groove_r - d.groove_w / 2, d.groove_r + d.groove_w / 2
    crystal = groove_profile(D[1], D[2], zf, zb, nphi, gi, go, d.groove_d)
    active = groove_profile(D[1] - D[3], D[2] - D[3], zf - D[3], zb + sep, nphi, gi - sep, go + sep, d.groove_d)
    # the z_slices side bands add vertices on straight segments only (no volume change)
    assert m.volume(3) == pytest.approx(faceted_volume(crystal, N), rel=1e-10)
    assert m.volume(4) == pytest.approx(faceted_volume(active, N), rel=1e-10)
    c = 0.5 * N * math.sin(2 * math.pi / N)
    assert m.volume(3) == pytest.approx(faceted_volume(rounded_profile(D[1], D[2], zf, zb, nphi), N)
                                        - d.groove_d * c * (go * go - gi * gi), rel=1e-10)
    M, nh = d.bolt_n_sides, d.n_bolt_holes
    ring = c * (d.flange_r_out ** 2 - d.flange_r_in ** 2)
    holes = nh * 0.5 * M * math.sin(2 * math.pi / M) * d.bolt_r ** 2
    f = W.STRESS_FLANGE_SOLID
    assert m.volume(f) == pytest.approx(d.flange_h * (ring - holes), rel=1e-10)
    assert m.euler(f) == 2 - 2 * (nh + 1) == -32
    for s in range(m.n_solid):
        assert m.open_edges(s) == 0, s
        if s != f:
            assert m.euler(s) == 2, s
    xyz, tri, ts, solids = m.arrays()
    assert solids["parent"][f] == 1 and solids["material"][f] == W.MAT_CU
    # the flange's top and bottom faces cover exactly the ring minus the holes
    area = 0.0
    for t in tri[ts == f]:
        a, b, cc = xyz[t[0]], xyz[t[1]], xyz[t[2]]
        n = np.cross(b - a, cc - a)
        if abs(n[2]) > 1e-9 * np.linalg.norm(n):
            area += 0.5 * abs(n[2])
    assert area == pytest.approx(2 * (ring - holes), rel=1e-10)
    # parity rule in the new features
    tc = 2 * math.pi * 0.5 / nh                      # hole 0 centre angle
    hx, hy = d.bolt_rc * math.cos(tc), d.bolt_rc * math.sin(tc)
    zmid = d.flange_z_top - d.flange_h / 2
    cases = [
        ((hx, hy, zmid), 1),                                           # inside a bolt hole
        ((d.flange_r_in + 0.2, 0.0, zmid), f),                         # flange material
        ((d.flange_r_out + 0.2, 0.0, zmid), 1),                        # beyond the flange
        ((d.groove_r, 0.0, zb + d.groove_d / 2), 1),                   # in the groove channel
        ((d.groove_r, 0.0, zb + d.groove_d + sep / 2), 3),             # dead layer over the groove
        ((d.groove_r, 0.0, zb + d.groove_d + 3 * sep), 4),             # active Ge above it
        ((gi - sep / 2, 0.0, zb + d.groove_d / 2), 3),                 # dead wall of the groove
    ]
    dirs = [(0, 0, 1), (0.3, -0.5, 0.81), (-1, 0, 0.02), (0.1, 0.99, -0.05)]
    for p, want in cases:
        for dd in dirs:
            n = np.array(dd, dtype=float)
            n /= np.linalg.norm(n)
            assert m.locate(p, n) == want, (p, dd)


def test_detector2_triangle_counts_in_the_paper_range(orc):
    """Sec. 3.3 prints the triangle count of detector #2 at two mesh densities:
    4416 at (N_theta, N_phi) = (32, 10) and 13440 at (64, 20).  The paper does not
    list the components behind them, so they bound a sanity range, not an exact
    value: ours (endcap, holder cup, crystal, active volume, bore contact and
    bore vacuum, flat end faces as concentric rings at 64 segments) are within 30 %
    of both and grow by a similar factor."""
    import dataclasses
    counts = []
    for (nt, nphi), paper in (((32, 10), 4416), ((64, 20), 13440)):
        m = det(orc, dataclasses.replace(W.DET2, n_theta=nt, n_phi=nphi))
        counts.append(m.n_tri)
        assert 0.7 * paper <= m.n_tri <= 1.3 * paper, (nt, nphi, m.n_tri, paper)
    assert counts == [3456, 12968]
    assert 0.7 * 13440 / 4416 <= counts[1] / counts[0] <= 1.3 * 13440 / 4416


def _prism_clip(o, d, N, R, z_lo, z_hi):
    """Cyrus-Beck clipping of the line o + t d against the regular N-gon prism
    (vertex i at angle 2 pi i / N, radius R) between z_lo and z_hi: (t_in, t_out)."""
    apo = R * math.cos(math.pi / N)
    planes = [(np.array([math.cos(2 * math.pi * (i + 0.5) / N), math.sin(2 * math.pi * (i + 0.5) / N), 0.0]), apo)
              for i in range(N)]
    planes += [(np.array([0.0, 0.0, 1.0]), z_hi), (np.array([0.0, 0.0, -1.0]), -z_lo)]
    t_in, t_out = -math.inf, math.inf
    for n, off in planes:
        dn, num = n @ d, off - n @ o
        if dn == 0.0:
            if num < 0:
                return math.inf, -math.inf
            continue
        t = num / dn
        if dn < 0:
            t_in = max(t_in, t)
        else:
            t_out = min(t_out, t)
    return t_in, t_out


def test_nearest_hit_against_prism_clipping(orc):
    """The FP64 brute-force nearest hit (the reference of the GPU distance tests)
    against the closed-form clipping of rays by the convex 48-gon prism of the
    bare cylinder: from outside the first hit enters at t_in, from inside it
    leaves at t_out; with t_min past t_in the next hit is the exit; the
    excluded triangle is skipped."""
    m = det(orc, W.BARE_CYLINDER)
    N, R, L = 48, 30.0, 60.0
    rng = np.random.default_rng(3)
    n_in = n_out = 0
    for _ in range(1500):
        if rng.random() < 0.5:                       # outside, aimed at a point inside
            u = rng.normal(size=3)
            o = np.array([0.0, 0.0, -30.0]) + 120.0 * u / np.linalg.norm(u)
            tgt = np.array([*(rng.uniform(-20, 20, 2)), rng.uniform(-55, -5)])
            d = (tgt - o) / np.linalg.norm(tgt - o)
        else:                                        # inside, any direction
            o = np.array([*(rng.uniform(-20, 20, 2)), rng.uniform(-55, -5)])
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
        t_in, t_out = _prism_clip(o, d, N, R, -L, 0.0)
        k, t, ent = m.nearest_hit(tuple(o), tuple(d), 0.0, -1)
        if t_in > 0:
            n_out += 1
            assert k >= 0 and ent == 1 and t == pytest.approx(t_in, rel=1e-12, abs=1e-12)
            k2, t2, ent2 = m.nearest_hit(tuple(o), tuple(d), t_in + 1e-6, -1)
            assert ent2 == 0 and t2 == pytest.approx(t_out, rel=1e-12, abs=1e-12)
            k3, t3, _ = m.nearest_hit(tuple(o), tuple(d), 0.0, k)
            assert k3 != k and t3 >= t - 1e-9
        else:
            n_in += 1
            assert k >= 0 and ent == 0 and t == pytest.approx(t_out, rel=1e-12, abs=1e-12)
    assert n_in > 500 and n_out > 500


def test_open_edges_detects_holes_and_flips(orc):
    """The closedness check is not vacuous: a box with one triangle removed has
    its three edges unmatched; a box with one triangle flipped has directed
    edges that repeat instead of reversing."""
    xyz, tri, ts = W.box_mesh([(-1, -2, -3, 1, 2, 3)])
    holed = orc.Mesh.from_arrays(xyz, tri[1:], ts[1:], [1], [1], [0], [-1])
    assert holed.open_edges(0) == 3
    flipped_tri = tri.copy()
    flipped_tri[0] = flipped_tri[0][::-1]
    flipped = orc.Mesh.from_arrays(xyz, flipped_tri, ts, [1], [1], [0], [-1])
    assert flipped.open_edges(0) > 0
