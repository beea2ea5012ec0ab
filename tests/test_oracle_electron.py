"""Pins of the oracle's charged-particle model (continuous slowing down, the
stand-in for the paper's electron transport, Sec. 2.4.1 physics list).

* Stopping power and CSDA range of water against the published NIST ESTAR
  values (tests/golden/estar_water_electrons.txt).  The model leaves out the
  density-effect correction, which lowers the collision stopping power by about
  1 % at 1 MeV in water, so there it must sit above ESTAR by at most 2 %.
* The tabulated range and its inversion against a brute-force integration of
  dT/ds = -rho S(T) (Runge-Kutta, fine steps) and a trapezoid quadrature of
  1/S over a fine grid: checks the table, its interpolation and the bisection
  independently of how the table was built.
* Track geometry against closed forms on meshes whose distances are known: a
  track leaving the bare cylinder through its top face, one stopping inside,
  one crossing from the active coax volume into its dead layer, density scale,
  the weight of the pair, and the cut below which nothing is tracked.
* Transport invariants: energy conservation per history, identical photon
  histories in both models.
"""
import math
import os

import numpy as np
import pytest

from paper_2605_25963_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "estar_water_electrons.txt")
WATER, GE = 4, 1          # material codes (slots of W.MATERIAL_CODES)
RHO_GE = 5.323


@pytest.fixture(scope="module")
def tab(orc):
    assert tuple(W.MATERIAL_CODES) == (0, 1, 2, 3, 4)
    return orc.Tables.build(W.MATERIAL_CODES)


def estar():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return [(float(a) * 1e3, float(b), float(c)) for a, b, c in rows]


def test_water_stopping_power_and_range_match_estar(orc, tab):
    for T, s_col, r_csda in estar():
        col, tot = orc.e_stopping(WATER, T)
        if T < 500.0:
            assert col == pytest.approx(s_col, rel=0.005), (T, col)
        else:
            assert 1.0 <= col / s_col <= 1.02, (T, col)      # no density effect
        assert tot > col
        r = tab.e_range(WATER, T) / 10.0                     # mm -> g/cm^2 at rho = 1
        assert r == pytest.approx(r_csda, rel=0.03 if T < 50.0 else 0.015), (T, r)


def test_stopping_power_shape(orc):
    # falls with energy up to ~1 MeV, the radiative share grows like Z T
    s = [orc.e_stopping(GE, T)[0] for T in (2.0, 10.0, 100.0, 500.0)]
    assert all(a > b for a, b in zip(s, s[1:]))
    c, t = orc.e_stopping(GE, 2000.0)
    assert (t - c) / c == pytest.approx(32 * 2.0 / 800.0, rel=1e-12)
    c, t = orc.e_stopping(0, 100.0)
    assert c == 0.0 and t == 0.0
    with pytest.raises(ValueError):
        orc.e_stopping(99, 100.0)


def _rk4_energy_after(orc, code, rho, T, L, n=20000):
    """T after L mm by integrating dT/ds = -100 rho S_tot(T) keV/mm."""
    h = L / n

    def f(x):
        return -100.0 * rho * orc.e_stopping(code, max(x, 1e-9))[1]

    for _ in range(n):
        k1 = f(T); k2 = f(T + 0.5 * h * k1); k3 = f(T + 0.5 * h * k2); k4 = f(T + h * k3)
        T += h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return T


def test_range_table_and_inversion_against_brute_force(orc, tab):
    for T0, L in ((1000.0, 0.5), (300.0, 0.12), (50.0, 0.004)):
        want = _rk4_energy_after(orc, GE, RHO_GE, T0, L)
        got = tab.e_energy_after(GE, T0, L)
        assert got == pytest.approx(want, rel=2e-5, abs=1e-3), (T0, L, got, want)
    # range = T_min / S(T_min) + integral of dT / S, trapezoid on a fine grid in T
    for T0 in (20.0, 662.0, 2500.0):
        x = np.linspace(orc.E_TMIN, T0, 200001)
        y = np.array([1.0 / orc.e_stopping(GE, v)[1] for v in x[::100]])
        xs = x[::100]
        integral = np.sum(0.5 * (y[1:] + y[:-1]) * np.diff(xs)) * 1e-3          # g/cm^2
        r0 = orc.E_TMIN * 1e-3 / orc.e_stopping(GE, orc.E_TMIN)[1]
        want = 10.0 * (r0 + integral) / RHO_GE
        assert tab.e_range(GE, T0) == pytest.approx(want, rel=2e-5), T0
    # monotone, exhausted range, vacuum
    assert tab.e_energy_after(GE, 500.0, 10.0) == 0.0
    assert tab.e_energy_after(0, 500.0, 10.0) == 500.0
    assert math.isinf(tab.e_range(0, 500.0))
    Ts = [tab.e_energy_after(GE, 800.0, L) for L in np.linspace(0.0, 1.0, 11)]
    assert all(a > b for a, b in zip(Ts, Ts[1:])) and Ts[0] == pytest.approx(800.0, rel=1e-12)


@pytest.fixture(scope="module")
def bare(orc):
    return orc.Mesh.build(orc.Det(**W.BARE_CYLINDER.as_dict()))


@pytest.fixture(scope="module")
def coax(orc):
    return orc.Mesh.build(orc.Det(**W.COAX_P.as_dict()))


def test_track_leaving_through_the_top_face(orc, tab, bare):
    # bare Ge cylinder z in [-60, 0], world (vacuum) above: 0.3 mm of Ge, then out
    T, d = 1000.0, 0.3
    act, allp, esc = orc.e_track(bare, tab, (0.1, 0.2, -d), (0.0, 0.0, 1.0), T, 0)
    left = tab.e_energy_after(GE, T, d)
    assert act == pytest.approx(T - left, rel=1e-9) and allp == pytest.approx(act, rel=1e-12)
    assert esc == pytest.approx(left, rel=1e-9) and act + esc == pytest.approx(T, rel=1e-12)
    # downward it stops long before the bottom face
    act, allp, esc = orc.e_track(bare, tab, (0.1, 0.2, -d), (0.0, 0.0, -1.0), T, 0)
    assert act == T and esc == 0.0
    # density scale 1.5 of the crystal's group (2): the same path costs 1.5 x the range
    act, _, esc = orc.e_track(bare, tab, (0.1, 0.2, -d), (0.0, 0.0, 1.0), T, 0, group_scale=(1.0, 1.0, 1.5))
    assert esc == pytest.approx(tab.e_energy_after(GE, T, 1.5 * d), rel=1e-9)
    # two identical particles on one line (pair production)
    a2, p2, e2 = orc.e_track(bare, tab, (0.1, 0.2, -d), (0.0, 0.0, 1.0), T, 0, weight=2.0)
    assert a2 == pytest.approx(2 * (T - left), rel=1e-9) and e2 == pytest.approx(2 * left, rel=1e-9)
    # below the tracking cut: deposited where it is, in the given region
    a, p, e = orc.e_track(bare, tab, (0.1, 0.2, -d), (0.0, 0.0, 1.0), 0.5 * orc.E_TMIN, 0)
    assert a == p == 0.5 * orc.E_TMIN and e == 0.0
    a, p, e = orc.e_track(bare, tab, (0.1, 0.2, 5.0), (0.0, 0.0, 1.0), 0.5 * orc.E_TMIN, -1)
    assert a == 0.0 and p == 0.5 * orc.E_TMIN


def test_track_from_active_volume_into_dead_layer(orc, tab, coax):
    # coax active Ge: 128-gon of vertex radius 29.8 (the 0.7 mm dead layer outside it)
    # at mid-height; the side facet between the vertices at angles 0 and a = 2 pi / 128,
    # hit along the direction phi, lies at R cos(a/2) / cos(phi - a/2)
    a = 2.0 * math.pi / 128
    phi = 0.3 * a
    u = (math.cos(phi), math.sin(phi), 0.0)
    r0, z = 29.5, -37.0
    d_active = 29.8 * math.cos(a / 2) / math.cos(phi - a / 2) - r0
    T = 1500.0
    act, allp, esc = orc.e_track(coax, tab, (r0 * u[0], r0 * u[1], z), u, T, 4)
    assert act == pytest.approx(T - tab.e_energy_after(GE, T, d_active), rel=1e-7)
    assert allp > act + 1.0            # the dead layer (inactive Ge) takes the next 0.7 mm
    assert allp + esc == pytest.approx(T, rel=1e-12)


def test_transport_invariants_with_tracks(orc, tab, coax):
    src = orc.Source(kind=W.COAX_POINT_25.kind, pos=W.COAX_POINT_25.pos, dir=W.COAX_POINT_25.dir)
    for E in (122.0, 1332.0):
        r0 = orc.transport(coax, tab, src, E, 20000, want_edep=True)
        r1 = orc.transport(coax, tab, src, E, 20000, want_edep=True, e_model=1)
        assert r1.tally["n_err"] == 0 and r1.tally["max_rel_energy_err"] < 1e-12
        # the tracks draw no random numbers: the photon histories are the same
        for k in ("n_segments", "n_interactions", "n_crossings", "n_first_pe", "n_first_compton", "n_first_pair"):
            assert r0.tally[k] == r1.tally[k], k
        # a history whose deposits all stay put is scored the same in both models
        same = np.isclose(r0.edep, r1.edep, rtol=0, atol=1e-9)
        assert 0.9 < same.mean() < 1.0
        # the pair can only appear above threshold; tracks move energy between regions
        assert r1.tally["sum_dep_all"] + r1.tally["sum_esc"] == pytest.approx(20000 * E, rel=1e-12)
    with pytest.raises(ValueError):
        orc.transport(coax, orc.Tables.from_array(tab.array()), src, 662.0, 10, e_model=1)


def test_compton_electron_direction_in_a_thin_slab(orc):
    """The recoil electron of a Compton scattering runs along E d - E' d'
    (momentum conservation), at cos(phi_e) = (E - E' c) / |E d - E' d'| to the
    photon: a pencil beam along +z enters a 0.3 mm active Ge slab whose photon
    table is Compton-only just at E (so the photon scatters once and leaves);
    the electron of T = E - E' born at depth z0 runs forward and, if its range
    allows, leaves through the top face after L = (h - z0) / cos(phi_e) with
    T'(T, L) (the range functions pinned above).  The mean active deposit per
    scattering matches the Klein-Nishina quadrature over cos(theta) and depth."""
    E, h, mu_c = 662.0, 0.3, 0.05
    k = E / 510.99895
    n_grid = 200_000
    t = orc.Tables.build(W.MATERIAL_CODES, n_grid)
    Eg = np.exp(np.linspace(math.log(10.0), math.log(3000.0), n_grid))
    j = int(np.searchsorted(Eg, E)) - 1
    mu = np.zeros((len(W.MATERIAL_CODES), 3, n_grid), np.float32)
    mu[GE, 1, j:] = mu_c
    t.set_mu(mu)
    xyz, tri, ts = W.box_mesh([(-50, -50, 0.0, 50, 50, h)])
    m = orc.Mesh.from_arrays(xyz, tri, ts, [GE], [1], [-1], [-1])
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, -1.0), dir=(0, 0, 1.0))
    r = orc.transport(m, t, src, E, 2_000_000, want_edep=True, e_model=1)
    T_ = r.tally
    assert T_["n_err"] == 0 and T_["n_first_pe"] == 0
    dep = r.edep[r.edep > 0]
    assert len(dep) == T_["n_first_compton"] > 20_000
    # quadrature: midpoints in cos(theta) (Klein-Nishina weight) and depth (exp(-mu z0))
    nc, nz = 1000, 40
    c = -1 + (np.arange(nc) + 0.5) * 2 / nc
    P = 1 / (1 + k * (1 - c))
    w = P * P * (P + 1 / P - (1 - c * c))
    Ep = E * P
    Te = E - Ep
    cos_e = (E - Ep * c) / np.sqrt(E * E + Ep * Ep - 2 * E * Ep * c)
    z0 = (np.arange(nz) + 0.5) * h / nz
    wz = np.exp(-mu_c * z0)
    mean_c = np.empty(nc)
    for i in range(nc):
        if Te[i] < orc.E_TMIN:
            mean_c[i] = Te[i]
            continue
        d_i = [Te[i] - t.e_energy_after(GE, Te[i], (h - z) / cos_e[i]) for z in z0]
        mean_c[i] = np.dot(wz, d_i) / wz.sum()
    expect = np.dot(w, mean_c) / w.sum()
    assert abs(dep.mean() - expect) < 4 * dep.std() / math.sqrt(len(dep)) + 1e-4 * expect, (dep.mean(), expect)
    assert 0.2 * (E - E / (1 + k)) < expect < E - E / (1 + 2 * k)    # a real fraction escapes
