"""Pins of the oracle's transport against closed forms (CPU only).

  * narrow-beam slab transmission: P(E_dep > 0) = 1 - exp(-mu_tot x), and
    across two density-scaled slabs;
  * black absorber: FEPE = (solid angle of the meshed top face) / 4 pi, from
    the Van Oosterom-Strackee formula summed over the fan triangles;
  * Kahn sampler: chi-square against bin integrals of the Klein-Nishina
    angular distribution;
  * first-interaction process frequencies = mu_i / mu_tot;
  * Compton angle in transport: backscatter fraction and energies against
    the textbook Klein-Nishina formula;
  * pair production: deposit E - 2 mc^2 and two 511 keV photons;
  * energy conservation per history, parity rule == nesting-tree rule;
  * density-perturbation gradient: the slab identity dFEPE/ds = -mu x FEPE
    and central finite differences with common random numbers;
  * source sampling moments.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2605_25963_gb300 import workloads as W

MEC2 = 510.99895


def zsig(a, b, sa, sb):
    return abs(a - b) / math.sqrt(sa * sa + sb * sb)


def slab_mesh(orc, boxes, materials, active, groups=None):
    xyz, tri, ts = W.box_mesh(boxes)
    n = len(boxes)
    groups = groups if groups is not None else [-1] * n
    return orc.Mesh.from_arrays(xyz, tri, ts, materials, active, groups, [-1] * n)


def test_slab_transmission(orc):
    """Pencil beam normal to an active Ge slab of 0.5, 0.7 or 1 mean free path:
    P(E_dep > 0) = 1 - exp(-mu_tot x) exactly; 1e7 histories, within 3 sigma."""
    t = orc.Tables.build(W.MATERIAL_CODES)
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, 10.0), dir=(0, 0, -1.0))
    for E, n_mfp in ((59.5, 0.5), (662.0, 0.7), (1332.0, 1.0)):
        mu = sum(t.eval(W.MAT_GE, E))
        x = n_mfp / mu
        m = slab_mesh(orc, [(-1e3, -1e3, -x, 1e3, 1e3, 0.0)], [W.MAT_GE], [1])
        N = 10_000_000
        r = orc.transport(m, t, src, E, N)
        p_int = 1 - r.tally["n_zero"] / N
        expect = 1 - math.exp(-mu * x)
        sig = math.sqrt(expect * (1 - expect) / N)
        assert abs(p_int - expect) < 3 * sig, (E, p_int, expect)
        assert r.tally["n_err"] == 0


@pytest.mark.parametrize("s1,s2", [(1.0, 1.0), (1.7, 1.0), (0.4, 2.5)])
def test_density_scaled_two_slab_transmission(orc, s1, s2):
    """Free flight across a boundary with density scales (Sec. 2.4.1 free
    flight; the scales of the gradient's density groups): photoabsorption-only
    slabs, the first inactive (group 0, scale s1, thickness x1), the second
    active (group 1, scale s2, thickness x2).  A photon deposits exactly when it
    crosses the first slab and is absorbed in the second:
    P = exp(-s1 mu1 x1) (1 - exp(-s2 mu2 x2))."""
    x1, x2, mu1, mu2 = 3.0, 2.0, 0.2, 0.35
    mu = np.zeros((3, 3, 1000), np.float32)
    mu[1, 0, :] = mu1
    mu[2, 0, :] = mu2
    t = orc.Tables.from_array(mu)
    m = slab_mesh(orc, [(-50, -50, -x1, 50, 50, 0.0), (-50, -50, -x1 - 1.0 - x2, 50, 50, -x1 - 1.0)],
                  [1, 2], [0, 1], groups=[0, 1])
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, 5.0), dir=(0, 0, -1.0))
    N = 400_000
    r = orc.transport(m, t, src, 662.0, N, group_scale=(s1, s2))
    p = 1 - r.tally["n_zero"] / N
    expect = math.exp(-s1 * mu1 * x1) * (1 - math.exp(-s2 * mu2 * x2))
    assert abs(p - expect) < 4 * math.sqrt(expect * (1 - expect) / N), (p, expect)
    assert r.tally["n_first_pe"] == N - r.tally["n_first_none"]


def vos_solid_angle(obs, tri_pts):
    """Van Oosterom & Strackee (1983): solid angle of a triangle seen from obs."""
    a, b, c = (np.asarray(p, float) - obs for p in tri_pts)
    la, lb, lc = (np.linalg.norm(v) for v in (a, b, c))
    num = abs(np.dot(a, np.cross(b, c)))
    den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
    return 2 * math.atan2(num, den)


def test_black_absorber_solid_angle(orc):
    m = orc.Mesh.build(orc.Det(**W.BARE_CYLINDER.as_dict()))
    mu = np.zeros((2, 3, 1000), np.float32)
    mu[1, 0, :] = 1e6                      # photoabsorption only, mean free path 1 nm
    t = orc.Tables.from_array(mu)
    src = orc.Source(kind=W.SRC_POINT, pos=(0, 0, 100.0))
    N = 10_000_000
    r = orc.transport(m, t, src, 662.0, N)
    xyz, tri, ts, _ = m.arrays()
    top = [f for f in tri if np.allclose(xyz[f][:, 2], 0.0)]
    assert len(top) == 48
    omega = sum(vos_solid_angle(np.array([0, 0, 100.0]), xyz[f]) for f in top)
    expect = omega / (4 * math.pi)
    disk = (1 - 100 / math.hypot(100, 30)) / 2
    assert expect == pytest.approx(disk, rel=3e-3)       # polygon -> disk at O(N^-2)
    sig = math.sqrt(expect * (1 - expect) / N)
    assert abs(r.fepe - expect) < 3 * sig
    assert r.tally["n_fep"] + r.tally["n_zero"] == N


@pytest.mark.parametrize("E", [59.5, 662.0, 1332.0, 2900.0])
def test_kahn_sampler_klein_nishina(orc, E):
    """1e7 samples of cos(theta) per energy against the bin integrals of the
    Klein-Nishina distribution; the four energies form one family of tests, so
    each must reach p > 0.01 / 4 (Bonferroni)."""
    k = E / MEC2
    n = 10_000_000
    x = orc.kahn_samples(k, n, seed=5)
    assert np.all(x >= 1.0) and np.all(x <= 1 + 2 * k + 1e-12)
    c = 1 - (x - 1) / k
    edges = np.linspace(-1, 1, 41)
    obs, _ = np.histogram(c, bins=edges)
    tot = orc.sigma_kn(k)
    p = np.array([integrate.quad(lambda cc: orc.dsigma_kn_dcos(k, cc), a, b, epsabs=0, epsrel=1e-12)[0] / tot
                  for a, b in zip(edges[:-1], edges[1:])])
    assert p.sum() == pytest.approx(1.0, rel=1e-9)
    chi = stats.chisquare(obs, p * n)
    assert chi.pvalue > 0.01 / 4, chi


def test_first_interaction_frequencies(orc):
    E = 1332.0
    m = slab_mesh(orc, [(-1e4, -1e4, -1e4, 1e4, 1e4, 0.0)], [W.MAT_GE], [1])
    t = orc.Tables.build(W.MATERIAL_CODES)
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, 1.0), dir=(0, 0, -1.0))
    N = 10_000_000
    r = orc.transport(m, t, src, E, N)
    mu = np.array(t.eval(W.MAT_GE, E))
    obs = [r.tally["n_first_pe"], r.tally["n_first_compton"], r.tally["n_first_pair"]]
    assert sum(obs) == N
    chi = stats.chisquare(obs, mu / mu.sum() * N)
    assert chi.pvalue > 0.01, (obs, mu / mu.sum() * N)


def kn_textbook(k, c):
    """Klein-Nishina dsigma/dOmega over r_e^2/2 (Klein & Nishina 1929), written
    here from the textbook: P^2 (P + 1/P - sin^2 theta), P = E'/E."""
    P = 1.0 / (1.0 + k * (1.0 - c))
    return P * P * (P + 1.0 / P - (1.0 - c * c))


@pytest.mark.parametrize("E,alpha", [(59.5, 0.0), (662.0, 0.0), (1332.0, 0.0), (59.5, 1.0), (662.0, 1.0)])
def test_compton_angle_backscatter_fraction(orc, E, alpha):
    """The scattering angle inside transport (not the sampler alone): a pencil
    beam at angle alpha to +z crosses a thin Compton-only slab z in [0, 0.1]
    whose cross section vanishes just below E (so every photon scatters once at
    most); a black, active catcher 10 m wide fills z < -2, behind the beam's
    origin.  A history deposits in the catcher exactly when its scattered
    photon heads to -z, with E' = E / (1 + k (1 - cos theta)) deposited.  For
    uniform azimuth the probability of heading to -z at polar cosine c about a
    beam at alpha is arccos(cot(alpha) c / sin(theta)) / pi (a step at c = 0
    for alpha = 0), so the deposit fraction is that weighted by Klein-Nishina
    over c; the tilted beam (with a y component) takes the general branch of
    the direction rotation.  Every deposit lies in [E/(1+2k), E]; for alpha = 0
    in [E/(1+2k), E/(1+k)] with the backward average of E' as mean."""
    k = E / MEC2
    # 200,000 log-spaced grid points: the slab's cross section is 0.02 / mm from
    # the grid point below E up and zero below the one before it, so only a
    # photon scattered by less than ~6e-5 in relative energy could scatter again
    n_grid = 200_000
    Eg = np.exp(np.linspace(math.log(10.0), math.log(3000.0), n_grid))
    j = int(np.searchsorted(Eg, E)) - 1
    mu = np.zeros((3, 3, n_grid), np.float32)
    mu[1, 1, j:] = 0.02                          # scatterer: Compton only, 0.1 mm -> 0.2 %
    mu[2, 0, :] = 1e3                            # catcher: photoabsorption, 1 um mean free path
    t = orc.Tables.from_array(mu)
    m = slab_mesh(orc, [(-50, -50, 0.0, 50, 50, 0.1), (-5e3, -5e3, -100.0, 5e3, 5e3, -2.0)],
                  [1, 2], [0, 1])
    beta = 0.7
    d = (math.sin(alpha) * math.cos(beta), math.sin(alpha) * math.sin(beta), math.cos(alpha))
    src = orc.Source(kind=W.SRC_PENCIL, pos=(-d[0] / d[2], -d[1] / d[2], -1.0), dir=d)
    N = 10_000_000
    r = orc.transport(m, t, src, E, N, want_edep=True)
    T = r.tally
    assert T["n_err"] == 0 and T["n_first_pe"] == 0 and T["n_first_pair"] == 0
    n_c = T["n_first_compton"]
    assert n_c > 10_000
    w = lambda c: kn_textbook(k, c)
    if alpha == 0.0:
        heads_down = lambda c: 1.0 if c < 0 else 0.0
    else:
        heads_down = lambda c: math.acos(min(1.0, max(-1.0, c / math.tan(alpha) /
                                                       math.sqrt(max(1e-300, 1 - c * c))))) / math.pi
    tot = integrate.quad(w, -1, 1)[0]
    down = integrate.quad(lambda c: w(c) * heads_down(c), -1, 1, points=[0.0], limit=200)[0]
    F = down / tot
    dep = r.edep[r.edep > 0]
    f = len(dep) / n_c
    assert abs(f - F) < 4 * math.sqrt(F * (1 - F) / n_c), (f, F)
    assert dep.min() >= E / (1 + 2 * k) * (1 - 1e-12) and dep.max() <= E * (1 + 1e-12)
    if alpha == 0.0:
        assert dep.max() <= E / (1 + k) * (1 + 1e-12)
        Ep = lambda c: E / (1 + k * (1 - c))
        mean = integrate.quad(lambda c: Ep(c) * w(c), -1, 0)[0] / down
        sd = math.sqrt(integrate.quad(lambda c: (Ep(c) - mean) ** 2 * w(c), -1, 0)[0] / down)
        assert abs(dep.mean() - mean) < 4 * sd / math.sqrt(len(dep)), (dep.mean(), mean)


def _box_hit_fraction(E, d, box, mu_s, slab_t, n_c=1000, n_phi=1000, n_depth=4):
    """Klein-Nishina-weighted fraction of single scatterings of a beam along d
    (through the origin; scattering points weighted exp(-mu_s s) along its path
    through the slab z in [0, slab_t]) whose ray hits the box, and the mean
    E' of those: midpoint quadrature over cos(theta), azimuth and depth, with
    the test's own frame and ray-box slab test."""
    k = E / MEC2
    d = np.asarray(d, float)
    e1 = np.cross(d, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    c = -1 + (np.arange(n_c) + 0.5) * 2 / n_c
    w = kn_textbook(k, c)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    sn = np.sqrt(1 - c * c)
    n = c[:, None, None] * d + sn[:, None, None] * (np.cos(phi)[None, :, None] * e1 +
                                                   np.sin(phi)[None, :, None] * e2)
    lo, hi = np.array(box[:3], float), np.array(box[3:], float)
    path = slab_t / d[2]
    hits = e_sum = total = 0.0
    for j in range(n_depth):
        sd = (j + 0.5) / n_depth * path
        wd = math.exp(-mu_s * sd)
        p = d * sd
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - p) / n, (hi - p) / n
        t_in = np.nanmax(np.minimum(t1, t2), axis=-1)
        t_out = np.nanmin(np.maximum(t1, t2), axis=-1)
        h = (w[:, None] * (t_out >= np.maximum(t_in, 0.0))).sum(axis=1)
        hits += wd * h.sum()
        e_sum += wd * (h * E / (1 + k * (1 - c))).sum()
        total += wd * w.sum() * n_phi
    return hits / total, e_sum / hits


def test_compton_direction_into_a_finite_catcher(orc):
    """The full scattered direction, not only its hemisphere: the tilted beam
    of the test above (alpha = 1, with a y component) scatters once in the thin
    slab, and a black, active 40 mm cube off the beam's plane, 30-70 mm below
    the slab, catches the photons whose rays meet it.  The fraction that
    deposits and their mean energy match the Klein-Nishina quadrature over
    the directions that hit the cube (about 2.5 % of the scatterings)."""
    E = 662.0
    n_grid = 200_000
    Eg = np.exp(np.linspace(math.log(10.0), math.log(3000.0), n_grid))
    j = int(np.searchsorted(Eg, E)) - 1
    mu = np.zeros((3, 3, n_grid), np.float32)
    mu[1, 1, j:] = 0.1
    mu[2, 0, :] = 1e3
    t = orc.Tables.from_array(mu)
    box = (-40.0, 20.0, -70.0, 0.0, 60.0, -30.0)
    m = slab_mesh(orc, [(-50, -50, 0.0, 50, 50, 0.1), box], [1, 2], [0, 1])
    alpha, beta = 1.0, 0.7
    d = (math.sin(alpha) * math.cos(beta), math.sin(alpha) * math.sin(beta), math.cos(alpha))
    src = orc.Source(kind=W.SRC_PENCIL, pos=(-d[0] / d[2], -d[1] / d[2], -1.0), dir=d)
    r = orc.transport(m, t, src, E, 10_000_000, want_edep=True)
    T = r.tally
    assert T["n_err"] == 0 and T["n_first_pe"] == 0
    n_c = T["n_first_compton"]
    F, mean = _box_hit_fraction(E, d, box, 0.1, 0.1)
    dep = r.edep[r.edep > 0]
    f = len(dep) / n_c
    assert abs(f - F) < 4 * math.sqrt(F * (1 - F) / n_c), (f, F)
    assert abs(dep.mean() - mean) < 4 * dep.std() / math.sqrt(len(dep)), (dep.mean(), mean)


def test_dos_gradient_interaction_term(orc):
    """The interaction part of the density-perturbation score: an active slab
    that only photoabsorbs (group 0, mu x = 0.6), so every interacting photon
    is in the full-energy peak and FEPE(s) = 1 - exp(-s mu x); hence
    dFEPE/ds = mu x exp(-s mu x), carried entirely by the score 1/s - mu d of
    the absorbing step."""
    x, mu0 = 2.0, 0.3
    mu = np.zeros((2, 3, 1000), np.float32)
    mu[1, 0, :] = mu0
    t = orc.Tables.from_array(mu)
    m = slab_mesh(orc, [(-50, -50, -x, 50, 50, 0.0)], [1], [1], groups=[0])
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, 5.0), dir=(0, 0, -1.0))
    for s_ in (1.0, 1.5):
        r = orc.transport(m, t, src, 662.0, 400_000, group_scale=(s_,))
        fe = 1 - math.exp(-s_ * mu0 * x)
        assert abs(r.fepe - fe) < 4 * math.sqrt(fe * (1 - fe) / 400_000)
        expect = mu0 * x * math.exp(-s_ * mu0 * x)
        assert abs(r.dfepe(0) - expect) < 4 * r.dfepe_sigma(0), (s_, r.dfepe(0), expect)


def test_pair_production_deposits(orc):
    """Pair-only above threshold, black absorber below 600 keV: every interacting
    1332 keV photon deposits E - 2 mc^2 and both 511 keV photons are absorbed."""
    m = slab_mesh(orc, [(-1e3, -1e3, -1e3, 1e3, 1e3, 0.0)], [W.MAT_GE], [1])
    mu = np.zeros((2, 3, 1000), np.float32)
    lnE = np.linspace(math.log(10), math.log(3000), 1000)
    E = np.exp(lnE)
    mu[1, 2, E > 1100] = 0.5
    mu[1, 0, E < 600] = 1e3
    t = orc.Tables.from_array(mu)
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, 1.0), dir=(0, 0, -1.0))
    r = orc.transport(m, t, src, 1332.0, 20_000, want_edep=True)
    assert r.tally["n_first_pair"] == 20_000
    # a 511 keV photon escapes only from pair events within ~1 um of the surface
    assert r.fepe > 0.999
    allowed = np.array([1332.0, 1332.0 - MEC2, 1332.0 - 2 * MEC2])
    assert np.all(np.min(np.abs(r.edep[:, None] - allowed[None, :]), axis=1) < 1e-9)
    assert r.tally["max_rel_energy_err"] < 1e-12
    # thin active layer: annihilation photons leave, deposit is exactly E - 2 mc^2
    m2 = slab_mesh(orc, [(-1e3, -1e3, -1e3, 1e3, 1e3, 0.0)], [W.MAT_GE], [1])
    mu2 = np.zeros((2, 3, 1000), np.float32)
    mu2[1, 2, E > 1100] = 0.5
    t2 = orc.Tables.from_array(mu2)
    r2 = orc.transport(m2, t2, src, 1332.0, 5_000, want_edep=True)
    assert np.allclose(r2.edep, 1332.0 - 2 * MEC2, rtol=0, atol=1e-9)
    assert r2.tally["sum_esc"] == pytest.approx(5_000 * 2 * MEC2, rel=1e-12)


def _peak_excess(spec, E, n_bins=4096, e_max=3000.0):
    """Counts in the bin of energy E above the mean of the bins 3-12 away on both
    sides, in units of that mean's Poisson sigma."""
    b = int(E * n_bins / e_max)
    side = np.r_[spec[b - 12:b - 2], spec[b + 3:b + 13]].astype(float)
    mu = side.mean()
    return (spec[b] - mu) / math.sqrt(max(mu, 1.0))


def test_escape_peaks_in_the_coax_spectrum(orc):
    """Pair production in the coax at 1332 keV leaves single- and double-escape
    peaks at E - 511 and E - 1022 keV in the pulse-height spectrum (one or both
    annihilation photons leave the crystal); at 662 keV, below the threshold,
    there is none at E - 511.  A pencil beam parallel to the axis at r = 15 mm
    (between the bore and the crystal's side) crosses the whole crystal length."""
    m = orc.Mesh.build(orc.Det(**W.COAX_P.as_dict()))
    t = orc.Tables.build(W.MATERIAL_CODES)
    src = orc.Source(kind=W.SRC_PENCIL, pos=(15.0, 0, 25.0), dir=(0, 0, -1.0))
    r = orc.transport(m, t, src, 1332.0, 300_000)
    assert r.tally["n_first_pair"] > 0 and r.tally["n_err"] == 0
    assert _peak_excess(r.spectrum, 1332.0 - MEC2) > 5
    assert _peak_excess(r.spectrum, 1332.0 - 2 * MEC2) > 5
    assert abs(_peak_excess(r.spectrum, 1000.0)) < 4              # no peak where none belongs
    r6 = orc.transport(m, t, src, 662.0, 100_000)
    assert r6.tally["n_first_pair"] == 0
    assert _peak_excess(r6.spectrum, 662.0 - MEC2) < 4


@pytest.mark.parametrize("E", [59.5, 1332.0])
def test_coax_energy_conservation_and_parity(orc, E):
    m = orc.Mesh.build(orc.Det(**W.GRAD_DET.as_dict()))
    t = orc.Tables.build(W.MATERIAL_CODES)
    for src in (orc.Source(kind=W.SRC_POINT, pos=(0, 0, 25.0)),
                orc.Source(kind=W.SRC_PRISM, pos=(0, 0, 0.01), radius=35.0, height=40.0, n_sides=128)):
        r = orc.transport(m, t, src, E, 3000)
        T = r.tally
        assert T["n_err"] == 0
        assert T["n_parity_mismatch"] == 0
        assert T["max_rel_energy_err"] < 1e-12
        assert T["n_crossings"] > 0 and T["n_interactions"] > 0


def test_source_moments(orc):
    N = 20000
    disk = orc.Source(kind=W.SRC_DISK, pos=(1.0, -2.0, 10.0), radius=30.0)
    P = np.array([orc.sample_birth(disk, 9, h)[0] for h in range(N)])
    r2 = (P[:, 0] - 1) ** 2 + (P[:, 1] + 2) ** 2
    assert r2.max() <= 900.0 and np.all(P[:, 2] == 10.0)
    assert r2.mean() == pytest.approx(450.0, rel=0.02)           # E[r^2] = R^2 / 2
    prism = orc.Source(kind=W.SRC_PRISM, pos=(0, 0, 1.0), radius=35.0, height=40.0, n_sides=8)
    P = np.array([orc.sample_birth(prism, 9, h)[0] for h in range(N)])
    assert P[:, 2].min() >= 1.0 and P[:, 2].max() <= 41.0
    assert P[:, 2].mean() == pytest.approx(21.0, abs=0.3)
    # inside the octagon: |(x,y) . n_k| <= apothem for every edge normal
    apo = 35.0 * math.cos(math.pi / 8)
    for kk in range(8):
        a = 2 * math.pi * (kk + 0.5) / 8
        assert np.all(P[:, 0] * math.cos(a) + P[:, 1] * math.sin(a) <= apo + 1e-9)
    # uniform in area: the fraction inside radius apo/2 equals its area fraction
    inner = np.mean(np.hypot(P[:, 0], P[:, 1]) < apo / 2)
    area_oct = 8 / 2 * 35.0 ** 2 * math.sin(2 * math.pi / 8)
    assert inner == pytest.approx(math.pi * (apo / 2) ** 2 / area_oct, abs=0.015)
    dirs = np.array([orc.sample_birth(disk, 9, h)[1] for h in range(N)])
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0)
    assert abs(dirs[:, 2].mean()) < 0.02 and dirs[:, 2].var() == pytest.approx(1 / 3, rel=0.03)


def test_point_and_pencil_sources(orc):
    """Point: birth at the point, directions uniform on the sphere -- every
    octant holds 1/8 of them and each Cartesian component has mean 0 and
    variance 1/3 (a half-range azimuth or a sign slip fails the octant count).
    Pencil: birth at its origin along its direction, exactly."""
    N = 40000
    pt = orc.Source(kind=W.SRC_POINT, pos=(3.0, -4.0, 25.0))
    B = [orc.sample_birth(pt, 5, h) for h in range(N)]
    P = np.array([b[0] for b in B])
    D = np.array([b[1] for b in B])
    assert np.all(P == np.array([3.0, -4.0, 25.0]))
    assert np.allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-12)
    for c in range(3):
        assert abs(D[:, c].mean()) < 0.015
        assert D[:, c].var() == pytest.approx(1 / 3, rel=0.03)
    octant = (D[:, 0] > 0) * 4 + (D[:, 1] > 0) * 2 + (D[:, 2] > 0)
    counts = np.bincount(octant, minlength=8)
    assert np.all(np.abs(counts - N / 8) < 5 * math.sqrt(N / 8 * 7 / 8))
    # transport draws from the pinned stream layout: a point source takes words
    # 0 and 1 of history (seed, hid, inst) as cos(theta) = 2 u - 1, phi = 2 pi u
    for seed, hid, inst in ((5, 0, 0), (0x1122334455667788, 0x0000000A00000003, 7), (1, 2 ** 40 + 5, 3)):
        w = orc.stream_words(seed, hid, inst, 2)
        d = orc.sample_birth(pt, seed, hid, inst)[1]
        assert d[2] == 2.0 * orc.u01(w[0]) - 1.0
        assert math.atan2(d[1], d[0]) % (2 * math.pi) == pytest.approx(2 * math.pi * orc.u01(w[1]), abs=1e-12)
    u = np.array([1.0, 2.0, -2.0]) / 3.0
    pen = orc.Source(kind=W.SRC_PENCIL, pos=(0.5, 0.25, -7.0), dir=tuple(u))
    for h in (0, 1, 77, 123456):
        p, d = orc.sample_birth(pen, 5, h)
        assert np.all(p == np.array([0.5, 0.25, -7.0]))
        assert np.allclose(d, u, rtol=0, atol=1e-15)


def test_dos_gradient_slab_identity(orc):
    """Al slab (group 0) in front of a Ge slab: FEPE(s) = exp(-s mu x) K,
    so dFEPE/ds = -mu x FEPE exactly (within 3 sigma, 2e6 histories).  Central
    finite differences (+-1 %, common random numbers: the same history ids at
    both scales), with their sigma from 100 batch means, agree with the
    density-perturbation estimate within 3 combined sigma."""
    x = 2.0
    m = slab_mesh(orc, [(-50, -50, -x, 50, 50, 0.0), (-50, -50, -40, 50, 50, -x - 1.0)],
                  [W.MAT_AL, W.MAT_GE], [0, 1], groups=[0, 1])
    t = orc.Tables.build(W.MATERIAL_CODES)
    src = orc.Source(kind=W.SRC_PENCIL, pos=(0, 0, 5.0), dir=(0, 0, -1.0))
    E, N = 122.0, 2_000_000
    r = orc.transport(m, t, src, E, N, group_scale=(1.0, 1.0))
    mu = sum(t.eval(W.MAT_AL, E))
    expect = -mu * x * r.fepe
    g, sg = r.dfepe(0), r.dfepe_sigma(0)
    assert abs(g - expect) < 3 * sg, (g, expect, sg)
    h, B = 0.01, 100
    n = N // B
    fd = []
    for b in range(B):
        fp = orc.transport(m, t, src, E, n, history_offset=b * n, group_scale=(1 + h, 1.0)).fepe
        fm = orc.transport(m, t, src, E, n, history_offset=b * n, group_scale=(1 - h, 1.0)).fepe
        fd.append((fp - fm) / (2 * h))
    fd = np.array(fd)
    s_fd = fd.std(ddof=1) / math.sqrt(B)
    assert abs(fd.mean() - g) < 3 * math.hypot(s_fd, sg), (fd.mean(), s_fd, g, sg)


def test_history_offset_partitions_exactly(orc):
    """Counter-based streams: two halves with history offsets add up to one run."""
    m = orc.Mesh.build(orc.Det(**W.BARE_CYLINDER.as_dict()))
    t = orc.Tables.build(W.MATERIAL_CODES)
    src = orc.Source(kind=W.SRC_POINT, pos=(0, 0, 100.0))
    full = orc.transport(m, t, src, 662.0, 20000)
    a = orc.transport(m, t, src, 662.0, 12000)
    b = orc.transport(m, t, src, 662.0, 8000, history_offset=12000)
    for k in ("n_fep", "n_zero", "n_over", "n_crossings", "n_interactions"):
        assert full.tally[k] == a.tally[k] + b.tally[k]
    assert np.array_equal(full.spectrum, a.spectrum + b.spectrum)


def test_oracle_struct_layouts_match_header(orc, tmp_path):
    """The oracle's ctypes mirrors have the sizes and offsets gcc gives oracle.h."""
    import ctypes as C
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    pairs = (("orc_detparams", orc.DetParams), ("orc_mesh", orc.MeshC), ("orc_tables", orc.TablesC),
             ("orc_source", orc.SourceC), ("orc_opts", orc.OptsC), ("orc_tally", orc.TallyC))
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "oracle.h"', "int main(void) {"]
    for name, cls in pairs:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.dirname(os.path.abspath(orc.__file__))
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in filter(None, subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")):
        name, key, val = line.split()
        got[(name, key)] = int(val)
    for name, cls in pairs:
        assert C.sizeof(cls) == got[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == got[(name, field)], (name, field)
