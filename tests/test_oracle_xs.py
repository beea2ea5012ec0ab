"""Pins of the oracle's closed-form cross sections and tables (CPU only).

Klein-Nishina: the closed-form total is checked against a numerical quadrature
of the differential formula, and the differential formula against the
Thomson limit.  Photoabsorption and pair production are synthetic model
definitions; they are pinned by their scaling laws and by one value each
computed here from the textbook form of each model with CODATA constants.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2605_25963_gb300 import workloads as W

# cross sections are ~1e-24 cm^2: every pytest.approx below sets abs=0, since its
# default absolute tolerance of 1e-12 would accept any such value

MEC2 = 510.99895
RE = 2.8179403262e-13
ALPHA = 1 / 137.035999084
NA = 6.02214076e23


@pytest.mark.parametrize("E", [10.0, 59.5, 122.0, 511.0, 662.0, 1332.0, 2900.0])
def test_kn_total_equals_integral_of_differential(orc, E):
    k = E / MEC2
    q, err = integrate.quad(lambda c: orc.dsigma_kn_dcos(k, c), -1.0, 1.0, epsabs=0, epsrel=1e-13,
                            limit=200)
    assert orc.sigma_kn(k) == pytest.approx(q, rel=1e-10, abs=0)


def test_kn_thomson_limit(orc):
    sigma_T = 8 * math.pi / 3 * RE ** 2
    # low-energy expansion (Heitler, The Quantum Theory of Radiation):
    # sigma / sigma_T = 1 - 2k + 26/5 k^2 - 133/10 k^3 + 1144/35 k^4 - ...; at k = 3e-3
    # the omitted terms are ~2e-11 and the closed form's FP64 cancellation ~1e-16 / k^3
    k = 3e-3
    series = 1 - 2 * k + 26 / 5 * k ** 2 - 133 / 10 * k ** 3 + 1144 / 35 * k ** 4
    assert orc.sigma_kn(k) == pytest.approx(sigma_T * series, rel=1e-9, abs=0)
    for c in (-1.0, -0.3, 0.0, 0.5, 1.0):
        assert orc.dsigma_kn_dcos(1e-9, c) == pytest.approx(math.pi * RE ** 2 * (1 + c * c), rel=1e-8, abs=0)
    # forward scattering is unchanged by recoil: P = 1 at c = 1
    assert orc.dsigma_kn_dcos(2.0, 1.0) == pytest.approx(2 * math.pi * RE ** 2, rel=1e-12, abs=0)


def test_photoabsorption_model(orc):
    # Heitler's K-shell Born formula (32 pi sqrt2 / 3) r_e^2 alpha^4 Z^5 (mc^2/E)^(7/2), x 5/4
    E, Z = 100.0, 32
    ref = 1.25 * (32 * math.pi * math.sqrt(2) / 3) * RE ** 2 * ALPHA ** 4 * Z ** 5 * (MEC2 / E) ** 3.5
    assert orc.sigma_pe(Z, E) == pytest.approx(ref, rel=1e-12, abs=0)
    assert orc.sigma_pe(29, 200.0) / orc.sigma_pe(29, 100.0) == pytest.approx(2 ** -3.5, rel=1e-12)
    assert orc.sigma_pe(32, 300.0) / orc.sigma_pe(16, 300.0) == pytest.approx(32.0, rel=1e-12)


def test_pair_model(orc):
    assert orc.sigma_pair(32, 1000.0) == 0.0
    assert orc.sigma_pair(32, 2 * MEC2) == 0.0
    E = 2000.0
    k = E / MEC2
    ref = (2 * math.pi / 3) * ALPHA * RE ** 2 * 32 ** 2 * ((k - 2) / k) ** 3
    assert orc.sigma_pair(32, E) == pytest.approx(ref, rel=1e-12, abs=0)
    assert orc.sigma_pair(13, E) / orc.sigma_pair(26, E) == pytest.approx(0.25, rel=1e-12)


def test_material_compositions(orc):
    E = 662.0
    k = E / MEC2
    # Ge: electron density rho N_A Z / A
    ne = 5.323 * NA * 32 / 72.630
    assert orc.mu(W.MAT_GE, E)[1] == pytest.approx(0.1 * ne * orc.sigma_kn(k), rel=1e-12, abs=0)
    # water: 10 electrons per molecule of molar mass 2*1.008 + 15.999
    ne_w = 1.0 * NA * 10 / (2 * 1.008 + 15.999)
    assert orc.mu(W.MAT_WATER, E)[1] == pytest.approx(0.1 * ne_w * orc.sigma_kn(k), rel=1e-12, abs=0)
    n_w = NA / (2 * 1.008 + 15.999)
    pe_w = 0.1 * n_w * (2 * orc.sigma_pe(1, E) + orc.sigma_pe(8, E))
    assert orc.mu(W.MAT_WATER, E)[0] == pytest.approx(pe_w, rel=1e-12, abs=0)
    assert orc.mu(W.MAT_VACUUM, E) == (0.0, 0.0, 0.0)
    # total attenuation of Ge at 662 keV is of the order of the real value (~0.4 /cm)
    assert 0.02 < sum(orc.mu(W.MAT_GE, E)) < 0.08


def test_tables_grid_and_interpolation(orc):
    t = orc.Tables.build(W.MATERIAL_CODES, 1000, 10.0, 3000.0)
    a = t.array()
    assert a.shape == (5, 3, 1000)
    assert not a[0].any()
    step = (math.log(3000.0) - math.log(10.0)) / 999
    for g in (0, 1, 417, 998, 999):
        E = math.exp(math.log(10.0) + g * step)
        exact = orc.mu(W.MAT_GE, E)
        # stored values are the closed forms rounded to binary32
        for c in range(3):
            assert a[1, c, g] == np.float32(exact[c])
        v = t.eval(1, E)
        for c in range(2):
            assert v[c] == pytest.approx(float(a[1, c, g]), rel=1e-12, abs=0)
    # linear interpolation in ln E: error bounded by (step^2/8) max |f''| ~ 12.25 f step^2/8
    rng = np.random.default_rng(3)
    for E in np.exp(rng.uniform(math.log(10.0), math.log(3000.0), 200)):
        ex = orc.mu(W.MAT_GE, E)
        v = t.eval(1, E)
        assert sum(v) == pytest.approx(sum(ex), rel=1e-4)
        if E <= 2 * MEC2:
            assert v[2] == 0.0
