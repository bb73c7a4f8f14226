"""Pins of the oracle's RAMBO phase-space generator (Kleiss, Stirling, Ellis).

Momentum conservation, on-shell masses, the closed-form flat massless volume
(pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!), the closed-form massive two-body
volume pi |k| / sqrt(s), uniformity of the two-body angle and of the
three-body Dalitz plot, and the massive three-body volume against an
independent Dalitz-area integral (phase space = pi^2 * area in (E1, E2)).
"""
import math

import numpy as np
import pytest

from helpers import mdot, rambo_gamma
from paper_2106_12631_gb300 import inputs as I

MT = I.SM_PARAMS["mt"]


boost_gamma = rambo_gamma


EPS = np.finfo(float).eps


@pytest.mark.parametrize("proc,nr,ecm", [(1, 8, 500.0), (2, 8, 1500.0), (3, 12, 1500.0),
                                         (4, 16, 1500.0)])
def test_conservation_and_mass_shell(orc, proc, nr, ecm):
    nev = 5000
    rnd = I.uniforms(11, nr, nev)
    mom, w = orc.rambo(proc, rnd, ecm)
    nfin = mom.shape[0] - 2
    tol = 8 * EPS * (1 + boost_gamma(rnd, nfin) ** 2)
    tot = mom[2:].sum(axis=0)
    assert np.all(np.abs(tot[0] - ecm) <= tol * ecm)
    assert np.all(np.max(np.abs(tot[1:]), axis=0) <= tol * ecm)
    np.testing.assert_allclose(mom[0], [[ecm / 2], [0], [0], [ecm / 2]] * np.ones((1, nev)))
    np.testing.assert_allclose(mom[1], [[ecm / 2], [0], [0], [-ecm / 2]] * np.ones((1, nev)))
    masses = {1: [0, 0], 2: [MT, MT], 3: [MT, MT, 0], 4: [MT, MT, 0, 0]}[proc]
    for i, m in enumerate(masses):
        p = mom[2 + i]
        assert np.all(np.abs(mdot(p, p) - m * m) <= tol * ecm ** 2)
    assert np.all(w > 0) and np.all(np.isfinite(w))


@pytest.mark.parametrize("n", [2, 3, 4])
def test_massless_weight_closed_form(orc, n):
    # massless final states: use e+e- -> mu+mu- (n=2); for n=3,4 build the
    # massless configuration by setting mt = 0
    proc = {2: 1, 3: 3, 4: 4}[n]
    prm = orc.params(mt=0.0)
    rnd = I.uniforms(12, 4 * n, 500)
    s = 1000.0 ** 2
    _, w = orc.rambo(proc, rnd, 1000.0, prm)
    w0 = (math.pi / 2) ** (n - 1) * s ** (n - 2) / (math.factorial(n - 1) * math.factorial(n - 2))
    np.testing.assert_allclose(w, w0, rtol=1e-14)


def test_massive_two_body_weight(orc):
    rnd = I.uniforms(13, 8, 500)
    ecm = 1500.0
    mom, w = orc.rambo(2, rnd, ecm)
    tol = 8 * EPS * (1 + boost_gamma(rnd, 2) ** 2)
    k = np.linalg.norm(mom[2, 1:], axis=0)
    kexact = math.sqrt(ecm ** 2 / 4 - MT ** 2)
    assert np.all(np.abs(k / kexact - 1) <= tol)
    assert np.all(np.abs(w / (math.pi * kexact / ecm) - 1) <= tol)


def test_two_body_angle_uniform(orc):
    from scipy import stats
    rnd = I.uniforms(14, 8, 50000)
    mom, _ = orc.rambo(1, rnd, 500.0)
    c = mom[3, 3] / mom[3, 0]
    assert stats.kstest((c + 1) / 2, "uniform").pvalue > 1e-4
    phi = np.arctan2(mom[3, 2], mom[3, 1])
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4


def test_three_body_dalitz_uniform(orc):
    """Massless 3-body: (E1, E2) uniform on the triangle -> P(E1 <= x) = (2x/ecm)^2."""
    from scipy import stats
    prm = orc.params(mt=0.0)
    ecm = 1000.0
    rnd = I.uniforms(15, 12, 50000)
    mom, _ = orc.rambo(3, rnd, ecm, prm)
    e1 = mom[2, 0]
    assert np.all(e1 <= ecm / 2 * (1 + 1e-12))
    assert stats.kstest(e1, lambda x: np.clip(2 * x / ecm, 0, 1) ** 2).pvalue > 1e-4


def _dalitz_area(ecm, m1, m2, m3, n=4000):
    """Area of the allowed (E1, E2) region, by the triangle condition on |p|'s."""
    e1 = np.linspace(m1, ecm, n + 1)
    e1 = 0.5 * (e1[1:] + e1[:-1])
    area = 0.0
    de1 = (ecm - m1) / n
    for x in e1:
        p1 = math.sqrt(max(x * x - m1 * m1, 0.0))
        e2 = np.linspace(m2, ecm - x - m3, n + 1)
        if e2[-1] <= e2[0]:
            continue
        e2m = 0.5 * (e2[1:] + e2[:-1])
        p2 = np.sqrt(np.maximum(e2m ** 2 - m2 * m2, 0.0))
        e3 = ecm - x - e2m
        p3 = np.sqrt(np.maximum(e3 ** 2 - m3 * m3, 0.0))
        ok = (p3 <= p1 + p2) & (p3 >= np.abs(p1 - p2))
        area += ok.sum() * (e2[1] - e2[0]) * de1
    return area


def test_massive_three_body_volume(orc):
    ecm = 1500.0
    nev = 200000
    rnd = I.uniforms(16, 12, nev)
    _, w = orc.rambo(3, rnd, ecm)
    mc = w.mean()
    err = w.std() / math.sqrt(nev)
    exact = math.pi ** 2 * _dalitz_area(ecm, MT, MT, 0.0, n=1500)
    assert abs(mc - exact) < 5 * err + 2e-3 * exact


def test_below_threshold_rejected(orc):
    rnd = I.uniforms(17, 8, 4)
    with pytest.raises(ValueError):
        orc.rambo(2, rnd, 300.0)
