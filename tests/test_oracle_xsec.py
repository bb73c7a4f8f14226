"""Pins of the oracle's cross section and unweighting (Sec. 3: the weighted
events of a run give the cross section; unweighted events follow |M|^2).

* e+e- -> mu+mu- total cross section: pure QED 4 pi alpha^2 / (3 s), and with
  the Z the textbook chiral form (4 pi alpha^2 / 3 s) (1/4) sum_ij |A_ij|^2,
  A_ij = Q_e Q_mu + g_i g_j / (sw^2 cw^2) s / (s - M^2 + i M Gamma).
* gg -> t tbar (Gamma_t = 0): the closed-form |M|^2 integrated by Gauss-Legendre
  quadrature over the two-body phase space (1/2s)(beta/16 pi) int dcos.
  Both compare with the oracle's Monte Carlo over RAMBO (within 5 sigma).
* Unweighting: a hand-worked example; the kept fraction mean(x)/max(x);
  kept e+e- -> mu+mu- (QED) events have <cos^2 theta> = 2/5 (1 + cos^2 shape).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2106_12631_gb300 import inputs as I

P = I.SM_PARAMS
ALPHA = 1.0 / P["alpha_inv"]


def mc(orc, proc, ecm, n, seed, prm):
    rnd = I.uniforms(seed, 4 * (oracle.NPAR[proc] - 2), n)
    mom, wgt = orc.rambo(proc, rnd, ecm, prm)
    me = orc.me(proc, mom, prm, nthreads=8)
    return mom, wgt, me, oracle.cross_section(proc, ecm, me, wgt)


def test_xsec_ee_pure_qed(orc):
    ecm = 500.0
    prm = orc.params(mz=1.0e9, wz=0.0)
    _, _, _, (sig, err) = mc(orc, 1, ecm, 1 << 15, 9101, prm)
    ref = 4 * math.pi * ALPHA ** 2 / (3 * ecm ** 2) * oracle.HBARC2_PB
    assert err / sig < 2e-3
    assert abs(sig - ref) < 5 * err, (sig, ref, err)


def test_xsec_ee_gamma_z(orc):
    ecm = 500.0
    prm = orc.params()
    _, _, _, (sig, err) = mc(orc, 1, ecm, 1 << 15, 9102, prm)
    s, sw2 = ecm ** 2, P["sw2"]
    cw2 = 1 - sw2
    chi = s / complex(s - P["mz"] ** 2, P["mz"] * P["wz"])
    q = -1.0
    g = {"L": -0.5 - q * sw2, "R": -q * sw2}  # T3 - Q sw^2, -Q sw^2 (charged leptons)
    a2 = sum(abs(q * q + g[i] * g[j] / (sw2 * cw2) * chi) ** 2 for i in "LR" for j in "LR")
    ref = 4 * math.pi * ALPHA ** 2 / (3 * s) * a2 / 4 * oracle.HBARC2_PB
    assert abs(sig - ref) < 5 * err, (sig, ref, err)
    assert abs(ref / (4 * math.pi * ALPHA ** 2 / (3 * s) * oracle.HBARC2_PB) - 1) > 0.05  # the Z matters here


def gg_tt_closed_form(c, ecm, mt):
    s = ecm ** 2
    rho = 4 * mt ** 2 / s
    beta = math.sqrt(1 - rho)
    t1, t2 = (1 - beta * c) / 2, (1 + beta * c) / 2
    g4 = (4 * math.pi * P["alpha_s"]) ** 2
    return g4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))


def test_xsec_gg_tt_quadrature(orc):
    ecm, mt = 1500.0, P["mt"]
    prm = orc.params(wt=0.0)
    _, _, _, (sig, err) = mc(orc, 2, ecm, 1 << 14, 9103, prm)
    x, w = np.polynomial.legendre.leggauss(64)
    integral = sum(wi * gg_tt_closed_form(xi, ecm, mt) for xi, wi in zip(x, w))
    beta = math.sqrt(1 - 4 * mt ** 2 / ecm ** 2)
    ref = integral * beta / (16 * math.pi) / (2 * ecm ** 2) * oracle.HBARC2_PB
    assert err / sig < 2e-2
    assert abs(sig - ref) < 5 * err, (sig, ref, err)


def test_unweight_hand_example():
    me = np.array([0.0, 1.0, 2.0, 4.0, 3.0])
    w = np.array([1.0, 1.0, 1.0, 1.0, 0.5])
    u = np.array([0.1, 0.3, 0.6, 0.99, 0.2])
    # max x = 4: kept iff 4 u < x -> 0.4<0 no, 1.2<1 no, 2.4<2 no, 3.96<4 yes, 0.8<1.5 yes
    np.testing.assert_array_equal(oracle.unweight(me, w, u), [3, 4])
    assert oracle.unweight(np.zeros(3), np.ones(3), np.full(3, 0.5)).size == 0
    assert oracle.unweight(np.zeros(0), np.zeros(0), np.zeros(0)).size == 0


def test_unweight_distribution(orc):
    ecm, n = 500.0, 1 << 15
    prm = orc.params(mz=1.0e9, wz=0.0)
    mom, wgt, me, _ = mc(orc, 1, ecm, n, 9104, prm)
    u = I.uniforms(9104, 64, n)[63]
    kept = oracle.unweight(me, wgt, u)
    x = wgt * me
    frac = x.mean() / x.max()  # expected kept fraction
    assert abs(kept.size / n - frac) < 5 * math.sqrt(frac * (1 - frac) / n)
    c = mom[2, 3, kept] / mom[2, 0, kept]  # cos theta of the mu+
    c2 = np.mean(c ** 2)  # 1 + cos^2 theta: <cos^2> = 2/5, variance of cos^2 = 9/35 - 4/25
    assert abs(c2 - 0.4) < 5 * math.sqrt((9 / 35 - 4 / 25) / kept.size), c2


def test_choose_helicity_hand_example():
    ph = np.array([[1.0, 0.0, 2.0], [0.0, 0.0, 2.0], [3.0, 0.0, 0.0], [4.0, 0.0, 4.0]])  # (nhel=4, nevt=3)
    mask = np.array([1, 0, 1, 1])  # helicity 1 is not good
    # event 0: good sums 1, 4, 8 -> u=0.5 -> target 4 -> first run > 4 is h=3
    # event 1: all zero -> -1; event 2: runs 2, 2, 6 (h=1 skipped) -> u=0.2 -> 1.2 -> h=0
    np.testing.assert_array_equal(oracle.choose_helicity(ph, mask, np.array([0.5, 0.3, 0.2])), [3, -1, 0])
    # u = 0 picks the first good helicity with |M_h|^2 > 0; u -> 1 the last one
    np.testing.assert_array_equal(oracle.choose_helicity(ph, mask, np.array([0.0, 0.0, 0.0])), [0, -1, 0])
    np.testing.assert_array_equal(oracle.choose_helicity(ph, mask, np.full(3, 1 - 2 ** -53)), [3, -1, 3])


def test_choose_helicity_frequencies(orc):
    # one gg -> t tbar point, many uniforms: the chosen helicities follow |M_h|^2 / |M|^2
    rnd = I.uniforms(9105, 4 * 2, 1)
    mom, _ = orc.rambo(2, rnd, 1500.0)
    me, ph = orc.me(2, mom, per_helicity=True)
    n = 1 << 14
    u = I.uniforms(9106, 1, n)[0]
    mask = (ph[:, 0] > 0).astype(np.int32)
    h = oracle.choose_helicity(np.repeat(ph, n, axis=1), mask, u)
    p = ph[:, 0] / ph[:, 0].sum()
    for k in range(ph.shape[0]):
        f = np.mean(h == k)
        assert abs(f - p[k]) < 5 * math.sqrt(p[k] * (1 - p[k]) / n) + 1e-12, (k, f, p[k])
