"""Pins of the oracle's colour-flow decomposition (Sec. 2, colour-flow method:
the full-colour amplitude is a sum over colour flows, M = sum_s J_s chi_s,
chi_s a chain of SU(3) generators between the top and antitop colours) and of
the colour-flow choice built on it.

* The diagrams' explicit colour tensors lie in the span of the chains
  (projection residual at rounding level).
* J^dagger C J with the explicit-SU(3) chain colour matrix C gives back the
  oracle's colour-summed |M_h|^2 of every helicity (all four processes).
* gg -> t tbar (massive, Gamma_t = 0), textbook colour-ordered amplitudes: with
  t1 = 2 p_g1.p_t / s, t2 = 1 - t1, rho = 4 m^2 / s and
  F = t1^2 + t2^2 + rho - rho^2 / (4 t1 t2), summed over helicities
  |J_(12)|^2 = 8 g^4 F t2 / t1, |J_(21)|^2 = 8 g^4 F t1 / t2 and
  Re J_(12) conj(J_(21)) = 8 g^4 F, where (12) is the chain T^{a1} T^{a2}
  with gluon 1 next to the top.  Their sum is the abelian gamma gamma -> t tbar
  form 8 g^4 F / (t1 t2).
* Bose symmetry of gg -> t tbar g g: exchanging the two final gluons (momenta
  and helicities) maps every flow onto the flow with those two gluons
  exchanged in its chain.
* The choice: a hand example and its frequencies at one phase-space point.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2106_12631_gb300 import inputs as I

P = I.SM_PARAMS
NORM = {1: 4.0, 2: 256.0, 3: 256.0, 4: 512.0}  # helicity x colour average x symmetry
NG = {1: 0, 2: 2, 3: 3, 4: 4}
ECM = {1: 500.0, 2: 1500.0, 3: 1500.0, 4: 1500.0}


def events(orc, proc, n, seed, prm=None):
    rnd = I.uniforms(seed, 4 * (oracle.NPAR[proc] - 2), n)
    return orc.rambo(proc, rnd, ECM[proc], prm)[0]


@pytest.mark.parametrize("proc", [1, 2, 3, 4])
def test_projection_residual(orc, proc):
    nf, res = oracle.colour_flow_info(proc)
    assert nf == math.factorial(NG[proc])
    assert res < 1e-13


@pytest.mark.parametrize("proc,n", [(1, 5), (2, 6), (3, 4), (4, 2)])
def test_flows_reproduce_colour_sum(orc, proc, n):
    mom = events(orc, proc, n, 9201 + proc)
    _, ph = orc.me(proc, mom, per_helicity=True)
    jf = oracle.colour_flows(proc, mom, nthreads=4)
    C = oracle.chain_colour_matrix(NG[proc]).real if NG[proc] else np.ones((1, 1))
    got = np.einsum("hse,st,hte->he", jf.conj(), C, jf).real / NORM[proc]
    np.testing.assert_allclose(got, ph, rtol=1e-11, atol=1e-14 * np.abs(ph).max())


def test_gg_tt_colour_ordered_closed_forms(orc):
    prm = orc.params(wt=0.0)
    mom = events(orc, 2, 8, 9210, prm)
    jf = oracle.colour_flows(2, mom, prm)
    s, mt = ECM[2] ** 2, P["mt"]
    g4 = (4 * math.pi * P["alpha_s"]) ** 2
    dot = lambda a, b: a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]
    t1 = 2 * dot(mom[0], mom[2]) / s
    t2 = 1 - t1
    rho = 4 * mt ** 2 / s
    F = t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2)
    a12 = np.sum(np.abs(jf[:, 0]) ** 2, axis=0)
    a21 = np.sum(np.abs(jf[:, 1]) ** 2, axis=0)
    x = np.sum((jf[:, 0] * jf[:, 1].conj()).real, axis=0)
    np.testing.assert_allclose(a12, 8 * g4 * F * t2 / t1, rtol=1e-12)
    np.testing.assert_allclose(a21, 8 * g4 * F * t1 / t2, rtol=1e-12)
    np.testing.assert_allclose(x, 8 * g4 * F, rtol=1e-12)
    assert np.all(np.abs(t1 - t2) > 1e-3)  # the two flows are told apart


def test_gg_ttgg_bose_symmetry(orc):
    mom = events(orc, 4, 2, 9220)
    swapped = mom[[0, 1, 2, 3, 5, 4]].copy()
    jf = oracle.colour_flows(4, mom)
    js = oracle.colour_flows(4, swapped)
    perms = list(itertools.permutations(range(4)))  # chains over gluon legs (0, 1, 4, 5)
    swap = {0: 0, 1: 1, 2: 3, 3: 2}
    fmap = [perms.index(tuple(swap[k] for k in p)) for p in perms]
    nl = 6
    for h in range(1 << nl):
        bits = [(h >> (nl - 1 - i)) & 1 for i in range(nl)]
        bits[4], bits[5] = bits[5], bits[4]
        hs = sum(b << (nl - 1 - i) for i, b in enumerate(bits))
        np.testing.assert_allclose(js[hs][fmap], jf[h], rtol=1e-10, atol=1e-12 * np.abs(jf).max())


def test_choose_colour_hand_example():
    jf = np.zeros((2, 3, 3), complex)  # (nhel, nflow, nevt)
    jf[0, :, 0] = [1, 1j, 2]           # w = 1, 1, 4 (+ helicity 1 below)
    jf[1, :, 0] = [0, 1, 0]            # w = 1, 2, 4 with both helicities
    jf[1, :, 2] = [3, 0, 0]
    mask = np.array([1, 1])
    # event 0 (w = 1, 2, 4; sum 7): u = 0.5 -> 3.5 -> runs 1, 3, 7 -> flow 2
    # event 1: all zero -> -1; event 2: w = 9, 0, 0 -> flow 0 for any u
    np.testing.assert_array_equal(oracle.choose_colour(jf, mask, np.array([0.5, 0.5, 0.99])), [2, -1, 0])
    # only helicity 0 (w = 1, 1, 4; sum 6): u = 0.3 -> 1.8 -> runs 1, 2 -> flow 1
    np.testing.assert_array_equal(oracle.choose_colour(jf, np.array([1, 0]), np.array([0.3, 0.3, 0.3])),
                                  [1, -1, -1])


def test_choose_colour_frequencies(orc):
    mom = events(orc, 3, 1, 9230)
    jf = oracle.colour_flows(3, mom)
    mask = np.ones(jf.shape[0], dtype=np.int32)
    n = 1 << 14
    u = I.uniforms(9231, 1, n)[0]
    c = oracle.choose_colour(np.repeat(jf, n, axis=2), mask, u)
    w = np.sum(np.abs(jf[:, :, 0]) ** 2, axis=0)
    p = w / w.sum()
    for k in range(len(p)):
        f = np.mean(c == k)
        assert abs(f - p[k]) < 5 * math.sqrt(p[k] * (1 - p[k]) / n) + 1e-12, (k, f, p[k])
