"""Pins of the oracle's squared matrix elements.

* e+e- -> mu+mu- (photon + Z): textbook helicity closed form and its pure-QED
  limit 2 e^4 (t^2 + u^2) / s^2; exactly four of sixteen helicities survive
  (Fig. 1 caption).
* gg -> t tbar at Gamma_t = 0: the LO closed form (Combridge 1979; Ellis,
  Stirling, Webber) and its massless limit.
* gg -> t tbar (g (g)): Ward identity (one gluon polarisation replaced by its
  momentum gives a zero colour-dressed amplitude), Lorentz invariance under
  boosts and rotations (Gamma_t = 0), parity, Bose symmetry of identical gluons.
* Colour: chain-basis matrix closed forms (diagonal N C_F^n, two-gluon
  off-diagonal -2/3), rank of the diagram colour Gram matrix = number of
  colour flows.
* Diagram / helicity counts printed with the paper's processes.
"""
import json
import math
import os

import numpy as np
import pytest

from helpers import boost, mdot, rotate, two_body
from paper_2106_12631_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
FACTS = json.load(open(os.path.join(HERE, "golden", "paper_facts.json")))["processes"]
P = I.SM_PARAMS
NR = {1: 8, 2: 8, 3: 12, 4: 16}
ECM = {1: 500.0, 2: 1500.0, 3: 1500.0, 4: 1500.0}


@pytest.mark.parametrize("proc", [1, 2, 3, 4])
def test_counts(orc, proc):
    info = orc.process_info(proc)
    assert info["ndiagrams"] == FACTS[str(proc)]["ndiagrams"]
    assert info["nhel"] == FACTS[str(proc)]["nhel"]


def _ee_closed_form(mom, mz, wz):
    e2 = 4 * math.pi / P["alpha_inv"]
    sw2 = P["sw2"]
    cw2 = 1 - sw2
    gl, gr = -0.5 + sw2, sw2
    s = mdot(mom[0] + mom[1], mom[0] + mom[1])
    t = mdot(mom[1] - mom[3], mom[1] - mom[3])   # (p_e- - p_mu-)^2
    u = mdot(mom[1] - mom[2], mom[1] - mom[2])   # (p_e- - p_mu+)^2
    D = s - mz ** 2 + 1j * mz * wz

    def A(gi, gj):
        return e2 / s + e2 / (sw2 * cw2) * gi * gj / D

    return (u ** 2 * (abs(A(gl, gl)) ** 2 + abs(A(gr, gr)) ** 2)
            + t ** 2 * (abs(A(gl, gr)) ** 2 + abs(A(gr, gl)) ** 2)), s, t, u


def _angles(seed, n):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.999, 0.999, n), rng.uniform(0, 2 * math.pi, n)


def test_ee_mumu_closed_form(orc):
    # exactly on-shell momenta built from angles (RAMBO output is on shell only to
    # ~1e-12 when the boost is ill-conditioned; that is pinned in test_oracle_rambo)
    mom = two_body(500.0, 0.0, *_angles(21, 300))
    me, ph = orc.me(1, mom, per_helicity=True)
    cf, *_ = _ee_closed_form(mom, P["mz"], P["wz"])
    np.testing.assert_allclose(me, cf, rtol=1e-13)
    np.testing.assert_allclose(ph.sum(axis=0), me, rtol=1e-15)
    # the same through RAMBO momenta: agreement limited by their mass-shell rounding
    rnd = I.uniforms(21, 8, 300)
    mr, _ = orc.rambo(1, rnd, 500.0)
    np.testing.assert_allclose(orc.me(1, mr), _ee_closed_form(mr, P["mz"], P["wz"])[0],
                               rtol=1e-11)
    # exactly four helicity combinations are non-zero, the same for all events
    nz = np.any(ph != 0, axis=1)
    assert nz.sum() == FACTS["1"]["nhel_allowed"]
    assert np.all((ph != 0) == nz[:, None])
    # which ones: e+/e- opposite and mu+/mu- opposite helicities
    for h in np.nonzero(nz)[0]:
        bits = [(h >> (3 - i)) & 1 for i in range(4)]
        assert bits[0] != bits[1] and bits[2] != bits[3]


def test_ee_mumu_qed_limit(orc):
    prm = orc.params(mz=1.0e9, wz=0.0)
    mom = two_body(500.0, 0.0, *_angles(22, 100))
    me = orc.me(1, mom, prm)
    e2 = 4 * math.pi / P["alpha_inv"]
    s = mdot(mom[0] + mom[1], mom[0] + mom[1])
    t = mdot(mom[1] - mom[3], mom[1] - mom[3])
    u = mdot(mom[1] - mom[2], mom[1] - mom[2])
    np.testing.assert_allclose(me, 2 * e2 ** 2 * (t ** 2 + u ** 2) / s ** 2, rtol=1e-10)


def test_gg_tt_closed_form(orc):
    prm = orc.params(wt=0.0)
    mom = two_body(1500.0, P["mt"], *_angles(23, 300))
    me = orc.me(2, mom, prm)
    g4 = (4 * math.pi * P["alpha_s"]) ** 2
    s = mdot(mom[0] + mom[1], mom[0] + mom[1])
    t1 = 2 * mdot(mom[0], mom[2]) / s
    t2 = 2 * mdot(mom[1], mom[2]) / s
    rho = 4 * P["mt"] ** 2 / s
    cf = g4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    np.testing.assert_allclose(me, cf, rtol=1e-12)


def test_gg_tt_massless_limit(orc):
    prm = orc.params(wt=0.0, mt=0.0)
    mom = two_body(1500.0, 0.0, *_angles(24, 200))
    me = orc.me(2, mom, prm)
    g4 = (4 * math.pi * P["alpha_s"]) ** 2
    s = mdot(mom[0] + mom[1], mom[0] + mom[1])
    t = mdot(mom[0] - mom[2], mom[0] - mom[2])
    u = mdot(mom[1] - mom[2], mom[1] - mom[2])
    cf = g4 * ((t * t + u * u) / (6 * t * u) - 3 * (t * t + u * u) / (8 * s * s))
    np.testing.assert_allclose(me, cf, rtol=1e-12)


def _colour_projector(orc, proc):
    # the colour sum is a^T CC a* = a^H conj(CC) a
    CC = orc.colour_gram(proc).conj()
    lam, U = np.linalg.eigh(CC)
    keep = lam > 1e-9 * lam.max()
    return np.sqrt(lam[keep])[:, None] * U[:, keep].conj().T, int(keep.sum())


@pytest.mark.parametrize("proc", [2, 3, 4])
def test_colour_gram_rank(orc, proc):
    _, rank = _colour_projector(orc, proc)
    assert rank == FACTS[str(proc)]["ncolor"]


@pytest.mark.parametrize("proc", [2, 3, 4])
def test_ward_identity(orc, proc):
    prm = orc.params(wt=0.0)
    rnd = I.uniforms(25, NR[proc], 2)
    mom, _ = orc.rambo(proc, rnd, 1500.0, prm)
    Pj, _ = _colour_projector(orc, proc)
    npar = mom.shape[0]
    gluons = [l for l in range(npar) if l not in (2, 3)]
    step = {2: 1, 3: 3, 4: 7}[proc]
    control = 0.0
    for ev in range(2):
        m1 = mom[:, :, ev]
        for leg in gluons:
            for h in range(0, 1 << npar, step):
                aw = orc.amplitudes(proc, m1, h, prm, pol_override=m1[leg].astype(complex),
                                    pol_leg=leg)
                scale = np.linalg.norm(np.abs(Pj) @ np.abs(aw))
                assert np.linalg.norm(Pj @ aw) < 1e-12 * scale
                # control: with the physical polarisation the amplitude does not vanish
                a = orc.amplitudes(proc, m1, h, prm)
                control = max(control, np.linalg.norm(Pj @ a) / np.linalg.norm(np.abs(Pj) @ np.abs(a)))
    assert control > 1e-2


@pytest.mark.parametrize("proc", [1, 2, 3, 4])
def test_lorentz_and_parity(orc, proc):
    prm = orc.params(wt=0.0)
    nev = {1: 20, 2: 20, 3: 8, 4: 3}[proc]
    rnd = I.uniforms(26, NR[proc], nev)
    mom, _ = orc.rambo(proc, rnd, ECM[proc], prm)
    me = orc.me(proc, mom, prm)
    npar = mom.shape[0]
    for beta, axis, ang in (([0.3, -0.2, 0.35], [1, 2, 3], 0.7), ([-0.45, 0.1, 0.0], [0, 1, 0], 2.1)):
        mb = np.stack([rotate(boost(mom[l], beta), axis, ang) for l in range(npar)])
        np.testing.assert_allclose(orc.me(proc, mb, prm), me, rtol=1e-11)
    mp = mom.copy()
    mp[:, 1:] *= -1
    np.testing.assert_allclose(orc.me(proc, mp, prm), me, rtol=1e-12)


def test_width_breaks_lorentz_only_slightly(orc):
    """With Gamma_t != 0 the helicity sum is frame dependent at O(Gamma/m); a sanity bound."""
    rnd = I.uniforms(27, 8, 20)
    mom, _ = orc.rambo(2, rnd, 1500.0)
    me = orc.me(2, mom)
    mb = np.stack([boost(mom[l], [0.3, -0.2, 0.35]) for l in range(4)])
    d = np.max(np.abs(orc.me(2, mb) / me - 1))
    assert 1e-12 < d < 1e-3


@pytest.mark.parametrize("proc", [2, 3, 4])
def test_bose_symmetry(orc, proc):
    nev = {2: 20, 3: 6, 4: 3}[proc]
    rnd = I.uniforms(28, NR[proc], nev)
    mom, _ = orc.rambo(proc, rnd, 1500.0)
    me = orc.me(proc, mom)
    sw = mom.copy()
    sw[[0, 1]] = sw[[1, 0]]
    np.testing.assert_allclose(orc.me(proc, sw), me, rtol=1e-12)
    if proc == 4:
        sw = mom.copy()
        sw[[4, 5]] = sw[[5, 4]]
        np.testing.assert_allclose(orc.me(proc, sw), me, rtol=1e-12)


@pytest.mark.parametrize("ng", [1, 2, 3, 4])
def test_chain_colour_matrix(orc, ng):
    C = orc.chain_colour_matrix(ng)
    n = math.factorial(ng)
    assert C.shape == (n, n)
    assert np.max(np.abs(C.imag)) < 1e-12
    C = C.real
    np.testing.assert_allclose(C, C.T, atol=1e-12)
    np.testing.assert_allclose(np.diag(C), 3 * (4 / 3) ** ng, rtol=1e-13)  # N C_F^n
    if ng == 2:
        np.testing.assert_allclose(C[0, 1], -2 / 3, rtol=1e-13)  # N C_F (C_F - N/2)
    ev = np.linalg.eigvalsh(C)
    assert ev.min() > 1e-9  # chains independent for SU(3), n <= 4
