"""Pins of the oracle's Dirac algebra, external wavefunctions and SU(3) colour.

These are textbook identities, independent of how the oracle builds the
objects: Clifford algebra, Dirac equation, spinor normalisation and
completeness, helicity eigen-property, transversality of polarisation vectors;
Gell-Mann normalisation, structure constants, Casimir and Jacobi identities.
"""
import numpy as np
import pytest

from helpers import mdot

G = np.diag([1.0, -1.0, -1.0, -1.0])


@pytest.fixture(scope="module")
def gam(orc):
    return orc.gamma()


def slash(gam, p):
    return sum(G[m, m] * p[m] * gam[m] for m in range(4))


def test_clifford(gam):
    for m in range(4):
        for n in range(4):
            anti = gam[m] @ gam[n] + gam[n] @ gam[m]
            np.testing.assert_allclose(anti, 2 * G[m, n] * np.eye(4), atol=1e-15)
    g5 = 1j * gam[0] @ gam[1] @ gam[2] @ gam[3]
    np.testing.assert_allclose(g5, gam[4], atol=1e-15)
    # upper components left-handed: P_L = (1 - g5)/2 projects on the upper pair
    np.testing.assert_allclose((np.eye(4) - gam[4]) / 2, np.diag([1, 1, 0, 0]), atol=1e-15)


def _momenta(rng, m, n=20):
    out = []
    for _ in range(n):
        v = rng.normal(size=3) * rng.uniform(1, 500)
        out.append(np.array([np.sqrt(v @ v + m * m), *v]))
    out.append(np.array([np.sqrt(100.0 ** 2 + m * m), 0, 0, -100.0]))  # along -z
    out.append(np.array([np.sqrt(100.0 ** 2 + m * m), 0, 0, 100.0]))   # along +z
    return out


@pytest.mark.parametrize("m", [0.0, 173.0])
def test_dirac_equation_and_normalisation(orc, gam, m):
    rng = np.random.default_rng(1)
    g0 = gam[0]
    for p in _momenta(rng, m):
        ps = slash(gam, p)
        uu = np.zeros((4, 4), complex)
        vv = np.zeros((4, 4), complex)
        for lam in (-1, 1):
            u = orc.wavefunction("u", p, m, lam)
            v = orc.wavefunction("v", p, m, lam)
            scale = p[0]
            np.testing.assert_allclose((ps - m * np.eye(4)) @ u, 0, atol=1e-12 * scale)
            np.testing.assert_allclose((ps + m * np.eye(4)) @ v, 0, atol=1e-12 * scale)
            ubar = u.conj() @ g0
            vbar = v.conj() @ g0
            assert abs(ubar @ u - 2 * m) < 1e-12 * scale
            assert abs(vbar @ v + 2 * m) < 1e-12 * scale
            # helicity: (Sigma . p^) u = lam u,  (Sigma . p^) v = -lam v
            pp = np.linalg.norm(p[1:])
            sig = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
            hs = sum(p[k + 1] / pp * sig[k] for k in range(3))
            H = np.kron(np.eye(2), hs)
            np.testing.assert_allclose(H @ u, lam * u, atol=1e-12 * np.sqrt(scale))
            np.testing.assert_allclose(H @ v, -lam * v, atol=1e-12 * np.sqrt(scale))
            uu += np.outer(u, ubar)
            vv += np.outer(v, vbar)
        # completeness
        np.testing.assert_allclose(uu, ps + m * np.eye(4), atol=1e-12 * p[0])
        np.testing.assert_allclose(vv, ps - m * np.eye(4), atol=1e-12 * p[0])


def test_massless_chirality_exact(orc):
    """For m = 0 the helicity +1 spinor u has exactly vanishing left components."""
    rng = np.random.default_rng(2)
    for p in _momenta(rng, 0.0):
        u = orc.wavefunction("u", p, 0.0, +1)
        assert u[0] == 0 and u[1] == 0
        u = orc.wavefunction("u", p, 0.0, -1)
        assert u[2] == 0 and u[3] == 0


def test_polarisation_vectors(orc):
    rng = np.random.default_rng(3)
    for k in _momenta(rng, 0.0):
        eps = {lam: orc.wavefunction("eps", k, 0.0, lam) for lam in (-1, 1)}
        for lam in (-1, 1):
            e = eps[lam]
            assert abs(e[0]) == 0
            assert abs(mdot(k, e)) < 1e-12 * k[0]
            assert abs(mdot(e, e.conj()) + 1) < 1e-14
        assert abs(mdot(eps[1], eps[-1].conj())) < 1e-14
        # helicity: (S.k^) v = i k^ x v has eigenvalue lam on eps(k, lam)
        kh = k[1:] / np.linalg.norm(k[1:])
        Sk = 1j * np.array([[0, -kh[2], kh[1]], [kh[2], 0, -kh[0]], [-kh[1], kh[0], 0]])
        for lam in (-1, 1):
            np.testing.assert_allclose(Sk @ eps[lam][1:], lam * eps[lam][1:], atol=1e-14)


def test_su3_generators(orc):
    T, f = orc.su3()
    for a in range(8):
        np.testing.assert_allclose(T[a], T[a].conj().T, atol=1e-15)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
    cas = sum(T[a] @ T[a] for a in range(8))
    np.testing.assert_allclose(cas, 4.0 / 3.0 * np.eye(3), atol=1e-15)
    # [T^a, T^b] = i f^abc T^c
    for a in range(8):
        for b in range(8):
            lhs = T[a] @ T[b] - T[b] @ T[a]
            rhs = 1j * sum(f[a, b, c] * T[c] for c in range(8))
            np.testing.assert_allclose(lhs, rhs, atol=1e-15)


def test_structure_constants(orc):
    _, f = orc.su3()
    assert abs(f[0, 1, 2] - 1.0) < 1e-15
    assert abs(f[3, 4, 7] - np.sqrt(3) / 2) < 1e-15
    assert abs(f[0, 3, 6] - 0.5) < 1e-15
    np.testing.assert_allclose(f, -np.transpose(f, (1, 0, 2)), atol=1e-15)
    np.testing.assert_allclose(f, -np.transpose(f, (0, 2, 1)), atol=1e-15)
    # f^acd f^bcd = N delta^ab
    np.testing.assert_allclose(np.einsum("acd,bcd->ab", f, f), 3 * np.eye(8), atol=1e-14)
    # Jacobi
    j = (np.einsum("abe,ecd->abcd", f, f) + np.einsum("bce,ead->abcd", f, f)
         + np.einsum("cae,ebd->abcd", f, f))
    assert np.max(np.abs(j)) < 1e-14
