"""Pins of the oracle's dual-number gradient and event accumulation.

d(me)/d(random numbers) by forward-mode dual numbers through RAMBO (massive,
with its Newton step) and the amplitudes must agree with central finite
differences of the plain FP64 oracle; rows RAMBO does not consume get an
exactly zero derivative.  The event sum must match an exactly rounded sum.
"""
import math

import numpy as np
import pytest

from paper_2106_12631_gb300 import inputs as I


@pytest.mark.parametrize("proc,nr", [(2, 8), (3, 16)])
def test_dual_gradient_matches_central_differences(orc, proc, nr):
    rnd = I.uniforms(31, nr, 6)
    rnd = np.clip(rnd, 1e-3, 1 - 1e-3)
    me, g = orc.me_grad(proc, rnd, 1500.0)
    me0 = orc.me(proc, orc.rambo(proc, rnd, 1500.0)[0])
    np.testing.assert_allclose(me, me0, rtol=1e-14)
    h = 1e-6
    used = 4 * (orc.NPAR[proc] - 2)
    fd = np.zeros_like(g)
    for k in range(used):
        rp, rm = rnd.copy(), rnd.copy()
        rp[k] += h
        rm[k] -= h
        fd[k] = (orc.me(proc, orc.rambo(proc, rp, 1500.0)[0])
                 - orc.me(proc, orc.rambo(proc, rm, 1500.0)[0])) / (2 * h)
    err = np.max(np.abs(g - fd), axis=0) / np.max(np.abs(fd), axis=0)
    assert np.all(err < 1e-6)
    assert np.all(g[used:] == 0.0)


def test_event_sum(orc):
    rng = np.random.default_rng(4)
    me = rng.exponential(size=100001)
    w = rng.uniform(0.5, 2.0, size=100001)
    out = orc.event_sum(me, w)
    x = me * w
    assert abs(out[0] - math.fsum(x)) <= 1e-14 * math.fsum(x)
    assert abs(out[1] - math.fsum(x * x)) <= 1e-14 * math.fsum(x * x)
    assert out[2] == 100001
    assert np.all(orc.event_sum(np.zeros(0), np.zeros(0)) == 0)
