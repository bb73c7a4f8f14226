"""The oracle's colour-ordered amplitudes against the Parke-Taylor formula.

At m_t = 0 and Gamma_t = 0, gg -> t t~ g and gg -> t t~ g g are the
one-quark-line amplitudes 0 -> q q~ + n gluons (all momenta outgoing; an
incoming gluon of helicity h is an outgoing one of helicity -h).  Their full
colour decomposition over the chains (T^{a_s1} .. T^{a_sn})_{i_q j_q~} is exact
at tree level, and the oracle projects its explicit colour tensors onto those
chains (Sec. 2, colour-flow decomposition).  For the MHV configurations (two
negative helicities: one of the quarks and one gluon j) the Parke-Taylor
formula gives the partial amplitude of the cyclic ordering (q, s_1, .., s_n, q~)
as

    |A| = C |<f j>|^3 |<f' j>| / (|<q s_1>| |<s_1 s_2>| .. |<s_n q~>| |<q~ q>|),

f the quark with j's helicity, f' the other one, C common to all helicities
and orderings of a process (couplings, normalisation); the anti-MHV
configurations (two positive helicities) are its parity image, with |[ab]| =
|<ab>| (Parke and Taylor, Phys. Rev. Lett. 56 (1986) 2459; Mangano and Parke,
Phys. Rept. 200 (1991) 301, for the quark line).  Only magnitudes enter, with
|<ab>|^2 = |2 p_a.p_b| for crossed momenta too, so no spinor phase convention
is involved.  Every other helicity of gg -> t t~ g vanishes (quark helicity
conservation, and all-but-one equal helicities); for gg -> t t~ g g the NMHV
configurations have no one-term formula and are pinned elsewhere (Ward,
Lorentz, Bose and explicit-colour tests).
"""
import itertools
import math

import numpy as np
import pytest

from helpers import mdot
from paper_2106_12631_gb300 import inputs as I

TOP, TBAR = 2, 3


def all_outgoing(h: int, npar: int):
    """Leg helicities of helicity index h (leg 0 is the highest bit, set = +1),
    the two incoming gluons crossed to outgoing."""
    hel = [1 if (h >> (npar - 1 - k)) & 1 else -1 for k in range(npar)]
    hel[0], hel[1] = -hel[0], -hel[1]
    return hel


def special_legs(out, gluons):
    """(j, f, f') of an MHV or anti-MHV configuration, else None."""
    if out[TOP] == out[TBAR]:
        return None
    for sign in (-1, 1):  # MHV: the lone negative gluon; anti-MHV: the lone positive one
        odd = [g for g in gluons if out[g] == sign]
        if len(odd) == 1 and sum(1 for x in out if x == sign) == 2:
            f = TOP if out[TOP] == sign else TBAR
            return odd[0], f, TBAR if f == TOP else TOP
    return None


@pytest.mark.parametrize("proc", [3, 4])
def test_parke_taylor_ratios(orc, proc):
    npar = {3: 5, 4: 6}[proc]
    gluons = [0, 1] + list(range(4, npar))
    orderings = list(itertools.permutations(gluons))  # the oracle's flow order: lexicographic
    prm = orc.params(mt=0.0, wt=0.0)
    nevt = 4
    mom, _ = orc.rambo(proc, I.uniforms(9100 + proc, 4 * (npar - 2), nevt), 1500.0, prm)
    jf = orc.colour_flows(proc, mom, prm, nthreads=4)
    assert jf.shape == (1 << npar, len(orderings), nevt)
    nmhv = 0
    for e in range(nevt):
        p = mom[:, :, e]

        def ang(a, b):
            return math.sqrt(abs(2.0 * mdot(p[a], p[b])))

        scale = np.abs(jf[:, :, e]).max()
        ratios = []
        for h in range(1 << npar):
            out = all_outgoing(h, npar)
            sp = special_legs(out, gluons)
            if sp is None:
                nneg = sum(1 for x in out if x < 0)
                if proc == 4 and out[TOP] != out[TBAR] and nneg == 3:
                    nmhv += 1  # NMHV: no one-term formula
                    continue
                assert np.abs(jf[h, :, e]).max() <= 1e-12 * scale, (h, out)
                continue
            j, f, fp = sp
            num = ang(f, j) ** 3 * ang(fp, j)
            for k, sigma in enumerate(orderings):
                cyc = [TOP, *sigma, TBAR]
                den = math.prod(ang(cyc[i], cyc[(i + 1) % len(cyc)]) for i in range(len(cyc)))
                ratios.append(abs(jf[h, k, e]) / (num / den))
        ratios = np.array(ratios)
        # one constant for every MHV / anti-MHV helicity and every ordering
        assert len(ratios) == (2 * 2 * (npar - 2)) * len(orderings)
        assert ratios.max() / ratios.min() - 1 <= 1e-10, (ratios.min(), ratios.max())
    if proc == 4:
        assert nmhv == nevt * 2 * 6  # C(4,2) gluon pairs x 2 quark helicities per event


def test_parke_taylor_detects_a_wrong_ordering(orc):
    """Control: the same ratios with the chain read in the other direction
    (q, s_n, .., s_1, q~) are not constant, so the test above fixes the
    orientation of the chains as well."""
    proc, npar = 3, 5
    gluons = [0, 1, 4]
    orderings = list(itertools.permutations(gluons))
    prm = orc.params(mt=0.0, wt=0.0)
    mom, _ = orc.rambo(proc, I.uniforms(9200, 12, 1), 1500.0, prm)
    jf = orc.colour_flows(proc, mom, prm)
    p = mom[:, :, 0]

    def ang(a, b):
        return math.sqrt(abs(2.0 * mdot(p[a], p[b])))

    ratios = []
    for h in range(1 << npar):
        sp = special_legs(all_outgoing(h, npar), gluons)
        if sp is None:
            continue
        j, f, fp = sp
        num = ang(f, j) ** 3 * ang(fp, j)
        for k, sigma in enumerate(orderings):
            cyc = [TOP, *reversed(sigma), TBAR]
            den = math.prod(ang(cyc[i], cyc[(i + 1) % len(cyc)]) for i in range(len(cyc)))
            ratios.append(abs(jf[h, k, 0]) / (num / den))
    assert max(ratios) / min(ratios) - 1 > 1e-3
