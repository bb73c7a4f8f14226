"""The batched entry point for an external integrator (Sec. 5: an existing
event generator hands its own phase-space points over, event by event, and
gets their matrix elements back), through the C ABI.

* Momenta as an array of structures give the same me, bit for bit, as the
  structure-of-arrays call on the same momenta, in every mode; asking for a
  helicity choice changes no me.
* The helicity chosen per event equals the oracle's inverse-CDF choice over its
  own per-helicity |M_h|^2 with the same uniforms, except where u * |M|^2 falls
  within the mode's error of a boundary of the running sum (FP64: 1e-12 or
  4 d_rot relative up to 1e-9, d_rot the event's own conditioning; mixed: 1e-4).
* The colour flow chosen per event likewise equals the oracle's choice over its
  own colour-flow weights w_s = sum over the good helicities of |J_s|^2, the
  oracle's J_s projected from explicit colour tensors (Sec. 2, colour-flow
  method), except within the mode's error of a boundary (FP64: 1e-9 or
  100 d_rot; mixed: 1e-4).
* For one phase-space point and many uniforms the chosen helicities follow
  |M_h|^2 / |M|^2 and the chosen flows w_s / sum w (5 sigma each).
* Edge cases: only vanishing helicities in the mask (me = 0, choices -1),
  no events, and a choice asked of a mode that has none (error).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import MIXED_MAX_REL, fp64_tol, oracle_conditioning
from paper_2106_12631_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NR = {1: 8, 2: 8, 3: 12, 4: 16}
ECM = {1: 500.0, 2: 1500.0, 3: 1500.0, 4: 1500.0}
NAME = {1: "ee_mumu", 2: "gg_tt", 3: "gg_ttg", 4: "gg_ttgg"}
HS_MODES = ["fp64", "mixed", "mixed_simt", "mixed_tc"]


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12631_gb300 import mg as M
    M.lib()
    return M


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_mask(mg, proc):
    rnd = I.uniforms(I.filter_seed_of(NAME[proc]), NR[proc], 16)
    mom, _ = mg.rambo(proc, dev(rnd), ECM[proc])
    return mg.filter_helicities(proc, mom)


def aos(mom_soa):
    """(npar, 4, nevt) -> (nevt, npar, 4)"""
    return np.ascontiguousarray(np.transpose(mom_soa, (2, 0, 1)))


@pytest.mark.parametrize("mode", HS_MODES + ["fp64_unrolled", "mixed_unrolled"])
@pytest.mark.parametrize("proc,nevt", [(1, 1), (1, 1031), (2, 4099), (3, 257), (4, 67)])
def test_aos_equals_soa(mg, orc, proc, nevt, mode):
    rnd = I.uniforms(91 + proc, NR[proc], nevt)
    mom, _ = orc.rambo(proc, rnd, ECM[proc])
    mask = gpu_mask(mg, proc)
    want = host(mg.sigmakin(proc, dev(mom), mask, mode=mode))
    got = host(mg.matrix_elements_batch(proc, dev(aos(mom)), mask, mode=mode))
    np.testing.assert_array_equal(got, want)
    if mode in HS_MODES:
        u = I.uniforms(95 + proc, 2, nevt)
        me2, _, _ = mg.matrix_elements_batch(proc, dev(aos(mom)), mask, mode=mode, hel_rnd=dev(u[0]),
                                             col_rnd=dev(u[1]))
        np.testing.assert_array_equal(host(me2), want)


def check_choice(got, want, weights, u, tol, max_bad):
    """got: GPU indices; weights: the oracle's (n, nevt) weights in order."""
    nevt = weights.shape[1]
    cum = np.cumsum(weights, axis=0)
    tot = cum[-1]
    target = u * tot
    e = np.arange(nevt)
    assert np.all(got >= 0)
    hi = cum[got, e]
    lo = np.where(got > 0, cum[np.maximum(got - 1, 0), e], 0.0)
    assert np.all(lo - tol * tot <= target) and np.all(target <= hi + tol * tot)
    bad = got != want
    assert bad.mean() <= max_bad + 1.0 / nevt, bad.sum()
    return int(bad.sum())


@pytest.mark.parametrize("mode", HS_MODES)
@pytest.mark.parametrize("proc,nevt", [(1, 2000), (2, 4099), (3, 513), (4, 131)])
def test_choices(mg, orc, proc, nevt, mode):
    rnd = I.uniforms(101 + proc, NR[proc], nevt)
    mom, _ = orc.rambo(proc, rnd, ECM[proc])
    _, ph = orc.me(proc, mom, per_helicity=True, nthreads=8)
    jf = oracle.colour_flows(proc, mom, nthreads=8)
    _, d_rot = oracle_conditioning(orc, proc, mom)
    mask = gpu_mask(mg, proc)
    mask_h = host(mask)
    u = I.uniforms(105 + proc, 2, nevt)
    _, hel, col = mg.matrix_elements_batch(proc, dev(aos(mom)), mask, mode=mode, hel_rnd=dev(u[0]),
                                           col_rnd=dev(u[1]))
    hel, col = host(hel), host(col)
    assert np.all(mask_h[hel] != 0)
    fp64 = mode == "fp64"
    good = (mask_h != 0)[:, None]
    nb = check_choice(hel, oracle.choose_helicity(ph, mask_h, u[0]), np.where(good, ph, 0.0), u[0],
                      fp64_tol(d_rot) if fp64 else MIXED_MAX_REL, 0.0 if fp64 else 0.01)
    w = np.sum(np.where(good[:, :, None], np.abs(jf) ** 2, 0.0), axis=0)
    nc = check_choice(col, oracle.choose_colour(jf, mask_h, u[1]), w, u[1],
                      np.maximum(1e-9, 100 * d_rot) if fp64 else MIXED_MAX_REL, 0.0 if fp64 else 0.01)
    print("proc %d %s: %d helicity and %d colour choices of %d differ from the oracle's" % (proc, mode, nb, nc, nevt))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_choice_frequencies(mg, orc, mode):
    proc, n = 3, 1 << 16
    rnd = I.uniforms(111, NR[proc], 1)
    mom, _ = orc.rambo(proc, rnd, ECM[proc])
    _, ph = orc.me(proc, mom, per_helicity=True)
    jf = oracle.colour_flows(proc, mom)
    mask = gpu_mask(mg, proc)
    u = I.uniforms(112, 2, n)
    rep = np.repeat(aos(mom), n, axis=0)
    me, hel, col = mg.matrix_elements_batch(proc, dev(rep), mask, mode=mode, hel_rnd=dev(u[0]), col_rnd=dev(u[1]))
    me, hel, col = host(me), host(hel), host(col)
    assert np.all(me == me[0])
    good = host(mask) != 0
    for got, w in ((hel, ph[:, 0] * good), (col, np.sum(np.abs(jf[good, :, 0]) ** 2, axis=0))):
        p = w / w.sum()
        counts = np.bincount(got, minlength=len(p))
        assert counts.size == len(p)
        for k in range(len(p)):
            assert abs(counts[k] / n - p[k]) <= 5 * math.sqrt(p[k] * (1 - p[k]) / n) + 1e-12, (k, counts[k], p[k])


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_vanishing_helicities_and_empty(mg, orc, mode):
    proc, nevt = 1, 100
    rnd = I.uniforms(121, NR[proc], nevt)
    mom, _ = orc.rambo(proc, rnd, ECM[proc])
    zero = 1 - host(gpu_mask(mg, proc))  # the helicities whose amplitude vanishes
    assert zero.sum() == 12
    u = dev(I.uniforms(122, 1, nevt)[0])
    me, hel, col = mg.matrix_elements_batch(proc, dev(aos(mom)), dev(zero.astype(np.int32)), mode=mode, hel_rnd=u,
                                            col_rnd=u)
    assert np.all(host(me) == 0)
    assert np.all(host(hel) == -1) and np.all(host(col) == -1)
    # no good helicity at all
    none = torch.zeros(16, dtype=torch.int32, device="cuda")
    me, hel, col = mg.matrix_elements_batch(proc, dev(aos(mom)), none, mode=mode, hel_rnd=u, col_rnd=u)
    assert np.all(host(me) == 0)
    assert np.all(host(hel) == -1) and np.all(host(col) == -1)
    empty = torch.zeros((0, 4, 4), dtype=torch.float64, device="cuda")
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    me0, hel0, col0 = mg.matrix_elements_batch(proc, empty, gpu_mask(mg, proc), mode=mode, hel_rnd=z, col_rnd=z)
    assert me0.numel() == 0 and hel0.numel() == 0 and col0.numel() == 0


def test_choice_needs_helicity_shared_mode(mg):
    proc = 2
    mom = torch.zeros((8, 4, 4), dtype=torch.float64, device="cuda")
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError):
        mg.matrix_elements_batch(proc, mom, gpu_mask(mg, proc), mode="fp64_unrolled", hel_rnd=u)
    with pytest.raises(mg.MGError):
        mg.matrix_elements_batch(proc, mom, gpu_mask(mg, proc), mode="mixed_unrolled", col_rnd=u)
