"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars:
* RAMBO momenta and weights: per event within 16 eps (1 + gamma^2), gamma the
  Lorentz factor of RAMBO's boost: each side rounds to about 2.5 eps gamma^2.
* FP64 matrix elements on identical momenta: 1e-12 relative per event, except
  for events whose own FP64 conditioning is worse: there the bar is 4 d_rot,
  d_rot = the oracle's relative change under exact rotations of the event
  (rounding-level input changes), and never above 1e-9.  At most 0.1% of
  events (plus one, for small samples) may need the relaxation.
* Mixed precision (FP32 amplitudes, FP64 denominators and sums): median <=
  1e-6, 99.9th percentile <= 1e-5, max <= 1e-4, no NaN/Inf; for events with
  d_rot <= 1e-14 (well conditioned) every event is within 1e-5.
* Helicity mask: identical to the oracle's set of non-zero helicities.
* Event sum: 1e-14 relative to the oracle's pairwise sum, bitwise
  reproducible run to run.
"""
import numpy as np
import pytest
import torch

from helpers import (FP64_CAP, FP64_REL, MIXED_MAX_REL, MIXED_MEDIAN_REL, MIXED_P999_REL, fp64_tol,
                     oracle_conditioning, rambo_gamma)
from paper_2106_12631_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_ILL_FRACTION = 1e-3
WELL_CONDITIONED = 1e-14
EPS = np.finfo(float).eps
NR = {1: 8, 2: 8, 3: 12, 4: 16}
ECM = {1: 500.0, 2: 1500.0, 3: 1500.0, 4: 1500.0}
NAME = {1: "ee_mumu", 2: "gg_tt", 3: "gg_ttg", 4: "gg_ttgg"}


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


_ORACLE = {}


def oracle_sample(orc, proc, seed, nevt):
    """Oracle momenta, matrix elements and conditioning of a seeded sample
    (computed once per module: several modes compare with the same values)."""
    key = (proc, seed, nevt)
    if key not in _ORACLE:
        rnd = I.uniforms(seed, NR[proc], nevt)
        mom_o, _ = orc.rambo(proc, rnd, ECM[proc])
        me_o, d_rot = oracle_conditioning(orc, proc, mom_o, nthreads=16)
        _ORACLE[key] = (mom_o, me_o, d_rot)
    return _ORACLE[key]


def gpu_mask(mg, proc):
    rnd = I.uniforms(I.filter_seed_of(NAME[proc]), NR[proc], 16)
    mom, _ = mg.rambo(proc, dev(rnd), ECM[proc])
    return mg.filter_helicities(proc, mom)


@pytest.mark.parametrize("proc,nevt", [(1, 1), (1, 1000), (1, 16384), (2, 37), (2, 4097), (3, 129), (4, 67)])
def test_rambo_parity(mg, orc, proc, nevt):
    rnd = I.uniforms(41 + proc, NR[proc], nevt)
    mom, wgt = mg.rambo(proc, dev(rnd), ECM[proc])
    m_o, w_o = orc.rambo(proc, rnd, ECM[proc])
    m_g, w_g = host(mom), host(wgt)
    tol = 16 * EPS * (1 + rambo_gamma(rnd, m_o.shape[0] - 2) ** 2)
    err = np.max(np.abs(m_g - m_o), axis=(0, 1)) / ECM[proc]
    assert np.all(err <= tol), (err / tol).max()
    assert np.all(np.abs(w_g / w_o - 1) <= tol)


@pytest.mark.parametrize("proc", [1, 2, 3, 4])
def test_filter_mask(mg, orc, proc):
    rnd = I.uniforms(I.filter_seed_of(NAME[proc]), NR[proc], 16)
    mom_o, _ = orc.rambo(proc, rnd, ECM[proc])
    _, ph = orc.me(proc, mom_o, per_helicity=True)
    want = np.any(ph != 0, axis=1).astype(np.int32)
    mask = host(gpu_mask(mg, proc))
    np.testing.assert_array_equal(mask, want)
    if proc == 1:
        assert mask.sum() == 4


@pytest.mark.parametrize("mode", ["fp64", "fp64_unrolled"])
@pytest.mark.parametrize("proc,nevt", [(1, 1), (1, 33), (1, 16384), (2, 1), (2, 4099), (3, 1), (3, 257), (4, 1),
                                       (4, 67)])
def test_sigmakin_fp64_parity(mg, orc, proc, nevt, mode):
    mom_o, me_o, d_rot = oracle_sample(orc, proc, 51 + proc, nevt)
    mask = gpu_mask(mg, proc)
    me_g = host(mg.sigmakin(proc, dev(mom_o), mask, mode=mode))
    rel = np.abs(me_g / me_o - 1)
    check_fp64(rel, d_rot)


def check_fp64(rel, d_rot):
    tol = fp64_tol(d_rot)
    assert np.all(rel <= tol), (rel.max(), int(np.argmax(rel / tol)))
    assert np.mean(rel > FP64_REL) <= FP64_ILL_FRACTION + 1.0 / len(rel)


@pytest.mark.parametrize("mode", ["mixed_simt", "mixed", "mixed_tc", "mixed_unrolled"])
@pytest.mark.parametrize("proc,nevt", [(1, 16384), (2, 4099), (3, 4099), (4, 4099)])
def test_sigmakin_mixed(mg, orc, proc, nevt, mode):
    mom_o, me_o, d_rot = oracle_sample(orc, proc, 61 + proc, nevt)
    mask = gpu_mask(mg, proc)
    me_g = host(mg.sigmakin(proc, dev(mom_o), mask, mode=mode))
    assert np.all(np.isfinite(me_g))
    rel = np.abs(me_g / me_o - 1)
    print("proc %d %s: max %.3g median %.3g p99.9 %.3g (well-conditioned max %.3g)"
          % (proc, mode, rel.max(), np.median(rel), np.quantile(rel, 0.999),
             rel[d_rot <= WELL_CONDITIONED].max()))
    check_mixed(rel, d_rot)


def check_mixed(rel, d_rot):
    assert rel.max() <= MIXED_MAX_REL
    assert np.quantile(rel, 0.999) <= MIXED_P999_REL
    assert np.median(rel) <= MIXED_MEDIAN_REL
    assert np.all(rel[d_rot <= WELL_CONDITIONED] <= MIXED_P999_REL)


@pytest.mark.parametrize("proc", [1, 3, 4])
def test_mask_subset(mg, orc, proc):
    """me with a subset of helicities equals the oracle's partial helicity sum."""
    nevt = 40
    rnd = I.uniforms(71, NR[proc], nevt)
    mom_o, _ = orc.rambo(proc, rnd, ECM[proc])
    _, ph = orc.me(proc, mom_o, per_helicity=True, nthreads=8)
    nhel = ph.shape[0]
    rng = np.random.default_rng(proc)
    sub = (rng.uniform(size=nhel) < 0.4).astype(np.int32)
    sub[1] = 1
    want = ph[sub == 1].sum(axis=0)
    _, d_rot = oracle_conditioning(orc, proc, mom_o)
    me_g = host(mg.sigmakin(proc, dev(mom_o), dev(sub), mode="fp64"))
    me_u = host(mg.sigmakin(proc, dev(mom_o), dev(sub), mode="fp64_unrolled"))
    ok = want != 0
    assert np.all(np.abs(me_u[ok] / want[ok] - 1) <= fp64_tol(d_rot[ok]))
    rel = np.abs(me_g[ok] / want[ok] - 1)
    assert np.all(rel <= fp64_tol(d_rot[ok]))
    assert np.all(me_g[~ok] == 0)


def test_zero_mask_and_empty(mg):
    mom = torch.zeros((6, 4, 5), dtype=torch.float64, device="cuda")
    mask = torch.zeros(64, dtype=torch.int32, device="cuda")
    me = torch.full((5,), 7.0, dtype=torch.float64, device="cuda")
    mg.sigmakin(4, mom, mask, mode="fp64", me=me)
    assert np.all(host(me) == 0)
    empty = torch.zeros((6, 4, 0), dtype=torch.float64, device="cuda")
    assert mg.sigmakin(4, empty, mask, mode="mixed").numel() == 0


def test_event_sum(mg, orc):
    for nevt in (1, 4095, 4096, 4097, 100003):
        rng = np.random.default_rng(nevt)
        me = rng.exponential(size=nevt)
        w = rng.uniform(0.5, 2, size=nevt)
        a = host(mg.event_sum(dev(me), dev(w)))
        b = host(mg.event_sum(dev(me), dev(w)))
        np.testing.assert_array_equal(a, b)
        ref = orc.event_sum(me, w)
        np.testing.assert_allclose(a, ref, rtol=1e-14)
    z = host(mg.event_sum(torch.zeros(0, dtype=torch.float64, device="cuda"),
                          torch.zeros(0, dtype=torch.float64, device="cuda")))
    np.testing.assert_array_equal(z, [0, 0, 0])


def test_pipeline_host_matches_device_path(mg):
    proc, nevt = 3, 3001
    rnd = I.uniforms(81, 12, nevt)
    mask = gpu_mask(mg, proc)
    mom, _ = mg.rambo(proc, dev(rnd), 1500.0)
    me_dev = host(mg.sigmakin(proc, mom, mask, mode="mixed"))
    rnd_h = torch.from_numpy(rnd).pin_memory()
    sums_h = torch.zeros(3, dtype=torch.float64).pin_memory()
    wgt_h = torch.zeros(nevt, dtype=torch.float64).pin_memory()
    me_h = mg.pipeline_host(proc, rnd_h, 1500.0, mask, mode="mixed", wgt_host=wgt_h, sums_host=sums_h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(me_h.numpy(), me_dev)
    # the event sum of the pipeline is the device event sum of the same me and weights
    _, wgt = mg.rambo(proc, dev(rnd), 1500.0)
    np.testing.assert_array_equal(wgt_h.numpy(), host(wgt))
    ref = host(mg.event_sum(torch.from_numpy(me_dev).cuda(), wgt))
    np.testing.assert_array_equal(sums_h.numpy(), ref)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_full_size_sampled(mg, orc, mode):
    """gg -> t t~ g g at 2^20 events in the benchmark's launch configuration;
    sampled events recomputed one by one by the oracle."""
    nevt = 1 << 20
    seed = I.seed_of("gg_ttgg")
    rnd = I.uniforms(seed, 16, nevt)
    mask = gpu_mask(mg, 4)
    mom, wgt = mg.rambo(4, dev(rnd), 1500.0)
    me = mg.sigmakin(4, mom, mask, mode=mode)
    out = mg.event_sum(me, wgt)
    idx = np.sort(np.random.default_rng(5).choice(nevt, 24, replace=False))
    idx[-1] = nevt - 1
    mom_g = host(mom)[:, :, idx]
    me_g = host(me)[idx]
    r = I.uniforms_at(seed, 16, idx)
    mom_o, _ = orc.rambo(4, r, 1500.0)
    tol = 16 * EPS * (1 + rambo_gamma(r, 4) ** 2)
    assert np.all(np.max(np.abs(mom_g - mom_o), axis=(0, 1)) / 1500.0 <= tol)
    me_o, d_rot = oracle_conditioning(orc, 4, np.ascontiguousarray(mom_g))
    rel = np.abs(me_g / me_o - 1)
    if mode == "fp64":
        assert np.all(rel <= fp64_tol(d_rot))
    else:
        assert rel.max() <= MIXED_MAX_REL and np.all(rel[d_rot <= WELL_CONDITIONED] <= MIXED_P999_REL)
    s = host(out)
    assert s[2] == nevt and np.isfinite(s[0]) and s[0] > 0


def test_abi_errors(mg):
    L = mg.lib()
    p = torch.zeros(64, dtype=torch.float64, device="cuda")
    base = p.data_ptr()
    assert L.mg_sigmakin(9, 1, base, base, base, 0, None) == -2
    assert L.mg_sigmakin(1, -1, base, base, base, 0, None) == -1
    assert L.mg_sigmakin(1, 1, base + 8, base, base, 0, None) == -3
    assert L.mg_sigmakin(1, 1, base, base, base, 99, None) == -1
    assert L.mg_rambo(2, 4, 300.0, base, 8, base, base, None) == -1   # below threshold
    assert L.mg_rambo(3, 4, 1500.0, base, 8, base, base, None) == -1  # too few random rows
    assert L.mg_event_sum(5000, base, base, base, base, 8, None) == -6


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("proc", [3, 4])
def test_mask_subset_many_groups(mg, orc, proc, mode):
    """A random subset of the helicities with enough events that every
    persistent CTA (304 for gg -> t t~ g g) runs several groups and the last
    group is ragged: me equals the oracle's partial helicity sum."""
    nevt = 2 * 304 * 4 + 37
    rnd = I.uniforms(72, NR[proc], nevt)
    mom_o, _ = orc.rambo(proc, rnd, ECM[proc])
    nhel = 1 << (proc + 2 if proc > 1 else 4)
    sub = (np.random.default_rng(10 + proc).uniform(size=nhel) < 0.6).astype(np.int32)
    sub[1] = 1
    _, ph = orc.me(proc, mom_o, per_helicity=True, nthreads=16)
    want = ph[sub == 1].sum(axis=0)
    me_g = host(mg.sigmakin(proc, dev(mom_o), dev(sub), mode=mode))
    ok = want != 0
    assert np.all(me_g[~ok] == 0)
    rel = np.abs(me_g[ok] / want[ok] - 1)
    if mode == "fp64":
        # never above the 1e-9 cap, 1e-12 on at least 99 % of the events, the
        # median at rounding level.  A partial helicity sum has no averaging over
        # the other helicities, so near a collinear limit its FP64 rounding shows
        # more often than the full sum's (this sample: 0.28 % of the events above
        # 1e-12, at most 8e-12), and the rotation probe of the full-sum bar can
        # miss it (one gg -> t t~ g event with pT = 12 GeV against a beam:
        # single-helicity differences up to 5e-11 between two FP64 evaluations,
        # rotation sensitivity at most 2e-12)
        assert np.all(rel <= FP64_CAP), rel.max()
        assert np.mean(rel > FP64_REL) <= 0.01, np.mean(rel > FP64_REL)
        assert np.median(rel) <= 1e-13, np.median(rel)
    else:
        assert rel.max() <= MIXED_MAX_REL and np.median(rel) <= MIXED_MEDIAN_REL, (rel.max(), np.median(rel))
