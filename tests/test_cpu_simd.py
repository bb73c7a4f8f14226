"""The SIMD CPU build of the helicity-shared program (libmg_cpu.so: the GPU
path's wavefunction, current and contraction routines compiled for the host
cores, several events per vector; Sec. 4's vectorised C++ build) against the
FP64 oracle.

* FP64: 1e-12 relative per event, or 4 d_rot where the event's own FP64
  conditioning is worse (d_rot as in the GPU parity tests).
* FP32 amplitudes (FP64 momentum sums, propagators, helicity sum): median
  <= 1e-6, max <= 1e-4 on these samples.
* A subset of helicities gives the oracle's partial helicity sum; no good
  helicity gives zeros; results do not depend on the thread count (every
  vector of events is independent); event counts that do not fill the last
  vector are handled.
"""
import numpy as np
import pytest

from helpers import fp64_tol, oracle_conditioning
from paper_2106_12631_gb300 import cpu_simd
from paper_2106_12631_gb300 import inputs as I

NR = {1: 8, 2: 8, 3: 12, 4: 16}
ECM = {1: 500.0, 2: 1500.0, 3: 1500.0, 4: 1500.0}


def sample(orc, proc, nevt, seed):
    rnd = I.uniforms(seed, NR[proc], nevt)
    mom, _ = orc.rambo(proc, rnd, ECM[proc])
    return mom


def good_mask(orc, proc):
    mom = sample(orc, proc, 16, 7000 + proc)
    _, ph = orc.me(proc, mom, per_helicity=True, nthreads=4)
    return (np.abs(ph).max(axis=1) > 0).astype(np.int32)


@pytest.mark.parametrize("proc,nevt", [(1, 1), (1, 1001), (2, 37), (2, 515), (3, 67), (4, 13)])
def test_fp64_parity(orc, proc, nevt):
    mom = sample(orc, proc, nevt, 7100 + proc)
    me_o, d_rot = oracle_conditioning(orc, proc, mom)
    me = cpu_simd.sigmakin(proc, mom, good_mask(orc, proc), "fp64", nthreads=4)
    rel = np.abs(me / me_o - 1)
    assert np.all(rel <= fp64_tol(d_rot)), rel.max()


@pytest.mark.parametrize("proc,nevt", [(1, 1001), (2, 515), (3, 67), (4, 13)])
def test_fp32_parity(orc, proc, nevt):
    mom = sample(orc, proc, nevt, 7200 + proc)
    me_o = orc.me(proc, mom, nthreads=4)
    me = cpu_simd.sigmakin(proc, mom, good_mask(orc, proc), "fp32", nthreads=4)
    rel = np.abs(me / me_o - 1)
    assert np.all(np.isfinite(me))
    assert np.median(rel) <= 1e-6 and rel.max() <= 1e-4, (np.median(rel), rel.max())


@pytest.mark.parametrize("proc", [1, 3])
def test_helicity_subset_and_zero_mask(orc, proc):
    mom = sample(orc, proc, 21, 7300 + proc)
    _, ph = orc.me(proc, mom, per_helicity=True, nthreads=4)
    rng = np.random.default_rng(proc)
    sub = (rng.uniform(size=ph.shape[0]) < 0.5).astype(np.int32)
    want = ph[sub == 1].sum(axis=0)
    got = cpu_simd.sigmakin(proc, mom, sub, "fp64", nthreads=2)
    ok = want != 0
    np.testing.assert_allclose(got[ok], want[ok], rtol=1e-11)
    assert np.all(got[~ok] == 0)
    zero = cpu_simd.sigmakin(proc, mom, np.zeros(ph.shape[0], np.int32), "fp32")
    assert np.all(zero == 0)


def test_threads_and_tails(orc):
    proc = 2
    lanes = cpu_simd.lanes("fp32")
    mom = sample(orc, proc, 5 * lanes + 3, 7400)
    mask = good_mask(orc, proc)
    a = cpu_simd.sigmakin(proc, mom, mask, "fp32", nthreads=1)
    b = cpu_simd.sigmakin(proc, mom, mask, "fp32", nthreads=3)
    np.testing.assert_array_equal(a, b)
    # the events of a partly filled last vector equal the same events computed alone
    tail = cpu_simd.sigmakin(proc, np.ascontiguousarray(mom[:, :, -3:]), mask, "fp32", nthreads=1)
    np.testing.assert_array_equal(tail, a[-3:])
    assert cpu_simd.sigmakin(proc, mom[:, :, :0], mask, "fp32").size == 0
