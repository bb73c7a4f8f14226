"""Device RNG + RAMBO, cross section and unweighting against the oracle.

* mg_rambo_seeded draws the same uniforms as inputs.uniforms (the counter-based
  generator, implemented independently on the device) and gives bit-identical
  momenta and weights to mg_rambo on those uniforms.
* mg_cross_section from the FP64 path's event sums equals the oracle's cross
  section of its own matrix elements on the same events (FP64 parity).
* mg_unweight keeps exactly the oracle's indices (bit-exact index work) for
  seeded synthetic weights at ragged and full sizes; on physics weights the
  kept sets agree except for events within FP64 rounding of the threshold.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_12631_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ECM = {1: 500.0, 2: 1500.0, 3: 1500.0, 4: 1500.0}


@pytest.fixture(scope="module")
def mg():
    from paper_2106_12631_gb300 import mg as m
    m.lib()
    return m


@pytest.mark.parametrize("proc,nevt,first", [(1, 1, 0), (2, 129, 7), (3, 5000, 1 << 33), (4, 1025, 3)])
def test_rambo_seeded_equals_buffered(mg, proc, nevt, first):
    seed = 4242 + proc
    nr = 4 * (oracle.NPAR[proc] - 2)
    rnd = torch.from_numpy(I.uniforms(seed, nr, nevt, first_event=first)).cuda()
    mom_b, wgt_b = mg.rambo(proc, rnd, ECM[proc])
    mom_s, wgt_s = mg.rambo_seeded(proc, nevt, ECM[proc], seed, first)
    torch.cuda.synchronize()
    assert torch.equal(mom_s, mom_b) and torch.equal(wgt_s, wgt_b)


@pytest.mark.parametrize("proc,nevt", [(1, 16384), (3, 1000)])
def test_cross_section_matches_oracle(mg, orc, proc, nevt):
    seed = 777 + proc
    mom, wgt = mg.rambo_seeded(proc, nevt, ECM[proc], seed)
    mask = mg.filter_helicities(proc, mom[:, :, :16].contiguous())
    me = mg.sigmakin(proc, mom, mask, mode="fp64")
    xs = mg.cross_section(proc, ECM[proc], mg.event_sum(me, wgt)).cpu().numpy()
    rnd = I.uniforms(seed, 4 * (oracle.NPAR[proc] - 2), nevt)
    mom_o, wgt_o = orc.rambo(proc, rnd, ECM[proc])
    ref = oracle.cross_section(proc, ECM[proc], orc.me(proc, mom_o, nthreads=16), wgt_o)
    np.testing.assert_allclose(xs, ref, rtol=1e-11, atol=0)


def synthetic_weights(nevt, first, seed=5150):
    r = I.uniforms(seed, 3, nevt, first_event=first)
    me = np.exp(12.0 * (r[0] - 0.5)) * (r[1] > 0.05)  # heavy tail, some exact zeros
    return me, r[2]


@pytest.mark.parametrize("nevt,first", [(1, 0), (1023, 0), (1024, 5), (1025, 0), (4097, 1 << 40), (1 << 20, 3)])
def test_unweight_bit_exact(mg, nevt, first):
    seed = 9909
    me, w = synthetic_weights(nevt, first)
    idx, cnt = mg.unweight(torch.from_numpy(me).cuda(), torch.from_numpy(w).cuda(), seed, first)
    n = int(cnt.item())
    ref = oracle.unweight(me, w, I.uniforms(seed, 64, nevt, first_event=first)[63])
    assert n == ref.size
    np.testing.assert_array_equal(idx[:n].cpu().numpy(), ref)


def test_unweight_edge_cases(mg):
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    _, cnt = mg.unweight(e, e, 1)
    assert int(cnt.item()) == 0
    z = torch.zeros(3000, dtype=torch.float64, device="cuda")
    _, cnt = mg.unweight(z, torch.ones_like(z), 1)
    assert int(cnt.item()) == 0
    one = torch.ones(3000, dtype=torch.float64, device="cuda")
    idx, cnt = mg.unweight(one, one, 1)  # every x = max x: u < 1 always keeps
    assert int(cnt.item()) == 3000
    assert torch.equal(idx, torch.arange(3000, device="cuda"))


def test_unweight_physics(mg, orc):
    proc, nevt, seed = 1, 16384, 31337
    mom, wgt = mg.rambo_seeded(proc, nevt, ECM[proc], seed)
    mask = mg.filter_helicities(proc, mom[:, :, :16].contiguous())
    me = mg.sigmakin(proc, mom, mask, mode="fp64")
    idx, cnt = mg.unweight(me, wgt, seed)
    kept = set(idx[: int(cnt.item())].cpu().numpy().tolist())
    rnd = I.uniforms(seed, 8, nevt)
    mom_o, wgt_o = orc.rambo(proc, rnd, ECM[proc])
    me_o = orc.me(proc, mom_o, nthreads=16)
    u = I.uniforms(seed, 64, nevt)[63]
    ref = set(oracle.unweight(me_o, wgt_o, u).tolist())
    x = wgt_o * me_o
    near = set(np.nonzero(np.abs(u * x.max() - x) <= 1e-10 * x.max())[0].tolist())
    assert kept ^ ref <= near
    assert len(kept) > 1000
