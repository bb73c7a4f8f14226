"""RAMBO and SIGMAKIN in one kernel (mg_sigmakin_rambo, mg_sigmakin_seeded),
through the C ABI: me and the phase-space weight equal, bit for bit, RAMBO
(mg_rambo or mg_rambo_seeded) followed by mg_sigmakin, for every process in
the helicity-shared modes, on batches that leave a ragged last group and on
the full gg -> t t~ g g workload; the per-helicity modes and bad arguments are
refused."""
import numpy as np
import pytest
import torch

from paper_2106_12631_gb300 import inputs as I

pytestmark = pytest.mark.gpu

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


def gpu_mask(mg, proc):
    rnd = I.uniforms(I.filter_seed_of(NAME[proc]), NR[proc], 16)
    mom, _ = mg.rambo(proc, torch.from_numpy(rnd).cuda(), ECM[proc])
    return mg.filter_helicities(proc, mom)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_tc"])
@pytest.mark.parametrize("proc,nevt", [(1, 1), (1, 4099), (2, 37), (2, 20001), (3, 1), (3, 5003), (4, 3), (4, 4099)])
def test_fused_buffered_equals_two_kernels(mg, proc, nevt, mode):
    rnd = torch.from_numpy(I.uniforms(201 + proc, 16, nevt)).cuda()  # 16 rows: extra rows are ignored
    mask = gpu_mask(mg, proc)
    mom, wgt = mg.rambo(proc, rnd, ECM[proc])
    me = mg.sigmakin(proc, mom, mask, mode=mode)
    me_f, wgt_f = mg.sigmakin_rambo(proc, rnd, ECM[proc], mask, mode=mode)
    np.testing.assert_array_equal(host(wgt_f), host(wgt))
    np.testing.assert_array_equal(host(me_f), host(me))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("proc,nevt,first", [(1, 777, 0), (2, 4097, 12345), (3, 3001, 7), (4, 1029, 1 << 40)])
def test_fused_seeded_equals_two_kernels(mg, proc, nevt, first, mode):
    seed = I.seed_of(NAME[proc])
    mask = gpu_mask(mg, proc)
    mom, wgt = mg.rambo_seeded(proc, nevt, ECM[proc], seed, first)
    me = mg.sigmakin(proc, mom, mask, mode=mode)
    me_f, wgt_f = mg.sigmakin_seeded(proc, nevt, ECM[proc], seed, mask, mode=mode, first_event=first)
    np.testing.assert_array_equal(host(wgt_f), host(wgt))
    np.testing.assert_array_equal(host(me_f), host(me))


def test_fused_full_workload(mg):
    """gg -> t t~ g g at 2^20 events (every CTA runs many groups, the next
    group's RAMBO in flight behind each)."""
    nevt = 1 << 20
    rnd = torch.from_numpy(I.uniforms(I.seed_of("gg_ttgg"), 16, nevt)).cuda()
    mask = gpu_mask(mg, 4)
    mom, wgt = mg.rambo(4, rnd, 1500.0)
    me = mg.sigmakin(4, mom, mask, mode="mixed")
    me_f, wgt_f = mg.sigmakin_rambo(4, rnd, 1500.0, mask, mode="mixed")
    assert torch.equal(wgt_f, wgt) and torch.equal(me_f, me)


def test_fused_zero_mask_and_errors(mg):
    rnd = torch.from_numpy(I.uniforms(5, 16, 300)).cuda()
    zero = torch.zeros(64, dtype=torch.int32, device="cuda")
    me, wgt = mg.sigmakin_rambo(4, rnd, 1500.0, zero, mode="mixed")
    _, wgt2 = mg.rambo(4, rnd, 1500.0)
    assert np.all(host(me) == 0)
    np.testing.assert_array_equal(host(wgt), host(wgt2))
    L = mg.lib()
    mask = gpu_mask(mg, 4)
    p = rnd.data_ptr()
    for mode in (3, 4, 9):  # per-helicity modes and an unknown one
        assert L.mg_sigmakin_rambo(4, 300, 1500.0, p, 16, mask.data_ptr(), mode, p, p, None) == -1
    assert L.mg_sigmakin_rambo(4, 300, 1500.0, p, 12, mask.data_ptr(), 1, p, p, None) == -1  # too few rows
    assert L.mg_sigmakin_rambo(4, 300, 300.0, p, 16, mask.data_ptr(), 1, p, p, None) == -1  # below threshold
    assert L.mg_sigmakin_seeded(4, 300, 1500.0, 1, -1, mask.data_ptr(), 1, p, p, None) == -1
    assert L.mg_sigmakin_rambo(9, 300, 1500.0, p, 16, mask.data_ptr(), 1, p, p, None) == -2
    assert L.mg_sigmakin_rambo(4, 300, 1500.0, p + 8, 16, mask.data_ptr(), 1, p, p, None) == -3
    assert L.mg_sigmakin_rambo(4, 0, 1500.0, p, 16, mask.data_ptr(), 1, p, p, None) == 0
