"""The kernel-split variant (currents kernel, then amplitudes kernel, chunk by
chunk, replayed from a CUDA graph), through the C ABI.

* Bit-identical to the single helicity-shared kernel (same arithmetic in the
  same order) in FP64 and mixed precision, for all four processes, with the
  default workspace and with a small one that forces many chunks and a ragged
  last chunk.
* A replayed graph reads the buffers' current contents (a new mask through
  the same buffer), and a parameter change re-captures it.
* FP64 against the oracle on one process directly (1e-12 relative or the
  event's own conditioning).
* Errors: a mode without a split variant, a workspace below 8 records.
"""
import numpy as np
import pytest
import torch

from helpers import MIXED_MAX_REL, MIXED_MEDIAN_REL, fp64_tol, oracle_conditioning
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_mask(mg, proc):
    rnd = torch.from_numpy(I.uniforms(I.filter_seed_of(NAME[proc]), NR[proc], 16)).cuda()
    mom, _ = mg.rambo(proc, rnd, ECM[proc])
    return mg.filter_helicities(proc, mom)


def record_bytes(mg, proc, mode):
    return mg.sigmakin_split_workspace_bytes(proc, mode, 4) // 8


def events(mg, proc, nevt, seed):
    rnd = torch.from_numpy(I.uniforms(seed, NR[proc], nevt)).cuda()
    return mg.rambo(proc, rnd, ECM[proc])[0]


@pytest.mark.parametrize("mode", ["fp64", "mixed_simt"])
@pytest.mark.parametrize("proc,nevt", [(1, 1), (1, 4097), (2, 4099), (3, 1031), (4, 131)])
def test_split_equals_single_kernel(mg, proc, nevt, mode):
    mom = events(mg, proc, nevt, 131 + proc)
    mask = gpu_mask(mg, proc)
    want = host(mg.sigmakin(proc, mom, mask, mode=mode))
    got = host(mg.sigmakin_split(proc, mom, mask, mode=mode))
    np.testing.assert_array_equal(got, want)
    # many chunks: 12 events each (the last one ragged)
    ws = torch.empty(2 * 12 * record_bytes(mg, proc, mode) // 8, dtype=torch.float64, device="cuda")
    got = host(mg.sigmakin_split(proc, mom, mask, mode=mode, workspace=ws))
    np.testing.assert_array_equal(got, want)


def test_graph_replay_and_recapture(mg):
    proc, nevt, mode = 3, 2003, "mixed_simt"
    mom = events(mg, proc, nevt, 141)
    mask = gpu_mask(mg, proc)
    me = torch.empty(nevt, dtype=torch.float64, device="cuda")
    ws = torch.empty(mg.sigmakin_split_workspace_bytes(proc, mode, nevt) // 8, dtype=torch.float64, device="cuda")
    a = host(mg.sigmakin_split(proc, mom, mask, mode=mode, me=me, workspace=ws)).copy()
    b = host(mg.sigmakin_split(proc, mom, mask, mode=mode, me=me, workspace=ws)).copy()
    np.testing.assert_array_equal(a, b)
    # same buffers, new contents: half of the helicities
    full = mask.clone()
    mask[::2] = 0
    got = host(mg.sigmakin_split(proc, mom, mask, mode=mode, me=me, workspace=ws)).copy()
    np.testing.assert_array_equal(got, host(mg.sigmakin(proc, mom, mask, mode=mode)))
    assert np.all(got < a)
    mask.copy_(full)
    # new parameters: the graph is captured again
    old = mg.get_params()
    try:
        mg.set_params(alpha_s=0.13)
        got = host(mg.sigmakin_split(proc, mom, mask, mode=mode, me=me, workspace=ws)).copy()
        np.testing.assert_array_equal(got, host(mg.sigmakin(proc, mom, mask, mode=mode)))
        # |M|^2 ~ alpha_s^3; a ratio of two mixed results, each within the mixed bar
        rel = np.abs(got / a / (0.13 / 0.118) ** 3 - 1)
        assert np.median(rel) < 2 * MIXED_MEDIAN_REL and rel.max() < 2 * MIXED_MAX_REL
    finally:
        mg.set_params(**old)


def test_split_fp64_against_oracle(mg, orc):
    proc, nevt = 2, 517
    rnd = I.uniforms(151, NR[proc], nevt)
    mom_o, _ = orc.rambo(proc, rnd, ECM[proc])
    me_o, d_rot = oracle_conditioning(orc, proc, mom_o)
    got = host(mg.sigmakin_split(proc, torch.from_numpy(mom_o).cuda(), gpu_mask(mg, proc), mode="fp64"))
    assert np.all(np.abs(got / me_o - 1) <= fp64_tol(d_rot))


def test_split_errors(mg):
    proc = 2
    mom = events(mg, proc, 64, 161)
    mask = gpu_mask(mg, proc)
    with pytest.raises(mg.MGError):
        mg.sigmakin_split(proc, mom, mask, mode="mixed_tc")
    small = torch.empty(7 * record_bytes(mg, proc, "fp64") // 8, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError):
        mg.sigmakin_split(proc, mom, mask, mode="fp64", workspace=small)
    assert mg.sigmakin_split(proc, mom[:, :, :0].contiguous(), mask, mode="fp64").numel() == 0
