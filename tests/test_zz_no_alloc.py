"""The allocation-free event sum (mg_event_sum_noalloc) against mg_event_sum.

mg_event_sum_noalloc is for callers that cannot allocate device memory (a
stream being captured into a CUDA graph, a host program whose device memory
belongs to another framework's pool, a loop that must not trigger the
synchronisation of cudaMalloc): it keeps its partial sums in a fixed array
inside the library instead of caller scratch.  This file runs last so that a
failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_event_sum_matches_scratch_version():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12631_gb300 import mg
    L = mg.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row; the second is smaller, so the shared array still
    # holds partials of the first call beyond the ones the second writes
    for call, nevt in enumerate((300007, 4097)):
        rng = np.random.default_rng(call)
        me = torch.from_numpy(rng.exponential(size=nevt)).cuda()
        w = torch.from_numpy(rng.uniform(0.5, 2.0, size=nevt)).cuda()
        want = mg.event_sum(me, w).cpu().numpy()
        out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        rc = L.mg_event_sum_noalloc(nevt, me.data_ptr(), w.data_ptr(), out.data_ptr(), stream)
        assert rc == 0, mg.lib().mg_status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-14)
    # beyond the stated maximum: a clear error, nothing launched
    nmax = L.mg_event_sum_noalloc_max_events()
    assert nmax == 1 << 26
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    fake = ctypes.c_void_p(out.data_ptr())
    assert L.mg_event_sum_noalloc(nmax + 1, fake, fake, out.data_ptr(), stream) == -6


def test_noalloc_edges_and_binding():
    """No events (pass 2 alone: (0, 0, 0)), exactly the largest batch the
    fixed array holds (every partial slot in use; 1 GiB of inputs), and the
    Python binding, each bit for bit against mg_event_sum."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12631_gb300 import mg
    empty = torch.zeros(0, dtype=torch.float64, device="cuda")
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    mg.event_sum_noalloc(empty, empty, out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), [0.0, 0.0, 0.0])
    nmax = int(mg.lib().mg_event_sum_noalloc_max_events())
    g = torch.Generator(device="cuda").manual_seed(2106)
    for nevt in (nmax, 5):
        me = torch.rand(nevt, dtype=torch.float64, device="cuda", generator=g)
        w = torch.rand(nevt, dtype=torch.float64, device="cuda", generator=g) + 0.5
        got = mg.event_sum_noalloc(me, w).cpu().numpy()
        want = mg.event_sum(me, w).cpu().numpy()
        np.testing.assert_array_equal(got, want)
        assert got[2] == nevt
        del me, w
