"""Adjoint gradient d me / d rnd (gg -> t t~ and gg -> t t~ g) against the oracle.

The default modes run the helicity-shared adjoint, modes *_unrolled the
per-helicity one.  Bars (per event, normwise over the random rows k):
  |g - g_ref|_inf / |g_ref|_inf <= 1e-4 for the FP32 forward + adjoint
  (tested against the oracle's forward-mode dual-number gradient and against
  central finite differences h = 1e-6 of the FP64 oracle), <= 1e-9 for the
  FP64 adjoint against the dual-number gradient; rows RAMBO does not consume
  are exactly 0; the matrix elements returned with the gradient equal the
  SIGMAKIN ones.  Events with a random number within 1e-3 of 0 or 1 are left
  out of the finite-difference comparison (the +-h points must stay inside
  (0, 1)).
"""
import numpy as np
import pytest
import torch

from paper_2106_12631_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NR = {2: 8, 3: 12}


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12631_gb300 import mg as M
    M.lib()
    return M


def mask_for(mg, proc, nrows):
    rnd = I.uniforms(I.filter_seed_of({2: "gg_tt", 3: "gg_ttg"}[proc]), nrows, 16)
    mom, _ = mg.rambo(proc, torch.from_numpy(rnd).cuda(), 1500.0)
    return mg.filter_helicities(proc, mom)


def normwise(g, ref):
    return np.max(np.abs(g - ref), axis=0) / np.max(np.abs(ref), axis=0)


@pytest.mark.parametrize("proc,nevt", [(2, 33), (3, 37)])
@pytest.mark.parametrize("mode,bar", [("fp64", 1e-9), ("mixed", 1e-4), ("fp64_unrolled", 1e-9),
                                      ("mixed_unrolled", 1e-4)])
def test_adjoint_vs_dual(mg, orc, proc, nevt, mode, bar):
    nrows = 16
    rnd = I.uniforms(I.seed_of("gg_ttg_grad") + proc, nrows, nevt)
    mask = mask_for(mg, proc, nrows)
    g, me = mg.sigmakin_grad(proc, torch.from_numpy(rnd).cuda(), 1500.0, mask, mode=mode)
    torch.cuda.synchronize()
    g, me = g.cpu().numpy(), me.cpu().numpy()
    me_o, g_o = orc.me_grad(proc, rnd, 1500.0, nthreads=8)
    used = 4 * (orc.NPAR[proc] - 2)
    assert np.all(g[used:] == 0.0)
    err = normwise(g[:used], g_o[:used])
    print("proc %d %s: max normwise err %.3g median %.3g" % (proc, mode, err.max(), np.median(err)))
    assert np.all(err <= bar), (err.max(), int(err.argmax()))
    np.testing.assert_allclose(me, me_o, rtol=1e-9 if mode.startswith("fp64") else 1e-4)


def test_adjoint_vs_finite_differences(mg, orc):
    proc, nevt, nrows, h = 3, 24, 12, 1e-6
    rnd = I.uniforms(I.seed_of("gg_ttg_grad"), nrows, 200)
    keep = np.all((rnd > 1e-3) & (rnd < 1 - 1e-3), axis=0)
    rnd = np.ascontiguousarray(rnd[:, keep][:, :nevt])
    mask = mask_for(mg, proc, nrows)
    g, _ = mg.sigmakin_grad(proc, torch.from_numpy(rnd).cuda(), 1500.0, mask, mode="mixed")
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    fd = np.zeros_like(g)
    for k in range(nrows):
        rp, rm = rnd.copy(), rnd.copy()
        rp[k] += h
        rm[k] -= h
        fd[k] = (orc.me(proc, orc.rambo(proc, rp, 1500.0)[0]) - orc.me(proc, orc.rambo(proc, rm, 1500.0)[0])) / (2 * h)
    err = normwise(g, fd)
    print("fd: max %.3g median %.3g" % (err.max(), np.median(err)))
    assert np.all(err <= 1e-4)


def test_me_matches_sigmakin_and_gout_scaling(mg):
    proc, nevt = 3, 1000
    rnd = torch.from_numpy(I.uniforms(77, 16, nevt)).cuda()
    mask = mask_for(mg, proc, 16)
    g1, me1 = mg.sigmakin_grad(proc, rnd, 1500.0, mask, mode="fp64")
    mom, _ = mg.rambo(proc, rnd, 1500.0)
    me_s = mg.sigmakin(proc, mom, mask, mode="fp64")
    gout = torch.linspace(-2.0, 3.0, nevt, dtype=torch.float64, device="cuda")
    g2, _ = mg.sigmakin_grad(proc, rnd, 1500.0, mask, mode="fp64", gout=gout)
    torch.cuda.synchronize()
    np.testing.assert_allclose(me1.cpu().numpy(), me_s.cpu().numpy(), rtol=1e-13)
    # gout is applied before the (linear) RAMBO adjoint: equal up to rounding,
    # normwise per event (the adjoint sums terms that cancel, and its shared
    # atomics may add in a different order in the two calls)
    a, b = g2.cpu().numpy(), (g1 * gout).cpu().numpy()
    assert np.all(np.max(np.abs(a - b), axis=0) <= 1e-9 * np.max(np.abs(b), axis=0))


def test_autograd_function(mg):
    proc, nevt = 3, 300
    rnd = torch.from_numpy(I.uniforms(78, 16, nevt)).cuda().requires_grad_(True)
    mask = mask_for(mg, proc, 16)
    me = mg.matrix_element(rnd, proc, 1500.0, mask, "mixed")
    w = torch.linspace(0.5, 1.5, nevt, dtype=torch.float64, device="cuda")
    (me * w).sum().backward()
    g_ref, _ = mg.sigmakin_grad(proc, rnd.detach(), 1500.0, mask, mode="mixed", gout=w)
    torch.cuda.synchronize()
    # the adjoint accumulates shared variants with atomics: two calls agree to
    # FP32 rounding (normwise per event), not bit for bit
    a, b = rnd.grad.cpu().numpy(), g_ref.cpu().numpy()
    assert np.all(np.max(np.abs(a - b), axis=0) <= 1e-5 * np.max(np.abs(b), axis=0))


def test_grad_unsupported_process(mg):
    L = mg.lib()
    p = torch.zeros(64, dtype=torch.float64, device="cuda").data_ptr()
    assert L.mg_sigmakin_grad(4, 1, 1500.0, p, 16, p, None, p, None, 1, None) == -2
    assert L.mg_sigmakin_grad(1, 1, 500.0, p, 16, p, None, p, None, 1, None) == -2


@pytest.mark.parametrize("proc,mode", [(2, "fp64"), (3, "fp64"), (3, "mixed")])
def test_helicity_subsets_add_up(mg, proc, mode):
    """The gradient is linear in the helicity sum: the gradients for two
    complementary helicity masks add up to the full one (the masked runs take
    the adjoint's path for incomplete helicity sets, the full one its warp-sum
    path, which the oracle comparisons pin)."""
    nevt, nrows = 301, 16
    rnd = torch.from_numpy(I.uniforms(I.seed_of("gg_ttg_grad") + 10 * proc, nrows, nevt)).cuda()
    full = mask_for(mg, proc, nrows)
    nhel = full.numel()
    a = full.clone()
    a[torch.arange(nhel, device="cuda") % 3 == 0] = 0
    b = full - a
    g, me = mg.sigmakin_grad(proc, rnd, 1500.0, full, mode=mode)
    ga, mea = mg.sigmakin_grad(proc, rnd, 1500.0, a, mode=mode)
    gb, meb = mg.sigmakin_grad(proc, rnd, 1500.0, b, mode=mode)
    torch.cuda.synchronize()
    bar = 1e-12 if mode == "fp64" else 1e-5
    np.testing.assert_allclose((mea + meb).cpu().numpy(), me.cpu().numpy(), rtol=bar)
    s, ref = (ga + gb).cpu().numpy(), g.cpu().numpy()
    assert np.all(np.max(np.abs(s - ref), axis=0) <= bar * np.max(np.abs(ref), axis=0))


@pytest.mark.parametrize("mode,bar", [("mixed", 1e-4), ("fp64", 1e-9)])
def test_adjoint_full_size_sampled(mg, orc, mode, bar):
    """The gradient workload at full size (gg -> t t~ g, 2^18 events, 16 random
    rows) in the benchmark's launch configuration; 32 sampled events, the
    first and the last among them, recomputed one by one by the oracle's
    dual numbers from their own uniforms."""
    proc, nevt, nrows = 3, 1 << 18, 16
    seed = I.seed_of("gg_ttg_grad")
    mask = mask_for(mg, proc, nrows)
    rnd = torch.from_numpy(I.uniforms(seed, nrows, nevt)).cuda()
    g, me = mg.sigmakin_grad(proc, rnd, 1500.0, mask, mode=mode)
    idx = np.sort(np.random.default_rng(7).choice(nevt, 32, replace=False))
    idx[0], idx[-1] = 0, nevt - 1
    g = g.cpu().numpy()[:, idx]
    me = me.cpu().numpy()[idx]
    me_o, g_o = orc.me_grad(proc, I.uniforms_at(seed, nrows, idx), 1500.0, nthreads=8)
    used = 4 * (orc.NPAR[proc] - 2)
    assert np.all(g[used:] == 0.0)
    err = normwise(g[:used], g_o[:used])
    assert np.all(err <= bar), (err.max(), int(idx[err.argmax()]))
    np.testing.assert_allclose(me, me_o, rtol=1e-9 if mode == "fp64" else 1e-4)
