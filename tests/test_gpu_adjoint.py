"""CUDA adjoint vs the FP64 oracle's reverse-mode gradients (themselves pinned by finite
differences), and projected-gradient refinement on the device vs the oracle's.

Tolerance: |g_gpu - g_oracle| <= 1e-4 * max|g_oracle| per problem (the GPU forward runs in FP32 with
the outward margin, the oracle in FP64 without it)."""
import numpy as np
import pytest
import torch

from oracle import reach as orc
from paper_2605_25346_b300 import workloads as wl

pytestmark = pytest.mark.gpu
GTOL = 1e-4


def _api():
    from paper_2605_25346_b300 import api
    return api


def _interior_alpha(p, seed):
    a0 = orc.chord_alpha(p)
    g = torch.Generator().manual_seed(seed)
    a = (a0 + 0.2 * (torch.rand(a0.shape, generator=g, dtype=torch.float64) - 0.5)).clamp(0.05, 0.95)
    return a.float().double()


def _grad_close(g, o, tol=GTOL):
    o = np.asarray(o, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    scale = max(np.abs(o).max(), 1e-30)
    err = np.abs(g - o) / scale
    assert err.max() <= tol, f"gradient max err {err.max():.3e} (scale {scale:.3e})"


@pytest.mark.parametrize("widths", [[3, 12, 10, 2], [4, 24, 24, 24, 3], [2, 1, 1]])
def test_dalpha_matches_oracle(widths):
    p = wl.random_problem(61, widths, D=12, H=4, eps=0.3)
    alpha = _interior_alpha(p, 0)
    _, ga_o, _ = orc.value_and_grad(p, alpha)
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, _ = r.backward()
    _grad_close(ga, ga_o.numpy())


def test_dbeta_and_dalpha_with_splits():
    p = wl.random_problem(62, [6, 40, 40, 3], D=24, H=5, eps=0.2)
    rng = np.random.default_rng(3)
    p.splits = wl.branch_splits(p, rng, max_k=6)
    p.beta = rng.uniform(0.05, 0.5, size=p.splits.nnz).astype(np.float32).astype(np.float64)
    alpha = _interior_alpha(p, 1)
    _, ga_o, gb_o = orc.value_and_grad(p, alpha, torch.as_tensor(p.beta))
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, gb = r.backward()
    assert p.splits.nnz > 20
    _grad_close(ga, ga_o.numpy())
    _grad_close(gb, gb_o.numpy())


def test_upstream_gradients():
    p = wl.random_problem(63, [3, 16, 16, 2], D=8, H=3, eps=0.3)
    alpha = _interior_alpha(p, 2)
    rng = np.random.default_rng(0)
    wlo = rng.normal(size=(p.D, p.H + 1, p.n))
    whi = rng.normal(size=(p.D, p.H + 1, p.n))
    a = alpha.clone().requires_grad_(True)
    res = orc.reach(p, alpha=a, mode=orc.MODE_USER)
    (res["lo"] * torch.as_tensor(wlo) + res["hi"] * torch.as_tensor(whi)).sum().backward()
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, _ = r.backward(wlo=wlo, whi=whi)
    _grad_close(ga, a.grad.numpy())


def test_autograd_function_matches_backward():
    api = _api()
    p = wl.random_problem(64, [3, 16, 16, 2], D=8, H=3, eps=0.3)
    alpha = _interior_alpha(p, 3).float()
    r = api.Reach(0).load(p)
    a = alpha.cuda().requires_grad_(True)
    b = torch.zeros(0, device="cuda", requires_grad=True)
    lo, hi = api.bounds(r, a, b)
    V = (hi[:, 1:] - lo[:, 1:]).sum()
    V.backward()
    r.set_alpha(alpha.numpy())
    ga, _ = r.backward()
    np.testing.assert_allclose(a.grad.cpu().numpy(), ga, rtol=1e-6, atol=1e-6 * np.abs(ga).max())
    _, ga_o, _ = orc.value_and_grad(p, alpha.double())
    _grad_close(a.grad.cpu().numpy(), ga_o.numpy())


def test_autograd_two_forwards_then_backward_of_the_first():
    # each output's gradient is taken at the slopes its own forward call was given
    api = _api()
    p = wl.random_problem(66, [3, 16, 16, 2], D=8, H=3, eps=0.3)
    a1 = _interior_alpha(p, 5).float()
    a2 = _interior_alpha(p, 6).float()
    r = api.Reach(0).load(p)
    x1 = a1.cuda().requires_grad_(True)
    x2 = a2.cuda().requires_grad_(True)
    b = torch.zeros(0, device="cuda", requires_grad=True)
    lo1, hi1 = api.bounds(r, x1, b)
    lo2, hi2 = api.bounds(r, x2, b)
    (hi1[:, 1:] - lo1[:, 1:]).sum().backward()
    r.set_alpha(a1.numpy())
    g1, _ = r.backward()
    np.testing.assert_allclose(x1.grad.cpu().numpy(), g1, rtol=1e-6, atol=1e-6 * np.abs(g1).max())
    (hi2[:, 1:] - lo2[:, 1:]).sum().backward()
    r.set_alpha(a2.numpy())
    g2, _ = r.backward()
    np.testing.assert_allclose(x2.grad.cpu().numpy(), g2, rtol=1e-6, atol=1e-6 * np.abs(g2).max())
    assert np.abs(g1 - g2).max() > 1e-3 * np.abs(g1).max()


def test_refinement_cartpole_subset():
    p = wl.cartpole_diff()
    sub = p.subset(np.arange(0, p.D, 16))  # 64 of the 1024 sub-boxes
    steps, lr = 20, 0.1
    ref = orc.optimize_slopes(sub, steps, lr, 0.0)
    r = _api().Reach(0).load(sub)
    hist = r.optimize(steps, lr, 0.0)
    h_o = np.array(ref["V_hist"])
    assert (np.diff(hist) <= 0).all()
    assert hist[-1] < hist[0]
    np.testing.assert_allclose(hist[0], h_o[0], rtol=5e-4)  # V includes the outward box margin
    np.testing.assert_allclose(hist, h_o, rtol=2e-3)
    # the installed best slopes reproduce the best objective
    V = r.objective()
    np.testing.assert_allclose(V.sum(), hist[-1], rtol=1e-6)


def test_refinement_from_perturbed_start_matches_oracle():
    # From slopes 0.05 off the chord point, refinement lowers V by 15-20 % (the chord point itself is
    # already a local minimum, see the design notes); the device's V history follows the oracle's
    # projected gradient from the same start.
    p = wl.cartpole_diff()
    sub = p.subset(np.arange(0, p.D, 16))
    a0 = orc.chord_alpha(sub)
    start = torch.where(a0 > 0, (a0 + 0.05).clamp(0.0, 1.0), a0).float().double()
    steps, lr = 20, 0.1
    ref = orc.optimize_slopes(sub, steps, lr, 0.0, alpha0=start)
    r = _api().Reach(0).load(sub)
    r.set_alpha(start.float().numpy())
    hist = r.optimize(steps, lr, 0.0)
    h_o = np.array(ref["V_hist"])
    assert h_o[-1] < 0.9 * h_o[0]
    assert (np.diff(hist) <= 0).all()
    np.testing.assert_allclose(hist, h_o, rtol=1e-3)


# Wide controllers: the forward-with-tape and reverse kernels keep their per-domain working set in
# per-CTA slabs of global memory when it does not fit in shared memory.

def test_dalpha_wide_controller():
    p = wl.random_problem(65, [4, 300, 300, 2], D=6, H=3, eps=0.2)
    alpha = _interior_alpha(p, 4)
    _, ga_o, _ = orc.value_and_grad(p, alpha)
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, _ = r.backward()
    _grad_close(ga, ga_o.numpy())


def test_dalpha_wide_controller_three_hidden_ragged():
    # three hidden layers of widths that are no multiple of the 128 x 128 tiles or the 32-wide K
    # slices of the slab kernels' shared-memory products
    p = wl.random_problem(66, [3, 200, 150, 130, 2], D=4, H=3, eps=0.2)
    alpha = _interior_alpha(p, 6)
    _, ga_o, _ = orc.value_and_grad(p, alpha)
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, _ = r.backward()
    _grad_close(ga, ga_o.numpy())


def test_branch12_gradients_subset():
    import dataclasses
    p = dataclasses.replace(wl.quadrotor_branch(only=np.arange(4)), H=4)
    rng = np.random.default_rng(5)
    p.beta = rng.uniform(0.0, 0.005, size=p.splits.nnz).astype(np.float32).astype(np.float64)
    alpha = _interior_alpha(p, 5)
    _, ga_o, gb_o = orc.value_and_grad(p, alpha, torch.as_tensor(p.beta))
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, gb = r.backward()
    _grad_close(ga, ga_o.numpy())
    if p.splits.nnz:
        _grad_close(gb, gb_o.numpy())


def test_large16_gradient_subset():
    import dataclasses
    p = dataclasses.replace(wl.large16().subset(np.arange(2)), H=3)
    alpha = _interior_alpha(p, 6)
    _, ga_o, _ = orc.value_and_grad(p, alpha)
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    ga, _ = r.backward()
    _grad_close(ga, ga_o.numpy())


def test_large16_refinement_subset():
    import dataclasses
    p = dataclasses.replace(wl.large16().subset(np.arange(0, 262144, 65536)), H=3)
    # the chord slopes sit at a kink of every unstable neuron's intercept, where the subgradient
    # need not descend: start both sides from perturbed slopes
    alpha = _interior_alpha(p, 7)
    steps, lr = 3, 1.0
    ref = orc.optimize_slopes(p, steps, lr, 0.0, alpha0=alpha)
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    hist = r.optimize(steps, lr, 0.0)
    h_o = np.array(ref["V_hist"])
    assert (np.diff(hist) <= 0).all()
    assert hist[-1] < hist[0]
    np.testing.assert_allclose(hist, h_o, rtol=2e-3)
