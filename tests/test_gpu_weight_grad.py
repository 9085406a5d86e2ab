"""dV/dW_l and dV/db_l of the controller from the CUDA reverse sweep (dr_get_weight_gradient) vs the
FP64 oracle's reverse-mode gradient (value_and_weight_grad, pinned by finite differences).

The certified-training loss of Sec. V-A differentiates the tube proxy with respect to the model's
parameters; these tests cover the fused kernels' shapes (one and several hidden layers, a
single-neuron layer), split constraints with multipliers, the global-memory slab kernels of wide
controllers, CHORD slopes (the slopes themselves depend on the pre-activation bounds), and a sweep
cut into several launches.

Tolerance: per layer, |g_gpu - g_oracle| <= 1e-4 * max|g_oracle| over all layers' weights and
biases (the same bar as the slope gradients; the GPU forward runs in FP32 with the outward margin,
the oracle in FP64 without it), and 1e-3 of the layer's own largest entry.
"""
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


def _check(gW, gb, oW, ob):
    oW = [np.asarray(x, dtype=np.float64) for x in oW]
    ob = [np.asarray(x, dtype=np.float64) for x in ob]
    scale = max(max(np.abs(x).max() for x in oW), max(np.abs(x).max() for x in ob))
    assert scale > 0
    for l, (g, o) in enumerate(list(zip(gW, oW)) + list(zip(gb, ob))):
        assert g.shape == o.shape, (l, g.shape, o.shape)
        err = np.abs(g - o)
        assert err.max() <= GTOL * scale, f"entry {l}: max err {err.max():.3e} (scale {scale:.3e})"
        own = max(np.abs(o).max(), 1e-30)
        assert err.max() <= 1e-3 * own or err.max() <= GTOL * scale * 1e-2, \
            f"entry {l}: max err {err.max():.3e} against its own scale {own:.3e}"


def _gpu(p, alpha=None, chunk=0, mode=None):
    r = _api().Reach(0).load(p, mode=mode)
    if alpha is not None:
        r.set_alpha(alpha.float().numpy())
    r.set_options(mode=3 if alpha is not None else mode, chunk=chunk, weight_grad=1)
    r.backward()
    gW, gb = r.weight_gradient()
    r.close()
    return gW, gb


@pytest.mark.parametrize("widths", [[3, 12, 10, 2], [4, 24, 24, 24, 3], [2, 1, 1], [2, 16, 2]])
def test_weight_gradient_matches_oracle(widths):
    p = wl.random_problem(71, widths, D=12, H=4, eps=0.3)
    alpha = _interior_alpha(p, 0)
    _, oW, ob = orc.value_and_weight_grad(p, alpha)
    gW, gb = _gpu(p, alpha)
    _check(gW, gb, oW, ob)


def test_weight_gradient_with_splits():
    p = wl.random_problem(72, [6, 40, 40, 3], D=24, H=5, eps=0.2)
    rng = np.random.default_rng(3)
    p.splits = wl.branch_splits(p, rng, max_k=6)
    p.beta = rng.uniform(0.05, 0.5, size=p.splits.nnz).astype(np.float32).astype(np.float64)
    assert p.splits.nnz > 20
    alpha = _interior_alpha(p, 1)
    _, oW, ob = orc.value_and_weight_grad(p, alpha, torch.as_tensor(p.beta))
    gW, gb = _gpu(p, alpha)
    _check(gW, gb, oW, ob)


def test_weight_gradient_chord_slopes():
    # outside user slopes the slope of each unstable neuron is u / (u - l), a function of the weights too
    p = wl.random_problem(73, [3, 16, 16, 2], D=8, H=3, eps=0.3)
    _, oW, ob = orc.value_and_weight_grad(p)
    gW, gb = _gpu(p)
    _check(gW, gb, oW, ob)


def test_weight_gradient_in_several_launches():
    # 12 domains in launches of at most 5: the slices of each launch add to the same sums
    p = wl.random_problem(74, [3, 12, 10, 2], D=12, H=4, eps=0.3)
    alpha = _interior_alpha(p, 2)
    _, oW, ob = orc.value_and_weight_grad(p, alpha)
    gW, gb = _gpu(p, alpha, chunk=5)
    _check(gW, gb, oW, ob)
    gW1, gb1 = _gpu(p, alpha)
    for x, y in zip(gW + gb, gW1 + gb1):
        np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-12 * max(np.abs(y).max(), 1.0))


def test_weight_gradient_wide_controller_slabs():
    p = wl.random_problem(75, [4, 300, 300, 2], D=4, H=3, eps=0.2)
    alpha = _interior_alpha(p, 4)
    _, oW, ob = orc.value_and_weight_grad(p, alpha)
    gW, gb = _gpu(p, alpha)
    _check(gW, gb, oW, ob)


def test_weight_gradient_requires_the_option():
    from paper_2605_25346_b300 import _lib
    p = wl.random_problem(76, [3, 8, 2], D=2, H=2, eps=0.3)
    r = _api().Reach(0).load(p)
    r.backward()
    with pytest.raises(RuntimeError):
        r.weight_gradient()
    r.set_options(weight_grad=1)
    r.backward()
    gW, gb = r.weight_gradient()
    assert [g.shape for g in gW] == [w.shape for w in p.W] and [g.shape for g in gb] == [x.shape for x in p.b]
    # a new controller invalidates it
    r.load(p)
    with pytest.raises(RuntimeError):
        r.weight_gradient()
    r.close()
    assert _lib.DR_ERR_STATE != 0
