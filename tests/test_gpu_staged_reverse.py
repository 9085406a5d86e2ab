"""The staged reverse sweep: the keep-mode forward pass of a chunk, the per-domain reverse kernels
and the reverse chain GEMM (tcgen05 3xTF32 with the reverse epilogue for targets whose width is a
multiple of 32, CUDA cores otherwise), against the FP64 oracle's reverse-mode gradients (pinned by
finite differences on the CPU) at 1e-4 of the largest entry, and against the fused reverse kernels.

Small controllers are sent through it with set_options(reverse=2); wide ones take it by default
(tests/test_gpu_adjoint.py covers those workloads)."""
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
    return (a0 + 0.2 * (torch.rand(a0.shape, generator=g, dtype=torch.float64) - 0.5)).clamp(0.05, 0.95).float().double()


def _grad_close(g, o, tol=GTOL):
    o = np.asarray(o, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    scale = max(np.abs(o).max(), 1e-30)
    err = np.abs(g - o) / scale
    assert err.max() <= tol, f"gradient max err {err.max():.3e} (scale {scale:.3e})"


def _reach(p, alpha=None, precision=0, reverse=2, chunk=0, stream=None):
    r = _api().Reach(0, stream=stream).load(p, precision=precision)
    r.set_options(precision=precision, reverse=reverse, chunk=chunk)
    if alpha is not None:
        r.set_alpha(alpha.float().numpy())
    return r


# widths: targets on the tensor cores with 32-row segments (64, 96, 128: uniform and domain-straddling
# 128-row tiles, ragged columns) and with one segment per domain (2, 8 or 16 rows), targets on CUDA
# cores (3 rows; 40 and 72 rows), and four hidden layers
@pytest.mark.parametrize("widths", [[4, 64, 64, 2], [3, 96, 64, 128, 3], [3, 64, 50, 96, 2], [3, 40, 72, 2],
                                    [2, 32, 64, 32, 64, 2], [3, 64, 64, 8], [4, 16, 64, 16, 4]])
@pytest.mark.parametrize("precision", [0, 1])
def test_staged_dalpha_matches_oracle(widths, precision):
    p = wl.random_problem(71, widths, D=10, H=4, eps=0.25)
    alpha = _interior_alpha(p, 0)
    _, ga_o, _ = orc.value_and_grad(p, alpha)
    r = _reach(p, alpha, precision)
    ga, _ = r.backward()
    _grad_close(ga, ga_o.numpy())
    # the keep-mode forward pass leaves the pass's outputs, as dr_compute_bounds does
    V = r.objective()
    r.close()
    V_o = orc.reach(p, alpha=alpha, mode=orc.MODE_USER)["V"].numpy()
    np.testing.assert_allclose(V, V_o, rtol=5e-4)  # V includes the outward box margin


def test_staged_dbeta_with_splits():
    p = wl.random_problem(72, [6, 64, 96, 3], D=16, H=5, eps=0.2)
    rng = np.random.default_rng(7)
    p.splits = wl.branch_splits(p, rng, max_k=6)
    p.beta = rng.uniform(0.05, 0.5, size=p.splits.nnz).astype(np.float32).astype(np.float64)
    alpha = _interior_alpha(p, 1)
    _, ga_o, gb_o = orc.value_and_grad(p, alpha, torch.as_tensor(p.beta))
    r = _reach(p, alpha)
    ga, gb = r.backward()
    r.close()
    assert p.splits.nnz > 20
    _grad_close(ga, ga_o.numpy())
    _grad_close(gb, gb_o.numpy())


def test_staged_upstream_and_shift_gradients():
    # DT neural dynamics with planned inputs: dV/d(centre shift) per step (its action rows are
    # dV/du_t), under random upstream weights of the bounds
    rng = np.random.default_rng(4)
    n, k = 4, 2
    W, b = wl.mlp(rng, [n + k, 64, 96, n], f32=True, out_gain=0.5)
    xhat = rng.uniform(-1, 1, size=(6, n))
    p = wl.neural_dynamics("dt-staged", W, b, n, k, xhat - 0.05, xhat + 0.05, rng.uniform(-1, 1, size=(6, 3, k)),
                           residual=True)
    alpha = _interior_alpha(p, 2)
    wlo = rng.normal(size=(p.D, p.H + 1, p.n))
    whi = rng.normal(size=(p.D, p.H + 1, p.n))
    a = alpha.clone().requires_grad_(True)
    res = orc.reach(p, alpha=a, mode=orc.MODE_USER)
    (res["lo"] * torch.as_tensor(wlo) + res["hi"] * torch.as_tensor(whi)).sum().backward()
    r = _reach(p, alpha)
    ga, _ = r.backward(wlo=wlo, whi=whi)
    _grad_close(ga, a.grad.numpy())
    _, g_o = orc.value_and_shift_grad(p, alpha=alpha)
    r.backward()
    g = r.shift_gradient()
    r.close()
    _grad_close(g, g_o.numpy())
    assert np.abs(g[:, :p.H, n:]).max() > 1e-3 * np.abs(g_o.numpy()).max()


def test_staged_matches_fused_reverse_and_chunks():
    p = wl.random_problem(73, [5, 128, 128, 128, 4], D=12, H=4, eps=0.2)
    alpha = _interior_alpha(p, 3)
    r = _reach(p, alpha, reverse=1)
    g_fused, _ = r.backward()
    r.close()
    r = _reach(p, alpha)
    g_one, _ = r.backward()
    r.close()
    r = _reach(p, alpha, chunk=5)  # three chunks, the last one short
    g_chunked, _ = r.backward()
    r.close()
    _grad_close(g_one, g_fused, tol=2e-5)
    # per-domain arithmetic does not depend on how the domains are chunked
    np.testing.assert_allclose(g_chunked, g_one, rtol=0, atol=1e-6 * np.abs(g_one).max())


def test_staged_refinement_matches_oracle():
    p = wl.random_problem(74, [4, 64, 96, 2], D=8, H=4, eps=0.25)
    alpha = _interior_alpha(p, 4)
    steps, lr = 4, 0.5
    ref = orc.optimize_slopes(p, steps, lr, 0.0, alpha0=alpha)
    r = _reach(p, alpha, stream=torch.cuda.Stream())  # a stream of its own: the steps can be captured
    hist = r.optimize(steps, lr, 0.0)
    replays = r.graph_replays()
    r.close()
    h_o = np.array(ref["V_hist"])
    assert (np.diff(hist) <= 0).all()
    np.testing.assert_allclose(hist, h_o, rtol=2e-3)
    assert replays >= steps - 1  # steps after the first replayed from one captured step
