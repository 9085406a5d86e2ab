"""Discrete-time neural dynamics with planned inputs (Alg. 2) and MPC action samples (Sec. V-B), on
the GPU, through per-step offsets of the dynamics over the state augmented by the planned input.

* Bounds: the T-pushing-shaped model 7-96-96-96-5 (state 5, action 2) over 128 random initial boxes
  with their own action sequences, H = 10, on the fused kernels and on the staged tensor-core path,
  element by element against the FP64 oracle (1e-5 relative, zero-slack containment of the oracle's
  box), and 10^4 simulated trajectories inside the GPU machines.
* MPC batching: 1024 action-sequence samples from one initial box in one call.
* Gradients: dV/d(centre shift) per step, whose action rows are dV/du_t, against the oracle's
  reverse-mode gradient (pinned by finite differences on the CPU) at 1e-4 of the largest entry, with
  fixed user slopes; the fused and the global-slab reverse kernels.
"""
import numpy as np
import pytest
import torch

from oracle import reach as orc
from paper_2605_25346_b300 import workloads as wl

from test_gpu_parity import compare, gpu_bounds

pytestmark = pytest.mark.gpu
TCORE = 2


def _api():
    from paper_2605_25346_b300 import api
    return api


@pytest.mark.parametrize("precision", [0, TCORE])
def test_tpush_dt_bounds(precision):
    p = wl.tpush_dt()
    g = gpu_bounds(p, precision=precision, chunk=64 if precision else 0)
    compare(p, g, orc.reach(p))
    dom, xs, _ = wl.sample_trajectories(p, 10000, 31)
    assert ((xs >= g["lo"][dom]) & (xs <= g["hi"][dom])).all()


def test_mpc_samples_in_one_call():
    p = wl.tpush_mpc()
    g = gpu_bounds(p)
    compare(p, g, orc.reach(p))
    # every sample starts from the same state box; the action rows carry each sample's next input
    n = p.meta["state_dims"]
    np.testing.assert_array_equal(g["lo"][:, 0, :n], np.repeat(p.lo[:1, :n], p.D, 0))
    acts_next = p.eoff[:, :-1, n:]
    mag = np.abs(acts_next)
    assert (np.abs(g["lo"][:, 1:p.H, n:] - acts_next) <= 2.0 ** -17 * (mag + 1.0)).all()


def _interior_alpha(p, seed):
    a0 = orc.chord_alpha(p)
    gen = torch.Generator().manual_seed(seed)
    return (a0 + 0.2 * (torch.rand(a0.shape, generator=gen, dtype=torch.float64) - 0.5)).clamp(0.05, 0.95).float().double()


@pytest.mark.parametrize("case", ["tpush", "wide"])
def test_shift_gradient_matches_oracle(case):
    if case == "tpush":
        p = wl.tpush_dt(D=16, H=6)
    else:  # working set beyond shared memory: the reverse kernel runs out of global slabs
        rng = np.random.default_rng(4)
        n, k = 4, 2
        W, b = wl.mlp(rng, [n + k, 300, 300, n], f32=True, out_gain=0.5)
        xhat = rng.uniform(-1, 1, size=(6, n))
        p = wl.neural_dynamics("wide-dt", W, b, n, k, xhat - 0.05, xhat + 0.05, rng.uniform(-1, 1, size=(6, 3, k)),
                               residual=True)
    alpha = _interior_alpha(p, 2)
    _, g_o = orc.value_and_shift_grad(p, alpha=alpha)
    r = _api().Reach(0).load(p)
    r.set_alpha(alpha.float().numpy())
    r.backward()
    g = r.shift_gradient()
    r.close()
    g_o = g_o.numpy()
    scale = np.abs(g_o).max()
    assert scale > 0
    assert np.abs(g - g_o).max() <= 1e-4 * scale, np.abs(g - g_o).max() / scale
    # the action rows (dV/du_t) are not all zero
    n = p.meta["state_dims"]
    assert np.abs(g[:, :p.H, n:]).max() > 1e-3 * scale


def test_offsets_follow_the_boxes_and_horizon():
    api = _api()
    from paper_2605_25346_b300 import _lib
    p = wl.tpush_dt(D=8, H=4)
    r = api.Reach(0).load(p)
    with pytest.raises(_lib.DiffReachError) as e:
        r.shift_gradient()  # no backward yet
    assert e.value.code == _lib.DR_ERR_STATE
    bad = p.eoff.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(_lib.DiffReachError) as e:
        r.set_step_offsets(bad)
    assert e.value.code == _lib.DR_ERR_NONFINITE
    with_off = r.bounds(on_device=False)
    r.set_step_offsets(None)
    without = r.bounds(on_device=False)
    without["V"] = r.objective()
    assert np.abs(with_off["lo"] - without["lo"]).max() > 0.1
    q = wl.tpush_dt(D=8, H=4)
    q.eoff = None
    compare(q, without, orc.reach(q))
    r.close()
