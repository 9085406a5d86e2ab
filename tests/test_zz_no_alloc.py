"""The allocation-free slope gradient (dr_slope_gradient_static).

Some callers may not allocate device memory at all: code that runs inside a memory pool it manages
itself, or a control loop with a deadline, where a cudaMalloc/cudaFree can synchronise the device
and stall it.  Such callers hand in every input and output buffer and the library uses a fixed
scratch array reserved when it is loaded.  This test checks, through the C ABI, that the gradient
it returns agrees with the context-based dr_backward, on two calls in a row (the shared scratch is
reused), and that an oversized problem is refused before any device work.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _args(lib_mod, p, dev_bufs):
    a = lib_mod.dr_static_args()
    a.L = p.L
    for i, w in enumerate(p.widths):
        a.widths[i] = w
    for name in ("W", "b", "A", "B", "e", "lo", "hi", "alpha", "dalpha", "V"):
        setattr(a, name, ctypes.c_void_p(dev_bufs[name].data_ptr()))
    a.D = p.D
    a.H = p.H
    a.margin_rho = 0.0
    a.stream = None
    return a


def test_static_gradient_matches_backward_on_two_calls():
    from paper_2605_25346_b300 import _lib, api
    from paper_2605_25346_b300 import workloads as wl

    p = wl.random_problem(71, [3, 20, 16, 2], D=24, H=5, eps=0.3)
    r = api.Reach(0).load(p)
    chord = r.get_alpha()
    alpha = np.clip(chord + 0.1 * (np.random.default_rng(0).random(chord.shape) - 0.5), 0.05, 0.95).astype(np.float32)
    r.set_alpha(alpha)
    ref, _ = r.backward()
    r.bounds(on_device=False)
    V_ref = r.objective()
    r.close()

    dev = "cuda:0"
    f32 = dict(dtype=torch.float32, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    bufs = {
        "W": torch.cat([torch.as_tensor(w, **f32).reshape(-1) for w in p.W]),
        "b": torch.cat([torch.as_tensor(x, **f32).reshape(-1) for x in p.b]),
        "A": torch.as_tensor(p.A, **f64).contiguous(),
        "B": torch.as_tensor(p.B, **f64).contiguous(),
        "e": torch.as_tensor(p.e, **f64).contiguous(),
        "lo": torch.as_tensor(p.lo, **f64).contiguous(),
        "hi": torch.as_tensor(p.hi, **f64).contiguous(),
        "alpha": torch.as_tensor(alpha, **f32).contiguous(),
        "dalpha": torch.empty(alpha.shape, **f32),
        "V": torch.empty(p.D, **f64),
    }
    lib = _lib.load()
    args = _args(_lib, p, bufs)
    scale = np.abs(ref).max()
    for _call in range(2):
        bufs["dalpha"].fill_(float("nan"))
        bufs["V"].fill_(float("nan"))
        torch.cuda.synchronize()
        rc = lib.dr_slope_gradient_static(ctypes.byref(args))
        assert rc == _lib.DR_OK, lib.dr_last_error(None)
        torch.cuda.synchronize()
        got = bufs["dalpha"].cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-4 * scale
        # the objective at these slopes, as the context-based bound pass reports it
        V = bufs["V"].cpu().numpy()
        np.testing.assert_allclose(V, V_ref, rtol=1e-5)


def test_static_gradient_rejects_oversized_problem():
    from paper_2605_25346_b300 import _lib
    from paper_2605_25346_b300 import workloads as wl

    p = wl.random_problem(72, [3, 8, 2], D=4, H=3)
    dev = "cuda:0"
    dummy = {k: torch.zeros(4, dtype=torch.float64, device=dev) for k in ("W", "b", "A", "B", "e", "lo", "hi", "alpha",
                                                                          "dalpha", "V")}
    lib = _lib.load()
    args = _args(_lib, p, dummy)
    args.D = 10 ** 7
    rc = lib.dr_slope_gradient_static(ctypes.byref(args))
    assert rc == _lib.DR_ERR_SHAPE
    assert b"static limit" in lib.dr_last_error(None)
