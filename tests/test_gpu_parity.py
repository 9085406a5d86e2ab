"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (floating point): |gpu - oracle| <= 1e-5 * max(|o_lo|, |o_hi|, o_hi - o_lo) for every
domain, step and coordinate.  Soundness against the oracle: the box computed on the GPU is never tighter than the
oracle's, i.e. g_lo <= o_lo and g_hi >= o_hi (the reported boxes carry the outward margin 2^-18 of
their L1 magnitude, sized to cover the FP32 pass's deviation from FP64).  Status words are compared
exactly.
"""
import numpy as np
import pytest
import torch

from oracle import reach as orc
from paper_2605_25346_b300 import workloads as wl

pytestmark = pytest.mark.gpu

RTOL = 1e-5
RHO = 0.0  # no slack: the box computed on the GPU must enclose the oracle's box


def _api():
    from paper_2605_25346_b300 import api
    return api


def gpu_bounds(prob, mode=None, alpha=None, on_device=True, rho=None, precision=0, chunk=0, tuning=0):
    api = _api()
    r = api.Reach(0)
    r.load(prob, mode=mode, rho=rho, precision=precision)
    if chunk or tuning:
        r.set_options(mode=prob.mode if mode is None else mode, precision=precision, rho=rho, chunk=chunk, tuning=tuning)
    if alpha is not None:
        r.set_alpha(alpha)
    out = r.bounds(on_device=on_device)
    V = r.objective()
    res = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
    res["V"] = V
    r.close()
    return res


def compare(prob, g, o, rtol=RTOL, rho=RHO, check_hull=True):
    olo, ohi = o["lo"].detach().numpy(), o["hi"].detach().numpy()
    glo, ghi = g["lo"], g["hi"]
    scale = np.maximum(np.maximum(np.abs(olo), np.abs(ohi)), ohi - olo)
    err = np.maximum(np.abs(glo - olo), np.abs(ghi - ohi)) / np.maximum(scale, 1e-300)
    assert np.isfinite(glo).all() and np.isfinite(ghi).all()
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= rtol, f"max rel err {err.max():.3e} at {worst}"
    mag = np.abs(olo) + np.abs(ohi)
    assert (glo <= olo + rho * mag).all(), "GPU lower bound tighter than the oracle beyond the margin"
    assert (ghi >= ohi - rho * mag).all(), "GPU upper bound tighter than the oracle beyond the margin"
    # the method's status bits (non-finite, infeasible); DR_STATUS_MARGIN is the GPU's own numerics flag
    np.testing.assert_array_equal(g["status"].astype(np.int64) & 3, o["status"].numpy())
    assert not (g["status"].astype(np.int64) & 4).any(), "calibrated margin's range left on a parity case"
    # V sums box widths, which carry the outward box margin (about 2 * 2^-18 * |centre| per entry;
    # for point boxes the widths are nothing but the margin)
    oV = o["V"].detach().numpy()
    vmag = (np.abs(olo) + np.abs(ohi))[:, 1:, :].sum(axis=(1, 2))
    assert (np.abs(g["V"] - oV) <= 5e-4 * np.abs(oV) + 2.0 ** -16 * vmag).all()
    if check_hull:
        hl, hh = o["hull_lo"].numpy(), o["hull_hi"].numpy()
        hs = np.maximum(np.maximum(np.abs(hl), np.abs(hh)), hh - hl)  # the same per-entry scale as the boxes
        assert (np.abs(g["hull_lo"] - o["hull_lo"].numpy()) <= rtol * hs).all()
        assert (np.abs(g["hull_hi"] - o["hull_hi"].numpy()) <= rtol * hs).all()
    return float(err.max())


def test_double_integrator_adaptive():
    p = wl.double_integrator_tiny()
    compare(p, gpu_bounds(p), orc.reach(p))


def test_quad6_all_domains():
    p = wl.quad6_batched()
    compare(p, gpu_bounds(p), orc.reach(p))


def test_cartpole_all_domains():
    p = wl.cartpole_diff()
    compare(p, gpu_bounds(p), orc.reach(p))


SHAPES = [[5, 37, 23, 3], [3, 16, 2], [7, 96, 96, 96, 2], [2, 128, 128, 1], [4, 1, 1, 1]]
# The adaptive slope (1 if u >= -l else 0) jumps at u = -l, so FP32 rounding may pick the other slope
# there; it is compared only on nets with at most two hidden layers, where no neuron sits that close.
CASES = [(w, m) for w in SHAPES for m in (orc.MODE_CHORD, orc.MODE_ZERO)] + \
        [(w, orc.MODE_ADAPTIVE) for w in SHAPES if len(w) <= 4]


@pytest.mark.parametrize("widths,mode", CASES)
def test_random_shapes(widths, mode):
    p = wl.random_problem(hash((tuple(widths), mode)) % 1000, widths, D=77, H=5, eps=0.15, mode=mode)
    compare(p, gpu_bounds(p), orc.reach(p))


def test_user_slopes():
    p = wl.random_problem(3, [4, 33, 17, 2], D=40, H=6, eps=0.3)
    g = torch.Generator().manual_seed(0)
    alpha = torch.rand(p.D, p.H, p.hidden, generator=g, dtype=torch.float64)
    alpha32 = alpha.float().numpy()
    o = orc.reach(p, alpha=torch.as_tensor(alpha32, dtype=torch.float64), mode=orc.MODE_USER)
    compare(p, gpu_bounds(p, alpha=alpha32), o)


def test_chord_slopes_roundtrip_bitwise():
    api = _api()
    p = wl.random_problem(4, [3, 20, 20, 2], D=16, H=5, eps=0.3)
    r = api.Reach(0).load(p)
    ref = r.bounds(on_device=False)
    a = r.get_alpha()
    r.set_alpha(a)
    out = r.bounds(on_device=False)
    np.testing.assert_array_equal(ref["lo"], out["lo"])
    np.testing.assert_array_equal(ref["hi"], out["hi"])


def _with_splits(p, seed, beta_scale):
    rng = np.random.default_rng(seed)
    p.splits = wl.branch_splits(p, rng, max_k=6)
    p.beta = rng.uniform(0, beta_scale, size=p.splits.nnz) if beta_scale > 0 else np.zeros(p.splits.nnz)
    p.beta = p.beta.astype(np.float32).astype(np.float64)
    return p


@pytest.mark.parametrize("beta_scale", [0.0, 0.5])
def test_split_domains(beta_scale):
    p = _with_splits(wl.random_problem(8, [6, 40, 40, 3], D=64, H=6, eps=0.2), 1, beta_scale)
    assert p.splits.nnz > 50
    compare(p, gpu_bounds(p), orc.reach(p))


# Launch variants of the bounds-only pass, forced through dr_options.tuning = 2 + v: v = 0..2 one warp
# per domain (16, 8, 4 warps per CTA; two hidden layers), v = 3 several domains per CTA.
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_launch_variants_on_workloads(variant):
    for p in (wl.double_integrator_tiny(), wl.quad6_batched(), wl.cartpole_diff()):
        compare(p, gpu_bounds(p, tuning=2 + variant), orc.reach(p))


@pytest.mark.parametrize("variant,widths,mode", [(v, w, m) for v in (0, 2, 3) for w, m in (
    ([5, 37, 23, 3], orc.MODE_CHORD), ([2, 128, 128, 1], orc.MODE_ZERO), ([4, 1, 1, 1], orc.MODE_ADAPTIVE))] +
    [(2, [8, 100, 60, 8], orc.MODE_CHORD)])  # 16 warps of this width exceed shared memory; 4 fit
def test_launch_variants_random_shapes(variant, widths, mode):
    p = wl.random_problem(hash((tuple(widths), mode, 7)) % 1000, widths, D=45, H=5, eps=0.15, mode=mode)
    compare(p, gpu_bounds(p, tuning=2 + variant), orc.reach(p))


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("beta_scale", [0.0, 0.5])
def test_launch_variants_split_domains(variant, beta_scale):
    p = _with_splits(wl.random_problem(8, [6, 40, 40, 3], D=64, H=6, eps=0.2), 1, beta_scale)
    compare(p, gpu_bounds(p, tuning=2 + variant), orc.reach(p))


def test_launch_variant_user_slopes():
    p = wl.random_problem(3, [4, 33, 17, 2], D=40, H=6, eps=0.3)
    g = torch.Generator().manual_seed(0)
    alpha32 = torch.rand(p.D, p.H, p.hidden, generator=g, dtype=torch.float64).float().numpy()
    o = orc.reach(p, alpha=torch.as_tensor(alpha32, dtype=torch.float64), mode=orc.MODE_USER)
    compare(p, gpu_bounds(p, alpha=alpha32, tuning=2), o)


def test_launch_variant_that_does_not_fit_is_an_error():
    api = _api()
    p = wl.random_problem(9, [3, 16, 16, 16, 2], D=4, H=2)  # three hidden layers: no warp variant
    r = api.Reach(0).load(p)
    with pytest.raises(RuntimeError, match="does not fit"):
        r.set_options(mode=p.mode, tuning=2)
        r.bounds()
    r.close()


def test_host_and_device_outputs_identical():
    p = wl.random_problem(5, [4, 24, 24, 2], D=33, H=4)
    a = gpu_bounds(p, on_device=True)
    b = gpu_bounds(p, on_device=False)
    np.testing.assert_array_equal(a["lo"], b["lo"])
    np.testing.assert_array_equal(a["hi"], b["hi"])


def test_gpu_bounds_contain_trajectories():
    p = wl.quad6_batched()
    sub = p.subset(np.arange(0, p.D, 16))
    g = gpu_bounds(sub)
    dom, xs, _ = wl.sample_trajectories(sub, 10000, 7)
    assert ((xs >= g["lo"][dom]) & (xs <= g["hi"][dom])).all()


def test_empty_domain_set():
    api = _api()
    p = wl.random_problem(6, [3, 8, 2], D=4, H=3)
    q = p.subset(np.arange(0))
    r = api.Reach(0).load(q)
    out = r.bounds(on_device=False)
    assert out["lo"].shape == (0, 4, 3)


def test_invalid_arguments_are_errors():
    api = _api()
    from paper_2605_25346_b300 import _lib
    p = wl.random_problem(6, [3, 8, 2], D=4, H=3)
    bad = p.subset(np.arange(4))
    bad.lo = bad.lo.copy()
    bad.lo[1, 0] = np.nan
    with pytest.raises(_lib.DiffReachError) as e:
        api.Reach(0).load(bad)
    assert e.value.code == _lib.DR_ERR_NONFINITE
    inv = p.subset(np.arange(4))
    inv.lo, inv.hi = inv.hi.copy(), inv.lo.copy()
    with pytest.raises(_lib.DiffReachError) as e:
        api.Reach(0).load(inv)
    assert e.value.code == _lib.DR_ERR_ARG
    sp = _with_splits(p.subset(np.arange(4)), 0, 0.0)
    sp.splits.layer = sp.splits.layer.copy()
    if sp.splits.nnz:
        sp.splits.layer[0] = 2  # not a hidden layer of a 2-layer controller
        with pytest.raises(_lib.DiffReachError) as e:
            api.Reach(0).load(sp)
        assert e.value.code == _lib.DR_ERR_ARG
    r = api.Reach(0)
    r.set_options(mode=None, mem_cap=1024)
    with pytest.raises(_lib.DiffReachError) as e:
        r.load(wl.quad6_batched())
    assert e.value.code == _lib.DR_ERR_OOM


# ---- staged path (per-phase kernels over domain chunks; wide controllers) -----------------------
STAGED = 1  # DR_PREC_SIMT: staged path with the CUDA-core chain GEMM


@pytest.mark.parametrize("name", ["quad6_batched", "cartpole_diff"])
def test_staged_path_narrow_workloads(name):
    p = wl.WORKLOADS[name]()
    sub = p.subset(np.arange(0, p.D, 4))
    compare(sub, gpu_bounds(sub, precision=STAGED, chunk=97), orc.reach(sub))


@pytest.mark.parametrize("widths,mode", [([5, 37, 23, 3], orc.MODE_CHORD), ([7, 96, 96, 96, 2], orc.MODE_ZERO),
                                         ([3, 70, 130, 65, 2], orc.MODE_CHORD)])
def test_staged_path_random_shapes(widths, mode):
    p = wl.random_problem(hash(tuple(widths)) % 1000, widths, D=45, H=4, eps=0.15, mode=mode)
    compare(p, gpu_bounds(p, precision=STAGED, chunk=16), orc.reach(p))


@pytest.mark.parametrize("beta_scale", [0.0, 0.005])
def test_branch12_split_domains(beta_scale):
    idx = np.arange(0, 65536, 1021)[:64]
    p = wl.quadrotor_branch(only=idx)
    if beta_scale > 0:
        p.beta = np.random.default_rng(5).uniform(0, beta_scale, size=p.splits.nnz).astype(np.float32).astype(np.float64)
    assert p.splits.nnz > 500
    # Arbitrary (unoptimised) multipliers widen the tube: at 0.5 the dual bound diverges over 30 steps,
    # at 0.02 plain FP32 arithmetic already drifts 8e-6 from FP64 by the last step; 0.005 stays at 2e-6.
    compare(p, gpu_bounds(p), orc.reach(p))


def test_large16_subset():
    p = wl.large16()
    sub = p.subset(np.arange(0, p.D, p.D // 8))
    compare(sub, gpu_bounds(sub), orc.reach(sub))


# ---- staged path with the tcgen05 3xTF32 chain (the default for wide controllers) --------------
TCORE = 2  # DR_PREC_TF32X3


@pytest.mark.parametrize("name", ["quad6_batched", "cartpole_diff"])
def test_tensor_core_path_narrow_workloads(name):
    p = wl.WORKLOADS[name]()
    sub = p.subset(np.arange(0, p.D, 4))
    compare(sub, gpu_bounds(sub, precision=TCORE, chunk=257), orc.reach(sub))


# [20, ...]: more than 16 states, so the last chain level is not folded into the GEMM epilogue;
# [16, 48, 130, 90, 4]: exactly 16 states with a 48-wide first layer (32-column epilogue tiles).
@pytest.mark.parametrize("widths,mode", [([5, 37, 23, 3], orc.MODE_CHORD), ([7, 96, 96, 96, 2], orc.MODE_ZERO),
                                         ([3, 70, 130, 65, 2], orc.MODE_CHORD), ([9, 300, 40, 5], orc.MODE_CHORD),
                                         ([20, 64, 48, 40, 3], orc.MODE_CHORD), ([16, 48, 130, 90, 4], orc.MODE_CHORD)])
def test_tensor_core_path_random_shapes(widths, mode):
    p = wl.random_problem(hash(tuple(widths)) % 1000 + 1, widths, D=45, H=4, eps=0.15, mode=mode)
    compare(p, gpu_bounds(p, precision=TCORE, chunk=16), orc.reach(p))


# 128 domains of 160-row chain levels: R = 20,480 stacked rows in 128-row tiles, at least two
# 128 x 128 tiles per SM, so the chain levels run in the persistent GEMM (epilogues overlapped with
# the next tile).  160 rows per domain leave most row tiles spanning two domains (per-row slopes).
# n = 4 folds the last level into the epilogue (W_1 product); n = 20 ends on a plain GEMM.
# 256-wide levels on 80 domains: 160 row tiles x 2 column tiles, also persistent.
@pytest.mark.parametrize("widths,D", [([4, 160, 160, 160, 160, 2], 128), ([20, 160, 160, 160, 2], 128),
                                      ([4, 256, 256, 256, 256, 2], 80), ([20, 256, 256, 256, 2], 80)])
def test_tensor_core_path_persistent_gemm(widths, D):
    p = wl.random_problem(hash(tuple(widths)) % 1000 + 2, widths, D=D, H=2, eps=0.15, mode=orc.MODE_CHORD)
    compare(p, gpu_bounds(p, precision=TCORE, chunk=D), orc.reach(p))


# The staged tensor-core path in the launch configuration bench.py times for the two wide workloads
# (16-512x4-8: the first 2048 of 262,144 sub-boxes, H = 50, two lanes of 1024 domains, persistent
# chain GEMMs; 12-256x3-4: 4096 of the 65,536 branch domains, H = 30), checked on sampled domains
# that span both lanes and the chunk edges, each against the oracle run on that domain alone
# (domains are independent through every step).
def _sampled(prob, g, idx):
    return {"lo": g["lo"][idx], "hi": g["hi"][idx], "status": g["status"][idx], "V": g["V"][idx]}


def test_large16_bench_configuration_sampled():
    p = wl.large16().subset(np.arange(2048))
    g = gpu_bounds(p)
    idx = np.array([0, 1, 511, 1023, 1024, 1535, 2047])
    o = orc.reach(p.subset(idx))
    compare(p.subset(idx), _sampled(p, g, idx), o, check_hull=False)
    # soundness headroom over the 50 steps: the GPU machines enclose the oracle's with at least a quarter
    # of the outward margin (2^-18 of the entry's magnitude) to spare
    olo, ohi = o["lo"].numpy(), o["hi"].numpy()
    m = 2.0 ** -18 * np.maximum(np.abs(olo), np.abs(ohi))
    used = 1.0 - np.minimum((olo - g["lo"][idx]) / m, (g["hi"][idx] - ohi) / m)[:, 1:]
    assert used.max() <= 0.75, f"outward margin used up to {used.max():.2f}"


def test_branch12_bench_configuration_sampled():
    p = wl.quadrotor_branch(only=np.arange(4096))
    g = gpu_bounds(p)
    idx = np.array([0, 5, 1023, 2047, 2048, 3071, 4090, 4095])
    compare(p.subset(idx), _sampled(p, g, idx), orc.reach(p.subset(idx)), check_hull=False)


# ---- degenerate cases of the method, on the fused and on the staged tensor-core path -----------
PATHS = [0, TCORE]  # DR_PREC_AUTO (fused kernels for these sizes), DR_PREC_TF32X3 (staged)


@pytest.mark.parametrize("precision", PATHS)
def test_point_boxes(precision):
    # lo == hi: P = 0, every neuron stable, the bounds are the single trajectory (plus the margins);
    # mixed with ordinary boxes in the same launch
    p = wl.random_problem(21, [4, 48, 40, 2], D=24, H=6, eps=0.2)
    p.hi = p.hi.copy()
    p.hi[::2] = p.lo[::2]
    compare(p, gpu_bounds(p, precision=precision, chunk=16 if precision else 0), orc.reach(p))


@pytest.mark.parametrize("precision", PATHS)
def test_linear_controller(precision):
    # L = 1: no ReLU, the controller is affine and the TM is exact (no relaxation, no chain)
    p = wl.random_problem(22, [5, 3], D=16, H=8, eps=0.2)
    compare(p, gpu_bounds(p, precision=precision), orc.reach(p))


@pytest.mark.parametrize("precision", PATHS)
def test_dead_and_saturated_layers(precision):
    # biases below / above the first layer's pre-activation range on every step: all of its neurons
    # inactive (the controller is a constant) or all active (no relaxation in that layer).  Shifts of
    # +-50 put intermediate values ~300x above the box scale, where the calibrated box margin no
    # longer covers the FP32 / 3xTF32 rounding (a known limit of the calibrated margin).
    for shift in (-6.0, 6.0):
        p = wl.random_problem(23, [4, 40, 36, 2], D=12, H=5, eps=0.1)
        p.b = [bb.copy() for bb in p.b]
        p.b[0] = p.b[0] + shift
        compare(p, gpu_bounds(p, precision=precision), orc.reach(p))


@pytest.mark.parametrize("precision", PATHS)
def test_margin_status_flags_large_intermediate_values(precision):
    # first-layer biases shifted by +-50: rows sum terms several hundred times the Taylor model's scale,
    # beyond the calibrated range of the default margin -> DR_STATUS_MARGIN on the affected domains
    for shift in (-50.0, 50.0):
        p = wl.random_problem(23, [4, 40, 36, 2], D=12, H=5, eps=0.1)
        p.b = [bb.copy() for bb in p.b]
        p.b[0] = p.b[0] + shift
        g = gpu_bounds(p, precision=precision)
        assert (g["status"].astype(np.int64) & 4).any()


@pytest.mark.parametrize("precision", PATHS)
def test_single_domain_single_step(precision):
    p = wl.random_problem(24, [3, 33, 2], D=1, H=1, eps=0.3)
    compare(p, gpu_bounds(p, precision=precision), orc.reach(p))


def test_large16_all_sub_boxes_one_step_sampled():
    # every one of the 262,144 sub-boxes in one call (the largest domain count of the workloads; many
    # lane chunks of the staged path), one step, checked on domains spread over the whole range
    import dataclasses
    p = dataclasses.replace(wl.large16(), H=1)
    g = gpu_bounds(p)
    idx = np.array([0, 1, 65535, 131072, 199999, 262142, 262143])
    compare(p.subset(idx), _sampled(p, g, idx), orc.reach(p.subset(idx)), check_hull=False)


def test_tensor_core_bounds_contain_trajectories():
    # soundness of the staged 3xTF32 path itself (not only agreement with the oracle): simulated
    # trajectories from sub-boxes of the 16-512x4-8 workload stay inside the GPU machines
    import dataclasses
    p = dataclasses.replace(wl.large16().subset(np.arange(0, 262144, 32768)), H=10)
    g = gpu_bounds(p)
    dom, xs, _ = wl.sample_trajectories(p, 4000, 11)
    assert ((xs >= g["lo"][dom]) & (xs <= g["hi"][dom])).all()


# ---- the tensor-core GEMM's launch shapes: each shape the autotuner may pick, forced for every GEMM
# of the staged path (dr_options.tuning = 100 + g: 1 persistent 128 x 128, 2 / 3 / 4 one 128 x 128 /
# 64 / 32 tile per CTA), and the autotuner itself (tuning = 0) with its report
@pytest.mark.parametrize("shape", [1, 2, 3, 4])
def test_tensor_core_gemm_launch_shapes(shape):
    p = wl.random_problem(77, [6, 256, 256, 256, 3], D=48, H=2, eps=0.15)
    compare(p, gpu_bounds(p, precision=TCORE, chunk=24, tuning=100 + shape), orc.reach(p))


def test_gemm_autotuner_picks_and_reports():
    api = _api()
    p = wl.random_problem(78, [6, 256, 256, 200, 3], D=64, H=2, eps=0.15)
    compare(p, gpu_bounds(p, precision=TCORE), orc.reach(p))
    rep = api.gemm_tuning_report()
    assert "epi1" in rep and "epi2" in rep and "variant" in rep, rep
