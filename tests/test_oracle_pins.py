"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics, not by the oracle itself.

* hand-derived one-step example (shared-slope relaxation, Sec. IV-C; Thm. 3);
* closed forms: a controller without ReLU, or with every neuron stably active, makes the TM exact,
  so each box equals the exact range of the affine closed loop, attained at the initial box's
  vertices (brute force over all 2^n vertices);
* interval arithmetic: with zero slopes and one hidden layer without stably-active neurons the
  first box equals plain interval propagation exactly; with zero slopes the bounds are never
  looser than interval propagation at any depth or step;
* brute force: simulated trajectories stay inside every bound (soundness, Thm. 2/3), including
  split domains with arbitrary beta >= 0 (trajectories that satisfy the splits);
* refinement: keep-best projected gradient never increases V; zero slopes are inclusion-monotone
  under input splitting at the first step;
* derivatives: reverse-mode dV/dalpha and dV/dbeta agree with central finite differences;
* the split dual and empty domains (a reading: the paper only cites beta-CROWN): a hand-derived
  two-step example with one split and beta in {0, 3}, where beta = 3 reaches the exact lower bound;
  a split that contradicts its box sets the INFEASIBLE bit and leaves the domain out of the hull;
* the adaptive slope's tie u = -l takes slope 1 (hand-derived box);
* planted mistakes in the oracle are caught by these pins: dropped intercept, swapped
  Lambda+/-, wrong chord slope, the split dual's linear term dropped from EvalInt or from the
  intermediate bounds, no infeasibility check, the adaptive tie taking slope 0.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import reach as orc
from paper_2605_25346_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand_problem(mode):
    g = json.load(open(os.path.join(GOLDEN, "hand_example.json")))
    W = [np.array(g["W1"]), np.array(g["W2"])]
    b = [np.array(g["b1"]), np.array(g["b2"])]
    return g, wl.Problem("hand", [1, 1, 1], W, b, np.array(g["A"]), np.array(g["B"]), np.zeros(1),
                         np.array([g["lo"]]), np.array([g["hi"]]), 1, mode=mode)


@pytest.mark.parametrize("name,mode", [("chord", orc.MODE_CHORD), ("adaptive", orc.MODE_ADAPTIVE),
                                       ("zero", orc.MODE_ZERO)])
def test_hand_example(name, mode):
    g, p = _hand_problem(mode)
    r = orc.reach(p, keep_intermediate=True)
    assert r["l"][0, 0, 0].item() == pytest.approx(g["layer1_bounds"][0], abs=1e-15)
    assert r["u"][0, 0, 0].item() == pytest.approx(g["layer1_bounds"][1], abs=1e-15)
    assert r["lo"][0, 1, 0].item() == pytest.approx(g["box1"][name][0], abs=1e-14)
    assert r["hi"][0, 1, 0].item() == pytest.approx(g["box1"][name][1], abs=1e-14)
    assert r["lo"][0, 1, 0].item() <= g["true_range"][0] and r["hi"][0, 1, 0].item() >= g["true_range"][1]


def _vertex_box(prob, d):
    """Exact per-step box of an affine closed loop: min/max over the images of all box vertices."""
    V = wl.box_vertices(prob.lo[d], prob.hi[d])
    x = V.copy()
    out = [(x.min(0), x.max(0))]
    for _ in range(prob.H):
        h = x
        for l in range(prob.L):
            z = h @ prob.W[l].T + prob.b[l]
            h = np.maximum(z, 0) if l < prob.L - 1 else z
        x = x @ prob.A.T + h @ prob.B.T + prob.e
        out.append((x.min(0), x.max(0)))
    return out


def test_closed_form_linear_controller():
    # L = 1: pi(x) = W1 x + b1, the TM is exact and the remainder stays 0.
    for seed in range(3):
        p = wl.random_problem(seed, [4, 3], D=3, H=6, eps=0.3)
        p.e = np.random.default_rng(seed).normal(size=4) * 0.1
        r = orc.reach(p)
        for d in range(p.D):
            ref = _vertex_box(p, d)
            for t in range(p.H + 1):
                np.testing.assert_allclose(r["lo"][d, t].numpy(), ref[t][0], rtol=1e-12, atol=1e-12)
                np.testing.assert_allclose(r["hi"][d, t].numpy(), ref[t][1], rtol=1e-12, atol=1e-12)


def test_closed_form_all_active():
    # Large positive hidden biases keep every neuron active: the network is affine on the tube.
    p = wl.random_problem(7, [3, 6, 5, 2], D=2, H=5, eps=0.2)
    p.b = [p.b[0] + 40.0, p.b[1] + 60.0 * np.abs(p.W[1]).sum(1) + 40.0, p.b[2]]
    for mode in (orc.MODE_CHORD, orc.MODE_ZERO, orc.MODE_ADAPTIVE):
        r = orc.reach(p, mode=mode, keep_intermediate=True)
        assert bool((r["l"] > 0).all()), "precondition: all neurons stably active"
        for d in range(p.D):
            ref = _vertex_box(p, d)
            for t in range(p.H + 1):
                np.testing.assert_allclose(r["lo"][d, t].numpy(), ref[t][0], rtol=1e-11, atol=1e-10)
                np.testing.assert_allclose(r["hi"][d, t].numpy(), ref[t][1], rtol=1e-11, atol=1e-10)


def test_ibp_identity_one_hidden_layer():
    # ZERO slopes, one hidden layer, biases centring every pre-activation at 0 (no active neuron):
    # the controller bound is interval arithmetic, and the first box equals IBP exactly.
    for seed in range(4):
        p = wl.random_problem(100 + seed, [3, 7, 2], D=4, H=1, eps=0.3, mode=orc.MODE_ZERO)
        c = 0.5 * (p.lo + p.hi)
        # one centring bias per problem: use a single domain per problem instance
        for d in range(p.D):
            q = p.subset([d])
            q.b = [-(p.W[0] @ c[d]), p.b[1]]
            r = orc.reach(q, keep_intermediate=True)
            assert bool((r["l"] < 0).all()), "precondition: no stably-active neuron"
            ib = orc.ibp_reach(q)
            np.testing.assert_allclose(r["lo"][0, 1].numpy(), ib["lo"][0, 1].numpy(), rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(r["hi"][0, 1].numpy(), ib["hi"][0, 1].numpy(), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("widths", [[3, 8, 2], [4, 10, 10, 3], [2, 6, 6, 6, 1]])
def test_zero_slopes_never_looser_than_ibp(widths):
    p = wl.random_problem(5, widths, D=16, H=6, eps=0.2, mode=orc.MODE_ZERO)
    r = orc.reach(p)
    ib = orc.ibp_reach(p)
    scale = 1e-12 * (1 + ib["hi"].abs())
    assert bool((r["lo"] >= ib["lo"] - scale).all())
    assert bool((r["hi"] <= ib["hi"] + scale).all())


def _contained(prob, res, n_traj, seed, splits_ok=None):
    dom, xs, pre = wl.sample_trajectories(prob, n_traj, seed)
    lo = res["lo"].detach().numpy()[dom]
    hi = res["hi"].detach().numpy()[dom]
    tol = 1e-9 * (1 + np.abs(lo) + np.abs(hi))
    inside = (xs >= lo - tol) & (xs <= hi + tol)
    ok = inside.all(axis=(1, 2))
    if splits_ok is not None:
        keep = splits_ok(dom, pre)
        return bool(ok[keep].all()), int(keep.sum())
    return bool(ok.all()), n_traj


@pytest.mark.parametrize("mode", [orc.MODE_CHORD, orc.MODE_ADAPTIVE, orc.MODE_ZERO, orc.MODE_USER])
def test_containment_random(mode):
    p = wl.random_problem(11, [3, 12, 12, 2], D=8, H=8, eps=0.15, mode=mode)
    alpha = None
    if mode == orc.MODE_USER:
        alpha = torch.rand(p.D, p.H, p.hidden, dtype=torch.float64, generator=torch.Generator().manual_seed(3))
    r = orc.reach(p, alpha=alpha)
    ok, n = _contained(p, r, 10000, 1)
    assert ok and n == 10000


def test_containment_double_integrator_grid():
    p = wl.double_integrator_tiny()
    r = orc.reach(p)
    g = np.linspace(0, 1, 201)
    X0 = np.stack(np.meshgrid(0.9 + 0.2 * g, -0.1 + 0.2 * g, indexing="ij"), -1).reshape(-1, 2)
    x = X0
    for t in range(1, p.H + 1):
        h = x
        for l in range(p.L):
            z = h @ p.W[l].T + p.b[l]
            h = np.maximum(z, 0) if l < p.L - 1 else z
        x = x @ p.A.T + h @ p.B.T
        assert (x >= r["lo"][0, t].numpy() - 1e-12).all() and (x <= r["hi"][0, t].numpy() + 1e-12).all()


@pytest.mark.parametrize("name", ["quad6_batched", "cartpole_diff"])
def test_containment_workloads(name):
    p = wl.WORKLOADS[name]()
    sub = p.subset(np.arange(0, p.D, p.D // 32))
    r = orc.reach(sub)
    ok, n = _contained(sub, r, 10000, {"quad6_batched": 2, "cartpole_diff": 3}[name])
    assert ok


def _split_filter(prob):
    sp = prob.splits
    offs = np.concatenate([[0], np.cumsum(prob.widths[1:-1])])

    def keep(dom, pre):
        res = np.ones(len(dom), dtype=bool)
        for i, d in enumerate(dom):
            for k in range(sp.row_ptr[d], sp.row_ptr[d + 1]):
                z = pre[i, sp.t[k], offs[sp.layer[k] - 1] + sp.neuron[k]]
                if sp.sign[k] * z < 0:
                    res[i] = False
                    break
        return res
    return keep


def test_containment_split_domains_with_beta():
    p = wl.quadrotor_branch(only=np.arange(0, 65536, 97)[:600])
    counts = np.diff(p.splits.row_ptr)
    sel = np.nonzero((counts >= 1) & (counts <= 5))[0][:6]
    q = p.subset(sel)
    rng = np.random.default_rng(0)
    beta = torch.as_tensor(rng.uniform(0, 2.0, size=q.splits.nnz))
    r = orc.reach(q, beta=beta)
    assert int((r["status"] & orc.STATUS_INFEASIBLE).sum()) == 0
    ok, n = _contained(q, r, 20000, 3, splits_ok=_split_filter(q))
    assert ok and n > 200


def test_refinement_monotone_and_improves():
    p = wl.random_problem(21, [3, 10, 10, 2], D=6, H=5, eps=0.3)
    out = orc.optimize_slopes(p, steps=8, lr_alpha=0.05, lr_beta=0.0)
    h = np.array(out["V_hist"])
    assert (np.diff(h) <= 1e-12).all()
    assert h[-1] < h[0]
    # the kept slopes reproduce the kept objective
    r = orc.reach(p, alpha=out["alpha"], mode=orc.MODE_USER)
    np.testing.assert_allclose(r["V"].numpy(), out["best_V"].numpy(), rtol=1e-12)


def test_zero_slopes_inclusion_monotone_first_step():
    p = wl.random_problem(31, [2, 9, 9, 2], D=1, H=1, eps=0.4, mode=orc.MODE_ZERO)
    c = 0.5 * (p.lo[0] + p.hi[0])
    lo, hi = wl.box_grid(c, 0.5 * (p.hi[0, 0] - p.lo[0, 0]), [3, 3])
    lo[:, 1] = np.interp(lo[:, 1], [c[1] - 0.5 * (p.hi[0, 0] - p.lo[0, 0]), c[1] + 0.5 * (p.hi[0, 0] - p.lo[0, 0])], [p.lo[0, 1], p.hi[0, 1]])
    hi[:, 1] = np.interp(hi[:, 1], [c[1] - 0.5 * (p.hi[0, 0] - p.lo[0, 0]), c[1] + 0.5 * (p.hi[0, 0] - p.lo[0, 0])], [p.lo[0, 1], p.hi[0, 1]])
    q = wl.Problem("split", p.widths, p.W, p.b, p.A, p.B, p.e, lo, hi, 1, mode=orc.MODE_ZERO)
    whole = orc.reach(p)
    parts = orc.reach(q)
    assert bool((parts["hull_lo"][1] >= whole["lo"][0, 1] - 1e-12).all())
    assert bool((parts["hull_hi"][1] <= whole["hi"][0, 1] + 1e-12).all())


def _interior_alpha(p, seed):
    a0 = orc.chord_alpha(p)
    g = torch.Generator().manual_seed(seed)
    return (a0 + 0.2 * (torch.rand(a0.shape, generator=g, dtype=torch.float64) - 0.5)).clamp(0.05, 0.95)


def test_fd_gradient_alpha():
    p = wl.random_problem(41, [3, 8, 8, 2], D=2, H=3, eps=0.4)
    alpha = _interior_alpha(p, 0)
    res, ga, _ = orc.value_and_grad(p, alpha)
    flat = ga.reshape(-1)
    nz = torch.nonzero(flat).reshape(-1).numpy()
    assert len(nz) > 10
    rng = np.random.default_rng(0)
    coords = rng.choice(nz, size=min(16, len(nz)), replace=False)
    fd, ok = orc.finite_difference(p, alpha, None, coords, eps=1e-4)
    assert ok.sum() >= 8
    an = flat.numpy()[coords]
    err = np.abs(fd - an)[ok] / np.maximum(1e-12, np.abs(an[ok]).max())
    assert err.max() < 1e-6
    # coordinates with zero gradient are flat under FD too
    zc = np.setdiff1d(np.arange(flat.numel()), nz)[:4]
    fd0, ok0 = orc.finite_difference(p, alpha, None, zc, eps=1e-4)
    assert np.abs(fd0[ok0]).max(initial=0) < 1e-9


def test_fd_gradient_beta():
    p = wl.quadrotor_branch(only=np.arange(0, 65536, 131)[:200])
    counts = np.diff(p.splits.row_ptr)
    sel = np.nonzero(counts >= 3)[0][:2]
    q = p.subset(sel)
    q.H = 4
    keep = q.splits.t < q.H
    q = _restrict_splits(q, keep)
    alpha = _interior_alpha(q, 1)
    beta = torch.as_tensor(np.random.default_rng(2).uniform(0.05, 0.5, size=q.splits.nnz))
    res, ga, gb = orc.value_and_grad(q, alpha, beta)
    assert q.splits.nnz >= 2 and float(gb.abs().max()) > 0
    coords = np.arange(q.splits.nnz)[:8]
    fd, ok = orc.finite_difference(q, alpha, beta, coords, eps=1e-4, which="beta")
    assert ok.sum() >= 2
    an = gb.numpy()[coords]
    err = np.abs(fd - an)[ok] / np.maximum(1e-12, np.abs(an).max())
    assert err.max() < 1e-6


def _restrict_splits(q, keep):
    sp = q.splits
    dom = np.repeat(np.arange(q.D), np.diff(sp.row_ptr))[keep]
    row_ptr = np.zeros(q.D + 1, dtype=np.int64)
    np.add.at(row_ptr, dom + 1, 1)
    q.splits = wl.Splits(np.cumsum(row_ptr), sp.t[keep], sp.layer[keep], sp.neuron[keep], sp.sign[keep])
    q.beta = np.zeros(q.splits.nnz)
    return q


# ---------------------------------------------------------------------------------------------
# planted mistakes: each must break at least one pin above
# ---------------------------------------------------------------------------------------------

def _hand_box(mode):
    _, p = _hand_problem(mode)
    r = orc.reach(p)
    return r["lo"][0, 1, 0].item(), r["hi"][0, 1, 0].item()


def test_planted_dropped_intercept(monkeypatch):
    real = orc.relax

    def no_intercept(l, u, alpha, mode):
        s, d, a, un, br = real(l, u, alpha, mode)
        return s, torch.zeros_like(d), a, un, br
    monkeypatch.setattr(orc, "relax", no_intercept)
    lo, hi = _hand_box(orc.MODE_CHORD)
    assert not (lo <= -2.0 and hi >= 3.0)  # no longer encloses the exact range


def test_planted_swapped_lambda_split(monkeypatch):
    p = wl.random_problem(11, [3, 12, 12, 2], D=8, H=8, eps=0.15)
    real_pos, real_neg = orc.pos, orc.neg
    monkeypatch.setattr(orc, "pos", real_neg)
    monkeypatch.setattr(orc, "neg", real_pos)
    ok, _ = _contained(p, orc.reach(p), 10000, 1)
    assert not ok


def test_planted_wrong_chord(monkeypatch):
    real = orc.relax

    def bad(l, u, alpha, mode):
        if mode == orc.MODE_CHORD:
            unstable = (l < 0) & (u > 0)
            a = torch.where(unstable, -l / torch.where(unstable, u - l, torch.ones_like(l)), torch.zeros_like(l))
            return real(l, u, a, orc.MODE_USER)
        return real(l, u, alpha, mode)
    monkeypatch.setattr(orc, "relax", bad)
    lo, hi = _hand_box(orc.MODE_CHORD)
    assert (lo, hi) != pytest.approx((-2.75, 3.0))


# ---------------------------------------------------------------------------------------------
# split dual, infeasible domains, hull and the adaptive tie: hand-derived goldens
# ---------------------------------------------------------------------------------------------

def _golden(name):
    return json.load(open(os.path.join(GOLDEN, name)))


def _scalar_net(g):
    return [np.array(g["W1"]), np.array(g["W2"])], [np.array(g["b1"]), np.array(g["b2"])]


def _split_dual_problem(g, beta):
    W, b = _scalar_net(g)
    s = g["split"]
    sp = wl.Splits(np.array([0, 1], np.int64), np.array([s["t"]], np.int32), np.array([s["layer"]], np.int32),
                   np.array([s["neuron"]], np.int32), np.array([s["sign"]], np.int32))
    return wl.Problem("split-dual", [1, 1, 1], W, b, np.array(g["A"]), np.array(g["B"]), np.zeros(1),
                      np.array([g["lo"]]), np.array([g["hi"]]), g["H"], mode=orc.MODE_CHORD, splits=sp,
                      beta=np.array([beta]))


def _split_dual_matches(case):
    """True iff the oracle reproduces every hand-derived value of one split-dual case."""
    g = _golden("split_dual_example.json")
    c = g["cases"][case]
    r = orc.reach(_split_dual_problem(g, c["beta"]), keep_intermediate=True)
    ok = True
    for t, (l, u) in enumerate(c["layer1_bounds"]):
        ok &= abs(r["l"][0, t, 0].item() - l) <= 1e-13 and abs(r["u"][0, t, 0].item() - u) <= 1e-13
    for t, (lo, hi) in enumerate(c["box"]):
        ok &= abs(r["lo"][0, t, 0].item() - lo) <= 1e-13 and abs(r["hi"][0, t, 0].item() - hi) <= 1e-13
    return bool(ok), r


@pytest.mark.parametrize("case", ["beta3", "beta0"])
def test_split_dual_hand_example(case):
    ok, r = _split_dual_matches(case)
    assert ok
    g = _golden("split_dual_example.json")
    assert int(r["status"][0]) == 0
    for t, (lo, hi) in enumerate(g["true_range"]):
        assert r["lo"][0, t, 0].item() <= lo and r["hi"][0, t, 0].item() >= hi


def test_split_dual_tightens_the_lower_bound():
    # beta = 3 reaches the exact minimum of x_1 over the split domain; beta = 0 does not
    g = _golden("split_dual_example.json")
    r3 = orc.reach(_split_dual_problem(g, 3.0))
    r0 = orc.reach(_split_dual_problem(g, 0.0))
    assert r3["lo"][0, 1, 0].item() == pytest.approx(g["true_range"][1][0], abs=1e-14)
    assert r3["lo"][0, 1, 0].item() > r0["lo"][0, 1, 0].item() + 1.0


def _infeasible_problem():
    g = _golden("infeasible_split_example.json")
    W, b = _scalar_net(g)
    s = g["splits"]
    sp = wl.Splits(np.array(s["row_ptr"], np.int64), np.array(s["t"], np.int32), np.array(s["layer"], np.int32),
                   np.array(s["neuron"], np.int32), np.array(s["sign"], np.int32))
    p = wl.Problem("infeasible", [1, 1, 1], W, b, np.array(g["A"]), np.array(g["B"]), np.zeros(1),
                   np.array(g["lo"]), np.array(g["hi"]), g["H"], mode=orc.MODE_CHORD, splits=sp)
    return g, p


def _infeasible_matches():
    g, p = _infeasible_problem()
    r = orc.reach(p)
    ok = [int(x) for x in r["status"]] == g["status"]
    for t, (lo, hi) in enumerate(g["hull"]):
        ok &= abs(r["hull_lo"][t, 0].item() - lo) <= 1e-14 and abs(r["hull_hi"][t, 0].item() - hi) <= 1e-14
    return bool(ok)


def test_infeasible_split_flagged_and_excluded_from_hull():
    assert _infeasible_matches()


def _adaptive_tie_box():
    g = _golden("adaptive_tie_example.json")
    W, b = _scalar_net(g)
    p = wl.Problem("tie", [1, 1, 1], W, b, np.array(g["A"]), np.array(g["B"]), np.zeros(1),
                   np.array([g["lo"]]), np.array([g["hi"]]), g["H"], mode=orc.MODE_ADAPTIVE)
    r = orc.reach(p, keep_intermediate=True)
    return g, r


def test_adaptive_tie_takes_slope_one():
    g, r = _adaptive_tie_box()
    assert (r["l"][0, 0, 0].item(), r["u"][0, 0, 0].item()) == tuple(g["layer1_bounds"])
    assert r["lo"][0, 1, 0].item() == pytest.approx(g["box1"][0], abs=1e-14)
    assert r["hi"][0, 1, 0].item() == pytest.approx(g["box1"][1], abs=1e-14)


def _mutate(monkeypatch, fn_name, edits):
    """Install a copy of oracle function `fn_name` with textual edits (old -> new) applied."""
    import inspect
    src = inspect.getsource(getattr(orc, fn_name))
    for old, new in edits:
        assert old in src, f"mutation target not found: {old!r}"
        src = src.replace(old, new)
    ns = dict(vars(orc))
    exec(compile(src, orc.__file__, "exec"), ns)
    monkeypatch.setattr(orc, fn_name, ns[fn_name])


def test_planted_dual_dropped_in_evalint(monkeypatch):
    _mutate(monkeypatch, "reach", [("pm = P - v[:, None, :]", "pm = P"), ("pp = P + v[:, None, :]", "pp = P")])
    assert not _split_dual_matches("beta3")[0]


def test_planted_dual_dropped_in_intermediate_bounds(monkeypatch):
    _mutate(monkeypatch, "reach", [("gm = G - v[:, None, :]", "gm = G"), ("gp = G + v[:, None, :]", "gp = G")])
    assert not _split_dual_matches("beta3")[0]


def test_planted_no_infeasibility_check(monkeypatch):
    _mutate(monkeypatch, "reach", [("bad = (l > u).any(-1)", "bad = torch.zeros_like((l > u).any(-1))")])
    assert not _infeasible_matches()


def test_planted_adaptive_tie_takes_zero(monkeypatch):
    _mutate(monkeypatch, "relax", [("a = torch.where(u >= -l, one, zero)", "a = torch.where(u > -l, one, zero)")])
    g, r = _adaptive_tie_box()
    assert (r["lo"][0, 1, 0].item(), r["hi"][0, 1, 0].item()) == pytest.approx(tuple(g["box1_if_tie_took_zero"]))


# ---------------------------------------------------------------------------------------------
# per-step offsets: DT neural dynamics with planned inputs (Alg. 2), MPC action samples (Sec. V-B)
# ---------------------------------------------------------------------------------------------

def _linear_dt(seed=0, D=3, H=5):
    """x_{t+1} = W [x; u_t] + b with planned inputs: the network is affine, so the TM is exact."""
    rng = np.random.default_rng(seed)
    n, k = 3, 2
    W = [rng.normal(size=(n, n + k)) * 0.5]
    b = [rng.normal(size=n) * 0.1]
    xhat = rng.uniform(-1, 1, size=(D, n))
    r = rng.uniform(0.05, 0.2, size=(D, n))
    acts = rng.uniform(-1, 1, size=(D, H, k))
    return wl.neural_dynamics("lin-dt", W, b, n, k, xhat - r, xhat + r, acts), acts


def test_offsets_closed_form_linear_dynamics():
    p, acts = _linear_dt()
    n = 3
    r = orc.reach(p)
    for d in range(p.D):
        X = wl.box_vertices(p.lo[d, :n], p.hi[d, :n])
        for t in range(p.H):
            X = np.concatenate([X, np.repeat(acts[d, t][None], len(X), 0)], 1) @ p.W[0].T + p.b[0]
            np.testing.assert_allclose(r["lo"][d, t + 1, :n].numpy(), X.min(0), rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(r["hi"][d, t + 1, :n].numpy(), X.max(0), rtol=1e-12, atol=1e-12)
            if t + 1 < p.H:  # the action rows carry the next planned input exactly
                np.testing.assert_allclose(r["lo"][d, t + 1, n:].numpy(), acts[d, t + 1], atol=1e-15)
                np.testing.assert_allclose(r["hi"][d, t + 1, n:].numpy(), acts[d, t + 1], atol=1e-15)


def test_constant_offsets_equal_the_affine_term():
    p = wl.random_problem(91, [3, 12, 2], D=5, H=4, eps=0.2)
    e = np.array([0.3, -0.2, 0.1])
    q = wl.random_problem(91, [3, 12, 2], D=5, H=4, eps=0.2)
    q.eoff = np.broadcast_to(e, (q.D, q.H, 3)).copy()
    p.e = e
    a, b = orc.reach(p), orc.reach(q)
    np.testing.assert_array_equal(a["lo"].numpy(), b["lo"].numpy())
    np.testing.assert_array_equal(a["hi"].numpy(), b["hi"].numpy())


def test_tpush_dt_trajectories_contained():
    p = wl.tpush_dt(D=16)
    r = orc.reach(p)
    ok, n = _contained(p, r, 10000, 5)
    assert ok and n == 10000


def test_shift_gradient_matches_finite_differences():
    p = wl.tpush_dt(D=2, H=4)
    res, g = orc.value_and_shift_grad(p)
    n = 5
    flat = g.reshape(-1)
    # action rows (dV/du_t) and state rows, at steps 0 (initial centre) and later
    coords = [np.ravel_multi_index((d, t, i), g.shape) for d in range(2) for t in (0, 1, 3) for i in (0, 2, n, n + 1)]
    base = torch.zeros(p.D, p.H + 1, p.n, dtype=torch.float64)
    h = 1e-6
    fd = []
    for c in coords:
        vals = []
        for sg in (1.0, -1.0):
            sh = base.clone().reshape(-1)
            sh[c] += sg * h
            vals.append(float(orc.reach(p, shift=sh.reshape(base.shape))["V"].sum()))
        fd.append((vals[0] - vals[1]) / (2 * h))
    an = flat.numpy()[coords]
    assert np.abs(an).max() > 0
    np.testing.assert_allclose(fd, an, rtol=1e-5, atol=1e-6 * np.abs(an).max())


def test_weight_gradient_matches_finite_differences():
    # dV/dtheta of the controller (certified training, Sec. V-A) at fixed interior slopes
    p = wl.random_problem(47, [3, 8, 8, 2], D=3, H=3, eps=0.3)
    alpha = _interior_alpha(p, 4)
    _, gW, gb = orc.value_and_weight_grad(p, alpha)
    rng = np.random.default_rng(1)
    h = 1e-6
    checked = 0
    for layer in range(p.L):
        for which, grads, arrays in (("W", gW, p.W), ("b", gb, p.b)):
            flat = grads[layer].reshape(-1).numpy()
            for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
                vals = []
                for sg in (1.0, -1.0):
                    Ws = [torch.as_tensor(w).clone() for w in p.W]
                    bs = [torch.as_tensor(x).clone() for x in p.b]
                    tgt = Ws if which == "W" else bs
                    tgt[layer].view(-1)[idx] += sg * h
                    vals.append(float(orc.reach(p, alpha=alpha, mode=orc.MODE_USER, params=(Ws, bs))["V"].sum()))
                fd = (vals[0] - vals[1]) / (2 * h)
                assert abs(fd - flat[idx]) <= 1e-5 * max(1.0, abs(flat[idx])), (layer, which, idx, fd, flat[idx])
                checked += 1
    assert checked >= 10 and max(float(g.abs().max()) for g in gW) > 0
