"""CUDA-graph capture and replay of dr_compute_bounds (a context on its own stream): the plain first
call, the capturing second call and the replays give bitwise-identical boxes, equal to a context with
graphs disabled; new box values under the same domain count are picked up by the replay; a change of
options forces a new capture.  Host outputs (on_device = 0) synchronise the stream."""
import numpy as np
import pytest
import torch

from paper_2605_25346_b300 import workloads as wl

pytestmark = pytest.mark.gpu
TCORE = 2  # DR_PREC_TF32X3


def _api():
    from paper_2605_25346_b300 import api
    return api


def _reach(p, graphs, precision=0, chunk=0):
    api = _api()
    r = api.Reach(0, stream=torch.cuda.Stream()).load(p, precision=precision)
    r.set_options(mode=p.mode, precision=precision, chunk=chunk, graphs=graphs)
    return r


def _same(a, b):
    for k in ("lo", "hi", "hull_lo", "hull_hi", "status"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("case", ["fused", "staged", "staged_auto_chunk"])
def test_replay_matches_plain_launches(case):
    if case == "fused":
        p, prec, chunk = wl.random_problem(71, [5, 40, 30, 3], D=300, H=6, eps=0.2), 0, 0
    elif case == "staged":
        p, prec, chunk = wl.random_problem(72, [6, 96, 80, 64, 2], D=300, H=4, eps=0.15), TCORE, 64
    else:  # the chunk chosen from the device's free memory on the plain call is kept while capturing
        p, prec, chunk = wl.random_problem(75, [6, 96, 80, 64, 2], D=300, H=4, eps=0.15), TCORE, 0
    ref = _reach(p, graphs=1, precision=prec, chunk=chunk)
    want = ref.bounds(on_device=False)
    ref.close()
    r = _reach(p, graphs=0, precision=prec, chunk=chunk)
    launches = []
    for _ in range(4):  # plain, capture, replay, replay
        l0 = r.launches()
        got = r.bounds(on_device=False)
        launches.append(r.launches() - l0)
        _same(got, want)
    assert len(set(launches)) == 1 and launches[0] > 0
    assert r.graph_replays() == 2  # calls 3 and 4
    r.close()


def test_replay_reads_new_boxes_and_recaptures_on_new_options():
    p = wl.random_problem(73, [4, 32, 32, 2], D=200, H=5, eps=0.2)
    q = wl.random_problem(74, [4, 32, 32, 2], D=200, H=5, eps=0.3)
    q.W, q.b, q.A, q.B, q.e = p.W, p.b, p.A, p.B, p.e  # same system, different boxes
    r = _reach(p, graphs=0)
    for _ in range(3):
        r.bounds(on_device=False)
    lo, hi = np.ascontiguousarray(q.lo), np.ascontiguousarray(q.hi)
    r._c(r.lib.dr_set_boxes(r.ctx, q.D, _api()._ptr(lo), _api()._ptr(hi), 0))
    got = r.bounds(on_device=False)
    ref = _reach(q, graphs=1)
    _same(got, ref.bounds(on_device=False))
    # a different outward margin changes kernel arguments: the next calls must not replay the old graph
    r.set_options(mode=q.mode, box_margin=2.0 ** -16)
    ref.set_options(mode=q.mode, box_margin=2.0 ** -16, graphs=1)
    want = ref.bounds(on_device=False)
    n0 = r.graph_replays()
    for _ in range(3):
        _same(r.bounds(on_device=False), want)
    assert r.graph_replays() == n0 + 1  # plain, capture, replay
    r.close()
    ref.close()


# Refinement: the first projected-gradient step runs plain, the others replay one captured step.
# The V history, the kept slopes and multipliers and the final bounds equal those of a context with
# graphs disabled, bit for bit; the shared-memory and the global-slab (wide controller) reverse
# kernels, with and without split multipliers.
@pytest.mark.parametrize("case", ["fused", "slab", "splits"])
def test_refinement_steps_replayed_from_a_graph(case):
    if case == "fused":
        p, lrb = wl.random_problem(81, [4, 24, 24, 2], D=40, H=4, eps=0.3), 0.0
    elif case == "slab":
        p, lrb = wl.random_problem(82, [4, 300, 300, 2], D=6, H=3, eps=0.2), 0.0
    else:
        p = wl.random_problem(83, [6, 40, 40, 3], D=24, H=5, eps=0.2)
        rng = np.random.default_rng(3)
        p.splits = wl.branch_splits(p, rng, max_k=6)
        p.beta = rng.uniform(0.0, 0.05, size=p.splits.nnz).astype(np.float32).astype(np.float64)
        lrb = 0.01
    steps = 5
    out = {}
    for graphs in (1, 0):
        r = _reach(p, graphs=graphs)
        with torch.cuda.stream(r.stream):
            a0 = r.get_alpha()
            g = torch.Generator().manual_seed(1)
            alpha = np.clip(a0 + 0.1 * (torch.rand(a0.shape, generator=g).numpy() - 0.5), 0.0, 1.0).astype(np.float32)
            r.set_alpha(alpha)
            replays0 = r.graph_replays()
            hist = r.optimize(steps, 0.05, lrb)
            replays = r.graph_replays() - replays0
            out[graphs] = (hist, r.get_alpha(), r.get_beta(), r.bounds(on_device=False), replays)
        r.close()
    h1, a1, b1, o1, rep1 = out[1]
    h0, a0, b0, o0, rep0 = out[0]
    assert rep1 == 0 and rep0 == steps - 1
    np.testing.assert_array_equal(h0, h1)
    np.testing.assert_array_equal(a0, a1)
    np.testing.assert_array_equal(b0, b1)
    _same(o0, o1)
    assert (np.diff(h0) <= 0).all()
