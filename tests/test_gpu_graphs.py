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
