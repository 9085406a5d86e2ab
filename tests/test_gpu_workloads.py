"""The five workloads at their stated sizes, on the GPU, against the FP64 oracle and against simulation.

* Parity in the launch configuration the benchmark times: the headline step (16,384 of the 262,144
  sub-boxes of the 16-512x4-8 workload, H = 50, two lanes of domain chunks, persistent tensor-core
  GEMMs, replayed from a CUDA graph on a side stream) and all 65,536 branch domains of the
  12-256x3-4 workload (H = 30, 0..32 splits each), each checked on sampled domains spread over the
  whole range (lane and chunk edges, domains with no split and with 32 splits) against the oracle
  run on those domains alone: domains are independent through every step, so a domain's bounds do
  not depend on which other domains share the launch.
* Soundness of the GPU machines themselves: 10^4 simulated trajectories per workload (FP64, initial
  states uniform in the union of the domain boxes) stay inside the boxes of their domain at every
  step; for branch domains only trajectories that satisfy all of the domain's split signs count, and
  draws continue until 10^4 of those have been checked.

Tolerance: the same 1e-5 relative per box entry and zero-slack containment of the oracle's box as
the other parity tests.
"""
import numpy as np
import pytest
import torch

from oracle import reach as orc
from paper_2605_25346_b300 import workloads as wl

from test_gpu_parity import compare, gpu_bounds

pytestmark = pytest.mark.gpu


def _bench_configuration_bounds(prob, calls=3):
    """dr_compute_bounds as the benchmark issues it: a side stream, device outputs, the third call a
    replay of the CUDA graph captured on the second."""
    from paper_2605_25346_b300 import api
    stream = torch.cuda.Stream()
    r = api.Reach(0, stream=stream).load(prob)
    with torch.cuda.stream(stream):
        for _ in range(calls):
            out = r.bounds(on_device=True)
        torch.cuda.synchronize()
    replays = r.graph_replays()
    V = r.objective()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["V"] = V
    r.close()
    return res, replays


def _sampled(g, idx):
    return {"lo": g["lo"][idx], "hi": g["hi"][idx], "status": g["status"][idx], "V": g["V"][idx]}


def _enclosed(prob, g, n_traj, seed, keep=None):
    dom, xs, pre = wl.sample_trajectories(prob, n_traj, seed)
    inside = ((xs >= g["lo"][dom]) & (xs <= g["hi"][dom])).all(axis=(1, 2))
    if keep is not None:
        k = keep(dom, pre)
        return bool(inside[k].all()), int(k.sum())
    return bool(inside.all()), n_traj


def test_large16_headline_chunk():
    p = wl.large16().subset(np.arange(16384))
    g, replays = _bench_configuration_bounds(p)
    assert replays >= 1
    assert np.isfinite(g["lo"]).all() and np.isfinite(g["hi"]).all()
    rng = np.random.default_rng(0)
    edges = np.array([0, 1, 1023, 4095, 8191, 8192, 8193, 12287, 16382, 16383])
    idx = np.unique(np.concatenate([edges, rng.choice(16384, size=8, replace=False)]))
    assert len(idx) >= 16
    o = orc.reach(p.subset(idx))
    compare(p.subset(idx), _sampled(g, idx), o, check_hull=False)
    # outward-margin headroom over the 50 steps (the margin is 2^-18 of the entry's magnitude)
    olo, ohi = o["lo"].numpy(), o["hi"].numpy()
    m = 2.0 ** -18 * np.maximum(np.abs(olo), np.abs(ohi))
    used = 1.0 - np.minimum((olo - g["lo"][idx]) / m, (g["hi"][idx] - ohi) / m)[:, 1:]
    assert used.max() <= 0.75, f"outward margin used up to {used.max():.2f}"
    # the hull over all 16,384 domains encloses every sampled domain's oracle box
    assert (g["hull_lo"][None] <= olo).all() and (g["hull_hi"][None] >= ohi).all()
    ok, n = _enclosed(p, g, 10000, 21)
    assert ok and n == 10000


def _split_filter(prob):
    sp = prob.splits
    offs = np.concatenate([[0], np.cumsum(prob.widths[1:-1])])

    def keep(dom, pre):
        res = np.ones(len(dom), dtype=bool)
        for i, d in enumerate(dom):
            for k in range(sp.row_ptr[d], sp.row_ptr[d + 1]):
                if sp.sign[k] * pre[i, sp.t[k], offs[sp.layer[k] - 1] + sp.neuron[k]] < 0:
                    res[i] = False
                    break
        return res
    return keep


def test_branch12_all_domains():
    p = wl.quadrotor_branch()
    assert p.D == 65536
    counts = np.diff(p.splits.row_ptr)
    assert counts.min() == 0 and counts.max() == 32
    g, replays = _bench_configuration_bounds(p)
    assert replays >= 1
    rng = np.random.default_rng(1)
    none = np.nonzero(counts == 0)[0]
    full = np.nonzero(counts == 32)[0]
    idx = np.unique(np.concatenate([[0, 65535], none[[0, len(none) // 2, -1]], full[[0, len(full) // 2, -1]],
                                    rng.choice(65536, size=12, replace=False)]))
    assert len(idx) >= 16
    compare(p.subset(idx), _sampled(g, idx), orc.reach(p.subset(idx)), check_hull=False)
    # 10^4 trajectories that satisfy all of their domain's split signs (about 6 % of uniform draws do)
    kept, seed = 0, 100
    while kept < 10000 and seed < 140:
        ok, n = _enclosed(p, g, 10000, seed, keep=_split_filter(p))
        assert ok
        kept += n
        seed += 1
    assert kept >= 10000


def test_double_integrator_grid_enclosed():
    # the tiny workload: a 201 x 201 grid of initial states (40,401 trajectories) inside the GPU machines
    p = wl.double_integrator_tiny()
    g = gpu_bounds(p)
    t = np.linspace(0, 1, 201)
    x = np.stack(np.meshgrid(p.lo[0, 0] + (p.hi[0, 0] - p.lo[0, 0]) * t, p.lo[0, 1] + (p.hi[0, 1] - p.lo[0, 1]) * t,
                             indexing="ij"), -1).reshape(-1, 2)
    for step in range(1, p.H + 1):
        h = x
        for l in range(p.L):
            z = h @ p.W[l].T + p.b[l]
            h = np.maximum(z, 0) if l < p.L - 1 else z
        x = x @ p.A.T + h @ p.B.T + p.e
        assert (x >= g["lo"][0, step]).all() and (x <= g["hi"][0, step]).all()


@pytest.mark.parametrize("name,seed", [("quad6_batched", 23), ("cartpole_diff", 24)])
def test_batched_workloads_enclosed(name, seed):
    p = wl.WORKLOADS[name]()
    g = gpu_bounds(p)
    ok, n = _enclosed(p, g, 10000, seed)
    assert ok and n == 10000
