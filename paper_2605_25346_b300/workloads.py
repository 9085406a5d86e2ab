"""Seeded synthetic workloads for closed-loop discrete-time reachability.

This module only *draws inputs*: controller weights, the linear dynamics
x_{t+1} = A x + B u + e, the initial sub-box grid, and the branch-domain split
lists.  It contains none of the bound-propagation arithmetic, so both the FP64
oracle (``oracle/``) and the CUDA path can consume the same problems without
sharing any code of the method itself.

The problems are shaped like the paper's workloads:

* the initial set is a box B_eps(x_hat) = {x : x_hat - eps <= x <= x_hat + eps}
  (Problem statement, Sec. III-A), optionally partitioned into a uniform grid
  of sub-boxes ("input splitting", Sec. VI-A and Table I);
* the closed loop is x_{t+1} = A x_t + B pi(x_t) + e with a ReLU MLP pi, the
  discrete-time neural feedback case of Sec. IV-E;
* branch domains carry ReLU split constraints (t, layer, neuron, sign), each
  restricting the domain to sign * z_{layer,neuron}(x_t) >= 0.

Random draws use ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MODE_ADAPTIVE = 0
MODE_CHORD = 1
MODE_ZERO = 2
MODE_USER = 3
MODE_NAMES = {"adaptive": MODE_ADAPTIVE, "chord": MODE_CHORD, "zero": MODE_ZERO, "user": MODE_USER}


@dataclass
class Splits:
    """Ragged per-domain ReLU split lists in CSR form.

    ``row_ptr[d]:row_ptr[d+1]`` indexes domain d's splits, sorted by (t, layer,
    neuron).  ``layer`` is the 1-based hidden-layer index (1..L-1), ``neuron``
    is 0-based, ``sign`` is +1 (z >= 0) or -1 (z <= 0).
    """

    row_ptr: np.ndarray  # int64 [D+1]
    t: np.ndarray  # int32 [nnz]
    layer: np.ndarray  # int32 [nnz]
    neuron: np.ndarray  # int32 [nnz]
    sign: np.ndarray  # int32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def subset(self, idx: np.ndarray) -> "Splits":
        idx = np.asarray(idx, dtype=np.int64)
        counts = self.row_ptr[idx + 1] - self.row_ptr[idx]
        row_ptr = np.zeros(len(idx) + 1, dtype=np.int64)
        row_ptr[1:] = np.cumsum(counts)
        sel = np.concatenate([np.arange(self.row_ptr[i], self.row_ptr[i + 1]) for i in idx]) if len(idx) else np.zeros(0, np.int64)
        sel = sel.astype(np.int64)
        return Splits(row_ptr, self.t[sel].copy(), self.layer[sel].copy(), self.neuron[sel].copy(), self.sign[sel].copy())


@dataclass
class Problem:
    name: str
    widths: List[int]  # n_0 = n (state), ..., n_L = m (control)
    W: List[np.ndarray]  # float64 [n_l, n_{l-1}], l = 1..L (index 0 is layer 1)
    b: List[np.ndarray]  # float64 [n_l]
    A: np.ndarray  # float64 [n, n]
    B: np.ndarray  # float64 [n, m]
    e: np.ndarray  # float64 [n]
    lo: np.ndarray  # float64 [D, n]
    hi: np.ndarray  # float64 [D, n]
    H: int
    mode: int = MODE_CHORD
    splits: Optional[Splits] = None
    beta: Optional[np.ndarray] = None  # float64 [nnz] (>= 0); None = zeros
    alpha_steps: int = 0
    lr_alpha: float = 0.1
    lr_beta: float = 0.1
    meta: dict = field(default_factory=dict)
    eoff: Optional[np.ndarray] = None  # float64 [D, H, n] per-step offsets: x_{t+1} = A x + B pi(x) + e + eoff[d, t]

    @property
    def D(self) -> int:
        return int(self.lo.shape[0])

    @property
    def n(self) -> int:
        return int(self.widths[0])

    @property
    def m(self) -> int:
        return int(self.widths[-1])

    @property
    def L(self) -> int:
        return len(self.W)

    @property
    def hidden(self) -> int:
        return int(sum(self.widths[1:-1]))

    def subset(self, idx) -> "Problem":
        """The same problem restricted to the domains ``idx`` (bounds per domain are independent)."""
        idx = np.asarray(idx, dtype=np.int64)
        sp = self.splits.subset(idx) if self.splits is not None else None
        beta = None
        if self.beta is not None and self.splits is not None:
            sel = np.concatenate([np.arange(self.splits.row_ptr[i], self.splits.row_ptr[i + 1]) for i in idx]) if len(idx) else np.zeros(0, np.int64)
            beta = self.beta[sel.astype(np.int64)].copy()
        return Problem(self.name + f"[{len(idx)}]", list(self.widths), self.W, self.b, self.A, self.B, self.e,
                       self.lo[idx].copy(), self.hi[idx].copy(), self.H, self.mode, sp, beta,
                       self.alpha_steps, self.lr_alpha, self.lr_beta, dict(self.meta, subset=True),
                       None if self.eoff is None else self.eoff[idx].copy())


# ---------------------------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------------------------

def mlp(rng: np.random.Generator, widths: List[int], f32: bool, bias_std: float = 0.1,
        hidden_gain: float = 1.0, out_gain: float = 1.0):
    """Random-init ReLU MLP: W_l ~ N(0, g_l^2/fan_in), b_l ~ N(0, bias_std^2) (output bias scaled
    by out_gain).  g_1 = 1, g_l = hidden_gain for the hidden-to-hidden layers and out_gain for
    the output layer; all gains 1 is the plain N(0, 1/fan_in) initialisation.

    With ``f32`` the values are rounded to float32 (and kept as float64) so that an
    FP32 device path and the FP64 oracle start from bit-identical parameters.
    """
    W, b = [], []
    L = len(widths) - 1
    for l in range(1, len(widths)):
        g = 1.0 if l == 1 else (out_gain if l == L else hidden_gain)
        w = rng.normal(0.0, g / np.sqrt(widths[l - 1]), size=(widths[l], widths[l - 1]))
        bb = rng.normal(0.0, bias_std, size=(widths[l],)) * (out_gain if l == L else 1.0)
        if f32:
            w = w.astype(np.float32).astype(np.float64)
            bb = bb.astype(np.float32).astype(np.float64)
        W.append(np.ascontiguousarray(w))
        b.append(np.ascontiguousarray(bb))
    return W, b


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with R's diagonal signs fixed."""
    q, r = np.linalg.qr(rng.normal(size=(n, n)))
    return q * np.sign(np.diag(r))[None, :]


def mixing_dynamics(rng: np.random.Generator, n: int, rho: float = 0.97, kappa: float = 0.1) -> np.ndarray:
    """Random stable A = rho [(1-kappa) S + kappa R]: S a random signed permutation, R a Gaussian
    matrix with unit row L1 norms.  Every row of |A| sums to at most rho < 1, so A contracts the
    infinity norm and interval remainders pushed through A do not grow (a dense rotation would
    inflate them by the row sums of |Q|, about 2 for n = 16, at every step).
    """
    S = np.zeros((n, n))
    S[np.arange(n), rng.permutation(n)] = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    G = rng.normal(size=(n, n))
    R = G / np.abs(G).sum(axis=1, keepdims=True)
    return rho * ((1.0 - kappa) * S + kappa * R)


def box_grid(center: np.ndarray, eps: float, parts: List[int]):
    """Uniform grid partition of [center-eps, center+eps] into prod(parts) sub-boxes.

    Cells are enumerated in C order (last coordinate fastest).
    """
    n = len(center)
    assert len(parts) == n
    edges = [np.linspace(center[i] - eps, center[i] + eps, parts[i] + 1) for i in range(n)]
    idx = np.indices(parts).reshape(n, -1).T  # [D, n]
    lo = np.stack([edges[i][idx[:, i]] for i in range(n)], axis=1)
    hi = np.stack([edges[i][idx[:, i] + 1] for i in range(n)], axis=1)
    return np.ascontiguousarray(lo), np.ascontiguousarray(hi)


def nominal_preactivations(prob: Problem, x0: np.ndarray, dom: Optional[np.ndarray] = None) -> List[np.ndarray]:
    """Pre-activations of every hidden layer along the nominal closed-loop trajectories from x0.

    Plain point evaluation of the system (no bounds); returns a list over t of
    arrays [D, hidden] (hidden layers concatenated).  ``dom`` names the domain of each row of x0
    (for the per-step offsets; default: row i is domain i).
    """
    x = x0.copy()
    out = []
    for _t in range(prob.H):
        h = x
        zs = []
        for l in range(prob.L):
            z = h @ prob.W[l].T + prob.b[l]
            if l < prob.L - 1:
                zs.append(z)
                h = np.maximum(z, 0.0)
            else:
                u = z
        out.append(np.concatenate(zs, axis=1) if zs else np.zeros((x.shape[0], 0)))
        x = x @ prob.A.T + u @ prob.B.T + prob.e + _offset(prob, dom, _t)
    return out


def _offset(prob: Problem, dom, t: int):
    """The per-step dynamics offsets of the given domains at step t (0 when the problem has none)."""
    if prob.eoff is None:
        return 0.0
    return prob.eoff[np.arange(prob.D) if dom is None else dom, t]


def branch_splits(prob: Problem, rng: np.random.Generator, max_k: int = 32, pool: int = 4,
                  only: Optional[np.ndarray] = None) -> Splits:
    """Draw 0..max_k ReLU splits per domain (count uniform), at neurons near their switching point.

    For each domain the nominal trajectory from the sub-box centre is simulated and
    the ``pool * max_k`` (t, layer, neuron) positions with the smallest |pre-activation|
    form the candidate pool; k of them are drawn without replacement and each gets a
    random sign.  All random numbers are drawn for every domain up front, so a
    domain's splits do not depend on which other domains are generated; ``only`` restricts the
    (costly) simulation to those domains and returns their split lists in that order.
    """
    D = prob.D
    hidden = prob.widths[1:-1]
    offs = np.concatenate([[0], np.cumsum(hidden)])
    counts = rng.integers(0, max_k + 1, size=D)
    keys = rng.random(size=(D, pool * max_k))
    signs = np.where(rng.random(size=(D, max_k)) < 0.5, -1, 1).astype(np.int32)
    sel = np.arange(D) if only is None else np.asarray(only, dtype=np.int64)
    centre = 0.5 * (prob.lo[sel] + prob.hi[sel])
    rows_t, rows_l, rows_j, rows_s = [], [], [], []
    row_ptr = np.zeros(len(sel) + 1, dtype=np.int64)
    chunk = 4096
    for c0 in range(0, len(sel), chunk):
        c1 = min(len(sel), c0 + chunk)
        z = nominal_preactivations(prob, centre[c0:c1], sel[c0:c1])  # H x [c, hid]
        za = np.abs(np.stack(z, axis=1)).reshape(c1 - c0, -1)  # [c, H*hid]
        kk = min(pool * max_k, za.shape[1] - 1)
        cand = np.argpartition(za, kk, axis=1)[:, : pool * max_k]
        cand = np.take_along_axis(cand, np.argsort(np.take_along_axis(za, cand, 1), axis=1, kind="stable"), 1)
        for i in range(c0, c1):
            d = int(sel[i])
            k = min(int(counts[d]), cand.shape[1])
            order = np.argsort(keys[d][: cand.shape[1]], kind="stable")[:k]
            flat = np.sort(cand[i - c0][order])  # sorted by (t, hidden index)
            t = flat // offs[-1]
            hid = flat % offs[-1]
            layer = np.searchsorted(offs, hid, side="right")  # 1-based hidden layer
            neuron = hid - offs[layer - 1]
            rows_t.append(t.astype(np.int32))
            rows_l.append(layer.astype(np.int32))
            rows_j.append(neuron.astype(np.int32))
            rows_s.append(signs[d, :k])
            row_ptr[i + 1] = row_ptr[i] + k
    cat = lambda xs: np.concatenate(xs).astype(np.int32) if xs else np.zeros(0, np.int32)
    return Splits(row_ptr, cat(rows_t), cat(rows_l), cat(rows_j), cat(rows_s))


def sample_trajectories(prob: Problem, n_traj: int, seed: int):
    """Uniform initial states in the union of the domain boxes, simulated in FP64.

    Returns (dom [N], xs [N, H+1, n], pre [N, H, hidden]); ``dom`` is one domain whose
    box contains x0 (initial states are drawn inside a randomly chosen domain box).
    """
    rng = np.random.default_rng(seed)
    dom = rng.integers(0, prob.D, size=n_traj)
    u01 = rng.random(size=(n_traj, prob.n))
    x0 = prob.lo[dom] + u01 * (prob.hi[dom] - prob.lo[dom])
    xs = [x0]
    pre = nominal_preactivations(prob, x0, dom)
    x = x0
    for _t in range(prob.H):
        h = x
        for l in range(prob.L):
            z = h @ prob.W[l].T + prob.b[l]
            h = np.maximum(z, 0.0) if l < prob.L - 1 else z
        x = x @ prob.A.T + h @ prob.B.T + prob.e + _offset(prob, dom, _t)
        xs.append(x)
    return dom, np.stack(xs, axis=1), np.stack(pre, axis=1)


def box_vertices(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    n = lo.shape[0]
    bits = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(bool)
    return np.where(bits, hi[None, :], lo[None, :])


# ---------------------------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------------------------

SEED_BASE = 20260


def double_integrator_tiny() -> Problem:
    """2-state double integrator (dt = 0.1, exact zero-order hold), controller 2-16-16-1 with FP64
    weights, one box [0.9,1.1]x[-0.1,0.1], horizon 5, fixed adaptive slopes."""
    rng = np.random.default_rng(SEED_BASE + 1)
    widths = [2, 16, 16, 1]
    W, b = mlp(rng, widths, f32=False)
    A = np.array([[1.0, 0.1], [0.0, 1.0]])
    B = np.array([[0.005], [0.1]])
    lo = np.array([[0.9, -0.1]])
    hi = np.array([[1.1, 0.1]])
    return Problem("double-integrator 2-16-16-1, 1 box, H=5", widths, W, b, A, B, np.zeros(2), lo, hi, 5,
                   mode=MODE_ADAPTIVE)


def quad6_batched(parts: int = 4) -> Problem:
    """6-state random stable linear dynamics (A = mixing_dynamics, B = 0.1 N(0,1) 6x3), controller
    6-64-64-3 (FP32 weights, N(0, 1/fan_in), output gain 0.5), B_0.1(x_hat) split into a uniform
    parts^6 grid (4096 sub-boxes), H = 10."""
    rng = np.random.default_rng(SEED_BASE + 2)
    widths = [6, 64, 64, 3]
    W, b = mlp(rng, widths, f32=True, out_gain=0.5)
    A = mixing_dynamics(rng, 6)
    B = 0.1 * rng.normal(size=(6, 3))
    xhat = rng.uniform(-1, 1, size=6)
    lo, hi = box_grid(xhat, 0.1, [parts] * 6)
    return Problem(f"quad6 6-64-64-3, {lo.shape[0]} sub-boxes, H=10", widths, W, b, A, B, np.zeros(6), lo, hi, 10,
                   mode=MODE_CHORD)


def cartpole_linear(dt: float = 0.02, mc: float = 1.0, mp: float = 0.1, l: float = 0.5, g: float = 9.81):
    """Cart-pole linearised about the upright pole, forward Euler.

    State (x, x_dot, theta, theta_dot), inputs (cart force F, pivot torque tau).  From
    the mass matrix [[mc+mp, mp l], [mp l, mp l^2]] and generalised forces (F, tau + mp g l theta).
    """
    Ac = np.zeros((4, 4))
    Ac[0, 1] = 1.0
    Ac[1, 2] = -mp * g / mc
    Ac[2, 3] = 1.0
    Ac[3, 2] = (mc + mp) * g / (mc * l)
    Bc = np.zeros((4, 2))
    Bc[1, 0] = 1.0 / mc
    Bc[3, 0] = -1.0 / (mc * l)
    Bc[1, 1] = -1.0 / (mc * l)
    Bc[3, 1] = (mc + mp) / (mc * mp * l * l)
    return np.eye(4) + dt * Ac, dt * Bc


def cartpole_diff(alpha_steps: int = 20) -> Problem:
    """Linearised cart-pole, controller 4-128-128-2 (FP32 weights), 1024 = 4x4x8x8 sub-boxes, H = 20,
    alpha refinement by projected gradient."""
    rng = np.random.default_rng(SEED_BASE + 3)
    widths = [4, 128, 128, 2]
    W, b = mlp(rng, widths, f32=True, out_gain=0.3)
    A, B = cartpole_linear()
    xhat = rng.uniform(-1, 1, size=4)
    lo, hi = box_grid(xhat, 0.1, [4, 4, 8, 8])
    return Problem("cart-pole 4-128-128-2, 1024 sub-boxes, H=20", widths, W, b, A, B, np.zeros(4), lo, hi, 20,
                   mode=MODE_CHORD, alpha_steps=alpha_steps)


def quadrotor_hover(dt: float = 0.02, mass: float = 1.0, J=(0.01, 0.01, 0.02), g: float = 9.81):
    """12-state quadrotor hover linearisation, forward Euler.

    State (px, py, pz, phi, theta, psi, vx, vy, vz, p, q, r); inputs (delta thrust, roll, pitch, yaw
    torques): vx' = g theta, vy' = -g phi, vz' = du1/m, angle rates = body rates, p' = u2/Jx, ...
    """
    Ac = np.zeros((12, 12))
    Ac[0, 6] = Ac[1, 7] = Ac[2, 8] = 1.0
    Ac[3, 9] = Ac[4, 10] = Ac[5, 11] = 1.0
    Ac[6, 4] = g
    Ac[7, 3] = -g
    Bc = np.zeros((12, 4))
    Bc[8, 0] = 1.0 / mass
    Bc[9, 1] = 1.0 / J[0]
    Bc[10, 2] = 1.0 / J[1]
    Bc[11, 3] = 1.0 / J[2]
    return np.eye(12) + dt * Ac, dt * Bc


def quadrotor_branch(D_grid=(4, 4, 4, 4, 2, 2, 2, 2, 2, 2, 2, 2), max_splits: int = 32,
                     with_splits: bool = True, only: Optional[np.ndarray] = None) -> Problem:
    """12-state random stable linear dynamics (A = mixing_dynamics, B = 0.1 N(0,1) 12x4), controller
    12-256-256-256-4 (FP32 weights; hidden gain 0.7, bias std 0.5, output gain 0.3), 65536 branch
    domains (4^4 * 2^8 grid) with 0..32 ReLU splits each, H = 30, beta multipliers initialised to 0.

    The hover linearisation of a quadrotor (a chain of integrators) is only marginally stable and
    an untrained controller does not stabilise it: the certified tube then diverges (width ~1e49
    at t = 30, past the FP32 range), so a random stable 12-state system stands in for it.
    """
    rng = np.random.default_rng(SEED_BASE + 4)
    widths = [12, 256, 256, 256, 4]
    W, b = mlp(rng, widths, f32=True, bias_std=0.5, hidden_gain=0.7, out_gain=0.3)
    A = mixing_dynamics(rng, 12)
    B = 0.1 * rng.normal(size=(12, 4))
    xhat = rng.uniform(-1, 1, size=12)
    lo, hi = box_grid(xhat, 0.1, list(D_grid))
    prob = Problem(f"branch12 12-256-256-256-4, {lo.shape[0]} branch domains, H=30", widths, W, b, A, B,
                   np.zeros(12), lo, hi, 30, mode=MODE_CHORD)
    if with_splits:
        sp = branch_splits(prob, rng, max_k=max_splits, only=only)
        if only is not None:
            prob = Problem(prob.name + f"[{len(only)}]", widths, W, b, A, B, np.zeros(12), lo[only], hi[only], 30,
                           mode=MODE_CHORD, meta=dict(subset=True))
        prob.splits = sp
        prob.beta = np.zeros(sp.nnz)
    elif only is not None:
        prob = prob.subset(only)
    return prob


def large16(D_grid=(4, 4) + (2,) * 14, alpha_steps: int = 10) -> Problem:
    """16-state random stable linear dynamics (A = mixing_dynamics, B = 0.1 N(0,1) 16x8), controller
    16-512-512-512-512-8 (FP32 weights; hidden gain 0.5, bias std 0.5, output gain 0.2), 262144
    sub-boxes (4^2 * 2^14 grid), H = 50, 10 alpha steps."""
    rng = np.random.default_rng(SEED_BASE + 5)
    widths = [16, 512, 512, 512, 512, 8]
    W, b = mlp(rng, widths, f32=True, bias_std=0.5, hidden_gain=0.5, out_gain=0.2)
    A = mixing_dynamics(rng, 16)
    B = 0.1 * rng.normal(size=(16, 8))
    xhat = rng.uniform(-1, 1, size=16)
    lo, hi = box_grid(xhat, 0.1, list(D_grid))
    return Problem(f"large 16-512x4-8, {lo.shape[0]} sub-boxes, H=50", widths, W, b, A, B, np.zeros(16), lo, hi,
                   50, mode=MODE_CHORD, alpha_steps=alpha_steps)


def neural_dynamics(name: str, W, b, n: int, k: int, lo: np.ndarray, hi: np.ndarray, actions: np.ndarray,
                    mode: int = MODE_CHORD, residual: bool = False) -> Problem:
    """Discrete-time neural dynamics x_{t+1} = f(x_t, u_t) (or x_t + f(x_t, u_t) with ``residual``) with
    planned inputs u_t per domain (Alg. 2), written as a closed loop over the augmented state
    y = [x; u] of size n + k:

        y_{t+1} = A y_t + B f(y_t) + eoff[d, t],   A = [[I or 0, 0], [0, 0]],  B = [[I_n], [0]],
        eoff[d, t] = [0; u_{d, t+1}] (u_{d, H} = 0),  initial box [lo_d; u_{d, 0}] x [hi_d; u_{d, 0}].

    f is the MLP with input width n + k (widths[0]) and output width n; actions [D, H, k].  Each domain
    is one action sequence (an MPC sample) with its own initial box.
    """
    D, H = actions.shape[0], actions.shape[1]
    N = n + k
    A = np.zeros((N, N))
    if residual:
        A[:n, :n] = np.eye(n)
    B = np.zeros((N, n))
    B[:n, :n] = np.eye(n)
    eoff = np.zeros((D, H, N))
    eoff[:, :H - 1, n:] = actions[:, 1:, :]
    lo_a = np.concatenate([lo, actions[:, 0, :]], axis=1)
    hi_a = np.concatenate([hi, actions[:, 0, :]], axis=1)
    widths = [N] + [w.shape[0] for w in W]
    return Problem(name, widths, W, b, A, B, np.zeros(N), lo_a, hi_a, H, mode=mode,
                   meta=dict(state_dims=n, action_dims=k), eoff=eoff)


def tpush_dt(D: int = 128, H: int = 10, eps: float = 0.05, seed_offset: int = 0) -> Problem:
    """The paper's DT benchmark shape (Sec. VI-A with the T-pushing model of App. D): neural dynamics
    with state (T pose: position, orientation; pusher position) n = 5, action (pusher velocity) k = 2,
    residual MLP x_{t+1} = x_t + f(x_t, u_t), f 7-96-96-96-5 with random weights (FP32 values; hidden
    gain 0.7, output gain 0.2), D random initial boxes B_eps(x_hat), x_hat ~ U[-1, 1]^5, eps = 0.05 (the
    T-pushing planning perturbation of Sec. VI-D), action sequences u ~ U[-1, 1]^2, horizon 10.

    An untrained direct-form model x_{t+1} = f(x_t, u_t) either blows the tube up (N(0, 1/fan_in)
    gains: width 4e9 after 10 steps) or collapses it to a point (small output gain: width 1e-9); the
    residual form with these gains keeps the tube near its initial size (width 0.11 -> 0.22 over 10
    steps) with about 13 % of the neurons unstable."""
    rng = np.random.default_rng(SEED_BASE + 6 + seed_offset)
    n, k = 5, 2
    W, b = mlp(rng, [n + k, 96, 96, 96, n], f32=True, hidden_gain=0.7, out_gain=0.2)
    xhat = rng.uniform(-1, 1, size=(D, n))
    actions = rng.uniform(-1, 1, size=(D, H, k))
    return neural_dynamics(f"tpush-dt 7-96x3-5 (residual), {D} boxes x action sequences, H={H}", W, b, n, k,
                           xhat - eps, xhat + eps, actions, residual=True)


def tpush_mpc(samples: int = 1024, H: int = 10, eps: float = 0.05) -> Problem:
    """Sampling-based MPC over the T-pushing DT dynamics (Sec. V-B): one nominal initial box
    B_eps(x_hat) and `samples` candidate action sequences u ~ U[-1, 1]^{H x 2}, each a domain."""
    base = tpush_dt(D=1, H=H, eps=eps)
    rng = np.random.default_rng(SEED_BASE + 7)
    n, k = 5, 2
    xhat = 0.5 * (base.lo[0, :n] + base.hi[0, :n])
    actions = rng.uniform(-1, 1, size=(samples, H, k))
    lo = np.repeat((xhat - eps)[None], samples, axis=0)
    hi = np.repeat((xhat + eps)[None], samples, axis=0)
    return neural_dynamics(f"tpush-mpc 7-96x3-5 (residual), {samples} action samples, H={H}", base.W, base.b, n, k,
                           lo, hi, actions, residual=True)


def random_problem(seed: int, widths, D: int, H: int, eps: float = 0.1, mode: int = MODE_CHORD,
                   f32: bool = True, rho: float = 0.97, b_scale: float = 0.1, out_gain: float = 0.5) -> Problem:
    """Small random closed loop for tests: random boxes of radius ~eps around U[-1,1]^n centres."""
    rng = np.random.default_rng(seed)
    W, b = mlp(rng, list(widths), f32=f32, out_gain=out_gain)
    n, m = widths[0], widths[-1]
    A = mixing_dynamics(rng, n, rho)
    B = b_scale * rng.normal(size=(n, m))
    c = rng.uniform(-1, 1, size=(D, n))
    r = eps * rng.uniform(0.25, 1.0, size=(D, n))
    return Problem(f"random{tuple(widths)} D={D} H={H}", list(widths), W, b, A, B, np.zeros(n), c - r, c + r, H,
                   mode=mode)


WORKLOADS = {
    "double_integrator_tiny": double_integrator_tiny,
    "quad6_batched": quad6_batched,
    "cartpole_diff": cartpole_diff,
    "quadrotor_branch": quadrotor_branch,
    "large16": large16,
    "tpush_dt": tpush_dt,
    "tpush_mpc": tpush_mpc,
}
