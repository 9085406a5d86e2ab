"""FP64 CPU oracle for closed-loop discrete-time reachability with shared-slope CROWN Taylor models.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow reference that the CUDA
path is checked against.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the library itself never does, and it shares no
code with the CUDA path (the only common module is the seeded input generator,
which holds none of the method's arithmetic).

What it computes (the paper: Sec. IV-A linear Taylor models, Thm. 2 CROWN bounds,
Thm. 3 CROWN with a linear-TM input and its proof in App. B, Alg. 2 stepwise
discrete-time reachability, Sec. IV-E closed-loop remark, Sec. V-A tube-volume
proxy), for each domain d independently:

  a1  BuildLinearTM: x = c + P zeta + r, zeta in [-1,1]^n, r in [I_lo, I_hi];
      c = (lo+hi)/2, P = diag((hi-lo)/2), I = 0                 (Alg. 2; Alg. 3 normalisation)
  for t = 0..H-1:
    for each layer l = 1..L of the controller (target of the bound):
      a4  backward chain: Lambda = W_l, kappa = b_l; for m = l-1..1:
            kappa_hi += Lambda^+ d_m ; kappa_lo += Lambda^- d_m
            Lambda_s = Lambda diag(s_m); kappa += Lambda_s b_m; Lambda = Lambda_s W_m     (Thm. 2)
      a5  concretise over the TM input (Thm. 3): G = Lambda P, a = Lambda c,
            [R_lo, R_hi] = Lambda (x) [I];  l = a + kappa_lo + R_lo - |G|_1,
            u = a + kappa_hi + R_hi + |G|_1   (plus the split dual, see below)
      a3  shared-slope relaxation of a hidden layer: stable neurons exact; unstable
            neurons lower alpha z, upper alpha z + max(-alpha l, (1-alpha) u)  (Sec. IV-C)
      a6  output layer: controller TM  P_u = G, c_u = a + (k_lo+k_hi)/2,
            I_u = +-(k_hi-k_lo)/2 + [R_lo, R_hi]                           (Thm. 3, App. B)
    a7  dynamics: P' = A P + B P_u, c' = A c + B c_u + e + e_{d,t}, I' = A (x) [I] + B (x) [I_u]
        (e_{d,t}: optional per-domain, per-step offsets; with the state augmented by the planned
        input, y = [x; u], they carry the planned inputs u_k of Alg. 2 into a neural dynamics model)
    a8  EvalInt: box_{t+1} = c' +- |P'|_1 + [I']                          (Alg. 2)
  a9  hull over domains; V_d = sum_{t=1..H} sum_i width(box_{t,i})           (Sec. V-A)

Readings where the paper is silent (each restated in the design notes):
  * slope modes: CHORD alpha = u/(u-l); ADAPTIVE alpha = 1 if u >= -l else 0; ZERO
    alpha = 0; USER alpha given per (domain, step, hidden neuron).
  * ReLU split (t, layer, j, sign): after layer `layer` of step t is concretised,
    the neuron's bound is clipped (sign>0: l = max(l,0); sign<0: u = min(u,0)) and
    the valid constraint g^T zeta + h >= 0 (g = sign*G_j, h = sign>0 ? a+k_hi+R_hi :
    -(a+k_lo+R_lo)) is recorded.  Every later concretisation of p^T zeta over
    [-1,1]^n uses the Lagrangian dual with one multiplier beta_k >= 0 per split:
    min >= -|p - v|_1 - w, max <= |p + v|_1 + w, v = sum beta_k g_k, w = sum beta_k h_k.
  * tie rules (subgradients): |0|' = 0, Lambda^+ and Lambda^- have zero slope at 0,
    the intercept max(-alpha l, (1-alpha) u) takes the first branch on a tie,
    classification is l >= 0 -> active, else u <= 0 -> inactive, else unstable.

Gradients dV/dalpha, dV/dbeta are obtained by reverse-mode automatic
differentiation of this FP64 forward pass and pinned by central finite differences.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional

import numpy as np
import torch

MODE_ADAPTIVE, MODE_CHORD, MODE_ZERO, MODE_USER = 0, 1, 2, 3
STATUS_NONFINITE = 1
STATUS_INFEASIBLE = 2

_F64 = torch.float64


def _t(x) -> torch.Tensor:
    return torch.as_tensor(np.asarray(x), dtype=_F64)


def pos(x: torch.Tensor) -> torch.Tensor:
    """x^+ with zero slope at 0."""
    return torch.where(x > 0, x, torch.zeros_like(x))


def neg(x: torch.Tensor) -> torch.Tensor:
    """x^- with zero slope at 0."""
    return torch.where(x < 0, x, torch.zeros_like(x))


def interval_matvec(M: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor):
    """Interval product M (x) [lo, hi] (exact range of M r over the box r in [lo, hi]).

    M: [..., k, n], lo/hi: [..., n] -> ([..., k], [..., k]).
    """
    Mp, Mn = pos(M), neg(M)
    out_lo = (Mp @ lo.unsqueeze(-1) + Mn @ hi.unsqueeze(-1)).squeeze(-1)
    out_hi = (Mp @ hi.unsqueeze(-1) + Mn @ lo.unsqueeze(-1)).squeeze(-1)
    return out_lo, out_hi


def relax(l: torch.Tensor, u: torch.Tensor, alpha: Optional[torch.Tensor], mode: int):
    """Shared-slope ReLU relaxation (Sec. IV-C shared-slope constraint).

    Returns (s, d): alpha z <= relu(z) <= alpha z + d on [l, u] for unstable neurons
    (s = alpha), s = 1, d = 0 for l >= 0 and s = 0, d = 0 for u <= 0.
    """
    active = l >= 0
    inactive = (~active) & (u <= 0)
    unstable = ~(active | inactive)
    one = torch.ones_like(l)
    zero = torch.zeros_like(l)
    if mode == MODE_CHORD:
        den = torch.where(unstable, u - l, one)
        a = torch.where(unstable, u / den, zero)
    elif mode == MODE_ADAPTIVE:
        a = torch.where(u >= -l, one, zero)
    elif mode == MODE_ZERO:
        a = zero
    elif mode == MODE_USER:
        a = alpha
    else:
        raise ValueError(mode)
    s = torch.where(active, one, torch.where(unstable, a, zero))
    br1 = -a * l
    br2 = (1.0 - a) * u
    d = torch.where(unstable, torch.where(br1 >= br2, br1, br2), zero)
    return s, d, a, unstable, (br1 >= br2)


class _SplitIndex:
    """Splits grouped by (t, layer) for vectorised application."""

    def __init__(self, prob, dom_index: np.ndarray):
        self.groups: Dict[tuple, tuple] = {}
        sp = prob.splits
        if sp is None or sp.nnz == 0:
            return
        D = prob.D
        dom = np.repeat(np.arange(D), np.diff(sp.row_ptr))
        keys = {}
        for k in range(sp.nnz):
            keys.setdefault((int(sp.t[k]), int(sp.layer[k])), []).append(k)
        for key, ks in keys.items():
            ks = np.asarray(ks, dtype=np.int64)
            self.groups[key] = (torch.as_tensor(ks), torch.as_tensor(dom[ks]),
                                torch.as_tensor(sp.neuron[ks].astype(np.int64)),
                                torch.as_tensor(sp.sign[ks].astype(np.int64)))


def reach(prob, alpha: Optional[torch.Tensor] = None, beta: Optional[torch.Tensor] = None,
          mode: Optional[int] = None, record: Optional[list] = None, keep_intermediate: bool = False,
          shift: Optional[torch.Tensor] = None, params: Optional[tuple] = None):
    """Bounds for every domain, step and coordinate (Alg. 2 with the closed loop of Sec. IV-E).

    alpha: [D, H, hidden] (MODE_USER only); beta: [nnz] split multipliers (>= 0) or None.
    shift: optional [D, H+1, n] shift of the TM centre, added to c_0 (entry 0) and to c_{t+1} after
    the dynamics of step t (entry t+1), on top of the problem's offsets; used to differentiate V
    with respect to the initial centre and the per-step offsets.
    params: optional (W list, b list) of FP64 tensors replacing the controller's weights and biases
    (to differentiate V with respect to them).
    Returns a dict with lo/hi [D, H+1, n], V [D], status [D] (int64), hull_lo/hull_hi [H+1, n],
    alpha_used [D, H, hidden] (the slopes in effect; zeros at stable neurons),
    and optionally the intermediate pre-activation bounds l/u [D, H, hidden].
    """
    mode = prob.mode if mode is None else mode
    D, n, H, L = prob.D, prob.n, prob.H, prob.L
    widths = prob.widths
    W = [_t(w) for w in prob.W] if params is None else list(params[0])
    b = [_t(x) for x in prob.b] if params is None else list(params[1])
    A, B, e = _t(prob.A), _t(prob.B), _t(prob.e)
    offs = np.concatenate([[0], np.cumsum(widths[1:-1])]).astype(int)
    if mode == MODE_USER and alpha is None:
        raise ValueError("MODE_USER needs alpha")
    splits = _SplitIndex(prob, np.arange(D))
    if beta is None:
        nnz = prob.splits.nnz if prob.splits is not None else 0
        beta = torch.zeros(nnz, dtype=_F64) if prob.beta is None else _t(prob.beta)

    lo0, hi0 = _t(prob.lo), _t(prob.hi)
    eoff = _t(prob.eoff) if getattr(prob, "eoff", None) is not None else None
    # a1: BuildLinearTM over the normalised box
    c = 0.5 * (lo0 + hi0)
    if shift is not None:
        c = c + shift[:, 0, :]
        lo0, hi0 = lo0 + shift[:, 0, :], hi0 + shift[:, 0, :]
    P = torch.diag_embed(0.5 * (hi0 - lo0))
    Ilo = torch.zeros(D, n, dtype=_F64)
    Ihi = torch.zeros(D, n, dtype=_F64)
    v = torch.zeros(D, n, dtype=_F64)
    w = torch.zeros(D, dtype=_F64)
    status = torch.zeros(D, dtype=torch.int64)
    los, his = [lo0], [hi0]
    alpha_used = torch.zeros(D, H, int(offs[-1]), dtype=_F64)
    inter_l, inter_u = [], []

    for t in range(H):
        rs: List[Optional[torch.Tensor]] = [None] * L  # slopes s_m (1-based hidden index m)
        rd: List[Optional[torch.Tensor]] = [None] * L  # intercepts d_m
        step_l, step_u, step_a = [], [], []
        for ell in range(1, L + 1):
            # a4: backward chain from target layer ell down to the input
            Lam = W[ell - 1].expand(D, -1, -1)
            klo = b[ell - 1].expand(D, -1)
            khi = klo
            for m in range(ell - 1, 0, -1):
                s_m, d_m = rs[m], rd[m]
                khi = khi + (pos(Lam) * d_m[:, None, :]).sum(-1)
                klo = klo + (neg(Lam) * d_m[:, None, :]).sum(-1)
                if record is not None:
                    record.append(Lam > 0)
                    record.append(Lam < 0)
                Lam_s = Lam * s_m[:, None, :]
                kb = (Lam_s @ b[m - 1].unsqueeze(-1)).squeeze(-1)
                klo = klo + kb
                khi = khi + kb
                Lam = Lam_s @ W[m - 1]
            # a5: concretisation over the linear TM input (Thm. 3)
            G = Lam @ P
            a = (Lam @ c.unsqueeze(-1)).squeeze(-1)
            Rlo, Rhi = interval_matvec(Lam, Ilo, Ihi)
            if record is not None:
                record.append(Lam > 0)
                record.append(Lam < 0)
            if ell < L:
                gm = G - v[:, None, :]
                gp = G + v[:, None, :]
                if record is not None:
                    record.append(gm > 0)
                    record.append(gp > 0)
                l = a + klo + Rlo - gm.abs().sum(-1) - w[:, None]
                u = a + khi + Rhi + gp.abs().sum(-1) + w[:, None]
                grp = splits.groups.get((t, ell))
                if grp is not None:
                    ks, dom, j, sg = grp
                    # the valid constraint g^T zeta + h >= 0 recorded for each split
                    hh = torch.where(sg > 0, (a + khi + Rhi)[dom, j], -(a + klo + Rlo)[dom, j])
                    gg = sg[:, None].to(_F64) * G[dom, j, :]
                    bk = beta[ks]
                    v = v.index_add(0, dom, bk[:, None] * gg)
                    w = w.index_add(0, dom, bk * hh)
                    posm = torch.zeros(D, widths[ell], dtype=torch.bool)
                    negm = torch.zeros(D, widths[ell], dtype=torch.bool)
                    posm[dom[sg > 0], j[sg > 0]] = True
                    negm[dom[sg < 0], j[sg < 0]] = True
                    l = torch.where(posm & (l < 0), torch.zeros_like(l), l)
                    u = torch.where(negm & (u > 0), torch.zeros_like(u), u)
                # l > u (after clipping, or from a dual certificate) proves the domain empty
                bad = (l > u).any(-1)
                status = torch.where(bad, status | STATUS_INFEASIBLE, status)
                al = alpha[:, t, offs[ell - 1]:offs[ell]] if mode == MODE_USER else None
                s, d, a_used, unstable, br = relax(l, u, al, mode)
                if record is not None:
                    record.append(unstable)
                    record.append(l >= 0)
                    record.append(br)
                rs[ell], rd[ell] = s, d
                step_a.append(torch.where(unstable, a_used, torch.zeros_like(a_used)).detach())
                step_l.append(l)
                step_u.append(u)
            else:
                # a6: controller output as a linear TM
                Pu = G
                cu = a + 0.5 * (klo + khi)
                Iulo = 0.5 * (klo - khi) + Rlo
                Iuhi = 0.5 * (khi - klo) + Rhi
        if step_a:
            alpha_used[:, t, :] = torch.cat(step_a, dim=1)
        if keep_intermediate and step_l:
            inter_l.append(torch.cat(step_l, dim=1))
            inter_u.append(torch.cat(step_u, dim=1))
        # a7: linear dynamics on the TM
        P_n = A @ P + B @ Pu
        c_n = c @ A.T + cu @ B.T + e
        if eoff is not None:
            c_n = c_n + eoff[:, t, :]
        if shift is not None:
            c_n = c_n + shift[:, t + 1, :]
        aLo, aHi = interval_matvec(A, Ilo, Ihi)
        bLo, bHi = interval_matvec(B, Iulo, Iuhi)
        P, c, Ilo, Ihi = P_n, c_n, aLo + bLo, aHi + bHi
        # a8: EvalInt (with the split dual)
        pm = P - v[:, None, :]
        pp = P + v[:, None, :]
        if record is not None:
            record.append(pm > 0)
            record.append(pp > 0)
        los.append(c + Ilo - pm.abs().sum(-1) - w[:, None])
        his.append(c + Ihi + pp.abs().sum(-1) + w[:, None])
        status = torch.where((los[-1] > his[-1]).any(-1), status | STATUS_INFEASIBLE, status)

    lo = torch.stack(los, dim=1)
    hi = torch.stack(his, dim=1)
    fin = torch.isfinite(lo).all(-1).all(-1) & torch.isfinite(hi).all(-1).all(-1)
    status = torch.where(fin, status, status | STATUS_NONFINITE)
    V = (hi[:, 1:, :] - lo[:, 1:, :]).sum(-1).sum(-1)
    feas = (status & STATUS_INFEASIBLE) == 0
    with torch.no_grad():
        if bool(feas.any()):
            hull_lo = lo.detach()[feas].min(dim=0).values
            hull_hi = hi.detach()[feas].max(dim=0).values
        else:
            hull_lo = torch.full((H + 1, n), math.inf, dtype=_F64)
            hull_hi = torch.full((H + 1, n), -math.inf, dtype=_F64)
    out = dict(lo=lo, hi=hi, V=V, status=status, hull_lo=hull_lo, hull_hi=hull_hi, alpha_used=alpha_used)
    if keep_intermediate:
        out["l"] = torch.stack(inter_l, dim=1) if inter_l else None
        out["u"] = torch.stack(inter_u, dim=1) if inter_u else None
    return out


def reach_chunked(prob, chunk: int = 512, **kw):
    """``reach`` over domain chunks (domains are independent; this only bounds memory)."""
    if prob.D <= chunk:
        return reach(prob, **kw)
    parts = []
    for c0 in range(0, prob.D, chunk):
        idx = np.arange(c0, min(prob.D, c0 + chunk))
        sub_kw = dict(kw)
        if sub_kw.get("alpha") is not None:
            sub_kw["alpha"] = sub_kw["alpha"][c0:c0 + len(idx)]
        if sub_kw.get("beta") is not None and prob.splits is not None:
            rp = prob.splits.row_ptr
            sub_kw["beta"] = sub_kw["beta"][int(rp[c0]):int(rp[c0 + len(idx)])]
        parts.append(reach(prob.subset(idx), **sub_kw))
    out = {}
    for k in ("lo", "hi", "V", "status", "alpha_used"):
        out[k] = torch.cat([p[k] for p in parts], dim=0)
    feas = (out["status"] & STATUS_INFEASIBLE) == 0
    out["hull_lo"] = out["lo"][feas].min(dim=0).values
    out["hull_hi"] = out["hi"][feas].max(dim=0).values
    return out


def value_and_grad(prob, alpha: torch.Tensor, beta: Optional[torch.Tensor] = None):
    """V per domain and dV/dalpha, dV/dbeta (reverse-mode AD of the FP64 forward, USER slopes)."""
    a = alpha.detach().clone().requires_grad_(True)
    nnz = prob.splits.nnz if prob.splits is not None else 0
    if beta is None:
        beta = torch.zeros(nnz, dtype=_F64) if prob.beta is None else _t(prob.beta)
    bt = beta.detach().clone().requires_grad_(True)
    res = reach(prob, alpha=a, beta=bt, mode=MODE_USER)
    res["V"].sum().backward()
    ga = a.grad if a.grad is not None else torch.zeros_like(a)
    gb = bt.grad if bt.grad is not None else torch.zeros_like(bt)
    return res, ga, gb


def value_and_shift_grad(prob, alpha: Optional[torch.Tensor] = None, beta: Optional[torch.Tensor] = None):
    """V per domain and dV/dshift [D, H+1, n]: the gradient of V with respect to a shift of the TM
    centre at step t (t = 0: the initial box centre; t >= 1: the offset added after step t-1).  For a
    neural dynamics model over the state augmented by the planned input (workloads.neural_dynamics)
    its action rows are dV/du_t, t = 0..H-1 (reverse-mode AD of the FP64 forward pass)."""
    sh = torch.zeros(prob.D, prob.H + 1, prob.n, dtype=_F64, requires_grad=True)
    kw = dict(mode=MODE_USER, alpha=alpha) if alpha is not None else {}
    res = reach(prob, beta=beta, shift=sh, **kw)
    res["V"].sum().backward()
    return res, sh.grad


def value_and_weight_grad(prob, alpha: Optional[torch.Tensor] = None, beta: Optional[torch.Tensor] = None):
    """V per domain and dV/dW_l, dV/db_l of the controller (V summed over domains; the certified-training
    loss of Sec. V-A differentiates the tube proxy with respect to the model's parameters), by
    reverse-mode AD of the FP64 forward pass (user slopes held fixed when alpha is given)."""
    W = [_t(w).clone().requires_grad_(True) for w in prob.W]
    b = [_t(x).clone().requires_grad_(True) for x in prob.b]
    kw = dict(mode=MODE_USER, alpha=alpha) if alpha is not None else {}
    res = reach(prob, beta=beta, params=(W, b), **kw)
    res["V"].sum().backward()
    return res, [w.grad for w in W], [x.grad for x in b]


def chord_alpha(prob) -> torch.Tensor:
    """The CHORD slopes of the unrefined pass, used as the starting point of refinement."""
    return reach(prob, mode=MODE_CHORD)["alpha_used"]


def optimize_slopes(prob, steps: int, lr_alpha: float, lr_beta: float,
                    alpha0: Optional[torch.Tensor] = None, beta0: Optional[torch.Tensor] = None):
    """Projected-gradient refinement of the slopes (Sec. VI-A "gradient-based refinement").

    alpha <- clip(alpha - lr_alpha g_alpha, 0, 1), beta <- max(beta - lr_beta g_beta, 0);
    keep-best per domain.  Returns V_hist [steps+1] (sum of the per-domain best V after each
    evaluation), the best alpha/beta, and the final best bounds.
    """
    alpha = chord_alpha(prob) if alpha0 is None else alpha0.clone()
    nnz = prob.splits.nnz if prob.splits is not None else 0
    beta = (torch.zeros(nnz, dtype=_F64) if prob.beta is None else _t(prob.beta)) if beta0 is None else beta0.clone()
    dom_of_split = torch.as_tensor(np.repeat(np.arange(prob.D), np.diff(prob.splits.row_ptr))) if nnz else None
    best_V = torch.full((prob.D,), math.inf, dtype=_F64)
    best_alpha = alpha.clone()
    best_beta = beta.clone()
    hist = []
    for it in range(steps + 1):
        res, ga, gb = value_and_grad(prob, alpha, beta)
        V = res["V"].detach()
        better = V < best_V
        best_V = torch.where(better, V, best_V)
        best_alpha[better] = alpha[better]
        if nnz:
            bsel = better[dom_of_split]
            best_beta[bsel] = beta[bsel]
        hist.append(float(best_V.sum()))
        if it == steps:
            break
        alpha = (alpha - lr_alpha * ga).clamp(0.0, 1.0)
        if nnz:
            beta = (beta - lr_beta * gb).clamp(min=0.0)
    return dict(V_hist=hist, alpha=best_alpha, beta=best_beta, best_V=best_V)


def finite_difference(prob, alpha: torch.Tensor, beta: Optional[torch.Tensor], coords, eps: float = 1e-4,
                      which: str = "alpha", shrink: int = 3):
    """Central differences of V (summed over domains) at the given flat coordinates.

    Returns (fd values, ok mask): ok says the activation / sign pattern of the whole pass is
    identical at both evaluation points (no kink inside [-h, +h]).  When a kink lies inside,
    the step h is divided by 10, up to ``shrink`` times, before the coordinate is given up.
    """
    vals, ok = [], []
    base = alpha if which == "alpha" else beta
    for k in coords:
        h = eps
        for _attempt in range(shrink + 1):
            pts, pats = [], []
            for sgn in (1.0, -1.0):
                x = base.detach().clone().reshape(-1)
                x[k] += sgn * h
                x = x.reshape(base.shape)
                rec: list = []
                if which == "alpha":
                    r = reach(prob, alpha=x, beta=beta, mode=MODE_USER, record=rec)
                else:
                    r = reach(prob, alpha=alpha, beta=x, mode=MODE_USER, record=rec)
                pts.append(float(r["V"].sum()))
                pats.append(rec)
            same = all(bool(torch.equal(p, q)) for p, q in zip(pats[0], pats[1]))
            if same:
                break
            h = h / 10.0
        vals.append((pts[0] - pts[1]) / (2 * h))
        ok.append(same)
    return np.array(vals), np.array(ok)


def ibp_reach(prob) -> Dict[str, torch.Tensor]:
    """Plain interval arithmetic through pi and the dynamics (used only for invariants)."""
    lo, hi = _t(prob.lo), _t(prob.hi)
    W = [_t(w) for w in prob.W]
    b = [_t(x) for x in prob.b]
    A, B, e = _t(prob.A), _t(prob.B), _t(prob.e)
    los, his = [lo], [hi]
    for _t_ in range(prob.H):
        hlo, hhi = lo, hi
        for l in range(prob.L):
            zl, zh = interval_matvec(W[l], hlo, hhi)
            zl, zh = zl + b[l], zh + b[l]
            if l < prob.L - 1:
                hlo, hhi = zl.clamp(min=0), zh.clamp(min=0)
            else:
                ulo, uhi = zl, zh
        al, ah = interval_matvec(A, lo, hi)
        bl, bh = interval_matvec(B, ulo, uhi)
        off = _t(prob.eoff)[:, _t_, :] if getattr(prob, "eoff", None) is not None else 0.0
        lo, hi = al + bl + e + off, ah + bh + e + off
        los.append(lo)
        his.append(hi)
    return dict(lo=torch.stack(los, 1), hi=torch.stack(his, 1))
