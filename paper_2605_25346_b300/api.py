"""Python front end of the CUDA library: marshals a ``workloads.Problem`` across the C ABI.

Device memory and streams come from PyTorch; every step of the bound computation runs in
the library's kernels.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import check

BOX_MARGIN = 2.0 ** -18  # default outward margin of reported boxes (relative to their L1 magnitude)
_MODE = {0: _lib.DR_SLOPE_ADAPTIVE, 1: _lib.DR_SLOPE_CHORD, 2: _lib.DR_SLOPE_ZERO, 3: _lib.DR_SLOPE_USER}


def _ptr(a) -> ctypes.c_void_p:
    if isinstance(a, torch.Tensor):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


class Reach:
    """One library context (one device, one stream) holding a loaded problem."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self.lib = _lib.load()
        self.ctx = ctypes.c_void_p()
        self.stream = stream
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        code = self.lib.dr_create(ctypes.byref(self.ctx), device, s)
        if code != _lib.DR_OK:
            raise _lib.DiffReachError(code, self.lib.dr_last_error(None).decode())
        self.device = device
        self.prob = None

    def close(self):
        if self.ctx:
            self.lib.dr_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, code):
        return check(self.ctx, code)

    # ---- problem upload -------------------------------------------------------------------
    def set_options(self, mode: Optional[int] = None, precision: int = _lib.DR_PREC_AUTO, rho: Optional[float] = None,
                    chunk: int = 0, mem_cap: int = 0, box_margin: Optional[float] = None, tuning: int = 0,
                    graphs: int = 0, timing: int = 0, rigorous: int = 0, weight_grad: int = 0, reverse: int = 0):
        o = _lib.dr_options()
        o.weight_grad = weight_grad
        o.reverse = reverse
        o.tuning = tuning
        o.graphs = graphs
        o.timing = timing
        o.rigorous = rigorous
        o.slope_mode = _MODE[mode] if mode is not None else _lib.DR_SLOPE_CHORD
        o.precision = precision
        o.margin_rho = 0.0 if rho is None else rho
        o.chunk_domains = chunk
        o.mem_cap_bytes = mem_cap
        o.box_margin = BOX_MARGIN if box_margin is None else box_margin
        self._c(self.lib.dr_set_options(self.ctx, ctypes.byref(o)))

    def load(self, prob, mode: Optional[int] = None, rho: Optional[float] = None, precision: int = _lib.DR_PREC_AUTO,
             boxes_on_device: bool = False):
        self.prob = prob
        widths = np.asarray(prob.widths, dtype=np.int32)
        self._keep = [np.ascontiguousarray(w, dtype=np.float64) for w in prob.W] + \
                     [np.ascontiguousarray(b, dtype=np.float64) for b in prob.b]
        L = prob.L
        Wp = (ctypes.c_void_p * L)(*[x.ctypes.data for x in self._keep[:L]])
        bp = (ctypes.c_void_p * L)(*[x.ctypes.data for x in self._keep[L:]])
        self._c(self.lib.dr_set_horizon(self.ctx, prob.H))
        self._c(self.lib.dr_load_controller(self.ctx, L, _ptr(widths), Wp, bp, _lib.DR_F64))
        A = np.ascontiguousarray(prob.A, dtype=np.float64)
        B = np.ascontiguousarray(prob.B, dtype=np.float64)
        e = np.ascontiguousarray(prob.e, dtype=np.float64)
        self._c(self.lib.dr_load_dynamics(self.ctx, prob.n, prob.m, _ptr(A), _ptr(B), _ptr(e)))
        m0 = prob.mode if mode is None else mode
        m0 = 1 if m0 == 3 else m0  # user slopes are installed with set_alpha after the boxes
        self.set_options(m0, precision, rho)
        if boxes_on_device:
            lo = torch.as_tensor(prob.lo, dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
            hi = torch.as_tensor(prob.hi, dtype=torch.float64, device=f"cuda:{self.device}").contiguous()
            self._c(self.lib.dr_set_boxes(self.ctx, prob.D, _ptr(lo), _ptr(hi), 1))
            torch.cuda.synchronize()
        else:
            lo = np.ascontiguousarray(prob.lo, dtype=np.float64)
            hi = np.ascontiguousarray(prob.hi, dtype=np.float64)
            self._c(self.lib.dr_set_boxes(self.ctx, prob.D, _ptr(lo), _ptr(hi), 0))
        if prob.splits is not None:
            self.set_splits(prob.splits, prob.beta)
        if getattr(prob, "eoff", None) is not None:
            self.set_step_offsets(prob.eoff)
        # dr_set_boxes resets the slope mode to the default; restore the requested one
        self.set_options(m0, precision, rho)
        return self

    def set_splits(self, splits, beta=None):
        nnz = splits.nnz
        rec = np.zeros((max(nnz, 1), 4), dtype=np.int32)
        rec[:nnz, 0] = splits.t
        rec[:nnz, 1] = splits.layer
        rec[:nnz, 2] = splits.neuron
        rec[:nnz, 3] = splits.sign
        rp = np.ascontiguousarray(splits.row_ptr, dtype=np.int64)
        bt = None if beta is None else np.ascontiguousarray(beta, dtype=np.float32)
        self._c(self.lib.dr_set_splits(self.ctx, _ptr(rp), _ptr(rec), None if bt is None else _ptr(bt)))

    def set_step_offsets(self, eoff):
        """Per-step dynamics offsets [D, H, n] (numpy host array or CUDA tensor); None removes them."""
        if eoff is None:
            self._c(self.lib.dr_set_step_offsets(self.ctx, None, 0))
        elif isinstance(eoff, torch.Tensor):
            e = eoff.to(torch.float64).contiguous()
            self._c(self.lib.dr_set_step_offsets(self.ctx, _ptr(e), 1))
            torch.cuda.synchronize()
        else:
            e = np.ascontiguousarray(eoff, dtype=np.float64)
            self._c(self.lib.dr_set_step_offsets(self.ctx, _ptr(e), 0))

    def shift_gradient(self) -> np.ndarray:
        """dV/d(shift of the TM centre at step t) [D, H+1, n] of the last backward() call."""
        p = self.prob
        g = np.empty((p.D, p.H + 1, p.n))
        self._c(self.lib.dr_get_shift_gradient(self.ctx, _ptr(g), 0))
        return g

    def weight_gradient(self):
        """dV/dW_l, dV/db_l of the controller (lists of numpy arrays shaped like the problem's W, b),
        summed over domains, of the last backward() call made with set_options(weight_grad=1)."""
        p = self.prob
        w = p.widths
        nW = sum(int(w[l + 1]) * int(w[l]) for l in range(p.L))
        nb = sum(int(w[l + 1]) for l in range(p.L))
        gW = np.empty(nW)
        gb = np.empty(nb)
        self._c(self.lib.dr_get_weight_gradient(self.ctx, _ptr(gW), _ptr(gb), 0))
        outW, outb, oW, ob = [], [], 0, 0
        for l in range(p.L):
            r, k = int(w[l + 1]), int(w[l])
            outW.append(gW[oW:oW + r * k].reshape(r, k))
            outb.append(gb[ob:ob + r])
            oW += r * k
            ob += r
        return outW, outb

    # ---- computation ---------------------------------------------------------------------
    def bounds(self, on_device: bool = True, hull: bool = True):
        """Boxes [D, H+1, n], hull [H+1, n] x2 and status [D] (device tensors, or numpy on host)."""
        p = self.prob
        D, H, n = p.D, p.H, p.n
        if on_device:
            dev = f"cuda:{self.device}"
            lo = torch.empty(D, H + 1, n, dtype=torch.float64, device=dev)
            hi = torch.empty_like(lo)
            hl = torch.empty(H + 1, n, dtype=torch.float64, device=dev)
            hh = torch.empty_like(hl)
            st = torch.empty(D, dtype=torch.int32, device=dev)
        else:
            lo = np.empty((D, H + 1, n))
            hi = np.empty_like(lo)
            hl = np.empty((H + 1, n))
            hh = np.empty_like(hl)
            st = np.empty(D, dtype=np.uint32)
        self._c(self.lib.dr_compute_bounds(self.ctx, _ptr(lo), _ptr(hi), _ptr(hl) if hull else None,
                                           _ptr(hh) if hull else None, _ptr(st), 1 if on_device else 0))
        return dict(lo=lo, hi=hi, hull_lo=hl, hull_hi=hh, status=st)

    def objective(self) -> np.ndarray:
        V = np.empty(self.prob.D)
        self._c(self.lib.dr_get_objective(self.ctx, _ptr(V), 0))
        return V

    def get_alpha(self) -> np.ndarray:
        p = self.prob
        a = np.empty((p.D, p.H, p.hidden), dtype=np.float32)
        self._c(self.lib.dr_get_alpha(self.ctx, _ptr(a), 0))
        return a

    def set_alpha(self, alpha):
        a = np.ascontiguousarray(alpha, dtype=np.float32)
        self._c(self.lib.dr_set_alpha(self.ctx, _ptr(a), 0))

    def get_beta(self) -> np.ndarray:
        p = self.prob
        nnz = p.splits.nnz if p.splits is not None else 0
        b = np.empty(max(nnz, 1), dtype=np.float32)
        self._c(self.lib.dr_get_beta(self.ctx, _ptr(b), 0))
        return b[:nnz]

    def set_beta(self, beta):
        b = np.ascontiguousarray(beta, dtype=np.float32)
        self._c(self.lib.dr_set_beta(self.ctx, _ptr(b), 0))

    def backward(self, wlo=None, whi=None):
        """dV/dalpha [D, H, hidden] and dV/dbeta [nnz] at the current slopes (host numpy).

        wlo/whi: optional upstream gradients [D, H+1, n] of the lower/upper bounds (default: the
        tube-volume proxy, -1/+1 on steps 1..H)."""
        p = self.prob
        nnz = p.splits.nnz if p.splits is not None else 0
        ga = np.empty((p.D, p.H, p.hidden), dtype=np.float32)
        gb = np.empty(max(nnz, 1), dtype=np.float32)
        wl = None if wlo is None else np.ascontiguousarray(wlo, dtype=np.float64)
        wh = None if whi is None else np.ascontiguousarray(whi, dtype=np.float64)
        self._c(self.lib.dr_backward(self.ctx, None if wl is None else _ptr(wl), None if wh is None else _ptr(wh),
                                     _ptr(ga), _ptr(gb), 0))
        return ga, gb[:nnz]

    def optimize(self, steps: int, lr_alpha: float, lr_beta: float = 0.0):
        hist = np.empty(steps + 1)
        self._c(self.lib.dr_optimize_slopes(self.ctx, steps, lr_alpha, lr_beta, _ptr(hist)))
        return hist

    def launches(self) -> int:
        return int(self.lib.dr_kernel_launches(self.ctx))

    def graph_replays(self) -> int:
        return int(self.lib.dr_graph_replays(self.ctx))

    def kernel_timing(self, which: int = _lib.DR_KT_GEMM_ALL, min_rows: int = 0):
        """(launches, total ms, algorithmic FLOP) of the timed tensor-core GEMM launches of a class with
        at least `min_rows` rows (timing is switched on with set_options(timing=1))."""
        nl, ms, fl = ctypes.c_int64(0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._c(self.lib.dr_kernel_timing(self.ctx, which, min_rows, ctypes.byref(nl), ctypes.byref(ms),
                                          ctypes.byref(fl)))
        return int(nl.value), float(ms.value), float(fl.value)


def gemm_tuning_report() -> str:
    """The tensor-core GEMM autotuner's choices so far in this process (one line per GEMM shape)."""
    lib = _lib.load()
    need = int(lib.dr_gemm_tuning_report(None, 0))
    buf = ctypes.create_string_buffer(max(need, 1))
    lib.dr_gemm_tuning_report(buf, need)
    return buf.value.decode()


class BoundsFunction(torch.autograd.Function):
    """Differentiable bounds: (alpha, beta) -> (lo, hi), backward through the library's adjoint.

    alpha [D, H, hidden] float32 and beta [nnz] float32 are CUDA tensors; lo/hi [D, H+1, n]
    float64.  The backward pass hands torch's upstream gradients of lo and hi to dr_backward at the
    slopes and multipliers this forward call was given (saved with the graph), so several forward
    calls on one Reach before a backward each get their own gradient.
    """

    @staticmethod
    def _install(reach: "Reach", a: torch.Tensor, b: torch.Tensor):
        reach._c(reach.lib.dr_set_alpha(reach.ctx, _ptr(a), 1))
        if b.numel():
            reach._c(reach.lib.dr_set_beta(reach.ctx, _ptr(b), 1))

    @staticmethod
    def forward(ctx, reach: "Reach", alpha: torch.Tensor, beta: torch.Tensor):
        a = alpha.detach().to(torch.float32).contiguous()
        b = beta.detach().to(torch.float32).contiguous()
        BoundsFunction._install(reach, a, b)
        out = reach.bounds(on_device=True, hull=False)
        ctx.reach = reach
        ctx.dtypes = (alpha.dtype, beta.dtype)
        ctx.save_for_backward(a, b)
        return out["lo"], out["hi"]

    @staticmethod
    def backward(ctx, glo, ghi):
        r = ctx.reach
        p = r.prob
        a, b = ctx.saved_tensors
        dev = f"cuda:{r.device}"
        zeros = torch.zeros(p.D, p.H + 1, p.n, dtype=torch.float64, device=dev)
        wlo = (glo if glo is not None else zeros).to(torch.float64).contiguous()
        whi = (ghi if ghi is not None else zeros).to(torch.float64).contiguous()
        ga = torch.empty(a.shape, dtype=torch.float32, device=dev)
        gb = torch.empty(max(1, b.numel()), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        BoundsFunction._install(r, a, b)
        r._c(r.lib.dr_backward(r.ctx, _ptr(wlo), _ptr(whi), _ptr(ga), _ptr(gb), 1))
        return None, ga.to(ctx.dtypes[0]), gb[: b.numel()].reshape(b.shape).to(ctx.dtypes[1])


def bounds(reach: "Reach", alpha: torch.Tensor, beta: torch.Tensor):
    """(lo, hi) with autograd through the CUDA adjoint (see BoundsFunction)."""
    return BoundsFunction.apply(reach, alpha, beta)
