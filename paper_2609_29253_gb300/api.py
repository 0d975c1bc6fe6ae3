"""Python API over the C ABI: plans, operator calls and autograd.

Tensors are torch CUDA tensors (float32, contiguous).  Workspaces are
allocated through torch and handed to the library, which allocates nothing per
call.  Every operator step runs in the CUDA library (``_lib``); nothing here
computes.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from .workloads import Workload


def system_taps(w: Workload, device=None) -> np.ndarray:
    """Discrete system kernel h-bar (Eq. def_bh) computed on the GPU, FP64."""
    taps = torch.empty(w.T, dtype=torch.float64, device=device or "cuda")
    _lib.pat_system_kernel(w.rbf_kind, w.kappa, w.eir_kind, w.eir_par, w.c, w.fs, w.U, w.n_lo, taps)
    return taps.cpu().numpy()


def system_taps_dc(w: Workload, device=None) -> torch.Tensor:
    """d h-bar / dc for the workload's tap window, computed on the GPU, FP64
    (device tensor, the argument of Plan.forward_dc)."""
    dtaps = torch.empty(w.T, dtype=torch.float64, device=device or "cuda")
    _lib.pat_system_kernel_dc(w.rbf_kind, w.kappa, w.eir_kind, w.eir_par, w.c, w.fs, w.U, w.n_lo, dtaps)
    return dtaps


class Plan:
    """An operator A (and A^T) for one grid, one set of transducer positions
    and one time axis; see pat_plan_create in include/pat.h."""

    def __init__(self, w: Workload, taps: np.ndarray | None = None, allow_clip: bool = False, conv_tc: bool = False,
                 piecewise_planes: int = 0, device=None):
        self.w = w
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            if taps is None:
                taps = system_taps(w, self.device)
            self.taps = np.ascontiguousarray(taps, dtype=np.float64)
            flags = (_lib.PAT_FLAG_ALLOW_CLIP if allow_clip else 0) | (_lib.PAT_FLAG_CONV_TC if conv_tc else 0) | \
                    (_lib.PAT_FLAG_PIECEWISE_PLANES if piecewise_planes > 0 else 0)
            self.handle = _lib.pat_plan_create(w.n, w.origin, w.pitch, w.tx, w.c, w.fs, w.t0, w.L, w.U, w.dl,
                                               w.method, w.q1, w.q2, flags, w.kappa, self.taps, w.n_lo,
                                               np_planes=piecewise_planes)
        self.info = _lib.pat_plan_get_info(self.handle)
        self._ws = {}
        self.N, self.K, self.L, self.UL = w.N, w.K, w.L, w.UL

    def close(self):
        if getattr(self, "handle", None) is not None:
            _lib.pat_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, op: int) -> torch.Tensor:
        need = _lib.pat_workspace_bytes(self.handle, op)
        ws = self._ws.get(op)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self._ws[op] = ws
        return ws

    def _f32(self, t, n):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"expected a contiguous float32 CUDA tensor with {n} elements")
        return t

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        x = self._f32(x, self.N)
        s = out if out is not None else torch.empty((self.K, self.L), dtype=torch.float32, device=self.device)
        _lib.pat_forward(self.handle, x, s, self.workspace(_lib.PAT_OP_FORWARD))
        return s

    def adjoint(self, s: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        s = self._f32(s, self.K * self.L)
        z = out if out is not None else torch.empty(self.N, dtype=torch.float32, device=self.device)
        _lib.pat_adjoint(self.handle, s, z, self.workspace(_lib.PAT_OP_ADJOINT))
        return z

    def forward_geometric(self, x: torch.Tensor) -> torch.Tensor:
        x = self._f32(x, self.N)
        f = torch.empty((self.K, self.UL), dtype=torch.float32, device=self.device)
        _lib.pat_forward_geometric(self.handle, x, f, self.workspace(_lib.PAT_OP_FORWARD))
        return f

    def adjoint_geometric(self, v: torch.Tensor) -> torch.Tensor:
        v = self._f32(v, self.K * self.UL)
        z = torch.empty(self.N, dtype=torch.float32, device=self.device)
        _lib.pat_adjoint_geometric(self.handle, v, z, self.workspace(_lib.PAT_OP_ADJOINT))
        return z

    def conv_forward(self, f: torch.Tensor) -> torch.Tensor:
        f = self._f32(f, self.K * self.UL)
        s = torch.empty((self.K, self.L), dtype=torch.float32, device=self.device)
        _lib.pat_conv_forward(self.handle, f, s)
        return s

    def conv_split(self, f: torch.Tensor) -> torch.Tensor:
        """f [K][U L] as the BF16 hi and lo planes of pat_conv_split (int16
        storage, [2][K][ld]; tensor-core plans only)."""
        f = self._f32(f, self.K * self.UL)
        n = _lib.pat_workspace_bytes(self.handle, _lib.PAT_OP_CONV_SPLIT) // 2
        planes = torch.empty(n, dtype=torch.int16, device=self.device)
        _lib.pat_conv_split(self.handle, f, planes)
        return planes

    def conv_forward_split(self, planes: torch.Tensor) -> torch.Tensor:
        """s [K][L] from the planes of conv_split (pat_conv_forward_split)."""
        s = torch.empty((self.K, self.L), dtype=torch.float32, device=self.device)
        _lib.pat_conv_forward_split(self.handle, planes, s)
        return s

    def conv_forward_split_withheld(self, planes: torch.Tensor) -> torch.Tensor:
        """The give-up path of the split-plane kernel (pat_conv_forward_split_withheld):
        s is undefined afterwards and info["tc_error"] non-zero."""
        s = torch.empty((self.K, self.L), dtype=torch.float32, device=self.device)
        _lib.pat_conv_forward_split_withheld(self.handle, planes, s)
        return s

    def clear_tc_error(self) -> None:
        _lib.pat_plan_clear_tc_error(self.handle)

    def conv_adjoint(self, s: torch.Tensor) -> torch.Tensor:
        s = self._f32(s, self.K * self.L)
        v = torch.empty((self.K, self.UL), dtype=torch.float32, device=self.device)
        _lib.pat_conv_adjoint(self.handle, s, v)
        return v

    def forward_dc(self, x: torch.Tensor, dtaps: torch.Tensor | None = None) -> torch.Tensor:
        """d(A x)/dc at the plan's speed of sound (see pat_forward_dc)."""
        x = self._f32(x, self.N)
        if dtaps is None:
            dtaps = self._dtaps()
        ds = torch.empty((self.K, self.L), dtype=torch.float32, device=self.device)
        _lib.pat_forward_dc(self.handle, x, dtaps, ds, self.workspace(_lib.PAT_OP_FORWARD_DC))
        return ds

    def autotune(self, x: torch.Tensor | None = None) -> dict:
        """Pick the fastest launch shapes for this plan (pat_plan_autotune)."""
        x = self._f32(x, self.N) if x is not None else torch.ones(self.N, dtype=torch.float32, device=self.device)
        _lib.pat_plan_autotune(self.handle, x, self.workspace(_lib.PAT_OP_AUTOTUNE))
        self.info = _lib.pat_plan_get_info(self.handle)
        return {"fwd_blocks": self.info["fwd_blocks"], "adj_blocks": self.info["adj_blocks"]}

    def _dtaps(self) -> torch.Tensor:
        if getattr(self, "_dtaps_t", None) is None:
            with torch.cuda.device(self.device):
                self._dtaps_t = system_taps_dc(self.w, self.device)
        return self._dtaps_t

    def recon(self, s: torch.Tensor, x0: torch.Tensor | None = None, iters: int = 50, lambda_R: float = 0.0,
              step: float = 0.0) -> torch.Tensor:
        """Projected FISTA for Eq. (nnls_tik); step <= 0 estimates 1/|A^T A + lambda|."""
        s = self._f32(s, self.K * self.L)
        x = x0.clone() if x0 is not None else torch.zeros(self.N, dtype=torch.float32, device=self.device)
        _lib.pat_recon(self.handle, s, x, iters, lambda_R, step, self.workspace(_lib.PAT_OP_RECON))
        return x


def recon_batch(plans: list, s_list: list, x0_list: list | None = None, iters: int = 50, lambdas=None,
                steps=None) -> list:
    """Projected FISTA for several independent problems (pat_recon_batch):
    one CUDA graph per iteration of all problems, each on its own branch."""
    xs = [x0.clone() if x0 is not None else torch.zeros(p.N, dtype=torch.float32, device=p.device)
          for p, x0 in zip(plans, x0_list or [None] * len(plans))]
    s_list = [p._f32(s, p.K * p.L) for p, s in zip(plans, s_list)]
    ws = [p.workspace(_lib.PAT_OP_RECON) for p in plans]
    lambdas = lambdas if lambdas is not None else [0.0] * len(plans)
    _lib.pat_recon_batch([p.handle for p in plans], s_list, xs, iters, lambdas, steps, ws)
    return xs


def plan_from_workload(w: Workload, **kw) -> Plan:
    return Plan(w, **kw)


class PatForward(torch.autograd.Function):
    """s = A x with backward A^T (the exact transpose, App. G)."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, gs):
        return ctx.plan.adjoint(gs.contiguous()), None


class PatForwardSpeed(torch.autograd.Function):
    """s = A(c) x with gradients for x (A^T, App. G) and for the speed of
    sound c (the scalar <ds, dA/dc x>, pat_forward_dc).  c is a 0-d tensor
    equal to the plan's speed of sound; the plan fixes the bins."""

    @staticmethod
    def forward(ctx, x, c, plan):
        if abs(float(c) - plan.w.c) > 1e-9 * plan.w.c:
            raise ValueError(f"c = {float(c)} differs from the plan's {plan.w.c}: build a plan at this c")
        ctx.plan = plan
        ctx.save_for_backward(x)
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, gs):
        (x,) = ctx.saved_tensors
        gs = gs.contiguous()
        gx = ctx.plan.adjoint(gs) if ctx.needs_input_grad[0] else None
        gc = None
        if ctx.needs_input_grad[1]:
            ds = ctx.plan.forward_dc(x.detach().contiguous())
            gc = (gs.double() * ds.double()).sum().to(torch.float32)
        return gx, gc, None


def forward(plan: Plan, x: torch.Tensor, c: torch.Tensor | None = None) -> torch.Tensor:
    """s = A x; with c (a 0-d tensor) the speed of sound is differentiable too."""
    if c is None:
        return PatForward.apply(x, plan)
    return PatForwardSpeed.apply(x, c, plan)


def adjoint(plan: Plan, s: torch.Tensor) -> torch.Tensor:
    return plan.adjoint(s.contiguous())
