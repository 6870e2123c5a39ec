"""Python front end of the learnable multigrid (torch tensors in, torch out).

Every numerical step runs in libmg.so's CUDA kernels; this module passes
pointers, sizes and the current torch stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L
from .hierarchy import Hierarchy


@dataclass
class LMGParams:
    """Theta of Sec. 3: per level l < J-1: theta_l, eta_l and (w1, w2) of the
    SAGEConvs Phi_B, Phi_R, Phi_P; nu_pre/nu_post smoothing steps."""
    theta: np.ndarray
    eta: np.ndarray
    wB: np.ndarray
    wR: np.ndarray
    wP: np.ndarray
    nu_pre: int = 2
    nu_post: int = 2

    @staticmethod
    def identity(J: int, omega: float = 2.0 / 3.0, nu: int = 2) -> "LMGParams":
        """Sec. 3.4: W1 = 1, W2 = 0, theta = omega, eta = 1 (classical cycle)."""
        m = J - 1
        w = np.tile([1.0, 0.0], (m, 1))
        return LMGParams(np.full(m, omega), np.ones(m), w.copy(), w.copy(), w.copy(), nu, nu)

    @property
    def J(self) -> int:
        return int(self.theta.size) + 1

    def flat(self) -> np.ndarray:
        """[J-1][8]: theta, eta, wB1, wB2, wR1, wR2, wP1, wP2."""
        return np.concatenate([self.theta[:, None], self.eta[:, None], self.wB, self.wR, self.wP],
                              axis=1).ravel()

    @staticmethod
    def from_flat(x, nu_pre: int = 2, nu_post: int = 2) -> "LMGParams":
        x = np.asarray(x, dtype=np.float64).reshape(-1, 8)
        return LMGParams(x[:, 0].copy(), x[:, 1].copy(), x[:, 2:4].copy(), x[:, 4:6].copy(),
                         x[:, 6:8].copy(), nu_pre, nu_post)

    def with_levels(self, J: int) -> "LMGParams":
        """Weight transfer to a hierarchy with J levels: levels beyond the
        trained ones copy the deepest trained level (Sec. 4.2 transfer rule)."""
        x = self.flat().reshape(-1, 8)
        if J - 1 <= x.shape[0]:
            y = x[:J - 1]
        else:
            y = np.concatenate([x, np.repeat(x[-1:], J - 1 - x.shape[0], axis=0)], 0)
        return LMGParams.from_flat(y, self.nu_pre, self.nu_post)

    def c_struct(self):
        arrs = [L.as_f64(a).ravel() for a in (self.theta, self.eta, self.wB, self.wR, self.wP)]
        p = L.Params(self.J, int(self.nu_pre), int(self.nu_post),
                     *[L.ptr(a, L.f64p) for a in arrs])
        return p, arrs


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class SolveInfo:
    status: int
    iters: np.ndarray
    relres: np.ndarray
    extra: dict = field(default_factory=dict)


class Solver:
    """A hierarchy resident on the current CUDA device.

    precision 64: the V-cycle runs in FP64; precision 32: in FP32, and solve()
    wraps it in FP64 iterative refinement."""

    def __init__(self, hier: Hierarchy, params: LMGParams, precision: int = 32,
                 max_batch: int = 1, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2608_29082_b300.Solver needs a CUDA device")
        self.lib = L.lib()
        self.hier = hier
        self.precision = int(precision)
        self.max_batch = int(max_batch)
        if isinstance(device, torch.device):
            self.device = device
        else:
            self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                       else int(device))
        self.dtype = torch.float64 if self.precision == 64 else torch.float32
        self.params = params
        h, Aarr, keep = hier.c_structs()
        p, pkeep = params.c_struct()
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.mg_setup(C.byref(ctx), C.byref(h), Aarr, C.byref(p), self.max_batch,
                                   self.precision, _stream_handle())
        L.check(st)
        self.ctx = ctx
        self.n = hier.sizes

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------------
    def set_params(self, params: LMGParams):
        p, keep = params.c_struct()
        L.check(self.lib.mg_set_params(self.ctx, C.byref(p)), self.ctx)
        self.params = params

    def set_cheb(self, coef: np.ndarray | None):
        """ChebConv smoother of degree K = coef.shape[1] - 1 (coef [J-1, K+1],
        level l's c_0..c_K), or None for the SAGEConv smoother (mg_set_cheb)."""
        if coef is None:
            L.check(self.lib.mg_set_cheb(self.ctx, 0, None), self.ctx)
            return
        c = np.ascontiguousarray(coef, dtype=np.float64)
        if c.ndim != 2 or c.shape[0] != self.hier.J - 1 or c.shape[1] < 2:
            raise ValueError(f"coef: expected shape ({self.hier.J - 1}, K+1) with K >= 1")
        L.check(self.lib.mg_set_cheb(self.ctx, c.shape[1] - 1, L.ptr(c, L.f64p)), self.ctx)

    def _vec(self, x: torch.Tensor, n: int, dtype, name: str) -> torch.Tensor:
        if x.device != self.device or x.dtype != dtype or not x.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous {dtype} tensor on {self.device}")
        if x.dim() == 1:
            x = x.view(-1, 1)
        if x.shape[0] != n or x.shape[1] < 1 or x.shape[1] > self.max_batch:
            raise ValueError(f"{name}: expected shape ({n}, 1..{self.max_batch}), got {tuple(x.shape)}")
        return x

    def vcycle(self, f: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
        """u <- LMG(A, f, u) in place (context precision)."""
        f2 = self._vec(f, self.n[0], self.dtype, "f")
        u2 = self._vec(u, self.n[0], self.dtype, "u")
        L.check(self.lib.mg_vcycle(self.ctx, C.c_void_p(f2.data_ptr()), C.c_void_p(u2.data_ptr()),
                                   f2.shape[1], _stream_handle()), self.ctx)
        return u

    def fmg(self, f: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
        """u <- one full multigrid application (nested iteration) on f; u's
        input is not read (context precision)."""
        f2 = self._vec(f, self.n[0], self.dtype, "f")
        u2 = self._vec(u, self.n[0], self.dtype, "u")
        L.check(self.lib.mg_fmg(self.ctx, C.c_void_p(f2.data_ptr()), C.c_void_p(u2.data_ptr()),
                                f2.shape[1], _stream_handle()), self.ctx)
        return u

    def solve(self, f: torch.Tensor, u: torch.Tensor | None = None, tol: float = 1e-8,
              max_iter: int = 100, method: str = "refine",
              restart: int = 30) -> tuple[torch.Tensor, SolveInfo]:
        """FP64 f, u (u = initial guess, zero if None) -> (u, info).
        method "refine": stationary cycles (FP64 context) or FP64 iterative
        refinement around FP32 cycles; "fcg": flexible CG with the cycle (or
        full multigrid, option "fcg_precond") as preconditioner; "fgmres":
        restarted flexible GMRES (restart) with the same preconditioners."""
        f2 = self._vec(f, self.n[0], torch.float64, "f")
        if u is None:
            u = torch.zeros_like(f)
        u2 = self._vec(u, self.n[0], torch.float64, "u")
        B = f2.shape[1]
        iters = np.zeros(B, dtype=np.int32)
        relres = np.zeros(B)
        if method == "fgmres":
            st = self.lib.mg_solve_fgmres(self.ctx, C.c_void_p(f2.data_ptr()),
                                          C.c_void_p(u2.data_ptr()), B, float(tol), int(max_iter),
                                          int(restart), L.ptr(iters, L.i32p),
                                          L.ptr(relres, L.f64p), _stream_handle())
        else:
            fn = {"refine": self.lib.mg_solve, "fcg": self.lib.mg_solve_fcg}[method]
            st = fn(self.ctx, C.c_void_p(f2.data_ptr()), C.c_void_p(u2.data_ptr()), B,
                    float(tol), int(max_iter), L.ptr(iters, L.i32p),
                    L.ptr(relres, L.f64p), _stream_handle())
        L.check(st, self.ctx, allow=(L.MG_OK, L.MG_NOT_CONVERGED))
        return u, SolveInfo(st, iters, relres)

    def solve_host(self, f: np.ndarray, u: np.ndarray | None = None, tol: float = 1e-8,
                   max_iter: int = 100) -> tuple[np.ndarray, SolveInfo]:
        """Host FP64 arrays (n, B): copies in, solves, copies out."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.ndim == 1:
            f = f[:, None]
        u = np.zeros_like(f) if u is None else np.ascontiguousarray(u, dtype=np.float64)
        B = f.shape[1]
        iters = np.zeros(B, dtype=np.int32)
        relres = np.zeros(B)
        st = self.lib.mg_solve_host(self.ctx, L.ptr(f, L.f64p), L.ptr(u, L.f64p), B, float(tol),
                                    int(max_iter), L.ptr(iters, L.i32p), L.ptr(relres, L.f64p),
                                    _stream_handle())
        L.check(st, self.ctx, allow=(L.MG_OK, L.MG_NOT_CONVERGED))
        return u, SolveInfo(st, iters, relres)

    def level_apply(self, level: int, op: str, x: torch.Tensor, y: torch.Tensor | None,
                    out: torch.Tensor):
        B = x.shape[1] if x.dim() == 2 else 1
        yp = C.c_void_p(y.data_ptr()) if y is not None else None
        L.check(self.lib.mg_level_apply(self.ctx, level, L.OPS[op], C.c_void_p(x.data_ptr()), yp,
                                        C.c_void_p(out.data_ptr()), B, _stream_handle()), self.ctx)
        return out

    def vcycle_profile(self, f: torch.Tensor, u: torch.Tensor) -> list[tuple[str, int, float]]:
        """One V-cycle with CUDA events around every kernel on the current
        stream: [(kernel name, level, ms)] in launch order."""
        f2 = self._vec(f, self.n[0], self.dtype, "f")
        u2 = self._vec(u, self.n[0], self.dtype, "u")
        cap = 4096
        buf = (L.KernelTime * cap)()
        n = C.c_int32(0)
        L.check(self.lib.mg_vcycle_profile(self.ctx, C.c_void_p(f2.data_ptr()),
                                           C.c_void_p(u2.data_ptr()), f2.shape[1], buf, cap,
                                           C.byref(n), _stream_handle()), self.ctx)
        return [(self.lib.mg_kernel_name(buf[k].kernel).decode(), buf[k].level, buf[k].ms)
                for k in range(n.value)]

    def set_option(self, name: str, value: int):
        """Launch-shape options ("tail_work", "pdl", "multi_rhs", "device_loop",
        "halo_rows"; results bitwise unchanged) and the flexible-CG
        preconditioner ("fcg_precond": 0 V-cycle, 1 full multigrid)."""
        L.check(self.lib.mg_set_option(self.ctx, L.OPTIONS[name], int(value)), self.ctx)

    # ------------------------------------------------------------ training
    def forward_record(self, f: torch.Tensor, u: torch.Tensor, n_cycles: int) -> torch.Tensor:
        """n_cycles cycles on u in place, recording per-level checkpoints."""
        f2 = self._vec(f, self.n[0], self.dtype, "f")
        u2 = self._vec(u, self.n[0], self.dtype, "u")
        L.check(self.lib.mg_forward_record(self.ctx, C.c_void_p(f2.data_ptr()),
                                           C.c_void_p(u2.data_ptr()), f2.shape[1], int(n_cycles),
                                           _stream_handle()), self.ctx)
        return u

    def backward(self, grad_u_out: torch.Tensor, n_cycles: int, want_inputs: bool = True):
        """Adjoint of the recorded cycles: (dL/du_0, dL/df, dL/dTheta [J-1, 8] FP64)."""
        g = self._vec(grad_u_out, self.n[0], self.dtype, "grad_u_out")
        gin = torch.empty_like(g) if want_inputs else None
        gf = torch.empty_like(g) if want_inputs else None
        gp = torch.empty((self.hier.J - 1, 8), dtype=torch.float64, device=self.device)
        L.check(self.lib.mg_vcycle_backward(
            self.ctx, int(n_cycles), C.c_void_p(g.data_ptr()),
            C.c_void_p(gin.data_ptr()) if gin is not None else None,
            C.c_void_p(gf.data_ptr()) if gf is not None else None,
            C.c_void_p(gp.data_ptr()), _stream_handle()), self.ctx)
        return gin, gf, gp

    def residual_loss(self, f: torch.Tensor, u: torch.Tensor, weights: torch.Tensor | None = None,
                      grad: bool = False):
        """(sum_b w_b ||f_b - A u_b||^2, per-rhs ||r_b||^2, gradient w.r.t. u or None),
        all device tensors."""
        f2 = self._vec(f, self.n[0], self.dtype, "f")
        u2 = self._vec(u, self.n[0], self.dtype, "u")
        B = f2.shape[1]
        per = torch.empty(B, dtype=torch.float64, device=self.device)
        loss = torch.empty((), dtype=torch.float64, device=self.device) if weights is not None else None
        g = torch.empty_like(u2) if (grad and weights is not None) else None
        L.check(self.lib.mg_residual_loss(
            self.ctx, C.c_void_p(f2.data_ptr()), C.c_void_p(u2.data_ptr()), B,
            C.c_void_p(weights.data_ptr()) if weights is not None else None,
            C.c_void_p(loss.data_ptr()) if loss is not None else None,
            C.c_void_p(per.data_ptr()), C.c_void_p(g.data_ptr()) if g is not None else None,
            _stream_handle()), self.ctx)
        return loss, per, g

    def kernel_launches(self) -> int:
        return int(self.lib.mg_kernel_launches(self.ctx))
