"""Two features per node (d = 2): the learnable cycle on complex systems.

Binding of the mg2_* entry points of libmg.so (include/mg.h).  The Helmholtz
setting of Sec. 4.2 carries (Re u, Im u) as two node features, and every
SAGEConv holds W_1, W_2 in R^{2x2} (Sec. 3.2).  The host set-up runs in the
library's native complex Galerkin and elimination helpers (the drop rule on
complex moduli); this module only marshals arrays.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .solver import SolveInfo, _stream_handle

DROP_TOL = 1e-12


@dataclass
class Hierarchy2:
    """Interior complex operators A[l], real prolongations P[l] (l < J-1) and
    1/deg per level (graph of the operator before Dirichlet elimination)."""
    A: list
    P: list
    inv_deg: list

    @property
    def J(self) -> int:
        return len(self.A)

    @property
    def sizes(self) -> list[int]:
        return [a.shape[0] for a in self.A]

    @staticmethod
    def from_problem(problem, drop_tol: float = DROP_TOL) -> "Hierarchy2":
        """Duck-typed: .mesh.levels[l].{nv, boundary, parent}, .A_full
        (scipy CSR, complex, all vertices of the finest level).  Every step
        of the set-up runs in libmg.so (mg_eliminate_complex, mg_prolongation,
        mg_galerkin_complex); numpy only holds arrays."""
        lib = L.lib()
        lv = problem.mesh.levels
        Af = L.HostCSRComplex.from_scipy(problem.A_full.tocsr().astype(np.complex128))
        A, P, inv_deg = [], [], []
        for lev, ML in enumerate(lv):
            bnd = np.ascontiguousarray(ML.boundary, dtype=np.uint8)
            deg = np.zeros(int((bnd == 0).sum()))
            o = L.CSROwned()
            L.check(lib.mg_eliminate_complex(C.byref(Af.c), L.ptr(bnd, L.u8p), drop_tol, C.byref(o),
                                             L.ptr(deg, L.f64p)))
            A.append(L.take_owned_complex(o).to_scipy())
            inv_deg.append(deg)
            if lev < len(lv) - 1:
                par = L.as_i32(ML.parent)
                bc = np.ascontiguousarray(lv[lev + 1].boundary, dtype=np.uint8)
                o = L.CSROwned()
                L.check(lib.mg_prolongation(L.ptr(par, L.i32p), ML.nv, L.ptr(bnd, L.u8p),
                                            lv[lev + 1].nv, L.ptr(bc, L.u8p), C.byref(o)))
                P.append(L.take_owned(o).to_scipy())
                o = L.CSROwned()
                L.check(lib.mg_galerkin_complex(C.byref(Af.c), L.ptr(par, L.i32p), lv[lev + 1].nv,
                                                drop_tol, C.byref(o)))
                Af = L.take_owned_complex(o)
        return Hierarchy2(A, P, inv_deg)


@dataclass
class Params2:
    """theta[l], eta[l]; WB, WR, WP of shape (J-1, 2, 2, 2) = per level
    (W_1, W_2), each acting on the feature column (Re, Im)."""
    theta: np.ndarray
    eta: np.ndarray
    WB: np.ndarray
    WR: np.ndarray
    WP: np.ndarray
    nu_pre: int = 1
    nu_post: int = 1

    @staticmethod
    def identity(J: int, omega: float = 2.0 / 3.0, nu: int = 1) -> "Params2":
        """W_1 = I, W_2 = 0, theta = omega, eta = 1: the classical
        damped-Jacobi cycle on the complex system."""
        W = np.zeros((J - 1, 2, 2, 2))
        W[:, 0] = np.eye(2)
        return Params2(np.full(J - 1, omega), np.ones(J - 1), W.copy(), W.copy(), W.copy(),
                       nu, nu)


class Solver2:
    """A device-resident complex hierarchy and its two-feature cycle (FP64
    or FP32); vectors are torch complex128 / complex64 tensors (n, nrhs)."""

    def __init__(self, hier: Hierarchy2, params: Params2, precision: int = 64,
                 max_batch: int = 1):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2608_29082_b300.Solver2 needs a CUDA device")
        self.lib = L.lib()
        self.hier = hier
        self.precision = int(precision)
        self.max_batch = int(max_batch)
        self.dtype = torch.complex128 if self.precision == 64 else torch.complex64
        self.n = hier.sizes
        keep = []
        levels = (L.Level2 * hier.J)()
        for lev in range(hier.J):
            A = hier.A[lev]
            arrs = [L.as_i32(A.indptr), L.as_i32(A.indices),
                    np.ascontiguousarray(np.stack([A.data.real, A.data.imag], 1).ravel()),
                    L.as_f64(hier.inv_deg[lev])]
            keep += arrs
            lv = levels[lev]
            lv.n = A.shape[0]
            lv.A_indptr, lv.A_indices = L.ptr(arrs[0], L.i32p), L.ptr(arrs[1], L.i32p)
            lv.A_vals, lv.inv_deg = L.ptr(arrs[2], L.f64p), L.ptr(arrs[3], L.f64p)
            if lev < hier.J - 1:
                P = hier.P[lev].tocsr()
                pa = [L.as_i32(P.indptr), L.as_i32(P.indices), L.as_f64(P.data)]
                keep += pa
                lv.P_indptr, lv.P_indices = L.ptr(pa[0], L.i32p), L.ptr(pa[1], L.i32p)
                lv.P_vals = L.ptr(pa[2], L.f64p)
        ctx = C.c_void_p()
        L.check(self.lib.mg2_setup(C.byref(ctx), hier.J, levels, self.max_batch, self.precision))
        self.ctx = ctx
        self.set_params(params)

    def set_params(self, p: Params2):
        m = self.hier.J - 1
        arrs = [L.as_f64(p.theta), L.as_f64(p.eta)] + [L.as_f64(np.asarray(W).reshape(m * 8))
                                                      for W in (p.WB, p.WR, p.WP)]
        if arrs[0].size != m or arrs[1].size != m:
            raise ValueError(f"theta, eta: expected {m} levels")
        L.check(self.lib.mg2_set_params(self.ctx, *[L.ptr(a, L.f64p) for a in arrs],
                                        int(p.nu_pre), int(p.nu_post)))
        self.params = p

    def set_option(self, name: str, value: int):
        """Launch shapes of the cycle ("pdl", "multi_rhs", "tail_work";
        mg2_set_option)."""
        if name not in ("pdl", "multi_rhs", "tail_work"):
            raise ValueError(f"unknown two-feature option {name!r}")
        L.check(self.lib.mg2_set_option(self.ctx, L.OPTIONS[name], int(value)))

    def _check_cycle_args(self, f: torch.Tensor, u: torch.Tensor):
        for name, x in (("f", f), ("u", u)):
            if (x.dtype != self.dtype or not x.is_cuda or not x.is_contiguous() or x.dim() != 2
                    or x.shape[0] != self.n[0] or not 1 <= x.shape[1] <= self.max_batch):
                raise ValueError(f"{name}: expected a contiguous {self.dtype} CUDA tensor "
                                 f"({self.n[0]}, 1..{self.max_batch})")
        if f.shape != u.shape:
            raise ValueError("f and u differ in shape")

    def vcycle(self, f: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
        """u <- one two-feature cycle (Algorithm 2) on level 0, in place."""
        self._check_cycle_args(f, u)
        L.check(self.lib.mg2_vcycle(self.ctx, C.c_void_p(f.data_ptr()), C.c_void_p(u.data_ptr()),
                                    f.shape[1], _stream_handle()))
        return u

    def vcycle_profile(self, f: torch.Tensor, u: torch.Tensor) -> list[tuple[str, int, float]]:
        """One cycle with CUDA events around every kernel: [(name, level, ms)]."""
        self._check_cycle_args(f, u)
        cap = 4096
        buf = (L.KernelTime * cap)()
        n = C.c_int32(0)
        L.check(self.lib.mg2_vcycle_profile(self.ctx, C.c_void_p(f.data_ptr()),
                                            C.c_void_p(u.data_ptr()), f.shape[1], buf, cap,
                                            C.byref(n), _stream_handle()))
        return [(self.lib.mg_kernel_name(buf[k].kernel).decode(), buf[k].level, buf[k].ms)
                for k in range(n.value)]

    def solve_fgmres(self, f: torch.Tensor, u: torch.Tensor | None = None, tol: float = 1e-8,
                     max_iter: int = 300, restart: int = 30,
                     precond: str = "vcycle") -> tuple[torch.Tensor, SolveInfo]:
        """Restarted flexible GMRES on the real 2n form with the two-feature
        cycle ("vcycle") or full multigrid ("fmg") as right preconditioner
        (mg2_solve_fgmres).  f, u: complex128 CUDA tensors (n, nrhs)."""
        if u is None:
            u = torch.zeros_like(f)
        for name, x in (("f", f), ("u", u)):
            if (x.dtype != torch.complex128 or not x.is_cuda or not x.is_contiguous()
                    or x.dim() != 2 or x.shape[0] != self.n[0]
                    or not 1 <= x.shape[1] <= self.max_batch):
                raise ValueError(f"{name}: expected a contiguous complex128 CUDA tensor "
                                 f"({self.n[0]}, 1..{self.max_batch})")
        if f.shape != u.shape:
            raise ValueError("f and u differ in shape")
        B = f.shape[1]
        iters = np.zeros(B, dtype=np.int32)
        relres = np.zeros(B)
        st = self.lib.mg2_solve_fgmres(self.ctx, C.c_void_p(f.data_ptr()),
                                       C.c_void_p(u.data_ptr()), B, float(tol), int(max_iter),
                                       int(restart), {"vcycle": 0, "fmg": 1}[precond],
                                       L.ptr(iters, L.i32p), L.ptr(relres, L.f64p),
                                       _stream_handle())
        L.check(st, None, allow=(L.MG_OK, L.MG_NOT_CONVERGED))
        return u, SolveInfo(st, iters, relres)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mg2_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
