"""Stacked contexts for serving: one operator per request on a structured
square mesh (binding of mg_setup_square, mg_square_set_block and
mg_solve_blocks).

A SquareBatch holds `slots` independent systems -div(k grad u) = f on the
same N x N right-triangle mesh of the unit square.  Each slot gets its own
operator on the device from its element coefficients (assembly, Galerkin
coarsening, degrees and the coarsest inverse all run in libmg.so's kernels);
one solve call iterates every occupied slot to its own tolerance.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .solver import LMGParams, SolveInfo, _stream_handle


def levels_for(N: int) -> int:
    """Levels from N x N down to 3 x 3 vertices."""
    J, n = 1, N
    while n > 3:
        if (n - 1) % 2:
            raise ValueError(f"{N} x {N} does not coarsen to 3 x 3")
        n = (n - 1) // 2 + 1
        J += 1
    return J


class SquareBatch:
    def __init__(self, N: int, slots: int, params: LMGParams, precision: int = 32, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("SquareBatch needs a CUDA device")
        self.lib = L.lib()
        self.N, self.slots, self.precision = int(N), int(slots), int(precision)
        self.J = levels_for(self.N)
        if isinstance(device, torch.device):
            self.device = device
        else:
            self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                       else int(device))
        self.m = (self.N - 2) ** 2
        self.params = params.with_levels(self.J)
        p, keep = self.params.c_struct()
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.mg_setup_square(C.byref(ctx), self.N, self.J, self.slots, C.byref(p),
                                             self.precision, _stream_handle()))
        self.ctx = ctx
        sizes = (C.c_int32 * self.J)()
        Jout = C.c_int32(0)
        L.check(self.lib.mg_level_sizes(self.ctx, C.byref(Jout), sizes), self.ctx)
        self.sizes = [int(sizes[k]) for k in range(self.J)]

    @property
    def n_elements(self) -> int:
        return 2 * (self.N - 1) ** 2

    def set_block(self, block: int, ke: torch.Tensor):
        """Writes block `block`'s operator from its element coefficients
        (device FP64 [2 (N-1)^2], the square mesh's element order)."""
        if ke.device != self.device or ke.dtype != torch.float64 or not ke.is_contiguous() \
                or ke.numel() != self.n_elements:
            raise ValueError(f"ke: expected a contiguous FP64 tensor of {self.n_elements} "
                             f"elements on {self.device}")
        L.check(self.lib.mg_square_set_block(self.ctx, int(block), C.c_void_p(ke.data_ptr()),
                                             _stream_handle()), self.ctx)

    def solve(self, f: torch.Tensor, u: torch.Tensor, tol: float = 1e-8,
              max_iter: int = 100, nblocks: int | None = None) -> SolveInfo:
        """f, u: device FP64 stacks [slots * m] (u: initial guess, updated).
        Only the leading `nblocks` blocks (all if None) are iterated; the
        returned counts and residuals of the others are zero."""
        for x, nm in ((f, "f"), (u, "u")):
            if x.device != self.device or x.dtype != torch.float64 or not x.is_contiguous() \
                    or x.numel() != self.slots * self.m:
                raise ValueError(f"{nm}: expected a contiguous FP64 stack of "
                                 f"{self.slots * self.m} values on {self.device}")
        k = self.slots if nblocks is None else int(nblocks)
        iters = np.zeros(self.slots, dtype=np.int32)
        relres = np.zeros(self.slots)
        st = self.lib.mg_solve_blocks(self.ctx, k, C.c_void_p(f.data_ptr()),
                                      C.c_void_p(u.data_ptr()), float(tol), int(max_iter),
                                      L.ptr(iters, L.i32p), L.ptr(relres, L.f64p),
                                      _stream_handle())
        L.check(st, self.ctx, allow=(L.MG_OK, L.MG_NOT_CONVERGED))
        return SolveInfo(st, iters, relres)

    def vcycle(self, f: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
        """One cycle of Algorithm 2 on every block, u in place (context
        precision, stacks [slots * m])."""
        L.check(self.lib.mg_vcycle(self.ctx, C.c_void_p(f.data_ptr()), C.c_void_p(u.data_ptr()), 1,
                                   _stream_handle()), self.ctx)
        return u

    def vcycle_profile(self, f: torch.Tensor, u: torch.Tensor) -> list[tuple[str, int, float]]:
        """One cycle with CUDA events around every kernel: [(name, level, ms)]."""
        cap = 4096
        buf = (L.KernelTime * cap)()
        n = C.c_int32(0)
        L.check(self.lib.mg_vcycle_profile(self.ctx, C.c_void_p(f.data_ptr()),
                                           C.c_void_p(u.data_ptr()), 1, buf, cap, C.byref(n),
                                           _stream_handle()), self.ctx)
        return [(self.lib.mg_kernel_name(buf[k].kernel).decode(), buf[k].level, buf[k].ms)
                for k in range(n.value)]

    def level_apply(self, level: int, op: str, x: torch.Tensor, y: torch.Tensor | None,
                    out: torch.Tensor):
        yp = C.c_void_p(y.data_ptr()) if y is not None else None
        L.check(self.lib.mg_level_apply(self.ctx, level, L.OPS[op], C.c_void_p(x.data_ptr()), yp,
                                        C.c_void_p(out.data_ptr()), 1, _stream_handle()), self.ctx)
        return out

    def set_option(self, name: str, value: int):
        L.check(self.lib.mg_set_option(self.ctx, L.OPTIONS[name], int(value)), self.ctx)

    def kernel_launches(self) -> int:
        return int(self.lib.mg_kernel_launches(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
