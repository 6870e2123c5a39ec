"""Host set-up of a multigrid hierarchy from a nested mesh hierarchy.

Calls the native set-up helpers of libmg.so (Galerkin coarsening, Dirichlet
elimination, interior prolongation, graph degree); numpy only holds arrays.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib as L

DROP_TOL = 1e-12


@dataclass
class Hierarchy:
    """Interior operators A[l], prolongations P[l] (l < J-1) and 1/deg per level."""
    A: list            # list[_lib.HostCSR]
    P: list            # list[_lib.HostCSR], J-1 entries
    inv_deg: list      # list[np.ndarray]

    @property
    def J(self) -> int:
        return len(self.A)

    @property
    def sizes(self) -> list[int]:
        return [a.shape[0] for a in self.A]

    @staticmethod
    def from_mesh(A_full_indptr, A_full_indices, A_full_data, nv: list[int],
                  boundary: list[np.ndarray], parent: list[np.ndarray],
                  drop_tol: float = DROP_TOL) -> "Hierarchy":
        """A_full_*: finest operator over all vertices (CSR, FP64).  nv[l],
        boundary[l] (bool per vertex) and parent[l] ((nv[l], 2) fine->coarse
        map, l < J-1) describe the nested meshes, finest first."""
        lib = L.lib()
        J = len(nv)
        Af = L.HostCSR(A_full_indptr, A_full_indices, A_full_data, (nv[0], nv[0]))
        A, P, inv_deg = [], [], []
        for lev in range(J):
            bnd = np.ascontiguousarray(boundary[lev], dtype=np.uint8)
            n_int = int((bnd == 0).sum())
            deg = np.zeros(n_int)
            o = L.CSROwned()
            L.check(lib.mg_eliminate(C.byref(Af.c), L.ptr(bnd, L.u8p), drop_tol, C.byref(o),
                                     L.ptr(deg, L.f64p)))
            A.append(L.take_owned(o))
            inv_deg.append(deg)
            if lev < J - 1:
                par = L.as_i32(parent[lev])
                bc = np.ascontiguousarray(boundary[lev + 1], dtype=np.uint8)
                o = L.CSROwned()
                L.check(lib.mg_prolongation(L.ptr(par, L.i32p), nv[lev], L.ptr(bnd, L.u8p),
                                            nv[lev + 1], L.ptr(bc, L.u8p), C.byref(o)))
                P.append(L.take_owned(o))
                o = L.CSROwned()
                L.check(lib.mg_galerkin(C.byref(Af.c), L.ptr(par, L.i32p), nv[lev + 1], drop_tol,
                                        C.byref(o)))
                Af = L.take_owned(o)
        return Hierarchy(A, P, inv_deg)

    @staticmethod
    def from_problem(problem, drop_tol: float = DROP_TOL) -> "Hierarchy":
        """Duck-typed: .mesh.levels[l].{nv, boundary, parent} and .A_full (scipy CSR)."""
        Af = problem.A_full.tocsr()
        lv = problem.mesh.levels
        return Hierarchy.from_mesh(Af.indptr, Af.indices, Af.data, [x.nv for x in lv],
                                   [x.boundary for x in lv],
                                   [x.parent for x in lv[:-1]], drop_tol)

    def c_structs(self):
        """(mg_hierarchy, mg_csr[J], keep-alive list)."""
        J = self.J
        Parr = (L.CSR * max(J - 1, 1))(*[p.c for p in self.P])
        deg_ptrs = (L.f64p * J)(*[L.ptr(d, L.f64p) for d in self.inv_deg])
        Aarr = (L.CSR * J)(*[a.c for a in self.A])
        h = L.Hier(J, Parr, deg_ptrs)
        return h, Aarr, [Parr, deg_ptrs, Aarr]

    def footprint_bytes(self, max_batch: int, precision: int) -> int:
        h, Aarr, keep = self.c_structs()
        out = C.c_size_t(0)
        L.check(L.lib().mg_footprint_bytes(C.byref(h), Aarr, max_batch, precision, C.byref(out)))
        return int(out.value)
