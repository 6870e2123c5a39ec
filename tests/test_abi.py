"""The C ABI: the library loads and exports every function include/mg.h declares;
argument validation that needs no GPU."""
import ctypes as C
import os
import re

import numpy as np

from paper_2608_29082_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:mg_status|void|int64_t)\s+(mg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_are_rejected_without_gpu():
    lib = L.lib()
    ctx = C.c_void_p()
    st = lib.mg_setup(C.byref(ctx), None, None, None, 1, 64, None)
    assert st == -1 and not ctx.value
    assert "NULL" in L.last_error()
    # a bad parent index in the Galerkin helper
    A = L.HostCSR([0, 1, 2], [0, 1], [1.0, 1.0], (2, 2))
    par = np.array([[0, -1], [5, -1]], dtype=np.int32)
    o = L.CSROwned()
    st = lib.mg_galerkin(C.byref(A.c), L.ptr(par, L.i32p), 2, 1e-12, C.byref(o))
    assert st == -1
    assert "parent" in L.last_error()


def test_galerkin_helper_small():
    """1D P1 hat functions: P^T A P of the 3-point Laplacian over all vertices."""
    n = 5
    A = np.diag([1, 2, 2, 2, 1.0]) - np.diag(np.ones(4), 1) - np.diag(np.ones(4), -1)
    import scipy.sparse as sp
    Af = L.HostCSR.from_scipy(sp.csr_matrix(A))
    par = np.array([[0, -1], [0, 1], [1, -1], [1, 2], [2, -1]], dtype=np.int32)
    o = L.CSROwned()
    L.check(L.lib().mg_galerkin(C.byref(Af.c), L.ptr(par, L.i32p), 3, 1e-12, C.byref(o)))
    Ac = L.take_owned(o).to_scipy().toarray()
    ref = 0.5 * (np.diag([1, 2, 1.0]) - np.diag(np.ones(2), 1) - np.diag(np.ones(2), -1))
    assert np.allclose(Ac, ref, atol=1e-15)
