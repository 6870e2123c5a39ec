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
        names += re.findall(r"^\s*(?:mg_status|void|int64_t|int32_t)\s+(mg2?_\w+)\s*\(", src,
                            flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_release_build_has_no_index_checks_and_debug_build_exports_the_abi():
    """mg_debug_bounds reports a release build without touching the device;
    the index-checked build, when it has been built, exports the same
    functions."""
    lib = L.lib()
    w = C.c_uint64(5)
    assert lib.mg_debug_bounds(C.byref(w)) == 0 and w.value == 0
    assert lib.mg_debug_bounds(None) == 0
    dbg = os.path.join(os.path.dirname(L.LIB_PATH), "libmg_debug.so")
    if os.path.exists(dbg):
        d = C.CDLL(dbg)
        missing = [n for n in declared_functions() if not hasattr(d, n)]
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


def test_noalloc_rejects_overlapping_f_and_u_without_gpu():
    """mg_smooth_noalloc checks its arguments before any CUDA call: f and u
    whose [n][nrhs] ranges overlap (equal or shifted by less than their
    length) are rejected, so these stand-in addresses are never used."""
    lib = L.lib()
    base = 1 << 40
    n, nrhs = 100, 2
    nbytes = n * nrhs * 8
    fake = C.c_void_p(base)
    for shift in (0, 8, nbytes - 8, -8, -(nbytes - 8)):
        st = lib.mg_smooth_noalloc(n, fake, fake, fake, fake, C.c_void_p(base),
                                   C.c_void_p(base + shift), nrhs, 1, 1.0, 1.0, 1.0, 0.0, None)
        assert st == -1, shift
        assert "overlap" in L.last_error()


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


def test_two_feature_entry_points_reject_bad_input_without_gpu():
    """mg2_setup validates every array before its first CUDA call; the other
    mg2 entry points and mg_set_cheb reject a NULL context."""
    lib = L.lib()
    assert "mg2_setup" in declared_functions() and "mg2_solve_fgmres" in declared_functions()
    ctx = C.c_void_p()
    assert lib.mg2_setup(C.byref(ctx), 0, None, 1, 64) == -1 and not ctx.value
    # one level, 2 x 2 complex operator with a column index out of range
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 7], dtype=np.int32)
    av = np.array([1.0, 0.0, 1.0, 0.0])
    deg = np.ones(2)
    lv = (L.Level2 * 1)()
    lv[0].n = 2
    lv[0].A_indptr, lv[0].A_indices = L.ptr(rp, L.i32p), L.ptr(ci, L.i32p)
    lv[0].A_vals, lv[0].inv_deg = L.ptr(av, L.f64p), L.ptr(deg, L.f64p)
    assert lib.mg2_setup(C.byref(ctx), 1, lv, 1, 64) == -1
    assert "column" in L.last_error()
    # two levels without a prolongation on level 0
    lv2 = (L.Level2 * 2)()
    for k in range(2):
        lv2[k].n = 2
        lv2[k].A_indptr, lv2[k].A_indices = L.ptr(rp, L.i32p), L.ptr(np.array([0, 1], dtype=np.int32), L.i32p)
        lv2[k].A_vals, lv2[k].inv_deg = L.ptr(av, L.f64p), L.ptr(deg, L.f64p)
    assert lib.mg2_setup(C.byref(ctx), 2, lv2, 1, 64) == -1
    assert "prolongation" in L.last_error()
    assert lib.mg2_setup(C.byref(ctx), 1, lv2, 1, 16) == -1  # precision
    x = np.zeros(4)
    assert lib.mg2_set_params(None, L.ptr(x, L.f64p), L.ptr(x, L.f64p), L.ptr(x, L.f64p),
                              L.ptr(x, L.f64p), L.ptr(x, L.f64p), 1, 1) == -1
    assert lib.mg2_vcycle(None, None, None, 1, None) == -1
    assert lib.mg2_solve_fgmres(None, None, None, 1, 1e-8, 10, 10, 0, None, None, None) == -1
    assert lib.mg_set_cheb(None, 2, L.ptr(x, L.f64p)) == -1


def _two_level(AJ):
    """A 2-level hierarchy: the 3-point 1D Laplacian on 3 rows, P = hat
    function of the middle row, and the given coarsest operator (1 x 1 or
    2 x 2, dense)."""
    import scipy.sparse as sp
    A0 = L.HostCSR.from_scipy(sp.csr_matrix(np.array([[2.0, -1, 0], [-1, 2, -1], [0, -1, 2]])))
    nJ = AJ.shape[0]
    P = L.HostCSR.from_scipy(sp.csr_matrix(np.ones((3, nJ)) * 0.5))
    AJc = L.HostCSR.from_scipy(sp.csr_matrix(AJ))
    deg0, degJ = np.full(3, 0.5), np.full(nJ, 1.0)
    Parr = (L.CSR * 1)(P.c)
    degs = (L.f64p * 2)(L.ptr(deg0, L.f64p), L.ptr(degJ, L.f64p))
    Aarr = (L.CSR * 2)(A0.c, AJc.c)
    h = L.Hier(2, Parr, degs)
    keep = [A0, P, AJc, deg0, degJ, Parr, degs, Aarr]
    return h, Aarr, keep


def test_setup_rejects_indefinite_coarsest_operator_without_gpu():
    """Failure detection on the host: a coarsest operator that is not SPD
    (indefinite, or singular) makes mg_setup return MG_ERR_NOT_SPD before any
    device allocation; a non-positive diagonal entry (the smoother divides by
    it) is rejected earlier as MG_ERR_INVALID.  No context is returned."""
    from paper_2608_29082_b300 import LMGParams
    lib = L.lib()
    cases = ((np.array([[1.0, 2.0], [2.0, 1.0]]), -3, "not SPD"),
             (np.array([[1.0, 1.0], [1.0, 1.0]]), -3, "not SPD"),
             (np.array([[-1.0]]), -1, "non-positive diagonal"))
    for AJ, want, msg in cases:
        h, Aarr, keep = _two_level(AJ)
        prm = LMGParams.identity(2)
        p, pkeep = prm.c_struct()
        for prec in (64, 32):
            ctx = C.c_void_p()
            st = lib.mg_setup(C.byref(ctx), C.byref(h), Aarr, C.byref(p), 1, prec, None)
            assert st == want and not ctx.value, (AJ, prec, st)
            assert msg in L.last_error()


def test_two_feature_setup_rejects_singular_coarsest_operator_without_gpu():
    """mg2_setup inverts the complex coarsest operator on the host before
    any CUDA call: an exactly singular one gives MG_ERR_NOT_SPD, a zero
    diagonal MG_ERR_INVALID."""
    lib = L.lib()
    rp = np.array([0, 2, 4], dtype=np.int32)
    ci = np.array([0, 1, 0, 1], dtype=np.int32)
    deg = np.ones(2)
    singular = np.array([1.0, 1.0, 2.0, 2.0, 1.0, 1.0, 2.0, 2.0])  # rows (1+i, 2+2i) twice
    zero_diag = np.array([0.0, 0.0, 1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    for vals, want, msg in ((singular, -3, "singular"), (zero_diag, -1, "zero diagonal")):
        lv = (L.Level2 * 1)()
        lv[0].n = 2
        lv[0].A_indptr, lv[0].A_indices = L.ptr(rp, L.i32p), L.ptr(ci, L.i32p)
        lv[0].A_vals, lv[0].inv_deg = L.ptr(vals, L.f64p), L.ptr(deg, L.f64p)
        for prec in (64, 32):
            ctx = C.c_void_p()
            assert lib.mg2_setup(C.byref(ctx), 1, lv, 1, prec) == want and not ctx.value
            assert msg in L.last_error()
