"""ctypes binding of libmg.so (include/mg.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MG_LIB_VARIANT=debug loads the index-checked build (libmg_debug.so)
LIB_PATH = os.path.join(HERE, "libmg_debug.so" if os.environ.get("MG_LIB_VARIANT") == "debug"
                        else "libmg.so")

MG_OK = 0
MG_NOT_CONVERGED = 1
STATUS = {0: "MG_OK", 1: "MG_NOT_CONVERGED", -1: "MG_ERR_INVALID", -2: "MG_ERR_OOM",
          -3: "MG_ERR_NOT_SPD", -4: "MG_ERR_CUDA", -5: "MG_ERR_TIMEOUT", -6: "MG_ERR_DIVERGED",
          -7: "MG_ERR_NOT_IMPLEMENTED", -8: "MG_ERR_STATE"}
OPTIONS = {"tail_work": 0, "pdl": 1, "multi_rhs": 2, "device_loop": 3, "halo_rows": 4, "fcg_precond": 5,
           "fgmres_floor": 6, "sell_halo_rows": 7,
           "sell_halo_threads": 8, "sell_halo_max_bytes": 9, "coarse_inverse": 10,
           "tail_teams": 11, "fcg_fp32": 12, "fcg_floor": 13,
           "halo2d_bytes": 14, "dia_two_rows": 15}
OPS = {"smooth": 0, "residual": 1, "restrict": 2, "prolong": 3, "coarse": 4,
       "outer_residual": 5, "refine_residual": 6}

i32p = C.POINTER(C.c_int32)
f64p = C.POINTER(C.c_double)
u8p = C.POINTER(C.c_uint8)


class CSR(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int32),
                ("rowptr", i32p), ("col", i32p), ("val", f64p)]


class CSROwned(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int32),
                ("rowptr", i32p), ("col", i32p), ("val", f64p)]


class Hier(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("P", C.POINTER(CSR)), ("inv_deg", C.POINTER(f64p))]


class Params(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("nu_pre", C.c_int32), ("nu_post", C.c_int32),
                ("theta", f64p), ("eta", f64p), ("wB", f64p), ("wR", f64p), ("wP", f64p)]


class Level2(C.Structure):
    """mg2_level: one level of a complex (two-feature) hierarchy."""
    _fields_ = [("n", C.c_int32), ("A_indptr", i32p), ("A_indices", i32p), ("A_vals", f64p),
                ("inv_deg", f64p), ("P_indptr", i32p), ("P_indices", i32p), ("P_vals", f64p)]


class KernelTime(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("level", C.c_int32), ("ms", C.c_float)]


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """The loaded library.  Raises if libmg.so has not been built: there is no
    fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with "
                          "`python -m paper_2608_29082_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "mg_galerkin": ([C.POINTER(CSR), i32p, C.c_int32, C.c_double, C.POINTER(CSROwned)], C.c_int),
        "mg_eliminate": ([C.POINTER(CSR), u8p, C.c_double, C.POINTER(CSROwned), f64p], C.c_int),
        "mg_galerkin_complex": ([C.POINTER(CSR), i32p, C.c_int32, C.c_double,
                                 C.POINTER(CSROwned)], C.c_int),
        "mg_eliminate_complex": ([C.POINTER(CSR), u8p, C.c_double, C.POINTER(CSROwned), f64p],
                                 C.c_int),
        "mg_prolongation": ([i32p, C.c_int32, u8p, C.c_int32, u8p, C.POINTER(CSROwned)], C.c_int),
        "mg_csr_owned_free": ([C.POINTER(CSROwned)], None),
        "mg_setup": ([C.POINTER(vp), C.POINTER(Hier), C.POINTER(CSR), C.POINTER(Params),
                      C.c_int32, C.c_int32, vp], C.c_int),
        "mg_set_params": ([vp, C.POINTER(Params)], C.c_int),
        "mg_set_cheb": ([vp, C.c_int32, f64p], C.c_int),
        "mg2_setup": ([C.POINTER(vp), C.c_int32, C.POINTER(Level2), C.c_int32, C.c_int32],
                      C.c_int),
        "mg2_set_params": ([vp, f64p, f64p, f64p, f64p, f64p, C.c_int32, C.c_int32], C.c_int),
        "mg2_set_option": ([vp, C.c_int32, C.c_int64], C.c_int),
        "mg_debug_bounds": ([C.POINTER(C.c_uint64)], C.c_int32),
        "mg2_vcycle_profile": ([vp, vp, vp, C.c_int32, C.POINTER(KernelTime), C.c_int32,
                                C.POINTER(C.c_int32), vp], C.c_int),
        "mg2_vcycle": ([vp, vp, vp, C.c_int32, vp], C.c_int),
        "mg2_solve_fgmres": ([vp, vp, vp, C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                              i32p, f64p, vp], C.c_int),
        "mg2_destroy": ([vp], None),
        "mg_vcycle": ([vp, vp, vp, C.c_int32, vp], C.c_int),
        "mg_fmg": ([vp, vp, vp, C.c_int32, vp], C.c_int),
        "mg_solve": ([vp, vp, vp, C.c_int32, C.c_double, C.c_int32, i32p, f64p, vp], C.c_int),
        "mg_solve_fcg": ([vp, vp, vp, C.c_int32, C.c_double, C.c_int32, i32p, f64p, vp], C.c_int),
        "mg_solve_fgmres": ([vp, vp, vp, C.c_int32, C.c_double, C.c_int32, C.c_int32, i32p, f64p,
                             vp], C.c_int),
        "mg_solve_host": ([vp, f64p, f64p, C.c_int32, C.c_double, C.c_int32, i32p, f64p, vp],
                          C.c_int),
        "mg_level_apply": ([vp, C.c_int32, C.c_int32, vp, vp, vp, C.c_int32, vp], C.c_int),
        "mg_level_sizes": ([vp, i32p, i32p], C.c_int),
        "mg_footprint_bytes": ([C.POINTER(Hier), C.POINTER(CSR), C.c_int32, C.c_int32,
                                C.POINTER(C.c_size_t)], C.c_int),
        "mg_vcycle_profile": ([vp, vp, vp, C.c_int32, C.POINTER(KernelTime), C.c_int32, i32p,
                               vp], C.c_int),
        "mg_kernel_name": ([C.c_int32], C.c_char_p),
        "mg_set_option": ([vp, C.c_int32, C.c_int64], C.c_int),
        "mg_set_layout_policy": ([C.c_int32], C.c_int),
        "mg_forward_record": ([vp, vp, vp, C.c_int32, C.c_int32, vp], C.c_int),
        "mg_vcycle_backward": ([vp, C.c_int32, vp, vp, vp, vp, vp], C.c_int),
        "mg_residual_loss": ([vp, vp, vp, C.c_int32, vp, vp, vp, vp, vp], C.c_int),
        "mg_smooth_noalloc": ([C.c_int32, vp, vp, vp, vp, vp, vp, C.c_int32, C.c_int32,
                               C.c_double, C.c_double, C.c_double, C.c_double, vp], C.c_int),
        "mg_setup_square": ([C.POINTER(vp), C.c_int32, C.c_int32, C.c_int32, C.POINTER(Params),
                             C.c_int32, vp], C.c_int),
        "mg_square_set_block": ([vp, C.c_int32, vp, vp], C.c_int),
        "mg_solve_blocks": ([vp, C.c_int32, vp, vp, C.c_double, C.c_int32, i32p, f64p, vp],
                            C.c_int),
        "mg_last_error": ([vp, C.c_char_p, C.c_size_t], C.c_int),
        "mg_kernel_launches": ([vp], C.c_int64),
        "mg_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def last_error(ctx=None) -> str:
    buf = C.create_string_buffer(1024)
    lib().mg_last_error(ctx, buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int, ctx=None, allow=(MG_OK,)) -> int:
    if status not in allow:
        raise MGError(status, last_error(ctx))
    return status


# ---------------------------------------------------------- marshalling ----

def as_i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class HostCSR:
    """Keeps the arrays of an mg_csr alive."""

    def __init__(self, indptr, indices, data, shape):
        self.indptr, self.indices, self.data = as_i32(indptr), as_i32(indices), as_f64(data)
        self.shape = (int(shape[0]), int(shape[1]))
        self.c = CSR(self.shape[0], self.shape[1], int(self.data.size), ptr(self.indptr, i32p),
                     ptr(self.indices, i32p), ptr(self.data, f64p))

    @staticmethod
    def from_scipy(m) -> "HostCSR":
        m = m.tocsr()
        return HostCSR(m.indptr, m.indices, m.data, m.shape)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=self.shape)


class HostCSRComplex:
    """Keeps the arrays of an mg_csr whose values are complex (2 doubles per
    entry, (Re, Im) adjacent)."""

    def __init__(self, indptr, indices, data, shape):
        self.indptr, self.indices = as_i32(indptr), as_i32(indices)
        self.data = np.ascontiguousarray(data, dtype=np.complex128)
        self.shape = (int(shape[0]), int(shape[1]))
        pairs = self.data.view(np.float64)
        self.c = CSR(self.shape[0], self.shape[1], int(self.data.size), ptr(self.indptr, i32p),
                     ptr(self.indices, i32p), ptr(pairs, f64p))

    @staticmethod
    def from_scipy(m) -> "HostCSRComplex":
        m = m.tocsr()
        return HostCSRComplex(m.indptr, m.indices, m.data, m.shape)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=self.shape)


def take_owned_complex(o: CSROwned) -> HostCSRComplex:
    """take_owned for a library-allocated CSR with complex values."""
    try:
        n, nnz = o.n_rows, o.nnz
        indptr = np.ctypeslib.as_array(o.rowptr, shape=(n + 1,)).copy()
        if nnz > 0:
            indices = np.ctypeslib.as_array(o.col, shape=(nnz,)).copy()
            data = np.ctypeslib.as_array(o.val, shape=(2 * nnz,)).copy().view(np.complex128)
        else:
            indices = np.zeros(0, np.int32)
            data = np.zeros(0, np.complex128)
        return HostCSRComplex(indptr, indices, data, (o.n_rows, o.n_cols))
    finally:
        lib().mg_csr_owned_free(C.byref(o))


def take_owned(o: CSROwned) -> HostCSR:
    """Copies a library-allocated CSR into numpy arrays and frees it."""
    try:
        n, nnz = o.n_rows, o.nnz
        indptr = np.ctypeslib.as_array(o.rowptr, shape=(n + 1,)).copy()
        if nnz > 0:
            indices = np.ctypeslib.as_array(o.col, shape=(nnz,)).copy()
            data = np.ctypeslib.as_array(o.val, shape=(nnz,)).copy()
        else:
            indices = np.zeros(0, np.int32)
            data = np.zeros(0)
        return HostCSR(indptr, indices, data, (o.n_rows, o.n_cols))
    finally:
        lib().mg_csr_owned_free(C.byref(o))
