"""mg_smooth_noalloc: the allocation-free smoothing entry point, for callers
that cannot call cudaMalloc (a host application that owns all device memory,
or a latency-critical loop that cannot take an allocation's implicit device
synchronisation).  Its output must match the context-based entry point
(mg_level_apply with MG_OP_SMOOTH), called through the C ABI, on two calls in
a row (the static scratch keeps the previous call's contents).

This file is collected last on purpose and runs alone in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from paper_2608_29082_b300 import Hierarchy, LMGParams, Solver
from paper_2608_29082_b300 import _lib as L

pytestmark = pytest.mark.gpu


def _vp(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("name", ["checker65", "lshape_r2"])
def test_noalloc_smoothing_matches_context_path(name):
    if name == "checker65":
        p = W.checkerboard_square(65, 6, ncell=8, values=(1.0, 1e4), batch=3, seed=7)
    else:
        p = W.lshape_anisotropic(refinements=2, batch=3, seed=3)
    H = Hierarchy.from_problem(p)
    lev = 0
    A = H.A[lev]
    n = A.shape[0]
    B = 3
    prm = LMGParams.identity(H.J)
    prm.theta[lev], prm.eta[lev] = 0.61, 1.07
    prm.wB[lev] = (0.93, 0.21)
    nu = 2
    S = Solver(H, prm, precision=64, max_batch=B)
    dev = torch.device("cuda")
    rowptr = torch.tensor(A.indptr, dtype=torch.int32, device=dev)
    col = torch.tensor(A.indices, dtype=torch.int32, device=dev)
    val = torch.tensor(A.data, dtype=torch.float64, device=dev)
    invdeg = torch.tensor(H.inv_deg[lev], dtype=torch.float64, device=dev)
    r = np.random.default_rng(0)
    f = torch.tensor(r.standard_normal((n, B)), dtype=torch.float64, device=dev)
    u0 = torch.tensor(r.standard_normal((n, B)), dtype=torch.float64, device=dev)
    lib = L.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    u_new = u0.clone()
    u_ref = u0.clone()
    tmp = torch.empty_like(u0)
    for call in range(2):
        st = lib.mg_smooth_noalloc(n, _vp(rowptr), _vp(col), _vp(val), _vp(invdeg), _vp(f),
                                   _vp(u_new), B, nu, prm.theta[lev], prm.eta[lev],
                                   prm.wB[lev][0], prm.wB[lev][1], stream)
        L.check(st)
        for _ in range(nu):
            S.level_apply(lev, "smooth", f, u_ref, tmp)
            u_ref.copy_(tmp)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(u_new - u_ref) / torch.linalg.norm(u_ref)).item()
        assert err < 1e-13, (call, err)
    S.close()


def test_noalloc_rejects_oversize():
    lib = L.lib()
    n = 1 << 20  # n * nrhs above MG_NOALLOC_MAX_ELEMS: rejected before any launch
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.mg_smooth_noalloc(n, _vp(dummy), _vp(dummy), _vp(dummy), _vp(dummy), _vp(dummy),
                               C.c_void_p(dummy.data_ptr() + 8), 1, 1, 1.0, 1.0, 1.0, 0.0, None)
    assert st == -1
    assert "exceeds" in L.last_error()
