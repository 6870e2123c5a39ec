"""Child process of tests/test_gpu_debug_build.py: runs a set of cycles and
solves through whichever library MG_LIB_VARIANT selects and prints one JSON
line with the results' digests and the library's bounds record."""
import ctypes as C
import hashlib
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads as W  # noqa: E402
from paper_2608_29082_b300 import Hierarchy, LMGParams, Solver, _lib  # noqa: E402
from paper_2608_29082_b300.features2 import Hierarchy2, Params2, Solver2  # noqa: E402
from paper_2608_29082_b300.square import SquareBatch  # noqa: E402


def digest(t: torch.Tensor) -> str:
    return hashlib.sha256(t.detach().cpu().contiguous().numpy().tobytes()).hexdigest()[:16]


def params(J, seed):
    r = np.random.default_rng(seed)
    p = LMGParams.identity(J)
    for w in (p.wB, p.wR, p.wP):
        w[:, 1] += 0.1 * r.uniform(-1, 1, J - 1)
    return p


out = {}
for name, prob in (("checker65", W.checkerboard_square(65, 6, ncell=8, values=(1.0, 1e4), batch=3,
                                                       seed=3)),
                   ("lshape_r2", W.lshape_anisotropic(refinements=2, batch=3, seed=2))):
    hier = Hierarchy.from_problem(prob)
    for prec in (32, 64):
        S = Solver(hier, params(hier.J, 5), precision=prec, max_batch=3)
        S.set_option("sell_halo_rows", 64 if name == "lshape_r2" else 0)
        dt = torch.float32 if prec == 32 else torch.float64
        f = torch.tensor(prob.f, dtype=dt, device="cuda")
        u = torch.zeros_like(f)
        for _ in range(2):
            S.vcycle(f, u)
        f64 = torch.tensor(prob.f, dtype=torch.float64, device="cuda")
        res = [digest(u)]
        for method in ("refine", "fcg", "fgmres"):
            uu, info = S.solve(f64, tol=1e-8, max_iter=300, method=method)
            res += [digest(uu), int(info.iters.max())]
        out[f"{name}_fp{prec}"] = res
        S.close()
p2 = W.helmholtz_square(33, 3, k=2 * np.pi, batch=2, seed=3)
S2 = Solver2(Hierarchy2.from_problem(p2), Params2.identity(3), precision=32, max_batch=2)
f2 = torch.tensor(p2.f, dtype=torch.complex64, device="cuda")
u2 = torch.zeros_like(f2)
S2.vcycle(f2, u2)
out["features2"] = [digest(torch.view_as_real(u2))]
S2.close()
B = SquareBatch(33, 2, LMGParams.identity(5), precision=32)
k = torch.ones(B.n_elements, dtype=torch.float64, device="cuda")
for b in range(2):
    B.set_block(b, k)
fs = torch.ones(2 * B.m, dtype=torch.float64, device="cuda")
us = torch.zeros_like(fs)
info = B.solve(fs, us, tol=1e-8, max_iter=100)
out["square"] = [digest(us), int(info.iters.max())]
B.close()
word = C.c_uint64(7)
out["bounds"] = [int(_lib.lib().mg_debug_bounds(C.byref(word))), int(word.value)]
out["library"] = os.path.basename(_lib.LIB_PATH)
print(json.dumps(out))
