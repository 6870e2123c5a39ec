"""ChebConv smoother (mg_set_cheb) against the FP64 oracle, through the C ABI.

Tolerances as in the SAGEConv parity tests: single FP64 steps 1e-13
relative, FP64 cycles 1e-12, the FP32 cycle within 1e-5 of the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2608_29082_b300 import Hierarchy, LMGParams, MGError, Solver

pytestmark = pytest.mark.gpu

DEV = "cuda"

CASES = {
    "poisson33": lambda: W.poisson_square(33, 4, batch=3, seed=1),
    "checker65": lambda: W.checkerboard_square(65, 6, ncell=8, values=(1.0, 1e4), batch=2, seed=3),
    "lshape_r2": lambda: W.lshape_anisotropic(refinements=2, batch=2, seed=2),
}
_cache = {}


def problem(name):
    if name not in _cache:
        p = CASES[name]()
        _cache[name] = (p, O.build_hierarchy(p), Hierarchy.from_problem(p))
    return _cache[name]


def t64(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def params(J, seed, spread=0.2):
    r = np.random.default_rng(seed)
    p = LMGParams.identity(J)
    m = J - 1
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, m))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, m))
    for w in (p.wR, p.wP):
        w[:, 0] += spread * r.uniform(-1, 1, m)
        w[:, 1] += spread * r.uniform(-1, 1, m)
    return p


def cheb_coef(J, K, seed, spread=0.2):
    c = spread * np.random.default_rng(100 + seed).uniform(-1, 1, (J - 1, K + 1))
    c[:, 0] += 1.0
    return c


def to_oracle(p: LMGParams, cheb) -> O.Params:
    return O.Params(p.theta.copy(), p.eta.copy(), p.wB.copy(), p.wR.copy(), p.wP.copy(),
                    p.nu_pre, p.nu_post, None if cheb is None else np.array(cheb))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("K", [1, 2, 5])
def test_cheb_smooth_step_fp64(name, K):
    p, Ho, Hp = problem(name)
    prm = params(Hp.J, 3)
    c = cheb_coef(Hp.J, K, K)
    po = to_oracle(prm, c)
    S = Solver(Hp, prm, precision=64, max_batch=4)
    S.set_cheb(c)
    r = np.random.default_rng(0)
    for lev in range(Hp.J - 1):
        Lo = Ho.levels[lev]
        n = Hp.sizes[lev]
        f, u = r.standard_normal((n, 3)), r.standard_normal((n, 3))
        out = torch.empty((n, 3), dtype=torch.float64, device=DEV)
        S.level_apply(lev, "smooth", t64(f), t64(u), out)
        ref = O.smooth(Lo, f, u, po.theta[lev], po.eta[lev], po.wB[lev], po.cheb[lev])
        assert rel(out.cpu().numpy(), ref) < 1e-13, lev
    S.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("K", [2, 4])
def test_cheb_vcycle_parity(name, prec, K):
    """Per-cycle parity of the whole cycle with the ChebConv smoother on every
    level (DIA and SELL levels, multi-rhs batches)."""
    p, Ho, Hp = problem(name)
    prm = params(Hp.J, 7)
    c = cheb_coef(Hp.J, K, 7 + K)
    po = to_oracle(prm, c)
    f = p.f
    S = Solver(Hp, prm, precision=prec, max_batch=f.shape[1])
    S.set_cheb(c)
    dt = torch.float64 if prec == 64 else torch.float32
    fg = t64(f).to(dt)
    ug = torch.zeros_like(fg)
    fo = f if prec == 64 else f.astype(np.float32).astype(np.float64)
    uo = np.zeros_like(f)
    tol = 1e-12 if prec == 64 else 1e-5
    for m in range(4):
        S.vcycle(fg, ug)
        uo = O.vcycle(Ho, po, fo, uo)
        assert rel(ug.double().cpu().numpy(), uo) < tol, m
    S.close()


def test_cheb_degree_one_is_sage_and_switch_back():
    """Degree 1 with (c_0, c_1) is the SAGEConv smoother with (c_0, -c_1);
    switching the smoother back (K = 0) restores the SAGEConv cycle bitwise."""
    p, Ho, Hp = problem("checker65")
    prm = params(Hp.J, 5)
    c = cheb_coef(Hp.J, 1, 5)
    sage = params(Hp.J, 5)
    sage.wB[:, 0], sage.wB[:, 1] = c[:, 0], -c[:, 1]
    f = t64(p.f)
    Sc = Solver(Hp, prm, precision=64, max_batch=2)
    Ss = Solver(Hp, sage, precision=64, max_batch=2)
    u_s0 = torch.zeros_like(f)
    Ss.vcycle(f, u_s0)
    Sc.set_cheb(c)
    uc, us = torch.zeros_like(f), torch.zeros_like(f)
    for _ in range(3):
        Sc.vcycle(f, uc)
        Ss.vcycle(f, us)
    assert rel(uc.cpu().numpy(), us.cpu().numpy()) < 1e-12
    # back to SAGEConv with the same Theta as Ss: bitwise the first cycle of Ss
    Sc.set_params(sage)
    Sc.set_cheb(None)
    u1 = torch.zeros_like(f)
    Sc.vcycle(f, u1)
    assert torch.equal(u1, u_s0)
    Sc.close()
    Ss.close()


@pytest.mark.parametrize("method", ["refine", "fcg", "fgmres"])
def test_cheb_solves_reach_tolerance(method):
    """The FP32 cycle with a degree-3 ChebConv smoother inside the FP64 outer
    loops reaches 1e-8, re-checked by the oracle."""
    p, Ho, Hp = problem("lshape_r2")
    prm = LMGParams.identity(Hp.J)
    c = np.tile([1.0, 0.1, 0.05, 0.0], (Hp.J - 1, 1))
    S = Solver(Hp, prm, precision=32, max_batch=p.f.shape[1])
    S.set_cheb(c)
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=300, method=method)
    assert info.status == 0
    assert (O.relres(Ho, p.f, u.cpu().numpy()) < 1e-8).all()
    S.close()


def test_cheb_rejects_bad_input_and_training():
    p, Ho, Hp = problem("poisson33")
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=64, max_batch=3)
    with pytest.raises(MGError):
        S.set_cheb(np.ones((Hp.J - 1, 10)))  # degree 9 > MG_CHEB_MAX_DEGREE
    bad = np.ones((Hp.J - 1, 3))
    bad[0, 1] = np.nan
    with pytest.raises(MGError):
        S.set_cheb(bad)
    with pytest.raises(ValueError):
        S.set_cheb(np.ones((Hp.J, 3)))
    S.set_cheb(np.tile([1.0, 0.2, 0.0], (Hp.J - 1, 1)))
    f = t64(p.f)
    with pytest.raises(MGError):
        S.forward_record(f, torch.zeros_like(f), 2)
    S.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("tile", [2, 4, 8])
def test_cheb_multi_rhs_tile_bitwise(prec, tile):
    """The right-hand-side-tiled Chebyshev pass computes every entry with the
    scalar pass's arithmetic: cycles agree bitwise for every tile width."""
    p, Ho, Hp = problem("checker65")
    prm = params(Hp.J, 9)
    c = cheb_coef(Hp.J, 3, 9)
    f = np.random.default_rng(4).standard_normal((Hp.sizes[0], 8))
    dt = torch.float64 if prec == 64 else torch.float32
    res = []
    for opt in (0, tile):
        S = Solver(Hp, prm, precision=prec, max_batch=8)
        S.set_cheb(c)
        S.set_option("multi_rhs", opt)
        u = torch.zeros((Hp.sizes[0], 8), dtype=dt, device=DEV)
        fg = t64(f).to(dt)
        for _ in range(2):
            S.vcycle(fg, u)
        res.append(u)
        S.close()
    assert torch.equal(res[0], res[1])
