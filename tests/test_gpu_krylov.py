"""The refinement step and the Krylov outer loops of the CUDA path against the
FP64 oracle, step by step and iterate by iterate, through the C ABI; solves on
a caller's non-blocking stream; failure detection on host-built inputs.

Tolerances: a single FP64 step 1e-13 relative; the scaled FP32 copy of the
refinement residual bitwise equal to float(2^-s r) of the FP64 residual the
same kernels compute, and within one FP32 rounding of float(2^-s r) of the
oracle's residual; FP64 Krylov iterates 1e-10 relative to the oracle's (the
two sides differ only in rounding order: CGS2 against MGS, and the order of
the dot-product sums), FGMRES residual estimates within 1e-10 ||f||.
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


def rand_params(J, seed, spread):
    r = np.random.default_rng(seed)
    p = LMGParams.identity(J)
    m = J - 1
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, m))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, m))
    for w in (p.wB, p.wR, p.wP):
        w[:, 0] += spread * r.uniform(-1, 1, m)
        w[:, 1] += spread * r.uniform(-1, 1, m)
    return p


def to_oracle(p: LMGParams) -> O.Params:
    return O.Params(p.theta.copy(), p.eta.copy(), p.wB.copy(), p.wR.copy(), p.wP.copy(),
                    p.nu_pre, p.nu_post)


def t64(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def ilogb(x: float) -> int:
    """Unbiased binary exponent of a positive finite x (C's ilogb)."""
    return int(np.frexp(x)[1]) - 1


# ------------------------------------------------------ refinement step ----

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_refinement_residual_step(name, prec):
    """The FP64 residual of the refinement (a7) element by element against
    f - A u, and its scaled FP32 copy, the FP32 cycle's input."""
    p, Ho, Hp = problem(name)
    A = Ho.levels[0].A
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=prec, max_batch=4)
    r = np.random.default_rng(7)
    n = Hp.sizes[0]
    f = r.standard_normal((n, 4)) * np.array([1.0, 1e-6, 3e5, 1.0])
    f[:, 3] = 0.0  # ||f|| = 0: scale exponent 0
    u = r.standard_normal((n, 4))
    ref = f - A @ u
    out = torch.empty((n, 4), dtype=torch.float64, device=DEV)
    S.level_apply(0, "outer_residual", t64(f), t64(u), out)
    rg = out.cpu().numpy()
    scale = np.abs(f) + abs(A) @ np.abs(u)
    assert np.all(np.abs(rg - ref) <= 1e-13 * scale), name
    assert np.linalg.norm(rg - ref) <= 1e-13 * np.linalg.norm(ref)
    rhat = torch.empty((n, 4), dtype=torch.float32, device=DEV)
    S.level_apply(0, "refine_residual", t64(f), t64(u), rhat)
    rh = rhat.cpu().numpy()
    fn = np.linalg.norm(f, axis=0)
    s = np.array([ilogb(x) if x > 0 else 0 for x in fn])
    assert s[3] == 0
    # bitwise: float(2^-s r) of the FP64 residual (2^-s r is exact in FP64)
    assert np.array_equal(rh, (rg * np.ldexp(1.0, -s)).astype(np.float32))
    # against the oracle's residual: at most one FP32 rounding apart
    ro = (ref * np.ldexp(1.0, -s)).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(ro).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(rh.astype(np.float64) - ro) <= ulp + 1e-45)
    S.close()


# ------------------------------------------------- FCG, iterate by iterate --

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("which", ["identity", "learned"])
def test_fcg_iterates_match_oracle(name, which):
    """FP64 flexible CG with the FP64 cycle as preconditioner: after k
    iterations (max_iter = k) every right-hand side's iterate equals the
    oracle's FCG(1) iterate u_k."""
    p, Ho, Hp = problem(name)
    prm = LMGParams.identity(Hp.J) if which == "identity" else rand_params(Hp.J, 47, 0.05)
    po = to_oracle(prm)
    A = Ho.levels[0].A
    B = p.f.shape[1]
    S = Solver(Hp, prm, precision=64, max_batch=B)
    M = lambda v: O.vcycle(Ho, po, v[:, None], np.zeros((v.size, 1)))[:, 0]  # noqa: E731
    K = 10
    ref = [O.fcg(A, p.f[:, b], M, 1e-300, max_iter=K)[3] for b in range(B)]
    for k in (1, 2, 3, 5, 7, 10):
        u, info = S.solve(t64(p.f), tol=1e-300, max_iter=k, method="fcg")
        assert info.status == 1 and np.all(info.iters == k)
        ug = u.cpu().numpy()
        for b in range(B):
            uo = ref[b][k - 1]
            err = np.linalg.norm(ug[:, b] - uo) / np.linalg.norm(uo)
            assert err < 1e-10, (name, which, k, b, err)
            # the reported relres is the true residual of that iterate
            rr = np.linalg.norm(p.f[:, b] - A @ ug[:, b]) / np.linalg.norm(p.f[:, b])
            assert abs(info.relres[b] - rr) <= 1e-10 * rr + 1e-13
    S.close()


# ---------------------------------------------- FGMRES, iterate by iterate --

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pc", [0, 1])
def test_fgmres_iterates_and_estimates_match_oracle(name, pc):
    """FP64 FGMRES(5) with the learnable cycle (pc 0) or FMG (pc 1): after
    k Arnoldi steps, across restarts, each right-hand side's iterate equals
    the oracle FGMRES's, and its residual equals the oracle's residual
    estimate |g_{k+1}| (the least-squares residual of step k)."""
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 29, 0.2) if pc == 0 else rand_params(Hp.J, 23, 0.05)
    po = to_oracle(prm)
    A = Ho.levels[0].A
    B = p.f.shape[1]
    if pc:
        M = lambda v: O.fmg(Ho, po, v[:, None])[:, 0]  # noqa: E731
    else:
        M = lambda v: O.vcycle(Ho, po, v[:, None], np.zeros((v.size, 1)))[:, 0]  # noqa: E731
    S = Solver(Hp, prm, precision=64, max_batch=B)
    S.set_option("fcg_precond", pc)
    fn = np.linalg.norm(p.f, axis=0)
    _, _, hist_full = zip(*[O.fgmres(A, p.f[:, b], M, 1e-300, restart=5, max_iter=12)
                            for b in range(B)])
    for k in (1, 2, 4, 5, 6, 9, 12):
        u, info = S.solve(t64(p.f), tol=1e-300, max_iter=k, method="fgmres", restart=5)
        assert info.status == 1 and np.all(info.iters == k)
        ug = u.cpu().numpy()
        for b in range(B):
            uo, its, hist = O.fgmres(A, p.f[:, b], M, 1e-300, restart=5, max_iter=k)
            assert its == k
            assert np.array_equal(hist, hist_full[b][:k])  # the oracle is prefix-stable
            err = np.linalg.norm(ug[:, b] - uo) / np.linalg.norm(uo)
            assert err < 1e-10, (name, pc, k, b, err)
            assert abs(info.relres[b] - hist[-1] / fn[b]) <= 1e-10, (name, pc, k, b)
    S.close()


# ----------------------------------------------- a caller's own stream ----

@pytest.mark.parametrize("method", ["refine", "fcg", "fcg32", "fgmres"])
@pytest.mark.parametrize("prec", [64, 32])
def test_solve_on_nonblocking_stream_reports_its_own_results(method, prec):
    """On a torch stream (non-blocking with respect to the legacy default
    stream) the iteration counts and residuals a solve returns are those of
    that solve: they match the oracle's residual of the returned iterate,
    not the state a previous solve left behind."""
    p, Ho, Hp = problem("checker65")
    prm = rand_params(Hp.J, 17, 0.05)
    B = p.f.shape[1]
    S = Solver(Hp, prm, precision=prec, max_batch=B)
    if method == "fcg32":  # flexible CG with FP32 vectors
        S.set_option("fcg_fp32", 1)
        method = "fcg"
    # a previous solve with a looser tolerance leaves other counts behind
    S.solve(t64(p.f), tol=1e-2, max_iter=300, method=method, restart=10)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        f = t64(2.0 * p.f[:, ::-1])
        u, info = S.solve(f, tol=1e-9, max_iter=300, method=method, restart=10)
        un = u.cpu().numpy()  # the copy waits for `side`
    assert info.status == 0
    rr = O.relres(Ho, 2.0 * p.f[:, ::-1], un)
    assert np.all(rr < 1e-9), rr
    assert np.allclose(info.relres, rr, rtol=1e-6, atol=0.0), (info.relres, rr)
    _, ref = S.solve(f, tol=1e-9, max_iter=300, method=method, restart=10)
    assert np.array_equal(info.iters, ref.iters)
    S.close()


# ------------------------------------------------- failure detection ------

@pytest.mark.parametrize("method", ["refine", "fcg", "fcg32", "fgmres"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("where", ["f", "u"])
def test_nonfinite_input_returns_diverged(method, prec, where):
    """A NaN or Inf in a host-built right-hand side or initial guess is a
    non-finite residual: the solve returns MG_ERR_DIVERGED (no device fault),
    and the context keeps working for the next solve ("fcg32": flexible CG
    with FP32 vectors, whose first FP64 restart meets the non-finite
    residual)."""
    p, Ho, Hp = problem("checker65")
    B = p.f.shape[1]
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=prec, max_batch=B)
    if method == "fcg32":
        S.set_option("fcg_fp32", 1)
        method = "fcg"
    f = np.array(p.f)
    u0 = np.zeros_like(f)
    if where == "f":
        f[17, 1] = np.nan
    else:
        u0[5, 0] = np.inf
    with pytest.raises(MGError) as e:
        S.solve(t64(f), t64(u0), tol=1e-8, max_iter=50, method=method, restart=10)
    assert e.value.status == -6, e.value  # MG_ERR_DIVERGED
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=300, method=method, restart=10)
    assert info.status == 0
    assert np.all(O.relres(Ho, p.f, u.cpu().numpy()) < 1e-8)
    S.close()
