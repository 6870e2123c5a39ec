"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 per-cycle parity 1e-12 relative (||r_gpu - r_orc|| / ||f||
and ||u_gpu - u_orc|| / ||u_orc||); single FP64 steps 1e-13 relative; the FP32
cycle is compared with the FP64 oracle and must stay within 1e-5 relative
(FP32 unit round-off 6e-8 times the growth of a few dozen operations).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle as O
import workloads as W
from paper_2608_29082_b300 import Hierarchy, LMGParams, MGError, Solver

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rand_params(J, seed, spread=0.3, conv=True):
    r = np.random.default_rng(seed)
    p = LMGParams.identity(J)
    m = J - 1
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, m))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, m))
    for w in (p.wB, p.wR, p.wP):
        w[:, 0] += spread * r.uniform(-1, 1, m)
        if conv:
            w[:, 1] += spread * r.uniform(-1, 1, m)
    return p


def to_oracle(p: LMGParams) -> O.Params:
    return O.Params(p.theta.copy(), p.eta.copy(), p.wB.copy(), p.wR.copy(), p.wP.copy(),
                    p.nu_pre, p.nu_post)


CASES = {
    "poisson33": lambda: W.poisson_square(33, 4, batch=3, seed=1),
    "checker65": lambda: W.checkerboard_square(65, 6, ncell=8, values=(1.0, 1e4), batch=2, seed=3),
    "lognormal65": lambda: W.lognormal_square(65, seed=5, batch=2),
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


def rel(a, b, scale=None):
    s = np.linalg.norm(b) if scale is None else scale
    return np.linalg.norm(a - b) / max(s, 1e-300)


# ------------------------------------------------------------- steps ------

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("conv", [False, True])
def test_single_steps_fp64(name, conv):
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 3, conv=conv)
    po = to_oracle(prm)
    S = Solver(Hp, prm, precision=64, max_batch=4)
    r = np.random.default_rng(0)
    for lev in range(Hp.J - 1):
        Lo = Ho.levels[lev]
        n, nc = Hp.sizes[lev], Hp.sizes[lev + 1]
        f, u = r.standard_normal((n, 3)), r.standard_normal((n, 3))
        ec = r.standard_normal((nc, 3))
        out = torch.empty((n, 3), dtype=torch.float64, device=DEV)
        S.level_apply(lev, "smooth", t64(f), t64(u), out)
        ref = O.smooth(Lo, f, u, po.theta[lev], po.eta[lev], po.wB[lev])
        assert rel(out.cpu().numpy(), ref) < 1e-13, ("smooth", lev)
        S.level_apply(lev, "residual", t64(f), t64(u), out)
        assert rel(out.cpu().numpy(), f - Lo.A @ u) < 1e-13, ("residual", lev)
        outc = torch.empty((nc, 3), dtype=torch.float64, device=DEV)
        S.level_apply(lev, "restrict", t64(f), None, outc)
        ref = Lo.P.T @ O.conv(Lo, f, po.wR[lev][0], po.wR[lev][1])
        assert rel(outc.cpu().numpy(), ref) < 1e-13, ("restrict", lev)
        S.level_apply(lev, "prolong", t64(ec), t64(u), out)
        ref = u + O.conv(Lo, Lo.P @ ec, po.wP[lev][0], po.wP[lev][1])
        assert rel(out.cpu().numpy(), ref) < 1e-13, ("prolong", lev)
    nJ = Hp.sizes[-1]
    fJ = r.standard_normal((nJ, 3))
    outJ = torch.empty((nJ, 3), dtype=torch.float64, device=DEV)
    S.level_apply(Hp.J - 1, "coarse", t64(fJ), None, outJ)
    assert rel(outJ.cpu().numpy(), sla.cho_solve(Ho.chol, fJ)) < 1e-13
    S.close()


# ------------------------------------------------------------- cycles -----

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("which", ["identity", "learned"])
def test_vcycle_fp64_per_cycle_parity(name, which):
    p, Ho, Hp = problem(name)
    prm = LMGParams.identity(Hp.J) if which == "identity" else rand_params(Hp.J, 11, 0.2)
    po = to_oracle(prm)
    f = p.f
    S = Solver(Hp, prm, precision=64, max_batch=f.shape[1])
    fg = t64(f)
    ug = torch.zeros_like(fg)
    uo = np.zeros_like(f)
    fn = np.linalg.norm(f)
    for m in range(8):
        S.vcycle(fg, ug)
        uo = O.vcycle(Ho, po, f, uo)
        ugn = ug.cpu().numpy()
        ro, rg = O.residual(Ho, f, uo), O.residual(Ho, f, ugn)
        assert np.linalg.norm(rg - ro) / fn < 1e-12, m
        assert rel(ugn, uo) < 1e-12, m
    S.close()


def test_batch_independence_bitwise():
    p, Ho, Hp = problem("checker65")
    prm = rand_params(Hp.J, 5, 0.2)
    f = np.random.default_rng(9).standard_normal((Hp.sizes[0], 5))
    S5 = Solver(Hp, prm, precision=64, max_batch=5)
    S1 = Solver(Hp, prm, precision=64, max_batch=1)
    u5 = torch.zeros((Hp.sizes[0], 5), dtype=torch.float64, device=DEV)
    S5.vcycle(t64(f), u5)
    S5.vcycle(t64(f), u5)
    for b in range(5):
        u1 = torch.zeros((Hp.sizes[0], 1), dtype=torch.float64, device=DEV)
        f1 = t64(f[:, [b]])
        S1.vcycle(f1, u1)
        S1.vcycle(f1, u1)
        assert torch.equal(u1[:, 0], u5[:, b])


@pytest.mark.parametrize("name", ["poisson33", "checker65", "lshape_r2"])
def test_vcycle_fp32_error_vs_oracle(name):
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 13, 0.2)
    po = to_oracle(prm)
    f = p.f
    S = Solver(Hp, prm, precision=32, max_batch=f.shape[1])
    fg = torch.tensor(f, dtype=torch.float32, device=DEV)
    ug = torch.zeros_like(fg)
    uo = np.zeros_like(f)
    for m in range(3):
        # one FP32 cycle from the same FP32-representable iterate
        uo = O.vcycle(Ho, po, f.astype(np.float32).astype(np.float64),
                      ug.double().cpu().numpy())
        S.vcycle(fg, ug)
        err = rel(ug.double().cpu().numpy(), uo)
        assert err < 1e-5, (m, err)
    S.close()


# ------------------------------------------------------------- solves -----

def test_plain_fp64_solve_matches_oracle_iterations():
    p, Ho, Hp = problem("poisson33")
    prm = LMGParams.identity(Hp.J)
    S = Solver(Hp, prm, precision=64, max_batch=3)
    u, info = S.solve(t64(p.f), tol=1e-10, max_iter=100)
    ref = O.solve_vcycles(Ho, to_oracle(prm), p.f, 1e-10)
    assert info.status == 0
    assert np.array_equal(info.iters, ref.iters)
    rr = O.relres(Ho, p.f, u.cpu().numpy())
    assert (rr < 1e-10).all()
    assert np.allclose(info.relres, rr, rtol=1e-6)


@pytest.mark.parametrize("name", ["checker65", "lognormal65", "lshape_r2"])
def test_fp32_refinement_reaches_tolerance(name):
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 17, 0.05)
    S = Solver(Hp, prm, precision=32, max_batch=p.f.shape[1])
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=400)
    assert info.status == 0
    rr = O.relres(Ho, p.f, u.cpu().numpy())  # re-evaluated by the oracle in FP64
    assert (rr < 1e-8).all(), rr
    ref = O.solve_refinement(Ho, to_oracle(prm), p.f, 1e-8, max_iter=400)
    # FP32 inner cycles: iteration counts within a few of the FP64 oracle's
    assert np.all(np.abs(info.iters - ref.iters) <= max(2, 0.1 * ref.iters.max()))


@pytest.mark.parametrize("name", ["checker65", "lognormal65", "lshape_r2"])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_fp32_refinement_replays_bitwise(name, nrhs):
    """The FP32 refinement loop (one captured graph: the cycle, u += 2^s c,
    the FP64 residual with the next cycle's scaled residual and first
    smoothing delta, the test) equals, bitwise, a host replay of Algorithm
    2 inside iterative refinement through entry points that fold nothing:
    r = f - A u in FP64, s = ilogb ||r||, c = one FP32 cycle on float(2^-s r)
    from zero, u += 2^s c."""
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 23, 0.05)
    f = t64(np.random.default_rng(31).standard_normal((Hp.sizes[0], nrhs)))
    S = Solver(Hp, prm, precision=32, max_batch=nrhs)
    K = 4
    u = torch.zeros_like(f)
    r = torch.empty_like(f)
    for _ in range(K):
        S.level_apply(0, "outer_residual", f, u, r)
        rn = np.sqrt((r.cpu().numpy() ** 2).sum(axis=0))
        sexp = np.frexp(rn)[1] - 1  # ilogb
        scale = torch.tensor(np.ldexp(1.0, -sexp), dtype=torch.float64, device=DEV)
        rhat = (r * scale).float()
        c = torch.zeros_like(rhat)
        S.vcycle(rhat, c)
        u = u + c.double() / scale
    us, info = S.solve(f, tol=1e-300, max_iter=K)
    assert np.array_equal(info.iters, np.full(nrhs, K))
    assert torch.equal(us, u), (name, (us - u).abs().max().item())
    S.close()


def test_solve_result_independent_of_batch():
    p, Ho, Hp = problem("lognormal65")
    prm = rand_params(Hp.J, 19, 0.05)
    f = np.random.default_rng(4).standard_normal((Hp.sizes[0], 4))
    f[:, 2] *= 1e-3  # different scale and convergence history
    S4 = Solver(Hp, prm, precision=32, max_batch=4)
    S1 = Solver(Hp, prm, precision=32, max_batch=1)
    u4, i4 = S4.solve(t64(f), tol=1e-8, max_iter=200)
    for b in range(4):
        u1, i1 = S1.solve(t64(f[:, [b]]), tol=1e-8, max_iter=200)
        assert i1.iters[0] == i4.iters[b]
        assert torch.equal(u1[:, 0], u4[:, b])


def test_solve_host_equals_device():
    p, Ho, Hp = problem("checker65")
    prm = LMGParams.identity(Hp.J)
    S = Solver(Hp, prm, precision=32, max_batch=2)
    ud, infod = S.solve(t64(p.f), tol=1e-8, max_iter=400)
    uh, infoh = S.solve_host(p.f, tol=1e-8, max_iter=400)
    assert np.array_equal(ud.cpu().numpy(), uh)
    assert np.array_equal(infod.iters, infoh.iters)


# ------------------------------------------------------------ edge cases --

def test_odd_and_zero_smoothing_steps():
    p, Ho, Hp = problem("checker65")
    for nu_pre, nu_post in [(1, 0), (0, 3), (3, 1)]:
        for conv in (False, True):
            prm = rand_params(Hp.J, 23, 0.2, conv=conv)
            prm.nu_pre, prm.nu_post = nu_pre, nu_post
            po = to_oracle(prm)
            S = Solver(Hp, prm, precision=64, max_batch=2)
            ug = torch.zeros((Hp.sizes[0], 2), dtype=torch.float64, device=DEV)
            S.vcycle(t64(p.f), ug)
            S.vcycle(t64(p.f), ug)
            uo = O.vcycle(Ho, po, p.f, O.vcycle(Ho, po, p.f, np.zeros_like(p.f)))
            assert rel(ug.cpu().numpy(), uo) < 1e-12, (nu_pre, nu_post, conv)
            S.close()


def test_set_params_switches_kernels():
    p, Ho, Hp = problem("poisson33")
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=64, max_batch=3)
    for k, prm in enumerate([LMGParams.identity(Hp.J), rand_params(Hp.J, 29, 0.2),
                             LMGParams.identity(Hp.J), rand_params(Hp.J, 31, 0.2, conv=False)]):
        S.set_params(prm)
        ug = torch.zeros((Hp.sizes[0], 3), dtype=torch.float64, device=DEV)
        S.vcycle(t64(p.f), ug)
        uo = O.vcycle(Ho, to_oracle(prm), p.f, np.zeros_like(p.f))
        assert rel(ug.cpu().numpy(), uo) < 1e-12, k


def test_invalid_calls_raise():
    p, Ho, Hp = problem("poisson33")
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=64, max_batch=2)
    f = torch.zeros((Hp.sizes[0], 3), dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        S.vcycle(f, torch.zeros_like(f))  # batch 3 > max_batch 2
    with pytest.raises(MGError):
        S.level_apply(0, "coarse", f[:, :1].contiguous(), None, torch.zeros_like(f[:, :1]))
    bad = LMGParams.identity(Hp.J + 1)
    with pytest.raises(MGError):
        S.set_params(bad)


def test_zero_rhs_and_not_converged():
    p, Ho, Hp = problem("checker65")
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=32, max_batch=2)
    f = torch.zeros((Hp.sizes[0], 2), dtype=torch.float64, device=DEV)
    f[:, 1] = 1.0
    u, info = S.solve(f, tol=1e-8, max_iter=2)
    assert info.status == 1  # MG_NOT_CONVERGED: column 1 needs more than 2 iterations
    assert info.iters[0] == 0 and info.iters[1] == 2
    assert torch.all(u[:, 0] == 0)


# ------------------------------------------------- full-size workload -----

@pytest.mark.slow
def test_full_size_checkerboard_513():
    """The 513^2, 9-level jump-coefficient workload in the benchmark's launch
    configuration: one FP64 cycle against the oracle, and the FP32 + FP64
    refinement solve re-checked by the oracle."""
    p = W.checkerboard_square()
    Ho = O.build_hierarchy(p)
    Hp = Hierarchy.from_problem(p)
    prm = LMGParams.identity(Hp.J)
    S64 = Solver(Hp, prm, precision=64, max_batch=1)
    ug = torch.zeros((Hp.sizes[0], 1), dtype=torch.float64, device=DEV)
    S64.vcycle(t64(p.f), ug)
    uo = O.vcycle(Ho, to_oracle(prm), p.f, np.zeros_like(p.f))
    assert rel(ug.cpu().numpy(), uo) < 1e-12
    S64.close()
    S32 = Solver(Hp, prm, precision=32, max_batch=1)
    u, info = S32.solve(t64(p.f), tol=1e-8, max_iter=400)
    assert info.status == 0
    assert O.relres(Ho, p.f, u.cpu().numpy())[0] < 1e-8
    # 5 rhs at this size take the per-rhs reduction blocks, 1 rhs the merged
    # reduce-and-test block: the same sums in the same order, so every rhs is
    # bitwise its solve alone (refinement and flexible CG)
    f5 = np.concatenate([p.f, np.random.default_rng(21).standard_normal((Hp.sizes[0], 4))], 1)
    S5 = Solver(Hp, prm, precision=32, max_batch=5)
    for method in ("refine", "fcg"):
        u5, i5 = S5.solve(t64(f5), tol=1e-8, max_iter=400, method=method)
        for b in (0, 3):
            u1, i1 = S32.solve(t64(f5[:, [b]]), tol=1e-8, max_iter=400, method=method)
            assert torch.equal(u1[:, 0], u5[:, b]), (method, b)
            assert i1.iters[0] == i5.iters[b] and i1.relres[0] == i5.relres[b]
    S5.close()


# ------------------------------------------------------ flexible CG outer --

@pytest.mark.parametrize("name", ["checker65", "lognormal65", "lshape_r2"])
@pytest.mark.parametrize("prec", [64, 32])
def test_fcg_reaches_tolerance_with_fewer_iterations(name, prec):
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 47, 0.05)
    S = Solver(Hp, prm, precision=prec, max_batch=p.f.shape[1])
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=400, method="fcg")
    assert info.status == 0
    rr = O.relres(Ho, p.f, u.cpu().numpy())  # true residual, re-evaluated by the oracle
    assert (rr < 1e-8).all(), rr
    assert np.allclose(info.relres, rr, rtol=1e-6)
    _, info_r = S.solve(t64(p.f), tol=1e-8, max_iter=400, method="refine")
    assert info.iters.max() <= info_r.iters.max()


@pytest.mark.parametrize("nrhs", [3, 12, 16])
@pytest.mark.parametrize("fp32", [1, 0])
def test_fcg_result_independent_of_batch(nrhs, fp32):
    """Each right-hand side's FCG result and count are bitwise those of its
    solve alone, with FP32 vectors (right-hand-side tiles of 1, 4 and 8
    columns in the product q = A p for 3, 12 and 16 rhs; 1 alone) and with
    FP64 vectors."""
    p, Ho, Hp = problem("lognormal65")
    prm = rand_params(Hp.J, 53, 0.05)
    f = np.random.default_rng(8).standard_normal((Hp.sizes[0], nrhs))
    f[:, 1] *= 1e-4
    S3 = Solver(Hp, prm, precision=32, max_batch=nrhs)
    S1 = Solver(Hp, prm, precision=32, max_batch=1)
    for S in (S3, S1):
        S.set_option("fcg_fp32", fp32)
    u3, i3 = S3.solve(t64(f), tol=1e-8, max_iter=200, method="fcg")
    for b in sorted({0, 1, 2, nrhs - 1}):
        u1, i1 = S1.solve(t64(f[:, [b]]), tol=1e-8, max_iter=200, method="fcg")
        assert i1.iters[0] == i3.iters[b], (b, i1.iters, i3.iters)
        assert torch.equal(u1[:, 0], u3[:, b]), b


@pytest.mark.parametrize("name", ["poisson33", "checker65", "lshape_r2"])
def test_fcg_fp32_vectors_against_fp64_vectors(name):
    """Precision-32 FCG with FP32 vectors and FP64 restarts (the default) and
    with FP64 vectors both reach 1e-8 for every right-hand side, re-checked
    by the oracle from the returned iterate; the reported relres is the
    restart's FP64 residual (the oracle's within 1e-6 relative); the FP32
    form takes at most a few steps more (a restart drops the one kept
    direction).  Phase floors 10^-3 .. 10^-6 and none all converge."""
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 61, 0.05)
    S = Solver(Hp, prm, precision=32, max_batch=p.f.shape[1])
    out = {}
    for fp32, floor in ((0, 4), (1, 4), (1, 3), (1, 6), (1, 0)):
        S.set_option("fcg_fp32", fp32)
        S.set_option("fcg_floor", floor)
        u, info = S.solve(t64(p.f), tol=1e-8, max_iter=400, method="fcg")
        assert info.status == 0, (fp32, floor)
        rr = O.relres(Ho, p.f, u.cpu().numpy())
        assert (rr < 1e-8).all(), (fp32, floor, rr)
        assert np.allclose(info.relres, rr, rtol=1e-6, atol=0.0), (fp32, floor)
        out[(fp32, floor)] = info.iters.max()
    assert out[(1, 4)] <= out[(0, 4)] + 5, out
    for bad in (-1, 16):
        with pytest.raises(MGError):
            S.set_option("fcg_floor", bad)
    with pytest.raises(MGError):
        S.set_option("fcg_fp32", 3)
    S.close()


def test_fcg_fp32_last_iteration_restarts():
    """Stopped by max_iter, the FP32 form still folds its correction into u
    and reports the FP64 residual of that u (MG_NOT_CONVERGED), which the
    oracle re-computes; the count is max_iter."""
    p, Ho, Hp = problem("checker65")
    prm = rand_params(Hp.J, 61, 0.05)
    S = Solver(Hp, prm, precision=32, max_batch=p.f.shape[1])
    S.set_option("fcg_fp32", 1)
    for k in (1, 3, 7):
        u, info = S.solve(t64(p.f), tol=1e-14, max_iter=k, method="fcg")
        assert info.status == 1 and (info.iters == k).all(), (k, info.iters)
        rr = O.relres(Ho, p.f, u.cpu().numpy())
        assert np.allclose(info.relres, rr, rtol=1e-6, atol=0.0), (k, info.relres, rr)
        assert np.isfinite(rr).all()
    S.close()


@pytest.mark.parametrize("inverse", [1, 0])
@pytest.mark.parametrize("nrhs", [1, 4, 16])
def test_coarse_solve_matches_cholesky(inverse, nrhs):
    """The L-shape coarsest level (161 rows): the explicit-inverse product
    (default) and the shared-memory packed-factor substitutions (option off,
    one block per right-hand side) both give scipy's Cholesky solve to
    1e-13; the cycle with the inverse stays within 1e-12 of the oracle's,
    and in the small-levels block (tail) it is bitwise the grid kernel's."""
    p, Ho, Hp = problem("lshape_r2")
    prm = rand_params(Hp.J, 59)
    S = Solver(Hp, prm, precision=64, max_batch=16)
    S.set_option("coarse_inverse", inverse)
    nJ = Hp.sizes[-1]
    fJ = np.random.default_rng(2).standard_normal((nJ, nrhs))
    out = torch.empty((nJ, nrhs), dtype=torch.float64, device=DEV)
    S.level_apply(Hp.J - 1, "coarse", t64(fJ), None, out)
    assert rel(out.cpu().numpy(), sla.cho_solve(Ho.chol, fJ)) < 1e-13
    f = p.f[:, :1] if nrhs == 1 else np.concatenate([p.f] * (nrhs // 2), axis=1)
    outs = []
    for tail in (0, 1 << 30):
        S.set_option("tail_work", tail)
        ug = torch.zeros((Hp.sizes[0], nrhs), dtype=torch.float64, device=DEV)
        S.vcycle(t64(f), ug)
        outs.append(ug.clone())
    assert torch.equal(outs[0], outs[1])
    uo = O.vcycle(Ho, to_oracle(prm), f, np.zeros_like(f))
    assert rel(outs[0].cpu().numpy(), uo) < 1e-12
    with pytest.raises(MGError):
        S.set_option("coarse_inverse", 2)
    S.close()


# --------------------------------------------------------- launch options --

@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("conv", [False, True])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_launch_options_are_bitwise_neutral(prec, conv, nrhs):
    """The single-block small-level kernel, programmatic dependent launch, the
    multi-rhs tiles and the halo-fused DIA steps (tiles of many blocks, a tile
    narrower than the finest level's halo that falls back there, one block per
    level) change launch
    shapes only: the cycle and the solve are bitwise identical."""
    p, Ho, Hp = problem("checker65")
    prm = rand_params(Hp.J, 37, 0.1, conv=conv)
    dt = torch.float64 if prec == 64 else torch.float32
    outs = []
    f4 = np.concatenate([p.f, 0.5 * p.f[:, ::-1]], axis=1)[:, :nrhs]
    for tail, pdl, mrhs, halo, teams in [(8192, 1, 1, 2048, 1), (0, 1, 1, 2048, 1),
                                         (8192, 0, 1, 2048, 1), (1 << 30, 1, 1, 2048, 1),
                                         (8192, 1, 0, 2048, 1), (0, 1, 0, 2048, 1),
                                         (8192, 1, 1, 0, 1), (0, 1, 1, 256, 1), (0, 1, 0, 50, 1),
                                         (0, 0, 1, 1 << 20, 1), (8192, 1, 1, 2048, 0),
                                         (1 << 30, 1, 1, 2048, 0)]:
        S = Solver(Hp, prm, precision=prec, max_batch=4)
        S.set_option("tail_work", tail)
        S.set_option("tail_teams", teams)
        S.set_option("pdl", pdl)
        S.set_option("multi_rhs", mrhs)
        S.set_option("halo_rows", halo)
        u = torch.zeros((Hp.sizes[0], nrhs), dtype=dt, device=DEV)
        f = torch.tensor(f4, dtype=dt, device=DEV)
        S.vcycle(f, u)
        S.vcycle(f, u)
        us, info = S.solve(t64(p.f), tol=1e-9, max_iter=300)
        outs.append((u.clone(), us.clone(), info.iters.copy()))
        S.close()
    for u, us, it in outs[1:]:
        assert torch.equal(u, outs[0][0])
        assert torch.equal(us, outs[0][1])
        assert np.array_equal(it, outs[0][2])


@pytest.mark.parametrize("name", ["poisson33", "checker65", "lognormal65"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_halo2d_tiles_are_bitwise_neutral(name, prec, nrhs):
    """The 2D-tiled fused steps on DIA levels (forced on every grid level:
    the byte threshold 1, no 1D halo, no single-block kernel; tiles wider
    and taller than the coarse grids, ragged last tiles, 5- and 7-point
    offsets) give the two-kernel cycle and solve bitwise, with and without
    the convolutions."""
    p, Ho, Hp = problem(name)
    dt = torch.float64 if prec == 64 else torch.float32
    f = np.random.default_rng(nrhs).standard_normal((Hp.sizes[0], nrhs))
    for conv in (True, False):
        prm = rand_params(Hp.J, 41, 0.1, conv=conv)
        outs = []
        for bytes_ in (0, 1):
            S = Solver(Hp, prm, precision=prec, max_batch=nrhs)
            S.set_option("tail_work", 0)
            S.set_option("halo_rows", 0)
            S.set_option("halo2d_bytes", bytes_)
            u = torch.zeros((Hp.sizes[0], nrhs), dtype=dt, device=DEV)
            fd = torch.tensor(f, dtype=dt, device=DEV)
            for _ in range(3):
                S.vcycle(fd, u)
            us, info = S.solve(t64(f), tol=1e-9, max_iter=300)
            outs.append((u.clone(), us.clone(), info.iters.copy()))
            S.close()
        assert torch.isfinite(outs[0][0]).all()
        assert torch.equal(outs[1][0], outs[0][0]), (name, conv)
        assert torch.equal(outs[1][1], outs[0][1]), (name, conv)
        assert np.array_equal(outs[1][2], outs[0][2])


@pytest.mark.parametrize("name", ["poisson33", "checker65", "lognormal65"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("grid_only", [True, False])
def test_dia_two_rows_are_bitwise_neutral(name, prec, grid_only):
    """One right-hand side on DIA levels: the kernels taking two rows per
    thread (residual, SAGEConv update, Phi_R, Phi_P with the update; odd
    row counts leave one row to the last thread) give the one-row kernels'
    cycle, refinement, FCG and FGMRES solves bitwise, with and without the
    convolutions; grid_only runs every level as grid kernels."""
    p, Ho, Hp = problem(name)
    dt = torch.float64 if prec == 64 else torch.float32
    f = np.random.default_rng(5).standard_normal((Hp.sizes[0], 1))
    for conv in (True, False):
        prm = rand_params(Hp.J, 43, 0.1, conv=conv)
        outs = []
        for two in (0, 1):
            S = Solver(Hp, prm, precision=prec, max_batch=1)
            if grid_only:
                S.set_option("tail_work", 0)
                S.set_option("halo_rows", 0)
            S.set_option("dia_two_rows", two)
            u = torch.zeros((Hp.sizes[0], 1), dtype=dt, device=DEV)
            fd = torch.tensor(f, dtype=dt, device=DEV)
            for _ in range(3):
                S.vcycle(fd, u)
            res = [u.clone()]
            for method in ("refine", "fcg", "fgmres"):
                us, info = S.solve(t64(f), tol=1e-9, max_iter=300, method=method)
                res += [us.clone(), info.iters.copy()]
            outs.append(res)
            S.close()
        assert torch.isfinite(outs[0][0]).all()
        for a, b in zip(outs[1], outs[0]):
            if isinstance(a, torch.Tensor):
                assert torch.equal(a, b), (name, conv)
            else:
                assert np.array_equal(a, b), (name, conv)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("method", ["refine", "fcg"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_host_driven_loop_matches_device_loop(prec, method, nrhs):
    """A solve whose iterations the host drives (plain graphs, the flag read
    after every iteration) is bitwise the solve whose loop is a device while
    node: same iterate, iteration counts and residuals."""
    p, Ho, Hp = problem("checker65")
    prm = rand_params(Hp.J, 67, 0.1)
    f = t64(np.random.default_rng(8).standard_normal((Hp.sizes[0], nrhs)))
    res = []
    for loop in (1, 0):
        S = Solver(Hp, prm, precision=prec, max_batch=nrhs)
        S.set_option("device_loop", loop)
        u, info = S.solve(f, tol=1e-9, max_iter=300, method=method)
        n0 = S.kernel_launches()
        u2, info2 = S.solve(f, tol=1e-9, max_iter=300, method=method)
        res.append((u.clone(), info.iters.copy(), info.relres.copy(), S.kernel_launches() - n0))
        assert torch.equal(u, u2)
        S.close()
    (ua, ia, ra, ka), (ub, ib, rb, kb) = res
    assert torch.equal(ua, ub)
    assert np.array_equal(ia, ib) and np.array_equal(ra, rb)
    assert ia.max() > 1 and (ra < 1e-9).all()
    assert ka == kb  # both forms count the same kernels


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nrhs", [12, 16])
def test_multi_rhs_tiles_are_bitwise_neutral(prec, nrhs):
    """Every right-hand-side tile width (several adjacent lanes per row, a
    non-power-of-two lane count for 12 rhs) gives the one-thread-per-(row,
    rhs) cycle bitwise, on a SELL level (L-shape) and on DIA levels."""
    from paper_2608_29082_b300._lib import MGError
    for name in ("lshape_r2", "checker65"):
        p, Ho, Hp = problem(name)
        prm = rand_params(Hp.J, 61, 0.1, conv=True)
        dt = torch.float64 if prec == 64 else torch.float32
        f = torch.tensor(np.random.default_rng(5).standard_normal((Hp.sizes[0], nrhs)),
                         dtype=dt, device=DEV)
        S = Solver(Hp, prm, precision=prec, max_batch=nrhs)
        S.set_option("tail_work", 0)
        outs = []
        for tile in (0, 1, 2, 4, 8, 16):
            S.set_option("multi_rhs", tile)
            u = torch.zeros_like(f)
            S.vcycle(f, u)
            S.vcycle(f, u)
            outs.append(u.clone())
        with pytest.raises(MGError):
            S.set_option("multi_rhs", 3)
        S.close()
        assert torch.isfinite(outs[0]).all()
        for u in outs[1:]:
            assert torch.equal(u, outs[0])


@pytest.mark.parametrize("prec", [64, 32])
def test_dia_and_sell_layouts_agree_bitwise(prec):
    """Structured levels are stored as DIA by default; forcing SELL-32 must
    give bitwise the same cycle, solve and parameter gradient."""
    from paper_2608_29082_b300 import _lib as Lb
    p, Ho, Hp = problem("checker65")
    prm = rand_params(Hp.J, 43, 0.1)
    dt = torch.float64 if prec == 64 else torch.float32
    outs = []
    try:
        for policy in (0, 1):
            Lb.check(Lb.lib().mg_set_layout_policy(policy))
            S = Solver(Hp, prm, precision=prec, max_batch=2)
            f = torch.tensor(p.f, dtype=dt, device=DEV)
            u = torch.zeros_like(f)
            S.vcycle(f, u)
            us, info = S.solve(t64(p.f), tol=1e-9, max_iter=300)
            u2 = torch.zeros_like(f)
            S.forward_record(f, u2, 2)
            _, _, gp = S.backward(torch.ones_like(f), 2, want_inputs=False)
            outs.append((u, us, gp))
            S.close()
    finally:
        Lb.lib().mg_set_layout_policy(0)
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_whole_cycle_in_one_block_matches_oracle():
    """Tiny hierarchy: with the tail threshold above level 0 the entire cycle
    runs in one thread block; FP64 parity with the oracle still holds."""
    p, Ho, Hp = problem("poisson33")
    prm = rand_params(Hp.J, 41, 0.2)
    S = Solver(Hp, prm, precision=64, max_batch=3)
    S.set_option("tail_work", 1 << 30)
    f = t64(p.f)
    u = torch.zeros_like(f)
    uo = np.zeros_like(p.f)
    for m in range(4):
        S.vcycle(f, u)
        uo = O.vcycle(Ho, to_oracle(prm), p.f, uo)
        assert rel(u.cpu().numpy(), uo) < 1e-12


# ------------------------------------------------------ full multigrid -----

@pytest.mark.parametrize("name", ["poisson33", "checker65", "lshape_r2"])
def test_fmg_matches_oracle(name):
    """One full multigrid application (mg_fmg) against the oracle's nested
    iteration: FP64 to 1e-12, FP32 within 1e-5; repeated calls are the same
    (u's input is not read); with and without the small-levels block (a cycle
    started inside it from a nonzero guess) the result is bitwise equal."""
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 71, 0.2)
    f = p.f
    ref = O.fmg(Ho, to_oracle(prm), f)
    S = Solver(Hp, prm, precision=64, max_batch=f.shape[1])
    u = torch.zeros((Hp.sizes[0], f.shape[1]), dtype=torch.float64, device=DEV)
    S.fmg(t64(f), u)
    assert rel(u.cpu().numpy(), ref) < 1e-12
    u2 = torch.full_like(u, 7.0)
    S.fmg(t64(f), u2)
    assert torch.equal(u, u2)
    S.set_option("tail_work", 0)
    u3 = torch.zeros_like(u)
    S.fmg(t64(f), u3)
    assert torch.equal(u, u3)
    S.close()
    S32 = Solver(Hp, prm, precision=32, max_batch=f.shape[1])
    f32 = torch.tensor(f, dtype=torch.float32, device=DEV)
    u32 = torch.zeros_like(f32)
    S32.fmg(f32, u32)
    ref32 = O.fmg(Ho, to_oracle(prm), f.astype(np.float32).astype(np.float64))
    assert rel(u32.double().cpu().numpy(), ref32) < 1e-5
    S32.close()


@pytest.mark.parametrize("name", ["checker65", "lognormal65", "lshape_r2"])
@pytest.mark.parametrize("prec", [64, 32])
def test_fcg_with_fmg_preconditioner(name, prec):
    """Flexible CG preconditioned by full multigrid reaches 1e-8 (re-checked
    by the oracle) in no more iterations than with the V-cycle."""
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 23, 0.05)
    S = Solver(Hp, prm, precision=prec, max_batch=p.f.shape[1])
    _, iv = S.solve(t64(p.f), tol=1e-8, max_iter=300, method="fcg")
    S.set_option("fcg_precond", 1)
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=300, method="fcg")
    assert info.status == 0
    assert (O.relres(Ho, p.f, u.cpu().numpy()) < 1e-8).all()
    assert info.iters.max() <= iv.iters.max()
    with pytest.raises(MGError):
        S.set_option("fcg_precond", 2)
    S.close()


# ------------------------------------------------------ flexible GMRES -----

@pytest.mark.parametrize("name", ["checker65", "lognormal65", "lshape_r2"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("pc", [0, 1])
def test_fgmres_reaches_tolerance(name, prec, pc):
    """Restarted flexible GMRES with a nonsymmetric learnable V-cycle (pc 0)
    or full multigrid (pc 1) as preconditioner reaches 1e-8 (re-checked by
    the oracle); in FP64 each right-hand side takes the oracle FGMRES's
    iteration count to within one step (CGS2 here, MGS there)."""
    p, Ho, Hp = problem(name)
    # a nonsymmetric learnable cycle; with FMG a milder Theta (FMG with the
    # 0.2-spread one is no preconditioner at all: the oracle's FGMRES
    # stagnates at relres 0.99 with it, and so does this one)
    prm = rand_params(Hp.J, 29, 0.2) if pc == 0 else rand_params(Hp.J, 23, 0.05)
    S = Solver(Hp, prm, precision=prec, max_batch=p.f.shape[1])
    S.set_option("fcg_precond", pc)
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=300, method="fgmres", restart=10)
    assert info.status == 0
    assert (O.relres(Ho, p.f, u.cpu().numpy()) < 1e-8).all()
    if prec == 64:
        po = to_oracle(prm)
        if pc:
            M = lambda v: O.fmg(Ho, po, v[:, None])[:, 0]  # noqa: E731
        else:
            M = lambda v: O.vcycle(Ho, po, v[:, None], np.zeros((v.size, 1)))[:, 0]  # noqa: E731
        for b in range(p.f.shape[1]):
            _, its, _ = O.fgmres(Ho.levels[0].A, p.f[:, b], M, 1e-8, restart=10, max_iter=300)
            assert abs(int(info.iters[b]) - its) <= 1, (b, info.iters[b], its)
    with pytest.raises(MGError):
        S.solve(t64(p.f), tol=1e-8, method="fgmres", restart=0)
    S.close()


def test_fgmres_zero_rhs_and_not_converged():
    p, Ho, Hp = problem("checker65")
    S = Solver(Hp, LMGParams.identity(Hp.J), precision=32, max_batch=2)
    f = np.array(p.f)
    f[:, 1] = 0.0
    u, info = S.solve(t64(f), tol=1e-8, max_iter=300, method="fgmres", restart=10)
    assert info.status == 0 and info.iters[1] == 0 and torch.all(u[:, 1] == 0)
    u, info = S.solve(t64(p.f), tol=1e-14, max_iter=3, method="fgmres", restart=10)
    assert info.status == 1 and info.iters.max() == 3
    S.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", ["lognormal65", "poisson33"])
def test_fgmres_batch_independent(name, prec):
    """A right-hand side's FGMRES run does not depend on the rest of the
    batch: the reductions group terms independently of B, and a right-hand
    side whose cycle ended early waits with its own columns only."""
    p, Ho, Hp = problem(name)
    assert p.f.shape[1] >= 2
    S = Solver(Hp, rand_params(Hp.J, 29, 0.2), precision=prec, max_batch=p.f.shape[1])
    ub, ib = S.solve(t64(p.f), tol=1e-8, max_iter=300, method="fgmres", restart=8)
    assert ib.status == 0
    for b in range(p.f.shape[1]):
        u1, i1 = S.solve(t64(p.f[:, b:b + 1]), tol=1e-8, max_iter=300, method="fgmres",
                         restart=8)
        assert int(i1.iters[0]) == int(ib.iters[b])
        assert torch.equal(u1[:, 0], ub[:, b])
    S.close()


@pytest.mark.gpu
@pytest.mark.parametrize("floor", [0, 7])
def test_fgmres_fp32_floor(floor):
    """FP32 cycles with another floor (0: none) still reach 1e-8 through the
    FP64 restarts; out-of-range floors are rejected."""
    p, Ho, Hp = problem("checker65")
    S = Solver(Hp, rand_params(Hp.J, 29, 0.2), precision=32, max_batch=p.f.shape[1])
    S.set_option("fgmres_floor", floor)
    u, info = S.solve(t64(p.f), tol=1e-8, max_iter=300, method="fgmres", restart=10)
    assert info.status == 0
    assert (O.relres(Ho, p.f, u.cpu().numpy()) < 1e-8).all()
    for bad in (-1, 16):
        with pytest.raises(MGError):
            S.set_option("fgmres_floor", bad)
    S.close()


# ------------------------------------------------- SELL halo-tiled steps --

CASES["lshape_r3"] = lambda: W.lshape_anisotropic(refinements=3, batch=2, seed=4)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("conv", [False, True])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_sell_halo_tiles_are_bitwise_neutral(prec, conv, nrhs):
    """On SELL levels (the jittered L-shape) the halo-tiled fused steps
    (one kernel per smoothing step, residual + Phi_R, P e_c + Phi_P) give
    bitwise the two-kernel cycle and solve, for every tile size (tiles
    smaller than a halo, a ragged last tile, one tile for a whole level)
    and right-hand-side tile width (16 rhs: 8 per thread; 3: one)."""
    for name in ("lshape_r2", "lshape_r3"):
        p, Ho, Hp = problem(name)
        prm = rand_params(Hp.J, 73, 0.1, conv=conv)
        dt = torch.float64 if prec == 64 else torch.float32
        f = np.random.default_rng(nrhs).standard_normal((Hp.sizes[0], nrhs))
        outs = []
        for rows in (0, 32, 96, 256, 1024, 8192):
            S = Solver(Hp, prm, precision=prec, max_batch=nrhs)
            S.set_option("sell_halo_rows", rows)
            S.set_option("tail_work", 0)  # every level a grid level
            u = torch.zeros((Hp.sizes[0], nrhs), dtype=dt, device=DEV)
            fd = torch.tensor(f, dtype=dt, device=DEV)
            S.vcycle(fd, u)
            S.vcycle(fd, u)
            us, info = S.solve(t64(f), tol=1e-9, max_iter=100, method="fcg")
            outs.append((u.clone(), us.clone(), info.iters.copy()))
            S.close()
        assert torch.isfinite(outs[0][0]).all()
        for u, us, it in outs[1:]:
            assert torch.equal(u, outs[0][0]), name
            assert torch.equal(us, outs[0][1]), name
            assert np.array_equal(it, outs[0][2]), name


def test_sell_halo_cycle_matches_oracle_and_steps():
    """The fused SELL path against the oracle directly: single FP64 smoothing
    steps (1e-13) and cycles (1e-12) on the L-shape, and the option is
    validated."""
    p, Ho, Hp = problem("lshape_r3")
    prm = rand_params(Hp.J, 79, 0.2)
    po = to_oracle(prm)
    S = Solver(Hp, prm, precision=64, max_batch=2)
    S.set_option("sell_halo_rows", 64)
    r = np.random.default_rng(3)
    for lev in range(Hp.J - 1):
        n = Hp.sizes[lev]
        f, u = r.standard_normal((n, 2)), r.standard_normal((n, 2))
        out = torch.empty((n, 2), dtype=torch.float64, device=DEV)
        S.level_apply(lev, "smooth", t64(f), t64(u), out)
        ref = O.smooth(Ho.levels[lev], f, u, po.theta[lev], po.eta[lev], po.wB[lev])
        assert rel(out.cpu().numpy(), ref) < 1e-13, lev
    ug = torch.zeros((Hp.sizes[0], 2), dtype=torch.float64, device=DEV)
    uo = np.zeros_like(p.f)
    for m in range(4):
        S.vcycle(t64(p.f), ug)
        uo = O.vcycle(Ho, po, p.f, uo)
        assert rel(ug.cpu().numpy(), uo) < 1e-12, m
    for bad in (-32, 33, 8224):
        with pytest.raises(MGError):
            S.set_option("sell_halo_rows", bad)
    S.close()
