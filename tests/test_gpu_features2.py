"""Two features per node (mg2_*) against the FP64 oracle, through the C ABI.

The complex Helmholtz operator with impedance boundary (Sec. 4.2) and
random two-feature weights W_1, W_2 in R^{2x2}.  Per-cycle parity: the GPU
cycle and the oracle cycle map the same iterate; FP64 within 1e-12
relative.  FP32 against the FP64 oracle applied to the FP32 input: 1e-5 for
the cycle from zero; afterwards FP32 rounds f - A u relative to
||A|| ||u||, so the bound scales with the residual's cancellation factor
c = (||f|| + ||A||_inf ||u||) / ||f - A u||: max(1e-5, 5e-7 c), about
8 FP32 unit round-offs per unit of c (measured: at most 4).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2608_29082_b300 import MGError
from paper_2608_29082_b300.features2 import Hierarchy2, Params2, Solver2

pytestmark = pytest.mark.gpu

CASES = {
    "helmholtz33": lambda: W.helmholtz_square(33, 3, k=2 * np.pi, batch=2, seed=3),
    "helmholtz65": lambda: W.helmholtz_square(65, 4, k=4 * np.pi, batch=3, seed=4),
}
_cache = {}


def problem(name):
    if name not in _cache:
        p = CASES[name]()
        _cache[name] = (p, O.build_hierarchy(p), Hierarchy2.from_problem(p))
    return _cache[name]


def params(J, seed, spread=0.3):
    r = np.random.default_rng(seed)
    p = Params2.identity(J)
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, J - 1))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, J - 1))
    for Wt in (p.WB, p.WR, p.WP):
        Wt += spread * r.uniform(-1, 1, Wt.shape)
    return p


def to_oracle(p: Params2) -> O.Params2:
    return O.Params2(p.theta.copy(), p.eta.copy(), p.WB.copy(), p.WR.copy(), p.WP.copy(),
                     p.nu_pre, p.nu_post)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nu", [(1, 1), (1, 2)])
def test_two_feature_cycle_parity(name, prec, nu):
    p, Ho, Hp = problem(name)
    prm = params(Hp.J, 11)
    prm.nu_pre, prm.nu_post = nu
    po = to_oracle(prm)
    S = Solver2(Hp, prm, precision=prec, max_batch=p.f.shape[1])
    dt = torch.complex128 if prec == 64 else torch.complex64
    f = torch.tensor(p.f, dtype=dt, device="cuda")
    fo = f.cpu().numpy().astype(np.complex128)
    u = torch.zeros_like(f)
    A = Ho.levels[0].A
    nA = abs(A).sum(axis=1).max()
    for m in range(3):
        u_in = u.cpu().numpy().astype(np.complex128)
        S.vcycle(f, u)
        ref = O.vcycle2(Ho, po, fo, u_in)
        if prec == 64:
            tol = 1e-12
        else:
            c = (np.linalg.norm(fo) + nA * np.linalg.norm(u_in)) / np.linalg.norm(fo - A @ u_in)
            tol = max(1e-5, 5e-7 * c)
        assert rel(u.cpu().numpy().astype(np.complex128), ref) < tol, m
    S.close()


def test_classical_cycle_reduces_error():
    """W_1 = I, W_2 = 0 (the classical cycle) on a mildly indefinite system:
    the FP64 cycle as a stationary iteration decreases the residual, and
    agrees with the oracle's iterates."""
    p = W.helmholtz_square(33, 3, k=np.pi, batch=1, seed=0)
    Ho, Hp = O.build_hierarchy(p), Hierarchy2.from_problem(p)
    prm = Params2.identity(Hp.J)
    S = Solver2(Hp, prm, precision=64, max_batch=1)
    f = torch.tensor(p.f, dtype=torch.complex128, device="cuda")
    u = torch.zeros_like(f)
    uo = np.zeros_like(p.f)
    A = Ho.levels[0].A
    r0 = np.linalg.norm(p.f)
    for _ in range(6):
        S.vcycle(f, u)
        uo = O.vcycle2(Ho, to_oracle(prm), p.f, uo)
    ug = u.cpu().numpy()
    assert rel(ug, uo) < 1e-12
    assert np.linalg.norm(p.f - A @ ug) < 0.5 * r0
    S.close()


def test_two_feature_errors():
    p, Ho, Hp = problem("helmholtz33")
    S = Solver2(Hp, params(Hp.J, 1), precision=64, max_batch=2)
    f = torch.tensor(p.f, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        S.vcycle(f.to(torch.complex64), torch.zeros_like(f).to(torch.complex64))
    with pytest.raises(ValueError):
        S.vcycle(torch.zeros((Hp.sizes[0], 3), dtype=torch.complex128, device="cuda"),
                 torch.zeros((Hp.sizes[0], 3), dtype=torch.complex128, device="cuda"))
    bad = params(Hp.J, 1)
    bad.WB[0, 0, 0, 0] = np.inf
    with pytest.raises(MGError):
        S.set_params(bad)
    S.close()


def test_set_params_recaptures_the_cycle():
    """The cycle is replayed from a graph per (f, u, nrhs); new parameters
    must reach the next cycle on the same buffers."""
    p, Ho, Hp = problem("helmholtz33")
    a, b = params(Hp.J, 21), params(Hp.J, 22)
    S = Solver2(Hp, a, precision=64, max_batch=p.f.shape[1])
    f = torch.tensor(p.f, dtype=torch.complex128, device="cuda")
    u = torch.zeros_like(f)
    S.vcycle(f, u)
    u_in = u.cpu().numpy()
    S.set_params(b)
    S.vcycle(f, u)
    assert rel(u.cpu().numpy(), O.vcycle2(Ho, to_oracle(b), p.f, u_in)) < 1e-12
    S.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("precond", ["vcycle", "fmg"])
@pytest.mark.parametrize("which", ["classical", "random"])
def test_fgmres2_reaches_tolerance(prec, precond, which):
    """FGMRES on the real 2n form with the two-feature cycle or FMG as right
    preconditioner reaches 1e-8 (re-checked against the oracle's operator);
    in FP64 each right-hand side takes the oracle's iteration count to within
    one step (CGS2 here, MGS there)."""
    p = W.helmholtz_square(33, 3, k=2 * np.pi, batch=2, seed=1)
    Ho, Hp = O.build_hierarchy(p), Hierarchy2.from_problem(p)
    prm = Params2.identity(Hp.J) if which == "classical" else params(Hp.J, 4, 0.1)
    S = Solver2(Hp, prm, precision=prec, max_batch=2)
    f = torch.tensor(p.f, dtype=torch.complex128, device="cuda")
    u, info = S.solve_fgmres(f, tol=1e-8, precond=precond)
    assert info.status == 0
    A = Ho.levels[0].A
    ug = u.cpu().numpy()
    for b in range(2):
        assert np.linalg.norm(p.f[:, b] - A @ ug[:, b]) / np.linalg.norm(p.f[:, b]) < 1e-8
        if prec == 64:
            _, its, _ = O.fgmres2(Ho, to_oracle(prm), p.f[:, b], 1e-8, precond=precond)
            assert abs(int(info.iters[b]) - its) <= 1, (b, info.iters[b], its)
    S.close()


def test_fgmres2_zero_rhs_and_not_converged():
    p = W.helmholtz_square(33, 3, k=2 * np.pi, batch=2, seed=1)
    Hp = Hierarchy2.from_problem(p)
    S = Solver2(Hp, Params2.identity(Hp.J), precision=32, max_batch=2)
    f = np.array(p.f)
    f[:, 1] = 0.0
    u, info = S.solve_fgmres(torch.tensor(f, dtype=torch.complex128, device="cuda"), tol=1e-8)
    assert info.status == 0 and info.iters[1] == 0 and torch.all(u[:, 1] == 0)
    ft = torch.tensor(p.f, dtype=torch.complex128, device="cuda")
    u, info = S.solve_fgmres(ft, tol=1e-14, max_iter=3, restart=10)
    assert info.status == 1 and info.iters.max() == 3
    with pytest.raises(MGError):
        S.solve_fgmres(ft, restart=0)
    S.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 8, 16])
def test_tiles_and_pdl_are_bitwise_neutral(prec, nrhs):
    """Right-hand-side tiles (4 complex values per thread in FP32, 2 in FP64,
    the widest dividing nrhs), programmatic dependent launch and the
    single-block kernel for the small levels (option; threshold 2048, and
    every level of the 65^2 hierarchy from level 0 on) give bitwise the cycle,
    full multigrid and FGMRES of the one-thread-per-(row, rhs) plain grid
    launches."""
    p, Ho, Hp = problem("helmholtz65")
    prm = params(Hp.J, 19)
    dt = torch.complex128 if prec == 64 else torch.complex64
    r = np.random.default_rng(nrhs)
    fc = r.standard_normal((Hp.sizes[0], nrhs)) + 1j * r.standard_normal((Hp.sizes[0], nrhs))
    outs = []
    for tile, pdl, tail in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (1, 1, 2048),
                            (0, 1, 1 << 20)):
        S = Solver2(Hp, prm, precision=prec, max_batch=nrhs)
        S.set_option("multi_rhs", tile)
        S.set_option("pdl", pdl)
        S.set_option("tail_work", tail)
        f = torch.tensor(fc, dtype=dt, device="cuda")
        u = torch.zeros_like(f)
        for _ in range(3):
            S.vcycle(f, u)
        f64 = torch.tensor(fc, dtype=torch.complex128, device="cuda")
        ug, ig = S.solve_fgmres(f64, tol=1e-8, max_iter=200, restart=10, precond="fmg")
        outs.append((u.clone(), ug.clone(), ig.iters.copy()))
        S.close()
    assert torch.isfinite(torch.view_as_real(outs[0][0])).all()
    for u, ug, it in outs[1:]:
        assert torch.equal(u, outs[0][0])
        assert torch.equal(ug, outs[0][1])
        assert np.array_equal(it, outs[0][2])


def test_two_feature_option_errors():
    p, Ho, Hp = problem("helmholtz33")
    S = Solver2(Hp, params(Hp.J, 3), precision=32, max_batch=2)
    with pytest.raises(MGError):
        S.set_option("multi_rhs", 2)
    with pytest.raises(ValueError):
        S.set_option("halo_rows", 0)
    with pytest.raises(MGError):
        S.set_option("tail_work", -1)
    S.close()
