"""Hand-written adjoint of the unrolled V-cycle (mg_forward_record /
mg_vcycle_backward / mg_residual_loss) against the oracle.

FP64: parameter gradient vs the oracle's complex-step derivative (exact to
rounding) at 1e-10 relative (max-norm over the gradient), and vs central
finite differences of the GPU loss at 1e-5; input adjoints vs the linearity
identity <ubar, u_K(x + d) - u_K(x)> = <grad_x, d> at 1e-11.
FP32: the gradient's error against the oracle is stated (< 2e-3 relative).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2608_29082_b300 import Hierarchy, LMGParams, Solver
from paper_2608_29082_b300.training import (ParamMap, ResidualLoss, Trainer,
                                            UnrolledCycles)

pytestmark = pytest.mark.gpu
DEV = "cuda"


def rand_params(J, seed, spread=0.2):
    r = np.random.default_rng(seed)
    p = LMGParams.identity(J)
    m = J - 1
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, m))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, m))
    for w in (p.wB, p.wR, p.wP):
        w[:, 0] += spread * r.uniform(-1, 1, m)
        w[:, 1] += spread * r.uniform(-1, 1, m)
    return p


def to_oracle(p):
    return O.Params(p.theta.copy(), p.eta.copy(), p.wB.copy(), p.wR.copy(), p.wP.copy(),
                    p.nu_pre, p.nu_post)


CASES = {
    "checker33": lambda: W.checkerboard_square(33, 4, ncell=4, values=(1.0, 1e3), batch=3, seed=2),
    "lshape_r1": lambda: W.lshape_anisotropic(refinements=1, batch=2, seed=1),
}
_cache = {}


def problem(name):
    if name not in _cache:
        p = CASES[name]()
        _cache[name] = (p, O.build_hierarchy(p), Hierarchy.from_problem(p))
    return _cache[name]


def gpu_loss_grad(S, f, K, u0=None):
    f_t = torch.tensor(f, dtype=S.dtype, device=DEV)
    u = torch.zeros_like(f_t) if u0 is None else torch.tensor(u0, dtype=S.dtype, device=DEV)
    _, r0, _ = S.residual_loss(f_t, u)
    w = 1.0 / (f.shape[1] * r0)
    S.forward_record(f_t, u, K)
    loss, _, gu = S.residual_loss(f_t, u, w, grad=True)
    _, _, gp = S.backward(gu, K, want_inputs=False)
    return loss.item(), gp.cpu().numpy().ravel()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nu", [(2, 2), (1, 2)])
def test_param_gradient_fp64_vs_complex_step(name, nu):
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 5)
    prm.nu_pre, prm.nu_post = nu
    K = 2
    S = Solver(Hp, prm, precision=64, max_batch=p.batch)
    loss, g = gpu_loss_grad(S, p.f, K)
    lo, go = O.loss_gradient_complex_step(Ho, to_oracle(prm), p.f, K)
    assert abs(loss - lo) <= 1e-12 * lo
    assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max(), np.abs(g - go).max() / np.abs(go).max()
    S.close()


def test_param_gradient_fp64_vs_central_differences():
    p, Ho, Hp = problem("checker33")
    prm = rand_params(Hp.J, 7)
    K = 3
    S = Solver(Hp, prm, precision=64, max_batch=p.batch)
    _, g = gpu_loss_grad(S, p.f, K)
    x = prm.flat()
    fd = np.zeros_like(x)
    for k in range(x.size):
        h = 1e-6 * max(1.0, abs(x[k]))
        vals = []
        for sgn in (1, -1):
            y = x.copy()
            y[k] += sgn * h
            S.set_params(LMGParams.from_flat(y))
            vals.append(gpu_loss_grad(S, p.f, K)[0])
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-5 * np.abs(g).max()
    S.close()


def test_input_adjoints_fp64():
    """u_K is affine in (u_0, f): check grad_u0 and grad_f along random
    directions against the exact difference."""
    p, Ho, Hp = problem("checker33")
    prm = rand_params(Hp.J, 9)
    K = 3
    S = Solver(Hp, prm, precision=64, max_batch=p.batch)
    r = np.random.default_rng(0)
    n, B = p.f.shape
    f = torch.tensor(p.f, dtype=torch.float64, device=DEV)
    u0 = torch.tensor(r.standard_normal((n, B)), dtype=torch.float64, device=DEV)
    ubar = torch.tensor(r.standard_normal((n, B)), dtype=torch.float64, device=DEV)
    du = torch.tensor(r.standard_normal((n, B)), dtype=torch.float64, device=DEV)
    df = torch.tensor(r.standard_normal((n, B)), dtype=torch.float64, device=DEV)

    def run(ff, uu):
        u = uu.clone()
        S.forward_record(ff, u, K)
        return u

    base = run(f, u0)
    gin, gf, _ = S.backward(ubar, K)
    lhs_u = torch.sum(ubar * (run(f, u0 + du) - base)).item()
    lhs_f = torch.sum(ubar * (run(f + df, u0) - base)).item()
    rhs_u = torch.sum(gin * du).item()
    rhs_f = torch.sum(gf * df).item()
    assert abs(lhs_u - rhs_u) <= 1e-11 * max(abs(lhs_u), 1.0)
    assert abs(lhs_f - rhs_f) <= 1e-11 * max(abs(lhs_f), 1.0)
    S.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_multi_rhs_adjoint_matches_per_element_adjoint(prec, name):
    """With 8 right-hand sides the adjoint runs its multi-rhs kernels (a row
    and a tile of rhs per thread); with the option off, one thread per (row,
    rhs).  Input adjoints are the same bitwise; the parameter gradients sum
    the same terms in another order (FP64: 1e-12 relative, FP32: 1e-5)."""
    p, Ho, Hp = problem(name)
    prm = rand_params(Hp.J, 13)
    K = 3
    r = np.random.default_rng(4)
    n = Hp.sizes[0]
    dt = torch.float64 if prec == 64 else torch.float32
    f = torch.tensor(r.standard_normal((n, 8)), dtype=dt, device=DEV)
    u0 = torch.tensor(r.standard_normal((n, 8)), dtype=dt, device=DEV)
    ubar = torch.tensor(r.standard_normal((n, 8)), dtype=dt, device=DEV)
    out = []
    for mrhs in (1, 0):
        S = Solver(Hp, prm, precision=prec, max_batch=8)
        S.set_option("multi_rhs", mrhs)
        u = u0.clone()
        S.forward_record(f, u, K)
        gin, gf, gp = S.backward(ubar, K)
        out.append((u, gin, gf, gp.cpu().numpy().ravel()))
        S.close()
    (ua, ga, fa, pa), (ub, gb, fb, pb) = out
    assert torch.equal(ua, ub)
    assert torch.equal(ga, gb) and torch.equal(fa, fb)
    tol = 1e-12 if prec == 64 else 1e-5
    assert np.abs(pa - pb).max() <= tol * np.abs(pb).max()


def test_param_gradient_fp32_error_stated():
    p, Ho, Hp = problem("checker33")
    prm = rand_params(Hp.J, 11)
    K = 2
    S = Solver(Hp, prm, precision=32, max_batch=p.batch)
    _, g = gpu_loss_grad(S, p.f, K)
    _, go = O.loss_gradient_complex_step(Ho, to_oracle(prm), p.f, K)
    err = np.abs(g - go).max() / np.abs(go).max()
    assert err < 2e-3, err
    S.close()


def test_autograd_function_matches_direct_path():
    p, Ho, Hp = problem("checker33")
    prm = rand_params(Hp.J, 13)
    K = 2
    S = Solver(Hp, prm, precision=64, max_batch=p.batch)
    _, g_direct = gpu_loss_grad(S, p.f, K)
    theta = torch.tensor(prm.flat().reshape(-1, 8), dtype=torch.float64, requires_grad=True)
    f = torch.tensor(p.f, dtype=torch.float64, device=DEV)
    u0 = torch.zeros_like(f)
    _, r0, _ = S.residual_loss(f, u0)
    w = 1.0 / (p.batch * r0)
    uK = UnrolledCycles.apply(theta, f, u0, S, K)
    loss = ResidualLoss.apply(uK, f, w, S)
    loss.backward()
    assert np.abs(theta.grad.numpy().ravel() - g_direct).max() <= 1e-12 * np.abs(g_direct).max()
    S.close()


def test_backward_requires_matching_forward():
    p, Ho, Hp = problem("checker33")
    S = Solver(Hp, rand_params(Hp.J, 1), precision=64, max_batch=p.batch)
    f = torch.tensor(p.f, dtype=torch.float64, device=DEV)
    from paper_2608_29082_b300 import MGError
    with pytest.raises(MGError):
        S.backward(torch.zeros_like(f), 2)
    u = torch.zeros_like(f)
    S.forward_record(f, u, 2)
    S.set_params(rand_params(Hp.J, 2))
    with pytest.raises(MGError):
        S.backward(torch.zeros_like(f), 2)
    S.close()


def test_training_improves_the_cycle():
    """Rprop on the unrolled loss (Algorithm 3) lowers the 10-cycle residual
    reduction of a jump-coefficient problem, and the trained cycle needs fewer
    refinement iterations (re-checked by the oracle)."""
    p = W.checkerboard_square(65, 6, ncell=8, values=(1.0, 1e4), batch=8, seed=21)
    Hp = Hierarchy.from_problem(p)
    Ho = O.build_hierarchy(p)
    prm0 = LMGParams.identity(Hp.J)
    S = Solver(Hp, prm0, precision=32, max_batch=8)
    f = torch.tensor(p.f, dtype=torch.float32, device=DEV)
    tr = Trainer(S, ParamMap(Hp.J, shared=("wB1", "wB2", "wR1", "wR2", "wP1", "wP2")),
                 n_cycles=4)
    log = tr.train(f, prm0, max_epochs=60)
    assert log.best_loss < 0.5 * log.losses[0]
    test = np.random.default_rng(99).standard_normal((Hp.sizes[0], 1))
    S64 = Solver(Hp, prm0, precision=32, max_batch=1)
    _, i0 = S64.solve(torch.tensor(test, device=DEV), tol=1e-8, max_iter=400)
    S64.set_params(log.params)
    u1, i1 = S64.solve(torch.tensor(test, device=DEV), tol=1e-8, max_iter=400)
    assert i1.iters[0] < i0.iters[0]
    assert O.relres(Ho, test, u1.cpu().numpy())[0] < 1e-8
