"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares it with an
independent form (closed-form spectra, dense error-propagation matrices,
direct solves, complex-step derivatives vs finite differences, invariants).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle as O
import workloads as W
from workloads import fields, meshes


@pytest.fixture(scope="module")
def poisson33():
    p = W.poisson_square(33, 4, batch=3, seed=1)
    return p, O.build_hierarchy(p)


@pytest.fixture(scope="module")
def checker17():
    p = W.checkerboard_square(N=17, J=3, ncell=4, values=(1.0, 1e4), batch=2, seed=2)
    return p, O.build_hierarchy(p)


def random_params(J, seed, spread=0.3):
    r = np.random.default_rng(seed)
    p = O.Params.identity(J)
    m = J - 1
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, m))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, m))
    for w in (p.wB, p.wR, p.wP):
        w[:, 0] += spread * r.uniform(-1, 1, m)
        w[:, 1] += spread * r.uniform(-1, 1, m)
    return p


# ---------------------------------------------------------------- setup ----

def test_p1_poisson_is_five_point(poisson33):
    """P1 on right triangles gives the (4, -1) five-point stencil exactly."""
    p, H = poisson33
    A = H.levels[0].A.toarray()
    N = 31
    T = 2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    ref = np.kron(np.eye(N), T) + np.kron(T, np.eye(N))
    assert np.array_equal(A, ref)


@pytest.mark.parametrize("case", ["poisson", "checker"])
def test_galerkin_equals_rediscretisation(case):
    """Nested P1 with P = natural inclusion: P^T A P equals the stiffness
    matrix assembled directly on the coarse mesh (coefficient aligned with it)."""
    N = 33
    if case == "poisson":
        p = W.poisson_square(N, 3)
        kc = None
        Lc = p.mesh.levels[1]
    else:
        p = W.checkerboard_square(N, 3, ncell=4, values=(1.0, 1e4), seed=5)
        Lc = p.mesh.levels[1]
        kc = fields.checkerboard(Lc, 4, (1.0, 1e4), 5)
    H = O.build_hierarchy(p)
    Ac = fields.assemble_p1(Lc, k=kc)
    I = Lc.interior
    ref = Ac[I][:, I].toarray()
    got = H.levels[1].A.toarray()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_prolongation_column_sums(poisson33):
    """Each coarse vertex away from the boundary spreads to itself (1) and its
    six fine edge midpoints (1/2): column sums of P are 4."""
    _, H = poisson33
    P = H.levels[0].P
    cs = np.asarray(P.sum(axis=0)).ravel().reshape(15, 15)
    assert np.allclose(cs[1:-1, 1:-1], 4.0)
    assert (P.getnnz(axis=1) <= 2).all()


def test_degree_counts_full_stencil(poisson33):
    """Degree counts every algebraic neighbour including eliminated Dirichlet
    vertices: 4 everywhere for the five-point stencil."""
    _, H = poisson33
    for L in H.levels:
        assert np.all(1.0 / L.inv_deg == 4.0)


# ------------------------------------------------------------- smoother ----

def dense_smoother(L, theta, eta, wB):
    n = L.A.shape[0]
    I = np.eye(n)
    return O.smooth(L, np.zeros((n, n)), I, theta, eta, wB)  # f = 0: u -> S u


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_smoother_spectrum_closed_form(poisson33, seed):
    """Eq. (eigenvalue-S): sigma = 1 - eta theta (w1 + w2 lambda_hat) lambda with
    lambda = 1 - (cos p pi h + cos q pi h)/2 and lambda_hat = 1 - lambda for the
    five-point Laplacian, for arbitrary (w1, w2, theta, eta)."""
    _, H = poisson33
    r = np.random.default_rng(seed)
    theta, eta = r.uniform(0.3, 1.0), r.uniform(0.5, 1.5)
    wB = (r.uniform(0.5, 1.5), r.uniform(-0.8, 0.8))
    S = dense_smoother(H.levels[0], theta, eta, wB)
    h = 1.0 / 32
    pq = np.arange(1, 32)
    lam = 1 - (np.cos(pq[:, None] * np.pi * h) + np.cos(pq[None, :] * np.pi * h)) / 2
    lam_hat = 1 - lam
    sigma = 1 - eta * theta * (wB[0] + wB[1] * lam_hat) * lam
    ev = np.sort(np.linalg.eigvals(S).real)
    assert np.abs(ev - np.sort(sigma.ravel())).max() < 1e-12


def test_proposition_learnable_smoother_beats_optimal_jacobi(poisson33):
    """Proposition (Sec. 3.3): min over (w1, w2, eta, theta) of rho(S) is at
    most rho(S_{omega*}).  On the five-point Laplacian both minima have
    closed forms over the spectrum [a, b] of D_A^{-1} A, mu = (b+a)/(b-a):
    damped Jacobi gives 1/mu at omega* = 2/(a+b); the learnable factor
    1 - eta theta (w1 + w2 (1 - lambda)) lambda is a quadratic with value 1
    at 0, whose minimax on [a, b] is the shifted Chebyshev polynomial, value
    1/T_2(mu) = 1/(2 mu^2 - 1) (strictly smaller, the Remark's frequency-
    dependent damping).  The oracle's smoother at the parameters realising
    each has exactly these spectral radii."""
    _, H = poisson33
    L = H.levels[0]
    h = 1.0 / 32
    a, b = 1 - np.cos(np.pi * h), 1 + np.cos(np.pi * h)
    mu, sc = (b + a) / (b - a), 2.0 / (b - a)
    rho_j = np.abs(np.linalg.eigvals(dense_smoother(L, 2.0 / (a + b), 1.0, (1.0, 0.0)))).max()
    assert abs(rho_j - 1.0 / mu) < 1e-12
    t2 = 2 * mu * mu - 1
    w2 = 2 * sc * sc / t2
    w1 = 4 * mu * sc / t2 - w2
    rho_l = np.abs(np.linalg.eigvals(dense_smoother(L, 1.0, 1.0, (w1, w2)))).max()
    assert abs(rho_l - 1.0 / t2) < 1e-12
    assert rho_l < rho_j


def test_jacobi_recovery(poisson33):
    """Remark (recovery of classical methods): w1=1, w2=0, theta=omega, eta=1
    gives S = I - omega D_A^{-1} A with eigenvalues 1 - omega lambda."""
    _, H = poisson33
    L = H.levels[0]
    omega = 2.0 / 3.0
    S = dense_smoother(L, omega, 1.0, (1.0, 0.0))
    ref = np.eye(961) - omega * (L.A.toarray() / L.diag[:, None])
    assert np.abs(S - ref).max() < 1e-15


# ------------------------------------------------------ ChebConv smoother ----

def ring_level(n):
    import scipy.sparse as sp
    i = np.arange(n)
    G = sp.csr_matrix((np.ones(2 * n), (np.r_[i, i], np.r_[(i + 1) % n, (i - 1) % n])),
                      shape=(n, n))
    return O.Level(A=G, diag=np.ones(n), G=G, inv_deg=np.full(n, 0.5), P=None)


@pytest.mark.parametrize("K", [1, 2, 5])
def test_cheb_conv_ring_modes(K):
    """On a ring every Fourier mode is an eigenvector of the mean operator
    D_g^{-1} A_g with eigenvalue cos(theta), so Lhat = -D_g^{-1} A_g acts as
    cos(pi - theta) and T_k(Lhat) as cos(k (pi - theta)), because
    T_k(cos phi) = cos(k phi)."""
    n = 24
    L = ring_level(n)
    c = np.random.default_rng(K).uniform(-1, 1, K + 1)
    i = np.arange(n)
    for m in range(n // 2 + 1):
        th = 2 * np.pi * m / n
        for v in (np.cos(th * i), np.sin(th * i)):
            if np.abs(v).max() < 1e-9:
                continue
            got = O.cheb_conv(L, v[:, None], c)[:, 0]
            ref = sum(c[k] * np.cos(k * (np.pi - th)) for k in range(K + 1)) * v
            assert np.abs(got - ref).max() < 1e-12, (K, m)


def test_cheb_degree_one_is_sage(poisson33):
    """Degree 1: c_0 I + c_1 Lhat = c_0 I - c_1 D_g^{-1} A_g, the SAGEConv
    mean with w1 = c_0, w2 = -c_1 (the degree-1 polynomial of the Sec. 3.3
    remark)."""
    _, H = poisson33
    L = H.levels[0]
    x = np.random.default_rng(3).standard_normal((L.A.shape[0], 2))
    assert np.array_equal(O.cheb_conv(L, x, [0.8, 0.35]), O.conv(L, x, 0.8, -0.35))


@pytest.mark.parametrize("seed", [0, 1])
def test_cheb_smoother_spectrum_closed_form(poisson33, seed):
    """Degree-3 ChebConv smoother on the five-point Laplacian (Sec. 3.3
    remark: a degree-K polynomial smoother): with lambda = 1 - (cos p pi h +
    cos q pi h)/2 the eigenvalues of D_A^{-1} A and lambda_hat = 1 - lambda
    those of D_g^{-1} A_g, sigma = 1 - eta theta poly lambda where
    poly = sum_k c_k cos(k arccos(-lambda_hat))."""
    _, H = poisson33
    r = np.random.default_rng(10 + seed)
    theta, eta = r.uniform(0.3, 1.0), r.uniform(0.5, 1.5)
    c = r.uniform(-0.5, 0.5, 4)
    c[0] += 1.0
    L = H.levels[0]
    n = L.A.shape[0]
    S = O.smooth(L, np.zeros((n, n)), np.eye(n), theta, eta, None, c)
    h = 1.0 / 32
    pq = np.arange(1, 32)
    lam = 1 - (np.cos(pq[:, None] * np.pi * h) + np.cos(pq[None, :] * np.pi * h)) / 2
    lam_hat = 1 - lam
    poly = sum(c[k] * np.cos(k * np.arccos(-lam_hat)) for k in range(4))
    sigma = 1 - eta * theta * poly * lam
    ev = np.sort(np.linalg.eigvals(S).real)
    assert np.abs(ev - np.sort(sigma.ravel())).max() < 1e-12


def test_cheb_identity_polynomial_is_jacobi_cycle(poisson33):
    """Coefficients (1, 0, 0): Phi_B = T_0 = I, so the cycle is the SAGEConv
    cycle with W1 = 1, W2 = 0 (damped Jacobi smoothing, Sec. 3 remark)."""
    p, H = poisson33
    th = random_params(H.J, 5)
    th.wB[:, 0], th.wB[:, 1] = 1.0, 0.0
    tc = th.copy()
    tc.cheb = np.tile([1.0, 0.0, 0.0], (H.J - 1, 1))
    u0 = np.zeros_like(p.f)
    assert np.array_equal(O.vcycle(H, th, p.f, u0), O.vcycle(H, tc, p.f, u0))


# ---------------------------------------------------------------- cycle ----

def dense_error_propagation(H, p):
    """E_l = S_l^nu_post (I - C_l) S_l^nu_pre with
    C_l = Phi_P P (I - E_{l+1}) A_{l+1}^{-1} P^T Phi_R A_l, E_J = 0."""
    J = H.J
    E = np.zeros((H.levels[-1].A.shape[0],) * 2)
    for lev in range(J - 2, -1, -1):
        L, Lc = H.levels[lev], H.levels[lev + 1]
        A = L.A.toarray()
        n = A.shape[0]
        Ag = L.inv_deg[:, None] * L.G.toarray()
        phi = lambda w: w[0] * np.eye(n) + w[1] * Ag  # noqa: E731
        S = np.eye(n) - p.eta[lev] * p.theta[lev] * phi(p.wB[lev]) @ (A / L.diag[:, None])
        P = L.P.toarray()
        Ac = Lc.A.toarray()
        C = phi(p.wP[lev]) @ P @ (np.eye(Ac.shape[0]) - E) @ np.linalg.solve(Ac, P.T @ phi(p.wR[lev]) @ A)
        E = np.linalg.matrix_power(S, p.nu_post) @ (np.eye(n) - C) @ np.linalg.matrix_power(S, p.nu_pre)
    return E


def dense_fmg(H, p):
    """Full multigrid as dense matrices: f_l = P^T Phi_R f_{l-1}; u_{J-1} =
    A_{J-1}^{-1} f_{J-1}; on level l one V-cycle from u0 = Phi_P P u_{l+1}, i.e.
    u_l = E_l u0 + (I - E_l) A_l^{-1} f_l with E_l the error propagation of
    the V-cycle started on level l (E_{J-1} = 0).  Returns the matrix f -> u."""
    J = H.J
    mats = []
    E = np.zeros((H.levels[-1].A.shape[0],) * 2)
    Es = [None] * J
    Es[J - 1] = E
    for lev in range(J - 2, -1, -1):  # E_l, the same recursion as dense_error_propagation
        L, Lc = H.levels[lev], H.levels[lev + 1]
        A = L.A.toarray()
        n = A.shape[0]
        Ag = L.inv_deg[:, None] * L.G.toarray()
        phi = lambda w: w[0] * np.eye(n) + w[1] * Ag  # noqa: E731
        S = np.eye(n) - p.eta[lev] * p.theta[lev] * phi(p.wB[lev]) @ (A / L.diag[:, None])
        P = L.P.toarray()
        Ac = Lc.A.toarray()
        C = phi(p.wP[lev]) @ P @ (np.eye(Ac.shape[0]) - Es[lev + 1]) @ np.linalg.solve(
            Ac, P.T @ phi(p.wR[lev]) @ A)
        Es[lev] = np.linalg.matrix_power(S, p.nu_post) @ (np.eye(n) - C) @ \
            np.linalg.matrix_power(S, p.nu_pre)
    # restriction of f to every level
    Rs = [np.eye(H.levels[0].A.shape[0])]
    for lev in range(J - 1):
        L = H.levels[lev]
        n = L.A.shape[0]
        phiR = p.wR[lev][0] * np.eye(n) + p.wR[lev][1] * (L.inv_deg[:, None] * L.G.toarray())
        Rs.append(L.P.toarray().T @ phiR @ Rs[lev])
    M = np.linalg.solve(H.levels[J - 1].A.toarray(), Rs[J - 1])
    for lev in range(J - 2, -1, -1):
        L = H.levels[lev]
        A = L.A.toarray()
        n = A.shape[0]
        phiP = p.wP[lev][0] * np.eye(n) + p.wP[lev][1] * (L.inv_deg[:, None] * L.G.toarray())
        U0 = phiP @ L.P.toarray() @ M
        M = Es[lev] @ U0 + (np.eye(n) - Es[lev]) @ np.linalg.solve(A, Rs[lev])
    return M


@pytest.mark.parametrize("which", ["identity", "random"])
def test_fmg_matches_dense_nested_iteration(poisson33, checker17, which):
    """Full multigrid (the Sec. 4.2 preconditioner) against its dense construction
    from the per-level error propagation matrices, on Poisson and on a jump
    coefficient; and it is linear in f."""
    for case, seed in ((poisson33, 5), (checker17, 6)):
        prob, H = case
        th = O.Params.identity(H.J) if which == "identity" else random_params(H.J, seed)
        n = H.levels[0].A.shape[0]
        f = np.random.default_rng(seed).standard_normal((n, 2))
        got = O.fmg(H, th, f)
        ref = dense_fmg(H, th) @ f
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        g2 = O.fmg(H, th, 2.0 * f[:, :1] - 3.0 * f[:, 1:])
        assert np.abs(g2 - (2.0 * got[:, :1] - 3.0 * got[:, 1:])).max() <= 1e-12 * np.abs(got).max()


@pytest.mark.parametrize("which", ["identity", "random"])
def test_vcycle_matches_dense_error_propagation(poisson33, which):
    p, H = poisson33
    th = O.Params.identity(H.J) if which == "identity" else random_params(H.J, 7)
    E = dense_error_propagation(H, th)
    A = H.levels[0].A.toarray()
    r = np.random.default_rng(3)
    f = r.standard_normal((961, 2))
    u0 = r.standard_normal((961, 2))
    ustar = np.linalg.solve(A, f)
    got = O.vcycle(H, th, f, u0)
    ref = ustar + E @ (u0 - ustar)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_vcycle_dense_on_jump_coefficients(checker17):
    p, H = checker17
    th = random_params(H.J, 11)
    E = dense_error_propagation(H, th)
    A = H.levels[0].A.toarray()
    f = p.f
    u0 = np.random.default_rng(0).standard_normal(f.shape)
    ustar = np.linalg.solve(A, f)
    got = O.vcycle(H, th, f, u0)
    ref = ustar + E @ (u0 - ustar)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_jacobi_equivalent_reproduces_classical_factor(poisson33):
    """With the identity initialisation the learnable cycle is the classical
    damped-Jacobi V-cycle (Sec. 3.4): its observed asymptotic factor equals the
    spectral radius of Algorithm 1's error propagation built with B = omega D^{-1}
    and no convolutions."""
    _, H = poisson33
    J = H.J
    omega = 2.0 / 3.0
    E = np.zeros((H.levels[-1].A.shape[0],) * 2)
    for lev in range(J - 2, -1, -1):
        L, Lc = H.levels[lev], H.levels[lev + 1]
        A = L.A.toarray()
        n = A.shape[0]
        S = np.eye(n) - omega * A / np.diag(A)[:, None]
        P = L.P.toarray()
        Ac = P.T @ A @ P
        CGC = np.eye(n) - P @ (np.eye(Ac.shape[0]) - E) @ np.linalg.solve(Ac, P.T @ A)
        E = S @ S @ CGC @ S @ S
    rho = np.abs(np.linalg.eigvals(E)).max()
    th = O.Params.identity(J)
    n = E.shape[0]
    E_orc = O.vcycle(H, th, np.zeros((n, n)), np.eye(n))  # f = 0: error -> E error
    assert np.abs(E_orc - E).max() < 1e-13
    rho_orc = np.abs(np.linalg.eigvals(E_orc)).max()
    assert abs(rho_orc - rho) < 1e-10
    assert rho < 0.35


def test_converges_to_direct_solve(poisson33):
    p, H = poisson33
    res = O.solve_vcycles(H, O.Params.identity(H.J), p.f, 1e-10)
    assert (res.relres < 1e-10).all()
    ref = spla.spsolve(H.levels[0].A.tocsc(), p.f)
    assert np.abs(res.u - ref).max() <= 1e-9 * np.abs(ref).max()


def test_refinement_converges(checker17):
    p, H = checker17
    res = O.solve_refinement(H, random_params(H.J, 3, 0.1), p.f, 1e-10)
    assert (res.relres < 1e-10).all()
    ref = np.linalg.solve(H.levels[0].A.toarray(), p.f)
    assert np.abs(res.u - ref).max() <= 1e-8 * np.abs(ref).max()


# ----------------------------------------------------------- invariants ----

def test_linearity(poisson33):
    _, H = poisson33
    th = random_params(H.J, 5)
    r = np.random.default_rng(4)
    f1, f2, u1, u2 = (r.standard_normal((961, 1)) for _ in range(4))
    a, b = 0.7, -1.3
    lhs = O.vcycle(H, th, a * f1 + b * f2, a * u1 + b * u2)
    rhs = a * O.vcycle(H, th, f1, u1) + b * O.vcycle(H, th, f2, u2)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_identity_cycle_is_symmetric(poisson33):
    """R = P^T, symmetric smoother, nu_pre = nu_post: M = (I - E) A^{-1} is SPD."""
    _, H = poisson33
    th = O.Params.identity(H.J)
    n = 961
    M = O.vcycle(H, th, np.eye(n), np.zeros((n, n)))  # columns M e_k
    assert np.abs(M - M.T).max() < 1e-13 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_permutation_equivariance():
    """Relabelling the finest vertices relabels the result (mean aggregation is
    permutation invariant)."""
    p = W.checkerboard_square(N=17, J=3, ncell=4, values=(1.0, 1e4), batch=1, seed=9)
    H = O.build_hierarchy(p)
    th = random_params(H.J, 13)
    L0 = p.mesh.levels[0]
    perm = np.random.default_rng(0).permutation(L0.nv)   # new -> old
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    L0p = meshes.MeshLevel(L0.xy[perm], inv[L0.tri], L0.boundary[perm], L0.parent[perm])
    Hm = meshes.MeshHierarchy([L0p] + p.mesh.levels[1:])
    Ap = p.A_full[perm][:, perm].tocsr()
    # interior DOF order of the permuted mesh, expressed in old interior indices
    old_int = {v: k for k, v in enumerate(L0.interior)}
    dof_perm = np.array([old_int[perm[v]] for v in L0p.interior])
    pp = W.Problem("perm", Hm, Ap, p.f[dof_perm], {})
    Hp = O.build_hierarchy(pp)
    u0 = np.random.default_rng(1).standard_normal(p.f.shape)
    got = O.vcycle(Hp, th, pp.f, u0[dof_perm])
    ref = O.vcycle(H, th, p.f, u0)[dof_perm]
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


# ------------------------------------------------------------- gradient ----

def test_unrolled_loss_dense(poisson33):
    """r_K = A E^K A^{-1} f from u_0 = 0, so the loss has a dense closed form."""
    p, H = poisson33
    th = random_params(H.J, 21, 0.2)
    E = dense_error_propagation(H, th)
    A = H.levels[0].A.toarray()
    f = p.f
    rK = A @ np.linalg.matrix_power(E, 3) @ np.linalg.solve(A, f)
    ref = ((rK * rK).sum(0) / (f * f).sum(0)).mean()
    got = O.unrolled_loss(H, th, f, 3)
    assert abs(got - ref) < 1e-11 * ref


def test_complex_step_gradient_matches_finite_differences(checker17):
    p, H = checker17
    th = random_params(H.J, 17, 0.2)
    loss, g_cs = O.loss_gradient_complex_step(H, th, p.f, 2)
    g_fd = O.loss_gradient_fd(H, th, p.f, 2)
    scale = np.abs(g_cs).max()
    assert np.abs(g_cs - g_fd).max() < 1e-6 * scale
    assert loss > 0


def test_shared_weight_gradient_is_sum_over_levels(checker17):
    """Sharing one SAGEConv across levels: the derivative along the shared
    direction (all levels perturbed at once) equals the sum of the per-level
    derivatives."""
    p, H = checker17
    th = random_params(H.J, 19, 0.2)
    _, g = O.loss_gradient_complex_step(H, th, p.f, 2)
    g = g.reshape(H.J - 1, 8)
    x = th.flat().astype(np.complex128).reshape(H.J - 1, 8)
    x[:, 5] += 1e-30j  # wR2 at every level
    lc = O.unrolled_loss(H, O.Params.from_flat(x.ravel()), p.f.astype(np.complex128), 2)
    assert abs(np.imag(lc) / 1e-30 - g[:, 5].sum()) < 1e-12 * max(1.0, abs(g[:, 5]).sum())


def test_fgmres_reduces_to_gmres_and_exact_preconditioner(poisson33):
    """Without preconditioning the oracle's FGMRES is GMRES: its residual
    estimates equal scipy's GMRES residual history (restart 20); with the
    exact inverse as preconditioner it converges in one step."""
    p, H = poisson33
    A = H.levels[0].A.tocsc()
    f = p.f[:, 0]
    u, its, hist = O.fgmres(A, f, lambda v: v, 1e-8, restart=20, max_iter=60)
    ref = []
    spla.gmres(A, f, rtol=1e-8, restart=20, maxiter=3, callback=lambda x: ref.append(x),
               callback_type="pr_norm")
    ref = np.array(ref) * np.linalg.norm(f)  # scipy reports ||r|| / ||f||
    k = min(len(ref), len(hist), 40)
    assert k >= 20
    assert np.abs(hist[:k] - ref[:k]).max() <= 1e-10 * np.linalg.norm(f)
    # at the end of a restart cycle the estimate is the true residual
    assert abs(np.linalg.norm(f - A @ u) - hist[-1]) <= 1e-10 * np.linalg.norm(f)
    lu = spla.splu(A)
    u1, its1, _ = O.fgmres(A, f, lu.solve, 1e-10, restart=5, max_iter=10)
    assert its1 == 1 and np.linalg.norm(f - A @ u1) < 1e-10 * np.linalg.norm(f)


def test_fgmres_with_fmg_preconditioner(checker17):
    """FGMRES with the learnable FMG (random Theta, a nonsymmetric
    preconditioner) converges to the tolerance."""
    p, H = checker17
    th = random_params(H.J, 9)
    A = H.levels[0].A
    f = p.f[:, 0]
    u, its, hist = O.fgmres(A, f, lambda v: O.fmg(H, th, v[:, None])[:, 0], 1e-10, restart=10)
    assert np.linalg.norm(f - A @ u) < 1e-9 * np.linalg.norm(f)
    assert its < 60


def _cg_iterates(A, f, M=None, k=15):
    """scipy's (preconditioned) conjugate gradients from zero: the first k
    iterates, recorded by its callback."""
    xs = []
    spla.cg(A, f, rtol=1e-300, atol=0.0, maxiter=k, M=M, callback=lambda x: xs.append(x.copy()))
    return xs


def test_fcg_identity_preconditioner_is_cg(poisson33):
    """FCG(1) with the identity as preconditioner is the conjugate gradient
    method: its iterates equal scipy's CG iterates."""
    p, H = poisson33
    A = H.levels[0].A
    f = p.f[:, 0]
    ref = _cg_iterates(A, f, k=15)
    _, its, hist, us = O.fcg(A, f, lambda v: v.copy(), 1e-300, max_iter=15)
    assert its == 15 and len(ref) == 15
    for k in range(15):
        assert np.linalg.norm(us[k] - ref[k]) <= 1e-10 * np.linalg.norm(ref[k]), k
        # the recurrence residual is the true residual (exact arithmetic)
        assert abs(hist[k] - np.linalg.norm(f - A @ us[k])) <= 1e-10 * np.linalg.norm(f), k


def test_fcg_fixed_spd_preconditioner_is_pcg(checker17):
    """With a fixed SPD preconditioner (symmetric Gauss-Seidel on the
    jump-coefficient operator) FCG(1) is preconditioned CG: same iterates as
    scipy's PCG with the same operator."""
    p, H = checker17
    A = H.levels[0].A.tocsr()
    Ad = A.toarray()
    Lo = np.tril(Ad)
    Dg = np.diag(Ad)

    def sgs(v):
        return sla.solve_triangular(Lo.T, Dg * sla.solve_triangular(Lo, v, lower=True),
                                    lower=False)
    f = p.f[:, 1]
    M = spla.LinearOperator(A.shape, matvec=sgs)
    ref = _cg_iterates(A, f, M=M, k=8)
    _, its, _, us = O.fcg(A, f, sgs, 1e-300, max_iter=8)
    assert its == 8 and len(ref) == 8
    for k in range(8):
        assert np.linalg.norm(us[k] - ref[k]) <= 1e-10 * np.linalg.norm(ref[k]), k


def test_fcg_exact_preconditioner_converges_in_one_step(checker17):
    p, H = checker17
    A = H.levels[0].A.tocsc()
    f = p.f[:, 0]
    u, its, hist, _ = O.fcg(A, f, spla.splu(A).solve, 1e-12)
    assert its == 1 and np.linalg.norm(f - A @ u) < 1e-12 * np.linalg.norm(f)


def test_fcg_variable_preconditioner_orthogonality(checker17):
    """With a variable, nonsymmetric preconditioner (the learnable cycle with
    random Theta) FCG(1) still makes each new direction d_i = (u_{i+1} -
    u_i)/alpha_i A-orthogonal to the previous one and each new residual
    orthogonal to the last direction: the two properties that fix beta and
    alpha.  It converges to the tolerance."""
    p, H = checker17
    th = random_params(H.J, 31, 0.1)
    A = H.levels[0].A
    f = p.f[:, 0]
    M = lambda v: O.vcycle(H, th, v[:, None], np.zeros((v.size, 1)))[:, 0]  # noqa: E731
    u, its, hist, us = O.fcg(A, f, M, 1e-10, max_iter=200)
    assert np.linalg.norm(f - A @ u) < 1e-9 * np.linalg.norm(f)
    us = [np.zeros_like(f)] + us
    anorm = lambda x: np.sqrt(x @ (A @ x))  # noqa: E731
    for i in range(1, min(len(us) - 1, 12)):
        d_prev, d = us[i] - us[i - 1], us[i + 1] - us[i]
        assert abs(d @ (A @ d_prev)) <= 1e-10 * anorm(d) * anorm(d_prev), i
        r_next = f - A @ us[i + 1]
        assert abs(d @ r_next) <= 1e-10 * np.linalg.norm(d) * np.linalg.norm(f), i


# ------------------------------------------ two features per node (d = 2) ----

@pytest.fixture(scope="module", params=[2, 3])
def helmholtz17(request):
    p = W.helmholtz_square(17, request.param, k=2 * np.pi, batch=2, seed=3)
    return p, O.build_hierarchy(p)


def random_params2(J, seed, spread=0.3):
    r = np.random.default_rng(seed)
    p = O.Params2.identity(J)
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, J - 1))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, J - 1))
    for Wt in (p.WB, p.WR, p.WP):
        Wt += spread * r.uniform(-1, 1, Wt.shape)
    return p


def test_helmholtz_operator(helmholtz17):
    """K - k^2 M - i k B is complex symmetric; its imaginary part lives on the
    boundary (the impedance term) and integrates to -k times the perimeter;
    coarse operators are the Galerkin products P^T A P (Sec. 2.2)."""
    p, H = helmholtz17
    A = H.levels[0].A
    assert abs(A - A.T).max() == 0
    k = p.info["wave_number"]
    assert abs(A.imag.sum() + k * 4.0) < 1e-12
    for lev in range(H.J - 1):
        L = H.levels[lev]
        ref = (L.P.T @ L.A @ L.P).toarray()
        assert np.abs(H.levels[lev + 1].A.toarray() - ref).max() < 1e-12 * np.abs(ref).max()


def test_conv2_complex_weights_are_complex_products(helmholtz17):
    """W = [[a, -b], [b, a]] acts on (Re, Im) as multiplication by a + ib, so
    W_1, W_2 of that form give the scalar SAGEConv with complex weights."""
    _, H = helmholtz17
    L = H.levels[0]
    n = L.A.shape[0]
    r = np.random.default_rng(1)
    x = r.standard_normal((n, 2)) + 1j * r.standard_normal((n, 2))
    a, b, c, d = 0.7, -0.4, 0.3, 0.9
    Wt = np.array([[[a, -b], [b, a]], [[c, -d], [d, c]]])
    assert np.abs(O.conv2(L, x, Wt) - O.conv(L, x, a + 1j * b, c + 1j * d)).max() < 1e-14


def test_conv2_orientation(helmholtz17):
    """W_1 = [[0, 1], [0, 0]], W_2 = 0 maps the feature vector (Re, Im) to
    (Im, 0): W acts on feature columns, not transposed."""
    _, H = helmholtz17
    L = H.levels[0]
    n = L.A.shape[0]
    r = np.random.default_rng(2)
    x = r.standard_normal((n, 3)) + 1j * r.standard_normal((n, 3))
    Wt = np.zeros((2, 2, 2))
    Wt[0] = [[0.0, 1.0], [0.0, 0.0]]
    assert np.array_equal(O.conv2(L, x, Wt), x.imag + 0j)


def real_form(Z):
    """Complex n x m -> the real 2n x 2m map on [Re; Im]."""
    return np.block([[Z.real, -Z.imag], [Z.imag, Z.real]])


def conv2_matrix(L, Wt):
    """C(W) = W_1 (x) I + W_2 (x) D_g^{-1} A_g on [Re; Im] (features outer)."""
    n = L.A.shape[0]
    return np.kron(Wt[0], np.eye(n)) + np.kron(Wt[1], L.inv_deg[:, None] * L.G.toarray())


def dense_error2(H, p, lev=0):
    """E_l = S^nu_post (I - C_P P (I - E_{l+1}) A_{l+1}^{-1} P^T C_R A_l)
    S^nu_pre in the real 2n form, E_J = 0, S = I - eta theta C_B D_A^{-1} A."""
    L = H.levels[lev]
    n2 = 2 * L.A.shape[0]
    A = real_form(L.A.toarray())
    S = np.eye(n2) - p.eta[lev] * p.theta[lev] * conv2_matrix(L, p.WB[lev]) @ \
        real_form(np.diag(1.0 / L.diag)) @ A
    P = np.kron(np.eye(2), L.P.toarray())
    Ac = real_form(H.levels[lev + 1].A.toarray())
    inner = np.eye(Ac.shape[0]) if lev + 1 == H.J - 1 else \
        np.eye(Ac.shape[0]) - dense_error2(H, p, lev + 1)
    cgc = np.eye(n2) - conv2_matrix(L, p.WP[lev]) @ P @ inner @ np.linalg.solve(
        Ac, P.T @ conv2_matrix(L, p.WR[lev]) @ A)
    return (np.linalg.matrix_power(S, p.nu_post) @ cgc @ np.linalg.matrix_power(S, p.nu_pre))


@pytest.mark.parametrize("seed", [0, 1])
def test_vcycle2_dense_error_propagation(helmholtz17, seed):
    """The two-feature cycle on the complex Helmholtz system against its error
    propagation built densely in the real 2n form, applied to every real
    basis direction (u = e_k and u = i e_k, f = 0)."""
    _, H = helmholtz17
    th = random_params2(H.J, seed)
    th.nu_pre, th.nu_post = 1, 2
    n = H.levels[0].A.shape[0]
    U = np.concatenate([np.eye(n), 1j * np.eye(n)], axis=1)
    out = O.vcycle2(H, th, np.zeros_like(U), U)
    Eo = np.concatenate([out.real, out.imag], axis=0)
    E = dense_error2(H, th)
    assert np.abs(E - Eo).max() < 1e-10 * max(1.0, np.abs(E).max())


@pytest.mark.parametrize("precond", ["vcycle", "fmg"])
@pytest.mark.parametrize("which", ["classical", "random"])
def test_fgmres2_reaches_the_direct_solution(precond, which):
    """FGMRES on the real 2n form with the two-feature cycle or FMG as the
    right preconditioner converges to scipy's direct complex solve."""
    import scipy.sparse.linalg as spla_
    p = W.helmholtz_square(33, 3, k=2 * np.pi, batch=2, seed=1)
    H = O.build_hierarchy(p)
    th = O.Params2.identity(H.J) if which == "classical" else random_params2(H.J, 4, 0.1)
    A = H.levels[0].A.tocsc()
    for b in range(2):
        ex = spla_.spsolve(A, p.f[:, b])
        u, its, hist = O.fgmres2(H, th, p.f[:, b], 1e-10, precond=precond)
        assert hist[-1] < 1e-10 * np.linalg.norm(p.f[:, b]) and its < 60
        assert np.linalg.norm(u - ex) / np.linalg.norm(ex) < 1e-8


def dense_fmg2(H, p, lev=0):
    """FMG map f -> u in the real 2n form: f_{l+1} = P^T C_R f_l, u_J =
    A_J^{-1} f_J, and on level l one cycle from u_0 = C_P P u_{l+1}; a
    consistent cycle is affine, u = E_l (u_0 - u*) + u*, u* = A_l^{-1} f_l."""
    L = H.levels[lev]
    A = real_form(L.A.toarray())
    Ainv = np.linalg.inv(A)
    if lev == H.J - 1:
        return Ainv
    P = np.kron(np.eye(2), L.P.toarray())
    R = P.T @ conv2_matrix(L, p.WR[lev])
    U0 = conv2_matrix(L, p.WP[lev]) @ P @ dense_fmg2(H, p, lev + 1) @ R
    E = dense_error2(H, p, lev)
    return E @ (U0 - Ainv) + Ainv


@pytest.mark.parametrize("seed", [0, 1])
def test_fmg2_dense_nested_iteration(helmholtz17, seed):
    _, H = helmholtz17
    th = random_params2(H.J, 30 + seed)
    n = H.levels[0].A.shape[0]
    F = np.concatenate([np.eye(n), 1j * np.eye(n)], axis=1)
    out = O.fmg2(H, th, F)
    Mo = np.concatenate([out.real, out.imag], axis=0)
    M = dense_fmg2(H, th)
    assert np.abs(M - Mo).max() < 1e-10 * max(1.0, np.abs(M).max())


def test_cheb_coefficient_gradient(checker17):
    """Gradients of the unrolled loss (Algorithm 3) in the ChebConv
    smoother's coefficients: complex step equals central differences; with
    the ChebConv smoother on, the unused SAGEConv smoother weights W_B have
    exactly zero gradient and the other parameters' gradients still agree."""
    p, H = checker17
    th = random_params(H.J, 8, 0.2)
    th.cheb = np.tile([1.0, 0.15, -0.05], (H.J - 1, 1))
    gc = O.cheb_gradient_complex_step(H, th, p.f, 2)
    gf = O.cheb_gradient_fd(H, th, p.f, 2)
    assert np.abs(gc - gf).max() < 1e-5 * np.abs(gc).max()
    loss, g = O.loss_gradient_complex_step(H, th, p.f, 2)
    assert loss == O.unrolled_loss(H, th, p.f, 2)
    g = g.reshape(-1, 8)
    assert np.all(g[:, 2:4] == 0.0)
    gfd = O.loss_gradient_fd(H, th, p.f, 2).reshape(-1, 8)
    assert np.abs(g - gfd).max() < 1e-5 * np.abs(g).max()
