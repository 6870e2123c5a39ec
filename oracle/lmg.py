"""Oracle: plain, slow FP64 CPU implementation of the learnable multigrid.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, the package's smoke check and the benchmark's CPU-baseline leg do.
It shares no code with the CUDA path: it builds its own prolongation, Galerkin
coarse operators, graphs and coarsest-level factorisation from the inputs
produced by `workloads`, with scipy sparse products as the only primitives.

Every function follows the paper's definitions in the paper's order:

  graph of A (Sec. 2.1)        E = {(i,j): A_ij != 0, i != j}
  prolongation (Sec. 2.2)      P_l = natural inclusion of the coarse P1 space
  restriction (Sec. 2.2)       R_l = P_l^T
  Galerkin coarsening (Sec. 2.2)  A_{l+1} = R_l A_l P_l
  SAGEConv, mean (Sec. 3.2)    Phi(x)_i = w1 x_i + w2 mean_{j in N(i)} x_j
                               (matrix form, Eq. graph-conv-matrix:
                                Phi = w1 I + w2 D_g^{-1} A_g)
  learnable smoother (Sec. 3)  delta = theta B (f - A u),  B = D_A^{-1};
                               u <- u + eta Phi_B(delta)
  ChebConv smoother (Sec. 3.3, remark on polynomial smoothers)
                               Phi_B(delta) = sum_k c_k T_k(Lhat) delta,
                               Lhat = D_g^{-1} L_g - I = -D_g^{-1} A_g
  learnable transfers (Sec. 3) r_c = R Phi_R(r);  e = Phi_P(P e_c)
  learnable V-cycle            Algorithm 2
  training loss                mean_b ||r_K||^2 / ||r_0||^2 after K cycles

Readings where the paper is silent or ambiguous (kept identical in the CUDA
path and listed with reasons in the design notes):
  * the convolution graph is the algebraic graph of each level's operator,
    after dropping |A_ij| <= 1e-12 max(|A_ii|, |A_jj|) (exact zeros of P1 on
    right triangles, and round-off from Galerkin products);
  * deg_i counts the neighbours of i in that graph before the Dirichlet rows
    and columns are removed, so the mean divides by the full stencil count
    while the removed boundary values enter as zero;
  * the convolutions carry no bias, so the cycle is linear in (f, u);
  * the coarsest level is solved exactly by a dense Cholesky factorisation;
  * ChebConv uses the random-walk normalised Laplacian D_g^{-1} L_g (the
    mean aggregation of the SAGEConv smoother) scaled by lambda_max = 2, and
    "order K" is the polynomial degree K (coefficients c_0..c_K), so degree 1
    is the SAGEConv smoother with w1 = c_0, w2 = -c_1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

DROP_TOL = 1e-12


# ---------------------------------------------------------------- setup ----

def prolongation_full(parent: np.ndarray, nv_coarse: int) -> sp.csr_matrix:
    """Natural inclusion of the coarse P1 space in the fine one (Sec. 2.2): a
    fine vertex on a coarse vertex takes its value, a fine vertex at the
    midpoint of a coarse edge takes the mean of the edge's two end values."""
    rows, cols, vals = [], [], []
    for i, (a, b) in enumerate(parent):
        if b < 0:
            rows.append(i); cols.append(a); vals.append(1.0)
        else:
            rows += [i, i]; cols += [a, b]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(parent.shape[0], nv_coarse))


def drop_small(A: sp.csr_matrix) -> sp.csr_matrix:
    """Remove off-diagonal entries that are zero up to round-off."""
    C = A.tocoo()
    d = np.abs(A.diagonal())
    off = C.row != C.col
    small = np.abs(C.data) <= DROP_TOL * np.maximum(d[C.row], d[C.col])
    keep = ~(off & small)
    return sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)


@dataclass
class Level:
    A: sp.csr_matrix            # operator on interior DOFs
    diag: np.ndarray            # D_A
    G: sp.csr_matrix            # 0/1 adjacency of the algebraic graph (interior)
    inv_deg: np.ndarray         # 1/deg_i, deg over the graph before elimination
    P: sp.csr_matrix | None     # interior fine x interior coarse


@dataclass
class Hierarchy:
    levels: list[Level]
    chol: tuple | None          # cho_factor of A_J (dense), real SPD operators
    lu: tuple | None = None     # lu_factor of A_J, complex (Helmholtz) operators

    @property
    def J(self) -> int:
        return len(self.levels)


def build_hierarchy(problem) -> Hierarchy:
    """Levels 1..J of Sec. 2.2 from the mesh hierarchy and the finest stiffness
    matrix over all vertices; Dirichlet rows/columns are removed per level."""
    mesh = problem.mesh
    A_full = drop_small(problem.A_full.tocsr())
    levels = []
    for lev, ML in enumerate(mesh.levels):
        I = ML.interior
        pattern = sp.csr_matrix((np.ones(A_full.nnz), A_full.indices.copy(),
                                 A_full.indptr.copy()), shape=A_full.shape)
        pattern.setdiag(0)
        pattern.eliminate_zeros()
        deg = np.asarray(pattern.sum(axis=1)).ravel()[I]
        A = A_full[I][:, I].tocsr()
        G = pattern[I][:, I].tocsr()
        P = None
        if lev < mesh.J - 1:
            nvc = mesh.levels[lev + 1].nv
            P_full = prolongation_full(ML.parent, nvc)
            Ic = mesh.levels[lev + 1].interior
            P = P_full[I][:, Ic].tocsr()
            A_full = drop_small((P_full.T @ A_full @ P_full).tocsr())
        levels.append(Level(A=A, diag=A.diagonal().copy(), G=G, inv_deg=1.0 / deg, P=P))
    AJ = levels[-1].A.toarray()
    if np.iscomplexobj(AJ):  # complex symmetric, not Hermitian: LU
        return Hierarchy(levels, None, sla.lu_factor(AJ))
    return Hierarchy(levels, sla.cho_factor(AJ, lower=True))


# ----------------------------------------------------------- parameters ----

@dataclass
class Params:
    """Theta = {theta_l, eta_l, Theta_B,l, Theta_R,l, Theta_P,l : l = 1..J-1}
    (Sec. 3).  With scalar features each SAGEConv holds (w1, w2)."""
    theta: np.ndarray
    eta: np.ndarray
    wB: np.ndarray
    wR: np.ndarray
    wP: np.ndarray
    nu_pre: int = 2
    nu_post: int = 2
    # ChebConv smoother coefficients c_{l,0..K} per level (J-1, K+1); None:
    # the SAGEConv smoother with wB
    cheb: np.ndarray | None = None

    @staticmethod
    def identity(J: int, omega: float = 2.0 / 3.0, nu: int = 2) -> "Params":
        """Initialisation of Sec. 3.4: W1 = I, W2 = 0, theta = omega, eta = 1,
        which makes the learnable cycle the classical damped-Jacobi V-cycle."""
        m = J - 1
        one = np.tile([1.0, 0.0], (m, 1))
        return Params(np.full(m, omega), np.ones(m), one.copy(), one.copy(), one.copy(), nu, nu)

    def copy(self) -> "Params":
        return Params(self.theta.copy(), self.eta.copy(), self.wB.copy(), self.wR.copy(),
                      self.wP.copy(), self.nu_pre, self.nu_post,
                      None if self.cheb is None else self.cheb.copy())

    def astype(self, dtype) -> "Params":
        return Params(self.theta.astype(dtype), self.eta.astype(dtype), self.wB.astype(dtype),
                      self.wR.astype(dtype), self.wP.astype(dtype), self.nu_pre, self.nu_post,
                      None if self.cheb is None else self.cheb.astype(dtype))

    # flat view used for gradients: per level [theta, eta, wB1, wB2, wR1, wR2, wP1, wP2]
    def flat(self) -> np.ndarray:
        return np.concatenate([self.theta[:, None], self.eta[:, None], self.wB, self.wR,
                               self.wP], axis=1).ravel()

    @staticmethod
    def from_flat(x: np.ndarray, nu_pre: int = 2, nu_post: int = 2) -> "Params":
        x = np.asarray(x).reshape(-1, 8)
        return Params(x[:, 0].copy(), x[:, 1].copy(), x[:, 2:4].copy(), x[:, 4:6].copy(),
                      x[:, 6:8].copy(), nu_pre, nu_post)


# ---------------------------------------------------------------- cycle ----

def conv(L: Level, x: np.ndarray, w1, w2) -> np.ndarray:
    """SAGEConv with mean aggregation (Sec. 3.2): w1 x_i + w2 mean_{N(i)} x_j."""
    return w1 * x + w2 * (L.inv_deg[:, None] * (L.G @ x))


def lap_hat(L: Level, x: np.ndarray) -> np.ndarray:
    """The scaled normalised graph Laplacian of ChebConv with lambda_max = 2:
    Lhat x = (D_g^{-1} L_g - I) x = -D_g^{-1} A_g x, L_g = D_g - A_g."""
    return -(L.inv_deg[:, None] * (L.G @ x))


def cheb_conv(L: Level, x: np.ndarray, c) -> np.ndarray:
    """ChebConv of degree K = len(c) - 1 >= 1 (Defferrard et al.; Sec. 3.3):
    sum_k c_k T_k(Lhat) x with the Chebyshev recurrence T_0 = I,
    T_1 = Lhat, T_k = 2 Lhat T_{k-1} - T_{k-2}."""
    t_prev, t = x, lap_hat(L, x)
    out = c[0] * t_prev + c[1] * t
    for k in range(2, len(c)):
        t_prev, t = t, 2.0 * lap_hat(L, t) - t_prev
        out = out + c[k] * t
    return out


def smooth(L: Level, f, u, theta, eta, wB, cheb=None):
    """One learnable smoothing step (Sec. 3): delta = theta D_A^{-1}(f - A u),
    u <- u + eta Phi_B(delta); Phi_B is SAGEConv (wB) or, with cheb, the
    ChebConv polynomial smoother."""
    delta = theta * (f - L.A @ u) / L.diag[:, None]
    if cheb is not None:
        return u + eta * cheb_conv(L, delta, cheb)
    return u + eta * conv(L, delta, wB[0], wB[1])


def lmg(H: Hierarchy, p: Params, lev: int, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Algorithm 2, u = LMG(A_l, f, u, l, Theta); lev is 0-based (paper l-1)."""
    if lev == H.J - 1:
        return sla.cho_solve(H.chol, f)
    L = H.levels[lev]
    cb = None if p.cheb is None else p.cheb[lev]
    for _ in range(p.nu_pre):
        u = smooth(L, f, u, p.theta[lev], p.eta[lev], p.wB[lev], cb)
    r = f - L.A @ u
    rc = L.P.T @ conv(L, r, p.wR[lev][0], p.wR[lev][1])
    ec = lmg(H, p, lev + 1, rc, np.zeros_like(rc))
    e = conv(L, L.P @ ec, p.wP[lev][0], p.wP[lev][1])
    u = u + e
    for _ in range(p.nu_post):
        u = smooth(L, f, u, p.theta[lev], p.eta[lev], p.wB[lev], cb)
    return u


def vcycle(H: Hierarchy, p: Params, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    return lmg(H, p, 0, f, u)


# -------------------------------------------- two features per node (d = 2) ----

@dataclass
class Params2:
    """Theta with two features per node: each SAGEConv holds W_1, W_2 in
    R^{2x2} (Sec. 3.2).  The Helmholtz experiment (Sec. 4.2) carries the real
    and imaginary parts of the complex solution as the two features.
    WB, WR, WP: (J-1, 2, 2, 2), per level (W_1, W_2)."""
    theta: np.ndarray
    eta: np.ndarray
    WB: np.ndarray
    WR: np.ndarray
    WP: np.ndarray
    nu_pre: int = 1
    nu_post: int = 1

    @staticmethod
    def identity(J: int, omega: float = 2.0 / 3.0, nu: int = 1) -> "Params2":
        """W_1 = I, W_2 = 0, theta = omega, eta = 1 (the initialisation of the
        Helmholtz experiment): the classical damped-Jacobi cycle on the complex
        system."""
        W = np.zeros((J - 1, 2, 2, 2))
        W[:, 0] = np.eye(2)
        return Params2(np.full(J - 1, omega), np.ones(J - 1), W.copy(), W.copy(), W.copy(), nu, nu)


def features(x: np.ndarray) -> np.ndarray:
    """Complex (n, B) -> node features (n, B, 2) = (Re, Im)."""
    return np.stack([x.real, x.imag], axis=-1)


def conv2(L: Level, x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """SAGEConv, mean aggregation, two features per node (Sec. 3.2):
    Phi(x)_i = W_1 x_i + W_2 mean_{N(i)} x_j for the feature vectors
    x_i = (Re, Im) of the complex input; returns the complex form."""
    n, B = x.shape
    X = features(x)
    mean = (L.inv_deg[:, None] * (L.G @ X.reshape(n, 2 * B))).reshape(n, B, 2)
    Y = np.einsum("pq,nbq->nbp", W[0], X) + np.einsum("pq,nbq->nbp", W[1], mean)
    return Y[..., 0] + 1j * Y[..., 1]


def smooth2(L: Level, f, u, theta, eta, WB):
    """Learnable smoothing step (Sec. 3) on a complex system with two-feature
    convolutions: delta = theta D_A^{-1}(f - A u) in complex arithmetic,
    u <- u + eta Phi_B(delta)."""
    delta = theta * (f - L.A @ u) / L.diag[:, None]
    return u + eta * conv2(L, delta, WB)


def lmg2(H: Hierarchy, p: Params2, lev: int, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Algorithm 2 with two features per node on a complex operator; the
    coarsest level is solved exactly (dense LU)."""
    if lev == H.J - 1:
        return sla.lu_solve(H.lu, f)
    L = H.levels[lev]
    for _ in range(p.nu_pre):
        u = smooth2(L, f, u, p.theta[lev], p.eta[lev], p.WB[lev])
    r = f - L.A @ u
    rc = L.P.T @ conv2(L, r, p.WR[lev])
    ec = lmg2(H, p, lev + 1, rc, np.zeros_like(rc))
    u = u + conv2(L, L.P @ ec, p.WP[lev])
    for _ in range(p.nu_post):
        u = smooth2(L, f, u, p.theta[lev], p.eta[lev], p.WB[lev])
    return u


def vcycle2(H: Hierarchy, p: Params2, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    return lmg2(H, p, 0, f, u)


def fmg2(H: Hierarchy, p: Params2, f: np.ndarray) -> np.ndarray:
    """Full multigrid with two-feature convolutions: f restricted to every
    level by P^T Phi_R, the coarsest level solved exactly, on each finer level
    Phi_P(P u_{l+1}) from a zero iterate as the initial guess of one cycle
    started on that level (the FMG of the Sec. 4.2 preconditioner table,
    tab:helmholtz-results-precond)."""
    J = H.J
    fs = [f]
    for lev in range(J - 1):
        L = H.levels[lev]
        fs.append(L.P.T @ conv2(L, fs[lev], p.WR[lev]))
    u = sla.lu_solve(H.lu, fs[J - 1])
    for lev in range(J - 2, -1, -1):
        L = H.levels[lev]
        u = lmg2(H, p, lev, fs[lev], conv2(L, L.P @ u, p.WP[lev]))
    return u


def real_vec(z: np.ndarray) -> np.ndarray:
    """Complex (n,) -> the real 2n vector [Re z; Im z]."""
    return np.concatenate([z.real, z.imag])


def complex_vec(v: np.ndarray) -> np.ndarray:
    """The real 2n vector [Re; Im] -> complex (n,)."""
    n = v.shape[0] // 2
    return v[:n] + 1j * v[n:]


def fgmres2(H: Hierarchy, p: Params2, f: np.ndarray, tol: float, precond: str = "vcycle",
            restart: int = 30, max_iter: int = 300):
    """FGMRES on a complex system with the two-feature cycle (or FMG) as the
    right preconditioner, one right-hand side f (complex, 1-D).  With W_1, W_2
    mixing the features the preconditioner is real-linear, not complex-linear,
    so the Krylov method runs on the equivalent real system of size 2n,
    [[Re A, -Im A], [Im A, Re A]] [Re u; Im u] = [Re f; Im f], with real inner
    products.  Returns (u complex, iterations, residual estimates)."""
    A = H.levels[0].A
    Ar = sp.bmat([[A.real, -A.imag], [A.imag, A.real]]).tocsr()

    def M(v):
        z = complex_vec(v)[:, None]
        if precond == "fmg":
            out = fmg2(H, p, z)
        else:
            out = lmg2(H, p, 0, z, np.zeros_like(z))
        return real_vec(out[:, 0])

    u, its, hist = fgmres(Ar, real_vec(f), M, tol, restart=restart, max_iter=max_iter)
    return complex_vec(u), its, hist


def fmg(H: Hierarchy, p: Params, f: np.ndarray) -> np.ndarray:
    """Full multigrid (nested iteration), the preconditioner of the Krylov
    experiments of Sec. 4.2 (tab:helmholtz-results-precond).  The right-hand
    side goes to every level through the cycle's restriction P^T Phi_R; the
    coarsest level is solved exactly; on each finer level the coarser
    solution, through the cycle's prolongation Phi_P P, is the initial guess
    of one V-cycle (Algorithm 2 started on that level).  One V-cycle per
    level, as in the paper."""
    J = H.J
    fs = [f]
    for lev in range(J - 1):
        L = H.levels[lev]
        fs.append(L.P.T @ conv(L, fs[lev], p.wR[lev][0], p.wR[lev][1]))
    u = sla.cho_solve(H.chol, fs[J - 1])
    for lev in range(J - 2, -1, -1):
        L = H.levels[lev]
        u0 = conv(L, L.P @ u, p.wP[lev][0], p.wP[lev][1])
        u = lmg(H, p, lev, fs[lev], u0)
    return u


def fgmres(A, f: np.ndarray, precond, tol: float, restart: int = 30, max_iter: int = 300):
    """Restarted flexible GMRES with right preconditioning (Saad 1993), the
    outer Krylov method the paper pairs with its V-cycle and FMG
    preconditioners (Sec. 4.2, tab:helmholtz-results-precond), for one
    right-hand side f (1-D).  precond(v)
    returns z ~ A^{-1} v and may change between calls.  Modified Gram-Schmidt
    Arnoldi, Givens rotations on the Hessenberg matrix; stops when the
    recurrence's residual estimate |g_{j+1}| < tol ||f||, or after max_iter
    inner steps.  Returns (u, iterations, residual estimates per step)."""
    n = f.shape[0]
    u = np.zeros(n)
    fn = np.linalg.norm(f)
    hist, its = [], 0
    while its < max_iter:
        r = f - A @ u
        beta = np.linalg.norm(r)
        if beta < tol * fn:
            break
        V = np.zeros((n, restart + 1))
        Z = np.zeros((n, restart))
        Hm = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / beta
        jl = -1
        for j in range(restart):
            Z[:, j] = precond(V[:, j])
            w = A @ Z[:, j]
            for i in range(j + 1):
                Hm[i, j] = w @ V[:, i]
                w = w - Hm[i, j] * V[:, i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] > 0:
                V[:, j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            rr = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = (Hm[j, j] / rr, Hm[j + 1, j] / rr) if rr > 0 else (1.0, 0.0)
            Hm[j, j], Hm[j + 1, j] = rr, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            jl = j
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) < tol * fn or its >= max_iter:
                break
        y = np.linalg.solve(np.triu(Hm[:jl + 1, :jl + 1]), g[:jl + 1])
        u = u + Z[:, :jl + 1] @ y
        if hist and hist[-1] < tol * fn:
            break
    return u, its, np.array(hist)


def fcg(A, f: np.ndarray, precond, tol: float, max_iter: int = 300, mmax: int = 1):
    """Flexible conjugate gradients, FCG(mmax) of Notay (SIAM J. Sci. Comput.
    22, 2000), for one right-hand side f (1-D) from u = 0.  The paper pairs its
    cycle with FGMRES (Sec. 4.2); for the SPD operators of this path flexible
    CG is the symmetric counterpart.  precond(v) returns z ~ A^{-1} v and may
    change between calls.  Iteration i:
        z_i = precond(r_i)
        d_i = z_i - sum_{k = i-m_i .. i-1} (z_i, A d_k) / (d_k, A d_k) d_k,
              m_i = min(i, mmax)   (explicit A-orthogonalisation against the
                                    last mmax directions)
        alpha_i = (d_i, r_i) / (d_i, A d_i)
        u_{i+1} = u_i + alpha_i d_i,   r_{i+1} = r_i - alpha_i A d_i
    stopping as soon as the recurrence residual ||r_{i+1}|| < tol ||f||, or
    after max_iter iterations (r_0 = f is tested first).  Returns
    (u, iterations, recurrence residual norms per iteration, iterates u_1..)."""
    u = np.zeros_like(f)
    r = f.copy()
    fn = np.linalg.norm(f)
    D, AD = [], []  # last mmax directions and their images
    hist, iterates = [], []
    if not np.linalg.norm(r) < tol * fn:
        for _ in range(max_iter):
            z = precond(r)
            d = z.copy()
            for dk, qk in zip(D, AD):
                d = d - (z @ qk) / (dk @ qk) * dk
            q = A @ d
            alpha = (d @ r) / (d @ q)
            u = u + alpha * d
            r = r - alpha * q
            D.append(d)
            AD.append(q)
            if len(D) > mmax:
                D.pop(0)
                AD.pop(0)
            hist.append(np.linalg.norm(r))
            iterates.append(u.copy())
            if hist[-1] < tol * fn:
                break
    return u, len(hist), np.array(hist), iterates


def residual(H: Hierarchy, f, u):
    return f - H.levels[0].A @ u


def relres(H: Hierarchy, f, u) -> np.ndarray:
    """||f - A u||_2 / ||f||_2 per right-hand side (column)."""
    r = residual(H, f, u)
    return np.sqrt((r * r).sum(0)) / np.sqrt((f * f).sum(0))


@dataclass
class SolveResult:
    u: np.ndarray
    iters: np.ndarray
    relres: np.ndarray
    history: list = field(default_factory=list)


def solve_vcycles(H: Hierarchy, p: Params, f: np.ndarray, tol: float,
                  max_iter: int = 200) -> SolveResult:
    """Stationary iteration u^m = LMG(A, f, u^{m-1}) from u^0 = 0, each column
    stopping as soon as ||f - A u||/||f|| < tol (checked before each cycle)."""
    u = np.zeros_like(f)
    B = f.shape[1]
    iters = np.zeros(B, dtype=np.int64)
    active = np.ones(B, dtype=bool)
    hist = []
    for _ in range(max_iter + 1):
        rr = relres(H, f, u)
        hist.append(rr.copy())
        active &= rr >= tol
        if not active.any():
            break
        if iters[active].max() >= max_iter:
            break
        cols = np.flatnonzero(active)
        u[:, cols] = vcycle(H, p, f[:, cols], u[:, cols])
        iters[cols] += 1
    return SolveResult(u, iters, relres(H, f, u), hist)


def solve_refinement(H: Hierarchy, p: Params, f: np.ndarray, tol: float,
                     max_iter: int = 100) -> SolveResult:
    """Iterative refinement with the V-cycle as the inner solve: r = f - A u,
    c = LMG(A, r, 0), u <- u + c, until ||r||/||f|| < tol (per column).  In the
    oracle every step is FP64; the CUDA path runs the inner cycle in FP32."""
    u = np.zeros_like(f)
    B = f.shape[1]
    iters = np.zeros(B, dtype=np.int64)
    active = np.ones(B, dtype=bool)
    hist = []
    for _ in range(max_iter + 1):
        r = residual(H, f, u)
        rr = np.sqrt((r * r).sum(0)) / np.sqrt((f * f).sum(0))
        hist.append(rr.copy())
        active &= rr >= tol
        if not active.any() or iters[active].max() >= max_iter:
            break
        cols = np.flatnonzero(active)
        c = vcycle(H, p, r[:, cols], np.zeros((f.shape[0], cols.size), dtype=f.dtype))
        u[:, cols] += c
        iters[cols] += 1
    return SolveResult(u, iters, relres(H, f, u), hist)


# -------------------------------------------------------------- training ----

def unrolled_loss(H: Hierarchy, p: Params, f: np.ndarray, K: int,
                  u0: np.ndarray | None = None) -> np.ndarray:
    """Loss of K unrolled cycles: mean over columns of ||r_K||^2 / ||r_0||^2,
    with r_k = f - A u_k, u_{k+1} = LMG(A, f, u_k).  Written with x*x instead
    of |x|^2 so that it stays analytic (complex-step differentiable)."""
    u = np.zeros_like(f) if u0 is None else u0
    r0 = residual(H, f, u)
    n0 = (r0 * r0).sum(0)
    for _ in range(K):
        u = vcycle(H, p, f, u)
    r = residual(H, f, u)
    return ((r * r).sum(0) / n0).mean()


def loss_gradient_complex_step(H: Hierarchy, p: Params, f: np.ndarray, K: int,
                               u0: np.ndarray | None = None, h: float = 1e-30):
    """d loss / d Theta by complex-step differentiation: for each flat
    parameter x_k, Im L(x + i h e_k) / h.  The loss is a polynomial in Theta,
    so this is exact to rounding, independent of any hand-written adjoint."""
    x = p.flat()
    g = np.zeros_like(x)
    fc = f.astype(np.complex128)
    u0c = None if u0 is None else u0.astype(np.complex128)
    for k in range(x.size):
        xc = x.astype(np.complex128)
        xc[k] += 1j * h
        pc = _same_smoother(Params.from_flat(xc, p.nu_pre, p.nu_post), p)
        g[k] = np.imag(unrolled_loss(H, pc, fc, K, u0c)) / h
    return unrolled_loss(H, p, f, K, u0), g


def _same_smoother(q: Params, p: Params) -> Params:
    """q with p's smoother choice (the ChebConv coefficients are not part of
    the flat Theta vector)."""
    q.cheb = None if p.cheb is None else p.cheb.astype(q.theta.dtype)
    return q


def cheb_gradient_complex_step(H: Hierarchy, p: Params, f: np.ndarray, K: int,
                               u0: np.ndarray | None = None, h: float = 1e-30) -> np.ndarray:
    """d loss / d c_{l,k} of the ChebConv smoother's coefficients by complex
    step (the loss is a polynomial in them, so exact to rounding)."""
    g = np.zeros_like(p.cheb)
    fc = f.astype(np.complex128)
    u0c = None if u0 is None else u0.astype(np.complex128)
    for idx in np.ndindex(*p.cheb.shape):
        pc = p.astype(np.complex128)
        pc.cheb[idx] += 1j * h
        g[idx] = np.imag(unrolled_loss(H, pc, fc, K, u0c)) / h
    return g


def cheb_gradient_fd(H: Hierarchy, p: Params, f: np.ndarray, K: int,
                     u0: np.ndarray | None = None, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of the same loss in the ChebConv coefficients."""
    g = np.zeros_like(p.cheb)
    for idx in np.ndindex(*p.cheb.shape):
        step = h * max(1.0, abs(p.cheb[idx]))
        pp, pm = p.copy(), p.copy()
        pp.cheb[idx] += step
        pm.cheb[idx] -= step
        g[idx] = (unrolled_loss(H, pp, f, K, u0) - unrolled_loss(H, pm, f, K, u0)) / (2 * step)
    return g


def loss_gradient_fd(H: Hierarchy, p: Params, f: np.ndarray, K: int,
                     u0: np.ndarray | None = None, h: float = 1e-6):
    """Central finite differences of the same loss (second-order accurate)."""
    x = p.flat()
    g = np.zeros_like(x)
    for k in range(x.size):
        xp, xm = x.copy(), x.copy()
        step = h * max(1.0, abs(x[k]))
        xp[k] += step
        xm[k] -= step
        lp = unrolled_loss(H, _same_smoother(Params.from_flat(xp, p.nu_pre, p.nu_post), p), f,
                           K, u0)
        lm = unrolled_loss(H, _same_smoother(Params.from_flat(xm, p.nu_pre, p.nu_post), p), f,
                           K, u0)
        g[k] = (lp - lm) / (2 * step)
    return g
