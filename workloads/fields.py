"""Seeded coefficient fields, P1 stiffness assembly and right-hand sides.

The linear system A u = f is the input of the multigrid method (the paper's
Eq. (1.1) and Algorithm 3's "Given: system matrix A, right-hand side f").
This module produces it: the P1 finite-element stiffness matrix of
-div(K grad u) on the finest mesh, before the Dirichlet rows and columns are
removed, and i.i.d. N(0,1) right-hand sides on the interior vertices.
Everything the multigrid method derives from A (prolongation, Galerkin coarse
operators, graphs, smoothers) is left to its two implementations.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .meshes import MeshLevel, _rng


def centroids(L: MeshLevel) -> np.ndarray:
    return L.xy[L.tri].mean(axis=1)


def checkerboard(L: MeshLevel, ncell: int, values: tuple[float, float], seed: int,
                 domain=((0.0, 1.0), (0.0, 1.0))) -> np.ndarray:
    """Piecewise-constant isotropic coefficient per element: ncell x ncell cells,
    each independently values[0] or values[1] with probability 1/2."""
    table = _rng(seed, 0).integers(0, 2, size=(ncell, ncell))
    c = centroids(L)
    (x0, x1), (y0, y1) = domain
    ix = np.clip(np.floor((c[:, 0] - x0) / (x1 - x0) * ncell).astype(int), 0, ncell - 1)
    iy = np.clip(np.floor((c[:, 1] - y0) / (y1 - y0) * ncell).astype(int), 0, ncell - 1)
    return np.asarray(values, dtype=np.float64)[table[iy, ix]]


def lognormal(L: MeshLevel, sigma: float, corr_len: float, seed: int,
              n_features: int = 512) -> np.ndarray:
    """k = exp(sigma * g) per element, g a unit-variance Gaussian field with
    covariance exp(-|x-y|^2 / (2 corr_len^2)), drawn as n_features random
    Fourier features and evaluated at element centroids."""
    r = _rng(seed, 0)
    w = r.standard_normal((n_features, 2)) / corr_len
    b = r.uniform(0.0, 2.0 * np.pi, size=n_features)
    c = centroids(L)
    g = _rff_tensor_grid(c, w, b)
    if g is None:
        g = np.empty(c.shape[0])
        step = 65536
        for s in range(0, c.shape[0], step):
            g[s:s + step] = np.cos(c[s:s + step] @ w.T + b).sum(1)
    return np.exp(sigma * np.sqrt(2.0 / n_features) * g)


def _rff_tensor_grid(c: np.ndarray, w: np.ndarray, b: np.ndarray):
    """sum_m cos(w_m . c + b_m) for centroids that form a few tensor grids
    (uniform square meshes: one grid per triangle orientation), as
    Re(Ey diag(e^{ib}) Ex^T), a complex matrix product; None otherwise."""
    xs, xi = np.unique(np.round(c[:, 0], 12), return_inverse=True)
    ys, yi = np.unique(np.round(c[:, 1], 12), return_inverse=True)
    if xs.size * ys.size > 8 * c.shape[0] or xs.size * ys.size > 2 ** 26:
        return None
    ex = np.exp(1j * np.outer(xs, w[:, 0]))              # (nx, M)
    ey = np.exp(1j * np.outer(ys, w[:, 1]) + 1j * b)     # (ny, M)
    G = (ey @ ex.T).real                                  # (ny, nx)
    return G[yi, xi]


def rotated_anisotropy(eps: float, angle_deg: float) -> np.ndarray:
    t = np.deg2rad(angle_deg)
    R = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
    return R @ np.diag([1.0, eps]) @ R.T


def assemble_p1(L: MeshLevel, k: np.ndarray | None = None,
                K: np.ndarray | None = None) -> sp.csr_matrix:
    """P1 stiffness matrix over all vertices (no boundary conditions applied):
    A_ab = sum_T |T| grad(phi_a)^T K_T grad(phi_b).  k: per-element scalar
    coefficient (isotropic); K: one constant 2x2 tensor.  Default k = 1."""
    p = L.xy[L.tri]  # (nt, 3, 2)
    x, y = p[:, :, 0], p[:, :, 1]
    two_area = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    gx = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], 1) / two_area[:, None]
    gy = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], 1) / two_area[:, None]
    area = 0.5 * np.abs(two_area)
    if K is not None:
        Kxx, Kxy, Kyy = K[0, 0], 0.5 * (K[0, 1] + K[1, 0]), K[1, 1]
        ke = (Kxx * gx[:, :, None] * gx[:, None, :] + Kyy * gy[:, :, None] * gy[:, None, :]
              + Kxy * (gx[:, :, None] * gy[:, None, :] + gy[:, :, None] * gx[:, None, :]))
        ke *= area[:, None, None]
    else:
        kk = np.ones(L.tri.shape[0]) if k is None else np.asarray(k, dtype=np.float64)
        ke = (gx[:, :, None] * gx[:, None, :] + gy[:, :, None] * gy[:, None, :])
        ke *= (area * kk)[:, None, None]
    rows = np.repeat(L.tri, 3, axis=1).ravel()
    cols = np.tile(L.tri, (1, 3)).ravel()
    A = sp.coo_matrix((ke.ravel(), (rows, cols)), shape=(L.nv, L.nv)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble_mass_p1(L: MeshLevel) -> sp.csr_matrix:
    """P1 mass matrix over all vertices: M_ab = int phi_a phi_b, per element
    |T|/12 (1 + delta_ab)."""
    p = L.xy[L.tri]
    x, y = p[:, :, 0], p[:, :, 1]
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0])
                        - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    me = (np.ones((3, 3)) + np.eye(3))[None] * (area / 12.0)[:, None, None]
    rows = np.repeat(L.tri, 3, axis=1).ravel()
    cols = np.tile(L.tri, (1, 3)).ravel()
    M = sp.coo_matrix((me.ravel(), (rows, cols)), shape=(L.nv, L.nv)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def boundary_edges(L: MeshLevel) -> np.ndarray:
    """(ne, 2) vertex pairs of the edges that belong to one triangle only."""
    e = np.concatenate([L.tri[:, [0, 1]], L.tri[:, [1, 2]], L.tri[:, [2, 0]]], 0)
    e = np.sort(e, axis=1)
    u, cnt = np.unique(e, axis=0, return_counts=True)
    return u[cnt == 1]


def assemble_boundary_mass_p1(L: MeshLevel) -> sp.csr_matrix:
    """P1 boundary mass over the domain boundary: int_{boundary} phi_a phi_b,
    per boundary edge |e|/6 (1 + delta_ab)."""
    e = boundary_edges(L)
    ln = np.linalg.norm(L.xy[e[:, 0]] - L.xy[e[:, 1]], axis=1)
    be = (np.ones((2, 2)) + np.eye(2))[None] * (ln / 6.0)[:, None, None]
    rows = np.repeat(e, 2, axis=1).ravel()
    cols = np.tile(e, (1, 2)).ravel()
    Bm = sp.coo_matrix((be.ravel(), (rows, cols)), shape=(L.nv, L.nv)).tocsr()
    Bm.sum_duplicates()
    Bm.sort_indices()
    return Bm


def disk_source(xy: np.ndarray, centers, r_s: float = 0.02, eps_s: float = 0.001) -> np.ndarray:
    """Smoothed disk sources of the Helmholtz experiment (Sec. 4.2): 100 (1 -
    prod_c tanh((|x - c|^2 - r_s^2) / eps_s)); one centre for training, two
    for testing."""
    t = np.ones(xy.shape[0])
    for c in centers:
        t = t * np.tanh((((xy - np.asarray(c)) ** 2).sum(1) - r_s ** 2) / eps_s)
    return 100.0 * (1.0 - t)


def rhs(n: int, batch: int, seed: int) -> np.ndarray:
    """f ~ N(0,1) i.i.d. per interior DOF and right-hand side, shape (n, batch),
    right-hand-side index fastest (the node-feature layout X[n][B])."""
    return _rng(seed, 1).standard_normal((n, batch))
