"""Seeded synthetic meshes and nested mesh hierarchies.

This module generates inputs only: vertex coordinates, triangles, Dirichlet
boundary flags and, between consecutive levels of a uniformly refined
hierarchy, the map from each fine vertex to the coarse vertices it sits on or
between.  It holds none of the multigrid method's arithmetic (no prolongation
matrices, no coarse operators, no graphs); both the oracle and the CUDA path
build those themselves from what is produced here.

Level numbering follows the paper (Sec. 2.2): index 0 here is the finest level
(the paper's level 1) and the last index is the coarsest (level J).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class MeshLevel:
    """One level of a nested triangulation.

    xy        (nv, 2) float64 vertex coordinates
    tri       (nt, 3) int64 vertex indices, counter-clockwise or not
    boundary  (nv,) bool, True on the Dirichlet boundary
    parent    (nv, 2) int64 or None.  For every vertex of this level, the
              vertices of the next-coarser level it comes from: (c, -1) when
              it coincides with coarse vertex c, (a, b) when it is the
              midpoint of the coarse edge a-b.  None on the coarsest level.
    """

    xy: np.ndarray
    tri: np.ndarray
    boundary: np.ndarray
    parent: np.ndarray | None = None

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    @property
    def interior(self) -> np.ndarray:
        """Indices of the interior vertices in vertex order: the DOF ordering."""
        return np.flatnonzero(~self.boundary)


@dataclass
class MeshHierarchy:
    levels: list[MeshLevel] = field(default_factory=list)  # [0] finest

    @property
    def J(self) -> int:
        return len(self.levels)


def _rng(seed: int, stream: int) -> np.random.Generator:
    """Independent, reproducible streams: 0 coefficients, 1 sources, 2 mesh
    jitter, 3 initial guesses, 4 arrivals."""
    return np.random.default_rng([int(seed), int(stream)])


# --------------------------------------------------------------------------
# Uniform right-triangle meshes of the unit square
# --------------------------------------------------------------------------

def square_level(N: int) -> MeshLevel:
    """N x N vertices on [0,1]^2 (h = 1/(N-1)); vertex (i, j) has index
    j*N + i (x fastest).  Each cell is split by its SW->NE diagonal."""
    i = np.arange(N)
    X, Y = np.meshgrid(i, i, indexing="xy")  # Y[j, i] = j
    xy = np.stack([X.ravel() / (N - 1), Y.ravel() / (N - 1)], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(N - 1), np.arange(N - 1), indexing="xy")
    v00 = (cj * N + ci).ravel()
    v10, v01 = v00 + 1, v00 + N
    v11 = v01 + 1
    tri = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    # order triangles cell by cell (lower then upper) for a stable assembly order
    nc = v00.size
    order = np.stack([np.arange(nc), np.arange(nc) + nc], 1).ravel()
    tri = tri[order].astype(np.int64)
    bnd = (X == 0) | (X == N - 1) | (Y == 0) | (Y == N - 1)
    return MeshLevel(xy=xy, tri=tri, boundary=bnd.ravel())


def square_parent(N: int) -> np.ndarray:
    """Fine (N x N) -> coarse ((N+1)/2 x (N+1)/2) vertex parent map for the
    uniform refinement that splits every coarse triangle into four."""
    assert (N - 1) % 2 == 0
    Nc = (N - 1) // 2 + 1
    i = np.arange(N)
    I, Jj = np.meshgrid(i, i, indexing="xy")
    I, Jj = I.ravel(), Jj.ravel()
    par = np.full((N * N, 2), -1, dtype=np.int64)
    ie, je = I % 2 == 0, Jj % 2 == 0
    m = ie & je
    par[m, 0] = (Jj[m] // 2) * Nc + I[m] // 2
    m = ~ie & je  # horizontal coarse edge
    par[m, 0] = (Jj[m] // 2) * Nc + (I[m] - 1) // 2
    par[m, 1] = (Jj[m] // 2) * Nc + (I[m] + 1) // 2
    m = ie & ~je  # vertical coarse edge
    par[m, 0] = ((Jj[m] - 1) // 2) * Nc + I[m] // 2
    par[m, 1] = ((Jj[m] + 1) // 2) * Nc + I[m] // 2
    m = ~ie & ~je  # SW->NE diagonal of a coarse cell
    par[m, 0] = ((Jj[m] - 1) // 2) * Nc + (I[m] - 1) // 2
    par[m, 1] = ((Jj[m] + 1) // 2) * Nc + (I[m] + 1) // 2
    return par


def square_hierarchy(N: int, J: int) -> MeshHierarchy:
    """J nested uniform meshes of the unit square, finest N x N vertices."""
    levels = []
    n = N
    for lev in range(J):
        L = square_level(n)
        if lev < J - 1:
            if (n - 1) % 2:
                raise ValueError(f"cannot coarsen a {n}x{n} mesh {J - 1} times")
            L.parent = square_parent(n)
            n = (n - 1) // 2 + 1
        levels.append(L)
    return MeshHierarchy(levels)


# --------------------------------------------------------------------------
# Unstructured: red refinement of a jittered L-shaped coarse triangulation
# --------------------------------------------------------------------------

def _boundary_from_edges(nv: int, tri: np.ndarray):
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 0)
    e.sort(axis=1)
    ue, inv, cnt = np.unique(e, axis=0, return_inverse=True, return_counts=True)
    bnd = np.zeros(nv, dtype=bool)
    be = ue[cnt == 1]
    bnd[be.ravel()] = True
    return ue, inv.reshape(3, -1).T, cnt, bnd


def lshape_coarse(h_inv: int = 8, jitter: float = 0.2, seed: int = 0) -> MeshLevel:
    """Structured triangulation (h = 1/h_inv) of [-1,1]^2 minus (0,1]x(0,1]
    with SW->NE diagonals; interior vertices moved by U(-jitter*h, jitter*h)
    per coordinate from the seed."""
    n = 2 * h_inv + 1
    h = 1.0 / h_inv
    g = np.arange(n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    x = -1.0 + X.ravel() * h
    y = -1.0 + Y.ravel() * h
    keep = ~((x > 1e-12) & (y > 1e-12))
    newid = -np.ones(n * n, dtype=np.int64)
    newid[keep] = np.arange(keep.sum())
    tris = []
    for j in range(n - 1):
        for i in range(n - 1):
            x0, y0 = -1.0 + i * h, -1.0 + j * h
            if x0 > -1e-12 and y0 > -1e-12:
                continue  # cell inside the removed quadrant
            v00 = j * n + i
            v10, v01, v11 = v00 + 1, v00 + n, v00 + n + 1
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    tri = newid[np.array(tris, dtype=np.int64)]
    xy = np.stack([x[keep], y[keep]], 1)
    _, _, _, bnd = _boundary_from_edges(xy.shape[0], tri)
    r = _rng(seed, 2)
    d = r.uniform(-jitter * h, jitter * h, size=xy.shape)
    xy = xy + np.where(bnd[:, None], 0.0, d)
    return MeshLevel(xy=xy, tri=tri, boundary=bnd)


def _morton_order(xy: np.ndarray) -> np.ndarray:
    lo = xy.min(0)
    span = (xy.max(0) - lo).max()
    q = np.floor((xy - lo) / span * (2 ** 20 - 1)).astype(np.uint64)

    def spread(v):
        v = v & np.uint64(0xFFFFF)
        out = np.zeros_like(v)
        for b in range(20):
            out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        return out

    key = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))
    return np.argsort(key, kind="stable")


def red_refine(coarse: MeshLevel, reorder: bool = True) -> MeshLevel:
    """Split every triangle into four through its edge midpoints.  Returns the
    fine level with .parent filled in (fine -> coarse).  With reorder=True the
    fine vertices are renumbered along a Morton curve for memory locality."""
    nvc = coarse.nv
    ue, tri_edge, cnt, _ = _boundary_from_edges(nvc, coarse.tri)
    mid = nvc + np.arange(ue.shape[0])
    xy = np.concatenate([coarse.xy, 0.5 * (coarse.xy[ue[:, 0]] + coarse.xy[ue[:, 1]])], 0)
    bnd = np.concatenate([coarse.boundary, cnt == 1])
    par = np.concatenate([
        np.stack([np.arange(nvc), -np.ones(nvc, dtype=np.int64)], 1),
        ue.astype(np.int64)], 0)
    a, b, c = coarse.tri[:, 0], coarse.tri[:, 1], coarse.tri[:, 2]
    mab, mbc, mca = mid[tri_edge[:, 0]], mid[tri_edge[:, 1]], mid[tri_edge[:, 2]]
    tri = np.concatenate([
        np.stack([a, mab, mca], 1), np.stack([mab, b, mbc], 1),
        np.stack([mca, mbc, c], 1), np.stack([mab, mbc, mca], 1)], 0)
    if reorder:
        perm = _morton_order(xy)          # new -> old
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)  # old -> new
        xy, bnd, par = xy[perm], bnd[perm], par[perm]
        tri = inv[tri]
    return MeshLevel(xy=xy, tri=tri.astype(np.int64), boundary=bnd, parent=par)


def lshape_hierarchy(refinements: int = 7, h_inv: int = 8, jitter: float = 0.2,
                     seed: int = 0) -> MeshHierarchy:
    coarse = lshape_coarse(h_inv, jitter, seed)
    chain = [coarse]
    for _ in range(refinements):
        chain.append(red_refine(chain[-1]))
    # chain[k].parent maps chain[k] -> chain[k-1]; hierarchy wants finest first
    levels = []
    for k in range(len(chain) - 1, -1, -1):
        L = chain[k]
        levels.append(MeshLevel(xy=L.xy, tri=L.tri, boundary=L.boundary, parent=L.parent))
    levels[-1].parent = None
    return MeshHierarchy(levels)
