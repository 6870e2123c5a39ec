"""Named synthetic workloads shaped like the paper's model problems.

Each builder returns a Problem: a nested mesh hierarchy, the finest-level P1
stiffness matrix over all vertices and seeded right-hand sides on the interior
vertices.  The five workloads and their sizes:

  poisson_square      -Laplace u = f, 33x33 nodes (961 DOF), 4 levels
  checkerboard_square -div(k grad u) = f, 513x513 (261121 DOF), 9 levels,
                      k in {1, 1e4} on an 8x8 checkerboard
  training_square     257x257 (65025 DOF), 8 levels, Poisson or a 4x4
                      {1, 1e3} checkerboard, 64 right-hand sides
  lognormal_square    65^2 .. 1025^2, k = exp(1.5 g), g a Gaussian field
                      with correlation length 0.1 (serving requests)
  lshape_anisotropic  jittered L-shape, 7 red refinements (about 3.1M DOF),
                      8 levels, K = R(30 deg) diag(1, 1e-3) R(30 deg)^T
  helmholtz_square    -Laplace u - k^2 u = f with the impedance condition
                      du/dn - i k u = 0 on the unit square centred at the
                      origin: complex A = K - k^2 M - i k B, every vertex a
                      DOF; column 0 the smoothed-disk training source, the
                      others seeded complex N(0, 1)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fields, meshes


@dataclass
class Problem:
    name: str
    mesh: meshes.MeshHierarchy
    A_full: sp.csr_matrix          # finest level, all vertices, FP64
    f: np.ndarray                  # (n_interior, batch) FP64
    info: dict

    @property
    def J(self) -> int:
        return self.mesh.J

    @property
    def n(self) -> int:
        return int(self.f.shape[0])

    @property
    def batch(self) -> int:
        return int(self.f.shape[1])


def poisson_square(N: int = 33, J: int = 4, batch: int = 1, seed: int = 0) -> Problem:
    H = meshes.square_hierarchy(N, J)
    A = fields.assemble_p1(H.levels[0])
    n = H.levels[0].interior.size
    return Problem(f"poisson_{N}", H, A, fields.rhs(n, batch, seed),
                   dict(N=N, J=J, batch=batch, seed=seed, coefficient="1"))


def checkerboard_square(N: int = 513, J: int = 9, ncell: int = 8,
                        values=(1.0, 1e4), batch: int = 1, seed: int = 0) -> Problem:
    H = meshes.square_hierarchy(N, J)
    k = fields.checkerboard(H.levels[0], ncell, values, seed)
    A = fields.assemble_p1(H.levels[0], k=k)
    n = H.levels[0].interior.size
    return Problem(f"checker{ncell}_{N}", H, A, fields.rhs(n, batch, seed),
                   dict(N=N, J=J, batch=batch, seed=seed,
                        coefficient=f"checkerboard {ncell}x{ncell} {values}"))


def training_square(kind: str = "poisson", N: int = 257, J: int = 8, batch: int = 64,
                    seed: int = 0) -> Problem:
    if kind == "poisson":
        return poisson_square(N, J, batch, seed)
    return checkerboard_square(N, J, 4, (1.0, 1e3), batch, seed)


def lognormal_square(N: int, seed: int, sigma: float = 1.5, corr_len: float = 0.1,
                     batch: int = 1, J: int | None = None) -> Problem:
    J = J if J is not None else int(round(np.log2(N - 1)))
    H = meshes.square_hierarchy(N, J)
    k = fields.lognormal(H.levels[0], sigma, corr_len, seed)
    A = fields.assemble_p1(H.levels[0], k=k)
    n = H.levels[0].interior.size
    return Problem(f"lognormal_{N}_s{seed}", H, A, fields.rhs(n, batch, seed),
                   dict(N=N, J=J, batch=batch, seed=seed,
                        coefficient=f"lognormal sigma={sigma} corr={corr_len}"))


def square_with_coefficients(N: int, k: np.ndarray, f: np.ndarray, J: int | None = None,
                             name: str = "square") -> Problem:
    """-div(k grad u) = f on the N x N square mesh with given element
    coefficients k (the mesh's element order: cells x fastest, lower then
    upper triangle) and interior source f ((n,) or (n, batch)); J levels
    down to 3 x 3 vertices by default.  A serving request's system."""
    J = J if J is not None else int(round(np.log2(N - 1)))
    H = meshes.square_hierarchy(N, J)
    A = fields.assemble_p1(H.levels[0], k=np.asarray(k, dtype=np.float64))
    f = np.asarray(f, dtype=np.float64)
    return Problem(name, H, A, f[:, None] if f.ndim == 1 else f,
                   dict(N=N, J=J, coefficient="given per element"))


def lshape_anisotropic(refinements: int = 7, batch: int = 16, seed: int = 0,
                       eps: float = 1e-3, angle: float = 30.0) -> Problem:
    H = meshes.lshape_hierarchy(refinements, 8, 0.2, seed)
    K = fields.rotated_anisotropy(eps, angle)
    A = fields.assemble_p1(H.levels[0], K=K)
    n = H.levels[0].interior.size
    return Problem(f"lshape_r{refinements}", H, A, fields.rhs(n, batch, seed),
                   dict(refinements=refinements, J=H.J, batch=batch, seed=seed,
                        coefficient=f"anisotropic diag(1,{eps}) rotated {angle} deg"))


def helmholtz_square(N: int = 33, J: int = 3, k: float = 2 * np.pi, batch: int = 1,
                     seed: int = 0) -> Problem:
    """Helmholtz with the impedance boundary condition (Sec. 4.2) on uniform
    meshes of [-1/2, 1/2]^2.  The impedance condition keeps every vertex a
    DOF (no Dirichlet boundary).  A_full is complex symmetric:
    K - k^2 M - i k B with the P1 stiffness, mass and boundary-edge mass."""
    H = meshes.square_hierarchy(N, J)
    for L in H.levels:
        L.xy = L.xy - 0.5
        L.boundary = np.zeros(L.nv, dtype=bool)
    L0 = H.levels[0]
    A = (fields.assemble_p1(L0).astype(np.complex128) - k * k * fields.assemble_mass_p1(L0)
         - 1j * k * fields.assemble_boundary_mass_p1(L0)).tocsr()
    A.sort_indices()
    M = fields.assemble_mass_p1(L0)
    f = np.zeros((L0.nv, batch), dtype=np.complex128)
    f[:, 0] = M @ fields.disk_source(L0.xy, [(0.0, 0.0)])
    if batch > 1:
        r = meshes._rng(seed, 1)
        f[:, 1:] = r.standard_normal((L0.nv, batch - 1)) + 1j * r.standard_normal((L0.nv, batch - 1))
    return Problem(f"helmholtz_{N}", H, A, f,
                   dict(N=N, J=J, batch=batch, seed=seed, wave_number=k,
                        coefficient="Helmholtz, impedance boundary"))
