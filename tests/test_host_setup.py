"""Native host set-up (libmg.so helpers, no GPU) against the oracle's setup."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2608_29082_b300 import Hierarchy


def _cases():
    return [
        ("poisson33", lambda: W.poisson_square(33, 4)),
        ("checker65", lambda: W.checkerboard_square(65, 6, ncell=8, values=(1.0, 1e4), seed=3)),
        ("lognormal33", lambda: W.lognormal_square(33, seed=4)),
        ("lshape_r2", lambda: W.lshape_anisotropic(refinements=2, batch=1, seed=1)),
    ]


@pytest.mark.parametrize("name,make", _cases())
def test_hierarchy_matches_oracle(name, make):
    p = make()
    Ho = O.build_hierarchy(p)
    Hp = Hierarchy.from_problem(p)
    assert Hp.J == Ho.J
    for lev in range(Ho.J):
        Ao = Ho.levels[lev].A.toarray()
        Ap = Hp.A[lev].to_scipy().toarray()
        assert Ap.shape == Ao.shape
        assert np.abs(Ap - Ao).max() <= 1e-13 * np.abs(Ao).max(), lev
        # same graph: same pattern
        assert np.array_equal(Ap != 0, Ao != 0), lev
        assert np.allclose(Hp.inv_deg[lev], Ho.levels[lev].inv_deg, rtol=0, atol=0), lev
        if lev < Ho.J - 1:
            Po = Ho.levels[lev].P.toarray()
            Pp = Hp.P[lev].to_scipy().toarray()
            assert np.array_equal(Pp, Po), lev


def test_lshape_sizes():
    p = W.lshape_anisotropic(refinements=3, batch=1)
    Hp = Hierarchy.from_problem(p)
    assert Hp.sizes[-1] == 161
    # anisotropic rotated tensor couples along every mesh edge
    A0 = Hp.A[0].to_scipy()
    assert A0.getnnz(axis=1).max() >= 7


def test_footprint_positive():
    p = W.poisson_square(33, 4)
    Hp = Hierarchy.from_problem(p)
    b64 = Hp.footprint_bytes(4, 64)
    b32 = Hp.footprint_bytes(4, 32)
    assert b64 > 0 and b32 > 0


@pytest.mark.parametrize("N,J", [(17, 2), (33, 3)])
def test_complex_hierarchy_matches_oracle(N, J):
    """The two-feature path's host set-up (native Galerkin on the real and
    imaginary parts, merged, round-off dropped on complex magnitudes) gives
    the oracle's complex hierarchy: same patterns, degrees and P."""
    import oracle as O
    import workloads as W
    from paper_2608_29082_b300.features2 import Hierarchy2
    p = W.helmholtz_square(N, J, k=2 * np.pi, batch=1, seed=0)
    Ho, Hp = O.build_hierarchy(p), Hierarchy2.from_problem(p)
    assert Hp.J == Ho.J == J
    for lev in range(J):
        a, b = Ho.levels[lev].A, Hp.A[lev]
        assert ((a != 0) != (b != 0)).nnz == 0
        assert abs(a - b).max() <= 1e-15 * abs(a).max()
        assert np.array_equal(Ho.levels[lev].inv_deg, Hp.inv_deg[lev])
        if lev < J - 1:
            assert abs(Ho.levels[lev].P - Hp.P[lev]).max() == 0
