"""Host-side training logic (no GPU): parameter sharing maps and Rprop."""
import numpy as np
import torch

from paper_2608_29082_b300.solver import LMGParams
from paper_2608_29082_b300.training import ParamMap, Rprop


def test_parammap_roundtrip_and_shared_gradient():
    J = 5
    pm = ParamMap(J, shared=("wB1", "wB2", "wR1", "wR2", "wP1", "wP2"))
    assert pm.size == 2 * (J - 1) + 6
    p = LMGParams.identity(J)
    flat = p.flat()
    z = pm.gather(flat)
    assert np.array_equal(pm.scatter(z, flat), flat)
    g = np.arange((J - 1) * 8, dtype=float)
    gz = pm.reduce_grad(g)
    gm = g.reshape(J - 1, 8)
    # shared wR2 (column 5) sums over levels; per-level theta keeps each level
    assert gz[pm.index[0, 5]] == gm[:, 5].sum()
    assert np.array_equal(gz[pm.index[:, 0]], gm[:, 0])


def test_parammap_frozen_columns():
    J = 4
    pm = ParamMap(J, train=("wR1", "wR2", "wP1", "wP2"), shared=("wR1", "wR2", "wP1", "wP2"))
    assert pm.size == 4
    flat = LMGParams.identity(J).flat()
    z = pm.gather(flat) + 1.0
    out = pm.scatter(z, flat).reshape(J - 1, 8)
    assert np.all(out[:, 0] == 2.0 / 3.0)        # theta frozen
    assert np.all(out[:, 4] == 2.0)              # wR1 shared and moved


def test_rprop_matches_torch_rprop():
    """Same update rule as torch.optim.Rprop (lr 0.01, etas (0.5, 1.2))."""
    r = np.random.default_rng(0)
    x0 = r.standard_normal(7)
    grads = [r.standard_normal(7) for _ in range(12)]
    mine = Rprop(7, lr=0.01)
    z = x0.copy()
    t = torch.tensor(x0, requires_grad=True)
    opt = torch.optim.Rprop([t], lr=0.01, etas=(0.5, 1.2), step_sizes=(1e-6, 50.0))
    for g in grads:
        z = mine.update(z, g)
        opt.zero_grad()
        t.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(z, t.detach().numpy(), rtol=0, atol=1e-14)
