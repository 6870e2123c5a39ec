"""Continuous-batching server with an operator per request: each result equals
the same system solved alone (bitwise), the oracle re-checks sampled results,
and admission respects the device budget."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2608_29082_b300 import LMGParams
from paper_2608_29082_b300.serve import Request, Server, make_pools, summarize
from paper_2608_29082_b300.square import SquareBatch

pytestmark = pytest.mark.gpu

CLASSES = [65, 129]


@pytest.fixture(scope="module")
def pools():
    coefs, src = make_pools(CLASSES, coefs_per_class=3, srcs_per_class=3, seed=5)
    p = LMGParams.identity(7)
    p.wB[:, 1] = 0.1   # exercise the graph convolutions
    p.wR[:, 1] = 0.05
    p.wP[:, 1] = -0.05
    return coefs, src, p


def requests(n, spacing=0.0005):
    return [Request(i, CLASSES[i % 2], (i // 2) % 3, i % 3, spacing * i) for i in range(n)]


def test_result_in_mix_equals_result_alone(pools):
    coefs, src, params = pools
    srv = Server(coefs, src, params, slots=4, iters_per_tick=2, keep_results=True)
    srv.warm()
    done = srv.run(requests(24))
    srv.close()
    assert len(done) == 24
    assert all(r.relres < 1e-8 for r in done)
    alone = {}
    for r in done:
        if r.klass not in alone:
            alone[r.klass] = SquareBatch(r.klass, 1, params, precision=32)
        A1 = alone[r.klass]
        A1.set_block(0, torch.tensor(coefs[(r.klass, r.coef)], dtype=torch.float64,
                                     device="cuda"))
        u = torch.zeros(A1.m, dtype=torch.float64, device="cuda")
        f = torch.tensor(src[(r.klass, r.src)], dtype=torch.float64, device="cuda")
        info = A1.solve(f, u, tol=1e-8, max_iter=400)
        assert int(info.iters[0]) == r.iters
        assert np.array_equal(u.cpu().numpy(), r.u)
    for A1 in alone.values():
        A1.close()


def test_oracle_rechecks_sampled_results(pools):
    coefs, src, params = pools
    srv = Server(coefs, src, params, slots=4, iters_per_tick=3, keep_results=True)
    done = srv.run(requests(8, spacing=0.0))
    srv.close()
    for r in done[:4]:
        p = W.square_with_coefficients(r.klass, coefs[(r.klass, r.coef)], src[(r.klass, r.src)])
        H = O.build_hierarchy(p)
        assert O.relres(H, p.f, r.u[:, None])[0] < 1e-8


def test_admission_respects_device_budget(pools):
    """A budget for a single two-slot context: ten requests of one class still
    all complete, the reserved bytes never exceed the budget."""
    coefs, src, params = pools
    c = {k: v for k, v in coefs.items() if k[0] == 65}
    s = {k: v for k, v in src.items() if k[0] == 65}
    probe = Server(c, s, params, slots=2)
    need = probe.need[65]
    srv = Server(c, s, params, slots=2, iters_per_tick=2, budget_bytes=need)
    reqs = [Request(i, 65, i % 3, i % 3, 0.0002 * i) for i in range(10)]
    done = srv.run(reqs)
    srv.close()
    assert len(done) == 10 and all(r.relres < 1e-8 for r in done)
    assert srv.peak <= need
    stats = summarize(done, 1.0)
    assert stats["solves"] == 10 and stats["p99_ms"] >= stats["p50_ms"]
