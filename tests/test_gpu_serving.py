"""Continuous-batching server: results equal solving alone, admission by
device budget, results re-checked by the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2608_29082_b300 import LMGParams, Solver
from paper_2608_29082_b300.serve import Request, Server, make_pools, summarize

pytestmark = pytest.mark.gpu

CLASSES = [65, 129]


@pytest.fixture(scope="module")
def pools():
    hier, src, probs = make_pools(CLASSES, ops_per_class=2, srcs_per_class=3, seed=5)
    J = max(h.J for h in hier.values())
    p = LMGParams.identity(J)
    p.wB[:, 1] = 0.1   # exercise the graph convolutions
    p.wR[:, 1] = 0.05
    p.wP[:, 1] = -0.05
    return hier, src, probs, p


def requests(n, spacing=0.0005):
    return [Request(i, CLASSES[i % 2], (i // 2) % 2, i % 3, spacing * i) for i in range(n)]


def test_result_in_mix_equals_result_alone(pools):
    hier, src, probs, params = pools
    srv = Server(hier, src, params, slots=4, iters_per_tick=2, keep_results=True)
    srv.warm()
    done = srv.run(requests(24))
    srv.close()
    assert len(done) == 24
    assert all(r.relres < 1e-8 for r in done)
    alone = {}
    for r in done:
        key = (r.klass, r.op)
        if key not in alone:
            alone[key] = Solver(hier[key], params.with_levels(hier[key].J), precision=32,
                                max_batch=1)
        f = torch.tensor(src[(r.klass, r.src)][:, None], dtype=torch.float64, device="cuda")
        u, info = alone[key].solve(f, tol=1e-8, max_iter=400)
        assert int(info.iters[0]) == r.iters
        assert np.array_equal(u[:, 0].cpu().numpy(), r.u)
    for S in alone.values():
        S.close()


def test_oracle_rechecks_sampled_results(pools):
    hier, src, probs, params = pools
    srv = Server(hier, src, params, slots=4, iters_per_tick=3, keep_results=True)
    done = srv.run(requests(8, spacing=0.0))
    srv.close()
    for r in done[:4]:
        H = O.build_hierarchy(probs[(r.klass, r.op)])
        f = src[(r.klass, r.src)][:, None]
        assert O.relres(H, f, r.u[:, None])[0] < 1e-8


def test_admission_respects_device_budget(pools):
    """A budget for a single operator context: requests for two operators of
    one class still all complete, contexts are swapped as they go idle, and
    the reserved bytes never exceed the budget."""
    hier, src, probs, params = pools
    h = {k: v for k, v in hier.items() if k[0] == 65}
    s = {k: v for k, v in src.items() if k[0] == 65}
    probe = Server(h, s, params, slots=2)
    need = max(probe.need.values())
    srv = Server(h, s, params, slots=2, iters_per_tick=2, budget_bytes=need)
    reqs = [Request(i, 65, i % 2, i % 3, 0.0002 * i) for i in range(10)]
    done = srv.run(reqs)
    srv.close()
    assert len(done) == 10 and all(r.relres < 1e-8 for r in done)
    assert srv.peak <= need
    stats = summarize(done, 1.0)
    assert stats["solves"] == 10 and stats["p99_ms"] >= stats["p50_ms"]
