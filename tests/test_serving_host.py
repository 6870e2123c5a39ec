"""Host logic of the continuous-batching server, without a GPU.

The server's budget accounting, context reuse (LRU), eviction of idle
contexts under memory pressure and admission into free slots are plain
host code.  These tests build Server / ClassWorker / OperatorContext objects
without their CUDA constructors (a fake solver, CPU tensors) and drive the
real methods.
"""
import threading
import time
from collections import OrderedDict, deque

import torch

from paper_2608_29082_b300.serve import ClassWorker, OperatorContext, Request, Server


class FakeSolver:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def fake_server(budget, need, slots=1, n=4, klass=65):
    S = object.__new__(Server)
    S.budget, S.in_use, S.peak, S.pressure = budget, 0, 0, False
    S.mem_lock = threading.Lock()
    S.classes = [klass]
    S.contexts = {klass: OrderedDict()}
    S.need = need
    S.slots = slots
    S.idle_evict_s = 0.0
    S.sources = {(klass, s): torch.full((n,), float(s + 1), dtype=torch.float64)
                 for s in range(4)}
    S.done, S.done_lock = [], threading.Lock()
    created = []

    def create(key):
        ctx = object.__new__(OperatorContext)
        ctx.key, ctx.S, ctx.n = key, slots, n
        ctx.f = torch.zeros((n, slots), dtype=torch.float64)
        ctx.u = torch.ones((n, slots), dtype=torch.float64)
        ctx.req = [None] * slots
        ctx.bytes = need[key]
        ctx.last_used = time.perf_counter()
        ctx.solver = FakeSolver()
        S.contexts[key[0]][key] = ctx
        created.append(key)
        return ctx

    S.create = create
    return S, created


def fake_worker(S, klass=65):
    w = object.__new__(ClassWorker)
    w.server, w.klass = S, klass
    w.queue, w.lock = deque(), threading.Lock()
    w.stop, w.error = False, None
    return w


def test_budget_accounting():
    S, _ = fake_server(budget=100, need={})
    assert S.reserve(60) and S.in_use == 60
    assert not S.reserve(50) and S.in_use == 60
    assert S.reserve(40) and S.in_use == 100 and S.peak == 100
    S.pressure = True
    S.release(60)
    assert S.in_use == 40 and not S.pressure and S.peak == 100


def test_admission_waits_then_evicts_an_idle_context():
    """Two contexts fit the budget.  A request for a third operator waits
    (and flags memory pressure) while both are busy; once one finishes, the
    idle context is evicted, its bytes released, and the request admitted
    into a fresh context with its source and a zero iterate."""
    need = {(65, op): 40 for op in range(3)}
    S, created = fake_server(budget=80, need=need)
    w = fake_worker(S)
    reqs = [Request(rid=i, klass=65, op=i, src=i) for i in range(3)]
    for r in reqs:
        w.submit(r)
    w._admit()
    assert created == [(65, 0), (65, 1)]
    assert list(w.queue) == [reqs[2]] and S.pressure and S.in_use == 80
    c0 = S.contexts[65][(65, 0)]
    assert c0.req[0] is reqs[0] and torch.equal(c0.f[:, 0], S.sources[(65, 0)])
    assert torch.all(c0.u[:, 0] == 0) and reqs[0].t_admit > 0
    # request 0 finishes: its context becomes idle and evictable
    c0.req[0] = None
    w._admit()
    assert created == [(65, 0), (65, 1), (65, 2)]
    assert (65, 0) not in S.contexts[65] and c0.solver.closed
    assert S.in_use == 80 and not w.queue
    assert S.contexts[65][(65, 2)].req[0] is reqs[2]


def test_resident_context_is_reused_and_moved_to_the_lru_end():
    need = {(65, op): 10 for op in range(2)}
    S, created = fake_server(budget=100, need=need, slots=2)
    w = fake_worker(S)
    a, b, c = (Request(rid=i, klass=65, op=op, src=0) for i, op in enumerate((0, 1, 0)))
    for r in (a, b):
        w.submit(r)
    w._admit()
    assert list(S.contexts[65]) == [(65, 0), (65, 1)]
    w.submit(c)
    w._admit()
    assert created == [(65, 0), (65, 1)]                 # no new context for op 0
    assert list(S.contexts[65]) == [(65, 1), (65, 0)]    # op 0 is now most recent
    assert S.contexts[65][(65, 0)].req == [a, c]


def test_waiting_requests_keep_their_order():
    """Requests that cannot be admitted go back to the head of the queue in
    arrival order, ahead of later submissions."""
    need = {(65, 0): 50}
    S, _ = fake_server(budget=50, need=need, slots=1)
    w = fake_worker(S)
    rs = [Request(rid=i, klass=65, op=0, src=0) for i in range(4)]
    for r in rs[:3]:
        w.submit(r)
    w._admit()
    assert list(w.queue) == rs[1:3]
    w.submit(rs[3])
    w._admit()                                           # the slot is still busy
    assert list(w.queue) == rs[1:4]
