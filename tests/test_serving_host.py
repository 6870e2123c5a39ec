"""Host logic of the continuous-batching server, without a GPU.

The server's budget accounting, admission into free slots of a class's
stacked contexts, creation of contexts within the budget and eviction of
idle ones under memory pressure are plain host code.  These tests build
Server / ClassWorker / BatchContext objects without their CUDA constructors
(a fake stacked batch that records its set-up calls, CPU tensors) and drive
the real methods.
"""
import threading
import time
from collections import OrderedDict, deque

import numpy as np
import torch

from paper_2608_29082_b300.serve import BatchContext, ClassWorker, Request, Server, batch_footprint
from paper_2608_29082_b300.solver import SolveInfo


class FakeBatch:
    def __init__(self):
        self.closed = False
        self.blocks = []

    def set_block(self, k, ke):
        self.blocks.append((k, float(ke[0])))

    def close(self):
        self.closed = True


def fake_server(budget, need, slots=1, m=4, klass=65):
    S = object.__new__(Server)
    S.budget, S.in_use, S.peak, S.pressure = budget, 0, 0, False
    S.mem_lock = threading.Lock()
    S.classes = [klass]
    S.contexts = {klass: OrderedDict()}
    S.need = need
    S.slots = {klass: slots}
    S.idle_evict_s = 0.0
    S.coefs = {(klass, c): torch.full((6,), float(10 + c), dtype=torch.float64)
               for c in range(4)}
    S.sources = {(klass, s): torch.full((m,), float(s + 1), dtype=torch.float64)
                 for s in range(4)}
    S.done, S.done_lock = [], threading.Lock()
    S._serial = 0
    S.grow = True
    created = []

    def create(k):
        ctx = object.__new__(BatchContext)
        ctx.klass, ctx.S, ctx.m = k, slots, m
        ctx.f = torch.zeros(slots * m, dtype=torch.float64)
        ctx.u = torch.ones(slots * m, dtype=torch.float64)
        ctx.ke = torch.zeros(6, dtype=torch.float64)
        ctx.req = [None] * slots
        ctx.bytes = need[k]
        ctx.last_used = time.perf_counter()
        ctx.batch = FakeBatch()
        S._serial += 1
        S.contexts[k][(k, S._serial)] = ctx
        created.append((k, S._serial))
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


def test_admission_builds_each_request_operator_in_its_slot():
    """Every admitted request gets its own block: its coefficients are staged
    and written into that block (one set-up call per request), its source
    fills the block of f and its iterate starts at zero."""
    S, created = fake_server(budget=100, need={65: 40}, slots=3)
    w = fake_worker(S)
    reqs = [Request(rid=i, klass=65, coef=i, src=i) for i in range(3)]
    for r in reqs:
        w.submit(r)
    w._admit()
    assert created == [(65, 1)]
    ctx = S.contexts[65][(65, 1)]
    assert ctx.req == reqs
    assert ctx.batch.blocks == [(0, 10.0), (1, 11.0), (2, 12.0)]
    for k in range(3):
        assert torch.all(ctx.block(ctx.f, k) == float(k + 1))
        assert torch.all(ctx.block(ctx.u, k) == 0)
        assert reqs[k].t_admit > 0


def test_full_context_opens_another_then_waits_then_reuses_the_freed_slot():
    """One slot per context, two contexts fit the budget.  A third request
    waits (and flags memory pressure) while both are busy; once one request
    finishes, the waiting request takes the freed slot of that resident
    context: no new context, no eviction."""
    S, created = fake_server(budget=80, need={65: 40}, slots=1)
    w = fake_worker(S)
    reqs = [Request(rid=i, klass=65, coef=i, src=i) for i in range(3)]
    for r in reqs:
        w.submit(r)
    w._admit()
    assert created == [(65, 1), (65, 2)]
    assert list(w.queue) == [reqs[2]] and S.pressure and S.in_use == 80
    c1 = S.contexts[65][(65, 1)]
    c1.req[0] = None          # request 0 finishes
    w._admit()
    assert created == [(65, 1), (65, 2)]
    assert c1.req[0] is reqs[2] and not w.queue and not c1.batch.closed
    assert c1.batch.blocks[-1] == (0, 12.0)


def test_memory_pressure_evicts_an_idle_context_of_another_class():
    """Class 129 cannot reserve a context while an idle class-65 context holds
    the budget: it flags pressure, the class-65 worker evicts its idle
    context (as its loop does under pressure), and the class-129 request is
    admitted."""
    S, created = fake_server(budget=60, need={65: 40, 129: 50}, slots=1)
    S.classes = [65, 129]
    S.contexts[129] = OrderedDict()
    S.slots[129] = 1
    S.coefs.update({(129, 0): torch.full((6,), 7.0, dtype=torch.float64)})
    S.sources.update({(129, 0): torch.full((4,), 9.0, dtype=torch.float64)})
    w65, w129 = fake_worker(S, 65), fake_worker(S, 129)
    a = Request(rid=0, klass=65, coef=0, src=0)
    w65.submit(a)
    w65._admit()
    S.contexts[65][(65, 1)].req[0] = None     # a finished: idle context
    b = Request(rid=1, klass=129, coef=0, src=0)
    w129.submit(b)
    w129._admit()
    assert list(w129.queue) == [b] and S.pressure and S.in_use == 40
    w65._evict_idle(older_than=0.0)
    assert not S.contexts[65] and S.in_use == 0 and not S.pressure
    w129._admit()
    assert not w129.queue and S.in_use == 50
    assert created == [(65, 1), (129, 2)]


def test_free_slot_of_a_resident_context_is_reused_first():
    S, created = fake_server(budget=100, need={65: 10}, slots=2)
    w = fake_worker(S)
    a, b, c = (Request(rid=i, klass=65, coef=i, src=0) for i in range(3))
    for r in (a, b):
        w.submit(r)
    w._admit()
    ctx = S.contexts[65][(65, 1)]
    ctx.req[0] = None          # a finishes
    w.submit(c)
    w._admit()
    assert created == [(65, 1)]               # no new context
    assert ctx.req == [c, b]
    assert ctx.batch.blocks[-1] == (0, 12.0)  # c's own operator in slot 0


def test_without_growth_a_full_class_waits_for_a_slot():
    """With growth off (contexts warmed ahead of time) a class whose contexts
    are full queues its requests even while the budget has room."""
    S, created = fake_server(budget=1000, need={65: 40}, slots=1)
    S.grow = False
    w = fake_worker(S)
    rs = [Request(rid=i, klass=65, coef=0, src=0) for i in range(2)]
    for r in rs:
        w.submit(r)
    w._admit()
    assert created == [(65, 1)]               # the class had no context yet
    assert list(w.queue) == rs[1:] and S.in_use == 40


def test_waiting_requests_keep_their_order():
    """Requests that cannot be admitted go back to the head of the queue in
    arrival order, ahead of later submissions."""
    S, _ = fake_server(budget=50, need={65: 50}, slots=1)
    w = fake_worker(S)
    rs = [Request(rid=i, klass=65, coef=0, src=0) for i in range(4)]
    for r in rs[:3]:
        w.submit(r)
    w._admit()
    assert list(w.queue) == rs[1:3]
    w.submit(rs[3])
    w._admit()                                # the slot is still busy
    assert list(w.queue) == rs[1:4]


def test_footprint_grows_with_slots_and_size():
    assert batch_footprint(129, 8, 32) > batch_footprint(65, 8, 32) > 0
    assert batch_footprint(65, 16, 32) > batch_footprint(65, 8, 32)


def test_tick_iterates_the_leading_blocks_up_to_the_last_occupied_slot():
    """Admission fills the lowest free slot; a tick passes the count of
    leading blocks up to the last occupied slot (holes below it included)."""
    S, _ = fake_server(budget=100, need={65: 10}, slots=4)
    w = fake_worker(S)
    rs = [Request(rid=i, klass=65, coef=0, src=0) for i in range(3)]
    for r in rs:
        w.submit(r)
    w._admit()
    ctx = S.contexts[65][(65, 1)]
    assert ctx.lead == 3
    seen = []

    def solve(f, u, tol, max_iter, nblocks):
        seen.append(nblocks)
        it = np.zeros(4, dtype=np.int32)
        it[:nblocks] = 1
        rr = np.zeros(4)
        rr[:nblocks] = 1.0
        return SolveInfo(1, it, rr)

    ctx.batch.solve = solve
    S.tol, S.max_iter, S.iters_per_tick, S.keep_results = 1e-8, 100, 1, False
    ctx.req[2] = None                     # the last request leaves
    assert ctx.lead == 2
    ctx.req[0] = None                     # a hole below the last occupied slot
    assert ctx.lead == 2 and ctx.busy == 1
    w._tick()
    assert seen == [2] and rs[1].iters == 1
    ctx.req[1] = None
    assert ctx.lead == 0


def test_tick_block_counts_are_multiples_of_an_eighth():
    """A tick's block count is the lead rounded up to a multiple of S / 8
    (at most 8 solve graphs per context), and capture builds exactly those."""
    S, _ = fake_server(budget=1000, need={65: 10}, slots=64)
    ctx = S.create(65)
    calls = []
    ctx.batch.solve = lambda f, u, tol, max_iter, nblocks: calls.append(nblocks)
    for lead, want in ((1, 8), (8, 8), (9, 16), (63, 64), (64, 64)):
        ctx.req = [None] * 64
        ctx.req[lead - 1] = object()
        assert ctx.tick_blocks == want, (lead, ctx.tick_blocks)
    ctx.capture()
    assert calls == [8, 16, 24, 32, 40, 48, 56, 64]
    S4, _ = fake_server(budget=1000, need={65: 10}, slots=4)
    c4 = S4.create(65)
    c4.req = [None, None, object(), None]
    assert c4.quantum == 1 and c4.tick_blocks == 3

