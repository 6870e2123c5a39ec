"""Continuous-batching solve server.

Requests (a size class, an operator of that class, a right-hand side) arrive
over time.  Each resident operator is one libmg context with S right-hand-side
slots; a slot holds one request's f and iterate u as a column of X[n][S].  One
worker thread and one CUDA stream per size class loops:

  1. admit waiting requests into free slots of their operator's context (a
     new context is created only if the device budget allows it, else the
     request waits and idle contexts are evicted);
  2. tick: run `iters_per_tick` FP64-refinement iterations (FP32 learned
     V-cycles) on every context that has occupied slots (mg_solve with a
     small max_iter, warm-started from the slot's iterate);
  3. retire the slots whose relative residual met the tolerance.

Requests join and leave a batch between iterations while other requests of
the same context keep iterating, and the size classes' streams run
concurrently on the device.  Every column is computed by the same arithmetic
whatever the batch holds, and re-starting a solve rescales the FP32 residual
by an exact power of two, so a request's result in the mix equals its result
when solved alone.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np
import torch

from .hierarchy import Hierarchy
from .solver import LMGParams, Solver


@dataclass
class Request:
    rid: int
    klass: int            # mesh size N (N x N nodes)
    op: int               # operator index within the class pool
    src: int              # source index within the class pool
    t_arrival: float = 0.0
    t_admit: float = -1.0
    t_done: float = -1.0
    iters: int = 0
    relres: float = float("nan")
    u: np.ndarray | None = None


class OperatorContext:
    """One resident operator with S right-hand-side slots."""

    def __init__(self, key, hier: Hierarchy, params: LMGParams, slots: int, device, nbytes: int):
        self.key = key
        self.solver = Solver(hier, params.with_levels(hier.J), precision=32, max_batch=slots,
                             device=device)
        n = hier.sizes[0]
        self.n = n
        self.S = slots
        self.f = torch.zeros((n, slots), dtype=torch.float64, device=device)
        self.u = torch.zeros((n, slots), dtype=torch.float64, device=device)
        self.req: list[Request | None] = [None] * slots
        self.bytes = nbytes
        self.last_used = time.perf_counter()

    @property
    def busy(self) -> int:
        return sum(r is not None for r in self.req)

    def free_slot(self) -> int:
        for k, r in enumerate(self.req):
            if r is None:
                return k
        return -1

    def close(self):
        self.solver.close()


class ClassWorker(threading.Thread):
    """Serves one size class on its own CUDA stream; only this thread touches
    the contexts of its class while it runs."""

    def __init__(self, server: "Server", klass: int):
        super().__init__(daemon=True)
        self.server = server
        self.klass = klass
        self.queue: deque[Request] = deque()
        self.lock = threading.Lock()
        # the smaller half of the size classes gets a high-priority stream, so
        # their short kernels are scheduled ahead of the large classes' full-
        # GPU kernels instead of queueing behind them (latency of small
        # requests); priorities change scheduling only, never results
        small = klass <= server.classes[(len(server.classes) - 1) // 2]
        self.stream = torch.cuda.Stream(device=server.device, priority=-1 if small else 0)
        self.stop = False
        self.error: BaseException | None = None

    def submit(self, r: Request):
        with self.lock:
            self.queue.append(r)

    def _evict_idle(self, older_than: float = 0.0):
        S = self.server
        now = time.perf_counter()
        for key, c in list(S.contexts[self.klass].items()):
            if c.busy == 0 and now - c.last_used >= older_than:
                S.drop(self.klass, key)

    def _context_for(self, op: int) -> OperatorContext | None:
        S = self.server
        key = (self.klass, op)
        ctx = S.contexts[self.klass].get(key)
        if ctx is not None:
            S.contexts[self.klass].move_to_end(key)
            return ctx
        if not S.reserve(S.need[key]):
            self._evict_idle()
            if not S.reserve(S.need[key]):
                S.pressure = True
                return None
        return S.create(key)

    def _admit(self):
        S = self.server
        with self.lock:
            waiting = list(self.queue)
            self.queue.clear()
        keep = []
        for r in waiting:
            ctx = self._context_for(r.op)
            slot = ctx.free_slot() if ctx is not None else -1
            if slot < 0:
                keep.append(r)
                continue
            ctx.req[slot] = r
            ctx.f[:, slot].copy_(S.sources[(self.klass, r.src)])
            ctx.u[:, slot].zero_()
            r.t_admit = time.perf_counter()
        if keep:
            with self.lock:
                self.queue.extendleft(reversed(keep))

    def _tick(self):
        S = self.server
        for ctx in list(S.contexts[self.klass].values()):
            if ctx.busy == 0:
                continue
            _, info = ctx.solver.solve(ctx.f, ctx.u, tol=S.tol, max_iter=S.iters_per_tick)
            ctx.last_used = time.perf_counter()
            for k, r in enumerate(ctx.req):
                if r is None:
                    continue
                r.iters += int(info.iters[k])
                r.relres = float(info.relres[k])
                if r.relres < S.tol or r.iters >= S.max_iter:
                    if S.keep_results:
                        r.u = ctx.u[:, k].cpu().numpy()
                    else:
                        torch.cuda.current_stream().synchronize()
                    r.t_done = time.perf_counter()
                    ctx.req[k] = None
                    ctx.f[:, k].zero_()
                    ctx.u[:, k].zero_()
                    S.finish(r)

    def run(self):
        S = self.server
        try:
            with torch.cuda.device(S.device), torch.cuda.stream(self.stream):
                while True:
                    self._admit()
                    busy = any(c.busy for c in S.contexts[self.klass].values())
                    if busy:
                        self._tick()
                    else:
                        with self.lock:
                            empty = not self.queue
                        if self.stop and empty:
                            break
                        if not empty and not S.contexts[self.klass] and S.in_use == 0:
                            raise RuntimeError("device budget too small for one operator")
                        time.sleep(50e-6)
                    if S.pressure:  # another class is waiting for memory
                        self._evict_idle(older_than=S.idle_evict_s)
        except BaseException as e:  # surfaced by Server.run
            self.error = e


class Server:
    """Pools of operators per size class (resident contexts created on demand
    within a device-memory budget, or ahead of time by warm()), and one worker
    thread per class during run()."""

    def __init__(self, hierarchies: dict, sources: dict, params,
                 slots: int = 8, tol: float = 1e-8, iters_per_tick: int = 6,
                 max_iter: int = 400, budget_bytes: int | None = None, device=None,
                 keep_results: bool = False, idle_evict_s: float = 0.02):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.hierarchies = hierarchies          # (klass, op) -> Hierarchy
        self.sources = {k: torch.as_tensor(v, dtype=torch.float64).to(self.device)
                        for k, v in sources.items()}  # (klass, src) -> (n,) f
        self.params = params  # LMGParams, or {size class: LMGParams}
        self.slots = slots
        self.tol = tol
        self.iters_per_tick = iters_per_tick
        self.max_iter = max_iter
        free, total = torch.cuda.mem_get_info(self.device)
        self.budget = int(budget_bytes if budget_bytes is not None else 0.5 * free)
        self.in_use = 0
        self.peak = 0
        self.pressure = False
        self.idle_evict_s = idle_evict_s
        self.mem_lock = threading.Lock()
        self.done: list[Request] = []
        self.done_lock = threading.Lock()
        self.keep_results = keep_results
        self.classes = sorted({k for k, _ in hierarchies})
        self.contexts = {k: OrderedDict() for k in self.classes}
        # admission footprint of an operator context: library workspace plus
        # the slots' f and u columns
        self.need = {key: h.footprint_bytes(slots, 32) + 2 * h.sizes[0] * slots * 8
                     for key, h in hierarchies.items()}

    def reserve(self, nbytes: int) -> bool:
        with self.mem_lock:
            if self.in_use + nbytes > self.budget:
                return False
            self.in_use += nbytes
            self.peak = max(self.peak, self.in_use)
            return True

    def release(self, nbytes: int):
        with self.mem_lock:
            self.in_use -= nbytes
            self.pressure = False

    def create(self, key) -> OperatorContext:
        """Sets up a context whose bytes are already reserved."""
        prm = self.params[key[0]] if isinstance(self.params, dict) else self.params
        ctx = OperatorContext(key, self.hierarchies[key], prm, self.slots, self.device,
                              self.need[key])
        self.contexts[key[0]][key] = ctx
        return ctx

    def drop(self, klass, key):
        ctx = self.contexts[klass].pop(key)
        ctx.close()
        self.release(ctx.bytes)

    def warm(self, keys=None):
        """Creates contexts ahead of time (as many as the budget allows)."""
        for key in keys if keys is not None else self.hierarchies:
            if key not in self.contexts[key[0]] and self.reserve(self.need[key]):
                self.create(key)

    def close(self):
        for k in self.classes:
            for key in list(self.contexts[k]):
                self.drop(k, key)

    def finish(self, r: Request):
        with self.done_lock:
            self.done.append(r)

    def run(self, requests: list[Request], t0: float | None = None) -> list[Request]:
        """Replays requests at their arrival times (seconds from t0) and
        returns them completed, in request order."""
        self.done = []
        workers = {k: ClassWorker(self, k) for k in self.classes}
        for w in workers.values():
            w.start()
        t0 = time.perf_counter() if t0 is None else t0
        for r in sorted(requests, key=lambda q: q.t_arrival):
            delay = t0 + r.t_arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            r.t_arrival = t0 + r.t_arrival
            workers[r.klass].submit(r)
        for w in workers.values():
            w.stop = True
        for w in workers.values():
            w.join()
        for w in workers.values():
            if w.error is not None:
                raise w.error
        return sorted(self.done, key=lambda q: q.rid)


# ------------------------------------------------------------- workload ----

def make_pools(classes, ops_per_class: int, srcs_per_class: int, seed: int = 0):
    """Seeded lognormal operators (sigma 1.5, correlation 0.1) and N(0,1)
    sources for each size class N in classes."""
    import workloads as W
    from workloads import fields
    hier, src, probs = {}, {}, {}
    for N in classes:
        for op in range(ops_per_class):
            p = W.lognormal_square(N, seed=seed * 1000 + op + 17 * N, batch=1)
            hier[(N, op)] = Hierarchy.from_problem(p)
            probs[(N, op)] = p
        n = hier[(N, 0)].sizes[0]
        for s in range(srcs_per_class):
            src[(N, s)] = fields.rhs(n, 1, seed * 1000 + 500 + s + 17 * N)[:, 0]
    return hier, src, probs


def poisson_requests(rate: float, duration: float, classes, ops_per_class: int,
                     srcs_per_class: int, seed: int = 0) -> list[Request]:
    """Poisson arrivals (exponential gaps) of uniformly drawn classes,
    operators and sources."""
    r = np.random.default_rng([seed, 4])
    t, out, k = 0.0, [], 0
    while True:
        t += r.exponential(1.0 / rate)
        if t > duration:
            break
        out.append(Request(k, int(classes[r.integers(len(classes))]),
                           int(r.integers(ops_per_class)), int(r.integers(srcs_per_class)), t))
        k += 1
    return out


def summarize(done: list[Request], wall: float) -> dict:
    lat = np.array([r.t_done - r.t_arrival for r in done]) * 1e3
    per = {}
    for N in sorted({r.klass for r in done}):
        l = np.array([r.t_done - r.t_arrival for r in done if r.klass == N]) * 1e3
        it = np.array([r.iters for r in done if r.klass == N])
        per[str(N)] = {"n": int(l.size), "p50_ms": round(float(np.percentile(l, 50)), 3),
                       "p99_ms": round(float(np.percentile(l, 99)), 3),
                       "mean_iters": round(float(it.mean()), 2)}
    return {"solves": len(done), "solves_per_s": round(len(done) / wall, 2),
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_relres": float(max(r.relres for r in done)), "per_class": per}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=5.0)
    ap.add_argument("--classes", default="65,129,257,513,1025")
    ap.add_argument("--ops", type=int, default=2)
    ap.add_argument("--srcs", type=int, default=4)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--iters-per-tick", type=int, default=6)
    ap.add_argument("--params", default=None,
                    help="parameter set of every class (default: the package's trained set)")
    ap.add_argument("--class-params", default=None,
                    help="per-class sets N=path[,N=path]; default: the 1025^2 class uses the "
                         "set trained on a 1025^2 lognormal operator")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    from . import trained
    classes = [int(x) for x in a.classes.split(",")]
    t_setup = time.perf_counter()
    hier, src, _ = make_pools(classes, a.ops, a.srcs, a.seed)
    base = trained.load(a.params, max(h.J for h in hier.values()))
    spec = a.class_params
    if spec is None and os.path.exists(trained.LOGNORMAL1025):
        spec = f"1025={trained.LOGNORMAL1025}"
    over = dict((int(k), v) for k, v in (x.split("=", 1) for x in spec.split(","))) if spec else {}
    params = {k: trained.read(over[k]) if k in over else base for k in classes}
    t_setup = time.perf_counter() - t_setup
    reqs = poisson_requests(a.rate, a.duration, classes, a.ops, a.srcs, a.seed)
    srv = Server(hier, src, params, slots=a.slots, iters_per_tick=a.iters_per_tick)
    srv.warm()
    # warm-up: one request per operator (captures the solve graphs), not timed
    srv.run([Request(-1 - i, k[0], k[1], 0, 0.0) for i, k in enumerate(hier)])
    t0 = time.perf_counter()
    done = srv.run(reqs, t0)
    wall = time.perf_counter() - t0
    srv.close()
    out = {"metric": "continuous-batching solves to 1e-8 (learned FP32 V-cycle + FP64 refinement)",
           "offered_rate_per_s": a.rate, "duration_s": a.duration, "classes": classes,
           "operators_per_class": a.ops, "slots": a.slots, "iters_per_tick": a.iters_per_tick,
           "wall_s": round(wall, 3), "setup_s": round(t_setup, 2),
           "peak_device_bytes": srv.peak, "budget_bytes": srv.budget,
           "params": {str(k): os.path.basename(over[k]) if k in over else
                      trained.describe(a.params).split(":")[0] for k in classes}}
    out.update(summarize(done, wall))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
