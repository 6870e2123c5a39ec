"""Continuous-batching solve server with an operator per request.

Every request brings its own system: a size class N (an N x N right-triangle
mesh of the unit square), its element coefficients k and its source f.  The
server keeps, per size class, stacked contexts (square.SquareBatch) of S
slots each; a slot is one block of the stack, i.e. one request's operator on
every level of the hierarchy.  One worker thread and one CUDA stream per
size class loops:

  1. admit waiting requests into free slots: copy the request's coefficients
     and source to the device, build its operator in the slot's block on the
     GPU (P1 assembly, Galerkin coarsening, degrees, coarsest inverse:
     mg_square_set_block) and clear the slot's iterate.  A new context is
     created only while the device budget allows it; under memory pressure
     idle contexts (of any class) are evicted;
  2. tick: one mg_solve_blocks call per context with occupied slots (over its
     leading blocks up to the last occupied one, rounded up to a multiple of
     an eighth of the context; admission fills the lowest free slot) runs
     `iters_per_tick` FP64-refinement iterations (FP32 learned V-cycles) on
     all of its requests at once, each block masked and tested on its own;
  3. retire the slots whose relative residual met the tolerance.

So a request's latency contains its upload, its operator set-up and its
iterations.  Requests join and leave a stack between iterations while the
other blocks keep iterating, and the size classes' streams run concurrently
on the device.  A block's arithmetic never reads another block, and
restarting a solve rescales its FP32 residual by an exact power of two, so a
request's result in the mix equals its result solved alone.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass

import numpy as np
import torch

from .solver import LMGParams
from .square import SquareBatch, levels_for


@dataclass
class Request:
    rid: int
    klass: int            # mesh size N (N x N vertices)
    coef: int             # coefficient field within the class pool
    src: int              # source within the class pool
    t_arrival: float = 0.0
    t_admit: float = -1.0
    t_done: float = -1.0
    iters: int = 0
    relres: float = float("nan")
    u: np.ndarray | None = None


def batch_footprint(N: int, slots: int, precision: int) -> int:
    """Device bytes of a stacked context (an upper estimate): per level the
    DIA values (at most 6 diagonals), diagonal, 1/diagonal, 1/degree and four
    work vectors in the context precision, transfer lists, the FP64 finest
    copy and refinement vectors, the set-up scratch (7-point stencils over all
    vertices), plus the server's f, u stacks and coefficient staging."""
    b = 4 if precision == 32 else 8
    total, n = 0, N
    while True:
        m = (n - 2) ** 2 * slots
        total += m * (6 + 3 + 4) * b + m * 2 * (4 + b) * 2 + n * n * 7 * 8
        if n <= 3:
            break
        n = (n - 1) // 2 + 1
    m0 = (N - 2) ** 2 * slots
    total += m0 * (6 + 2) * 8 + m0 * 3 * 8 + m0 * 2 * 4 + slots * slots * 8
    total += 2 * m0 * 8 + 2 * (N - 1) ** 2 * 8
    return int(total * 1.1) + (1 << 20)


class BatchContext:
    """One stacked context of a size class, its slots and device stacks."""

    def __init__(self, klass: int, slots: int, params: LMGParams, device, nbytes: int):
        self.klass = klass
        self.batch = SquareBatch(klass, slots, params, precision=32, device=device)
        self.m = self.batch.m
        self.S = slots
        self.f = torch.zeros(slots * self.m, dtype=torch.float64, device=device)
        self.u = torch.zeros(slots * self.m, dtype=torch.float64, device=device)
        self.ke = torch.empty(self.batch.n_elements, dtype=torch.float64, device=device)
        self.req: list[Request | None] = [None] * slots
        self.bytes = nbytes
        self.last_used = time.perf_counter()

    @property
    def busy(self) -> int:
        return sum(r is not None for r in self.req)

    def free_slot(self) -> int:
        """The lowest free slot: occupied slots stay packed towards the front,
        so a tick iterates the leading blocks only (lead)."""
        for k, r in enumerate(self.req):
            if r is None:
                return k
        return -1

    @property
    def lead(self) -> int:
        """Leading blocks up to the last occupied slot."""
        for k in range(self.S - 1, -1, -1):
            if self.req[k] is not None:
                return k + 1
        return 0

    @property
    def quantum(self) -> int:
        return max(1, self.S // 8)

    @property
    def tick_blocks(self) -> int:
        """Blocks a tick iterates: lead rounded up to a multiple of S / 8, so
        that a context uses at most 8 solve graphs (one per block count)."""
        q = self.quantum
        return min(self.S, -(-self.lead // q) * q)

    def capture(self):
        """Builds the solve graph of every block count a tick can use (on the
        context's zero stacks: every block idle, no iterations)."""
        for k in range(self.quantum, self.S + 1, self.quantum):
            self.batch.solve(self.f, self.u, tol=1e-8, max_iter=1, nblocks=k)

    def block(self, x: torch.Tensor, k: int) -> torch.Tensor:
        return x[k * self.m:(k + 1) * self.m]

    def close(self):
        self.batch.close()


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

    def _slot(self) -> tuple[BatchContext | None, int]:
        """A context of this class with a free slot (a new one if the budget
        allows), most recently used first."""
        S = self.server
        for key in reversed(S.contexts[self.klass]):
            ctx = S.contexts[self.klass][key]
            k = ctx.free_slot()
            if k >= 0:
                S.contexts[self.klass].move_to_end(key)
                return ctx, k
        if S.contexts[self.klass] and not S.grow:
            return None, -1  # wait for a slot of the resident contexts
        need = S.need[self.klass]
        if not S.reserve(need):
            self._evict_idle()
            if not S.reserve(need):
                S.pressure = True
                return None, -1
        ctx = S.create(self.klass)
        return ctx, ctx.free_slot()

    def _admit(self):
        S = self.server
        with self.lock:
            waiting = list(self.queue)
            self.queue.clear()
        keep = []
        for r in waiting:
            ctx, k = self._slot()
            if ctx is None:
                keep.append(r)
                continue
            ctx.req[k] = r
            r.t_admit = time.perf_counter()
            # the request's data to the device, its operator into block k
            ctx.ke.copy_(S.coefs[(self.klass, r.coef)], non_blocking=True)
            ctx.batch.set_block(k, ctx.ke)
            ctx.block(ctx.f, k).copy_(S.sources[(self.klass, r.src)], non_blocking=True)
            ctx.block(ctx.u, k).zero_()
        if keep:
            with self.lock:
                self.queue.extendleft(reversed(keep))

    def _tick(self):
        S = self.server
        for ctx in list(S.contexts[self.klass].values()):
            if ctx.busy == 0:
                continue
            info = ctx.batch.solve(ctx.f, ctx.u, tol=S.tol, max_iter=S.iters_per_tick,
                                   nblocks=ctx.tick_blocks)
            ctx.last_used = time.perf_counter()
            for k, r in enumerate(ctx.req):
                if r is None:
                    continue
                r.iters += int(info.iters[k])
                r.relres = float(info.relres[k])
                if r.relres < S.tol or r.iters >= S.max_iter:
                    if S.keep_results:
                        r.u = ctx.block(ctx.u, k).cpu().numpy()
                    r.t_done = time.perf_counter()
                    ctx.req[k] = None
                    ctx.block(ctx.f, k).zero_()  # idle block: no iterations
                    ctx.block(ctx.u, k).zero_()
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
                            raise RuntimeError("device budget too small for one context")
                        time.sleep(50e-6)
                    if S.pressure:  # another class is waiting for memory
                        self._evict_idle(older_than=S.idle_evict_s)
        except BaseException as e:  # surfaced by Server.run
            self.error = e


class Server:
    """Stacked contexts per size class (created on demand within a device
    memory budget, or ahead of time by warm()), and one worker thread per
    class during run().  coefs[(N, i)] and sources[(N, j)] are the pools the
    requests draw their data from (host arrays, pinned for the uploads)."""

    def __init__(self, coefs: dict, sources: dict, params, slots=8, tol: float = 1e-8,
                 iters_per_tick: int = 6, max_iter: int = 400, budget_bytes: int | None = None,
                 device=None, keep_results: bool = False, idle_evict_s: float = 0.02,
                 grow: bool = True):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.coefs = {k: torch.as_tensor(v, dtype=torch.float64).pin_memory()
                      for k, v in coefs.items()}
        self.sources = {k: torch.as_tensor(v, dtype=torch.float64).pin_memory()
                        for k, v in sources.items()}
        self.params = params  # LMGParams, or {size class: LMGParams}
        self.classes = sorted({k for k, _ in coefs})
        self.slots = slots if isinstance(slots, dict) else {k: int(slots) for k in self.classes}
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
        self.contexts = {k: OrderedDict() for k in self.classes}
        self.need = {k: batch_footprint(k, self.slots[k], 32) for k in self.classes}
        self._serial = 0
        # grow: a class whose contexts are all full creates another one (within
        # the budget) instead of waiting for a slot; building a context takes
        # host time (seconds for the largest class), so a server that warmed
        # its contexts ahead of time turns it off
        self.grow = grow

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

    def create(self, klass: int) -> BatchContext:
        """Sets up a context whose bytes are already reserved."""
        prm = self.params[klass] if isinstance(self.params, dict) else self.params
        ctx = BatchContext(klass, self.slots[klass], prm, self.device, self.need[klass])
        self._serial += 1
        self.contexts[klass][(klass, self._serial)] = ctx
        return ctx

    def drop(self, klass, key):
        ctx = self.contexts[klass].pop(key)
        ctx.close()
        self.release(ctx.bytes)

    def warm(self, per_class=1):
        """Creates contexts ahead of time (as many as the budget allows):
        per_class contexts for every class, or {class: count}."""
        for k in self.classes:
            count = per_class.get(k, 1) if isinstance(per_class, dict) else int(per_class)
            for _ in range(count):
                if self.reserve(self.need[k]):
                    self.create(k).capture()

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

def make_pools(classes, coefs_per_class: int, srcs_per_class: int, seed: int = 0,
               device=None):
    """Seeded lognormal element coefficients (sigma 1.5, correlation 0.1) and
    N(0,1) interior sources for each size class N.  The random-Fourier-
    feature fields are evaluated on the GPU with torch (input generation
    only, outside any timed region)."""
    from workloads import fields, meshes
    dev = torch.device("cuda") if device is None else device
    coefs, src = {}, {}
    for N in classes:
        L = meshes.square_level(N)
        c = torch.tensor(fields.centroids(L), dtype=torch.float64, device=dev)
        for i in range(coefs_per_class):
            r = np.random.default_rng([seed * 1000 + i + 17 * N, 0])
            M = 512
            w = torch.tensor(r.standard_normal((M, 2)) / 0.1, dtype=torch.float64, device=dev)
            b = torch.tensor(r.uniform(0.0, 2.0 * np.pi, size=M), dtype=torch.float64, device=dev)
            g = torch.zeros(c.shape[0], dtype=torch.float64, device=dev)
            for s in range(0, c.shape[0], 1 << 18):
                g[s:s + (1 << 18)] = torch.cos(c[s:s + (1 << 18)] @ w.T + b).sum(1)
            coefs[(N, i)] = torch.exp(1.5 * np.sqrt(2.0 / M) * g).cpu().numpy()
        n = (N - 2) ** 2
        for j in range(srcs_per_class):
            src[(N, j)] = fields.rhs(n, 1, seed * 1000 + 500 + j + 17 * N)[:, 0]
    return coefs, src


def poisson_requests(rate: float, duration: float, classes, coefs_per_class: int,
                     srcs_per_class: int, seed: int = 0) -> list[Request]:
    """Poisson arrivals (exponential gaps) of uniformly drawn classes,
    coefficient fields and sources."""
    r = np.random.default_rng([seed, 4])
    t, out, k = 0.0, [], 0
    while True:
        t += r.exponential(1.0 / rate)
        if t > duration:
            break
        out.append(Request(k, int(classes[r.integers(len(classes))]),
                           int(r.integers(coefs_per_class)), int(r.integers(srcs_per_class)), t))
        k += 1
    return out


def summarize(done: list[Request], wall: float) -> dict:
    lat = np.array([r.t_done - r.t_arrival for r in done]) * 1e3
    per = {}
    for N in sorted({r.klass for r in done}):
        l = np.array([r.t_done - r.t_arrival for r in done if r.klass == N]) * 1e3
        it = np.array([r.iters for r in done if r.klass == N])
        wait = np.array([r.t_admit - r.t_arrival for r in done if r.klass == N]) * 1e3
        per[str(N)] = {"n": int(l.size), "p50_ms": round(float(np.percentile(l, 50)), 3),
                       "p99_ms": round(float(np.percentile(l, 99)), 3),
                       "p50_wait_ms": round(float(np.percentile(wait, 50)), 3),
                       "p50_service_ms": round(float(np.percentile(l - wait, 50)), 3),
                       "mean_iters": round(float(it.mean()), 2)}
    return {"solves": len(done), "solves_per_s": round(len(done) / wall, 2),
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_relres": float(max(r.relres for r in done)), "per_class": per}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--classes", default="65,129,257,513,1025")
    ap.add_argument("--coefs", type=int, default=16, help="coefficient fields per class pool")
    ap.add_argument("--srcs", type=int, default=8)
    ap.add_argument("--slots", default="65=64,129=64,257=32,513=16,1025=8",
                    help="slots per context, N=S[,N=S] (or one number for all)")
    ap.add_argument("--contexts", default="65=1,129=1,257=1,513=2,1025=3",
                    help="stacked contexts created per class before the run, N=K[,N=K]")
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
    if "=" in a.slots:
        slots = {int(k): int(v) for k, v in (x.split("=") for x in a.slots.split(","))}
        slots = {k: slots.get(k, 8) for k in classes}
    else:
        slots = {k: int(a.slots) for k in classes}
    t_setup = time.perf_counter()
    coefs, src = make_pools(classes, a.coefs, a.srcs, a.seed)
    base = trained.load(a.params, max(levels_for(k) for k in classes))
    spec = a.class_params
    if spec is None and os.path.exists(trained.LOGNORMAL1025):
        spec = f"1025={trained.LOGNORMAL1025}"
    over = dict((int(k), v) for k, v in (x.split("=", 1) for x in spec.split(","))) if spec else {}
    params = {k: trained.read(over[k]) if k in over else base for k in classes}
    t_setup = time.perf_counter() - t_setup
    reqs = poisson_requests(a.rate, a.duration, classes, a.coefs, a.srcs, a.seed)
    ctxs = {int(k): int(v) for k, v in (x.split("=") for x in a.contexts.split(","))}
    srv = Server(coefs, src, params, slots=slots, iters_per_tick=a.iters_per_tick, grow=False)
    t_warm = time.perf_counter()
    srv.warm({k: ctxs.get(k, 1) for k in classes})
    t_warm = time.perf_counter() - t_warm
    # warm-up: a few requests per class (captures the solve graphs), not timed
    srv.run([Request(-1 - i, k, i % a.coefs, 0, 0.0)
             for i, k in enumerate(c for c in classes for _ in range(2))])
    t0 = time.perf_counter()
    done = srv.run(reqs, t0)
    wall = time.perf_counter() - t0
    launches = sum(c.batch.kernel_launches() for k in classes for c in srv.contexts[k].values())
    n_ctx = {str(k): len(srv.contexts[k]) for k in classes}
    srv.close()
    out = {"metric": "continuous-batching solves to 1e-8, an operator per request (learned FP32 "
                     "V-cycle + FP64 refinement; operator set-up on the GPU inside the latency)",
           "offered_rate_per_s": a.rate, "duration_s": a.duration, "classes": classes,
           "coefficient_pool_per_class": a.coefs, "slots": slots,
           "iters_per_tick": a.iters_per_tick,
           "contexts": n_ctx,
           "wall_s": round(wall, 3), "pool_setup_s": round(t_setup, 2),
           "context_setup_s": round(t_warm, 2),
           "peak_device_bytes": srv.peak, "budget_bytes": srv.budget,
           "kernel_launches_resident_contexts": launches,
           "params": {str(k): os.path.basename(over[k]) if k in over else
                      trained.describe(a.params).split(":")[0] for k in classes}}
    out.update(summarize(done, wall))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
