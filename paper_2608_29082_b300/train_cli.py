"""Train Theta on a synthetic workload and write a checkpoint.

    python -m paper_2608_29082_b300.train_cli --workload checker513 \
        --out paper_2608_29082_b300/params/checker513_learned.json

Training follows Algorithm 3 with K unrolled cycles per epoch on a batch of
seeded N(0,1) right-hand sides (a different seed from the evaluation source),
FP32 forward/adjoint, Rprop.  After training, the refinement solve of the
evaluation source is timed with the identity and the trained parameters.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2608_29082_b300 import Hierarchy, LMGParams, Solver, trained  # noqa: E402
from paper_2608_29082_b300.training import ParamMap, Trainer  # noqa: E402

PRESETS = {
    "all": dict(train=("theta", "eta", "wB1", "wB2", "wR1", "wR2", "wP1", "wP2"), shared=()),
    "shared_conv": dict(train=("theta", "eta", "wB1", "wB2", "wR1", "wR2", "wP1", "wP2"),
                        shared=("wB1", "wB2", "wR1", "wR2", "wP1", "wP2")),
    "rps": dict(train=("eta", "wB1", "wB2", "wR1", "wR2", "wP1", "wP2"),
                shared=("wR1", "wR2", "wP1", "wP2")),
    "rp": dict(train=("wR1", "wR2", "wP1", "wP2"), shared=("wR1", "wR2", "wP1", "wP2")),
}


def make(workload: str, batch: int, seed: int):
    import workloads as W
    if workload == "checker513":
        return W.checkerboard_square(513, 9, 8, (1.0, 1e4), batch=batch, seed=seed)
    if workload == "checker257":
        return W.checkerboard_square(257, 8, 8, (1.0, 1e4), batch=batch, seed=seed)
    if workload == "train257_checker":
        return W.training_square("checker", batch=batch, seed=seed)
    if workload == "train257_poisson":
        return W.training_square("poisson", batch=batch, seed=seed)
    if workload == "lshape7":  # the anisotropic L-shape, 7 red refinements (3141633 DOF)
        return W.lshape_anisotropic(refinements=7, batch=batch, seed=seed)
    if workload.startswith("lognormal"):  # lognormal513, lognormal1025 (serving classes)
        return W.lognormal_square(int(workload[len("lognormal"):]), seed=seed, batch=batch)
    raise ValueError(workload)


def solve_iters(S: Solver, f: torch.Tensor, params: LMGParams, tol=1e-8):
    S.set_params(params)
    u, info = S.solve(f, tol=tol, max_iter=400)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u.zero_()
    u, info = S.solve(f, u, tol=tol, max_iter=400)
    torch.cuda.synchronize()
    return int(info.iters.max()), float(info.relres.max()), (time.perf_counter() - t0) * 1e3


def train(workload="checker513", preset="all", epochs=100, K=10, batch=8, seed=1000, lr=0.01,
          eval_seed=0, verbose=True, carry_u=False):
    """Trains on the workload's operator (coefficient seed eval_seed) with
    `batch` N(0,1) right-hand sides drawn from `seed`."""
    from workloads import fields
    ev = make(workload, 1, eval_seed)
    prob = ev
    hier = Hierarchy.from_problem(prob)
    J = hier.J
    p0 = LMGParams.identity(J)
    S = Solver(hier, p0, precision=32, max_batch=max(batch, 1))
    f = torch.tensor(fields.rhs(hier.sizes[0], batch, seed), dtype=torch.float32, device="cuda")
    pm = ParamMap(J, **PRESETS[preset])
    tr = Trainer(S, pm, n_cycles=K, lr=lr, carry_u=carry_u)
    t0 = time.perf_counter()
    log = tr.train(f, p0, max_epochs=epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # evaluation source: the workload's own right-hand side
    fe = torch.tensor(ev.f, dtype=torch.float64, device="cuda")
    it0, rr0, ms0 = solve_iters(S, fe, p0)
    it1, rr1, ms1 = solve_iters(S, fe, log.params)
    res = dict(workload=workload, preset=preset, epochs=len(log.losses), K=K, batch=batch,
               carry_u=carry_u,
               loss0=log.losses[0], best_loss=log.best_loss, train_s=round(t_train, 3),
               iters_identity=it0, iters_trained=it1, relres_trained=rr1,
               ms_identity=round(ms0, 3), ms_trained=round(ms1, 3))
    if verbose:
        print(json.dumps(res), flush=True)
    S.close()
    return log.params, res


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="checker513")
    ap.add_argument("--preset", default="all", choices=list(PRESETS))
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--lr", type=float, default=0.01)
    ap.add_argument("--carry-u", action="store_true")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    params, res = train(a.workload, a.preset, a.epochs, a.K, a.batch, a.seed, a.lr,
                        carry_u=a.carry_u)
    if a.out:
        trained.save(params, a.out, trained_on=(
            f"{a.workload}, preset {a.preset}, {res['epochs']} Rprop epochs, K={a.K} unrolled "
            f"cycles, {a.batch} N(0,1) rhs (seed {a.seed}); refinement iterations "
            f"{res['iters_identity']} -> {res['iters_trained']}"))
