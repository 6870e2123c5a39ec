"""Measurements of the other workloads (one JSON line each).

    python -m paper_2608_29082_b300.workload_bench lshape [--refinements 7 --batch 16]
        Jittered L-shape, anisotropic diffusion (about 3.1M DOF at 7 red
        refinements), 16 right-hand sides: Theta trained on the operator
        (Algorithm 3), then time to 1e-8 for the learned FP32 cycle in FP64
        refinement and for the plain FP64 multigrid, and per-kernel achieved
        bandwidth (algorithmic bytes / CUDA-event time) against the measured
        HBM peak.  The working set is far larger than L2.
    python -m paper_2608_29082_b300.workload_bench training [--kind checker --batch 64]
        One training step of Algorithm 3 on the 257^2 workloads: K = 10
        unrolled FP32 cycles with per-level checkpoints, the residual loss
        and the hand-written adjoint, for 64 right-hand sides.
    python -m paper_2608_29082_b300.workload_bench cheb [--refinements 7 --batch 16]
        ChebConv smoother (mg_set_cheb) of degree 1, 2, 4 against the
        SAGEConv smoother: FP32 cycle time on the L-shape (16 rhs) and on the
        513^2 checkerboard (1 rhs), and the level-0 Chebyshev pass's achieved
        bandwidth against the measured HBM peak.
    python -m paper_2608_29082_b300.workload_bench features2
        Two features per node (mg2_*): the Helmholtz operator with impedance
        boundary at the paper's resolution (h = 1/256, k = 16 pi, J = 5);
        cycle time in FP32 and FP64 for 1 and 16 right-hand sides, and time
        to 1e-8 with FGMRES and the cycle or FMG (129^2, k = 8 pi, J = 3).
    python -m paper_2608_29082_b300.workload_bench profile_case
        A short, fixed case for a profiler's kernel captures: on the L-shape
        (3.1M DOF, 16 rhs, FP32) one cycle with a degree-2 ChebConv smoother,
        then one FGMRES(4) cycle (4 Arnoldi steps) with the V-cycle.
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

from paper_2608_29082_b300 import Hierarchy, LMGParams, Solver  # noqa: E402
from paper_2608_29082_b300.training import ParamMap, Trainer  # noqa: E402
from paper_2608_29082_b300.train_cli import PRESETS  # noqa: E402


def hbm_peak() -> float:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6400.0


def level_bytes(name: str, hier, lev: int, B: int, b: int) -> float:
    """Algorithmic bytes of one launch (each array read or written once)."""
    n = hier.sizes[lev]
    A = hier.A[lev]
    nnz_off = A.data.size - n
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    m = A.indices != rows
    col_b = 0 if np.unique(A.indices[m] - rows[m]).size <= 8 else 4
    nc = hier.sizes[lev + 1] if lev + 1 < hier.J else 0
    nnzP = hier.P[lev].data.size if lev < hier.J - 1 else 0
    # the mean aggregation's neighbour test: SELL column indices, or on
    # DIA levels one mask byte per row
    mean_b = nnz_off * col_b if col_b else n
    table = {
        "jacobi_smooth": nnz_off * (col_b + b) + 2 * n * b + 3 * B * n * b,
        "residual_scaled": nnz_off * (col_b + b) + 2 * n * b + 3 * B * n * b,
        "sage_conv_update": mean_b + n * b + 3 * B * n * b,
        "cheb_conv_update": mean_b + n * b + 5 * B * n * b,
        "residual": nnz_off * (col_b + b) + n * b + 3 * B * n * b,
        "restrict_conv_fine": mean_b + n * b + 2 * B * n * b,
        "restrict_conv": nnzP * (4 + b) + B * n * b + B * nc * b,
        "prolong_fine": nnzP * (4 + b) + B * nc * b + B * n * b,
        "prolong_conv": mean_b + n * b + 3 * B * n * b,
        "outer_residual_fp64": nnz_off * (col_b + 8) + 2 * n * 8 + B * n * 24,
        "smooth_halo": nnz_off * (col_b + b) + 3 * n * b + 3 * B * n * b,
        "restrict_conv_halo": nnz_off * (col_b + b) + 2 * n * b + 3 * B * n * b,
        "prolong_halo": nnzP * (4 + b) + mean_b + n * b + B * nc * b
                        + 2 * B * n * b,
    }
    return table.get(name, float("nan"))


def kernel_table(S: Solver, hier, f: torch.Tensor, reps: int = 3):
    B = f.shape[1]
    b = 4 if S.precision == 32 else 8
    u = torch.zeros_like(f)
    agg = {}
    for _ in range(reps):
        u.zero_()
        for name, lev, ms in S.vcycle_profile(f, u):
            a = agg.setdefault((name, lev), [0.0, 0])
            a[0] += ms
            a[1] += 1
    peak = hbm_peak()
    out = []
    total = sum(v[0] for v in agg.values()) / reps
    for (name, lev), (ms, cnt) in sorted(agg.items(), key=lambda kv: -kv[1][0]):
        per = ms / cnt
        nb = level_bytes(name, hier, lev, B, b)
        gbs = nb / (per * 1e-3) / 1e9 if np.isfinite(nb) else None
        out.append({"kernel": name, "level": lev, "launches_per_cycle": cnt / reps,
                    "us_per_launch": round(per * 1e3, 2), "share": round(ms / reps / total, 4),
                    "algorithmic_MB": round(nb / 1e6, 2) if np.isfinite(nb) else None,
                    "GBps": round(gbs, 1) if gbs else None,
                    "frac_of_hbm": round(gbs / peak, 3) if gbs else None})
    return out, total * 1e3


def timed_solve(S: Solver, f64: torch.Tensor, tol: float, reps: int = 3, method="refine"):
    u = torch.zeros_like(f64)
    S.solve(f64, u, tol=tol, max_iter=400, method=method)
    ms = []
    for _ in range(reps):
        u.zero_()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        _, info = S.solve(f64, u, tol=tol, max_iter=400, method=method)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms)), info, u


def run_lshape(a):
    import workloads as W
    from workloads import fields
    t0 = time.perf_counter()
    prob = W.lshape_anisotropic(refinements=a.refinements, batch=a.batch, seed=a.seed)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    hier = Hierarchy.from_problem(prob)
    t_setup = time.perf_counter() - t0
    J = hier.J
    dev = torch.device("cuda")
    plain = LMGParams.identity(J)
    learned, training = plain, None
    if a.cycles_only:
        # a few FP32 cycles with convolutions on every level (profiling target)
        p = LMGParams.identity(J)
        p.wB[:, 1], p.wR[:, 1], p.wP[:, 1] = 0.1, 0.05, -0.05
        S = Solver(hier, p, precision=32, max_batch=a.batch)
        if a.sell_halo_rows:
            S.set_option("sell_halo_rows", a.sell_halo_rows)
        f = torch.tensor(prob.f, dtype=torch.float32, device=dev)
        u = torch.zeros_like(f)
        for _ in range(a.cycles_only):
            S.vcycle(f, u)
        kt, cyc = kernel_table(S, hier, f, reps=1)
        torch.cuda.synchronize()
        print(json.dumps({"workload": f"L-shape r{a.refinements}, {hier.sizes[0]} DOF, "
                          f"{a.batch} rhs", "cycle_us_profiled": round(cyc, 1),
                          "kernels_fp32": kt[:6]}), flush=True)
        return
    if a.train_epochs > 0:
        ftr = torch.tensor(fields.rhs(hier.sizes[0], a.train_batch, 1000 + a.seed),
                           dtype=torch.float32, device=dev)
        Str = Solver(hier, plain, precision=32, max_batch=a.train_batch)
        t0 = time.perf_counter()
        log = Trainer(Str, ParamMap(J, **PRESETS[a.preset]), n_cycles=a.K).train(
            ftr, plain, max_epochs=a.train_epochs)
        torch.cuda.synchronize()
        training = {"preset": a.preset, "epochs": len(log.losses), "K": a.K,
                    "rhs": a.train_batch, "seconds": round(time.perf_counter() - t0, 2),
                    "loss_ratio": float(log.best_loss / log.losses[0])}
        learned = log.params
        Str.close()
    f64 = torch.tensor(prob.f, dtype=torch.float64, device=dev)
    S32 = Solver(hier, learned, precision=32, max_batch=a.batch)
    ms32, info32, u32 = timed_solve(S32, f64, a.tol)
    kt32, cyc32 = kernel_table(S32, hier, f64.float())
    msf32, infof32, uf32 = timed_solve(S32, f64, a.tol, method="fcg")
    S32.set_option("fcg_precond", 1)  # full multigrid as the preconditioner
    msg32, infog32, ug32 = timed_solve(S32, f64, a.tol, method="fcg")
    # restarted flexible GMRES(30) takes the nonsymmetric preconditioners as they are
    msq32, infoq32, uq32 = timed_solve(S32, f64, a.tol, method="fgmres")
    S32.set_option("fcg_precond", 0)
    msr32, infor32, ur32 = timed_solve(S32, f64, a.tol, method="fgmres")
    S64 = Solver(hier, plain, precision=64, max_batch=a.batch)
    ms64, info64, _ = timed_solve(S64, f64, a.tol)
    msf64, infof64, _ = timed_solve(S64, f64, a.tol, method="fcg")
    kt64, cyc64 = kernel_table(S64, hier, f64)
    # the final relative residuals recomputed on the host (FP64) from the
    # workload's own finest operator, not from the solver's device copy
    I = prob.mesh.levels[0].interior
    A_int = prob.A_full.tocsr()[I][:, I]

    def recheck(uu):
        un = uu.cpu().numpy()
        r = prob.f - A_int @ un
        return np.sqrt((r * r).sum(0)) / np.sqrt((prob.f * prob.f).sum(0))
    rr = recheck(u32)
    rrf = recheck(uf32)
    rrg = recheck(ug32)
    rrr = recheck(ur32)
    rrq = recheck(uq32)
    out = {"workload": f"L-shape anisotropic, {a.refinements} red refinements, {hier.sizes[0]} DOF, "
                       f"{J} levels, {a.batch} rhs, tol {a.tol}",
           "levels": hier.sizes, "generate_s": round(t_gen, 1), "setup_s": round(t_setup, 1),
           "training": training,
           "learned_fp32_ms": round(ms32, 3), "learned_iters": int(info32.iters.max()),
           "plain_fp64_ms": round(ms64, 3), "plain_iters": int(info64.iters.max()),
           "speedup": round(ms64 / ms32, 3), "max_relres_recheck": float(rr.max()),
           "learned_fp32_fcg_ms": round(msf32, 3), "learned_fcg_iters": int(infof32.iters.max()),
           "max_relres_recheck_fcg": float(rrf.max()),
           "learned_fp32_fcg_fmg_ms": round(msg32, 3),
           "learned_fcg_fmg_iters": int(infog32.iters.max()),
           "max_relres_recheck_fcg_fmg": float(rrg.max()),
           "learned_fp32_fgmres_ms": round(msr32, 3),
           "learned_fgmres_iters": int(infor32.iters.max()),
           "max_relres_recheck_fgmres": float(rrr.max()),
           "learned_fp32_fgmres_fmg_ms": round(msq32, 3),
           "learned_fgmres_fmg_iters": int(infoq32.iters.max()),
           "max_relres_recheck_fgmres_fmg": float(rrq.max()),
           "plain_fp64_fcg_ms": round(msf64, 3), "plain_fcg_iters": int(infof64.iters.max()),
           "speedup_fcg_learned_vs_plain_stationary": round(ms64 / msf32, 3),
           "cycle_us_fp32_profiled": round(cyc32, 1), "cycle_us_fp64_profiled": round(cyc64, 1),
           "hbm_peak_gbs": hbm_peak(), "kernels_fp32": kt32[:8], "kernels_fp64": kt64[:6]}
    print(json.dumps(out), flush=True)


def cycle_ms(S: Solver, f: torch.Tensor, reps: int = 20) -> float:
    """Median CUDA-event time of one FP32 cycle (graph replay), from zero."""
    u = torch.zeros_like(f)
    for _ in range(3):
        S.vcycle(f, u)
    ms = []
    for _ in range(reps):
        u.zero_()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        S.vcycle(f, u)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms))


def run_cheb(a):
    import workloads as W
    dev = torch.device("cuda")
    out = {"workload": "ChebConv smoother vs SAGEConv, FP32 cycle, identity-initialised "
                       "coefficients (c_0 = 1, c_k = 0.1 / k)"}
    for tag, prob in (("lshape", W.lshape_anisotropic(refinements=a.refinements, batch=a.batch,
                                                       seed=a.seed)),
                      ("checker513", W.checkerboard_square(N=513, J=9, ncell=8,
                                                           values=(1.0, 1e4), batch=1,
                                                           seed=a.seed))):
        hier = Hierarchy.from_problem(prob)
        S = Solver(hier, LMGParams.identity(hier.J), precision=32, max_batch=prob.f.shape[1])
        f = torch.tensor(prob.f, dtype=torch.float32, device=dev)
        res = {"dof": hier.sizes[0], "rhs": prob.f.shape[1], "sage_cycle_ms": cycle_ms(S, f)}
        for K in (1, 2, 4):
            c = np.zeros((hier.J - 1, K + 1))
            c[:, 0] = 1.0
            c[:, 1:] = 0.1 / np.arange(1, K + 1)
            S.set_cheb(c)
            res[f"cheb{K}_cycle_ms"] = cycle_ms(S, f)
            if K == 4 and tag == "lshape":
                kt, _ = kernel_table(S, hier, f)
                res["cheb4_level0"] = [r for r in kt if r["level"] == 0][:4]
        S.close()
        out[tag] = res
    out["hbm_peak_gbs"] = hbm_peak()
    print(json.dumps(out), flush=True)


def run_profile_case(a):
    import workloads as W
    prob = W.lshape_anisotropic(refinements=a.refinements, batch=a.batch, seed=a.seed)
    hier = Hierarchy.from_problem(prob)
    S = Solver(hier, LMGParams.identity(hier.J), precision=32, max_batch=a.batch)
    f32 = torch.tensor(prob.f, dtype=torch.float32, device="cuda")
    f64 = torch.tensor(prob.f, dtype=torch.float64, device="cuda")
    c = np.zeros((hier.J - 1, 3))
    c[:, 0], c[:, 1:] = 1.0, 0.1
    S.set_cheb(c)
    S.vcycle(f32, torch.zeros_like(f32))
    S.set_cheb(None)
    _, info = S.solve(f64, torch.zeros_like(f64), tol=1e-12, max_iter=4, method="fgmres",
                      restart=4)
    # flexible CG with FP32 vectors, iterations driven from the host (plain
    # graphs, which a profiler traces): a first restart, a few FP32 steps,
    # the forced restart of the last one
    S.set_option("device_loop", 0)
    _, info_c = S.solve(f64, torch.zeros_like(f64), tol=1e-12, max_iter=a.fcg_steps,
                        method="fcg")
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"L-shape {hier.sizes[0]} DOF, {a.batch} rhs",
                      "fgmres_steps": int(info.iters.max()),
                      "fcg_steps": int(info_c.iters.max())}), flush=True)
    S.close()
    if a.features2:
        # the two-feature cycle on 1025^2 vertices, 16 rhs, FP32: three cycles
        from paper_2608_29082_b300.features2 import Hierarchy2, Params2, Solver2
        p2 = W.helmholtz_square(1025, 6, k=16 * np.pi, batch=16, seed=a.seed)
        h2 = Hierarchy2.from_problem(p2)
        prm = Params2.identity(h2.J)
        prm.WB[:, 1] = 0.1 * np.eye(2)
        S2 = Solver2(h2, prm, precision=32, max_batch=16)
        f2 = torch.tensor(p2.f, dtype=torch.complex64, device="cuda")
        u2 = torch.zeros_like(f2)
        for _ in range(3):
            S2.vcycle(f2, u2)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": f"two features, {h2.sizes[0]} DOF, 16 rhs",
                          "max_abs_u": float(u2.abs().max())}), flush=True)
        S2.close()


def level_bytes2(name: str, hier, lev: int, B: int, b: int) -> float:
    """Algorithmic bytes of one two-feature launch: CSR row pointers and
    column indices (4 B), complex matrix values (2 b), real P / P^T values
    (b), complex vectors (2 b per entry), each array read or written once."""
    A = hier.A[lev]
    n, nnz = A.shape[0], A.nnz
    c2 = 2 * b
    nc = hier.sizes[lev + 1] if lev + 1 < hier.J else 0
    nnzP = hier.P[lev].nnz if lev < hier.J - 1 else 0
    rp = (n + 1) * 4
    table = {
        "residual_scaled": rp + nnz * (4 + c2) + n * c2 + 3 * B * n * c2,
        "residual": rp + nnz * (4 + c2) + 3 * B * n * c2,
        "sage_conv_update": rp + nnz * 4 + n * b + 3 * B * n * c2,
        "restrict_conv_fine": rp + nnz * 4 + n * b + 2 * B * n * c2,
        "restrict_conv": (nc + 1) * 4 + nnzP * (4 + b) + B * n * c2 + B * nc * c2,
        "prolong_fine": rp + nnzP * (4 + b) + B * nc * c2 + B * n * c2,
        "prolong_conv": rp + nnz * 4 + n * b + 3 * B * n * c2,
    }
    return table.get(name, float("nan"))


def features2_roofline(a):
    """Per-kernel time (CUDA events around each launch of an eager cycle) and
    algorithmic GB/s of the two-feature cycle on a case whose level-0 vectors
    exceed L2: Helmholtz with impedance boundary on roof_N^2 vertices, 16
    rhs, FP32."""
    import workloads as W
    from paper_2608_29082_b300.features2 import Hierarchy2, Params2, Solver2
    B = 16
    prob = W.helmholtz_square(a.roof_N, a.roof_J, k=a.roof_k_over_pi * np.pi, batch=B,
                              seed=a.seed)
    hier = Hierarchy2.from_problem(prob)
    prm = Params2.identity(hier.J)
    prm.WB[:, 1] = 0.1 * np.eye(2)
    prm.WR[:, 1] = 0.05 * np.eye(2)
    prm.WP[:, 1] = -0.05 * np.eye(2)
    S = Solver2(hier, prm, precision=32, max_batch=B)
    f = torch.tensor(prob.f, dtype=torch.complex64, device="cuda")
    u = torch.zeros_like(f)
    for _ in range(3):
        S.vcycle(f, u)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    ms = []
    for _ in range(10):
        u.zero_()
        e0.record()
        S.vcycle(f, u)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    agg, reps = {}, 3
    for _ in range(reps):
        u.zero_()
        for name, lev, t in S.vcycle_profile(f, u):
            x = agg.setdefault((name, lev), [0.0, 0])
            x[0] += t
            x[1] += 1
    S.close()
    peak = hbm_peak()
    total = sum(v[0] for v in agg.values()) / reps
    rows = []
    for (name, lev), (t, cnt) in sorted(agg.items(), key=lambda kv: -kv[1][0]):
        per = t / cnt
        nb = level_bytes2(name, hier, lev, B, 4)
        gbs = nb / (per * 1e-3) / 1e9 if np.isfinite(nb) else None
        rows.append({"kernel": name, "level": lev, "us_per_launch": round(per * 1e3, 2),
                     "share": round(t / reps / total, 4),
                     "algorithmic_MB": round(nb / 1e6, 2) if np.isfinite(nb) else None,
                     "GBps": round(gbs, 1) if gbs else None,
                     "frac_of_hbm": round(gbs / peak, 3) if gbs else None})
    return {"workload": f"Helmholtz, impedance boundary, {a.roof_N}x{a.roof_N} vertices "
                        f"({hier.sizes[0]} DOF), k = {a.roof_k_over_pi:g} pi, J = {hier.J}, "
                        f"{B} rhs, FP32, two features",
            "cycle_ms_graph": round(float(np.median(ms)), 3),
            "cycle_ms_eager_events": round(total, 3), "hbm_peak_gbs": peak,
            "kernels": rows[:10]}


def run_features2(a):
    import workloads as W
    from paper_2608_29082_b300.features2 import Hierarchy2, Params2, Solver2
    if a.roof_N:
        print(json.dumps({"roofline": features2_roofline(a)}), flush=True)
    out = {"workload": f"Helmholtz, impedance boundary, {a.N}x{a.N} vertices (h = 1/{a.N - 1}), "
                       f"k = {a.k_over_pi:g} pi, J = {a.J}, two features (Re, Im), W_1 = I, "
                       "W_2 = 0.1 on the smoother"}
    for B in (1, 16):
        prob = W.helmholtz_square(a.N, a.J, k=a.k_over_pi * np.pi, batch=B, seed=a.seed)
        hier = Hierarchy2.from_problem(prob)
        prm = Params2.identity(hier.J)
        prm.WB[:, 1] = 0.1 * np.eye(2)
        for prec in (32, 64):
            S = Solver2(hier, prm, precision=prec, max_batch=B)
            dt = torch.complex64 if prec == 32 else torch.complex128
            f = torch.tensor(prob.f, dtype=dt, device="cuda")
            u = torch.zeros_like(f)
            for _ in range(3):
                S.vcycle(f, u)
            ms = []
            for _ in range(20):
                u.zero_()
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record()
                S.vcycle(f, u)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            out[f"fp{prec}_rhs{B}_cycle_ms"] = round(float(np.median(ms)), 4)
            S.close()
        out["dof"] = hier.sizes[0]
        out["levels"] = hier.sizes
    # time to 1e-8 with FGMRES(30), classical two-feature weights, FP32
    # cycle: half the resolution at the same k h (129^2, k = 8 pi), on a
    # hierarchy shallow enough for Jacobi-type smoothing on every level
    # (coarsest h = 1/32; the paper's deeper runs use GMRES smoothers)
    Jk = a.krylov_J
    out["fgmres_workload"] = (f"{a.krylov_N}x{a.krylov_N}, k = {a.krylov_k_over_pi:g} pi, "
                              f"J = {Jk}, FP32 cycle, FGMRES(30), tol 1e-8")
    for B in (1, 16):
        prob = W.helmholtz_square(a.krylov_N, Jk, k=a.krylov_k_over_pi * np.pi, batch=B,
                                  seed=a.seed)
        hier = Hierarchy2.from_problem(prob)
        S = Solver2(hier, Params2.identity(hier.J), precision=32, max_batch=B)
        f = torch.tensor(prob.f, dtype=torch.complex128, device="cuda")
        for pc in ("vcycle", "fmg"):
            u = torch.zeros_like(f)
            S.solve_fgmres(f, u, tol=1e-8, precond=pc)
            ms = []
            for _ in range(3):
                u.zero_()
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record()
                _, info = S.solve_fgmres(f, u, tol=1e-8, precond=pc)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            out[f"fgmres_{pc}_J{Jk}_rhs{B}"] = {"ms": round(float(np.median(ms)), 3),
                                               "iters": int(info.iters.max()),
                                               "relres": float(info.relres.max())}
        S.close()
    print(json.dumps(out), flush=True)


def run_training(a):
    import workloads as W
    prob = W.training_square(a.kind, N=257, J=8, batch=a.batch, seed=a.seed)
    hier = Hierarchy.from_problem(prob)
    J = hier.J
    p = LMGParams.identity(J)
    S = Solver(hier, p, precision=32, max_batch=a.batch)
    f = torch.tensor(prob.f, dtype=torch.float32, device="cuda")
    tr = Trainer(S, ParamMap(J, shared=("wB1", "wB2", "wR1", "wR2", "wP1", "wP2")), n_cycles=a.K)
    for _ in range(2):
        tr.loss_and_grad(p, f, torch.zeros_like(f))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    for _ in range(a.steps):
        loss, g, _ = tr.loss_and_grad(p, f, torch.zeros_like(f))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    t0 = time.perf_counter()
    log = tr.train(f, p, max_epochs=a.epochs)
    t_train = time.perf_counter() - t0
    print(json.dumps({"workload": f"training {a.kind} 257^2, {J} levels, {a.batch} rhs, K={a.K}",
                      "ms_per_training_step": round(ms, 3), "loss0": log.losses[0],
                      "best_loss": log.best_loss, "epochs": len(log.losses),
                      "train_seconds": round(t_train, 2)}), flush=True)



# Algorithmic bytes per row of the stacked square levels' main kernels for
# one rhs in FP32 (interior rows: six off-diagonals; DIA, so no column
# indices): residual_scaled reads f, u, six values, diagonal and its
# inverse and writes delta; sage_conv_update reads the neighbour mask, 1/deg,
# delta and u and writes u; residual reads f, u, six values and the diagonal
# and writes r.
STACKED_ROW_BYTES = {"residual_scaled": 44, "sage_conv_update": 17, "residual": 40}


def run_stacked(a):
    """An S-slot stacked context of N x N meshes (one seeded lognormal
    operator per slot, set up on the device): the per-kernel table of an
    eager FP32 cycle, the graph-replayed cycle and optionally one solve of
    every slot to 1e-8."""
    print(json.dumps(stacked_report(a)), flush=True)


def stacked_report(a) -> dict:
    """run_stacked's measurements as a dict (fields of a: N, slots, cycles,
    solve, two_rows, halo2d_bytes, host_loop, seed)."""
    from . import serve, trained
    from .square import SquareBatch
    N, S = a.N, a.slots
    coefs, src = serve.make_pools([N], min(S, 4), 1, a.seed)
    p = trained.read(trained.LOGNORMAL1025) if os.path.exists(trained.LOGNORMAL1025) \
        else trained.load(None, 12)
    sb = SquareBatch(N, S, p, precision=32)
    for k in range(S):
        sb.set_block(k, torch.tensor(coefs[(N, k % min(S, 4))], dtype=torch.float64,
                                     device=sb.device))
    sb.set_option("dia_two_rows", a.two_rows)
    sb.set_option("halo2d_bytes", a.halo2d_bytes)
    if a.host_loop:  # plain graphs per iteration (profilers skip conditional nodes)
        sb.set_option("device_loop", 0)
    g = torch.Generator(device=sb.device).manual_seed(a.seed)
    f = torch.randn(S * sb.m, dtype=torch.float32, device=sb.device, generator=g)
    u = torch.zeros_like(f)
    for _ in range(a.cycles):
        sb.vcycle(f, u)
    torch.cuda.synchronize()
    agg = {}
    for _ in range(3):
        u.zero_()
        for name, lev, ms in sb.vcycle_profile(f, u):
            r = agg.setdefault((name, lev), [0.0, 0])
            r[0] += ms
            r[1] += 1
    peak = hbm_peak()
    rows = []
    for (name, lev), (ms, cnt) in sorted(agg.items(), key=lambda kv: -kv[1][0]):
        us = 1e3 * ms / cnt
        rb = STACKED_ROW_BYTES.get(name) if lev == 0 else None
        gbs = rb * sb.sizes[0] / (us * 1e-6) / 1e9 if rb else None
        rows.append({"kernel": name, "level": lev, "launches_per_cycle": cnt // 3,
                     "us_per_launch": round(us, 2),
                     "GBps": round(gbs, 1) if gbs else None,
                     "frac_of_hbm": round(gbs / peak, 3) if gbs else None})
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(10):
        sb.vcycle(f, u)
    e1.record()
    torch.cuda.synchronize()
    out = {"workload": f"stacked {S} x {N}^2 lognormal, {sb.J} levels, FP32 cycle",
           "rows": sb.sizes[0], "graph_cycle_ms": round(e0.elapsed_time(e1) / 10, 4),
           "hbm_peak_gbs": peak, "kernels": rows[:16]}
    if a.solve:
        f64 = torch.tensor(np.concatenate([src[(N, 0)]] * S), dtype=torch.float64,
                           device=sb.device)
        u64 = torch.zeros_like(f64)
        sb.solve(f64, u64, tol=1e-8, max_iter=100)
        u64.zero_()
        torch.cuda.synchronize()
        e0.record()
        info = sb.solve(f64, u64, tol=1e-8, max_iter=100)
        e1.record()
        torch.cuda.synchronize()
        out["solve_ms"] = round(e0.elapsed_time(e1), 3)
        out["solve_iters_max"] = int(info.iters.max())
    sb.close()
    return out

if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    l = sub.add_parser("lshape")
    l.add_argument("--refinements", type=int, default=7)
    l.add_argument("--batch", type=int, default=16)
    l.add_argument("--tol", type=float, default=1e-8)
    l.add_argument("--train-epochs", type=int, default=60)
    l.add_argument("--train-batch", type=int, default=4)
    l.add_argument("--K", type=int, default=10)
    l.add_argument("--preset", default="shared_conv")
    l.add_argument("--seed", type=int, default=0)
    l.add_argument("--sell-halo-rows", type=int, default=0,
                   help="with --cycles-only: the fused SELL steps' tile rows (0: two kernels)")
    l.add_argument("--cycles-only", type=int, default=0,
                   help="only run this many FP32 cycles and the per-kernel table")
    t = sub.add_parser("training")
    t.add_argument("--kind", default="checker")
    t.add_argument("--batch", type=int, default=64)
    t.add_argument("--K", type=int, default=10)
    t.add_argument("--steps", type=int, default=5)
    t.add_argument("--epochs", type=int, default=30)
    t.add_argument("--seed", type=int, default=0)
    c = sub.add_parser("cheb")
    c.add_argument("--refinements", type=int, default=7)
    c.add_argument("--batch", type=int, default=16)
    c.add_argument("--seed", type=int, default=0)
    f2 = sub.add_parser("features2")
    f2.add_argument("--N", type=int, default=257)
    f2.add_argument("--J", type=int, default=5)
    f2.add_argument("--k-over-pi", type=float, default=16.0)
    f2.add_argument("--seed", type=int, default=0)
    f2.add_argument("--krylov-J", type=int, default=3)
    f2.add_argument("--krylov-N", type=int, default=129)
    f2.add_argument("--krylov-k-over-pi", type=float, default=8.0)
    f2.add_argument("--roof-N", type=int, default=1025,
                    help="size of the per-kernel roofline case (0: skip)")
    f2.add_argument("--roof-J", type=int, default=6)
    f2.add_argument("--roof-k-over-pi", type=float, default=16.0)
    pc = sub.add_parser("profile_case")
    pc.add_argument("--refinements", type=int, default=7)
    pc.add_argument("--batch", type=int, default=16)
    pc.add_argument("--seed", type=int, default=0)
    pc.add_argument("--fcg-steps", type=int, default=3)
    pc.add_argument("--features2", type=int, default=1,
                    help="also run three two-feature cycles on 1025^2 vertices")
    sq = sub.add_parser("stacked")
    sq.add_argument("--N", type=int, default=1025)
    sq.add_argument("--slots", type=int, default=8)
    sq.add_argument("--cycles", type=int, default=2, help="warm-up cycles")
    sq.add_argument("--solve", type=int, default=1)
    sq.add_argument("--two-rows", type=int, default=1)
    sq.add_argument("--halo2d-bytes", type=int, default=0)
    sq.add_argument("--host-loop", action="store_true",
                    help="iterate the solve from the host (for profilers)")
    sq.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    {"lshape": run_lshape, "training": run_training, "cheb": run_cheb,
     "profile_case": run_profile_case, "features2": run_features2,
     "stacked": run_stacked}[a.cmd](a)
