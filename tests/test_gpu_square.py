"""Stacked contexts (one operator per request on the square mesh) against the
oracle: the device set-up (P1 assembly, Galerkin coarsening, drop rule,
degrees, coarsest inverse) level by level, the cycle per block, block
solves that equal each system solved alone, bitwise, and solves over the
leading blocks that equal solves over all of them, through the C ABI.

Tolerances: FP64 operator application and single steps 1e-13 relative per
block (the device sums the Galerkin products in another order than the
oracle's sparse products); FP64 cycles 1e-12; FP32 cycles 1e-5; solves to
1e-8 re-evaluated by the oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2608_29082_b300 import LMGParams
from paper_2608_29082_b300.square import SquareBatch, levels_for
from workloads import fields, meshes

pytestmark = pytest.mark.gpu

DEV = "cuda"


def coefficients(N, kind, seed):
    L = meshes.square_level(N)
    if kind == "poisson":
        return np.ones(L.tri.shape[0])
    if kind == "checker":
        return fields.checkerboard(L, 4, (1.0, 1e3), seed)
    return fields.lognormal(L, 1.5, 0.1, seed)


def systems(N, kinds, seed=0):
    n = (N - 2) ** 2
    out = []
    for b, kind in enumerate(kinds):
        k = coefficients(N, kind, seed + b)
        f = fields.rhs(n, 1, seed + 100 + b)[:, 0]
        p = W.square_with_coefficients(N, k, f)
        out.append((k, f, p, O.build_hierarchy(p)))
    return out


def rand_params(J, seed, spread=0.2):
    r = np.random.default_rng(seed)
    p = LMGParams.identity(J)
    m = J - 1
    p.theta = p.theta * (1 + spread * r.uniform(-1, 1, m))
    p.eta = p.eta * (1 + spread * r.uniform(-1, 1, m))
    for w in (p.wB, p.wR, p.wP):
        w[:, 0] += spread * r.uniform(-1, 1, m)
        w[:, 1] += spread * r.uniform(-1, 1, m)
    return p


def to_oracle(p):
    return O.Params(p.theta.copy(), p.eta.copy(), p.wB.copy(), p.wR.copy(), p.wP.copy(),
                    p.nu_pre, p.nu_post)


def t64(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def fill(batch, sys_list):
    for b, (k, f, p, H) in enumerate(sys_list):
        batch.set_block(b, t64(k))


@pytest.mark.parametrize("N", [17, 33])
def test_device_setup_matches_oracle_per_level(N):
    """For every level and block: A u (the residual step with f = 0), the
    learnable smoothing step (diagonal, 1/diagonal and 1/degree through the
    SAGEConv mean) and the coarsest solve equal the oracle's for that
    block's own system."""
    sys_list = systems(N, ["lognormal", "checker", "poisson"], seed=3)
    J = levels_for(N)
    prm = rand_params(J, 5)
    po = to_oracle(prm)
    S = SquareBatch(N, 3, prm, precision=64)
    fill(S, sys_list)
    r = np.random.default_rng(1)
    for lev in range(J):
        m = S.sizes[lev] // 3
        u = r.standard_normal(3 * m)
        f = r.standard_normal(3 * m)
        out = torch.empty(3 * m, dtype=torch.float64, device=DEV)
        if lev == J - 1:
            S.level_apply(lev, "coarse", t64(f), None, out)
            for b, (_, _, _, H) in enumerate(sys_list):
                ref = f[b * m:(b + 1) * m] / H.levels[lev].A.toarray()[0, 0]
                got = out.cpu().numpy()[b * m:(b + 1) * m]
                assert np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max(), (lev, b)
            continue
        S.level_apply(lev, "residual", t64(np.zeros(3 * m)), t64(u), out)
        got = -out.cpu().numpy()
        for b, (_, _, _, H) in enumerate(sys_list):
            ref = H.levels[lev].A @ u[b * m:(b + 1) * m]
            err = np.linalg.norm(got[b * m:(b + 1) * m] - ref) / np.linalg.norm(ref)
            assert err < 1e-13, (N, lev, b, err)
        S.level_apply(lev, "smooth", t64(f), t64(u), out)
        got = out.cpu().numpy()
        for b, (_, _, _, H) in enumerate(sys_list):
            sl = slice(b * m, (b + 1) * m)
            ref = O.smooth(H.levels[lev], f[sl, None], u[sl, None], po.theta[lev], po.eta[lev],
                           po.wB[lev])[:, 0]
            err = np.linalg.norm(got[sl] - ref) / np.linalg.norm(ref)
            assert err < 1e-13, (N, lev, b, err)
    S.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_cycle_per_block_matches_oracle(prec):
    N = 33
    sys_list = systems(N, ["lognormal", "lognormal", "checker", "lognormal"], seed=11)
    J = levels_for(N)
    prm = rand_params(J, 7)
    po = to_oracle(prm)
    S = SquareBatch(N, 4, prm, precision=prec)
    fill(S, sys_list)
    m = S.m
    fs = np.concatenate([f for (_, f, _, _) in sys_list])
    dt = torch.float64 if prec == 64 else torch.float32
    fd = torch.tensor(fs, dtype=dt, device=DEV)
    u = torch.zeros(4 * m, dtype=dt, device=DEV)
    uo = [np.zeros((m, 1)) for _ in sys_list]
    for cyc in range(3):
        if prec == 32:  # the oracle from the same FP32-representable iterate
            cur = u.double().cpu().numpy()
            uo = [cur[b * m:(b + 1) * m, None] for b in range(4)]
        S.vcycle(fd, u)
        got = u.double().cpu().numpy()
        for b, (_, f, p, H) in enumerate(sys_list):
            fo = f.astype(np.float32).astype(np.float64) if prec == 32 else f
            uo[b] = O.vcycle(H, po, fo[:, None], uo[b])
            err = np.linalg.norm(got[b * m:(b + 1) * m] - uo[b][:, 0]) / np.linalg.norm(uo[b])
            assert err < (1e-12 if prec == 64 else 1e-5), (prec, cyc, b, err)
    S.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_block_solves_in_the_mix_equal_alone(prec):
    """Four systems in one stacked context, iterated in ticks of 3 with
    systems entering and leaving between ticks, give each system's result
    solved alone in a one-slot context in one call: same iterate bitwise,
    same iteration count; the oracle re-checks relres < 1e-8.  An idle block
    (f = 0) takes no iterations."""
    N = 65
    kinds = ["lognormal", "lognormal", "checker", "lognormal"]
    sys_list = systems(N, kinds, seed=21)
    J = levels_for(N)
    prm = LMGParams.identity(J)
    prm.wB[:, 1], prm.wR[:, 1], prm.wP[:, 1] = 0.1, 0.05, -0.05
    S = SquareBatch(N, 4, prm, precision=prec)
    m = S.m
    f = torch.zeros(4 * m, dtype=torch.float64, device=DEV)
    u = torch.zeros_like(f)
    iters = np.zeros(4, dtype=int)
    done = {}
    # block b enters at tick 2 b; ticks of 3 iterations
    for tick in range(200):
        for b in range(4):
            if tick == 2 * b:
                S.set_block(b, t64(sys_list[b][0]))
                f[b * m:(b + 1) * m] = t64(sys_list[b][1])
                u[b * m:(b + 1) * m] = 0
        info = S.solve(f, u, tol=1e-8, max_iter=3)
        for b in range(4):
            if tick < 2 * b or b in done:
                assert info.iters[b] == 0
                continue
            iters[b] += info.iters[b]
            if info.relres[b] < 1e-8:
                done[b] = u[b * m:(b + 1) * m].cpu().numpy().copy()
                f[b * m:(b + 1) * m] = 0
                u[b * m:(b + 1) * m] = 0
        if len(done) == 4:
            break
    assert len(done) == 4
    S.close()
    for b, (k, fb, p, H) in enumerate(sys_list):
        A1 = SquareBatch(N, 1, prm, precision=prec)
        A1.set_block(0, t64(k))
        ua = torch.zeros(m, dtype=torch.float64, device=DEV)
        info = A1.solve(t64(fb), ua, tol=1e-8, max_iter=400)
        assert int(info.iters[0]) == iters[b], (b, info.iters, iters)
        assert np.array_equal(ua.cpu().numpy(), done[b]), b
        assert O.relres(H, fb[:, None], done[b][:, None])[0] < 1e-8
        A1.close()


@pytest.mark.parametrize("N,prec", [(33, 32), (65, 32), (33, 64)])
def test_leading_blocks_solve_equals_whole_context(N, prec):
    """A solve over the leading k blocks (views of every level with fewer rows
    and the whole level's strides; on 33^2 with k = 1 every level runs in the
    single-block kernel, whose shared-memory copy then takes the strided
    rows) gives those blocks the results of a solve over all blocks: same
    iterates bitwise, same counts.  The other blocks' iterates are not
    touched, and their counts are reported as zero."""
    kinds = ["lognormal", "checker", "lognormal", "poisson", "lognormal"]
    sys_list = systems(N, kinds, seed=31)
    prm = LMGParams.identity(levels_for(N))
    prm.wB[:, 1], prm.wR[:, 1], prm.wP[:, 1] = 0.1, 0.05, -0.05
    S = SquareBatch(N, 5, prm, precision=prec)
    fill(S, sys_list)
    m = S.m
    f = t64(np.concatenate([x[1] for x in sys_list]))
    u_all = torch.zeros_like(f)
    info_all = S.solve(f, u_all, tol=1e-8, max_iter=300)
    assert info_all.status == 0
    for k in (1, 3, 5):
        u = torch.full_like(f, 7.0)
        u[:k * m] = 0
        info = S.solve(f, u, tol=1e-8, max_iter=300, nblocks=k)
        assert info.status == 0
        assert np.array_equal(info.iters[:k], info_all.iters[:k]), (k, info.iters, info_all.iters)
        assert np.all(info.iters[k:] == 0)
        assert torch.equal(u[:k * m], u_all[:k * m]), k
        assert torch.all(u[k * m:] == 7.0), k
    for b, (_, fb, _, H) in enumerate(sys_list):
        assert O.relres(H, fb[:, None], u_all[b * m:(b + 1) * m].cpu().numpy()[:, None])[0] < 1e-8
    S.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_stacked_halo2d_is_bitwise_neutral(prec):
    """On a stacked context (a grid of width N - 2 and slots (N - 2) rows,
    zero couplings between blocks) the 2D-tiled fused steps give the
    two-kernel block solve bitwise, for all blocks and for leading blocks."""
    N = 65
    sys_list = systems(N, ["lognormal", "checker", "lognormal"], seed=7)
    prm = LMGParams.identity(levels_for(N))
    prm.wB[:, 1], prm.wR[:, 1], prm.wP[:, 1] = 0.1, 0.05, -0.05
    f = t64(np.concatenate([x[1] for x in sys_list]))
    outs = []
    for bytes_ in (0, 1):
        S = SquareBatch(N, 3, prm, precision=prec)
        fill(S, sys_list)
        S.set_option("tail_work", 0)
        S.set_option("halo_rows", 0)
        S.set_option("halo2d_bytes", bytes_)
        res = []
        for k in (3, 2):
            u = torch.zeros_like(f)
            info = S.solve(f, u, tol=1e-8, max_iter=300, nblocks=k)
            res.append((u.clone(), info.iters.copy()))
        outs.append(res)
        S.close()
    for (u1, i1), (u0, i0) in zip(outs[1], outs[0]):
        assert torch.equal(u1, u0) and np.array_equal(i1, i0)


@pytest.mark.parametrize("prec", [32, 64])
def test_stacked_two_rows_are_bitwise_neutral(prec):
    """On a stacked context (one right-hand side per block, DIA levels of
    odd row counts) the two-rows-per-thread kernels give the one-row
    kernels' block solves bitwise, for all blocks and for leading blocks."""
    N = 65
    sys_list = systems(N, ["lognormal", "checker", "lognormal"], seed=9)
    prm = LMGParams.identity(levels_for(N))
    prm.wB[:, 1], prm.wR[:, 1], prm.wP[:, 1] = 0.1, 0.05, -0.05
    f = t64(np.concatenate([x[1] for x in sys_list]))
    outs = []
    for two in (0, 1):
        S = SquareBatch(N, 3, prm, precision=prec)
        fill(S, sys_list)
        S.set_option("tail_work", 0)
        S.set_option("dia_two_rows", two)
        res = []
        for k in (3, 2):
            u = torch.zeros_like(f)
            info = S.solve(f, u, tol=1e-8, max_iter=300, nblocks=k)
            res.append((u.clone(), info.iters.copy()))
        outs.append(res)
        S.close()
    for (u1, i1), (u0, i0) in zip(outs[1], outs[0]):
        assert torch.equal(u1, u0) and np.array_equal(i1, i0)


def test_stacked_refinement_replays_bitwise():
    """The stacked FP32 refinement loop (the cycle over all blocks, u += 2^s_b
    c, the per-block FP64 residual with the next cycle's scaled residual and
    first smoothing delta, the per-block test) equals, bitwise, a host
    replay through entry points that fold nothing: r = f - A u in FP64,
    s_b = ilogb ||r_b||, one FP32 cycle of the stack on float(2^-s_b r_b)
    from zero, u_b += 2^s_b c_b."""
    N = 65
    sys_list = systems(N, ["lognormal", "checker", "poisson"], seed=11)
    S = SquareBatch(N, 3, rand_params(levels_for(N), 5, 0.1), precision=32)
    fill(S, sys_list)
    m = S.m
    f = t64(np.concatenate([x[1] for x in sys_list]))
    K = 4
    u = torch.zeros_like(f)
    r = torch.empty_like(f)
    for _ in range(K):
        S.level_apply(0, "outer_residual", f, u, r)
        rn = np.sqrt((r.cpu().numpy().reshape(3, m) ** 2).sum(axis=1))
        sexp = np.frexp(rn)[1] - 1  # ilogb per block
        scale = torch.tensor(np.repeat(np.ldexp(1.0, -sexp), m), dtype=torch.float64, device=DEV)
        rhat = (r * scale).float()
        c = torch.zeros_like(rhat)
        S.vcycle(rhat, c)
        u = u + c.double() / scale
    us = torch.zeros_like(f)
    info = S.solve(f, us, tol=1e-300, max_iter=K)
    assert np.array_equal(info.iters, np.full(3, K))
    assert torch.equal(us, u), (us - u).abs().max().item()
    S.close()


def test_invalid_square_arguments():
    from paper_2608_29082_b300._lib import MGError
    with pytest.raises(MGError):
        SquareBatch(33, 0, LMGParams.identity(5))
    S = SquareBatch(17, 2, LMGParams.identity(4))
    with pytest.raises(ValueError):
        S.set_block(0, torch.zeros(10, dtype=torch.float64, device=DEV))
    with pytest.raises(MGError):
        S.set_block(2, torch.ones(S.n_elements, dtype=torch.float64, device=DEV))
    f = torch.zeros(2 * S.m, dtype=torch.float64, device=DEV)
    u = torch.zeros_like(f)
    for k in (0, 3, -1):
        with pytest.raises(MGError):
            S.solve(f, u, nblocks=k)
    S.close()


def test_contexts_created_and_solved_from_several_threads():
    """Set-up, graph capture and destruction on one thread while another
    thread captures and launches its own solves (the serving pattern): every
    thread's results equal the same work done on one thread, bitwise."""
    import threading
    N = 33
    sys_list = systems(N, ["lognormal", "checker"], seed=41)
    prm = LMGParams.identity(levels_for(N))
    prm.wB[:, 1] = 0.1

    def work(seed, out):
        torch.cuda.set_device(0)
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            res = []
            for rep in range(3):
                S = SquareBatch(N, 2, prm, precision=32)
                fill(S, sys_list)
                f = t64(np.concatenate([x[1] for x in sys_list]) * (1 + seed))
                u = torch.zeros_like(f)
                for k in (1, 2):
                    S.solve(f, u, tol=1e-8, max_iter=100, nblocks=k)
                res.append(u.cpu().numpy().copy())
                S.close()
            side.synchronize()
        out[seed] = res

    alone = {}
    for seed in range(3):
        work(seed, alone)
    together = {}
    threads = [threading.Thread(target=work, args=(seed, together)) for seed in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for seed in range(3):
        for a, b in zip(alone[seed], together[seed]):
            assert np.array_equal(a, b), seed
