"""Training of Theta (Algorithm 3) through the hand-written adjoint.

UnrolledCycles is a torch.autograd.Function around mg_forward_record /
mg_vcycle_backward; ResidualLoss around mg_residual_loss.  Trainer runs the
paper's loop with Rprop (Sec. 3.1) on the host over the few dozen scalars of
Theta; every vector operation runs in libmg.so.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .solver import LMGParams, Solver

# column order of the flat parameter block
COLS = {"theta": 0, "eta": 1, "wB1": 2, "wB2": 3, "wR1": 4, "wR2": 5, "wP1": 6, "wP2": 7}


class UnrolledCycles(torch.autograd.Function):
    """u_K = LMG^K(f, u_0; Theta).  theta_flat: CPU FP64 tensor [J-1, 8]."""

    @staticmethod
    def forward(ctx, theta_flat, f, u0, solver: Solver, n_cycles: int):
        p = solver.params
        solver.set_params(LMGParams.from_flat(theta_flat.detach().cpu().numpy(), p.nu_pre,
                                              p.nu_post))
        u = u0.detach().clone()
        solver.forward_record(f.detach(), u, n_cycles)
        ctx.solver, ctx.n_cycles = solver, n_cycles
        return u

    @staticmethod
    def backward(ctx, grad_u):
        gin, gf, gp = ctx.solver.backward(grad_u.contiguous(), ctx.n_cycles)
        return gp.cpu(), gf, gin, None, None


class ResidualLoss(torch.autograd.Function):
    """sum_b w_b ||f_b - A u_b||^2 (a device FP64 scalar); gradient w.r.t. u
    computed by the library alongside the value."""

    @staticmethod
    def forward(ctx, u, f, weights, solver: Solver):
        loss, _, g = solver.residual_loss(f.detach(), u.detach(), weights, grad=True)
        ctx.save_for_backward(g)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (g,) = ctx.saved_tensors
        return g * grad_loss.to(g.dtype), None, None, None


@dataclass
class ParamMap:
    """Which entries of Theta [J-1, 8] are trained and which share one value
    across levels.  train: column names that are trained; shared: column names
    whose value is one scalar for every level (e.g. the SAGEConv weights)."""
    J: int
    train: tuple = ("theta", "eta", "wB1", "wB2", "wR1", "wR2", "wP1", "wP2")
    shared: tuple = ()
    index: np.ndarray = field(init=False)  # [J-1, 8] -> z index or -1

    def __post_init__(self):
        idx = -np.ones((self.J - 1, 8), dtype=np.int64)
        k = 0
        for name, col in COLS.items():
            if name not in self.train:
                continue
            if name in self.shared:
                idx[:, col] = k
                k += 1
            else:
                idx[:, col] = np.arange(k, k + self.J - 1)
                k += self.J - 1
        self.index = idx
        self.size = k

    def gather(self, flat: np.ndarray) -> np.ndarray:
        x = flat.reshape(self.J - 1, 8)
        z = np.zeros(self.size)
        for (l, c), k in np.ndenumerate(self.index):
            if k >= 0:
                z[k] = x[l, c]  # shared: last level wins (all equal by construction)
        return z

    def scatter(self, z: np.ndarray, flat: np.ndarray) -> np.ndarray:
        x = flat.reshape(self.J - 1, 8).copy()
        m = self.index >= 0
        x[m] = z[self.index[m]]
        return x.ravel()

    def reduce_grad(self, g: np.ndarray) -> np.ndarray:
        """dL/dz: per-level gradients summed over the levels sharing a value."""
        gz = np.zeros(self.size)
        m = self.index >= 0
        np.add.at(gz, self.index[m], g.reshape(self.J - 1, 8)[m])
        return gz


class Rprop:
    """Resilient backpropagation (Riedmiller & Braun): per-parameter step
    sizes grown by eta_plus while the gradient keeps its sign, shrunk by
    eta_minus (and the step skipped) when it flips."""

    def __init__(self, n: int, lr: float = 0.01, etas=(0.5, 1.2), step_sizes=(1e-6, 50.0)):
        self.step = np.full(n, lr)
        self.prev = np.zeros(n)
        self.etaminus, self.etaplus = etas
        self.smin, self.smax = step_sizes

    def update(self, z: np.ndarray, g: np.ndarray) -> np.ndarray:
        g = g.copy()
        s = g * self.prev
        self.step = np.where(s > 0, np.minimum(self.step * self.etaplus, self.smax),
                             np.where(s < 0, np.maximum(self.step * self.etaminus, self.smin),
                                      self.step))
        g[s < 0] = 0.0
        self.prev = g
        return z - np.sign(g) * self.step


@dataclass
class TrainLog:
    losses: list = field(default_factory=list)
    params: LMGParams | None = None
    epochs: int = 0


class Trainer:
    """Algorithm 3 with K unrolled cycles per epoch: u_0 = 0 (or carried over
    when carry_u), u_K = LMG^K(f, u_0), loss = mean_b ||r_K||^2/||r_0||^2,
    gradient by the adjoint, Rprop step.  Stops when loss/loss_0 <= rel_tol
    or after max_epochs."""

    def __init__(self, solver: Solver, pmap: ParamMap, n_cycles: int = 10, lr: float = 0.01,
                 carry_u: bool = False):
        self.S = solver
        self.pmap = pmap
        self.K = n_cycles
        self.carry_u = carry_u
        self.opt = Rprop(pmap.size, lr=lr)

    def loss_and_grad(self, params: LMGParams, f: torch.Tensor, u0: torch.Tensor):
        S = self.S
        S.set_params(params)
        _, r0, _ = S.residual_loss(f, u0)
        w = 1.0 / (f.shape[1] * r0)
        u = u0.clone()
        S.forward_record(f, u, self.K)
        loss, _, gu = S.residual_loss(f, u, w, grad=True)
        _, _, gp = S.backward(gu, self.K, want_inputs=False)
        return float(loss.item()), gp.cpu().numpy().ravel(), u

    def train(self, f: torch.Tensor, params: LMGParams, max_epochs: int = 100,
              rel_tol: float = 1e-6, log_every: int = 0) -> TrainLog:
        flat = params.flat()
        z = self.pmap.gather(flat)
        u0 = torch.zeros_like(f)
        log = TrainLog()
        loss0 = None
        best_loss, best_z = np.inf, z.copy()
        for ep in range(max_epochs):
            p = LMGParams.from_flat(self.pmap.scatter(z, flat), params.nu_pre, params.nu_post)
            loss, g, u = self.loss_and_grad(p, f, u0)
            log.losses.append(loss)
            if loss0 is None:
                loss0 = loss
            if not np.isfinite(loss):
                break
            if loss < best_loss:
                best_loss, best_z = loss, z.copy()
            if log_every and ep % log_every == 0:
                print(f"epoch {ep:4d} loss {loss:.6e}")
            if loss <= rel_tol * loss0:
                break
            z = self.opt.update(z, self.pmap.reduce_grad(g))
            if self.carry_u:
                u0 = u.detach()
            log.epochs = ep + 1
        # the best evaluated parameters (the last update is never evaluated)
        log.params = LMGParams.from_flat(self.pmap.scatter(best_z, flat), params.nu_pre,
                                         params.nu_post)
        log.best_loss = best_loss
        return log
