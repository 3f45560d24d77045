"""Differentiable simulation: gradient of a pose-matching loss with respect to
every per-element stiffness parameter (the quantity the paper's adjoint
Gauss-Newton material fitting consumes, Sec. 6.1).

The forward pass runs N time steps solved to equilibrium (PD iterations
followed by Newton steps with an FP64 residual, `pd_equilibrium_step`),
keeping only the FP64 state (x, v) every `checkpoint_every` steps.  The backward pass walks the
segments from the last one, recomputes each segment's positions from its
checkpoint, and runs the adjoint recurrence backwards through them
(`pd_adjoint_step`).  Parameterisation: gamma_s = theta, gamma_v =
volume_ratio * theta, so dL/dtheta = dL/dgamma_s + volume_ratio dL/dgamma_v.
"""
from __future__ import annotations

import numpy as np
import torch

from .sim import Adjoint, Mesh


class DiffSim:
    def __init__(self, rest, tets, pinned, tet_domain, n_domains, density, dt, pin_targets_fn, n_steps,
                 x0=None, v0=None, gravity=(0.0, 0.0, -9.81), volume_ratio=10.0, checkpoint_every=10,
                 n_pd_iter=10, n_newton=3, cg_iters=30, store_all=False):
        self.mesh = Mesh(rest, tets, pinned, tet_domain, n_domains, density)
        self.adj = Adjoint(self.mesh, cg_iters)
        self.dt = float(dt)
        self.pins = pin_targets_fn
        self.N = int(n_steps)
        self.C = max(1, int(checkpoint_every))
        self.gravity = tuple(float(g) for g in gravity)
        self.ratio = float(volume_ratio)
        self.n_pd, self.n_newton = int(n_pd_iter), int(n_newton)
        self.store_all = store_all
        n_v = self.mesh.n_v
        self.x0 = torch.as_tensor(np.asarray(rest if x0 is None else x0), dtype=torch.float32, device="cuda")
        self.v0 = torch.zeros((n_v, 3), device="cuda") if v0 is None else torch.as_tensor(v0, dtype=torch.float32,
                                                                                            device="cuda")
        self._pins_dev = [None] * self.N

    def _pin(self, n):
        if self._pins_dev[n] is None:
            p = self.pins(n)
            self._pins_dev[n] = None if p is None else torch.as_tensor(p, dtype=torch.float32, device="cuda")
        return self._pins_dev[n]

    def set_theta(self, theta: torch.Tensor):
        th = theta.detach().to(device="cuda", dtype=torch.float32).contiguous()
        self.mesh.set_materials(th, self.ratio * th)
        self.mesh.prefactor(self.dt)

    def forward(self, theta, targets):
        """Returns (loss tensor, checkpoints, stored positions or None)."""
        self.set_theta(theta)
        m, a = self.mesh, self.adj
        a.set_state64(self.x0.double(), self.v0.double())
        ckpts = {0: a.get_state64()}
        stored = [] if self.store_all else None
        loss = torch.zeros(1, device="cuda", dtype=torch.float64)
        x = torch.empty((m.n_v, 3), device="cuda")
        for n in range(self.N):
            a.equilibrium_step(self._pin(n), self.gravity, self.n_pd, self.n_newton, x_out=x)
            a.pose_misfit_accumulate(x, targets[n + 1], loss)
            if stored is not None:
                stored.append((x.clone(), a.get_state64()[0]))
            if (n + 1) % self.C == 0 and n + 1 < self.N:
                ckpts[n + 1] = a.get_state64()      # FP64 checkpoints: the recomputation is bitwise the original
        return loss.reshape(()), ckpts, stored

    def backward(self, ckpts, stored, targets):
        m, a = self.mesh, self.adj
        gs = torch.zeros(m.n_t, device="cuda")
        gv = torch.zeros(m.n_t, device="cuda")
        a.reset()
        x = torch.empty((m.n_v, 3), device="cuda")
        dl = torch.empty((m.n_v, 3), device="cuda")
        scratch = torch.zeros(1, device="cuda", dtype=torch.float64)
        for start in sorted(ckpts, reverse=True):
            end = min(start + self.C, self.N)
            if stored is not None:
                xs = stored[start:end]
            else:
                a.set_state64(*ckpts[start])
                xs = []
                for n in range(start, end):
                    a.equilibrium_step(self._pin(n), self.gravity, self.n_pd, self.n_newton, x_out=x)
                    xs.append((x.clone(), a.get_state64()[0]))
            for n in range(end - 1, start - 1, -1):
                xn, xn64 = xs[n - start]
                a.pose_misfit_accumulate(xn, targets[n + 1], scratch, dl)   # dL/dx_n = 2 (x_n - xhat_n), 0 on pins
                a.step64(xn64, dl, gs, gv)
        return gs, gv


class PoseLoss(torch.autograd.Function):
    """L(theta) = sum_{n=1..N} sum_{free v} ||x_{n,v}(theta) - xhat_{n,v}||^2."""

    @staticmethod
    def forward(ctx, theta, sim: DiffSim, targets):
        loss, ckpts, stored = sim.forward(theta, targets)
        ctx.sim, ctx.ckpts, ctx.stored, ctx.targets = sim, ckpts, stored, targets
        ctx.theta_device = theta.device
        return loss.to(theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        sim = ctx.sim
        gs, gv = sim.backward(ctx.ckpts, ctx.stored, ctx.targets)
        g = sim.adj.tied_gradient(gs, gv, sim.ratio, scale=grad_out)
        return g.to(device=ctx.theta_device), None, None


def pose_loss(theta: torch.Tensor, sim: DiffSim, targets) -> torch.Tensor:
    return PoseLoss.apply(theta, sim, targets)
