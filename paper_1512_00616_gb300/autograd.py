"""torch.autograd.Function for mu -> (J_E, J_T) on the manifold of periodic solutions.

Forward: for every motion vector of the batch, Newton-Krylov shooting (Algorithm primal)
to a periodic initial state (warm-started by a callable or by the previous solution),
then the cycle-averaged flapping energy J_E = -W/T and thrust J_T = -J_x/T (Eq. qoi).
Backward: the periodic adjoint of every batch entry in one batched call
(pp_periodic_adjoint_batched; Algorithms dual and grad) for
F = g_E J_E + g_T J_T, i.e. weights (-g_E/T, -g_T/T) on (W, J_x); the linearization
is recomputed from the saved periodic state by a primal sweep (checkpointed every K
steps when the context's checkpoint_stride is K > 0).  Every step runs in libpp; this
module only orchestrates calls of the C ABI.
"""
import numpy as np
import torch

from . import api as A


class PeriodicSolver:
    """Context + mesh + period discretization shared by forward and backward."""

    def __init__(self, mesh, p, kin, Nt, tol=1e-10, T=5.0, device=0, warm_start=None, **cfg):
        self.cfg = A.pp_config_default(p=p, kin=kin, T=T, device=device, **cfg)
        self.ctx = A.pp_create(self.cfg)
        self.mesh = A.pp_mesh_create(self.ctx, mesh.verts, mesh.tris, mesh.ftag)
        self.ne, self.np, self.nu = A.pp_mesh_info(self.mesh)
        self.Nt, self.tol, self.T = Nt, tol, T
        self.device = torch.device(f"cuda:{device}")
        self.warm_start = warm_start      # callable mu -> device tensor [nu] or None
        self.last_u0 = None
        self.history = []

    def shoot(self, mu):
        guess = None
        if self.warm_start is not None:
            guess = self.warm_start(mu)
        elif self.last_u0 is not None:
            guess = self.last_u0.clone()
        u0 = torch.empty(self.nu, dtype=torch.float64, device=self.device)
        qoi, st = A.pp_shoot_nk(self.ctx, self.mesh, np.asarray(mu, dtype=np.float64), self.Nt, self.tol, u0,
                                u0_guess=guess)
        self.last_u0 = u0
        self.history.append(st)
        return u0, qoi

    def gradient(self, mu, u0, weights):
        F, g, st = A.pp_periodic_adjoint(self.ctx, self.mesh, np.asarray(mu, dtype=np.float64), self.Nt,
                                         np.asarray(weights, dtype=np.float64), u0=u0)
        return F, g

    def close(self):
        if self.ctx is not None:
            A.pp_mesh_destroy(self.mesh)
            A.pp_destroy(self.ctx)
            self.ctx = None


class PeriodicQoI(torch.autograd.Function):
    """apply(mu [B, n_mu] float64, solver) -> [B, 2] = (J_E, J_T) per motion vector."""

    @staticmethod
    def forward(ctx, mu, solver):
        mus = mu.detach().cpu().numpy().astype(np.float64)
        out = np.zeros((mus.shape[0], 2))
        u0s = []
        for b, m in enumerate(mus):
            u0, qoi = solver.shoot(m)
            out[b] = qoi[2], qoi[3]
            u0s.append(u0)
        ctx.solver = solver
        ctx.mus = mus
        ctx.u0s = u0s
        return torch.tensor(out, dtype=torch.float64, device=mu.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().cpu().numpy().astype(np.float64)
        solver = ctx.solver
        grads = np.zeros_like(ctx.mus)
        live = [b for b in range(len(ctx.mus)) if np.any(g[b])]
        if live:
            # one batched call: the periodic adjoint of every live entry (pp_periodic_adjoint_batched)
            w = np.stack([[-g[b, 0] / solver.T, -g[b, 1] / solver.T] for b in live])
            u0 = torch.cat([ctx.u0s[b] for b in live])
            _, gl = A.pp_periodic_adjoint_batched(solver.ctx, solver.mesh, ctx.mus[live], solver.Nt, w, u0)
            grads[live] = gl
        return torch.tensor(grads, dtype=torch.float64, device=grad_out.device), None
