"""Shared helpers for the GPU tests: build contexts and meshes through the
C-ABI binding, and seeded inputs from pp_inputs (no oracle arithmetic here)."""
import numpy as np

from pp_inputs import CONFIGS, KIN_FOURIER6, config_mesh, config_mu, free_stream_state, state_perturbation

PARITY_TOL = 1e-10   # relative FP64 parity bar (max-norm of the difference / max-norm of the reference)

TIGHT = dict(newton_tol=1e-13, newton_maxit=30, gmres_rtol=1e-6, gmres_restart=40, gmres_maxit=2000,
             lin_rtol=1e-13, nk_gmres_rtol=1e-8, nk_restart=40, nk_max_newton=20, nk_max_krylov=200,
             adj_tol=1e-13, adj_restart=40, adj_maxit=400)


def api():
    from paper_1512_00616_gb300 import api as A
    return A


def make(p, kin, mesh, **cfg):
    A = api()
    c = A.pp_config_default(p=p, kin=kin, **cfg)
    ctx = A.pp_create(c)
    m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
    return A, ctx, m


def to_dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x).reshape(-1), dtype=torch.float64, device="cuda")


def to_host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def perturbed_state(nt, p, seed, amp=1e-2):
    return (free_stream_state(nt, p) + state_perturbation(nt, p, seed, amp=amp)).reshape(-1)
