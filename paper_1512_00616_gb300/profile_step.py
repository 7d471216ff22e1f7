"""One primal sweep plus one adjoint sweep (F = J_E, dF/dmu) on a named workload, for
profiler captures.  Usage:

    python -m paper_1512_00616_gb300.profile_step CONFIG NT [fp64|mixed]

NT below the workload's own number of steps shortens the period with the same time step
(T scaled by NT / Nt, the motion amplitudes by the same factor), so that a capture of
the same kernels holds a few GB of device memory instead of the whole period's
linearization.  Starts from the free stream.
"""
import sys

import numpy as np
import torch

from . import api as A


def main(argv):
    from pp_inputs import CONFIGS, PHYS, config_mesh, config_mu, free_stream_state
    name, Nt = argv[0], int(argv[1])
    prec = argv[2] if len(argv) > 2 else "fp64"
    c = CONFIGS[name]
    mesh = config_mesh(name)
    mu = config_mu(name)
    T = PHYS["T"] * Nt / c["Nt"]
    if Nt < c["Nt"]:
        mu = mu * (T / PHYS["T"])
    cfg = A.pp_config_default(p=c["p"], kin=c["kin"], T=T,
                              precision=A.PP_PREC_MIXED if prec == "mixed" else A.PP_PREC_FP64)
    ctx = A.pp_create(cfg)
    m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
    ne, _, nu = A.pp_mesh_info(m)
    u0 = torch.tensor(free_stream_state(ne, c["p"]).reshape(-1), dtype=torch.float64, device="cuda")
    uN, lamN, lam0 = torch.zeros_like(u0), torch.zeros_like(u0), torch.zeros_like(u0)
    torch.cuda.synchronize()
    A.pp_primal_period(ctx, m, mu, u0, Nt, u_final=uN)
    A.pp_adjoint_sweep(ctx, lamN, lam0, weights=np.array([-1.0 / T, 0.0]), n_mu=len(mu))
    torch.cuda.synchronize()
    print("ok", float(uN.norm()), float(lam0.norm()), A.pp_sweep_counts(ctx))
    A.pp_mesh_destroy(m)
    A.pp_destroy(ctx)


if __name__ == "__main__":
    main(sys.argv[1:])
