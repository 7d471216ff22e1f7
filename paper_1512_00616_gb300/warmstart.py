"""Learned warm start for Newton-Krylov shooting.

A small network maps the motion parameters mu to the POD coefficients of the periodic
initial state u0(mu).  The POD basis comes from a snapshot set of periodic states
produced by the GPU shooter itself.  Every arithmetic step runs in libpp kernels:

* snapshot Gram matrix, modes, projections and reconstructions: FP64 GEMMs
  (pp_gemm_f64);
* eigen-decomposition of the Gram matrix: one-block Jacobi (pp_syevj_f64);
* network forward and backward passes and Adam: pp_gemm_f32, pp_bias_act_f32,
  pp_gelu_backward_f32, pp_colsum_f32, pp_mse_f32, pp_adam_f32.

A prediction is used only if the shooting residual it starts from is small enough.
The first primal sweep of pp_shoot_nk evaluates that residual.  If it exceeds the
gate, the shooting is redone from the cold start (the steady state), as in the paper's
procedure.  So this module only ever improves the initial guess; it never changes the
periodic solution.

``python -m paper_1512_00616_gb300.warmstart --config c0`` runs the experiment.  It
generates data with the GPU shooter, trains, then compares NK iterations and wall time
on held-out mu against the steady-state cold start.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import api as A


# ------------------------------------------------------------------------------ POD
class POD:
    """Method of snapshots: D = S - mean, G = D^T D, G = V L V^T, modes Phi = D V L^{-1/2}."""

    def __init__(self, snapshots, n_modes):
        # snapshots: [n_snap, nu] float64 CUDA tensor (one periodic state per row)
        S = snapshots.contiguous()
        n, nu = S.shape
        dev = S.device
        ones = torch.ones(1, n, dtype=torch.float64, device=dev)
        self.mean = torch.zeros(1, nu, dtype=torch.float64, device=dev)
        A.pp_gemm(ones, S, self.mean, alpha=1.0 / n)            # mean = 1^T S / n
        D = S.clone()
        A.pp_gemm(ones, self.mean, D, ta=True, alpha=-1.0, beta=1.0)  # D = S - 1 mean
        G = torch.zeros(n, n, dtype=torch.float64, device=dev)
        A.pp_gemm(D, D, G, tb=True)                             # G = D D^T (rows are snapshots)
        V = torch.zeros_like(G)
        w = torch.zeros(n, dtype=torch.float64, device=dev)
        A.pp_syevj_f64(G, V, w)
        wh = w.cpu().numpy()
        order = np.argsort(-wh)[:min(n_modes, n - 1)]
        order = order[wh[order] > 1e-12 * wh[order[0]]]          # centred snapshots have rank <= n - 1
        Vk = V[:, torch.as_tensor(order, device=dev)].contiguous()          # [n, k] (gather)
        Vk_scaled = Vk.clone()
        inv_sqrt = torch.tensor(1.0 / np.sqrt(np.maximum(wh[order], 1e-300)), dtype=torch.float64, device=dev)
        diag = torch.diag(inv_sqrt)
        A.pp_gemm(Vk, diag, Vk_scaled)                          # Vk L^{-1/2}
        self.modes = torch.zeros(len(order), nu, dtype=torch.float64, device=dev)
        A.pp_gemm(Vk_scaled, D, self.modes, ta=True)            # orthonormal rows = L^{-1/2} Vk^T D
        self.energy = wh[order] / np.maximum(wh, 0).sum()

    def project(self, U):
        """U [m, nu] -> coefficients [m, k]."""
        C = torch.zeros(U.shape[0], self.modes.shape[0], dtype=torch.float64, device=U.device)
        A.pp_gemm(U.contiguous(), self.modes, C, tb=True)
        mc = torch.zeros(1, self.modes.shape[0], dtype=torch.float64, device=U.device)
        A.pp_gemm(self.mean, self.modes, mc, tb=True)
        ones = torch.ones(U.shape[0], 1, dtype=torch.float64, device=U.device)
        A.pp_gemm(ones, mc, C, alpha=-1.0, beta=1.0)            # C = (U - 1 mean) Phi^T
        return C

    def reconstruct(self, coef):
        """coefficients [m, k] -> states [m, nu]."""
        U = self.mean.expand(coef.shape[0], -1).contiguous().clone()
        A.pp_gemm(coef.contiguous(), self.modes, U, beta=1.0)   # U = 1 mean + coef Phi
        return U


# ------------------------------------------------------------------------------ network
class MLP:
    """sizes[0] -> ... -> sizes[-1] with GELU hidden activations, FP32, row-major."""

    def __init__(self, sizes, seed=0, device="cuda"):
        g = np.random.default_rng(seed)
        self.params = []
        for fi, fo in zip(sizes[:-1], sizes[1:]):
            lim = np.sqrt(6.0 / (fi + fo))
            W = torch.tensor(g.uniform(-lim, lim, (fi, fo)), dtype=torch.float32, device=device)
            b = torch.zeros(fo, dtype=torch.float32, device=device)
            self.params.append([W, b])
        self.m = [[torch.zeros_like(p) for p in layer] for layer in self.params]
        self.v = [[torch.zeros_like(p) for p in layer] for layer in self.params]
        self.step = 0

    def forward(self, X):
        self.cache = []
        H = X.contiguous()
        for li, (W, b) in enumerate(self.params):
            Z = torch.zeros(H.shape[0], W.shape[1], dtype=torch.float32, device=H.device)
            A.pp_gemm(H, W, Z)
            Hn = torch.empty_like(Z)
            A.pp_bias_act_f32(Z, b, Hn, li < len(self.params) - 1)
            self.cache.append((H, Z))
            H = Hn
        return H

    def backward(self, dY):
        grads = [None] * len(self.params)
        dH = dY.contiguous()
        for li in range(len(self.params) - 1, -1, -1):
            Hin, Z = self.cache[li]
            if li == len(self.params) - 1:
                dZ = dH
            else:
                dZ = torch.empty_like(Z)
                A.pp_gelu_backward_f32(Z, dH, dZ)
            W = self.params[li][0]
            dW = torch.zeros_like(W)
            A.pp_gemm(Hin, dZ, dW, ta=True)
            db = torch.zeros_like(self.params[li][1])
            A.pp_colsum_f32(dZ, db)
            grads[li] = (dW, db)
            if li > 0:
                dHn = torch.zeros_like(Hin)
                A.pp_gemm(dZ, W, dHn, tb=True)
                dH = dHn
        return grads

    def loss_and_grads(self, X, T):
        Y = self.forward(X)
        dY = torch.empty_like(Y)
        loss = torch.zeros(1, dtype=torch.float32, device=Y.device)
        A.pp_mse_f32(Y, T.contiguous(), dY, loss)
        return loss, self.backward(dY)

    def adam_step(self, grads, lr):
        self.step += 1
        for li, (gW, gb) in enumerate(grads):
            for pi, g in enumerate((gW, gb)):
                A.pp_adam_f32(self.params[li][pi], g, self.m[li][pi], self.v[li][pi], lr, self.step)


# ------------------------------------------------------------------------------ warm start
class LearnedWarmStart:
    def __init__(self, n_modes=64, hidden=256, seed=0):
        self.n_modes, self.hidden, self.seed = n_modes, hidden, seed

    def fit(self, mus, u0s, epochs=3000, lr=2e-3, log=None):
        """mus [n, n_mu] numpy, u0s [n, nu] float64 CUDA tensor of periodic states."""
        self.pod = POD(u0s, self.n_modes)
        k = self.pod.modes.shape[0]
        coef = self.pod.project(u0s).cpu().numpy()
        self.mu_mean, self.mu_std = mus.mean(0), mus.std(0) + 1e-12
        self.c_mean, self.c_std = coef.mean(0), coef.std(0) + 1e-12
        X = torch.tensor((mus - self.mu_mean) / self.mu_std, dtype=torch.float32, device=u0s.device)
        Y = torch.tensor((coef - self.c_mean) / self.c_std, dtype=torch.float32, device=u0s.device)
        self.net = MLP([mus.shape[1], self.hidden, self.hidden, k], seed=self.seed, device=u0s.device)
        self.losses = []
        for ep in range(epochs):
            loss, grads = self.net.loss_and_grads(X, Y)
            # cosine decay of the learning rate to 1% over the run
            lr_ep = lr * (0.01 + 0.99 * 0.5 * (1.0 + np.cos(np.pi * ep / max(epochs - 1, 1))))
            self.net.adam_step(grads, lr_ep)
            if ep % 100 == 0 or ep == epochs - 1:
                self.losses.append(float(loss.item()))
        return self

    def __call__(self, mu):
        X = torch.tensor(((np.atleast_2d(mu) - self.mu_mean) / self.mu_std), dtype=torch.float32,
                         device=self.pod.mean.device)
        c = self.net.forward(X).cpu().numpy().astype(np.float64) * self.c_std + self.c_mean
        coef = torch.tensor(c, dtype=torch.float64, device=self.pod.mean.device)
        return self.pod.reconstruct(coef)[0].contiguous()


def shoot_with_warm_start(ctx, mesh, mu, Nt, tol, predictor=None, gate=1e-2):
    """NK shooting from the learned prediction; falls back to the cold start (steady
    state) when the RMS periodicity residual at the prediction, ||R||_2 / sqrt(N_u),
    exceeds `gate`.  The first primal sweep of the shooting evaluates that residual; if
    it fails the gate, the shooting restarts cold (that sweep is counted)."""
    nu = A.pp_mesh_info(mesh)[2]
    u0 = torch.empty(nu, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    used = "cold"
    if predictor is not None:
        guess = predictor(mu)
        qoi, st = A.pp_shoot_nk(ctx, mesh, mu, Nt, tol, u0, u0_guess=guess, raise_on_noconv=False)
        pred_res = st["residual"][0]
        if pred_res / np.sqrt(nu) <= gate and st["status"] == A.PP_OK:
            used = "learned"
        else:
            first = st
            qoi, st = A.pp_shoot_nk(ctx, mesh, mu, Nt, tol, u0)
            st["newton_iters"] += first["newton_iters"] + 1
            st["krylov_iters"] += first["krylov_iters"]
            used = "fallback"
        st["prediction_residual"] = pred_res
    else:
        qoi, st = A.pp_shoot_nk(ctx, mesh, mu, Nt, tol, u0)
    torch.cuda.synchronize()
    return u0, qoi, st, used, time.perf_counter() - t0


def lhs(n, lo, hi, seed):
    """Latin-hypercube samples in the box [lo, hi]."""
    g = np.random.default_rng(seed)
    d = len(lo)
    u = (np.stack([g.permutation(n) for _ in range(d)], 1) + g.uniform(0, 1, (n, d))) / n
    return lo + u * (hi - lo)


def experiment(config="c0", n_train=96, n_test=16, tol=1e-8, epochs=6000, seed=44):
    """Data generation with the GPU shooter, POD + network training, then per held-out mu
    the time to a periodic gradient (u0 with ||R|| <= tol, then the periodic adjoint for
    J_E) by (a) plain FP64 from the steady-state cold start, (b) mixed precision from the
    learned warm start and (c) FP64 from the learned warm start."""
    from pp_inputs import CONFIGS, KIN_FOURIER6, MU_F6_BASE, MU_F6_SCALE, config_mesh
    c = CONFIGS[config]
    mesh = config_mesh(config)
    T = 5.0
    ctxs, meshes = {}, {}
    for name, prec in (("fp64", A.PP_PREC_FP64), ("mixed", A.PP_PREC_MIXED)):
        ctxs[name] = A.pp_create(A.pp_config_default(p=c["p"], kin=KIN_FOURIER6, precision=prec, adj_tol=1e-10))
        meshes[name] = A.pp_mesh_create(ctxs[name], mesh.verts, mesh.tris, mesh.ftag)
    lo, hi = MU_F6_BASE - 0.2 * MU_F6_SCALE, MU_F6_BASE + 0.2 * MU_F6_SCALE
    train = lhs(n_train, lo, hi, seed)
    test = lhs(n_test, lo, hi, seed + 1)
    nu = A.pp_mesh_info(meshes["mixed"])[2]
    # data generation (mixed precision, continuation from the previous periodic state)
    U = torch.empty(n_train, nu, dtype=torch.float64, device="cuda")
    prev = None
    t0 = time.perf_counter()
    for i in np.argsort(train[:, 0]):
        u0 = torch.empty(nu, dtype=torch.float64, device="cuda")
        A.pp_shoot_nk(ctxs["mixed"], meshes["mixed"], train[i], c["Nt"], 1e-10, u0, u0_guess=prev)
        U[i] = u0
        prev = u0
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    ws = LearnedWarmStart(n_modes=64).fit(train, U, epochs=epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    w = np.array([-1.0 / T, 0.0])  # F = J_E
    rows = []
    for mu in test:
        # (a) plain FP64, cold start
        t0 = time.perf_counter()
        _, _, st_a, _, _ = shoot_with_warm_start(ctxs["fp64"], meshes["fp64"], mu, c["Nt"], tol)
        _, g_a, _ = A.pp_periodic_adjoint(ctxs["fp64"], meshes["fp64"], mu, c["Nt"], w)
        t_a = time.perf_counter() - t0
        # (b) mixed precision, learned warm start
        t0 = time.perf_counter()
        _, _, st_b, used, _ = shoot_with_warm_start(ctxs["mixed"], meshes["mixed"], mu, c["Nt"], tol, predictor=ws)
        _, g_b, _ = A.pp_periodic_adjoint(ctxs["mixed"], meshes["mixed"], mu, c["Nt"], w)
        t_b = time.perf_counter() - t0
        # (c) FP64, learned warm start (the warm start's own effect)
        t0 = time.perf_counter()
        _, _, st_c, _, _ = shoot_with_warm_start(ctxs["fp64"], meshes["fp64"], mu, c["Nt"], tol, predictor=ws)
        _, g_c, _ = A.pp_periodic_adjoint(ctxs["fp64"], meshes["fp64"], mu, c["Nt"], w)
        t_c = time.perf_counter() - t0
        rows.append(dict(plain_newton=st_a["newton_iters"], plain_tangent_sweeps=st_a["krylov_iters"],
                         plain_s=t_a, learned_newton=st_b["newton_iters"],
                         learned_tangent_sweeps=st_b["krylov_iters"], learned_s=t_b,
                         fp64_learned_newton=st_c["newton_iters"], fp64_learned_tangent_sweeps=st_c["krylov_iters"],
                         fp64_learned_s=t_c,
                         grad_rel_diff_fp64_learned=float(np.linalg.norm(g_c - g_a) / np.linalg.norm(g_a)),
                         first_residual_plain=st_a["residual"][0],
                         first_residual_learned=st_b.get("prediction_residual", st_b["residual"][0]),
                         grad_rel_diff=float(np.linalg.norm(g_b - g_a) / np.linalg.norm(g_a)), used=used))
    for name in ctxs:
        A.pp_mesh_destroy(meshes[name])
        A.pp_destroy(ctxs[name])
    agg = {k: float(np.mean([r[k] for r in rows])) for k in rows[0] if k != "used"}
    agg["grad_rel_diff_max"] = float(np.max([r["grad_rel_diff"] for r in rows]))
    return dict(config=config, n_train=n_train, n_test=n_test, tol=tol, data_s=t_data, train_s=t_train,
                final_loss=ws.losses[-1], pod_modes=int(ws.pod.modes.shape[0]),
                pod_energy=float(ws.pod.energy.sum()), fallbacks=sum(r["used"] != "learned" for r in rows),
                mean=agg)


def cold_time_to_gradient(config="c1", n_test=1, tol=1e-8, seed=45):
    """Time to a periodic gradient from the steady-state cold start, plain FP64 against
    mixed precision, on held-out mu of the +-20% box (no network: for workloads where
    generating a training set does not fit the available GPU time)."""
    from pp_inputs import CONFIGS, KIN_FOURIER6, MU_F6_BASE, MU_F6_SCALE, config_mesh
    c = CONFIGS[config]
    mesh = config_mesh(config)
    T = 5.0
    lo, hi = MU_F6_BASE - 0.2 * MU_F6_SCALE, MU_F6_BASE + 0.2 * MU_F6_SCALE
    test = lhs(n_test, lo, hi, seed)
    w = np.array([-1.0 / T, 0.0])  # F = J_E
    rows = []
    grads = {}
    for name, prec in (("fp64", A.PP_PREC_FP64), ("mixed", A.PP_PREC_MIXED)):
        ctx = A.pp_create(A.pp_config_default(p=c["p"], kin=KIN_FOURIER6, precision=prec, adj_tol=1e-10))
        m = A.pp_mesh_create(ctx, mesh.verts, mesh.tris, mesh.ftag)
        for i, mu in enumerate(test):
            t0 = time.perf_counter()
            _, _, st, _, _ = shoot_with_warm_start(ctx, m, mu, c["Nt"], tol)
            t1 = time.perf_counter()
            F, g, ast = A.pp_periodic_adjoint(ctx, m, mu, c["Nt"], w)
            t2 = time.perf_counter()
            grads[(name, i)] = g
            rows.append(dict(precision=name, mu=i, newton=st["newton_iters"], tangent_sweeps=st["krylov_iters"],
                             periodicity=st["residual"][-1], shoot_s=t1 - t0, adjoint_s=t2 - t1,
                             total_s=t2 - t0, J_E=F))
        A.pp_mesh_destroy(m)
        A.pp_destroy(ctx)
    for r in rows:
        if r["precision"] == "mixed":
            ga, gb = grads[("fp64", r["mu"])], grads[("mixed", r["mu"])]
            r["grad_rel_diff_vs_fp64"] = float(np.linalg.norm(gb - ga) / np.linalg.norm(ga))
    return dict(config=config, tol=tol, rows=rows)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c0")
    ap.add_argument("--train", type=int, default=96)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--cold-only", action="store_true",
                    help="plain FP64 against mixed precision from the cold start, no network")
    a = ap.parse_args()
    if a.cold_only:
        print(json.dumps(cold_time_to_gradient(a.config, a.test)))
    else:
        print(json.dumps(experiment(a.config, a.train, a.test, epochs=a.epochs)))


if __name__ == "__main__":
    main()
