"""Learned warm start: the hand-written network, Adam, eigensolver and POD kernels
against the NumPy oracle, and the gain of the trained predictor over the cold start."""
import numpy as np
import pytest

from oracle import mlp as OM

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_mlp_loss_gradients_and_adam_match_oracle():
    from paper_1512_00616_gb300.warmstart import MLP
    from paper_1512_00616_gb300 import api as A
    net = MLP([6, 256, 256, 64], seed=3)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((32, 6))
    T = rng.standard_normal((32, 64))
    Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
    Tg = torch.tensor(T, dtype=torch.float32, device="cuda")
    loss, grads = net.loss_and_grads(Xg, Tg)
    params = [(W.double().cpu().numpy(), b.double().cpu().numpy()) for W, b in net.params]
    ref_loss, ref_grads = OM.loss_and_grads(params, X, T)
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    for (gW, gb), (rW, rb) in zip(grads, ref_grads):
        assert np.max(np.abs(gW.double().cpu().numpy() - rW)) <= 1e-5 * np.max(np.abs(rW))
        assert np.max(np.abs(gb.double().cpu().numpy() - rb)) <= 1e-5 * np.max(np.abs(rb)) + 1e-9
    # one Adam step on the first weight matrix
    W0 = net.params[0][0].double().cpu().numpy()
    net.adam_step(grads, lr=1e-3)
    rW, _, _ = OM.adam(W0, grads[0][0].double().cpu().numpy(), 0.0, 0.0, 1, 1e-3)
    assert np.max(np.abs(net.params[0][0].double().cpu().numpy() - rW)) <= 1e-6


def test_jacobi_eigensolver_and_pod():
    from paper_1512_00616_gb300 import api as A
    from paper_1512_00616_gb300.warmstart import POD
    rng = np.random.default_rng(1)
    B = rng.standard_normal((96, 96))
    S = B @ B.T
    G = torch.tensor(S, dtype=torch.float64, device="cuda")
    V = torch.zeros_like(G)
    w = torch.zeros(96, dtype=torch.float64, device="cuda")
    A.pp_syevj_f64(G, V, w)
    wn, Vn = w.cpu().numpy(), V.cpu().numpy()
    assert np.allclose(np.sort(wn), np.linalg.eigvalsh(S), rtol=1e-11, atol=1e-10 * np.abs(wn).max())
    assert np.linalg.norm(S @ Vn - Vn * wn) <= 1e-10 * np.linalg.norm(S)
    # POD of snapshots lying in a 5-dimensional affine space: 5 modes reproduce them exactly
    base = rng.standard_normal((5, 300))
    snaps = rng.standard_normal((40, 5)) @ base + rng.standard_normal(300)
    U = torch.tensor(snaps, dtype=torch.float64, device="cuda")
    pod = POD(U, 5)
    Mm = pod.modes.cpu().numpy()
    assert np.allclose(Mm @ Mm.T, np.eye(5), atol=1e-10)
    rec = pod.reconstruct(pod.project(U)).cpu().numpy()
    assert np.max(np.abs(rec - snaps)) <= 1e-9 * np.max(np.abs(snaps))


@pytest.mark.parametrize("n", [257, 512])
def test_jacobi_eigensolver_multi_block(n):
    """n > 256 (the 512-snapshot Gram matrix of the configured POD): the multi-CTA sweeps
    against LAPACK's symmetric eigensolver, with a clustered spectrum like a Gram matrix."""
    from paper_1512_00616_gb300 import api as A
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.exp(-np.linspace(0.0, 20.0, n)) * rng.uniform(0.5, 1.5, n)   # decaying, like POD
    S = (Q * lam) @ Q.T
    S = 0.5 * (S + S.T)
    G = torch.tensor(S, dtype=torch.float64, device="cuda")
    V = torch.zeros_like(G)
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    A.pp_syevj_f64(G, V, w)
    wn, Vn = w.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.eigvalsh(S)
    assert np.max(np.abs(np.sort(wn) - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.linalg.norm(S @ Vn - Vn * wn) <= 1e-11 * np.linalg.norm(S)
    assert np.max(np.abs(Vn.T @ Vn - np.eye(n))) <= 1e-11


def test_learned_warm_start_beats_cold_start():
    from paper_1512_00616_gb300.warmstart import experiment
    r = experiment("tiny", n_train=24, n_test=3, tol=1e-8, epochs=4000)
    print(r)
    assert r["fallbacks"] == 0
    assert r["mean"]["learned_newton"] < r["mean"]["plain_newton"]
    assert r["mean"]["first_residual_learned"] < r["mean"]["first_residual_plain"]
    # both paths reach the same periodic gradient (1e-6 accuracy target)
    assert r["mean"]["grad_rel_diff_max"] <= 1e-6
