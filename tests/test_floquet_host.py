"""The library's Hessenberg QR (the eigenvalue step of pp_floquet), host code run on the
CPU through the C ABI: every computed eigenvalue is an exact eigenvalue of a nearby matrix
(smallest singular value of H - lambda I at round-off level), symmetric tridiagonal
matrices give LAPACK's eigenvalues, and a companion matrix gives its polynomial's roots."""
import numpy as np
import pytest

A = pytest.importorskip("paper_1512_00616_gb300.api")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 200])
def test_backward_stable_on_random_hessenberg(n):
    rng = np.random.default_rng(n)
    H = np.triu(rng.standard_normal((n, n)), -1)
    ev = A.pp_hessenberg_eigvals(H)
    assert len(ev) == n
    scale = np.linalg.norm(H, 2)
    for lam in ev:
        smin = np.linalg.svd(H - lam * np.eye(n), compute_uv=False)[-1]
        assert smin <= 1e-12 * scale
    # conjugate pairs stay paired: the spectrum of a real matrix is closed under conjugation
    assert np.allclose(np.sort_complex(ev), np.sort_complex(np.conj(ev)), atol=1e-10 * scale)


def test_symmetric_tridiagonal_matches_lapack():
    rng = np.random.default_rng(7)
    n = 60
    d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
    H = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ev = np.sort(A.pp_hessenberg_eigvals(H).real)
    assert np.max(np.abs(ev - np.linalg.eigvalsh(H))) <= 1e-12 * np.max(np.abs(ev))


def test_companion_matrix_roots():
    roots = np.array([0.9, 0.5 + 0.3j, 0.5 - 0.3j, -0.2, 0.05j, -0.05j])
    c = np.real(np.poly(roots))                      # monic coefficients
    n = len(roots)
    H = np.zeros((n, n))
    H[0, :] = -c[1:]
    H[np.arange(1, n), np.arange(n - 1)] = 1.0      # upper Hessenberg companion form
    ev = A.pp_hessenberg_eigvals(H)
    for r in roots:
        assert np.min(np.abs(ev - r)) <= 1e-10
