"""Pins for the DIRK3 tableau (Eqs. dirk, dirk-stage; scheme reading: Alexander 1977)."""
import os

import numpy as np

from oracle.dirk import tableau, dirk_step_scalar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dirk3_alexander.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_tableau_matches_published_values():
    A, b, c = tableau()
    g = _golden()
    assert abs(A[0, 0] - g["gamma"]) < 1e-10
    assert abs(c[1] - g["c2"]) < 1e-9
    assert abs(b[0] - g["b1"]) < 1e-9
    assert abs(b[1] - g["b2"]) < 1e-9


def test_order_conditions_and_stiff_accuracy():
    A, b, c = tableau()
    assert np.allclose(A.sum(1), c, atol=1e-15)
    assert abs(b.sum() - 1.0) < 1e-15
    assert abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c**2 - 1.0 / 3.0) < 1e-15
    assert abs(b @ A @ c - 1.0 / 6.0) < 1e-15
    assert np.allclose(A[-1], b, atol=0)          # stiffly accurate
    assert np.allclose(np.triu(A, 1), 0.0)        # diagonally implicit
    # L-stability: R(z) -> 1 - b^T A^{-1} 1 = 0 as z -> -inf
    assert abs(1.0 - b @ np.linalg.solve(A, np.ones(3))) < 1e-13


def _prothero_robinson_error(lam, n):
    f = lambda y, t: lam * (y - np.cos(t)) - np.sin(t)
    dfdy = lambda y, t: lam
    y, t, T = 1.0, 0.0, 1.0
    dt = T / n
    for _ in range(n):
        y = dirk_step_scalar(f, dfdy, y, t, dt)
        t += dt
    return abs(y - np.cos(T))


def test_observed_third_order():
    errs = [_prothero_robinson_error(-1.0, n) for n in (10, 20, 40, 80)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(7.0 < r < 9.0 for r in ratios), ratios
    # stiff case stays accurate (L-stable, stiffly accurate)
    assert _prothero_robinson_error(-1e4, 20) < 1e-6
