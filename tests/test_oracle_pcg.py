"""The oracle's Jacobi-preconditioned CG (the local solver of Fig. 1C)
against a direct solve on the masked subspace, its exact-arithmetic
termination bound, a diagonal system (one step), b = 0, and the SPD check."""
import numpy as np
import pytest

from oracle.mps import NotSPD, pcg


def _system(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = np.geomspace(1e-2, 10.0, n)
    A = (Q * lam) @ Q.T
    mask = rng.random(n) > 0.25
    return A, mask, rng


def test_matches_direct_solve_on_the_masked_subspace():
    A, mask, rng = _system(40, 1)
    b = rng.normal(size=40) * mask
    x0 = rng.normal(size=40)
    Am = A[np.ix_(mask, mask)]
    want = np.linalg.solve(Am, b[mask])
    x, it = pcg(lambda v: A @ v, b, x0, np.diag(A).copy(), mask, 1e-13, 1000)
    assert np.all(x[~mask] == 0.0)
    assert np.abs(x[mask] - want).max() < 1e-9 * np.abs(want).max()
    assert it <= 3 * int(mask.sum())


def test_diagonal_system_converges_in_one_step():
    d = np.linspace(1.0, 5.0, 12)
    mask = np.ones(12, dtype=bool)
    b = np.arange(1.0, 13.0)
    x, it = pcg(lambda v: d * v, b, np.zeros(12), d, mask, 1e-14, 50)
    assert it == 1 and np.allclose(x, b / d, rtol=0, atol=1e-14)


def test_zero_rhs_and_indefinite_operator():
    A, mask, rng = _system(20, 2)
    x, it = pcg(lambda v: A @ v, np.zeros(20), rng.normal(size=20), np.diag(A).copy(), mask, 1e-12, 100)
    assert it == 0 and not x.any()
    # a direction of negative curvature: -I with a positive preconditioner
    with pytest.raises(NotSPD):
        pcg(lambda v: -v, rng.normal(size=20) * mask, np.zeros(20), np.ones(20), mask, 1e-12, 200)
