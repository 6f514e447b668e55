"""Pins of the small dense steps (oracle side)."""
import numpy as np
import pytest

from oracle import dense


def spd(q, seed, cond=1e6):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((q, q)))
    ev = np.logspace(0, np.log10(cond), q)
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("q", [1, 3, 16, 48])
def test_scaled_cholesky_reconstructs(q):
    G = spd(q, q)
    R = dense.scaled_cholesky(G)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.max(np.abs(R.T @ R - G)) <= 1e-13 * np.max(np.abs(G))


def test_scaled_cholesky_is_scale_invariant():
    """Section 2.2: the factorisation must be invariant to column scaling."""
    G = spd(12, 1)
    d = 2.0 ** np.arange(-20, 28, 4)        # powers of two: the scaling itself is exact
    R1 = dense.scaled_cholesky(G)
    R2 = dense.scaled_cholesky(d[:, None] * G * d[None, :])
    assert np.array_equal(R2, R1 * d[None, :])


def test_scaled_cholesky_handles_badly_scaled_columns():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((500, 6)) * np.array([1e-12, 1, 1e6, 1e-3, 1e9, 1e-7])
    R = dense.scaled_cholesky(W.T @ W)
    Q = dense.apply_inverse_upper(W, R)
    assert np.max(np.abs(Q.T @ Q - np.eye(6))) < 1e-12


def test_scaled_cholesky_breakdown():
    W = np.random.default_rng(4).standard_normal((50, 4))
    W[:, 3] = W[:, 1]
    with pytest.raises(dense.Breakdown):
        dense.scaled_cholesky(W.T @ W)
    with pytest.raises(dense.Breakdown):
        dense.scaled_cholesky(np.array([[1.0, np.nan], [np.nan, 1.0]]))


def test_rayleigh_ritz_generalized():
    q, m = 24, 8
    rng = np.random.default_rng(5)
    A0 = rng.standard_normal((q, q))
    gA = A0 + A0.T
    gB = spd(q, 6, cond=1e3)
    lam, C = dense.rayleigh_ritz(gA, gB, m)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(gA @ C - gB @ C * lam[None, :])) < 1e-10 * np.max(np.abs(gA))
    assert np.max(np.abs(C.T @ gB @ C - np.eye(m))) < 1e-11
    # eigenvalues of the non-symmetric gB^-1 gA by a general (different) eigensolver
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(gB, gA)).real)[:m]
    assert np.max(np.abs(ev - lam)) < 1e-8 * np.max(np.abs(ev))


def test_rayleigh_ritz_reduces_to_standard_problem():
    A0 = np.random.default_rng(7).standard_normal((10, 10))
    gA = A0 + A0.T
    lam, C = dense.rayleigh_ritz(gA, np.eye(10), 4)
    assert np.allclose(lam, np.linalg.eigvalsh(gA)[:4], rtol=0, atol=1e-13)
