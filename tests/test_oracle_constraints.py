"""Pins of the oracle's constraint steps (Section 2.2 the constraint projections, the hard locking of
Section 2.3) against brute force.

The ground truth is a dense eigendecomposition of the 7-point Laplacian assembled here as a
Kronecker sum of 1-D second differences (independently of the oracle's stencil code), on a
6 x 7 x 8 box whose low eigenvalues are simple.  With Y = the first l eigenvectors the
constrained iteration must return eigenpairs l .. l+m-1; Y replaced by Y M (another basis of the
same span, badly scaled) must give the same result, which fails if the (Y^T Y)^-1 factor of the
projector is dropped or transposed; calling the solver again with the computed eigenvectors as
constraints (the repeated calls the paper recommends for many eigenpairs) must continue the
spectrum.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import lobpcg as olob, rng  # noqa: E402

DIMS = (6, 7, 8)


def kron_laplacian(dims, scale):
    nx, ny, nz = dims

    def d2(k):
        return 2 * np.eye(k) - np.eye(k, k, 1) - np.eye(k, k, -1)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    # point index p = i + nx (j + ny k): x fastest, so x is the last Kronecker factor
    return scale * (np.kron(np.kron(Iz, Iy), d2(nx)) + np.kron(np.kron(Iz, d2(ny)), Ix) +
                    np.kron(np.kron(d2(nz), Iy), Ix))


@pytest.fixture(scope="module")
def truth():
    A = olob.Laplace7(DIMS, 1.0)
    M = kron_laplacian(DIMS, 1.0)
    mu, V = np.linalg.eigh(M)
    gaps = np.diff(mu[:16]) / mu[1:16]
    assert np.all(gaps > 1e-3)          # simple eigenvalues: single vectors are comparable
    return A, mu, V


def test_constrained_iteration_returns_the_next_eigenpairs(truth):
    A, mu, V = truth
    l, m = 5, 4
    Y = V[:, :l]
    res = olob.lobpcg(A, rng.uniform_block(2, A.n, m), 1e-10, 400, Y=Y)
    assert res.status == "converged"
    assert np.max(np.abs(res.lam - mu[l:l + m]) / mu[l:l + m]) < 1e-12
    assert np.max(np.abs(Y.T @ res.X)) < 1e-12
    for j in range(m):      # each eigenvector up to sign
        c = abs(float(V[:, l + j] @ res.X[:, j]))
        assert c > 1 - 1e-12


def test_constraint_projection_keeps_a_mixing_preconditioner_out_of_span_y(truth):
    """A diagonal preconditioner that does not commute with A puts components of span(Y) into
    T R; only the constraint projection of W keeps them out (without it the iteration drifts to the locked pairs)."""
    A, mu, V = truth
    l, m = 5, 4
    Y = V[:, :l]
    d = np.random.default_rng(11).uniform(0.3, 3.0, A.n)
    res = olob.lobpcg(A, rng.uniform_block(2, A.n, m), 1e-10, 400, T=lambda R: R * d[:, None], Y=Y)
    assert res.status == "converged"
    assert np.max(np.abs(res.lam - mu[l:l + m]) / mu[l:l + m]) < 1e-12
    assert np.max(np.abs(Y.T @ res.X)) < 1e-11


def test_constraints_depend_only_on_their_span(truth):
    A, mu, V = truth
    l, m = 5, 4
    Y = V[:, :l]
    g = np.random.default_rng(7)
    M = g.standard_normal((l, l)) @ np.diag([1e3, 1.0, 1e-3, 10.0, 0.1])
    Y2 = Y @ M                           # same span, far from orthonormal
    a = olob.lobpcg(A, rng.uniform_block(2, A.n, m), 1e-10, 400, Y=Y)
    b = olob.lobpcg(A, rng.uniform_block(2, A.n, m), 1e-10, 400, Y=Y2)
    assert b.status == "converged"
    assert np.max(np.abs(a.lam - b.lam) / a.lam) < 1e-12
    assert abs(a.iters - b.iters) <= 1
    assert np.max(np.abs(Y.T @ b.X)) < 1e-11
    # the projector with the (Y^T Y)^-1 factor dropped is not a projector for this Y2: a check
    # that the test above could tell the difference
    V0 = rng.uniform_block(3, A.n, 2)
    wrong = V0 - Y2 @ (Y2.T @ V0)
    assert np.max(np.abs(Y.T @ wrong)) > 1.0


def test_repeated_calls_continue_the_spectrum(truth):
    """Hard locking by repeated calls: each call's eigenvectors become constraints of the next."""
    A, mu, V = truth
    m, tol = 4, 1e-10
    Ys = np.zeros((A.n, 0))
    found = []
    for call in range(3):
        res = olob.lobpcg(A, rng.uniform_block(2 + call, A.n, m), tol, 400, Y=Ys if Ys.shape[1] else None)
        assert res.status == "converged"
        found.extend(res.lam)
        Ys = np.hstack([Ys, res.X])
    found = np.array(found)
    # the locked vectors carry errors ~ tol^2-level in lambda and ~ tol / gap in angle; the later
    # eigenvalues stay within the Rayleigh-quotient error of those angles
    assert np.max(np.abs(found - mu[:3 * m]) / mu[:3 * m]) < 1e-12
    assert np.max(np.abs(Ys.T @ Ys - np.eye(3 * m))) < 1e-9


def test_dependent_constraints_break_down(truth):
    A, mu, V = truth
    Y = np.hstack([V[:, :3], V[:, :1] * 2.0])
    res = olob.lobpcg(A, rng.uniform_block(2, A.n, 3), 1e-8, 50, Y=Y)
    assert res.status == "breakdown"
