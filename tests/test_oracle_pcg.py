"""Pins of the oracle's inner-PCG preconditioner (Section 4.2) against what conjugate gradients
must compute, independently of the recurrences: the k-th iterate minimises the A-norm of the
error over the Krylov space K_k(M A, M b) (a Galerkin solve on an explicit, orthonormalised
Krylov basis), k = 1 is the closed-form scaled step alpha M b, enough iterations solve A x = b,
and k = 0 is the direct preconditioner.  Then LOBPCG with it: same eigenpairs, and fewer outer
iterations than with the direct preconditioner.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import laplace, lobpcg as olob, multigrid, pcg, rng  # noqa: E402

DIMS = (8, 7, 6)


def setup():
    scale = laplace.default_scale(DIMS)
    A = olob.Laplace7(DIMS, scale)
    M = multigrid.VCycle(DIMS, scale, 2)
    Ad = laplace.dense_matrix(DIMS, scale)
    return A, M, Ad


def galerkin_krylov(Ad, Md, b, k):
    """argmin_{x in K_k(M A, M b)} ||x - A^-1 b||_A via an orthonormal Krylov basis."""
    v = Md @ b
    K = [v]
    for _ in range(k - 1):
        K.append(Md @ (Ad @ K[-1]))
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    y = np.linalg.solve(Q.T @ Ad @ Q, Q.T @ b)
    return Q @ y


def test_k0_is_the_direct_preconditioner():
    A, M, _ = setup()
    B = rng.uniform_block(3, A.n, 3)
    assert np.array_equal(pcg.pcg_columns(A, M, B, 0), M(B))


def test_k1_is_the_optimal_multiple_of_mb():
    A, M, Ad = setup()
    b = rng.uniform_block(4, A.n, 1)[:, 0]
    z = M(b[:, None])[:, 0]
    alpha = (b @ z) / (z @ (Ad @ z))
    x = pcg.pcg_columns(A, M, b[:, None], 1)[:, 0]
    assert np.max(np.abs(x - alpha * z)) <= 1e-13 * np.max(np.abs(x))


def test_iterates_are_the_krylov_galerkin_solutions():
    A, M, Ad = setup()
    Md = M(np.eye(A.n))                       # the V-cycle as a dense matrix (it is linear)
    B = rng.uniform_block(5, A.n, 2)
    for k in (2, 4, 7):
        X = pcg.pcg_columns(A, M, B, k)
        for j in range(2):
            want = galerkin_krylov(Ad, Md, B[:, j], k)
            assert np.max(np.abs(X[:, j] - want)) <= 1e-9 * np.max(np.abs(want)), k
    # and without a preconditioner it is plain CG (M = I)
    ident = lambda R: R.copy()  # noqa: E731
    X = pcg.pcg_columns(A, ident, B, 6)
    want = galerkin_krylov(Ad, np.eye(A.n), B[:, 0], 6)
    assert np.max(np.abs(X[:, 0] - want)) <= 1e-9 * np.max(np.abs(want))


def test_many_iterations_solve_the_system():
    A, M, Ad = setup()
    B = rng.uniform_block(6, A.n, 2)
    X = pcg.pcg_columns(A, M, B, 60)
    assert np.max(np.abs(Ad @ X - B)) <= 1e-10 * np.max(np.abs(B))
    # the A-norm of the error decreases monotonically with k
    Xs = np.linalg.solve(Ad, B[:, :1])
    errs = []
    for k in range(0, 12):
        Xk = pcg.pcg_columns(A, M, B[:, :1], k) if k else np.zeros_like(Xs)     # k = 0 here: x_0 = 0
        E = Xk - Xs
        errs.append(float(E[:, 0] @ (Ad @ E[:, 0])))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))


def test_lobpcg_with_inner_pcg():
    A, M, _ = setup()
    m, tol = 4, 1e-10
    X0 = rng.uniform_block(2, A.n, m)
    direct = olob.lobpcg(A, X0, tol, 300, T=M)
    k0 = olob.lobpcg(A, X0, tol, 300, T=pcg.InnerPCG(A, M, 0))
    assert np.array_equal(direct.lam, k0.lam) and direct.iters == k0.iters
    exact = laplace.exact_eigenvalues(DIMS, A.scale, m)
    iters = [direct.iters]
    for k in (2, 6):
        r = olob.lobpcg(A, X0, tol, 300, T=pcg.InnerPCG(A, M, k))
        assert r.status == "converged"
        assert np.max(np.abs(r.lam - exact) / exact) < 1e-12
        iters.append(r.iters)
    # better inner solves cut the outer iterations against the direct V-cycle (the count is not
    # monotone in k: LOBPCG stays linearly convergent even with T = A^-1, Section 4.2)
    assert iters[1] < iters[0] and iters[2] < iters[0], iters
