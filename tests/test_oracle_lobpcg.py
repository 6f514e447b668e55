"""Pins of the oracle LOBPCG iteration (Sections 2.2, 2.3 and 4.1)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import laplace, lobpcg as L, multigrid, rng

EPS = np.finfo(np.float64).eps


def kron_sum_matrix(dims, scale):
    nx, ny, nz = dims
    T = lambda n: 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    I = np.eye
    return scale * (np.kron(I(nz), np.kron(I(ny), T(nx))) + np.kron(I(nz), np.kron(T(ny), I(nx)))
                    + np.kron(T(nz), np.kron(I(ny), I(nx))))


def max_angle(U, V):
    return float(np.max(scipy.linalg.subspace_angles(U, V)))


@pytest.mark.parametrize("precond", [False, True])
def test_small_grid_matches_brute_force(precond):
    dims, m = (6, 7, 8), 5
    A = L.Laplace7(dims, 1.0)
    T = multigrid.VCycle(dims, 1.0, 2) if precond else None
    res = L.lobpcg(A, rng.uniform_block(2, A.n, m), 1e-9, 300, T=T)
    assert res.status == "converged"
    ev, V = np.linalg.eigh(kron_sum_matrix(dims, 1.0))
    assert np.max(np.abs(res.lam - ev[:m]) / ev[:m]) < 1e-12
    # distinct eigenvalues on this machine: compare eigenvectors one by one
    for j in range(m):
        assert max_angle(res.X[:, [j]], V[:, [j]]) < 1e-6
    assert np.all(res.resid <= 1e-9 * np.abs(res.lam) * (1 + 1e-6))


@pytest.fixture(scope="module")
def c1_run():
    """48^3 interior grid, m = 8, 4-level V-cycle, relative tol 1e-8, seed 2."""
    dims = (48, 48, 48)
    A = L.Laplace7(dims)
    T = multigrid.VCycle(dims, A.scale, 4)
    res = L.lobpcg(A, rng.uniform_block(2, A.n, 8), 1e-8, 200, T=T, record=True)
    return dims, A, res


@pytest.mark.slow
def test_c1_against_closed_form(c1_run):
    dims, A, res = c1_run
    assert res.status == "converged"
    exact = laplace.exact_eigenvalues(dims, A.scale, 8)
    assert np.max(np.abs(res.lam - exact) / exact) < 1e-12
    # The final check recomputes every residual from A X once J is empty and sends failing
    # columns back, so every returned residual meets the tolerance.
    assert np.all(res.resid <= 1e-8 * np.abs(res.lam))
    # complete clusters (1 + 3 + 3) against the exact eigenspaces
    for idx in ([0], [1, 2, 3], [4, 5, 6]):
        E = laplace.exact_eigenspace(dims, A.scale, exact[idx[0]], max_index=4)
        assert E.shape[1] == len(idx)
        assert max_angle(res.X[:, idx], E) < 1e-6
    # the cut cluster (1 of the 3-fold (1,1,3) eigenvalue) lies inside its eigenspace
    E = laplace.exact_eigenspace(dims, A.scale, exact[7], max_index=4)
    assert E.shape[1] == 3
    x = res.X[:, 7]
    assert np.linalg.norm(x - E @ (E.T @ x)) < 1e-6


@pytest.mark.slow
def test_c1_invariants_every_iteration(c1_run):
    dims, A, res = c1_run
    exact = laplace.exact_eigenvalues(dims, A.scale, 8)
    # Ritz values come from Gram entries that are sums of n products: their rounding error
    # is of order sqrt(n) * eps relative, which sets the slack of both inequalities.
    slack = np.sqrt(A.n) * EPS
    prev = None
    for h in res.history:
        assert h["orth"] <= 1e-12                                   # X^T X = I
        assert np.all(h["lam"] >= exact * (1 - slack))               # Courant-Fischer
        if prev is not None:
            assert np.all(h["lam"] <= prev * (1 + slack))            # non-increasing
        prev = h["lam"]
    # J only shrinks while columns remain active; it can grow only at the final check
    segment = []
    for h in res.history:
        segment.append(len(h["J"]))
        if "recheck_J" in h:
            assert segment == sorted(segment, reverse=True)
            segment = []
    assert segment == sorted(segment, reverse=True)


def test_final_check_sends_failing_locked_columns_back():
    """Soft locking (Section 2.3) keeps locked columns in the Rayleigh-Ritz basis, so a column
    that passed its test can be rotated above the tolerance afterwards.  On this 16^3 start the
    printed rule (exit once J is empty) returns a column above tol; the final check finds it with a
    fresh A X, reactivates it, and the returned residuals -- recomputed here with the independently
    assembled dense operator -- all meet the tolerance."""
    dims, m, tol = (16, 16, 16), 4, 1e-8
    A = L.Laplace7(dims)
    T = multigrid.VCycle(dims, A.scale, 3)
    X0 = rng.uniform_block(2, A.n, m)
    M = kron_sum_matrix(dims, A.scale)
    literal = L.lobpcg(A, X0, tol, 300, T=T, final_check=False)
    checked = L.lobpcg(A, X0, tol, 300, T=T, record=True)
    assert literal.status == checked.status == "converged"
    r_lit = np.linalg.norm(M @ literal.X - literal.X * literal.lam, axis=0)
    r_chk = np.linalg.norm(M @ checked.X - checked.X * checked.lam, axis=0)
    assert np.max(r_lit / literal.lam) > tol                  # the printed rule misses it here
    assert np.all(r_chk <= tol * checked.lam * (1 + 1e-6))
    rechecks = [h["recheck_J"] for h in checked.history if "recheck_J" in h]
    assert rechecks[0] and rechecks[-1] == []                 # one reactivation, then a clean check
    assert checked.iters > literal.iters
    exact = laplace.exact_eigenvalues(dims, A.scale, m)
    assert np.max(np.abs(checked.lam - exact) / exact) < 1e-12


@pytest.mark.slow
@pytest.mark.parametrize("dims", [(16, 16, 16), (16, 17, 18)])
def test_paper_accuracy_claim_reduced_size(dims):
    """Section 4.1: 50 smallest eigenpairs, tol 1e-6 on the residual norm, relative
    eigenvalue error below 1e-8, both with multiplicities (cube) and clusters (box)."""
    A = L.Laplace7(dims, 1.0)
    T = multigrid.VCycle(dims, 1.0, 3)
    res = L.lobpcg(A, rng.uniform_block(2, A.n, 50), 1e-6, 300, T=T, tol_mode="absolute")
    assert res.status == "converged"
    exact = laplace.exact_eigenvalues(dims, 1.0, 50)
    assert np.max(np.abs(res.lam - exact) / exact) < 1e-8


def test_soft_locked_pairs_keep_improving():
    """Section 2.3 (figure of soft locking at residual 1e-1, m = 10): locked pairs stay in
    the Rayleigh-Ritz basis and their eigenvalue errors do not grow."""
    dims, m = (12, 12, 12), 10
    A = L.Laplace7(dims, 1.0)
    T = multigrid.VCycle(dims, 1.0, 2)
    res = L.lobpcg(A, rng.uniform_block(3, A.n, m), 5e-3, 100, T=T, tol_mode="absolute", record=True)
    assert res.status == "converged"
    exact = laplace.exact_eigenvalues(dims, 1.0, m)
    err = np.array([h["lam"] - exact for h in res.history])
    lock_k = {}
    for h, nxt in zip(res.history, res.history[1:]):
        for j in set(h["J"]) - set(nxt["J"]):
            lock_k[j] = h["k"]
    assert len(lock_k) >= 5
    improved = 0
    for j, k in lock_k.items():
        after = err[k:, j]
        assert np.all(after[1:] <= after[:-1] + np.sqrt(A.n) * EPS * exact[j])
        improved += after[-1] < 0.5 * after[0]
    assert improved >= 1


def test_paper_gram_variant_agrees_with_explicit():
    """The Gram blocks as printed (Lambda and I blocks) vs the explicit Gram blocks."""
    dims = (20, 20, 20)
    A = L.Laplace7(dims)
    T = multigrid.VCycle(dims, A.scale, 3)
    X0 = rng.uniform_block(2, A.n, 8)
    r1 = L.lobpcg(A, X0, 1e-8, 200, T=T, gram="explicit")
    r2 = L.lobpcg(A, X0, 1e-8, 200, T=T, gram="paper")
    assert r1.status == r2.status == "converged"
    assert np.max(np.abs(r1.lam - r2.lam) / r1.lam) < 1e-12
    assert abs(r1.iters - r2.iters) <= 1


def test_preconditioner_cuts_iterations():
    """Section 4.2: without preconditioning LOBPCG needs far more iterations."""
    dims = (16, 16, 16)
    A = L.Laplace7(dims)
    X0 = rng.uniform_block(4, A.n, 4)
    with_t = L.lobpcg(A, X0, 1e-8, 400, T=multigrid.VCycle(dims, A.scale, 3))
    without = L.lobpcg(A, X0, 1e-8, 400, T=None)
    assert with_t.status == "converged"
    assert without.iters > 2 * with_t.iters


def test_status_outcomes():
    dims = (6, 6, 6)
    A = L.Laplace7(dims)
    X0 = rng.uniform_block(2, A.n, 4)
    dup = X0.copy()
    dup[:, 3] = dup[:, 1]
    assert L.lobpcg(A, dup, 1e-8, 50).status == "breakdown"
    bad = X0.copy()
    bad[5, 2] = np.nan
    assert L.lobpcg(A, bad, 1e-8, 50).status == "nonfinite"
    one = L.lobpcg(A, X0, 1e-8, 1)
    assert one.status == "not_converged" and one.iters == 1
    assert np.all(np.isfinite(one.lam)) and np.max(np.abs(one.X.T @ one.X - np.eye(4))) < 1e-12


def test_absolute_and_relative_tolerance_modes():
    dims = (8, 8, 8)
    A = L.Laplace7(dims)
    X0 = rng.uniform_block(2, A.n, 3)
    T = multigrid.VCycle(dims, A.scale, 2)
    rel = L.lobpcg(A, X0, 1e-6, 100, T=T)
    ab = L.lobpcg(A, X0, 1e-6, 100, T=T, tol_mode="absolute")
    assert np.all(rel.resid <= 1e-6 * rel.lam * (1 + 1e-6))
    assert np.all(ab.resid <= 1e-6 * (1 + 1e-6))
    assert ab.iters >= rel.iters     # lambda ~ 1e2 here, so the absolute test is stricter


def test_exact_eigenspace_start_converges_at_pass_zero():
    """X0 spanning the exact eigenspace of the m smallest eigenvalues: every residual is at the
    rounding level at pass k = 0, so the loop exits there with iters = 0 and the closed-form
    eigenvalues (the exit test of the residuals and the soft-locking test, reading R11)."""
    dims = (5, 6, 7)                               # distinct axes: the smallest eigenvalues are simple
    A = L.Laplace7(dims)
    modes = laplace.exact_modes(dims, A.scale, 3)
    X0 = np.stack([laplace.exact_eigenvector(dims, abc) for _, abc in modes], axis=1)
    X0 = X0 @ np.array([[1.0, 0.3, -0.2], [0.0, 2.0, 0.5], [0.0, 0.0, 0.7]])   # any basis of the space
    r = L.lobpcg(A, X0, 1e-8, 50, T=multigrid.VCycle(dims, A.scale, 2))
    assert r.status == "converged" and r.iters == 0
    want = np.array([lam for lam, _ in modes])
    assert np.max(np.abs(r.lam - want) / want) < 1e-13


def test_maxit_zero_only_checks_the_start():
    dims = (6, 5, 4)
    A = L.Laplace7(dims)
    X0 = rng.uniform_block(2, A.n, 3)
    r = L.lobpcg(A, X0, 1e-8, 0)
    assert r.status == "not_converged" and r.iters == 0
    # the result is the Rayleigh-Ritz of the start (the set-up): orthonormal X, Ritz values of span(X0)
    assert np.max(np.abs(r.X.T @ r.X - np.eye(3))) < 1e-12
    Q, _ = np.linalg.qr(X0)
    H = Q.T @ A(Q)
    assert np.max(np.abs(r.lam - np.linalg.eigvalsh(0.5 * (H + H.T))) / r.lam) < 1e-12


@pytest.mark.parametrize("dims,m", [((7, 5, 3), 1), ((2, 1, 1), 1), ((2, 2, 1), 2), ((3, 2, 1), 3)])
def test_single_vector_and_largest_block(dims, m):
    """m = 1 (plain locally optimal preconditioned CG on one vector), tiny grids, and the largest
    block m = n / 2: the m smallest eigenvalues of the dense operator."""
    A = L.Laplace7(dims)
    X0 = rng.uniform_block(3, A.n, m)
    r = L.lobpcg(A, X0, 1e-10, 200, T=multigrid.VCycle(dims, A.scale, 1))
    assert r.status == "converged"
    want = np.linalg.eigvalsh(laplace.dense_matrix(dims, A.scale))[:m]
    assert np.max(np.abs(r.lam - want) / want) < 1e-12
