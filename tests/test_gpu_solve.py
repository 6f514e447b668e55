"""End-to-end parity of the CUDA LOBPCG solve with the CPU oracle, through the C ABI.

Bars (float64 form): eigenvalues within 1e-10 relative of the oracle and of the closed form of
Section 4.1; eigenvectors within 1e-6 in subspace angle over complete eigenvalue clusters (a
cluster cut by the block has no unique basis; there each computed vector must lie in the exact
eigenspace); iteration counts within 10% of the oracle's on the same seeded initial block.
"""
import ctypes

import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import laplace, lobpcg as olob, multigrid, rng  # noqa: E402
from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import LobpcgError, Solver  # noqa: E402


def angle(U, V):
    return float(np.max(scipy.linalg.subspace_angles(U, V)))


def oracle_run(dims, scale, m, tol, maxit, levels, seed=2, tol_mode="relative", gram="explicit"):
    A = olob.Laplace7(dims, scale)
    T = multigrid.VCycle(dims, A.scale, levels) if levels else None
    return olob.lobpcg(A, rng.uniform_block(seed, A.n, m), tol, maxit, T=T, tol_mode=tol_mode, gram=gram)


def within_10pct(a, b):
    return abs(a - b) <= max(1, round(0.1 * b))


@pytest.mark.parametrize("dims,scale,m,levels", [((6, 7, 8), 1.0, 5, None), ((6, 7, 8), 1.0, 5, 2),
                                                 ((12, 11, 10), 1.0, 6, 2), ((16, 16, 16), None, 4, 3)])
def test_small_solves_match_oracle(dims, scale, m, levels):
    tol, maxit = 1e-9, 300
    s = Solver(dims, scale=scale, levels=levels, precond="gmg" if levels else "none")
    out = s.solve(m, tol=tol, maxit=maxit, seed=2)
    ref = oracle_run(dims, s.scale, m, tol, maxit, levels)
    assert out["status_name"] == "ok" and ref.status == "converged"
    lam = np.array(out["lam"])
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10
    exact = laplace.exact_eigenvalues(dims, s.scale, m)
    assert np.max(np.abs(lam - exact) / exact) < 1e-10
    assert within_10pct(out["iters"], ref.iters), (out["iters"], ref.iters)
    assert out["max_rel_resid"] <= tol * (1 + 1e-6)
    X = out["X"].cpu().numpy().T
    for c in laplace.eigen_clusters(exact):
        if c[-1] < m - 1 or len(laplace.exact_eigenspace(dims, s.scale, exact[c[0]], max_index=8).T) == len(c):
            assert angle(X[:, c], ref.X[:, c]) < 1e-6


@pytest.fixture(scope="module")
def c1():
    """48^3 interior grid, m = 8, 4-level V-cycle (2+2 weighted-Jacobi sweeps, w = 2/3), tol 1e-8."""
    dims, m, tol = (48, 48, 48), 8, 1e-8
    s = Solver(dims, levels=4)
    out = s.solve(m, tol=tol, maxit=200, seed=2)
    s.close()
    ref = oracle_run(dims, laplace.default_scale(dims), m, tol, 200, 4)
    return dims, out, ref


def test_c1_eigenvalues_and_iterations(c1):
    dims, out, ref = c1
    lam = np.array(out["lam"])
    exact = laplace.exact_eigenvalues(dims, laplace.default_scale(dims), 8)
    assert out["status_name"] == "ok"
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10
    assert np.max(np.abs(lam - exact) / exact) < 1e-10
    assert within_10pct(out["iters"], ref.iters), (out["iters"], ref.iters)
    # the final check (every residual from a fresh A X once J is empty) holds every column to tol
    assert out["max_rel_resid"] <= 1e-8 * (1 + 1e-6)
    assert np.all(np.array(out["resid"]) <= 1e-8 * lam * (1 + 1e-6))


def test_c1_eigenvectors(c1):
    dims, out, ref = c1
    scale = laplace.default_scale(dims)
    X = out["X"].cpu().numpy().T
    assert np.max(np.abs(X.T @ X - np.eye(8))) < 1e-12
    exact = laplace.exact_eigenvalues(dims, scale, 8)
    for idx in ([0], [1, 2, 3], [4, 5, 6]):           # complete clusters
        assert angle(X[:, idx], ref.X[:, idx]) < 1e-6
        E = laplace.exact_eigenspace(dims, scale, exact[idx[0]], max_index=4)
        assert angle(X[:, idx], E) < 1e-6
    E = laplace.exact_eigenspace(dims, scale, exact[7], max_index=4)   # cut 3-fold cluster
    assert np.linalg.norm(X[:, 7] - E @ (E.T @ X[:, 7])) < 1e-6


def test_c2_full_size_properties():
    """128^3 (2,097,152 unknowns), m = 16, 6-level V-cycle, tol 1e-8: the bench workload."""
    dims, m = (128, 128, 128), 16
    s = Solver(dims, levels=6)
    out = s.solve(m, tol=1e-8, maxit=200, seed=2)
    scale = laplace.default_scale(dims)
    exact = laplace.exact_eigenvalues(dims, scale, m)
    lam = np.array(out["lam"])
    assert out["status_name"] == "ok"
    assert np.max(np.abs(lam - exact) / exact) < 1e-10
    assert out["max_rel_resid"] <= 1e-8 * (1 + 1e-6)
    Xd = out["X"]
    G = (Xd @ Xd.T).cpu().numpy()
    assert np.max(np.abs(G - np.eye(m))) < 1e-12
    X = Xd.cpu().numpy().T
    for c in laplace.eigen_clusters(exact)[:5]:       # complete clusters 1, 3, 3, 3, 1
        E = laplace.exact_eigenspace(dims, scale, exact[c[0]], max_index=4)
        assert E.shape[1] == len(c)
        assert angle(X[:, c], E) < 1e-6
    s.close()


def test_paper_gram_variant_matches_explicit():
    dims = (20, 20, 20)
    r = {}
    for g in ("explicit", "paper"):
        s = Solver(dims, levels=3, gram=g)
        r[g] = s.solve(8, tol=1e-8, maxit=200, seed=2)
        s.close()
    a, b = np.array(r["explicit"]["lam"]), np.array(r["paper"]["lam"])
    # The two forms of the Gram blocks round differently; near convergence the basis [X, W, P]
    # is ill conditioned and the Ritz values inherit eps * cond of the scaled Gram B, so the
    # forms agree to a few thousand ulps, well inside the 1e-10 bound against the oracle.
    assert np.max(np.abs(a - b) / a) < 1e-11
    assert abs(r["explicit"]["iters"] - r["paper"]["iters"]) <= 1
    ref = oracle_run(dims, laplace.default_scale(dims), 8, 1e-8, 200, 3, gram="paper")
    assert np.max(np.abs(b - ref.lam) / ref.lam) < 1e-10


def test_soft_locking_matches_oracle():
    """Section 2.3 demo shape: m = 10, loose tolerance, locked pairs keep improving."""
    dims, m = (12, 12, 12), 10
    s = Solver(dims, scale=1.0, levels=2, tol_mode="absolute")
    out = s.solve(m, tol=5e-3, maxit=100, seed=3)
    ref = oracle_run(dims, 1.0, m, 5e-3, 100, 2, seed=3, tol_mode="absolute")
    lam = np.array(out["lam"])
    assert out["status_name"] == "ok"
    assert out["iters"] == ref.iters
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10


def test_solve_is_deterministic():
    s = Solver((24, 24, 24), levels=3)
    a = s.solve(6, tol=1e-8, maxit=100, seed=4)
    b = s.solve(6, tol=1e-8, maxit=100, seed=4)
    assert a["lam"] == b["lam"] and a["iters"] == b["iters"]
    assert torch.equal(a["X"], b["X"])


def test_stepwise_api_matches_solve():
    s = Solver((16, 16, 16), levels=3)
    full = s.solve(4, tol=1e-8, maxit=100, seed=2)
    s.begin(4, tol=1e-8, seed=2)
    rc = capi.NOT_CONVERGED
    while rc == capi.NOT_CONVERGED:
        rc = s.iterate(1)
    s.finish()
    step = s.result()
    assert step["lam"] == full["lam"] and step["iters"] == full["iters"]


def test_fixed_work_with_zero_tolerance():
    s = Solver((16, 16, 16), levels=3)
    s.begin(4, tol=0.0, seed=2)
    assert s.iterate(7) == capi.NOT_CONVERGED
    assert s.info.iters == 7 and s.info.active == 4


def test_status_outcomes():
    dims = (8, 8, 8)
    s = Solver(dims, levels=2)
    out = s.solve(4, tol=1e-8, maxit=1, seed=2)
    assert out["status_name"] == "not_converged" and out["iters"] == 1
    X = out["X"].cpu().numpy().T
    assert np.max(np.abs(X.T @ X - np.eye(4))) < 1e-12
    X0 = torch.from_numpy(rng.uniform_block(2, s.n, 4).T.copy())
    X0[3] = X0[1]
    s.set_initial(X0)
    with pytest.raises(LobpcgError) as e:
        s.solve(4, tol=1e-8, maxit=10)
    assert e.value.code == capi.ERR_BREAKDOWN
    X0 = torch.from_numpy(rng.uniform_block(2, s.n, 4).T.copy())
    X0[2, 5] = float("nan")
    s.set_initial(X0)
    with pytest.raises(LobpcgError) as e:
        s.solve(4, tol=1e-8, maxit=10)
    assert e.value.code == capi.ERR_NONFINITE
    for bad in (0, 101, 300):
        with pytest.raises(LobpcgError) as e:
            s.solve(bad, tol=1e-8, maxit=10)
        assert e.value.code == capi.ERR_ARG
    with pytest.raises(LobpcgError):
        s.solve(4, tol=-1.0, maxit=10)
    s.close()


def test_call_order_and_allocator_failure():
    h = ctypes.c_void_p()
    assert capi.lobpcg_create(ctypes.byref(h), 0, None, None, capi.FP64) == capi.OK
    assert capi.lobpcg_solve(h, 4, 1e-8, 10, 2, None) == capi.ERR_STATE
    lam = (ctypes.c_double * 4)()
    assert capi.lobpcg_get_eigenpairs(h, lam, None, 0, 0, None) == capi.ERR_STATE
    assert capi.lobpcg_set_preconditioner(h, capi.PRECOND_GMG, 2, 2, 2, 2 / 3) == capi.ERR_STATE
    capi.lobpcg_destroy(h)
    # an allocator that always fails -> LOBPCG_ERR_OOM, handle stays usable for destroy
    fail = capi.Allocator(None, capi.ALLOC_FN(lambda c, n, s: None), capi.FREE_FN(lambda c, p, n, s: None))
    assert capi.lobpcg_create(ctypes.byref(h), 0, None, ctypes.byref(fail), capi.FP64) == capi.OK
    assert capi.lobpcg_set_operator(h, capi.LAPLACE7, 8, 8, 8, 1.0, None) == capi.OK
    assert capi.lobpcg_solve(h, 4, 1e-8, 10, 2, None) == capi.ERR_OOM
    assert "allocation" in capi.lobpcg_last_error(h)
    assert capi.lobpcg_destroy(h) == capi.OK


@pytest.mark.parametrize("dims,m", [((14, 13, 12), 40), ((12, 12, 11), 64)])
def test_wide_blocks_match_oracle(dims, m):
    """Blocks wider than 32 columns (Rayleigh-Ritz bases up to 3m = 192, the Gram split into
    several thread blocks per row range, the Cholesky factors of 40..64 columns): eigenvalues
    within 1e-10 of the oracle and of the dense eigenvalues, iterations within 10 %."""
    tol, maxit = 1e-8, 300
    s = Solver(dims, scale=1.0, levels=2)
    out = s.solve(m, tol=tol, maxit=maxit, seed=2)
    s.close()
    ref = oracle_run(dims, 1.0, m, tol, maxit, 2)
    assert out["status_name"] == "ok" and ref.status == "converged"
    lam = np.array(out["lam"])
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10
    want = np.linalg.eigvalsh(laplace.dense_matrix(dims, 1.0))[:m]
    assert np.max(np.abs(lam - want) / want) < 1e-10
    assert within_10pct(out["iters"], ref.iters), (out["iters"], ref.iters)
    assert out["max_rel_resid"] <= tol * (1 + 1e-6)


def test_mixed_form_caps_the_block_at_32():
    s = Solver((16, 16, 16), levels=3, precision="mixed")
    with pytest.raises(LobpcgError) as e:
        s.solve(33, tol=1e-8, maxit=10)
    assert e.value.code == capi.ERR_ARG
    s.close()
