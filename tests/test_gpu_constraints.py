"""Constraints / hard locking (Section 2.2 the constraint projections, Section 2.3) on the GPU.

Parity with the oracle (oracle/lobpcg.py with Y) on the same seeded start: eigenvalues 1e-10
relative, iteration counts within 10 %, eigenvectors within the residual / gap bound, and X
orthogonal to the constraints.  Y is a block of closed-form eigenvectors (sine products of
Section 4.1) of a box with distinct sides, so the constrained spectrum is known exactly: the
eigenvalues after the l smallest.  Also: a badly scaled basis of the same span gives the same
result, repeated calls continue the spectrum, the mixed form, and argument / breakdown errors.
"""
import os
import sys

import numpy as np
import pytest
import scipy.linalg
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import laplace, lobpcg as olob, multigrid, rng  # noqa: E402
from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402

pytestmark = pytest.mark.gpu


def exact_block(dims, scale, count):
    modes = laplace.exact_modes(dims, scale, count)
    lam = np.array([lm for lm, _ in modes])
    V = np.stack([laplace.exact_eigenvector(dims, abc) for _, abc in modes], axis=1)
    return lam, V


@pytest.mark.parametrize("dims,l,m,levels", [((16, 17, 18), 4, 6, 2), ((24, 22, 20), 7, 5, 3)],
                         ids=["16x17x18-l4", "24x22x20-l7"])
def test_constrained_solve_matches_oracle(dims, l, m, levels):
    tol = 1e-10
    s = Solver(dims, levels=levels)
    lam_all, V = exact_block(dims, s.scale, l + m + 1)
    assert np.all(np.diff(lam_all) / lam_all[1:] > 1e-4)        # simple eigenvalues on this machine
    Y = V[:, :l]
    s.set_constraints(Y.T)
    out = s.solve(m, tol=tol, maxit=300, seed=2)
    A = olob.Laplace7(dims, s.scale)
    ref = olob.lobpcg(A, rng.uniform_block(2, A.n, m), tol, 300, T=multigrid.VCycle(dims, s.scale, levels), Y=Y)
    assert out["status_name"] == "ok" and ref.status == "converged"
    lam = np.array(out["lam"])
    want = lam_all[l:l + m]
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10
    assert np.max(np.abs(lam - want) / want) < 1e-10
    assert abs(out["iters"] - ref.iters) <= max(1, round(0.1 * ref.iters))
    X = out["X"].cpu().numpy().T
    assert np.max(np.abs(Y.T @ X)) < 1e-12
    gaps = np.minimum(np.diff(lam_all)[l:l + m], np.diff(lam_all)[l - 1:l + m - 1])
    for j in range(m):
        a = float(np.max(scipy.linalg.subspace_angles(X[:, j:j + 1], V[:, l + j:l + j + 1])))
        assert a <= 2.0 * out["resid"][j] / gaps[j] + 1e-12, (j, a)
    s.close()


def test_constraints_depend_only_on_their_span():
    dims, l, m = (16, 17, 18), 4, 6
    s = Solver(dims, levels=2)
    lam_all, V = exact_block(dims, s.scale, l + m)
    Y = V[:, :l]
    M = np.random.default_rng(7).standard_normal((l, l)) @ np.diag([1e3, 1.0, 1e-3, 10.0])
    s.set_constraints(Y.T)
    a = s.solve(m, tol=1e-10, maxit=300, seed=2)
    s.set_constraints(torch.tensor((Y @ M).T))
    b = s.solve(m, tol=1e-10, maxit=300, seed=2)
    assert np.max(np.abs(np.array(a["lam"]) - np.array(b["lam"])) / np.array(a["lam"])) < 1e-11
    assert abs(a["iters"] - b["iters"]) <= 1
    assert np.max(np.abs(Y.T @ b["X"].cpu().numpy().T)) < 1e-12
    # removing the constraints brings back the smallest eigenpairs
    s.set_constraints(None)
    c = s.solve(m, tol=1e-10, maxit=300, seed=2)
    assert np.max(np.abs(np.array(c["lam"]) - lam_all[:m]) / lam_all[:m]) < 1e-10
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_repeated_calls_continue_the_spectrum(precision):
    """The paper's recipe for many eigenpairs: each call's eigenvectors constrain the next."""
    dims, m, calls = (40, 36, 34), 6, 3
    tol = 1e-10 if precision == "fp64" else 1e-8
    s = Solver(dims, levels=3, precision=precision)
    lam_all = laplace.exact_eigenvalues(dims, s.scale, m * calls + 1)
    assert np.all(np.diff(lam_all) / lam_all[1:] > 1e-4)
    Ys = np.zeros((s.n, 0))
    found = []
    for call in range(calls):
        s.set_constraints(Ys.T if Ys.shape[1] else None)
        out = s.solve(m, tol=tol, maxit=300, seed=2 + call)
        assert out["status_name"] == "ok", (call, out["status_name"])
        X = out["X"].cpu().numpy().T
        if Ys.shape[1]:
            assert np.max(np.abs(Ys.T @ X)) < 1e-12
        found.extend(out["lam"])
        Ys = np.hstack([Ys, X])
    found = np.array(found)
    # eigenvalue errors of the locked vectors are second order in their residuals
    assert np.max(np.abs(found - lam_all[:m * calls]) / lam_all[:m * calls]) < 1e-12
    s.close()


def test_constraint_argument_errors():
    dims = (10, 9, 8)
    s = Solver(dims, levels=2)
    n = s.n
    assert capi.lobpcg_set_constraints(s.h, None, 2, n, 1) == capi.ERR_ARG          # NULL with l > 0
    Y = torch.zeros((n // 2, n), dtype=torch.float64)
    import ctypes
    assert capi.lobpcg_set_constraints(s.h, ctypes.c_void_p(Y.data_ptr()), n // 2, n, 1) == capi.ERR_ARG
    assert capi.lobpcg_set_constraints(s.h, ctypes.c_void_p(Y.data_ptr()), 2, n - 1, 1) == capi.ERR_ARG
    # m + l too large for the grid
    big = torch.randn((n // 2 - 3, n), dtype=torch.float64)
    s.set_constraints(big)
    assert capi.lobpcg_solve(s.h, 6, 1e-8, 50, 2, None) == capi.ERR_ARG
    # linearly dependent constraints: breakdown at the solve
    v = torch.randn((1, n), dtype=torch.float64)
    s.set_constraints(torch.cat([v, 2.0 * v, torch.randn((1, n), dtype=torch.float64)]))
    assert capi.lobpcg_solve(s.h, 4, 1e-8, 50, 2, None) == capi.ERR_BREAKDOWN
    s.set_constraints(None)
    assert capi.lobpcg_solve(s.h, 4, 1e-8, 200, 2, None) in (capi.OK, capi.NOT_CONVERGED)
    s.close()
