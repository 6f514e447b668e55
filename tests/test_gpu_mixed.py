"""End-to-end parity of the mixed-precision form with the float64 CPU oracle.

Mixed form: X, AX and the small matrices in float64; W, AW, P, AP and the finest V-cycle level
in float32, coarser V-cycle levels stored in bfloat16; Gram products in float32 with compensated
sums; a float64 correction sweep confirms convergence.  Bars: eigenvalues within 1e-9 relative of
the oracle, subspace angles below 1e-6 over complete eigenvalue clusters, and -- because the
float64 sweep re-tests every column at the end -- every final residual within the tolerance.
The mixed form is meant for large grids, where the float32 roundings average out over many
unknowns; on grids of a few thousand points its attainable residual can stay above 1e-8.
"""
import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import laplace, lobpcg as olob, multigrid, rng  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402


def angle(U, V):
    return float(np.max(scipy.linalg.subspace_angles(U, V)))


def oracle_run(dims, scale, m, tol, maxit, levels, seed=2):
    A = olob.Laplace7(dims, scale)
    T = multigrid.VCycle(dims, A.scale, levels)
    return olob.lobpcg(A, rng.uniform_block(seed, A.n, m), tol, maxit, T=T)


def complete_clusters(dims, scale, exact, m):
    out = []
    for c in laplace.eigen_clusters(exact):
        full = laplace.exact_eigenspace(dims, scale, exact[c[0]], max_index=8).shape[1]
        if full == len(c):
            out.append(c)
    return out


# nx = 42 is not a multiple of 4: the per-point residual and stencil kernels instead of the
# float4 ones
@pytest.mark.parametrize("dims,scale,m,levels", [((40, 36, 34), None, 6, 3), ((42, 36, 34), None, 6, 3), ((48, 48, 48), None, 8, 4)])
@pytest.mark.parametrize("engine", ["tensor", "simt"])
def test_mixed_matches_fp64_oracle(dims, scale, m, levels, engine):
    tol = 1e-8
    s = Solver(dims, scale=scale, levels=levels, precision="mixed", gram_engine=engine)
    out = s.solve(m, tol=tol, maxit=200, seed=2)
    ref = oracle_run(dims, s.scale, m, tol, 200, levels)
    assert out["status_name"] == "ok", out
    assert out["fp64_sweeps"] >= 1
    lam = np.array(out["lam"])
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-9
    exact = laplace.exact_eigenvalues(dims, s.scale, m)
    assert np.max(np.abs(lam - exact) / exact) < 1e-9
    assert out["max_rel_resid"] <= tol * (1 + 1e-6)
    X = out["X"].cpu().numpy().T
    assert np.max(np.abs(X.T @ X - np.eye(m))) < 1e-12
    for c in complete_clusters(dims, s.scale, exact, m):
        assert angle(X[:, c], ref.X[:, c]) < 1e-6
    s.close()


@pytest.mark.parametrize("engine", ["auto", "tensor", "simt"])
def test_mixed_c2_full_size(engine):
    """128^3 (2,097,152 unknowns), m = 16, 6-level V-cycle: the bench workload in mixed form."""
    dims, m = (128, 128, 128), 16
    s = Solver(dims, levels=6, precision="mixed", gram_engine=engine)
    out = s.solve(m, tol=1e-8, maxit=200, seed=2)
    scale = laplace.default_scale(dims)
    exact = laplace.exact_eigenvalues(dims, scale, m)
    lam = np.array(out["lam"])
    assert out["status_name"] == "ok"
    assert np.max(np.abs(lam - exact) / exact) < 1e-9
    assert out["max_rel_resid"] <= 1e-8 * (1 + 1e-6)
    X = out["X"].cpu().numpy().T
    for c in laplace.eigen_clusters(exact)[:5]:       # complete clusters 1, 3, 3, 3, 1
        E = laplace.exact_eigenspace(dims, scale, exact[c[0]], max_index=4)
        assert angle(X[:, c], E) < 1e-6
    s.close()


def test_mixed_is_deterministic():
    s = Solver((24, 24, 24), levels=3, precision="mixed")
    a = s.solve(6, tol=1e-8, maxit=100, seed=4)
    b = s.solve(6, tol=1e-8, maxit=100, seed=4)
    assert a["lam"] == b["lam"] and a["iters"] == b["iters"]
    assert torch.equal(a["X"], b["X"])
    s.close()
