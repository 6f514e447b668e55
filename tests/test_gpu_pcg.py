"""Inner-PCG preconditioning (Section 4.2) on the GPU against the oracle (oracle/pcg.py).

The preconditioner itself: T_k(R) through lobpcg_op_precond against the oracle's k PCG iterations
preconditioned by the oracle's V-cycle (the two V-cycles agree to rounding, and k CG steps
amplify rounding only mildly at these k): 1e-11 relative.  The solver: eigenvalues 1e-10 relative
and iteration counts within 10 % of the oracle with the same inner iteration count, fewer outer
iterations than the direct V-cycle, and argument errors.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import laplace, lobpcg as olob, multigrid, pcg, rng  # noqa: E402
from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import dev, empty, host, ptr  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [0, 1, 3, 8])
def test_inner_pcg_operator_matches_oracle(k):
    dims, levels, m = (20, 18, 16), 3, 3
    s = Solver(dims, levels=levels)
    s.set_inner_pcg(k)
    n = s.n
    R = np.random.default_rng(5).standard_normal((n, m))
    E = empty(m, n)
    assert capi.lobpcg_op_precond(s.h, m, ptr(dev(R)), n, ptr(E), n) == capi.OK
    A = olob.Laplace7(dims, s.scale)
    want = pcg.pcg_columns(A, multigrid.VCycle(dims, s.scale, levels), R, k)
    got = host(E, n)
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want)), k
    s.close()


@pytest.mark.parametrize("k", [2, 6])
def test_solve_with_inner_pcg_matches_oracle(k):
    dims, levels, m, tol = (24, 24, 24), 3, 6, 1e-10
    s = Solver(dims, levels=levels)
    s.set_inner_pcg(k)
    out = s.solve(m, tol=tol, maxit=300, seed=2)
    A = olob.Laplace7(dims, s.scale)
    M = multigrid.VCycle(dims, s.scale, levels)
    ref = olob.lobpcg(A, rng.uniform_block(2, A.n, m), tol, 300, T=pcg.InnerPCG(A, M, k))
    assert out["status_name"] == "ok" and ref.status == "converged"
    lam = np.array(out["lam"])
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10
    exact = laplace.exact_eigenvalues(dims, s.scale, m)
    assert np.max(np.abs(lam - exact) / exact) < 1e-10
    assert abs(out["iters"] - ref.iters) <= max(1, round(0.1 * ref.iters))
    # and fewer outer iterations than the direct V-cycle
    s.set_inner_pcg(0)
    direct = s.solve(m, tol=tol, maxit=300, seed=2, with_vectors=False)
    assert out["iters"] < direct["iters"]
    s.close()


def test_inner_pcg_argument_errors():
    s = Solver((8, 8, 8), levels=2)
    assert capi.lobpcg_set_inner_pcg(s.h, -1) == capi.ERR_ARG
    assert capi.lobpcg_set_inner_pcg(s.h, 10001) == capi.ERR_ARG
    s.close()
    mx = Solver((16, 16, 16), levels=2, precision="mixed")
    assert capi.lobpcg_set_inner_pcg(mx.h, 3) == capi.ERR_ARG
    assert capi.lobpcg_set_inner_pcg(mx.h, 0) == capi.OK
    mx.close()
