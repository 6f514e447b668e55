"""Failure detection without a GPU fault: the bounded stage waits of the TMA-staged float32
kernels (the SIMT Gram tiles and the streamed block products of the mixed form).

With the handle's wait limit at 0 polls every stage wait gives up at once: the kernel lets the
copies it still has in flight land (under its own, unchanged bound), records the failure in the
handle's status word and returns, and the call reports LOBPCG_ERR_TIMEOUT.  Nothing hangs and
nothing faults, so the context stays usable: the same handle with the default limit restored,
and a new handle, compute correct results afterwards.  The tensor-core engine is not selected
here (its bounds are fixed).
"""
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import laplace  # noqa: E402
from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import LobpcgError, Solver  # noqa: E402
from tests.gpu_util import ptr  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev32(X, ld):
    n, w = X.shape
    T = torch.full((w, ld), float("nan"), dtype=torch.float32)
    T[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T.astype(np.float32)))
    return T.cuda()


def _gram_f32(s, S, V, ld):
    w, b = S.shape[1], V.shape[1]
    Sd, Vd = _dev32(S, ld), _dev32(V, ld)
    C = torch.full((b, w), float("nan"), dtype=torch.float64, device="cuda")
    G = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    rc = capi.lobpcg_op_gram_f32(s.h, ptr(Sd), w, None, 0, ptr(Vd), b, ld, ptr(C), ptr(G))
    return rc, C.cpu().numpy().T, G.cpu().numpy().T


def test_gram_f32_wait_timeout_then_recovers():
    dims = (48, 48, 48)
    s = Solver(dims, precond="none", precision="mixed", gram_engine="simt")
    n, ld = s.n, s.n + 4
    g = np.random.default_rng(5)
    S = g.standard_normal((n, 8)).astype(np.float32).astype(np.float64)
    V = g.standard_normal((n, 8)).astype(np.float32).astype(np.float64)
    assert capi.lobpcg_set_wait_limit(s.h, 0) == capi.OK
    rc, _, _ = _gram_f32(s, S, V, ld)
    assert rc == capi.ERR_TIMEOUT, rc
    assert "bounded wait" in capi.lobpcg_last_error(s.h)
    nS, nV = np.linalg.norm(S, axis=0), np.linalg.norm(V, axis=0)
    # default limit restored on the same handle, then a new handle: correct products
    assert capi.lobpcg_set_wait_limit(s.h, -1) == capi.OK
    s2 = Solver(dims, precond="none", precision="mixed", gram_engine="simt")
    for h in (s, s2):
        rc, C, G = _gram_f32(h, S, V, ld)
        assert rc == capi.OK, capi.lobpcg_last_error(h.h)
        assert np.all(np.abs(C - S.T @ V) <= 1e-6 * np.outer(nS, nV))
        assert np.all(np.abs(G - V.T @ V) <= 1e-6 * np.outer(nV, nV))
    s.close()
    s2.close()


def test_mixed_solve_wait_timeout_then_recovers():
    """A whole mixed-form solve: its first pass runs the Gram tiles and the streamed products,
    every stage wait gives up, and the solve returns LOBPCG_ERR_TIMEOUT; with the default limit
    the same handle then converges to the closed-form eigenvalues."""
    dims, m = (24, 24, 24), 6
    s = Solver(dims, levels=3, precision="mixed", gram_engine="simt")
    assert capi.lobpcg_set_wait_limit(s.h, 0) == capi.OK
    with pytest.raises(LobpcgError) as e:
        s.solve(m, tol=1e-8, maxit=50, seed=2, with_vectors=False)
    assert e.value.code == capi.ERR_TIMEOUT
    assert capi.lobpcg_set_wait_limit(s.h, -1) == capi.OK
    out = s.solve(m, tol=1e-8, maxit=200, seed=2, with_vectors=False)
    assert out["status_name"] == "ok"
    exact = laplace.exact_eigenvalues(dims, laplace.default_scale(dims), m)
    assert np.max(np.abs(np.array(out["lam"]) - exact) / exact) < 1e-9
    s.close()
