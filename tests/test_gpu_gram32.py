"""Float32 Gram kernels of the mixed form through the C ABI, both engines: the SIMT tiles
(k_gram32.cu) and the tcgen05 tensor-core form (k_gram_tc.cu).

Inputs are float32 blocks; the expected values are float64 products of the same float32 values
(the plain definitions S^T V, V^T V) and, for the residual form, the oracle's Gram matrices of
the Gram matrices of the Rayleigh-Ritz basis (upper block triangle, symmetrised diagonal blocks) of the basis [X W P] with
X = Xh + Xl.  The residual form equals them in exact arithmetic; the bounds allow the float32
rounding of the inputs R, AW, AP and the arithmetic of the engine, relative to |s_i| |t_j|:
  SIMT: float32 products, compensated sums: 1e-6;
  tensor cores: 3 x TF32 products (2^-20) and float32 accumulation in tensor memory that rounds
  toward zero at each of the at most 96 MMA steps of a 256-point chunk (96 * 2^-23 of the
  chunk's sum of |s_k t_k|): 1.3e-5;
and 1e-12 for the double-float X^T X block (same kernel under both engines).
"""
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import laplace, lobpcg as olob  # noqa: E402
from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import ptr  # noqa: E402

pytestmark = pytest.mark.gpu

ENGINE_TOL = {"simt": 1e-6, "tensor": 1.3e-5}


def dev32(X, ld):
    """numpy (n, w) -> float32 cuda tensor (w, ld), row j = column j (padding NaN)."""
    n, w = X.shape
    T = torch.full((max(w, 1), ld), float("nan"), dtype=torch.float32)
    T[:w, :n] = torch.from_numpy(np.ascontiguousarray(X.T.astype(np.float32)))
    return T.cuda()


def f32(X):
    return X.astype(np.float32).astype(np.float64)


def ld_for(n):
    return ((n + 3) // 4) * 4 + 4


@pytest.mark.parametrize("dims,w0,w1,b", [((12, 11, 10), 6, 0, 5), ((12, 11, 10), 6, 5, 5), ((48, 48, 48), 8, 8, 8),
                                          ((40, 36, 34), 16, 16, 16), ((128, 128, 128), 16, 16, 16),
                                          ((20, 20, 20), 32, 32, 32), ((7, 7, 7), 1, 0, 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
@pytest.mark.parametrize("engine", ["tensor", "simt"])
def test_gram_f32_cross_and_vtv(dims, w0, w1, b, engine):
    tol = ENGINE_TOL[engine]
    s = Solver(dims, precond="none", gram_engine=engine)
    n, ld = s.n, ld_for(s.n)
    g = np.random.default_rng(11)
    S = f32(g.standard_normal((n, w0 + w1)) * g.uniform(0.1, 10, w0 + w1)[None, :])
    V = f32(g.standard_normal((n, b)))
    S0, S1, Vd = dev32(S[:, :w0], ld), dev32(S[:, w0:], ld) if w1 else None, dev32(V, ld)
    C = torch.full((b, w0 + w1), float("nan"), dtype=torch.float64, device="cuda")   # column-major (w0+w1) x b
    G = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    rc = capi.lobpcg_op_gram_f32(s.h, ptr(S0), w0, ptr(S1), w1, ptr(Vd), b, ld, ptr(C), ptr(G))
    assert rc == capi.OK, capi.lobpcg_last_error(s.h)
    Cg, Gg = C.cpu().numpy().T, G.cpu().numpy().T
    nS, nV = np.linalg.norm(S, axis=0), np.linalg.norm(V, axis=0)
    assert np.all(np.abs(Cg - S.T @ V) <= tol * np.outer(nS, nV))
    assert np.all(np.abs(Gg - V.T @ V) <= tol * np.outer(nV, nV))
    assert np.array_equal(Gg, Gg.T)
    s.close()


def residual_form_inputs(dims, m, b, bp, seed, near=False):
    """X (float64, as hi / lo planes), W, P float32, T = [R AW AP] float32, Lambda."""
    g = np.random.default_rng(seed)
    scale = laplace.default_scale(dims)
    n = int(np.prod(dims))
    if near:   # X close to eigenvectors: R small, as near convergence
        modes = laplace.exact_modes(dims, scale, m)
        lam = np.array([lm for lm, _ in modes])
        X = np.stack([laplace.exact_eigenvector(dims, abc) for _, abc in modes], axis=1)
        X = X + 1e-6 * g.standard_normal((n, m))
    else:
        X = g.standard_normal((n, m))
        lam = np.sort(g.uniform(1, 100, m))
    Xh = X.astype(np.float32)
    Xl = (X - Xh.astype(np.float64)).astype(np.float32)
    X = Xh.astype(np.float64) + Xl.astype(np.float64)
    W = f32(g.standard_normal((n, b)))
    P = f32(g.standard_normal((n, bp)))
    A = olob.Laplace7(dims, scale)
    AX, AW, AP = A(X), A(W), A(P)
    R = AX - X * lam[None, :]
    return dict(X=X, Xh=Xh, Xl=Xl, W=W, P=P, AX=AX, AW=AW, AP=AP, R=R, lam=lam, n=n)


@pytest.mark.parametrize("dims,m,b,bp,near", [((12, 11, 10), 6, 5, 5, False), ((12, 11, 10), 4, 4, 0, False),
                                              ((40, 36, 34), 8, 8, 8, True), ((48, 48, 48), 16, 16, 16, False),
                                              ((128, 128, 128), 16, 16, 16, True), ((40, 40, 40), 32, 32, 32, False),
                                              ((9, 9, 9), 1, 1, 1, False)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
@pytest.mark.parametrize("engine", ["tensor", "simt"])
def test_gram_residual_form_matches_oracle_gram(dims, m, b, bp, near, engine):
    tol = ENGINE_TOL[engine]
    s = Solver(dims, precond="none", gram_engine=engine)
    d = residual_form_inputs(dims, m, b, bp, seed=3, near=near)
    n, ld, q = d["n"], ld_for(d["n"]), m + b + bp
    blk = {k: dev32(d[k], ld) for k in ("Xh", "Xl", "W", "R", "AW")}
    blk["P"] = dev32(d["P"], ld) if bp else None
    blk["AP"] = dev32(d["AP"], ld) if bp else None
    lam = torch.tensor(d["lam"], dtype=torch.float64, device="cuda")
    gA = torch.full((q, q), float("nan"), dtype=torch.float64, device="cuda")
    gB = torch.full((q, q), float("nan"), dtype=torch.float64, device="cuda")
    rc = capi.lobpcg_op_gram_residual(s.h, *[ptr(blk[k]) for k in ("Xh", "Xl", "W", "P", "R", "AW", "AP")], ld,
                                      m, b, bp, ptr(lam), ptr(gA), ptr(gB))
    assert rc == capi.OK, capi.lobpcg_last_error(s.h)
    GA, GB = gA.cpu().numpy().T, gB.cpu().numpy().T
    Sb = [d["X"], d["W"]] + ([d["P"]] if bp else [])
    ASb = [d["AX"], d["AW"]] + ([d["AP"]] if bp else [])
    wantA = olob.upper_block_gram(Sb, ASb)
    S = np.concatenate(Sb, axis=1)
    T = np.concatenate([d["R"], d["AW"]] + ([d["AP"]] if bp else []), axis=1)
    wantB = S.T @ S
    nS, nT = np.linalg.norm(S, axis=0), np.linalg.norm(T, axis=0)
    lamq = np.concatenate([d["lam"], np.zeros(q - m)])
    # gramB: double-float X^T X, float32 elsewhere
    bound_b = tol * np.outer(nS, nS)
    bound_b[:m, :m] = 1e-12 * np.outer(nS[:m], nS[:m])
    assert np.all(np.abs(GB - wantB) <= bound_b)
    # gramA: the float32 part scales with |s_i| |t_j|; the Lambda X^T S part with the gramB error
    bound_a = tol * (np.outer(nS, nT) + np.outer(nT, nS)) + np.abs(lamq)[:, None] * bound_b + \
        np.abs(lamq)[None, :] * bound_b
    assert np.all(np.abs(GA - wantA) <= bound_a)
    assert np.array_equal(GA, GA.T) and np.array_equal(GB, GB.T)
    # deterministic: a second call gives the same bits
    gA2, gB2 = torch.empty_like(gA), torch.empty_like(gB)
    rc = capi.lobpcg_op_gram_residual(s.h, *[ptr(blk[k]) for k in ("Xh", "Xl", "W", "P", "R", "AW", "AP")], ld,
                                      m, b, bp, ptr(lam), ptr(gA2), ptr(gB2))
    assert rc == capi.OK
    assert torch.equal(gA, gA2) and torch.equal(gB, gB2)
    s.close()


def test_gram_f32_rejects_bad_arguments():
    s = Solver((8, 8, 8), precond="none")
    ld = ld_for(s.n)
    V = dev32(np.ones((s.n, 2)), ld)
    G = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    assert capi.lobpcg_op_gram_f32(s.h, None, 0, None, 0, ptr(V), 0, ld, None, ptr(G)) == capi.ERR_ARG
    assert capi.lobpcg_op_gram_f32(s.h, None, 0, None, 0, ptr(V), 2, s.n - 1, None, ptr(G)) == capi.ERR_ARG
    assert capi.lobpcg_op_gram_f32(s.h, None, 2, None, 0, ptr(V), 2, ld, None, ptr(G)) == capi.ERR_ARG
    s.close()
