"""Property pins of the oracle's operators on random grid shapes (hypothesis; skipped where it is
not installed).  Each property fails for a plausible indexing mistake that fixed shapes can hide:

* A is symmetric, <A u, v> = <u, A v>, on boxes with distinct, odd and even axes (a swapped
  neighbour stride or a missing boundary term breaks it);
* restriction is the adjoint of prolongation over 8, <R f, c> = <f, P c> / 8 (a transposed
  operand, an off-by-one coarse index or a wrong weight breaks it);
* P reproduces a coarse field exactly at the fine points that sit on coarse points (fine index 2I
  for coarse I, 1-based);
* the V-cycle T is symmetric and positive definite (Section 2.1.1 asks it of T) for random shapes
  and depths.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import laplace, multigrid  # noqa: E402

dims3 = st.tuples(st.integers(1, 9), st.integers(1, 9), st.integers(1, 9))
coarsenable = st.tuples(st.integers(2, 11), st.integers(2, 11), st.integers(2, 11))


@settings(max_examples=40, deadline=None)
@given(dims=dims3, seed=st.integers(0, 2 ** 32 - 1), scale=st.floats(0.5, 100.0))
def test_stencil_is_symmetric(dims, seed, scale):
    g = np.random.default_rng(seed)
    n = laplace.npoints(dims)
    u, v = g.standard_normal((n, 1)), g.standard_normal((n, 1))
    lhs = float(laplace.apply(u, dims, scale)[:, 0] @ v[:, 0])
    rhs = float(u[:, 0] @ laplace.apply(v, dims, scale)[:, 0])
    assert abs(lhs - rhs) <= 1e-12 * scale * n


@settings(max_examples=40, deadline=None)
@given(dims=coarsenable, seed=st.integers(0, 2 ** 32 - 1))
def test_restriction_is_adjoint_of_prolongation(dims, seed):
    dc = tuple(d // 2 for d in dims)
    g = np.random.default_rng(seed)
    f = g.standard_normal((laplace.npoints(dims), 2))
    c = g.standard_normal((laplace.npoints(dc), 2))
    lhs = np.sum(multigrid.restrict(f, dims, dc) * c)
    rhs = np.sum(f * multigrid.prolong(c, dc, dims)) / 8.0
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(f).sum() + np.abs(c).sum())


@settings(max_examples=30, deadline=None)
@given(dims=coarsenable, seed=st.integers(0, 2 ** 32 - 1))
def test_prolongation_injects_on_coarse_points(dims, seed):
    dc = tuple(d // 2 for d in dims)
    c = np.random.default_rng(seed).standard_normal((laplace.npoints(dc), 1))
    F = multigrid.prolong(c, dc, dims)[:, 0].reshape(dims[2], dims[1], dims[0])
    C = c[:, 0].reshape(dc[2], dc[1], dc[0])
    # coarse I (1-based) sits on fine 2I (1-based), i.e. 0-based fine index 2I - 1
    assert np.array_equal(F[1::2, 1::2, 1::2][:dc[2], :dc[1], :dc[0]], C)


@settings(max_examples=15, deadline=None)
@given(dims=st.tuples(st.integers(4, 9), st.integers(4, 9), st.integers(4, 9)), levels=st.integers(1, 3),
       seed=st.integers(0, 2 ** 32 - 1))
def test_vcycle_symmetric_positive_definite(dims, levels, seed):
    if min(multigrid.level_dims(dims, 1)[0]) // 2 ** (levels - 1) < 1:
        levels = 1
    scale = laplace.default_scale(dims)
    T = multigrid.VCycle(dims, scale, levels)
    n = laplace.npoints(dims)
    g = np.random.default_rng(seed)
    U = g.standard_normal((n, 3))
    TU = T(U)
    G = U.T @ TU
    assert np.max(np.abs(G - G.T)) <= 1e-12 * np.max(np.abs(G))
    assert np.all(np.linalg.eigvalsh(0.5 * (G + G.T)) > 0)
