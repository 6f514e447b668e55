"""Pins of the V-cycle preconditioner T (oracle side).

The dense operators below are built independently of ``oracle.multigrid``:
the 1-D prolongation from the coarse hat basis functions, 3-D transfer
operators by Kronecker products, and the V-cycle composed as a matrix
expression of smoother, restriction, coarse solve and prolongation.
"""
import numpy as np
import pytest

from oracle import laplace, multigrid


def hat_prolongation(nf):
    """Column I is the coarse hat function centred at fine node 2I (half-width 2)."""
    nc = nf // 2
    i = np.arange(1, nf + 1)[:, None]
    I = np.arange(1, nc + 1)[None, :]
    return np.maximum(0.0, 1.0 - np.abs(i - 2 * I) / 2.0)


def kron3(Px, Py, Pz):
    return np.kron(Pz, np.kron(Py, Px))


def dense_vcycle(dims, scale, levels, nu=2, omega=2.0 / 3.0):
    """The V-cycle as a dense matrix: V = M^nu G + B_nu, G = B_nu + P C R (I - A B_nu)."""
    n = laplace.npoints(dims)
    A = laplace.dense_matrix(dims, scale)
    if levels == 1:
        return np.linalg.inv(A)
    dc = tuple(d // 2 for d in dims)
    P = kron3(hat_prolongation(dims[0]), hat_prolongation(dims[1]), hat_prolongation(dims[2]))
    R = P.T / 8.0
    C = dense_vcycle(dc, scale / 4.0, levels - 1, nu, omega)
    Dinv = omega / (6.0 * scale)
    M = np.eye(n) - Dinv * A
    B = sum(np.linalg.matrix_power(M, t) for t in range(nu)) * Dinv
    G = B + P @ C @ R @ (np.eye(n) - A @ B)
    return np.linalg.matrix_power(M, nu) @ G + B


@pytest.mark.parametrize("nf", [1, 2, 5, 8, 9, 48])
def test_prolongation_1d_equals_hat_basis(nf):
    assert np.array_equal(multigrid.prolongation_1d(nf), hat_prolongation(nf))


def test_level_dims_match_workload_level_counts():
    assert multigrid.level_dims((48, 48, 48), 4)[-1] == (6, 6, 6)
    assert multigrid.level_dims((128,) * 3, 6)[-1] == (4, 4, 4)
    assert multigrid.level_dims((256,) * 3, 7)[-1] == (4, 4, 4)
    assert multigrid.level_dims((464,) * 3, 8)[-1] == (3, 3, 3)
    with pytest.raises(ValueError):
        multigrid.level_dims((4, 4, 4), 4)


def test_prolongation_exact_on_trilinear_functions():
    dims_f, dims_c = (9, 11, 7), (4, 5, 3)
    # a trilinear function sampled at coarse nodes (fine coordinates 2I, 2J, 2K)
    I, J, K = [np.arange(1, d + 1) for d in dims_c]
    f = lambda x, y, z: 0.3 + 0.7 * x - 0.2 * y + 0.45 * z + 0.05 * x * y * z
    fc = f(2 * I[None, None, :], 2 * J[None, :, None], 2 * K[:, None, None]).ravel()[:, None]
    ff = multigrid.prolong(fc, dims_c, dims_f)[:, 0].reshape(dims_f[2], dims_f[1], dims_f[0])
    i, j, k = [np.arange(1, d + 1) for d in dims_f]
    want = f(i[None, None, :], j[None, :, None], k[:, None, None])
    # exact wherever the fine node lies between two coarse nodes on every axis
    sl = (slice(1, 2 * dims_c[2]), slice(1, 2 * dims_c[1]), slice(1, 2 * dims_c[0]))
    assert np.max(np.abs(ff[sl] - want[sl])) < 1e-13


def test_restriction_is_full_weighting():
    dims_f, dims_c = (9, 9, 9), (4, 4, 4)
    ones = np.ones((laplace.npoints(dims_f), 1))
    rc = multigrid.restrict(ones, dims_f, dims_c)[:, 0]
    assert np.allclose(rc, 1.0, atol=1e-15, rtol=0)     # odd grid: every stencil is interior
    # weights of one coarse point: 1/8 centre, 1/16 faces, 1/32 edges, 1/64 corners
    e = np.zeros((laplace.npoints(dims_f), 1))
    e[3 + 9 * (3 + 9 * 3), 0] = 1.0                       # fine (4,4,4) 1-based = coarse (2,2,2)
    w = multigrid.restrict(e, dims_f, dims_c)[:, 0].reshape(4, 4, 4)
    assert w[1, 1, 1] == 1.0 / 8.0
    e[:] = 0.0
    e[2 + 9 * (3 + 9 * 3), 0] = 1.0                       # fine (3,4,4): face neighbour
    assert multigrid.restrict(e, dims_f, dims_c)[:, 0].reshape(4, 4, 4)[1, 1, 1] == 1.0 / 16.0


@pytest.mark.parametrize("dims,levels", [((7, 7, 7), 2), ((8, 6, 5), 2), ((8, 8, 8), 3), ((7, 9, 8), 3),
                                         ((16, 14, 12), 4)])
def test_vcycle_matches_dense_assembly(dims, levels):
    s = 2.0 + sum(dims)
    T = multigrid.VCycle(dims, s, levels)
    n = laplace.npoints(dims)
    got = T(np.eye(n))
    want = dense_vcycle(dims, s, levels)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("dims,levels", [((7, 7, 7), 3), ((8, 8, 8), 3), ((6, 9, 7), 2)])
def test_vcycle_symmetric_positive_definite(dims, levels):
    """Section 2.1.1 requires T linear, symmetric and positive definite."""
    T = multigrid.VCycle(dims, 1.0, levels)
    V = T(np.eye(laplace.npoints(dims)))
    assert np.max(np.abs(V - V.T)) <= 1e-14 * np.max(np.abs(V))
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0.0


def test_vcycle_contraction_on_nested_grid():
    """On 2^k - 1 grids the V(2,2) cycle contracts at about the Jacobi smoothing bound.

    omega = 2/3 Jacobi damps the 3-D high frequencies by at most 1 - omega/3 = 7/9
    per sweep, so four sweeps give about (7/9)^4 = 0.37.
    """
    dims = (15, 15, 15)
    s = laplace.default_scale(dims)
    T = multigrid.VCycle(dims, s, 3)
    n = laplace.npoints(dims)
    V = T(np.eye(n))
    E = np.eye(n) - V @ laplace.dense_matrix(dims, s)
    rho = np.max(np.abs(np.linalg.eigvals(E)))
    assert 0.2 < rho < (7.0 / 9.0) ** 4 + 0.02
