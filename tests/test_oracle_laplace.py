"""Pins of the 7-point operator and its closed-form spectrum (Section 4.1)."""
import numpy as np
import pytest

from oracle import laplace


def kron_sum_matrix(dims, scale):
    """Dense operator built independently as a Kronecker sum of 1-D second differences.

    Linear index p = i + nx*(j + ny*k) makes x the fastest axis, so the x term is
    I_z (x) I_y (x) T_x  (numpy's kron puts the second factor's index fastest).
    """
    nx, ny, nz = dims

    def T(n):
        return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)

    I = np.eye
    return scale * (np.kron(I(nz), np.kron(I(ny), T(nx)))
                    + np.kron(I(nz), np.kron(T(ny), I(nx)))
                    + np.kron(T(nz), np.kron(I(ny), I(nx))))


@pytest.mark.parametrize("dims", [(3, 4, 5), (5, 4, 3), (6, 6, 6), (1, 7, 2)])
def test_stencil_matches_kronecker_sum(dims):
    s = 3.7
    assert np.array_equal(laplace.dense_matrix(dims, s), kron_sum_matrix(dims, s))


@pytest.mark.parametrize("dims,scale", [((6, 6, 6), 1.0), ((4, 5, 7), 1.0), ((7, 7, 7), None)])
def test_closed_form_eigenvalues_match_dense_eigensolve(dims, scale):
    s = laplace.default_scale(dims) if scale is None else scale
    n = laplace.npoints(dims)
    want = np.linalg.eigvalsh(kron_sum_matrix(dims, s))
    got = laplace.exact_eigenvalues(dims, s, n)
    assert np.max(np.abs(got - want) / want) < 1e-13


def test_default_scale_is_h_minus_two_for_cube():
    assert laplace.default_scale((48, 48, 48)) == 49.0 ** 2
    assert laplace.default_scale((96, 80, 64)) == 1.0


def test_sine_products_are_eigenvectors():
    dims, s = (9, 8, 7), 2.5
    for lam, abc in laplace.exact_modes(dims, s, 12):
        v = laplace.exact_eigenvector(dims, abc)
        r = laplace.apply(v, dims, s) - lam * v
        assert np.linalg.norm(r) < 1e-12 * lam
        assert abs(np.linalg.norm(v) - 1.0) < 1e-14


def test_multiplicities_of_cube_spectrum():
    # Lowest cube modes: (1,1,1) simple, (1,1,2) 3-fold, (1,2,2) 3-fold, (1,1,3) 3-fold,
    # (2,2,2) simple, (1,2,3) 6-fold, ...  Cumulative counts 1,4,7,10,11,17,20,23,26,32:
    # m = 8 cuts the (1,1,3) cluster, m = 16 cuts the (1,2,3) cluster, m = 32 ends on a cluster.
    lam = laplace.exact_eigenvalues((48, 48, 48), 49.0 ** 2, 40)
    sizes = [len(c) for c in laplace.eigen_clusters(lam)]
    assert sizes[:10] == [1, 3, 3, 3, 1, 6, 3, 3, 3, 6]
