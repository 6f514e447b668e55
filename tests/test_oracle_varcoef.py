"""Pins of the variable-coefficient oracle (oracle/varcoef.py) and of the kappa generator.

* kappa = const reduces the operator to the constant-coefficient Laplacian (scale = kappa) and the
  coarse faces to kappa / 4 (the constant operator's s / 4 rule);
* the operator is symmetric and its diagonal is the sum of the six face coefficients;
* the eigenvalue gradient (first-order perturbation of a simple eigenvalue) against per-face
  central finite differences of a dense eigensolver on a small box;
* harmonic averaging along the face normal on a field that varies only along that axis;
* the variable-coefficient V-cycle is a symmetric positive definite matrix;
* the oracle LOBPCG with that V-cycle against a dense eigensolver.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import laplace, lobpcg as olob, multigrid, rng, varcoef  # noqa: E402
from paper_0705_2626_gb300 import fields  # noqa: E402


def const_kappa(dims, c):
    return np.full(fields.num_faces(dims), float(c))


@pytest.mark.parametrize("dims", [(3, 4, 5), (6, 5, 4), (7, 7, 7)])
def test_constant_kappa_is_the_laplacian(dims):
    U = np.random.default_rng(0).standard_normal((int(np.prod(dims)), 3))
    assert np.allclose(varcoef.apply(U, dims, const_kappa(dims, 2.5)), laplace.apply(U, dims, 2.5),
                       rtol=0, atol=1e-13)


def test_symmetric_and_diagonal():
    dims = (4, 3, 5)
    kappa = fields.random_kappa(dims, seed=1, length=2.0)
    A = varcoef.dense_matrix(dims, kappa)
    assert np.array_equal(A, A.T)
    assert np.allclose(np.diag(A), varcoef.diagonal(dims, kappa), rtol=1e-15)
    assert np.all(np.linalg.eigvalsh(A) > 0)


def test_gradient_matches_finite_differences():
    dims = (3, 4, 5)
    kappa = fields.random_kappa(dims, seed=3, length=2.0)
    lam, V = np.linalg.eigh(varcoef.dense_matrix(dims, kappa))
    assert lam[1] - lam[0] > 1e-3 * lam[0]          # simple smallest eigenvalue
    g = varcoef.grad(V[:, :1], dims, [1.0])
    eps = 1e-6
    fd = np.empty_like(kappa)
    for f in range(kappa.size):
        kp, km = kappa.copy(), kappa.copy()
        kp[f] += eps
        km[f] -= eps
        fd[f] = (np.linalg.eigvalsh(varcoef.dense_matrix(dims, kp))[0]
                 - np.linalg.eigvalsh(varcoef.dense_matrix(dims, km))[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-7 * np.max(np.abs(g))
    # the cluster-trace weights: w = (1, 1) on two eigenvectors equals the sum of their gradients
    g2 = varcoef.grad(V[:, :2], dims, [1.0, 1.0])
    assert np.allclose(g2, g + varcoef.grad(V[:, 1:2], dims, [1.0]), rtol=1e-14, atol=0)


def test_coarse_faces_constant_and_harmonic():
    dims_f, dims_c = (8, 6, 7), (4, 3, 3)
    kc = varcoef.coarse_kappa(dims_f, const_kappa(dims_f, 3.0), dims_c)
    assert kc.size == fields.num_faces(dims_c)
    assert np.allclose(kc, 0.75, rtol=1e-15)
    # kappa varying only along x on the x-faces: coarse x-face F = harmonic mean of fine 2F, 2F+1
    nx, ny, nz = dims_f
    kx = np.tile(1.0 + np.arange(nx + 1, dtype=float), (nz, ny, 1))
    kappa = np.concatenate([kx.ravel(), np.ones(nx * (ny + 1) * nz), np.ones(nx * ny * (nz + 1))])
    Kx, Ky, Kz = varcoef.split(varcoef.coarse_kappa(dims_f, kappa, dims_c), dims_c)
    for F in range(dims_c[0] + 1):
        a, b = 1.0 + 2 * F, 1.0 + (2 * F + 1 if 2 * F + 1 <= nx else 2 * F)
        want = (2.0 / (1.0 / a + 1.0 / b)) if 2 * F + 1 <= nx else a
        assert np.allclose(Kx[:, :, F], want / 4.0, rtol=1e-15)
    assert np.allclose(Ky, 0.25) and np.allclose(Kz, 0.25)


def test_vcycle_is_spd():
    dims = (8, 7, 6)
    kappa = fields.random_kappa(dims, seed=5, length=3.0)
    T = varcoef.VCycleVar(dims, kappa, levels=3)
    n = int(np.prod(dims))
    M = T(np.eye(n))
    assert np.max(np.abs(M - M.T)) <= 1e-13 * np.max(np.abs(M))
    assert np.min(np.linalg.eigvalsh(0.5 * (M + M.T))) > 0


def test_lobpcg_with_vcycle_matches_dense():
    dims, m = (8, 7, 6), 4
    kappa = fields.random_kappa(dims, seed=7, length=3.0)
    A = varcoef.VarCoef7(dims, kappa)
    T = varcoef.VCycleVar(dims, kappa, levels=2)
    res = olob.lobpcg(A, rng.uniform_block(2, A.n, m), 1e-10, 300, T=T)
    want = np.linalg.eigvalsh(varcoef.dense_matrix(dims, kappa))[:m]
    assert res.status == "converged"
    assert np.max(np.abs(res.lam - want) / want) < 1e-12


def test_random_kappa_field_statistics():
    dims = (20, 18, 16)
    logk = fields.gaussian_log_field(dims, seed=11, length=4.0)
    assert logk.shape == (dims[2] + 2, dims[1] + 2, dims[0] + 2)
    assert abs(logk.mean()) < 1e-12 and abs(logk.std() - 1.0) < 1e-12
    kappa = fields.random_kappa(dims, seed=11, length=4.0)
    assert kappa.size == fields.num_faces(dims) and np.all(kappa > 0)
    # deterministic in the seed
    assert np.array_equal(kappa, fields.random_kappa(dims, seed=11, length=4.0))
