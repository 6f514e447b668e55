"""Pins of the variable-coefficient oracle (oracle/varcoef.py) and of the kappa generator.

* kappa = const reduces the operator to the constant-coefficient Laplacian (scale = kappa) and the
  coarse faces to kappa / 4 (the constant operator's s / 4 rule);
* the operator is symmetric and its diagonal is the sum of the six face coefficients;
* the eigenvalue gradient (first-order perturbation of a simple eigenvalue) against per-face
  central finite differences of a dense eigensolver on a small box;
* harmonic averaging along the face normal on a field that varies only along that axis;
* the operator assembled entry by entry from the face list (A[p,q] = -kappa_f for the face f
  between p and q, kappa_f added to both diagonals, boundary faces to one);
* coarse face values computed by hand on a 2 x 3 x 2 box whose kappa varies across the face
  normals (the 1/4, 1/2, 1/4 weights and their renormalisation where a line leaves the box);
* the V-cycle against a dense matrix built from the face-list operators, for two and three levels;
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


def face_list_matrix(dims, kappa):
    """A assembled from the face list: the face f between cells p and q adds kappa_f to A[p,p] and
    A[q,q] and -kappa_f to A[p,q] and A[q,p]; a face on the boundary adds kappa_f to A[p,p] only.
    Face layout: x-faces (f, j, k) between cells (f-1, j, k) and (f, j, k), then y-faces, then
    z-faces, x fastest in each part."""
    nx, ny, nz = dims
    n = nx * ny * nz
    A = np.zeros((n, n))
    cell = lambda i, j, k: i + nx * (j + ny * k)
    faces = []
    for k in range(nz):
        for j in range(ny):
            for f in range(nx + 1):
                faces.append((cell(f - 1, j, k) if f > 0 else None, cell(f, j, k) if f < nx else None))
    for k in range(nz):
        for f in range(ny + 1):
            for i in range(nx):
                faces.append((cell(i, f - 1, k) if f > 0 else None, cell(i, f, k) if f < ny else None))
    for f in range(nz + 1):
        for j in range(ny):
            for i in range(nx):
                faces.append((cell(i, j, f - 1) if f > 0 else None, cell(i, j, f) if f < nz else None))
    assert len(faces) == kappa.size
    for (p, q), kf in zip(faces, kappa):
        for a in (p, q):
            if a is not None:
                A[a, a] += kf
        if p is not None and q is not None:
            A[p, q] -= kf
            A[q, p] -= kf
    return A


@pytest.mark.parametrize("dims", [(3, 4, 5), (5, 2, 3), (1, 4, 2)])
def test_operator_matches_face_list_assembly(dims):
    kappa = fields.random_kappa(dims, seed=4, length=2.0)
    A = face_list_matrix(dims, kappa)
    B = varcoef.dense_matrix(dims, kappa)
    assert np.max(np.abs(A - B)) <= 1e-14 * np.max(np.abs(A))
    # every off-diagonal entry is minus one face coefficient (or zero)
    off = B[~np.eye(B.shape[0], dtype=bool)]
    assert np.all(np.isin(-off[off != 0], kappa))


def test_coarse_faces_by_hand_with_kappa_varying_across():
    """Fine box 2 x 3 x 2 -> coarse 1 x 1 x 1 (two coarse faces per direction).  Coarse lines sit on
    fine line 1 of each across-axis; the offsets -1, 0, +1 weigh 1/4, 1/2, 1/4, and a fine line
    outside the box (index 2 of a 2-point axis) is dropped with the weights renormalised (3/4).

    x-faces: kappa_x(f, y, z) = c(y, z), c(., 0) = 1, 2, 3 and c(., 1) = 4, 8, 12 (constant along
      x, so the harmonic mean along x is c itself).  y-weights 1/4, 1/2, 1/4 give 2 (z = 0) and
      8 (z = 1); z-weights 1/4, 1/2 over 3/4: (2/4 + 8/2) / (3/4) = 6; / 4 -> 1.5 for both faces.
    y-faces: kappa_y(x, f, z) = d(x, z), d(0, 0) = 1, d(1, 0) = 3, d(0, 1) = 5, d(1, 1) = 7.  x- and
      z-weights both 1/4, 1/2 over 3/4: (1/4 (1/4 + 3/2) + 1/2 (5/4 + 7/2)) / (9/16) = 5; / 4 ->
      1.25 for both faces.
    z-faces: kappa_z(x, y, f) = g(x, y) h(f), g(0, .) = 2, 4, 6, g(1, .) = 1, h = 1, 3, 2.  Coarse
      face 0 spans fine faces 0 and 1: harmonic mean 2 / (1/g + 1/(3g)) = 1.5 g; coarse face 1 has
      fine face 2 only: 2 g.  y-weights give g -> 4 (x = 0), 1 (x = 1); x-weights 1/4, 1/2 over
      3/4: (4/4 + 1/2) / (3/4) = 2.  So 1.5 * 2 / 4 = 0.75 and 2 * 2 / 4 = 1.0.
    Equal weights of 1/3 instead would give 1.25, 1.0 and 0.9375 / 1.25; no renormalisation would
    give 1.125, 0.703 and 0.5625 / 0.75."""
    dims_f, dims_c = (2, 3, 2), (1, 1, 1)
    kx = np.empty((2, 3, 3))
    c = {0: [1.0, 2.0, 3.0], 1: [4.0, 8.0, 12.0]}
    for z in range(2):
        for y in range(3):
            kx[z, y, :] = c[z][y]
    ky = np.empty((2, 4, 2))
    d = {(0, 0): 1.0, (1, 0): 3.0, (0, 1): 5.0, (1, 1): 7.0}
    for z in range(2):
        for x in range(2):
            ky[z, :, x] = d[(x, z)]
    kz = np.empty((3, 3, 2))
    g = {0: [2.0, 4.0, 6.0], 1: [1.0, 1.0, 1.0]}
    h = [1.0, 3.0, 2.0]
    for f in range(3):
        for y in range(3):
            for x in range(2):
                kz[f, y, x] = g[x][y] * h[f]
    kappa = np.concatenate([kx.ravel(), ky.ravel(), kz.ravel()])
    Kx, Ky, Kz = varcoef.split(varcoef.coarse_kappa(dims_f, kappa, dims_c), dims_c)
    assert np.allclose(Kx.ravel(), [1.5, 1.5], rtol=1e-15, atol=0)
    assert np.allclose(Ky.ravel(), [1.25, 1.25], rtol=1e-15, atol=0)
    assert np.allclose(Kz.ravel(), [0.75, 1.0], rtol=1e-15, atol=0)


def dense_vcycle_var(dims, kappa, levels, nu=2, omega=2.0 / 3.0):
    """The variable-coefficient V-cycle as a dense matrix from the face-list operators:
    V = M^nu G + B_nu, G = B_nu + P C R (I - A B_nu), Jacobi diagonal D = diag(A), coarse operator
    from the coarse faces; exact inverse on the coarsest level."""
    from tests.test_oracle_multigrid import hat_prolongation, kron3
    A = face_list_matrix(dims, kappa)
    n = A.shape[0]
    if levels == 1:
        return np.linalg.inv(A)
    dc = tuple(x // 2 for x in dims)
    P = kron3(hat_prolongation(dims[0]), hat_prolongation(dims[1]), hat_prolongation(dims[2]))
    R = P.T / 8.0
    C = dense_vcycle_var(dc, varcoef.coarse_kappa(dims, kappa, dc), levels - 1, nu, omega)
    Dinv = omega / np.diag(A)
    M = np.eye(n) - Dinv[:, None] * A
    B = sum(np.linalg.matrix_power(M, t) for t in range(nu)) @ np.diag(Dinv)
    G = B + P @ C @ R @ (np.eye(n) - A @ B)
    return np.linalg.matrix_power(M, nu) @ G + B


@pytest.mark.parametrize("dims,levels", [((6, 5, 4), 2), ((8, 7, 6), 3)])
def test_vcycle_matches_dense_face_list_assembly(dims, levels):
    kappa = fields.random_kappa(dims, seed=9, length=2.5)
    T = varcoef.VCycleVar(dims, kappa, levels=levels)
    n = int(np.prod(dims))
    V = dense_vcycle_var(dims, kappa, levels)
    M = T(np.eye(n))
    assert np.max(np.abs(M - V)) <= 1e-12 * np.max(np.abs(V))
