"""Small dense steps of the algorithm: scale-invariant Cholesky and Rayleigh-Ritz.

TEST INFRASTRUCTURE ONLY (see the package header).

* ``scaled_cholesky`` -- the Cholesky factor used for the orthonormalisation of
  X, W and P (Section 2.2).  The paper requires the factorisation
  to be invariant to column scaling, or else an explicit normalisation of the
  columns first (Section 2.2, discussion after the algorithm).  Reading used:
  always normalise, i.e. D = diag(G)^-1/2, R' = chol(D G D) (upper),
  R = R' D^-1, so that G = R^T R and  X R^-1 = X D R'^-1.
  Numerical breakdown (the paper only warns of it): on the unit-diagonal
  matrix D G D, any pivot (the square of a diagonal entry of R') at or below
  q * eps (q = order, eps = 2^-52) counts as failure.
* ``rayleigh_ritz`` -- the Rayleigh-Ritz step (Section 2.2): gramA C = gramB C Lambda, the first m
  eigenvalues ascending, C gramB-orthonormal.  The library routine
  scipy.linalg.eigh (LAPACK sygvd) is the step.

Pinned by: reconstruction G = R^T R and exact invariance under column scaling;
the generalized eigen-equations and gramB-orthonormality of C; reduction to the
standard symmetric eigenproblem when gramB = I.
"""

import numpy as np
import scipy.linalg


class Breakdown(Exception):
    """A Gram matrix that should be positive definite is not (numerically)."""


def scaled_cholesky(G):
    """Upper-triangular R with G = R^T R, computed on the unit-diagonal scaling of G."""
    G = np.asarray(G, dtype=np.float64)
    if not np.all(np.isfinite(G)):
        raise Breakdown("non-finite Gram matrix")
    dg = np.diag(G).copy()
    if np.any(dg <= 0.0):
        raise Breakdown("non-positive diagonal in Gram matrix")
    d = 1.0 / np.sqrt(dg)
    S = d[:, None] * G * d[None, :]
    try:
        L = np.linalg.cholesky(S)
    except np.linalg.LinAlgError as exc:
        raise Breakdown(str(exc)) from exc
    q = G.shape[0]
    if np.min(np.diag(L)) ** 2 <= q * np.finfo(np.float64).eps:
        raise Breakdown("numerically singular Gram matrix")
    Rp = L.T
    return Rp / d[None, :]          # R = R' D^-1  (column k of R' divided by d_k)


def apply_inverse_upper(X, R):
    """X R^-1 for upper-triangular R (triangular solve, no explicit inverse)."""
    return scipy.linalg.solve_triangular(R, X.T, trans="T", lower=False).T


def symmetrize(G):
    return 0.5 * (G + G.T)


def rayleigh_ritz(gramA, gramB, m):
    """(Lambda[m], C[:, :m]) of gramA C = gramB C Lambda, ascending, C^T gramB C = I."""
    try:
        lam, C = scipy.linalg.eigh(gramA, gramB)
    except np.linalg.LinAlgError as exc:
        raise Breakdown(str(exc)) from exc
    return lam[:m], C[:, :m]
