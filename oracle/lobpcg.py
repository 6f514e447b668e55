"""Block LOBPCG with soft locking, B = I, optional constraints.

TEST INFRASTRUCTURE ONLY (see the package header).

Follows the algorithm of Section 2.2 ("The Detailed Description of the LOBPCG
Algorithm", the algorithm of Section 2.2) with B = I (so BX = X, BW = W, BP = P and 6m vectors
are stored, as the paper notes after the algorithm).  Soft locking as in
Section 2.3: only the active columns J get residuals, preconditioned residuals
and directions; all m columns of X stay in the Rayleigh-Ritz basis.  A
constraint block Y (l linearly independent columns; the hard locking of
Section 2.3) enters in the constraint projection of X, X = X - Y (Y^T Y)^-1 (Y^T X), and in the constraint projection of W,
W_J = W_J - Y (Y^T Y)^-1 (Y^T W_J); without Y both steps are empty.

Readings of points the paper leaves open (each listed in the design notes):
* convergence test (the soft-locking test): column j leaves J when ||A x_j - lambda_j x_j||_2
  <= tol * |lambda_j| (``tol_mode="relative"``, default) or <= tol
  (``"absolute"``, the paper's literal wording); J only shrinks while columns
  remain active.
* final check (``final_check=True``, default): soft-locked columns stay in the
  Rayleigh-Ritz basis (Section 2.3), and inside a cluster of equal Ritz values
  the Rayleigh-Ritz rotation can move part of an active column's error into a locked
  one after its test.  So when J empties, every residual is recomputed from a
  fresh A X (which also replaces the implicitly updated AX of the update of AX);
  columns above the tolerance re-enter J and the iteration continues; the solve
  is converged only when this check passes, so every returned residual meets
  the tolerance (the target the paper's tests state, Section 4.1).
  ``final_check=False`` keeps the printed rule (exit as soon as J is empty).
* loop bound (the iteration loop, k = 0..MaxIterations): the pass k = maxit performs only
  the residuals and the soft-locking test; ``iters`` is the k at which J became empty.
* Gram blocks (the Gram blocks): the paper prints only the upper block triangle of
  gramA (the blocks below the diagonal are its transposes); those blocks are
  computed, including the diagonal blocks the paper sets to Lambda and I, which
  are symmetrised (G + G^T)/2 (the explicit variant the paper reports as more
  accurate).  gramB = S^T S.  ``gram="paper"`` sets the diagonal blocks as
  printed in the algorithm.
* Cholesky (the orthonormalisations of X, W and P): scale-invariant via unit-diagonal scaling.
* breakdown: if chol(P_J^T P_J) or the Rayleigh-Ritz with P fails, the P block
  is dropped for that iteration (the form without P at k = 0); if
  chol(X^T X) or chol(W_J^T W_J) fails the solve stops with status "breakdown".
* at exit every residual is recomputed from A X (not the implicitly updated AX).
* constraints: (Y^T Y)^-1 is applied through the scale-invariant Cholesky factor
  of Y^T Y; if that factorisation fails (Y not linearly independent) the solve
  stops with status "breakdown" before the orthonormalisation of X.
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import laplace
from .dense import Breakdown, scaled_cholesky, apply_inverse_upper, symmetrize, rayleigh_ritz


@dataclass
class Result:
    lam: np.ndarray
    X: np.ndarray
    iters: int
    status: str                     # "converged" | "not_converged" | "breakdown" | "nonfinite"
    resid: np.ndarray               # final ||A x_j - lambda_j x_j||, from A X
    history: list = field(default_factory=list)


class Laplace7:
    """The operator A as a callable on (n, m) blocks."""

    def __init__(self, dims, scale=None):
        self.dims = tuple(int(d) for d in dims)
        self.scale = laplace.default_scale(self.dims) if scale is None else float(scale)
        self.n = laplace.npoints(self.dims)

    def __call__(self, U):
        return laplace.apply(U, self.dims, self.scale)


def upper_block_gram(S, AS):
    """gramA of the Gram blocks as printed: blocks S_I^T AS_J for I <= J, lower blocks by symmetry,
    diagonal blocks symmetrised."""
    widths = [b.shape[1] for b in S]
    offs = np.concatenate([[0], np.cumsum(widths)])
    q = int(offs[-1])
    G = np.empty((q, q))
    for I in range(len(S)):
        for J in range(I, len(S)):
            blk = S[I].T @ AS[J]
            if I == J:
                blk = symmetrize(blk)
            G[offs[I]:offs[I + 1], offs[J]:offs[J + 1]] = blk
            G[offs[J]:offs[J + 1], offs[I]:offs[I + 1]] = blk.T
    return G


def constraint_projector(Y):
    """V -> V - Y (Y^T Y)^-1 (Y^T V) (the constraint projections with B = I), with Y^T Y = R^T R from the
    scale-invariant Cholesky; raises Breakdown if Y^T Y is not positive definite."""
    R = scaled_cholesky(Y.T @ Y)

    def project(V):
        C = Y.T @ V
        Z = scipy.linalg.solve_triangular(R, scipy.linalg.solve_triangular(R, C, trans="T"))
        return V - Y @ Z
    return project


def _converged(norm, lam, tol, tol_mode):
    bound = tol * abs(lam) if tol_mode == "relative" else tol
    return norm <= bound


def lobpcg(A, X0, tol, maxit, T=None, tol_mode="relative", gram="explicit", record=False, on_pass=None, Y=None,
           final_check=True):
    """Smallest m = X0.shape[1] eigenpairs of the operator A, preconditioner T (None = identity),
    in the complement of the constraint block Y ((n, l) array or None).

    ``on_pass(k)`` (optional) is called at the end of pass k, for timing only.
    """
    X = np.array(X0, dtype=np.float64, copy=True)
    n, m = X.shape
    hist = []
    if not np.all(np.isfinite(X)):
        return Result(np.full(m, np.nan), X, 0, "nonfinite", np.full(m, np.nan))
    precond = (lambda R: R) if T is None else T
    constrain = None
    if Y is not None and Y.shape[1] > 0:
        try:
            constrain = constraint_projector(np.asarray(Y, dtype=np.float64))
        except Breakdown:
            return Result(np.full(m, np.nan), X, 0, "breakdown", np.full(m, np.nan))
        # constraints: project the initial block
        X = constrain(X)

    # orthonormalise X (B = I): R = chol(X^T X), X = X R^-1, AX = A X
    try:
        R = scaled_cholesky(X.T @ X)
    except Breakdown:
        return Result(np.full(m, np.nan), X, 0, "breakdown", np.full(m, np.nan))
    X = apply_inverse_upper(X, R)
    AX = A(X)
    # initial Ritz vectors from (X^T AX) TMP = TMP Lambda
    lam, TMP = rayleigh_ritz(symmetrize(X.T @ AX), np.eye(m), m)
    X = X @ TMP
    AX = AX @ TMP
    # all columns active
    J = list(range(m))
    P = AP = None
    iters, status = maxit, "not_converged"

    for k in range(0, maxit + 1):
        # residuals of the active columns
        W = AX[:, J] - X[:, J] * lam[J][None, :]
        norms = np.linalg.norm(W, axis=0)
        if not (np.all(np.isfinite(norms)) and np.all(np.isfinite(lam))):
            status, iters = "nonfinite", k
            break
        # soft-lock converged columns; exit when none is left
        keep = [t for t, j in enumerate(J) if not _converged(norms[t], lam[j], tol, tol_mode)]
        if record:
            hist.append(dict(k=k, lam=lam.copy(), J=list(J), norms=norms.copy(),
                             orth=float(np.max(np.abs(X.T @ X - np.eye(m)))), dropped_p=False))
        J = [J[t] for t in keep]
        W = W[:, keep]
        if not J and final_check:
            # Final check: residuals of all m columns from a fresh A X; failing columns re-enter.
            AX = A(X)
            Rall = AX - X * lam[None, :]
            norms_all = np.linalg.norm(Rall, axis=0)
            J = [j for j in range(m) if not _converged(norms_all[j], lam[j], tol, tol_mode)]
            W = Rall[:, J]
            if record:
                hist[-1]["recheck_J"] = list(J)
        if not J:
            status, iters = "converged", k
            break
        if k == maxit:
            break
        # precondition
        W = precond(W)
        # constraints: project the preconditioned residuals
        if constrain is not None:
            W = constrain(W)
        # orthonormalise W_J
        try:
            R = scaled_cholesky(W.T @ W)
        except Breakdown:
            status, iters = "breakdown", k
            break
        W = apply_inverse_upper(W, R)
        # AW_J = A W_J
        AW = A(W)
        # orthonormalise P_J and update AP_J (k > 0)
        use_p = k > 0
        if use_p:
            PJ, APJ = P[:, J], AP[:, J]
            try:
                R = scaled_cholesky(PJ.T @ PJ)
                PJ = apply_inverse_upper(PJ, R)
                APJ = apply_inverse_upper(APJ, R)
            except Breakdown:
                use_p = False
        # Gram matrices of the basis and the Rayleigh-Ritz eigenproblem
        dropped = False
        while True:
            S = [X, W] + ([PJ] if use_p else [])
            AS = [AX, AW] + ([APJ] if use_p else [])
            Sm = np.hstack(S)
            gramA = upper_block_gram(S, AS)
            gramB = symmetrize(Sm.T @ Sm)
            if gram == "paper":
                gramA[:m, :m] = np.diag(lam)
                off = 0
                for blk in S:
                    w = blk.shape[1]
                    gramB[off:off + w, off:off + w] = np.eye(w)
                    off += w
            try:
                lam, C = rayleigh_ritz(gramA, gramB, m)
                break
            except Breakdown:
                if use_p:
                    use_p, dropped = False, True
                    continue
                status, iters = "breakdown", k
                lam = None
                break
        if lam is None:
            lam = hist[-1]["lam"] if hist else np.full(m, np.nan)
            break
        if record and dropped:
            hist[-1]["dropped_p"] = True
        # Ritz vectors: the update of X and P
        b = len(J)
        CX, CW = C[:m], C[m:m + b]
        P = W @ CW
        AP = AW @ CW
        if use_p:
            CP = C[m + b:m + 2 * b]
            P = P + PJ @ CP
            AP = AP + APJ @ CP
        X = X @ CX + P
        AX = AX @ CX + AP
        if on_pass is not None:
            on_pass(k)

    resid = np.linalg.norm(A(X) - X * lam[None, :], axis=0)
    return Result(lam, X, iters, status, resid, hist)
