"""Inner preconditioned conjugate gradients as the LOBPCG preconditioner (Section 4.2).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's Section 4.2 ("Performance Versus the Number of Inner Iterations") applies the
preconditioner x = T b either directly or through a PCG solve of A x = b, so that T approximates
A^-1 better with more inner iterations (and becomes a nonlinear map of b, which Section 2.1
allows for LOBPCG).  Here T_k(b) = x_k, the k-th iterate of PCG for A x = b from x_0 = 0
preconditioned by M (the V-cycle), column by column; k = 0 means T = M applied directly.

PCG (the textbook recurrences, written out): r_0 = b, z_0 = M r_0, p_0 = z_0, and for i = 0..k-1
  alpha_i = (r_i . z_i) / (p_i . A p_i),  x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i - alpha_i A p_i,
  z_{i+1} = M r_{i+1},  beta_i = (r_{i+1} . z_{i+1}) / (r_i . z_i),  p_{i+1} = z_{i+1} + beta_i p_i.
A column stops early (keeps its x) once p . A p <= 0 or r . z <= 0 (exact convergence, or a
breakdown of a non-definite M); no other tolerance is applied -- the paper fixes the iteration
count, not a residual target.
"""

import numpy as np


def pcg_columns(A, M, B, k):
    """X = T_k(B) for the (n, b) block B: k PCG iterations per column (k = 0: M(B))."""
    B = np.asarray(B, dtype=np.float64)
    if k == 0:
        return M(B)
    X = np.zeros_like(B)
    R = B.copy()
    Z = M(R)
    P = Z.copy()
    rz = np.sum(R * Z, axis=0)
    active = rz > 0
    for _ in range(k):
        if not np.any(active):
            break
        AP = A(P)
        pap = np.sum(P * AP, axis=0)
        active &= pap > 0
        alpha = np.where(active, rz / np.where(active, pap, 1.0), 0.0)
        X += P * alpha[None, :]
        R -= AP * alpha[None, :]
        Z = M(R)
        rz_new = np.sum(R * Z, axis=0)
        active &= rz_new > 0
        beta = np.where(active, rz_new / np.where(rz > 0, rz, 1.0), 0.0)
        P = Z + P * beta[None, :]
        rz = rz_new
    return X


class InnerPCG:
    """The preconditioner T_k as a callable on (n, m) blocks."""

    def __init__(self, A, M, k):
        self.A, self.M, self.k = A, M, int(k)

    def __call__(self, B):
        return pcg_columns(self.A, self.M, B, self.k)
