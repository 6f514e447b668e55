"""Geometric-multigrid V-cycle preconditioner T on the structured grid.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper applies hypre/PETSc preconditioners (BoomerAMG, SMG, PFMG, Schwarz;
Sections 4.2-4.4, Appendix D).  This project replaces them by a plain
geometric V-cycle; the paper fixes only the properties T must have: linear,
symmetric and positive definite (Section 2.1.1).  Definition used (this
project's reading, since the paper is silent):

* Levels l = 0..L-1.  Level l+1 has floor(n/2) points per axis of level l;
  coarse index I (1-based) sits on fine index 2I.  Operator on level l is the
  same 7-point stencil with scale s_{l+1} = s_l / 4 (mesh width doubles).
* 1-D prolongation P[i, I] = 1 if i = 2I, 1/2 if |i - 2I| = 1, else 0
  (1-based; coarse boundary values are zero).  3-D P is the tensor product
  (trilinear interpolation); restriction is R = P^T / 8 (full weighting).
* Smoother: weighted Jacobi  e <- e + omega D^-1 (r - A_l e),  D = 6 s_l,
  omega = 2/3, nu_pre sweeps from e = 0 and nu_post sweeps after the coarse
  correction (nu_pre = nu_post keeps T symmetric).
* Coarsest level: exact solve with a dense Cholesky factor of A_{L-1}.

Pinned by: dense two- and three-level operators assembled independently from
Kronecker products; symmetry and positive definiteness of T; exactness of P on
trilinear functions; the unit row sums of R.  Values beyond those pins are
"parity unpinned": the paper does not define this V-cycle.
"""

import numpy as np
import scipy.linalg

from . import laplace

MAX_COARSEST = 4096


def level_dims(dims, levels):
    """Grid dimensions of each level, finest first."""
    out = [tuple(int(d) for d in dims)]
    for _ in range(1, levels):
        nxt = tuple(d // 2 for d in out[-1])
        if min(nxt) < 1:
            raise ValueError(f"grid {dims} cannot be coarsened to {levels} levels")
        out.append(nxt)
    return out


def prolongation_1d(nf):
    """Dense (nf, nc) 1-D prolongation matrix, nc = nf // 2."""
    nc = nf // 2
    P = np.zeros((nf, nc))
    for I in range(1, nc + 1):          # 1-based coarse index
        for i in (2 * I - 1, 2 * I, 2 * I + 1):   # 1-based fine neighbours
            if 1 <= i <= nf:
                P[i - 1, I - 1] = 1.0 if i == 2 * I else 0.5
    return P


def _along(u, M, axis):
    """Apply matrix M (rows out, cols in) along one grid axis of u (m, nz, ny, nx)."""
    return np.moveaxis(np.tensordot(M, u, axes=([1], [axis])), 0, axis)


def prolong(Ec, dims_c, dims_f):
    """P Ec for an (nc, m) coarse block -> (nf, m) fine block."""
    u = Ec.T.reshape(Ec.shape[1], dims_c[2], dims_c[1], dims_c[0])
    u = _along(u, prolongation_1d(dims_f[0]), 3)
    u = _along(u, prolongation_1d(dims_f[1]), 2)
    u = _along(u, prolongation_1d(dims_f[2]), 1)
    return np.ascontiguousarray(u.reshape(u.shape[0], -1).T)


def restrict(Rf, dims_f, dims_c):
    """R Rf = P^T Rf / 8 for an (nf, m) fine block -> (nc, m) coarse block."""
    u = Rf.T.reshape(Rf.shape[1], dims_f[2], dims_f[1], dims_f[0])
    u = _along(u, prolongation_1d(dims_f[0]).T, 3)
    u = _along(u, prolongation_1d(dims_f[1]).T, 2)
    u = _along(u, prolongation_1d(dims_f[2]).T, 1)
    return np.ascontiguousarray(u.reshape(u.shape[0], -1).T) / 8.0


class VCycle:
    """The preconditioner T as a callable on (n, m) blocks."""

    def __init__(self, dims, scale, levels, nu_pre=2, nu_post=2, omega=2.0 / 3.0):
        self.dims = level_dims(dims, levels)
        self.scales = [scale / 4.0 ** l for l in range(levels)]
        self.levels = levels
        self.nu_pre, self.nu_post, self.omega = nu_pre, nu_post, omega
        nc = laplace.npoints(self.dims[-1])
        if nc > MAX_COARSEST:
            raise ValueError(f"coarsest level has {nc} points (> {MAX_COARSEST}); add levels")
        Ac = laplace.dense_matrix(self.dims[-1], self.scales[-1])
        self.coarse_factor = scipy.linalg.cho_factor(Ac, lower=False)

    def _jacobi(self, l, r, e):
        d = 6.0 * self.scales[l]
        return e + (self.omega / d) * (r - laplace.apply(e, self.dims[l], self.scales[l]))

    def _cycle(self, l, r):
        if l == self.levels - 1:
            return scipy.linalg.cho_solve(self.coarse_factor, r)
        e = np.zeros_like(r)
        for _ in range(self.nu_pre):
            e = self._jacobi(l, r, e)
        res = r - laplace.apply(e, self.dims[l], self.scales[l])
        rc = restrict(res, self.dims[l], self.dims[l + 1])
        ec = self._cycle(l + 1, rc)
        e = e + prolong(ec, self.dims[l + 1], self.dims[l])
        for _ in range(self.nu_post):
            e = self._jacobi(l, r, e)
        return e

    def __call__(self, R):
        R = np.asarray(R, dtype=np.float64)
        if R.ndim == 1:
            return self._cycle(0, R[:, None])[:, 0]
        return self._cycle(0, R)
