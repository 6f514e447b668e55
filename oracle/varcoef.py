"""Variable-coefficient 7-point operator -div(kappa grad u), its V-cycle and the eigenvalue gradient.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's model problem is the constant-coefficient Laplacian (Section 4); this is the
differentiated operator the project adds beside it (unit spacing h = 1, Dirichlet: the
eigenvector is zero on the ghost layer around the box):

    (A u)_p = sum over the 6 faces f of p of kappa_f (u_p - u_q),   u_q = 0 outside the box,

with kappa given per face in the layout of paper_0705_2626_gb300.fields (x-, y-, z-faces).

Eigenvalue derivative (first-order perturbation of a symmetric eigenproblem with unit-norm
eigenvector x_i; dA/dkappa_f = (e_p - e_q)(e_p - e_q)^T, or e_p e_p^T on a boundary face):

    d lambda_i / d kappa_f = (x_i,p - x_i,q)^2    (x_i,q = 0 on boundary faces),

valid for a simple eigenvalue; for a cluster of equal eigenvalues the sum over the cluster is
basis-invariant.  grad(w) returns sum_i w_i (x_i,p - x_i,q)^2.

V-cycle (this project's reading; the paper has no variable-coefficient preconditioner): levels,
transfer operators and smoother as in multigrid.VCycle, with the Jacobi diagonal
D_p = sum of the 6 face coefficients of p, and rediscretised coarse operators whose faces are
  * along the face normal: the harmonic mean of the two fine faces the coarse face spans
    (two conductances in series over twice the length; one face where the coarse grid is not
    nested at the far end of an even-sized axis);
  * across it: the average of those line values over the fine lines at offsets -1, 0, +1 with
    weights 1/4, 1/2, 1/4 (lines outside the box dropped, weights renormalised);
  * divided by 4 (mesh width 2h), so that kappa = const reproduces the constant operator's
    s_{l+1} = s_l / 4.
"""

import numpy as np
import scipy.linalg

from . import multigrid


def split(kappa, dims):
    nx, ny, nz = dims
    cx, cy = (nx + 1) * ny * nz, nx * (ny + 1) * nz
    cz = nx * ny * (nz + 1)
    kappa = np.asarray(kappa, dtype=np.float64)
    assert kappa.size == cx + cy + cz
    return (kappa[:cx].reshape(nz, ny, nx + 1), kappa[cx:cx + cy].reshape(nz, ny + 1, nx),
            kappa[cx + cy:].reshape(nz + 1, ny, nx))


def _padded(U, dims):
    nx, ny, nz = dims
    m = U.shape[1]
    g = np.zeros((m, nz + 2, ny + 2, nx + 2))
    g[:, 1:-1, 1:-1, 1:-1] = U.T.reshape(m, nz, ny, nx)
    return g


def apply(U, dims, kappa):
    """A U for an (n, m) block."""
    U = np.asarray(U, dtype=np.float64)
    vec = U.ndim == 1
    if vec:
        U = U[:, None]
    kx, ky, kz = split(kappa, dims)
    g = _padded(U, dims)
    c = g[:, 1:-1, 1:-1, 1:-1]
    fx = kx * (g[:, 1:-1, 1:-1, 1:] - g[:, 1:-1, 1:-1, :-1])     # kappa_f (u_right - u_left)
    fy = ky * (g[:, 1:-1, 1:, 1:-1] - g[:, 1:-1, :-1, 1:-1])
    fz = kz * (g[:, 1:, 1:-1, 1:-1] - g[:, :-1, 1:-1, 1:-1])
    out = (fx[..., :-1] - fx[..., 1:]) + (fy[:, :, :-1, :] - fy[:, :, 1:, :]) + (fz[:, :-1] - fz[:, 1:])
    del c
    out = out.reshape(U.shape[1], -1).T
    return out[:, 0] if vec else out


def diagonal(dims, kappa):
    kx, ky, kz = split(kappa, dims)
    d = (kx[:, :, :-1] + kx[:, :, 1:]) + (ky[:, :-1, :] + ky[:, 1:, :]) + (kz[:-1] + kz[1:])
    return d.ravel()


def dense_matrix(dims, kappa):
    n = int(np.prod(dims))
    return apply(np.eye(n), dims, kappa)


def grad(X, dims, w):
    """sum_i w_i (x_i,p - x_i,q)^2 per face (same layout as kappa)."""
    X = np.asarray(X, dtype=np.float64)
    g = _padded(X, dims)
    w = np.asarray(w, dtype=np.float64)
    dx = (g[:, 1:-1, 1:-1, 1:] - g[:, 1:-1, 1:-1, :-1]) ** 2
    dy = (g[:, 1:-1, 1:, 1:-1] - g[:, 1:-1, :-1, 1:-1]) ** 2
    dz = (g[:, 1:, 1:-1, 1:-1] - g[:, :-1, 1:-1, 1:-1]) ** 2
    return np.concatenate([np.tensordot(w, dx, axes=1).ravel(), np.tensordot(w, dy, axes=1).ravel(),
                           np.tensordot(w, dz, axes=1).ravel()])


def _coarse_axis_faces(k, axis_len_f, axis_len_c, along, across):
    """Coarse face values for faces normal to one axis.  `k` is the fine face array moved so that
    its axes are (across0, across1, along) with the along axis of length n_f + 1."""
    nf, nc = axis_len_f, axis_len_c
    a0f, a1f = k.shape[0], k.shape[1]
    a0c, a1c = across
    # along: coarse face F (0..nc) spans fine faces 2F and 2F + 1 (0-based)
    line = np.empty((a0f, a1f, nc + 1))
    for F in range(nc + 1):
        fs = [f for f in (2 * F, 2 * F + 1) if f <= nf]
        if len(fs) == 2:
            line[:, :, F] = 2.0 / (1.0 / k[:, :, fs[0]] + 1.0 / k[:, :, fs[1]])
        else:
            line[:, :, F] = k[:, :, fs[0]]
    # across: coarse line J (0-based) sits on fine 2J + 1; offsets -1, 0, +1 weighted 1/4, 1/2, 1/4
    def avg(arr, nfine, ncoarse, axis):
        out_shape = list(arr.shape)
        out_shape[axis] = ncoarse
        out = np.zeros(out_shape)
        for J in range(ncoarse):
            tot = 0.0
            acc = 0.0
            for off, wgt in ((-1, 0.25), (0, 0.5), (1, 0.25)):
                j = 2 * J + 1 + off
                if 0 <= j < nfine:
                    acc = acc + wgt * np.take(arr, j, axis=axis)
                    tot += wgt
            idx = [slice(None)] * arr.ndim
            idx[axis] = J
            out[tuple(idx)] = acc / tot
        return out
    line = avg(line, a0f, a0c, 0)
    line = avg(line, a1f, a1c, 1)
    return line / 4.0


def coarse_kappa(dims_f, kappa, dims_c):
    """Face coefficients of the rediscretised operator on the next coarser level."""
    nx, ny, nz = dims_f
    cx, cy, cz = dims_c
    kx, ky, kz = split(kappa, dims_f)
    # x-faces: array (nz, ny, nx+1) -> across axes (z, y), along x
    Kx = _coarse_axis_faces(kx, nx, cx, 2, (cz, cy))                              # (cz, cy, cx+1)
    # y-faces: (nz, ny+1, nx) -> across (z, x), along y
    Ky = _coarse_axis_faces(np.moveaxis(ky, 1, 2), ny, cy, 1, (cz, cx))           # (cz, cx, cy+1)
    Ky = np.moveaxis(Ky, 2, 1)                                                    # (cz, cy+1, cx)
    # z-faces: (nz+1, ny, nx) -> across (y, x), along z
    Kz = _coarse_axis_faces(np.moveaxis(kz, 0, 2), nz, cz, 0, (cy, cx))           # (cy, cx, cz+1)
    Kz = np.moveaxis(Kz, 2, 0)                                                    # (cz+1, cy, cx)
    return np.concatenate([Kx.ravel(), Ky.ravel(), Kz.ravel()])


class VarCoef7:
    """The operator A as a callable on (n, m) blocks."""

    def __init__(self, dims, kappa):
        self.dims = tuple(int(d) for d in dims)
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.n = int(np.prod(self.dims))

    def __call__(self, U):
        return apply(U, self.dims, self.kappa)


class VCycleVar:
    """The V-cycle preconditioner of the variable-coefficient operator, on (n, m) blocks."""

    def __init__(self, dims, kappa, levels, nu_pre=2, nu_post=2, omega=2.0 / 3.0):
        self.dims = multigrid.level_dims(dims, levels)
        self.kappas = [np.asarray(kappa, dtype=np.float64)]
        for l in range(1, levels):
            self.kappas.append(coarse_kappa(self.dims[l - 1], self.kappas[-1], self.dims[l]))
        self.diags = [diagonal(d, k) for d, k in zip(self.dims, self.kappas)]
        self.levels = levels
        self.nu_pre, self.nu_post, self.omega = nu_pre, nu_post, omega
        nc = int(np.prod(self.dims[-1]))
        if nc > multigrid.MAX_COARSEST:
            raise ValueError(f"coarsest level has {nc} points; add levels")
        self.coarse_factor = scipy.linalg.cho_factor(dense_matrix(self.dims[-1], self.kappas[-1]), lower=False)

    def _jacobi(self, l, r, e):
        return e + self.omega * (r - apply(e, self.dims[l], self.kappas[l])) / self.diags[l][:, None]

    def _cycle(self, l, r):
        if l == self.levels - 1:
            return scipy.linalg.cho_solve(self.coarse_factor, r)
        e = np.zeros_like(r)
        for _ in range(self.nu_pre):
            e = self._jacobi(l, r, e)
        res = r - apply(e, self.dims[l], self.kappas[l])
        ec = self._cycle(l + 1, multigrid.restrict(res, self.dims[l], self.dims[l + 1]))
        e = e + multigrid.prolong(ec, self.dims[l + 1], self.dims[l])
        for _ in range(self.nu_post):
            e = self._jacobi(l, r, e)
        return e

    def __call__(self, R):
        R = np.asarray(R, dtype=np.float64)
        if R.ndim == 1:
            return self._cycle(0, R[:, None])[:, 0]
        return self._cycle(0, R)
