"""The 7-point finite-difference Dirichlet Laplacian and its closed-form eigenpairs.

TEST INFRASTRUCTURE ONLY (see the package header).

Model problem of the paper (Section 4): the 3-D 7-point Laplacian on an
nx x ny x nz interior grid with Dirichlet boundaries.  Grid point (i, j, k),
0-based interior indices, has linear index p = i + nx*(j + ny*k); a block of
vectors is an (n, m) float64 array whose column c is one grid function.

Operator (scaled stencil):   (A u)_p = s * (6 u_p - sum of the 6 neighbours),
neighbours outside the interior count as zero.  With s = 1 the eigenvalues are
exactly the paper's formula (Section 4.1):

    lambda_{a,b,c} = 4 [ sin^2(a pi / (2(nx+1))) + sin^2(b pi / (2(ny+1)))
                         + sin^2(c pi / (2(nz+1))) ],   1 <= a <= nx, ...

and for the cube with s = h^-2, h = 1/(n+1), they are (4/h^2) * sum sin^2(...).
The eigenvectors are the products sin(a pi x) sin(b pi y) sin(c pi z) with
x = (i+1)/(nx+1) (textbook; not printed in the paper).

Pinned by: a Kronecker-sum assembly of the dense matrix on small grids, and
the closed form against a dense symmetric eigensolve.
"""

import itertools
import numpy as np


def npoints(dims):
    nx, ny, nz = dims
    return nx * ny * nz


def default_scale(dims):
    """h^-2 for the cube, h = 1/(n+1); 1.0 (the paper's unscaled formula) otherwise."""
    nx, ny, nz = dims
    if nx == ny == nz:
        return float(nx + 1) ** 2
    return 1.0


def _as_grid(U, dims):
    nx, ny, nz = dims
    m = U.shape[1]
    return U.T.reshape(m, nz, ny, nx)


def _as_block(u, dims):
    m = u.shape[0]
    return np.ascontiguousarray(u.reshape(m, npoints(dims)).T)


def apply(U, dims, scale):
    """A U for an (n, m) block U: the 7-point stencil with zero Dirichlet data."""
    U = np.asarray(U, dtype=np.float64)
    if U.ndim == 1:
        return apply(U[:, None], dims, scale)[:, 0]
    u = _as_grid(U, dims)
    m, nz, ny, nx = u.shape
    pad = np.zeros((m, nz + 2, ny + 2, nx + 2))
    pad[:, 1:-1, 1:-1, 1:-1] = u
    nbr = (pad[:, 1:-1, 1:-1, :-2] + pad[:, 1:-1, 1:-1, 2:]      # x - 1, x + 1
           + pad[:, 1:-1, :-2, 1:-1] + pad[:, 1:-1, 2:, 1:-1]    # y - 1, y + 1
           + pad[:, :-2, 1:-1, 1:-1] + pad[:, 2:, 1:-1, 1:-1])   # z - 1, z + 1
    return _as_block(scale * (6.0 * u - nbr), dims)


def dense_matrix(dims, scale):
    """Dense n x n matrix of the operator, assembled by applying it to unit vectors."""
    n = npoints(dims)
    return apply(np.eye(n), dims, scale)


def exact_eigenvalues(dims, scale, count):
    """The ``count`` smallest eigenvalues (ascending), from the closed form of Section 4.1."""
    nx, ny, nz = dims
    lim = [min(d, count) for d in dims]
    sx = np.sin(np.arange(1, lim[0] + 1) * np.pi / (2 * (nx + 1))) ** 2
    sy = np.sin(np.arange(1, lim[1] + 1) * np.pi / (2 * (ny + 1))) ** 2
    sz = np.sin(np.arange(1, lim[2] + 1) * np.pi / (2 * (nz + 1))) ** 2
    lam = 4.0 * scale * (sx[:, None, None] + sy[None, :, None] + sz[None, None, :])
    return np.sort(lam.ravel())[:count]


def exact_modes(dims, scale, count):
    """[(lambda, (a, b, c))] for the ``count`` smallest eigenvalues, ascending."""
    nx, ny, nz = dims
    lim = [min(d, count) for d in dims]
    out = []
    for a, b, c in itertools.product(range(1, lim[0] + 1), range(1, lim[1] + 1), range(1, lim[2] + 1)):
        lam = 4.0 * scale * (np.sin(a * np.pi / (2 * (nx + 1))) ** 2
                             + np.sin(b * np.pi / (2 * (ny + 1))) ** 2
                             + np.sin(c * np.pi / (2 * (nz + 1))) ** 2)
        out.append((lam, (a, b, c)))
    out.sort(key=lambda t: t[0])
    return out[:count]


def exact_eigenvector(dims, abc):
    """Unit-norm sine-product eigenvector for mode (a, b, c), as a length-n vector."""
    nx, ny, nz = dims
    a, b, c = abc
    x = np.arange(1, nx + 1) / (nx + 1)
    y = np.arange(1, ny + 1) / (ny + 1)
    z = np.arange(1, nz + 1) / (nz + 1)
    v = (np.sin(c * np.pi * z)[:, None, None] * np.sin(b * np.pi * y)[None, :, None]
         * np.sin(a * np.pi * x)[None, None, :]).ravel()
    return v / np.linalg.norm(v)


def eigen_clusters(lams, rtol=1e-9):
    """Group indices of an ascending eigenvalue list into clusters of (numerically) equal values."""
    clusters, cur = [], [0]
    for i in range(1, len(lams)):
        if abs(lams[i] - lams[cur[0]]) <= rtol * abs(lams[cur[0]]):
            cur.append(i)
        else:
            clusters.append(cur)
            cur = [i]
    clusters.append(cur)
    return clusters


def exact_eigenspace(dims, scale, lam, rtol=1e-9, max_index=None):
    """Orthonormal basis (n, d) of the exact eigenspace of eigenvalue ``lam`` (all modes that equal it)."""
    nx, ny, nz = dims
    lim = max_index or max(nx, ny, nz)
    vecs = []
    for a in range(1, min(nx, lim) + 1):
        for b in range(1, min(ny, lim) + 1):
            for c in range(1, min(nz, lim) + 1):
                mu = 4.0 * scale * (np.sin(a * np.pi / (2 * (nx + 1))) ** 2
                                    + np.sin(b * np.pi / (2 * (ny + 1))) ** 2
                                    + np.sin(c * np.pi / (2 * (nz + 1))) ** 2)
                if abs(mu - lam) <= rtol * abs(lam):
                    vecs.append(exact_eigenvector(dims, (a, b, c)))
    return np.stack(vecs, axis=1)
