"""Seeded synthetic inputs of the variable-coefficient operator -div(kappa grad u).

This module only generates inputs; it holds none of the eigensolver's arithmetic, and both the
CUDA path and the float64 oracle take its arrays as given.

Face layout (one float64 array, three consecutive parts, x fastest inside each part):
  x-faces: (nx+1) * ny * nz, face (f, j, k) between cells (f-1, j, k) and (f, j, k), f = 0..nx;
  y-faces: nx * (ny+1) * nz, face (i, f, k) between cells (i, f-1, k) and (i, f, k);
  z-faces: nx * ny * (nz+1), face (i, j, f) between cells (i, j, f-1) and (i, j, f).
Cells are the interior points 0..n-1 of each axis; index -1 and n are the ghost layer, where the
eigenvector is zero (Dirichlet), so the first and last face of every line are boundary faces.
"""
import numpy as np


def face_counts(dims):
    nx, ny, nz = dims
    return (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1)


def num_faces(dims):
    return sum(face_counts(dims))


def split_faces(kappa, dims):
    """Views (kx, ky, kz) shaped (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx)."""
    nx, ny, nz = dims
    cx, cy, cz = face_counts(dims)
    kappa = np.asarray(kappa)
    return (kappa[:cx].reshape(nz, ny, nx + 1), kappa[cx:cx + cy].reshape(nz, ny + 1, nx),
            kappa[cx + cy:cx + cy + cz].reshape(nz + 1, ny, nx))


def gaussian_log_field(dims, seed, length=8.0, std=1.0):
    """log kappa on the node lattice with its ghost layer, shape (nz+2, ny+2, nx+2): seeded white
    noise convolved separably with a Gaussian of standard deviation length / sqrt(2) (so that the
    covariance is exp(-r^2 / (2 length^2)), squared-exponential), then shifted to mean 0 and
    scaled to the given standard deviation."""
    nx, ny, nz = dims
    g = np.random.default_rng(seed)
    w = g.standard_normal((nz + 2, ny + 2, nx + 2))
    s = length / np.sqrt(2.0)
    r = int(np.ceil(4 * s))
    t = np.arange(-r, r + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (t / s) ** 2)
    ker /= ker.sum()
    for axis in range(3):     # zero-padded convolution, output aligned with the input
        w = np.apply_along_axis(lambda v: np.convolve(v, ker, mode="full")[r:r + v.size], axis, w)
    w -= w.mean()
    w *= std / w.std()
    return w


def faces_from_nodes(node, dims):
    """Face coefficients kappa_f = (kappa_p + kappa_q) / 2 from node values on the lattice with its
    ghost layer (shape (nz+2, ny+2, nx+2)), in the layout above."""
    nx, ny, nz = dims
    c = node
    kx = 0.5 * (c[1:nz + 1, 1:ny + 1, 0:nx + 1] + c[1:nz + 1, 1:ny + 1, 1:nx + 2])
    ky = 0.5 * (c[1:nz + 1, 0:ny + 1, 1:nx + 1] + c[1:nz + 1, 1:ny + 2, 1:nx + 1])
    kz = 0.5 * (c[0:nz + 1, 1:ny + 1, 1:nx + 1] + c[1:nz + 2, 1:ny + 1, 1:nx + 1])
    return np.concatenate([kx.ravel(), ky.ravel(), kz.ravel()])


def random_kappa(dims, seed, length=8.0, std=1.0):
    """Face coefficients of kappa = exp(log field) for the box `dims` (float64, layout above)."""
    return faces_from_nodes(np.exp(gaussian_log_field(dims, seed, length, std)), dims)
