"""Variable-coefficient operator -div(kappa grad u) and its eigenvalue gradient on the GPU.

Parity with the oracle (oracle/varcoef.py): the operator, the V-cycle, a full solve, and the
gradient formula; then the gradient against finite differences of the GPU eigensolver itself: a
central difference along a dense random direction over all faces at the 96 x 80 x 64 box with a
Gaussian log-kappa field (length 8 cells, standard deviation 1), and per-face differences on a
small box.
"""
import os
import sys

import numpy as np
import pytest
import scipy.linalg
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import lobpcg as olob, rng, varcoef  # noqa: E402
from paper_0705_2626_gb300 import capi, fields  # noqa: E402
from paper_0705_2626_gb300.autograd import eigenvalues  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import dev, empty, host, ptr  # noqa: E402

pytestmark = pytest.mark.gpu

BOX5 = (96, 80, 64)


def angle(A, B):
    return float(np.max(scipy.linalg.subspace_angles(A, B)))


@pytest.mark.parametrize("dims,length", [((5, 6, 7), 2.0), ((16, 14, 12), 4.0), (BOX5, 8.0)])
def test_varcoef_spmv_matches_oracle(dims, length):
    kappa = fields.random_kappa(dims, seed=1, length=length)
    s = Solver(dims, kappa=kappa, precond="none")
    n, m = s.n, 3
    X = np.random.default_rng(2).standard_normal((n, m))
    Y = empty(m, n)
    assert capi.lobpcg_op_stencil(s.h, m, ptr(dev(X)), n, ptr(Y), n) == capi.OK
    want = varcoef.apply(X, dims, kappa)
    assert np.max(np.abs(host(Y, n) - want)) <= 1e-14 * np.max(np.abs(want))
    s.close()


def test_varcoef_vcycle_matches_oracle():
    dims, levels, m = (16, 14, 12), 3, 3
    kappa = fields.random_kappa(dims, seed=4, length=4.0)
    s = Solver(dims, kappa=kappa, levels=levels)
    n = s.n
    R = np.random.default_rng(5).standard_normal((n, m))
    E = empty(m, n)
    assert capi.lobpcg_op_precond(s.h, m, ptr(dev(R)), n, ptr(E), n) == capi.OK
    want = varcoef.VCycleVar(dims, kappa, levels)(R)
    assert np.max(np.abs(host(E, n) - want)) <= 1e-12 * np.max(np.abs(want))
    s.close()


def test_varcoef_solve_and_gradient_match_oracle():
    dims, m, levels, tol = (24, 20, 16), 6, 3, 1e-11
    kappa = fields.random_kappa(dims, seed=6, length=8.0)
    s = Solver(dims, kappa=kappa, levels=levels)
    out = s.solve(m, tol=tol, maxit=400, seed=2)
    A = varcoef.VarCoef7(dims, kappa)
    ref = olob.lobpcg(A, rng.uniform_block(2, A.n, m), tol, 400, T=varcoef.VCycleVar(dims, kappa, levels))
    lam = np.array(out["lam"])
    assert out["status_name"] == "ok" and ref.status == "converged"
    assert np.max(np.abs(lam - ref.lam) / ref.lam) < 1e-10
    assert abs(out["iters"] - ref.iters) <= max(1, round(0.1 * ref.iters))
    X = out["X"].cpu().numpy().T
    gaps = np.diff(ref.lam) / ref.lam[1:]
    assert np.all(gaps > 1e-3)                          # simple eigenvalues for this field
    # eigenvector angles: a unit vector with residual r_j is within r_j / gap_j of the exact
    # eigenvector (gap_j to the nearest other eigenvalue; the last column's gap to lambda_{m+1}
    # is unknown and it is left out).  The residuals are the final ones recomputed from A X by
    # both solvers (soft-locked columns can end above tol, Section 2.3 / R13).
    angles = []
    for j in range(m - 1):
        gap = min(abs(ref.lam[j] - ref.lam[k]) for k in range(m) if k != j)
        a = angle(X[:, j:j + 1], ref.X[:, j:j + 1])
        assert a <= 1.5 * (out["resid"][j] + ref.resid[j]) / gap + 1e-13, (j, a)
        angles.append(a)
    # the gradient kernel against the formula on the same (GPU) eigenvectors: rounding only
    for w in [np.eye(m)[0], np.eye(m)[m - 1], np.ones(m)]:
        g = s.eig_grad(w).cpu().numpy()
        want = varcoef.grad(X, dims, w)
        assert np.max(np.abs(g - want)) <= 1e-13 * np.max(np.abs(want))
    # and against the oracle's eigenvectors, within what the angles allow: with dx = x - x_ref,
    # |(x_q - x_p)^2 - (x_ref,q - x_ref,p)^2| <= 2 |x_ref,q - x_ref,p| |dx_q - dx_p| + |dx_q - dx_p|^2
    for j in range(m - 1):
        g = s.eig_grad(np.eye(m)[j]).cpu().numpy()
        want = varcoef.grad(ref.X, dims, np.eye(m)[j])
        dmax = 2 * 2 * np.sin(angles[j] / 2) * 1.0001   # |dx_q - dx_p| <= 2 ||dx||_2, unit vectors, signs aligned
        bound = 2 * np.sqrt(np.max(want)) * dmax + dmax ** 2 + 1e-13 * np.max(want)
        assert np.max(np.abs(g - want)) <= bound
    s.close()


def test_gradient_directional_fd_box5():
    """Central difference (the initial blocke-6) along a dense random direction over all 1,493,504 faces."""
    dims, m = BOX5, 6
    kappa = fields.random_kappa(dims, seed=3, length=8.0, std=1.0)
    assert kappa.size == 1493504
    u = np.random.default_rng(9).uniform(0.0, 1.0, kappa.size)
    d = kappa * (0.5 + u)                                 # positive-biased dense direction
    eps, tol = 1e-6, 1e-10

    def lam_of(k):
        s = Solver(dims, kappa=k)
        out = s.solve(m, tol=tol, maxit=400, seed=2, with_vectors=False)
        assert out["status_name"] == "ok"
        return s, np.array(out["lam"])

    s0, lam0 = lam_of(kappa)
    G = np.stack([s0.eig_grad(np.eye(m)[j]).cpu().numpy() for j in range(m)])
    s0.close()
    sp, lp = lam_of(kappa + eps * d)
    sp.close()
    sm, lm = lam_of(kappa - eps * d)
    sm.close()
    fd = (lp - lm) / (2 * eps)
    an = G @ d
    gaps = np.diff(lam0) / lam0[1:]
    simple = np.concatenate([[gaps[0] > 1e-3], (gaps[:-1] > 1e-3) & (gaps[1:] > 1e-3), [gaps[-1] > 1e-3]])
    assert simple.sum() >= 3
    assert np.max(np.abs(fd - an)[simple] / np.abs(an[simple])) < 1e-6
    # the sum over all m (trace) is basis-invariant even where eigenvalues are close
    assert abs(fd.sum() - an.sum()) / abs(an.sum()) < 1e-6


def test_gradient_per_face_fd_small_box():
    """Per-face central differences of the GPU eigensolver on a small box.  Bound: the derivative
    of one face is about lambda / #faces, and eigenvalues carry about 1e-14 lambda of solver
    noise, so the difference quotient is good to ~1e-14 lambda / eps relative to that."""
    dims, m, eps = (8, 7, 6), 2, 1e-5
    kappa = fields.random_kappa(dims, seed=12, length=3.0)
    s = Solver(dims, kappa=kappa)
    out = s.solve(m, tol=1e-13, maxit=500, seed=2, with_vectors=False)
    g = s.eig_grad([1.0, 0.0]).cpu().numpy()
    s.close()
    lam0 = out["lam"][0]
    faces = np.random.default_rng(13).choice(kappa.size, 8, replace=False)
    for f in faces:
        vals = []
        for sign in (+1, -1):
            k = kappa.copy()
            k[f] += sign * eps
            sf = Solver(dims, kappa=k)
            vals.append(sf.solve(m, tol=1e-13, maxit=500, seed=2, with_vectors=False)["lam"][0])
            sf.close()
        fd = (vals[0] - vals[1]) / (2 * eps)
        bound = 1e-6 * abs(g[f]) + 4e-14 * lam0 / eps
        assert abs(fd - g[f]) <= bound, (f, fd, g[f], bound)


def test_autograd_backward_equals_library_gradient():
    dims, m = (16, 14, 12), 4
    kappa = torch.tensor(fields.random_kappa(dims, seed=21, length=4.0), device="cuda", requires_grad=True)
    lam = eigenvalues(kappa, dims, m, tol=1e-11)
    w = torch.tensor([1.0, 0.5, 0.25, 2.0], dtype=torch.float64, device="cuda")
    (lam * w).sum().backward()
    s = Solver(dims, kappa=kappa.detach())
    out = s.solve(m, tol=1e-11, maxit=400, seed=2, with_vectors=False)
    g = s.eig_grad(w.cpu().tolist())
    s.close()
    assert np.allclose(np.array(out["lam"]), lam.detach().cpu().numpy(), rtol=1e-13, atol=0)
    assert torch.allclose(kappa.grad, g, rtol=1e-9, atol=1e-9 * float(g.abs().max()))


def test_varcoef_argument_errors():
    import ctypes
    dims = (6, 5, 4)
    kappa = fields.random_kappa(dims, seed=1, length=2.0)
    with pytest.raises(Exception):
        Solver(dims, kappa=kappa, precision="mixed")
    s = Solver(dims, kappa=kappa)
    g = torch.empty(kappa.size, dtype=torch.float64, device="cuda")
    w = (ctypes.c_double * 1)(1.0)
    assert capi.lobpcg_eig_grad_kappa(s.h, w, ptr(g)) == capi.ERR_STATE    # nothing solved yet
    s.close()
    c = Solver(dims)                                                         # constant operator
    c.solve(1, tol=1e-8, with_vectors=False)
    assert capi.lobpcg_eig_grad_kappa(c.h, w, ptr(g)) == capi.ERR_STATE
    c.close()
