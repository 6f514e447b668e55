"""Eigenvalues of the variable-coefficient operator as a differentiable torch function.

``eigenvalues(kappa, dims, m)`` solves A(kappa) x = lambda x for the m smallest eigenpairs with the
CUDA LOBPCG (float64) and returns lambda as a tensor; its backward pass returns
d(sum_j g_j lambda_j)/d kappa = sum_j g_j (x_j,p - x_j,q)^2 per face from the eigenvectors of the
finished solve, which the solver handle keeps (the eigenvectors are checkpointed once; no
iteration history is stored).  The formula is the first-order perturbation of a simple
eigenvalue; for a cluster of equal eigenvalues only gradients that weight the cluster's members
equally (its trace) are independent of the basis chosen inside it.
"""
import torch

from .solver import Solver


class _Eigenvalues(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, dims, m, tol, maxit, seed, levels):
        s = Solver(dims, kappa=kappa.detach(), levels=levels, device=kappa.device.index or 0)
        out = s.solve(m, tol=tol, maxit=maxit, seed=seed, with_vectors=False)
        if out["status_name"] != "ok":
            raise RuntimeError(f"eigensolve did not converge: {out['status_name']}")
        ctx.solver = s
        return torch.tensor(out["lam"], dtype=torch.float64, device=kappa.device)

    @staticmethod
    def backward(ctx, grad_lam):
        g = ctx.solver.eig_grad(grad_lam.detach().double().cpu().tolist())
        return g.to(grad_lam.device), None, None, None, None, None, None


def eigenvalues(kappa, dims, m, tol=1e-10, maxit=400, seed=2, levels=None):
    """The m smallest eigenvalues of -div(kappa grad u) on the box `dims` (unit spacing,
    Dirichlet), differentiable with respect to the face coefficients `kappa` (float64 tensor on a
    CUDA device, layout of paper_0705_2626_gb300.fields)."""
    return _Eigenvalues.apply(kappa, tuple(int(d) for d in dims), int(m), float(tol), int(maxit), int(seed),
                              levels)
