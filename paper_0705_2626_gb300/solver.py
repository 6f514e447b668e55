"""Python front end of the GB300 LOBPCG library.

``Solver`` owns one C handle (include/lobpcg_gb300.h).  PyTorch supplies the device memory
(the handle's workspace comes from torch's caching allocator through the C allocator
callback) and the CUDA stream; every step of the iteration runs in the CUDA library.
Blocks of vectors cross the boundary as torch tensors of shape (m, ld): row j of the tensor is
column j of the column-major n-by-m block.
"""
import ctypes

import torch

from . import capi


class LobpcgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{capi.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc, h=None, allow=(capi.OK,)):
    if rc not in allow:
        raise LobpcgError(rc, capi.lobpcg_last_error(h))
    return rc


class _TorchAllocator:
    """C allocator callbacks backed by torch's caching allocator on one device."""

    def __init__(self, device):
        self.device = device

        def _alloc(ctx, size, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(size), self.device, int(stream or 0))
            except Exception:  # the C side maps NULL to LOBPCG_ERR_OOM
                return None

        def _free(ctx, ptr, size, stream):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._alloc = capi.ALLOC_FN(_alloc)
        self._free = capi.FREE_FN(_free)
        self.struct = capi.Allocator(None, self._alloc, self._free)


def default_scale(dims):
    nx, ny, nz = dims
    return float(nx + 1) ** 2 if nx == ny == nz else 1.0


class Solver:
    """LOBPCG for the m smallest eigenpairs of the 7-point Dirichlet Laplacian on `dims`."""

    def __init__(self, dims, scale=None, precond="gmg", levels=None, nu=2, omega=2.0 / 3.0,
                 device=0, stream=None, tol_mode="relative", gram="explicit", phase_timing=False,
                 torch_allocator=True, precision="fp64", kappa=None, gram_engine="auto"):
        """kappa: face coefficients of the variable-coefficient operator -div(kappa grad u) (unit
        spacing; layout of paper_0705_2626_gb300.fields), a float64 numpy array or torch tensor;
        None selects the constant-coefficient Laplacian.  gram_engine: "auto" (tensor cores for wide
        stacks), "tensor" (tcgen05, 3 x TF32, whenever the blocks fit) or "simt" for the float32 Gram
        products of the mixed form."""
        if precision not in ("fp64", "mixed"):
            raise ValueError(f"precision must be 'fp64' or 'mixed', not {precision!r}")
        self.precision = precision
        self.dims = tuple(int(d) for d in dims)
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self.varcoef = kappa is not None
        self.scale = (1.0 if self.varcoef else default_scale(self.dims)) if scale is None else float(scale)
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._alloc = _TorchAllocator(device) if torch_allocator else None
        h = ctypes.c_void_p()
        _check(capi.lobpcg_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                  ctypes.byref(self._alloc.struct) if self._alloc else None,
                                  capi.MIXED if precision == "mixed" else capi.FP64))
        self.h = h
        if self.varcoef:
            kt = torch.as_tensor(kappa, dtype=torch.float64)
            kt = kt.detach().to(self.device).contiguous()
            torch.cuda.current_stream(self.device).synchronize()
            _check(capi.lobpcg_set_operator(h, capi.VARCOEF7, *self.dims, self.scale,
                                            ctypes.c_void_p(kt.data_ptr())), h)
        else:
            _check(capi.lobpcg_set_operator(h, capi.LAPLACE7, *self.dims, self.scale, None), h)
        if precond == "gmg":
            if levels is None:
                levels = 1
                d = list(self.dims)
                while min(d) // 2 >= 3 and levels < 24:
                    d = [x // 2 for x in d]
                    levels += 1
                # the variable-coefficient coarsest level is solved with a dense inverse
                while self.varcoef and d[0] * d[1] * d[2] > 512 and min(d) // 2 >= 1:
                    d = [x // 2 for x in d]
                    levels += 1
            _check(capi.lobpcg_set_preconditioner(h, capi.PRECOND_GMG, levels, nu, nu, omega), h)
        elif precond is None or precond == "none":
            _check(capi.lobpcg_set_preconditioner(h, capi.PRECOND_NONE, 1, 1, 1, 1.0), h)
        else:
            raise ValueError(f"unknown preconditioner {precond!r}")
        self.levels = levels if precond == "gmg" else 1
        _check(capi.lobpcg_set_options(h, capi.TOL_RELATIVE if tol_mode == "relative" else capi.TOL_ABSOLUTE,
                                       capi.GRAM_EXPLICIT if gram == "explicit" else capi.GRAM_PAPER,
                                       1 if phase_timing else 0), h)
        engines = {"auto": capi.ENGINE_AUTO, "simt": capi.ENGINE_SIMT, "tensor": capi.ENGINE_TENSOR}
        if gram_engine not in engines:
            raise ValueError(f"gram_engine must be one of {sorted(engines)}, not {gram_engine!r}")
        _check(capi.lobpcg_set_gram_engine(h, engines[gram_engine]), h)
        self.m = None
        self.info = capi.Info()

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            capi.lobpcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- solving
    def set_initial(self, X0):
        """X0: (m, n) float64 tensor (host or device), row j = column j of the block."""
        X0 = X0.contiguous()
        on_host = 0 if X0.is_cuda else 1
        _check(capi.lobpcg_set_initial(self.h, ctypes.c_void_p(X0.data_ptr()), X0.shape[0], X0.shape[1],
                                       on_host), self.h)

    def set_inner_pcg(self, iters):
        """The preconditioning as `iters` inner PCG iterations preconditioned by the V-cycle (0: V-cycle directly)."""
        _check(capi.lobpcg_set_inner_pcg(self.h, int(iters)), self.h)

    def set_constraints(self, Y):
        """Constraint block (hard locking, the constraint projections): Y an (l, n) float64 tensor (host or
        device), row j = column j; None or l = 0 removes the constraints."""
        if Y is None:
            _check(capi.lobpcg_set_constraints(self.h, None, 0, self.n, 0), self.h)
            return
        Y = torch.as_tensor(Y, dtype=torch.float64).contiguous()
        if Y.dim() != 2 or Y.shape[1] != self.n:
            raise ValueError(f"Y must have shape (l, {self.n})")
        on_host = 0 if Y.is_cuda else 1
        if Y.is_cuda:
            torch.cuda.current_stream(self.device).synchronize()
        _check(capi.lobpcg_set_constraints(self.h, ctypes.c_void_p(Y.data_ptr()) if Y.shape[0] else None,
                                           Y.shape[0], self.n, on_host), self.h)

    def solve(self, m, tol=1e-8, maxit=200, seed=2, with_vectors=True):
        rc = capi.lobpcg_solve(self.h, m, tol, maxit, seed, ctypes.byref(self.info))
        self.m = m
        _check(rc, self.h, allow=(capi.OK, capi.NOT_CONVERGED))
        return self.result(with_vectors)

    def begin(self, m, tol=1e-8, seed=2):
        _check(capi.lobpcg_begin(self.h, m, tol, seed), self.h)
        self.m = m

    def iterate(self, steps):
        rc = capi.lobpcg_iterate(self.h, steps, ctypes.byref(self.info))
        _check(rc, self.h, allow=(capi.OK, capi.NOT_CONVERGED))
        return rc

    def set_options(self, tol_mode="relative", gram="explicit", phase_timing=False):
        _check(capi.lobpcg_set_options(self.h, capi.TOL_RELATIVE if tol_mode == "relative" else capi.TOL_ABSOLUTE,
                                       capi.GRAM_EXPLICIT if gram == "explicit" else capi.GRAM_PAPER,
                                       1 if phase_timing else 0), self.h)

    def finish(self):
        rc = capi.lobpcg_finish(self.h, ctypes.byref(self.info))
        _check(rc, self.h, allow=(capi.OK, capi.NOT_CONVERGED))
        return rc

    def eig_grad(self, w):
        """Gradient of sum_j w[j] lambda_j with respect to the face coefficients (variable-
        coefficient operator, after a finished solve), as a float64 tensor on the device."""
        w = [float(x) for x in w]
        assert len(w) == self.m
        wa = (ctypes.c_double * self.m)(*w)
        from .fields import num_faces
        g = torch.empty(num_faces(self.dims), dtype=torch.float64, device=self.device)
        torch.cuda.current_stream(self.device).synchronize()
        _check(capi.lobpcg_eig_grad_kappa(self.h, wa, ctypes.c_void_p(g.data_ptr())), self.h)
        return g

    def result(self, with_vectors=True):
        m = self.m
        lam = (ctypes.c_double * m)()
        res = (ctypes.c_double * m)()
        X = None
        if with_vectors:
            X = torch.empty((m, self.n), dtype=torch.float64, device=self.device)
            torch.cuda.current_stream(self.device).synchronize()
            _check(capi.lobpcg_get_eigenpairs(self.h, lam, ctypes.c_void_p(X.data_ptr()), self.n, 0, res), self.h)
        else:
            _check(capi.lobpcg_get_eigenpairs(self.h, lam, None, self.n, 0, res), self.h)
        return dict(lam=list(lam), resid=list(res), X=X, iters=self.info.iters, status=self.info.status,
                    status_name=capi.STATUS_NAMES.get(self.info.status), active=self.info.active,
                    p_dropped=self.info.p_dropped, fp64_sweeps=self.info.fp64_sweeps,
                    setup_ms=self.info.setup_ms, solve_ms=self.info.solve_ms,
                    max_rel_resid=self.info.max_rel_resid, kernel_launches=self.info.kernel_launches,
                    phase_ms=dict(zip(capi.PHASE_NAMES, list(self.info.phase_ms))))
