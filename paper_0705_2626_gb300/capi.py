"""ctypes binding of liblobpcg_gb300.so -- argument marshalling only.

Every function here has the name and argument order of the C entry point declared in
include/lobpcg_gb300.h and does nothing but convert arguments; all computation runs in the
CUDA library.  Loading fails loudly (RuntimeError) when the library has not been built: there
is no fallback implementation.
"""
import ctypes
import os

from .build import LIB_PATH

c_int, c_int64, c_uint64, c_double, c_void_p, c_size_t = (
    ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)
c_dp = ctypes.POINTER(ctypes.c_double)

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_BREAKDOWN, ERR_NONFINITE, ERR_STATE, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "ok", 1: "not_converged", -1: "err_arg", -2: "err_oom", -3: "err_cuda",
                -4: "breakdown", -5: "nonfinite", -6: "err_state", -7: "err_timeout"}
FP64, MIXED = 0, 1
LAPLACE7, VARCOEF7 = 0, 1
PRECOND_NONE, PRECOND_GMG = 0, 1
TOL_RELATIVE, TOL_ABSOLUTE = 0, 1
GRAM_EXPLICIT, GRAM_PAPER = 0, 1
ENGINE_AUTO, ENGINE_SIMT, ENGINE_TENSOR = 0, 1, 2
MAX_M = 100
MAX_M_MIXED = 32
NPHASES = 8
PHASE_NAMES = ["residual", "precond", "cholqr_w", "spmv", "cholqr_p", "gram", "rayleigh_ritz", "update"]

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_size_t, c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("ctx", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("active", ctypes.c_int32),
                ("p_dropped", ctypes.c_int32), ("fp64_sweeps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_rel_resid", c_double), ("setup_ms", c_double),
                ("solve_ms", c_double), ("kernel_launches", ctypes.c_int64), ("phase_ms", c_double * NPHASES)]


_SIGNATURES = {
    "lobpcg_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_void_p, ctypes.POINTER(Allocator), c_int]),
    "lobpcg_set_operator": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_double, c_void_p]),
    "lobpcg_set_preconditioner": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_double]),
    "lobpcg_set_options": (c_int, [c_void_p, c_int, c_int, c_int]),
    "lobpcg_set_gram_engine": (c_int, [c_void_p, c_int]),
    "lobpcg_set_wait_limit": (c_int, [c_void_p, c_int]),
    "lobpcg_set_inner_pcg": (c_int, [c_void_p, c_int]),
    "lobpcg_set_initial": (c_int, [c_void_p, c_void_p, c_int, c_int64, c_int]),
    "lobpcg_set_constraints": (c_int, [c_void_p, c_void_p, c_int, c_int64, c_int]),
    "lobpcg_solve": (c_int, [c_void_p, c_int, c_double, c_int, c_uint64, ctypes.POINTER(Info)]),
    "lobpcg_begin": (c_int, [c_void_p, c_int, c_double, c_uint64]),
    "lobpcg_iterate": (c_int, [c_void_p, c_int, ctypes.POINTER(Info)]),
    "lobpcg_finish": (c_int, [c_void_p, ctypes.POINTER(Info)]),
    "lobpcg_get_eigenpairs": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_void_p]),
    "lobpcg_eig_grad_kappa": (c_int, [c_void_p, c_void_p, c_void_p]),
    "lobpcg_last_error": (ctypes.c_char_p, [c_void_p]),
    "lobpcg_destroy": (c_int, [c_void_p]),
    "lobpcg_op_random_block": (c_int, [c_void_p, c_uint64, c_int, c_void_p, c_int64]),
    "lobpcg_op_stencil": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p, c_int64]),
    "lobpcg_op_precond": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p, c_int64]),
    "lobpcg_op_precond_f32": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p, c_int64]),
    "lobpcg_op_stencil_f32": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p, c_int64]),
    "lobpcg_op_residual": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int), c_void_p, c_void_p, c_int64,
                                   c_void_p, c_void_p, c_int64, c_void_p]),
    "lobpcg_op_gram": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_int64, c_int, c_int, c_int, c_void_p, c_void_p]),
    "lobpcg_op_gram_f32": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_int64,
                                   c_void_p, c_void_p]),
    "lobpcg_op_gram_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_int64, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "lobpcg_op_cholqr": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int64]),
    "lobpcg_op_update": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int, c_int, c_int,
                                 c_void_p, c_void_p, c_void_p]),
    "lobpcg_op_rayleigh_ritz": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lobpcg_gram_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                    c_int64, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
}

_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                " (the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return sorted(_SIGNATURES)


def _call(name, *args):
    return getattr(lib(), name)(*args)


# Thin wrappers with the C names (pointer arguments are ints or ctypes objects).
def lobpcg_create(handle_out, device, stream, alloc, precision):
    return _call("lobpcg_create", handle_out, device, stream, alloc, precision)


def lobpcg_set_operator(h, kind, nx, ny, nz, scale, kappa_faces=None):
    return _call("lobpcg_set_operator", h, kind, nx, ny, nz, scale, kappa_faces)


def lobpcg_set_preconditioner(h, kind, levels, nu_pre, nu_post, omega):
    return _call("lobpcg_set_preconditioner", h, kind, levels, nu_pre, nu_post, omega)


def lobpcg_set_options(h, tol_mode, gram_mode, phase_timing):
    return _call("lobpcg_set_options", h, tol_mode, gram_mode, phase_timing)


def lobpcg_set_gram_engine(h, engine):
    return _call("lobpcg_set_gram_engine", h, engine)


def lobpcg_set_wait_limit(h, polls):
    return _call("lobpcg_set_wait_limit", h, polls)


def lobpcg_set_inner_pcg(h, iters):
    return _call("lobpcg_set_inner_pcg", h, iters)


def lobpcg_set_initial(h, X0, m, ldx, on_host):
    return _call("lobpcg_set_initial", h, X0, m, ldx, on_host)


def lobpcg_set_constraints(h, Y, l, ldy, on_host):
    return _call("lobpcg_set_constraints", h, Y, l, ldy, on_host)


def lobpcg_solve(h, m, tol, maxit, seed, info):
    return _call("lobpcg_solve", h, m, tol, maxit, seed, info)


def lobpcg_begin(h, m, tol, seed):
    return _call("lobpcg_begin", h, m, tol, seed)


def lobpcg_iterate(h, steps, info):
    return _call("lobpcg_iterate", h, steps, info)


def lobpcg_finish(h, info):
    return _call("lobpcg_finish", h, info)


def lobpcg_get_eigenpairs(h, lam, X, ldx, x_on_host, resid):
    return _call("lobpcg_get_eigenpairs", h, lam, X, ldx, x_on_host, resid)


def lobpcg_last_error(h):
    s = _call("lobpcg_last_error", h)
    return s.decode() if s else ""


def lobpcg_destroy(h):
    return _call("lobpcg_destroy", h)


def lobpcg_op_random_block(h, seed, m, X, ldx):
    return _call("lobpcg_op_random_block", h, seed, m, X, ldx)


def lobpcg_op_stencil(h, ncols, X, ldx, Y, ldy):
    return _call("lobpcg_op_stencil", h, ncols, X, ldx, Y, ldy)


def lobpcg_op_precond(h, ncols, R, ldr, E, lde):
    return _call("lobpcg_op_precond", h, ncols, R, ldr, E, lde)


def lobpcg_op_precond_f32(h, ncols, R, ldr, E, lde):
    return _call("lobpcg_op_precond_f32", h, ncols, R, ldr, E, lde)


def lobpcg_op_stencil_f32(h, ncols, X, ldx, Y, ldy):
    return _call("lobpcg_op_stencil_f32", h, ncols, X, ldx, Y, ldy)


def lobpcg_op_residual(h, ncols, cols, X, AX, ld, lam, W, ldw, norms):
    return _call("lobpcg_op_residual", h, ncols, cols, X, AX, ld, lam, W, ldw, norms)


def lobpcg_op_gram(h, S0, S1, S2, AS0, AS1, AS2, ld, w0, w1, w2, gramA, gramB):
    return _call("lobpcg_op_gram", h, S0, S1, S2, AS0, AS1, AS2, ld, w0, w1, w2, gramA, gramB)


def lobpcg_eig_grad_kappa(h, w, grad_faces):
    return _call("lobpcg_eig_grad_kappa", h, w, grad_faces)


def lobpcg_op_gram_f32(h, S0, w0, S1, w1, V, b, ld, C, G):
    return _call("lobpcg_op_gram_f32", h, S0, w0, S1, w1, V, b, ld, C, G)


def lobpcg_op_gram_residual(h, Xh, Xl, W, P, R, AW, AP, ld, m, b, bp, lam, gramA, gramB):
    return _call("lobpcg_op_gram_residual", h, Xh, Xl, W, P, R, AW, AP, ld, m, b, bp, lam, gramA, gramB)


def lobpcg_op_cholqr(h, b, V, AV, ld):
    return _call("lobpcg_op_cholqr", h, b, V, AV, ld)


def lobpcg_op_update(h, S0, S1, S2, ld, w0, w1, w2, m, C, Xout, Pout):
    return _call("lobpcg_op_update", h, S0, S1, S2, ld, w0, w1, w2, m, C, Xout, Pout)


def lobpcg_op_rayleigh_ritz(h, q, m, gramA, gramB, lam, C):
    return _call("lobpcg_op_rayleigh_ritz", h, q, m, gramA, gramB, lam, C)


def lobpcg_gram_noalloc(S0, S1, S2, AS0, AS1, AS2, n, ld, w0, w1, w2, gramA, gramB, stream):
    return _call("lobpcg_gram_noalloc", S0, S1, S2, AS0, AS1, AS2, n, ld, w0, w1, w2, gramA, gramB, stream)
