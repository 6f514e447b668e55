"""Float64 Ritz update (Section 2.2) through the C ABI, against its definition
X = [S0 S1 S2] C and P = [S1 S2] C(w0:, :).

With the default engine, bases of at most 32 columns and at most 28 outputs run on the tensor
cores: every grid point is split into 8 signed 7-bit digits under its largest exponent over the
q columns, every coefficient column under its own, and the digit levels s + t <= 8 are summed
exactly.  Per output the error is then below (q + 4) 2^-54 max_k |S(p, k)| max_k |C(k, j)|
(the digits' rounding, the dropped levels and the 14 dropped integer bits) plus the final
rounding, 2^-53 |Y|.  The float64 FMA kernel (the SIMT engine, and wider shapes) stays within
q 2^-52 sum_k |S(p, k)| |C(k, j)|.  References are formed in long double.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import dev, host, ptr  # noqa: E402

ENGINES = {"auto": capi.ENGINE_AUTO, "simt": capi.ENGINE_SIMT}


def make(dims, engine="auto"):
    s = Solver(dims, precond="none")
    assert capi.lobpcg_set_gram_engine(s.h, ENGINES[engine]) == capi.OK
    return s


def ld_of(n):
    return (n + 31) // 32 * 32


def run_update(s, S, widths, C, with_p, ld=None):
    """Device call; returns (X, P or None) as numpy (n, m)."""
    n, q = S.shape
    m = C.shape[1]
    ld = ld_of(n) if ld is None else ld
    blocks, off = [], 0
    for w in widths:
        blocks.append(dev(S[:, off:off + w], ld) if w else None)
        off += w
    Cd = torch.from_numpy(np.asfortranarray(C).ravel(order="F").copy()).cuda()
    Xd = torch.full((m, ld), float("nan"), dtype=torch.float64, device="cuda")
    Pd = torch.full((m, ld), float("nan"), dtype=torch.float64, device="cuda") if with_p else None
    rc = capi.lobpcg_op_update(s.h, *[ptr(b) for b in blocks], ld, *widths, m, ptr(Cd), ptr(Xd), ptr(Pd))
    assert rc == capi.OK, rc
    return host(Xd, n), (host(Pd, n) if with_p else None)


def reference(S, C):
    return S.astype(np.longdouble) @ C.astype(np.longdouble)


def digit_bound(S, C, Y, rowmax):
    q = S.shape[1]
    colmax = np.max(np.abs(C), axis=0)
    return (q + 4) * 2.0 ** -54 * np.outer(rowmax, colmax) + 2.0 ** -53 * np.abs(Y)


def fma_bound(S, C):
    q = S.shape[1]
    return q * 2.0 ** -52 * (np.abs(S) @ np.abs(C))


def check(S, C, Y, w0=0):
    """Y against S(:, w0:) C(w0:, :); the digit frame of a grid point is its largest entry over
    all q columns of S, also for the P outputs (w0 > 0)."""
    Sx, Cx = S[:, w0:], C[w0:, :]
    want = reference(Sx, Cx)
    err = np.abs(Y.astype(np.longdouble) - want).astype(np.float64)
    rowmax = np.max(np.abs(S), axis=1)
    bnd = np.maximum(digit_bound(S, Cx, want.astype(np.float64), rowmax), fma_bound(Sx, Cx))
    assert np.all(err <= bnd), float(np.max(err / np.maximum(bnd, 1e-300)))


def basis(n, q, seed, spread=3.0):
    g = np.random.default_rng(seed)
    S = g.standard_normal((n, q)) * 10.0 ** g.uniform(-spread, spread, q)[None, :]
    S[::97, :] = 0.0                         # rows of zeros
    S[5::101, q // 2] = 0.0                  # single zero entries
    return S


@pytest.mark.parametrize("dims,widths,m,with_p", [
    ((40, 36, 34), (8, 8, 8), 8, True),       # the 464^3 shape (q = 24, 16 outputs), ragged tail
    ((40, 36, 34), (8, 4, 4), 8, True),       # W and P narrower than X
    ((40, 36, 34), (5, 2, 0), 4, False),      # odd q, no P block
    ((33, 33, 33), (10, 10, 10), 10, True),   # q = 30, 20 outputs: the float64 FMA kernel
    ((33, 33, 33), (8, 6, 6), 10, True),      # q = 20, 20 outputs (N = 192)
    ((20, 20, 20), (1, 0, 0), 1, False),
    ((20, 20, 20), (14, 9, 9), 14, True),     # 28 outputs, q = 32: beyond the shared memory
    ((24, 24, 24), (16, 16, 16), 16, True),   # q = 48: the float64 FMA kernel
    ((5, 4, 3), (3, 3, 3), 3, True),          # fewer points than one tile
])
@pytest.mark.parametrize("engine", ["auto", "simt"])
def test_update_matches_definition(dims, widths, m, with_p, engine):
    s = make(dims, engine)
    n, q = s.n, sum(widths)
    S = basis(n, q, 7 + q)
    C = np.random.default_rng(8).standard_normal((q, m)) * 10.0 ** np.random.default_rng(9).uniform(-2, 2, m)
    X, P = run_update(s, S, widths, C, with_p)
    check(S, C, X)
    if with_p:
        check(S, C, P, w0=widths[0])


def test_update_in_place_matches_out_of_place():
    """X over S0 and P over S2 (as the solver calls it) give the same bits as separate outputs."""
    dims, widths, m = (40, 36, 34), (8, 8, 8), 8
    s = make(dims)
    n, q = s.n, sum(widths)
    ld = ld_of(n)
    S = basis(n, q, 11, spread=1.0)
    C = np.random.default_rng(12).standard_normal((q, m))
    X, P = run_update(s, S, widths, C, True)
    blocks = [dev(S[:, 0:8], ld), dev(S[:, 8:16], ld), dev(S[:, 16:24], ld)]
    Cd = torch.from_numpy(C.ravel(order="F").copy()).cuda()
    rc = capi.lobpcg_op_update(s.h, *[ptr(b) for b in blocks], ld, *widths, m, ptr(Cd), ptr(blocks[0]),
                               ptr(blocks[2]))
    assert rc == capi.OK
    assert np.array_equal(host(blocks[0], n), X)
    assert np.array_equal(host(blocks[2], n), P)


def test_update_digit_extremes():
    """Every entry with a full 53-bit mantissa ((2 - 2^-52) 2^e, its digits near 127) and equal
    exponents along each row and column: the level sums reach their largest values (about
    8 q 127^2), and their float32 sums must stay exact.  Signs are random, rows and columns
    carry different exponents."""
    dims, widths, m = (40, 36, 34), (8, 8, 8), 8
    s = make(dims)
    n, q = s.n, sum(widths)
    g = np.random.default_rng(13)
    full = 2.0 - 2.0 ** -52
    S = full * np.ldexp(1.0, g.integers(-20, 20, n))[:, None] * g.choice([-1.0, 1.0], (n, q))
    S[::2] = np.abs(S[::2])                              # same-sign rows: the largest sums
    C = full * np.ldexp(1.0, g.integers(-5, 5, m))[None, :] * g.choice([-1.0, 1.0], (q, m))
    C[:, 0] = np.abs(C[:, 0])
    X, P = run_update(s, S, widths, C, True)
    check(S, C, X)
    check(S, C, P, w0=8)
    # same-sign rows against a same-sign column: the exact sum is q times the product
    want = np.longdouble(q) * np.abs(S[::2, 0]).astype(np.longdouble) * np.longdouble(C[0, 0])
    err = np.abs(X[::2, 0].astype(np.longdouble) - want).astype(np.float64)
    assert np.all(err <= (q + 4) * 2.0 ** -54 * np.abs(S[::2, 0]) * C[0, 0] + 2.0 ** -53 * want.astype(np.float64))


@pytest.mark.parametrize("dims,q", [((48, 48, 48), 24), ((40, 36, 34), 16)])
def test_update_engines_agree_on_grid_functions(dims, q):
    """Sine modes plus noise, each column at its own scale (the kind of basis LOBPCG builds), and
    Ritz-vector-like coefficients: both engines inside the bound, and within 1e-13 of each other
    relative to max_k |S(p, k)| max_k |C(k, j)|."""
    n = dims[0] * dims[1] * dims[2]
    nx, ny, nz = dims
    ii, jj, kk = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1), indexing="ij")
    g = np.random.default_rng(14)
    cols = []
    for c in range(q):
        a, b, d = 1 + c % 3, 1 + (c // 3) % 3, 1 + c // 9
        f = np.sin(a * np.pi * ii / (nx + 1)) * np.sin(b * np.pi * jj / (ny + 1)) * np.sin(d * np.pi * kk / (nz + 1))
        cols.append(f.transpose(2, 1, 0).ravel() * 10.0 ** g.uniform(-2, 2) + 1e-4 * g.standard_normal(n))
    S = np.stack(cols, axis=1)
    m = q // 3
    C = np.linalg.qr(g.standard_normal((q, q)))[0][:, :m]
    widths = (m, m, q - 2 * m)
    outs = {}
    for engine in ("auto", "simt"):
        s = make(dims, engine)
        outs[engine] = run_update(s, S, widths, C, True)
        check(S, C, outs[engine][0])
        check(S, C, outs[engine][1], w0=m)
        s.close()
    scale = np.outer(np.max(np.abs(S), axis=1), np.max(np.abs(C), axis=0))
    assert np.all(np.abs(outs["auto"][0] - outs["simt"][0]) <= 1e-13 * scale)


def test_update_nonfinite_rows():
    """A NaN or an infinity in a row of S makes that row's outputs non-finite; rows of zeros give
    exact zeros."""
    dims, widths, m = (40, 36, 34), (8, 8, 8), 8
    s = make(dims)
    n, q = s.n, sum(widths)
    S = basis(n, q, 15, spread=1.0)
    S[10, 3] = np.nan
    S[300, 20] = np.inf
    C = np.random.default_rng(16).standard_normal((q, m))
    X, P = run_update(s, S, widths, C, True)
    assert not np.any(np.isfinite(X[10])) and not np.any(np.isfinite(X[300]))
    assert not np.any(np.isfinite(P[300]))
    ok = np.ones(n, bool)
    ok[[10, 300]] = False
    assert np.all(np.isfinite(X[ok])) and np.all(X[0] == 0.0) and np.all(X[97] == 0.0)
    check(S[ok], C, X[ok])
