"""The tensor-core float64 kernels against the exact-integer numpy model of their digit scheme
(`tests/test_digit_product_model.py`), through the C ABI.

The update kernel's arithmetic is exact up to its one conversion per output (digit products,
level sums in float32 below 2^22, the level assembly in 64-bit integers), so its outputs must
equal the model's bit for bit.  The Gram kernel sums the float64 parts of its exponent windows
in its own order and mirrors one triangle, so it must agree with the model to within those
additions and the model's truncation of the other triangle: far tighter than the 2 n eps bar of
the float64 Gram tests, tight enough that a wrong digit, frame or shift would show.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import dev, host, ptr  # noqa: E402
from tests.test_digit_product_model import WIN_PTS, gram_model, grid_columns, model_product  # noqa: E402


def basis(n, q, seed, spread):
    g = np.random.default_rng(seed)
    S = g.standard_normal((n, q)) * 10.0 ** g.uniform(-spread, spread, q)[None, :]
    S[::97] = 0.0
    S[5::101, q // 2] = 0.0
    return S


@pytest.mark.parametrize("dims,widths,m", [((40, 36, 34), (8, 8, 8), 8), ((33, 33, 33), (8, 6, 6), 10),
                                           ((20, 20, 20), (5, 2, 0), 4)])
def test_update_equals_the_digit_model_bit_for_bit(dims, widths, m):
    s = Solver(dims, precond="none")
    assert capi.lobpcg_set_gram_engine(s.h, capi.ENGINE_AUTO) == capi.OK
    n, q = s.n, sum(widths)
    ld = (n + 31) // 32 * 32
    S = basis(n, q, 21 + q, 3.0)
    C = np.random.default_rng(22).standard_normal((q, m)) * 10.0 ** np.random.default_rng(23).uniform(-2, 2, m)
    blocks, off = [], 0
    for w in widths:
        blocks.append(dev(S[:, off:off + w], ld) if w else None)
        off += w
    Cd = torch.from_numpy(np.asfortranarray(C).ravel(order="F").copy()).cuda()
    with_p = widths[1] + widths[2] > 0
    Xd = torch.full((m, ld), float("nan"), dtype=torch.float64, device="cuda")
    Pd = torch.full((m, ld), float("nan"), dtype=torch.float64, device="cuda") if with_p else None
    rc = capi.lobpcg_op_update(s.h, *[ptr(b) for b in blocks], ld, *widths, m, ptr(Cd), ptr(Xd), ptr(Pd))
    assert rc == capi.OK
    X = host(Xd, n)
    wantX, _ = model_product(S, C)
    assert np.array_equal(X, wantX), float(np.max(np.abs(X - wantX)))
    if with_p:
        CP = C.copy()
        CP[:widths[0]] = 0.0
        wantP, _ = model_product(S, CP)
        assert np.array_equal(host(Pd, n), wantP)
    s.close()


@pytest.mark.parametrize("kind", ["grid", "random"])
def test_gram_agrees_with_the_digit_model(kind):
    dims, widths = (40, 36, 34), (8, 8, 8)
    s = Solver(dims, precond="none")
    assert capi.lobpcg_set_gram_engine(s.h, capi.ENGINE_AUTO) == capi.OK
    n, q = s.n, sum(widths)
    if kind == "grid":
        X = grid_columns(*dims, 2 * q, 24)
    else:
        g = np.random.default_rng(25)
        X = g.standard_normal((n, 2 * q)) * 10.0 ** g.uniform(-4, 4, 2 * q)[None, :]
        X[::97] = 0.0
    S, AS = X[:, :q], X[:, q:]
    ld = n + 2
    blocks, ablocks, off = [], [], 0
    for w in widths:
        blocks.append(dev(S[:, off:off + w], ld))
        ablocks.append(dev(AS[:, off:off + w], ld))
        off += w
    gA = torch.empty((q, q), dtype=torch.float64, device="cuda")
    gB = torch.empty((q, q), dtype=torch.float64, device="cuda")
    rc = capi.lobpcg_op_gram(s.h, *[ptr(b) for b in blocks], *[ptr(b) for b in ablocks], ld, *widths,
                             ptr(gA), ptr(gB))
    assert rc == capi.OK
    GA, GB = gA.cpu().numpy().T, gB.cpu().numpy().T
    MB, partsB = gram_model(S, S)
    MA, partsA = gram_model(S, AS)

    def tol(parts):
        # reassociation of the float64 parts, plus the other triangle's truncation (16 units of
        # 2^(E_i + E_j - 52) per window in each of the two orders)
        t = 0.0
        for part, ei, ej, Le, _ in parts:
            nw = -(-Le.shape[0] // WIN_PTS)
            t = t + 4 * 2.0 ** -53 * np.abs(part) + \
                32 * nw * np.ldexp(1.0, (ei[:, None] + ej[None, :] - 2096).astype(int))
        return t

    tB = tol(partsB)
    assert np.all(np.abs(GB - MB) <= tB), float(np.max(np.abs(GB - MB) / tB))
    offs = np.concatenate([[0], np.cumsum(widths)])
    tA = tol(partsA)
    for I in range(3):
        for J in range(I + 1, 3):                      # the blocks S_I^T AS_J as printed (I < J)
            sl = (slice(offs[I], offs[I + 1]), slice(offs[J], offs[J + 1]))
            assert np.all(np.abs(GA[sl] - MA[sl]) <= tA[sl]), float(np.max(np.abs(GA[sl] - MA[sl]) / tA[sl]))
    s.close()
