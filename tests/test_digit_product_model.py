"""The error model of the float64 products by error-free digit splitting (Ozaki, Ogita and Oishi,
Numer. Algorithms 59, 2012), checked on the CPU with exact integer arithmetic.

The tensor-core Ritz update computes Y = S C (Section 2.2, the Ritz update) by writing every
entry of a row p of S in the frame of the row's largest exponent E_p as 8 signed 7-bit digits
(56 bits rounded to nearest), every column j of C likewise in its own frame F_j, keeping the digit
levels L = s + t <= 8, rounding the level sum T to 2^-56 of the frame and converting once to
float64.  The GPU tests (`test_gpu_update.py`) hold the kernel to
    |Y - S C| <= (q + 4) 2^-54 max_k |S(p, k)| max_k |C(k, j)| + 2^-53 |S C|.
This file computes the same scheme in numpy integers, independently of the CUDA sources, and
checks that the bound holds with a margin for the model itself (so the GPU tests do not pass by a
loose tolerance), that it is not vacuous (the model's error does reach a fair part of it on
full-mantissa inputs), and that every level sum stays below 2^22, which keeps the tensor cores'
float32 sums exact for q <= 32.  The second part does the same for the tensor-core float64 Gram
(windowed frames, every digit pair kept, truncated integer combination): its error stays inside
the bound derived from those steps, far inside the 2 n eps bar of the GPU Gram tests, and within
one eps of sum_p |x_i(p)| |y_j(p)| on grid functions and on random columns.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

LEVELS = 9


def exponent_field(x):
    return ((x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)


def digits(x, emax):
    """Signed 7-bit digits d_0..d_7 of x in the frame of the exponent field emax (broadcast
    against x): F = round(|x| 2^(56 - E)), E = emax - 1022, u_s = bits 49 - 7 s .. 55 - 7 s."""
    bits = x.view(np.uint64)
    e = exponent_field(x)
    sign = np.where((bits >> np.uint64(63)) != 0, -1, 1).astype(np.int64)
    mant = (bits & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    m3 = mant << np.uint64(3)
    sh = emax - e
    s = np.clip(sh, 0, 63).astype(np.uint64)
    half = (np.uint64(1) << s) >> np.uint64(1)
    F = (m3 + half) >> s
    F = np.where((e == 0) | (sh >= 60), np.uint64(0), F)
    out = np.empty(x.shape + (8,), dtype=np.int64)
    for k in range(8):
        out[..., k] = ((F >> np.uint64(49 - 7 * k)) & np.uint64(127)).astype(np.int64) * sign
    return out


def model_product(S, C):
    """Y = S C as the digit scheme forms it; also the level sums D_L (n, m, 9)."""
    es, ec = exponent_field(S), exponent_field(C)
    em = np.max(np.where(es > 0, es, -(1 << 20)), axis=1)                 # row frames
    cj = np.max(np.where(ec > 0, ec, -(1 << 20)), axis=0)                 # column frames
    dS = digits(S, em[:, None])                                           # (n, q, 8)
    dC = digits(C, cj[None, :])                                           # (q, m, 8)
    D = np.zeros((S.shape[0], C.shape[1], LEVELS), dtype=np.int64)
    for s in range(8):
        for t in range(8):
            if s + t < LEVELS:
                D[:, :, s + t] += dS[:, :, s] @ dC[:, :, t]
    a1 = D[..., 0] * 128 + D[..., 1]
    a2 = D[..., 2] * 128 + D[..., 3]
    lo14 = D[..., 5] * 128 + D[..., 6] + ((D[..., 7] * 128 + D[..., 8] + 8192) >> 14)   # to nearest
    t = a1 * (1 << 35) + a2 * (1 << 21) + D[..., 4] * (1 << 14) + lo14
    ex = em[:, None] + cj[None, :] - 2100
    Y = np.ldexp(t.astype(np.float64), ex)                                # one rounding, exact scaling
    Y[(em[:, None] < 0) | (cj[None, :] < 0)] = 0.0
    return Y, D


def bound(S, C, ref):
    q = S.shape[1]
    return (q + 4) * 2.0 ** -54 * np.outer(np.max(np.abs(S), axis=1), np.max(np.abs(C), axis=0)) + \
        2.0 ** -53 * np.abs(ref)


def reference(S, C):
    return (S.astype(np.longdouble) @ C.astype(np.longdouble))


def basis(n, q, seed, spread):
    g = np.random.default_rng(seed)
    S = g.standard_normal((n, q)) * 10.0 ** g.uniform(-spread, spread, q)[None, :]
    S[::37] = 0.0
    S[3::41, q // 2] = 0.0
    return S


@pytest.mark.parametrize("n,q,m,spread,seed", [(3000, 24, 16, 3.0, 1), (2000, 32, 28, 1.0, 2),
                                               (2000, 8, 8, 5.0, 3), (500, 1, 1, 0.0, 4)])
def test_model_within_the_kernel_bound(n, q, m, spread, seed):
    S = basis(n, q, seed, spread)
    C = np.random.default_rng(seed + 10).standard_normal((q, m)) * 10.0 ** \
        np.random.default_rng(seed + 20).uniform(-2, 2, m)
    Y, D = model_product(S, C)
    ref = reference(S, C)
    err = np.abs(Y.astype(np.longdouble) - ref).astype(np.float64)
    bnd = bound(S, C, ref.astype(np.float64))
    assert np.all(err <= 0.5 * bnd), float(np.max(err / bnd))          # margin for the model itself
    assert np.all(Y[::37] == 0.0)                                         # rows of zeros stay exact zeros
    assert np.max(np.abs(D)) < 2 ** 22


def test_full_mantissa_digits_stay_exact_and_use_the_bound():
    """Every entry (2 - 2^-52) 2^e with the exponent shared along rows and columns: F = 2^56 - 8,
    so digits 0-6 are 127 and digit 7 is 120 in magnitude; the level sums reach their largest
    values (level 7: q (6 127^2 + 2 127 120), under the 8 q 127^2 < 2^22 of any input for q = 32),
    and the dropped levels make the error a visible part of the bound."""
    g = np.random.default_rng(5)
    n, q, m = 400, 32, 28
    full = 2.0 - 2.0 ** -52
    S = full * np.ldexp(1.0, g.integers(-20, 20, n))[:, None] * np.ones((n, q))
    S[1::2] *= g.choice([-1.0, 1.0], (n // 2, q))
    C = full * np.ldexp(1.0, g.integers(-5, 5, m))[None, :] * np.ones((q, m))
    Y, D = model_product(S, C)
    assert np.max(np.abs(D)) == q * (6 * 127 ** 2 + 2 * 127 * 120) and 8 * q * 127 ** 2 < 2 ** 22
    ref = reference(S, C)
    err = np.abs(Y.astype(np.longdouble) - ref).astype(np.float64)
    bnd = bound(S, C, ref.astype(np.float64))
    assert np.all(err <= bnd)
    assert np.max(err / bnd) > 0.05                                       # the bound is not vacuous


def test_digits_reassemble_to_the_rounded_value():
    """sum_s d_s 2^(7 (7 - s)) 2^(E - 56) is x rounded to 2^(E - 56): within 2^(E - 57) of x."""
    g = np.random.default_rng(6)
    x = g.standard_normal(5000) * 10.0 ** g.uniform(-8, 8, 5000)
    x[::50] = 0.0
    emax = int(np.max(exponent_field(x)))
    d = digits(x, np.full(x.shape, emax))
    E = emax - 1022
    F = sum(d[:, s] * (1 << (7 * (7 - s))) for s in range(8))          # int64, |F| <= 2^56
    exact = np.ldexp(x.astype(np.longdouble), 56 - E)                    # x 2^(56 - E), exact
    assert np.all(np.abs(F.astype(np.longdouble) - exact) <= 0.5)
    assert np.all(np.abs(d) <= 127) and np.all(F[::50] == 0)


# ---------------------------------------------------------------- the float64 Gram (tensor cores)
# Per column and exponent window of 16384 points the frame is the column's largest exponent field
# there; per accumulation window of 1024 points every digit-pair sum D_st(i, j) is exact; line s
# of column i contributes hi 2^(17 - 7 s) + lo 2^(-11 - 7 s) (each shift a floor) with
# hi = sum_{t<4} D_st 2^(7 (3 - t)) and lo = sum_{t>=4} D_st 2^(7 (7 - t)), in units of
# 2^(E_i + E_j - 52); the windows of one exponent window are summed exactly, converted to
# float64 once and added to the entry.

EXP_PTS, WIN_PTS = 16384, 1024


def gram_model(L, R):
    n, qa = L.shape
    qb = R.shape[1]
    G = np.zeros((qa, qb))
    parts = []
    for e0 in range(0, n, EXP_PTS):
        Le, Re = L[e0:e0 + EXP_PTS], R[e0:e0 + EXP_PTS]
        ei, ej = exponent_field(Le).max(axis=0), exponent_field(Re).max(axis=0)
        dL, dR = digits(Le, ei[None, :]), digits(Re, ej[None, :])
        acc = np.zeros((qa, qb), dtype=object)
        for w0 in range(0, Le.shape[0], WIN_PTS):
            D = np.einsum("pis,pjt->isjt", dL[w0:w0 + WIN_PTS], dR[w0:w0 + WIN_PTS])    # exact int64
            assert np.max(np.abs(D)) < 2 ** 24
            c = np.zeros((qa, qb), dtype=np.int64)
            for s in range(8):
                hi = sum(D[:, s, :, t] * (1 << (7 * (3 - t))) for t in range(4))
                lo = sum(D[:, s, :, t] * (1 << (7 * (7 - t))) for t in range(4, 8))
                shl = 17 - 7 * s
                c += (hi << shl) if shl >= 0 else (hi >> -shl)
                c += lo >> (11 + 7 * s)
            acc = acc + c.astype(object)
        part = np.array([[np.ldexp(float(acc[i, j]), int(ei[i] + ej[j] - 2096)) for j in range(qb)]
                         for i in range(qa)])
        parts.append((part, ei, ej, Le, Re))
        G += part
    return G, parts


def gram_model_bound(parts):
    """Digit rounding (2^(E - 57) per element against the other column's absolute sum), the
    dropped products of two rounding errors, the truncation (at most 16 units per window), and the
    float64 conversions and additions of the exponent windows' parts."""
    tot, absparts = 0.0, 0.0
    k = len(parts)
    for part, ei, ej, Le, Re in parts:
        Ei, Ej = ei.astype(float) - 1022, ej.astype(float) - 1022
        sx, sy = np.abs(Le).sum(axis=0), np.abs(Re).sum(axis=0)
        nw = -(-Le.shape[0] // WIN_PTS)
        scale = np.ldexp(1.0, (Ei[:, None] + Ej[None, :]).astype(int))
        tot = tot + np.ldexp(1.0, (Ei - 57).astype(int))[:, None] * sy[None, :] + \
            np.ldexp(1.0, (Ej - 57).astype(int))[None, :] * sx[:, None] + \
            scale * (2.0 ** -114 * Le.shape[0] + 16 * nw * 2.0 ** -52)
        absparts = absparts + np.abs(part)
    return tot + (k + 1) * 2.0 ** -53 * absparts


def grid_columns(nx, ny, nz, q, seed):
    """Sine modes with noise, each column at its own scale: the kind of basis LOBPCG builds."""
    g = np.random.default_rng(seed)
    ii, jj, kk = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1), indexing="ij")
    cols = []
    for c in range(q):
        a, b, d = 1 + c % 3, 1 + (c // 3) % 3, 1 + c // 9
        f = np.sin(a * np.pi * ii / (nx + 1)) * np.sin(b * np.pi * jj / (ny + 1)) * np.sin(d * np.pi * kk / (nz + 1))
        cols.append(f.transpose(2, 1, 0).ravel() * 10.0 ** g.uniform(-3, 3) + 1e-5 * g.standard_normal(f.size))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("kind", ["grid", "random"])
def test_gram_model_within_its_bound_and_the_float64_test_bound(kind):
    if kind == "grid":
        X = grid_columns(40, 36, 34, 12, 7)                    # 48,960 points: 3 exponent windows, ragged
    else:
        g = np.random.default_rng(8)
        X = g.standard_normal((40000, 12)) * 10.0 ** g.uniform(-4, 4, 12)[None, :]
        X[::97] = 0.0
    L, R = X[:, :6], X
    G, parts = gram_model(L, R)
    want = L.astype(np.longdouble).T @ R.astype(np.longdouble)
    err = np.abs(G.astype(np.longdouble) - want).astype(np.float64)
    mb = gram_model_bound(parts)
    assert np.all(err <= mb), float(np.max(err / mb))
    n = X.shape[0]
    eps = np.finfo(np.float64).eps
    gpu_bound = 2 * n * eps * np.outer(np.linalg.norm(L, axis=0), np.linalg.norm(R, axis=0))
    assert np.all(mb <= 1e-3 * gpu_bound)                      # far inside the GPU test's bar
    # float64 quality: on these bases the scheme stays within one eps of sum_p |x_i| |y_j| (the
    # float64 product L^T R in numpy reaches about 2 eps on the same data)
    absdot = np.abs(L).T @ np.abs(R)
    assert np.all(err <= eps * absdot), float(np.max(err / (eps * absdot)))
