"""Per-kernel parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances follow from the float64 arithmetic: the two sides sum in different orders, so an
entry built from k products differs by at most about k * eps times the sum of the magnitudes
of its terms.  Integer work (the SplitMix64 block) must match bit for bit.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dense, laplace, lobpcg as olob, multigrid, rng  # noqa: E402
from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import dev, empty, host, ptr  # noqa: E402

EPS = np.finfo(np.float64).eps


def make(dims, scale=1.0, levels=None, precond="gmg"):
    return Solver(dims, scale=scale, levels=levels, precond=precond)


@pytest.mark.parametrize("dims,m,seed", [((7, 9, 5), 3, 2), ((48, 48, 48), 8, 2),
                                         ((5, 4, 3), 2, 2 ** 64 - 1), ((33, 1, 2), 5, 12345)])
def test_random_block_bit_exact(dims, m, seed):
    s = make(dims, precond="none")
    n = s.n
    ld = n + 3
    T = empty(m, ld)
    assert capi.lobpcg_op_random_block(s.h, seed, m, ptr(T), ld) == capi.OK
    got = host(T, n)
    want = rng.uniform_block(seed, n, m)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("dims,m", [((5, 7, 9), 3), ((33, 33, 33), 4), ((1, 1, 7), 2), ((17, 3, 70), 5),
                                    ((128, 128, 128), 16)])
def test_stencil_matches_oracle(dims, m):
    s = make(dims, scale=3.25, precond="none")
    n = s.n
    X = np.random.default_rng(1).uniform(-1, 1, (n, m))
    ld = n + 7
    Xd, Yd = dev(X, ld), empty(m, ld)
    assert capi.lobpcg_op_stencil(s.h, m, ptr(Xd), ld, ptr(Yd), ld) == capi.OK
    got = host(Yd, n)
    want = laplace.apply(X, dims, 3.25)
    bound = 16 * EPS * 3.25 * 12 * np.max(np.abs(X))
    assert np.max(np.abs(got - want)) <= bound
    assert torch.isnan(Yd[:, n:]).all()          # padding rows untouched


@pytest.mark.parametrize("dims,m", [((24, 13, 11), 3), ((8, 8, 70), 2), ((36, 17, 65), 5), ((4, 1, 1), 1),
                                    ((33, 33, 33), 4), ((128, 128, 128), 16)])
@pytest.mark.parametrize("ld_kind", ["vec", "odd"])
def test_stencil_f32_matches_oracle(dims, m, ld_kind):
    """The mixed form's float32 SpMV against the float64 operator on the same float32 inputs.
    With nx divisible by 4 and a leading dimension divisible by 4 the float4-row kernel runs
    (ragged runs of 2 or 4 planes, odd ny / nz here); an odd leading dimension takes the scalar
    kernel.  Bound: a few float32 roundings of the six neighbour differences, their sum and the
    scaling, 16 eps32 * s * 12 * max|x|."""
    s = Solver(dims, scale=3.25, precond="none", precision="mixed")
    n = s.n
    ld = (n + 3) // 4 * 4 + 4 if ld_kind == "vec" else n + 7
    X = np.random.default_rng(3).uniform(-1, 1, (n, m)).astype(np.float32)
    Xd = torch.full((m, ld), float("nan"), dtype=torch.float32, device="cuda")
    Xd[:, :n] = torch.tensor(np.ascontiguousarray(X.T), device="cuda")
    Yd = torch.full((m, ld), float("nan"), dtype=torch.float32, device="cuda")
    assert capi.lobpcg_op_stencil_f32(s.h, m, ptr(Xd), ld, ptr(Yd), ld) == capi.OK
    got = Yd[:, :n].cpu().numpy().T.astype(np.float64)
    want = laplace.apply(X.astype(np.float64), dims, 3.25)
    bound = 16 * np.finfo(np.float32).eps * 3.25 * 12 * np.max(np.abs(X))
    assert np.max(np.abs(got - want)) <= bound
    assert torch.isnan(Yd[:, n:]).all()          # padding rows untouched
    s.close()


def test_stencil_f32_needs_mixed_handle():
    s = make((8, 8, 8), scale=1.0, precond="none")
    X = torch.zeros((1, 512), dtype=torch.float32, device="cuda")
    assert capi.lobpcg_op_stencil_f32(s.h, 1, ptr(X), 512, ptr(X), 512) == capi.ERR_ARG


@pytest.mark.parametrize("dims,levels,m", [((7, 7, 7), 1, 3), ((8, 8, 8), 2, 2), ((16, 16, 16), 3, 4),
                                           ((15, 17, 13), 3, 3), ((48, 48, 48), 4, 8),
                                           ((128, 128, 128), 6, 16)])
def test_vcycle_matches_oracle(dims, levels, m):
    scale = laplace.default_scale(dims)
    s = make(dims, scale=scale, levels=levels)
    n = s.n
    R = np.random.default_rng(2).standard_normal((n, m))
    Rd, Ed = dev(R), empty(m, n)
    assert capi.lobpcg_op_precond(s.h, m, ptr(Rd), n, ptr(Ed), n) == capi.OK
    got = host(Ed, n)
    want = multigrid.VCycle(dims, scale, levels)(R)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("dims,levels,m", [((9, 7, 6), 2, 2), ((15, 17, 13), 3, 3), ((40, 36, 34), 3, 4),
                                           ((44, 27, 21), 3, 3), ((72, 34, 66), 4, 4), ((128, 128, 128), 6, 16)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_mixed_vcycle_matches_oracle(dims, levels, m):
    """The mixed form's V-cycle (float32 level 0, bfloat16 coarse levels) against the float64
    oracle V-cycle: the bfloat16 storage of the coarse
    corrections (8 significant bits) bounds the difference, about 2^-9 of the coarse part; an
    indexing error in any level would show as O(1)."""
    scale = laplace.default_scale(dims)
    s = Solver(dims, scale=scale, levels=levels, precision="mixed")
    n = s.n
    g = np.random.default_rng(2)
    for kind in ("random", "smooth"):
        if kind == "random":
            R = g.standard_normal((n, m))
        else:   # smooth right-hand sides: the coarse correction carries most of T R
            R = np.stack([laplace.exact_eigenvector(dims, (1 + j % 2, 1 + j % 3, 1)) for j in range(m)], axis=1)
            R += 0.01 * g.standard_normal((n, m))
        R32 = R.astype(np.float32)
        Rd = torch.tensor(np.ascontiguousarray(R32.T), device="cuda")
        Ed = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        assert capi.lobpcg_op_precond_f32(s.h, m, ptr(Rd), n, ptr(Ed), n) == capi.OK
        got = Ed.cpu().numpy().T.astype(np.float64)
        want = multigrid.VCycle(dims, scale, levels)(R32.astype(np.float64))
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert rel <= 1e-2, (kind, rel)
        assert np.max(np.abs(got - want)) <= 3e-2 * np.max(np.abs(want)), kind
    s.close()


def test_identity_preconditioner_copies():
    s = make((6, 5, 4), precond="none")
    R = np.random.default_rng(3).standard_normal((s.n, 3))
    Rd, Ed = dev(R), empty(3, s.n)
    assert capi.lobpcg_op_precond(s.h, 3, ptr(Rd), s.n, ptr(Ed), s.n) == capi.OK
    assert np.array_equal(host(Ed, s.n), R)


@pytest.mark.parametrize("dims,m,cols", [((9, 8, 7), 5, [0, 2, 3]), ((64, 64, 64), 16, list(range(16))),
                                         ((3, 3, 3), 4, [3])])
def test_residual_and_norms(dims, m, cols):
    s = make(dims, precond="none")
    n = s.n
    g = np.random.default_rng(4)
    X, AX = g.standard_normal((n, m)), g.standard_normal((n, m))
    lam = g.uniform(1, 50, m)
    ld = n + 1
    Xd, AXd, Wd = dev(X, ld), dev(AX, ld), empty(len(cols), ld)
    lamd = torch.from_numpy(lam).cuda()
    norms = (ctypes.c_double * len(cols))()
    c_cols = (ctypes.c_int * len(cols))(*cols)
    rc = capi.lobpcg_op_residual(s.h, len(cols), c_cols, ptr(Xd), ptr(AXd), ld, ptr(lamd), ptr(Wd), ld, norms)
    assert rc == capi.OK
    W = AX[:, cols] - X[:, cols] * lam[cols][None, :]
    assert np.max(np.abs(host(Wd, n) - W)) <= 4 * EPS * np.max(np.abs(AX) + np.abs(X) * lam.max())
    want = np.linalg.norm(W, axis=0)
    assert np.max(np.abs(np.array(norms[:]) - want) / want) <= 4 * n * EPS


@pytest.mark.parametrize("dims,widths", [((33, 33, 33), (8, 5, 5)), ((10, 9, 8), (3, 0, 0)),
                                         ((16, 16, 16), (4, 4, 0)), ((128, 128, 128), (16, 16, 16)),
                                         ((20, 20, 20), (32, 32, 32)), ((2, 3, 5), (7, 1, 2)),
                                         ((20, 19, 18), (50, 50, 50)), ((12, 12, 12), (100, 100, 100)),
                                         ((64, 64, 64), (8, 0, 0)), ((30, 30, 30), (16, 16, 12))])
def test_gram_matches_definition(dims, widths):
    s = make(dims, precond="none")
    n = s.n
    q = sum(widths)
    g = np.random.default_rng(5)
    S = g.standard_normal((n, q)) * g.uniform(0.1, 10, q)[None, :]
    AS = g.standard_normal((n, q))
    ld = n + 2
    blocks, ablocks, off = [], [], 0
    for w in widths:
        blocks.append(dev(S[:, off:off + w], ld) if w else None)
        ablocks.append(dev(AS[:, off:off + w], ld) if w else None)
        off += w
    gA = torch.empty((q, q), dtype=torch.float64, device="cuda")
    gB = torch.empty((q, q), dtype=torch.float64, device="cuda")
    rc = capi.lobpcg_op_gram(s.h, *[ptr(b) for b in blocks], *[ptr(b) for b in ablocks], ld, *widths,
                             ptr(gA), ptr(gB))
    assert rc == capi.OK
    # device matrices are column-major: element (i, j) at i + q*j -> transpose of the row-major view
    GA, GB = gA.cpu().numpy().T, gB.cpu().numpy().T
    offs = np.concatenate([[0], np.cumsum(widths)])
    Sb = [S[:, offs[i]:offs[i + 1]] for i in range(3) if widths[i]]
    ASb = [AS[:, offs[i]:offs[i + 1]] for i in range(3) if widths[i]]
    wantA = olob.upper_block_gram(Sb, ASb)      # the Gram blocks as printed: upper block triangle
    wantB = S.T @ S
    nrmS, nrmA = np.linalg.norm(S, axis=0), np.linalg.norm(AS, axis=0)
    boundA = 2 * n * EPS * (np.outer(nrmS, nrmA) + np.outer(nrmA, nrmS)) / 2
    boundB = 2 * n * EPS * np.outer(nrmS, nrmS)
    assert np.all(np.abs(GA - wantA) <= boundA)
    assert np.all(np.abs(GB - wantB) <= boundB)
    assert np.array_equal(GA, GA.T) and np.array_equal(GB, GB.T)


def test_gram_is_deterministic():
    s = make((40, 40, 40), precond="none")
    n, q = s.n, 12
    S = np.random.default_rng(6).standard_normal((n, q))
    Sd = dev(S)
    outs = []
    for _ in range(3):
        gB = torch.empty((q, q), dtype=torch.float64, device="cuda")
        assert capi.lobpcg_op_gram(s.h, ptr(Sd), None, None, None, None, None, n, q, 0, 0, None, ptr(gB)) == 0
        outs.append(gB.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("dims,b", [((20, 20, 20), 6), ((9, 9, 9), 1), ((32, 32, 32), 32), ((128, 128, 128), 16),
                                   ((24, 24, 24), 100), ((40, 40, 40), 50), ((24, 24, 24), 44), ((30, 20, 25), 41)])
def test_cholqr_matches_oracle(dims, b):
    s = make(dims, precond="none")
    n = s.n
    g = np.random.default_rng(7)
    V = g.standard_normal((n, b)) * np.logspace(-9, 6, b)[None, :]
    AV = g.standard_normal((n, b))
    Vd, AVd = dev(V), dev(AV)
    assert capi.lobpcg_op_cholqr(s.h, b, ptr(Vd), ptr(AVd), n) == capi.OK
    R = dense.scaled_cholesky(V.T @ V)
    Q = dense.apply_inverse_upper(V, R)
    AQ = dense.apply_inverse_upper(AV, R)
    got, agot = host(Vd, n), host(AVd, n)
    assert np.max(np.abs(got - Q)) <= 1e-10 * np.max(np.abs(Q))
    assert np.max(np.abs(agot - AQ)) <= 1e-10 * np.max(np.abs(AQ))
    assert np.max(np.abs(got.T @ got - np.eye(b))) < 1e-12


def test_cholqr_breakdown_leaves_block_untouched():
    s = make((10, 10, 10), precond="none")
    V = np.random.default_rng(8).standard_normal((s.n, 4))
    V[:, 2] = V[:, 0]
    Vd = dev(V)
    assert capi.lobpcg_op_cholqr(s.h, 4, ptr(Vd), None, s.n) == capi.ERR_BREAKDOWN
    assert np.array_equal(host(Vd, s.n), V)


def _sym_pair(q, seed, cluster=False):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((q, q)))
    ev = np.sort(g.uniform(1, 100, q))
    if cluster:
        ev[2:5] = ev[2]
        ev[7:9] = ev[7] * (1 + 1e-13)
    A = (Q * ev) @ Q.T
    Q2, _ = np.linalg.qr(g.standard_normal((q, q)))
    B = (Q2 * g.uniform(0.5, 2.0, q)) @ Q2.T
    return 0.5 * (A + A.T), 0.5 * (B + B.T)


@pytest.mark.parametrize("q,m,cluster", [(24, 8, False), (48, 16, False), (96, 32, False), (48, 16, True),
                                         (5, 5, False), (1, 1, False), (120, 40, False), (150, 50, True),
                                         (240, 80, False), (300, 100, True)])
def test_rayleigh_ritz_matches_oracle(q, m, cluster):
    s = make((4, 4, 4), precond="none")
    A, B = _sym_pair(q, q + m, cluster)
    Ad = torch.from_numpy(A.T.copy()).cuda()
    Bd = torch.from_numpy(B.T.copy()).cuda()
    lamd = torch.empty(m, dtype=torch.float64, device="cuda")
    Cd = torch.empty((m, q), dtype=torch.float64, device="cuda")
    assert capi.lobpcg_op_rayleigh_ritz(s.h, q, m, ptr(Ad), ptr(Bd), ptr(lamd), ptr(Cd)) == capi.OK
    lam, C = lamd.cpu().numpy(), Cd.cpu().numpy().T
    wl, wC = dense.rayleigh_ritz(A, B, m)
    scale = np.max(np.abs(wl))
    assert np.max(np.abs(lam - wl)) <= 1e-12 * scale
    assert np.max(np.abs(C.T @ B @ C - np.eye(m))) <= 1e-12
    assert np.max(np.abs(A @ C - B @ C * lam[None, :])) <= 1e-11 * scale
    if not cluster:   # distinct eigenvalues: vectors agree up to sign
        for j in range(m):
            assert abs(abs(C[:, j] @ B @ wC[:, j]) - 1.0) < 1e-10


def test_rayleigh_ritz_breakdown_on_indefinite_gramB():
    s = make((4, 4, 4), precond="none")
    A, B = _sym_pair(12, 3)
    B[0, 0] = -1.0
    Ad, Bd = torch.from_numpy(A.T.copy()).cuda(), torch.from_numpy(B.T.copy()).cuda()
    lamd = torch.empty(4, dtype=torch.float64, device="cuda")
    Cd = torch.empty((4, 12), dtype=torch.float64, device="cuda")
    assert capi.lobpcg_op_rayleigh_ritz(s.h, 12, 4, ptr(Ad), ptr(Bd), ptr(lamd), ptr(Cd)) == capi.ERR_BREAKDOWN


def _gram_b(s, S, engine):
    capi.lobpcg_set_gram_engine(s.h, {"auto": capi.ENGINE_AUTO, "simt": capi.ENGINE_SIMT}[engine])
    n, q = S.shape
    Sd = dev(S)
    gB = torch.empty((q, q), dtype=torch.float64, device="cuda")
    assert capi.lobpcg_op_gram(s.h, ptr(Sd), None, None, None, None, None, n, q, 0, 0, None, ptr(gB)) == capi.OK
    return gB.cpu().numpy().T


def test_gram_tensor_digits_are_summed_exactly():
    """Every digit of 1 - 2^-56 is 127, so a window of 1024 equal points drives every digit-pair
    sum of the tensor-core Gram to 1024 * 127^2 = 16,516,096, just below 2^24; with the signs
    alternating the partial sums swing over the whole range.  The float32 accumulators must keep
    every unit: the entries must equal the float64 sums to rounding (a lost unit would show at
    about 1e-7 relative).  64 x 64 x 40 points give every thread block at least one full
    window."""
    s = make((64, 64, 40), precond="none")
    n = s.n
    v = 1.0 - 2.0 ** -56
    S = np.empty((n, 4))
    S[:, 0] = v
    S[:, 1] = v * np.where(np.arange(n) % 2, -1.0, 1.0)
    S[:, 2] = v * np.where(np.arange(n) < n // 2, 1.0, -1.0)
    S[:, 3] = np.random.default_rng(3).uniform(-1.0, 1.0, n)
    G = _gram_b(s, S, "auto")
    want = S.T @ S
    assert np.max(np.abs(G - want)) <= 1e-14 * n


@pytest.mark.parametrize("dims,q", [((48, 48, 48), 8), ((64, 64, 64), 24), ((40, 36, 34), 48), ((7, 5, 3), 3)])
def test_gram_engines_agree_on_grid_functions(dims, q):
    """Tensor-core digit products against the float64 FMA pipe on smooth grid functions (sine
    modes plus noise, the kind of basis LOBPCG builds): both within float64 rounding of the
    definition, to 1e-14 relative to |s_i| |s_j|."""
    s = make(dims, precond="none")
    n = s.n
    g = np.random.default_rng(4)
    nx, ny, nz = dims
    ii, jj, kk = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1), indexing="ij")
    cols = []
    for c in range(q):
        a, b, d = 1 + c % 3, 1 + (c // 3) % 3, 1 + c // 9
        f = np.sin(a * np.pi * ii / (nx + 1)) * np.sin(b * np.pi * jj / (ny + 1)) * np.sin(d * np.pi * kk / (nz + 1))
        cols.append(f.transpose(2, 1, 0).ravel() * 10.0 ** g.uniform(-3, 3) + 1e-3 * g.standard_normal(n))
    S = np.stack(cols, axis=1)
    nrm = np.linalg.norm(S, axis=0)
    want = S.T @ S
    for engine in ("auto", "simt"):
        G = _gram_b(s, S, engine)
        assert np.all(np.abs(G - want) <= 1e-13 * np.outer(nrm, nrm)), engine
