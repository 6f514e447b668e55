"""The allocation-free Gram entry point against the handle-based one.

lobpcg_gram_noalloc serves callers that may not allocate device memory (host callbacks,
applications whose pool owns all device memory, callers without a handle).  It keeps its
partial sums in one fixed device array that every call reuses, so this test makes two calls in a
row with different shapes and checks both against lobpcg_op_gram, with the tolerance of the Gram
parity test, and checks that the device's free memory is the same before and after each call
(after one first call, which loads the library's code onto the device and looks up the array's
address).  The file name sorts last so that a run stopping at its first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0705_2626_gb300 import capi  # noqa: E402
from paper_0705_2626_gb300.solver import Solver  # noqa: E402
from tests.gpu_util import dev, ptr  # noqa: E402

EPS = np.finfo(np.float64).eps


def _blocks(S, AS, widths, ld):
    blocks, ablocks, off = [], [], 0
    for w in widths:
        blocks.append(dev(S[:, off:off + w], ld) if w else None)
        ablocks.append(dev(AS[:, off:off + w], ld) if w else None)
        off += w
    return blocks, ablocks


@pytest.mark.parametrize("dims", [(33, 33, 33)])
def test_noalloc_gram_matches_handle_gram_twice(dims):
    s = Solver(dims, precond="none")
    n = s.n
    stream = torch.cuda.current_stream().cuda_stream
    # first call: module load and address lookup (not measured)
    x = torch.ones((1, n), dtype=torch.float64, device="cuda")
    g1 = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    assert capi.lobpcg_gram_noalloc(ptr(x), None, None, None, None, None, n, n, 1, 0, 0, None, ptr(g1),
                                    ctypes.c_void_p(stream)) == capi.OK
    torch.cuda.synchronize()
    assert abs(g1.item() - n) <= 1e-12 * n
    for call, widths in enumerate([(8, 5, 5), (16, 16, 16)]):
        q = sum(widths)
        g = np.random.default_rng(100 + call)
        S = g.standard_normal((n, q)) * g.uniform(0.1, 10, q)[None, :]
        AS = g.standard_normal((n, q))
        ld = n + 3
        bl, abl = _blocks(S, AS, widths, ld)
        outs = {}
        for which in ("handle", "noalloc"):
            gA = torch.full((q, q), float("nan"), dtype=torch.float64, device="cuda")
            gB = torch.full((q, q), float("nan"), dtype=torch.float64, device="cuda")
            args = [ptr(b) for b in bl] + [ptr(b) for b in abl]
            if which == "handle":
                rc = capi.lobpcg_op_gram(s.h, *args, ld, *widths, ptr(gA), ptr(gB))
            else:
                torch.cuda.synchronize()
                free_before = torch.cuda.mem_get_info()[0]
                rc = capi.lobpcg_gram_noalloc(*args, n, ld, *widths, ptr(gA), ptr(gB), ctypes.c_void_p(stream))
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info()[0] == free_before      # nothing was allocated
            assert rc == capi.OK, capi.lobpcg_last_error(None)
            outs[which] = (gA.cpu().numpy().T, gB.cpu().numpy().T)
        nrmS, nrmA = np.linalg.norm(S, axis=0), np.linalg.norm(AS, axis=0)
        boundA = 4 * n * EPS * (np.outer(nrmS, nrmA) + np.outer(nrmA, nrmS)) / 2
        boundB = 4 * n * EPS * np.outer(nrmS, nrmS)
        assert np.all(np.abs(outs["noalloc"][0] - outs["handle"][0]) <= boundA)
        assert np.all(np.abs(outs["noalloc"][1] - outs["handle"][1]) <= boundB)
    s.close()


def test_noalloc_gram_rejects_too_wide_basis():
    x = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
    g = torch.zeros((97, 97), dtype=torch.float64, device="cuda")
    rc = capi.lobpcg_gram_noalloc(ptr(x), ptr(x), ptr(x), None, None, None, 64, 64, 33, 32, 32, None, ptr(g), None)
    assert rc == capi.ERR_ARG
    assert "maximum" in capi.lobpcg_last_error(None)
