"""Helpers of the GPU tests: move column-major numpy blocks to and from device tensors."""
import ctypes

import numpy as np
import torch


def dev(X, ld=None):
    """numpy (n, m) float64 -> cuda tensor (m, ld); row j holds column j (ld >= n, pad = NaN)."""
    n, m = X.shape
    ld = n if ld is None else ld
    T = torch.full((m, ld), float("nan"), dtype=torch.float64)
    T[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T))
    return T.cuda()


def host(T, n):
    return T[:, :n].cpu().numpy().T.copy()


def ptr(T):
    return ctypes.c_void_p(T.data_ptr()) if T is not None else None


def empty(m, ld):
    return torch.full((m, ld), float("nan"), dtype=torch.float64, device="cuda")
