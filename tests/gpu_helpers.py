"""Helpers shared by the GPU tests: move numpy ciphertexts to the device, call
the C-ABI hot path through the binding, bring results back."""
from __future__ import annotations

import numpy as np

from paper_2505_07329_b300 import phe


def to_dev_u64(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_matmul(ctx, w, direction, A, B, rows, flags=phe.PHE_OUT_SWITCHED, stream=None):
    """Run phe_matmul on host arrays A, B [T, L, N]; returns (mask, body) as numpy."""
    import torch
    T, L, N = A.shape
    dA, dB = to_dev_u64(A), to_dev_u64(B)
    odt = torch.int32 if flags == phe.PHE_OUT_SWITCHED else torch.int64
    om = torch.empty((T, rows, N), dtype=odt, device="cuda")
    ob = torch.empty((T, rows), dtype=odt, device="cuda")
    phe.phe_matmul(ctx, w, direction, T, dA, dB, om, ob, flags, stream)
    torch.cuda.synchronize()
    npdt = np.uint32 if flags == phe.PHE_OUT_SWITCHED else np.uint64
    return om.cpu().numpy().view(npdt), ob.cpu().numpy().view(npdt)
