"""phe_matmul_noalloc: the variant for callers that cannot allocate device
memory while serving (their HBM is owned by another allocator, or their loop
must not touch the CUDA allocator after start-up).  It keeps its scratch in a
fixed device array instead of allocating; its results must equal
phe_matmul's exactly (integer outputs), also on a second call that finds the
first call's data still in the shared array.

This file is collected last on purpose (pytest orders files by name)."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu
Q = synth.Q60


@pytest.fixture(scope="module")
def env():
    from paper_2505_07329_b300 import build
    build.build()
    ctx = phe.phe_ctx_create(4096, Q, 32, 0)
    W = synth.weights(300, 5000, seed=77)  # forward L = 2, backward L = 1
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
    yield ctx, w
    phe.phe_weights_free(w)
    phe.phe_ctx_destroy(ctx)


def _run(fn, ctx, w, direction, A, B, flags):
    import torch
    T, L, N = A.shape
    rows = phe.phe_weights_shape(w, direction)[0]
    odt = torch.int32 if flags == phe.PHE_OUT_SWITCHED else torch.int64
    om = torch.full((T, rows, N), -1, dtype=odt, device="cuda")
    ob = torch.full((T, rows), -1, dtype=odt, device="cuda")
    fn(ctx, w, direction, T, to_dev_u64(A), to_dev_u64(B), om, ob, flags)
    torch.cuda.synchronize()
    return om.cpu().numpy(), ob.cpu().numpy()


def test_noalloc_equals_phe_matmul_on_two_calls_in_a_row(env):
    ctx, w = env
    cases = [(phe.PHE_FWD, 40, phe.PHE_OUT_SWITCHED, 1), (phe.PHE_BWD, 17, phe.PHE_OUT_RAW, 2)]
    for direction, T, flags, seed in cases:
        L = phe.phe_weights_shape(w, direction)[2]
        A = synth.uniform_words((T, L, 4096), Q, 100 + seed)
        B = synth.uniform_words((T, L, 4096), Q, 200 + seed)
        ref_m, ref_b = _run(phe.phe_matmul, ctx, w, direction, A, B, flags)
        got_m, got_b = _run(phe.phe_matmul_noalloc, ctx, w, direction, A, B, flags)
        assert np.array_equal(got_m, ref_m)
        assert np.array_equal(got_b, ref_b)


def test_noalloc_rejects_requests_beyond_its_scratch(env):
    import torch
    ctx, w = env
    L = phe.phe_weights_shape(w, phe.PHE_FWD)[2]
    T = phe.PHE_NOALLOC_MAX_SCRATCH_BYTES // (L * 4096 * 8) + 1
    dummy = torch.empty(8, dtype=torch.int64, device="cuda")
    with pytest.raises(phe.PheError) as ei:
        phe.phe_matmul_noalloc(ctx, w, phe.PHE_FWD, T, dummy, dummy, dummy, dummy)
    assert ei.value.status == phe.PHE_EINVAL
    assert "exceeds the fixed scratch" in str(ei.value)
