"""phe_matmul_noalloc: the variant for callers that cannot allocate device
memory while serving (their HBM is owned by another allocator, or their loop
must not touch the CUDA allocator after start-up).  It keeps its scratch in a
fixed device array instead of allocating; its results must equal
phe_matmul's exactly (integer outputs), also on a second call that finds the
first call's data still in the shared array, and the oracle's.

This file is collected last on purpose (pytest orders files by name)."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu
N = 4096
MODULI = {"prime": (synth.Q60, None), "rns": (synth.Q_RNS, (synth.RNS_P1, synth.RNS_P2))}


@pytest.fixture(scope="module", params=sorted(MODULI))
def env(request):
    from paper_2505_07329_b300 import build
    build.build()
    q, rns = MODULI[request.param]
    ctx = phe.phe_ctx_create(N, q, 32, 0, rns=rns)
    W = synth.weights(300, 5000, seed=77)  # forward L = 2, backward L = 1
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
    yield ctx, w, W, q
    phe.phe_weights_free(w)
    phe.phe_ctx_destroy(ctx)


def _bufs(w, direction, T, flags):
    import torch
    rows = phe.phe_weights_shape(w, direction)[0]
    odt = torch.int32 if flags == phe.PHE_OUT_SWITCHED else torch.int64
    return (torch.full((T, rows, N), -1, dtype=odt, device="cuda"),
            torch.full((T, rows), -1, dtype=odt, device="cuda"))


def _run(fn, ctx, w, direction, dA, dB, flags, T):
    import torch
    om, ob = _bufs(w, direction, T, flags)
    fn(ctx, w, direction, T, dA, dB, om, ob, flags)
    torch.cuda.synchronize()
    return om.cpu().numpy(), ob.cpu().numpy()


def test_noalloc_equals_phe_matmul_on_two_calls_in_a_row(env):
    ctx, w, _, q = env
    cases = [(phe.PHE_FWD, 40, phe.PHE_OUT_SWITCHED, 1), (phe.PHE_BWD, 17, phe.PHE_OUT_RAW, 2)]
    for direction, T, flags, seed in cases:
        L = phe.phe_weights_shape(w, direction)[2]
        A = synth.uniform_words((T, L, N), q, 100 + seed)
        B = synth.uniform_words((T, L, N), q, 200 + seed)
        dA, dB = to_dev_u64(A), to_dev_u64(B)
        ref_m, ref_b = _run(phe.phe_matmul, ctx, w, direction, dA, dB, flags, T)
        got_m, got_b = _run(phe.phe_matmul_noalloc, ctx, w, direction, dA, dB, flags, T)
        assert np.array_equal(got_m, ref_m)
        assert np.array_equal(got_b, ref_b)


def test_noalloc_matches_the_oracle(env, orc):
    # sampled (token, row) outputs against the CPU oracle, raw and switched
    ctx, w, W, q = env
    T = 6
    A = synth.uniform_words((T, 2, N), q, 31)
    B = synth.uniform_words((T, 2, N), q, 32)
    dA, dB = to_dev_u64(A), to_dev_u64(B)
    raw_m, raw_b = _run(phe.phe_matmul_noalloc, ctx, w, phe.PHE_FWD, dA, dB, phe.PHE_OUT_RAW, T)
    sw_m, sw_b = _run(phe.phe_matmul_noalloc, ctx, w, phe.PHE_FWD, dA, dB, phe.PHE_OUT_SWITCHED, T)
    pairs = np.array([[t, j] for t in (0, T - 1) for j in (0, 151, 299)], dtype=np.int64)
    # the oracle's NTT products need a prime q; the RNS q takes the schoolbook definition
    ea, eb = orc.lwedot_pairs(W, A, B, pairs, q, method=1 if q == synth.Q60 else 0)
    for n, (t, j) in enumerate(pairs):
        assert np.array_equal(raw_m[t, j].view(np.uint64), ea[n])
        assert int(raw_b[t, j].view(np.uint64)) == int(eb[n])
        assert np.array_equal(sw_m[t, j].view(np.uint32).astype(np.uint64), orc.modswitch(ea[n], q, 32))
        assert int(sw_b[t, j].view(np.uint32)) == int(orc.modswitch(np.array([eb[n]], dtype=np.uint64), q, 32)[0])


def test_noalloc_takes_no_memory_and_records_no_trace(env):
    import torch
    ctx, w, _, q = env
    T = 8
    A = synth.uniform_words((T, 2, N), q, 41)
    B = synth.uniform_words((T, 2, N), q, 42)
    dA, dB = to_dev_u64(A), to_dev_u64(B)
    om, ob = _bufs(w, phe.PHE_FWD, T, phe.PHE_OUT_SWITCHED)
    phe.phe_matmul_noalloc(ctx, w, phe.PHE_FWD, T, dA, dB, om, ob)  # warm
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    phe.phe_trace_enable(ctx, True)
    try:
        phe.phe_matmul_noalloc(ctx, w, phe.PHE_FWD, T, dA, dB, om, ob)
        torch.cuda.synchronize()
        assert phe.phe_trace_read(ctx) == {}
    finally:
        phe.phe_trace_enable(ctx, False)
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_requests_beyond_its_scratch(env):
    import torch
    ctx, w, _, _ = env
    L = phe.phe_weights_shape(w, phe.PHE_FWD)[2]
    T = phe.PHE_NOALLOC_MAX_SCRATCH_BYTES // (L * N * 8) + 1
    dummy = torch.empty(8, dtype=torch.int64, device="cuda")
    with pytest.raises(phe.PheError) as ei:
        phe.phe_matmul_noalloc(ctx, w, phe.PHE_FWD, T, dummy, dummy, dummy, dummy)
    assert ei.value.status == phe.PHE_EINVAL
    assert "exceeds the fixed scratch" in str(ei.value)
