"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for
bit, on the same seeded inputs.  Integer results must match exactly."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import gpu_matmul, to_dev, to_dev_u64

pytestmark = pytest.mark.gpu
Q = synth.Q60


@pytest.fixture(scope="module")
def lib():
    from paper_2505_07329_b300 import build
    build.build()
    return phe.lib()


@pytest.fixture(scope="module")
def ctxs(lib):
    made = {}

    def get(N, k=32):
        if (N, k) not in made:
            made[(N, k)] = phe.phe_ctx_create(N, Q, k, 0)
        return made[(N, k)]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _oracle_all(orc, W, A, B, method=0):
    return orc.lwedot_all(W, A, B, Q, method)


def _check_both_modes(orc, ctx, w, direction, Wdir, A, B, k=32, method=0):
    rows = Wdir.shape[0]
    ea, eb = _oracle_all(orc, Wdir, A, B, method)
    ga, gb = gpu_matmul(ctx, w, direction, A, B, rows, phe.PHE_OUT_RAW)
    assert np.array_equal(ga, ea), "raw masks differ"
    assert np.array_equal(gb, eb), "raw bodies differ"
    sa, sb = gpu_matmul(ctx, w, direction, A, B, rows, phe.PHE_OUT_SWITCHED)
    assert np.array_equal(sa.astype(np.uint64), orc.modswitch(ea, Q, k)), "switched masks differ"
    assert np.array_equal(sb.astype(np.uint64), orc.modswitch(eb, Q, k)), "switched bodies differ"


def test_toy_workload_full_parity(orc, ctxs):
    # N=1024, W 256x256, 16 tokens, encrypted by the oracle: every output word.
    wl = synth.WORKLOADS["toy"]
    N, (name, d_in, d_out), T = wl.ring.N, wl.projections[0], wl.tokens
    L = synth.blocks(d_in, N)
    W = synth.weights(d_out, d_in)
    X = synth.activations(T, d_in)
    S = synth.secret_key(N)
    A = synth.masks(T, L, N, Q)
    E = synth.noise(T, L, N)
    B = orc.encrypt_vectors(A, S, E, X, Q, wl.ring.delta)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        _check_both_modes(orc, ctx, w, phe.PHE_FWD, W, A, B)
        # and the switched result decrypts to W x mod t
        sa, sb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out)
        Y = X.astype(np.int64) @ W.astype(np.int64).T
        for t in range(T):
            for j in range(0, d_out, 17):
                v = orc.lwe_phase(sa[t, j].astype(np.uint64), int(sb[t, j]), S, 2 ** 32)
                assert (orc.decode(v, 2 ** 32, synth.T_PLAIN) - int(Y[t, j])) % synth.T_PLAIN == 0
    finally:
        phe.phe_weights_free(w)


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192])
def test_every_ring_degree(orc, ctxs, N):
    # Two blocks with a ragged tail (d_in = N + 5), 3 rows, 2 tokens.
    d_in, d_out, T = N + 5, 3, 2
    L = synth.blocks(d_in, N)
    W = synth.weights(d_out, d_in, seed=N)
    A = synth.uniform_words((T, L, N), Q, N + 1)
    B = synth.uniform_words((T, L, N), Q, N + 2)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        _check_both_modes(orc, ctx, w, phe.PHE_FWD, W, A, B, method=1 if N >= 4096 else 0)
    finally:
        phe.phe_weights_free(w)


@pytest.mark.parametrize("N", [256, 1024, 2048])
@pytest.mark.parametrize("T", [1, 2, 3])
def test_fewer_tokens_than_transform_slots(orc, ctxs, N, T):
    # At N <= 2048 a block holds 4096/N transform slots; with fewer tokens the
    # idle slots take adjacent rows.  d_out = 21 leaves a ragged last row
    # group, and T = 3 a ragged last token round.
    d_in, d_out = N // 2 + 3, 21
    L = synth.blocks(d_in, N)
    W = synth.weights(d_out, d_in, seed=N + T)
    A = synth.uniform_words((T, L, N), Q, 10 * N + T)
    B = synth.uniform_words((T, L, N), Q, 10 * N + T + 1)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        _check_both_modes(orc, ctx, w, phe.PHE_FWD, W, A, B)
    finally:
        phe.phe_weights_free(w)


@pytest.mark.parametrize("d_in,d_out,T", [(300, 37, 19), (256, 129, 17), (700, 5, 33)])
def test_ragged_forward_and_backward(orc, ctxs, d_in, d_out, T):
    # Shapes that leave partial row tiles (128), token chunks (16) and blocks.
    N = 256
    W = synth.weights(d_out, d_in, seed=d_in)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
    try:
        assert phe.phe_weights_shape(w, phe.PHE_FWD) == (d_out, d_in, synth.blocks(d_in, N))
        assert phe.phe_weights_shape(w, phe.PHE_BWD) == (d_in, d_out, synth.blocks(d_out, N))
        L = synth.blocks(d_in, N)
        A = synth.uniform_words((T, L, N), Q, 1)
        B = synth.uniform_words((T, L, N), Q, 2)
        _check_both_modes(orc, ctx, w, phe.PHE_FWD, W, A, B)
        Lb = synth.blocks(d_out, N)
        Ag = synth.uniform_words((T, Lb, N), Q, 3)
        Bg = synth.uniform_words((T, Lb, N), Q, 4)
        _check_both_modes(orc, ctx, w, phe.PHE_BWD, np.ascontiguousarray(W.T), Ag, Bg)
    finally:
        phe.phe_weights_free(w)


def test_output_modulus_26_bits(orc, ctxs):
    N, d_in, d_out, T = 512, 600, 9, 5
    W = synth.weights(d_out, d_in, seed=26)
    L = synth.blocks(d_in, N)
    A = synth.uniform_words((T, L, N), Q, 261)
    B = synth.uniform_words((T, L, N), Q, 262)
    ctx = ctxs(N, 26)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        _check_both_modes(orc, ctx, w, phe.PHE_FWD, W, A, B, k=26)
    finally:
        phe.phe_weights_free(w)


def test_extreme_inputs(orc, ctxs):
    # Words at 0, q-1 and above q (reduced on load), weights at -128/127.
    N, d_in, d_out, T = 256, 256, 4, 3
    W = np.full((d_out, d_in), 127, dtype=np.int8)
    W[1, :] = -128
    W[2, ::2] = -128
    W[3, :] = 0
    A = np.full((T, 1, N), Q - 1, dtype=np.uint64)
    A[1] = 0
    A[2] = np.uint64((1 << 64) - 1)  # reduced mod q by the kernel
    B = np.full((T, 1, N), Q - 1, dtype=np.uint64)
    B[2] = np.uint64((1 << 64) - 1)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        Ar = A % np.uint64(Q)
        Br = B % np.uint64(Q)
        ea, eb = orc.lwedot_all(W, Ar, Br, Q)
        ga, gb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out, phe.PHE_OUT_RAW)
        assert np.array_equal(ga, ea) and np.array_equal(gb, eb)
        assert not ga[1].any()  # zero mask in, zero mask out
    finally:
        phe.phe_weights_free(w)


def test_zero_tokens_is_a_noop(ctxs):
    ctx = ctxs(256)
    w = phe.phe_weights_upload(ctx, synth.weights(4, 8), phe.PHE_DIR_FWD_BIT)
    try:
        phe.phe_matmul(ctx, w, phe.PHE_FWD, 0, None, None, None, None)
        with pytest.raises(phe.PheError) as ei:
            phe.phe_matmul(ctx, w, phe.PHE_BWD, 1, 1, 1, 1, 1)
        assert ei.value.status == phe.PHE_EINVAL
    finally:
        phe.phe_weights_free(w)


def test_modswitch_kernel(orc, ctxs):
    import torch
    for k in (32, 26, 1):
        ctx = ctxs(1024, k)
        words = np.concatenate([np.array([0, 1, Q // 2, Q // 2 + 1, Q - 1, Q, 2 ** 64 - 1], dtype=np.uint64),
                                synth.uniform_words(100000, Q, k)])
        d_in = to_dev_u64(words)
        d_out = torch.empty(words.shape[0], dtype=torch.int32, device="cuda")
        phe.phe_modswitch(ctx, d_in, d_out, words.shape[0])
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got, orc.modswitch(words % np.uint64(Q), Q, k))


def test_client_encrypt_matches_oracle(orc, ctxs):
    import torch
    for N, d, T in [(256, 300, 3), (1024, 1024, 2)]:
        L = synth.blocks(d, N)
        S = synth.secret_key(N)
        A = synth.masks(T, L, N, Q)
        E = synth.noise(T, L, N)
        X = synth.activations(T, d)
        delta = Q // synth.T_PLAIN
        expect = orc.encrypt_vectors(A, S, E, X, Q, delta)
        ctx = ctxs(N)
        dB = torch.empty((T, L, N), dtype=torch.int64, device="cuda")
        phe.phe_client_encrypt(ctx, T, d, to_dev_u64(A), to_dev(S.astype(np.int8)), to_dev(E.astype(np.int32)),
                               to_dev(X), delta, dB)
        torch.cuda.synchronize()
        assert np.array_equal(dB.cpu().numpy().view(np.uint64), expect)


def test_q_proj_full_size_sampled(orc, ctxs):
    # Llama-3.2-1B q_proj at full size (N=4096, W 2048x2048, 1024 tokens) in
    # the configuration the benchmark times: sampled (token, row) outputs,
    # forward and backward, against the oracle one by one.
    import torch
    wl = synth.WORKLOADS["q_proj"]
    N, (name, d_in, d_out), T = wl.ring.N, wl.projections[0], wl.tokens
    W = synth.weights(d_out, d_in)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
    try:
        for direction, Wd in ((phe.PHE_FWD, W), (phe.PHE_BWD, np.ascontiguousarray(W.T))):
            rows, cols = Wd.shape
            L = synth.blocks(cols, N)
            A = synth.uniform_words((T, L, N), Q, 40 + direction)
            B = synth.uniform_words((T, L, N), Q, 50 + direction)
            dA, dB = to_dev_u64(A), to_dev_u64(B)
            om = torch.empty((T, rows, N), dtype=torch.int32, device="cuda")
            ob = torch.empty((T, rows), dtype=torch.int32, device="cuda")
            phe.phe_matmul(ctx, w, direction, T, dA, dB, om, ob)
            torch.cuda.synchronize()
            r = np.random.default_rng(7 + direction)
            pairs = np.stack([r.integers(0, T, 12), r.integers(0, rows, 12)], axis=1)
            pairs[0] = (T - 1, rows - 1)
            pairs[1] = (0, 0)
            ea, eb = orc.lwedot_pairs(Wd, A, B, pairs, Q, method=1)
            for n, (t, j) in enumerate(pairs):
                got_a = om[t, j].cpu().numpy().view(np.uint32).astype(np.uint64)
                got_b = np.uint64(np.uint32(ob[t, j].item() & 0xffffffff))
                assert np.array_equal(got_a, orc.modswitch(ea[n], Q, 32)), (direction, t, j)
                assert got_b == orc.modswitch(eb[n:n + 1], Q, 32)[0], (direction, t, j)
    finally:
        phe.phe_weights_free(w)
