"""GPU: the test library's client-side calls (libphe_test.so only): the
seeded key generator draws the stated distributions, and an encryption under
its key, pushed through the server path, decrypts to W x mod t (the oracle's
decryption)."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import gpu_matmul, to_dev, to_dev_u64

pytestmark = pytest.mark.gpu
N = 1024


@pytest.fixture(scope="module")
def ctx():
    from paper_2505_07329_b300 import build
    build.build()
    c = phe.phe_ctx_create(N, synth.Q60, 32, 0)
    yield c
    phe.phe_ctx_destroy(c)


def test_keygen_distributions(ctx):
    t = phe.phe_test_keygen(ctx, N, 7, phe.PHE_KEY_TERNARY)
    assert set(np.unique(t)) <= {-1, 0, 1}
    counts = [int(np.sum(t == v)) for v in (-1, 0, 1)]
    assert all(0.25 * N < c < 0.42 * N for c in counts), counts
    assert np.array_equal(t, phe.phe_test_keygen(ctx, N, 7, phe.PHE_KEY_TERNARY))
    assert not np.array_equal(t, phe.phe_test_keygen(ctx, N, 8, phe.PHE_KEY_TERNARY))
    b = phe.phe_test_keygen(ctx, N, 7, phe.PHE_KEY_BINARY)
    assert set(np.unique(b)) <= {0, 1} and 0.4 * N < int(b.sum()) < 0.6 * N


def test_encryption_under_the_generated_key_decrypts(orc, ctx):
    q = synth.Q60
    T, d_in, d_out = 3, 700, 33
    S = phe.phe_test_keygen(ctx, N, 11).astype(np.int64)
    W = synth.weights(d_out, d_in, seed=5)
    X = synth.activations(T, d_in, seed=6)
    L = synth.blocks(d_in, N)
    A = synth.masks(T, L, N, q, seed=7)
    E = synth.noise(T, L, N, seed=8)
    import torch
    dB = torch.empty((T, L, N), dtype=torch.int64, device="cuda")
    phe.phe_client_encrypt(ctx, T, d_in, to_dev_u64(A), to_dev(S.astype(np.int8)), to_dev(E.astype(np.int32)),
                           to_dev(X), q // synth.T_PLAIN, dB)
    torch.cuda.synchronize()
    B = dB.cpu().numpy().view(np.uint64)
    assert np.array_equal(B, orc.encrypt_vectors(A, S, E, X, q, q // synth.T_PLAIN))
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        sa, sb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out)
    finally:
        phe.phe_weights_free(w)
    Y = X.astype(np.int64) @ W.astype(np.int64).T
    for t in range(T):
        for j in range(d_out):
            v = orc.lwe_phase(sa[t, j].astype(np.uint64), int(sb[t, j]), S, 2 ** 32)
            assert (orc.decode(v, 2 ** 32, synth.T_PLAIN) - int(Y[t, j])) % synth.T_PLAIN == 0
