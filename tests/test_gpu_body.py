"""GPU parity of the bodies b'_tj = sum_k W[j,k] B_t[k] (mod q), which run on
the tensor cores as an exact bf16 digit GEMM (tcgen05.mma, fp32 accumulation
in chunks of 1024 columns), against the CPU oracle's Eq. (LWEdot), word for
word; the fused dp4a bodies (small launch groups) must give the same words.
The cases push the fp32 accumulators to their largest magnitude, cross the
chunk boundaries, and leave ragged row, token and column tails."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import gpu_matmul

pytestmark = pytest.mark.gpu
N = 1024
MODULI = {"prime": (synth.Q60, None), "rns": (synth.Q_RNS, (synth.RNS_P1, synth.RNS_P2))}


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(name):
        if name not in made:
            q, rns = MODULI[name]
            made[name] = phe.phe_ctx_create(N, q, 32, 0, rns=rns)
        return made[name]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _extreme_body(q):
    """A word below q whose balanced base-256 digits are -128 in every byte
    but the top one: the largest |digit| the GEMM meets."""
    v = 0x80 | sum(0x7F << (8 * l) for l in range(1, 7))
    top = 0x0F
    while (v | (top << 56)) >= q:
        top -= 1
    return v | (top << 56)


def _check(orc, ctx, q, W, A, B, direction=phe.PHE_FWD, Wdir=None):
    """Bodies on the tensor cores (forced, whatever the size) against the
    oracle, raw and switched; the fused bodies must give the same words."""
    Wdir = W if Wdir is None else Wdir
    rows = Wdir.shape[0]
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
    try:
        # the oracle's NTT products need a prime q; the RNS q takes the schoolbook definition
        ea, eb = orc.lwedot_all(Wdir, A, B, q, 1 if q == synth.Q60 else 0)
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_TENSOR)
        ga, gb = gpu_matmul(ctx, w, direction, A, B, rows, phe.PHE_OUT_RAW)
        assert np.array_equal(gb, eb), "raw bodies differ"
        assert np.array_equal(ga, ea), "raw masks differ"
        sa, sb = gpu_matmul(ctx, w, direction, A, B, rows, phe.PHE_OUT_SWITCHED)
        assert np.array_equal(sb.astype(np.uint64), orc.modswitch(eb, q, 32)), "switched bodies differ"
        assert phe.phe_ctx_status(ctx) == 0
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_FUSED)
        fa, fb = gpu_matmul(ctx, w, direction, A, B, rows, phe.PHE_OUT_SWITCHED)
        assert np.array_equal(fb, sb) and np.array_equal(fa, sa), "fused bodies differ"
    finally:
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_AUTO)
        phe.phe_weights_free(w)


@pytest.mark.parametrize("modulus", sorted(MODULI))
@pytest.mark.parametrize("d_in", [1024, 2048, 3071])
def test_largest_accumulator_magnitudes(orc, ctxs, modulus, d_in):
    # every weight +-127 and every digit -128: each 1024-column chunk sums to
    # +-127 * 128 * 1024 = 16 646 144, just below 2^24
    q = MODULI[modulus][0]
    rows, T = 130, 3
    L = synth.blocks(d_in, N)
    W = np.full((rows, d_in), -127, dtype=np.int8)
    W[1::2] = 127
    A = synth.uniform_words((T, L, N), q, 5)
    B = np.full((T, L, N), _extreme_body(q), dtype=np.uint64)
    _check(orc, ctxs(modulus), q, W, A, B)


@pytest.mark.parametrize("modulus", sorted(MODULI))
@pytest.mark.parametrize("d_in,rows,T", [(1, 1, 1), (7, 129, 2), (1023, 127, 33), (1025, 300, 5),
                                         (2049, 64, 17), (4100, 9, 9)])
def test_ragged_shapes(orc, ctxs, modulus, d_in, rows, T):
    # column tails inside a 64-column stage and across 1024-column chunks,
    # row tails inside a 128-row tile, token tails inside a token tile
    q = MODULI[modulus][0]
    L = synth.blocks(d_in, N)
    W = synth.weights(rows, d_in, seed=d_in + rows)
    A = synth.uniform_words((T, L, N), q, d_in)
    B = synth.uniform_words((T, L, N), q, d_in + 1)
    _check(orc, ctxs(modulus), q, W, A, B)


def test_backward_bodies_and_unreduced_words(orc, ctxs):
    # backward: the GEMM runs on W^T (uploaded transposed); body words at and
    # above q are reduced before the digit split
    q = synth.Q60
    d_out, d_in, T = 1500, 200, 4
    W = synth.weights(d_out, d_in, seed=3)
    L = synth.blocks(d_out, N)
    A = synth.uniform_words((T, L, N), q, 8)
    B = synth.uniform_words((T, L, N), q, 9)
    B[0, 0, :16] = np.array([q, q + 1, 2 ** 64 - 1, 2 ** 63] + [q - 1] * 12, dtype=np.uint64)
    _check(orc, ctxs("prime"), q, W, A, B, direction=phe.PHE_BWD, Wdir=np.ascontiguousarray(W.T))


def test_sixteen_chunks(orc, ctxs):
    # d_in = 16384, the upload limit: 16 fp32 chunks of 1024 columns, 32
    # tensor-memory columns each (4 tokens per tile)
    q = synth.Q_RNS
    rows, T, d_in = 5, 6, 16384
    L = synth.blocks(d_in, N)
    W = synth.weights(rows, d_in, seed=16)
    W[0] = -127
    A = synth.uniform_words((T, L, N), q, 16)
    B = synth.uniform_words((T, L, N), q, 17)
    B[:, :, :] = np.where(np.arange(N) % 2 == 0, _extreme_body(q), B)
    _check(orc, ctxs("rns"), q, W, A, B)


@pytest.mark.parametrize("d_in,rows,T", [(2048, 130, 3), (3000, 64, 9), (8192, 33, 2)])
def test_power_of_two_modulus(orc, d_in, rows, T):
    # the paper's q = 2^39 (N = 2048, computed exactly through p1 p2): bodies
    # reduced mod 2^39 before the digit split and recombined mod 2^39, the
    # switch a rounding shift to 2^26
    q, k, Np = 1 << 39, 26, 2048
    ctx = phe.phe_ctx_create(Np, q, k, 0, rns=(synth.RNS_P1, synth.RNS_P2))
    L = synth.blocks(d_in, Np)
    W = synth.weights(rows, d_in, seed=d_in)
    W[0] = -127
    A = synth.uniform_words((T, L, Np), q, 21)
    B = synth.uniform_words((T, L, Np), q, 22)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        ea, eb = orc.lwedot_all(W, A, B, q, 0)
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_TENSOR)
        ga, gb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, rows, phe.PHE_OUT_RAW)
        assert np.array_equal(gb, eb) and np.array_equal(ga, ea)
        sa, sb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, rows, phe.PHE_OUT_SWITCHED)
        assert np.array_equal(sb.astype(np.uint64), orc.modswitch(eb, q, k))
        assert phe.phe_ctx_status(ctx) == 0
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_FUSED)
        fa, fb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, rows, phe.PHE_OUT_SWITCHED)
        assert np.array_equal(fb, sb) and np.array_equal(fa, sa)
    finally:
        phe.phe_weights_free(w)
        phe.phe_ctx_destroy(ctx)


@pytest.mark.parametrize("Nr,d_in,rows,T", [(256, 700, 130, 5), (8192, 9000, 40, 3)])
def test_other_ring_degrees(orc, Nr, d_in, rows, T):
    # the bodies' token stride is L*N words: ring degrees at both ends, with
    # ragged last blocks, through the tensor cores and fused
    q = synth.Q60
    ctx = phe.phe_ctx_create(Nr, q, 32, 0)
    L = synth.blocks(d_in, Nr)
    W = synth.weights(rows, d_in, seed=Nr)
    A = synth.uniform_words((T, L, Nr), q, 31)
    B = synth.uniform_words((T, L, Nr), q, 32)
    try:
        _check(orc, ctx, q, W, A, B)
    finally:
        phe.phe_ctx_destroy(ctx)
