"""GPU: the paper's parameter set (Table cryptoparams, Sec. 4.4): N = 2048,
q = 2^39, q_out = 2^26, binary key, Delta = q / 2^27 (beta = 27 bits).

The power-of-two q has no NTT, so the kernels form the products exactly in Z
through the RNS modulus p1 p2 (centred lift of the masks) and reduce mod 2^39.

  - parity: the GPU outputs (raw mod 2^39, and switched to 2^26 by a rounding
    shift) equal the oracle's Eq. (LWEdot) + ModulusSwitch at q = 2^39, for
    full and seeded inputs, ragged shapes, lift edges and the largest block
    count the exact range allows (d_in = 8192, L = 4);
  - the bit-error experiment of Sec. 6.2: homomorphic dot products of random
    int8 vectors for d_in in {768, 2048, 8192}, decrypted and compared
    bitwise with the true values: bits 12 and up err on well under 1% of the
    outputs.
"""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu

Q39 = 1 << 39
KOUT = 26
BETA = 27
DELTA = Q39 >> BETA   # 2^12


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(N):
        if N not in made:
            made[N] = phe.phe_ctx_create(N, Q39, KOUT, 0, rns=(synth.RNS_P1, synth.RNS_P2))
        return made[N]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _run(ctx, w, direction, A, B, rows, flags, seeds=None):
    import torch
    T, L, N = B.shape
    odt = torch.int64 if flags == phe.PHE_OUT_RAW else torch.int32
    om = torch.empty((T, rows, N), dtype=odt, device="cuda")
    ob = torch.empty((T, rows), dtype=odt, device="cuda")
    if seeds is None:
        phe.phe_matmul(ctx, w, direction, T, to_dev_u64(A), to_dev_u64(B), om, ob, flags)
    else:
        phe.phe_matmul_seeded(ctx, w, direction, T, to_dev_u64(seeds), to_dev_u64(B), om, ob, flags)
    torch.cuda.synchronize()
    if flags == phe.PHE_OUT_RAW:
        return om.cpu().numpy().view(np.uint64), ob.cpu().numpy().view(np.uint64)
    return (om.cpu().numpy().view(np.uint32).astype(np.uint64),
            (ob.cpu().numpy().astype(np.int64) & 0xffffffff).astype(np.uint64))


@pytest.mark.parametrize("N,d_in,d_out,T", [(256, 300, 37, 3), (2048, 768, 5, 2)])
def test_pow2_products_match_oracle(orc, ctxs, N, d_in, d_out, T):
    ctx = ctxs(N)
    g = _rng(N + d_in)
    W = g.integers(-127, 128, (d_out, d_in)).astype(np.int8)
    L = synth.blocks(d_in, N)
    A = g.integers(0, Q39, (T, L, N), dtype=np.uint64)
    A[0, 0, :6] = [0, 1, Q39 - 1, Q39 // 2, Q39 // 2 - 1, Q39 // 2 + 1]   # edges of the centred lift
    B = g.integers(0, Q39, (T, L, N), dtype=np.uint64)
    w = phe.phe_weights_upload(ctx, W)
    try:
        ra, rb = _run(ctx, w, phe.PHE_FWD, A, B, d_out, phe.PHE_OUT_RAW)
        sa, sb = _run(ctx, w, phe.PHE_FWD, A, B, d_out, phe.PHE_OUT_SWITCHED)
        Wt = np.ascontiguousarray(W.T)
        Lb = synth.blocks(d_out, N)
        Ab = g.integers(0, Q39, (T, Lb, N), dtype=np.uint64)
        Bb = g.integers(0, Q39, (T, Lb, N), dtype=np.uint64)
        rab, rbb = _run(ctx, w, phe.PHE_BWD, Ab, Bb, d_in, phe.PHE_OUT_RAW)
    finally:
        phe.phe_weights_free(w)
    ea, eb = orc.lwedot_all(W, A, B, Q39)
    assert np.array_equal(ra, ea) and np.array_equal(rb, eb)
    assert np.array_equal(sa, orc.modswitch(ea, Q39, KOUT)) and np.array_equal(sb, orc.modswitch(eb, Q39, KOUT))
    pairs = np.array([(0, 0), (T - 1, d_in - 1), (0, d_in // 2)])
    eab, ebb = orc.lwedot_pairs(Wt, Ab, Bb, pairs, Q39)
    assert np.array_equal(np.stack([rab[t, j] for t, j in pairs]), eab)
    assert np.array_equal(np.array([rbb[t, j] for t, j in pairs]), ebb)


def test_pow2_seeded_and_largest_block_count(orc, ctxs):
    N, d_in, d_out, T = 2048, 8192, 3, 2     # L = 4: 4 * 2048 * 127 * 2^38 < p1 p2 / 2
    ctx = ctxs(N)
    g = _rng(5)
    W = g.integers(-127, 128, (d_out, d_in)).astype(np.int8)
    W[0] = 127                                  # the extreme row of the exact range
    L = synth.blocks(d_in, N)
    seeds = g.integers(0, 2 ** 64, (T, L), dtype=np.uint64)
    A = orc.expand_masks(seeds, N, Q39)
    B = g.integers(0, Q39, (T, L, N), dtype=np.uint64)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        sa, sb = _run(ctx, w, phe.PHE_FWD, A, B, d_out, phe.PHE_OUT_SWITCHED, seeds=seeds)
    finally:
        phe.phe_weights_free(w)
    pairs = np.array([(0, 0), (1, 0), (1, 2)])
    ea, eb = orc.lwedot_pairs(W, A, B, pairs, Q39)
    assert np.array_equal(np.stack([sa[t, j] for t, j in pairs]), orc.modswitch(ea, Q39, KOUT))
    assert np.array_equal(np.array([sb[t, j] for t, j in pairs]), orc.modswitch(eb, Q39, KOUT))


def test_pow2_rejects_blocks_beyond_the_exact_range(ctxs):
    # q = 2^42, N = 2048: L * 2048 * 127 * 2^41 < p1 p2 / 2 holds for L = 1 only
    ctx = phe.phe_ctx_create(2048, 1 << 42, 26, 0, rns=(synth.RNS_P1, synth.RNS_P2))
    try:
        w = phe.phe_weights_upload(ctx, np.zeros((2, 2048), np.int8), phe.PHE_DIR_FWD_BIT)
        phe.phe_weights_free(w)
        with pytest.raises(phe.PheError) as ei:
            phe.phe_weights_upload(ctx, np.zeros((2, 2049), np.int8), phe.PHE_DIR_FWD_BIT)
        assert ei.value.status == phe.PHE_EINVAL
    finally:
        phe.phe_ctx_destroy(ctx)
    # a key-switching key at q = 2^39 is held in exact slices: at N = n = 256,
    # base 2^13, one level, 256 * 256 * 2^12 * 2^(b-1) < p1 p2 / 2 gives
    # b = 31 bits, so two slices of the 40-bit balanced key
    k = phe.phe_ksk_upload(ctxs(256), np.zeros((256, 1, 256), np.uint64), np.zeros((256, 1, 256), np.uint64), 13, 1)
    try:
        assert phe.phe_ksk_device_bytes(k) == 2 * (256 * 2 * 256 * 16)
    finally:
        phe.phe_ksk_free(k)


def _bit_errors(y, dec, bits=BETA):
    """Fraction of outputs whose bit b (two's complement, `bits` wide) differs."""
    m = (1 << bits) - 1
    a, b = (y & m), (dec & m)
    return np.array([np.mean(((a >> k) & 1) != ((b >> k) & 1)) for k in range(bits)])


@pytest.mark.parametrize("d_in", [768, 2048, 8192])
def test_bit_error_rates_sec_6_2(orc, ctxs, d_in):
    N, T, rows = 2048, 4, 1024
    ctx = ctxs(N)
    g = _rng(62 + d_in)
    S = g.integers(0, 2, N)                      # binary key (Sec. 3.1)
    W = g.integers(-127, 128, (rows, d_in)).astype(np.int8)
    X = g.integers(-127, 128, (T, d_in)).astype(np.int8)
    L = synth.blocks(d_in, N)
    A = g.integers(0, Q39, (T, L, N), dtype=np.uint64)
    E = np.rint(g.normal(0, synth.SIGMA, (T, L, N))).astype(np.int64)
    B = orc.encrypt_vectors(A, S, E, X, Q39, DELTA)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        a, b = _run(ctx, w, phe.PHE_FWD, A, B, rows, phe.PHE_OUT_SWITCHED)
    finally:
        phe.phe_weights_free(w)
    # client: phase mod 2^26, message = phase * 2^27 / 2^26 = 2 * phase (mod 2^27)
    ph = (b.astype(np.int64) - (a.astype(np.int64) @ S.astype(np.int64))) % (1 << KOUT)
    dec = (2 * ph) % (1 << BETA)
    dec = np.where(dec >= 1 << (BETA - 1), dec - (1 << BETA), dec)
    y = X.astype(np.int64) @ W.astype(np.int64).T
    rates = _bit_errors(y.ravel(), dec.ravel())
    print(f"d_in={d_in} bit error rates (bit 0..21): " + " ".join(f"{r:.4f}" for r in rates[:22]))
    assert np.all(rates[12:] < 0.01), rates
    assert rates[0] > 0.3     # the LSB is lost to the switch (q_out / 2^beta = 1/2)
