"""GPU: output packing (Sec. 3.2 KeySwitching and Rotate, Eq. (pack_rotate))
against the oracle, bit for bit.

  - phe_pack on given LWE ciphertexts equals the oracle's packing sum
    (raw words mod q, and after the switch), for both moduli, several gadget
    shapes, ragged row groups and several tokens;
  - at N = 4096, sampled coefficients of full-size packs match the oracle's
    coefficient-by-coefficient evaluation;
  - phe_matmul_packed on real encryptions equals the oracle composition
    Eq. (LWEdot) -> packing -> switch, and decrypts to (W x) mod t;
  - token chunking inside phe_matmul_packed does not change the result.
"""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu

MODULI = {"prime": (synth.Q60, None), "rns": (synth.Q_RNS, (synth.RNS_P1, synth.RNS_P2)),
          "pow2": (1 << 39, (synth.RNS_P1, synth.RNS_P2))}   # q = 2^39: the key in exact slices


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(N, modulus):
        key = (N, modulus)
        if key not in made:
            q, rns = MODULI[modulus]
            made[key] = phe.phe_ctx_create(N, q, 32, 0, rns=rns)
        return made[key]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _gpu_pack(ctx, k, masks, bodies, N, flags):
    import torch
    T, rows = bodies.shape
    G = (rows + N - 1) // N
    odt = torch.int64 if flags == phe.PHE_OUT_RAW else torch.int32
    oa = torch.empty((T, G, N), dtype=odt, device="cuda")
    ob = torch.empty((T, G, N), dtype=odt, device="cuda")
    phe.phe_pack(ctx, k, T, rows, to_dev_u64(masks), to_dev_u64(bodies), oa, ob, flags)
    torch.cuda.synchronize()
    if flags == phe.PHE_OUT_RAW:
        return oa.cpu().numpy().view(np.uint64), ob.cpu().numpy().view(np.uint64)
    return (oa.cpu().numpy().view(np.uint32).astype(np.uint64), ob.cpu().numpy().view(np.uint32).astype(np.uint64))


@pytest.mark.parametrize("modulus,base_log,ell", [("rns", 26, 1), ("prime", 26, 1), ("rns", 13, 2),
                                                  ("prime", 10, 3), ("rns", 8, 4),
                                                  ("pow2", 26, 1), ("pow2", 13, 2), ("pow2", 8, 4)])
def test_pack_matches_oracle(orc, ctxs, modulus, base_log, ell):
    N, T, rows = 256, 2, 300          # two row groups per token, the second ragged (44 rows)
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    g = _rng(100 + ell)
    KA = g.integers(0, q, (N, ell, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, ell, N), dtype=np.uint64)
    masks = g.integers(0, q, (T, rows, N), dtype=np.uint64)
    bodies = g.integers(0, q, (T, rows), dtype=np.uint64)
    masks[0, 0, :4] = [0, q - 1, q // 2, (q + 1) // 2]   # switch edges
    k = phe.phe_ksk_upload(ctx, KA, KB, base_log, ell)
    try:
        raw_a, raw_b = _gpu_pack(ctx, k, masks, bodies, N, phe.PHE_OUT_RAW)
        sw_a, sw_b = _gpu_pack(ctx, k, masks, bodies, N, phe.PHE_OUT_SWITCHED)
    finally:
        phe.phe_ksk_free(k)
    for t in range(T):
        for grp in range(2):
            a = masks[t, grp * N:(grp + 1) * N]
            b = bodies[t, grp * N:(grp + 1) * N]
            ea, eb = orc.pack_coeffs(a, b, KA, KB, q, base_log, ell, np.arange(N))
            assert np.array_equal(raw_a[t, grp], ea) and np.array_equal(raw_b[t, grp], eb), (t, grp)
            assert np.array_equal(sw_a[t, grp], orc.modswitch(ea, q, 32))
            assert np.array_equal(sw_b[t, grp], orc.modswitch(eb, q, 32))


def test_matmul_packed_pow2_matches_oracle(orc, ctxs):
    # q = 2^39: Eq. (LWEdot) through p1 p2, the masks switched to 2^26 for
    # Decomp, the key in slices; compared word for word with the oracle's
    # composition (no decryption: with t = 2^16 the key-switching noise at
    # this q exceeds the plaintext margin)
    import torch
    N, T, q = 256, 2, 1 << 39
    ctx = ctxs(N, "pow2")
    g = _rng(41)
    W = synth.weights(300, 290, seed=42)
    L = synth.blocks(290, N)
    A = g.integers(0, q, (T, L, N), dtype=np.uint64)
    B = g.integers(0, q, (T, L, N), dtype=np.uint64)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        oa = torch.empty((T, 2, N), dtype=torch.int32, device="cuda")
        ob = torch.empty((T, 2, N), dtype=torch.int32, device="cuda")
        phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, to_dev_u64(A), to_dev_u64(B), oa, ob)
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    ga = oa.cpu().numpy().view(np.uint32).astype(np.uint64)
    gb = ob.cpu().numpy().view(np.uint32).astype(np.uint64)
    la, lb = orc.lwedot_all(W, A, B, q)
    for t in range(T):
        for grp in range(2):
            m = min(N, 300 - grp * N)
            ea, eb = orc.pack_coeffs(la[t, grp * N:grp * N + m], lb[t, grp * N:grp * N + m], KA, KB, q, 26, 1,
                                     np.arange(N))
            assert np.array_equal(ga[t, grp], orc.modswitch(ea, q, 32)), (t, grp)
            assert np.array_equal(gb[t, grp], orc.modswitch(eb, q, 32)), (t, grp)


@pytest.mark.parametrize("modulus", ["rns", "prime"])
def test_pack_full_size_sampled(orc, ctxs, modulus):
    N, T, rows = 4096, 2, 4096 + 100
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    g = _rng(7)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    masks = g.integers(0, q, (T, rows, N), dtype=np.uint64)
    bodies = g.integers(0, q, (T, rows), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        ga, gb = _gpu_pack(ctx, k, masks, bodies, N, phe.PHE_OUT_SWITCHED)
    finally:
        phe.phe_ksk_free(k)
    rs = np.array([0, 1, 99, 100, 2047, 4095])
    for t, grp in [(0, 0), (1, 1)]:
        a = masks[t, grp * N:(grp + 1) * N]
        b = bodies[t, grp * N:(grp + 1) * N]
        ea, eb = orc.pack_coeffs(a, b, KA, KB, q, 26, 1, rs)
        assert np.array_equal(ga[t, grp, rs], orc.modswitch(ea, q, 32)), (t, grp)
        assert np.array_equal(gb[t, grp, rs], orc.modswitch(eb, q, 32)), (t, grp)


def _encrypted_inputs(orc, N, T, d, q, seed):
    g = _rng(seed)
    S = g.integers(-1, 2, N)
    L = synth.blocks(d, N)
    A = g.integers(0, q, (T, L, N), dtype=np.uint64)
    E = np.rint(g.normal(0, synth.SIGMA, (T, L, N))).astype(np.int64)
    X = g.integers(-127, 128, (T, d)).astype(np.int8)
    B = orc.encrypt_vectors(A, S, E, X, q, q // synth.T_PLAIN)
    return S, A, B, X


@pytest.mark.parametrize("modulus", ["rns", "prime"])
@pytest.mark.parametrize("direction", [phe.PHE_FWD, phe.PHE_BWD])
def test_matmul_packed_end_to_end(orc, ctxs, modulus, direction):
    import torch
    N, T, t = 256, 3, synth.T_PLAIN
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    W = synth.weights(300, 290, seed=21)          # fwd: 300 rows (2 groups) of 290; bwd: 290 rows of 300
    Wd = W if direction == phe.PHE_FWD else np.ascontiguousarray(W.T)
    rows, cols = Wd.shape
    S, A, B, X = _encrypted_inputs(orc, N, T, cols, q, 22 + direction)
    g = _rng(23)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    E = np.rint(g.normal(0, synth.SIGMA, (N, 1, N))).astype(np.int64)
    KB = orc.ksk_encrypt(KA, E, S, S, q, 26, 1)
    w = phe.phe_weights_upload(ctx, W)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    G = (rows + N - 1) // N
    try:
        oa = torch.empty((T, G, N), dtype=torch.int32, device="cuda")
        ob = torch.empty((T, G, N), dtype=torch.int32, device="cuda")
        phe.phe_matmul_packed(ctx, w, k, direction, T, to_dev_u64(A), to_dev_u64(B), oa, ob)
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    ga = oa.cpu().numpy().view(np.uint32).astype(np.uint64)
    gb = ob.cpu().numpy().view(np.uint32).astype(np.uint64)
    la, lb = orc.lwedot_all(Wd, A, B, q)
    y = X.astype(np.int64) @ Wd.astype(np.int64).T
    Sq = np.array([s % (1 << 32) for s in S.tolist()], dtype=np.uint64)
    for tok in range(T):
        for grp in range(G):
            m = min(N, rows - grp * N)
            ea, eb = orc.pack_coeffs(la[tok, grp * N:grp * N + m], lb[tok, grp * N:grp * N + m], KA, KB, q, 26, 1,
                                     np.arange(N))
            assert np.array_equal(ga[tok, grp], orc.modswitch(ea, q, 32)), (tok, grp)
            assert np.array_equal(gb[tok, grp], orc.modswitch(eb, q, 32)), (tok, grp)
            AS = orc.negacyclic_mul(ga[tok, grp], Sq, 1 << 32)
            ph = [(int(bv) - int(av)) % (1 << 32) for bv, av in zip(gb[tok, grp], AS)]
            got = [orc.decode(v, 1 << 32, t) for v in ph]
            want = [((int(v) + t // 2) % t) - t // 2 for v in y[tok, grp * N:grp * N + m]] + [0] * (N - m)
            assert got == want, (tok, grp)


def test_matmul_packed_token_chunks_agree(ctxs):
    # 8192 switched mask rows x N words x 4 B = 134 MB per token: the 2 GiB
    # scratch holds 15 tokens, cut to 12 (24 RLWEs, whole blocks of the
    # key contraction), so 19 tokens run as two chunks.
    import torch
    N, T = 4096, 19
    ctx = ctxs(N, "rns")
    q = synth.Q_RNS
    W = synth.weights(8192, 2048, seed=31)
    g = _rng(32)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    A = torch.tensor(g.integers(0, q, (T, 1, N), dtype=np.uint64).view(np.int64), device="cuda")
    B = torch.tensor(g.integers(0, q, (T, 1, N), dtype=np.uint64).view(np.int64), device="cuda")
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        oa = torch.empty((T, 2, N), dtype=torch.int32, device="cuda")
        ob = torch.empty_like(oa)
        phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, A, B, oa, ob)
        ra = torch.empty_like(oa)
        rb = torch.empty_like(oa)
        raw_m = torch.empty((1, 8192, N), dtype=torch.int64, device="cuda")
        raw_b = torch.empty((1, 8192), dtype=torch.int64, device="cuda")
        for tok in range(T):   # one token at a time, through the two public steps
            phe.phe_matmul(ctx, w, phe.PHE_FWD, 1, A[tok:tok + 1], B[tok:tok + 1], raw_m, raw_b, phe.PHE_OUT_RAW)
            phe.phe_pack(ctx, k, 1, 8192, raw_m, raw_b, ra[tok:tok + 1], rb[tok:tok + 1])
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    assert torch.equal(oa, ra) and torch.equal(ob, rb)


def test_ksk_upload_rejects_bad_shapes(ctxs):
    ctx = ctxs(256, "rns")
    K = np.zeros((256, 1, 256), dtype=np.uint64)
    for base_log, ell in [(0, 1), (31, 1), (17, 2), (8, 5)]:
        with pytest.raises(phe.PheError) as ei:
            phe.phe_ksk_upload(ctx, np.zeros((256, ell, 256), np.uint64), np.zeros((256, ell, 256), np.uint64),
                               base_log, ell)
        assert ei.value.status == phe.PHE_EINVAL
    with pytest.raises(phe.PheError):
        phe.phe_ksk_upload(ctx, K[:128], K[:128], 26, 1)   # n != N


def test_matmul_packed_host_buffers_match_device_call(ctxs):
    import torch
    N, T = 256, 5
    ctx = ctxs(N, "rns")
    q = synth.Q_RNS
    W = synth.weights(300, 290, seed=41)
    g = _rng(42)
    KA = g.integers(0, q, (N, 2, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 2, N), dtype=np.uint64)
    A = g.integers(0, q, (T, 2, N), dtype=np.uint64)
    B = g.integers(0, q, (T, 2, N), dtype=np.uint64)
    w = phe.phe_weights_upload(ctx, W)
    k = phe.phe_ksk_upload(ctx, KA, KB, 13, 2)
    try:
        oa = torch.empty((T, 2, N), dtype=torch.int32, device="cuda")
        ob = torch.empty_like(oa)
        phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, to_dev_u64(A), to_dev_u64(B), oa, ob)
        torch.cuda.synchronize()
        hA = torch.from_numpy(A.view(np.int64)).pin_memory()
        hB = torch.from_numpy(B.view(np.int64)).pin_memory()
        ha = torch.empty((T, 2, N), dtype=torch.int32).pin_memory()
        hb = torch.empty_like(ha).pin_memory()
        phe.phe_matmul_packed_host(ctx, w, k, phe.PHE_FWD, T, hA, hB, ha, hb, tok_chunk=2)
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    assert torch.equal(ha, oa.cpu()) and torch.equal(hb, ob.cpu())


def test_pack_largest_ring_and_empty_calls(orc, ctxs):
    """N = 8192 (the largest ring: the finishing kernel's exchange buffer is
    above 48 KB of shared memory), 100 rows, sampled against the oracle; and
    T = 0 / rows = 0 calls return without launching anything."""
    N, T, rows = 8192, 1, 100
    q = synth.Q_RNS
    ctx = ctxs(N, "rns")
    g = _rng(81)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    masks = g.integers(0, q, (T, rows, N), dtype=np.uint64)
    bodies = g.integers(0, q, (T, rows), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        ga, gb = _gpu_pack(ctx, k, masks, bodies, N, phe.PHE_OUT_RAW)
        phe.phe_pack(ctx, k, 0, rows, None, None, None, None)
        phe.phe_pack(ctx, k, 3, 0, None, None, None, None)
    finally:
        phe.phe_ksk_free(k)
    rs = np.array([0, 1, 99, 100, 4096, 8191])
    ea, eb = orc.pack_coeffs(masks[0], bodies[0], KA, KB, q, 26, 1, rs)
    assert np.array_equal(ga[0, 0, rs], ea) and np.array_equal(gb[0, 0, rs], eb)


@pytest.mark.parametrize("modulus", ["rns", "prime"])
def test_matmul_packed_seeded_matches_mask_form(orc, ctxs, modulus):
    import torch
    N, T = 256, 3
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    g = _rng(91)
    W = synth.weights(290, 300, seed=92)
    KA = g.integers(0, q, (N, 2, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 2, N), dtype=np.uint64)
    seeds = g.integers(0, 2 ** 64, (T, 2), dtype=np.uint64)
    A = orc.expand_masks(seeds, N, q)
    B = g.integers(0, q, (T, 2, N), dtype=np.uint64)
    w = phe.phe_weights_upload(ctx, W)
    k = phe.phe_ksk_upload(ctx, KA, KB, 13, 2)
    try:
        oa = torch.empty((T, 2, N), dtype=torch.int64, device="cuda")
        ob = torch.empty_like(oa)
        phe.phe_matmul_packed_seeded(ctx, w, k, phe.PHE_FWD, T, to_dev_u64(seeds), to_dev_u64(B), oa, ob,
                                     phe.PHE_OUT_RAW)
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    la, lb = orc.lwedot_all(W, A, B, q)
    for t in range(T):
        for grp in range(2):
            m = min(N, 290 - grp * N)
            ea, eb = orc.pack_coeffs(la[t, grp * N:grp * N + m], lb[t, grp * N:grp * N + m], KA, KB, q, 13, 2,
                                     np.arange(N))
            assert np.array_equal(oa[t, grp].cpu().numpy().view(np.uint64), ea), (t, grp)
            assert np.array_equal(ob[t, grp].cpu().numpy().view(np.uint64), eb), (t, grp)


def test_pack_rejects_unaligned_masks(ctxs):
    import torch
    N = 256
    q = synth.Q_RNS
    ctx = ctxs(N, "rns")
    g = _rng(95)
    k = phe.phe_ksk_upload(ctx, g.integers(0, q, (N, 1, N), dtype=np.uint64),
                           g.integers(0, q, (N, 1, N), dtype=np.uint64), 26, 1)
    try:
        buf = torch.zeros(N * 40 + 1, dtype=torch.int64, device="cuda")
        body = torch.zeros(40, dtype=torch.int64, device="cuda")
        oa = torch.empty((1, 1, N), dtype=torch.int32, device="cuda")
        with pytest.raises(phe.PheError) as ei:
            phe.phe_pack(ctx, k, 1, 40, buf[1:].data_ptr(), body, oa, torch.empty_like(oa))   # 8-byte offset
        assert ei.value.status == phe.PHE_EINVAL and "aligned" in str(ei.value)
    finally:
        phe.phe_ksk_free(k)


def _gpu_pack_dense(ctx, k, masks, bodies, N, flags):
    """phe_pack with PHE_PACK_DENSE: outputs [units][N]."""
    import torch
    T, rows = bodies.shape
    units, tpu = phe.phe_pack_layout(N, rows, T, flags | phe.PHE_PACK_DENSE)
    odt = torch.int64 if flags == phe.PHE_OUT_RAW else torch.int32
    oa = torch.empty((units, N), dtype=odt, device="cuda")
    ob = torch.empty((units, N), dtype=odt, device="cuda")
    phe.phe_pack(ctx, k, T, rows, to_dev_u64(masks), to_dev_u64(bodies), oa, ob, flags | phe.PHE_PACK_DENSE)
    torch.cuda.synchronize()
    if flags == phe.PHE_OUT_RAW:
        return tpu, oa.cpu().numpy().view(np.uint64), ob.cpu().numpy().view(np.uint64)
    return (tpu, oa.cpu().numpy().view(np.uint32).astype(np.uint64),
            ob.cpu().numpy().view(np.uint32).astype(np.uint64))


@pytest.mark.parametrize("modulus,base_log,ell", [("rns", 26, 1), ("prime", 13, 2), ("pow2", 26, 1)])
@pytest.mark.parametrize("rows,T", [(60, 7), (128, 3), (1, 300)])
def test_dense_pack_matches_oracle(orc, ctxs, modulus, base_log, ell, rows, T):
    """Dense packing: the LWE outputs of floor(N/rows) consecutive tokens form
    one list of Eq. (pack_rotate), token t's row r at coefficient
    (t mod tpu)*rows + r; the last RLWE holds the remaining tokens and zeros.
    rows = 60 at N = 256: 4 tokens (240 coefficients) per RLWE, 7 tokens ->
    2 RLWEs; rows = N/2: 2 per RLWE; rows = 1: 256 per RLWE, 300 tokens ->
    2 RLWEs, the second with 44 coefficients."""
    N = 256
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    g = _rng(200 + rows + ell)
    KA = g.integers(0, q, (N, ell, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, ell, N), dtype=np.uint64)
    masks = g.integers(0, q, (T, rows, N), dtype=np.uint64)
    bodies = g.integers(0, q, (T, rows), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, base_log, ell)
    try:
        tpu, raw_a, raw_b = _gpu_pack_dense(ctx, k, masks, bodies, N, phe.PHE_OUT_RAW)
        _, sw_a, sw_b = _gpu_pack_dense(ctx, k, masks, bodies, N, phe.PHE_OUT_SWITCHED)
    finally:
        phe.phe_ksk_free(k)
    assert tpu == N // rows
    units = -(-T // tpu)
    assert raw_a.shape == (units, N)
    flat_a = masks.reshape(T * rows, N)
    flat_b = bodies.reshape(T * rows)
    for u in range(units):
        f0, f1 = u * tpu * rows, min((u + 1) * tpu * rows, T * rows)
        ea, eb = orc.pack_coeffs(flat_a[f0:f1], flat_b[f0:f1], KA, KB, q, base_log, ell, np.arange(N))
        assert np.array_equal(raw_a[u], ea) and np.array_equal(raw_b[u], eb), u
        assert np.array_equal(sw_a[u], orc.modswitch(ea, q, 32)), u
        assert np.array_equal(sw_b[u], orc.modswitch(eb, q, 32)), u


def test_dense_flag_changes_nothing_above_half_ring(ctxs):
    # rows > N/2 (here 129 and 300 at N = 256): one token per RLWE either way
    import torch
    N, T = 256, 3
    ctx = ctxs(N, "rns")
    q = synth.Q_RNS
    g = _rng(211)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        for rows in (129, 300):
            masks = g.integers(0, q, (T, rows, N), dtype=np.uint64)
            bodies = g.integers(0, q, (T, rows), dtype=np.uint64)
            assert phe.phe_pack_layout(N, rows, T, phe.PHE_PACK_DENSE) == (T * -(-rows // N), 1)
            ref = _gpu_pack(ctx, k, masks, bodies, N, phe.PHE_OUT_SWITCHED)
            _, da, db = _gpu_pack_dense(ctx, k, masks, bodies, N, phe.PHE_OUT_SWITCHED)
            assert np.array_equal(da, ref[0].reshape(-1, N)) and np.array_equal(db, ref[1].reshape(-1, N))
    finally:
        phe.phe_ksk_free(k)


@pytest.mark.parametrize("modulus", ["rns", "prime"])
def test_matmul_packed_dense_end_to_end(orc, ctxs, modulus):
    """Eq. (LWEdot) then dense packing on real encryptions: 100 output rows at
    N = 256 put 2 tokens in each RLWE (5 tokens -> 3 RLWEs); word for word
    against the oracle composition, and every coefficient decrypts to its
    token's (W x)_r mod t (zeros past the last token)."""
    import torch
    N, T, t = 256, 5, synth.T_PLAIN
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    W = synth.weights(100, 290, seed=221)
    rows, cols = W.shape
    S, A, B, X = _encrypted_inputs(orc, N, T, cols, q, 222)
    g = _rng(223)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    E = np.rint(g.normal(0, synth.SIGMA, (N, 1, N))).astype(np.int64)
    KB = orc.ksk_encrypt(KA, E, S, S, q, 26, 1)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    units, tpu = phe.phe_pack_layout(N, rows, T, phe.PHE_PACK_DENSE)
    assert (units, tpu) == (3, 2)
    try:
        oa = torch.empty((units, N), dtype=torch.int32, device="cuda")
        ob = torch.empty((units, N), dtype=torch.int32, device="cuda")
        phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, to_dev_u64(A), to_dev_u64(B), oa, ob,
                              phe.PHE_PACK_DENSE)
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    ga = oa.cpu().numpy().view(np.uint32).astype(np.uint64)
    gb = ob.cpu().numpy().view(np.uint32).astype(np.uint64)
    la, lb = orc.lwedot_all(W, A, B, q)
    fa, fb = la.reshape(T * rows, N), lb.reshape(T * rows)
    y = (X.astype(np.int64) @ W.astype(np.int64).T).reshape(T * rows)
    Sq = np.array([s % (1 << 32) for s in S.tolist()], dtype=np.uint64)
    for u in range(units):
        f0, f1 = u * tpu * rows, min((u + 1) * tpu * rows, T * rows)
        ea, eb = orc.pack_coeffs(fa[f0:f1], fb[f0:f1], KA, KB, q, 26, 1, np.arange(N))
        assert np.array_equal(ga[u], orc.modswitch(ea, q, 32)), u
        assert np.array_equal(gb[u], orc.modswitch(eb, q, 32)), u
        AS = orc.negacyclic_mul(ga[u], Sq, 1 << 32)
        got = [orc.decode((int(bv) - int(av)) % (1 << 32), 1 << 32, t) for bv, av in zip(gb[u], AS)]
        want = [((int(v) + t // 2) % t) - t // 2 for v in y[f0:f1]] + [0] * (N - (f1 - f0))
        assert got == want, u


def test_matmul_packed_dense_chunks_and_host_buffers_agree(ctxs):
    """2048 rows at N = 4096: 2 tokens per RLWE.  67 tokens need two token
    chunks of the 2 GiB scratch (about 33.6 MB a token; the first cut to 48
    tokens: whole RLWEs, whole blocks of the key contraction); the result equals
    phe_matmul (raw) then phe_pack, both dense, and the host-buffer call with
    3-token chunks (rounded to 2)."""
    import torch
    N, T, rows = 4096, 67, 2048
    ctx = ctxs(N, "rns")
    q = synth.Q_RNS
    W = synth.weights(rows, 2048, seed=231)
    g = _rng(232)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    A = torch.tensor(g.integers(0, q, (T, 1, N), dtype=np.uint64).view(np.int64), device="cuda")
    B = torch.tensor(g.integers(0, q, (T, 1, N), dtype=np.uint64).view(np.int64), device="cuda")
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    units, tpu = phe.phe_pack_layout(N, rows, T, phe.PHE_PACK_DENSE)
    assert (units, tpu) == (34, 2)
    try:
        oa = torch.empty((units, N), dtype=torch.int32, device="cuda")
        ob = torch.empty_like(oa)
        phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, A, B, oa, ob, phe.PHE_PACK_DENSE)
        raw_m = torch.empty((T, rows, N), dtype=torch.int64, device="cuda")
        raw_b = torch.empty((T, rows), dtype=torch.int64, device="cuda")
        phe.phe_matmul(ctx, w, phe.PHE_FWD, T, A, B, raw_m, raw_b, phe.PHE_OUT_RAW)
        ra = torch.empty_like(oa)
        rb = torch.empty_like(oa)
        phe.phe_pack(ctx, k, T, rows, raw_m, raw_b, ra, rb, phe.PHE_PACK_DENSE)
        torch.cuda.synchronize()
        del raw_m, raw_b
        ha = torch.empty((units, N), dtype=torch.int32).pin_memory()
        hb = torch.empty_like(ha).pin_memory()
        phe.phe_matmul_packed_host(ctx, w, k, phe.PHE_FWD, T, A.cpu().pin_memory(), B.cpu().pin_memory(), ha, hb,
                                   phe.PHE_PACK_DENSE, tok_chunk=3)
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
    assert torch.equal(oa, ra) and torch.equal(ob, rb)
    assert torch.equal(ha, oa.cpu()) and torch.equal(hb, ob.cpu())


def test_dense_pack_full_size_sampled(orc, ctxs):
    """Dense packing at N = 4096: 512 rows put 8 tokens in each RLWE, so 9
    tokens make 2 RLWEs, the second holding one token and zeros.  Sampled
    coefficients on both sides of each token boundary, against the oracle's
    coefficient-by-coefficient evaluation of the concatenated LWE list."""
    N, T, rows = 4096, 9, 512
    q = synth.Q_RNS
    ctx = ctxs(N, "rns")
    g = _rng(241)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    masks = g.integers(0, q, (T, rows, N), dtype=np.uint64)
    bodies = g.integers(0, q, (T, rows), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        tpu, ga, gb = _gpu_pack_dense(ctx, k, masks, bodies, N, phe.PHE_OUT_SWITCHED)
    finally:
        phe.phe_ksk_free(k)
    assert tpu == 8 and ga.shape == (2, N)
    flat_a, flat_b = masks.reshape(T * rows, N), bodies.reshape(T * rows)
    for u, rs in ((0, [0, 1, 511, 512, 1023, 1024, 3583, 3584, 4095]), (1, [0, 255, 511, 512, 2048, 4095])):
        f0, f1 = u * tpu * rows, min((u + 1) * tpu * rows, T * rows)
        rs = np.array(rs)
        ea, eb = orc.pack_coeffs(flat_a[f0:f1], flat_b[f0:f1], KA, KB, q, 26, 1, rs)
        assert np.array_equal(ga[u, rs], orc.modswitch(ea, q, 32)), u
        assert np.array_equal(gb[u, rs], orc.modswitch(eb, q, 32)), u
