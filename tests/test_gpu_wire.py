"""GPU: the wire format (Sec. 4.4 sizes, Sec. 4.5 bit-vector) against the
oracle's records, byte for byte.

  - phe_wire_pack equals the oracle's bit stream of the same fields;
  - phe_wire_unpack_inputs inverts the oracle's input records;
  - phe_matmul_wire at the paper's parameter set (N = 2048, q = 2^39,
    q_out = 2^26): 9992-byte input records in, LWE records out that unpack to
    the oracle's switched Eq. (LWEdot) outputs;
  - phe_matmul_wire with a key-switching key: RLWE records of 2N k-bit words
    equal to the packed phe_matmul_packed outputs.
"""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu
Q39 = 1 << 39


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(N, q, k):
        key = (N, q, k)
        if key not in made:
            rns = (synth.RNS_P1, synth.RNS_P2) if q in (Q39, synth.Q_RNS) else None
            made[key] = phe.phe_ctx_create(N, q, k, 0, rns=rns)
        return made[key]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _dev_bytes(n):
    import torch
    return torch.zeros(((n + 3) // 4,), dtype=torch.int32, device="cuda")


def _host_bytes(t, n):
    return t.cpu().numpy().view(np.uint8)[:n]


@pytest.mark.parametrize("k", [26, 32, 7])
def test_wire_pack_matches_oracle(orc, ctxs, k):
    import torch
    N = 256
    ctx = ctxs(N, synth.Q_RNS, k)
    g = _rng(k)
    n = 5
    a = g.integers(0, 1 << 32, (n, N), dtype=np.uint64).astype(np.uint32)
    b = g.integers(0, 1 << 32, (n, 1), dtype=np.uint64).astype(np.uint32)
    rec = phe.phe_wire_sizes(ctx)["lwe"]
    out = _dev_bytes(n * rec)
    phe.phe_wire_pack(ctx, torch.from_numpy(a.view(np.int32)).cuda(), N, torch.from_numpy(b.view(np.int32)).cuda(),
                      1, n, out)
    torch.cuda.synchronize()
    got = _host_bytes(out, n * rec)
    mask = (1 << k) - 1
    for r in range(n):
        fields = np.concatenate([a[r], b[r]]).astype(np.uint64) & np.uint64(mask)
        want = orc.pack_bits(fields, k)
        assert want.shape[0] == rec
        assert np.array_equal(got[r * rec:(r + 1) * rec], want), r


@pytest.mark.parametrize("q,bits", [(Q39, 39), (synth.Q_RNS, 60), (synth.Q60, 60)])
def test_wire_unpack_inverts_oracle_records(orc, ctxs, q, bits):
    import torch
    N = 256
    ctx = ctxs(N, q, 26)
    assert phe.phe_wire_sizes(ctx)["input"] == 8 + orc.wire_bytes(N, bits)
    g = _rng(bits)
    n = 6
    seeds = g.integers(0, 2 ** 64, n, dtype=np.uint64)
    B = g.integers(0, q, (n, N), dtype=np.uint64)
    B[0, :3] = [0, q - 1, 1]
    recs = np.concatenate([orc.wire_input_record(int(seeds[r]), B[r], bits) for r in range(n)])
    d_rec = torch.from_numpy(recs.view(np.int32).copy()).cuda()
    d_s = torch.empty(n, dtype=torch.int64, device="cuda")
    d_b = torch.empty((n, N), dtype=torch.int64, device="cuda")
    phe.phe_wire_unpack_inputs(ctx, d_rec, n, d_s, d_b)
    torch.cuda.synchronize()
    assert np.array_equal(d_s.cpu().numpy().view(np.uint64), seeds)
    assert np.array_equal(d_b.cpu().numpy().view(np.uint64), B)


def test_matmul_wire_paper_parameter_set(orc, ctxs):
    import torch
    N, k, T, d_in, d_out = 2048, 26, 2, 2500, 6      # L = 2 input records per token
    ctx = ctxs(N, Q39, k)
    sizes = phe.phe_wire_sizes(ctx)
    assert sizes["input"] == 9992 and sizes["rlwe"] == 13312      # the sizes printed in Sec. 4.4
    g = _rng(77)
    W = g.integers(-127, 128, (d_out, d_in)).astype(np.int8)
    L = synth.blocks(d_in, N)
    seeds = g.integers(0, 2 ** 64, (T, L), dtype=np.uint64)
    A = orc.expand_masks(seeds, N, Q39)
    B = g.integers(0, Q39, (T, L, N), dtype=np.uint64)
    recs = np.concatenate([orc.wire_input_record(int(seeds[t, i]), B[t, i], 39) for t in range(T) for i in range(L)])
    assert recs.shape[0] == T * L * 9992
    d_rec = torch.from_numpy(recs.view(np.int32).copy()).cuda()
    out = _dev_bytes(T * d_out * sizes["lwe"])
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        phe.phe_matmul_wire(ctx, w, None, phe.PHE_FWD, T, d_rec, out)
        torch.cuda.synchronize()
    finally:
        phe.phe_weights_free(w)
    got = _host_bytes(out, T * d_out * sizes["lwe"])
    assert sizes["lwe"] == orc.wire_bytes(N + 1, k)
    pairs = np.array([(0, 0), (1, d_out - 1), (1, 2)])
    ea, eb = orc.lwedot_pairs(W, A, B, pairs, Q39)
    for x, (t, j) in enumerate(pairs):
        r = t * d_out + j
        fields = orc.unpack_bits(got[r * sizes["lwe"]:(r + 1) * sizes["lwe"]], N + 1, k)
        assert np.array_equal(fields[:N], orc.modswitch(ea[x], Q39, k)), (t, j)
        assert fields[N] == orc.modswitch_one(int(eb[x]), Q39, k), (t, j)


def test_matmul_wire_packed_records_paper_modulus(orc, ctxs):
    # q = 2^39 -> 2^26 (the paper's moduli) with packing: seed + 39-bit body
    # records in, RLWE records of 2N 26-bit words out (13312 bytes at
    # N = 2048), equal to phe_matmul_packed's outputs bit-packed
    import torch
    N, k, T = 256, 26, 2
    ctx = ctxs(N, Q39, k)
    g = _rng(79)
    W = g.integers(-127, 128, (300, 290)).astype(np.int8)
    KA = g.integers(0, Q39, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, Q39, (N, 1, N), dtype=np.uint64)
    seeds = g.integers(0, 2 ** 64, (T, 2), dtype=np.uint64)
    A = orc.expand_masks(seeds, N, Q39)
    B = g.integers(0, Q39, (T, 2, N), dtype=np.uint64)
    recs = np.concatenate([orc.wire_input_record(int(seeds[t, i]), B[t, i], 39) for t in range(T) for i in range(2)])
    sizes = phe.phe_wire_sizes(ctx)
    assert sizes["rlwe"] == 2 * N * k // 8
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    kk = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        out = _dev_bytes(T * 2 * sizes["rlwe"])
        phe.phe_matmul_wire(ctx, w, kk, phe.PHE_FWD, T, torch.from_numpy(recs.view(np.int32).copy()).cuda(), out)
        oa = torch.empty((T, 2, N), dtype=torch.int32, device="cuda")
        ob = torch.empty_like(oa)
        phe.phe_matmul_packed(ctx, w, kk, phe.PHE_FWD, T, to_dev_u64(A), to_dev_u64(B), oa, ob)
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(kk)
        phe.phe_weights_free(w)
    got = _host_bytes(out, T * 2 * sizes["rlwe"])
    pa = oa.cpu().numpy().view(np.uint32).astype(np.uint64)
    pb = ob.cpu().numpy().view(np.uint32).astype(np.uint64)
    for t in range(T):
        for grp in range(2):
            r = t * 2 + grp
            want = orc.pack_bits(np.concatenate([pa[t, grp], pb[t, grp]]), k)
            assert np.array_equal(got[r * sizes["rlwe"]:(r + 1) * sizes["rlwe"]], want), (t, grp)


def test_matmul_wire_packed_records(orc, ctxs):
    import torch
    N, k, T = 256, 26, 3
    q = synth.Q_RNS
    ctx = ctxs(N, q, k)
    g = _rng(78)
    W = g.integers(-127, 128, (300, 290)).astype(np.int8)     # rows 300: two RLWE records per token
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    seeds = g.integers(0, 2 ** 64, (T, 2), dtype=np.uint64)
    A = orc.expand_masks(seeds, N, q)
    B = g.integers(0, q, (T, 2, N), dtype=np.uint64)
    recs = np.concatenate([orc.wire_input_record(int(seeds[t, i]), B[t, i], 60) for t in range(T) for i in range(2)])
    sizes = phe.phe_wire_sizes(ctx)
    assert sizes["rlwe"] == 2 * N * k // 8
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    kk = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        out = _dev_bytes(T * 2 * sizes["rlwe"])
        phe.phe_matmul_wire(ctx, w, kk, phe.PHE_FWD, T, torch.from_numpy(recs.view(np.int32).copy()).cuda(), out)
        oa = torch.empty((T, 2, N), dtype=torch.int32, device="cuda")
        ob = torch.empty_like(oa)
        phe.phe_matmul_packed(ctx, w, kk, phe.PHE_FWD, T, to_dev_u64(A), to_dev_u64(B), oa, ob)
        torch.cuda.synchronize()
    finally:
        phe.phe_ksk_free(kk)
        phe.phe_weights_free(w)
    got = _host_bytes(out, T * 2 * sizes["rlwe"])
    pa = oa.cpu().numpy().view(np.uint32).astype(np.uint64)
    pb = ob.cpu().numpy().view(np.uint32).astype(np.uint64)
    for t in range(T):
        for grp in range(2):
            r = t * 2 + grp
            want = orc.pack_bits(np.concatenate([pa[t, grp], pb[t, grp]]), k)
            assert np.array_equal(got[r * sizes["rlwe"]:(r + 1) * sizes["rlwe"]], want), (t, grp)
