"""GPU: every entry point writes only its own output words and leaves its
inputs as they were.

With no sanitizer on the GPU, each output buffer sits between two guard
regions of 4096 words filled with a fixed pattern.  After the call the guards
must still hold the pattern and the inputs must be unchanged.  The shapes are
ragged: rows not a multiple of 128, columns not a multiple of 8, odd token
counts, a last RLWE only partly filled.  The outputs' values are checked
against the oracle by the parity tests; here only where the calls write.
"""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu

GUARD = 4096
MODULI = {"prime": (synth.Q60, None), "rns": (synth.Q_RNS, (synth.RNS_P1, synth.RNS_P2)),
          "pow2": (1 << 39, (synth.RNS_P1, synth.RNS_P2))}


class Guarded:
    """A device (or pinned host) tensor of `shape` between two guard regions."""

    def __init__(self, shape, dtype, device="cuda"):
        import torch
        n = int(np.prod(shape)) if len(shape) else 1
        self.base = torch.empty(n + 2 * GUARD, dtype=dtype, device=device)
        if device == "cpu":
            self.base = self.base.pin_memory()
        self.pattern = torch.tensor(0x5A5AA5A5, dtype=torch.int64).to(dtype)
        self.base.fill_(self.pattern.item())
        self.view = self.base[GUARD:GUARD + n].view(shape)

    def intact(self) -> bool:
        import torch
        torch.cuda.synchronize()
        return bool((self.base[:GUARD] == self.pattern.item()).all()) and \
            bool((self.base[-GUARD:] == self.pattern.item()).all())


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(N, modulus):
        key = (N, modulus)
        if key not in made:
            q, rns = MODULI[modulus]
            made[key] = phe.phe_ctx_create(N, q, 32 if modulus != "pow2" else 26, 0, rns=rns)
        return made[key]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _inputs(q, T, L, N, seed):
    g = _rng(seed)
    return to_dev_u64(g.integers(0, q, (T, L, N), dtype=np.uint64)), to_dev_u64(g.integers(0, q, (T, L, N),
                                                                                             dtype=np.uint64))


@pytest.mark.parametrize("modulus", ["rns", "prime", "pow2"])
@pytest.mark.parametrize("path", [phe.PHE_BODY_TENSOR, phe.PHE_BODY_FUSED])
@pytest.mark.parametrize("flags", [phe.PHE_OUT_SWITCHED, phe.PHE_OUT_RAW])
def test_matmul_writes_only_its_outputs(ctxs, modulus, path, flags):
    import torch
    N, T = 256, 5
    q = MODULI[modulus][0]
    ctx = ctxs(N, modulus)
    W = synth.weights(300, 290, seed=301)          # fwd: 300 rows of 290; bwd: 290 rows of 300
    w = phe.phe_weights_upload(ctx, W)
    phe.phe_ctx_set_body_path(ctx, path)
    odt = torch.int32 if flags == phe.PHE_OUT_SWITCHED else torch.int64
    try:
        for direction, rows, cols in ((phe.PHE_FWD, 300, 290), (phe.PHE_BWD, 290, 300)):
            L = synth.blocks(cols, N)
            A, B = _inputs(q, T, L, N, 302 + direction)
            A0, B0 = A.clone(), B.clone()
            om, ob = Guarded((T, rows, N), odt), Guarded((T, rows), odt)
            phe.phe_matmul(ctx, w, direction, T, A, B, om.view, ob.view, flags)
            assert om.intact() and ob.intact(), (direction, "output guards")
            assert torch.equal(A, A0) and torch.equal(B, B0), (direction, "inputs changed")
    finally:
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_AUTO)
        phe.phe_weights_free(w)


@pytest.mark.parametrize("tune", [(16, 3), (4, 0)])
def test_plan_writes_only_its_outputs(ctxs, tune):
    """Three products of uneven token counts in one plan (one of them with no
    tokens), persistent grid and one CTA per tile, run and graph-replayed."""
    import torch
    N = 256
    q = MODULI["rns"][0]
    ctx = ctxs(N, "rns")
    W1, W2 = synth.weights(300, 290, seed=311), synth.weights(130, 700, seed=312)
    w1, w2 = phe.phe_weights_upload(ctx, W1), phe.phe_weights_upload(ctx, W2)
    stream = torch.cuda.Stream()
    try:
        shapes = [(w1, phe.PHE_FWD, 7, 300, 290), (w2, phe.PHE_BWD, 3, 700, 130), (w2, phe.PHE_FWD, 0, 130, 700)]
        jobs, guards, ins = [], [], []
        for n, (w, d, T, rows, cols) in enumerate(shapes):
            A, B = _inputs(q, max(T, 1), synth.blocks(cols, N), N, 313 + n)
            om, ob = Guarded((max(T, 1), rows, N), torch.int32), Guarded((max(T, 1), rows), torch.int32)
            jobs.append((w, d, T, A, B, om.view, ob.view))
            guards += [om, ob]
            ins.append((A, A.clone(), B, B.clone()))
        plan = phe.phe_plan_create(ctx, jobs, phe.PHE_OUT_SWITCHED, tune)
        try:
            phe.phe_plan_run(plan, stream)
            phe.phe_plan_graph(plan, stream)
            phe.phe_plan_graph(plan, stream)
            stream.synchronize()
        finally:
            phe.phe_plan_destroy(plan)
        assert all(g.intact() for g in guards)
        # the product with no tokens writes nothing at all
        assert all(bool((g.base == g.pattern.item()).all()) for g in guards[4:])
        assert all(torch.equal(a, a0) and torch.equal(b, b0) for a, a0, b, b0 in ins)
    finally:
        phe.phe_weights_free(w1)
        phe.phe_weights_free(w2)


@pytest.mark.parametrize("flags", [phe.PHE_OUT_SWITCHED, phe.PHE_OUT_SWITCHED | phe.PHE_PACK_DENSE,
                                   phe.PHE_OUT_RAW])
def test_packing_writes_only_its_outputs(ctxs, flags):
    """phe_pack on given LWE ciphertexts and phe_matmul_packed, one RLWE per
    token or dense (60 rows at N = 256: 4 tokens per RLWE, 7 tokens leave the
    last RLWE with 3)."""
    import torch
    N, T = 256, 7
    q = MODULI["rns"][0]
    ctx = ctxs(N, "rns")
    g = _rng(321)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    W = synth.weights(60, 290, seed=322)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    odt = torch.int64 if flags & phe.PHE_OUT_RAW else torch.int32
    try:
        units, _ = phe.phe_pack_layout(N, 60, T, flags)
        masks = to_dev_u64(g.integers(0, q, (T, 60, N), dtype=np.uint64))
        bodies = to_dev_u64(g.integers(0, q, (T, 60), dtype=np.uint64))
        m0, b0 = masks.clone(), bodies.clone()
        oa, ob = Guarded((units, N), odt), Guarded((units, N), odt)
        phe.phe_pack(ctx, k, T, 60, masks, bodies, oa.view, ob.view, flags)
        assert oa.intact() and ob.intact(), "phe_pack guards"
        assert torch.equal(masks, m0) and torch.equal(bodies, b0), "phe_pack inputs changed"
        A, B = _inputs(q, T, synth.blocks(290, N), N, 323)
        A0, B0 = A.clone(), B.clone()
        oa, ob = Guarded((units, N), odt), Guarded((units, N), odt)
        phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, A, B, oa.view, ob.view, flags)
        assert oa.intact() and ob.intact(), "phe_matmul_packed guards"
        assert torch.equal(A, A0) and torch.equal(B, B0), "phe_matmul_packed inputs changed"
    finally:
        phe.phe_weights_free(w)
        phe.phe_ksk_free(k)


def test_noalloc_modswitch_and_wire_write_only_their_outputs(ctxs):
    import torch
    N, T = 256, 3
    q = MODULI["rns"][0]
    ctx = ctxs(N, "rns")
    W = synth.weights(300, 290, seed=331)
    w = phe.phe_weights_upload(ctx, W)
    g = _rng(332)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        # the allocation-free entry point
        A, B = _inputs(q, T, 2, N, 333)
        A0, B0 = A.clone(), B.clone()
        om, ob = Guarded((T, 300, N), torch.int32), Guarded((T, 300), torch.int32)
        phe.phe_matmul_noalloc(ctx, w, phe.PHE_FWD, T, A, B, om.view, ob.view)
        assert om.intact() and ob.intact() and torch.equal(A, A0) and torch.equal(B, B0)
        # the unfused switch of 1001 words
        words = to_dev_u64(g.integers(0, q, (1001,), dtype=np.uint64))
        w0 = words.clone()
        out = Guarded((1001,), torch.int32)
        phe.phe_modswitch(ctx, words, out.view, 1001)
        assert out.intact() and torch.equal(words, w0)
        # wire records in (T x L input records), LWE records and packed RLWE records out
        sizes = phe.phe_wire_sizes(ctx)
        L = 2
        rec = torch.randint(-(1 << 31), 1 << 31, (T * L * sizes["input"] // 4,), dtype=torch.int64,
                            device="cuda").to(torch.int32)
        r0 = rec.clone()
        for kk, n_out in ((None, T * 300 * sizes["lwe"]), (k, T * 2 * sizes["rlwe"])):
            out = Guarded((n_out // 4,), torch.int32)
            phe.phe_matmul_wire(ctx, w, kk, phe.PHE_FWD, T, rec, out.view)
            assert out.intact(), "wire guards"
            assert torch.equal(rec, r0), "wire input changed"
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)


def test_host_buffer_calls_write_only_their_outputs(ctxs):
    """phe_matmul_host and phe_matmul_packed_host (dense) write their pinned
    host outputs and nothing around them, chunk after chunk."""
    import torch
    N, T = 256, 5
    q = MODULI["rns"][0]
    ctx = ctxs(N, "rns")
    W = synth.weights(100, 290, seed=341)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    g = _rng(342)
    KA = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    KB = g.integers(0, q, (N, 1, N), dtype=np.uint64)
    k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
    try:
        hA = torch.from_numpy(g.integers(0, q, (T, 2, N), dtype=np.uint64).view(np.int64)).pin_memory()
        hB = torch.from_numpy(g.integers(0, q, (T, 2, N), dtype=np.uint64).view(np.int64)).pin_memory()
        A0, B0 = hA.clone(), hB.clone()
        om, ob = Guarded((T, 100, N), torch.int32, "cpu"), Guarded((T, 100), torch.int32, "cpu")
        phe.phe_matmul_host(ctx, w, phe.PHE_FWD, T, hA, hB, om.view, ob.view, phe.PHE_OUT_SWITCHED,
                            max_chunk_bytes=2 * 100 * N * 4)
        assert om.intact() and ob.intact()
        units, _ = phe.phe_pack_layout(N, 100, T, phe.PHE_PACK_DENSE)
        oa, obb = Guarded((units, N), torch.int32, "cpu"), Guarded((units, N), torch.int32, "cpu")
        phe.phe_matmul_packed_host(ctx, w, k, phe.PHE_FWD, T, hA, hB, oa.view, obb.view, phe.PHE_PACK_DENSE,
                                   tok_chunk=2)
        assert oa.intact() and obb.intact()
        assert torch.equal(hA, A0) and torch.equal(hB, B0)
    finally:
        phe.phe_ksk_free(k)
        phe.phe_weights_free(w)
