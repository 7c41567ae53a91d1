"""GPU: seeded inputs (Sec. 3.1, masks regenerated from a 64-bit seed per
ciphertext).  The GPU keystream expansion matches the oracle's ChaCha20
reading, and the seeded product -- per call, in a plan and in the server --
matches the oracle on the expanded masks, bit for bit."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu
Q = synth.Q60


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(N):
        if N not in made:
            made[N] = phe.phe_ctx_create(N, Q, 32, 0)
        return made[N]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


def _seeds(shape, seed):
    return synth.rng(seed).integers(0, 2 ** 64, size=shape, dtype=np.uint64)


@pytest.mark.parametrize("N", [256, 1024, 4096])
def test_mask_expansion_matches_oracle(orc, ctxs, N):
    import torch
    seeds = _seeds(7, N)
    seeds[0] = 0
    seeds[1] = 2 ** 64 - 1
    out = torch.empty((7, N), dtype=torch.int64, device="cuda")
    phe.phe_expand_masks(ctxs(N), to_dev_u64(seeds), 7, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), orc.expand_masks(seeds, N, Q))


@pytest.mark.parametrize("N,d_in,d_out,T", [(256, 300, 37, 19), (4096, 2048, 16, 3)])
def test_seeded_product_matches_oracle(orc, ctxs, N, d_in, d_out, T):
    import torch
    ctx = ctxs(N)
    W = synth.weights(d_out, d_in, seed=N)
    L = synth.blocks(d_in, N)
    seeds = _seeds((T, L), 77 + N)
    A = orc.expand_masks(seeds, N, Q)
    B = synth.uniform_words((T, L, N), Q, 5)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        for flags in (phe.PHE_OUT_RAW, phe.PHE_OUT_SWITCHED):
            odt = torch.int64 if flags == phe.PHE_OUT_RAW else torch.int32
            om = torch.empty((T, d_out, N), dtype=odt, device="cuda")
            ob = torch.empty((T, d_out), dtype=odt, device="cuda")
            phe.phe_matmul_seeded(ctx, w, phe.PHE_FWD, T, to_dev_u64(seeds), to_dev_u64(B), om, ob, flags)
            torch.cuda.synchronize()
            if N <= 1024:
                ea, eb = orc.lwedot_all(W, A, B, Q)
                got_a, got_b = om.cpu().numpy(), ob.cpu().numpy()
            else:  # sampled outputs at N = 4096
                pairs = np.array([(0, 0), (T - 1, d_out - 1), (1, 7)])
                ea, eb = orc.lwedot_pairs(W, A, B, pairs, Q, method=1)
                got_a = np.stack([om[t, j].cpu().numpy() for t, j in pairs])
                got_b = np.array([ob[t, j].item() for t, j in pairs])
            if flags == phe.PHE_OUT_SWITCHED:
                ea, eb = orc.modswitch(ea, Q, 32), orc.modswitch(eb, Q, 32)
                got_a = got_a.view(np.uint32).astype(np.uint64)
                got_b = (got_b.astype(np.int64) & 0xffffffff).astype(np.uint64)
            else:
                got_a = got_a.view(np.uint64)
                got_b = got_b.astype(np.int64).view(np.uint64)
            assert np.array_equal(got_a, ea) and np.array_equal(got_b.reshape(eb.shape), eb)
    finally:
        phe.phe_weights_free(w)


def test_seeded_plan_and_server_match_the_mask_form(ctxs):
    import torch
    N = 1024
    ctx = ctxs(N)
    W = synth.weights(40, 1500, seed=3)
    L = synth.blocks(1500, N)
    T = 13
    seeds = _seeds((T, L), 9)
    dS = to_dev_u64(seeds)
    dA = torch.empty((T, L, N), dtype=torch.int64, device="cuda")
    phe.phe_expand_masks(ctx, dS, T * L, dA)
    dB = to_dev_u64(synth.uniform_words((T, L, N), Q, 10))
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        ref_m = torch.empty((T, 40, N), dtype=torch.int32, device="cuda")
        ref_b = torch.empty((T, 40), dtype=torch.int32, device="cuda")
        phe.phe_matmul(ctx, w, phe.PHE_FWD, T, dA, dB, ref_m, ref_b)
        pm, pb = torch.empty_like(ref_m), torch.empty_like(ref_b)
        plan = phe.phe_plan_create(ctx, [(w, phe.PHE_FWD, T, None, dB, pm, pb, dS)])
        phe.phe_plan_run(plan)
        torch.cuda.synchronize()
        phe.phe_plan_destroy(plan)
        assert torch.equal(pm, ref_m) and torch.equal(pb, ref_b)
        hm = torch.empty((T, 40, N), dtype=torch.int32).pin_memory()
        hb = torch.empty((T, 40), dtype=torch.int32).pin_memory()
        srv = phe.phe_server_create(ctx, 1 << 28, chunk_tokens=4)
        try:
            phe.phe_server_wait(srv, phe.phe_server_submit(srv, w, phe.PHE_FWD, T, None, dB, hm, hb, in_seeds=dS))
        finally:
            phe.phe_server_destroy(srv)
        assert torch.equal(hm, ref_m.cpu()) and torch.equal(hb, ref_b.cpu())
    finally:
        phe.phe_weights_free(w)
