"""GPU: the RNS form of the hot path (q = p1 p2, two 30-bit NTT primes, 32-bit
residue arithmetic, CRT before the switch) against the 64-bit form on the
same q -- identical words -- and against the oracle, including decryption."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import gpu_matmul, to_dev_u64

pytestmark = pytest.mark.gpu
Q = synth.Q_RNS
RNS = (synth.RNS_P1, synth.RNS_P2)


@pytest.fixture(scope="module")
def ctxs():
    from paper_2505_07329_b300 import build
    build.build()
    made = {}

    def get(N, force64=False, k=32):
        key = (N, force64, k)
        if key not in made:
            made[key] = phe.phe_ctx_create(N, Q, k, 0, rns=RNS, flags=phe.PHE_CTX_FORCE_U64 if force64 else 0)
        return made[key]
    yield get
    for c in made.values():
        phe.phe_ctx_destroy(c)


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192])
def test_rns_form_equals_u64_form(ctxs, N):
    d_in, d_out, T = N + 77, 19, 5
    W = synth.weights(d_out, d_in, seed=N)
    L = synth.blocks(d_in, N)
    A = synth.uniform_words((T, L, N), Q, N)
    B = synth.uniform_words((T, L, N), Q, N + 1)
    outs = []
    for force64 in (False, True):
        ctx = ctxs(N, force64)
        w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
        try:
            raw = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out, phe.PHE_OUT_RAW)
            sw = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out)
            Lb = synth.blocks(d_out, N)
            bwd = gpu_matmul(ctx, w, phe.PHE_BWD, A[:, :Lb], B[:, :Lb], d_in)
            outs.append((raw, sw, bwd))
        finally:
            phe.phe_weights_free(w)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("k", [31, 26, 1])
def test_rns_switch_to_other_output_moduli(ctxs, k):
    # the RNS epilogue switches from the CRT digits in 32-bit arithmetic;
    # compare with the 64-bit form's switch (itself checked against the oracle)
    N, d_in, d_out, T = 1024, 1100, 33, 7
    W = synth.weights(d_out, d_in, seed=k)
    A = synth.uniform_words((T, 2, N), Q, 100 + k)
    B = synth.uniform_words((T, 2, N), Q, 200 + k)
    got = []
    for force64 in (False, True):
        ctx = ctxs(N, force64, k)
        w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
        try:
            got.append(gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out))
        finally:
            phe.phe_weights_free(w)
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])
    assert int(got[0][0].max()) < 2 ** k


def test_rns_matches_oracle_and_decrypts(orc, ctxs):
    N, d_in, d_out, T = 1024, 1500, 24, 6
    L = synth.blocks(d_in, N)
    W = synth.weights(d_out, d_in, seed=3)
    X = synth.activations(T, d_in, seed=4)
    S = synth.secret_key(N)
    A = synth.masks(T, L, N, Q, seed=5)
    E = synth.noise(T, L, N, seed=6)
    delta = Q // synth.T_PLAIN
    B = orc.encrypt_vectors(A, S, E, X, Q, delta)
    ctx = ctxs(N)
    w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
    try:
        ga, gb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out, phe.PHE_OUT_RAW)
        ea, eb = orc.lwedot_all(W, A, B, Q)
        assert np.array_equal(ga, ea) and np.array_equal(gb, eb)
        sa, sb = gpu_matmul(ctx, w, phe.PHE_FWD, A, B, d_out)
        assert np.array_equal(sa.astype(np.uint64), orc.modswitch(ea, Q, 32))
        assert np.array_equal(sb.astype(np.uint64), orc.modswitch(eb, Q, 32))
        Y = X.astype(np.int64) @ W.astype(np.int64).T
        for t in range(T):
            for j in (0, 11, d_out - 1):
                v = orc.lwe_phase(sa[t, j].astype(np.uint64), int(sb[t, j]), S, 2 ** 32)
                assert (orc.decode(v, 2 ** 32, synth.T_PLAIN) - int(Y[t, j])) % synth.T_PLAIN == 0
    finally:
        phe.phe_weights_free(w)


def test_rns_plan_seeded_and_noalloc_paths(ctxs):
    import torch
    N, d_in, d_out, T = 4096, 2048, 48, 9
    W = synth.weights(d_out, d_in, seed=7)
    seeds = synth.rng(8).integers(0, 2 ** 64, size=(T, 1), dtype=np.uint64)
    B = synth.uniform_words((T, 1, N), Q, 9)
    res = []
    for force64 in (False, True):
        ctx = ctxs(N, force64)
        w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
        try:
            dS, dB = to_dev_u64(seeds), to_dev_u64(B)
            dA = torch.empty((T, 1, N), dtype=torch.int64, device="cuda")
            phe.phe_expand_masks(ctx, dS, T, dA)
            outs = []
            for kind in ("seeded", "plan", "noalloc"):
                om = torch.empty((T, d_out, N), dtype=torch.int32, device="cuda")
                ob = torch.empty((T, d_out), dtype=torch.int32, device="cuda")
                if kind == "seeded":
                    phe.phe_matmul_seeded(ctx, w, phe.PHE_FWD, T, dS, dB, om, ob)
                elif kind == "plan":
                    plan = phe.phe_plan_create(ctx, [(w, phe.PHE_FWD, T, dA, dB, om, ob)])
                    phe.phe_plan_run(plan)
                    torch.cuda.synchronize()
                    phe.phe_plan_destroy(plan)
                else:
                    phe.phe_matmul_noalloc(ctx, w, phe.PHE_FWD, T, dA, dB, om, ob)
                torch.cuda.synchronize()
                outs.append((om.cpu(), ob.cpu()))
            res.append(outs)
        finally:
            phe.phe_weights_free(w)
    for k in range(3):
        for f in range(2):
            assert torch.equal(res[0][k][f], res[1][0][f])


@pytest.mark.parametrize("k", [32, 26, 7, 1])
def test_rns_modswitch_near_ties(orc, ctxs, k):
    # phe_modswitch on an RNS context runs the fused epilogue's residue-form
    # switch; words whose c 2^k lies within a few q of (m + 1/2) q sit next to
    # a rounding boundary, where a quotient estimate off by one would show
    import torch
    ctx = ctxs(1024, False, k)
    rng = np.random.Generator(np.random.PCG64(500 + k))
    cs = [0, 1, Q - 1, Q // 2, Q // 2 + 1, Q // 2 - 1, synth.RNS_P1, synth.RNS_P2, Q - synth.RNS_P1,
          synth.RNS_P1 * (synth.RNS_P2 - 1)]
    for m in rng.integers(0, 1 << k, 400, dtype=np.uint64):
        base = ((2 * int(m) + 1) * Q) >> (k + 1)
        cs += [(base + d) % Q for d in range(-3, 4)]
    cs += [int(x) for x in rng.integers(0, Q, 4000, dtype=np.uint64)]
    c = np.array(cs, dtype=np.uint64)
    d_in = torch.from_numpy(c.view(np.int64).copy()).cuda()
    d_out = torch.empty(c.shape[0], dtype=torch.int32, device="cuda")
    phe.phe_modswitch(ctx, d_in, d_out, c.shape[0])
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got, orc.modswitch(c, Q, k))
