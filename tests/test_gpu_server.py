"""GPU: the served form (continuous batching).  A request's results are the
same alone and in a mix of concurrently admitted requests from other
projections and directions (integer results: bit for bit), equal the
per-call path's, and match the CPU oracle on sampled outputs."""
import time

import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import gpu_matmul, to_dev_u64

pytestmark = pytest.mark.gpu
Q = synth.Q60
N = 1024


@pytest.fixture(scope="module")
def env():
    from paper_2505_07329_b300 import build
    build.build()
    ctx = phe.phe_ctx_create(N, Q, 32, 0)
    Ws = [synth.weights(64, 300, seed=1), synth.weights(200, 1500, seed=2), synth.weights(50, 100, seed=3)]
    ws = [phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT) for W in Ws]
    yield ctx, Ws, ws
    for w in ws:
        phe.phe_weights_free(w)
    phe.phe_ctx_destroy(ctx)


def _request(Ws, ws, pi, direction, T, seed):
    import torch
    W = Ws[pi] if direction == phe.PHE_FWD else np.ascontiguousarray(Ws[pi].T)
    rows, cols = W.shape
    L = synth.blocks(cols, N)
    A = synth.uniform_words((T, L, N), Q, seed)
    B = synth.uniform_words((T, L, N), Q, seed + 1)
    hm = torch.full((T, rows, N), -1, dtype=torch.int32).pin_memory()
    hb = torch.full((T, rows), -1, dtype=torch.int32).pin_memory()
    return dict(pi=pi, dir=direction, T=T, W=W, A=A, B=B, dA=to_dev_u64(A), dB=to_dev_u64(B), hm=hm, hb=hb)


def _submit(srv, ws, r):
    return phe.phe_server_submit(srv, ws[r["pi"]], r["dir"], r["T"], r["dA"], r["dB"], r["hm"], r["hb"])


def _result(r):
    return r["hm"].numpy().view(np.uint32).copy(), r["hb"].numpy().view(np.uint32).copy()


def test_same_result_alone_and_in_the_mix(orc, env):
    ctx, Ws, ws = env
    budget = 256 << 20
    # alone
    R = _request(Ws, ws, 1, phe.PHE_FWD, 23, seed=10)
    srv = phe.phe_server_create(ctx, budget, chunk_tokens=4)
    try:
        phe.phe_server_wait(srv, _submit(srv, ws, R), 60000)
    finally:
        phe.phe_server_destroy(srv)
    alone = _result(R)
    # in a mix: the same request again plus six others, some arriving while
    # the first ones are on the GPU
    R2 = dict(R)
    import torch
    R2["hm"] = torch.full_like(R["hm"], -1).pin_memory()
    R2["hb"] = torch.full_like(R["hb"], -1).pin_memory()
    others = [_request(Ws, ws, 0, phe.PHE_FWD, 17, 20), _request(Ws, ws, 2, phe.PHE_BWD, 9, 30),
              _request(Ws, ws, 1, phe.PHE_BWD, 31, 40), _request(Ws, ws, 0, phe.PHE_BWD, 5, 50),
              _request(Ws, ws, 2, phe.PHE_FWD, 40, 60), _request(Ws, ws, 1, phe.PHE_FWD, 12, 70)]
    srv = phe.phe_server_create(ctx, budget, chunk_tokens=4)
    try:
        ids = [_submit(srv, ws, others[0]), _submit(srv, ws, others[1])]
        ids.append(_submit(srv, ws, R2))
        time.sleep(0.002)
        ids += [_submit(srv, ws, o) for o in others[2:]]
        for i in ids:
            phe.phe_server_wait(srv, i, 60000)
        st = phe.phe_server_stats(srv)
        assert st["completed"] == 7 and st["failed"] == 0
        assert st["peak_reserved_bytes"] <= budget
        assert st["iterations"] >= 2
    finally:
        phe.phe_server_destroy(srv)
    mixed = _result(R2)
    assert np.array_equal(mixed[0], alone[0]) and np.array_equal(mixed[1], alone[1])
    # every request equals the per-call path on the same inputs
    for r in [R] + others:
        ga, gb = gpu_matmul(ctx, ws[r["pi"]], r["dir"], r["A"], r["B"], r["W"].shape[0])
        got = _result(r) if r is not R else alone
        assert np.array_equal(got[0], ga) and np.array_equal(got[1], gb)
    # and the oracle on sampled outputs of R
    rng = np.random.default_rng(3)
    pairs = np.stack([rng.integers(0, R["T"], 24), rng.integers(0, R["W"].shape[0], 24)], axis=1)
    ea, eb = orc.lwedot_pairs(R["W"], R["A"], R["B"], pairs, Q)
    for n, (t, j) in enumerate(pairs):
        assert np.array_equal(alone[0][t, j].astype(np.uint64), orc.modswitch(ea[n], Q, 32))
        assert int(alone[1][t, j]) == int(orc.modswitch(eb[n:n + 1], Q, 32)[0])


def test_tight_budget_serialises_but_completes(env):
    ctx, Ws, ws = env
    r = _request(Ws, ws, 1, phe.PHE_FWD, 16, seed=90)
    # room for exactly one 4-token chunk of this request: transformed masks
    # (L = 2), mask and body outputs, and the bodies' bf16 digit rows (8 per
    # token, 1500 columns)
    one = 4 * 2 * N * 8 + 4 * 200 * N * 4 + 4 * 200 * 4 + 4 * 8 * 1504 * 2
    srv = phe.phe_server_create(ctx, one, chunk_tokens=4)
    try:
        phe.phe_server_wait(srv, _submit(srv, ws, r), 60000)
        st = phe.phe_server_stats(srv)
        assert st["peak_reserved_bytes"] == one and st["iterations"] == 4
    finally:
        phe.phe_server_destroy(srv)
    ga, gb = gpu_matmul(ctx, ws[1], phe.PHE_FWD, r["A"], r["B"], 200)
    got = _result(r)
    assert np.array_equal(got[0], ga) and np.array_equal(got[1], gb)


@pytest.mark.parametrize("q,rns,Nr", [(synth.Q_RNS, (synth.RNS_P1, synth.RNS_P2), 1024),
                                      (1 << 39, (synth.RNS_P1, synth.RNS_P2), 2048)])
def test_served_and_batched_forms_for_the_rns_and_power_of_two_moduli(q, rns, Nr):
    """The served form and a plan, with the benchmark's RNS modulus and with
    the paper's q = 2^39, equal the per-call path word for word."""
    import torch
    ctx = phe.phe_ctx_create(Nr, q, 26 if q == 1 << 39 else 32, 0, rns=rns)
    Ws = [synth.weights(70, 2100, seed=11), synth.weights(300, 500, seed=12)]
    ws = [phe.phe_weights_upload(ctx, W) for W in Ws]
    try:
        reqs = []
        for n, (pi, d, T) in enumerate([(0, phe.PHE_FWD, 9), (1, phe.PHE_BWD, 5), (1, phe.PHE_FWD, 13)]):
            W = Ws[pi] if d == phe.PHE_FWD else np.ascontiguousarray(Ws[pi].T)
            rows, cols = W.shape
            L = synth.blocks(cols, Nr)
            A = synth.uniform_words((T, L, Nr), q, 40 + n)
            B = synth.uniform_words((T, L, Nr), q, 60 + n)
            ref_m = torch.empty((T, rows, Nr), dtype=torch.int32, device="cuda")
            ref_b = torch.empty((T, rows), dtype=torch.int32, device="cuda")
            dA, dB = to_dev_u64(A), to_dev_u64(B)
            phe.phe_matmul(ctx, ws[pi], d, T, dA, dB, ref_m, ref_b)
            hm = torch.full((T, rows, Nr), -1, dtype=torch.int32).pin_memory()
            hb = torch.full((T, rows), -1, dtype=torch.int32).pin_memory()
            pm, pb = torch.empty_like(ref_m), torch.empty_like(ref_b)
            reqs.append(dict(pi=pi, d=d, T=T, dA=dA, dB=dB, ref=(ref_m, ref_b), host=(hm, hb), plan=(pm, pb)))
        torch.cuda.synchronize()
        srv = phe.phe_server_create(ctx, 1 << 30, chunk_tokens=4, tok_chunk=2)
        try:
            ids = [phe.phe_server_submit(srv, ws[r["pi"]], r["d"], r["T"], r["dA"], r["dB"], *r["host"]) for r in reqs]
            for i in ids:
                phe.phe_server_wait(srv, i, 120000)
        finally:
            phe.phe_server_destroy(srv)
        plan = phe.phe_plan_create(ctx, [(ws[r["pi"]], r["d"], r["T"], r["dA"], r["dB"], *r["plan"]) for r in reqs],
                                   phe.PHE_OUT_SWITCHED, (2, 0))
        try:
            phe.phe_plan_run(plan)
            torch.cuda.synchronize()
        finally:
            phe.phe_plan_destroy(plan)
        for r in reqs:
            assert torch.equal(r["host"][0], r["ref"][0].cpu()) and torch.equal(r["host"][1], r["ref"][1].cpu())
            assert torch.equal(r["plan"][0], r["ref"][0]) and torch.equal(r["plan"][1], r["ref"][1])
    finally:
        for w in ws:
            phe.phe_weights_free(w)
        phe.phe_ctx_destroy(ctx)


def test_persistent_grid_serves_the_same_words(env):
    # one CTA per SM walking the iteration's tiles from a counter: the same
    # words as the per-call path, for two requests of different shapes
    ctx, Ws, ws = env
    reqs = [_request(Ws, ws, 1, phe.PHE_FWD, 13, seed=70), _request(Ws, ws, 0, phe.PHE_BWD, 9, seed=71)]
    srv = phe.phe_server_create(ctx, 256 << 20, chunk_tokens=4, tok_chunk=2, blocks_per_sm=1)
    try:
        ids = [_submit(srv, ws, r) for r in reqs]
        for i in ids:
            phe.phe_server_wait(srv, i, 60000)
    finally:
        phe.phe_server_destroy(srv)
    for r in reqs:
        rows = r["W"].shape[0]
        ga, gb = gpu_matmul(ctx, ws[r["pi"]], r["dir"], r["A"], r["B"], rows)
        got = _result(r)
        assert np.array_equal(got[0], ga) and np.array_equal(got[1], gb)
