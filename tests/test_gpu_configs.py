"""GPU: parity at the workload shapes the benchmark and the model step use,
on sampled outputs the oracle computes one by one (RNS modulus, the
benchmark's form).

  - one Llama-3.2-1B layer: all seven projections, forward and backward, in
    one autotuned plan replayed from a CUDA graph (the benchmark's launch
    configuration, on a 32-token chunk);
  - the 16-layer step: all 16 layers' weights resident at once, a batch of 8
    sequences with uneven token counts drawn like the model workload's
    (U{64..2048}, scaled down 128x to keep the outputs in memory), one plan
    per layer over every projection, direction and sequence.
"""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu
N = 4096
Q = synth.Q_RNS


@pytest.fixture(scope="module")
def ctx():
    from paper_2505_07329_b300 import build
    build.build()
    c = phe.phe_ctx_create(N, Q, 32, 0, rns=(synth.RNS_P1, synth.RNS_P2))
    yield c
    phe.phe_ctx_destroy(c)


def _products():
    out = []
    for d in (phe.PHE_FWD, phe.PHE_BWD):
        for pi, (name, d_in, d_out) in enumerate(synth.LLAMA_PROJECTIONS):
            rows, cols = (d_out, d_in) if d == phe.PHE_FWD else (d_in, d_out)
            out.append((pi, d, rows, cols, synth.blocks(cols, N)))
    return out


def _check_samples(orc, W, d, A, B, om, ob, samples):
    Wd = W if d == phe.PHE_FWD else np.ascontiguousarray(W.T)
    pairs = np.array(samples)
    ea, eb = orc.lwedot_pairs(Wd, A, B, pairs, Q)
    for x, (t, j) in enumerate(pairs):
        got_a = om[t, j].cpu().numpy().view(np.uint32).astype(np.uint64)
        got_b = int(ob[t, j].item()) & 0xffffffff
        assert np.array_equal(got_a, orc.modswitch(ea[x], Q, 32)), (t, j)
        assert got_b == orc.modswitch_one(int(eb[x]), Q, 32), (t, j)


def test_layer_config_one_graph_plan(orc, ctx):
    import torch
    T = 32
    prods = _products()
    Ws = [synth.weights(d_out, d_in, seed=synth.SEED_W + pi)
          for pi, (_, d_in, d_out) in enumerate(synth.LLAMA_PROJECTIONS)]
    ws = [phe.phe_weights_upload(ctx, W) for W in Ws]
    try:
        jobs, host, outs = [], [], []
        for n, (pi, d, rows, cols, L) in enumerate(prods):
            A = synth.uniform_words((T, L, N), Q, 1000 + n)
            B = synth.uniform_words((T, L, N), Q, 2000 + n)
            om = torch.empty((T, rows, N), dtype=torch.int32, device="cuda")
            ob = torch.empty((T, rows), dtype=torch.int32, device="cuda")
            jobs.append((ws[pi], d, T, to_dev_u64(A), to_dev_u64(B), om, ob))
            host.append((A, B))
            outs.append((om, ob))
        stream = torch.cuda.Stream()
        tune, _ = phe.phe_autotune(ctx, jobs, phe.PHE_OUT_SWITCHED, 32, stream)
        plan = phe.phe_plan_create(ctx, jobs, phe.PHE_OUT_SWITCHED, tune)
        try:
            phe.phe_plan_graph(plan, stream)
            phe.phe_plan_graph(plan, stream)   # a replay of the captured graph
            torch.cuda.synchronize()
        finally:
            phe.phe_plan_destroy(plan)
        for n, (pi, d, rows, cols, L) in enumerate(prods):
            A, B = host[n]
            om, ob = outs[n]
            _check_samples(orc, Ws[pi], d, A, B, om, ob, [(0, 0), (T - 1, rows - 1), (T // 2, rows // 3)])
    finally:
        for w in ws:
            phe.phe_weights_free(w)
        outs = jobs = None
        torch.cuda.empty_cache()


def test_model_config_sixteen_layers_uneven_tokens(orc, ctx):
    import torch
    wl = synth.WORKLOADS["model"]
    layers = wl.extra["layers"]
    counts = [max(1, int(c) // 128) for c in synth.model_token_counts()]   # 8 sequences
    prods = _products()
    # every layer's weights resident at once (16 x 7 projections, both directions)
    Ws, ws = [], []
    for layer in range(layers):
        Ws.append([synth.weights(d_out, d_in, seed=synth.SEED_W + 100 * layer + pi)
                   for pi, (_, d_in, d_out) in enumerate(synth.LLAMA_PROJECTIONS)])
        ws.append([phe.phe_weights_upload(ctx, W) for W in Ws[-1]])
    try:
        Tmax = max(counts)
        outs = {(n, s): (torch.empty((counts[s], rows, N), dtype=torch.int32, device="cuda"),
                         torch.empty((counts[s], rows), dtype=torch.int32, device="cuda"))
                for n, (pi, d, rows, cols, L) in enumerate(prods) for s in range(len(counts))}
        stream = torch.cuda.Stream()
        for layer in range(layers):
            jobs, host = [], {}
            for n, (pi, d, rows, cols, L) in enumerate(prods):
                for s, T in enumerate(counts):
                    A = synth.uniform_words((T, L, N), Q, 10 ** 6 + 1000 * layer + 50 * n + s)
                    B = synth.uniform_words((T, L, N), Q, 2 * 10 ** 6 + 1000 * layer + 50 * n + s)
                    om, ob = outs[(n, s)]
                    jobs.append((ws[layer][pi], d, T, to_dev_u64(A), to_dev_u64(B), om, ob))
                    host[(n, s)] = (A, B)
            plan = phe.phe_plan_create(ctx, jobs, phe.PHE_OUT_SWITCHED, (8, 0))
            try:
                phe.phe_plan_run(plan, stream)
                torch.cuda.synchronize()
            finally:
                phe.phe_plan_destroy(plan)
            # two sampled outputs per layer, rotating over products and sequences
            for k in range(2):
                n = (3 * layer + 5 * k) % len(prods)
                s = (layer + k) % len(counts)
                pi, d, rows, cols, L = prods[n]
                A, B = host[(n, s)]
                om, ob = outs[(n, s)]
                _check_samples(orc, Ws[layer][pi], d, A, B, om, ob, [(counts[s] - 1, (7 * layer + k) % rows)])
        assert Tmax >= 1
    finally:
        for layer_ws in ws:
            for w in layer_ws:
                phe.phe_weights_free(w)
        outs = None
        torch.cuda.empty_cache()


def test_model_sequence_at_full_length(orc, ctx):
    # the longest sequence the model workload draws, at its full length, cut
    # into the model step's 128-token calls (the last one ragged), for three
    # products with one and two input blocks; every call's outputs are
    # sampled before the next call overwrites them
    import torch
    counts = [int(c) for c in synth.model_token_counts()]
    T = max(counts)
    chunk = 128
    picks = [(0, phe.PHE_FWD), (6, phe.PHE_FWD), (4, phe.PHE_BWD)]   # q fwd, down fwd (L=2), gate bwd (L=2)
    for k, (pi, d) in enumerate(picks):
        _, d_in, d_out = synth.LLAMA_PROJECTIONS[pi]
        W = synth.weights(d_out, d_in, seed=synth.SEED_W + 700 + pi)
        rows, cols = (d_out, d_in) if d == phe.PHE_FWD else (d_in, d_out)
        L = synth.blocks(cols, N)
        A = synth.uniform_words((T, L, N), Q, 3 * 10 ** 6 + k)
        B = synth.uniform_words((T, L, N), Q, 4 * 10 ** 6 + k)
        dA, dB = to_dev_u64(A), to_dev_u64(B)
        w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT if d == phe.PHE_FWD else phe.PHE_DIR_BWD_BIT)
        om = torch.empty((chunk, rows, N), dtype=torch.int32, device="cuda")
        ob = torch.empty((chunk, rows), dtype=torch.int32, device="cuda")
        try:
            got, pairs = [], []
            for c, t0 in enumerate(range(0, T, chunk)):
                tn = min(chunk, T - t0)
                phe.phe_matmul(ctx, w, d, tn, dA[t0:t0 + tn], dB[t0:t0 + tn], om, ob)
                torch.cuda.synchronize()
                for t, j in ((tn - 1, (37 * c) % rows), (tn // 2, rows - 1 - (11 * c) % rows)):
                    got.append((om[t, j].cpu().numpy().view(np.uint32).astype(np.uint64),
                                int(ob[t, j].item()) & 0xffffffff))
                    pairs.append((t0 + t, j))
            assert phe.phe_ctx_status(ctx) == 0
        finally:
            phe.phe_weights_free(w)
        Wd = W if d == phe.PHE_FWD else np.ascontiguousarray(W.T)
        ea, eb = orc.lwedot_pairs(Wd, A, B, np.array(pairs), Q)
        for x, (ga, gb) in enumerate(got):
            assert np.array_equal(ga, orc.modswitch(ea[x], Q, 32)), (pi, d, pairs[x])
            assert gb == orc.modswitch_one(int(eb[x]), Q, 32), (pi, d, pairs[x])
    assert T >= 1024  # the drawn batch has a long sequence
