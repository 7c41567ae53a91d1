"""GPU: the batched form (plans, CUDA-graph replay, autotuner) against the CPU
oracle, bit for bit.  Jobs have uneven token counts, shared inputs (several
products of one encrypted x) and both directions."""
import numpy as np
import pytest

import synth
from paper_2505_07329_b300 import phe
from tests.gpu_helpers import to_dev_u64

pytestmark = pytest.mark.gpu
Q = synth.Q60
N = 256


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2505_07329_b300 import build
    build.build()
    ctx = phe.phe_ctx_create(N, Q, 32, 0)
    # three "projections" sharing d_in = 300 (L = 2), like q/k/v of one x
    shapes = [(37, 300), (129, 300), (5, 300), (300, 70)]
    Ws = [synth.weights(do, di, seed=10 + i) for i, (do, di) in enumerate(shapes)]
    ws = [phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT) for W in Ws]
    stream = torch.cuda.Stream()
    yield ctx, Ws, ws, stream
    for w in ws:
        phe.phe_weights_free(w)
    phe.phe_ctx_destroy(ctx)


def _make_jobs(Ws, ws, flags, seed):
    """Jobs: fwd products 0,1,2 share one input x (T=19); bwd of product 1
    (T=7); fwd of product 3 (T=33); a skipped job (T=0)."""
    import torch
    odt = torch.int32 if flags == phe.PHE_OUT_SWITCHED else torch.int64
    T_x, T_g, T_3 = 19, 7, 33
    Ax = synth.uniform_words((T_x, 2, N), Q, seed)
    Bx = synth.uniform_words((T_x, 2, N), Q, seed + 1)
    Ag = synth.uniform_words((T_g, 1, N), Q, seed + 2)
    Bg = synth.uniform_words((T_g, 1, N), Q, seed + 3)
    A3 = synth.uniform_words((T_3, 1, N), Q, seed + 4)
    B3 = synth.uniform_words((T_3, 1, N), Q, seed + 5)
    dev = {k: to_dev_u64(v) for k, v in dict(Ax=Ax, Bx=Bx, Ag=Ag, Bg=Bg, A3=A3, B3=B3).items()}
    specs = [(0, phe.PHE_FWD, T_x, "Ax", "Bx"), (1, phe.PHE_FWD, T_x, "Ax", "Bx"), (2, phe.PHE_FWD, T_x, "Ax", "Bx"),
             (1, phe.PHE_BWD, T_g, "Ag", "Bg"), (3, phe.PHE_FWD, T_3, "A3", "B3"), (2, phe.PHE_BWD, 0, "Ag", "Bg")]
    jobs, outs, refs = [], [], []
    host = dict(Ax=Ax, Bx=Bx, Ag=Ag, Bg=Bg, A3=A3, B3=B3)
    for (pi, d, T, a, b) in specs:
        rows = Ws[pi].shape[0] if d == phe.PHE_FWD else Ws[pi].shape[1]
        om = torch.full((max(T, 1), rows, N), -1, dtype=odt, device="cuda")
        ob = torch.full((max(T, 1), rows), -1, dtype=odt, device="cuda")
        jobs.append((ws[pi], d, T, dev[a], dev[b], om, ob))
        outs.append((om, ob))
        Wd = Ws[pi] if d == phe.PHE_FWD else np.ascontiguousarray(Ws[pi].T)
        refs.append((Wd, host[a], host[b], T))
    return jobs, outs, refs, dev


def _check(orc, outs, refs, flags):
    import torch
    torch.cuda.synchronize()
    for (om, ob), (Wd, A, B, T) in zip(outs, refs):
        if T == 0:
            assert (om == -1).all()
            continue
        ea, eb = orc.lwedot_all(Wd, A, B, Q)
        if flags == phe.PHE_OUT_SWITCHED:
            ea, eb = orc.modswitch(ea, Q, 32), orc.modswitch(eb, Q, 32)
            ga = om.cpu().numpy().view(np.uint32).astype(np.uint64)
            gb = ob.cpu().numpy().view(np.uint32).astype(np.uint64)
        else:
            ga = om.cpu().numpy().view(np.uint64)
            gb = ob.cpu().numpy().view(np.uint64)
        assert np.array_equal(ga, ea) and np.array_equal(gb, eb)


@pytest.mark.parametrize("path", [phe.PHE_BODY_TENSOR, phe.PHE_BODY_FUSED])
@pytest.mark.parametrize("tune", [(16, 3), (4, 0), (64, 1), (1, 3)])
def test_plan_run_matches_oracle(orc, env, tune, path):
    ctx, Ws, ws, stream = env
    flags = phe.PHE_OUT_RAW if tune[0] == 4 else phe.PHE_OUT_SWITCHED
    jobs, outs, refs, _ = _make_jobs(Ws, ws, flags, seed=100 + tune[0])
    phe.phe_ctx_set_body_path(ctx, path)
    try:
        plan = phe.phe_plan_create(ctx, jobs, flags, tune)
    finally:
        phe.phe_ctx_set_body_path(ctx, phe.PHE_BODY_AUTO)
    try:
        info = phe.phe_plan_info(plan)
        assert info["tune"] == tune
        assert info["lwedot_launches"] == 1
        # x shared by three products: 3 distinct inputs, each with an input
        # transform (and, with tensor-core bodies, a digit-row kernel), then
        # the body GEMM (tensor-core bodies) and one lwedot launch
        assert info["launches"] == (8 if path == phe.PHE_BODY_TENSOR else 4)
        phe.phe_plan_run(plan, stream)
        stream.synchronize()
        _check(orc, outs, refs, flags)
    finally:
        phe.phe_plan_destroy(plan)


def test_plan_graph_replays_new_inputs(orc, env):
    import torch
    ctx, Ws, ws, stream = env
    flags = phe.PHE_OUT_SWITCHED
    jobs, outs, refs, dev = _make_jobs(Ws, ws, flags, seed=300)
    plan = phe.phe_plan_create(ctx, jobs, flags, (8, 3))
    try:
        phe.phe_plan_graph(plan, stream)   # capture + launch
        stream.synchronize()
        _check(orc, outs, refs, flags)
        # new data written into the same input buffers, then replay
        new = {}
        for key, seed in (("Ax", 401), ("Bx", 402), ("A3", 403)):
            new[key] = synth.uniform_words(tuple(dev[key].shape), Q, seed)
            dev[key].copy_(torch.from_numpy(new[key].view(np.int64)).cuda())
        for n in (0, 1, 2):  # the three products of x
            refs[n] = (refs[n][0], new["Ax"], new["Bx"], refs[n][3])
        refs[4] = (refs[4][0], new["A3"], refs[4][2], refs[4][3])
        torch.cuda.synchronize()
        phe.phe_plan_graph(plan, stream)   # replay
        stream.synchronize()
        _check(orc, outs, refs, flags)
    finally:
        phe.phe_plan_destroy(plan)


def test_autotune_picks_a_valid_shape_and_caches_it(orc, env):
    ctx, Ws, ws, stream = env
    jobs, outs, refs, _ = _make_jobs(Ws, ws, phe.PHE_OUT_SWITCHED, seed=500)
    best, ms = phe.phe_autotune(ctx, jobs, phe.PHE_OUT_SWITCHED, 16, stream)
    assert best[0] in (2, 4, 8, 16, 32, 64) and best[1] in (0, 3) and ms > 0
    cached, _ = phe.phe_autotune(ctx, jobs, phe.PHE_OUT_SWITCHED, 16, stream, timed=False)
    assert cached == best
    plan = phe.phe_plan_create(ctx, jobs, phe.PHE_OUT_SWITCHED, best)
    try:
        phe.phe_plan_run(plan, stream)
        stream.synchronize()
        _check(orc, outs, refs, phe.PHE_OUT_SWITCHED)
    finally:
        phe.phe_plan_destroy(plan)


def test_plan_rejects_bad_jobs(env):
    import torch
    ctx, Ws, ws, stream = env
    t = torch.empty(8, dtype=torch.int64, device="cuda")
    with pytest.raises(phe.PheError) as ei:
        phe.phe_plan_create(ctx, [(ws[0], 5, 1, t, t, t, t)])
    assert ei.value.status == phe.PHE_EINVAL
    with pytest.raises(phe.PheError):
        phe.phe_plan_create(ctx, [(ws[0], phe.PHE_FWD, 3, t, None, t, t)])
    with pytest.raises(phe.PheError):
        phe.phe_plan_create(ctx, [(ws[0], phe.PHE_FWD, 3, t, t, t, t)], tune=(0, 3))
