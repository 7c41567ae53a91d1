#!/usr/bin/env python
"""Benchmark: encrypted W.[x] tokens/s per Llama-3.2-1B layer on B300.

One step = the hot path over one batch: for every token, the encrypted
vector x clear matrix products of Eq. (LWEdot) with the fused ModulusSwitch
for all seven projections of one Llama-3.2-1B layer (q, k, v, o, gate, up,
down), forward W.[x] and backward W^T.[g]: 8 x 512 = 4096 tokens, N = 4096,
q = 2^60 - 2^14 + 1, q' = 2^32.  Inputs are real RLWE encryptions (made by the
library's client-side helper from seeded random keys, noise and int8
activations), resident in HBM before timing.  Outputs (721 MB per token) are
written in token chunks into per-projection device buffers that each chunk
overwrites, as a server streams results out.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs the same per-GPU workload on its own token
shard (weak scaling, no collective on the data path); rank 0 prints one JSON
line.  `--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "encrypted W·[x] tokens/s per Llama-1B layer; p50/p99 latency; % of roofline"
# DRAM bytes (read + write) of one lwedot_kernel launch of the batched form
# (all 14 products of the layer workload, RNS modulus) as a function of the
# launch's tokens T: a + b T, from ncu captures of the same launch at T = 2
# and T = 4 (dram__bytes_read.sum + dram__bytes_write.sum), one fit per grid
# policy (blocks per SM: 0 = one CTA per tile, 3 = the persistent grid).  a is
# what a launch reads once whatever its tokens (the encoded weights), b what
# each token adds (its transformed masks and its outputs).  In the captured
# launches every tile holds all of a row's T <= 4 tokens, which is the launch
# of any tokens-per-tile of at least 4, so a fit serves all of those.  Valid
# only for the kernel sources the counters were taken on (kernel_source_hash).
TRAFFIC_KERNEL_HASH = "1fb177aa8808c433"
TRAFFIC_FITS = {0: (3276.91e6, 755.400e6), 3: (3276.04e6, 750.738e6)}


def lwedot_alg_bytes(wl, T: int) -> float:
    """Algorithmic DRAM bytes of one batched lwedot launch over T tokens: the
    encoded weights once (16 bytes per word), each token's transformed input
    masks once (8 bytes per word, inputs shared across products counted
    once) and its switched output masks (4 bytes per word; the bodies come
    from the body GEMM)."""
    N = wl.ring.N
    what = sum(rows * L * N * 16 for _, _, _, rows, _, L in matmuls(wl))
    out = sum(rows * N * 4 for _, _, _, rows, _, _ in matmuls(wl))
    ahat = {key: L * N * 8 for (key, cols, L) in input_keys(wl).values()}
    return what + T * (out + sum(ahat.values()))


# The source text lwedot_kernel is built and launched from: the device header,
# and the parts of phe_kernels.cu from its launch bound to its end and from
# its launcher to the next one.
KERNEL_SOURCE_REGIONS = (
    ("// Resident threads per SM the register budget is sized for", "// Seeded masks written out in natural order"),
    ("template <int LOGN, int MODE, bool RNS>\nstatic cudaError_t lwedot_impl", "// The instantiated (mode, form) pairs"),
)


def _code_only(text: str) -> str:
    """C++ source without comments and whitespace runs (the sources' string
    literals hold no comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(kernels_text=None, device_text=None) -> str:
    """Hash of the code (comments and layout ignored) in the regions above."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2505_07329_b300", "csrc")
    if kernels_text is None:
        kernels_text = open(os.path.join(csrc, "phe_kernels.cu"), encoding="utf-8").read()
    if device_text is None:
        device_text = open(os.path.join(csrc, "phe_device.cuh"), encoding="utf-8").read()
    parts = [hashlib.sha256(_code_only(device_text).encode()).hexdigest()]
    for begin, end in KERNEL_SOURCE_REGIONS:
        i = kernels_text.index(begin)
        j = kernels_text.index(end, i)
        parts.append(hashlib.sha256(_code_only(kernels_text[i:j]).encode()).hexdigest())
    return hashlib.sha256((":".join(parts) + "\n").encode()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["layer", "q_proj", "toy", "model"], default="layer",
                    help="model: the 16-layer step (all 16 layers' weights resident, batch 8 with U{64..2048} "
                         "tokens per sequence; plain per-call form, --batch-chunk tokens per call)")
    ap.add_argument("--form", choices=["batched", "plain"], default="batched",
                    help="batched: one autotuned plan (persistent launch, CUDA graph) per token chunk over all "
                         "products; plain: one phe_matmul call per product and token chunk")
    ap.add_argument("--chunk", type=int, default=32, help="tokens per plain-form call")
    ap.add_argument("--batch-chunk", type=int, default=128, help="tokens per batched-form plan")
    ap.add_argument("--no-compare", action="store_true", help="skip the secondary measurement of the other form")
    ap.add_argument("--tune", default="",
                    help="fixed plan tuning 'tok_chunk,blocks_per_sm' instead of the autotuner's pick (profiling)")
    ap.add_argument("--small-batches", default="1,8,32",
                    help="token counts at which both forms run the layer's 14 products ('' to skip)")
    ap.add_argument("--tokens", type=int, default=0, help="override tokens per GPU (0 = the workload's)")
    ap.add_argument("--e2e-tokens", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--paper-table", type=int, default=1,
                    help="1: also time the shapes of the paper's timing table at its parameter set (N=2048, q=2^39)")
    ap.add_argument("--packed-tokens", type=int, default=64,
                    help="tokens of the packed-output measurement (Eq. (pack_rotate) after each product; 0 = skip)")
    ap.add_argument("--packed-chunk", type=int, default=32,
                    help="tokens per chunk of the packed host-buffer call (its two streams overlap chunks)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--modulus", choices=["rns", "prime"], default="rns",
                    help="rns: q = p1 p2 (two 30-bit NTT primes, 32-bit residue kernels); "
                         "prime: q = 2^60 - 2^14 + 1 (64-bit kernels)")
    ap.add_argument("--serve-requests", type=int, default=500, help="requests in the serving measurement (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean Poisson arrival rate, requests/s")
    ap.add_argument("--serve-light-load", type=float, default=0.6,
                    help="second serving measurement, below capacity: arrival rate as this fraction of the rate "
                         "served in the saturated run (same request count; 0 = skip)")
    ap.add_argument("--serve-bps", type=int, default=-1,
                    help="served form's persistent grid, blocks per SM (-1: the autotuned plans' choice)")
    ap.add_argument("--serving-only", action="store_true",
                    help="skip the timed layer steps' side measurements and run only the serving measurements")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload description
# ---------------------------------------------------------------------------

def matmuls(wl):
    """[(proj index, name, direction, rows, cols, L)] for every product of a step."""
    N = wl.ring.N
    out = []
    for d in wl.directions:
        for pi, (name, d_in, d_out) in enumerate(wl.projections):
            rows, cols = (d_out, d_in) if d == "fwd" else (d_in, d_out)
            out.append((pi, name, d, rows, cols, synth.blocks(cols, N)))
    return out


def input_keys(wl):
    """Distinct encrypted inputs: forward inputs are shared the way a Llama
    layer shares them (x -> q,k,v; h -> gate,up); each backward product gets
    its own gradient."""
    keys = {}
    share = {"q": "x", "k": "x", "v": "x", "o": "attn", "gate": "h", "up": "h", "down": "mlp"}
    for pi, name, d, rows, cols, L in matmuls(wl):
        key = ("fwd", share.get(name, name)) if d == "fwd" else ("bwd", name)
        keys[(pi, d)] = (key, cols, L)
    return keys


def modmuls_per_token(wl):
    """Algorithmic modular multiplications of the mask path per token: L*N
    pointwise products plus (N/2) log2 N inverse-transform butterflies per
    output row (the input transforms, L (N/2) log2 N per input block, are
    counted separately)."""
    N = wl.ring.N
    lg = int(math.log2(N))
    return sum(rows * (L * N + (N // 2) * lg) for _, _, _, rows, _, L in matmuls(wl))


def out_bytes_per_token(wl):
    N = wl.ring.N
    return sum(rows * (N + 1) * 4 for _, _, _, rows, _, _ in matmuls(wl))


def in_bytes_per_token(wl):
    N = wl.ring.N
    seen = {}
    for (pi, d), (key, cols, L) in input_keys(wl).items():
        seen[key] = 2 * L * N * 8
    return sum(seen.values())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_tokens_per_s(wl, seconds: float):
    """Time the CPU oracle (its NTT product path, as it stands) on a bounded
    sample of the workload's (token, row) products -- rounds over the 14
    projection/direction shapes, one batch of host-thread-count products per
    shape, until `seconds` of wall time are used -- and scale the mean time
    per product of each shape to the products of one token."""
    import oracle
    N, q = wl.ring.N, wl.ring.q
    threads = oracle.num_threads()
    mm = matmuls(wl)
    per_token_items = sum(rows for _, _, _, rows, _, _ in mm)
    r = np.random.default_rng(1)
    spent = {}
    count = {}
    t_start = time.perf_counter()
    rounds = 0
    while True:
        for (pi, name, d, rows, cols, L) in mm:
            W = synth.weights(64, cols, seed=pi)  # rows of the product's length
            A = synth.uniform_words((1, L, N), q, 2 * pi + rounds)
            B = synth.uniform_words((1, L, N), q, 2 * pi + 1 + rounds)
            n = max(threads, 1)
            pairs = np.stack([np.zeros(n, dtype=np.int64), r.integers(0, 64, n)], axis=1)
            t0 = time.perf_counter()
            oracle.lwedot_pairs(W, A, B, pairs, q, method=1)
            spent[(name, d)] = spent.get((name, d), 0.0) + time.perf_counter() - t0
            count[(name, d)] = count.get((name, d), 0) + n
        rounds += 1
        if time.perf_counter() - t_start > seconds:
            break
    sec_per_token = sum(rows * spent[(name, d)] / count[(name, d)] for (_, name, d, rows, _, _) in mm)
    elapsed = time.perf_counter() - t_start
    done = sum(count.values())
    # one product per call: the oracle's OpenMP loop then runs on one core
    one = 0.0
    for (pi, name, d, rows, cols, L) in mm:
        W = synth.weights(64, cols, seed=pi)
        A = synth.uniform_words((1, L, N), q, 7 * pi)
        B = synth.uniform_words((1, L, N), q, 7 * pi + 1)
        t0 = time.perf_counter()
        for j in range(3):
            oracle.lwedot_pairs(W, A, B, np.array([[0, j]], dtype=np.int64), q, method=1)
        one += rows * (time.perf_counter() - t0) / 3
    cpu_model = None
    try:
        with open("/proc/cpuinfo") as f:
            cpu_model = next((ln.split(":", 1)[1].strip() for ln in f if ln.startswith("model name")), None)
    except OSError:
        pass
    return {"value": 1.0 / sec_per_token, "unit": "tokens/s", "cores": threads, "kind": "oracle",
            "extrapolated": True, "products_sampled": done, "products_per_token": per_token_items,
            "modulus": "q = 2^60-2^14+1 (prime; the GPU line runs the RNS q = p1 p2 of the same size)",
            "single_core_value": 1.0 / one, "host_cpu": cpu_model, "host_logical_cpus": os.cpu_count(),
            "sample": f"{done} (token,row) products, {rounds} rounds over all {len(mm)} projection/direction "
                      f"shapes, oracle NTT path on {threads} host threads, {elapsed:.1f} s wall; per-shape "
                      f"mean time x rows, summed over the {per_token_items} products of one token; "
                      f"q = 2^60-2^14+1 (the oracle's NTT needs a prime; same word size as p1 p2)"}


def run_reference(args, wl, rank):
    if rank != 0:
        return 0
    t_all = time.perf_counter()
    vals = []
    for _ in range(args.warmup):
        oracle_tokens_per_s(wl, min(args.cpu_seconds, 5.0) / 2)
    for _ in range(args.steps):
        vals.append(oracle_tokens_per_s(wl, args.cpu_seconds / max(args.steps, 1)))
    value = statistics.median(v["value"] for v in vals)
    cb = dict(vals[-1])
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tokens/s", "n_gpus": args.gpus,
            "extrapolated": True,
            "sample": (f"{sum(v['products_sampled'] for v in vals)} (token,row) products over {args.steps} steps "
                       f"(about {cb['products_sampled'] / cb['products_per_token']:.4f} of one token's "
                       f"{cb['products_per_token']} products per step), scaled per shape to whole tokens; "
                       f"ms_per_step is that rate's time for the workload's {wl.tokens} tokens, not a measured step"),
            "modulus": cb["modulus"],
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value * wl.tokens,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (mod q)",
            "data": "synthetic",
            "config": workload_config(wl, argparse.Namespace(**{**vars(args), "modulus": "prime"}),
                                      form="CPU oracle, bounded sample (NTT path, extrapolated per token)"),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": "tokens/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line))
    return 0


def workload_config(wl, args, form):
    qdesc = (f"{synth.RNS_P1}*{synth.RNS_P2} (RNS, two 30-bit NTT primes)"
             if getattr(args, "modulus", "prime") == "rns" else "2^60-2^14+1 (prime)")
    return {"workload": f"llama3.2-1b-{wl.name}" if wl.name != "toy" else "toy",
            "description": wl.description, "tokens_per_gpu": args.tokens or wl.tokens,
            "N": wl.ring.N, "q": qdesc, "q_out": f"2^{wl.ring.log2_qout}",
            "projections": [f"{n} {di}->{do}" for n, di, do in wl.projections],
            "directions": list(wl.directions), "form": form, "plain_call_tokens": args.chunk,
            "l2": "inputs larger than L2 (encrypted inputs and encoded weights are several GB)"}


# ---------------------------------------------------------------------------
# the 16-layer step (configuration of the full model)
# ---------------------------------------------------------------------------

def run_model(args, wl, rank, world, local):
    """One step = every layer's 14 products (7 projections, forward and
    backward) over a batch of 8 sequences whose token counts are drawn from
    U{64..2048}, with all 16 layers' encoded weights resident in HBM.  Each
    sequence is cut into calls of --batch-chunk tokens per product (ragged
    last calls), plain per-call form.  The encrypted inputs of one layer are
    reused by every layer: the server's work does not depend on their values,
    and 16 layers' distinct inputs would add 16x their 8 GB."""
    import torch
    from paper_2505_07329_b300 import build, phe
    from paper_2505_07329_b300.dist import max_over_ranks
    build.build()
    phe.use_test_library()  # the client-side encryption that makes the synthetic inputs
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    N, layers = wl.ring.N, wl.extra["layers"]
    counts = [int(c) for c in synth.model_token_counts(wl.extra["batch"], wl.extra["tok_lo"], wl.extra["tok_hi"],
                                                       seed=synth.SEED_X + rank)]
    T = sum(counts)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(int)
    chunk = args.batch_chunk
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    q = synth.Q_RNS
    ctx = phe.phe_ctx_create(N, q, wl.ring.log2_qout, local, rns=(synth.RNS_P1, synth.RNS_P2))
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.SEED_MASK + rank)
    t_up = time.perf_counter()
    weights = []
    for layer in range(layers):
        weights.append([phe.phe_weights_upload(ctx, synth.weights(d_out, d_in, seed=synth.SEED_W + 100 * layer + pi),
                                               phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT)
                        for pi, (name, d_in, d_out) in enumerate(wl.projections)])
    torch.cuda.synchronize()
    upload_s = time.perf_counter() - t_up
    resident = sum(phe.phe_weights_device_bytes(w) for lw in weights for w in lw)
    S = torch.randint(-1, 2, (N,), device=dev, generator=gen, dtype=torch.int8)
    inputs = {}
    for (pi, d), (key, cols, L) in input_keys(wl).items():
        if key in inputs:
            continue
        A = torch.randint(0, q, (T, L, N), device=dev, generator=gen, dtype=torch.int64)
        E = torch.round(torch.randn((T, L, N), device=dev, generator=gen) * wl.ring.sigma).to(torch.int32)
        X = torch.randint(-127, 128, (T, cols), device=dev, generator=gen, dtype=torch.int8)
        B = torch.empty_like(A)
        phe.phe_client_encrypt(ctx, T, cols, A, S, E, X, q // wl.ring.t, B)
        inputs[key] = (A, B, X)
    keys = input_keys(wl)
    mm = matmuls(wl)
    outs = [(torch.empty((chunk, rows, N), dtype=torch.int32, device=dev),
             torch.empty((chunk, rows), dtype=torch.int32, device=dev)) for (_, _, _, rows, _, _) in mm]
    torch.cuda.synchronize()

    def step():
        for layer in range(layers):
            for s0, Ts in zip(starts, counts):
                for t0 in range(0, Ts, chunk):
                    tn = min(chunk, Ts - t0)
                    a = s0 + t0
                    for n, (pi, name, d, rows, cols, L) in enumerate(mm):
                        A, B, _ = inputs[keys[(pi, d)][0]]
                        phe.phe_matmul(ctx, weights[layer][pi], phe.PHE_FWD if d == "fwd" else phe.PHE_BWD, tn,
                                       A[a:a + tn], B[a:a + tn], outs[n][0], outs[n][1], phe.PHE_OUT_SWITCHED,
                                       stream)

    phe.phe_trace_enable(ctx, True)
    for _ in range(max(args.warmup, 0)):
        step()
        torch.cuda.synchronize()
        phe.phe_trace_read(ctx)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    alu = alu_probe(phe, local, "rns")
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tr = phe.phe_trace_read(ctx)
    phe.phe_trace_enable(ctx, False)
    if dist:
        dist.barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), device=dev)
    layer_tokens = T * layers * args.steps * world
    lw = tr.get("lwedot_kernel", {})
    modmuls = modmuls_per_token(wl) * T * layers * args.steps
    achieved = modmuls / (lw["total_ms"] / 1e3) / 1e9 if lw.get("total_ms") else None
    ub = unit_bound_gmodmul(clk.get("sm_max_mhz") or 2032.0)
    if rank == 0:
        line = {"metric": METRIC, "value": layer_tokens / (elapsed_ms / 1e3), "unit": "tokens/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64 mod q (u32 out mod 2^32)",
                "data": "synthetic (seeded RLWE encryptions of uniform int8 activations; uniform int8 weights)",
                "config": {"workload": "llama3.2-1b-model-step", "description": wl.description,
                           "layers": layers, "sequence_tokens": counts, "tokens_per_step": T,
                           "layer_tokens_per_step": T * layers, "N": N,
                           "q": f"{synth.RNS_P1}*{synth.RNS_P2} (RNS)", "q_out": "2^32",
                           "form": f"plain per-call, {chunk}-token phe_matmul calls per sequence and product",
                           "weights_resident_bytes": resident, "weights_upload_s": upload_s,
                           "inputs": "one layer's encrypted inputs, reused by every layer",
                           "l2": "inputs larger than L2"},
                "step_s": elapsed_ms / args.steps / 1e3,
                "sequence_tokens_s": T * args.steps * world / (elapsed_ms / 1e3),
                "roofline": {"bound": "alu", "unit": "Gmodmul/s", "achieved": achieved, "peak": alu["gmodmul"],
                             "frac": achieved / alu["gmodmul"] if achieved else None,
                             "unit_count_bound": ub, "frac_of_unit_count_bound": achieved / ub if achieved else None,
                             "peak_basis": f"phe_probe_alu in this run: {alu['bfly_per_s'] / 1e9:.1f} G 32-bit "
                                           f"butterflies/s / 2 residues", "traffic": None,
                             "share_of_step": lw.get("total_ms", 0.0) / elapsed_ms},
                "kernels": {k: {"launches": v["launches"], "total_ms": v["total_ms"]} for k, v in tr.items()},
                "gpu_launches": sum(v["launches"] for k, v in tr.items() if not k.startswith("phe_")),
                "clocks": clk, "paper_step_s": 3458.0,
                "paper_step_note": "Sec. 6.3: one training step of Llama-3.2-1B under HE, B = 1, C = 16 tokens, "
                                   "RTX 4060 Laptop GPU, packed outputs (context, not a like-for-like target)"}
        print(json.dumps(line))
    for lw_ in weights:
        for w in lw_:
            phe.phe_weights_free(w)
    phe.phe_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    wl = synth.WORKLOADS[args.workload]
    from paper_2505_07329_b300.dist import max_over_ranks, weak_scaling_range
    from paper_2505_07329_b300.dist import world as dist_world
    rank, world, local = dist_world()
    if args.impl == "reference":
        return run_reference(args, wl, rank)

    if wl.name == "model":
        return run_model(args, wl, rank, world, local)
    import torch
    from paper_2505_07329_b300 import build, phe
    build.build()
    phe.use_test_library()  # the client-side encryption that makes the synthetic inputs
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    N = wl.ring.N
    T = args.tokens or wl.tokens
    chunk = min(args.chunk, T)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.modulus == "rns":
        q = synth.Q_RNS
        ctx = phe.phe_ctx_create(N, q, wl.ring.log2_qout, local, rns=(synth.RNS_P1, synth.RNS_P2))
    else:
        q = wl.ring.q
        ctx = phe.phe_ctx_create(N, q, wl.ring.log2_qout, local)
    delta = q // wl.ring.t
    # this rank's shard of the global batch (weak scaling: T tokens per rank,
    # seeded by the shard's first token; no collective on the data path)
    shard = weak_scaling_range(T, rank)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.SEED_MASK + shard[0])

    # weights (public, int8) for every projection, both directions
    weights = []
    host_W = [synth.weights(d_out, d_in, seed=synth.SEED_W + pi) for pi, (name, d_in, d_out) in
              enumerate(wl.projections)]
    torch.cuda.synchronize()
    t_up = time.perf_counter()
    for W in host_W:
        weights.append(phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT | phe.PHE_DIR_BWD_BIT))
    torch.cuda.synchronize()
    upload = {"seconds": time.perf_counter() - t_up, "int8_bytes": int(sum(W.size for W in host_W)),
              "device_bytes": int(sum(phe.phe_weights_device_bytes(w) for w in weights)),
              "note": "one-time: both directions' int8 rows and N^-1 NTT(w_hat) with Shoup quotients, "
                      "host int8 in, device synchronized after the last upload"}
    del host_W

    # encrypted inputs: A uniform mod q, S ternary, E rounded Gaussian, x int8
    S = torch.randint(-1, 2, (N,), device=dev, generator=gen, dtype=torch.int8)
    inputs = {}
    for (pi, d), (key, cols, L) in input_keys(wl).items():
        if key in inputs:
            continue
        A = torch.randint(0, q, (T, L, N), device=dev, generator=gen, dtype=torch.int64)
        E = torch.round(torch.randn((T, L, N), device=dev, generator=gen) * wl.ring.sigma).to(torch.int32)
        X = torch.randint(-127, 128, (T, cols), device=dev, generator=gen, dtype=torch.int8)
        B = torch.empty_like(A)
        phe.phe_client_encrypt(ctx, T, cols, A, S, E, X, delta, B)
        inputs[key] = (A, B, X)
    keys = input_keys(wl)
    mm = matmuls(wl)
    bchunk = min(args.batch_chunk, T)
    uses_plans = args.form == "batched" or not args.no_compare
    out_tokens = max(chunk, bchunk) if uses_plans else chunk
    outs = []
    for (pi, name, d, rows, cols, L) in mm:
        outs.append((torch.empty((out_tokens, rows, N), dtype=torch.int32, device=dev),
                     torch.empty((out_tokens, rows), dtype=torch.int32, device=dev)))
    torch.cuda.synchronize()
    side = torch.cuda.Stream(dev)

    def plain_step():
        for t0 in range(0, T, chunk):
            tn = min(chunk, T - t0)
            for n, (pi, name, d, rows, cols, L) in enumerate(mm):
                A, B, _ = inputs[keys[(pi, d)][0]]
                dirc = phe.PHE_FWD if d == "fwd" else phe.PHE_BWD
                phe.phe_matmul(ctx, weights[pi], dirc, tn, A[t0:t0 + tn], B[t0:t0 + tn], outs[n][0], outs[n][1],
                               phe.PHE_OUT_SWITCHED, stream)

    def chunk_jobs(t0, tn):
        jobs = []
        for n, (pi, name, d, rows, cols, L) in enumerate(mm):
            A, B, _ = inputs[keys[(pi, d)][0]]
            dirc = phe.PHE_FWD if d == "fwd" else phe.PHE_BWD
            jobs.append((weights[pi], dirc, tn, A[t0:t0 + tn], B[t0:t0 + tn], outs[n][0], outs[n][1]))
        return jobs

    plans = []
    tuning = None
    tune_ms = None
    if uses_plans:
        # autotune on the first chunk's products (a 32-token sample), then one
        # plan per chunk: pointers into the resident inputs, shared outputs
        if args.tune:
            tuning, tune_ms = tuple(int(x) for x in args.tune.split(",")), None
        else:
            tuning, tune_ms = phe.phe_autotune(ctx, chunk_jobs(0, bchunk), phe.PHE_OUT_SWITCHED, 32, side)
        for t0 in range(0, T, bchunk):
            plans.append(phe.phe_plan_create(ctx, chunk_jobs(t0, min(bchunk, T - t0)), phe.PHE_OUT_SWITCHED, tuning))
        plan_modmuls = sum(phe.phe_plan_info(pl)["modmuls"] for pl in plans)
        assert plan_modmuls == modmuls_per_token(wl) * T

    def batched_step(graph=True):
        for pl in plans:
            if graph:
                phe.phe_plan_graph(pl, side)
            else:
                phe.phe_plan_run(pl, side)

    if args.serving_only:
        args.no_compare, args.small_batches, args.no_e2e = True, "", True
        args.paper_table, args.packed_tokens, args.no_cpu = 0, 0, True
    run_stream = side if args.form == "batched" else stream
    step = batched_step if args.form == "batched" else plain_step

    # Library tracing is on from the first warm-up step, so that the plans'
    # CUDA graphs are captured with event-record nodes around their lwedot
    # launches: every timed launch is then bracketed by CUDA events on its own
    # stream, for the plain form too.
    phe.phe_trace_enable(ctx, True)
    for _ in range(max(args.warmup, 0)):
        step()
        phe.phe_trace_read(ctx)
    torch.cuda.synchronize()

    # sanity: outputs of the last chunk's first product decrypt to W x mod t
    last_chunk = chunk if args.form == "plain" else bchunk
    check, noise = sanity_decrypt(wl, mm, inputs, keys, outs, S, T, last_chunk)

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # the roofline denominators, measured in this process right before the
    # timed region, under the same clock sampling
    alu = alu_probe(phe, local, args.modulus)
    tc_tflops = tensor_probe(phe, local)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms = []
    traces = []
    ev0.record(run_stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(run_stream)
        step()
        b.record(run_stream)
        step_ms.append((a, b))
        if args.form == "batched":
            traces.append(phe.phe_trace_read(ctx))  # graph events are re-recorded by the next replay
    ev1.record(run_stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if args.form != "batched":
        traces.append(phe.phe_trace_read(ctx))
    phe.phe_trace_enable(ctx, False)
    if dist:
        dist.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    step_ms = [a.elapsed_time(b) for a, b in step_ms]
    elapsed_ms = max_over_ranks(elapsed_ms, device=dev)
    total_tokens = T * args.steps * world
    value = total_tokens / (elapsed_ms / 1e3)

    trace = {}
    for tr in traces:
        for k, v in tr.items():
            agg = trace.setdefault(k, {"launches": 0, "total_ms": 0.0, "p50s": [], "p99s": []})
            agg["launches"] += v["launches"]
            agg["total_ms"] += v["total_ms"]
            agg["p50s"].append(v["p50_ms"])
            agg["p99s"].append(v["p99_ms"])
    for v in trace.values():
        v["p50_ms"] = statistics.median(v.pop("p50s"))
        v["p99_ms"] = max(v.pop("p99s"))
    lw = trace.get("lwedot_kernel", {})
    launches = lw.get("launches", 0)
    kernel_ms = lw.get("total_ms", 0.0)
    modmuls = modmuls_per_token(wl) * T * args.steps
    achieved = modmuls / (kernel_ms / 1e3) / 1e9 if kernel_ms else None
    peak = alu["gmodmul"]
    unit_bound = unit_bound_gmodmul(clk.get("sm_max_mhz") or 2032.0) if args.modulus == "rns" else None
    fit = TRAFFIC_FITS.get(tuning[1]) if tuning is not None and tuning[0] >= 4 else None
    traffic_ok = (kernel_source_hash() == TRAFFIC_KERNEL_HASH and wl.name == "layer"
                  and args.form == "batched" and args.modulus == "rns" and T % bchunk == 0 and fit is not None)
    roof = {"bound": "alu", "unit": "Gmodmul/s", "achieved": achieved, "peak": peak,
            "frac": (achieved / peak) if achieved and peak else None,
            "traffic": (fit[0] + fit[1] * bchunk) if traffic_ok else None,
            "traffic_alg_bytes": lwedot_alg_bytes(wl, bchunk),
            "traffic_basis": ("per launch of --batch-chunk tokens: a + b T from ncu DRAM counters of the same launch "
                              "at T = 2 and 4 (profiles/lwedot_kernel_rns_llama1b_layer_dram_traffic.md)"),
            "peak_basis": (f"measured in this run by phe_probe_alu: {alu['bfly_per_s'] / 1e9:.1f} G "
                           f"{alu['bfly']} register-only butterflies/s"
                           + (" / 2 residues per coefficient" if args.modulus == "rns" else "")
                           + "; unit: coefficient modmuls"),
            "unit_count_bound": unit_bound,
            "frac_of_unit_count_bound": (achieved / unit_bound) if achieved and unit_bound else None,
            "unit_count_basis": ("148 SMs x 64 FMA-heavy lanes / 4 lane-slots per 32-bit Shoup butterfly / "
                                 "2 residues x max SM clock" if unit_bound else None),
            "kernel_ms_per_launch": kernel_ms / launches if launches else None,
            "launches": launches,
            "share_of_step": kernel_ms / elapsed_ms if elapsed_ms else None,
            "out_write_GBps": out_bytes_per_token(wl) * T * args.steps / (kernel_ms / 1e3) / 1e9 if kernel_ms else None,
            "out_write_frac_of_hbm": (out_bytes_per_token(wl) * T * args.steps / (kernel_ms / 1e3) / 1e9 / HBM_GBPS
                                      if kernel_ms else None)}
    bg = trace.get("body_gemm_kernel", {})
    roof_body = None
    if bg.get("total_ms"):
        body_tflops = body_flops_per_token(wl) * T * args.steps / (bg["total_ms"] / 1e3) / 1e12
        roof_body = {"kernel": "body_gemm_kernel", "bound": "tensor", "unit": "TFLOP/s", "achieved": body_tflops,
                     "peak": BF16_TFLOPS_SUSTAINED, "frac": body_tflops / BF16_TFLOPS_SUSTAINED,
                     "peak_basis": "MEASURED_PEAKS bf16_tflops_sustained (cuBLAS bf16, kernel timed inside a long "
                                   "step)",
                     "probe_tflops": tc_tflops, "frac_of_probe": body_tflops / tc_tflops,
                     "probe_basis": "phe_probe_tensor in this run: back-to-back tcgen05.mma kind::f16, M128 N256 "
                                    "K16, one CTA per SM",
                     "int8_kind": int8_kind_check(),
                     "launches": bg.get("launches"), "ms_per_launch": bg["total_ms"] / bg["launches"],
                     "share_of_step": bg["total_ms"] / elapsed_ms,
                     "flops_basis": "2 x 8 base-256 digits x rows x cols per token and product"}
    if args.form == "batched":
        # graph replays: the input transforms run inside the graphs without
        # their own events; count them from the plans
        per_step = sum(phe.phe_plan_info(pl)["launches"] for pl in plans)
        gpu_launches = per_step * args.steps
    else:
        gpu_launches = sum(v["launches"] for k, v in trace.items() if not k.startswith("phe_"))

    other = None
    if not args.no_compare:
        # the other form, measured the same way (1 warm-up + 1 timed step)
        o_step = plain_step if args.form == "batched" else batched_step
        o_stream = stream if args.form == "batched" else side
        o_step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(o_stream)
        o_step()
        b.record(o_stream)
        torch.cuda.synchronize()
        o_ms = a.elapsed_time(b)
        other = {"form": "plain" if args.form == "batched" else "batched", "value": T / (o_ms / 1e3),
                 "ms_per_step": o_ms, "steps": 1, "warmup": 1}

    small = None
    if args.small_batches and wl.name == "layer" and rank == 0:
        sizes = [int(x) for x in args.small_batches.split(",") if x]
        small = measure_small_batches(phe, ctx, weights, mm, keys, inputs, outs,
                                      [t for t in sizes if t <= out_tokens], stream, side)

    e2e_unpacked = None
    if not args.no_e2e:
        e2e_unpacked = measure_e2e(phe, ctx, weights, wl, mm, keys, inputs, args.e2e_tokens, stream)

    paper_table = None
    if args.paper_table and rank == 0:
        paper_table = measure_paper_table(phe, dev)
        paper_table["wire"] = measure_wire_paper_set(phe, dev)

    packed = None
    if args.packed_tokens > 0:
        packed = measure_packed(phe, ctx, weights, wl, mm, keys, inputs, S, q, min(args.packed_tokens, T), stream,
                                gen, dev, alu, args.packed_chunk)
    # The end-to-end figure the line leads with is the paper's server path as
    # a client sees it: host buffers in, Eq. (LWEdot), the packing of
    # Eq. (pack_rotate) and the switch, packed RLWE results back to host.
    e2e = None
    e2e_dense = None
    if packed is not None and not args.no_e2e:
        e2e = dict(packed["e2e"])
        e2e["path"] = ("phe_matmul_packed_host over the layer's 14 products: pinned host inputs -> device, "
                       "Eq. (LWEdot), Eq. (pack_rotate), switch, packed RLWE results (one token per RLWE) "
                       "-> pinned host")
        e2e_dense = dict(packed["dense"]["e2e"])
        e2e_dense["path"] = "the same call with PHE_PACK_DENSE: floor(N/rows) tokens per RLWE where rows <= N/2"

    serving = None
    if args.serve_requests > 0 and wl.name == "layer":
        # release the batched plans' scratch first; the server allocates per chunk
        for pl in plans:
            phe.phe_plan_destroy(pl)
        plans = []
        sbps = args.serve_bps if args.serve_bps >= 0 else (tuning[1] if tuning else 0)
        serving = measure_serving(phe, ctx, weights, wl, inputs, keys, args.serve_requests, args.serve_rate, T,
                                  tuning[0] if tuning else 8, sbps)
        if args.serve_light_load > 0:
            # the same request mix below the capacity the saturated run
            # measured: latency without a standing queue
            light = args.serve_light_load * serving["served_req_s"]
            serving["light_load"] = measure_serving(phe, ctx, weights, wl, inputs, keys, args.serve_requests, light,
                                                    T, tuning[0] if tuning else 8, sbps)
            serving["light_load"]["rate_basis"] = (f"{args.serve_light_load} x the saturated run's served "
                                                   f"{serving['served_req_s']:.2f} req/s")
        # the plain per-call form on the first requests of the same stream
        n_plain = min(args.serve_requests, 100)
        serving["plain_same_stream"] = measure_serving_plain(phe, ctx, weights, wl, inputs, keys, args.serve_requests,
                                                             n_plain, T, stream)
        serving["served_over_plain"] = (serving["layer_equiv_tokens_s"] /
                                        serving["plain_same_stream"]["layer_equiv_tokens_s"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_tokens_per_s(wl, args.cpu_seconds)

    form_desc = ("batched: one autotuned plan per token chunk over all 14 products (one lwedot launch over "
                 "every tile of the chunk, persistent when the autotuner picks it; CUDA graph replay)"
                 if args.form == "batched"
                 else "plain per-call (one phe_matmul per projection and token chunk)")
    calls = trace.get("phe_plan_graph") if args.form == "batched" else trace.get("phe_matmul")
    calls = calls or {}
    if rank == 0:
        cfg = workload_config(wl, args, form=form_desc)
        cfg["batch_chunk"] = bchunk if args.form == "batched" else None
        cfg["tuning"] = {"tok_chunk": tuning[0], "blocks_per_sm": tuning[1],
                         "autotune_ms_per_token": tune_ms} if tuning else None
        line = {"metric": METRIC, "value": value, "unit": "tokens/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64 mod q (u32 out mod 2^32)",
                "data": "synthetic (seeded RLWE encryptions of uniform int8 activations; uniform int8 weights)",
                "config": cfg,
                "latency_ms": {"step_p50": statistics.median(step_ms), "step_max": max(step_ms),
                               "call_p50": calls.get("p50_ms"), "call_p99": calls.get("p99_ms"),
                               "call_tokens": bchunk if args.form == "batched" else chunk},
                "other_form": other,
                "small_batches": small,
                "weights_upload": upload,
                "serving": serving,
                "packed": packed,
                "paper_table": paper_table,
                "roofline": roof, "roofline_body": roof_body, "cpu_baseline": cpu, "e2e": e2e,
                "e2e_unpacked": e2e_unpacked, "e2e_packed_dense": e2e_dense, "gpu_launches": gpu_launches,
                "kernels": {k: {"launches": v["launches"], "total_ms": v["total_ms"]} for k, v in trace.items()},
                "clocks": clk, "sanity_decrypt": check, "noise": noise}
        print(json.dumps(line))
    for pl in plans:
        phe.phe_plan_destroy(pl)
    for w in weights:
        phe.phe_weights_free(w)
    phe.phe_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


# Measured HBM copy bandwidth (STREAM-style copy) and cuBLAS bf16 rates from
# MEASURED_PEAKS.json beside this file, else the figures recorded when this
# was written.
def _measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


_PEAKS = _measured_peaks()
HBM_GBPS = float(_PEAKS.get("hbm_gbs", 6505.6))
BF16_TFLOPS = float(_PEAKS.get("bf16_tflops", 1780.9))
BF16_TFLOPS_SUSTAINED = float(_PEAKS.get("bf16_tflops_sustained", 1397.9))


def alu_probe(phe, device: int, modulus: str, reps: int = 3) -> dict:
    """The ALU peak, measured in this process by the library's butterfly probe
    (phe_probe_alu: register-only Gentleman-Sande butterflies with the hot
    path's own arithmetic, at lwedot's occupancy), best of `reps`.  One
    coefficient modmul is two 32-bit butterflies in the RNS form (one per
    residue) and one 64-bit butterfly in the prime form."""
    form = 0 if modulus == "rns" else 1
    per_s = max(phe.phe_probe_alu(device, form) for _ in range(reps))
    return {"bfly_per_s": per_s, "gmodmul": per_s / (2.0 if modulus == "rns" else 1.0) / 1e9,
            "bfly": "32-bit" if modulus == "rns" else "64-bit"}


def unit_bound_gmodmul(sm_mhz: float, sms: int = 148) -> float:
    """Unit-count bound of the RNS form in coefficient modmuls/s: 64 FMA-heavy
    lanes per SM execute every 32-bit integer multiply; a 32-bit Shoup
    butterfly needs two low multiplies and one high multiply at half rate,
    4 lane-slots, so 16 butterflies per SM per clock, two per coefficient."""
    return sms * 8 * sm_mhz / 1e3


def tensor_probe(phe, device: int, reps: int = 3) -> float:
    """tcgen05.mma kind::f16 rate (bf16, fp32 accumulate, M 128 N 256 K 16)
    measured in this process, TFLOP/s, best of `reps`."""
    return max(phe.phe_probe_tensor(device) for _ in range(reps)) / 1e12


_I8_SNIPPET = r"""
#include <cstdint>
__global__ void k(uint32_t d, uint64_t a, uint64_t b, uint32_t i) {
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(i), "r"(i));
}
"""


def tensor_kind_check(kind: str, arch: str = "103a") -> str:
    """Whether ptxas accepts tcgen05.mma of this kind for sm_<arch>: compiles
    a one-instruction kernel with the toolchain of this machine."""
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.cu")
        with open(src, "w") as f:
            f.write(_I8_SNIPPET.replace("KIND", kind))
        try:
            r = subprocess.run([nvcc, "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", src, "-o",
                                os.path.join(d, "k.o")], capture_output=True, text=True, timeout=120)
        except (OSError, subprocess.TimeoutExpired) as e:
            return f"not checked: {e}"
    if r.returncode == 0:
        return f"kind::{kind} accepted by ptxas for sm_{arch}"
    msg = next((ln.split("error", 1)[1].strip(" :") for ln in (r.stdout + r.stderr).splitlines()
                if "error" in ln and "not supported" in ln), (r.stdout + r.stderr).strip().splitlines()[-1:])
    return f"kind::{kind} refused by ptxas for sm_{arch}: {msg}"


def int8_kind_check() -> str:
    return tensor_kind_check("i8")


def body_flops_per_token(wl) -> int:
    """Algorithmic flops of the bodies in the digit-GEMM form: 2 per MAC, one
    MAC per (row, column) per base-256 digit, 8 digits per word."""
    return sum(2 * 8 * rows * cols for _, _, _, rows, cols, _ in matmuls(wl))


def sanity_decrypt(wl, mm, inputs, keys, outs, S, T, chunk):
    """Decrypt a few outputs of the last chunk of the first product with the
    client's key and compare with W x mod t (plain integer arithmetic).  Also
    the noise of those outputs after the switch: e = phase - (q'/t) (W x mod
    t), centred; decryption is exact while |e| < q'/(2t)."""
    N = wl.ring.N
    pi, name, d, rows, cols, L = mm[0]
    A, B, X = inputs[keys[(pi, d)][0]]
    t0 = ((T - 1) // chunk) * chunk
    tn = T - t0
    om, ob = outs[0]
    W = synth.weights(*(wl.projections[pi][2], wl.projections[pi][1]), seed=synth.SEED_W + pi)
    Wd = W if d == "fwd" else W.T
    s = S.cpu().numpy().astype(np.int64)
    ok = 0
    tot = 0
    e_max = 0
    k = wl.ring.log2_qout
    t_plain = synth.T_PLAIN
    for t in range(min(tn, 2)):
        x = X[t0 + t].cpu().numpy().astype(np.int64)
        for j in sorted({0, rows // 2, rows - 1} | set(range(1, rows, max(1, rows // 16)))):
            a = om[t, j].cpu().numpy().view(np.uint32).astype(np.int64)
            b = int(ob[t, j].item()) & 0xffffffff
            v = (b - int(np.dot(a, s))) % (1 << k)
            y = int(np.dot(Wd[j].astype(np.int64), x))
            dec = ((v * t_plain + (1 << (k - 1))) >> k) % t_plain
            ok += int((dec - y) % t_plain == 0)
            e = (v - (y % t_plain) * ((1 << k) // t_plain)) % (1 << k)
            e_max = max(e_max, abs(e - (1 << k) if e >= (1 << (k - 1)) else e))
            tot += 1
    noise = {"outputs": tot, "max_abs": e_max, "log2_max_abs": math.log2(e_max) if e_max else None,
             "log2_budget": math.log2((1 << k) / (2 * t_plain)),
             "note": "after the switch to 2^k: e = phase - (2^k/t)(W x mod t), centred; exact decryption needs "
                     "|e| < 2^k/(2t)"}
    return f"{ok}/{tot}", noise


def measure_serving(phe, ctx, weights, wl, inputs, keys, n_requests, rate, T_avail, tok_chunk=8, blocks_per_sm=0):
    """The served form: requests from 64 clients arrive as a Poisson process
    (mean `rate` per second); each is one projection of the layer in one
    direction with U{64..2048} tokens (its inputs are slices of the resident
    encrypted inputs).  A bounded horizon of `n_requests` requests; results
    are computed and dropped.  Latency is submission -> last chunk done."""
    r = synth.rng(synth.SEED_ARRIVALS)
    gaps = r.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    projs = r.integers(0, len(wl.projections), size=n_requests)
    dirs = r.integers(0, 2, size=n_requests)
    toks = r.integers(64, 2049, size=n_requests)
    N = wl.ring.N
    srv = phe.phe_server_create(ctx, 24 << 30, chunk_tokens=32, tok_chunk=tok_chunk, blocks_per_sm=blocks_per_sm,
                                max_active=64,
                                max_jobs_per_iteration=64, max_queue=4096, wait_timeout_ms=600000)
    ids = []
    items = 0
    tokens = 0
    t0 = time.perf_counter()
    try:
        for k in range(n_requests):
            pi, d, Tk = int(projs[k]), ("fwd", "bwd")[int(dirs[k])], int(toks[k])
            key = keys[(pi, d)][0]
            A, B, _ = inputs[key]
            off = (k * 97) % max(1, T_avail - Tk + 1)
            name, d_in, d_out = wl.projections[pi]
            rows = d_out if d == "fwd" else d_in
            items += Tk * rows
            tokens += Tk
            delay = arrivals[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(phe.phe_server_submit(srv, weights[pi], phe.PHE_FWD if d == "fwd" else phe.PHE_BWD, Tk,
                                             A[off:off + Tk], B[off:off + Tk]))
        for i in ids:
            phe.phe_server_wait(srv, i, 600000)
        wall = time.perf_counter() - t0
        st = phe.phe_server_stats(srv)
    finally:
        phe.phe_server_destroy(srv)
    busy = st["busy_ms"] / 1e3
    per_layer_token = sum(rows for _, _, _, rows, _, _ in matmuls(wl))
    return {"requests": n_requests, "clients": 64, "offered_rate_req_s": rate,
            "offered_span_s": float(arrivals[-1]), "wall_s": wall, "served_req_s": n_requests / busy,
            "served_tokens_s": tokens / busy, "layer_equiv_tokens_s": items / busy / per_layer_token,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "mean_ms": st["mean_ms"],
            "iterations": st["iterations"], "mem_budget_bytes": 24 << 30,
            "grid": {"tok_chunk": tok_chunk, "blocks_per_sm": blocks_per_sm},
            "peak_reserved_bytes": st["peak_reserved_bytes"],
            # saturated: the queue takes long to drain after the last arrival
            "saturated": bool(wall - float(arrivals[-1]) > 0.25 * wall),
            "note": ("offered load above capacity: latency is mostly queueing; "
                     if wall - float(arrivals[-1]) > 0.25 * wall else
                     "offered load below capacity: latency is service time plus short waits, and the rates divide "
                     "by the server's busy time (idle waits between arrivals included); ") +
                    "tokens/s are tokens of single-projection requests; layer_equiv divides (token,row) items by "
                    "the 44032 of a layer token"}


def measure_serving_plain(phe, ctx, weights, wl, inputs, keys, n_stream, n_requests, T_avail, stream, chunk=32):
    """The plain per-call form on the first n_requests of the same request
    stream as an n_stream-request measure_serving run (same seed and draws, so
    the same projections, directions and token counts): every
    request already waiting, served one after another by phe_matmul calls of
    `chunk` tokens (the server's chunk size), results dropped.  Device time
    over the whole stream gives its throughput beside the served form's."""
    import torch
    r = synth.rng(synth.SEED_ARRIVALS)
    r.exponential(1.0, size=n_stream)  # the draws of the arrival gaps of an n_stream-request run
    projs = r.integers(0, len(wl.projections), size=n_stream)
    dirs = r.integers(0, 2, size=n_stream)
    toks = r.integers(64, 2049, size=n_stream)
    N = wl.ring.N
    max_rows = max(max(d_in, d_out) for _, d_in, d_out in wl.projections)
    om = torch.empty((chunk, max_rows, N), dtype=torch.int32, device=stream.device)
    ob = torch.empty((chunk, max_rows), dtype=torch.int32, device=stream.device)
    items = tokens = 0

    def run():
        for k in range(n_requests):
            pi, d, Tk = int(projs[k]), ("fwd", "bwd")[int(dirs[k])], int(toks[k])
            A, B, _ = inputs[keys[(pi, d)][0]]
            off = (k * 97) % max(1, T_avail - Tk + 1)
            for t0 in range(0, Tk, chunk):
                tn = min(chunk, Tk - t0)
                phe.phe_matmul(ctx, weights[pi], phe.PHE_FWD if d == "fwd" else phe.PHE_BWD, tn,
                               A[off + t0:off + t0 + tn], B[off + t0:off + t0 + tn], om, ob, phe.PHE_OUT_SWITCHED,
                               stream)
    for k in range(n_requests):
        pi, d, Tk = int(projs[k]), ("fwd", "bwd")[int(dirs[k])], int(toks[k])
        name, d_in, d_out = wl.projections[pi]
        items += Tk * (d_out if d == "fwd" else d_in)
        tokens += Tk
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    run()
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    per_layer_token = sum(rows for _, _, _, rows, _, _ in matmuls(wl))
    return {"requests": n_requests, "form": f"plain per-call, {chunk}-token phe_matmul calls, FIFO, all waiting",
            "served_req_s": n_requests / sec, "served_tokens_s": tokens / sec,
            "layer_equiv_tokens_s": items / sec / per_layer_token, "device_s": sec}


def measure_small_batches(phe, ctx, weights, mm, keys, inputs, outs, sizes, stream, side, reps=20):
    """Batched against plain at serving-size batches: the layer's 14 products
    over T tokens as one autotuned plan replayed from a CUDA graph, or as 14
    phe_matmul calls.  Device time per step over `reps` steps after 3 warm-up
    steps, each form on its own stream; at these sizes the inputs sit in L2
    for both forms."""
    import torch
    res = []
    for T in sizes:
        jobs = []
        for n, (pi, name, d, rows, cols, L) in enumerate(mm):
            A, B, _ = inputs[keys[(pi, d)][0]]
            dirc = phe.PHE_FWD if d == "fwd" else phe.PHE_BWD
            jobs.append((weights[pi], dirc, T, A[:T], B[:T], outs[n][0], outs[n][1]))
        tune, _ = phe.phe_autotune(ctx, jobs, phe.PHE_OUT_SWITCHED, T, side)
        plan = phe.phe_plan_create(ctx, jobs, phe.PHE_OUT_SWITCHED, tune)

        def plain():
            for (w, dirc, tn, A, B, om, ob) in jobs:
                phe.phe_matmul(ctx, w, dirc, tn, A, B, om, ob, phe.PHE_OUT_SWITCHED, stream)

        def batched():
            phe.phe_plan_graph(plan, side)

        r = {"tokens": T, "batched_tuning": list(tune)}
        try:
            for name, f, st in (("plain", plain, stream), ("batched", batched, side)):
                for _ in range(3):
                    f()
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(st)
                for _ in range(reps):
                    f()
                b.record(st)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / reps
                r[name] = {"ms_per_step": ms, "tokens_per_s": T / (ms / 1e3)}
        finally:
            phe.phe_plan_destroy(plan)
        r["batched_speedup"] = r["plain"]["ms_per_step"] / r["batched"]["ms_per_step"]
        res.append(r)
    return res


def measure_e2e(phe, ctx, weights, wl, mm, keys, inputs, tokens, stream):
    """Tokens/s through the host-buffer C-ABI call (phe_matmul_host): per step,
    pinned host inputs -> device, all products of the layer, results -> pinned
    host buffers; a bounded token sample because each token's results are
    721 MB."""
    import torch
    N = wl.ring.N
    host_in = {}
    h2d = 0
    for key, (A, B, X) in inputs.items():
        hA = A[:tokens].cpu().pin_memory()
        hB = B[:tokens].cpu().pin_memory()
        host_in[key] = (hA, hB)
    outs = []
    d2h = 0
    for (pi, name, d, rows, cols, L) in mm:
        outs.append((torch.empty((tokens, rows, N), dtype=torch.int32).pin_memory(),
                     torch.empty((tokens, rows), dtype=torch.int32).pin_memory()))
        d2h += tokens * rows * (N + 1) * 4
    for (pi, name, d, rows, cols, L) in mm:
        h2d += 2 * tokens * L * N * 8

    def step():
        for n, (pi, name, d, rows, cols, L) in enumerate(mm):
            hA, hB = host_in[keys[(pi, d)][0]]
            dirc = phe.PHE_FWD if d == "fwd" else phe.PHE_BWD
            phe.phe_matmul_host(ctx, weights[pi], dirc, tokens, hA, hB, outs[n][0], outs[n][1],
                                phe.PHE_OUT_SWITCHED, 1 << 30, stream)

    step()
    torch.cuda.synchronize()
    steps = 2
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": tokens * steps / dt, "unit": "tokens/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "tokens_per_step": tokens,
            "host_link_GBps": (h2d + d2h) * steps / dt / 1e9,
            "note": "host-buffer C-ABI call; every LWE result word of the layer's 14 products returns to pinned "
                    "host memory (unpacked outputs; `packed.e2e` has the path with Eq. (pack_rotate)); "
                    "host_link_GBps is the copied bytes over the whole step time, compute included"}


def _negacyclic_small(a, s, mod):
    """a * s in Z_mod[X]/(X^N + 1) for a small signed s (client-side decryption)."""
    a = a.astype(np.int64)
    acc = np.zeros(a.shape[0], dtype=np.int64)
    for k in np.nonzero(s)[0]:
        rolled = np.roll(a, k)
        rolled[:k] *= -1
        acc += int(s[k]) * rolled   # |acc| < N 2^32: no overflow
    return acc % mod


def client_ksk(phe, ctx, S, N, q, base_log, gen, dev):
    """Client side of the packing: KSK_i = RLWE_S(s_i round(q / 2^base_log)),
    i < N, for the LWE key s = S (what SampleExtract leaves) and one gadget
    level, made with the library's client encryption helper; host arrays
    [N][1][N]."""
    import torch
    g0 = (q + (1 << (base_log - 1))) >> base_log
    KA = torch.randint(0, q, (N, 1, N), device=dev, generator=gen, dtype=torch.int64)
    E = torch.round(torch.randn((N, 1, N), device=dev, generator=gen) * synth.SIGMA).to(torch.int32)
    X = torch.zeros((N, N), dtype=torch.int8, device=dev)
    X[:, 0] = S
    KB = torch.empty_like(KA)
    phe.phe_client_encrypt(ctx, N, N, KA, S, E, X, g0, KB)
    torch.cuda.synchronize()
    return KA.cpu().numpy().view(np.uint64), KB.cpu().numpy().view(np.uint64)


def measure_packed(phe, ctx, weights, wl, mm, keys, inputs, S, q, tokens, stream, gen, dev, alu, host_chunk=32):
    """The whole server path of the paper, Eq. (LWEdot) then the packing of
    Eq. (pack_rotate) and the switch: every product of the layer through
    phe_matmul_packed on `tokens` resident tokens (device-timed), then the
    same through the host-buffer call phe_matmul_packed_host (wall-clock,
    copies included).  Decomp: one level of base 2^26.  Two output layouts:
    one token per RLWE (the paper's), and dense packing (PHE_PACK_DENSE:
    floor(N/rows) tokens per RLWE for products of at most N/2 rows)."""
    import torch
    N = wl.ring.N
    base_log = 26
    KA, KB = client_ksk(phe, ctx, S, N, q, base_log, gen, dev)
    k = phe.phe_ksk_upload(ctx, KA, KB, base_log, 1)
    del KA, KB
    steps = 2
    lg = int(math.log2(N))
    host_in = {key: (A[:tokens].cpu().pin_memory(), B[:tokens].cpu().pin_memory())
               for key, (A, B, X) in inputs.items()}
    h2d = sum(2 * tokens * L * N * 8 for (_, _, _, _, _, L) in mm)

    def layout(flags):
        return [phe.phe_pack_layout(N, rows, tokens, flags)[0] for (_, _, _, rows, _, _) in mm]

    def run(flags):
        units = layout(flags)
        outs = [(torch.empty((u, N), dtype=torch.int32, device=dev), torch.empty((u, N), dtype=torch.int32, device=dev))
                for u in units]

        def step():
            for n, (pi, name, d, rows, cols, L) in enumerate(mm):
                A, B, _ = inputs[keys[(pi, d)][0]]
                phe.phe_matmul_packed(ctx, weights[pi], k, phe.PHE_FWD if d == "fwd" else phe.PHE_BWD, tokens,
                                      A[:tokens], B[:tokens], outs[n][0], outs[n][1], flags, stream)

        step()
        torch.cuda.synchronize()
        phe.phe_trace_enable(ctx, True)
        phe.phe_trace_read(ctx)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        tr = phe.phe_trace_read(ctx)
        phe.phe_trace_enable(ctx, False)
        kern = {n: round(v["total_ms"] / steps / tokens, 4) for n, v in tr.items() if n.endswith("_kernel")}
        # rooflines of the packing's two main kernels, per layer token: the
        # digit transforms (ALU: 32-bit butterflies, two residues) and the MAC
        # (HBM: transformed digits once, the key once per 8 units)
        upt = sum(units) / tokens   # units (output RLWEs) per layer token
        bfly = upt * N * (N // 2) * lg * 2
        mac_bytes = upt * (N * N * 8 + 2 * N * N * 16 / 8)
        roof = []
        if kern.get("input_ntt_kernel"):
            ach = bfly / (kern["input_ntt_kernel"] / 1e3) / 1e9
            peak = alu["bfly_per_s"] / 1e9  # this run's probe (32-bit butterflies)
            roof.append({"kernel": "input_ntt_kernel (digit rows)", "bound": "alu", "unit": "G 32-bit bfly/s",
                         "achieved": ach, "peak": peak, "frac": ach / peak,
                         "note": "the kernel time also holds the 16 input-mask transforms, < 1%"})
        if kern.get("pack_mac_kernel"):
            ach = mac_bytes / (kern["pack_mac_kernel"] / 1e3) / 1e9
            roof.append({"kernel": "pack_mac_kernel", "bound": "hbm", "unit": "GB/s", "achieved": ach,
                         "peak": HBM_GBPS, "frac": ach / HBM_GBPS})
        # client-side check: the first product's first RLWE, every token it holds
        pi, name, d, rows, cols, L = mm[0]
        _, tpu = phe.phe_pack_layout(N, rows, tokens, flags)
        _, _, X = inputs[keys[(pi, d)][0]]
        W = synth.weights(wl.projections[pi][2], wl.projections[pi][1], seed=synth.SEED_W + pi)
        Wd = W if d == "fwd" else W.T
        m = min(rows, N)
        y = np.concatenate([Wd[:m].astype(np.int64) @ X[t].cpu().numpy().astype(np.int64)
                            for t in range(min(tpu, tokens))])
        pa = outs[0][0][0].cpu().numpy().view(np.uint32)
        pb = outs[0][1][0].cpu().numpy().view(np.uint32).astype(np.int64)
        ph = (pb - _negacyclic_small(pa, S.cpu().numpy().astype(np.int64), 1 << 32)) % (1 << 32)
        t = synth.T_PLAIN
        dec = ((ph * t + (1 << 31)) >> 32) % t
        ok = int(np.sum((dec[:y.shape[0]] - y) % t == 0))
        zero = int(np.sum(dec[y.shape[0]:] == 0))
        # end to end with host buffers
        houts = [(torch.empty(o[0].shape, dtype=torch.int32).pin_memory(),
                  torch.empty(o[1].shape, dtype=torch.int32).pin_memory()) for o in outs]

        def host_step():
            for n, (pi, name, d, rows, cols, L) in enumerate(mm):
                hA, hB = host_in[keys[(pi, d)][0]]
                phe.phe_matmul_packed_host(ctx, weights[pi], k, phe.PHE_FWD if d == "fwd" else phe.PHE_BWD, tokens,
                                           hA, hB, houts[n][0], houts[n][1], flags, host_chunk, stream)

        host_step()
        t0 = time.perf_counter()
        for _ in range(steps):
            host_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out_bytes = sum(units) * 2 * N * 4
        return {"value": tokens * steps / (ms / 1e3), "unit": "tokens/s", "tokens": tokens,
                "ms_per_token": ms / steps / tokens, "kernel_ms_per_token": kern, "rlwe_per_token": upt,
                "roofline": roof, "out_bytes_per_token": out_bytes / tokens,
                "sanity_decrypt": f"{ok}/{y.shape[0]} coefficients of {min(tpu, tokens)} token(s), "
                                  f"{zero}/{N - y.shape[0]} unused zero",
                "e2e": {"value": tokens * steps / dt, "unit": "tokens/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": out_bytes, "tokens_per_step": tokens, "tok_chunk": host_chunk}}

    try:
        res = run(phe.PHE_OUT_SWITCHED)
        res["dense"] = run(phe.PHE_OUT_SWITCHED | phe.PHE_PACK_DENSE)
        res["dense"]["layout"] = ("PHE_PACK_DENSE: floor(N/rows) consecutive tokens per RLWE for products of at "
                                  "most N/2 rows (not in the paper, which packs one token per RLWE)")
        wire = measure_wire(phe, ctx, N, weights[mm[0][0]], k, mm[0], tokens, stream, dev)
    finally:
        phe.phe_ksk_free(k)
    res.update({"ksk": {"base_log": base_log, "ell": 1, "device_bytes": 2 * N * N * 16},
                "layout": "one token per RLWE (Eq. (pack_rotate) over a token's outputs)",
                "unpacked_out_bytes_per_token": out_bytes_per_token(wl), "wire": wire})
    return res


def measure_wire(phe, ctx, N, w, k, prod, tokens, stream, dev, reps=3):
    """phe_matmul_wire, device-timed: `tokens` tokens of one product from
    input records (8-byte seed + bodies at ceil(log2 q) bits) to output
    records: LWE records at log2_qout bits, or with the key k one packed RLWE
    record per group of N rows.  Every bit pattern of an input record is a
    valid record, so the inputs are random words."""
    import torch
    pi, name, d, rows, cols, L = prod
    sizes = phe.phe_wire_sizes(ctx)
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_X + 17)
    rec = torch.randint(-(1 << 31), 1 << 31, (tokens * L * sizes["input"] // 4,), device=dev, generator=g,
                        dtype=torch.int64).to(torch.int32)
    per_tok = ((rows + N - 1) // N) * sizes["rlwe"] if k is not None else rows * sizes["lwe"]
    out = torch.empty(((tokens * per_tok + 3) // 4,), dtype=torch.int32, device=dev)
    direction = phe.PHE_FWD if d == "fwd" else phe.PHE_BWD
    phe.phe_matmul_wire(ctx, w, k, direction, tokens, rec, out, stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        phe.phe_matmul_wire(ctx, w, k, direction, tokens, rec, out, stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    return {"value": tokens / (ms / 1e3), "unit": "tokens/s", "tokens": tokens, "product": f"{name} {d}",
            "records": "packed RLWE" if k is not None else "LWE",
            "in_bytes_per_token": L * sizes["input"], "out_bytes_per_token": per_tok}


def measure_wire_paper_set(phe, dev, tokens=64):
    """phe_matmul_wire at the paper's parameter set (N = 2048, q = 2^39 ->
    q_out = 2^26) on a 2048->2048 forward product, 9992-byte input records in:
    LWE records out, and packed RLWE records out (13312 bytes, the size Sec.
    4.4 counts; a random key-switching key of base 2^26, one level, in exact
    slices: the server's work does not depend on its values)."""
    import torch
    ctx = phe.phe_ctx_create(2048, 1 << 39, 26, dev.index or 0, rns=(synth.RNS_P1, synth.RNS_P2))
    stream = torch.cuda.current_stream(dev)
    prod = (0, "2048->2048", "fwd", 2048, 2048, 1)
    try:
        w = phe.phe_weights_upload(ctx, synth.weights(2048, 2048, seed=synth.SEED_W + 4096), phe.PHE_DIR_FWD_BIT)
        try:
            out = {"lwe": measure_wire(phe, ctx, 2048, w, None, prod, tokens, stream, dev)}
            kg = np.random.Generator(np.random.PCG64(synth.SEED_KEY + 40))
            k = phe.phe_ksk_upload(ctx, kg.integers(0, 1 << 39, (2048, 1, 2048), dtype=np.uint64),
                                   kg.integers(0, 1 << 39, (2048, 1, 2048), dtype=np.uint64), 26, 1)
            try:
                out["packed"] = measure_wire(phe, ctx, 2048, w, k, prod, tokens, stream, dev)
            finally:
                phe.phe_ksk_free(k)
            return out
        finally:
            phe.phe_weights_free(w)
    finally:
        phe.phe_ctx_destroy(ctx)


# Per-token latencies of W.[x] printed in Table fhe_matmul_timing (Sec. 6.3)
# for the paper's parameter set on its laptop GPU, including its output packing.
PAPER_TABLE = (((768, 768), 0.0809), ((3072, 768), 0.1528), ((2048, 2048), 0.2402), ((768, 3072), 0.3389),
               ((8192, 2048), 0.6368), ((2048, 8192), 1.0539))


def measure_paper_table(phe, dev, tokens=64):
    """The shapes of Table fhe_matmul_timing at the paper's parameter set
    (N = 2048, q = 2^39 computed through p1 p2, q_out = 2^26): one-token
    latency and throughput on `tokens` tokens (device-resident, CUDA events)
    of phe_matmul (LWE outputs) and of phe_matmul_packed (one packed RLWE per
    2048 rows, as the paper's timed path; base 2^26, one level, the key in
    4 exact slices).  The key-switching key is random words: the server's work
    does not depend on its values."""
    import torch
    ctx = phe.phe_ctx_create(2048, 1 << 39, 26, dev.index or 0, rns=(synth.RNS_P1, synth.RNS_P2))
    rows_out = []
    k = None
    try:
        stream = torch.cuda.current_stream(dev)
        kg = np.random.Generator(np.random.PCG64(synth.SEED_KEY + 39))
        KA = kg.integers(0, 1 << 39, (2048, 1, 2048), dtype=np.uint64)
        KB = kg.integers(0, 1 << 39, (2048, 1, 2048), dtype=np.uint64)
        k = phe.phe_ksk_upload(ctx, KA, KB, 26, 1)
        del KA, KB

        def timed(f, T, reps=5):
            for _ in range(2):
                f(T)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                f(T)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        for (d_in, d_out), paper_s in PAPER_TABLE:
            W = synth.weights(d_out, d_in, seed=synth.SEED_W + d_in + d_out)
            w = phe.phe_weights_upload(ctx, W, phe.PHE_DIR_FWD_BIT)
            L = synth.blocks(d_in, 2048)
            G = (d_out + 2047) // 2048
            g = torch.Generator(device=dev)
            g.manual_seed(d_in * 7 + d_out)
            A = torch.randint(0, 1 << 39, (tokens, L, 2048), device=dev, generator=g, dtype=torch.int64)
            B = torch.randint(0, 1 << 39, (tokens, L, 2048), device=dev, generator=g, dtype=torch.int64)
            om = torch.empty((tokens, d_out, 2048), dtype=torch.int32, device=dev)
            ob = torch.empty((tokens, d_out), dtype=torch.int32, device=dev)
            pa = torch.empty((tokens, G, 2048), dtype=torch.int32, device=dev)
            pb = torch.empty((tokens, G, 2048), dtype=torch.int32, device=dev)

            def lwe(T):
                phe.phe_matmul(ctx, w, phe.PHE_FWD, T, A, B, om, ob, phe.PHE_OUT_SWITCHED, stream)

            def packed(T):
                phe.phe_matmul_packed(ctx, w, k, phe.PHE_FWD, T, A, B, pa, pb, phe.PHE_OUT_SWITCHED, stream)

            res = {T: timed(lwe, T) for T in (1, tokens)}
            pres = {T: timed(packed, T, reps=3) for T in (1, tokens)}
            phe.phe_weights_free(w)
            rows_out.append({"shape": f"{d_in}->{d_out}", "paper_s_per_token": paper_s,
                             "latency_ms_1_token": res[1], "tokens_per_s": tokens / (res[tokens] / 1e3),
                             "packed_latency_ms_1_token": pres[1],
                             "packed_tokens_per_s": tokens / (pres[tokens] / 1e3)})
    finally:
        if k is not None:
            phe.phe_ksk_free(k)
        phe.phe_ctx_destroy(ctx)
    return {"params": "N=2048, q=2^39 (exact through p1 p2), q_out=2^26", "tokens": tokens, "rows": rows_out,
            "note": "paper times: laptop GPU, one token, with output packing; ours: one B300, LWE outputs and "
                    "packed RLWE outputs (base 2^26, one level, key in exact slices)"}


if __name__ == "__main__":
    sys.exit(main())
