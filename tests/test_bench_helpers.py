"""CPU checks of the benchmark's host-side arithmetic: the algorithmic work
and bytes it divides by, and the client-side decryption helper it uses for
the packed path's sanity check (against the oracle's negacyclic product)."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_layer_work_and_bytes():
    wl = synth.WORKLOADS["layer"]
    N = wl.ring.N
    mm = bench.matmuls(wl)
    assert len(mm) == 14
    rows = sum(r for _, _, _, r, _, _ in mm)
    assert rows == 44032                       # 23 552 forward + 20 480 backward output rows
    # L*N pointwise + (N/2) log2 N inverse-transform butterflies per output row
    want = sum(r * (L * N + (N // 2) * int(math.log2(N))) for _, _, _, r, _, L in mm)
    assert bench.modmuls_per_token(wl) == want
    assert bench.out_bytes_per_token(wl) == rows * (N + 1) * 4
    # inputs shared the way a layer shares them: x feeds q, k, v; h feeds gate, up
    keys = {v[0] for v in bench.input_keys(wl).values()}
    assert len(keys) == 11


def test_unit_count_bound_and_body_flops():
    # 148 SMs x 64 FMA-heavy lanes / 4 lane-slots per 32-bit Shoup butterfly
    # / 2 residues per coefficient, at 2032 MHz
    assert abs(bench.unit_bound_gmodmul(2032.0) - 148 * 64 / 4 / 2 * 2.032) < 1e-9
    wl = synth.WORKLOADS["layer"]
    macs = sum(rows * cols for _, _, _, rows, cols, _ in bench.matmuls(wl))
    assert macs == 2 * (2048 * 2048 * 2 + 2048 * 512 * 2 + 2048 * 8192 * 3)   # both directions
    assert bench.body_flops_per_token(wl) == 2 * 8 * macs


def test_int8_tensor_kind_is_refused_for_sm103a():
    # the toolchain of this image: tcgen05.mma kind::i8 does not assemble for
    # sm_103a (it does for sm_100a); the body GEMM uses kind::f16 with bf16 digits
    assert bench.tensor_kind_check("i8").startswith("kind::i8 refused by ptxas for sm_103a")
    assert bench.tensor_kind_check("f16") == "kind::f16 accepted by ptxas for sm_103a"


def test_client_decryption_product_matches_the_oracle(orc):
    rng = np.random.Generator(np.random.PCG64(5))
    N, mod = 64, 1 << 32
    a = rng.integers(0, mod, N, dtype=np.uint64)
    s = rng.integers(-1, 2, N)
    got = bench._negacyclic_small(a.astype(np.uint32), s, mod)
    sq = np.array([v % mod for v in s.tolist()], dtype=np.uint64)
    assert np.array_equal(got.astype(np.uint64), orc.negacyclic_mul(a, sq, mod))


def test_paper_table_is_the_papers_six_shapes():
    shapes = [shape for shape, _ in bench.PAPER_TABLE]
    assert shapes == [(768, 768), (3072, 768), (2048, 2048), (768, 3072), (8192, 2048), (2048, 8192)]
    assert all(t > 0 for _, t in bench.PAPER_TABLE)


def test_kernel_source_hash_covers_only_the_kernel_regions():
    # the traffic figure is tied to the code lwedot_kernel is built and
    # launched from: edits elsewhere in phe_kernels.cu keep the hash, code
    # edits inside the kernel or the device header change it
    csrc = os.path.join(bench.ROOT, "paper_2505_07329_b300", "csrc")
    k = open(os.path.join(csrc, "phe_kernels.cu"), encoding="utf-8").read()
    d = open(os.path.join(csrc, "phe_device.cuh"), encoding="utf-8").read()
    h = bench.kernel_source_hash(k, d)
    assert h == bench.kernel_source_hash()
    assert bench.kernel_source_hash(k + "\n// trailing comment\n", d) == h
    i = k.index("lwedot_kernel(const LweJobTable jt")
    assert bench.kernel_source_hash(k[:i] + " " + k[i:], d) == h          # layout only
    assert bench.kernel_source_hash(k[:i] + k[i:].replace("const u32 total = jt.prefix[jt.n];",
                                                          "const u32 total = jt.prefix[jt.n] + 0;", 1), d) != h
    j = k.index("static cudaError_t lwedot_impl")
    assert bench.kernel_source_hash(k[:j] + k[j:].replace("grid_limit > 0", "grid_limit >= 1", 1), d) != h
    # comments and layout do not count; code in the device header does
    assert bench.kernel_source_hash(k, d + "\n// a note\n/* another */\n") == h
    assert bench.kernel_source_hash(k, d + "\nconstexpr int kUnused = 1;\n") != h
