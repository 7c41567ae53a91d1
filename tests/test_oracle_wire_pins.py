"""Pins of the oracle's wire format (Sec. 4.4 sizes; Sec. 4.5 bit-vector).

  - the record sizes reproduce the byte counts the paper prints for its
    parameter set (tests/golden/wire_sizes_sec4_4.txt);
  - a packed record read as one little-endian integer equals
    sum_m v_m 2^(m*bits): the definition of the bit stream, checked with
    Python integers;
  - unpacking inverts packing, and the padding bits are zero;
  - an input record is the seed's 8 little-endian bytes and the packed body.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wire_sizes_sec4_4.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=")
            vals[k] = float(v) if "." in v else int(v)
    return vals


def test_sizes_match_the_paper(orc):
    g = _golden()
    N = g["N"]
    body = orc.wire_bytes(N, g["q_in_bits"])
    assert body == g["input_body_bytes"]
    assert g["seed_bytes"] + body == g["input_record_bytes"]
    comp = orc.wire_bytes(N, g["q_out_bits"])
    assert comp == g["output_component_bytes"]
    assert 2 * comp == g["output_rlwe_bytes"]
    assert g["output_plaintext_bytes"] == N * g["gamma_bits"] // 8
    assert round(g["input_record_bytes"] / g["input_plaintext_bytes"], 2) == g["input_expansion"]
    assert round(g["output_rlwe_bytes"] / g["output_plaintext_bytes"], 2) == g["output_expansion"]
    assert abs(16 * g["input_record_bytes"] / 1000 - g["tokens_16_input_kB"]) < 1.0


@pytest.mark.parametrize("bits", [1, 7, 26, 32, 39, 60, 64])
def test_bit_stream_is_the_little_endian_integer(orc, bits):
    rng = np.random.Generator(np.random.PCG64(bits))
    n = 97
    hi = (1 << bits) - 1
    v = [int(x) for x in rng.integers(0, 2 ** 63, n, dtype=np.uint64)]
    v = [(x * 2 + (x & 1)) & hi for x in v]
    v[0], v[-1] = hi, hi                                 # all-ones fields at both ends
    data = orc.pack_bits(np.array(v, dtype=np.uint64), bits)
    assert data.shape[0] == 4 * ((n * bits + 31) // 32)
    want = sum(x << (m * bits) for m, x in enumerate(v))
    assert int.from_bytes(data.tobytes(), "little") == want   # also: padding bits are zero
    assert np.array_equal(orc.unpack_bits(data, n, bits), np.array(v, dtype=np.uint64))


def test_input_record_layout(orc):
    rng = np.random.Generator(np.random.PCG64(3))
    B = rng.integers(0, 1 << 39, 2048, dtype=np.uint64)
    seed = 0x0123456789ABCDEF
    rec = orc.wire_input_record(seed, B, 39)
    assert rec.shape[0] == 9992
    assert int.from_bytes(rec[:8].tobytes(), "little") == seed
    assert np.array_equal(orc.unpack_bits(rec[8:], 2048, 39), B)
