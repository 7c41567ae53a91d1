"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and describes workload shapes; it holds none
of the method's arithmetic (no products, no encryption, no modulus switch).
The oracle and the CUDA path both consume what it returns.

Workloads (Llama-3.2-1B shapes: d = 2048, FFN m = 8192, 16 layers):
  toy          N=1024, W 256x256, 16 tokens                     (insecure, correctness)
  q_proj       N=4096, W 2048x2048, 4x256 tokens, fwd and bwd
  layer        N=4096, one layer's seven projections, 8x512 tokens, fwd and bwd
  model        N=4096, 16 layers x seven projections, batch 8 with U{64..2048} tokens
  serving      64 clients, Poisson arrivals, projection/direction/token count per request

Distributions (uniform int8 stands in for the symmetric 8-bit quantised
tensors of the paper's workloads; the paper's datasets and weights are not
used):
  W, x, g   uniform integers in [-127, 127]            numpy PCG64
  S         ternary, uniform over {-1, 0, 1} (or binary {0, 1})
  A         uniform in [0, q)
  E         round(sigma * N(0, 1)), sigma = 3.2        (rounded Gaussian)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_KEY = 0x5EED0001
SEED_MASK = 0x5EED0002
SEED_ERR = 0x5EED0003
SEED_W = 0x5EED0004
SEED_X = 0x5EED0005
SEED_ARRIVALS = 0x5EED0006

# 2^60 - 2^14 + 1: prime, = 1 mod 2^14, so it carries negacyclic NTTs up to N = 8192.
Q60 = (1 << 60) - (1 << 14) + 1
# An RNS ciphertext modulus of the same size: two 30-bit primes = 1 mod 2^14.
RNS_P1, RNS_P2 = 1073643521, 1073692673
Q_RNS = RNS_P1 * RNS_P2
T_PLAIN = 1 << 16          # plaintext modulus t
LOG2_QOUT = 32             # output modulus q' = 2^32
SIGMA = 3.2

LLAMA_D = 2048
LLAMA_M = 8192
LLAMA_LAYERS = 16
# (name, d_in, d_out) of one Llama-3.2-1B layer's projections.
LLAMA_PROJECTIONS = (
    ("q", 2048, 2048),
    ("k", 2048, 512),
    ("v", 2048, 512),
    ("o", 2048, 2048),
    ("gate", 2048, 8192),
    ("up", 2048, 8192),
    ("down", 8192, 2048),
)


@dataclass(frozen=True)
class RingParams:
    N: int
    q: int = Q60
    t: int = T_PLAIN
    log2_qout: int = LOG2_QOUT
    sigma: float = SIGMA
    key: str = "ternary"

    @property
    def delta(self) -> int:
        return self.q // self.t


@dataclass(frozen=True)
class Workload:
    name: str
    ring: RingParams
    projections: tuple            # ((name, d_in, d_out), ...)
    tokens: int
    directions: tuple = ("fwd",)
    description: str = ""
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "toy": Workload("toy", RingParams(N=1024), (("w", 256, 256),), 16, ("fwd",),
                    "single encrypted matvec, insecure toy params: W 256x256, 16 tokens, N=1024"),
    "q_proj": Workload("q_proj", RingParams(N=4096), (("q", 2048, 2048),), 1024, ("fwd", "bwd"),
                       "Llama-3.2-1B q_proj 2048x2048, 4x256 tokens, N=4096, fwd and bwd"),
    "layer": Workload("layer", RingParams(N=4096), LLAMA_PROJECTIONS, 4096, ("fwd", "bwd"),
                      "one Llama-3.2-1B layer (q,k,v,o,gate,up,down), 8x512 tokens, N=4096, fwd and bwd"),
    "model": Workload("model", RingParams(N=4096), LLAMA_PROJECTIONS, 8 * 1056, ("fwd", "bwd"),
                      "16 layers x 7 projections, batch 8 with U{64..2048} tokens, N=4096",
                      {"layers": LLAMA_LAYERS, "batch": 8, "tok_lo": 64, "tok_hi": 2048}),
    "serving": Workload("serving", RingParams(N=4096), LLAMA_PROJECTIONS, 0, ("fwd", "bwd"),
                        "64 clients, Poisson arrivals mean 200 req/s, 64..2048 tokens per request",
                        {"clients": 64, "rate": 200.0, "tok_lo": 64, "tok_hi": 2048}),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def weights(d_out: int, d_in: int, seed: int = SEED_W) -> np.ndarray:
    """int8 W [d_out, d_in], uniform in [-127, 127]."""
    return rng(seed).integers(-127, 128, size=(d_out, d_in), dtype=np.int64).astype(np.int8)


def activations(T: int, d: int, seed: int = SEED_X) -> np.ndarray:
    """int8 x (or g) [T, d], uniform in [-127, 127]."""
    return rng(seed).integers(-127, 128, size=(T, d), dtype=np.int64).astype(np.int8)


def secret_key(N: int, kind: str = "ternary", seed: int = SEED_KEY) -> np.ndarray:
    if kind == "ternary":
        return rng(seed).integers(-1, 2, size=N, dtype=np.int64)
    if kind == "binary":
        return rng(seed).integers(0, 2, size=N, dtype=np.int64)
    if kind == "zero":
        return np.zeros(N, dtype=np.int64)
    raise ValueError(kind)


def masks(T: int, L: int, N: int, q: int, seed: int = SEED_MASK) -> np.ndarray:
    """Uniform masks A [T, L, N] in [0, q)."""
    return rng(seed).integers(0, q, size=(T, L, N), dtype=np.uint64)


def noise(T: int, L: int, N: int, sigma: float = SIGMA, seed: int = SEED_ERR) -> np.ndarray:
    """Rounded Gaussian noise E [T, L, N] (int64)."""
    return np.rint(rng(seed).normal(0.0, sigma, size=(T, L, N))).astype(np.int64)


def uniform_words(shape, q: int, seed: int) -> np.ndarray:
    """Uniform words in [0, q): stands in for ciphertext components whose
    distribution is uniform mod q (masks, and bodies under RLWE)."""
    return rng(seed).integers(0, q, size=shape, dtype=np.uint64)


def blocks(d: int, N: int) -> int:
    """L = ceil(d / N)."""
    return (d + N - 1) // N


def model_token_counts(batch: int = 8, lo: int = 64, hi: int = 2048, seed: int = SEED_X) -> np.ndarray:
    return rng(seed).integers(lo, hi + 1, size=batch)
