"""CPU oracle for the encrypted vector x clear matrix product of arXiv 2505.07329.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg import this package; the product library never does.  The
arithmetic lives in ``phe_oracle.c`` (exact 128-bit integer arithmetic, no
lazy reduction); this module compiles it with gcc on first use and wraps it
with numpy arrays.  It shares no code or constants with the CUDA library.

Functions and the passages they follow:
  negacyclic_mul / negacyclic_mul_ntt    product in R_q = Z_q[X]/(X^N+1)   Sec. 3.1
  sample_extract                          SampleExtract(RLWE, h)           Sec. 3.2
  encode_weight_block                     w_hat_ij[k] = w_j[iN+N-1-k]      Sec. 4.3.1
  lwedot_pairs                            Eq. (LWEdot)                     Sec. 4.3.1
  lwedot_closed_form                      the same result written out term by term
  modswitch                               ModulusSwitch q -> 2^k           Sec. 3.2 / 4.3.1
  rlwe_encrypt, lwe_phase, decode         RLWE / LWE definitions           Sec. 3.1
  expand_mask, chacha20_block             mask from a seed (PRNG read as ChaCha20, RFC 8439)  Sec. 3.1
  gadget, decompose                       Decomp (read as TFHE's approximate signed gadget)  Sec. 3.2
  ksk_encrypt, keyswitch, rotate          KeySwitching, Rotate             Sec. 3.2
  pack, pack_coeffs                       sum_j Rotate(KeySwitching(LWE_j), j)   Eq. (pack_rotate)
  wire_bytes, pack_bits, unpack_bits,     bit-packed wire records          Sec. 4.4, Sec. 4.5
  wire_input_record

Parity status: every function above is pinned by tests/test_oracle_pins.py
(closed forms, library routines, brute force, exact noise identity).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile phe_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            L.oracle_powmod.restype = ctypes.c_uint64
            L.oracle_powmod.argtypes = [ctypes.c_uint64] * 3
            L.oracle_is_prime.restype = ctypes.c_int
            L.oracle_is_prime.argtypes = [ctypes.c_uint64]
            L.oracle_find_psi.restype = ctypes.c_uint64
            L.oracle_find_psi.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            L.oracle_negacyclic_mul.argtypes = [_u64p, _u64p, _u64p, ctypes.c_uint32, ctypes.c_uint64]
            L.oracle_negacyclic_mul_ntt.argtypes = [_u64p, _u64p, _u64p, ctypes.c_uint32, ctypes.c_uint64]
            L.oracle_ntt_forward.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_ntt_inverse.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_sample_extract.argtypes = [_u64p, _u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                                _u64p, _u64p]
            L.oracle_encode_weight_block.argtypes = [_i8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _i64p]
            L.oracle_lwedot_pairs.argtypes = [_i8p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, ctypes.c_uint32,
                                              ctypes.c_uint64, ctypes.c_int, _u32p, ctypes.c_uint64, _u64p, _u64p]
            L.oracle_lwedot_closed_form.argtypes = [_i8p, ctypes.c_uint32, _u64p, _u64p, ctypes.c_uint32,
                                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p]
            L.oracle_modswitch.restype = ctypes.c_uint64
            L.oracle_modswitch.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            L.oracle_modswitch_array.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            L.oracle_rlwe_encrypt.argtypes = [_u64p, _i64p, _i64p, _i64p, ctypes.c_uint32, ctypes.c_uint64,
                                              ctypes.c_uint64, _u64p]
            L.oracle_lwe_phase.restype = ctypes.c_uint64
            L.oracle_lwe_phase.argtypes = [_u64p, ctypes.c_uint64, _i64p, ctypes.c_uint32, ctypes.c_uint64]
            L.oracle_decode.restype = ctypes.c_int64
            L.oracle_decode.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_chacha20_block.argtypes = [_u32p, ctypes.c_uint32, _u32p, _u32p]
            L.oracle_expand_mask.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _u64p]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_wire_bytes.restype = ctypes.c_uint64
            L.oracle_wire_bytes.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            L.oracle_pack_bits.argtypes = [_u64p, ctypes.c_uint64, ctypes.c_uint32, _u8p]
            L.oracle_unpack_bits.argtypes = [_u8p, ctypes.c_uint64, ctypes.c_uint32, _u64p]
            L.oracle_wire_input_record.argtypes = [ctypes.c_uint64, _u64p, ctypes.c_uint32, ctypes.c_uint32, _u8p]
            L.oracle_gadget.restype = ctypes.c_uint64
            L.oracle_gadget.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_decompose.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _i64p]
            L.oracle_ksk_encrypt.argtypes = [_u64p, _i64p, _i64p, ctypes.c_uint32, _i64p, ctypes.c_uint32,
                                             ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u64p]
            L.oracle_keyswitch.argtypes = [_u64p, ctypes.c_uint64, ctypes.c_uint32, _u64p, _u64p, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p]
            L.oracle_rotate.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, _u64p]
            L.oracle_pack.argtypes = [_u64p, _u64p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p]
            L.oracle_pack_coeffs.argtypes = [_u64p, _u64p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p,
                                             ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             _u32p, ctypes.c_uint32, _u64p, _u64p]
            _lib = L
    return _lib


def _p(a: np.ndarray, ptype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ptype)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _i8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int8))


# --- modular helpers -------------------------------------------------------

def powmod(b: int, e: int, q: int) -> int:
    return int(lib().oracle_powmod(b, e, q))


def is_prime(n: int) -> bool:
    return bool(lib().oracle_is_prime(n))


def find_psi(q: int, N: int) -> int:
    return int(lib().oracle_find_psi(q, N))


# --- ring products ---------------------------------------------------------

def negacyclic_mul(a, b, q: int) -> np.ndarray:
    """Schoolbook product in Z_q[X]/(X^N+1)."""
    a, b = _u64(a), _u64(b)
    N = a.shape[0]
    c = np.zeros(N, dtype=np.uint64)
    lib().oracle_negacyclic_mul(_p(a, _u64p), _p(b, _u64p), _p(c, _u64p), N, q)
    return c


def negacyclic_mul_ntt(a, b, q: int) -> np.ndarray:
    """The same product through the oracle's textbook negacyclic NTT."""
    a, b = _u64(a), _u64(b)
    N = a.shape[0]
    c = np.zeros(N, dtype=np.uint64)
    lib().oracle_negacyclic_mul_ntt(_p(a, _u64p), _p(b, _u64p), _p(c, _u64p), N, q)
    return c


def ntt_forward(a, q: int, psi: int) -> np.ndarray:
    a = _u64(a).copy()
    lib().oracle_ntt_forward(_p(a, _u64p), a.shape[0], q, psi)
    return a


def ntt_inverse(a, q: int, psi: int) -> np.ndarray:
    a = _u64(a).copy()
    lib().oracle_ntt_inverse(_p(a, _u64p), a.shape[0], q, psi)
    return a


def sample_extract(A, B, h: int, q: int):
    """SampleExtract(RLWE(A,B), h) -> (a', b') per the paper's two-branch formula."""
    A, B = _u64(A), _u64(B)
    N = A.shape[0]
    a = np.zeros(N, dtype=np.uint64)
    b = np.zeros(1, dtype=np.uint64)
    lib().oracle_sample_extract(_p(A, _u64p), _p(B, _u64p), N, h, q, _p(a, _u64p), _p(b, _u64p))
    return a, int(b[0])


def encode_weight_block(w_row, i: int, N: int) -> np.ndarray:
    w_row = _i8(w_row)
    out = np.zeros(N, dtype=np.int64)
    lib().oracle_encode_weight_block(_p(w_row, _i8p), w_row.shape[0], i, N, _p(out, _i64p))
    return out


# --- Eq. (LWEdot) ------------------------------------------------------------

def lwedot_pairs(W, A, B, pairs, q: int, method: int = 0):
    """LWE(x_t . w_j) mod q for each (t, j) in ``pairs``.

    W: [d_out, d_in] int8.  A, B: [T, L, N] uint64.  pairs: [P, 2] (t, j).
    Returns (a [P, N] uint64, b [P] uint64), before any modulus switch.
    method 0 = schoolbook products (definition), 1 = products through the NTT.
    """
    W = _i8(W)
    A, B = _u64(A), _u64(B)
    d_out, d_in = W.shape
    T, L, N = A.shape
    assert B.shape == A.shape and L == (d_in + N - 1) // N
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.uint32).reshape(-1, 2))
    P = pairs.shape[0]
    a = np.zeros((P, N), dtype=np.uint64)
    b = np.zeros(P, dtype=np.uint64)
    lib().oracle_lwedot_pairs(_p(W, _i8p), d_out, d_in, _p(A, _u64p), _p(B, _u64p), N, q, method,
                              _p(pairs, _u32p), P, _p(a, _u64p), _p(b, _u64p))
    return a, b


def lwedot_all(W, A, B, q: int, method: int = 0):
    """Every (t, j): returns a [T, d_out, N], b [T, d_out] (mod q)."""
    T = np.asarray(A).shape[0]
    d_out = np.asarray(W).shape[0]
    tt, jj = np.meshgrid(np.arange(T), np.arange(d_out), indexing="ij")
    pairs = np.stack([tt.ravel(), jj.ravel()], axis=1)
    a, b = lwedot_pairs(W, A, B, pairs, q, method)
    N = np.asarray(A).shape[2]
    return a.reshape(T, d_out, N), b.reshape(T, d_out)


def lwedot_closed_form(W, A, B, t: int, j: int, q: int):
    W = _i8(W)
    A, B = _u64(A), _u64(B)
    d_out, d_in = W.shape
    N = A.shape[2]
    a = np.zeros(N, dtype=np.uint64)
    b = np.zeros(1, dtype=np.uint64)
    lib().oracle_lwedot_closed_form(_p(W, _i8p), d_in, _p(A, _u64p), _p(B, _u64p), N, q, t, j,
                                    _p(a, _u64p), _p(b, _u64p))
    return a, int(b[0])


# --- ModulusSwitch -----------------------------------------------------------

def modswitch(c, q: int, log2_qout: int) -> np.ndarray:
    c = _u64(c)
    flat = c.ravel()
    out = np.zeros_like(flat)
    lib().oracle_modswitch_array(_p(flat, _u64p), _p(out, _u64p), flat.shape[0], q, log2_qout)
    return out.reshape(c.shape)


def modswitch_one(c: int, q: int, log2_qout: int) -> int:
    return int(lib().oracle_modswitch(c, q, log2_qout))


# --- client side (tests only) --------------------------------------------------

def rlwe_encrypt(A, S, E, M, q: int, delta: int) -> np.ndarray:
    """B = A*S + E + Delta*M (mod q) for one block."""
    A, S, E, M = _u64(A), _i64(S), _i64(E), _i64(M)
    N = A.shape[0]
    B = np.zeros(N, dtype=np.uint64)
    lib().oracle_rlwe_encrypt(_p(A, _u64p), _p(S, _i64p), _p(E, _i64p), _p(M, _i64p), N, q, delta, _p(B, _u64p))
    return B


def encrypt_vectors(A, S, E, X, q: int, delta: int) -> np.ndarray:
    """Encrypt T vectors block by block (Sec. 4.3.1 block split, zero padding).

    A: [T, L, N] masks; S: [N] key; E: [T, L, N] noise; X: [T, d] int8 messages.
    Returns the bodies B [T, L, N]."""
    A = _u64(A)
    T, L, N = A.shape
    X = np.asarray(X)
    d = X.shape[1]
    B = np.zeros_like(A)
    for t in range(T):
        for i in range(L):
            M = np.zeros(N, dtype=np.int64)
            seg = X[t, i * N:min(d, (i + 1) * N)].astype(np.int64)
            M[:seg.shape[0]] = seg
            B[t, i] = rlwe_encrypt(A[t, i], S, E[t, i], M, q, delta)
    return B


def lwe_phase(a, b: int, s, Q: int) -> int:
    a, s = _u64(a), _i64(s)
    return int(lib().oracle_lwe_phase(_p(a, _u64p), b, _p(s, _i64p), a.shape[0], Q))


def decode(v: int, Q: int, t: int) -> int:
    return int(lib().oracle_decode(v, Q, t))


# --- seeded masks --------------------------------------------------------------

def chacha20_block(key_words, counter: int, nonce_words) -> np.ndarray:
    key = np.ascontiguousarray(np.asarray(key_words, dtype=np.uint32))
    nonce = np.ascontiguousarray(np.asarray(nonce_words, dtype=np.uint32))
    out = np.zeros(16, dtype=np.uint32)
    lib().oracle_chacha20_block(_p(key, _u32p), counter, _p(nonce, _u32p), _p(out, _u32p))
    return out


def expand_mask(seed: int, N: int, q: int) -> np.ndarray:
    """Mask of one ciphertext from its 64-bit seed (ChaCha20 keystream, nonce 0)."""
    A = np.zeros(N, dtype=np.uint64)
    lib().oracle_expand_mask(seed, N, q, _p(A, _u64p))
    return A


def expand_masks(seeds, N: int, q: int) -> np.ndarray:
    """Masks for an array of seeds, shape seeds.shape + (N,)."""
    seeds = np.asarray(seeds, dtype=np.uint64)
    out = np.zeros(seeds.shape + (N,), dtype=np.uint64)
    for idx in np.ndindex(seeds.shape):
        out[idx] = expand_mask(int(seeds[idx]), N, q)
    return out


# --- output packing ------------------------------------------------------------

def gadget(q: int, base_log: int, l: int) -> int:
    return int(lib().oracle_gadget(q, base_log, l))


def decompose(a: int, q: int, base_log: int, ell: int) -> np.ndarray:
    d = np.zeros(ell, dtype=np.int64)
    lib().oracle_decompose(a, q, base_log, ell, _p(d, _i64p))
    return d


def ksk_encrypt(KA, E, s, S2, q: int, base_log: int, ell: int) -> np.ndarray:
    """KB [n][ell][N] of the key-switching key s -> S2 with masks KA and noise E."""
    KA, E, s, S2 = _u64(KA), _i64(E), _i64(s), _i64(S2)
    n, N = s.shape[0], S2.shape[0]
    assert KA.shape == (n, ell, N) and E.shape == (n, ell, N)
    KB = np.zeros((n, ell, N), dtype=np.uint64)
    lib().oracle_ksk_encrypt(_p(KA, _u64p), _p(E, _i64p), _p(s, _i64p), n, _p(S2, _i64p), N, q, base_log, ell,
                             _p(KB, _u64p))
    return KB


def keyswitch(a, b: int, KA, KB, q: int, base_log: int, ell: int):
    a, KA, KB = _u64(a), _u64(KA), _u64(KB)
    n, N = a.shape[0], KA.shape[2]
    A_out = np.zeros(N, dtype=np.uint64)
    B_out = np.zeros(N, dtype=np.uint64)
    lib().oracle_keyswitch(_p(a, _u64p), b, n, _p(KA, _u64p), _p(KB, _u64p), N, q, base_log, ell,
                           _p(A_out, _u64p), _p(B_out, _u64p))
    return A_out, B_out


def rotate(P, k: int, q: int) -> np.ndarray:
    P = _u64(P)
    out = np.zeros_like(P)
    lib().oracle_rotate(_p(P, _u64p), P.shape[0], k, q, _p(out, _u64p))
    return out


def pack(a, b, KA, KB, q: int, base_log: int, ell: int):
    """(A, B) = sum_j Rotate(KeySwitching((a_j, b_j)), j) for a: [m][n], b: [m]."""
    a, b, KA, KB = _u64(a), _u64(b), _u64(KA), _u64(KB)
    m, n = a.shape
    N = KA.shape[2]
    A_out = np.zeros(N, dtype=np.uint64)
    B_out = np.zeros(N, dtype=np.uint64)
    lib().oracle_pack(_p(a, _u64p), _p(b, _u64p), m, n, _p(KA, _u64p), _p(KB, _u64p), N, q, base_log, ell,
                      _p(A_out, _u64p), _p(B_out, _u64p))
    return A_out, B_out


def pack_coeffs(a, b, KA, KB, q: int, base_log: int, ell: int, rs):
    """Coefficients rs of the packed (A, B), evaluated one by one."""
    a, b, KA, KB = _u64(a), _u64(b), _u64(KA), _u64(KB)
    rs = np.ascontiguousarray(np.asarray(rs, dtype=np.uint32))
    m, n = a.shape
    N = KA.shape[2]
    A_out = np.zeros(rs.shape[0], dtype=np.uint64)
    B_out = np.zeros(rs.shape[0], dtype=np.uint64)
    lib().oracle_pack_coeffs(_p(a, _u64p), _p(b, _u64p), m, n, _p(KA, _u64p), _p(KB, _u64p), N, q, base_log, ell,
                             _p(rs, _u32p), rs.shape[0], _p(A_out, _u64p), _p(B_out, _u64p))
    return A_out, B_out


# --- wire format ----------------------------------------------------------------

def wire_bytes(fields: int, bits: int) -> int:
    return int(lib().oracle_wire_bytes(fields, bits))


def pack_bits(v, bits: int) -> np.ndarray:
    v = _u64(v).ravel()
    out = np.zeros(wire_bytes(v.shape[0], bits), dtype=np.uint8)
    lib().oracle_pack_bits(_p(v, _u64p), v.shape[0], bits, _p(out, _u8p))
    return out


def unpack_bits(data, n: int, bits: int) -> np.ndarray:
    data = np.ascontiguousarray(np.asarray(data, dtype=np.uint8))
    v = np.zeros(n, dtype=np.uint64)
    lib().oracle_unpack_bits(_p(data, _u8p), n, bits, _p(v, _u64p))
    return v


def wire_input_record(seed: int, B, bits_q: int) -> np.ndarray:
    B = _u64(B)
    out = np.zeros(8 + wire_bytes(B.shape[0], bits_q), dtype=np.uint8)
    lib().oracle_wire_input_record(seed, _p(B, _u64p), B.shape[0], bits_q, _p(out, _u8p))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())
