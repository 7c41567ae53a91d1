"""Pins of the oracle's output packing: Decomp, KeySwitching and Rotate
(Sec. 3.2) and the packing sum of Eq. (pack_rotate).

Each pin is fixed by mathematics outside the oracle's own code:
  - with q = B^ell the gadget decomposition is the textbook signed base-B
    representation, exact;
  - for other q the reconstruction error obeys the analytic bound
    q/(2 B^ell) + ell B/4;
  - Rotate by k is the negacyclic product with the monomial X^k;
  - KeySwitching preserves the phase: exactly when Decomp is exact and the
    key carries no noise, within the noise bound otherwise;
  - packed ciphertexts decrypt, coefficient j, to the message of LWE_j, which
    for the product outputs is (W x)_j mod t from a plain integer matmul.
"""
import numpy as np
import pytest

import synth

Q = synth.Q60


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _centered(v, q):
    v %= q
    return v - q if v > q // 2 else v


def _phase_poly(orc, A, B, S, q):
    """B - A*S in R_q with S small signed (the RLWE phase)."""
    Sq = np.array([s % q for s in S.tolist()], dtype=np.uint64)
    AS = orc.negacyclic_mul(A, Sq, q)
    return [(int(b) - int(x)) % q for b, x in zip(B, AS)]


@pytest.mark.parametrize("base_log,ell", [(6, 4), (8, 3), (12, 2), (24, 1)])
def test_decompose_is_signed_base_B_when_q_is_B_to_the_ell(orc, base_log, ell):
    q = 1 << (base_log * ell)
    B = 1 << base_log
    vals = [0, 1, q - 1, q // 2, q // 2 - 1, B // 2, B // 2 - 1] + [int(v) for v in _rng(1).integers(0, q, 200)]
    for a in vals:
        d = orc.decompose(a, q, base_log, ell)
        assert all(-B // 2 <= int(x) < B // 2 for x in d)
        assert sum(int(x) * B ** (ell - 1 - l) for l, x in enumerate(d)) % q == a
    for l in range(ell):
        assert orc.gadget(q, base_log, l) == B ** (ell - 1 - l)


@pytest.mark.parametrize("q", [Q, synth.Q_RNS, (1 << 39)])
@pytest.mark.parametrize("base_log,ell", [(26, 1), (13, 2), (8, 3), (5, 4)])
def test_decompose_reconstruction_error_bound(orc, q, base_log, ell):
    B = 1 << base_log
    bound = q / (2 * B ** ell) + ell * B / 4 + 1
    vals = [0, 1, q - 1, q // 2, (q + 1) // 2] + [int(v) for v in _rng(2).integers(0, q, 300, dtype=np.uint64)]
    worst = 0
    for a in vals:
        d = orc.decompose(a, q, base_log, ell)
        assert all(-B // 2 <= int(x) < B // 2 for x in d)
        rec = sum(int(x) * orc.gadget(q, base_log, l) for l, x in enumerate(d))
        err = abs(_centered(a - rec, q))
        worst = max(worst, err)
        assert err <= bound, (a, err, bound)
    # the bound is not vacuous: the rounding error does reach a good part of it
    assert worst > 0.1 * (q / (2 * B ** ell))


def test_rotate_is_the_monomial_product(orc):
    N = 32
    P = _rng(3).integers(0, Q, N, dtype=np.uint64)
    for k in [0, 1, 5, N - 1, N, N + 3, 2 * N - 1]:
        mono = np.zeros(N, dtype=np.uint64)
        if k < N:
            mono[k] = 1
        else:
            mono[k - N] = Q - 1  # X^k = -X^(k-N)
        assert np.array_equal(orc.rotate(P, k, Q), orc.negacyclic_mul(P, mono, Q))
    # X^N = -1 and rotations compose
    neg = np.array([(Q - int(v)) % Q for v in P], dtype=np.uint64)
    assert np.array_equal(orc.rotate(P, N, Q), neg)
    assert np.array_equal(orc.rotate(orc.rotate(P, 7, Q), 9, Q), orc.rotate(P, 16, Q))


def _ksk(orc, n, N, q, base_log, ell, s, S2, sigma, seed):
    g = _rng(seed)
    KA = g.integers(0, q, (n, ell, N), dtype=np.uint64)
    E = np.rint(g.normal(0, sigma, (n, ell, N))).astype(np.int64) if sigma > 0 else np.zeros((n, ell, N), np.int64)
    return KA, orc.ksk_encrypt(KA, E, s, S2, q, base_log, ell), E


def test_keyswitch_preserves_the_phase_exactly_without_noise(orc):
    # q = B^ell: Decomp is exact; noiseless key: the phase moves over unchanged.
    base_log, ell = 6, 4
    q = 1 << 24
    n, N = 48, 32
    g = _rng(4)
    s = g.integers(-1, 2, n)
    S2 = g.integers(-1, 2, N)
    KA, KB, _ = _ksk(orc, n, N, q, base_log, ell, s, S2, 0.0, 5)
    for trial in range(4):
        a = g.integers(0, q, n, dtype=np.uint64)
        b = int(g.integers(0, q))
        A2, B2 = orc.keyswitch(a, b, KA, KB, q, base_log, ell)
        ph = _phase_poly(orc, A2, B2, S2, q)
        assert ph[0] == orc.lwe_phase(a, b, s, q)
        assert all(v == 0 for v in ph[1:])


@pytest.mark.parametrize("base_log,ell", [(26, 1), (13, 2)])
def test_keyswitch_noise_within_the_bound(orc, base_log, ell):
    n, N = 64, 64
    g = _rng(6)
    s = g.integers(-1, 2, n)
    S2 = g.integers(-1, 2, N)
    KA, KB, E = _ksk(orc, n, N, Q, base_log, ell, s, S2, synth.SIGMA, 7)
    B = 1 << base_log
    a = g.integers(0, Q, n, dtype=np.uint64)
    b = int(g.integers(0, Q))
    A2, B2 = orc.keyswitch(a, b, KA, KB, Q, base_log, ell)
    ph = _phase_poly(orc, A2, B2, S2, Q)
    want = orc.lwe_phase(a, b, s, Q)
    # rounding of Decomp times |s_i|, plus digits times the key noise
    digits = np.array([orc.decompose(int(x), Q, base_log, ell) for x in a])
    rnd = int(np.abs(s).sum()) * (Q / (2 * B ** ell) + ell * B / 4)
    for c in range(N):
        noise = int(np.abs(digits).sum(axis=None) * np.abs(E[:, :, c]).max())
        diff = abs(_centered(ph[c] - (want if c == 0 else 0), Q))
        assert diff <= (rnd if c == 0 else 0) + noise + 1


def _product_lwes(orc, N, d_in, m, q, t, seed):
    """LWE outputs of Eq. (LWEdot) for one token: a [m][N], b [m], plus W, x, S."""
    g = _rng(seed)
    S = g.integers(-1, 2, N)
    W = g.integers(-127, 128, (m, d_in)).astype(np.int8)
    X = g.integers(-127, 128, (1, d_in)).astype(np.int8)
    L = synth.blocks(d_in, N)
    A = g.integers(0, q, (1, L, N), dtype=np.uint64)
    E = np.rint(g.normal(0, synth.SIGMA, (1, L, N))).astype(np.int64)
    Bc = orc.encrypt_vectors(A, S, E, X, q, q // t)
    a, b = orc.lwedot_all(W, A, Bc, q)
    return a[0], b[0], W, X[0], S


@pytest.mark.parametrize("N,d_in,m", [(64, 64, 64), (64, 150, 37)])
def test_packed_ciphertext_decrypts_to_the_product(orc, N, d_in, m):
    t = synth.T_PLAIN
    base_log, ell = 26, 1
    a, b, W, x, S = _product_lwes(orc, N, d_in, m, Q, t, 8 + m)
    KA, KB, _ = _ksk(orc, N, N, Q, base_log, ell, S, S, synth.SIGMA, 9)
    A, B = orc.pack(a, b, KA, KB, Q, base_log, ell)
    y = (W.astype(np.int64) @ x.astype(np.int64))
    want = [((int(v) + t // 2) % t) - t // 2 for v in y] + [0] * (N - m)
    ph = _phase_poly(orc, A, B, S, Q)
    assert [orc.decode(v, Q, t) for v in ph] == want
    # and after the ModulusSwitch of Eq. (pack_rotate) to q' = 2^32
    A2, B2 = orc.modswitch(A, Q, 32), orc.modswitch(B, Q, 32)
    ph2 = _phase_poly(orc, A2, B2, S, 1 << 32)
    assert [orc.decode(v, 1 << 32, t) for v in ph2] == want


@pytest.mark.parametrize("base_log,ell", [(8, 3), (13, 3)])
def test_packing_is_exact_when_decomp_is(orc, base_log, ell):
    # q = B^ell (2^24, and the paper's 2^39) and a noiseless key: coefficient
    # j of the packed phase equals the phase of LWE_j exactly, and the unused
    # coefficients are 0.
    q = 1 << (base_log * ell)
    N, n, m = 32, 32, 20
    g = _rng(10)
    S = g.integers(-1, 2, N)
    KA, KB, _ = _ksk(orc, n, N, q, base_log, ell, S, S, 0.0, 11)
    a = g.integers(0, q, (m, n), dtype=np.uint64)
    b = g.integers(0, q, m, dtype=np.uint64)
    A, B = orc.pack(a, b, KA, KB, q, base_log, ell)
    ph = _phase_poly(orc, A, B, S, q)
    assert ph[:m] == [orc.lwe_phase(a[j], int(b[j]), S, q) for j in range(m)]
    assert all(v == 0 for v in ph[m:])


def test_single_lwe_pack_is_its_keyswitch_and_coeffs_agree(orc):
    N, n = 32, 32
    g = _rng(12)
    S = g.integers(-1, 2, N)
    KA, KB, _ = _ksk(orc, n, N, Q, 13, 2, S, S, synth.SIGMA, 13)
    a = g.integers(0, Q, (1, n), dtype=np.uint64)
    b = g.integers(0, Q, 1, dtype=np.uint64)
    A, B = orc.pack(a, b, KA, KB, Q, 13, 2)
    A1, B1 = orc.keyswitch(a[0], int(b[0]), KA, KB, Q, 13, 2)
    assert np.array_equal(A, A1) and np.array_equal(B, B1)
    m = 23
    a = g.integers(0, Q, (m, n), dtype=np.uint64)
    b = g.integers(0, Q, m, dtype=np.uint64)
    A, B = orc.pack(a, b, KA, KB, Q, 13, 2)
    rs = [0, 1, 5, 22, 23, N - 1]
    Ac, Bc = orc.pack_coeffs(a, b, KA, KB, Q, 13, 2, rs)
    assert np.array_equal(Ac, A[rs]) and np.array_equal(Bc, B[rs])
