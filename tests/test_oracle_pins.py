"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- a closed form, a library routine, brute force on tiny inputs,
or an exact identity that follows from the definitions in the paper
(Sec. 3.1-3.2 and Eq. (LWEdot) in Sec. 4.3.1)."""
from fractions import Fraction

import numpy as np
import pytest
import sympy
from numpy.polynomial import polynomial as P

import synth

Q = synth.Q60
SMALL_Q = 7681  # = 1 + 15 * 2^9, prime: carries negacyclic NTTs up to N = 256


def _full_product_negacyclic(a, b, q):
    """Library route: the full product in Z[X] by numpy's polymul on Python
    ints, then the reduction X^N = -1 by folding the upper half."""
    N = len(a)
    full = P.polymul(np.array([int(v) for v in a], dtype=object), np.array([int(v) for v in b], dtype=object))
    full = list(full) + [0] * (2 * N - len(full))
    return np.array([(full[r] - full[r + N]) % q for r in range(N)], dtype=object)


# --- modulus and roots -------------------------------------------------------

def test_q60_is_an_ntt_prime(orc):
    assert orc.is_prime(Q) and sympy.isprime(Q)
    assert (Q - 1) % (2 * 8192) == 0
    assert Q < 2 ** 60


def test_is_prime_agrees_with_sympy(orc):
    r = np.random.default_rng(5)
    cands = [int(v) for v in r.integers(2, 2 ** 62, size=200, dtype=np.uint64)] + list(range(2, 300))
    cands += [2 ** 61 - 1, 2 ** 61 + 1, 1152921504606830593 + 2, 3215031751]  # 3215031751: strong pseudoprime to 2,3,5,7
    for n in cands:
        assert orc.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("N", [4, 16, 1024, 4096])
def test_psi_is_primitive_2n_th_root(orc, N):
    psi = orc.find_psi(Q, N)
    assert pow(psi, N, Q) == Q - 1
    assert pow(psi, 2 * N, Q) == 1


# --- negacyclic products -----------------------------------------------------

def test_negacyclic_hand_example(orc):
    # In Z[X]/(X^4+1): (1 + X) * X^3 = X^3 + X^4 = X^3 - 1.
    a = [1, 1, 0, 0]
    b = [0, 0, 0, 1]
    assert list(orc.negacyclic_mul(a, b, Q)) == [Q - 1, 0, 0, 1]
    assert list(orc.negacyclic_mul_ntt(a, b, Q)) == [Q - 1, 0, 0, 1]


@pytest.mark.parametrize("k", [0, 1, 5, 15])
def test_multiply_by_monomial_is_negacyclic_rotation(orc, k):
    # Rotate (Sec. 3.2): multiplication by X^k shifts coefficients up by k and
    # negates the ones that wrap past X^N.
    N = 16
    a = synth.uniform_words(N, Q, 11 + k)
    xk = np.zeros(N, dtype=np.uint64)
    xk[k] = 1
    c = orc.negacyclic_mul(a, xk, Q)
    for r in range(N):
        expect = int(a[r - k]) if r >= k else (Q - int(a[r - k + N])) % Q
        assert int(c[r]) == expect


@pytest.mark.parametrize("N", [4, 8, 16, 64])
def test_negacyclic_matches_numpy_polymul(orc, N):
    a = synth.uniform_words(N, Q, 100 + N)
    b = synth.uniform_words(N, Q, 200 + N)
    ref = _full_product_negacyclic(a, b, Q)
    assert [int(v) for v in orc.negacyclic_mul(a, b, Q)] == list(ref)
    assert [int(v) for v in orc.negacyclic_mul_ntt(a, b, Q)] == list(ref)


def test_negacyclic_ntt_small_prime(orc):
    N = 256
    a = synth.uniform_words(N, SMALL_Q, 1)
    b = synth.uniform_words(N, SMALL_Q, 2)
    ref = _full_product_negacyclic(a, b, SMALL_Q)
    assert [int(v) for v in orc.negacyclic_mul_ntt(a, b, SMALL_Q)] == list(ref)


@pytest.mark.parametrize("N", [8, 64])
def test_ntt_is_evaluation_at_odd_powers_of_psi(orc, N):
    # Negacyclic DFT: a_hat_k = a(psi^(2k+1)), the evaluation of a at the
    # roots of X^N + 1; checked with Python's pow, plus the round trip.
    psi = orc.find_psi(Q, N)
    a = synth.uniform_words(N, Q, 7 * N)
    fwd = orc.ntt_forward(a, Q, psi)
    for k in range(N):
        root = pow(psi, 2 * k + 1, Q)
        assert int(fwd[k]) == sum(int(a[u]) * pow(root, u, Q) for u in range(N)) % Q
    assert np.array_equal(orc.ntt_inverse(fwd, Q, psi), a)


# --- SampleExtract and the reversed-weight encoding ---------------------------

def _encrypt_block(orc, N, q, S, seed, msg=None, delta=None):
    A = synth.uniform_words(N, q, seed)
    E = np.rint(np.random.default_rng(seed).normal(0, 3.2, N)).astype(np.int64)
    M = msg if msg is not None else np.random.default_rng(seed + 1).integers(-127, 128, N)
    delta = delta if delta is not None else q // synth.T_PLAIN
    B = orc.rlwe_encrypt(A, S, E, M, q, delta)
    return A, B, E, np.asarray(M, dtype=np.int64), delta


@pytest.mark.parametrize("h", [0, 1, 17, 63])
def test_sample_extract_phase_is_coefficient_h(orc, h):
    # Under key S' = (S_0..S_{N-1}) the extracted LWE has phase
    # b' - <a', S'> = E_h + Delta*M_h exactly (Sec. 3.2); this checks both
    # index branches and the sign of the wrap-around branch.
    N = 64
    S = synth.secret_key(N, "ternary", seed=3)
    A, B, E, M, delta = _encrypt_block(orc, N, Q, S, 40 + h)
    a, b = orc.sample_extract(A, B, h, Q)
    phase = orc.lwe_phase(a, b, S, Q)
    assert phase == (int(E[h]) + delta * int(M[h])) % Q


def test_reversed_weight_encoding_matches_paper(orc):
    w = np.arange(-10, 10, dtype=np.int8)  # d_in = 20
    N = 8
    for i in range(3):
        enc = orc.encode_weight_block(w, i, N)
        for k in range(N):
            src = i * N + N - 1 - k
            assert enc[k] == (int(w[src]) if src < 20 else 0)


@pytest.mark.parametrize("k", [0, 5, 9, 15, 16, 23])
def test_one_hot_weight_gives_sample_extract_at_k(orc, k):
    # With W = e_j e_k^T, Eq. (LWEdot) must return SampleExtract(RLWE(x_hat_i), k mod N)
    # for block i = k // N, i.e. the paper's two-branch formula at h = k mod N.
    N, d_in, d_out, j = 16, 24, 3, 1
    A = synth.uniform_words((1, 2, N), Q, 9)
    B = synth.uniform_words((1, 2, N), Q, 10)
    W = np.zeros((d_out, d_in), dtype=np.int8)
    W[j, k] = 1
    a, b = orc.lwedot_pairs(W, A, B, [(0, j)], Q)
    ea, eb = orc.sample_extract(A[0, k // N], B[0, k // N], k % N, Q)
    assert np.array_equal(a[0], ea) and int(b[0]) == eb


def test_lwedot_brute_force_tiny(orc):
    # Tiny ragged case (d_in = 20, N = 8, L = 3): each block product is formed
    # by numpy's polymul on Python ints, folded mod X^N + 1, coefficient N-1-m
    # is read off and the blocks are summed.
    N, d_in, d_out, T = 8, 20, 5, 2
    L = synth.blocks(d_in, N)
    W = synth.weights(d_out, d_in, seed=4)
    A = synth.uniform_words((T, L, N), Q, 5)
    B = synth.uniform_words((T, L, N), Q, 6)
    a, b = orc.lwedot_all(W, A, B, Q)
    for t in range(T):
        for j in range(d_out):
            acc_a = [0] * N
            acc_b = 0
            for i in range(L):
                w_hat = [int(W[j, i * N + N - 1 - kk]) if i * N + N - 1 - kk < d_in else 0 for kk in range(N)]
                pa = _full_product_negacyclic(A[t, i], w_hat, Q)
                pb = _full_product_negacyclic(B[t, i], w_hat, Q)
                for m in range(N):
                    acc_a[m] = (acc_a[m] + int(pa[N - 1 - m])) % Q
                acc_b = (acc_b + int(pb[N - 1])) % Q
            assert [int(v) for v in a[t, j]] == acc_a
            assert int(b[t, j]) == acc_b


def test_lwedot_paths_agree(orc):
    # Schoolbook (method 0), NTT products (method 1) and the term-by-term
    # closed form agree on a ragged two-block case.
    N, d_in, d_out, T = 64, 100, 6, 3
    L = synth.blocks(d_in, N)
    W = synth.weights(d_out, d_in, seed=8)
    A = synth.uniform_words((T, L, N), Q, 12)
    B = synth.uniform_words((T, L, N), Q, 13)
    a0, b0 = orc.lwedot_all(W, A, B, Q, method=0)
    a1, b1 = orc.lwedot_all(W, A, B, Q, method=1)
    assert np.array_equal(a0, a1) and np.array_equal(b0, b1)
    for t, j in [(0, 0), (1, 3), (2, 5)]:
        ac, bc = orc.lwedot_closed_form(W, A, B, t, j, Q)
        assert np.array_equal(ac, a0[t, j]) and bc == int(b0[t, j])


# --- the whole path against plaintext arithmetic --------------------------------

def _encrypted_batch(orc, N, d_in, d_out, T, key="ternary", q=Q, zero_noise=False, seed=0):
    L = synth.blocks(d_in, N)
    S = synth.secret_key(N, key, seed=synth.SEED_KEY + seed)
    A = synth.masks(T, L, N, q, seed=synth.SEED_MASK + seed)
    E = synth.noise(T, L, N, seed=synth.SEED_ERR + seed)
    if zero_noise:
        E[:] = 0
    X = synth.activations(T, d_in, seed=synth.SEED_X + seed)
    W = synth.weights(d_out, d_in, seed=synth.SEED_W + seed)
    delta = q // synth.T_PLAIN
    B = orc.encrypt_vectors(A, S, E, X, q, delta)
    return W, X, S, A, E, B, delta


def _centered(v, q):
    v %= q
    return v - q if v > q // 2 else v


@pytest.mark.parametrize("N,d_in,d_out", [(64, 64, 8), (64, 150, 7), (256, 256, 4)])
def test_exact_noise_identity(orc, N, d_in, d_out):
    # b' - <a', S> - Delta*(W x)_j == sum_k W[j,k] E[k]   (mod q), exactly:
    # the phase of each output carries exactly the clear dot product and the
    # weighted input noise (Sec. 3.1 with Eq. (LWEdot)).
    T = 3
    W, X, S, A, E, B, delta = _encrypted_batch(orc, N, d_in, d_out, T, seed=N + d_in)
    a, b = orc.lwedot_all(W, A, B, Q)
    Y = X.astype(np.int64) @ W.astype(np.int64).T
    Eflat = E.reshape(T, -1)[:, :d_in]
    for t in range(T):
        for j in range(d_out):
            phase = orc.lwe_phase(a[t, j], int(b[t, j]), S, Q)
            lhs = _centered(phase - delta * int(Y[t, j]), Q)
            rhs = int(np.dot(W[j].astype(np.int64), Eflat[t]))
            assert lhs == rhs


def test_decrypts_to_clear_product_mod_t(orc):
    N, d_in, d_out, T = 256, 300, 9, 4
    W, X, S, A, E, B, delta = _encrypted_batch(orc, N, d_in, d_out, T, seed=77)
    a, b = orc.lwedot_all(W, A, B, Q)
    Y = X.astype(np.int64) @ W.astype(np.int64).T
    t_mod = synth.T_PLAIN
    for t in range(T):
        for j in range(d_out):
            got = orc.decode(orc.lwe_phase(a[t, j], int(b[t, j]), S, Q), Q, t_mod)
            assert got == _centered(int(Y[t, j]), t_mod) or (got - int(Y[t, j])) % t_mod == 0


def test_zero_key_and_noise_gives_scaled_product(orc):
    N, d_in, d_out, T = 64, 100, 5, 2
    W, X, S, A, E, B, delta = _encrypted_batch(orc, N, d_in, d_out, T, key="zero", zero_noise=True, seed=3)
    a, b = orc.lwedot_all(W, A, B, Q)
    Y = X.astype(np.int64) @ W.astype(np.int64).T
    for t in range(T):
        for j in range(d_out):
            assert int(b[t, j]) == (delta * int(Y[t, j])) % Q


def test_zero_mask_gives_zero_output_mask(orc):
    N, d_in, d_out, T = 64, 64, 4, 2
    W = synth.weights(d_out, d_in, seed=1)
    A = np.zeros((T, 1, N), dtype=np.uint64)
    B = synth.uniform_words((T, 1, N), Q, 2)
    a, b = orc.lwedot_all(W, A, B, Q)
    assert not a.any()


def test_linearity_in_w(orc):
    N, d_in, d_out, T = 64, 80, 4, 2
    L = synth.blocks(d_in, N)
    W1 = (synth.weights(d_out, d_in, seed=1) // 2).astype(np.int8)
    W2 = (synth.weights(d_out, d_in, seed=2) // 2).astype(np.int8)
    A = synth.uniform_words((T, L, N), Q, 3)
    B = synth.uniform_words((T, L, N), Q, 4)
    a1, b1 = orc.lwedot_all(W1, A, B, Q)
    a2, b2 = orc.lwedot_all(W2, A, B, Q)
    a3, b3 = orc.lwedot_all((W1.astype(np.int16) + W2).astype(np.int8), A, B, Q)
    s = (a1.astype(object) + a2.astype(object)) % Q
    assert np.array_equal(a3.astype(object), s)
    assert np.array_equal(b3.astype(object), (b1.astype(object) + b2.astype(object)) % Q)


# --- ModulusSwitch ----------------------------------------------------------------

@pytest.mark.parametrize("k", [26, 32, 1])
def test_modswitch_closed_form(orc, k):
    # c' = round(c * 2^k / q) (ties up) mod 2^k, checked with exact rationals.
    qs = [Q, 2 ** 39, (1 << 50) + 1]
    for q in qs:
        cs = [0, 1, 2, q // 2, q // 2 + 1, q - 1, q - 2] + [int(v) for v in synth.uniform_words(200, q, k)]
        got = orc.modswitch(np.array(cs, dtype=np.uint64), q, k)
        for c, g in zip(cs, got):
            x = Fraction(c * 2 ** k, q)
            expect = int(x + Fraction(1, 2)) if x.denominator != 1 else int(x)
            # floor(x + 1/2) for positive x
            expect = (x + Fraction(1, 2)).__floor__() % (2 ** k)
            assert int(g) == expect, (q, c)


def test_modswitch_ties_round_up_for_power_of_two_q(orc):
    # q = 2^39 -> 2^26: c mod 2^13 = 2^12 is an exact tie and rounds up.
    q, k = 2 ** 39, 26
    c = (5 << 13) | (1 << 12)
    assert orc.modswitch_one(c, q, k) == 6
    assert orc.modswitch_one(c - 1, q, k) == 5


def test_switched_outputs_still_decrypt(orc):
    # After switching every word of the LWE outputs to q' = 2^32, decryption
    # with modulus q' still yields (W x)_j mod t, and the rounding error of the
    # phase stays within (1 + ||S||_1)/2 of the rescaled phase.
    N, d_in, d_out, T = 256, 256, 6, 3
    W, X, S, A, E, B, delta = _encrypted_batch(orc, N, d_in, d_out, T, seed=91)
    a, b = orc.lwedot_all(W, A, B, Q)
    k = synth.LOG2_QOUT
    Qp = 2 ** k
    a_s = orc.modswitch(a, Q, k)
    b_s = orc.modswitch(b, Q, k)
    Y = X.astype(np.int64) @ W.astype(np.int64).T
    l1 = int(np.abs(S).sum())
    for t in range(T):
        for j in range(d_out):
            v = orc.lwe_phase(a[t, j], int(b[t, j]), S, Q)
            vs = orc.lwe_phase(a_s[t, j], int(b_s[t, j]), S, Qp)
            scaled = Fraction(v * Qp, Q)
            diff = Fraction(vs) - scaled
            # compare on the circle Z_{q'}
            diff = diff - Qp * round(diff / Qp)
            assert abs(diff) <= Fraction(1 + l1, 2)
            got = orc.decode(vs, Qp, synth.T_PLAIN)
            assert (got - int(Y[t, j])) % synth.T_PLAIN == 0


# --- seeded masks ---------------------------------------------------------------------

def test_chacha20_block_matches_cryptography_library(orc):
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms
    r = np.random.default_rng(1)
    for trial in range(4):
        key = r.integers(0, 2 ** 32, size=8, dtype=np.uint64).astype(np.uint32)
        nonce = r.integers(0, 2 ** 32, size=3, dtype=np.uint64).astype(np.uint32)
        counter = int(r.integers(0, 2 ** 31))
        full_nonce = counter.to_bytes(4, "little") + nonce.astype("<u4").tobytes()
        enc = Cipher(algorithms.ChaCha20(key.astype("<u4").tobytes(), full_nonce), mode=None).encryptor()
        ks = enc.update(b"\x00" * 64)
        assert np.array_equal(orc.chacha20_block(key, counter, nonce), np.frombuffer(ks, dtype="<u4"))


def test_expand_mask_reads_chacha_keystream(orc):
    # seeded mask: ChaCha20 keystream under key = seed, nonce = 0, 128 bits
    # per coefficient reduced mod q (reading of the unnamed PRNG of Sec. 3.1)
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms
    seed, N = 0x1234_5678_9ABC_DEF0, 64
    A = orc.expand_mask(seed, N, Q)
    key = seed.to_bytes(8, "little") + b"\x00" * 24
    ks = Cipher(algorithms.ChaCha20(key, b"\x00" * 16), mode=None).encryptor().update(b"\x00" * (16 * N))
    for m in range(N):
        v = int.from_bytes(ks[16 * m:16 * m + 16], "little")
        assert int(A[m]) == v % Q
    A39 = orc.expand_mask(seed, N, 2 ** 39)
    assert int(A39.max()) < 2 ** 39
    assert not np.array_equal(orc.expand_mask(seed + 1, N, Q), A)
