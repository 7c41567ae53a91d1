/*
 * phe_oracle.c -- plain, slow, exact CPU oracle for the server-side hot path
 * of "Private LoRA Fine-tuning of Open-Source LLMs with Homomorphic
 * Encryption" (arXiv 2505.07329).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or constant generator with the CUDA
 * library: every constant (primitive roots, N^-1, ...) is recomputed here.
 *
 * All arithmetic is exact integer arithmetic: products are formed in 128-bit
 * integers and reduced with the C '%' operator, so that each function can be
 * checked against the paper by eye.  There is no blocking, fusion or lazy
 * reduction.
 *
 * What each function follows:
 *   - RLWE / LWE ciphertexts, B = A*S + E + Delta*M ........ Sec. 3.1
 *   - SampleExtract(RLWE, h) (both index branches) .......... Sec. 3.2, SampleExtract equation
 *   - block split x -> x_hat_i, zero padding ................ Sec. 4.3.1
 *   - reversed weight encoding w_hat_ij[k] = w_j[iN+N-1-k] .. Sec. 4.3.1
 *   - LWE(x.w_j) = sum_i SampleExtract(RLWE(x_hat_i).w_hat_ij, N-1)  Eq. (LWEdot)
 *   - ModulusSwitch q -> q_out .............................. Sec. 3.2, Sec. 4.3.1
 *   - seeded mask generation ("Mask Generation via PRNG") ... Sec. 3.1; the PRNG
 *     is not named by the paper; this oracle reads it as the ChaCha20 block
 *     function of RFC 8439 (see oracle_expand_mask).
 *   - Decomp, KeySwitching, Rotate ........................... Sec. 3.2
 *   - output packing sum_j Rotate(KeySwitching(LWE_j), j) ..... Eq. (pack_rotate), Sec. 4.3.1
 *   - wire records: seed + bit-packed body in, bit-packed results out  Sec. 4.4, Sec. 4.5
 *
 * Parity pins (closed forms, library routines, brute force) live in tests/.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* Z_q arithmetic by definition                                              */
/* ------------------------------------------------------------------------ */

static uint64_t mod_add(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + b) % q); }
static uint64_t mod_sub(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + q - b) % q); }
static uint64_t mod_mul(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }

/* Reduce a signed 128-bit integer into [0, q). */
static uint64_t mod_i128(i128 v, uint64_t q) {
    i128 r = v % (i128)q;
    if (r < 0) r += (i128)q;
    return (uint64_t)r;
}

uint64_t oracle_powmod(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mod_mul(r, b, q);
        b = mod_mul(b, b, q);
        e >>= 1;
    }
    return r;
}

/* Deterministic Miller-Rabin for n < 2^64 (the first twelve primes as bases
 * are known to suffice below 3.3e24). */
int oracle_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 12; ++i) {
        uint64_t x = oracle_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; ++r) {
            x = mod_mul(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* A primitive 2N-th root of unity psi mod a prime q with q = 1 (mod 2N):
 * psi^N = -1.  Found by trying g = 2, 3, ... and taking g^((q-1)/2N). */
uint64_t oracle_find_psi(uint64_t q, uint32_t N) {
    uint64_t twoN = 2ull * N;
    if ((q - 1) % twoN != 0) return 0;
    for (uint64_t g = 2; g < 1000000; ++g) {
        uint64_t psi = oracle_powmod(g, (q - 1) / twoN, q);
        if (oracle_powmod(psi, N, q) == q - 1) return psi;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Negacyclic products in R_q = Z_q[X]/(X^N+1)                               */
/* ------------------------------------------------------------------------ */

/* c = a*b in R_q by the schoolbook definition
 *   c_r = sum_{u+v=r} a_u b_v - sum_{u+v=r+N} a_u b_v  (mod q).
 * Both operands are arbitrary elements of Z_q. */
void oracle_negacyclic_mul(const uint64_t* a, const uint64_t* b, uint64_t* c, uint32_t N, uint64_t q) {
    for (uint32_t r = 0; r < N; ++r) {
        uint64_t acc = 0;
        for (uint32_t u = 0; u < N; ++u) {
            if (u <= r) {
                acc = mod_add(acc, mod_mul(a[u], b[r - u], q), q);
            } else {
                acc = mod_sub(acc, mod_mul(a[u], b[r + N - u], q), q);
            }
        }
        c[r] = acc;
    }
}

/* c = a*w in Z[X]/(X^N+1) followed by reduction mod q, where w has small
 * signed integer coefficients (the clear weights).  Because w_b is congruent
 * to its signed value mod q, this equals the product in R_q; the sums are
 * exact in 128-bit integers (|a_u w_b| < 2^70, at most N <= 2^14 terms). */
static void negacyclic_mul_small(const uint64_t* a, const int64_t* w, uint64_t* c, uint32_t N, uint64_t q) {
    for (uint32_t r = 0; r < N; ++r) {
        i128 acc = 0;
        for (uint32_t u = 0; u < N; ++u) {
            if (u <= r) acc += (i128)a[u] * w[r - u];
            else        acc -= (i128)a[u] * w[r + N - u];
        }
        c[r] = mod_i128(acc, q);
    }
}

/* ------------------------------------------------------------------------ */
/* Number-theoretic transform (used by the oracle's NTT product path and by  */
/* the CPU baseline).  Textbook form: twist by psi^k, cyclic radix-2 DIT     */
/* transform with omega = psi^2 over a bit-reversed copy, and the inverse    */
/* with omega^-1, N^-1 and the untwist psi^-k.                               */
/* ------------------------------------------------------------------------ */

static uint32_t bit_reverse(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

static void cyclic_ntt(uint64_t* a, uint32_t N, uint64_t omega, uint64_t q) {
    int bits = 0;
    while ((1u << bits) < N) ++bits;
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t j = bit_reverse(i, bits);
        if (j > i) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (uint32_t len = 2; len <= N; len <<= 1) {
        uint64_t wl = oracle_powmod(omega, N / len, q);
        for (uint32_t s = 0; s < N; s += len) {
            uint64_t w = 1;
            for (uint32_t k = 0; k < len / 2; ++k) {
                uint64_t u = a[s + k];
                uint64_t v = mod_mul(a[s + k + len / 2], w, q);
                a[s + k] = mod_add(u, v, q);
                a[s + k + len / 2] = mod_sub(u, v, q);
                w = mod_mul(w, wl, q);
            }
        }
    }
}

/* Forward negacyclic NTT, natural order in and out: a_hat_k = sum_u a_u psi^{(2k+1)u}. */
void oracle_ntt_forward(uint64_t* a, uint32_t N, uint64_t q, uint64_t psi) {
    uint64_t t = 1;
    for (uint32_t u = 0; u < N; ++u) { a[u] = mod_mul(a[u], t, q); t = mod_mul(t, psi, q); }
    cyclic_ntt(a, N, mod_mul(psi, psi, q), q);
}

/* Inverse of oracle_ntt_forward. */
void oracle_ntt_inverse(uint64_t* a, uint32_t N, uint64_t q, uint64_t psi) {
    uint64_t psi_inv = oracle_powmod(psi, q - 2, q);
    cyclic_ntt(a, N, mod_mul(psi_inv, psi_inv, q), q);
    uint64_t n_inv = oracle_powmod(N % q, q - 2, q);
    uint64_t t = n_inv;
    for (uint32_t u = 0; u < N; ++u) { a[u] = mod_mul(a[u], t, q); t = mod_mul(t, psi_inv, q); }
}

/* c = a*b in R_q through the NTT (prime q = 1 mod 2N only). */
void oracle_negacyclic_mul_ntt(const uint64_t* a, const uint64_t* b, uint64_t* c, uint32_t N, uint64_t q) {
    uint64_t psi = oracle_find_psi(q, N);
    uint64_t* fa = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* fb = (uint64_t*)malloc(sizeof(uint64_t) * N);
    for (uint32_t u = 0; u < N; ++u) { fa[u] = a[u] % q; fb[u] = b[u] % q; }
    oracle_ntt_forward(fa, N, q, psi);
    oracle_ntt_forward(fb, N, q, psi);
    for (uint32_t u = 0; u < N; ++u) c[u] = mod_mul(fa[u], fb[u], q);
    oracle_ntt_inverse(c, N, q, psi);
    free(fa);
    free(fb);
}

/* ------------------------------------------------------------------------ */
/* SampleExtract (Sec. 3.2):                                                 */
/*   a'_m = A_{h-m}        for 0 <= m <= h                                   */
/*   a'_m = -A_{N+h-m}     for h <  m < N                                    */
/*   b'   = B_h                                                              */
/* ------------------------------------------------------------------------ */
void oracle_sample_extract(const uint64_t* A, const uint64_t* B, uint32_t N, uint32_t h, uint64_t q,
                           uint64_t* a_out, uint64_t* b_out) {
    for (uint32_t m = 0; m < N; ++m) {
        if (m <= h) a_out[m] = A[h - m] % q;
        else        a_out[m] = mod_sub(0, A[N + h - m] % q, q);
    }
    *b_out = B[h] % q;
}

/* Reversed weight block (Sec. 4.3.1): w_hat_ij[k] = w_j[iN + N-1-k], zero past d_in.
 * w_row is row j of W (length d_in); the result is a small signed polynomial. */
void oracle_encode_weight_block(const int8_t* w_row, uint32_t d_in, uint32_t i, uint32_t N, int64_t* w_hat) {
    for (uint32_t k = 0; k < N; ++k) {
        uint64_t src = (uint64_t)i * N + (N - 1 - k);
        w_hat[k] = (src < d_in) ? (int64_t)w_row[src] : 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. (LWEdot): LWE(x.w_j) = sum_i SampleExtract(RLWE(x_hat_i) . w_hat_ij, N-1)  */
/*                                                                          */
/* Inputs for one token: A, B of L = ceil(d_in/N) blocks, [L][N], in Z_q.    */
/* Output for row j: mask a'[N] and body b' (mod q).                         */
/* method 0: full negacyclic products of A_i and B_i with w_hat_ij, then     */
/*           SampleExtract at N-1, then the block sum (the definition).      */
/* method 1: the same products through the NTT (prime q only).               */
/* ------------------------------------------------------------------------ */
static void lwedot_one(const int8_t* w_row, uint32_t d_in, const uint64_t* A, const uint64_t* B,
                       uint32_t N, uint64_t q, int method, uint64_t* a_out, uint64_t* b_out) {
    uint32_t L = (d_in + N - 1) / N;
    int64_t* w_hat = (int64_t*)malloc(sizeof(int64_t) * N);
    uint64_t* w_hat_q = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* PA = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* PB = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* ea = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t eb = 0;
    for (uint32_t m = 0; m < N; ++m) a_out[m] = 0;
    *b_out = 0;
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t* Ai = A + (uint64_t)i * N;
        const uint64_t* Bi = B + (uint64_t)i * N;
        oracle_encode_weight_block(w_row, d_in, i, N, w_hat);
        if (method == 0) {
            negacyclic_mul_small(Ai, w_hat, PA, N, q);
            negacyclic_mul_small(Bi, w_hat, PB, N, q);
        } else {
            for (uint32_t k = 0; k < N; ++k) w_hat_q[k] = mod_i128((i128)w_hat[k], q);
            oracle_negacyclic_mul_ntt(Ai, w_hat_q, PA, N, q);
            oracle_negacyclic_mul_ntt(Bi, w_hat_q, PB, N, q);
        }
        oracle_sample_extract(PA, PB, N, N - 1, q, ea, &eb);
        for (uint32_t m = 0; m < N; ++m) a_out[m] = mod_add(a_out[m], ea[m], q);
        *b_out = mod_add(*b_out, eb, q);
    }
    free(w_hat); free(w_hat_q); free(PA); free(PB); free(ea);
}

/* Batch form over a list of (token, row) pairs.
 *   W      [d_out][d_in] int8, row-major (row j = w_j)
 *   A, B   [T][L][N] u64 in [0, q)
 *   pairs  [n_pairs][2] = (token t, row j)
 *   a_out  [n_pairs][N], b_out [n_pairs]   (mod q, before any modulus switch)
 * Pairs are independent; an OpenMP loop spreads them over host threads. */
void oracle_lwedot_pairs(const int8_t* W, uint32_t d_out, uint32_t d_in, const uint64_t* A, const uint64_t* B,
                         uint32_t N, uint64_t q, int method, const uint32_t* pairs, uint64_t n_pairs,
                         uint64_t* a_out, uint64_t* b_out) {
    (void)d_out;
    uint32_t L = (d_in + N - 1) / N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < (int64_t)n_pairs; ++p) {
        uint32_t t = pairs[2 * p], j = pairs[2 * p + 1];
        lwedot_one(W + (uint64_t)j * d_in, d_in, A + (uint64_t)t * L * N, B + (uint64_t)t * L * N, N, q, method,
                   a_out + (uint64_t)p * N, b_out + p);
    }
}

/* Second, independent path: the closed form of the same result,
 *   a'_j[m] = sum_k W[j,k] G[k,m],  b'_j = sum_k W[j,k] B[k]   (mod q)
 * with k = iN + kb and G[k,m] = A_i[kb-m] if kb >= m, else -A_i[kb-m+N].
 * It follows from writing out the product coefficient N-1-m of Eq. (LWEdot)
 * term by term. */
void oracle_lwedot_closed_form(const int8_t* W, uint32_t d_in, const uint64_t* A, const uint64_t* B, uint32_t N,
                               uint64_t q, uint32_t t, uint32_t j, uint64_t* a_out, uint64_t* b_out) {
    uint32_t L = (d_in + N - 1) / N;
    const int8_t* w = W + (uint64_t)j * d_in;
    const uint64_t* At = A + (uint64_t)t * L * N;
    const uint64_t* Bt = B + (uint64_t)t * L * N;
    for (uint32_t m = 0; m < N; ++m) {
        i128 acc = 0;
        for (uint32_t k = 0; k < d_in; ++k) {
            uint32_t i = k / N, kb = k % N;
            const uint64_t* Ai = At + (uint64_t)i * N;
            if (kb >= m) acc += (i128)w[k] * Ai[kb - m];
            else         acc -= (i128)w[k] * Ai[kb + N - m];
        }
        a_out[m] = mod_i128(acc, q);
    }
    i128 accb = 0;
    for (uint32_t k = 0; k < d_in; ++k) accb += (i128)w[k] * Bt[k];
    *b_out = mod_i128(accb, q);
}

/* ------------------------------------------------------------------------ */
/* ModulusSwitch q -> q_out = 2^k (Sec. 3.2): c' = floor((c*q_out + floor(q/2)) / q) mod q_out,  */
/* i.e. round(c*q_out/q) with ties rounded up; computed in exact 128-bit integers.               */
/* ------------------------------------------------------------------------ */
uint64_t oracle_modswitch(uint64_t c, uint64_t q, uint32_t log2_qout) {
    u128 num = ((u128)(c % q) << log2_qout) + (q / 2);
    u128 quo = num / q;
    u128 mask = (((u128)1) << log2_qout) - 1;
    return (uint64_t)(quo & mask);
}

void oracle_modswitch_array(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t q, uint32_t log2_qout) {
    for (uint64_t i = 0; i < n; ++i) out[i] = oracle_modswitch(in[i], q, log2_qout);
}

/* ------------------------------------------------------------------------ */
/* Client side (test only): RLWE encryption of one block and LWE decryption. */
/* ------------------------------------------------------------------------ */

/* B = A*S + E + Delta*M  (mod q)   (Sec. 3.1).  S, E, M are small signed
 * integer polynomials (key, noise, message); A is in Z_q. */
void oracle_rlwe_encrypt(const uint64_t* A, const int64_t* S, const int64_t* E, const int64_t* M, uint32_t N,
                         uint64_t q, uint64_t delta, uint64_t* B) {
    negacyclic_mul_small(A, S, B, N, q);
    for (uint32_t k = 0; k < N; ++k) {
        uint64_t em = mod_add(mod_i128((i128)E[k], q), mod_mul(delta % q, mod_i128((i128)M[k], q), q), q);
        B[k] = mod_add(B[k], em, q);
    }
}

/* Phase of an LWE ciphertext under key s (modulus Q given as Q_lo/Q_hi so
 * that Q = 2^64 is expressible; here Q <= 2^63 in practice):
 *   v = b - <a, s>  (mod Q). */
uint64_t oracle_lwe_phase(const uint64_t* a, uint64_t b, const int64_t* s, uint32_t n, uint64_t Q) {
    i128 acc = (i128)(b % Q);
    for (uint32_t m = 0; m < n; ++m) acc -= (i128)(a[m] % Q) * s[m];
    return mod_i128(acc, Q);
}

/* Decode a phase: round(t*v/Q) mod t, centred into [-t/2, t/2). */
int64_t oracle_decode(uint64_t v, uint64_t Q, uint64_t t) {
    u128 num = (u128)v * t + Q / 2;
    uint64_t m = (uint64_t)((num / Q) % t);
    int64_t r = (int64_t)m;
    if (m >= t / 2) r -= (int64_t)t;
    return r;
}

/* ------------------------------------------------------------------------ */
/* Seeded mask (Sec. 3.1, "Mask Generation via PRNG"), read as ChaCha20.      */
/* ------------------------------------------------------------------------ */

static uint32_t rotl32(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }

static void quarter_round(uint32_t* x, int a, int b, int c, int d) {
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 16);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 12);
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 8);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 7);
}

/* The ChaCha20 block function (RFC 8439, Sec. 2.3): 16 output words. */
void oracle_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3], uint32_t out[16]) {
    uint32_t init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                         key[0], key[1], key[2], key[3], key[4], key[5], key[6], key[7],
                         counter, nonce[0], nonce[1], nonce[2]};
    uint32_t x[16];
    memcpy(x, init, sizeof(x));
    for (int round = 0; round < 10; ++round) {
        quarter_round(x, 0, 4, 8, 12);
        quarter_round(x, 1, 5, 9, 13);
        quarter_round(x, 2, 6, 10, 14);
        quarter_round(x, 3, 7, 11, 15);
        quarter_round(x, 0, 5, 10, 15);
        quarter_round(x, 1, 6, 11, 12);
        quarter_round(x, 2, 7, 8, 13);
        quarter_round(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; ++i) out[i] = x[i] + init[i];
}

/* Mask polynomial A of one ciphertext from its 64-bit seed (Sec. 3.1: the
 * client sends the seed and the body; both sides regenerate A).  Each
 * ciphertext carries its own seed, so the expansion does not depend on where
 * the ciphertext sits in a batch: key = (seed lo, seed hi, 0, ..., 0),
 * nonce = 0; coefficient m takes the 128-bit little-endian integer formed by
 * words 4*(m%4) .. 4*(m%4)+3 of the block with counter m/4, reduced mod q. */
void oracle_expand_mask(uint64_t seed, uint32_t N, uint64_t q, uint64_t* A) {
    uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
    uint32_t nonce[3] = {0, 0, 0};
    uint32_t ks[16];
    for (uint32_t m = 0; m < N; ++m) {
        if (m % 4 == 0) oracle_chacha20_block(key, m / 4, nonce, ks);
        const uint32_t* w = ks + 4 * (m % 4);
        u128 v = (u128)w[0] | ((u128)w[1] << 32) | ((u128)w[2] << 64) | ((u128)w[3] << 96);
        A[m] = (uint64_t)(v % q);
    }
}

/* ------------------------------------------------------------------------ */
/* Output packing: KeySwitching and Rotate (Sec. 3.2), Eq. (pack_rotate).     */
/* ------------------------------------------------------------------------ */

/* The paper takes Decomp from TFHE without fixing it; this oracle reads it as
 * the approximate signed gadget decomposition with base B = 2^base_log and
 * ell levels (base_log * ell <= 62):
 *   a~ = ModulusSwitch of a from q to B^ell (the same rounding as above),
 *   digits d_0 (most significant) .. d_{ell-1} in [-B/2, B/2) with
 *   sum_l d_l B^(ell-1-l) = a~ (mod B^ell),
 * and the matching gadget g_l = round(q / B^(l+1)) (ties up), so that
 * sum_l d_l g_l = a (mod q) up to q/(2 B^ell) + ell B/4. */
uint64_t oracle_gadget(uint64_t q, uint32_t base_log, uint32_t l) {
    u128 den = (u128)1 << (base_log * (l + 1));
    return (uint64_t)(((u128)q + den / 2) / den);
}

void oracle_decompose(uint64_t a, uint64_t q, uint32_t base_log, uint32_t ell, int64_t* d) {
    uint64_t v = oracle_modswitch(a, q, base_log * ell);
    const uint64_t B = (uint64_t)1 << base_log;
    for (int l = (int)ell - 1; l >= 0; --l) {
        int64_t r = (int64_t)(v & (B - 1));
        v >>= base_log;
        if (r >= (int64_t)(B / 2)) {  /* signed digit: borrow from the next level */
            r -= (int64_t)B;
            v += 1;
        }
        d[l] = r;
    }
    /* a carry out of d_0 is a multiple of B^ell, i.e. of q after scaling: dropped */
}

/* Key-switching key (client side, test only): KSK_{i,l} is an RLWE encryption
 * under S2 of the constant polynomial s_i g_l:
 *   KB_{i,l} = KA_{i,l} * S2 + E_{i,l} + s_i g_l X^0   (mod q).
 * KA, E, KB are [n][ell][N]; s has n entries (the LWE key), S2 N (the target key). */
void oracle_ksk_encrypt(const uint64_t* KA, const int64_t* E, const int64_t* s, uint32_t n, const int64_t* S2,
                        uint32_t N, uint64_t q, uint32_t base_log, uint32_t ell, uint64_t* KB) {
    for (uint32_t i = 0; i < n; ++i) {
        for (uint32_t l = 0; l < ell; ++l) {
            const size_t o = ((size_t)i * ell + l) * N;
            negacyclic_mul_small(KA + o, S2, KB + o, N, q);
            for (uint32_t k = 0; k < N; ++k) KB[o + k] = mod_add(KB[o + k], mod_i128((i128)E[o + k], q), q);
            const uint64_t msg = mod_mul(mod_i128((i128)s[i], q), oracle_gadget(q, base_log, l) % q, q);
            KB[o] = mod_add(KB[o], msg, q);
        }
    }
}

/* KeySwitching of one LWE ciphertext (a, b) of dimension n (Sec. 3.2):
 *   (A', B') = (0, b) - sum_i Decomp(a_i) . KSK_i
 *            = (-sum_{i,l} d_{i,l} KA_{i,l},  b X^0 - sum_{i,l} d_{i,l} KB_{i,l}). */
void oracle_keyswitch(const uint64_t* a, uint64_t b, uint32_t n, const uint64_t* KA, const uint64_t* KB, uint32_t N,
                      uint64_t q, uint32_t base_log, uint32_t ell, uint64_t* A_out, uint64_t* B_out) {
    int64_t* d = (int64_t*)malloc(sizeof(int64_t) * ell);
    for (uint32_t k = 0; k < N; ++k) {
        A_out[k] = 0;
        B_out[k] = 0;
    }
    B_out[0] = b % q;
    for (uint32_t i = 0; i < n; ++i) {
        oracle_decompose(a[i], q, base_log, ell, d);
        for (uint32_t l = 0; l < ell; ++l) {
            const size_t o = ((size_t)i * ell + l) * N;
            const uint64_t dq = mod_i128((i128)d[l], q);
            for (uint32_t k = 0; k < N; ++k) {
                A_out[k] = mod_sub(A_out[k], mod_mul(dq, KA[o + k], q), q);
                B_out[k] = mod_sub(B_out[k], mod_mul(dq, KB[o + k], q), q);
            }
        }
    }
    free(d);
}

/* Rotate (Sec. 3.2): P X^k in R_q.  For 0 <= k < N coefficient r of the result
 * is P_{r-k} when r >= k and -P_{r-k+N} when r < k; X^N = -1 covers N <= k < 2N. */
void oracle_rotate(const uint64_t* P, uint32_t N, uint32_t k, uint64_t q, uint64_t* out) {
    const int negate_all = (k >= N);
    if (negate_all) k -= N;
    for (uint32_t r = 0; r < N; ++r) {
        uint64_t v = (r >= k) ? P[r - k] % q : mod_sub(0, P[r - k + N] % q, q);
        out[r] = negate_all ? mod_sub(0, v, q) : v;
    }
}

/* Eq. (pack_rotate) before its ModulusSwitch: m <= N LWE ciphertexts
 * (a_j, b_j) of dimension n become one RLWE ciphertext
 *   (A, B) = sum_{j<m} Rotate(KeySwitching(LWE_j), j)      (mod q),
 * so that coefficient j of its message is the message of LWE_j.
 * a: [m][n], b: [m]; KA, KB: [n][ell][N]. */
void oracle_pack(const uint64_t* a, const uint64_t* b, uint32_t m, uint32_t n, const uint64_t* KA, const uint64_t* KB,
                 uint32_t N, uint64_t q, uint32_t base_log, uint32_t ell, uint64_t* A_out, uint64_t* B_out) {
    uint64_t* ka = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* kb = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* ra = (uint64_t*)malloc(sizeof(uint64_t) * N);
    uint64_t* rb = (uint64_t*)malloc(sizeof(uint64_t) * N);
    for (uint32_t k = 0; k < N; ++k) {
        A_out[k] = 0;
        B_out[k] = 0;
    }
    for (uint32_t j = 0; j < m; ++j) {
        oracle_keyswitch(a + (size_t)j * n, b[j], n, KA, KB, N, q, base_log, ell, ka, kb);
        oracle_rotate(ka, N, j, q, ra);
        oracle_rotate(kb, N, j, q, rb);
        for (uint32_t k = 0; k < N; ++k) {
            A_out[k] = mod_add(A_out[k], ra[k], q);
            B_out[k] = mod_add(B_out[k], rb[k], q);
        }
    }
    free(ka);
    free(kb);
    free(ra);
    free(rb);
}

/* The same sum evaluated one coefficient at a time, for sampled checks at
 * sizes where oracle_pack is too slow.  Coefficient r of Rotate(P, j) is
 * P_{r-j} (r >= j) or -P_{r-j+N} (r < j), and coefficient c of
 * KeySwitching(LWE_j) is [c = 0] b_j - sum_{i,l} d_{i,l}(a_j[i]) K_{i,l}[c]. */
void oracle_pack_coeffs(const uint64_t* a, const uint64_t* b, uint32_t m, uint32_t n, const uint64_t* KA,
                        const uint64_t* KB, uint32_t N, uint64_t q, uint32_t base_log, uint32_t ell,
                        const uint32_t* rs, uint32_t n_rs, uint64_t* A_out, uint64_t* B_out) {
    int64_t* D = (int64_t*)malloc(sizeof(int64_t) * (size_t)m * n * ell);
    for (size_t ji = 0; ji < (size_t)m * n; ++ji) oracle_decompose(a[ji], q, base_log, ell, D + ji * ell);
#pragma omp parallel for schedule(dynamic, 1)
    for (uint32_t x = 0; x < n_rs; ++x) {
        const uint32_t r = rs[x];
        uint64_t accA = 0, accB = 0;
        for (uint32_t j = 0; j < m; ++j) {
            const int wrapped = r < j;
            const uint32_t c = wrapped ? r + N - j : r - j;
            uint64_t ca = 0, cb = (c == 0) ? b[j] % q : 0;
            for (uint32_t i = 0; i < n; ++i) {
                for (uint32_t l = 0; l < ell; ++l) {
                    const uint64_t dq = mod_i128((i128)D[((size_t)j * n + i) * ell + l], q);
                    const size_t o = ((size_t)i * ell + l) * N + c;
                    ca = mod_sub(ca, mod_mul(dq, KA[o], q), q);
                    cb = mod_sub(cb, mod_mul(dq, KB[o], q), q);
                }
            }
            if (wrapped) {
                ca = mod_sub(0, ca, q);
                cb = mod_sub(0, cb, q);
            }
            accA = mod_add(accA, ca, q);
            accB = mod_add(accB, cb, q);
        }
        A_out[x] = accA;
        B_out[x] = accB;
    }
    free(D);
}

/* ------------------------------------------------------------------------ */
/* Wire format (Sec. 4.4 sizes; Sec. 4.5: the result is "packed into a bit-  */
/* vector").  A record is a little-endian bit stream: field m of width `bits` */
/* occupies stream bits m*bits .. m*bits+bits-1, and stream bit j is bit     */
/* j mod 8 of byte j/8.  Records are padded with zero bits to a multiple of  */
/* 32 bits (the sizes printed in Sec. 4.4 need no padding).                  */
/* ------------------------------------------------------------------------ */

uint64_t oracle_wire_bytes(uint64_t fields, uint32_t bits) { return ((fields * bits + 31) / 32) * 4; }

void oracle_pack_bits(const uint64_t* v, uint64_t n, uint32_t bits, uint8_t* out) {
    const uint64_t nbytes = oracle_wire_bytes(n, bits);
    for (uint64_t i = 0; i < nbytes; ++i) out[i] = 0;
    for (uint64_t m = 0; m < n; ++m) {
        for (uint32_t b = 0; b < bits; ++b) {
            const uint64_t j = m * bits + b;
            if ((v[m] >> b) & 1u) out[j / 8] |= (uint8_t)(1u << (j % 8));
        }
    }
}

void oracle_unpack_bits(const uint8_t* in, uint64_t n, uint32_t bits, uint64_t* v) {
    for (uint64_t m = 0; m < n; ++m) {
        uint64_t x = 0;
        for (uint32_t b = 0; b < bits; ++b) {
            const uint64_t j = m * bits + b;
            if ((in[j / 8] >> (j % 8)) & 1u) x |= (uint64_t)1 << b;
        }
        v[m] = x;
    }
}

/* Input record of one RLWE block as the client sends it (Sec. 3.1 "Mask
 * Generation via PRNG", Sec. 4.4 input size): the 8-byte seed (little
 * endian), then the N body coefficients at bits_q = ceil(log2 q) bits each.
 * Size 8 + wire_bytes(N, bits_q); N = 2048, q = 2^39 gives 8 + 9984. */
void oracle_wire_input_record(uint64_t seed, const uint64_t* B, uint32_t N, uint32_t bits_q, uint8_t* out) {
    for (int i = 0; i < 8; ++i) out[i] = (uint8_t)(seed >> (8 * i));
    oracle_pack_bits(B, N, bits_q, out + 8);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
