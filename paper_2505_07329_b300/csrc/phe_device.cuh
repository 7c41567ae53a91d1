// Device-side modular arithmetic and register-blocked negacyclic NTT passes.
//
// Arithmetic follows published methods:
//   * Shoup's precomputed-quotient multiplication and Harvey's lazy
//     butterflies (D. Harvey, "Faster arithmetic for number-theoretic
//     transforms", J. Symb. Comp. 2014): values are kept in [0, 2q) or
//     [0, 4q) and only reduced where a bound requires it (q < 2^61).
//   * Negacyclic transforms with the psi-twist merged into the twiddles,
//     Cooley-Tukey forward (natural in, bit-reversed out) and
//     Gentleman-Sande inverse (bit-reversed in, natural out) (P. Longa,
//     M. Naehrig, "Speeding up the number theoretic transform for faster
//     ideal lattice-based cryptography", CANS 2016).
//   * Barrett's estimated quotient (P. Barrett, CRYPTO 1986) for the exact
//     rounding division of the modulus switch.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace phe {

using u64 = unsigned long long;
using u32 = unsigned int;

// Constants of one ring R_q = Z_q[X]/(X^N+1) and of the switch q -> 2^k.
struct RingConst {
  u64 q;          // ciphertext modulus, prime, 2^53 < q < 2^61, q = 1 mod 2N
  u64 q2;         // 2q
  u64 q4;         // 4q
  u64 half_q;     // floor(q/2)
  u64 ms_mu;      // floor(2^(64+s) / q), s = floor(log2 q): Barrett constant of the switch
  u64 red_mu;     // floor(2^64 / q): Barrett constant for reducing a 64-bit word
  u64 c30;        // 2^30 mod q (recombines the split body accumulators)
  u64 c30p;       // Shoup quotient of c30
  u64 c60;        // 2^60 mod q
  u64 c60p;       // Shoup quotient of c60
  u64 c64;        // 2^64 mod q (reduces 128-bit keystream words of seeded masks)
  u64 c64p;       // Shoup quotient of c64
  u64 c32;        // 2^32 mod q (recombines the byte-plane body parts)
  u64 c32p;       // Shoup quotient of c32
  u32 ms_s;       // s = floor(log2 q)
  u32 log2_qout;  // k: output modulus 2^k, 1 <= k <= 32
};

// x*w mod q in [0, 2q) for any 64-bit x, with w < q and wp = floor(w 2^64 / q).
__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q) {
  const u64 quo = __umul64hi(wp, x);
  return x * w - quo * q;
}

// Shoup product with a cheaper quotient estimate.  With x = x1 2^32 + x0 and
// wp = w1 2^32 + w0, the estimate w1 x1 + hi32(w1 x0) + hi32(w0 x1) drops
// the low x low partial product and the carries of the two cross terms, so
// it is at most 2 below floor(wp x / 2^64) and never above it: the result
// x w - quo q lies in [0, 4q).  One wide and two high-half 32-bit multiplies
// replace the four wide multiplies of a full 64x64 high product.
__device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q) {
  const u32 x0 = (u32)x, x1 = (u32)(x >> 32);
  const u32 w0 = (u32)wp, w1 = (u32)(wp >> 32);
  const u64 quo = (u64)w1 * x1 + __umulhi(w1, x0) + __umulhi(w0, x1);
  return x * w - quo * q;
}

// Gentleman-Sande butterfly kept in [0, 4q) (Harvey's lazy butterfly with
// one more factor of two of headroom, valid for 8q < 2^64).
// In: X, Y in [0, 4q).  Out: X <- X + Y, Y <- (X - Y) w, both in [0, 4q).
__device__ __forceinline__ void gs_bfly(u64& X, u64& Y, u64 w, u64 wp, u64 q, u64 q4) {
  u64 s = X + Y;
  s = (s >= q4) ? s - q4 : s;
  const u64 d = X - Y + q4;
  Y = mul_shoup_lazy(d, w, wp, q);
  X = s;
}

// Cooley-Tukey butterfly, Harvey's lazy form.  In: X, Y in [0, 4q).
// Out: X <- X + Y w, Y <- X - Y w, both in [0, 4q).
__device__ __forceinline__ void ct_bfly(u64& X, u64& Y, u64 w, u64 wp, u64 q, u64 q2) {
  const u64 x = (X >= q2) ? X - q2 : X;
  const u64 t = mul_shoup(Y, w, wp, q);
  X = x + t;
  Y = x - t + q2;
}

__device__ __forceinline__ u64 reduce_2q(u64 x, u64 q) { return (x >= q) ? x - q : x; }
__device__ __forceinline__ u64 reduce_4q(u64 x, u64 q, u64 q2) {
  x = (x >= q2) ? x - q2 : x;
  return (x >= q) ? x - q : x;
}

// Any 64-bit word to [0, q): quotient estimate floor(c floor(2^64/q) / 2^64)
// is at most one below floor(c/q) (Barrett), so one correction suffices.
__device__ __forceinline__ u64 reduce_word(u64 c, const RingConst& rc) {
  const u64 quo = __umul64hi(c, rc.red_mu);
  const u64 r = c - quo * rc.q;
  return (r >= rc.q) ? r - rc.q : r;
}

// ---------------------------------------------------------------------------
// 32-bit residue arithmetic for an RNS modulus q = p1 p2 (p_i < 2^30): the
// same Shoup / Harvey forms on 32-bit words, values kept in [0, 2p) or [0, 4p).
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 mul_shoup32(u32 x, u32 w, u32 wp, u32 p) {
  return x * w - __umulhi(wp, x) * p;  // [0, 2p) for any 32-bit x
}
__device__ __forceinline__ u32 sub_if32(u32 x, u32 m) { return min(x, x - m); }  // x < 2m -> [0, m)
__device__ __forceinline__ void gs_bfly32(u32& X, u32& Y, u32 w, u32 wp, u32 p, u32 p2) {
  const u32 s = sub_if32(X + Y, p2);
  const u32 d = X - Y + p2;
  Y = mul_shoup32(d, w, wp, p);
  X = s;
}
__device__ __forceinline__ void ct_bfly32(u32& X, u32& Y, u32 w, u32 wp, u32 p, u32 p2) {
  const u32 x = sub_if32(X, p2);
  const u32 t = mul_shoup32(Y, w, wp, p);
  X = x + t;
  Y = x - t + p2;
}

// Constants of the RNS modulus q = p1 p2 (p1 < p2 < 2^30, both = 1 mod 2N).
struct RnsConst {
  u32 p1, p2;
  u32 inv, invp;      // p1^-1 mod p2 and its Shoup quotient (CRT)
  u32 c32a, c32ap;    // 2^32 mod p1 and its Shoup quotient
  u32 c32b, c32bp;    // 2^32 mod p2 and its Shoup quotient
  // switch to 2^k from residues: 2^k = a1 p1 + b1 = a2 p2 + b2
  u32 a1, b1, b1p;    // b1p = floor(b1 2^32 / p1)
  u32 s2, mu2;        // s2 = bit length of p2; mu2 = floor(2^(32+s2) / p2) - 2^32
  u32 half1, half2;   // (p1 - 1)/2, (p2 - 1)/2
  u32 kbits, kmask;   // k and 2^k - 1
  // A power-of-two ciphertext modulus q = 2^p2k computed through p1 p2: the
  // products are exact integers below (p1 p2)/2 in magnitude, so the centred
  // CRT value reduced mod 2^p2k is the product mod q (p2k = 0: q = p1 p2).
  u32 p2k, p2shift;   // log2 q and log2 q - k
  u64 Q, Qhalf;       // p1 p2 and floor(p1 p2 / 2)
  u64 lift;           // p1 p2 - 2^p2k: centred lift of a word in [2^(p2k-1), 2^p2k)
};

// A word of [0, 2^61) to its residues (mod p1, mod p2).
__device__ __forceinline__ uint2 to_residues(u64 a, const RnsConst& k) {
  const u32 hi = (u32)(a >> 32), lo = (u32)a;  // hi < 2^29 < p_i
  const u32 r1 = sub_if32(sub_if32(lo, 2 * k.p1), k.p1);
  const u32 r2 = sub_if32(sub_if32(lo, 2 * k.p2), k.p2);
  const u32 h1 = sub_if32(mul_shoup32(hi, k.c32a, k.c32ap, k.p1), k.p1);
  const u32 h2 = sub_if32(mul_shoup32(hi, k.c32b, k.c32bp, k.p2), k.p2);
  return make_uint2(sub_if32(h1 + r1, k.p1), sub_if32(h2 + r2, k.p2));
}

// CRT: the unique c in [0, p1 p2) with c = c1 (mod p1), c = c2 (mod p2),
// for c1 in [0, p1), c2 in [0, p2): c = c1 + p1 h, h = (c2 - c1) p1^-1 mod p2.
__device__ __forceinline__ u32 crt_digit(u32 c1, u32 c2, const RnsConst& k) {
  const u32 d = sub_if32(c2 + k.p2 - c1, k.p2);  // c1 < p1 < p2
  return sub_if32(mul_shoup32(d, k.inv, k.invp, k.p2), k.p2);
}
// The same digit from a lazily reduced second residue, c2 in [0, 2 p2): the
// Shoup product takes c2 + 2 p2 - c1 in (0, 4 p2) as it is.
__device__ __forceinline__ u32 crt_digit_lazy(u32 c1, u32 c2, const RnsConst& k) {
  return sub_if32(mul_shoup32(c2 + 2 * k.p2 - c1, k.inv, k.invp, k.p2), k.p2);
}
__device__ __forceinline__ u64 from_residues(u32 c1, u32 c2, const RnsConst& k) {
  return (u64)c1 + (u64)k.p1 * crt_digit(c1, c2, k);
}

// ModulusSwitch q -> 2^k of c = c1 + p1 h given by its CRT digits, in 32-bit
// arithmetic only.  q is odd, so floor(q/2) = p1 (p2-1)/2 + (p1-1)/2, and
// floor(x / n) = floor(floor(x) / n) for an integer n gives
//   floor((c 2^k + floor(q/2)) / q) = floor(Z / p2),
//   Z = h 2^k + g + (p2-1)/2,  g = floor((c1 2^k + (p1-1)/2) / p1) <= 2^k.
// g: with 2^k = a1 p1 + b1, a Shoup product c1 b1 = s1 p1 + r1 leaves r1 in
// [0, 2 p1), so r1 + (p1-1)/2 adds 0, 1 or 2 whole p1.  floor(Z / p2): Z <
// 2^(32+s2) (p2 < 2^s2); the top word z = floor(Z / 2^s2) times
// mu = floor(2^(32+s2) / p2) in (2^32, 2^33) estimates it from below, off by
// less than 2^s2/p2 + z/2^32 + 1 < 4.  The remainder Z - Qe p2 < 4 p2 < 2^32
// is then exact in the low word and three comparisons finish the quotient.
// K32: k = 32 known at compile time (no variable shift, no final mask).
template <bool K32 = false>
__device__ __forceinline__ u32 rns_modswitch(u32 c1, u32 h, const RnsConst& k) {
  const u32 s1 = __umulhi(k.b1p, c1);
  const u32 r1 = c1 * k.b1 - s1 * k.p1;  // [0, 2 p1)
  const u32 v = r1 + k.half1;           // [0, 2.5 p1)
  const u32 g = c1 * k.a1 + s1 + (u32)(v >= k.p1) + (u32)(v >= 2 * k.p1);
  const u64 Z = ((u64)h << (K32 ? 32 : k.kbits)) + g + k.half2;
  const u32 z = (u32)(Z >> k.s2);
  const u32 Qe = z + __umulhi(z, k.mu2);
  const u32 r = (u32)Z - Qe * k.p2;      // [0, 4 p2)
  const u32 t = (u32)(r >= k.p2) + (u32)(r >= 2 * k.p2) + (u32)(r >= 3 * k.p2);
  return K32 ? Qe + t : (Qe + t) & k.kmask;
}

// Power-of-two q (RnsConst::p2k > 0).  Input word -> residues of its centred
// lift: a mod 2^p2k in [-2^(p2k-1), 2^(p2k-1)), represented mod p1 p2.
__device__ __forceinline__ uint2 pow2_residues(u64 a_mod_q, const RnsConst& k) {
  const u64 v = (a_mod_q >> (k.p2k - 1)) ? a_mod_q + k.lift : a_mod_q;
  return to_residues(v, k);
}
// CRT digits (c1, h) of an exact product -> its value mod 2^p2k: the centred
// representative of c = c1 + p1 h, taken mod 2^64 (2^p2k divides 2^64).
__device__ __forceinline__ u64 pow2_from_crt(u32 c1, u32 h, const RnsConst& k) {
  u64 c = (u64)c1 + (u64)k.p1 * h;
  if (c > k.Qhalf) c -= k.Q;  // wraps: the two's complement of a negative value
  return c & ((1ull << k.p2k) - 1);
}
// ModulusSwitch 2^p2k -> 2^k: floor((v + 2^(p2k-k-1)) / 2^(p2k-k)) mod 2^k.
__device__ __forceinline__ u32 pow2_modswitch(u64 v, const RnsConst& k) {
  return (u32)((v + (1ull << (k.p2shift - 1))) >> k.p2shift) & k.kmask;
}

// Arithmetic policies of the NTT passes.
struct Ring64 {
  using Word = u64;
  using Tw = ulonglong2;  // (w, floor(w 2^64 / q))
  u64 q, qb;              // qb: butterfly bound (2q forward, 4q inverse)
  __device__ __forceinline__ void gs(Word& X, Word& Y, const Tw& w) const { gs_bfly(X, Y, w.x, w.y, q, qb); }
  __device__ __forceinline__ void ct(Word& X, Word& Y, const Tw& w) const { ct_bfly(X, Y, w.x, w.y, q, qb); }
};
struct Ring2x32 {
  using Word = uint2;     // (residue mod p1, residue mod p2)
  using Tw = uint4;       // (w1, w1', w2, w2') with w' = floor(w 2^32 / p)
  u32 p1, p2;
  __device__ __forceinline__ void gs(Word& X, Word& Y, const Tw& w) const {
    gs_bfly32(X.x, Y.x, w.x, w.y, p1, 2 * p1);
    gs_bfly32(X.y, Y.y, w.z, w.w, p2, 2 * p2);
  }
  __device__ __forceinline__ void ct(Word& X, Word& Y, const Tw& w) const {
    ct_bfly32(X.x, Y.x, w.x, w.y, p1, 2 * p1);
    ct_bfly32(X.y, Y.y, w.z, w.w, p2, 2 * p2);
  }
};

// ModulusSwitch q -> 2^k of c in [0, q):
//   floor((c 2^k + floor(q/2)) / q) mod 2^k   (round half up).
// X = c 2^k + floor(q/2) < 2^(s+1+k) + 2^s.  With x' = floor(X / 2^s) <= 2^(k+1)
// and mu = floor(2^(64+s)/q), Qt = floor(x' mu / 2^64) satisfies
// floor(X/q) - 2 <= Qt <= floor(X/q); the remainder X - Qt q < 3q < 2^63 is
// formed in 64-bit arithmetic and corrected at most twice.  (A variant that
// forms Qt from two 32-bit wide products and selects measured slower on
// B300 than the full 64x64 high product.)
__device__ __forceinline__ u32 modswitch_word(u64 c, const RingConst& rc) {
  const u32 k = rc.log2_qout;
  const u64 lo0 = c << k;
  const u64 lo = lo0 + rc.half_q;
  const u64 hi = (c >> (64 - k)) + (lo < lo0 ? 1ull : 0ull);
  const u64 xs = (lo >> rc.ms_s) | (hi << (64 - rc.ms_s));
  u64 quo = __umul64hi(xs, rc.ms_mu);
  u64 r = lo - quo * rc.q;
  if (r >= rc.q) { r -= rc.q; ++quo; }
  if (r >= rc.q) { ++quo; }
  return (u32)(quo & ((k == 32) ? 0xffffffffull : ((1ull << k) - 1)));
}

// ---------------------------------------------------------------------------
// Seeded masks (Sec. 3.1, "Mask Generation via PRNG", read as ChaCha20 with
// the ciphertext's 64-bit seed as key and a zero nonce): coefficient m is the
// 128-bit little-endian integer in words 4(m%4)..4(m%4)+3 of keystream block
// m/4, reduced mod q.  The block function follows RFC 8439, Sec. 2.3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void chacha_quarter(u32& a, u32& b, u32& c, u32& d) {
  a += b; d ^= a; d = __funnelshift_l(d, d, 16);
  c += d; b ^= c; b = __funnelshift_l(b, b, 12);
  a += b; d ^= a; d = __funnelshift_l(d, d, 8);
  c += d; b ^= c; b = __funnelshift_l(b, b, 7);
}

// Keystream block `ctr` for key (seed, 0, ..., 0), nonce 0.
__device__ __forceinline__ void chacha20_block(u64 seed, u32 ctr, u32 (&o)[16]) {
  const u32 init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u, (u32)seed, (u32)(seed >> 32),
                        0u, 0u, 0u, 0u, 0u, 0u, ctr, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 16; ++i) o[i] = init[i];
#pragma unroll 2
  for (int r = 0; r < 10; ++r) {
    chacha_quarter(o[0], o[4], o[8], o[12]);
    chacha_quarter(o[1], o[5], o[9], o[13]);
    chacha_quarter(o[2], o[6], o[10], o[14]);
    chacha_quarter(o[3], o[7], o[11], o[15]);
    chacha_quarter(o[0], o[5], o[10], o[15]);
    chacha_quarter(o[1], o[6], o[11], o[12]);
    chacha_quarter(o[2], o[7], o[8], o[13]);
    chacha_quarter(o[3], o[4], o[9], o[14]);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) o[i] += init[i];
}

// (hi 2^64 + lo) mod q, for the 128-bit keystream words.
__device__ __forceinline__ u64 reduce_u128(u64 hi, u64 lo, const RingConst& rc) {
  const u64 h = reduce_2q(mul_shoup(reduce_word(hi, rc), rc.c64, rc.c64p, rc.q), rc.q);
  return reduce_2q(h + reduce_word(lo, rc), rc.q);
}

// The four mask coefficients 4*cb .. 4*cb+3 of the ciphertext with `seed`.
__device__ __forceinline__ void seeded_mask4(u64 seed, u32 cb, const RingConst& rc, u64 (&v)[4]) {
  u32 o[16];
  chacha20_block(seed, cb, o);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const u64 lo = (u64)o[4 * c] | ((u64)o[4 * c + 1] << 32);
    const u64 hi = (u64)o[4 * c + 2] | ((u64)o[4 * c + 3] << 32);
    v[c] = reduce_u128(hi, lo, rc);
  }
}

// ---------------------------------------------------------------------------
// Register-blocked NTT of size N = 2^LOGN: P = N/16 threads hold 16 words
// each.  Stages are grouped into passes of up to four; within a pass every
// thread owns complete butterfly groups and works in registers; between
// passes the words move through shared memory.
//
// Stage s (0 <= s < LOGN) pairs positions (j, j + 2^s) with bit s of j clear;
// both transforms use the twiddle at table index (N >> (s+1)) + (j >> (s+1)).
// ---------------------------------------------------------------------------
template <int LOGN>
struct Shape {
  static constexpr int N = 1 << LOGN;
  static constexpr int E = 16;                       // words per thread
  static constexpr int P = N / E;                    // threads per transform
  static constexpr int NPASS = (LOGN + 3) / 4;
  static constexpr int TPB = (P < 256) ? 256 : P;    // threads per block
  static constexpr int SLOTS = TPB / P;              // transforms in flight per block
  static constexpr int PADN = N + N / 16;            // one pad word per 16: conflict-free exchanges
};

template <int LOGN, int PASS>
struct PassShape {
  static constexpr int S0 = 4 * PASS;                               // first stage of the pass
  static constexpr int K = (LOGN - S0) < 4 ? (LOGN - S0) : 4;       // stages in the pass
  static constexpr int G = 1 << K;                                  // words per butterfly group
  static constexpr int U = 16 / G;                                  // groups per thread
};

// Position of local word e (= u*G + r) of thread p in pass PASS.
template <int LOGN, int PASS>
__device__ __forceinline__ int pass_pos(int p, int e) {
  using PS = PassShape<LOGN, PASS>;
  constexpr int P = Shape<LOGN>::P;
  const int u = e / PS::G, r = e % PS::G;
  const int g = u * P + p;
  const int base = ((g >> PS::S0) << (PS::S0 + PS::K)) | (g & ((1 << PS::S0) - 1));
  return base + (r << PS::S0);
}

__device__ __forceinline__ int pad_idx(int pos) { return pos + (pos >> 4); }

// Slot of the pass-0 twiddle used by stage st (0..3), twiddle b of the group.
__host__ __device__ constexpr int pass0_slot(int st, int b) { return (16 - (16 >> st)) + b; }

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// One stage of a pass: stage ST of pass PASS (ST counted inside the pass).
// Every twiddle is loaded once and applied to the 2^ST butterflies sharing it.
template <int LOGN, int PASS, int ST, bool INVERSE, class R>
__device__ __forceinline__ void pass_stage(typename R::Word (&x)[16], int p, const typename R::Tw* __restrict__ tw0,
                                           const typename R::Tw* __restrict__ twc, const R& ring) {
  using PS = PassShape<LOGN, PASS>;
  constexpr int N = Shape<LOGN>::N;
  constexpr int P = Shape<LOGN>::P;
  constexpr int s = PS::S0 + ST;
  constexpr int h = 1 << ST;
  constexpr int NB = PS::G >> (ST + 1);  // distinct twiddles per group
#pragma unroll
  for (int u = 0; u < PS::U; ++u) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      typename R::Tw w;
      if constexpr (PASS == 0) {
        w = __ldg(&tw0[pass0_slot(ST, b) * P + p]);
      } else {
        const int j = pass_pos<LOGN, PASS>(p, u * PS::G + b * 2 * h);
        w = __ldg(&twc[(N >> (s + 1)) + (j >> (s + 1))]);
      }
#pragma unroll
      for (int c = 0; c < h; ++c) {
        const int e0 = u * PS::G + b * 2 * h + c;
        if constexpr (INVERSE) ring.gs(x[e0], x[e0 + h], w);
        else ring.ct(x[e0], x[e0 + h], w);
      }
    }
  }
}

// Inverse (Gentleman-Sande) pass: stages S0 .. S0+K-1 ascending.
// tw0: pass-0 table, thread-major [15][P]; twc: compact table [N].
template <int LOGN, int PASS, class R>
__device__ __forceinline__ void gs_pass(typename R::Word (&x)[16], int p, const typename R::Tw* __restrict__ tw0,
                                        const typename R::Tw* __restrict__ twc, const R& ring) {
  static_for<0, PassShape<LOGN, PASS>::K>([&](auto st) {
    pass_stage<LOGN, PASS, decltype(st)::value, true>(x, p, tw0, twc, ring);
  });
}

// Forward (Cooley-Tukey) pass: stages S0+K-1 .. S0 descending.
template <int LOGN, int PASS, class R>
__device__ __forceinline__ void ct_pass(typename R::Word (&x)[16], int p, const typename R::Tw* __restrict__ tw0,
                                        const typename R::Tw* __restrict__ twc, const R& ring) {
  constexpr int K = PassShape<LOGN, PASS>::K;
  static_for<0, K>([&](auto i) {
    pass_stage<LOGN, PASS, K - 1 - decltype(i)::value, false>(x, p, tw0, twc, ring);
  });
}

// Move the 16 words of every thread from pass A's positions to pass B's.
// The barrier after the reads guards the buffer against the next writer.  An
// exchange followed by the exchange out of pass B needs none: that one writes
// exactly the pass-B positions, and each is rewritten by the thread that read
// it (TRAIL = false).
template <int LOGN, int PA, int PB, bool TRAIL = true, class W>
__device__ __forceinline__ void exchange(W (&x)[16], int p, W* __restrict__ buf) {
#pragma unroll
  for (int e = 0; e < 16; ++e) buf[pad_idx(pass_pos<LOGN, PA>(p, e))] = x[e];
  __syncthreads();
#pragma unroll
  for (int e = 0; e < 16; ++e) x[e] = buf[pad_idx(pass_pos<LOGN, PB>(p, e))];
  if constexpr (TRAIL) __syncthreads();
}

// Full inverse transform (no N^-1 scaling): bit-reversed in (pass-0 layout),
// natural order out (last-pass layout).  Values stay within the policy's
// inverse bound ([0, 4q) for Ring64, [0, 2p) for Ring2x32).
template <int LOGN, class R>
__device__ __forceinline__ void intt_regs(typename R::Word (&x)[16], int p, typename R::Word* buf,
                                          const typename R::Tw* tw0, const typename R::Tw* twc, const R& ring) {
  constexpr int NP = Shape<LOGN>::NPASS;
  gs_pass<LOGN, 0>(x, p, tw0, twc, ring);
  if constexpr (NP > 1) {
    exchange<LOGN, 0, 1, (NP == 2)>(x, p, buf);
    gs_pass<LOGN, 1>(x, p, tw0, twc, ring);
  }
  if constexpr (NP > 2) {
    exchange<LOGN, 1, 2, (NP == 3)>(x, p, buf);
    gs_pass<LOGN, 2>(x, p, tw0, twc, ring);
  }
  if constexpr (NP > 3) {
    exchange<LOGN, 2, 3, true>(x, p, buf);
    gs_pass<LOGN, 3>(x, p, tw0, twc, ring);
  }
}

// Full forward transform: natural order in (last-pass layout), bit-reversed
// out (pass-0 layout).  Values in [0, 4q) (or [0, 4p)) in and out.
template <int LOGN, class R>
__device__ __forceinline__ void ntt_regs(typename R::Word (&x)[16], int p, typename R::Word* buf,
                                         const typename R::Tw* tw0, const typename R::Tw* twc, const R& ring) {
  constexpr int NP = Shape<LOGN>::NPASS;
  if constexpr (NP > 3) {
    ct_pass<LOGN, 3>(x, p, tw0, twc, ring);
    exchange<LOGN, 3, 2, false>(x, p, buf);
  }
  if constexpr (NP > 2) {
    ct_pass<LOGN, 2>(x, p, tw0, twc, ring);
    exchange<LOGN, 2, 1, false>(x, p, buf);
  }
  if constexpr (NP > 1) {
    ct_pass<LOGN, 1>(x, p, tw0, twc, ring);
    exchange<LOGN, 1, 0, true>(x, p, buf);
  }
  ct_pass<LOGN, 0>(x, p, tw0, twc, ring);
}

// Layout of transformed inputs (A_hat): word r of pass-0 thread p of a block
// of N words, pair-interleaved so that a warp reads 512 contiguous bytes.
template <int LOGN>
__device__ __forceinline__ int ahat_idx(int p, int r) {
  return (((r >> 1) * Shape<LOGN>::P + p) << 1) | (r & 1);
}
// Layout of transformed weights (W_hat, stored as (w, w') pairs): pair r of thread p.
template <int LOGN>
__device__ __forceinline__ int what_idx(int p, int r) {
  return r * Shape<LOGN>::P + p;
}

}  // namespace phe
