// Output packing (Sec. 3.2 KeySwitching and Rotate, Eq. (pack_rotate)):
// the m <= N LWE outputs (a_j, b_j) of a group of rows become one RLWE
// ciphertext sum_j Rotate(KeySwitching(LWE_j), j), then ModulusSwitch.
//
// KeySwitching is linear in the digits of the masks and Rotate by j is the
// product with X^j, so the packed mask is
//   A = - sum_{i,l} D_il(X) KA_il(X),   D_il(X) = sum_j d_l(a_j[i]) X^j,
// and B = sum_j b_j X^j - sum_{i,l} D_il(X) KB_il(X): n*ell negacyclic
// products with the key-switching key instead of m*n*ell scalar-polynomial
// products.  Kernels:
//   pack_decompose_kernel  digits d_l(a_j[i]) of the masks, transposed so
//                          that D_il is a row over j (natural order, mod q)
// A unit is one output RLWE and the LWE ciphertexts it packs (PackGeom).
//   input_ntt_kernel       D_il (int32 digits) -> NTT domain
//   pack_mac_kernel        per NTT slot: sum over (i,l) of D_hat * KSK_hat
//                          (the key carries -N^-1 and Shoup quotients)
//   pack_finish_kernel     inverse NTT of A_hat and B_hat, + b_j X^j, switch
//   pack_finish_pow2_kernel  the same for q = 2^K, whose key is held in exact
//                          slices: each slice's contraction lifted centred
//                          by CRT, the slices combined mod 2^K
//   ksk_finish_kernel      upload: NTT(KSK) -> -N^-1 NTT(KSK) with quotients
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "phe_host.hpp"

using phe::u32;
using phe::u64;
using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;

struct phe_ksk {
  phe_ctx* ctx = nullptr;
  uint32_t n = 0, base_log = 0, ell = 0;
  phe::RingConst rcK{};  // the context's constants with the switch target 2^(base_log*ell)
  phe::RnsConst rkK{};
  void* khat = nullptr;  // [slices][n*ell][2][N] entries of 16 bytes (A then B), A_hat slot order
  uint64_t bytes = 0;
  // q = 2^K: the centred key is split into `slices` signed pieces of
  // slice_bits bits, KSK = sum_s 2^(slice_bits s) KSK_s, each small enough
  // that its contraction stays below (p1 p2)/2 and is exact through p1 p2.
  uint32_t slices = 1, slice_bits = 0;
};

namespace phe {

// Signed gadget digits of a (Sec. 3.2 Decomp, read as the approximate signed
// decomposition of TFHE): a~ = ModulusSwitch of a from q to B^ell, then
// base-B digits d_0 (most significant) .. d_{ell-1} in [-B/2, B/2); a carry
// out of d_0 is a multiple of B^ell and is dropped.  rcK is the context's
// constants with log2_qout = base_log * ell (<= 32).
// Signed gadget digits (Sec. 3.2 Decomp, read as the approximate signed
// decomposition of TFHE) of a~ = ModulusSwitch of a from q to B^ell: base-B
// digits d_0 (most significant) .. d_{ell-1} in [-B/2, B/2); a carry out of
// d_0 is a multiple of B^ell and is dropped.
template <int ELL>
__device__ __forceinline__ void signed_digits(u32 v, u32 base_log, int (&d)[ELL]) {
  const u32 B = 1u << base_log, half = B >> 1, mask = B - 1;
#pragma unroll
  for (int l = ELL - 1; l >= 0; --l) {
    int r = (int)(v & mask);
    v = (base_log < 32) ? (v >> base_log) : 0u;
    if ((u32)r >= half) {
      r -= (int)B;
      v += 1u;
    }
    d[l] = r;
  }
}

// Which LWE ciphertexts each unit (one output RLWE) packs.  The LWE outputs
// of a call are numbered f = t*rows + r (token t, output row r).  With
// G = ceil(rows/N) > 1, unit u is group g = u % G of token t = u / G: rows
// gN .. of that token.  With G = 1, unit u holds the outputs of `tpu`
// consecutive tokens, f = u*tpu*rows onwards: tpu = 1 packs each token on
// its own (Eq. (pack_rotate) per token), tpu = floor(N/rows) > 1 fills the
// ring with several tokens (dense packing).  Coefficient j of the unit's
// RLWE carries LWE f0 + j for j < m, and zero past m.
struct PackGeom {
  u32 rows;   // LWE outputs per token
  u32 G;      // ceil(rows / N)
  u32 tpu;    // tokens per unit (1 unless G = 1 and dense)
  u64 nflat;  // T * rows: the LWE outputs in the buffers the kernels index
};

__device__ __forceinline__ void unit_span(const PackGeom& pg, u32 N, u32 u, u64& f0, u32& m) {
  if (pg.G > 1) {
    const u32 t = u / pg.G, g = u % pg.G;
    f0 = (u64)t * pg.rows + (u64)g * N;
    m = min(N, pg.rows - g * N);
  } else {
    f0 = (u64)u * pg.tpu * pg.rows;
    m = (u32)min((u64)pg.tpu * pg.rows, pg.nflat - f0);
  }
}

// Masks [T][rows][N] -> digit rows D[u][i*ell + l][j] of the units
// u_base + u, holding the signed digit d_l(a_{f0+j}[i]) of the unit's LWE
// f0 + j for j < m and 0 past it (unit_span).  SWITCHED: the masks are already
// a~ (uint32, switched to B^ell by the product kernel's epilogue); otherwise
// they are words below q, switched here with rcK (log2_qout = base_log*ell).
// A block moves a 64 (i) x 32 (j) tile through shared memory, so that both
// the load (two words of i per thread) and the store (along j) are coalesced.
template <int ELL, bool SWITCHED>
__global__ void __launch_bounds__(256)
    pack_decompose_kernel(const void* __restrict__ maskv, PackGeom pg, u32 N, u32 u_base, u32 base_log,
                          RingConst rcK, RnsConst rkK, int32_t* __restrict__ D) {
  __shared__ int tile[ELL][64][33];
  const u32 u = blockIdx.z;  // unit within the chunk; D holds the chunk's units
  u64 f0;
  u32 mu;
  unit_span(pg, N, u_base + u, f0, mu);
  const u32 i0 = blockIdx.x * 64, j0 = blockIdx.y * 32;
  const u32 tx = threadIdx.x, ty = threadIdx.y;
  const size_t first = ((size_t)f0 + j0) * N + i0;  // mask word (LWE f0+j0, column i0)
#pragma unroll
  for (u32 m = 0; m < 4; ++m) {
    const u32 k = ty + 8 * m;
    int d0[ELL], d1[ELL];
    if (j0 + k < mu) {
      u32 v0, v1;
      if constexpr (SWITCHED) {
        const uint2 v = *reinterpret_cast<const uint2*>(static_cast<const u32*>(maskv) + first + (size_t)k * N + 2 * tx);
        v0 = v.x;
        v1 = v.y;
      } else {
        const ulonglong2 v =
            *reinterpret_cast<const ulonglong2*>(static_cast<const u64*>(maskv) + first + (size_t)k * N + 2 * tx);
        if (rkK.p2k) {  // q = 2^K: a rounding shift
          v0 = pow2_modswitch(v.x & (rcK.q - 1), rkK);
          v1 = pow2_modswitch(v.y & (rcK.q - 1), rkK);
        } else {
          v0 = modswitch_word(v.x, rcK);
          v1 = modswitch_word(v.y, rcK);
        }
      }
      signed_digits<ELL>(v0, base_log, d0);
      signed_digits<ELL>(v1, base_log, d1);
    } else {
#pragma unroll
      for (int l = 0; l < ELL; ++l) d0[l] = d1[l] = 0;
    }
#pragma unroll
    for (int l = 0; l < ELL; ++l) {
      tile[l][2 * tx][k] = d0[l];
      tile[l][2 * tx + 1][k] = d1[l];
    }
  }
  __syncthreads();
  int32_t* out = D + ((size_t)u * N + i0) * ELL * N + j0;
#pragma unroll
  for (u32 m = 0; m < 8; ++m) {
    const u32 k = ty + 8 * m;  // i = i0 + k
#pragma unroll
    for (int l = 0; l < ELL; ++l) out[((size_t)k * ELL + l) * N + tx] = tile[l][k][tx];
  }
}

// Key upload: NTT(KSK) words in A_hat slot order -> -N^-1 NTT(KSK), fully
// reduced, with Shoup quotients: (k1, k1', k2, k2') (RNS) or (k, k') mod q.
template <bool RNS>
__global__ void ksk_finish_kernel(const u64* __restrict__ src, void* __restrict__ dst, size_t n, RingConst rc,
                                  RnsConst rk, NInv ninv) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    if constexpr (RNS) {
      const uint2 x = reinterpret_cast<const uint2*>(src)[idx];
      u32 a1 = sub_if32(sub_if32(x.x, 2 * rk.p1), rk.p1);
      u32 a2 = sub_if32(sub_if32(x.y, 2 * rk.p2), rk.p2);
      a1 = sub_if32(mul_shoup32(a1, ninv.n1, ninv.n1p, rk.p1), rk.p1);
      a2 = sub_if32(mul_shoup32(a2, ninv.n2, ninv.n2p, rk.p2), rk.p2);
      a1 = a1 ? rk.p1 - a1 : 0u;
      a2 = a2 ? rk.p2 - a2 : 0u;
      reinterpret_cast<uint4*>(dst)[idx] =
          make_uint4(a1, (u32)(((u64)a1 << 32) / rk.p1), a2, (u32)(((u64)a2 << 32) / rk.p2));
    } else {
      u64 v = reduce_4q(src[idx], rc.q, rc.q2);
      v = reduce_2q(mul_shoup(v, ninv.n64, ninv.n64p, rc.q), rc.q);
      v = v ? rc.q - v : 0ull;
      u64 rem = v, quo = 0;  // floor(v 2^64 / q) by long division
      for (int b = 0; b < 64; ++b) {
        rem <<= 1;
        quo <<= 1;
        if (rem >= rc.q) {
          rem -= rc.q;
          quo |= 1ull;
        }
      }
      reinterpret_cast<ulonglong2*>(dst)[idx] = make_ulonglong2(v, quo);
    }
  }
}

// Asynchronous global -> shared copies (cp.async, sm_80 and later): each
// thread stages only the words it reads itself, so the pipeline needs no
// block barrier, only the thread's own wait_group.
__device__ __forceinline__ void cp_async16(void* smem, const void* g) {
  const u32 sa = (u32)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* g) {
  const u32 sa = (u32)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Per NTT slot s, unit u and segment g of the contraction:
//   P_hat[g][u][c][s] = sum_{r in segment g} D_hat[u][r][s] K_hat[r][c][s]   (c = 0: A, 1: B),
// fully reduced.  A block covers 256 slots, one segment and UB units, so each
// key entry it loads serves UB units; the segments (a split of the n*ell
// contraction) give enough blocks to fill the GPU and are summed by the
// finishing kernel.  The key entries (16 bytes) and transformed digits
// (8 bytes) of row r stream through a STAGES-deep ring in shared memory, so
// that a thread keeps STAGES-1 rows of loads in flight.
template <bool RNS, int UB, int STAGES>
__global__ void __launch_bounds__(256, 2)
    pack_mac_kernel(const u64* __restrict__ Dhat, const void* __restrict__ khatv, u32 nr, u32 rseg, u32 N, u32 units,
                    u64* __restrict__ Phat, RingConst rc, RnsConst rk) {
  extern __shared__ uint4 mac_smem[];
  uint4* sk = mac_smem;                                        // [STAGES][2][256] key entries
  uint2* sd = reinterpret_cast<uint2*>(mac_smem + STAGES * 2 * 256);  // [STAGES][UB][256] digit words
  const u32 tid = threadIdx.x;
  const u32 s = blockIdx.x * blockDim.x + tid;  // N is a multiple of 256: s < N
  const u32 seg = blockIdx.y, u0 = blockIdx.z * UB;
  const int nu = (int)min((u32)UB, units - u0);
  const u32 r0 = seg * rseg, r1 = min(nr, r0 + rseg);
  u64* part = Phat + (size_t)seg * units * 2 * N;
  const uint4* kh = reinterpret_cast<const uint4*>(khatv);
  const uint2* dh = reinterpret_cast<const uint2*>(Dhat);
  auto issue = [&](u32 r, int st) {
    cp_async16(&sk[(st * 2) * 256 + tid], &kh[((size_t)r * 2) * N + s]);
    cp_async16(&sk[(st * 2 + 1) * 256 + tid], &kh[((size_t)r * 2 + 1) * N + s]);
#pragma unroll
    for (int k = 0; k < UB; ++k)
      if (k < nu) cp_async8(&sd[(st * UB + k) * 256 + tid], &dh[((size_t)(u0 + k) * nr + r) * N + s]);
  };
#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) {
    if (r0 + st < r1) issue(r0 + st, st);
    cp_async_commit();
  }
  if constexpr (RNS) {
    const u32 p1 = rk.p1, p2 = rk.p2, p1x2 = 2 * rk.p1, p2x2 = 2 * rk.p2;
    u32 acc[UB][4];  // kept in [0, 2p): each Shoup product is below 2p
#pragma unroll
    for (int k = 0; k < UB; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0;
    for (u32 r = r0; r < r1; ++r) {
      const u32 rn = r + STAGES - 1;
      if (rn < r1) issue(rn, (int)((rn - r0) % STAGES));
      cp_async_commit();
      cp_async_wait<STAGES - 1>();
      const int st = (int)((r - r0) % STAGES);
      const uint4 ka = sk[(st * 2) * 256 + tid];
      const uint4 kb = sk[(st * 2 + 1) * 256 + tid];
#pragma unroll
      for (int k = 0; k < UB; ++k) {
        if (k < nu) {
          const uint2 d = sd[(st * UB + k) * 256 + tid];
          acc[k][0] = sub_if32(acc[k][0] + mul_shoup32(d.x, ka.x, ka.y, p1), p1x2);
          acc[k][1] = sub_if32(acc[k][1] + mul_shoup32(d.y, ka.z, ka.w, p2), p2x2);
          acc[k][2] = sub_if32(acc[k][2] + mul_shoup32(d.x, kb.x, kb.y, p1), p1x2);
          acc[k][3] = sub_if32(acc[k][3] + mul_shoup32(d.y, kb.z, kb.w, p2), p2x2);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      if (k < nu) {
        uint2* out = reinterpret_cast<uint2*>(part) + (size_t)(u0 + k) * 2 * N + s;
        out[0] = make_uint2(sub_if32(acc[k][0], p1), sub_if32(acc[k][1], p2));
        out[N] = make_uint2(sub_if32(acc[k][2], p1), sub_if32(acc[k][3], p2));
      }
    }
  } else {
    const u64 q = rc.q, q4 = rc.q4;
    u64 acc[UB][2];
#pragma unroll
    for (int k = 0; k < UB; ++k) acc[k][0] = acc[k][1] = 0;
    for (u32 r = r0; r < r1; ++r) {
      const u32 rn = r + STAGES - 1;
      if (rn < r1) issue(rn, (int)((rn - r0) % STAGES));
      cp_async_commit();
      cp_async_wait<STAGES - 1>();
      const int st = (int)((r - r0) % STAGES);
      const ulonglong2 ka = reinterpret_cast<const ulonglong2*>(sk)[(st * 2) * 256 + tid];
      const ulonglong2 kb = reinterpret_cast<const ulonglong2*>(sk)[(st * 2 + 1) * 256 + tid];
#pragma unroll
      for (int k = 0; k < UB; ++k) {
        if (k < nu) {
          const u64 d = reinterpret_cast<const u64*>(sd)[(st * UB + k) * 256 + tid];
          const u64 a = acc[k][0] + mul_shoup_lazy(d, ka.x, ka.y, q);  // each term < 4q, sum < 8q
          const u64 b = acc[k][1] + mul_shoup_lazy(d, kb.x, kb.y, q);
          acc[k][0] = (a >= q4) ? a - q4 : a;
          acc[k][1] = (b >= q4) ? b - q4 : b;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UB; ++k) {
      if (k < nu) {
        u64* out = part + (size_t)(u0 + k) * 2 * N + s;
        out[0] = reduce_4q(acc[k][0], q, rc.q2);
        out[N] = reduce_4q(acc[k][1], q, rc.q2);
      }
    }
  }
  cp_async_wait<0>();  // no copy outlives the block
}

// Inverse transform of P_hat[u][c] (c = 0: A, c = 1: B), + b_{f0+j} at
// coefficient j of B for the unit's LWEs, then the switch (or raw words).
// Block b = u*2 + c of the chunk; u_base is the chunk's first unit.
template <int LOGN, bool RNS, int MODE>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    pack_finish_kernel(const u64* __restrict__ Phat, u32 nseg, const u64* __restrict__ body, PackGeom pg,
                       u32 u_base, u32 units, void* __restrict__ out_a, void* __restrict__ out_b, RingConst rc,
                       RnsConst rk, const void* __restrict__ tw0v, const void* __restrict__ twcv) {
  using S = Shape<LOGN>;
  using R = std::conditional_t<RNS, Ring2x32, Ring64>;
  using W = typename R::Word;
  using Tw = typename R::Tw;
  constexpr int N = S::N;
  constexpr int P = S::P;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / P, p = threadIdx.x % P;
  W* buf = reinterpret_cast<W*>(smem + slot * S::PADN);
  const u32 b = blockIdx.x * S::SLOTS + slot;
  const bool active = b < 2 * units;
  W x[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if constexpr (RNS) x[r] = make_uint2(0u, 0u);
    else x[r] = 0;
  }
  if (active) {
    // the segments' partial sums, words (r, r+1) of thread p together as the
    // input transform laid them out
    for (u32 g = 0; g < nseg; ++g) {
      const u64* part = Phat + ((size_t)g * units * 2 + b) * N;
      if constexpr (RNS) {
        const uint4* ap = reinterpret_cast<const uint4*>(part);
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
          const uint4 v = ap[(r >> 1) * P + p];
          x[r] = make_uint2(sub_if32(x[r].x + v.x, rk.p1), sub_if32(x[r].y + v.y, rk.p2));
          x[r + 1] = make_uint2(sub_if32(x[r + 1].x + v.z, rk.p1), sub_if32(x[r + 1].y + v.w, rk.p2));
        }
      } else {
        const ulonglong2* ap = reinterpret_cast<const ulonglong2*>(part);
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
          const ulonglong2 v = ap[(r >> 1) * P + p];
          x[r] = reduce_2q(x[r] + v.x, rc.q);
          x[r + 1] = reduce_2q(x[r + 1] + v.y, rc.q);
        }
      }
    }
  }
  if constexpr (RNS) {
    intt_regs<LOGN>(x, p, buf, reinterpret_cast<const Tw*>(tw0v), reinterpret_cast<const Tw*>(twcv),
                    Ring2x32{rk.p1, rk.p2});
  } else {
    intt_regs<LOGN>(x, p, buf, reinterpret_cast<const Tw*>(tw0v), reinterpret_cast<const Tw*>(twcv),
                    Ring64{rc.q, rc.q4});
  }
  if (!active) return;
  const u32 u = u_base + b / 2, comp = b % 2;
  u64 f0;
  u32 mu;
  unit_span(pg, N, u, f0, mu);
  void* out = comp ? out_b : out_a;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const u32 pos = (u32)pass_pos<LOGN, NP - 1>(p, e);
    const bool add_body = comp == 1 && pos < mu;
    const size_t o = (size_t)u * N + pos;
    if constexpr (RNS) {
      u32 c1 = sub_if32(x[e].x, rk.p1), c2 = sub_if32(x[e].y, rk.p2);
      if (add_body) {
        const uint2 rb = to_residues(reduce_word(body[f0 + pos], rc), rk);
        c1 = sub_if32(sub_if32(c1 + rb.x, 2 * rk.p1), rk.p1);
        c2 = sub_if32(sub_if32(c2 + rb.y, 2 * rk.p2), rk.p2);
      }
      const u32 h = crt_digit(c1, c2, rk);
      if constexpr (MODE == kOutSwitched) reinterpret_cast<u32*>(out)[o] = rns_modswitch(c1, h, rk);
      else reinterpret_cast<u64*>(out)[o] = (u64)c1 + (u64)rk.p1 * h;
    } else {
      u64 c = reduce_4q(x[e], rc.q, rc.q2);
      if (add_body) c = reduce_2q(c + reduce_word(body[f0 + pos], rc), rc.q);
      if constexpr (MODE == kOutSwitched) reinterpret_cast<u32*>(out)[o] = modswitch_word(c, rc);
      else reinterpret_cast<u64*>(out)[o] = c;
    }
  }
}

// q = 2^K (the key in slices): per slice sl, the segments' partial sums are
// inverse-transformed and the CRT value (exact, below (p1 p2)/2 in magnitude)
// is lifted centred; the slices combine as sum_sl 2^(bits sl) value mod 2^64,
// which is exact mod 2^K.  Then b_{f0+j} joins coefficient j of B and the
// words are switched to 2^k (or left mod 2^K).  Block b = u*2 + c as above;
// slice sl's partial sums start at Phat + sl * slice_stride.
template <int LOGN, int MODE>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    pack_finish_pow2_kernel(const u64* __restrict__ Phat, u32 nseg, u32 slices, u32 bits, size_t slice_stride,
                            const u64* __restrict__ body, PackGeom pg, u32 u_base, u32 units,
                            void* __restrict__ out_a, void* __restrict__ out_b, RnsConst rk,
                            const void* __restrict__ tw0v, const void* __restrict__ twcv) {
  using S = Shape<LOGN>;
  using W = Ring2x32::Word;
  using Tw = Ring2x32::Tw;
  constexpr int N = S::N;
  constexpr int P = S::P;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / P, p = threadIdx.x % P;
  W* buf = reinterpret_cast<W*>(smem + slot * S::PADN);
  const u32 b = blockIdx.x * S::SLOTS + slot;
  const bool active = b < 2 * units;
  u64 acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0;
  for (u32 sl = 0; sl < slices; ++sl) {
    W x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) x[r] = make_uint2(0u, 0u);
    if (active) {
      for (u32 g = 0; g < nseg; ++g) {
        const uint4* ap = reinterpret_cast<const uint4*>(Phat + sl * slice_stride + ((size_t)g * units * 2 + b) * N);
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
          const uint4 v = ap[(r >> 1) * P + p];
          x[r] = make_uint2(sub_if32(x[r].x + v.x, rk.p1), sub_if32(x[r].y + v.y, rk.p2));
          x[r + 1] = make_uint2(sub_if32(x[r + 1].x + v.z, rk.p1), sub_if32(x[r + 1].y + v.w, rk.p2));
        }
      }
    }
    intt_regs<LOGN>(x, p, buf, reinterpret_cast<const Tw*>(tw0v), reinterpret_cast<const Tw*>(twcv),
                    Ring2x32{rk.p1, rk.p2});
    const u32 sh = bits * sl;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const u32 c1 = sub_if32(x[e].x, rk.p1);
      const u64 v = pow2_from_crt(c1, crt_digit_lazy(c1, x[e].y, rk), rk);  // centred value mod 2^K
      acc[e] += (sh < 64) ? (v << sh) : 0ull;
    }
  }
  if (!active) return;
  const u32 u = u_base + b / 2, comp = b % 2;
  u64 f0;
  u32 mu;
  unit_span(pg, N, u, f0, mu);
  void* out = comp ? out_b : out_a;
  const u64 qmask = (1ull << rk.p2k) - 1;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const u32 pos = (u32)pass_pos<LOGN, NP - 1>(p, e);
    u64 v = acc[e];
    if (comp == 1 && pos < mu) v += body[f0 + pos];
    v &= qmask;
    const size_t o = (size_t)u * N + pos;
    if constexpr (MODE == kOutSwitched) reinterpret_cast<u32*>(out)[o] = pow2_modswitch(v, rk);
    else reinterpret_cast<u64*>(out)[o] = v;
  }
}

}  // namespace phe

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
namespace {

using phe::Span;




constexpr int kMacUnits = 8;                        // units per pack_mac_kernel block
constexpr int kMacStages = 4;                       // rows in flight per pack_mac_kernel thread
constexpr size_t kMacSmem = (size_t)kMacStages * 256 * (2 * 16 + kMacUnits * 8);
constexpr uint64_t kPackScratchBytes = 4ull << 30;  // digit rows in flight per phe_pack chunk
constexpr uint64_t kLweScratchBytes = 2ull << 30;   // switched masks in flight per phe_matmul_packed chunk
constexpr uint32_t kPackFlags = PHE_OUT_RAW | PHE_PACK_DENSE;

cudaError_t launch_decompose(const phe_ctx* c, const phe_ksk* k, const void* mask, bool switched,
                             const phe::PackGeom& pg, u32 u_base, u32 cu, int32_t* D, cudaStream_t s) {
  const u32 N = c->prm.N;
  const dim3 grid(N / 64, N / 32, cu), block(32, 8);
#define PHE_DECOMP(E)                                                                                       \
  (switched ? phe::pack_decompose_kernel<E, true><<<grid, block, 0, s>>>(mask, pg, N, u_base, k->base_log, k->rcK, \
                                                                          k->rkK, D)                                 \
            : phe::pack_decompose_kernel<E, false><<<grid, block, 0, s>>>(mask, pg, N, u_base, k->base_log, k->rcK, \
                                                                           k->rkK, D))
  switch (k->ell) {
    case 1: PHE_DECOMP(1); break;
    case 2: PHE_DECOMP(2); break;
    case 3: PHE_DECOMP(3); break;
    default: PHE_DECOMP(4); break;
  }
#undef PHE_DECOMP
  return cudaGetLastError();
}

// Segments of the n*ell contraction for a chunk of `cu` units: as many blocks
// as fit in four per SM (two waves of two resident blocks), each segment at
// least 16 rows long.
u32 mac_segments(const phe_ctx* c, const phe_ksk* k, u32 cu) {
  const u32 nr = k->n * k->ell;
  const u32 base = (c->prm.N / 256) * ((cu + kMacUnits - 1) / kMacUnits);
  const u32 want = (4u * (u32)c->num_sms) / base;
  return std::max(1u, std::min(want, nr / 16));
}

cudaError_t launch_mac(const phe_ctx* c, const phe_ksk* k, const u64* Dhat, u32 cu, u32 nseg, u64* Phat,
                       cudaStream_t s, u32 slice = 0) {
  const u32 N = c->prm.N, nr = k->n * k->ell;
  const void* khat = static_cast<const char*>(k->khat) + (size_t)slice * nr * 2 * N * 16;
  const u32 rseg = (nr + nseg - 1) / nseg;
  const dim3 grid(N / 256, nseg, (cu + kMacUnits - 1) / kMacUnits);
  auto kern = c->rns ? phe::pack_mac_kernel<true, kMacUnits, kMacStages>
                     : phe::pack_mac_kernel<false, kMacUnits, kMacStages>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMacSmem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, kMacSmem, s>>>(Dhat, khat, nr, rseg, N, cu, Phat, c->rc, c->rk);
  return cudaGetLastError();
}

template <int LOGN, bool RNS, int MODE>
cudaError_t finish_one(const phe_ctx* c, const u64* Phat, u32 nseg, const u64* body, const phe::PackGeom& pg,
                       u32 u_base, u32 cu, void* oa, void* ob, cudaStream_t s) {
  using S = phe::Shape<LOGN>;
  const size_t smem = phe::lwedot_smem(LOGN);
  auto kern = phe::pack_finish_kernel<LOGN, RNS, MODE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const phe::Tables& tab = RNS ? c->tab32 : c->tab;
  const u32 blocks = (2 * cu + S::SLOTS - 1) / S::SLOTS;
  kern<<<blocks, S::TPB, smem, s>>>(Phat, nseg, body, pg, u_base, cu, oa, ob, c->rc, c->rk, tab.inv_0, tab.inv_c);
  return cudaGetLastError();
}

template <int LOGN, int MODE>
cudaError_t finish_pow2(const phe_ctx* c, const phe_ksk* k, const u64* Phat, u32 nseg, size_t slice_stride,
                        const u64* body, const phe::PackGeom& pg, u32 u_base, u32 cu, void* oa, void* ob,
                        cudaStream_t s) {
  using S = phe::Shape<LOGN>;
  const size_t smem = phe::lwedot_smem(LOGN);
  auto kern = phe::pack_finish_pow2_kernel<LOGN, MODE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const u32 blocks = (2 * cu + S::SLOTS - 1) / S::SLOTS;
  kern<<<blocks, S::TPB, smem, s>>>(Phat, nseg, k->slices, k->slice_bits, slice_stride, body, pg, u_base, cu, oa, ob,
                                    c->rk, c->tab32.inv_0, c->tab32.inv_c);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t finish_by_form(const phe_ctx* c, int mode, const u64* Phat, u32 nseg, const u64* body,
                           const phe::PackGeom& pg, u32 u_base, u32 cu, void* oa, void* ob, cudaStream_t s) {
  if (c->rns) {
    return mode == phe::kOutRaw ? finish_one<LOGN, true, phe::kOutRaw>(c, Phat, nseg, body, pg, u_base, cu, oa, ob, s)
                                : finish_one<LOGN, true, phe::kOutSwitched>(c, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
  }
  return mode == phe::kOutRaw ? finish_one<LOGN, false, phe::kOutRaw>(c, Phat, nseg, body, pg, u_base, cu, oa, ob, s)
                              : finish_one<LOGN, false, phe::kOutSwitched>(c, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
}

cudaError_t launch_finish(const phe_ctx* c, int mode, const u64* Phat, u32 nseg, const u64* body,
                          const phe::PackGeom& pg, u32 u_base, u32 cu, void* oa, void* ob, cudaStream_t s) {
  switch (c->logn) {
    case 8: return finish_by_form<8>(c, mode, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
    case 9: return finish_by_form<9>(c, mode, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
    case 10: return finish_by_form<10>(c, mode, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
    case 11: return finish_by_form<11>(c, mode, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
    case 12: return finish_by_form<12>(c, mode, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
    case 13: return finish_by_form<13>(c, mode, Phat, nseg, body, pg, u_base, cu, oa, ob, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_finish_pow2(const phe_ctx* c, const phe_ksk* k, int mode, const u64* Phat, u32 nseg,
                               size_t slice_stride, const u64* body, const phe::PackGeom& pg, u32 u_base, u32 cu,
                               void* oa, void* ob, cudaStream_t s) {
#define PHE_FIN2(L)                                                                                     \
  return mode == phe::kOutRaw                                                                          \
             ? finish_pow2<L, phe::kOutRaw>(c, k, Phat, nseg, slice_stride, body, pg, u_base, cu, oa, ob, s) \
             : finish_pow2<L, phe::kOutSwitched>(c, k, Phat, nseg, slice_stride, body, pg, u_base, cu, oa, ob, s)
  switch (c->logn) {
    case 8: PHE_FIN2(8);
    case 9: PHE_FIN2(9);
    case 10: PHE_FIN2(10);
    case 11: PHE_FIN2(11);
    case 12: PHE_FIN2(12);
    case 13: PHE_FIN2(13);
    default: return cudaErrorInvalidValue;
  }
#undef PHE_FIN2
}

// Tokens per unit: floor(N / rows) for dense packing of rows <= N/2, else 1.
u32 tokens_per_unit(u32 N, u32 rows, bool dense) { return (dense && 2 * rows <= N) ? N / rows : 1u; }

phe::PackGeom pack_geom(u32 N, u32 rows, u32 T, bool dense) {
  return phe::PackGeom{rows, (rows + N - 1) / N, tokens_per_unit(N, rows, dense), (u64)T * rows};
}

// Units (output RLWEs) of T tokens, and the units before token t0 (a
// multiple of tpu).
u64 pack_units(const phe::PackGeom& pg, u64 T) { return pg.G > 1 ? T * pg.G : (T + pg.tpu - 1) / pg.tpu; }
u64 units_before(const phe::PackGeom& pg, u64 t0) { return pg.G > 1 ? t0 * pg.G : t0 / pg.tpu; }

// The packing of T x rows LWE ciphertexts on `s`, in chunks of units.
cudaError_t pack_device(phe_ctx* c, const phe_ksk* k, u32 T, u32 rows, bool dense, const void* mask, bool switched,
                        const u64* body, void* oa, void* ob, int mode, cudaStream_t s) {
  const u32 N = c->prm.N, nr = k->n * k->ell;
  const phe::PackGeom pg = pack_geom(N, rows, T, dense);
  const u64 units = pack_units(pg, T);
  // per unit: int32 digit rows, then their transforms (8 bytes per word)
  const u64 unit_bytes = (u64)nr * N * (sizeof(int32_t) + sizeof(u64));
  // whole MAC blocks per chunk: each reads the key once for kMacUnits units
  u32 per = (u32)std::max<u64>(1, std::min<u64>(units, kPackScratchBytes / unit_bytes));
  if (per < units && per >= (u32)kMacUnits) per -= per % kMacUnits;
  Span call(c, phe::kKPackCall, s);
  u64* Dhat = nullptr;
  u64* Phat = nullptr;
  cudaError_t e = phe::ctx_malloc_async(c, &Dhat, (size_t)per * unit_bytes, s);
  if (e != cudaSuccess) return e;
  int32_t* D = reinterpret_cast<int32_t*>(Dhat + (size_t)per * nr * N);
  const u32 nseg_max = mac_segments(c, k, 1);  // the smallest chunk needs the most segments
  e = phe::ctx_malloc_async(c, &Phat, (size_t)k->slices * nseg_max * per * 2 * N * sizeof(u64), s);
  for (u64 u0 = 0; u0 < units && e == cudaSuccess; u0 += per) {
    const u32 cu = (u32)std::min<u64>(per, units - u0);
    {
      Span sp(c, phe::kKPackDecompose, s);
      e = launch_decompose(c, k, mask, switched, pg, (u32)u0, cu, D, s);
    }
    if (e == cudaSuccess) {
      Span sp(c, phe::kKInputNtt, s);
      phe::NttJob nj{nullptr, Dhat, cu * nr, nullptr, D};
      e = phe::launch_input_ntt(c, &nj, 1, s);
    }
    const u32 nseg = mac_segments(c, k, cu);
    const size_t slice_stride = (size_t)nseg * cu * 2 * N;  // words of one slice's partial sums
    for (u32 sl = 0; sl < k->slices && e == cudaSuccess; ++sl) {
      Span sp(c, phe::kKPackMac, s);
      e = launch_mac(c, k, Dhat, cu, nseg, Phat + sl * slice_stride, s, sl);
    }
    if (e == cudaSuccess) {
      Span sp(c, phe::kKPackFinish, s);
      e = c->pow2 ? launch_finish_pow2(c, k, mode, Phat, nseg, slice_stride, body, pg, (u32)u0, cu, oa, ob, s)
                  : launch_finish(c, mode, Phat, nseg, body, pg, (u32)u0, cu, oa, ob, s);
    }
  }
  cudaError_t f1 = Phat ? cudaFreeAsync(Phat, s) : cudaSuccess;
  cudaError_t f2 = cudaFreeAsync(Dhat, s);
  if (e != cudaSuccess) return e;
  return f1 != cudaSuccess ? f1 : f2;
}

// Eq. (LWEdot) with the masks switched straight to B^ell (what Decomp
// reads) and raw bodies, then the packing, token chunk by token chunk (a
// chunk holds whole units).
cudaError_t matmul_packed_device(phe_ctx* c, const phe_weights::Dir& D, const phe_ksk* k, u32 T, const u64* in_mask,
                                 const u64* in_seeds, const u64* in_body, void* oa, void* ob, int mode, bool dense,
                                 cudaStream_t s) {
  const u32 N = c->prm.N;
  const phe::PackGeom pg = pack_geom(N, D.rows, T, dense);
  const size_t osz = mode == phe::kOutRaw ? sizeof(u64) : sizeof(u32);
  const u64 ahat_tok = (u64)D.L * N * sizeof(u64), atil_tok = (u64)D.rows * N * sizeof(u32);
  const u64 dig_tok = phe::digit_bytes(1, D.cols);  // the bodies' digit rows (body GEMM)
  const u64 tok_bytes = ahat_tok + atil_tok + (u64)D.rows * sizeof(u64) + dig_tok;
  u32 per = (u32)std::max<u64>(1, std::min<u64>(T, kLweScratchBytes / tok_bytes));
  if (per < T) {
    per = std::max(pg.tpu, per / pg.tpu * pg.tpu);  // whole units per chunk
    // and, within 8 steps, whole MAC blocks (a key read per kMacUnits units)
    for (u32 p2 = per, n = 0; p2 >= pg.tpu && n < (u32)kMacUnits; p2 -= pg.tpu, ++n)
      if (pack_units(pg, p2) % kMacUnits == 0) {
        per = p2;
        break;
      }
  }
  per = std::min(per, T);
  Span call(c, phe::kKCall, s);
  char* scratch = nullptr;
  cudaError_t e = phe::ctx_malloc_async(c, &scratch, (size_t)per * tok_bytes + 256, s);
  if (e != cudaSuccess) return e;
  u64* ahat = reinterpret_cast<u64*>(scratch);
  u32* atil = reinterpret_cast<u32*>(scratch + (size_t)per * ahat_tok);
  u64* rawb = reinterpret_cast<u64*>(scratch + (size_t)per * (ahat_tok + atil_tok));
  char* digits = scratch + (((size_t)per * (ahat_tok + atil_tok + (u64)D.rows * sizeof(u64)) + 255) & ~(size_t)255);
  for (u32 t0 = 0; t0 < T && e == cudaSuccess; t0 += per) {
    const u32 tn = std::min(per, T - t0);
    {
      Span sp(c, phe::kKInputNtt, s);
      phe::NttJob nj{in_mask ? in_mask + (size_t)t0 * D.L * N : nullptr, ahat, tn * D.L,
                     in_seeds ? in_seeds + (size_t)t0 * D.L : nullptr};
      e = phe::launch_input_ntt(c, &nj, 1, s);
    }
    if (e == cudaSuccess) {
      phe::LweJobTable jt{};
      jt.n = 1;
      phe::LweJob& J = jt.j[0];
      J.what = D.what;
      J.ahat = ahat;
      J.out = atil;
      J.wrow = D.wrow;
      J.wbf = D.wbf;
      J.bin = in_body + (size_t)t0 * D.L * N;
      J.out_body = rawb;
      J.rows = D.rows;
      J.cols = D.cols;
      J.T = tn;
      J.L = D.L;
      J.tok_chunk = phe::kDefaultTokChunk;
      phe::set_lwe_tiles(J, c->logn);
      jt.prefix[0] = 0;
      jt.prefix[1] = J.tiles;
      const bool gemm = phe::body_on_tensor_cores(c, jt);
      if (gemm) phe::assign_body_scratch(jt, digits);
      Span sp(c, phe::kKLwedot, s);
      e = phe::launch_lwedot_packin2(c, jt, k->rcK, k->rkK, gemm, s);
    }
    if (e == cudaSuccess)
      e = pack_device(c, k, tn, D.rows, dense, atil, true, rawb,
                      static_cast<char*>(oa) + (size_t)units_before(pg, t0) * N * osz,
                      static_cast<char*>(ob) + (size_t)units_before(pg, t0) * N * osz, mode, s);
  }
  cudaError_t f = cudaFreeAsync(scratch, s);
  return e != cudaSuccess ? e : f;
}

phe_status check_ksk(const phe_ctx* c, const phe_ksk* k, const char* who) {
  if (!c || !k) return fail(PHE_EINVAL, "%s: null handle", who);
  if (k->ctx != c) return fail(PHE_EINVAL, "%s: key-switching key belongs to another context", who);
  return PHE_OK;
}

}  // namespace

extern "C" {

phe_status phe_ksk_upload(phe_ctx* c, const uint64_t* h_ka, const uint64_t* h_kb, uint32_t n, uint32_t base_log,
                          uint32_t ell, phe_ksk** out) {
  if (!c || !h_ka || !h_kb || !out) return fail(PHE_EINVAL, "phe_ksk_upload: null argument");
  *out = nullptr;
  const u32 N = c->prm.N;
  if (n != N) return fail(PHE_EINVAL, "phe_ksk_upload: n=%u must equal N=%u (LWE outputs of dimension N)", n, N);
  if (ell < 1 || ell > 4 || base_log < 1 || base_log > 30 || base_log * ell > 32)
    return fail(PHE_EINVAL, "phe_ksk_upload: base_log=%u ell=%u (need 1<=ell<=4, 1<=base_log<=30, product<=32)",
                base_log, ell);
  // the digit transform takes each residue of a digit d as p_i + d: |d| <= B/2 < p_i
  if (c->rns && (1ull << (base_log - 1)) >= std::min(c->rk.p1, c->rk.p2))
    return fail(PHE_EINVAL, "phe_ksk_upload: base_log=%u: digits of magnitude 2^%u reach the RNS prime %u", base_log,
                base_log - 1, std::min(c->rk.p1, c->rk.p2));
  const size_t nr = (size_t)n * ell, words = nr * 2 * N;
  // q = 2^K: slices of b bits with n ell N (B/2) 2^(b-1) below (p1 p2)/2
  u32 slices = 1, bits = 0;
  if (c->pow2) {
    const u32 K = c->rk.p2k;
    const double lim = std::log2((double)c->rk.Q / 2.0) - std::log2((double)nr * N) - (double)(base_log - 1);
    bits = (u32)std::floor(lim) + 1;  // 2^(bits-1) <= 2^lim
    while (bits > 1 && std::ldexp((double)nr * N, (int)(base_log - 1 + bits - 1)) >= (double)c->rk.Q / 2.0) --bits;
    if (bits < 2) return fail(PHE_EUNSUPPORTED, "phe_ksk_upload: base_log=%u ell=%u leave no exact key slice at N=%u",
                              base_log, ell, N);
    if (bits > K) bits = K;
    slices = (K + 1 + bits - 1) / bits;  // balanced digits of a K-bit centred value: K+1 bits
    if (slices > 8) return fail(PHE_EUNSUPPORTED, "phe_ksk_upload: %u key slices of %u bits needed", slices, bits);
  }
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  phe_ksk* k = new (std::nothrow) phe_ksk;
  if (!k) return fail(PHE_ENOMEM, "phe_ksk_upload: host allocation");
  k->ctx = c;
  k->n = n;
  k->base_log = base_log;
  k->ell = ell;
  k->slices = slices;
  k->slice_bits = bits;
  k->rcK = c->rc;
  k->rcK.log2_qout = base_log * ell;
  k->rkK = c->rk;
  if (c->rns) phe::set_switch_target(k->rkK, base_log * ell);
  if (c->pow2) k->rkK.p2shift = c->rk.p2k - base_log * ell;
  k->bytes = (u64)slices * words * 16;
  // the host words of one slice: rows r = i*ell + l of KA and KB interleaved
  std::vector<u64> host;
  if (c->pow2) {
    try {
      host.resize(words);
    } catch (...) {
      delete k;
      return fail(PHE_ENOMEM, "phe_ksk_upload: host staging");
    }
  }
  u64* tmp = nullptr;
  cudaError_t e = cudaMalloc((void**)&tmp, words * sizeof(u64));
  if (e == cudaSuccess) e = cudaMalloc(&k->khat, k->bytes);
  for (u32 sl = 0; sl < slices && e == cudaSuccess; ++sl) {
    if (!c->pow2) {
      e = cudaMemcpy2D(tmp, 2 * N * sizeof(u64), h_ka, N * sizeof(u64), N * sizeof(u64), nr, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy2D(tmp + N, 2 * N * sizeof(u64), h_kb, N * sizeof(u64), N * sizeof(u64), nr,
                         cudaMemcpyHostToDevice);
    } else {
      // slice sl of each centred word, as a word mod 2^K (the transform's
      // centred lift gives back the signed slice)
      const u32 K = c->rk.p2k;
      const u64 qmask = (1ull << K) - 1, half = 1ull << (bits - 1);
      for (size_t r = 0; r < nr; ++r)
        for (u32 comp = 0; comp < 2; ++comp) {
          const uint64_t* src = (comp ? h_kb : h_ka) + r * N;
          u64* dst = host.data() + (r * 2 + comp) * N;
          for (u32 m = 0; m < N; ++m) {
            const u64 w = src[m] & qmask;
            long long v = (w >> (K - 1)) ? (long long)w - (long long)(1ull << K) : (long long)w;  // centred
            long long d = 0;
            for (u32 t = 0; t <= sl; ++t) {
              const long long lo = (long long)((((u64)v + half) & ((1ull << bits) - 1)) - half);
              d = lo;
              v = (v - lo) >> bits;
            }
            dst[m] = (u64)d & qmask;
          }
        }
      e = cudaMemcpy(tmp, host.data(), words * sizeof(u64), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
      phe::NttJob nj{tmp, tmp, (u32)(nr * 2), nullptr};
      e = phe::launch_input_ntt(c, &nj, 1, 0);
    }
    if (e == cudaSuccess) {
      void* dst = static_cast<char*>(k->khat) + (size_t)sl * words * 16;
      const int blocks = (int)std::min<size_t>((words + 255) / 256, (size_t)c->num_sms * 8);
      if (c->rns) phe::ksk_finish_kernel<true><<<blocks, 256>>>(tmp, dst, words, c->rc, c->rk, c->ninv);
      else phe::ksk_finish_kernel<false><<<blocks, 256>>>(tmp, dst, words, c->rc, c->rk, c->ninv);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) {
    if (k->khat) cudaFree(k->khat);
    delete k;
    return cuda_fail(e, "phe_ksk_upload");
  }
  *out = k;
  return PHE_OK;
}

void phe_ksk_free(phe_ksk* k) {
  if (!k) return;
  DeviceGuard g(k->ctx->device);
  if (k->khat) cudaFree(k->khat);
  delete k;
}

uint64_t phe_ksk_device_bytes(const phe_ksk* k) { return k ? k->bytes : 0; }

phe_status phe_pack_layout(uint32_t N, uint32_t rows, uint32_t T, uint32_t flags, uint64_t* units,
                           uint32_t* tokens_per_unit) {
  if (N == 0 || (N & (N - 1)) || rows == 0) return fail(PHE_EINVAL, "phe_pack_layout: N=%u rows=%u", N, rows);
  if (flags & ~kPackFlags) return fail(PHE_EINVAL, "phe_pack_layout: flags=%u", flags);
  const phe::PackGeom pg = pack_geom(N, rows, T, flags & PHE_PACK_DENSE);
  if (units) *units = pack_units(pg, T);
  if (tokens_per_unit) *tokens_per_unit = pg.tpu;
  return PHE_OK;
}

phe_status phe_pack(phe_ctx* c, const phe_ksk* k, uint32_t T, uint32_t rows, const uint64_t* d_lwe_mask,
                    const uint64_t* d_lwe_body, void* d_out_a, void* d_out_b, uint32_t flags, void* stream) {
  phe_status st = check_ksk(c, k, "phe_pack");
  if (st != PHE_OK) return st;
  if (flags & ~kPackFlags) return fail(PHE_EINVAL, "phe_pack: flags=%u", flags);
  if (T == 0 || rows == 0) return PHE_OK;
  if (!d_lwe_mask || !d_lwe_body || !d_out_a || !d_out_b) return fail(PHE_EINVAL, "phe_pack: null buffer");
  if (reinterpret_cast<uintptr_t>(d_lwe_mask) % 16)
    return fail(PHE_EINVAL, "phe_pack: d_lwe_mask must be 16-byte aligned (the masks are read two words at a time)");
  const bool dense = flags & PHE_PACK_DENSE;
  const u64 units = pack_units(pack_geom(c->prm.N, rows, T, dense), T);
  if (units > (1u << 24)) return fail(PHE_EINVAL, "phe_pack: %llu output RLWEs exceed 2^24", (unsigned long long)units);
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = pack_device(c, k, T, rows, dense, d_lwe_mask, false, reinterpret_cast<const u64*>(d_lwe_body),
                              d_out_a, d_out_b, (flags & PHE_OUT_RAW) ? phe::kOutRaw : phe::kOutSwitched,
                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_pack");
  return PHE_OK;
}

phe_status phe_matmul_packed(phe_ctx* c, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                             const uint64_t* d_in_mask, const uint64_t* d_in_body, void* d_out_a, void* d_out_b,
                             uint32_t flags, void* stream) {
  phe_status st = check_ksk(c, k, "phe_matmul_packed");
  if (st != PHE_OK) return st;
  uint32_t rows = 0, cols = 0, L = 0;
  if (!w || w->ctx != c) return fail(PHE_EINVAL, "phe_matmul_packed: weights missing or of another context");
  if ((st = phe_weights_shape(w, dir, &rows, &cols, &L)) != PHE_OK) return st;
  if (flags & ~kPackFlags) return fail(PHE_EINVAL, "phe_matmul_packed: flags=%u", flags);
  if (T == 0) return PHE_OK;
  if (!d_in_mask || !d_in_body || !d_out_a || !d_out_b) return fail(PHE_EINVAL, "phe_matmul_packed: null buffer");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = matmul_packed_device(c, w->dir[dir], k, T, reinterpret_cast<const u64*>(d_in_mask), nullptr,
                                       reinterpret_cast<const u64*>(d_in_body), d_out_a, d_out_b,
                                       (flags & PHE_OUT_RAW) ? phe::kOutRaw : phe::kOutSwitched,
                                       flags & PHE_PACK_DENSE, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_packed");
  return PHE_OK;
}

phe_status phe_matmul_packed_seeded(phe_ctx* c, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                                    const uint64_t* d_in_seeds, const uint64_t* d_in_body, void* d_out_a,
                                    void* d_out_b, uint32_t flags, void* stream) {
  phe_status st = check_ksk(c, k, "phe_matmul_packed_seeded");
  if (st != PHE_OK) return st;
  uint32_t rows = 0, cols = 0, L = 0;
  if (!w || w->ctx != c) return fail(PHE_EINVAL, "phe_matmul_packed_seeded: weights missing or of another context");
  if ((st = phe_weights_shape(w, dir, &rows, &cols, &L)) != PHE_OK) return st;
  if (flags & ~kPackFlags) return fail(PHE_EINVAL, "phe_matmul_packed_seeded: flags=%u", flags);
  if (T == 0) return PHE_OK;
  if (!d_in_seeds || !d_in_body || !d_out_a || !d_out_b)
    return fail(PHE_EINVAL, "phe_matmul_packed_seeded: null buffer");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = matmul_packed_device(c, w->dir[dir], k, T, nullptr, reinterpret_cast<const u64*>(d_in_seeds),
                                       reinterpret_cast<const u64*>(d_in_body), d_out_a, d_out_b,
                                       (flags & PHE_OUT_RAW) ? phe::kOutRaw : phe::kOutSwitched,
                                       flags & PHE_PACK_DENSE, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_packed_seeded");
  return PHE_OK;
}

phe_status phe_matmul_packed_host(phe_ctx* c, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                                  const uint64_t* h_in_mask, const uint64_t* h_in_body, void* h_out_a,
                                  void* h_out_b, uint32_t flags, uint32_t tok_chunk, void* stream) {
  phe_status st = check_ksk(c, k, "phe_matmul_packed_host");
  if (st != PHE_OK) return st;
  uint32_t rows = 0, cols = 0, L = 0;
  if (!w || w->ctx != c) return fail(PHE_EINVAL, "phe_matmul_packed_host: weights missing or of another context");
  if ((st = phe_weights_shape(w, dir, &rows, &cols, &L)) != PHE_OK) return st;
  if (flags & ~kPackFlags) return fail(PHE_EINVAL, "phe_matmul_packed_host: flags=%u", flags);
  if (T == 0) return PHE_OK;
  if (!h_in_mask || !h_in_body || !h_out_a || !h_out_b) return fail(PHE_EINVAL, "phe_matmul_packed_host: null buffer");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const u32 N = c->prm.N;
  const phe::PackGeom pg = pack_geom(N, rows, T, flags & PHE_PACK_DENSE);
  const size_t osz = (flags & PHE_OUT_RAW) ? sizeof(u64) : sizeof(u32);
  const size_t in_tok = (size_t)L * N * sizeof(u64), out_unit = (size_t)N * osz;
  u32 tc = std::max(1u, std::min(tok_chunk ? tok_chunk : 8u, T));
  if (tc < T) tc = std::min(T, std::max(pg.tpu, tc / pg.tpu * pg.tpu));  // whole units per chunk
  cudaStream_t caller = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!c->side[i]) e = cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  cudaEvent_t ev = nullptr;
  if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  e = cudaEventRecord(ev, caller);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->side[i], ev, 0);
  // two buffer sets on the context's two side streams: the copies of one
  // chunk overlap the kernels of the next
  struct Buf { u64 *a = nullptr, *b = nullptr; char *oa = nullptr, *ob = nullptr; } buf[2];
  const u32 nchunks = (T + tc - 1) / tc;
  for (int i = 0; i < 2 && i < (int)nchunks && e == cudaSuccess; ++i) {
    cudaStream_t s = c->side[i];
    if ((e = phe::ctx_malloc_async(c, &buf[i].a, tc * in_tok, s)) != cudaSuccess) break;
    if ((e = phe::ctx_malloc_async(c, &buf[i].b, tc * in_tok, s)) != cudaSuccess) break;
    if ((e = phe::ctx_malloc_async(c, &buf[i].oa, pack_units(pg, tc) * out_unit, s)) != cudaSuccess) break;
    e = phe::ctx_malloc_async(c, &buf[i].ob, pack_units(pg, tc) * out_unit, s);
  }
  for (u32 n = 0; n < nchunks && e == cudaSuccess && st == PHE_OK; ++n) {
    const u32 t0 = n * tc, tn = std::min(tc, T - t0);
    cudaStream_t s = c->side[n % 2];
    Buf& B = buf[n % 2];
    if ((e = cudaMemcpyAsync(B.a, reinterpret_cast<const char*>(h_in_mask) + t0 * in_tok, tn * in_tok,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(B.b, reinterpret_cast<const char*>(h_in_body) + t0 * in_tok, tn * in_tok,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    st = phe_matmul_packed(c, w, k, dir, tn, reinterpret_cast<const uint64_t*>(B.a),
                           reinterpret_cast<const uint64_t*>(B.b), B.oa, B.ob, flags, s);
    if (st != PHE_OK) break;
    const size_t o0 = units_before(pg, t0) * out_unit, on = pack_units(pg, tn) * out_unit;
    if ((e = cudaMemcpyAsync(static_cast<char*>(h_out_a) + o0, B.oa, on, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      break;
    e = cudaMemcpyAsync(static_cast<char*>(h_out_b) + o0, B.ob, on, cudaMemcpyDeviceToHost, s);
  }
  for (int i = 0; i < 2; ++i) {
    cudaStream_t s = c->side[i];
    if (buf[i].a) cudaFreeAsync(buf[i].a, s);
    if (buf[i].b) cudaFreeAsync(buf[i].b, s);
    if (buf[i].oa) cudaFreeAsync(buf[i].oa, s);
    if (buf[i].ob) cudaFreeAsync(buf[i].ob, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
  }
  cudaEventDestroy(ev);
  if (st != PHE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_packed_host");
  return PHE_OK;
}

}  // extern "C"
