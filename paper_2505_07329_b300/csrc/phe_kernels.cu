// CUDA kernels of the hot path (sm_103a):
//   input_ntt_kernel   forward negacyclic NTT of the input masks A_ti (or of
//                      masks expanded from seeds)
//   weight_ntt_kernel  w_hat_ij (reversed weight blocks, Sec. 4.3.1) -> NTT domain, x N^-1
//   lwedot_kernel      Eq. (LWEdot): pointwise sum over blocks, inverse NTT,
//                      SampleExtract at N-1 (index reversal), ModulusSwitch --
//                      one fused pass per (token, row) for the masks; the
//                      bodies b'_tj = sum_k W[j,k] B_t[k] (mod q) come from
//                      the tensor-core GEMM of phe_body.cu (kBodyGemm), or,
//                      in the allocation-free entry point, from a dp4a dot
//                      product fused into this kernel
//   modswitch_kernel   unfused ModulusSwitch
//   expand_masks_kernel seeded masks written out
//
// Each transform kernel has two arithmetic forms: 64-bit words mod q (any
// NTT-friendly q < 2^61), and -- when q = p1 p2 is a product of two 30-bit
// NTT primes -- a pair of 32-bit residues (RNS), which halves the multiply
// work per butterfly; the epilogue returns to q by the CRT before the switch.
//
// Why the inverse NTT yields SampleExtract at N-1: with P = A_i * w_hat_ij
// in R_q, SampleExtract(., N-1) takes a'_m = P_{N-1-m} for every m (the
// second branch of the formula is empty at h = N-1) and b' = (B_i *
// w_hat_ij)_{N-1}.  The block sum commutes with the transform, so the kernel
// sums A_hat_ti . W_hat_ij over i in the NTT domain, runs one inverse
// transform per (token, row) and writes coefficient N-1-m to slot m.
#include <cstdio>
#include <type_traits>

#include "phe_host.hpp"

namespace phe {

template <bool RNS>
using RingOf = std::conditional_t<RNS, Ring2x32, Ring64>;

template <bool RNS>
__device__ __forceinline__ RingOf<RNS> make_ring(const RingConst& rc, const RnsConst& rk, bool inverse) {
  if constexpr (RNS) {
    return Ring2x32{rk.p1, rk.p2};
  } else {
    return Ring64{rc.q, inverse ? rc.q4 : rc.q2};
  }
}

// --------------------------------------------------------------------------
// Forward transform of input masks: [blocks][N] natural -> A_hat layout.
// --------------------------------------------------------------------------
template <int LOGN, bool RNS, bool P2 = false>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    input_ntt_kernel(NttJob job, RingConst rc, RnsConst rk, const void* __restrict__ tw0v,
                     const void* __restrict__ twcv) {
  static_assert(RNS || !P2, "a power-of-two q runs in the RNS form");
  using S = Shape<LOGN>;
  using R = RingOf<RNS>;
  using W = typename R::Word;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / S::P, p = threadIdx.x % S::P;
  u64* buf64 = smem + slot * S::PADN;
  W* buf = reinterpret_cast<W*>(buf64);
  const u32 b = blockIdx.x * S::SLOTS + slot;
  const bool active = b < job.blocks;
  u64 v[16];
  if (job.seeds) {
    // Seeded mask: each thread expands 4 keystream blocks (16 coefficients)
    // into shared memory in natural order, then loads its transform words.
    const u64 seed = active ? job.seeds[b] : 0ull;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const u32 cb = p + k * S::P;
      u64 m4[4];
      seeded_mask4(seed, cb, rc, m4);
#pragma unroll
      for (int c = 0; c < 4; ++c) buf64[pad_idx(4 * cb + c)] = m4[c];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = buf64[pad_idx(pass_pos<LOGN, NP - 1>(p, e))];
    __syncthreads();
  } else if (!job.digits) {
    const u64* src = job.src + (size_t)(active ? b : 0) * S::N;
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = active ? reduce_word(src[pass_pos<LOGN, NP - 1>(p, e)], rc) : 0ull;
  }
  W x[16];
  if (job.digits) {
    // small signed integers: in the RNS form (gadget digits, |d| <= 2^29 <
    // p_i) each residue is p_i + d, in (0, 2 p_i) as the first butterflies
    // take it; in the 64-bit form (|d| < 2^31) d or q + d
    const int32_t* src = job.digits + (size_t)(active ? b : 0) * S::N;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int d = active ? src[pass_pos<LOGN, NP - 1>(p, e)] : 0;
      if constexpr (RNS) x[e] = make_uint2(rk.p1 + d, rk.p2 + d);
      else x[e] = d < 0 ? rc.q - (u64)(-(long long)d) : (u64)d;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if constexpr (P2) x[e] = pow2_residues(v[e], rk);
      else if constexpr (RNS) x[e] = to_residues(v[e], rk);
      else x[e] = v[e];
    }
  }
  ntt_regs<LOGN>(x, p, buf, reinterpret_cast<const typename R::Tw*>(tw0v),
                 reinterpret_cast<const typename R::Tw*>(twcv), make_ring<RNS>(rc, rk, false));
  if (active) {
    // words (r, r+1) of a thread stored together: 16 bytes, a warp covers 512
    W* dst = reinterpret_cast<W*>(job.dst + (size_t)b * S::N);
#pragma unroll
    for (int r = 0; r < 16; r += 2) {
      W* d = dst + 2 * ((r >> 1) * S::P + p);
      d[0] = x[r];
      d[1] = x[r + 1];
    }
  }
}

// --------------------------------------------------------------------------
// Weight encoding: block i of output row j holds w_hat_ij[k] = W(j, iN+N-1-k)
// (zero past cols); W(j, k) = W[j*rs + k*cs] lets one kernel read W for the
// forward pass and W^T for the backward pass.  Output: N^-1 NTT(w_hat) with
// Shoup quotients, fully reduced: (w, w') pairs mod q, or (w1, w1', w2, w2')
// for the RNS form.  rev = 0 skips the reversal (the client's key
// polynomial in phe_client_encrypt).
// --------------------------------------------------------------------------
__device__ __forceinline__ u64 shoup_quotient(u64 w, u64 q) {
  // floor(w 2^64 / q) by restoring long division (w < q < 2^61).
  u64 rem = w, quo = 0;
#pragma unroll 8
  for (int i = 0; i < 64; ++i) {
    rem <<= 1;
    quo <<= 1;
    if (rem >= q) {
      rem -= q;
      quo |= 1ull;
    }
  }
  return quo;
}

template <int LOGN, bool RNS>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    weight_ntt_kernel(const int8_t* __restrict__ W, u32 rows, u32 cols, u32 rs, u32 cs, u32 L, int rev,
                      void* __restrict__ whatv, RingConst rc, RnsConst rk, NInv ninv, const void* __restrict__ tw0v,
                      const void* __restrict__ twcv) {
  using S = Shape<LOGN>;
  using R = RingOf<RNS>;
  using Wd = typename R::Word;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / S::P, p = threadIdx.x % S::P;
  Wd* buf = reinterpret_cast<Wd*>(smem + slot * S::PADN);
  const u32 b = blockIdx.x * S::SLOTS + slot;
  const bool active = b < rows * L;
  const u32 j = active ? b / L : 0, i = active ? b % L : 0;
  Wd x[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const u32 pos = (u32)pass_pos<LOGN, NP - 1>(p, e);
    const u32 k = i * S::N + (rev ? (S::N - 1 - pos) : pos);
    const int w = (active && k < cols) ? (int)W[(size_t)j * rs + (size_t)k * cs] : 0;
    if constexpr (RNS) {
      x[e] = make_uint2((w < 0) ? rk.p1 - (u32)(-w) : (u32)w, (w < 0) ? rk.p2 - (u32)(-w) : (u32)w);
    } else {
      x[e] = (w < 0) ? rc.q - (u64)(-w) : (u64)w;
    }
  }
  ntt_regs<LOGN>(x, p, buf, reinterpret_cast<const typename R::Tw*>(tw0v),
                 reinterpret_cast<const typename R::Tw*>(twcv), make_ring<RNS>(rc, rk, false));
  if (active) {
    if constexpr (RNS) {
      uint4* dst = reinterpret_cast<uint4*>(whatv) + (size_t)b * S::N;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        u32 a1 = sub_if32(sub_if32(x[r].x, 2 * rk.p1), rk.p1);
        u32 a2 = sub_if32(sub_if32(x[r].y, 2 * rk.p2), rk.p2);
        a1 = sub_if32(mul_shoup32(a1, ninv.n1, ninv.n1p, rk.p1), rk.p1);
        a2 = sub_if32(mul_shoup32(a2, ninv.n2, ninv.n2p, rk.p2), rk.p2);
        dst[what_idx<LOGN>(p, r)] = make_uint4(a1, (u32)(((u64)a1 << 32) / rk.p1), a2,
                                               (u32)(((u64)a2 << 32) / rk.p2));
      }
    } else {
      ulonglong2* dst = reinterpret_cast<ulonglong2*>(whatv) + (size_t)b * S::N;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        u64 v = reduce_4q(x[r], rc.q, rc.q2);
        v = reduce_2q(mul_shoup(v, ninv.n64, ninv.n64p, rc.q), rc.q);
        dst[what_idx<LOGN>(p, r)] = make_ulonglong2(v, shoup_quotient(v, rc.q));
      }
    }
  }
}

// --------------------------------------------------------------------------
// Eq. (LWEdot).  A tile is (job, output row, chunk of tokens); the block walks
// the chunk SLOTS tokens at a time.  Per (token, row):
//   mask  sum_i A_hat_ti . W_hat_ij in the NTT domain, inverse transform,
//         coefficient N-1-m to slot m (SampleExtract at N-1), switch;
//   body  coefficient N-1 of sum_i B_ti * w_hat_ij, i.e. the plain dot
//         product sum_k W(j,k) B_t[k], exact in three int64 partial sums
//         (any 64-bit word B = B2 2^60 + B1 2^30 + B0 with B0, B1 < 2^30,
//         B2 < 16; |sum| < 2^14 2^7 2^30 = 2^51 < q), reduced across the
//         block and switched.
// --------------------------------------------------------------------------
// Resident threads per SM the register budget is sized for: 3 blocks of 256
// (80 registers a thread).  A 512-thread block (N = 8192) gets one block's
// worth, not three: 3 x 512 threads would leave 40 registers and spill.
#ifndef PHE_LWEDOT_MIN_THREADS
#define PHE_LWEDOT_MIN_THREADS 768
#endif
template <int TPB>
constexpr int lwedot_min_blocks() { return (PHE_LWEDOT_MIN_THREADS / TPB) > 0 ? PHE_LWEDOT_MIN_THREADS / TPB : 1; }

// One thread's share of the body dot product of (token t, row).
__device__ __forceinline__ void body_partial(const LweJob& J, u32 row, u32 t, int p, int P, int N,
                                             long long (&acc)[3]) {
  acc[0] = acc[1] = acc[2] = 0;
  const int8_t* wr = J.wrow + (size_t)row * J.cols;
  const u64* bt = J.bin + (size_t)t * J.L * (size_t)N;
  for (u32 kk = p; kk < J.cols; kk += P) {
    const u64 b = __ldg(&bt[kk]);
    const int w = __ldg(&wr[kk]);
    acc[0] += (long long)w * (int)(b & 0x3fffffffull);
    acc[1] += (long long)w * (int)((b >> 30) & 0x3fffffffull);
    acc[2] += (long long)w * (int)(b >> 60);
  }
}

// Byte-plane form of the same dot product, for rows whose length is a
// multiple of 4 and 16-byte aligned bodies: four consecutive words B[k..k+3]
// are cut into their 8 byte planes (byte l of each word, one plane per 32-bit
// register, by byte permutes), and each plane meets the four int8 weights in
// one dp4a (signed x unsigned bytes, int32 accumulate).  The thread's sum
// sum_l acc_l 2^(8l) leaves as two int64 parts, lo (planes 0-3) + hi 2^32
// (planes 4-7); |acc_l| <= 2^21 for rows up to 16384.
__device__ __forceinline__ int dp4a_su(int a, u32 b, int c) {
  int d;
  asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ void planes4(u32 x0, u32 x1, u32 x2, u32 x3, u32 (&pl)[4]) {
  const u32 t01 = __byte_perm(x0, x1, 0x5140), t23 = __byte_perm(x2, x3, 0x5140);
  const u32 u01 = __byte_perm(x0, x1, 0x7362), u23 = __byte_perm(x2, x3, 0x7362);
  pl[0] = __byte_perm(t01, t23, 0x5410);
  pl[1] = __byte_perm(t01, t23, 0x7632);
  pl[2] = __byte_perm(u01, u23, 0x5410);
  pl[3] = __byte_perm(u01, u23, 0x7632);
}
__device__ __forceinline__ void body_partial_planes(const LweJob& J, u32 row, u32 t, int p, int P, int N,
                                                    long long (&acc)[3]) {
  const int8_t* wr = J.wrow + (size_t)row * J.cols;
  const u64* bt = J.bin + (size_t)t * J.L * (size_t)N;
  int a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (u32 k4 = 4 * (u32)p; k4 < J.cols; k4 += 4 * (u32)P) {
    const int w4 = __ldg(reinterpret_cast<const int*>(wr + k4));
    const ulonglong2 b01 = __ldg(reinterpret_cast<const ulonglong2*>(bt + k4));
    const ulonglong2 b23 = __ldg(reinterpret_cast<const ulonglong2*>(bt + k4 + 2));
    u32 lo[4], hi[4];
    planes4((u32)b01.x, (u32)b01.y, (u32)b23.x, (u32)b23.y, lo);
    planes4((u32)(b01.x >> 32), (u32)(b01.y >> 32), (u32)(b23.x >> 32), (u32)(b23.y >> 32), hi);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      a[l] = dp4a_su(w4, lo[l], a[l]);
      a[4 + l] = dp4a_su(w4, hi[l], a[4 + l]);
    }
  }
  acc[0] = (long long)a[0] + ((long long)a[1] << 8) + ((long long)a[2] << 16) + ((long long)a[3] << 24);
  acc[1] = (long long)a[4] + ((long long)a[5] << 8) + ((long long)a[6] << 16) + ((long long)a[7] << 24);
  acc[2] = 0;
}

// The body mod q from block-reduced parts: S0 + S1 2^32 (byte planes).  With
// rows of at most 2^14 int8 weights, |S0| < 2^14 2^7 2^32 = 2^53 and |S1| <
// 2^14 2^7 2^28, both below q (> 2^53 for these moduli), so a negative part
// is q minus its magnitude and no division is needed.
__device__ __forceinline__ u64 body_combine_planes(const long long (&S)[3], const RingConst& rc) {
  const u64 q = rc.q;
  const u64 v0 = (S[0] < 0) ? q - (u64)(-S[0]) : (u64)S[0];
  const u64 v1 = (S[1] < 0) ? q - (u64)(-S[1]) : (u64)S[1];
  const u64 h = reduce_2q(mul_shoup(v1, rc.c32, rc.c32p, q), q);
  return reduce_2q(v0 + h, q);
}

// The body mod q from the block-reduced partial sums S0 + S1 2^30 + S2 2^60
// (word split).
__device__ __forceinline__ u64 body_combine(const long long (&S)[3], const RingConst& rc) {
  const u64 q = rc.q;
  u64 v[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = (S[i] < 0) ? q - (u64)(-S[i]) : (u64)S[i];
  const u64 a = reduce_2q(mul_shoup(v[1], rc.c30, rc.c30p, q), q);
  const u64 b = reduce_2q(mul_shoup(v[2], rc.c60, rc.c60p, q), q);
  return reduce_2q(reduce_2q(v[0] + a, q) + b, q);
}

template <int LOGN, int MODE, bool RNS>
__global__ void __launch_bounds__(Shape<LOGN>::TPB, lwedot_min_blocks<Shape<LOGN>::TPB>())
    lwedot_kernel(const LweJobTable jt, RingConst rc, RnsConst rk, const void* __restrict__ tw0v,
                  const void* __restrict__ twcv) {
  constexpr int OUT = MODE & 3;                 // kOutSwitched, kOutRaw or kOutRing
  constexpr bool P2 = (MODE & kPow2) != 0;      // power-of-two q through the RNS modulus
  constexpr bool K32 = (MODE & kK32) != 0;      // q' = 2^32 (RNS switched outputs)
  static_assert(!K32 || (RNS && !P2 && OUT == kOutSwitched), "the 2^32 form is an RNS switched mode");
  static_assert(!(RNS && OUT == kOutRing), "client encryption runs in the 64-bit form");
  static_assert(RNS || !P2, "a power-of-two q runs in the RNS form");
  using S = Shape<LOGN>;
  using R = RingOf<RNS>;
  using W = typename R::Word;
  using Tw = typename R::Tw;
  constexpr int N = S::N;
  constexpr int P = S::P;
  constexpr int NP = S::NPASS;
  constexpr bool BODY = OUT != kOutRing && (MODE & kBodyGemm) == 0;  // body fused here
  constexpr int GW = (P < 32) ? P : 32;   // lanes of one body-reduction group
  constexpr int NGRP = P / GW;            // groups per transform
  extern __shared__ u64 smem[];
  __shared__ long long red[2][S::SLOTS][NGRP][3];
  const int slot = threadIdx.x / P, p = threadIdx.x % P;
  W* buf = reinterpret_cast<W*>(smem + slot * S::PADN);
  const Tw* tw0 = reinterpret_cast<const Tw*>(tw0v);
  const Tw* twc = reinterpret_cast<const Tw*>(twcv);
  const R ring = make_ring<RNS>(rc, rk, true);
  const u64 q = rc.q, q4 = rc.q4;
  const u32 total = jt.prefix[jt.n];
  u32 seq = 0;
  // Dynamic tiles (persistent launches): thread 0 takes the next tile from
  // the launch's counter; two slots, so that the slot a thread reads is not
  // the one thread 0 overwrites for the following tile.
  __shared__ u32 next_tile[2];
  u32 tile = blockIdx.x;
  if (jt.tile_counter) {
    if (threadIdx.x == 0) next_tile[0] = atomicAdd(jt.tile_counter, 1u);
    __syncthreads();
    tile = next_tile[0];
  }

  for (u32 round = 1; tile < total; ++round) {
    u32 k = 0;
    while (tile >= jt.prefix[k + 1]) ++k;
    const LweJob& J = jt.j[k];
    const u32 local = tile - jt.prefix[k];
    // The token chunks of one row are adjacent tiles: CTAs resident at the
    // same time share W_hat_j through L2, so a launch reads W_hat from HBM
    // about once however small the token chunk.
    // A tile is a group of RG adjacent rows times a chunk of tokens; the
    // block's slots take CS tokens of each of the RG rows per round.
    const u32 nch = (J.T + J.tok_chunk - 1) / J.tok_chunk;
    const u32 RG = J.row_group ? J.row_group : 1;
    const u32 CS = S::SLOTS / RG;
    const u32 row = (local / nch) * RG + slot / CS;
    const bool row_ok = row < J.rows;
    const u32 t0 = (local % nch) * J.tok_chunk;
    const u32 t1 = min(J.T, t0 + J.tok_chunk);
    const Tw* wrow = reinterpret_cast<const Tw*>(J.what) + (size_t)(row_ok ? row : 0) * J.L * N;
    const bool planes = (J.cols % 4 == 0) && ((reinterpret_cast<uintptr_t>(J.bin) & 15) == 0);
    const u32 iters = (t1 - t0 + CS - 1) / CS;

    for (u32 it = 0; it < iters; ++it, ++seq) {
      const u32 t = t0 + it * CS + slot % CS;
      const bool active = row_ok && t < t1;
      const int par = seq & 1;
      // the body first, while no transform words are live
      if constexpr (BODY) {
        long long acc[3] = {0, 0, 0};
        if (active) {
          if (planes) body_partial_planes(J, row, t, p, P, N, acc);
          else body_partial(J, row, t, p, P, N, acc);
        }
#pragma unroll
        for (int off = GW / 2; off > 0; off >>= 1) {
#pragma unroll
          for (int i = 0; i < 3; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off, GW);
        }
        if (p % GW == 0) {
#pragma unroll
          for (int i = 0; i < 3; ++i) red[par][slot][p / GW][i] = acc[i];
        }
      }
      W x[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if constexpr (RNS) x[r] = make_uint2(0u, 0u);
        else x[r] = 0;
      }
      if (active) {
        const u64* at = J.ahat + (size_t)t * J.L * N;
        // Block i's products; the first block's (each below 2p in the RNS
        // form, below 4q in the 64-bit form: the inverse transform's input
        // bound) are the accumulator as they stand, later ones are added and
        // reduced.
        auto block = [&](u32 i, auto first) {
          constexpr bool FIRST = decltype(first)::value;
          const Tw* wp = wrow + (size_t)i * N;
          if constexpr (RNS) {
            const uint4* ap = reinterpret_cast<const uint4*>(at + (size_t)i * N);
#pragma unroll
            for (int r = 0; r < 16; r += 2) {
              const uint4 av = __ldg(&ap[(r >> 1) * P + p]);  // (a1_r, a2_r, a1_r+1, a2_r+1)
              const uint4 w0 = __ldg(&wp[what_idx<LOGN>(p, r)]);
              const uint4 w1 = __ldg(&wp[what_idx<LOGN>(p, r + 1)]);
              const u32 m0 = mul_shoup32(av.x, w0.x, w0.y, rk.p1), m1 = mul_shoup32(av.y, w0.z, w0.w, rk.p2);
              const u32 m2 = mul_shoup32(av.z, w1.x, w1.y, rk.p1), m3 = mul_shoup32(av.w, w1.z, w1.w, rk.p2);
              if constexpr (FIRST) {
                x[r] = make_uint2(m0, m1);
                x[r + 1] = make_uint2(m2, m3);
              } else {
                x[r].x = sub_if32(x[r].x + m0, 2 * rk.p1);
                x[r].y = sub_if32(x[r].y + m1, 2 * rk.p2);
                x[r + 1].x = sub_if32(x[r + 1].x + m2, 2 * rk.p1);
                x[r + 1].y = sub_if32(x[r + 1].y + m3, 2 * rk.p2);
              }
            }
          } else {
            const ulonglong2* ap = reinterpret_cast<const ulonglong2*>(at + (size_t)i * N);
#pragma unroll
            for (int r = 0; r < 16; r += 2) {
              const ulonglong2 av = __ldg(&ap[(r >> 1) * P + p]);
              const ulonglong2 w0 = __ldg(&wp[what_idx<LOGN>(p, r)]);
              const ulonglong2 w1 = __ldg(&wp[what_idx<LOGN>(p, r + 1)]);
              const u64 m0 = mul_shoup_lazy(av.x, w0.x, w0.y, q), m1 = mul_shoup_lazy(av.y, w1.x, w1.y, q);
              if constexpr (FIRST) {
                x[r] = m0;
                x[r + 1] = m1;
              } else {
                const u64 s0 = x[r] + m0, s1 = x[r + 1] + m1;  // each term < 4q, sum < 8q
                x[r] = (s0 >= q4) ? s0 - q4 : s0;
                x[r + 1] = (s1 >= q4) ? s1 - q4 : s1;
              }
            }
          }
        };
        block(0u, std::true_type{});
        for (u32 i = 1; i < J.L; ++i) block(i, std::false_type{});
      }
      intt_regs<LOGN>(x, p, buf, tw0, twc, ring);  // barriers inside also order red[]
      if (active) {
        if constexpr (OUT == kOutSwitched || OUT == kOutRaw || OUT == kOutPackIn) {
          constexpr bool SWM = OUT == kOutSwitched || OUT == kOutPackIn;  // masks switched
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int pos = pass_pos<LOGN, NP - 1>(p, e);
            const size_t o = ((size_t)t * J.rows + row) * N + (N - 1 - pos);
            if constexpr (P2) {
              const u32 c1 = sub_if32(x[e].x, rk.p1);
              const u64 v = pow2_from_crt(c1, crt_digit_lazy(c1, x[e].y, rk), rk);
              if constexpr (SWM) reinterpret_cast<uint32_t*>(J.out)[o] = pow2_modswitch(v, rk);
              else reinterpret_cast<u64*>(J.out)[o] = v;
            } else if constexpr (RNS) {
              const u32 c1 = sub_if32(x[e].x, rk.p1);
              const u32 h = crt_digit_lazy(c1, x[e].y, rk);
              if constexpr (SWM) reinterpret_cast<uint32_t*>(J.out)[o] = rns_modswitch<K32>(c1, h, rk);
              else reinterpret_cast<u64*>(J.out)[o] = (u64)c1 + (u64)rk.p1 * h;
            } else {
              const u64 c = reduce_4q(x[e], q, rc.q2);
              if constexpr (SWM) reinterpret_cast<uint32_t*>(J.out)[o] = modswitch_word(c, rc);
              else reinterpret_cast<u64*>(J.out)[o] = c;
            }
          }
        } else if constexpr (!RNS) {
          // Ring product in natural order plus E + delta * x_hat: client-side
          // RLWE encryption (one row: the key); `t` runs over token blocks.
          const u32 Le = (J.msg_d + N - 1) / N;
          const u32 tok = t / Le, blk = t % Le;
          u64* out = reinterpret_cast<u64*>(J.out) + (size_t)t * N;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int pos = pass_pos<LOGN, NP - 1>(p, e);
            u64 v = reduce_4q(x[e], q, rc.q2);
            const int32_t ev = J.err[(size_t)t * N + pos];
            v += (ev < 0) ? q - (u64)(-(int64_t)ev) : (u64)ev;
            v = reduce_2q(v, q);
            const u32 mi = blk * N + pos;
            const int m = (mi < J.msg_d) ? (int)J.msg[(size_t)tok * J.msg_d + mi] : 0;
            const u64 mq = (m < 0) ? q - (u64)(-m) : (u64)m;
            v += reduce_2q(mul_shoup(mq, J.delta, J.delta_p, q), q);
            out[pos] = reduce_2q(v, q);
          }
        }
        if constexpr (BODY) {
          if (p == 0) {
            long long S3[3] = {0, 0, 0};
#pragma unroll
            for (int g = 0; g < NGRP; ++g) {
#pragma unroll
              for (int i = 0; i < 3; ++i) S3[i] += red[par][slot][g][i];
            }
            if constexpr (P2) {
              // the parts' sum mod 2^64 is exact mod q = 2^p2k
              const u64 v = (planes ? ((u64)S3[0] + ((u64)S3[1] << 32))
                                    : ((u64)S3[0] + ((u64)S3[1] << 30) + ((u64)S3[2] << 60))) & (rc.q - 1);
              if constexpr (OUT == kOutSwitched)
                reinterpret_cast<uint32_t*>(J.out_body)[(size_t)t * J.rows + row] = pow2_modswitch(v, rk);
              else
                reinterpret_cast<u64*>(J.out_body)[(size_t)t * J.rows + row] = v;
            } else {
              const u64 v = planes ? body_combine_planes(S3, rc) : body_combine(S3, rc);
              if constexpr (OUT == kOutSwitched)
                reinterpret_cast<uint32_t*>(J.out_body)[(size_t)t * J.rows + row] = modswitch_word(v, rc);
              else
                reinterpret_cast<u64*>(J.out_body)[(size_t)t * J.rows + row] = v;
            }
          }
        }
      }
    }
    if (jt.tile_counter) {
      if (threadIdx.x == 0) next_tile[round & 1] = atomicAdd(jt.tile_counter, 1u);
      __syncthreads();
      tile = next_tile[round & 1];
    } else {
      tile += gridDim.x;
    }
  }
}

// Seeded masks written out in natural order: masks[i][m], m < N.
__global__ void expand_masks_kernel(const u64* __restrict__ seeds, u32 n, u32 N, u64* __restrict__ masks,
                                    RingConst rc) {
  const size_t nblocks = (size_t)n * (N / 4);
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nblocks;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx / (N / 4);
    const u32 cb = (u32)(idx % (N / 4));
    u64 v[4];
    seeded_mask4(seeds[i], cb, rc, v);
    u64* out = masks + i * N + 4 * cb;
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = v[c];
  }
}

// Unfused switch of single words.  An RNS modulus takes the residue form of
// the fused epilogue: residues, CRT digit, 32-bit quotient estimate.
__global__ void modswitch_kernel(const u64* __restrict__ in, uint32_t* __restrict__ out, size_t n, RingConst rc,
                                 RnsConst rk, bool rns) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const u64 c = reduce_word(in[i], rc);
    if (rk.p2k) {
      out[i] = pow2_modswitch(c, rk);
    } else if (rns) {
      const uint2 r = to_residues(c, rk);
      out[i] = rns_modswitch(r.x, crt_digit_lazy(r.x, r.y, rk), rk);
    } else {
      out[i] = modswitch_word(c, rc);
    }
  }
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------
int lwedot_threads(int logn) { return (logn - 4 >= 8) ? (1 << (logn - 4)) : 256; }
size_t lwedot_smem(int logn) {
  const int N = 1 << logn;
  const int slots = lwedot_threads(logn) / (N / 16);
  return (size_t)slots * (N + N / 16) * sizeof(u64);
}

template <typename F>
static cudaError_t set_smem(F* f, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static const void* tw0_of(const phe_ctx* c, bool rns, bool inverse) {
  const Tables& t = rns ? c->tab32 : c->tab;
  return inverse ? (const void*)t.inv_0 : (const void*)t.fwd_0;
}
static const void* twc_of(const phe_ctx* c, bool rns, bool inverse) {
  const Tables& t = rns ? c->tab32 : c->tab;
  return inverse ? (const void*)t.inv_c : (const void*)t.fwd_c;
}

// Calls f(integral_constant<int, LOGN>) for the context's ring degree.
template <class F>
static cudaError_t by_logn(int logn, F&& f) {
  switch (logn) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 10: return f(std::integral_constant<int, 10>{});
    case 11: return f(std::integral_constant<int, 11>{});
    case 12: return f(std::integral_constant<int, 12>{});
    case 13: return f(std::integral_constant<int, 13>{});
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_input_ntt(const phe_ctx* c, const NttJob* jobs, int n, cudaStream_t s, bool force64) {
  const bool rns = c->rns && !force64;
  for (int i = 0; i < n; ++i) {
    if (jobs[i].blocks == 0) continue;
    const NttJob job = jobs[i];
    cudaError_t e = by_logn(c->logn, [&](auto lg) -> cudaError_t {
      constexpr int LOGN = decltype(lg)::value;
      using S = Shape<LOGN>;
      const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
      const u32 grid = (job.blocks + S::SLOTS - 1) / S::SLOTS;
      if (rns && c->pow2) {
        cudaError_t e2 = set_smem(input_ntt_kernel<LOGN, true, true>, smem);
        if (e2 != cudaSuccess) return e2;
        input_ntt_kernel<LOGN, true, true><<<grid, S::TPB, smem, s>>>(job, c->rc, c->rk, tw0_of(c, true, false),
                                                                      twc_of(c, true, false));
      } else if (rns) {
        cudaError_t e2 = set_smem(input_ntt_kernel<LOGN, true>, smem);
        if (e2 != cudaSuccess) return e2;
        input_ntt_kernel<LOGN, true><<<grid, S::TPB, smem, s>>>(job, c->rc, c->rk, tw0_of(c, true, false),
                                                                twc_of(c, true, false));
      } else {
        cudaError_t e2 = set_smem(input_ntt_kernel<LOGN, false>, smem);
        if (e2 != cudaSuccess) return e2;
        input_ntt_kernel<LOGN, false><<<grid, S::TPB, smem, s>>>(job, c->rc, c->rk, tw0_of(c, false, false),
                                                                 twc_of(c, false, false));
      }
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_weight_ntt(const phe_ctx* c, const int8_t* W, u32 rows, u32 cols, u32 rs, u32 cs, u32 L,
                              int rev, void* what, cudaStream_t s, bool force64) {
  const bool rns = c->rns && !force64;
  return by_logn(c->logn, [&](auto lg) -> cudaError_t {
    constexpr int LOGN = decltype(lg)::value;
    using S = Shape<LOGN>;
    const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
    const u32 grid = (rows * L + S::SLOTS - 1) / S::SLOTS;
    if (rns) {
      cudaError_t e = set_smem(weight_ntt_kernel<LOGN, true>, smem);
      if (e != cudaSuccess) return e;
      weight_ntt_kernel<LOGN, true><<<grid, S::TPB, smem, s>>>(W, rows, cols, rs, cs, L, rev, what, c->rc, c->rk,
                                                               c->ninv, tw0_of(c, true, false),
                                                               twc_of(c, true, false));
    } else {
      cudaError_t e = set_smem(weight_ntt_kernel<LOGN, false>, smem);
      if (e != cudaSuccess) return e;
      weight_ntt_kernel<LOGN, false><<<grid, S::TPB, smem, s>>>(W, rows, cols, rs, cs, L, rev, what, c->rc, c->rk,
                                                                c->ninv, tw0_of(c, false, false),
                                                                twc_of(c, false, false));
    }
    return cudaGetLastError();
  });
}

template <int LOGN, int MODE, bool RNS>
static cudaError_t lwedot_impl(const phe_ctx* c, const LweJobTable& jt, int grid_limit, const RingConst& rc,
                               const RnsConst& rk, cudaStream_t s) {
  using S = Shape<LOGN>;
  const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
  cudaError_t e = set_smem(lwedot_kernel<LOGN, MODE, RNS>, smem);
  if (e != cudaSuccess) return e;
  const u32 total = jt.prefix[jt.n];
  if (total == 0) return cudaSuccess;
  u32 grid = total;
  if (grid_limit > 0 && grid > (u32)grid_limit) grid = (u32)grid_limit;
  if (jt.tile_counter && grid < total) {
    // persistent: CTAs take tiles from the counter, zeroed for this launch
    e = cudaMemsetAsync(jt.tile_counter, 0, sizeof(u32), s);
    if (e != cudaSuccess) return e;
    lwedot_kernel<LOGN, MODE, RNS><<<grid, S::TPB, smem, s>>>(jt, rc, rk, tw0_of(c, RNS, true), twc_of(c, RNS, true));
  } else {
    LweJobTable one_per_tile = jt;  // a CTA per tile: no counter
    one_per_tile.tile_counter = nullptr;
    lwedot_kernel<LOGN, MODE, RNS><<<grid, S::TPB, smem, s>>>(one_per_tile, rc, rk, tw0_of(c, RNS, true),
                                                              twc_of(c, RNS, true));
  }
  return cudaGetLastError();
}

// The instantiated (mode, form) pairs: bodies fused in lwedot (no kBodyGemm:
// small launch groups, and the allocation-free entry point) or from the
// tensor-core GEMM (kBodyGemm).
#define PHE_LWEDOT_MODES(X)                                                                           \
  X(kOutSwitched, false) X(kOutRaw, false) X(kOutRing, false) X(kOutSwitched, true)                  \
  X(kOutSwitched | kK32, true) X(kOutRaw, true) X(kOutSwitched | kPow2, true) X(kOutRaw | kPow2, true) \
  X(kOutSwitched | kBodyGemm, false) X(kOutRaw | kBodyGemm, false) X(kOutSwitched | kBodyGemm, true) \
  X(kOutSwitched | kK32 | kBodyGemm, true) X(kOutRaw | kBodyGemm, true)                               \
  X(kOutSwitched | kPow2 | kBodyGemm, true) X(kOutRaw | kPow2 | kBodyGemm, true)                      \
  X(kOutPackIn | kBodyGemm, false) X(kOutPackIn | kBodyGemm, true) X(kOutPackIn | kPow2 | kBodyGemm, true) \
  X(kOutPackIn, false) X(kOutPackIn, true) X(kOutPackIn | kPow2, true)

template <int LOGN>
static cudaError_t lwedot_dispatch(const phe_ctx* c, const LweJobTable& jt, int mode, bool rns, int grid_limit,
                                   const RingConst& rc, const RnsConst& rk, cudaStream_t s) {
  const int key = mode | (rns ? 64 : 0);
#define PHE_CASE(M, R) \
  if (key == ((M) | ((R) ? 64 : 0))) return lwedot_impl<LOGN, (M), (R)>(c, jt, grid_limit, rc, rk, s);
  PHE_LWEDOT_MODES(PHE_CASE)
#undef PHE_CASE
  return cudaErrorInvalidValue;
}

// Adds the form flags (kPow2, kK32) the context implies to a call's mode
// (kOutSwitched / kOutRaw / kOutRing / kOutPackIn, optionally | kBodyGemm).
static int full_mode(const phe_ctx* c, int mode, bool rns) {
  const int out = mode & 3;
  if (rns && c->pow2) return mode | kPow2;
  if (rns && out == kOutSwitched && c->prm.log2_qout == 32) return mode | kK32;
  return mode;
}

cudaError_t launch_lwedot(const phe_ctx* c, const LweJobTable& jt, int mode, int grid_limit, cudaStream_t s,
                          bool force64) {
  const bool rns = c->rns && !force64 && (mode & 3) != kOutRing;
  return by_logn(c->logn, [&](auto lg) -> cudaError_t {
    return lwedot_dispatch<decltype(lg)::value>(c, jt, full_mode(c, mode, rns), rns, grid_limit, c->rc, c->rk, s);
  });
}

cudaError_t launch_lwedot_packin2(const phe_ctx* c, const LweJobTable& jt, const RingConst& rcK, const RnsConst& rkK,
                                  bool gemm, cudaStream_t s) {
  if (jt.prefix[jt.n] == 0) return cudaSuccess;
  if (gemm) {
    cudaError_t e = launch_body(c, jt, /*raw=*/true, c->rc, c->rk, s);
    if (e != cudaSuccess) return e;
  }
  return by_logn(c->logn, [&](auto lg) -> cudaError_t {
    const int mode = kOutPackIn | (gemm ? kBodyGemm : 0) | ((c->rns && c->pow2) ? kPow2 : 0);
    return lwedot_dispatch<decltype(lg)::value>(c, jt, mode, c->rns, 0, rcK, rkK, s);
  });
}

cudaError_t prepare_launches(const phe_ctx* c) {
  cudaError_t e = by_logn(c->logn, [&](auto lg) -> cudaError_t {
    constexpr int LOGN = decltype(lg)::value;
    using S = Shape<LOGN>;
    const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
    cudaError_t e2 = set_smem(input_ntt_kernel<LOGN, false>, smem);
    if (e2 == cudaSuccess) e2 = set_smem(input_ntt_kernel<LOGN, true>, smem);
    if (e2 == cudaSuccess) e2 = set_smem(input_ntt_kernel<LOGN, true, true>, smem);
    if (e2 == cudaSuccess) e2 = set_smem(weight_ntt_kernel<LOGN, false>, smem);
    if (e2 == cudaSuccess) e2 = set_smem(weight_ntt_kernel<LOGN, true>, smem);
#define PHE_PREP(M, R) \
  if (e2 == cudaSuccess) e2 = set_smem(lwedot_kernel<LOGN, (M), (R)>, smem);
    PHE_LWEDOT_MODES(PHE_PREP)
#undef PHE_PREP
    return e2;
  });
  if (e == cudaSuccess) e = prepare_body_launches();
  return e;
}

cudaError_t launch_expand_masks(const phe_ctx* c, const u64* seeds, u32 n, u64* masks, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t work = (size_t)n * (c->prm.N / 4);
  size_t blocks = (work + 255) / 256;
  const size_t cap = (size_t)c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  expand_masks_kernel<<<(unsigned)blocks, 256, 0, s>>>(seeds, n, c->prm.N, masks, c->rc);
  return cudaGetLastError();
}

cudaError_t launch_modswitch(const phe_ctx* c, const u64* in, uint32_t* out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  const size_t cap = (size_t)c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  modswitch_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, n, c->rc, c->rk, c->rns && !c->pow2);
  return cudaGetLastError();
}

}  // namespace phe
