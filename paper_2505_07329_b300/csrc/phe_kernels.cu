// CUDA kernels of the hot path (sm_103a):
//   input_ntt_kernel   forward negacyclic NTT of the input masks A_ti
//   weight_ntt_kernel  w_hat_ij (reversed weight blocks, Sec. 4.3.1) -> NTT domain, x N^-1
//   lwedot_kernel      Eq. (LWEdot): pointwise sum over blocks, inverse NTT,
//                      SampleExtract at N-1 (index reversal), ModulusSwitch --
//                      one fused pass per (token, row) for the masks
//                      and the bodies b'_tj = sum_k W[j,k] B_t[k] (mod q)
//   modswitch_kernel   unfused ModulusSwitch
//
// Why the inverse NTT yields SampleExtract at N-1: with P = A_i * w_hat_ij
// in R_q, SampleExtract(., N-1) takes a'_m = P_{N-1-m} for every m (the
// second branch of the formula is empty at h = N-1) and b' = (B_i *
// w_hat_ij)_{N-1}.  The block sum commutes with the transform, so the kernel
// sums A_hat_ti . W_hat_ij over i in the NTT domain, runs one inverse
// transform per (token, row) and writes coefficient N-1-m to slot m.
#include <cstdio>

#include "phe_host.hpp"

namespace phe {

// --------------------------------------------------------------------------
// Forward transform of input masks: [blocks][N] natural -> A_hat layout.
// --------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    input_ntt_kernel(NttJob job, RingConst rc, const ulonglong2* __restrict__ tw0,
                     const ulonglong2* __restrict__ twc) {
  using S = Shape<LOGN>;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / S::P, p = threadIdx.x % S::P;
  u64* buf = smem + slot * S::PADN;
  const u32 b = blockIdx.x * S::SLOTS + slot;
  const bool active = b < job.blocks;
  u64 x[16];
  if (job.seeds) {
    // Seeded mask: each thread expands 4 keystream blocks (16 coefficients)
    // into shared memory in natural order, then loads its transform words.
    const u64 seed = active ? job.seeds[b] : 0ull;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const u32 cb = p + k * S::P;
      u64 v[4];
      seeded_mask4(seed, cb, rc, v);
#pragma unroll
      for (int c = 0; c < 4; ++c) buf[pad_idx(4 * cb + c)] = v[c];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) x[e] = buf[pad_idx(pass_pos<LOGN, NP - 1>(p, e))];
    __syncthreads();
  } else {
    const u64* src = job.src + (size_t)(active ? b : 0) * S::N;
#pragma unroll
    for (int e = 0; e < 16; ++e) x[e] = active ? reduce_word(src[pass_pos<LOGN, NP - 1>(p, e)], rc) : 0ull;
  }
  ntt_regs<LOGN>(x, p, buf, tw0, twc, rc.q, rc.q2);
  if (active) {
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(job.dst + (size_t)b * S::N);
#pragma unroll
    for (int r = 0; r < 16; r += 2) dst[(r >> 1) * S::P + p] = make_ulonglong2(x[r], x[r + 1]);
  }
}

// --------------------------------------------------------------------------
// Weight encoding: block i of output row j holds w_hat_ij[k] = W(j, iN+N-1-k)
// (zero past cols); W(j, k) = W[j*rs + k*cs] lets one kernel read W for the
// forward pass and W^T for the backward pass.  Output: (N^-1 NTT(w_hat), Shoup
// quotient) pairs, fully reduced.  rev = 0 skips the reversal (the client's
// key polynomial in phe_client_encrypt).
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

template <int LOGN>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    weight_ntt_kernel(const int8_t* __restrict__ W, u32 rows, u32 cols, u32 rs, u32 cs, u32 L, int rev,
                      ulonglong2* __restrict__ what, RingConst rc, u64 ninv, u64 ninv_p,
                      const ulonglong2* __restrict__ tw0, const ulonglong2* __restrict__ twc) {
  using S = Shape<LOGN>;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / S::P, p = threadIdx.x % S::P;
  u64* buf = smem + slot * S::PADN;
  const u32 b = blockIdx.x * S::SLOTS + slot;
  const bool active = b < rows * L;
  const u32 j = active ? b / L : 0, i = active ? b % L : 0;
  u64 x[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const u32 pos = (u32)pass_pos<LOGN, NP - 1>(p, e);
    const u32 k = i * S::N + (rev ? (S::N - 1 - pos) : pos);
    const int w = (active && k < cols) ? (int)W[(size_t)j * rs + (size_t)k * cs] : 0;
    x[e] = (w < 0) ? rc.q - (u64)(-w) : (u64)w;
  }
  ntt_regs<LOGN>(x, p, buf, tw0, twc, rc.q, rc.q2);
  if (active) {
    ulonglong2* dst = what + (size_t)b * S::N;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      u64 v = reduce_4q(x[r], rc.q, rc.q2);
      v = reduce_2q(mul_shoup(v, ninv, ninv_p, rc.q), rc.q);
      dst[what_idx<LOGN>(p, r)] = make_ulonglong2(v, shoup_quotient(v, rc.q));
    }
  }
}

// --------------------------------------------------------------------------
// Eq. (LWEdot).  A tile is (job, output row, chunk of tokens); the block walks
// the chunk SLOTS tokens at a time.  Per (token, row):
//   mask  sum_i A_hat_ti . W_hat_ij in the NTT domain, inverse transform,
//         coefficient N-1-m to slot m (SampleExtract at N-1), switch;
//   body  coefficient N-1 of sum_i B_ti * w_hat_ij, i.e. the plain dot
//         product sum_k W(j,k) B_t[k], exact in two int64 partial sums
//         (B = Bh 2^30 + Bl; |sum| < 2^14 2^7 2^31 = 2^52 < q), reduced
//         across the block and switched.
// --------------------------------------------------------------------------
#ifndef PHE_LWEDOT_MIN_BLOCKS
#define PHE_LWEDOT_MIN_BLOCKS 3
#endif
template <int LOGN, int MODE>
__global__ void __launch_bounds__(Shape<LOGN>::TPB, PHE_LWEDOT_MIN_BLOCKS)
    lwedot_kernel(const LweJobTable jt, RingConst rc, const ulonglong2* __restrict__ tw0,
                  const ulonglong2* __restrict__ twc) {
  using S = Shape<LOGN>;
  constexpr int N = S::N;
  constexpr int P = S::P;
  constexpr int NP = S::NPASS;
  constexpr bool BODY = MODE != kOutRing;
  constexpr int GW = (P < 32) ? P : 32;   // lanes of one body-reduction group
  constexpr int NGRP = P / GW;            // groups per transform
  extern __shared__ u64 smem[];
  __shared__ long long red[2][S::SLOTS][NGRP][2];
  const int slot = threadIdx.x / P, p = threadIdx.x % P;
  u64* buf = smem + slot * S::PADN;
  const u64 q = rc.q, q4 = rc.q4;
  const u32 total = jt.prefix[jt.n];
  u32 seq = 0;

  for (u32 tile = blockIdx.x; tile < total; tile += gridDim.x) {
    u32 k = 0;
    while (tile >= jt.prefix[k + 1]) ++k;
    const LweJob& J = jt.j[k];
    const u32 local = tile - jt.prefix[k];
    const u32 row = local % J.rows;
    const u32 t0 = (local / J.rows) * J.tok_chunk;
    const u32 t1 = min(J.T, t0 + J.tok_chunk);
    const ulonglong2* wrow = J.what + (size_t)row * J.L * N;
    const u32 iters = (t1 - t0 + S::SLOTS - 1) / S::SLOTS;

    for (u32 it = 0; it < iters; ++it, ++seq) {
      const u32 t = t0 + it * S::SLOTS + slot;
      const bool active = t < t1;
      const int par = seq & 1;
      u64 x[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) x[r] = 0;
      if (active) {
        const u64* at = J.ahat + (size_t)t * J.L * N;
        for (u32 i = 0; i < J.L; ++i) {
          const ulonglong2* ap = reinterpret_cast<const ulonglong2*>(at + (size_t)i * N);
          const ulonglong2* wp = wrow + (size_t)i * N;
#pragma unroll
          for (int r = 0; r < 16; r += 2) {
            const ulonglong2 av = __ldg(&ap[(r >> 1) * P + p]);
            const ulonglong2 w0 = __ldg(&wp[what_idx<LOGN>(p, r)]);
            const ulonglong2 w1 = __ldg(&wp[what_idx<LOGN>(p, r + 1)]);
            const u64 s0 = x[r] + mul_shoup_lazy(av.x, w0.x, w0.y, q);
            const u64 s1 = x[r + 1] + mul_shoup_lazy(av.y, w1.x, w1.y, q);
            x[r] = (s0 >= q4) ? s0 - q4 : s0;
            x[r + 1] = (s1 >= q4) ? s1 - q4 : s1;
          }
        }
      }
      if constexpr (BODY) {
        long long al = 0, ah = 0;
        if (active) {
          const int8_t* wr = J.wrow + (size_t)row * J.cols;
          const u64* bt = J.bin + (size_t)t * J.L * N;
          for (u32 kk = p; kk < J.cols; kk += P) {
            const u64 b = reduce_word(__ldg(&bt[kk]), rc);
            const int w = __ldg(&wr[kk]);
            al += (long long)w * (int)(b & 0x3fffffffull);
            ah += (long long)w * (int)(b >> 30);
          }
        }
#pragma unroll
        for (int off = GW / 2; off > 0; off >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, off, GW);
          ah += __shfl_xor_sync(0xffffffffu, ah, off, GW);
        }
        if (p % GW == 0) {
          red[par][slot][p / GW][0] = al;
          red[par][slot][p / GW][1] = ah;
        }
      }
      intt_regs<LOGN>(x, p, buf, tw0, twc, q, q4);  // barriers inside also order red[]
      if (active) {
        if constexpr (MODE == kOutSwitched) {
          uint32_t* out = reinterpret_cast<uint32_t*>(J.out) + ((size_t)t * J.rows + row) * N;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int pos = pass_pos<LOGN, NP - 1>(p, e);
            out[N - 1 - pos] = modswitch_word(reduce_4q(x[e], q, rc.q2), rc);
          }
        } else if constexpr (MODE == kOutRaw) {
          u64* out = reinterpret_cast<u64*>(J.out) + ((size_t)t * J.rows + row) * N;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int pos = pass_pos<LOGN, NP - 1>(p, e);
            out[N - 1 - pos] = reduce_4q(x[e], q, rc.q2);
          }
        } else {
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
            long long hl = 0, ll = 0;
#pragma unroll
            for (int g = 0; g < NGRP; ++g) {
              ll += red[par][slot][g][0];
              hl += red[par][slot][g][1];
            }
            const u64 vh = (hl < 0) ? q - (u64)(-hl) : (u64)hl;
            const u64 vl = (ll < 0) ? q - (u64)(-ll) : (u64)ll;
            u64 v = reduce_2q(mul_shoup(vh, rc.c30, rc.c30p, q), q) + vl;
            v = reduce_2q(v, q);
            if constexpr (MODE == kOutSwitched)
              reinterpret_cast<uint32_t*>(J.out_body)[(size_t)t * J.rows + row] = modswitch_word(v, rc);
            else
              reinterpret_cast<u64*>(J.out_body)[(size_t)t * J.rows + row] = v;
          }
        }
      }
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

__global__ void modswitch_kernel(const u64* __restrict__ in, uint32_t* __restrict__ out, size_t n, RingConst rc) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = modswitch_word(reduce_word(in[i], rc), rc);
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

template <int LOGN>
static cudaError_t input_ntt_impl(const phe_ctx* c, const NttJob& job, cudaStream_t s) {
  using S = Shape<LOGN>;
  const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
  cudaError_t e = set_smem(input_ntt_kernel<LOGN>, smem);
  if (e != cudaSuccess) return e;
  const u32 grid = (job.blocks + S::SLOTS - 1) / S::SLOTS;
  input_ntt_kernel<LOGN><<<grid, S::TPB, smem, s>>>(job, c->rc, c->tab.fwd_0, c->tab.fwd_c);
  return cudaGetLastError();
}

cudaError_t launch_input_ntt(const phe_ctx* c, const NttJob* jobs, int n, cudaStream_t s) {
  for (int i = 0; i < n; ++i) {
    if (jobs[i].blocks == 0) continue;
    cudaError_t e;
    switch (c->logn) {
      case 8: e = input_ntt_impl<8>(c, jobs[i], s); break;
      case 9: e = input_ntt_impl<9>(c, jobs[i], s); break;
      case 10: e = input_ntt_impl<10>(c, jobs[i], s); break;
      case 11: e = input_ntt_impl<11>(c, jobs[i], s); break;
      case 12: e = input_ntt_impl<12>(c, jobs[i], s); break;
      case 13: e = input_ntt_impl<13>(c, jobs[i], s); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int LOGN>
static cudaError_t weight_ntt_impl(const phe_ctx* c, const int8_t* W, u32 rows, u32 cols, u32 rs, u32 cs, u32 L,
                                   int rev, ulonglong2* what, cudaStream_t s) {
  using S = Shape<LOGN>;
  const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
  cudaError_t e = set_smem(weight_ntt_kernel<LOGN>, smem);
  if (e != cudaSuccess) return e;
  const u32 blocks = rows * L;
  const u32 grid = (blocks + S::SLOTS - 1) / S::SLOTS;
  weight_ntt_kernel<LOGN><<<grid, S::TPB, smem, s>>>(W, rows, cols, rs, cs, L, rev, what, c->rc, c->n_inv, c->n_inv_p,
                                                     c->tab.fwd_0, c->tab.fwd_c);
  return cudaGetLastError();
}

cudaError_t launch_weight_ntt(const phe_ctx* c, const int8_t* W, u32 rows, u32 cols, u32 rs, u32 cs, u32 L,
                              int rev, ulonglong2* what, cudaStream_t s) {
  switch (c->logn) {
    case 8: return weight_ntt_impl<8>(c, W, rows, cols, rs, cs, L, rev, what, s);
    case 9: return weight_ntt_impl<9>(c, W, rows, cols, rs, cs, L, rev, what, s);
    case 10: return weight_ntt_impl<10>(c, W, rows, cols, rs, cs, L, rev, what, s);
    case 11: return weight_ntt_impl<11>(c, W, rows, cols, rs, cs, L, rev, what, s);
    case 12: return weight_ntt_impl<12>(c, W, rows, cols, rs, cs, L, rev, what, s);
    case 13: return weight_ntt_impl<13>(c, W, rows, cols, rs, cs, L, rev, what, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGN, int MODE>
static cudaError_t lwedot_impl(const phe_ctx* c, const LweJobTable& jt, int grid_limit, cudaStream_t s) {
  using S = Shape<LOGN>;
  const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
  cudaError_t e = set_smem(lwedot_kernel<LOGN, MODE>, smem);
  if (e != cudaSuccess) return e;
  const u32 total = jt.prefix[jt.n];
  if (total == 0) return cudaSuccess;
  u32 grid = total;
  if (grid_limit > 0 && grid > (u32)grid_limit) grid = (u32)grid_limit;
  lwedot_kernel<LOGN, MODE><<<grid, S::TPB, smem, s>>>(jt, c->rc, c->tab.inv_0, c->tab.inv_c);
  return cudaGetLastError();
}

template <int LOGN>
static cudaError_t lwedot_mode(const phe_ctx* c, const LweJobTable& jt, int mode, int grid_limit, cudaStream_t s) {
  switch (mode) {
    case kOutSwitched: return lwedot_impl<LOGN, kOutSwitched>(c, jt, grid_limit, s);
    case kOutRaw: return lwedot_impl<LOGN, kOutRaw>(c, jt, grid_limit, s);
    case kOutRing: return lwedot_impl<LOGN, kOutRing>(c, jt, grid_limit, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_lwedot(const phe_ctx* c, const LweJobTable& jt, int mode, int grid_limit, cudaStream_t s) {
  switch (c->logn) {
    case 8: return lwedot_mode<8>(c, jt, mode, grid_limit, s);
    case 9: return lwedot_mode<9>(c, jt, mode, grid_limit, s);
    case 10: return lwedot_mode<10>(c, jt, mode, grid_limit, s);
    case 11: return lwedot_mode<11>(c, jt, mode, grid_limit, s);
    case 12: return lwedot_mode<12>(c, jt, mode, grid_limit, s);
    case 13: return lwedot_mode<13>(c, jt, mode, grid_limit, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGN>
static cudaError_t prepare_impl() {
  using S = Shape<LOGN>;
  const size_t smem = (size_t)S::SLOTS * S::PADN * sizeof(u64);
  cudaError_t e = set_smem(input_ntt_kernel<LOGN>, smem);
  if (e == cudaSuccess) e = set_smem(weight_ntt_kernel<LOGN>, smem);
  if (e == cudaSuccess) e = set_smem(lwedot_kernel<LOGN, kOutSwitched>, smem);
  if (e == cudaSuccess) e = set_smem(lwedot_kernel<LOGN, kOutRaw>, smem);
  if (e == cudaSuccess) e = set_smem(lwedot_kernel<LOGN, kOutRing>, smem);
  return e;
}

cudaError_t prepare_launches(const phe_ctx* c) {
  switch (c->logn) {
    case 8: return prepare_impl<8>();
    case 9: return prepare_impl<9>();
    case 10: return prepare_impl<10>();
    case 11: return prepare_impl<11>();
    case 12: return prepare_impl<12>();
    case 13: return prepare_impl<13>();
    default: return cudaErrorInvalidValue;
  }
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
  modswitch_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, n, c->rc);
  return cudaGetLastError();
}

}  // namespace phe
