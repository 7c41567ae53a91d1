// CUDA kernels of the hot path (sm_103a):
//   input_ntt_kernel   forward negacyclic NTT of the input masks A_ti
//   weight_ntt_kernel  w_hat_ij (reversed weight blocks, Sec. 4.3.1) -> NTT domain, x N^-1
//   lwedot_kernel      Eq. (LWEdot) for the masks: pointwise sum over blocks,
//                      inverse NTT, SampleExtract at N-1 (index reversal),
//                      ModulusSwitch -- one fused pass per (token, row)
//   body_kernel        the bodies b'_tj = sum_k W[j,k] B_t[k] (mod q) + switch
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
  const u64* src = job.src + (size_t)(active ? b : 0) * S::N;
  u64 x[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) x[e] = active ? reduce_word(src[pass_pos<LOGN, NP - 1>(p, e)], rc) : 0ull;
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
// Eq. (LWEdot), masks.  A tile is (job, output row, chunk of tokens); the
// block walks the chunk SLOTS tokens at a time.
// --------------------------------------------------------------------------
template <int LOGN, int MODE>
__global__ void __launch_bounds__(Shape<LOGN>::TPB)
    lwedot_kernel(const LweJobTable jt, RingConst rc, const ulonglong2* __restrict__ tw0,
                  const ulonglong2* __restrict__ twc) {
  using S = Shape<LOGN>;
  constexpr int N = S::N;
  constexpr int P = S::P;
  constexpr int NP = S::NPASS;
  extern __shared__ u64 smem[];
  const int slot = threadIdx.x / P, p = threadIdx.x % P;
  u64* buf = smem + slot * S::PADN;
  const u64 q = rc.q, q2 = rc.q2;
  const u32 total = jt.prefix[jt.n];

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

    for (u32 it = 0; it < iters; ++it) {
      const u32 t = t0 + it * S::SLOTS + slot;
      const bool active = t < t1;
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
            u64 s0 = x[r] + mul_shoup(av.x, w0.x, w0.y, q);
            u64 s1 = x[r + 1] + mul_shoup(av.y, w1.x, w1.y, q);
            x[r] = (s0 >= q2) ? s0 - q2 : s0;
            x[r + 1] = (s1 >= q2) ? s1 - q2 : s1;
          }
        }
      }
      intt_regs<LOGN>(x, p, buf, tw0, twc, q, q2);
      if (active) {
        if constexpr (MODE == kOutSwitched) {
          uint32_t* out = reinterpret_cast<uint32_t*>(J.out) + ((size_t)t * J.rows + row) * N;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int pos = pass_pos<LOGN, NP - 1>(p, e);
            out[N - 1 - pos] = modswitch_word(reduce_2q(x[e], q), rc);
          }
        } else if constexpr (MODE == kOutRaw) {
          u64* out = reinterpret_cast<u64*>(J.out) + ((size_t)t * J.rows + row) * N;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int pos = pass_pos<LOGN, NP - 1>(p, e);
            out[N - 1 - pos] = reduce_2q(x[e], q);
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
            u64 v = reduce_2q(x[e], q);
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
      }
    }
  }
}

// --------------------------------------------------------------------------
// Bodies: b'_tj = sum_k W(j, k) B_t[k] (mod q), k < K (coefficient N-1 of the
// block products of Eq. (LWEdot) is the plain dot product over the blocks).
// Exact: B = Bh 2^30 + Bl with Bl < 2^30, Bh < 2^31; both partial sums are
// accumulated in int64 (|sum| < 2^14 * 2^7 * 2^31 = 2^52 < q) and recombined
// mod q.  Tile: 128 rows x 16 tokens per block of 256 threads; thread
// (tx, ty) owns rows j0+tx, j0+tx+64 and tokens t0+ty+4b (b < 4).
// --------------------------------------------------------------------------
constexpr int kBodyRows = 128, kBodyToks = 16, kBodyKC = 128;

template <int MODE>
__global__ void __launch_bounds__(256) body_kernel(const BodyJobTable jt, RingConst rc) {
  __shared__ int2 bs[kBodyToks][kBodyKC];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const u64 q = rc.q;
  const u32 total = jt.prefix[jt.n];
  for (u32 tile = blockIdx.x; tile < total; tile += gridDim.x) {
    u32 k = 0;
    while (tile >= jt.prefix[k + 1]) ++k;
    const BodyJob& J = jt.j[k];
    const u32 local = tile - jt.prefix[k];
    const u32 j0 = (local % J.tiles_r) * kBodyRows;
    const u32 t0 = (local / J.tiles_r) * kBodyToks;
    const u32 K4 = (J.K + 3) & ~3u;
    long long accl[2][4], acch[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) accl[a][b] = acch[a][b] = 0;

    for (u32 k0 = 0; k0 < K4; k0 += kBodyKC) {
      for (int idx = threadIdx.x; idx < kBodyToks * kBodyKC; idx += 256) {
        const int tt = idx / kBodyKC, kk = idx % kBodyKC;
        const u32 t = t0 + tt, kg = k0 + kk;
        const u64 v = (t < J.T && kg < J.K) ? reduce_word(J.B[(size_t)t * J.ldB + kg], rc) : 0ull;
        bs[tt][kk] = make_int2((int)(v & 0x3fffffffull), (int)(v >> 30));
      }
      __syncthreads();
      const u32 kmax = min((u32)kBodyKC, K4 - k0);
      for (u32 k4 = 0; k4 < kmax / 4; ++k4) {
        u32 wv[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const u32 j = j0 + tx + 64 * a;
          wv[a] = (j < J.R) ? __ldg(&J.wb[(size_t)(k0 / 4 + k4) * J.R + j]) : 0u;
        }
#pragma unroll
        for (int by = 0; by < 4; ++by) {
          int2 bv[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = bs[ty + 4 * b][4 * k4 + by];
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            const int w = (int)(signed char)(wv[a] >> (8 * by));
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              accl[a][b] += (long long)w * bv[b].x;
              acch[a][b] += (long long)w * bv[b].y;
            }
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const u32 j = j0 + tx + 64 * a, t = t0 + ty + 4 * b;
        if (j < J.R && t < J.T) {
          const long long hl = acch[a][b], ll = accl[a][b];
          const u64 vh = (hl < 0) ? q - (u64)(-hl) : (u64)hl;
          const u64 vl = (ll < 0) ? q - (u64)(-ll) : (u64)ll;
          u64 v = reduce_2q(mul_shoup(vh, rc.c30, rc.c30p, q), q) + vl;
          v = reduce_2q(v, q);
          if constexpr (MODE == kOutSwitched) {
            reinterpret_cast<uint32_t*>(J.out)[(size_t)t * J.R + j] = modswitch_word(v, rc);
          } else {
            reinterpret_cast<u64*>(J.out)[(size_t)t * J.R + j] = v;
          }
        }
      }
    }
  }
}

__global__ void modswitch_kernel(const u64* __restrict__ in, uint32_t* __restrict__ out, size_t n, RingConst rc) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = modswitch_word(reduce_word(in[i], rc), rc);
}

// Packed weights for the body product: wb[(k/4) R + j] holds W(j, k..k+3).
__global__ void pack_body_weights_kernel(const int8_t* __restrict__ W, u32 R, u32 K, u32 rs, u32 cs,
                                         uint32_t* __restrict__ wb) {
  const u32 K4 = (K + 3) / 4;
  const size_t n = (size_t)K4 * R;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const u32 j = (u32)(idx % R), k4 = (u32)(idx / R);
    u32 word = 0;
    for (int by = 0; by < 4; ++by) {
      const u32 k = 4 * k4 + by;
      const u32 v = (k < K) ? (u32)(uint8_t)W[(size_t)j * rs + (size_t)k * cs] : 0u;
      word |= v << (8 * by);
    }
    wb[idx] = word;
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

cudaError_t launch_body(const phe_ctx* c, const BodyJobTable& jt, int mode, cudaStream_t s) {
  const u32 total = jt.prefix[jt.n];
  if (total == 0) return cudaSuccess;
  if (mode == kOutSwitched) body_kernel<kOutSwitched><<<total, 256, 0, s>>>(jt, c->rc);
  else body_kernel<kOutRaw><<<total, 256, 0, s>>>(jt, c->rc);
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

cudaError_t launch_pack_body_weights(const int8_t* W, u32 R, u32 K, u32 rs, u32 cs, uint32_t* wb, cudaStream_t s) {
  const size_t n = (size_t)((K + 3) / 4) * R;
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  pack_body_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(W, R, K, rs, cs, wb);
  return cudaGetLastError();
}

}  // namespace phe
