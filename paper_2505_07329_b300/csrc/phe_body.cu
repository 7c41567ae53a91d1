// The body part of Eq. (LWEdot) on the tensor cores (sm_103a, tcgen05).
//
// For token t and output row j the LWE body is b'_tj = sum_k W[j,k] B_t[k]
// (mod q): coefficient N-1 of sum_i B_ti * w_hat_ij, written out as a dot
// product (Sec. 3.2 SampleExtract at h = N-1, Sec. 4.3.1).  Over a batch of
// tokens that is a dense integer GEMM, [rows x cols] int8 weights times
// [cols x T] words mod q, and it runs here as an exact limb GEMM:
//
//   * every body word, reduced mod q, is cut into 8 balanced base-256 digits
//     beta_l in [-128, 128) with B = sum_l beta_l 2^(8l) (the top digit takes
//     the last carry and stays below 2^6);
//   * W (|w| <= 127) and the digits are bf16 -- both exact -- and
//     tcgen05.mma kind::f16 multiplies them with fp32 accumulation in tensor
//     memory.  |w beta| <= 127 * 128, so every partial sum over a chunk of
//     1024 columns stays below 2^24 in magnitude, where fp32 represents every
//     integer: each chunk's accumulator is exact whatever the summation order;
//   * the epilogue converts each chunk's accumulator to an integer, sums the
//     chunks, recombines sum_l acc_l 2^(8l) mod q exactly and applies the
//     ModulusSwitch (Sec. 3.2).
//
// (The int8 tensor-core kind, tcgen05.mma kind::i8, is not accepted by ptxas
// for sm_103a; bf16 digits are the exact form available there.)
//
// Operand tiles are staged by TMA (cp.async.bulk.tensor, 128-byte swizzle)
// into a 4-stage shared-memory ring; one thread issues the loads, one thread
// issues the MMAs (M = 128 rows, N = 8 x tokens, K = 16 per instruction), and
// four warps read tensor memory back in the epilogue.  Every wait is bounded
// (phe_tc.cuh): on a time-out the kernel records an error bit in the
// context's status word, lets its in-flight copies and MMAs finish, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "phe_host.hpp"
#include "phe_tc.cuh"

namespace phe {

namespace {

constexpr int kBM = 128;               // rows per tile (MMA M)
constexpr int kBK = 64;                // columns per stage: one 128-byte swizzle row of bf16
constexpr int kStages = 4;
constexpr int kMaxBN = 256;            // MMA N: 8 digit rows per token
constexpr int kChunkBlocks = kBodyChunk / kBK;  // stages per exact fp32 chunk
constexpr u32 kStageA = kBM * kBK * 2;          // 16 KB
constexpr u32 kStageB = kMaxBN * kBK * 2;       // 32 KB
constexpr u32 kTmemCols = 512;
constexpr size_t kBodySmem = 1024 + (size_t)kStages * (kStageA + kStageB) + 256;

// Status bits written to the context's status word.
constexpr u32 kErrLoad = 1u, kErrMma = 2u, kErrEpilogue = 4u, kErrDrain = 8u;

struct BodyJob {
  CUtensorMap tmA;  // W as bf16, dims {cols, rows}, box {64, 128}
  CUtensorMap tmB;  // digit rows, dims {cols, T*8}, box {64, bn}
  void* out;        // [T][rows], u32 switched or u64 raw
  u32 rows, T, nk, bn, tok_tiles;
};
struct BodyTable {
  u32 n;
  u32 prefix[kMaxJobs + 1];
  BodyJob j[kMaxJobs];
};

__device__ __forceinline__ unsigned short bf16_bits(int v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
}

}  // namespace

// int8 weight rows [rows][cols] -> bf16 rows [rows][pitch] (zero past cols).
__global__ void weights_bf16_kernel(const int8_t* __restrict__ W, u32 rows, u32 cols, u32 pitch,
                                    unsigned short* __restrict__ out) {
  const size_t n = (size_t)rows * pitch;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const u32 r = (u32)(i / pitch), k = (u32)(i % pitch);
    out[i] = bf16_bits(k < cols ? (int)W[(size_t)r * cols + k] : 0);
  }
}

// Bodies [T][tok_words] (the first `cols` words of each token) -> balanced
// base-256 digits as bf16, digit row t*8+l, [T*8][pitch], zero past cols.
// Each thread takes 4 adjacent columns of one token and writes 8 bytes per
// digit row.
template <bool P2>
__global__ void body_digits_kernel(const u64* __restrict__ bin, u32 tok_words, u32 T, u32 cols, u32 pitch,
                                   unsigned short* __restrict__ dig, RingConst rc) {
  const u32 groups = pitch / 4;
  const size_t n = (size_t)T * groups;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const u32 t = (u32)(i / groups), k0 = 4 * (u32)(i % groups);
    const u64* bt = bin + (size_t)t * tok_words;
    unsigned short d[8][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const u32 k = k0 + c;
      u64 v = 0;
      if (k < cols) v = P2 ? (__ldg(&bt[k]) & (rc.q - 1)) : reduce_word(__ldg(&bt[k]), rc);
#pragma unroll
      for (int l = 0; l < 7; ++l) {
        int x = (int)(v & 255u);
        v >>= 8;
        if (x >= 128) {
          x -= 256;
          v += 1;
        }
        d[l][c] = bf16_bits(x);
      }
      d[7][c] = bf16_bits((int)v);  // v < 2^62 / 2^56 + 1
    }
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      uint2 w;
      w.x = (u32)d[l][0] | ((u32)d[l][1] << 16);
      w.y = (u32)d[l][2] | ((u32)d[l][3] << 16);
      *reinterpret_cast<uint2*>(dig + ((size_t)t * 8 + l) * pitch + k0) = w;
    }
  }
}

// One tile: 128 output rows x (bn / 8) tokens of one job.
template <bool P2, bool RAW>
__global__ void __launch_bounds__(128, 1)
    body_gemm_kernel(const __grid_constant__ BodyTable bt, const RingConst rc, const RnsConst rk, u32* status) {
  extern __shared__ __align__(1024) unsigned char body_smem[];
  const u32 raw = smem_addr(body_smem);
  const u32 base = (raw + 1023u) & ~1023u;
  const u32 sA = base, sB = base + kStages * kStageA;
  const u32 bars = sB + kStages * kStageB;
  const u32 done_bar = bars + 16 * kStages;
  const u32 tmem_slot = done_bar + 8;
  volatile u32* abort_flag = reinterpret_cast<volatile u32*>(body_smem + (tmem_slot + 4 - raw));
  auto full = [&](u32 s) { return bars + 8 * s; };
  auto empty = [&](u32 s) { return bars + 8 * (kStages + s); };

  u32 k = 0;
  while (blockIdx.x >= bt.prefix[k + 1]) ++k;
  const BodyJob& J = bt.j[k];
  const u32 local = blockIdx.x - bt.prefix[k];
  const u32 row0 = (local / J.tok_tiles) * kBM;
  const u32 tt = J.bn / 8;
  const u32 tok0 = (local % J.tok_tiles) * tt;
  const u32 warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (u32 s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
    tma_prefetch_desc(&J.tmA);
    tma_prefetch_desc(&J.tmB);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const u32 tmem = *reinterpret_cast<volatile u32*>(body_smem + (tmem_slot - raw));
  const u32 stage_bytes = kStageA + J.bn * (kBK * 2);

  if (warp == 0 && lane == 0) {
    // producer: W rows row0.., digit rows tok0*8.., 64 columns per stage
    u32 issued = 0;
    for (u32 kb = 0; kb < J.nk; ++kb) {
      const u32 s = kb % kStages;
      if (!mbar_wait(empty(s), ((kb / kStages) & 1) ^ 1)) {
        *abort_flag = 1;
        atomicOr(status, kErrLoad);
        break;
      }
      mbar_expect_tx(full(s), stage_bytes);
      tma_load_2d(sA + s * kStageA, &J.tmA, (int)(kb * kBK), (int)row0, full(s));
      tma_load_2d(sB + s * kStageB, &J.tmB, (int)(kb * kBK), (int)(tok0 * 8), full(s));
      issued = kb + 1;
    }
    // every issued copy has landed before the CTA may exit
    for (u32 kb = issued > (u32)kStages ? issued - kStages : 0; kb < issued; ++kb) {
      if (!mbar_wait(full(kb % kStages), (kb / kStages) & 1)) {
        *abort_flag = 1;
        atomicOr(status, kErrDrain);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: chunk c of kChunkBlocks stages accumulates into columns
    // [c*bn, (c+1)*bn) of tensor memory, exact in fp32
    const u32 idesc = idesc_bf16_f32(kBM, J.bn);
    for (u32 kb = 0; kb < J.nk; ++kb) {
      const u32 s = kb % kStages;
      if (!mbar_wait(full(s), (kb / kStages) & 1)) {
        *abort_flag = 1;
        atomicOr(status, kErrMma);
        break;
      }
      tc_fence_after();
      const u32 d = tmem + (kb / kChunkBlocks) * J.bn;
      const u64 ad = sw128_kmajor_desc(sA + s * kStageA), bd = sw128_kmajor_desc(sB + s * kStageB);
#pragma unroll
      for (u32 k4 = 0; k4 < kBK / 16; ++k4)  // 32 bytes of K per step inside the swizzle row
        mma_bf16(d, ad + 2 * k4, bd + 2 * k4, idesc, (kb % kChunkBlocks) | k4);
      mma_commit(empty(s));
    }
    mma_commit(done_bar);  // arrives when every MMA above has completed
  }
  __syncthreads();
  const bool ok_self = mbar_wait(done_bar, 0);
  if (!ok_self) atomicOr(status, kErrEpilogue);
  // tcgen05.ld is warp-collective: a warp reads tensor memory only if every
  // one of its threads saw the MMAs complete
  const bool ok = __all_sync(0xffffffffu, ok_self);
  tc_fence_after();
  if (ok && !*abort_flag) {
    // epilogue: thread = row row0 + threadIdx.x (tensor-memory lane)
    const u32 row = row0 + threadIdx.x;
    const u32 nch = (J.nk + kChunkBlocks - 1) / kChunkBlocks;
    const u32 ntok = (J.T - tok0 < tt) ? J.T - tok0 : tt;  // warp-uniform
    const u32 lane_base = tmem + ((warp * 32) << 16);
    for (u32 i = 0; i < ntok; ++i) {
      int a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (u32 c = 0; c < nch; ++c) {
        u32 r[8];
        tmem_ld8(lane_base + c * J.bn + i * 8, r);
        tmem_wait_ld();
#pragma unroll
        for (int l = 0; l < 8; ++l) a[l] += __float2int_rn(__uint_as_float(r[l]));
      }
      if (row < J.rows) {
        // |a_l| < 16 2^24, so each half is below 2^53 < q
        const long long lo = (long long)a[0] + ((long long)a[1] << 8) + ((long long)a[2] << 16) + ((long long)a[3] << 24);
        const long long hi = (long long)a[4] + ((long long)a[5] << 8) + ((long long)a[6] << 16) + ((long long)a[7] << 24);
        const size_t o = (size_t)(tok0 + i) * J.rows + row;
        if constexpr (P2) {
          const u64 v = ((u64)lo + ((u64)hi << 32)) & (rc.q - 1);  // exact mod q = 2^k
          if constexpr (RAW) reinterpret_cast<u64*>(J.out)[o] = v;
          else reinterpret_cast<u32*>(J.out)[o] = pow2_modswitch(v, rk);
        } else {
          const u64 q = rc.q;
          const u64 v0 = lo < 0 ? q - (u64)(-lo) : (u64)lo;
          const u64 v1 = hi < 0 ? q - (u64)(-hi) : (u64)hi;
          const u64 v = reduce_2q(v0 + reduce_2q(mul_shoup(v1, rc.c32, rc.c32p, q), q), q);
          if constexpr (RAW) reinterpret_cast<u64*>(J.out)[o] = v;
          else reinterpret_cast<u32*>(J.out)[o] = modswitch_word(v, rc);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// bf16 matrix [outer][pitch] (inner extent `inner` <= pitch), box {64, box_outer}.
cudaError_t encode_bf16_2d(CUtensorMap* m, const void* base, u64 inner, u64 outer, u32 pitch, u32 box_outer) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, box_outer};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// MMA N for a job: 8 digit rows per token, at most 256, and nch chunk
// accumulators of bn columns each within the 512 tensor-memory columns.
u32 body_bn(u32 cols, u32 T) {
  const u32 nch = (cols + kBodyChunk - 1) / kBodyChunk;
  u32 bn = kTmemCols / nch;
  if (bn > (u32)kMaxBN) bn = kMaxBN;
  bn &= ~15u;
  const u32 need = ((T * 8) + 15) & ~15u;
  return need < bn ? need : bn;
}

unsigned grid_for(size_t work, int num_sms) {
  size_t b = (work + 255) / 256;
  const size_t cap = (size_t)num_sms * 16;
  if (b > cap) b = cap;
  return (unsigned)(b ? b : 1);
}

}  // namespace

cudaError_t launch_weights_bf16(const phe_ctx* c, const int8_t* W, u32 rows, u32 cols, void* out, cudaStream_t s) {
  weights_bf16_kernel<<<grid_for((size_t)rows * digit_pitch(cols), c->num_sms), 256, 0, s>>>(
      W, rows, cols, digit_pitch(cols), static_cast<unsigned short*>(out));
  return cudaGetLastError();
}

size_t body_scratch_bytes(const LweJobTable& jt) {
  size_t total = 0;
  for (u32 i = 0; i < jt.n; ++i) {
    bool dup = false;
    for (u32 k = 0; k < i && !dup; ++k)
      dup = jt.j[k].bin == jt.j[i].bin && jt.j[k].T == jt.j[i].T && jt.j[k].cols == jt.j[i].cols;
    if (!dup) total += (digit_bytes(jt.j[i].T, jt.j[i].cols) + 255) & ~(size_t)255;
  }
  return total;
}

cudaError_t assign_body_scratch(LweJobTable& jt, void* scratch) {
  char* p = static_cast<char*>(scratch);
  for (u32 i = 0; i < jt.n; ++i) {
    LweJob& J = jt.j[i];
    J.digits = nullptr;
    for (u32 k = 0; k < i; ++k)
      if (jt.j[k].bin == J.bin && jt.j[k].T == J.T && jt.j[k].cols == J.cols) J.digits = jt.j[k].digits;
    if (!J.digits) {
      J.digits = p;
      J.digits_owner = 1;
      p += (digit_bytes(J.T, J.cols) + 255) & ~(size_t)255;
    } else {
      J.digits_owner = 0;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_body(const phe_ctx* c, const LweJobTable& jt, bool raw, const RingConst& rc, const RnsConst& rk,
                        cudaStream_t s) {
  // 1. digit rows of every distinct body input
  for (u32 i = 0; i < jt.n; ++i) {
    const LweJob& J = jt.j[i];
    if (!J.digits_owner || J.T == 0) continue;
    const u32 pitch = digit_pitch(J.cols);
    const unsigned g = grid_for((size_t)J.T * (pitch / 4), c->num_sms);
    if (c->pow2)
      body_digits_kernel<true><<<g, 256, 0, s>>>(J.bin, J.L * c->prm.N, J.T, J.cols, pitch,
                                                 static_cast<unsigned short*>(J.digits), rc);
    else
      body_digits_kernel<false><<<g, 256, 0, s>>>(J.bin, J.L * c->prm.N, J.T, J.cols, pitch,
                                                  static_cast<unsigned short*>(J.digits), rc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // 2. the GEMM over every job's tiles
  BodyTable* bt = new (std::nothrow) BodyTable();
  if (!bt) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaSuccess;
  bt->prefix[0] = 0;
  for (u32 i = 0; i < jt.n && e == cudaSuccess; ++i) {
    const LweJob& J = jt.j[i];
    if (J.T == 0) continue;
    BodyJob& B = bt->j[bt->n];
    const u32 pitch = digit_pitch(J.cols);
    B.rows = J.rows;
    B.T = J.T;
    B.nk = (J.cols + kBK - 1) / kBK;
    B.bn = body_bn(J.cols, J.T);
    B.tok_tiles = (J.T + B.bn / 8 - 1) / (B.bn / 8);
    B.out = J.out_body;
    e = encode_bf16_2d(&B.tmA, J.wbf, J.cols, J.rows, pitch, kBM);
    if (e == cudaSuccess) e = encode_bf16_2d(&B.tmB, J.digits, J.cols, (u64)J.T * 8, pitch, B.bn);
    const u32 tiles = ((J.rows + kBM - 1) / kBM) * B.tok_tiles;
    bt->prefix[bt->n + 1] = bt->prefix[bt->n] + tiles;
    bt->n++;
  }
  if (e == cudaSuccess && bt->n) {
    const u32 grid = bt->prefix[bt->n];
    auto launch = [&](auto kern) -> cudaError_t {
      cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBodySmem);
      if (e2 != cudaSuccess) return e2;
      kern<<<grid, 128, kBodySmem, s>>>(*bt, rc, rk, c->d_status);
      return cudaGetLastError();
    };
    if (c->pow2) e = raw ? launch(body_gemm_kernel<true, true>) : launch(body_gemm_kernel<true, false>);
    else e = raw ? launch(body_gemm_kernel<false, true>) : launch(body_gemm_kernel<false, false>);
  }
  delete bt;
  return e;
}

cudaError_t prepare_body_launches() {
  cudaError_t e = cudaFuncSetAttribute(body_gemm_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBodySmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(body_gemm_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBodySmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(body_gemm_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBodySmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(body_gemm_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBodySmem);
  return e;
}

}  // namespace phe
