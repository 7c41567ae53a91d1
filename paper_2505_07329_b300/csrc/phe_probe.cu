// Peak probes: the denominators of the rooflines the benchmark reports,
// measured on the GPU that runs the hot path, in the same process.
//
//   * ALU: register-only Gentleman-Sande butterflies -- the same gs_bfly32 /
//     gs_bfly the inverse transforms use (Shoup products with Harvey's lazy
//     reduction) -- in independent chains, over a sweep of chains per thread
//     (4 to 16) and resident blocks per SM (2 to 8, one full wave), so that
//     neither dependency latency nor occupancy caps the rate; the best
//     configuration's rate is reported.  Nothing but butterflies is issued,
//     so this is the rate a transform kernel could reach if it did nothing
//     else.
//   * Tensor: back-to-back tcgen05.mma kind::f16 (bf16 in, fp32 accumulate,
//     M = 128, N = 256, K = 16) on shared-memory operands into tensor memory,
//     one CTA per SM -- the instruction shape of the body GEMM.
#include <cuda_bf16.h>

#include "phe_host.hpp"
#include "phe_tc.cuh"

namespace phe {

namespace {

// CHAINS independent butterfly chains per thread, NTW distinct twiddles
// shared round-robin by the chains (the transforms reuse a twiddle across
// 2^stage butterflies too), at MINB blocks of 256 threads per SM.
template <bool RNS, int CHAINS, int NTW, int MINB>
__global__ void __launch_bounds__(256, MINB) bfly_probe_kernel(u32 iters, const uint4* __restrict__ tw, u64 q,
                                                               u32 p1, u32 p2, u64* __restrict__ sink) {
  const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (RNS) {
    const Ring2x32 ring{p1, p2};
    uint2 X[CHAINS], Y[CHAINS];
    uint4 w[NTW];
#pragma unroll
    for (int c = 0; c < NTW; ++c) w[c] = __ldg(&tw[(tid + c) & 255]);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      X[c] = make_uint2((tid * 7u + c) % p1, (tid * 5u + c) % p2);
      Y[c] = make_uint2((tid * 3u + c) % p1, (tid * 11u + c) % p2);
    }
    for (u32 i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) ring.gs(X[c], Y[c], w[c % NTW]);
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc ^= ((u64)X[c].x << 32 | Y[c].x) ^ ((u64)X[c].y << 32 | Y[c].y);
    sink[tid] = acc;
  } else {
    const Ring64 ring{q, 4 * q};
    u64 X[CHAINS], Y[CHAINS];
    ulonglong2 w[NTW];
#pragma unroll
    for (int c = 0; c < NTW; ++c) {
      const uint4 t = __ldg(&tw[(tid + c) & 255]);
      w[c] = make_ulonglong2(((u64)t.y << 32 | t.x) % q, (u64)t.z << 32 | t.w);  // (w, floor(w 2^64 / q))
    }
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      X[c] = ((u64)tid * 7 + c) % q;
      Y[c] = ((u64)tid * 3 + c) % q;
    }
    for (u32 i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) ring.gs(X[c], Y[c], w[c % NTW]);
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc ^= X[c] ^ Y[c];
    sink[tid] = acc;
  }
}

constexpr u32 kTcCols = 256;
constexpr u32 kTcA = 128 * 64 * 2, kTcB = 256 * 64 * 2;
// more shared memory than the operands need, so that one CTA runs per SM
constexpr size_t kTcSmem = 160 * 1024;

__global__ void __launch_bounds__(128, 1) tc_probe_kernel(u32 iters, u32* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const u32 raw = smem_addr(sm);
  const u32 base = (raw + 1023u) & ~1023u;
  unsigned char* g = sm + (base - raw);
  const u32 sA = base, sB = base + kTcA, bar = sB + kTcB, slot = bar + 8;
  // operands: small bf16 integers (the digit range), any layout
  for (u32 i = threadIdx.x; i < (kTcA + kTcB) / 2; i += blockDim.x)
    reinterpret_cast<__nv_bfloat16*>(g)[i] = __float2bfloat16_rn((float)((int)((i * 37u + blockIdx.x) % 255u) - 127));
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor-core reads
  if (threadIdx.x < 32) {
    tmem_alloc(slot, kTcCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const u32 tmem = *reinterpret_cast<volatile u32*>(g + (slot - base));
  if (threadIdx.x == 0) {
    const u32 idesc = idesc_bf16_f32(128, 256);
    const u64 ad = sw128_kmajor_desc(sA), bd = sw128_kmajor_desc(sB);
    for (u32 i = 0; i < iters; ++i) {
#pragma unroll
      for (u32 k4 = 0; k4 < 4; ++k4) mma_bf16(tmem, ad + 2 * k4, bd + 2 * k4, idesc, (i | k4) != 0);
    }
    mma_commit(bar);
  }
  __syncthreads();
  if (!mbar_wait(bar, 0, 4 * kWaitLimitNs)) atomicOr(status, 16u);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

template <class F>
cudaError_t best_ms(F&& launch, int reps, float* best) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  *best = 1e30f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && r > 0 && ms < *best) *best = ms;  // the first run warms up
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

}  // namespace

}  // namespace phe

extern "C" {

phe_status phe_probe_alu(int device, int form, uint32_t iters, double* per_s) {
  using namespace phe;
  if (!per_s || (form != 0 && form != 1)) return fail(PHE_EINVAL, "phe_probe_alu: bad argument");
  if (iters == 0) iters = 4096;
  DeviceGuard g(device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  const u32 max_threads = (u32)sms * 8 * 256;
  uint4* tw = nullptr;
  u64* sink = nullptr;
  e = cudaMalloc(&tw, 256 * sizeof(uint4));
  if (e == cudaSuccess) e = cudaMalloc(&sink, max_threads * sizeof(u64));
  // twiddles (w, w') mod p1, p2: any w below p with its Shoup quotient
  const u32 p1 = 1073643521u, p2 = 1073692673u;
  const u64 q = 1152921504606830593ull;  // 2^60 - 2^14 + 1
  if (e == cudaSuccess) {
    uint4 h[256];
    for (u32 i = 0; i < 256; ++i) {
      const u32 a = (u32)((i * 2654435761u) % p1), b = (u32)((i * 40503u + 7u) % p2);
      h[i] = make_uint4(a, (u32)(((u64)a << 32) / p1), b, (u32)(((u64)b << 32) / p2));
      if (form == 1) {  // 64-bit form: w in (x, y) and floor(w 2^64 / q) in (z, w)
        const u64 w = ((u64)a << 30 ^ b) % q;
        const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
        h[i] = make_uint4((u32)w, (u32)(w >> 32), (u32)(wp >> 32), (u32)wp);
      }
    }
    e = cudaMemcpy(tw, h, sizeof(h), cudaMemcpyHostToDevice);
  }
  // Sweep (chains per thread, blocks per SM): the best rate is the peak.
  // Threads per launch: blocks per SM x 256 x SMs, one full wave.
  double best = 0.0;
  auto run = [&](auto kern, int chains, int minb) -> cudaError_t {
    const u32 blocks = (u32)sms * minb, threads = blocks * 256;
    float ms = 0.f;
    cudaError_t e2 = best_ms(
        [&] {
          kern<<<blocks, 256>>>(iters, tw, q, p1, p2, sink);
          return cudaGetLastError();
        },
        4, &ms);
    if (e2 == cudaSuccess) {
      // RNS form: two 32-bit butterflies per chain step; 64-bit form: one
      const double rate = (double)threads * chains * iters * (form == 0 ? 2.0 : 1.0) / (ms * 1e-3);
      if (rate > best) best = rate;
    }
    return e2;
  };
  if (e == cudaSuccess) {
    // (chains, twiddles, blocks per SM): every configuration fits its
    // register budget without spilling (ptxas -v)
    if (form == 0) {
      e = run(bfly_probe_kernel<true, 8, 8, 3>, 8, 3);
      if (e == cudaSuccess) e = run(bfly_probe_kernel<true, 10, 2, 3>, 10, 3);
      if (e == cudaSuccess) e = run(bfly_probe_kernel<true, 8, 4, 4>, 8, 4);
      if (e == cudaSuccess) e = run(bfly_probe_kernel<true, 6, 2, 5>, 6, 5);
      if (e == cudaSuccess) e = run(bfly_probe_kernel<true, 4, 2, 6>, 4, 6);
    } else {
      e = run(bfly_probe_kernel<false, 8, 4, 2>, 8, 2);
      if (e == cudaSuccess) e = run(bfly_probe_kernel<false, 6, 2, 3>, 6, 3);
      if (e == cudaSuccess) e = run(bfly_probe_kernel<false, 4, 4, 4>, 4, 4);
    }
  }
  cudaFree(tw);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "phe_probe_alu");
  *per_s = best;
  return PHE_OK;
}

phe_status phe_probe_tensor(int device, uint32_t iters, double* flops_per_s) {
  using namespace phe;
  if (!flops_per_s) return fail(PHE_EINVAL, "phe_probe_tensor: null argument");
  if (iters == 0) iters = 20000;
  DeviceGuard g(device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  u32* status = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(u32));
  if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(u32));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  float ms = 0.f;
  if (e == cudaSuccess)
    e = best_ms(
        [&] {
          tc_probe_kernel<<<sms, 128, kTcSmem>>>(iters, status);
          return cudaGetLastError();
        },
        4, &ms);
  u32 st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(u32), cudaMemcpyDeviceToHost);
  cudaFree(status);
  if (e != cudaSuccess) return cuda_fail(e, "phe_probe_tensor");
  if (st) return fail(PHE_ETIMEOUT, "phe_probe_tensor: an MMA wait timed out (status 0x%x)", st);
  *flops_per_s = (double)sms * iters * 4 * (2.0 * 128 * 256 * 16) / (ms * 1e-3);
  return PHE_OK;
}

phe_status phe_ctx_status(phe_ctx* c, uint32_t* flags, int clear) {
  using namespace phe;
  if (!c || !flags) return fail(PHE_EINVAL, "phe_ctx_status: null argument");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(flags, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(c->d_status, 0, sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail(e, "phe_ctx_status");
  return PHE_OK;
}

}  // extern "C"
