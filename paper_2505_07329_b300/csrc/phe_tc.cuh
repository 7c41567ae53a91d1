// Inline-PTX wrappers for the Blackwell tensor-core path (sm_103a):
// mbarriers, TMA tiled loads (cp.async.bulk.tensor), tensor-memory (TMEM)
// allocation, tcgen05.mma issue and commit, and tcgen05.ld read-back.
//
// Every wait on an mbarrier is bounded: mbar_wait() gives up after `limit_ns`
// of %globaltimer (and after a hard iteration cap), so a kernel whose async
// copy or MMA never completes reports an error instead of hanging the GPU.
#pragma once

#include <cstdint>

#include "phe_device.cuh"

namespace phe {

// Wait limit of every mbarrier wait (normal waits take microseconds).
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u64 global_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(u32 bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Makes barrier initialisation visible to the async proxy (TMA, tcgen05).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u32 bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u32 bar, u32 parity) {
  u32 ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// True once the phase with this parity has completed; false after the limit.
static __device__ __noinline__ bool mbar_wait(u32 bar, u32 parity, u64 limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const u64 t0 = global_ns();
  for (u32 i = 1; i < (1u << 28); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15) == 0 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// 2-D tiled TMA load into this CTA's shared memory; completes `bar`'s
// transaction count.  c0 is the innermost coordinate (elements).
__device__ __forceinline__ void tma_load_2d(u32 dst, const void* tmap, int c0, int c1, u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<u64>(tmap)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(tmap)) : "memory");
}

// Tensor memory: one warp allocates `ncols` columns (a power of two >= 32)
// and writes the base address to shared memory at `dst`.
__device__ __forceinline__ void tmem_alloc(u32 dst, u32 ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(u32 taddr, u32 ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzling: rows of 128 bytes (64 bf16), 8-row groups 1024
// bytes apart.  The tile base must be 1024-byte aligned.  Fields: start
// address >> 4 (bits 0-13), leading byte offset >> 4 (16-29, unused for
// swizzled K-major tiles), stride byte offset >> 4 (32-45), descriptor
// version 1 (46-47), swizzle mode 2 = 128 B (61-63).
__device__ __forceinline__ u64 sw128_kmajor_desc(u32 saddr) {
  u64 d = (u64)((saddr & 0x3ffffu) >> 4);
  d |= (u64)1 << 16;
  d |= (u64)(1024 >> 4) << 32;
  d |= (u64)1 << 46;
  d |= (u64)2 << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16 with bf16 A and B (both
// K-major) and an fp32 accumulator: D format (bits 4-5) = 1 (F32), A format
// (7-9) = 1 (BF16), B format (10-12) = 1 (BF16), N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr u32 idesc_bf16_f32(u32 M, u32 N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 step, issued by one thread.
__device__ __forceinline__ void mma_bf16(u32 d_tmem, u64 adesc, u64 bdesc, u32 idesc, u32 accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on `bar` once every tcgen05.mma this thread issued so far completes.
__device__ __forceinline__ void mma_commit(u32 bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 8 consecutive 32-bit TMEM columns of this thread's lane (warp w reads
// lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld8(u32 taddr, u32 (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace phe
