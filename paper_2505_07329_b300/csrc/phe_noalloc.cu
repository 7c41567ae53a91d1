// phe_matmul_noalloc: the per-call hot path without any device allocation.
//
// Some callers cannot allocate device memory while they serve requests: a
// process whose HBM is already owned by another allocator (for example a
// PyTorch caching allocator or an inference server that reserved a fixed
// budget at start-up), where a library allocation could fail or fragment
// that budget, and latency-critical loops that must not touch the CUDA
// allocator after start-up.  This entry point takes its only scratch buffer
// (the transformed input masks A_hat) from a fixed array in device memory
// instead of cudaMallocAsync.  The paper has no counterpart: this is an
// engineering variant of phe_matmul.
#include <cstdarg>
#include <cstdio>

#include "phe_host.hpp"

using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;

namespace {

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  In host code its name is a host-side stand-in, not a device
// address, so the host side only ever passes the address returned by
// cudaGetSymbolAddress to the kernels.
constexpr size_t kScratchWords = PHE_NOALLOC_MAX_SCRATCH_BYTES / sizeof(phe::u64);
static __device__ __align__(256) phe::u64 g_scratch[kScratchWords];

// Device address of the scratch array in the current context.  Once the
// array's module is loaded (phe_ctx_create loads it on its device), the
// lookup allocates nothing; asking every call, rather than caching the
// address, keeps it right after a device reset or under another context.
phe_status scratch_address(phe::u64** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return fail(PHE_ECUDA, "phe_matmul_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  *out = static_cast<phe::u64*>(p);
  return PHE_OK;
}

}  // namespace

extern "C" phe_status phe_matmul_noalloc(phe_ctx* c, const phe_weights* w, int dir, uint32_t T,
                                         const uint64_t* d_in_mask, const uint64_t* d_in_body, void* d_out_mask,
                                         void* d_out_body, uint32_t flags, void* stream) {
  if (!c || !w) return fail(PHE_EINVAL, "phe_matmul_noalloc: null handle");
  if (w->ctx != c) return fail(PHE_EINVAL, "phe_matmul_noalloc: weights belong to another context");
  if (dir != PHE_FWD && dir != PHE_BWD) return fail(PHE_EINVAL, "phe_matmul_noalloc: bad direction");
  if (!(w->dirs & (1u << dir))) return fail(PHE_EINVAL, "phe_matmul_noalloc: direction was not uploaded");
  if (flags != PHE_OUT_SWITCHED && flags != PHE_OUT_RAW) return fail(PHE_EINVAL, "phe_matmul_noalloc: bad flags");
  if (T == 0) return PHE_OK;
  if (!d_in_mask || !d_in_body || !d_out_mask || !d_out_body)
    return fail(PHE_EINVAL, "phe_matmul_noalloc: null buffer");
  const phe_weights::Dir& D = w->dir[dir];
  const size_t words = (size_t)T * D.L * c->prm.N;
  if (words > kScratchWords)
    return fail(PHE_EINVAL, "phe_matmul_noalloc: T*L*N*8 = %zu bytes exceeds the fixed scratch of %zu bytes",
                words * 8, (size_t)PHE_NOALLOC_MAX_SCRATCH_BYTES);

  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != c->device) e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(PHE_ECUDA, "phe_matmul_noalloc: cudaSetDevice: %s", cudaGetErrorString(e));
  phe::u64* ahat = nullptr;
  phe_status st = scratch_address(&ahat);
  if (st == PHE_OK) {
    cudaStream_t s = (cudaStream_t)stream;
    // The input transform overwrites every scratch word this call reads, so
    // nothing left by an earlier call needs clearing.
    phe::NttJob nj{reinterpret_cast<const phe::u64*>(d_in_mask), ahat, T * D.L};
    e = phe::launch_input_ntt(c, &nj, 1, s);
    if (e == cudaSuccess) {
      phe::LweJobTable jt{};
      jt.n = 1;
      phe::LweJob& J = jt.j[0];
      J.what = D.what;
      J.ahat = ahat;
      J.out = d_out_mask;
      J.wrow = D.wrow;
      J.bin = reinterpret_cast<const phe::u64*>(d_in_body);
      J.out_body = d_out_body;
      J.rows = D.rows;
      J.cols = D.cols;
      J.T = T;
      J.L = D.L;
      J.tok_chunk = phe::kDefaultTokChunk;
      phe::set_lwe_tiles(J, c->logn);
      jt.prefix[1] = J.tiles;
      e = phe::launch_lwedot(c, jt, flags == PHE_OUT_RAW ? phe::kOutRaw : phe::kOutSwitched, 0, s);
    }
    if (e != cudaSuccess) st = fail(PHE_ECUDA, "phe_matmul_noalloc: launch: %s", cudaGetErrorString(e));
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return st;
}

namespace phe {
// Loads the scratch array's module on the current device (called by
// phe_ctx_create with the context's device current), so that the array's
// memory is reserved at set-up and no phe_matmul_noalloc call loads code or
// reserves memory itself.
cudaError_t noalloc_setup() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_scratch);
}
}  // namespace phe
