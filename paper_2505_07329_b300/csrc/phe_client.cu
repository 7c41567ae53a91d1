// Client-side helpers for tests and benchmarks: RLWE encryption of int8
// vectors (Sec. 3.1, blocks of Sec. 4.3.1) and a seeded secret key.  The
// server never holds the key (Sec. 5), so these calls are built only into the
// test library, libphe_test.so (-DPHE_TESTING); the production libphe.so
// exports nothing that takes a secret key.
#ifndef PHE_TESTING
#error "phe_client.cu belongs to the test library only: compile it with -DPHE_TESTING"
#endif
#include <cstdint>

#include "phe_host.hpp"

using phe::u32;
using phe::u64;
using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;

namespace {

// SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014): the generator of the test key.
u64 splitmix64(u64& state) {
  u64 z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

phe_status phe_test_keygen(phe_ctx* c, uint64_t seed, uint32_t kind, int8_t* h_sk) {
  if (!c || !h_sk) return fail(PHE_EINVAL, "phe_test_keygen: null argument");
  if (kind != PHE_KEY_BINARY && kind != PHE_KEY_TERNARY) return fail(PHE_EINVAL, "phe_test_keygen: kind=%u", kind);
  u64 st = seed;
  for (u32 m = 0; m < c->prm.N; ++m) {
    const u64 r = splitmix64(st);
    // ternary: floor(3 r / 2^64) in {0, 1, 2}, minus 1; binary: the top bit
    h_sk[m] = kind == PHE_KEY_TERNARY ? (int8_t)((int)(((unsigned __int128)r * 3) >> 64) - 1) : (int8_t)(r >> 63);
  }
  return PHE_OK;
}

phe_status phe_client_encrypt(phe_ctx* c, uint32_t T, uint32_t d, const uint64_t* d_A, const int8_t* d_S,
                              const int32_t* d_E, const int8_t* d_x, uint64_t delta, uint64_t* d_B, void* stream) {
  if (!c) return fail(PHE_EINVAL, "phe_client_encrypt: null context");
  if (c->pow2) return fail(PHE_EUNSUPPORTED, "phe_client_encrypt: no NTT mod q = 2^%u (encrypt on the client)",
                           c->rk.p2k);
  if (T == 0) return PHE_OK;
  if (d < 1 || d > 16384) return fail(PHE_EINVAL, "phe_client_encrypt: d=%u not in [1, 16384]", d);
  if (!d_A || !d_S || !d_E || !d_x || !d_B) return fail(PHE_EINVAL, "phe_client_encrypt: null buffer");
  if (delta >= c->prm.q) return fail(PHE_EINVAL, "phe_client_encrypt: delta must be < q");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const u32 N = c->prm.N;
  const u32 L = (d + N - 1) / N;
  const u32 blocks = T * L;
  u64* ahat = nullptr;
  ulonglong2* shat = nullptr;
  cudaError_t e = phe::ctx_malloc_async(c, &ahat, (size_t)blocks * N * sizeof(u64), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(A_hat)");
  e = phe::ctx_malloc_async(c, &shat, (size_t)N * sizeof(ulonglong2), s);
  if (e == cudaSuccess) {
    phe::NttJob nj{reinterpret_cast<const u64*>(d_A), ahat, blocks};
    e = phe::launch_input_ntt(c, &nj, 1, s, /*force64=*/true);
  }
  if (e == cudaSuccess) e = phe::launch_weight_ntt(c, d_S, 1, N, 0, 1, 1, 0, shat, s, /*force64=*/true);
  if (e == cudaSuccess) {
    phe::LweJobTable jt{};
    jt.n = 1;
    phe::LweJob& J = jt.j[0];
    J.what = shat;
    J.ahat = ahat;
    J.out = d_B;
    J.err = d_E;
    J.msg = d_x;
    J.delta = delta;
    J.delta_p = (u64)(((unsigned __int128)delta << 64) / c->prm.q);
    J.rows = 1;
    J.T = blocks;
    J.L = 1;
    J.tok_chunk = 16;
    J.msg_d = d;
    phe::set_lwe_tiles(J, c->logn);
    jt.prefix[1] = J.tiles;
    e = phe::launch_lwedot(c, jt, phe::kOutRing, 0, s, /*force64=*/true);
  }
  if (shat) cudaFreeAsync(shat, s);
  cudaFreeAsync(ahat, s);
  if (e != cudaSuccess) return cuda_fail(e, "phe_client_encrypt launch");
  return PHE_OK;
}

}  // extern "C"
