// Wire format (Sec. 4.4 sizes; Sec. 4.5: the result is "packed into a
// bit-vector"): records are little-endian bit streams of fixed-width fields,
// padded with zero bits to a multiple of 32.
//   input record   8-byte seed (little endian), then the N body coefficients
//                  at bits_q = ceil(log2 q) bits (Sec. 3.1: the client sends
//                  the seed and the body; N = 2048, q = 2^39: 9992 bytes)
//   LWE record     the N mask words then the body, at log2_qout bits
//   RLWE record    A then B (2N words) at log2_qout bits (N = 2048 at 26
//                  bits: 13312 bytes)
// Kernels: wire_pack_kernel (one thread per output word, gathering the
// fields that overlap it) and wire_unpack_kernel (one thread per field).
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "phe_host.hpp"

using phe::u32;
using phe::u64;
using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;

namespace phe {

// Records of fa fields from a (record r at a + r*fa) followed by fb fields
// from b (at b + r*fb), `bits` <= 32 wide, into wpr 32-bit words each.
__global__ void wire_pack_kernel(const u32* __restrict__ a, u32 fa, const u32* __restrict__ b, u32 fb,
                                 u64 n_records, u32 bits, u32 wpr, u32* __restrict__ out) {
  const u64 total = n_records * wpr;
  const u32 fields = fa + fb;
  const u64 mask = (bits == 32) ? 0xffffffffull : ((1ull << bits) - 1);
  for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (u64)gridDim.x * blockDim.x) {
    const u64 r = idx / wpr;
    const u32 w = (u32)(idx % wpr);
    const u64 lo = (u64)w * 32;
    const u32 f0 = (u32)(lo / bits);
    const u64 fe = (lo + 32 + bits - 1) / bits;
    const u32 f1 = (u32)(fe < fields ? fe : fields);
    u64 acc = 0;
    for (u32 f = f0; f < f1; ++f) {
      const u64 v = (u64)((f < fa) ? a[r * fa + f] : b[r * fb + (f - fa)]) & mask;
      const long long sh = (long long)f * bits - (long long)lo;  // in (-bits, 32)
      acc |= (sh >= 0) ? (v << sh) : (v >> (-sh));
    }
    out[idx] = (u32)acc;
  }
}

// Input records (2 seed words + wb body words each) -> seeds[r] and
// bodies[r*N + m] (fields of `bits` <= 64).
__global__ void wire_unpack_kernel(const u32* __restrict__ rec, u64 n_records, u32 N, u32 bits, u32 wb,
                                   u64* __restrict__ seeds, u64* __restrict__ bodies) {
  const u64 total = n_records * N;
  const u64 mask = (bits == 64) ? ~0ull : ((1ull << bits) - 1);
  for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (u64)gridDim.x * blockDim.x) {
    const u64 r = idx / N;
    const u32 m = (u32)(idx % N);
    const u32* R = rec + r * (2 + (u64)wb);
    if (m == 0) seeds[r] = (u64)R[0] | ((u64)R[1] << 32);
    const u64 o = (u64)m * bits;
    const u32 w0 = (u32)(o / 32), sh = (u32)(o % 32);
    const u32* B = R + 2;
    const u64 x0 = B[w0];
    const u64 x1 = (w0 + 1 < wb) ? B[w0 + 1] : 0;
    const u64 x2 = (w0 + 2 < wb) ? B[w0 + 2] : 0;
    const u64 lo = x0 | (x1 << 32);
    const u64 v = (lo >> sh) | (sh ? (x2 << (64 - sh)) : 0ull);  // sh + bits <= 95 bits: three words
    bodies[idx] = v & mask;
  }
}

}  // namespace phe

namespace {

using phe::Span;




u32 words_of(u64 fields, u32 bits) { return (u32)((fields * bits + 31) / 32); }

// bits of an input body word: ceil(log2 q) (K for q = 2^K)
u32 body_bits(const phe_ctx* c) {
  const u64 q = c->prm.q;
  u32 b = 0;
  while (b < 64 && ((q - 1) >> b)) ++b;
  return b;
}

unsigned grid_for(const phe_ctx* c, u64 work) {
  return (unsigned)std::max<u64>(1, std::min<u64>((work + 255) / 256, (u64)c->num_sms * 16));
}

cudaError_t pack_records(const phe_ctx* c, const u32* a, u32 fa, const u32* b, u32 fb, u64 n, void* out,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const u32 bits = c->prm.log2_qout, wpr = words_of(fa + fb, bits);
  phe::wire_pack_kernel<<<grid_for(c, n * wpr), 256, 0, s>>>(a, fa, b, fb, n, bits, wpr, static_cast<u32*>(out));
  return cudaGetLastError();
}

constexpr u64 kWireScratchBytes = 2ull << 30;

}  // namespace

extern "C" {

phe_status phe_wire_sizes(const phe_ctx* c, uint64_t* in_record, uint64_t* lwe_record, uint64_t* rlwe_record) {
  if (!c) return fail(PHE_EINVAL, "phe_wire_sizes: null context");
  const u32 N = c->prm.N, k = c->prm.log2_qout;
  if (in_record) *in_record = 8 + 4ull * words_of(N, body_bits(c));
  if (lwe_record) *lwe_record = 4ull * words_of(N + 1, k);
  if (rlwe_record) *rlwe_record = 4ull * words_of(2ull * N, k);
  return PHE_OK;
}

phe_status phe_wire_pack(phe_ctx* c, const uint32_t* d_a, uint32_t fa, const uint32_t* d_b, uint32_t fb,
                         uint64_t n_records, void* d_out, void* stream) {
  if (!c) return fail(PHE_EINVAL, "phe_wire_pack: null context");
  if (n_records == 0) return PHE_OK;
  if (fa + fb == 0 || (fa && !d_a) || (fb && !d_b) || !d_out) return fail(PHE_EINVAL, "phe_wire_pack: bad buffers");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = pack_records(c, d_a, fa, d_b, fb, n_records, d_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_wire_pack");
  return PHE_OK;
}

phe_status phe_wire_unpack_inputs(phe_ctx* c, const void* d_records, uint64_t n_records, uint64_t* d_seeds,
                                  uint64_t* d_bodies, void* stream) {
  if (!c) return fail(PHE_EINVAL, "phe_wire_unpack_inputs: null context");
  if (n_records == 0) return PHE_OK;
  if (!d_records || !d_seeds || !d_bodies) return fail(PHE_EINVAL, "phe_wire_unpack_inputs: null buffer");
  if (reinterpret_cast<uintptr_t>(d_records) % 4) return fail(PHE_EINVAL, "phe_wire_unpack_inputs: records not 4-byte aligned");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const u32 N = c->prm.N, bits = body_bits(c), wb = words_of(N, bits);
  phe::wire_unpack_kernel<<<grid_for(c, n_records * N), 256, 0, (cudaStream_t)stream>>>(
      static_cast<const u32*>(d_records), n_records, N, bits, wb, reinterpret_cast<u64*>(d_seeds),
      reinterpret_cast<u64*>(d_bodies));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "phe_wire_unpack_inputs");
  return PHE_OK;
}

phe_status phe_matmul_wire(phe_ctx* c, const phe_weights* w, const phe_ksk* k, int dir, uint32_t T,
                           const void* d_in_records, void* d_out_records, void* stream) {
  if (!c || !w || w->ctx != c) return fail(PHE_EINVAL, "phe_matmul_wire: null handle or weights of another context");
  uint32_t rows = 0, cols = 0, L = 0;
  phe_status st = phe_weights_shape(w, dir, &rows, &cols, &L);
  if (st != PHE_OK) return st;
  if (T == 0) return PHE_OK;
  if (!d_in_records || !d_out_records) return fail(PHE_EINVAL, "phe_matmul_wire: null buffer");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const u32 N = c->prm.N, G = (rows + N - 1) / N;
  uint64_t in_rec = 0, lwe_rec = 0, rlwe_rec = 0;
  phe_wire_sizes(c, &in_rec, &lwe_rec, &rlwe_rec);
  // per-token scratch: seeds and bodies, then the switched outputs (and, when
  // packing, the raw LWE outputs inside phe_pack's own scratch)
  const u64 in_tok = (u64)L * (N + 1) * 8;
  const u64 out_tok = k ? (u64)G * 2 * N * 4 : (u64)rows * (N + 1) * 4;
  const u32 per = (u32)std::max<u64>(1, std::min<u64>(T, kWireScratchBytes / (in_tok + out_tok)));
  char* scratch = nullptr;
  cudaError_t e = phe::ctx_malloc_async(c, &scratch, (size_t)per * (in_tok + out_tok), s);
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_wire: scratch");
  u64* seeds = reinterpret_cast<u64*>(scratch);
  u64* bodies = seeds + (size_t)per * L;
  char* outs = scratch + (size_t)per * in_tok;
  for (u32 t0 = 0; t0 < T && st == PHE_OK; t0 += per) {
    const u32 tn = std::min(per, T - t0);
    const char* rin = static_cast<const char*>(d_in_records) + (size_t)t0 * L * in_rec;
    st = phe_wire_unpack_inputs(c, rin, (u64)tn * L, reinterpret_cast<uint64_t*>(seeds),
                                reinterpret_cast<uint64_t*>(bodies), stream);
    if (st != PHE_OK) break;
    if (k) {
      u32* oa = reinterpret_cast<u32*>(outs);
      u32* ob = oa + (size_t)tn * G * N;
      st = phe_matmul_packed_seeded(c, w, k, dir, tn, reinterpret_cast<uint64_t*>(seeds),
                                    reinterpret_cast<uint64_t*>(bodies), oa, ob, PHE_OUT_SWITCHED, stream);
      if (st == PHE_OK) {
        // RLWE record g of token t: A then B of unit t*G + g
        e = pack_records(c, oa, N, ob, N, (u64)tn * G, static_cast<char*>(d_out_records) + (size_t)t0 * G * rlwe_rec,
                         s);
        if (e != cudaSuccess) st = cuda_fail(e, "phe_matmul_wire: pack");
      }
    } else {
      u32* om = reinterpret_cast<u32*>(outs);
      u32* ob = om + (size_t)tn * rows * N;
      st = phe_matmul_seeded(c, w, dir, tn, reinterpret_cast<uint64_t*>(seeds), reinterpret_cast<uint64_t*>(bodies),
                             om, ob, PHE_OUT_SWITCHED, stream);
      if (st == PHE_OK) {
        e = pack_records(c, om, N, ob, 1, (u64)tn * rows,
                         static_cast<char*>(d_out_records) + (size_t)t0 * rows * lwe_rec, s);
        if (e != cudaSuccess) st = cuda_fail(e, "phe_matmul_wire: pack");
      }
    }
  }
  e = cudaFreeAsync(scratch, s);
  if (st != PHE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_wire: free");
  return PHE_OK;
}

}  // extern "C"
