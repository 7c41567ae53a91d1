// C ABI of libphe (include/phe.h): parameter validation, twiddle tables,
// weight upload and the per-call hot path.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "phe_host.hpp"

using phe::u32;
using phe::u64;
using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;
typedef unsigned __int128 u128;

namespace {

thread_local std::string g_err;

// --- host modular arithmetic (parameter set-up only) ---------------------
u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
u64 powmod(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  for (; e; e >>= 1) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
  }
  return r;
}
// Miller-Rabin with the first twelve prime bases: exact for n < 3.3e24.
bool is_prime(u64 n) {
  const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : bases) {
    if (n % p == 0) return n == p;
  }
  u64 d = n - 1;
  int r = 0;
  while (!(d & 1)) { d >>= 1; ++r; }
  for (u64 a : bases) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int i = 1; i < r && witness; ++i) {
      x = mulmod(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}
u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
u32 shoup32(u32 w, u32 p) { return (u32)(((u64)w << 32) / p); }

// a^-1 mod m for gcd(a, m) = 1, by the extended Euclidean algorithm (m need
// not be prime).
u64 modinv(u64 a, u64 m) {
  __int128 t = 0, nt = 1, r = m, nr = a % m;
  while (nr != 0) {
    const __int128 qq = r / nr;
    __int128 tmp = t - qq * nt;
    t = nt;
    nt = tmp;
    tmp = r - qq * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += m;
  return (u64)t;
}

// The x mod p1 p2 with x = a (mod p1), x = b (mod p2).
u64 crt2(u64 a, u64 p1, u64 b, u64 p2) {
  const u64 h = mulmod((b + p2 - a % p2) % p2, modinv(p1 % p2, p2), p2);
  return a + p1 * h;
}
u32 bitrev(u32 x, int bits) {
  u32 r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}
int floor_log2(u64 x) { return 63 - __builtin_clzll(x); }

// Primitive 2N-th root of unity: the smallest g^((q-1)/2N) with order 2N,
// trying odd g from 3 upward.
u64 primitive_root_2n(u64 q, u32 N) {
  const u64 e = (q - 1) / (2ull * N);
  for (u64 g = 3; g < (1u << 20); g += 2) {
    const u64 psi = powmod(g, e, q);
    if (powmod(psi, N, q) == q - 1) return psi;
  }
  return 0;
}

phe_status upload(void** dptr, const void* host, size_t bytes);

// Compact and pass-0 tables (forward and inverse) from entry(brv(k), inverse).
// Pass-0 twiddles in thread-major order: slot (st, b) of thread p is the
// twiddle of stage st for butterfly group b of positions [16p, 16p+16).
template <class F>
phe_status build_tables(const phe_ctx* c, F entry, phe::Tables& tab) {
  const u32 N = c->prm.N;
  const int logn = c->logn;
  std::vector<ulonglong2> fwd(N), inv(N);
  for (u32 k = 0; k < N; ++k) {
    const u32 br = bitrev(k, logn);
    fwd[k] = entry(br, false);
    inv[k] = entry(br, true);
  }
  const u32 P = N / 16;
  std::vector<ulonglong2> fwd0(15 * P), inv0(15 * P);
  for (int st = 0; st < 4; ++st) {
    for (int b = 0; b < (8 >> st); ++b) {
      for (u32 p = 0; p < P; ++p) {
        const u32 idx = (N >> (st + 1)) + ((16 * p) >> (st + 1)) + b;
        fwd0[phe::pass0_slot(st, b) * P + p] = fwd[idx];
        inv0[phe::pass0_slot(st, b) * P + p] = inv[idx];
      }
    }
  }
  phe_status st;
  if ((st = upload((void**)&tab.fwd_c, fwd.data(), N * sizeof(ulonglong2))) != PHE_OK ||
      (st = upload((void**)&tab.inv_c, inv.data(), N * sizeof(ulonglong2))) != PHE_OK ||
      (st = upload((void**)&tab.fwd_0, fwd0.data(), fwd0.size() * sizeof(ulonglong2))) != PHE_OK ||
      (st = upload((void**)&tab.inv_0, inv0.data(), inv0.size() * sizeof(ulonglong2))) != PHE_OK)
    return st;
  return PHE_OK;
}

phe_status upload(void** dptr, const void* host, size_t bytes) {
  cudaError_t e = cudaMalloc(dptr, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tables)");
  e = cudaMemcpy(*dptr, host, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(tables)");
  return PHE_OK;
}

void free_tables(phe::Tables& t) {
  cudaFree(t.fwd_c);
  cudaFree(t.inv_c);
  cudaFree(t.fwd_0);
  cudaFree(t.inv_0);
  t = phe::Tables{};
}

phe_status check_dir(const phe_weights* w, int dir) {
  if (dir != PHE_FWD && dir != PHE_BWD) return fail(PHE_EINVAL, "direction %d is not PHE_FWD or PHE_BWD", dir);
  if (!(w->dirs & (1u << dir)))
    return fail(PHE_EINVAL, "direction %s was not uploaded", dir == PHE_FWD ? "PHE_FWD" : "PHE_BWD");
  return PHE_OK;
}

using phe::Span;

// The device form of the hot path for one projection.
cudaError_t matmul_device(phe_ctx* c, const phe_weights::Dir& D, u32 T, const u64* in_mask, const u64* in_body,
                          void* out_mask, void* out_body, int mode, cudaStream_t s, const u64* in_seeds = nullptr) {
  const u32 N = c->prm.N;
  Span call(c, phe::kKCall, s);
  phe::LweJobTable jt{};
  jt.n = 1;
  phe::LweJob& J = jt.j[0];
  J.what = D.what;
  J.out = out_mask;
  J.wrow = D.wrow;
  J.wbf = D.wbf;
  J.bin = in_body;
  J.out_body = out_body;
  J.rows = D.rows;
  J.cols = D.cols;
  J.T = T;
  J.L = D.L;
  J.tok_chunk = phe::kDefaultTokChunk;
  phe::set_lwe_tiles(J, c->logn);
  jt.prefix[0] = 0;
  jt.prefix[1] = J.tiles;
  // one scratch allocation: A_hat, then (bodies on the tensor cores) the
  // bodies' digit rows
  const bool gemm = phe::body_on_tensor_cores(c, jt);
  const size_t ahat_bytes = ((size_t)T * D.L * N * sizeof(u64) + 255) & ~(size_t)255;
  char* scratch = nullptr;
  cudaError_t e =
      phe::ctx_malloc_async(c, &scratch, ahat_bytes + (gemm ? phe::body_scratch_bytes(jt) : 0), s);
  if (e != cudaSuccess) return e;
  u64* ahat = reinterpret_cast<u64*>(scratch);
  J.ahat = ahat;
  if (gemm) phe::assign_body_scratch(jt, scratch + ahat_bytes);
  {
    Span sp(c, phe::kKInputNtt, s);
    phe::NttJob nj{in_mask, ahat, T * D.L, in_seeds};
    e = phe::launch_input_ntt(c, &nj, 1, s);
  }
  if (e == cudaSuccess && gemm) {
    Span sp(c, phe::kKBodyGemm, s);
    e = phe::launch_body(c, jt, mode == phe::kOutRaw, c->rc, c->rk, s);
  }
  if (e == cudaSuccess) {
    Span sp(c, phe::kKLwedot, s);
    e = phe::launch_lwedot(c, jt, mode | (gemm ? phe::kBodyGemm : 0), 0, s);
  }
  cudaError_t ef = cudaFreeAsync(scratch, s);
  return e != cudaSuccess ? e : ef;
}

phe_status check_matmul_args(phe_ctx* c, const phe_weights* w, int dir, uint32_t flags) {
  if (!c || !w) return fail(PHE_EINVAL, "phe_matmul: null handle");
  if (w->ctx != c) return fail(PHE_EINVAL, "phe_matmul: weights belong to another context");
  phe_status st = check_dir(w, dir);
  if (st != PHE_OK) return st;
  if (flags != PHE_OUT_SWITCHED && flags != PHE_OUT_RAW) return fail(PHE_EINVAL, "phe_matmul: flags=%u", flags);
  return PHE_OK;
}

}  // namespace

namespace phe {
void set_last_error(const char* msg) { g_err = msg; }

phe_status fail(phe_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

phe_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(PHE_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(PHE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void set_switch_target(RnsConst& k, u32 log2_target) {
  const u32 p1 = k.p1, p2 = k.p2;
  const u64 two_k = 1ull << log2_target;
  k.a1 = (u32)(two_k / p1);
  k.b1 = (u32)(two_k % p1);
  k.b1p = shoup32(k.b1, p1);
  k.s2 = 0;
  while ((p2 >> k.s2) != 0) ++k.s2;
  k.mu2 = (u32)(((1ull << (32 + k.s2)) / p2) - (1ull << 32));  // p2 < 2^30
  k.half1 = (p1 - 1) / 2;
  k.half2 = (p2 - 1) / 2;
  k.kbits = log2_target;
  k.kmask = (u32)(two_k - 1);
}
}  // namespace phe

extern "C" {

const char* phe_status_string(phe_status s) {
  switch (s) {
    case PHE_OK: return "PHE_OK";
    case PHE_EINVAL: return "PHE_EINVAL";
    case PHE_ENOMEM: return "PHE_ENOMEM";
    case PHE_EBUSY: return "PHE_EBUSY";
    case PHE_ETIMEOUT: return "PHE_ETIMEOUT";
    case PHE_ECUDA: return "PHE_ECUDA";
    case PHE_EUNSUPPORTED: return "PHE_EUNSUPPORTED";
  }
  return "PHE_UNKNOWN";
}

const char* phe_last_error(void) { return g_err.c_str(); }

phe_status phe_ctx_create(const phe_params* prm, int device, phe_ctx** out) {
  if (!prm || !out) return fail(PHE_EINVAL, "phe_ctx_create: null argument");
  *out = nullptr;
  const u32 N = prm->N;
  if (N < (1u << phe::kMinLogN) || N > (1u << phe::kMaxLogN) || (N & (N - 1)))
    return fail(PHE_EINVAL, "N=%u must be a power of two in [256, 8192]", N);
  const u64 q = prm->q;
  const bool rns_modulus = prm->rns_p1 || prm->rns_p2;
  const u32 p1 = std::min(prm->rns_p1, prm->rns_p2), p2 = std::max(prm->rns_p1, prm->rns_p2);
  // q = 2^k (the paper's parameter set): computed exactly through p1 p2
  const bool pow2 = q != 0 && (q & (q - 1)) == 0;
  if (pow2) {
    const u32 k = (u32)floor_log2(q);
    if (!rns_modulus) return fail(PHE_EINVAL, "q=2^%u needs rns_p1, rns_p2 (the modulus the products run in)", k);
    if (k < 8 || k > 62) return fail(PHE_EINVAL, "q=2^%u: need 8 <= k <= 62", k);
    if (prm->log2_qout < 1 || prm->log2_qout >= k)
      return fail(PHE_EINVAL, "q=2^%u: log2_qout=%u must be in [1, %u)", k, prm->log2_qout, k);
    if (prm->flags & PHE_CTX_FORCE_U64) return fail(PHE_EINVAL, "q=2^%u has no 64-bit form", k);
  } else {
    if (q <= (1ull << 53) || q >= (1ull << 61))
      return fail(PHE_EINVAL, "q=%llu must satisfy 2^53 < q < 2^61", (unsigned long long)q);
    if ((q - 1) % (2ull * N) != 0)
      return fail(PHE_EINVAL, "q=%llu is not 1 mod 2N=%u", (unsigned long long)q, 2 * N);
  }
  if (rns_modulus) {
    if (!p1 || p1 == p2 || p2 >= (1u << 30) || (!pow2 && (u64)p1 * p2 != q))
      return fail(PHE_EINVAL, "RNS modulus: need q = p1 * p2 with distinct p1, p2 < 2^30");
    if (!is_prime(p1) || !is_prime(p2)) return fail(PHE_EINVAL, "RNS modulus: p1 and p2 must be prime");
    if ((p1 - 1) % (2u * N) != 0 || (p2 - 1) % (2u * N) != 0)
      return fail(PHE_EINVAL, "RNS modulus: p1 and p2 must be 1 mod 2N=%u", 2 * N);
  } else if (!is_prime(q)) {
    return fail(PHE_EINVAL, "q=%llu is not prime (give rns_p1, rns_p2 for an RNS modulus)",
                (unsigned long long)q);
  }
  if (pow2) {
    // one block of products must stay below (p1 p2)/2 in magnitude: N 127 2^(k-1)
    const u128 bound = (u128)N * 127 * (q / 2);
    if (2 * bound >= (u128)p1 * p2)
      return fail(PHE_EINVAL, "q=%llu: N*127*q/2 must be below p1*p2/2 for exact products",
                  (unsigned long long)q);
  }
  if (prm->log2_qout < 1 || prm->log2_qout > 32) return fail(PHE_EINVAL, "log2_qout=%u not in [1, 32]", prm->log2_qout);
  if (prm->flags & ~PHE_CTX_FORCE_U64) return fail(PHE_EINVAL, "flags=%u", prm->flags);

  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(PHE_EINVAL, "device %d out of range (%d devices)", device, ndev);
  DeviceGuard g(device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");

  phe_ctx* c = new (std::nothrow) phe_ctx();
  if (!c) return fail(PHE_ENOMEM, "phe_ctx_create: host allocation");
  c->prm = *prm;
  c->device = device;
  c->logn = floor_log2(N);
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaDeviceGetAttribute"); }
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&c->pool, &props);
    uint64_t keep = UINT64_MAX;  // freed scratch stays mapped for the next call
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      if (c->pool) cudaMemPoolDestroy(c->pool);
      delete c;
      return cuda_fail(e, "cudaMemPoolCreate");
    }
  }
  e = cudaMalloc(&c->d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = phe::noalloc_setup();
  if (e != cudaSuccess) {
    cudaFree(c->d_status);
    cudaMemPoolDestroy(c->pool);
    delete c;
    return cuda_fail(e, "phe_ctx_create: status word");
  }

  phe::RingConst& rc = c->rc;
  rc.q = q;
  rc.q2 = 2 * q;
  rc.q4 = 4 * q;
  rc.half_q = q / 2;
  rc.ms_s = (u32)floor_log2(q);
  rc.ms_mu = pow2 ? 0 : (u64)(((u128)1 << (64 + rc.ms_s)) / q);  // the power-of-two switch is a shift
  rc.red_mu = (u64)(((u128)1 << 64) / q);
  rc.c30 = (1ull << 30) % q;
  rc.c30p = shoup(rc.c30, q);
  rc.c60 = (1ull << 60) % q;
  rc.c60p = shoup(rc.c60, q);
  rc.c64 = (u64)(((u128)1 << 64) % q);
  rc.c64p = shoup(rc.c64, q);
  rc.c32 = (1ull << 32) % q;
  rc.c32p = shoup(rc.c32, q);
  rc.log2_qout = prm->log2_qout;
  c->pow2 = pow2;
  if (!pow2) {
    c->n_inv = modinv(N, q);
    c->n_inv_p = shoup(c->n_inv, q);
    c->ninv.n64 = c->n_inv;
    c->ninv.n64p = c->n_inv_p;
  }

  // Primitive 2N-th root of unity mod q: directly for a prime q; for q = p1 p2
  // the CRT combination of the two primes' roots (its order is 2N in both).
  u64 psi = 0;
  u32 psi1 = 0, psi2 = 0;
  if (rns_modulus) {
    psi1 = (u32)primitive_root_2n(p1, N);
    psi2 = (u32)primitive_root_2n(p2, N);
    if (!psi1 || !psi2) { cudaFree(c->d_status); cudaMemPoolDestroy(c->pool); delete c; return fail(PHE_EINVAL, "no primitive 2N-th root of unity mod p1 or p2"); }
    if (!pow2) psi = crt2(psi1, p1, psi2, p2);
  } else {
    psi = primitive_root_2n(q, N);
  }
  if (!psi && !pow2) { cudaFree(c->d_status); cudaMemPoolDestroy(c->pool); delete c; return fail(PHE_EINVAL, "no primitive 2N-th root of unity found for q"); }

  // 64-bit tables mod q (none for q = 2^k: everything runs through p1 p2)
  phe_status st = pow2 ? PHE_OK : build_tables(c, [&](u32 br, bool inverse) -> ulonglong2 {
    const u64 root = inverse ? modinv(psi, q) : psi;
    const u64 a = powmod(root, br, q);
    return make_ulonglong2(a, shoup(a, q));
  }, c->tab);
  if (st == PHE_OK && rns_modulus) {
    phe::RnsConst& k = c->rk;
    k.p1 = p1;
    k.p2 = p2;
    k.inv = (u32)modinv(p1 % p2, p2);
    k.invp = shoup32(k.inv, p2);
    k.c32a = (u32)((1ull << 32) % p1);
    k.c32ap = shoup32(k.c32a, p1);
    k.c32b = (u32)((1ull << 32) % p2);
    k.c32bp = shoup32(k.c32b, p2);
    phe::set_switch_target(k, prm->log2_qout);
    if (pow2) {
      k.p2k = (u32)floor_log2(q);
      k.p2shift = k.p2k - prm->log2_qout;
      k.Q = (u64)p1 * p2;
      k.Qhalf = k.Q / 2;
      k.lift = k.Q - q;
    }
    c->ninv.n1 = (u32)modinv(N, p1);
    c->ninv.n1p = shoup32(c->ninv.n1, p1);
    c->ninv.n2 = (u32)modinv(N, p2);
    c->ninv.n2p = shoup32(c->ninv.n2, p2);
    const u64 i1 = modinv(psi1, p1), i2 = modinv(psi2, p2);
    st = build_tables(c, [&](u32 br, bool inverse) -> ulonglong2 {
      const u32 a = (u32)powmod(inverse ? i1 : psi1, br, p1);
      const u32 b = (u32)powmod(inverse ? i2 : psi2, br, p2);
      // (w1, w1', w2, w2') packed as two 64-bit words: bytes of a uint4
      const u64 lo = (u64)a | ((u64)shoup32(a, p1) << 32);
      const u64 hi = (u64)b | ((u64)shoup32(b, p2) << 32);
      return make_ulonglong2(lo, hi);
    }, c->tab32);
    c->rns = !(prm->flags & PHE_CTX_FORCE_U64);
  }
  if (st != PHE_OK) {
    free_tables(c->tab);
    free_tables(c->tab32);
    cudaFree(c->d_status);
    cudaMemPoolDestroy(c->pool);
    delete c;
    return st;
  }
  *out = c;
  return PHE_OK;
}

void phe_ctx_destroy(phe_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  for (auto& s : c->side)
    if (s) cudaStreamDestroy(s);
  for (auto& r : c->tracer.recs) {
    if (r.borrowed) continue;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->tracer.pool) cudaEventDestroy(e);
  free_tables(c->tab);
  free_tables(c->tab32);
  cudaFree(c->d_status);
  // a pool with frees still in flight is released once they complete
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
}

phe_status phe_weights_upload(phe_ctx* c, const int8_t* h_W, uint32_t d_out, uint32_t d_in, uint32_t dirs,
                              void* stream, phe_weights** out) {
  if (!c || !h_W || !out) return fail(PHE_EINVAL, "phe_weights_upload: null argument");
  *out = nullptr;
  if (d_out < 1 || d_in < 1 || d_out > 16384 || d_in > 16384)
    return fail(PHE_EINVAL, "weights %ux%u: dimensions must be in [1, 16384]", d_out, d_in);
  if (dirs == 0 || (dirs & ~3u)) return fail(PHE_EINVAL, "dirs=%u must be a non-empty subset of {FWD, BWD}", dirs);
  if (c->pow2) {
    // every product sum_i A_i w_hat_ij must stay an exact integer below p1 p2 / 2
    const u32 N0 = c->prm.N;
    for (int dir = 0; dir < 2; ++dir) {
      if (!(dirs & (1u << dir))) continue;
      const u32 cols = dir == PHE_FWD ? d_in : d_out;
      const u64 L = (cols + N0 - 1) / N0;
      if (2 * ((u128)L * N0 * 127 * (c->prm.q / 2)) >= (u128)c->rk.Q)
        return fail(PHE_EINVAL, "weights %ux%u: %llu blocks exceed the exact range of p1*p2 for q=2^%u", d_out,
                    d_in, (unsigned long long)L, c->rk.p2k);
    }
  }
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;

  phe_weights* w = new (std::nothrow) phe_weights();
  if (!w) return fail(PHE_ENOMEM, "phe_weights_upload: host allocation");
  w->ctx = c;
  w->d_out = d_out;
  w->d_in = d_in;
  w->dirs = dirs;
  const u32 N = c->prm.N;
  const size_t wbytes = (size_t)d_out * d_in;
  std::vector<int8_t> WT;
  if (dirs & PHE_DIR_BWD_BIT) {
    WT.resize(wbytes);
    for (u32 j = 0; j < d_out; ++j)
      for (u32 k = 0; k < d_in; ++k) WT[(size_t)k * d_out + j] = h_W[(size_t)j * d_in + k];
  }
  cudaError_t e = cudaSuccess;
  for (int dir = 0; dir < 2 && e == cudaSuccess; ++dir) {
    if (!(dirs & (1u << dir))) continue;
    phe_weights::Dir& D = w->dir[dir];
    D.rows = dir == PHE_FWD ? d_out : d_in;
    D.cols = dir == PHE_FWD ? d_in : d_out;
    D.L = (D.cols + N - 1) / N;
    const size_t what_bytes = (size_t)D.rows * D.L * N * sizeof(ulonglong2);
    if ((e = cudaMalloc(&D.what, what_bytes)) != cudaSuccess) break;
    if ((e = cudaMalloc(&D.wrow, wbytes)) != cudaSuccess) break;
    const size_t bf_bytes = (size_t)D.rows * phe::digit_pitch(D.cols) * 2;
    if ((e = cudaMalloc(&D.wbf, bf_bytes)) != cudaSuccess) break;
    w->bytes += what_bytes + wbytes + bf_bytes;
    const int8_t* src = dir == PHE_FWD ? h_W : WT.data();
    if ((e = cudaMemcpyAsync(D.wrow, src, wbytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = phe::launch_weight_ntt(c, D.wrow, D.rows, D.cols, D.cols, 1, D.L, 1, D.what, s)) != cudaSuccess) break;
    if ((e = phe::launch_weights_bf16(c, D.wrow, D.rows, D.cols, D.wbf, s)) != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    phe_weights_free(w);
    return cuda_fail(e, "phe_weights_upload");
  }
  *out = w;
  return PHE_OK;
}

void phe_weights_free(phe_weights* w) {
  if (!w) return;
  DeviceGuard g(w->ctx->device);
  for (auto& D : w->dir) {
    cudaFree(D.what);
    cudaFree(D.wrow);
    cudaFree(D.wbf);
  }
  delete w;
}

phe_status phe_weights_shape(const phe_weights* w, int dir, uint32_t* rows, uint32_t* cols, uint32_t* L) {
  if (!w) return fail(PHE_EINVAL, "phe_weights_shape: null handle");
  phe_status st = check_dir(w, dir);
  if (st != PHE_OK) return st;
  if (rows) *rows = w->dir[dir].rows;
  if (cols) *cols = w->dir[dir].cols;
  if (L) *L = w->dir[dir].L;
  return PHE_OK;
}

uint64_t phe_weights_device_bytes(const phe_weights* w) { return w ? w->bytes : 0; }

phe_status phe_matmul(phe_ctx* c, const phe_weights* w, int dir, uint32_t T, const uint64_t* d_in_mask,
                      const uint64_t* d_in_body, void* d_out_mask, void* d_out_body, uint32_t flags, void* stream) {
  phe_status st = check_matmul_args(c, w, dir, flags);
  if (st != PHE_OK) return st;
  if (T == 0) return PHE_OK;
  if (!d_in_mask || !d_in_body || !d_out_mask || !d_out_body) return fail(PHE_EINVAL, "phe_matmul: null buffer");
  if (T > (1u << 24)) return fail(PHE_EINVAL, "phe_matmul: T=%u exceeds 2^24", T);
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const int mode = flags == PHE_OUT_RAW ? phe::kOutRaw : phe::kOutSwitched;
  cudaError_t e = matmul_device(c, w->dir[dir], T, reinterpret_cast<const u64*>(d_in_mask),
                                reinterpret_cast<const u64*>(d_in_body), d_out_mask, d_out_body, mode,
                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul");
  return PHE_OK;
}

phe_status phe_matmul_seeded(phe_ctx* c, const phe_weights* w, int dir, uint32_t T, const uint64_t* d_in_seeds,
                             const uint64_t* d_in_body, void* d_out_mask, void* d_out_body, uint32_t flags,
                             void* stream) {
  phe_status st = check_matmul_args(c, w, dir, flags);
  if (st != PHE_OK) return st;
  if (T == 0) return PHE_OK;
  if (!d_in_seeds || !d_in_body || !d_out_mask || !d_out_body)
    return fail(PHE_EINVAL, "phe_matmul_seeded: null buffer");
  if (T > (1u << 24)) return fail(PHE_EINVAL, "phe_matmul_seeded: T=%u exceeds 2^24", T);
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const int mode = flags == PHE_OUT_RAW ? phe::kOutRaw : phe::kOutSwitched;
  cudaError_t e = matmul_device(c, w->dir[dir], T, nullptr, reinterpret_cast<const u64*>(d_in_body), d_out_mask,
                                d_out_body, mode, (cudaStream_t)stream, reinterpret_cast<const u64*>(d_in_seeds));
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_seeded");
  return PHE_OK;
}

phe_status phe_expand_masks(phe_ctx* c, const uint64_t* d_seeds, uint32_t n, uint64_t* d_masks, void* stream) {
  if (!c) return fail(PHE_EINVAL, "phe_expand_masks: null context");
  if (n == 0) return PHE_OK;
  if (!d_seeds || !d_masks) return fail(PHE_EINVAL, "phe_expand_masks: null buffer");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  Span sp(c, phe::kKExpand, (cudaStream_t)stream);
  cudaError_t e = phe::launch_expand_masks(c, reinterpret_cast<const u64*>(d_seeds), n,
                                           reinterpret_cast<u64*>(d_masks), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_expand_masks");
  return PHE_OK;
}

phe_status phe_matmul_host(phe_ctx* c, const phe_weights* w, int dir, uint32_t T, const uint64_t* h_in_mask,
                           const uint64_t* h_in_body, void* h_out_mask, void* h_out_body, uint32_t flags,
                           uint64_t max_chunk_bytes, void* stream) {
  phe_status st = check_matmul_args(c, w, dir, flags);
  if (st != PHE_OK) return st;
  if (T == 0) return PHE_OK;
  if (!h_in_mask || !h_in_body || !h_out_mask || !h_out_body) return fail(PHE_EINVAL, "phe_matmul_host: null buffer");
  if (T > (1u << 24)) return fail(PHE_EINVAL, "phe_matmul_host: T=%u exceeds 2^24", T);
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const phe_weights::Dir& D = w->dir[dir];
  const u32 N = c->prm.N;
  const int mode = flags == PHE_OUT_RAW ? phe::kOutRaw : phe::kOutSwitched;
  const size_t osz = mode == phe::kOutRaw ? 8 : 4;
  const size_t in_tok = (size_t)D.L * N * sizeof(u64);
  const size_t om_tok = (size_t)D.rows * N * osz, ob_tok = (size_t)D.rows * osz;
  if (max_chunk_bytes == 0) max_chunk_bytes = 1ull << 30;
  u32 tc = (u32)(max_chunk_bytes / (om_tok + ob_tok));
  if (tc < 1) tc = 1;
  if (tc > T) tc = T;
  cudaStream_t caller = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!c->side[i]) e = cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  cudaEvent_t ev = nullptr;
  if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  e = cudaEventRecord(ev, caller);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->side[i], ev, 0);
  // Two buffer sets on two streams: chunk n uses set n % 2, so the copies of
  // one chunk overlap the kernels of the next.
  struct Buf { u64 *a = nullptr, *b = nullptr; char *om = nullptr, *ob = nullptr; } buf[2];
  const u32 nchunks = (T + tc - 1) / tc;
  for (int i = 0; i < 2 && i < (int)nchunks && e == cudaSuccess; ++i) {
    cudaStream_t s = c->side[i];
    if ((e = phe::ctx_malloc_async(c, &buf[i].a, tc * in_tok, s)) != cudaSuccess) break;
    if ((e = phe::ctx_malloc_async(c, &buf[i].b, tc * in_tok, s)) != cudaSuccess) break;
    if ((e = phe::ctx_malloc_async(c, &buf[i].om, tc * om_tok, s)) != cudaSuccess) break;
    e = phe::ctx_malloc_async(c, &buf[i].ob, tc * ob_tok, s);
  }
  for (u32 n = 0; n < nchunks && e == cudaSuccess; ++n) {
    const u32 t0 = n * tc, tn = (T - t0 < tc) ? T - t0 : tc;
    cudaStream_t s = c->side[n % 2];
    Buf& B = buf[n % 2];
    const char* hm = reinterpret_cast<const char*>(h_in_mask) + t0 * in_tok;
    const char* hb = reinterpret_cast<const char*>(h_in_body) + t0 * in_tok;
    if ((e = cudaMemcpyAsync(B.a, hm, tn * in_tok, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(B.b, hb, tn * in_tok, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = matmul_device(c, D, tn, B.a, B.b, B.om, B.ob, mode, s)) != cudaSuccess) break;
    char* om = reinterpret_cast<char*>(h_out_mask) + t0 * om_tok;
    char* ob = reinterpret_cast<char*>(h_out_body) + t0 * ob_tok;
    if ((e = cudaMemcpyAsync(om, B.om, tn * om_tok, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    e = cudaMemcpyAsync(ob, B.ob, tn * ob_tok, cudaMemcpyDeviceToHost, s);
  }
  for (int i = 0; i < 2; ++i) {
    cudaStream_t s = c->side[i];
    cudaFreeAsync(buf[i].a, s);
    cudaFreeAsync(buf[i].b, s);
    cudaFreeAsync(buf[i].om, s);
    cudaFreeAsync(buf[i].ob, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
  }
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(e, "phe_matmul_host");
  return PHE_OK;
}

phe_status phe_ctx_set_body_path(phe_ctx* c, uint32_t path) {
  if (!c) return fail(PHE_EINVAL, "phe_ctx_set_body_path: null context");
  if (path != PHE_BODY_AUTO && path != PHE_BODY_TENSOR && path != PHE_BODY_FUSED)
    return fail(PHE_EINVAL, "phe_ctx_set_body_path: path=%u", path);
  c->body_path = path;
  return PHE_OK;
}

phe_status phe_trace_enable(phe_ctx* c, int on) {
  if (!c) return fail(PHE_EINVAL, "phe_trace_enable: null context");
  c->tracer.on = on != 0;
  return PHE_OK;
}

phe_status phe_trace_read(phe_ctx* c, phe_trace_entry* out, uint32_t cap, uint32_t* n_out) {
  if (!c || !n_out || (cap && !out)) return fail(PHE_EINVAL, "phe_trace_read: null argument");
  DeviceGuard g(c->device);
  std::vector<std::vector<double>> ms(phe::kKCount);
  cudaError_t err = cudaSuccess;
  for (const auto& r : c->tracer.recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    ms[r.kid].push_back(t);
    if (!r.borrowed) {
      c->tracer.pool.push_back(r.a);
      c->tracer.pool.push_back(r.b);
    }
  }
  c->tracer.recs.clear();
  if (err != cudaSuccess) return cuda_fail(err, "phe_trace_read");
  uint32_t n = 0;
  for (int k = 0; k < phe::kKCount; ++k) {
    if (ms[k].empty()) continue;
    if (n < cap) {
      auto& v = ms[k];
      std::sort(v.begin(), v.end());
      phe_trace_entry& E = out[n];
      std::memset(&E, 0, sizeof(E));
      std::snprintf(E.name, sizeof(E.name), "%s", phe::kernel_name(k));
      E.launches = v.size();
      for (double x : v) E.total_ms += x;
      auto rank = [&](double pct) { size_t i = (size_t)std::ceil(pct * v.size()); return v[i ? i - 1 : 0]; };
      E.p50_ms = rank(0.50);
      E.p99_ms = rank(0.99);
      E.max_ms = v.back();
    }
    ++n;
  }
  *n_out = n < cap ? n : cap;
  return PHE_OK;
}

phe_status phe_modswitch(phe_ctx* c, const uint64_t* d_in, uint32_t* d_out, size_t n, void* stream) {
  if (!c) return fail(PHE_EINVAL, "phe_modswitch: null context");
  if (n == 0) return PHE_OK;
  if (!d_in || !d_out) return fail(PHE_EINVAL, "phe_modswitch: null buffer");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  Span sp(c, phe::kKModswitch, (cudaStream_t)stream);
  cudaError_t e = phe::launch_modswitch(c, reinterpret_cast<const u64*>(d_in), d_out, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "phe_modswitch launch");
  return PHE_OK;
}

}  // extern "C"
