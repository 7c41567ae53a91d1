// Host-side structures of libphe shared by the C-ABI layer and the kernel
// launchers.  Not part of the public interface (include/phe.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "phe_device.cuh"
#include "../../include/phe.h"

namespace phe {

constexpr int kMaxJobs = 32;      // jobs in one batched launch (passed by value)
// Tokens per lwedot tile for the calls that do not autotune (on the layer
// workload, with all tiles of one row adjacent, 8-token tiles ran within 1%
// of the autotuner's best and 4% above 2-token tiles).
constexpr unsigned kDefaultTokChunk = 8;
constexpr int kMinLogN = 8;
// Columns per exact fp32 accumulation of the body GEMM: |w beta| <= 127*128,
// so a chunk's partial sums stay below 2^24 (phe_body.cu).
constexpr u32 kBodyChunk = 1024;
// Row pitch (elements) of the bf16 weight and digit rows: 16-byte aligned rows for TMA.
inline u32 digit_pitch(u32 cols) { return (cols + 7) & ~7u; }
inline size_t digit_bytes(u32 T, u32 cols) { return (size_t)T * 8 * digit_pitch(cols) * 2; }
// Below this many (token, row) outputs in one launch group the bodies stay
// fused in lwedot (a dp4a dot product): the body GEMM's two extra launches
// and its cold pipeline cost more than the ~11% of lwedot time the fused body
// takes.  One token of a 2048x8192 product (8192 outputs) is faster fused;
// one token of a whole layer (44 032 outputs) on the tensor cores.
constexpr unsigned long long kBodyGemmMinItems = 16384;
constexpr int kMaxLogN = 13;

// One matrix product of the hot path, as the lwedot kernel sees it.
struct LweJob {
  const ulonglong2* what;   // W_hat pairs [rows][L][N] (what_idx layout)
  const u64* ahat;          // A_hat [T][L][N] (ahat_idx layout)
  void* out;                // mask out: [T][rows][N] u32 (switched) or u64 (raw / ring product)
  const int8_t* wrow;       // clear weights of this direction, [rows][cols] int8 (body product)
  const u64* bin;           // input bodies, token t at bin + t*L*N
  void* out_body;           // [T][rows] u32 (switched) or u64 (raw)
  const int32_t* err;       // client encryption only: E [T*L][N]
  const int8_t* msg;        // client encryption only: x [T][msg_d]
  u64 delta, delta_p;       // client encryption only: delta and its Shoup quotient
  u32 rows, cols, T, L, tok_chunk, tiles, msg_d;
  u32 row_group;             // rows per tile (set_lwe_tiles)
  // Bodies on the tensor cores (phe_body.cu): the direction's weights as
  // bf16 rows [rows][digit_pitch(cols)], and scratch for the bodies' digit
  // rows [T*8][digit_pitch(cols)] (assign_body_scratch), written by the
  // first job of a table that reads these bodies (digits_owner).
  const void* wbf = nullptr;
  void* digits = nullptr;
  u32 digits_owner = 0;
};
struct LweJobTable {
  u32 n;
  u32 prefix[kMaxJobs + 1];  // tile prefix sums
  LweJob j[kMaxJobs];
  // Persistent launches (a grid smaller than the tiles): a device counter,
  // zero at the launch, from which each CTA takes its next tile, so that
  // tiles of unequal cost balance across the CTAs.  Null: a CTA takes tiles
  // blockIdx.x, + gridDim.x, ...
  u32* tile_counter = nullptr;
};

struct NttJob {             // forward transform of T*L input blocks
  const u64* src;           // natural order [blocks][N], or nullptr when `seeds` is given
  u64* dst;                 // A_hat layout [blocks][N]
  u32 blocks;
  const u64* seeds = nullptr;  // [blocks] 64-bit seeds: masks expanded on the fly
  const int32_t* digits = nullptr;  // [blocks][N] small signed integers instead of src (packing digits)
};

// kOutPackIn: masks switched to the gadget modulus B^ell (uint32, what
// Decomp reads) and bodies raw mod q (uint64), the inputs of the packing.
enum OutMode : int {
  kOutSwitched = 0, kOutRaw = 1, kOutRing = 2, kOutPackIn = 3, kPow2 = 4 /* flag: q = 2^k via the RNS form */,
  kK32 = 8 /* flag: switched outputs at q' = 2^32, the shift and mask known at compile time */,
  kBodyGemm = 16 /* flag: the bodies come from the tensor-core GEMM (launch_body), not from lwedot */
};

// Kernel names for tracing; kKCall brackets a whole phe_matmul call.
enum KernelId : int {
  kKInputNtt = 0, kKLwedot, kKModswitch, kKWeightNtt, kKExpand, kKCall, kKPlan, kKGraph,
  kKPackDecompose, kKPackMac, kKPackFinish, kKPackCall, kKBodyGemm, kKCount
};
inline const char* kernel_name(int k) {
  static const char* names[kKCount] = {"input_ntt_kernel", "lwedot_kernel", "modswitch_kernel", "weight_ntt_kernel",
                                       "expand_masks_kernel", "phe_matmul", "phe_plan_run", "phe_plan_graph",
                                       "pack_decompose_kernel", "pack_mac_kernel", "pack_finish_kernel",
                                       "phe_pack", "body_gemm_kernel"};
  return (k >= 0 && k < kKCount) ? names[k] : "?";
}
struct TraceRec {
  int kid;
  cudaEvent_t a, b;
  bool borrowed = false;  // events owned by a captured graph, not by the pool
};
struct Tracer {
  bool on = false;
  std::vector<TraceRec> recs;
  std::vector<cudaEvent_t> pool;
};

// Twiddle tables (16 bytes per entry): (w, w') mod q for the 64-bit form,
// (w1, w1', w2, w2') mod (p1, p2) for the RNS form.
struct Tables {
  ulonglong2* fwd_c = nullptr;  // psi^brv(k) and Shoup quotient, [N]
  ulonglong2* inv_c = nullptr;  // psi^-brv(k) and Shoup quotient, [N]
  ulonglong2* fwd_0 = nullptr;  // pass-0 forward twiddles, thread-major [15][P]
  ulonglong2* inv_0 = nullptr;  // pass-0 inverse twiddles, thread-major [15][P]
};

// N^-1 with Shoup quotients: mod q (64-bit form) and mod p1, p2 (RNS form).
struct NInv {
  u64 n64, n64p;
  u32 n1, n1p, n2, n2p;
};

}  // namespace phe

struct phe_ctx {
  phe_params prm;
  int device = 0;
  int logn = 0;
  phe::RingConst rc{};
  phe::u64 n_inv = 0, n_inv_p = 0;  // N^-1 mod q and its Shoup quotient
  phe::NInv ninv{};
  phe::Tables tab;        // 64-bit form (every context)
  bool rns = false;       // hot path in the RNS form (q = p1 p2, or q = 2^k computed through p1 p2)
  bool pow2 = false;      // q = 2^k: exact products through p1 p2, reduced mod 2^k (RnsConst::p2k)
  phe::RnsConst rk{};
  phe::Tables tab32;      // RNS form (RNS contexts)
  int num_sms = 0;
  cudaStream_t side[2] = {nullptr, nullptr};  // streams for overlapped host-buffer chunks
  // The context's own stream-ordered memory pool: scratch freed at the end of
  // a call stays mapped for the next one (the device's default pool would
  // release it at every synchronization and map it again).
  cudaMemPool_t pool = nullptr;
  // Status word the kernels with bounded waits set bits in (phe_body.cu):
  // nonzero means a wait timed out and that launch's outputs are not valid.
  uint32_t* d_status = nullptr;
  uint32_t body_path = PHE_BODY_AUTO;  // phe_ctx_set_body_path
  phe::Tracer tracer;
};

struct phe_weights {
  phe_ctx* ctx = nullptr;
  uint32_t d_out = 0, d_in = 0, dirs = 0;
  struct Dir {
    ulonglong2* what = nullptr;  // [rows][L][N] pairs
    int8_t* wrow = nullptr;      // [rows][cols] clear weights of the direction
    void* wbf = nullptr;         // [rows][digit_pitch(cols)] the same weights as bf16 (body GEMM)
    uint32_t rows = 0, cols = 0, L = 0;
  } dir[2];
  uint64_t bytes = 0;
};

namespace phe {

// An event from the context's pool (or a new one); nullptr if none can be made.
inline cudaEvent_t trace_event(phe_ctx* c) {
  if (!c->tracer.pool.empty()) {
    cudaEvent_t e = c->tracer.pool.back();
    c->tracer.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets one launch (or one call) with events on its stream while tracing is on.
struct Span {
  phe_ctx* c;
  int kid;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Span(phe_ctx* c_, int kid_, cudaStream_t s_) : c(c_), kid(kid_), s(s_) {
    if (c->tracer.on && (a = trace_event(c)) != nullptr) cudaEventRecord(a, s);
  }
  ~Span() {
    if (!a) return;
    cudaEvent_t b = trace_event(c);
    if (!b) {
      c->tracer.pool.push_back(a);
      return;
    }
    cudaEventRecord(b, s);
    c->tracer.recs.push_back({kid, a, b});
  }
};

// Scratch for one call, from the context's pool, ordered on `s` (release it
// with cudaFreeAsync on a stream ordered after its last use).
template <class T>
inline cudaError_t ctx_malloc_async(const phe_ctx* c, T** p, size_t bytes, cudaStream_t s) {
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, c->pool, s);
}

// Launchers (phe_kernels.cu).  All asynchronous on `s`.
// The hot-path launchers use the context's form (RNS when c->rns) unless
// force64 asks for the 64-bit form (client-side encryption).
cudaError_t launch_input_ntt(const phe_ctx* c, const NttJob* jobs, int n, cudaStream_t s, bool force64 = false);
cudaError_t launch_weight_ntt(const phe_ctx* c, const int8_t* W, u32 rows, u32 cols, u32 row_stride,
                              u32 col_stride, u32 L, int rev, void* what, cudaStream_t s, bool force64 = false);
cudaError_t launch_lwedot(const phe_ctx* c, const LweJobTable& jt, int mode, int grid_limit, cudaStream_t s,
                          bool force64 = false);

cudaError_t launch_modswitch(const phe_ctx* c, const u64* in, u32* out, size_t n, cudaStream_t s);
cudaError_t launch_expand_masks(const phe_ctx* c, const u64* seeds, u32 n, u64* masks, cudaStream_t s);
int lwedot_threads(int logn);

// Bodies on the tensor cores (phe_body.cu).
// int8 rows [rows][cols] -> bf16 rows [rows][digit_pitch(cols)].
cudaError_t launch_weights_bf16(const phe_ctx* c, const int8_t* W, u32 rows, u32 cols, void* out, cudaStream_t s);
// Scratch bytes for the digit rows of every distinct body input of jt, and
// the assignment of that scratch to the jobs (sets digits / digits_owner).
size_t body_scratch_bytes(const LweJobTable& jt);
cudaError_t assign_body_scratch(LweJobTable& jt, void* scratch);
// Digit rows of each distinct body input, then the body GEMM of every job:
// out_body[t][j] switched to 2^k (raw = false) or raw mod q (raw = true).
cudaError_t launch_body(const phe_ctx* c, const LweJobTable& jt, bool raw, const RingConst& rc, const RnsConst& rk,
                        cudaStream_t s);
cudaError_t prepare_body_launches();
// Whether a launch group's bodies run on the tensor cores (the GEMM) or fused
// in lwedot: the context's body path, else the group's size.
inline bool body_on_tensor_cores(const phe_ctx* c, const LweJobTable& jt) {
  if (c->body_path == PHE_BODY_TENSOR) return true;
  if (c->body_path == PHE_BODY_FUSED) return false;
  unsigned long long items = 0;
  for (u32 i = 0; i < jt.n; ++i) items += (unsigned long long)jt.j[i].rows * jt.j[i].T;
  return items >= kBodyGemmMinItems;
}
// Loads the allocation-free entry point's scratch array on the current device (phe_noalloc.cu).
cudaError_t noalloc_setup();
// lwedot in kOutPackIn mode, with the switch constants rcK / rkK of
// 2^(base_log*ell), and the bodies of the GEMM (launch_body first; jobs carry
// wbf and digits) or fused (gemm = false).
cudaError_t launch_lwedot_packin2(const phe_ctx* c, const LweJobTable& jt, const RingConst& rcK, const RnsConst& rkK,
                                  bool gemm, cudaStream_t s);

// Tiles of an lwedot job: (a group of row_group adjacent rows) x (a chunk of
// tok_chunk tokens).  A block holds SLOTS = threads / (N/16) transforms; when
// a chunk has fewer tokens than that, the idle slots take adjacent rows, so
// one token per call still fills the block at N <= 2048.
inline void set_lwe_tiles(LweJob& J, int logn) {
  const u32 slots = (u32)lwedot_threads(logn) / ((1u << logn) / 16);
  u32 c = J.tok_chunk < J.T ? J.tok_chunk : J.T;
  if (c == 0) c = 1;
  u32 cs = 1;  // tokens per slot round: the largest power of two <= min(c, slots)
  while (cs * 2 <= c && cs * 2 <= slots) cs *= 2;
  J.row_group = slots / cs;
  J.tiles = ((J.rows + J.row_group - 1) / J.row_group) * ((J.T + J.tok_chunk - 1) / J.tok_chunk);
}
// Sets the dynamic shared-memory limits of the context's kernels (needed
// before a launch is captured into a graph when a kernel exceeds 48 KB).
cudaError_t prepare_launches(const phe_ctx* c);
// Sets the calling thread's phe_last_error() message (phe_capi.cu).
void set_last_error(const char* msg);
// Sets the message from a printf-style format and returns s (phe_capi.cu).
phe_status fail(phe_status s, const char* fmt, ...);
// fail() with a CUDA error's text; an allocation failure maps to PHE_ENOMEM.
phe_status cuda_fail(cudaError_t e, const char* what);

// Makes a device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};
// Sets the constants of rns_modswitch in k (p1, p2 set) for the target
// modulus 2^log2_target, 1 <= log2_target <= 32 (phe_capi.cu).
void set_switch_target(RnsConst& k, u32 log2_target);
size_t lwedot_smem(int logn);

}  // namespace phe
