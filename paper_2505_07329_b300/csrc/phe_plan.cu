// Batched form of the hot path: many products -- every projection and both
// directions of a layer, with uneven token counts -- as one input-transform
// pass and one persistent lwedot launch per group of up to kMaxJobs
// products, optionally replayed from a CUDA graph; plus the autotuner that
// picks the tile shape (tokens per tile) and the persistent grid.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "phe_host.hpp"

using phe::u32;
using phe::u64;
using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;

struct phe_plan {
  phe_ctx* ctx = nullptr;
  uint32_t flags = 0;
  phe_tuning tune{};
  struct Input {
    const u64* mask = nullptr;
    const u64* seeds = nullptr;
    u32 blocks = 0;
    u64* ahat = nullptr;
  };
  std::vector<Input> inputs;
  std::vector<phe::LweJobTable> tables;
  std::vector<void*> body_scratch;  // digit rows of the bodies, one buffer per table (tensor-core bodies)
  std::vector<char> gemm;           // per table: bodies on the tensor cores, else fused in lwedot
  u32* tile_counters = nullptr;     // persistent grids: one tile counter per table
  std::vector<u32> grids;
  u64 scratch_bytes = 0;
  u64 modmuls = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // Timing events captured into the graph (event-record nodes around each
  // lwedot launch) when tracing was on at capture; each replay re-records them.
  std::vector<phe::TraceRec> graph_recs;
};

namespace {




phe_status check_job(const phe_ctx* c, const phe_job& j, uint32_t idx) {
  if (!j.w) return fail(PHE_EINVAL, "job %u: null weights", idx);
  if (j.w->ctx != c) return fail(PHE_EINVAL, "job %u: weights belong to another context", idx);
  if (j.dir != PHE_FWD && j.dir != PHE_BWD) return fail(PHE_EINVAL, "job %u: bad direction %d", idx, j.dir);
  if (!(j.w->dirs & (1u << j.dir))) return fail(PHE_EINVAL, "job %u: direction was not uploaded", idx);
  if (j.T > (1u << 24)) return fail(PHE_EINVAL, "job %u: T=%u exceeds 2^24", idx, j.T);
  if (j.T && ((!j.d_in_mask && !j.d_in_seeds) || !j.d_in_body || !j.d_out_mask || !j.d_out_body))
    return fail(PHE_EINVAL, "job %u: null buffer", idx);
  return PHE_OK;
}

void destroy_plan(phe_plan* p) {
  if (!p) return;
  DeviceGuard g(p->ctx->device);
  // drop pending trace records that point at this plan's events
  auto& recs = p->ctx->tracer.recs;
  for (const auto& gr : p->graph_recs)
    recs.erase(std::remove_if(recs.begin(), recs.end(), [&](const phe::TraceRec& r) { return r.a == gr.a; }),
               recs.end());
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (auto& r : p->graph_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto& in : p->inputs) cudaFree(in.ahat);
  for (void* b : p->body_scratch) cudaFree(b);
  cudaFree(p->tile_counters);
  delete p;
}

// trace: spans through the context's tracer (direct launches);
// capture_events: event-record nodes kept by the plan (graph capture).
cudaError_t run_plan(phe_plan* p, cudaStream_t s, bool trace, bool capture_events = false) {
  phe_ctx* c = p->ctx;
  cudaError_t e = cudaSuccess;
  for (auto& in : p->inputs) {
    phe::NttJob nj{in.mask, in.ahat, in.blocks, in.seeds};
    if (trace) {
      phe::Span sp(c, phe::kKInputNtt, s);
      e = phe::launch_input_ntt(c, &nj, 1, s);
    } else {
      e = phe::launch_input_ntt(c, &nj, 1, s);
    }
    if (e != cudaSuccess) return e;
  }
  const int mode = p->flags == PHE_OUT_RAW ? phe::kOutRaw : phe::kOutSwitched;
  const bool raw = mode == phe::kOutRaw;
  // Runs one launch group (the bodies' digit rows and GEMM, or the masks'
  // lwedot) bracketed by a span or by captured event-record nodes.
  auto bracket = [&](int kid, auto&& launch) -> cudaError_t {
    if (trace) {
      phe::Span sp(c, kid, s);
      return launch();
    }
    if (!capture_events) return launch();
    phe::TraceRec r{kid, nullptr, nullptr, true};
    cudaError_t e2 = cudaEventCreate(&r.a);
    if (e2 == cudaSuccess) e2 = cudaEventCreate(&r.b);
    if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal);
    if (e2 == cudaSuccess) e2 = launch();
    if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(r.b, s, cudaEventRecordExternal);
    if (r.a || r.b) p->graph_recs.push_back(r);
    return e2;
  };
  for (size_t t = 0; t < p->tables.size(); ++t) {
    const phe::LweJobTable& jt = p->tables[t];
    const bool gemm = p->gemm[t] != 0;
    if (gemm) e = bracket(phe::kKBodyGemm, [&] { return phe::launch_body(c, jt, raw, c->rc, c->rk, s); });
    if (e == cudaSuccess)
      e = bracket(phe::kKLwedot, [&] {
        return phe::launch_lwedot(c, jt, mode | (gemm ? phe::kBodyGemm : 0), (int)p->grids[t], s);
      });
    if (e != cudaSuccess) return e;
  }
  return e;
}

// Tuning results cached per ring, output mode and job-shape signature.
std::mutex g_tune_mutex;
std::map<std::string, phe_tuning>& tune_cache() {
  static std::map<std::string, phe_tuning> m;
  return m;
}

std::string signature(const phe_ctx* c, const phe_job* jobs, uint32_t n, uint32_t flags) {
  std::string s = std::to_string(c->device) + "/" + std::to_string(c->prm.N) + "/" + std::to_string(c->prm.q) + "/" +
                  std::to_string(flags);
  for (uint32_t i = 0; i < n; ++i) {
    const auto& D = jobs[i].w->dir[jobs[i].dir];
    s += ":" + std::to_string(D.rows) + "x" + std::to_string(D.L) + "x" + std::to_string(jobs[i].T > 0);
  }
  return s;
}

}  // namespace

extern "C" {

phe_status phe_plan_create(phe_ctx* c, const phe_job* jobs, uint32_t n_jobs, uint32_t flags, const phe_tuning* tune,
                           phe_plan** out) {
  if (!c || !out || (n_jobs && !jobs)) return fail(PHE_EINVAL, "phe_plan_create: null argument");
  *out = nullptr;
  if (flags != PHE_OUT_SWITCHED && flags != PHE_OUT_RAW) return fail(PHE_EINVAL, "phe_plan_create: flags=%u", flags);
  if (n_jobs > PHE_PLAN_MAX_JOBS) return fail(PHE_EINVAL, "phe_plan_create: %u jobs exceed %d", n_jobs, PHE_PLAN_MAX_JOBS);
  for (uint32_t i = 0; i < n_jobs; ++i) {
    phe_status st = check_job(c, jobs[i], i);
    if (st != PHE_OK) return st;
  }
  phe_tuning tn{16, 3};
  if (tune) tn = *tune;
  if (tn.tok_chunk < 1 || tn.tok_chunk > 4096) return fail(PHE_EINVAL, "phe_plan_create: tok_chunk=%u", tn.tok_chunk);
  if (tn.blocks_per_sm > 64) return fail(PHE_EINVAL, "phe_plan_create: blocks_per_sm=%u", tn.blocks_per_sm);
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaError_t e = phe::prepare_launches(c);
  if (e != cudaSuccess) return cuda_fail(e, "phe_plan_create: kernel attributes");

  phe_plan* p = new phe_plan();
  p->ctx = c;
  p->flags = flags;
  p->tune = tn;
  const u32 N = c->prm.N;
  const u32 logn = (u32)c->logn;
  phe::LweJobTable cur{};
  for (uint32_t i = 0; i < n_jobs; ++i) {
    const phe_job& j = jobs[i];
    if (j.T == 0) continue;
    const phe_weights::Dir& D = j.w->dir[j.dir];
    // one forward transform per distinct input
    const u64* seeds = reinterpret_cast<const u64*>(j.d_in_seeds);
    const u64* mask = seeds ? nullptr : reinterpret_cast<const u64*>(j.d_in_mask);
    const u32 blocks = j.T * D.L;
    size_t k = 0;
    for (; k < p->inputs.size(); ++k)
      if (p->inputs[k].mask == mask && p->inputs[k].seeds == seeds && p->inputs[k].blocks == blocks) break;
    if (k == p->inputs.size()) {
      phe_plan::Input in;
      in.mask = mask;
      in.seeds = seeds;
      in.blocks = blocks;
      e = cudaMalloc((void**)&in.ahat, (size_t)blocks * N * sizeof(u64));
      if (e != cudaSuccess) {
        destroy_plan(p);
        return cuda_fail(e, "phe_plan_create: cudaMalloc(A_hat)");
      }
      p->scratch_bytes += (u64)blocks * N * sizeof(u64);
      p->inputs.push_back(in);
    }
    phe::LweJob& J = cur.j[cur.n];
    J = phe::LweJob{};
    J.what = D.what;
    J.ahat = p->inputs[k].ahat;
    J.out = j.d_out_mask;
    J.wrow = D.wrow;
    J.wbf = D.wbf;
    J.bin = reinterpret_cast<const u64*>(j.d_in_body);
    J.out_body = j.d_out_body;
    J.rows = D.rows;
    J.cols = D.cols;
    J.T = j.T;
    J.L = D.L;
    J.tok_chunk = tn.tok_chunk;
    phe::set_lwe_tiles(J, c->logn);
    cur.prefix[cur.n + 1] = cur.prefix[cur.n] + J.tiles;
    cur.n++;
    p->modmuls += (u64)j.T * D.rows * ((u64)D.L * N + (u64)(N / 2) * logn);
    if (cur.n == phe::kMaxJobs) {
      p->tables.push_back(cur);
      cur = phe::LweJobTable{};
    }
  }
  if (cur.n) p->tables.push_back(cur);
  for (auto& t : p->tables) {
    // digit rows of each distinct body input of the table, resident with the plan
    const bool gemm = phe::body_on_tensor_cores(c, t);
    p->gemm.push_back(gemm ? 1 : 0);
    if (!gemm) {
      p->body_scratch.push_back(nullptr);
      continue;
    }
    void* b = nullptr;
    const size_t bytes = phe::body_scratch_bytes(t);
    e = cudaMalloc(&b, bytes ? bytes : 256);
    if (e != cudaSuccess) {
      destroy_plan(p);
      return cuda_fail(e, "phe_plan_create: cudaMalloc(body digit rows)");
    }
    p->body_scratch.push_back(b);
    p->scratch_bytes += bytes;
    phe::assign_body_scratch(t, b);
  }
  if (tn.blocks_per_sm && !p->tables.empty()) {
    e = cudaMalloc(&p->tile_counters, p->tables.size() * sizeof(u32));
    if (e != cudaSuccess) {
      destroy_plan(p);
      return cuda_fail(e, "phe_plan_create: cudaMalloc(tile counters)");
    }
  }
  for (size_t i = 0; i < p->tables.size(); ++i) {
    auto& t = p->tables[i];
    const u32 tiles = t.prefix[t.n];
    const u32 persistent = tn.blocks_per_sm ? (u32)c->num_sms * tn.blocks_per_sm : tiles;
    p->grids.push_back(std::min(tiles, persistent));
    if (p->tile_counters) t.tile_counter = p->tile_counters + i;
  }
  *out = p;
  return PHE_OK;
}

phe_status phe_plan_run(phe_plan* p, void* stream) {
  if (!p) return fail(PHE_EINVAL, "phe_plan_run: null plan");
  DeviceGuard g(p->ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  phe::Span call(p->ctx, phe::kKPlan, s);
  cudaError_t e = run_plan(p, s, true);
  if (e != cudaSuccess) return cuda_fail(e, "phe_plan_run");
  return PHE_OK;
}

phe_status phe_plan_graph(phe_plan* p, void* stream) {
  if (!p) return fail(PHE_EINVAL, "phe_plan_graph: null plan");
  if (!stream) return fail(PHE_EINVAL, "phe_plan_graph: needs a non-default stream to capture on");
  DeviceGuard g(p->ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!p->exec) {
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t er = run_plan(p, s, false, p->ctx->tracer.on);
    e = cudaStreamEndCapture(s, &p->graph);
    if (er != cudaSuccess) e = er;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
      if (p->graph) cudaGraphDestroy(p->graph);
      p->graph = nullptr;
      p->exec = nullptr;
      return cuda_fail(e, "phe_plan_graph: capture");
    }
  }
  {
    phe::Span call(p->ctx, phe::kKGraph, s);
    e = cudaGraphLaunch(p->exec, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  // The captured events now time this replay's launches; a later replay
  // overwrites them, so read the trace before replaying the plan again.
  if (p->ctx->tracer.on)
    for (const auto& r : p->graph_recs) p->ctx->tracer.recs.push_back(r);
  return PHE_OK;
}

phe_status phe_plan_info(const phe_plan* p, phe_plan_stats* st) {
  if (!p || !st) return fail(PHE_EINVAL, "phe_plan_info: null argument");
  // per table: lwedot; with tensor-core bodies also one digit-row kernel per
  // distinct body input and the body GEMM
  uint32_t launches = (uint32_t)p->inputs.size();
  for (size_t k = 0; k < p->tables.size(); ++k) {
    const auto& t = p->tables[k];
    launches += 1;
    if (!p->gemm[k]) continue;
    launches += 1;
    for (u32 i = 0; i < t.n; ++i) launches += t.j[i].digits_owner;
  }
  st->launches = launches;
  st->lwedot_launches = (uint32_t)p->tables.size();
  st->scratch_bytes = p->scratch_bytes;
  st->modmuls = p->modmuls;
  st->tune = p->tune;
  st->tiles = 0;
  for (auto& t : p->tables) st->tiles += t.prefix[t.n];
  return PHE_OK;
}

void phe_plan_destroy(phe_plan* p) { destroy_plan(p); }

phe_status phe_autotune(phe_ctx* c, const phe_job* jobs, uint32_t n_jobs, uint32_t flags, uint32_t sample_tokens,
                        void* stream, phe_tuning* best, double* best_ms_per_token) {
  if (!c || !best || (n_jobs && !jobs)) return fail(PHE_EINVAL, "phe_autotune: null argument");
  if (!stream) return fail(PHE_EINVAL, "phe_autotune: needs a non-default stream");
  for (uint32_t i = 0; i < n_jobs; ++i) {
    phe_status st = check_job(c, jobs[i], i);
    if (st != PHE_OK) return st;
  }
  const std::string sig = signature(c, jobs, n_jobs, flags);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto hit = tune_cache().find(sig);
    if (hit != tune_cache().end() && best_ms_per_token == nullptr) {
      *best = hit->second;
      return PHE_OK;
    }
  }
  if (sample_tokens == 0) sample_tokens = 64;
  // The sample: the first `sample_tokens` tokens of every job, same buffers.
  std::vector<phe_job> sample(jobs, jobs + n_jobs);
  uint64_t tokens = 0;
  for (auto& j : sample) {
    j.T = std::min(j.T, sample_tokens);
    tokens += j.T;
  }
  if (tokens == 0) return fail(PHE_EINVAL, "phe_autotune: no tokens");
  DeviceGuard g(c->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t chunks[] = {2, 4, 8, 16, 32, 64};
  // persistent grids first: a tie (their tiles balance through the counter)
  // keeps the single persistent launch
  const uint32_t bps[] = {3, 0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "phe_autotune: events");
  double best_t = 1e30;
  phe_tuning bt{16, 3};
  const bool was_on = c->tracer.on;
  c->tracer.on = false;
  phe_status status = PHE_OK;
  for (uint32_t ch : chunks) {
    for (uint32_t b : bps) {
      phe_tuning tn{ch, b};
      phe_plan* p = nullptr;
      status = phe_plan_create(c, sample.data(), n_jobs, flags, &tn, &p);
      if (status != PHE_OK) break;
      float ms = 0.f, acc = 0.f;
      e = run_plan(p, s, false);  // warm
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = run_plan(p, s, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        acc += ms;
      }
      destroy_plan(p);
      if (e != cudaSuccess) {
        status = cuda_fail(e, "phe_autotune: timing run");
        break;
      }
      if (acc < best_t) {
        best_t = acc;
        bt = tn;
      }
    }
    if (status != PHE_OK) break;
  }
  c->tracer.on = was_on;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != PHE_OK) return status;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    tune_cache()[sig] = bt;
  }
  *best = bt;
  if (best_ms_per_token) *best_ms_per_token = best_t / 2.0 / (double)tokens;
  return PHE_OK;
}

}  // extern "C"
