// Served form of the hot path: continuous batching of encrypted-matmul
// requests from many clients and layers.
//
// A worker thread runs iterations.  Each iteration takes the next token
// chunk of every admitted request that still has tokens (FIFO by arrival),
// as long as the chunk's device buffers fit the memory budget, and runs all
// of them as one batched launch (one input transform per chunk, one lwedot
// launch per group of 32 chunks).  Requests that arrive while others are on
// the GPU join at the next iteration; buffers are reserved per chunk and
// released when the chunk completes, so admission follows free memory.
// Two iterations are kept in flight on the server's stream, so the host
// prepares one while the GPU runs the other.  Every host wait is bounded.
//
// The simulated backend (config.simulate) runs the same scheduler with no
// GPU: a chunk "takes" sim_ns_per_item per (token, row) item.  It exists so
// that admission, ordering, back-pressure and timeouts can be tested on a
// machine without a GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "phe_host.hpp"

using phe::u32;
using phe::u64;
using phe::cuda_fail;
using phe::DeviceGuard;
using phe::fail;
using Clock = std::chrono::steady_clock;

namespace {


double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
  uint64_t id = 0;
  phe_request r{};
  u32 rows = 0, cols = 0, L = 0;
  u32 next_token = 0;   // first token not yet scheduled
  u32 done_tokens = 0;  // tokens whose results are complete
  u32 skips = 0;        // iterations in a row whose budget had no room for its next chunk
  // 0 waiting, 1 active, 2 done, 3 failed, 4 failing: the server failed but
  // work that may still read or write this request's buffers is in flight
  int state = 0;
  Clock::time_point t_submit, t_done;
};

struct ChunkJob {
  uint64_t id;
  u32 t0, tn;
  size_t bytes;    // reserved against the budget
  uint64_t items;  // (token, row) items of the chunk
  u64* ahat = nullptr;
  void* om = nullptr;
  void* ob = nullptr;
};

struct Iteration {
  std::vector<ChunkJob> jobs;
  cudaEvent_t done = nullptr;
  Clock::time_point t_ready;  // simulated backend: when the work "finishes"
};

}  // namespace

struct phe_server {
  phe_ctx* ctx = nullptr;
  phe_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> waiting;
  std::vector<uint64_t> active;
  std::map<uint64_t, Req> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  cudaStream_t stream = nullptr;
  u32* tile_counters = nullptr;  // persistent grids: one per launch group of an iteration
  // accounting
  uint64_t reserved = 0, peak_reserved = 0;
  uint64_t submitted = 0, completed = 0, tokens_completed = 0, iterations = 0, failed = 0;
  std::vector<double> latencies;
  bool have_first = false;
  Clock::time_point t_first, t_last;
  phe_status worker_status = PHE_OK;
};

namespace {

size_t chunk_bytes(const phe_server* s, const Req& q, u32 tn) {
  const size_t N = s->ctx ? s->ctx->prm.N : 1;  // the simulated backend may run without a context
  const size_t osz = s->cfg.flags == PHE_OUT_RAW ? 8 : 4;
  // A_hat, mask and body outputs, and the bodies' digit rows for the body GEMM
  return (size_t)tn * q.L * N * 8 + (size_t)tn * q.rows * N * osz + (size_t)tn * q.rows * osz +
         (q.cols ? phe::digit_bytes(tn, q.cols) : 0);
}

// Iterations in a row a request may be passed over for lack of budget before
// younger requests stop being admitted ahead of it.
constexpr u32 kMaxSkips = 4;

// Build the next iteration (called with the lock held).
void schedule(phe_server* s, Iteration& it) {
  while (!s->waiting.empty() && s->active.size() < s->cfg.max_active) {
    const uint64_t id = s->waiting.front();
    s->waiting.pop_front();
    s->reqs[id].state = 1;
    s->active.push_back(id);
  }
  for (uint64_t id : s->active) {
    if (it.jobs.size() >= s->cfg.max_jobs_per_iteration) break;
    Req& q = s->reqs[id];
    if (q.next_token >= q.r.T) continue;
    const u32 tn = std::min(s->cfg.chunk_tokens, q.r.T - q.next_token);
    const size_t need = chunk_bytes(s, q, tn);
    if (s->reserved + need > s->cfg.mem_budget_bytes) {
      // A smaller chunk of a younger request may still fit, unless this
      // request has been passed over too often: then nothing younger is
      // admitted until its chunk fits, so its wait stays bounded.
      if (++q.skips >= kMaxSkips) break;
      continue;
    }
    q.skips = 0;
    s->reserved += need;
    s->peak_reserved = std::max(s->peak_reserved, s->reserved);
    it.jobs.push_back({id, q.next_token, tn, need, (uint64_t)tn * q.rows});
    q.next_token += tn;
  }
}

// Frees the chunk buffers of an iteration that could not be launched whole.
void release_jobs(phe_server* s, Iteration& it) {
  for (auto& j : it.jobs) {
    if (j.ahat) cudaFreeAsync(j.ahat, s->stream);
    if (j.om) cudaFreeAsync(j.om, s->stream);
    if (j.ob) cudaFreeAsync(j.ob, s->stream);
    j.ahat = nullptr;
    j.om = j.ob = nullptr;
  }
}

cudaError_t launch_iteration(phe_server* s, Iteration& it) {
  phe_ctx* c = s->ctx;
  const u32 N = c->prm.N;
  const size_t osz = s->cfg.flags == PHE_OUT_RAW ? 8 : 4;
  cudaError_t e = cudaSuccess;
  std::vector<phe::LweJobTable> tables(1);
  for (auto& j : it.jobs) {
    Req* q;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      q = &s->reqs[j.id];
    }
    const phe_weights::Dir& D = q->r.w->dir[q->r.dir];
    if ((e = phe::ctx_malloc_async(s->ctx, &j.ahat, (size_t)j.tn * D.L * N * 8, s->stream)) != cudaSuccess) break;
    if ((e = phe::ctx_malloc_async(s->ctx, &j.om, (size_t)j.tn * D.rows * N * osz, s->stream)) != cudaSuccess) break;
    if ((e = phe::ctx_malloc_async(s->ctx, &j.ob, (size_t)j.tn * D.rows * osz, s->stream)) != cudaSuccess) break;
    const size_t tok_words = (size_t)D.L * N;
    phe::NttJob nj{nullptr, j.ahat, j.tn * D.L};
    if (q->r.d_in_seeds)
      nj.seeds = reinterpret_cast<const u64*>(q->r.d_in_seeds) + (size_t)j.t0 * D.L;
    else
      nj.src = reinterpret_cast<const u64*>(q->r.d_in_mask) + (size_t)j.t0 * tok_words;
    if ((e = phe::launch_input_ntt(c, &nj, 1, s->stream)) != cudaSuccess) break;
    phe::LweJobTable& t = tables.back();
    phe::LweJob& J = t.j[t.n];
    J = phe::LweJob{};
    J.what = D.what;
    J.ahat = j.ahat;
    J.out = j.om;
    J.wrow = D.wrow;
    J.wbf = D.wbf;
    J.bin = reinterpret_cast<const u64*>(q->r.d_in_body) + (size_t)j.t0 * tok_words;
    J.out_body = j.ob;
    J.rows = D.rows;
    J.cols = D.cols;
    J.T = j.tn;
    J.L = D.L;
    J.tok_chunk = s->cfg.tok_chunk;
    phe::set_lwe_tiles(J, c->logn);
    t.prefix[t.n + 1] = t.prefix[t.n] + J.tiles;
    if (++t.n == phe::kMaxJobs) tables.emplace_back();
  }
  const int mode = s->cfg.flags == PHE_OUT_RAW ? phe::kOutRaw : phe::kOutSwitched;
  for (auto& t : tables) {
    if (e != cudaSuccess) break;
    if (!t.n) continue;
    const u32 tiles = t.prefix[t.n];
    const u32 grid = s->cfg.blocks_per_sm ? std::min(tiles, (u32)c->num_sms * s->cfg.blocks_per_sm) : tiles;
    t.tile_counter = s->tile_counters ? s->tile_counters + (&t - tables.data()) : nullptr;
    const bool gemm = phe::body_on_tensor_cores(c, t);
    if (!gemm) {
      if ((e = phe::launch_lwedot(c, t, mode, (int)grid, s->stream)) != cudaSuccess) break;
      continue;
    }
    // the bodies' digit rows live for this table's launches only
    void* dig = nullptr;
    if ((e = phe::ctx_malloc_async(s->ctx, &dig, phe::body_scratch_bytes(t), s->stream)) != cudaSuccess) break;
    phe::assign_body_scratch(t, dig);
    e = phe::launch_body(c, t, mode == phe::kOutRaw, c->rc, c->rk, s->stream);
    if (e == cudaSuccess) e = phe::launch_lwedot(c, t, mode | phe::kBodyGemm, (int)grid, s->stream);
    cudaFreeAsync(dig, s->stream);
  }
  if (e != cudaSuccess) {
    release_jobs(s, it);
    return e;
  }
  // deliver: results of each chunk to the request's host buffers (if any)
  for (auto& j : it.jobs) {
    Req* q;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      q = &s->reqs[j.id];
    }
    if (q->r.h_out_mask) {
      char* hm = static_cast<char*>(q->r.h_out_mask) + (size_t)j.t0 * q->rows * N * osz;
      char* hb = static_cast<char*>(q->r.h_out_body) + (size_t)j.t0 * q->rows * osz;
      if ((e = cudaMemcpyAsync(hm, j.om, (size_t)j.tn * q->rows * N * osz, cudaMemcpyDeviceToHost, s->stream)) !=
          cudaSuccess)
        break;
      if ((e = cudaMemcpyAsync(hb, j.ob, (size_t)j.tn * q->rows * osz, cudaMemcpyDeviceToHost, s->stream)) !=
          cudaSuccess)
        break;
    }
  }
  release_jobs(s, it);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&it.done, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaEventRecord(it.done, s->stream);
}

// Wait for an iteration with a bound; true when it completed.
bool wait_iteration(phe_server* s, Iteration& it, phe_status* st) {
  const auto deadline = Clock::now() + std::chrono::milliseconds(s->cfg.wait_timeout_ms);
  if (s->cfg.simulate) {
    std::this_thread::sleep_until(std::min(it.t_ready, deadline));
    if (Clock::now() < it.t_ready) {
      *st = fail(PHE_ETIMEOUT, "phe_server: iteration did not finish within %u ms", s->cfg.wait_timeout_ms);
      return false;
    }
    return true;
  }
  for (;;) {
    cudaError_t e = cudaEventQuery(it.done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      *st = fail(PHE_ECUDA, "phe_server: %s", cudaGetErrorString(e));
      return false;
    }
    if (Clock::now() > deadline) {
      *st = fail(PHE_ETIMEOUT, "phe_server: iteration did not finish within %u ms", s->cfg.wait_timeout_ms);
      return false;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  cudaEventDestroy(it.done);
  return true;
}

void complete_iteration(phe_server* s, Iteration& it) {
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& j : it.jobs) {
    Req& q = s->reqs[j.id];
    s->reserved -= j.bytes;
    q.done_tokens += j.tn;
    if (q.done_tokens == q.r.T && q.state == 1) {
      q.state = 2;
      q.t_done = now;
      s->completed++;
      s->tokens_completed += q.r.T;
      s->latencies.push_back(ms_since(q.t_submit, now));
      s->active.erase(std::remove(s->active.begin(), s->active.end(), j.id), s->active.end());
    }
  }
  s->t_last = now;
  s->iterations++;
  s->cv_done.notify_all();
}

// The server failed: no request is admitted or scheduled any more.  Requests
// not yet done become "failing"; they are reported failed only once the work
// in flight -- which may still read their inputs and write their host
// buffers -- has drained (drain_and_fail).
void begin_failure(phe_server* s, phe_status st) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->worker_status = st;
  for (auto& kv : s->reqs)
    if (kv.second.state < 2) kv.second.state = 4;
  s->waiting.clear();
  s->active.clear();
}

// Waits, with a bound, until every iteration in flight has finished on the
// device (the simulated backend: until its finishing time), then reports
// the failing requests failed.  If the work does not drain within the bound
// the requests stay failing: their waits time out, and their buffers must
// stay valid until phe_server_destroy, which synchronises the stream.
void drain_and_fail(phe_server* s, std::deque<Iteration>& inflight) {
  const auto limit = std::chrono::milliseconds(std::max<uint64_t>(4ull * s->cfg.wait_timeout_ms, 3000));
  const auto deadline = Clock::now() + limit;
  bool drained = true;
  if (s->cfg.simulate) {
    for (auto& it : inflight) {
      if (it.t_ready > deadline) {
        drained = false;
        break;
      }
      std::this_thread::sleep_until(it.t_ready);
    }
  } else {
    for (;;) {
      const cudaError_t e = cudaStreamQuery(s->stream);
      if (e != cudaErrorNotReady) break;  // drained, or the stream itself failed (nothing runs any more)
      if (Clock::now() > deadline) {
        drained = false;
        break;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(500));
    }
    if (drained)
      for (auto& it : inflight)
        if (it.done) cudaEventDestroy(it.done);
  }
  inflight.clear();
  std::lock_guard<std::mutex> lk(s->mu);
  if (drained) {
    for (auto& kv : s->reqs)
      if (kv.second.state == 4) {
        kv.second.state = 3;
        s->failed++;
      }
  }
  s->cv_done.notify_all();
}

void worker_main(phe_server* s) {
  if (!s->cfg.simulate) cudaSetDevice(s->ctx->device);
  std::deque<Iteration> inflight;
  for (;;) {
    Iteration it;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      schedule(s, it);
      if (it.jobs.empty() && inflight.empty()) {
        if (s->stop && s->waiting.empty() && s->active.empty()) return;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      if (!it.jobs.empty() && !s->have_first) {
        s->have_first = true;
        s->t_first = Clock::now();
      }
    }
    const bool launched = !it.jobs.empty();
    if (launched) {
      if (s->cfg.simulate) {
        uint64_t items = 0;
        for (auto& j : it.jobs) items += j.items;
        const auto start = inflight.empty() ? Clock::now() : std::max(Clock::now(), inflight.back().t_ready);
        it.t_ready = start + std::chrono::nanoseconds((uint64_t)(s->cfg.sim_ns_per_item * (double)items));
      } else {
        cudaError_t e = launch_iteration(s, it);
        if (e != cudaSuccess) {
          begin_failure(s, fail(PHE_ECUDA, "phe_server: launch: %s", cudaGetErrorString(e)));
          drain_and_fail(s, inflight);
          return;
        }
      }
      inflight.push_back(std::move(it));
    }
    // keep two iterations in flight; otherwise complete the oldest
    if (inflight.size() >= 2 || (!inflight.empty() && !launched)) {
      phe_status st = PHE_OK;
      if (!wait_iteration(s, inflight.front(), &st)) {
        begin_failure(s, st);
        drain_and_fail(s, inflight);
        return;
      }
      complete_iteration(s, inflight.front());
      inflight.pop_front();
    }
  }
}

}  // namespace

extern "C" {

phe_status phe_server_create(phe_ctx* c, const phe_server_config* cfg, phe_server** out) {
  if (!cfg || !out) return fail(PHE_EINVAL, "phe_server_create: null argument");
  *out = nullptr;
  if (!cfg->simulate && !c) return fail(PHE_EINVAL, "phe_server_create: null context");
  if (cfg->chunk_tokens < 1 || cfg->max_active < 1 || cfg->max_jobs_per_iteration < 1 || cfg->mem_budget_bytes == 0 ||
      cfg->tok_chunk < 1 || cfg->max_queue < 1 || cfg->wait_timeout_ms < 1)
    return fail(PHE_EINVAL, "phe_server_create: a size in the config is zero");
  if (cfg->flags != PHE_OUT_SWITCHED && cfg->flags != PHE_OUT_RAW) return fail(PHE_EINVAL, "phe_server_create: flags");
  phe_server* s = new phe_server();
  s->ctx = c;
  s->cfg = *cfg;
  if (!cfg->simulate) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaError_t e = phe::prepare_launches(c);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    // launch groups of up to kMaxJobs chunks: counters for every group an iteration can have
    const size_t groups = cfg->max_jobs_per_iteration / phe::kMaxJobs + 1;
    if (e == cudaSuccess && cfg->blocks_per_sm) e = cudaMalloc(&s->tile_counters, groups * sizeof(u32));
    if (e != cudaSuccess) {
      if (s->stream) cudaStreamDestroy(s->stream);
      if (prev >= 0) cudaSetDevice(prev);
      delete s;
      return fail(PHE_ECUDA, "phe_server_create: %s", cudaGetErrorString(e));
    }
    if (prev >= 0) cudaSetDevice(prev);
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return PHE_OK;
}

phe_status phe_server_submit(phe_server* s, const phe_request* r, uint64_t* id) {
  if (!s || !r || !id) return fail(PHE_EINVAL, "phe_server_submit: null argument");
  Req q;
  q.r = *r;
  if (!s->cfg.simulate) {
    if (!r->w || r->w->ctx != s->ctx) return fail(PHE_EINVAL, "phe_server_submit: weights of another context");
    if (r->dir != PHE_FWD && r->dir != PHE_BWD) return fail(PHE_EINVAL, "phe_server_submit: bad direction");
    if (!(r->w->dirs & (1u << r->dir))) return fail(PHE_EINVAL, "phe_server_submit: direction not uploaded");
    if (r->T && ((!r->d_in_mask && !r->d_in_seeds) || !r->d_in_body))
      return fail(PHE_EINVAL, "phe_server_submit: null input");
    if ((r->h_out_mask == nullptr) != (r->h_out_body == nullptr))
      return fail(PHE_EINVAL, "phe_server_submit: give both host outputs or neither");
    const phe_weights::Dir& D = r->w->dir[r->dir];
    q.rows = D.rows;
    q.cols = D.cols;
    q.L = D.L;
  } else {
    q.rows = r->sim_rows ? r->sim_rows : 1;
    q.L = 1;
  }
  if (r->T > (1u << 24)) return fail(PHE_EINVAL, "phe_server_submit: T too large");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->worker_status != PHE_OK) return fail(s->worker_status, "phe_server_submit: server failed earlier");
  if (s->stop) return fail(PHE_EINVAL, "phe_server_submit: server is stopping");
  const size_t one = chunk_bytes(s, q, std::min(s->cfg.chunk_tokens, std::max(r->T, 1u)));
  if (one > s->cfg.mem_budget_bytes)
    return fail(PHE_ENOMEM, "phe_server_submit: one chunk (%zu bytes) exceeds the memory budget", one);
  if (s->waiting.size() >= s->cfg.max_queue) return fail(PHE_EBUSY, "phe_server_submit: queue full");
  q.id = s->next_id++;
  q.t_submit = Clock::now();
  s->submitted++;
  if (r->T == 0) {
    q.state = 2;
    q.t_done = q.t_submit;
    s->completed++;
    s->latencies.push_back(0.0);
    s->reqs[q.id] = q;
  } else {
    s->reqs[q.id] = q;
    s->waiting.push_back(q.id);
  }
  *id = q.id;
  s->cv_work.notify_one();
  return PHE_OK;
}

phe_status phe_server_wait(phe_server* s, uint64_t id, uint32_t timeout_ms, double* latency_ms) {
  if (!s) return fail(PHE_EINVAL, "phe_server_wait: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(PHE_EINVAL, "phe_server_wait: unknown request %llu", (unsigned long long)id);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [&] { return it->second.state == 2 || it->second.state == 3; });
  if (!ok) return fail(PHE_ETIMEOUT, "phe_server_wait: request %llu not done after %u ms", (unsigned long long)id,
                       timeout_ms);
  if (it->second.state == 3) return fail(s->worker_status, "phe_server_wait: request failed");
  if (latency_ms) *latency_ms = ms_since(it->second.t_submit, it->second.t_done);
  return PHE_OK;
}

phe_status phe_server_poll(phe_server* s, uint64_t id, int* done, double* latency_ms) {
  if (!s || !done) return fail(PHE_EINVAL, "phe_server_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(PHE_EINVAL, "phe_server_poll: unknown request");
  *done = it->second.state == 2 ? 1 : (it->second.state == 3 ? -1 : 0);
  if (latency_ms && it->second.state == 2) *latency_ms = ms_since(it->second.t_submit, it->second.t_done);
  return PHE_OK;
}

phe_status phe_server_stats(phe_server* s, phe_serving_stats* st) {
  if (!s || !st) return fail(PHE_EINVAL, "phe_server_stats: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->tokens_completed = s->tokens_completed;
  st->iterations = s->iterations;
  st->waiting = s->waiting.size();
  st->active = s->active.size();
  st->reserved_bytes = s->reserved;
  st->peak_reserved_bytes = s->peak_reserved;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto rank = [&](double p) {
      size_t i = (size_t)std::ceil(p * v.size());
      return v[i ? i - 1 : 0];
    };
    st->p50_ms = rank(0.50);
    st->p99_ms = rank(0.99);
    st->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_ms = sum / v.size();
  }
  if (s->have_first) st->busy_ms = ms_since(s->t_first, s->t_last);
  return PHE_OK;
}

void phe_server_destroy(phe_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->stream) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  if (s->tile_counters) cudaFree(s->tile_counters);
  delete s;
}

}  // extern "C"
