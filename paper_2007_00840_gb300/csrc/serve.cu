// Serving: continuous batching of incoming sparsity patterns.
//
// Requests are admitted in arrival order while their projected device memory
// (CSR copy, per-row workspace, row pool and outputs, global-tier label slots
// for large orders) fits under the configured cap.  Each of `streams` stream
// slots has a dispatcher thread that takes the admitted requests waiting at
// that moment (up to max_batch) and runs them as one batch (the multi-matrix
// traversal of gsofa_batch, with pooled workspace).  While one slot's batch is
// on the GPU the other slot gathers the requests that arrived meanwhile and
// launches them behind it (its CTAs start as the running batch's CTAs retire,
// and its size read-back and output assembly overlap the other batch's
// traversal), so requests start as soon as a slot and memory free up.  Latency
// is measured from submission to completion of the result.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gsofa.h"
#include "internal.cuh"

using Clock = std::chrono::steady_clock;

namespace gsofa {
namespace {

struct Request {
  uint64_t ticket = 0;
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rp = nullptr;      // device CSR used by the kernels
  const int32_t* ci = nullptr;
  const int32_t* h_rp = nullptr;    // host CSR to copy in (on_device == 0)
  const int32_t* h_ci = nullptr;
  int32_t* own = nullptr;           // server copy of a host CSR (rowptr then colidx)
  int64_t projected = 0;
  int64_t budget = 0;               // space-budget mode: mem_budget_bytes of this request (0: server default)
  Clock::time_point t_submit, t_done;
  bool done = false;
  int status = GSOFA_OK;
  gsofa_result res;
};

}  // namespace
}  // namespace gsofa

using namespace gsofa;

struct gsofa_server {
  gsofa_server_config cfg;
  int device = 0;
  int sms = 0;
  int32_t smem_max_n = 0;
  cudaMemPool_t mpool = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending, ready;
  std::unordered_map<uint64_t, Request*> live;
  int64_t in_use = 0;
  int32_t inflight = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  // statistics
  int64_t completed = 0, failed = 0, batches = 0, total_nnz = 0, total_rows = 0, launches = 0;
  int64_t peak_in_use = 0;
  std::vector<float> lat_ms;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace {

int64_t projected_bytes(const gsofa_server* S, int32_t n, int64_t nnz, bool host_input) {
  const int64_t csr = host_input ? 4 * ((int64_t)n + 1) + 4 * nnz : 0;
  const int64_t rows = 96 * (int64_t)n;                        // per-row workspace, scans, row pointers
  int64_t est = 64 * nnz + 16 * (int64_t)n;                    // projected nnz(L+U)
  const int64_t full = (int64_t)n * ((int64_t)n + 1);
  if (est > full) est = full;
  int64_t b = csr + rows + 8 * est + (1 << 20);                // row pool + L/U outputs
  if (n > S->smem_max_n) b += global_tier_bytes(n, &S->cfg.opts);  // global-tier slots, as a call would size them
  return b;
}

// Move pending requests to the ready queue while they fit.  Caller holds mu.
void admit(gsofa_server* S) {
  while (!S->pending.empty()) {
    Request* r = S->pending.front();
    if (S->inflight >= S->cfg.max_inflight || S->in_use + r->projected > S->cfg.mem_cap_bytes) break;
    S->pending.pop_front();
    S->in_use += r->projected;
    if (S->in_use > S->peak_in_use) S->peak_in_use = S->in_use;
    S->inflight++;
    S->ready.push_back(r);
  }
}

void worker_loop(gsofa_server* S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t st = S->streams[slot];
  std::vector<Request*> take;
  std::vector<int32_t> ns;
  std::vector<const int32_t*> rps, cis;
  std::vector<gsofa_result> outs;
  for (;;) {
    take.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->ready.empty() && S->stop) return;
      while (!S->ready.empty() && (int)take.size() < S->cfg.max_batch) {
        take.push_back(S->ready.front());
        S->ready.pop_front();
      }
    }
    // host inputs: copy into pooled device memory on this slot's stream
    const int k = (int)take.size();
    std::vector<int> rcs(k, GSOFA_OK);
    for (int i = 0; i < k; i++) {
      Request* r = take[i];
      if (!r->h_rp) continue;
      const size_t words = (size_t)r->n + 1 + (size_t)r->nnz;
      if (cudaMallocFromPoolAsync((void**)&r->own, 4 * (words > 0 ? words : 1), S->mpool, st) != cudaSuccess ||
          cudaMemcpyAsync(r->own, r->h_rp, 4 * ((size_t)r->n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          (r->nnz > 0 && cudaMemcpyAsync(r->own + r->n + 1, r->h_ci, 4 * (size_t)r->nnz, cudaMemcpyHostToDevice,
                                         st) != cudaSuccess)) {
        cudaGetLastError();
        rcs[i] = GSOFA_E_NOMEM;
        continue;
      }
      r->rp = r->own;
      r->ci = r->own + r->n + 1;
    }
    outs.assign(k, gsofa_result());
    // requests admitted in space-budget mode run alone with their own budget;
    // the others run as one batch
    ns.clear();
    rps.clear();
    cis.clear();
    std::vector<int> in_batch;
    for (int i = 0; i < k; i++) {
      if (take[i]->budget > 0 || rcs[i] != GSOFA_OK) continue;
      in_batch.push_back(i);
      ns.push_back(take[i]->n);
      rps.push_back(take[i]->rp);
      cis.push_back(take[i]->ci);
    }
    int64_t launches = 0;
    auto run_alone = [&](int i, const gsofa_options& o) {
      const int32_t n1 = take[i]->n;
      const int32_t* rp1 = take[i]->rp;
      const int32_t* ci1 = take[i]->ci;
      rcs[i] = batch_transient(1, &n1, &rp1, &ci1, &o, st, &outs[i]);
      if (rcs[i] == GSOFA_OK) launches += outs[i].stats.kernel_launches;
    };
    if (!in_batch.empty()) {
      std::vector<gsofa_result> bo(in_batch.size());
      const int brc =
          batch_transient((int32_t)in_batch.size(), ns.data(), rps.data(), cis.data(), &S->cfg.opts, st, bo.data());
      if (brc == GSOFA_OK) {
        launches += bo[0].stats.kernel_launches;  // the batch's total
        for (size_t j = 0; j < in_batch.size(); j++) outs[in_batch[j]] = bo[j];
      } else if (brc == GSOFA_E_INVAL && in_batch.size() > 1) {
        // a malformed pattern rejects the whole batch: run the members one by
        // one so that only the offending request fails, as it would alone
        for (int i : in_batch) run_alone(i, S->cfg.opts);
      } else {
        for (int i : in_batch) rcs[i] = brc;
      }
    }
    for (int i = 0; i < k; i++) {
      if (take[i]->budget == 0 || rcs[i] != GSOFA_OK) continue;
      gsofa_options o = S->cfg.opts;
      o.mem_budget_bytes = take[i]->budget;
      run_alone(i, o);
    }
    const int wrc = wait_stream(st);  // results complete
    for (int i = 0; i < k; i++) {
      if (rcs[i] == GSOFA_OK && wrc != GSOFA_OK) rcs[i] = wrc;
      if (rcs[i] != GSOFA_OK) gsofa_free(&outs[i]);
      else detach_result_stream(&outs[i]);  // results are freed stream-less
    }
    const Clock::time_point now = Clock::now();
    for (Request* r : take)
      if (r->own) {
        cudaFreeAsync(r->own, st);
        r->own = nullptr;
      }
    std::lock_guard<std::mutex> lk(S->mu);
    S->batches++;
    S->launches += launches;
    for (int i = 0; i < k; i++) {
      Request* r = take[i];
      r->t_done = now;
      r->status = rcs[i];
      if (rcs[i] == GSOFA_OK) {
        r->res = outs[i];
        S->completed++;
        S->total_nnz += outs[i].nnz_L + outs[i].nnz_U;
        S->total_rows += outs[i].n;
        S->lat_ms.push_back(std::chrono::duration<float, std::milli>(now - r->t_submit).count());
      } else {
        std::memset(&r->res, 0, sizeof(r->res));
        S->failed++;
      }
      r->done = true;
      S->in_use -= r->projected;
      S->inflight--;
    }
    S->t_last = now;
    admit(S);
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
}

float percentile(std::vector<float> v, double q) {
  if (v.empty()) return 0.f;
  std::sort(v.begin(), v.end());
  size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
  if (i >= v.size()) i = v.size() - 1;
  return v[i];
}

}  // namespace

extern "C" {

int gsofa_server_default_config(gsofa_server_config* cfg) {
  if (!cfg) return GSOFA_E_INVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->mem_cap_bytes = (int64_t)150 << 30;
  cfg->max_inflight = 8192;
  cfg->streams = 2;
  cfg->max_batch = 512;
  cfg->queue_capacity = 1 << 20;
  gsofa_default_options(&cfg->opts);
  return GSOFA_OK;
}

int gsofa_server_create(const gsofa_server_config* cfg, gsofa_server** out) {
  if (!out) return GSOFA_E_INVAL;
  *out = nullptr;
  gsofa_server* S = new gsofa_server();
  if (cfg) S->cfg = *cfg; else gsofa_server_default_config(&S->cfg);
  gsofa_server_config def;
  gsofa_server_default_config(&def);
  if (S->cfg.mem_cap_bytes <= 0) S->cfg.mem_cap_bytes = def.mem_cap_bytes;
  if (S->cfg.max_inflight <= 0) S->cfg.max_inflight = def.max_inflight;
  if (S->cfg.streams <= 0) S->cfg.streams = def.streams;
  if (S->cfg.streams > 16) S->cfg.streams = 16;
  if (S->cfg.max_batch <= 0) S->cfg.max_batch = def.max_batch;
  if (S->cfg.queue_capacity <= 0) S->cfg.queue_capacity = def.queue_capacity;
  if (S->cfg.opts.chunk_size == 0) S->cfg.opts.chunk_size = 128;
  if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return GSOFA_E_CUDA; }
  S->sms = device_sms();
  S->smem_max_n = smem_tier_max_order();
  if (S->sms <= 0) { delete S; return GSOFA_E_CUDA; }
  {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->mpool, &props) != cudaSuccess) { delete S; return GSOFA_E_CUDA; }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(S->mpool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  for (int i = 0; i < S->cfg.streams; i++) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
      cudaMemPoolDestroy(S->mpool);
      delete S;
      return GSOFA_E_CUDA;
    }
    S->streams.push_back(st);
  }
  for (int i = 0; i < S->cfg.streams; i++) S->workers.emplace_back(worker_loop, S, i);
  *out = S;
  return GSOFA_OK;
}

int gsofa_server_submit(gsofa_server* S, int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t on_device,
                        uint64_t* ticket) {
  if (!S || !ticket || n < 0 || !rowptr || (n > 0 && !colidx)) return GSOFA_E_INVAL;
  Request* r = new Request();
  r->n = n;
  if (on_device) {
    int32_t last = 0;
    if (cudaMemcpy(&last, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete r;
      return GSOFA_E_CUDA;
    }
    r->nnz = last;
    r->rp = rowptr;
    r->ci = colidx;
  } else {
    r->nnz = rowptr[n];
    r->h_rp = rowptr;
    r->h_ci = colidx;
  }
  if (r->nnz < 0) { delete r; return GSOFA_E_INVAL; }
  r->projected = projected_bytes(S, n, r->nnz, !on_device);
  if (r->projected > S->cfg.mem_cap_bytes && n > S->smem_max_n) {
    // space-budget mode (the concurrent-source budget of Section 5, Eq. 1): run
    // the request with as many global-tier slots as the cap leaves room for
    const int64_t base = r->projected - global_tier_bytes(n, &S->cfg.opts);
    const int64_t one = global_slot_bytes(n);
    const int64_t slots = one > 0 ? (S->cfg.mem_cap_bytes - base) / one : 0;
    if (slots >= 1) {
      r->budget = 2 * slots * one;  // the global tier takes half of mem_budget_bytes
      r->projected = base + slots * one;
    }
  }
  if (r->projected > S->cfg.mem_cap_bytes) { delete r; return GSOFA_E_NOMEM; }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) { delete r; return GSOFA_E_INVAL; }
  if ((int64_t)S->pending.size() >= S->cfg.queue_capacity) { delete r; return GSOFA_E_BUSY; }
  r->ticket = S->next_ticket++;
  r->t_submit = Clock::now();
  if (!S->have_first) { S->have_first = true; S->t_first = r->t_submit; }
  S->live[r->ticket] = r;
  S->pending.push_back(r);
  admit(S);
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return GSOFA_OK;
}

static int take_result(gsofa_server* S, std::unordered_map<uint64_t, Request*>::iterator it, gsofa_result* out,
                       double* latency_ms) {
  Request* r = it->second;
  const int st = r->status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  if (out) *out = r->res; else gsofa_free(&r->res);
  S->live.erase(it);
  delete r;
  return st;
}

int gsofa_server_poll(gsofa_server* S, uint64_t ticket, gsofa_result* out, double* latency_ms) {
  if (!S) return GSOFA_E_INVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) return GSOFA_E_NOTFOUND;
  if (!it->second->done) return GSOFA_E_PENDING;
  return take_result(S, it, out, latency_ms);
}

int gsofa_server_wait(gsofa_server* S, uint64_t ticket, double timeout_s, gsofa_result* out, double* latency_ms) {
  if (!S) return GSOFA_E_INVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) return GSOFA_E_NOTFOUND;
  Request* r = it->second;
  const auto limit = std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 600.0);
  if (!S->cv_done.wait_for(lk, limit, [&] { return r->done; })) return GSOFA_E_TIMEOUT;
  return take_result(S, S->live.find(ticket), out, latency_ms);
}

int gsofa_server_get_stats(gsofa_server* S, gsofa_server_stats* st) {
  if (!S || !st) return GSOFA_E_INVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->completed = S->completed;
  st->failed = S->failed;
  st->batches = S->batches;
  st->pending = (int64_t)S->pending.size();
  st->inflight = S->inflight;
  st->kernel_launches = (int32_t)std::min<int64_t>(S->launches, INT32_MAX);
  st->total_nnz = S->total_nnz;
  st->total_rows = S->total_rows;
  st->mem_in_use = S->in_use;
  st->peak_mem_in_use = S->peak_in_use;
  st->p50_ms = percentile(S->lat_ms, 0.50);
  st->p99_ms = percentile(S->lat_ms, 0.99);
  st->max_ms = percentile(S->lat_ms, 1.0);
  st->span_s = S->have_first ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
  return GSOFA_OK;
}

void gsofa_server_destroy(gsofa_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    // requests never admitted are dropped
    for (Request* r : S->pending) {
      S->live.erase(r->ticket);
      delete r;
    }
    S->pending.clear();
  }
  S->cv_work.notify_all();
  for (std::thread& t : S->workers) t.join();
  for (auto& kv : S->live) {
    gsofa_free(&kv.second->res);
    delete kv.second;
  }
  for (cudaStream_t st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaMemPoolDestroy(S->mpool);
  delete S;
}

}  // extern "C"
