// Serving: continuous batching of incoming sparsity patterns.
//
// Requests are admitted in arrival order while their projected device memory
// (CSR copy, per-row workspace, row pool and outputs) fits under the configured
// cap; the class-kernel slots of a batch or of a large request are charged
// while that work runs (fewer slots when the cap leaves less room), not while
// it waits.  Admitted requests wait in two
// queues: batchable ones (orders whose visited bitmaps fit on chip) and large
// ones.  Each of `streams` stream slots has a dispatcher thread; a free slot
// takes whichever queue holds the oldest request: every batchable request
// waiting at that moment (up to max_batch) as one batch (the multi-matrix
// traversal of gsofa_batch, with pooled workspace), or one large request alone
// on a high-priority stream and half of the traversal CTAs.  So a large request
// occupies one slot and part of the GPU while the others keep serving batches,
// instead of holding up the small requests batched with it.  While one slot's
// work is on the GPU another gathers the requests that arrived meanwhile and
// launches them beside it.  A batch's class-kernel slots are charged against
// the cap while it runs (fewer slots when the cap leaves less room).  Latency
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

// Device bytes of the results of one batch (or one large request), charged
// against the cap from completion until the last of them is collected: batch
// results share one block that is freed with the last member.
struct Charge {
  int64_t bytes = 0;
  int refs = 0;
};

struct Request {
  uint64_t ticket = 0;
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rp = nullptr;      // device CSR used by the kernels
  const int32_t* ci = nullptr;
  const int32_t* h_rp = nullptr;    // host CSR to copy in (on_device == 0)
  const int32_t* h_ci = nullptr;
  int32_t* own = nullptr;           // server copy of a host CSR (rowptr then colidx)
  int64_t projected = 0;             // bytes with the class slots of a large request
  int64_t slot_part = 0;             // of which class slots: charged while the request runs, not while it waits
  int64_t slot_one = 0;              // bytes of one of those slots
  int64_t est = 0;                  // projected nnz(L+U): the first row-pool size of its batch share
  int64_t budget = 0;               // space-budget mode: mem_budget_bytes of this request (0: server default)
  bool big = false;                 // runs alone (order above the on-chip limit)
  Charge* held = nullptr;           // result bytes charged until collected
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
  std::deque<Request*> pending, ready_small, ready_big;
  std::unordered_map<uint64_t, Request*> live;
  int64_t in_use = 0;
  int32_t inflight = 0;
  int32_t big_running = 0;                 // large requests on the GPU (at most one)
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;       // per slot: batches
  std::vector<cudaStream_t> streams_hi;    // per slot: large requests, at the highest stream priority
  // statistics
  int64_t completed = 0, failed = 0, batches = 0, total_nnz = 0, total_rows = 0, launches = 0;
  int64_t peak_in_use = 0;
  // device memory actually held: library pool at start, class slots at start, peak seen
  int64_t pool_base = 0, slots_base = 0, peak_device = 0;
  std::vector<float> lat_ms;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace {

// Projected nnz(L+U) of a pattern: 64 per stored entry plus 16 per row, at most
// the full triangle pair.
int64_t projected_entries(int32_t n, int64_t nnz) {
  int64_t est = 64 * nnz + 16 * (int64_t)n;
  const int64_t full = (int64_t)n * ((int64_t)n + 1);
  return est > full ? full : est;
}

int64_t projected_bytes(const gsofa_server* S, int32_t n, int64_t nnz, bool host_input) {
  const int64_t csr = host_input ? 4 * ((int64_t)n + 1) + 4 * nnz : 0;
  const int64_t rows = 96 * (int64_t)n;                        // per-row workspace, scans, row pointers
  const int64_t est = projected_entries(n, nnz);
  int64_t b = csr + rows + 8 * est + (1 << 20);                // row pool + L/U outputs
  if (n > S->smem_max_n) b += global_tier_bytes(n, &S->cfg.opts);  // global-tier slots, as a call would size them
  return b;
}

// Move pending requests to the ready queue while they fit.  Caller holds mu.
void admit(gsofa_server* S) {
  while (!S->pending.empty()) {
    Request* r = S->pending.front();
    const int64_t charge = r->projected - r->slot_part;
    if (S->inflight >= S->cfg.max_inflight || S->in_use + charge > S->cfg.mem_cap_bytes) break;
    S->pending.pop_front();
    S->in_use += charge;
    if (S->in_use > S->peak_in_use) S->peak_in_use = S->in_use;
    S->inflight++;
    (r->big ? S->ready_big : S->ready_small).push_back(r);
  }
}

// Device memory the server's work holds beyond what was held when it started:
// the library pool's high-water mark, class slots it made the library keep,
// and its own pool (host inputs).  Caller holds mu.
void sample_device(gsofa_server* S) {
  int64_t lib = library_pool_bytes(1, 0) - S->pool_base;
  if (lib < 0) lib = 0;
  int64_t slots = library_slot_bytes() - S->slots_base;
  if (slots < 0) slots = 0;
  uint64_t own = 0;
  if (cudaMemPoolGetAttribute(S->mpool, cudaMemPoolAttrUsedMemHigh, &own) != cudaSuccess) {
    cudaGetLastError();
    own = 0;
  }
  const int64_t d = lib + slots + (int64_t)own;
  if (d > S->peak_device) S->peak_device = d;
}

void worker_loop(gsofa_server* S, int slot) {
  cudaSetDevice(S->device);
  std::vector<Request*> take;
  std::vector<int32_t> ns;
  std::vector<const int32_t*> rps, cis;
  std::vector<gsofa_result> outs;
  for (;;) {
    take.clear();
    int64_t reserved = 0;   // class-slot bytes of a batch, charged while it runs
    int32_t batch_slots = 0;
    int64_t big_budget = 0;  // a large request's memory budget when the cap leaves fewer slots
    bool small = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // one large request at a time: large requests share the library's class
      // slots, so a second one would only wait for them on this slot's thread
      auto big_ok = [&] { return !S->ready_big.empty() && S->big_running == 0; };
      S->cv_work.wait(lk, [&] {
        return (S->stop && S->ready_small.empty() && S->ready_big.empty()) || !S->ready_small.empty() || big_ok();
      });
      if (S->ready_small.empty() && S->ready_big.empty() && S->stop) return;
      // the queue with the oldest request goes first
      small = !S->ready_small.empty() &&
              (!big_ok() || S->ready_small.front()->t_submit <= S->ready_big.front()->t_submit);
      if (!small) S->big_running++;
      if (small) {
        int32_t nmax = 0;
        while (!S->ready_small.empty() && (int)take.size() < S->cfg.max_batch) {
          take.push_back(S->ready_small.front());
          nmax = std::max(nmax, S->ready_small.front()->n);
          S->ready_small.pop_front();
        }
        // the batch's class-kernel slots: as many as the cap leaves room for
        const int64_t per = global_slot_bytes(nmax);
        batch_slots = batch_class_slots(nmax);
        const int64_t room = S->cfg.mem_cap_bytes - S->in_use;
        if (per > 0 && (int64_t)batch_slots * per > room) batch_slots = (int32_t)std::max<int64_t>(4, room / per);
        reserved = (int64_t)batch_slots * per;
        S->in_use += reserved;
        if (S->in_use > S->peak_in_use) S->peak_in_use = S->in_use;
      } else {
        Request* r = S->ready_big.front();
        take.push_back(r);
        S->ready_big.pop_front();
        // its class slots, charged while it runs: as many as the cap leaves room for
        if (r->slot_one > 0 && r->slot_part > 0) {
          const int64_t room = S->cfg.mem_cap_bytes - S->in_use;
          int64_t slots = r->slot_part / r->slot_one;
          if (slots * r->slot_one > room) {
            slots = std::max<int64_t>(1, room / r->slot_one);
            big_budget = 2 * slots * r->slot_one;  // the class kernel takes half of mem_budget_bytes
          }
          reserved = slots * r->slot_one;
          S->in_use += reserved;
          if (S->in_use > S->peak_in_use) S->peak_in_use = S->in_use;
        }
      }
    }
    // batches on the slot's stream, a large request on its high-priority one
    cudaStream_t st = small ? S->streams[slot] : S->streams_hi[slot];
    // host inputs: copy into pooled device memory on that stream
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
    int64_t launches = 0;
    auto run_alone = [&](int i, const gsofa_options& o) {
      const int32_t n1 = take[i]->n;
      const int32_t* rp1 = take[i]->rp;
      const int32_t* ci1 = take[i]->ci;
      rcs[i] = batch_transient(1, &n1, &rp1, &ci1, &o, st, &outs[i], &take[i]->est);
      if (rcs[i] == GSOFA_OK) launches += outs[i].stats.kernel_launches;
    };
    if (small) {
      // one batch of the small requests
      ns.clear();
      rps.clear();
      cis.clear();
      std::vector<int> in_batch;
      std::vector<int64_t> pe;
      for (int i = 0; i < k; i++) {
        if (rcs[i] != GSOFA_OK) continue;
        in_batch.push_back(i);
        pe.push_back(take[i]->est);
        ns.push_back(take[i]->n);
        rps.push_back(take[i]->rp);
        cis.push_back(take[i]->ci);
      }
      gsofa_options bo_opts = S->cfg.opts;
      if (batch_slots > 0) bo_opts.max_concurrent = batch_slots;
      if (!in_batch.empty()) {
        std::vector<gsofa_result> bo(in_batch.size());
        const int brc =
            batch_transient((int32_t)in_batch.size(), ns.data(), rps.data(), cis.data(), &bo_opts, st, bo.data(),
                            pe.data());
        if (brc == GSOFA_OK) {
          launches += bo[0].stats.kernel_launches;  // the batch's total
          for (size_t j = 0; j < in_batch.size(); j++) outs[in_batch[j]] = bo[j];
        } else if (brc == GSOFA_E_INVAL && in_batch.size() > 1) {
          // a malformed pattern rejects the whole batch: run the members one by
          // one so that only the offending request fails, as it would alone
          for (int i : in_batch) run_alone(i, bo_opts);
        } else {
          for (int i : in_batch) rcs[i] = brc;
        }
      }
    } else if (rcs[0] == GSOFA_OK) {
      // one large request alone (space-budget mode: with its own memory budget),
      // on half of the traversal CTAs so that batches keep running beside it:
      // its time is set by the serial class chains of its largest sources
      gsofa_options o = S->cfg.opts;
      if (take[0]->budget > 0) o.mem_budget_bytes = take[0]->budget;
      if (big_budget > 0) o.mem_budget_bytes = big_budget;
      if (o.max_ctas == 0) o.max_ctas = S->sms * 4;
      run_alone(0, o);
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
    sample_device(S);
    S->batches++;
    S->launches += launches;
    S->in_use -= reserved;
    if (!small) {
      S->big_running--;
      S->cv_work.notify_all();
    }
    Charge* ch = nullptr;
    for (int i = 0; i < k; i++) {
      if (rcs[i] != GSOFA_OK) continue;
      if (!ch) ch = new Charge();
      const gsofa_result& o = outs[i];
      ch->bytes += 16 * ((int64_t)o.n + 1) + 4 * (o.nnz_L + o.nnz_U) + 4 * (int64_t)o.n + 4 * ((int64_t)o.n_super + 1);
      ch->refs++;
    }
    for (int i = 0; i < k; i++) {
      Request* r = take[i];
      r->t_done = now;
      r->status = rcs[i];
      if (rcs[i] == GSOFA_OK) {
        r->held = ch;
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
      S->in_use -= r->projected - r->slot_part;
      S->inflight--;
    }
    if (ch) {  // the results stay charged until collected
      S->in_use += ch->bytes;
      if (S->in_use > S->peak_in_use) S->peak_in_use = S->in_use;
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
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
    cudaGetLastError();
    prio_lo = prio_hi = 0;
  }
  for (int i = 0; i < S->cfg.streams; i++) {
    cudaStream_t st = nullptr, sh = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sh, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
      cudaGetLastError();
      if (st) cudaStreamDestroy(st);
      for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
      for (cudaStream_t x : S->streams_hi) cudaStreamDestroy(x);
      cudaMemPoolDestroy(S->mpool);
      delete S;
      return GSOFA_E_CUDA;
    }
    S->streams.push_back(st);
    S->streams_hi.push_back(sh);
  }
  S->pool_base = library_pool_bytes(0, 1);  // in use now; the high-water mark restarts here
  S->slots_base = library_slot_bytes();
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
  r->est = projected_entries(n, r->nnz);
  r->projected = projected_bytes(S, n, r->nnz, !on_device);
  if (n > S->smem_max_n) {
    r->slot_part = global_tier_bytes(n, &S->cfg.opts);
    r->slot_one = global_slot_bytes(n);
  }
  if (r->projected > S->cfg.mem_cap_bytes && n > S->smem_max_n) {
    // space-budget mode (the concurrent-source budget of Section 5, Eq. 1): run
    // the request with as many global-tier slots as the cap leaves room for
    const int64_t base = r->projected - global_tier_bytes(n, &S->cfg.opts);
    const int64_t one = global_slot_bytes(n);
    const int64_t slots = one > 0 ? (S->cfg.mem_cap_bytes - base) / one : 0;
    if (slots >= 1) {
      r->budget = 2 * slots * one;  // the global tier takes half of mem_budget_bytes
      r->projected = base + slots * one;
      r->slot_part = slots * one;
    } else if (S->cfg.opts.host_spill >= 0) {
      // not even one whole slot: the slots' logs in host memory, their
      // visited bitmaps alone on the device (Section 6 external frontier)
      const int64_t dev = global_device_slot_bytes(n);
      const int64_t hs = dev > 0 ? (S->cfg.mem_cap_bytes - base) / dev : 0;
      if (hs >= 1) {
        r->budget = 2 * hs * dev;
        r->projected = base + hs * dev;
        r->slot_part = hs * dev;
        r->slot_one = dev;
      }
    }
  }
  if (r->projected > S->cfg.mem_cap_bytes) { delete r; return GSOFA_E_NOMEM; }
  r->big = n > S->smem_max_n || r->budget > 0;
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

// Caller holds mu.
static void release_charge(gsofa_server* S, Request* r) {
  Charge* ch = r->held;
  r->held = nullptr;
  if (!ch || --ch->refs > 0) return;
  S->in_use -= ch->bytes;
  delete ch;
  admit(S);
  S->cv_work.notify_all();
}

static int take_result(gsofa_server* S, std::unordered_map<uint64_t, Request*>::iterator it, gsofa_result* out,
                       double* latency_ms) {
  Request* r = it->second;
  const int st = r->status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  if (out) *out = r->res; else gsofa_free(&r->res);
  release_charge(S, r);
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
  sample_device(S);
  st->peak_device_bytes = S->peak_device;
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
    release_charge(S, kv.second);
    delete kv.second;
  }
  for (cudaStream_t st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaStream_t st : S->streams_hi) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaMemPoolDestroy(S->mpool);
  delete S;
}

}  // extern "C"
