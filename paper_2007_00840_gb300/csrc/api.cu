// Host side of libgsofa: argument checks, device memory, kernel sequencing
// and the extern "C" entry points declared in include/gsofa.h.
//
// One call = validate the CSR (Section 2.4 input) -> maxId traversal of every
// source row (Section 4; shared-memory tier for sources whose maxId array fits
// on chip, global tier for the rest) -> T3 supernode flags (Section 5) ->
// one read-back of the sizes -> prefix sums, row compaction into L/U CSR and
// the supernode list.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <unordered_map>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gsofa.h"
#include "internal.cuh"

namespace gsofa {


namespace {

struct Ctx {
  int device = 0;
  int sms = 0;
  int smem_optin = 0;
  cudaMemPool_t mpool = nullptr;
  // slots of the class-ordered kernel (persist across calls; every source
  // leaves its visited bitmap cleared)
  std::mutex gmu;
  uint32_t* g_V = nullptr;       // visited bitmaps, cap/32 words per slot
  uint32_t* g_VS = nullptr;      // their summaries, cap/1024 words per slot
  int32_t* g_log = nullptr;      // level overflow and L row, cap per slot
  int64_t g_cap = 0;
  int g_slots = 0;
  cudaEvent_t g_done = nullptr;
  // row-pool size that fitted last time, by matrix order
  std::mutex hmu;
  std::map<int32_t, long long> pool_hint;
  double rows_ratio = 0.0;  // largest pool entries per row seen (nnz(L+U) + 1 per row)
  std::atomic<int64_t> free_bytes{-1};  // device memory free when first asked (slot sizing)
  // single-matrix autotune: faster frontier order by (n, nnz)
  std::map<std::pair<int32_t, int64_t>, int> order_tuned;
};

std::mutex g_ctx_mu;
Ctx* g_ctx[128] = {nullptr};

// Device allocations shared by the results of one batch; freed with the last.
struct SharedBlock {
  std::atomic<int> refs{0};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<void*> ptrs;
};

struct Priv {
  cudaStream_t stream = nullptr;
  int device = 0;
  cudaMemPool_t mpool = nullptr;
  void* host_block = nullptr;   // host results: one pinned block holding every array
  size_t host_cap = 0;
  SharedBlock* shared = nullptr;  // batch results: arrays point into this block
};

// Pinned host blocks are expensive to create (page locking), so results of the
// host entry point reuse them: gsofa_free returns a block here.
struct PinnedCache {
  std::mutex mu;
  std::multimap<size_t, void*> blocks;
  size_t cached = 0;
  size_t limit = (size_t)8 << 30;
};
PinnedCache g_pinned;

void* pinned_get(size_t bytes, size_t* cap) {
  {
    std::lock_guard<std::mutex> lk(g_pinned.mu);
    auto it = g_pinned.blocks.lower_bound(bytes);
    if (it != g_pinned.blocks.end() && it->first <= 2 * bytes + (1 << 20)) {
      void* p = it->second;
      *cap = it->first;
      g_pinned.cached -= it->first;
      g_pinned.blocks.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *cap = bytes;
  return p;
}

void pinned_put(void* p, size_t cap) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(g_pinned.mu);
    if (g_pinned.cached + cap <= g_pinned.limit) {
      g_pinned.blocks.emplace(cap, p);
      g_pinned.cached += cap;
      return;
    }
  }
  cudaFreeHost(p);
}

double timeout_seconds() {
  const char* e = std::getenv("GSOFA_TIMEOUT_S");
  if (e) {
    const double v = std::atof(e);
    if (v > 0) return v;
  }
  return 600.0;
}

}  // namespace

// Bounded wait for all work queued on `st` (never an unbounded block).
int wait_stream(cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const double limit = timeout_seconds();
  int spins = 0;
  for (;;) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return GSOFA_OK;
    if (e != cudaErrorNotReady) return GSOFA_E_CUDA;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return GSOFA_E_TIMEOUT;
    if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

namespace {

Ctx* get_ctx(int* err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    *err = GSOFA_E_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  if (g_ctx[dev]) return g_ctx[dev];
  Ctx* c = new Ctx();
  c->device = dev;
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    delete c;
    *err = GSOFA_E_CUDA;
    return nullptr;
  }
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaMemPoolCreate(&c->mpool, &props) != cudaSuccess) {
    delete c;
    *err = GSOFA_E_CUDA;
    return nullptr;
  }
  uint64_t thr = UINT64_MAX;  // keep freed blocks for reuse by later calls
  cudaMemPoolSetAttribute(c->mpool, cudaMemPoolAttrReleaseThreshold, &thr);
  cudaEventCreateWithFlags(&c->g_done, cudaEventDisableTiming);
  g_ctx[dev] = c;
  return c;
}

template <typename T>
cudaError_t palloc(Ctx* c, T** p, size_t count, cudaStream_t st) {
  *p = nullptr;
  const size_t bytes = (count > 0 ? count : 1) * sizeof(T);
  return cudaMallocFromPoolAsync((void**)p, bytes, c->mpool, st);
}

template <typename T>
void pfree(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}

// First row-pool size for `rows` rows whose full rows hold at most `full`
// entries: per row, the larger of `floor_per_row` and 1.25 x the largest ratio
// seen on this device, plus 64K entries, so a stream of similar patterns stops
// overflowing (an overflow reruns the traversal).
long long pool_estimate(Ctx* c, long long rows, long long floor_per_row, long long full) {
  double per_row;
  {
    std::lock_guard<std::mutex> lk(c->hmu);
    per_row = 1.25 * c->rows_ratio;
  }
  if (per_row < (double)floor_per_row) per_row = (double)floor_per_row;
  long long cap = (long long)(per_row * (double)rows) + (1 << 16);
  if (full > 0 && cap > full) cap = full;
  if (cap < 1024) cap = 1024;
  return cap;
}

void note_pool_use(Ctx* c, unsigned long long used, long long rows) {
  if (rows <= 0) return;
  const double r = (double)used / (double)rows;
  std::lock_guard<std::mutex> lk(c->hmu);
  if (r > c->rows_ratio) c->rows_ratio = r;
}

// Bytes of one class-kernel slot of capacity cap (a multiple of 1024 vertices):
// visited bitmap, its summary, and the log (level overflow and L row).
int64_t slot_bytes(int64_t cap) { return cap / 8 + cap / 256 + 4 * cap; }

// Memory for global-tier slots: half of the caller's budget, else half of the
// device memory that is free or already held by slots, at most 96 GiB.
int64_t global_budget(const Ctx* c, const gsofa_options& o) {
  if (o.mem_budget_bytes > 0) return o.mem_budget_bytes / 2;
  int64_t b = (int64_t)96 << 30;
  // free memory is asked once per device (the query costs a few hundred
  // microseconds, as much as a whole small factorisation)
  int64_t fr = c->free_bytes.load();
  if (fr < 0) {
    size_t f = 0, tot = 0;
    if (cudaMemGetInfo(&f, &tot) == cudaSuccess) {
      const int64_t held = c->g_V ? (int64_t)c->g_slots * slot_bytes(c->g_cap) : 0;
      fr = (int64_t)f + held;
      int64_t expect = -1;
      const_cast<Ctx*>(c)->free_bytes.compare_exchange_strong(expect, fr);
    } else {
      cudaGetLastError();
      fr = 2 * b;
    }
  }
  if (fr / 2 < b) b = fr / 2;
  return b;
}

// Launch configuration of the class-ordered kernel for orders up to n_max.
struct ClassCfg {
  int vm = 0;            // where the visited bitmaps live: 0 shared memory, 1 global slots
  int warps_per_sm = 32; // register build (above 32: 48 registers)
  int qw = 128;          // shared queue entries per warp and level parity
  int vwords = 0;        // words of one visited bitmap (ceil(n_max / 32))
  int ctas_per_sm = 0;   // resident CTAs of four warps
};

constexpr int CLASS_VM_SMEM = 0, CLASS_VM_GLOBAL = 1;

// Device setting of the clean-head gathers for option clean_heads: automatic
// (0) gathers, with back-off, only where the visited bitmaps are in global
// memory (there a class head costs dependent L2 round trips; with shared
// bitmaps one class at a time was faster on every workload measured).
int clean_heads_mode(int opt, int vm) {
  if (opt < 0) return -1;
  if (opt == 0) return vm == CLASS_VM_GLOBAL ? 0 : -1;
  return opt == 1 ? 0 : 1;
}

ClassCfg class_config(const Ctx* c, int32_t n_max, int warps_per_sm, int queue = 0) {
  (void)c;
  ClassCfg k;
  k.warps_per_sm = warps_per_sm;
  if (queue > 0) k.qw = queue < 32 ? 32 : (queue > 1024 ? 1024 : queue & ~31);
  const int want = warps_per_sm / CLASS_WARPS_PER_CTA;
  const int words = (n_max + 31) / 32;
  const int occ_sv = trav_class_occupancy(CLASS_VM_SMEM, warps_per_sm, words, k.qw);
  if (occ_sv >= 4) {
    // whole bitmaps on chip while that keeps at least 16 warps per SM
    k.vm = CLASS_VM_SMEM;
    k.vwords = words;
    k.ctas_per_sm = occ_sv < want ? occ_sv : want;
  } else {
    // bitmaps in the global slots
    k.vm = CLASS_VM_GLOBAL;
    k.vwords = words;
    const int occ = trav_class_occupancy(CLASS_VM_GLOBAL, warps_per_sm, k.vwords, k.qw);
    k.ctas_per_sm = occ < want ? occ : want;
    // default queues: 512 entries hold most levels of a large source on chip
    // (1M ND grid 81 -> 79 ms; 768 and more took the L1 the records need)
    if (queue <= 0 && trav_class_occupancy(CLASS_VM_GLOBAL, warps_per_sm, k.vwords, 512) >= k.ctas_per_sm)
      k.qw = 512;

  }
  return k;
}

// Device bytes of a slot whose log lives in host memory: the visited bitmap
// and its summary only.
int64_t device_slot_bytes(int64_t cap) { return cap / 8 + cap / 256; }

// Slots (one warp each) of the class-ordered kernel for order n: a full wave
// of resident warps, within the budget (device bytes per slot: all of it, or
// the bitmaps alone when the logs are in host memory), at most 4 per CTA
// allowed by max_ctas.
int64_t global_slots(const Ctx* c, int32_t n, const gsofa_options& o, bool host_log = false) {
  const int64_t cap = ((int64_t)n + 1023) / 1024 * 1024;
  const ClassCfg k = class_config(c, n, o.warps_per_sm > 0 ? o.warps_per_sm : 32, o.list_capacity);
  int64_t slots = o.max_concurrent > 0 ? o.max_concurrent : (int64_t)c->sms * k.ctas_per_sm * CLASS_WARPS_PER_CTA;
  const int64_t fit = global_budget(c, o) / (host_log ? device_slot_bytes(cap) : slot_bytes(cap));
  if (slots > fit) slots = fit;
  if (o.max_ctas > 0 && slots > (int64_t)o.max_ctas * CLASS_WARPS_PER_CTA)
    slots = (int64_t)o.max_ctas * CLASS_WARPS_PER_CTA;
  return slots;
}

// Allocate class-kernel slot arrays (zeroed bitmaps) for `slots` x `cap`
// vertices; stream-ordered from the pool when `pool` is set, else cudaMalloc.
int alloc_slot_arrays(Ctx* c, int64_t cap, int64_t slots, uint32_t** V, uint32_t** VS, int32_t** log, bool pool,
                      cudaStream_t st) {
  *V = nullptr; *VS = nullptr; *log = nullptr;
  const size_t nV = (size_t)(cap / 32) * (size_t)slots, nVS = (size_t)(cap / 1024) * (size_t)slots;
  const size_t nQ = (size_t)cap * (size_t)slots;
  bool ok;
  if (pool) {
    ok = palloc(c, V, nV, st) == cudaSuccess && palloc(c, VS, nVS, st) == cudaSuccess &&
         palloc(c, log, nQ, st) == cudaSuccess;
  } else {
    ok = cudaMalloc(V, 4 * nV) == cudaSuccess && cudaMalloc(VS, 4 * nVS) == cudaSuccess &&
         cudaMalloc(log, 4 * nQ) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (void* q : {(void*)*V, (void*)*VS, (void*)*log})
      if (q) { if (pool) cudaFreeAsync(q, st); else cudaFree(q); }
    *V = nullptr; *VS = nullptr; *log = nullptr;
    return GSOFA_E_NOMEM;
  }
  if (cudaMemsetAsync(*V, 0, 4 * nV, st) != cudaSuccess || cudaMemsetAsync(*VS, 0, 4 * nVS, st) != cudaSuccess)
    return GSOFA_E_CUDA;
  return GSOFA_OK;
}

void free_slot_arrays(uint32_t*& V, uint32_t*& VS, int32_t*& log, bool pool, cudaStream_t st) {
  for (void* q : {(void*)V, (void*)VS, (void*)log})
    if (q) { if (pool) cudaFreeAsync(q, st); else cudaFree(q); }
  V = nullptr; VS = nullptr; log = nullptr;
}

// Make sure the context's class-kernel slots hold `slots` x `cap` vertices.  Caller holds gmu.
int ensure_slots(Ctx* c, int64_t cap, int slots, cudaStream_t st) {
  cap = (cap + 1023) / 1024 * 1024;
  if (c->g_V && c->g_cap >= cap && c->g_slots >= slots) return GSOFA_OK;
  // the previous user of the slots must be done before they are replaced
  cudaEventSynchronize(c->g_done);
  free_slot_arrays(c->g_V, c->g_VS, c->g_log, false, st);
  c->g_cap = 0; c->g_slots = 0;
  const int rc = alloc_slot_arrays(c, cap, slots, &c->g_V, &c->g_VS, &c->g_log, false, st);
  if (rc) return rc;
  c->g_cap = cap;
  c->g_slots = slots;
  return GSOFA_OK;
}

DevCounters* pinned_counters() {
  thread_local DevCounters* h = nullptr;
  if (!h) {
    if (cudaMallocHost(&h, sizeof(DevCounters)) != cudaSuccess) h = nullptr;
  }
  return h;
}

struct Events {
  bool on = false;
  cudaEvent_t e[8] = {nullptr};
  void create(bool enable) {
    on = enable;
    if (!on) return;
    for (auto& x : e) cudaEventCreate(&x);
  }
  void rec(int i, cudaStream_t st) {
    if (on) cudaEventRecord(e[i], st);
  }
  float ms(int a, int b) {
    float v = 0.f;
    if (on) cudaEventElapsedTime(&v, e[a], e[b]);
    return v;
  }
  ~Events() {
    if (on)
      for (auto& x : e) cudaEventDestroy(x);
  }
};

void zero_result(gsofa_result* out) { std::memset(out, 0, sizeof(*out)); }

struct Plan {
  int32_t S = 0;          // shared tier: sources [0, S)
  int label16 = 0;        // shared tier: 16-bit maxId
  int32_t list_cap = 0;   // shared tier: frontier list entries held on chip
  int smem_block = 512;
  int smem_grid = 0;
  int glob_block = 512;
  int glob_grid = 0;
  int async_sched = 0;    // shared tier: worklist schedule (the two lists form one ring >= S)
  ClassCfg cls;           // class-ordered kernel (sources S .. n-1)
  int32_t nbig = 0;       // of those, the largest expanded by four-warp CTA teams
  bool host_log = false;  // the slots' logs in pinned host memory (Section 6 external frontier)
};

}  // namespace

// Shared tier launch shape for sources [0, S): the (block, CTAs per SM) pair
// with the most resident threads (ties: more CTAs, i.e. more sources in
// flight), then the largest frontier list that keeps that occupancy.
int choose_smem_config(int sms, size_t limit, int32_t n, int32_t S, int label16, int threads_req, int* block,
                       int* occ_out, int32_t* cap_out) {
  (void)sms;
  const int stat = trav_smem_static_bytes();
  const int32_t min_cap = S < 1024 ? S : 1024;
  const size_t per_sm = 233472;  // 228 KB of shared memory per SM
  int best_block = 0, best_occ = 0;
  const int blocks[4] = {1024, 512, 256, threads_req};
  for (int bi = 0; bi < 4; bi++) {
    const int b = blocks[bi];
    if (b <= 0) continue;
    if (threads_req > 0 && b != threads_req) continue;
    const int occ = trav_smem_occupancy(b, trav_smem_bytes(n, S, min_cap, label16), label16);
    if (occ < 1) continue;
    if (occ * b > best_occ * best_block || (occ * b == best_occ * best_block && occ > best_occ)) {
      best_block = b;
      best_occ = occ;
    }
  }
  if (best_block == 0) return GSOFA_E_CUDA;
  size_t lim = per_sm / (size_t)best_occ;
  lim = lim > (size_t)stat + 1024 + 64 ? lim - (size_t)stat - 1024 - 64 : 0;
  if (lim > limit) lim = limit;
  int32_t cap = S;
  const size_t esz = label16 ? 2 : 4;
  const size_t fixed = trav_smem_bytes(n, S, 0, label16);
  if (fixed + 2 * esz * (size_t)cap > lim) cap = lim > fixed ? (int32_t)((lim - fixed) / (2 * esz)) : 0;
  if (cap < S) cap &= ~31;
  if (cap < min_cap) cap = min_cap;
  while (cap > min_cap && trav_smem_occupancy(best_block, trav_smem_bytes(n, S, cap, label16), label16) < best_occ)
    cap = (cap / 2 > min_cap) ? cap / 2 : min_cap;
  *block = best_block;
  *occ_out = best_occ;
  *cap_out = cap;
  return GSOFA_OK;
}

namespace {

int make_plan(Ctx* c, int32_t n, const gsofa_options& o, Plan* p) {
  const int stat = trav_smem_static_bytes();
  const int label16 = (n <= 65533 && o.label_bits != 32) ? 1 : 0;
  const size_t limit = (size_t)c->smem_optin - (size_t)stat - 64;
  int32_t S = trav_smem_max_S(n, limit, label16);
  if (o.smem_max_source > 0 && o.smem_max_source < S) S = o.smem_max_source;
  if (o.smem_max_source < 0 || o.frontier_order == 2) S = 0;  // every source in the class-ordered tier
  if (S > n) S = n;
  if (S < 0) S = 0;
  p->S = S;
  p->label16 = label16;
  if (S > 0) {
    int block = 0, occ = 0;
    int32_t cap = 0;
    const int rc = choose_smem_config(c->sms, limit, n, S, label16, o.threads_per_source, &block, &occ, &cap);
    if (rc) return rc;
    // a short shared list leaves more L1 for the rows; the rest spills to global memory
    const int32_t want = o.list_capacity > 0 ? o.list_capacity : 2048;
    if (want < cap) cap = want < 32 ? 32 : want;
    if (cap > S) cap = S;
    p->list_cap = cap;
    p->smem_block = block;
    p->smem_grid = c->sms * occ;
    if (o.schedule == 2 && label16 && S >= n && (o.expand_mode == 0 || o.expand_mode == 3) && !o.fill_first) {
      // worklist schedule: a ring of 2 x cap >= S entries, as many threads as fit
      const int32_t rcap = (S + 1) / 2 > 32 ? (S + 1) / 2 : 32;
      const size_t bytes = trav_smem_bytes(n, S, rcap, 1);
      const int tb = o.threads_per_source > 0 ? o.threads_per_source : 1024;
      const int aocc = bytes <= limit ? trav_smem_occupancy(tb, bytes, 1) : 0;
      if (aocc > 0) {
        p->async_sched = 1;
        p->list_cap = rcap;
        p->smem_block = tb;
        p->smem_grid = c->sms * aocc;
      }
    }
    if (o.max_ctas > 0 && o.max_ctas < p->smem_grid) p->smem_grid = o.max_ctas;
  }
  if (S < n) {
    // one warp per source (the largest: a CTA); a full wave of warps within the memory budget
    int64_t slots = global_slots(c, n, o);
    p->host_log = o.host_spill > 0 || (o.host_spill == 0 && slots < 1);
    if (p->host_log) slots = global_slots(c, n, o, true);
    if (slots < 1) return GSOFA_E_NOMEM;
    p->cls = class_config(c, n, o.warps_per_sm > 0 ? o.warps_per_sm : 32, o.list_capacity);
    p->glob_block = 32 * CLASS_WARPS_PER_CTA;
    p->glob_grid = (int)slots;  // slots (warps); small CTAs spread any slot count over every SM
    int64_t nbig = o.team_sources > 0 ? o.team_sources : 0;
    if (nbig > n - S) nbig = n - S;
    p->nbig = (int32_t)nbig;
  }
  return GSOFA_OK;
}

int check_options(const gsofa_options* in, gsofa_options* o) {
  gsofa_default_options(o);
  if (!in) return GSOFA_OK;
  if (in->chunk_size < 0 || in->threads_per_source < 0 || in->smem_max_source < -1 ||
      in->max_concurrent < 0 || in->mem_budget_bytes < 0)
    return GSOFA_E_INVAL;
  if (in->chunk_size) o->chunk_size = in->chunk_size;
  if (in->threads_per_source) {
    if (in->threads_per_source % 32 || in->threads_per_source < 64 || in->threads_per_source > 1024)
      return GSOFA_E_INVAL;
    o->threads_per_source = in->threads_per_source;
  }
  o->smem_max_source = in->smem_max_source;
  o->max_concurrent = in->max_concurrent;
  o->mem_budget_bytes = in->mem_budget_bytes;
  if (in->work_chunk < 0 || in->list_capacity < 0) return GSOFA_E_INVAL;
  if (in->max_ctas < 0 || in->frontier_order < 0 || in->frontier_order > 2) return GSOFA_E_INVAL;
  o->max_ctas = in->max_ctas;
  o->frontier_order = in->frontier_order;
  if (in->label_bits != 0 && in->label_bits != 16 && in->label_bits != 32) return GSOFA_E_INVAL;
  o->label_bits = in->label_bits;
  if (in->expand_mode < 0 || in->expand_mode > 3) return GSOFA_E_INVAL;
  o->expand_mode = in->expand_mode;
  if (in->schedule < 0 || in->schedule > 2) return GSOFA_E_INVAL;
  o->schedule = in->schedule;
  if (in->team_sources < -1) return GSOFA_E_INVAL;
  o->team_sources = in->team_sources;
  if (in->warps_per_sm != 0 && (in->warps_per_sm < 4 || in->warps_per_sm > 48 || in->warps_per_sm % 4))
    return GSOFA_E_INVAL;
  o->warps_per_sm = in->warps_per_sm;
  if (in->host_spill < -1 || in->host_spill > 1) return GSOFA_E_INVAL;
  o->host_spill = in->host_spill;
  if (in->clean_heads < -1 || in->clean_heads > 2) return GSOFA_E_INVAL;
  o->clean_heads = in->clean_heads;
  o->autotune = in->autotune ? 1 : 0;
  o->work_chunk = in->work_chunk;
  o->list_capacity = in->list_capacity;
  o->fill_first = in->fill_first ? 1 : 0;
  if (in->collect_stats < 0 || in->collect_stats > 2) return GSOFA_E_INVAL;
  o->collect_stats = in->collect_stats;
  o->validate = in->validate;
  if (o->chunk_size > 1024) return GSOFA_E_INVAL;
  return GSOFA_OK;
}

// ---------------------------------------------------------------- one matrix
int run_device(Ctx* c, int32_t n, const int32_t* d_rowptr, const int32_t* d_colidx, const gsofa_options& o,
               cudaStream_t st, gsofa_result* out, int64_t pool_entries = 0) {
  zero_result(out);
  Priv* pv = new Priv();
  pv->stream = st;
  pv->device = c->device;
  pv->mpool = c->mpool;
  out->_priv = pv;
  out->n = n;
  out->on_device = 1;
  out->err_detail = -1;

  Events ev;
  ev.create(o.collect_stats != 0);
  ev.rec(0, st);

  int rc = GSOFA_OK;
  cudaError_t ce = cudaSuccess;
  DevCounters* ctr = nullptr;
  int32_t* order = nullptr;
  uint32_t* pool = nullptr;
  int64_t* row_off = nullptr;
  int32_t *row_nL = nullptr, *row_nU = nullptr, *flags = nullptr;
  void* scan_tmp = nullptr;
  int64_t* flag_pos = nullptr;
  int32_t* spill = nullptr;
  int64_t spill_cap = 0;
  int4* ell = nullptr;
  int4* ellw = nullptr;  // class kernel, orders past 32,768 (16-bit offsets may not reach)
  DevCounters* h = pinned_counters();
  Plan plan;
  long long pool_cap = 0;
  bool have_global_lock = false;
  int nlaunch = 0;
  std::unique_lock<std::mutex> glk(c->gmu, std::defer_lock);
  // host-log slots (plan.host_log): bitmaps from the pool, logs in mapped pinned host memory
  uint32_t *hV = nullptr, *hVS = nullptr;
  int32_t* hlog_dev = nullptr;
  void* hlog_host = nullptr;
  int64_t hcap = 0;

#define CK(x)                        \
  do {                               \
    ce = (x);                        \
    if (ce != cudaSuccess) {         \
      rc = GSOFA_E_CUDA;             \
      goto fail;                     \
    }                                \
  } while (0)
#define LK(x)                        \
  do {                               \
    CK(x);                           \
    nlaunch++;                       \
  } while (0)

  if (!h) { rc = GSOFA_E_NOMEM; goto fail; }
  rc = make_plan(c, n, o, &plan);
  if (rc) goto fail;

  CK(palloc(c, &ctr, 1, st));
  CK(palloc(c, &order, (size_t)n, st));
  CK(palloc(c, &row_off, (size_t)n, st));
  CK(palloc(c, &row_nL, (size_t)n, st));
  CK(palloc(c, &row_nU, (size_t)n, st));
  CK(palloc(c, &flags, (size_t)n, st));
  CK(palloc(c, &out->fill_count, (size_t)n, st));
  {
    std::lock_guard<std::mutex> lk(c->hmu);
    auto it = c->pool_hint.find(n);
    if (it != c->pool_hint.end()) pool_cap = it->second;
  }
  // first size: the caller's estimate (a server's charge), else the learned ratio
  if (pool_cap == 0 && pool_entries > 0) pool_cap = pool_entries + (1 << 16);
  if (pool_cap == 0) pool_cap = pool_estimate(c, n, 256, (long long)n * (long long)(n + 1));
  CK(palloc(c, &pool, (size_t)pool_cap, st));
  if (plan.S > 0) {
    spill_cap = plan.S > plan.list_cap ? plan.S - plan.list_cap : 1;
    CK(palloc(c, &spill, (size_t)plan.smem_grid * 2 * (size_t)spill_cap, st));
  }
  if (n > 0 && (o.expand_mode == 0 || o.expand_mode == 3)) {
    if (plan.S < n && n > 32768) CK(palloc(c, &ellw, 2 * (size_t)n, st));
    if (plan.S > 0 || !ellw) CK(palloc(c, &ell, (size_t)n, st));
  }
  // order: shared tier [S-1 .. 0] then global tier [n-1 .. S] (largest source first)
  LK(launch_iota_desc(order, plan.S, plan.S, st));
  LK(launch_iota_desc(order + plan.S, n, n - plan.S, st));

  if (plan.S < n && plan.host_log) {
    // the external frontier of Section 6: each slot's log (level overflow and L
    // row) in host memory the kernel reads and writes directly; only the
    // visited bitmaps take device memory
    hcap = ((int64_t)n + 1023) / 1024 * 1024;
    const size_t slots = (size_t)plan.glob_grid;
    CK(palloc(c, &hV, (size_t)(hcap / 32) * slots, st));
    CK(palloc(c, &hVS, (size_t)(hcap / 1024) * slots, st));
    CK(cudaMemsetAsync(hV, 0, 4 * (size_t)(hcap / 32) * slots, st));
    CK(cudaMemsetAsync(hVS, 0, 4 * (size_t)(hcap / 1024) * slots, st));
    if (cudaHostAlloc(&hlog_host, 4 * (size_t)hcap * slots, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      hlog_host = nullptr;
      rc = GSOFA_E_NOMEM;
      goto fail;
    }
    CK(cudaHostGetDevicePointer((void**)&hlog_dev, hlog_host, 0));
  } else if (plan.S < n) {
    glk.lock();
    have_global_lock = true;
    rc = ensure_slots(c, n, plan.glob_grid, st);
    if (rc) goto fail;
    CK(cudaStreamWaitEvent(st, c->g_done, 0));
  }

  for (int attempt = 0; attempt < 3; attempt++) {
    LK(launch_init_counters(ctr, st));
    if (o.validate != 2 && attempt == 0) {
      ev.rec(1, st);
      LK(launch_validate(n, d_rowptr, d_colidx, ctr, st));
    } else {
      ev.rec(1, st);
    }
    if (ell && attempt == 0) LK(launch_build_ell(n, d_rowptr, d_colidx, ell, ctr, st));
    if (ellw && attempt == 0) LK(launch_build_ellw(n, d_rowptr, d_colidx, ellw, ctr, st));
    TravArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    a.rowptr = d_rowptr;
    a.colidx = d_colidx;
    a.pool = pool;
    a.pool_cap = pool_cap;
    a.row_off = row_off;
    a.row_nL = row_nL;
    a.row_nU = row_nU;
    a.fill_count = out->fill_count;
    a.ctr = ctr;
    a.fill_first = o.fill_first;
    a.collect_stats = o.collect_stats == 1;  // work counters (2: times only)
    ev.rec(2, st);
    if (plan.S < n) {
      a.order = order + plan.S;
      a.nsrc = n - plan.S;
      a.ell = ell;
      a.ellw = ellw;
      a.g_V = plan.host_log ? hV : c->g_V;
      a.g_VS = plan.host_log ? hVS : c->g_VS;
      a.g_log = plan.host_log ? hlog_dev : c->g_log;
      a.g_cap = plan.host_log ? hcap : c->g_cap;
      a.g_slots = plan.glob_grid;
      a.ct_qw = plan.cls.qw;
      a.ct_vwords = plan.cls.vwords;
      a.ct_nbig = plan.nbig;
      a.ct_heads = clean_heads_mode(o.clean_heads, plan.cls.vm);
      LK(launch_trav_class(a, (plan.glob_grid + CLASS_WARPS_PER_CTA - 1) / CLASS_WARPS_PER_CTA, plan.cls.vm,
                           plan.cls.warps_per_sm, st));
      if (!plan.host_log) CK(cudaEventRecord(c->g_done, st));
    }
    ev.rec(3, st);
    if (plan.S > 0) {
      a.order = order;
      a.nsrc = plan.S;
      a.S = plan.S;
      a.list_cap = plan.list_cap;
      a.spill = spill;
      a.spill_cap = spill_cap;
      a.chunk = o.work_chunk > 0 ? o.work_chunk : 1;
      a.expand_mode = o.expand_mode == 0 ? 3 : o.expand_mode;
      a.async_sched = plan.async_sched;
      a.ell = ell;
      LK(launch_trav_smem(a, plan.smem_grid, plan.smem_block, plan.label16, st));
    }
    ev.rec(4, st);
    LK(launch_supernode_flags(n, o.chunk_size, pool, row_off, row_nL, row_nU, flags, ctr, st));
    ev.rec(5, st);
    CK(cudaMemcpyAsync(h, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    rc = wait_stream(st);
    if (rc) goto fail;
    if (h->err & ERR_INPUT) {
      rc = GSOFA_E_INVAL;
      out->err_detail = h->err_row == INT_MAX ? -1 : h->err_row;
      goto fail;
    }
    if (h->err & ERR_NOCONV) { rc = GSOFA_E_NOCONVERGE; goto fail; }
    if (!(h->err & ERR_OVERFLOW)) break;
    // the pool was too small: the counts are exact now, grow it and run again
    out->stats.pool_retries++;
    pfree(pool, st);
    pool_cap = (long long)h->pool_cursor + 1024;
    CK(palloc(c, &pool, (size_t)pool_cap, st));
  }
  if (h->err & ERR_OVERFLOW) { rc = GSOFA_E_NOMEM; goto fail; }
  if (have_global_lock) { glk.unlock(); have_global_lock = false; }
  if (plan.host_log) {
    // the traversal is complete (its counters were read back)
    if (hlog_host) cudaFreeHost(hlog_host);
    hlog_host = nullptr;
    pfree(hV, st);
    pfree(hVS, st);
  }
  {
    std::lock_guard<std::mutex> lk(c->hmu);
    c->pool_hint[n] = (long long)h->pool_cursor + ((long long)h->pool_cursor >> 4) + 1024;
  }
  note_pool_use(c, h->pool_cursor, n);

  out->nnz_L = (int64_t)h->total_L;
  out->nnz_U = (int64_t)h->total_U;
  out->n_super = h->n_super;
  out->stats.vertices_expanded = (int64_t)h->expansions;
  out->stats.edges_scanned = (int64_t)h->edges;
  out->stats.levels = (int64_t)h->levels;
  out->stats.cycles_traverse = (int64_t)h->cyc_trav;
  out->stats.cycles_emit = (int64_t)h->cyc_emit;
  out->stats.traverse_launches = (plan.S > 0) + (plan.S < n);

  CK(palloc(c, &out->L_rowptr, (size_t)n + 1, st));
  CK(palloc(c, &out->U_rowptr, (size_t)n + 1, st));
  CK(palloc(c, &out->L_colidx, (size_t)out->nnz_L, st));
  CK(palloc(c, &out->U_colidx, (size_t)out->nnz_U, st));
  CK(palloc(c, &out->super_start, (size_t)out->n_super + 1, st));
  CK(palloc(c, &flag_pos, (size_t)n + 1, st));
  {
    size_t tb = scan_tmp_bytes(n);
    CK(cudaMallocFromPoolAsync(&scan_tmp, tb, c->mpool, st));
  }
  CK(launch_scan_i32_i64(row_nL, out->L_rowptr, n, scan_tmp, st));
  CK(launch_scan_i32_i64(row_nU, out->U_rowptr, n, scan_tmp, st));
  if (n > 0) nlaunch += 9;  // three scans of three kernels each
  LK(launch_compact(n, pool, row_off, row_nL, row_nU, out->L_rowptr, out->U_rowptr, out->L_colidx,
                    out->U_colidx, st));
  CK(launch_scan_i32_i64(flags, flag_pos, n, scan_tmp, st));
  LK(launch_scatter_starts(n, flags, flag_pos, out->super_start, st));
  ev.rec(6, st);
  out->stats.kernel_launches = nlaunch;

  pfree(ctr, st);
  pfree(order, st);
  pfree(pool, st);
  pfree(row_off, st);
  pfree(row_nL, st);
  pfree(row_nU, st);
  pfree(flags, st);
  pfree(flag_pos, st);
  pfree(spill, st);
  pfree(ell, st);
  pfree(ellw, st);
  if (scan_tmp) cudaFreeAsync(scan_tmp, st);
  scan_tmp = nullptr;

  if (o.collect_stats) {
    rc = wait_stream(st);
    if (rc) goto fail;
    out->stats.ms_validate = ev.ms(1, 2);
    out->stats.ms_traverse_global = ev.ms(2, 3);
    out->stats.ms_traverse_smem = ev.ms(3, 4);
    out->stats.ms_traverse = ev.ms(2, 4);
    out->stats.ms_supernode = ev.ms(4, 5);
    out->stats.ms_emit = ev.ms(5, 6);
    out->stats.ms_total = ev.ms(0, 6);
  }
  if (cudaGetLastError() != cudaSuccess) { rc = GSOFA_E_CUDA; goto fail; }
  return GSOFA_OK;

fail:
  cudaGetLastError();
  if (have_global_lock) glk.unlock();
  wait_stream(st);
  if (hlog_host) cudaFreeHost(hlog_host);
  pfree(hV, st);
  pfree(hVS, st);
  pfree(ctr, st);
  pfree(order, st);
  pfree(pool, st);
  pfree(row_off, st);
  pfree(row_nL, st);
  pfree(row_nU, st);
  pfree(flags, st);
  pfree(flag_pos, st);
  pfree(spill, st);
  pfree(ell, st);
  pfree(ellw, st);
  if (scan_tmp) cudaFreeAsync(scan_tmp, st);
  {
    const int32_t det = out->err_detail;
    gsofa_free(out);
    out->err_detail = det;
  }
  return rc;
#undef CK
}


// ------------------------------------------------------------------ batches
// Launch shape of the shared-memory traversal for one batch shape.
struct LaunchShape {
  int block = 512;
  int occ = 1;
  int32_t list_cap = 1024;
  int work_chunk = 1;
  int kernel = 0;   // 0: shared-memory breadth-first tier; 1: class-ordered warp tier
  int slots = 0;    // kernel 1: warps (sources in flight)
  int fill_first = 0;  // kernel 0: the fill-first check of Section 4 ("line 9.5"; same rows)
};

// Workspace and captured graph of one batch signature.
struct BatchPlan {
  bool transient = false;           // workspace from the stream-ordered pool, freed after one call
  cudaStream_t stream = nullptr;
  Ctx* ctx = nullptr;
  int max_ctas = 0;
  uint64_t sig = 0;
  uint64_t last_use = 0;
  int32_t B = 0;                    // matrices in the batched launch
  std::vector<int32_t> members;     // their indices in the caller's arrays
  std::vector<int64_t> row_base;
  int32_t n_max = 0;
  int64_t N = 0, chunks = 0;
  int label16 = 1;
  LaunchShape shape;
  MatDesc* d_mats = nullptr;
  int32_t* d_item_start = nullptr;
  int32_t* d_mat_order = nullptr;
  unsigned char* d_ctr = nullptr;   // DevCounters | per matrix [nL, nU] | per matrix n_super
  unsigned char* h_ctr = nullptr;   // pinned copy of d_ctr
  size_t ctr_bytes = 0;
  int64_t* row_off = nullptr;
  int32_t *row_nL = nullptr, *row_nU = nullptr, *flags = nullptr, *fill = nullptr;
  uint32_t* pool = nullptr;
  long long pool_cap = 0;
  int32_t* spill = nullptr;
  int64_t spill_cap = 0;
  int64_t spill_alloc = 0;
  int4* ell = nullptr;              // ELL records of every row (row_base + v)
  // class-ordered kernel slots (kernel 1)
  uint32_t* c_V = nullptr;
  uint32_t* c_VS = nullptr;
  int32_t* c_log = nullptr;
  int64_t c_cap = 0;
  int c_slots = 0;
  ClassCfg c_cfg;
  int grid = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the traversal launch (collect_stats)

  DevCounters* ctr() const { return (DevCounters*)d_ctr; }
  unsigned long long* mat_tot() const { return (unsigned long long*)(d_ctr + 256); }
  int32_t* mat_nsuper() const { return (int32_t*)(d_ctr + 256 + 16 * (size_t)B); }
  const DevCounters* hctr() const { return (const DevCounters*)h_ctr; }
  const unsigned long long* h_tot() const { return (const unsigned long long*)(h_ctr + 256); }
  const int32_t* h_nsuper() const { return (const int32_t*)(h_ctr + 256 + 16 * (size_t)B); }
};

void free_plan(BatchPlan* p) {
  if (p->transient) {
    for (void* q : {(void*)p->d_mats, (void*)p->d_item_start, (void*)p->d_mat_order, (void*)p->d_ctr,
                    (void*)p->row_off, (void*)p->row_nL, (void*)p->row_nU, (void*)p->flags, (void*)p->fill,
                    (void*)p->pool, (void*)p->spill, (void*)p->c_V, (void*)p->c_VS, (void*)p->c_log,
                    (void*)p->ell})
      if (q) cudaFreeAsync(q, p->stream);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    delete p;
    return;
  }
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  cudaFree(p->d_mats);
  cudaFree(p->d_item_start);
  cudaFree(p->d_mat_order);
  cudaFree(p->d_ctr);
  cudaFree(p->row_off);
  cudaFree(p->row_nL);
  cudaFree(p->row_nU);
  cudaFree(p->flags);
  cudaFree(p->fill);
  cudaFree(p->pool);
  cudaFree(p->spill);
  cudaFree(p->c_V);
  cudaFree(p->c_VS);
  cudaFree(p->c_log);
  cudaFree(p->ell);
  if (p->h_ctr) cudaFreeHost(p->h_ctr);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
}

struct BatchCache {
  std::mutex mu;
  std::unordered_map<uint64_t, BatchPlan*> plans;
  uint64_t clock = 0;
  std::map<uint64_t, LaunchShape> tuned;  // shape bucket -> fastest launch shape
  bool file_loaded = false;
};
BatchCache g_batch[128];

uint64_t mix64(uint64_t h, uint64_t v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h * 0xBF58476D1CE4E5B9ull;
}

uint64_t bucket_key(int32_t n_max, int64_t N, int label16) {
  int a = 0, b = 0;
  while ((1LL << a) < n_max) a++;
  while ((1LL << b) < N) b++;
  return ((uint64_t)a << 32) | ((uint64_t)b << 8) | (uint64_t)label16;
}

// Tuning results persist in the file named by GSOFA_TUNE_FILE (optional).
void load_tune_file(BatchCache& bc) {
  if (bc.file_loaded) return;
  bc.file_loaded = true;
  const char* f = std::getenv("GSOFA_TUNE_FILE");
  if (!f) return;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  unsigned long long key;
  int block, occ, cap, chunk, kernel, slots, ff;
  while (std::fscanf(fp, "%llx %d %d %d %d %d %d %d", &key, &block, &occ, &cap, &chunk, &kernel, &slots, &ff) == 8) {
    LaunchShape sh;
    sh.block = block; sh.occ = occ; sh.list_cap = cap; sh.work_chunk = chunk;
    sh.kernel = kernel; sh.slots = slots; sh.fill_first = ff;
    bc.tuned[key] = sh;
  }
  std::fclose(fp);
}

void save_tune_entry(uint64_t key, const LaunchShape& sh) {
  const char* f = std::getenv("GSOFA_TUNE_FILE");
  if (!f) return;
  FILE* fp = std::fopen(f, "a");
  if (!fp) return;
  // key, threads per source, CTAs per SM, list capacity, work chunk, kernel (0 CTA per
  // source, 1 class-ordered warp per source), class-kernel slots, fill-first check
  std::fprintf(fp, "%llx %d %d %d %d %d %d %d\n", (unsigned long long)key, sh.block, sh.occ, sh.list_cap,
               sh.work_chunk, sh.kernel, sh.slots, sh.fill_first);
  std::fclose(fp);
}

// Warps of the class-ordered kernel for orders up to n_max: per_sm per SM (as
// far as the shared bitmaps allow), within 8 GiB.
int class_slots(Ctx* c, int32_t n_max, int per_sm) {
  const int64_t cap = ((int64_t)n_max + 1023) / 1024 * 1024;
  const ClassCfg k = class_config(c, n_max, per_sm);
  int64_t slots = (int64_t)c->sms * k.ctas_per_sm * CLASS_WARPS_PER_CTA;
  const int64_t fit = ((int64_t)8 << 30) / slot_bytes(cap);
  if (slots > fit) slots = fit;
  return (int)slots;
}

// Launch shapes worth timing for a batch whose largest order is n_max.
std::vector<LaunchShape> candidate_shapes(Ctx* c, int32_t n_max, int label16, size_t limit, int order) {
  std::vector<LaunchShape> out;
  const int blocks[3] = {256, 512, 1024};
  for (int b : (order == 2 ? std::vector<int>{} : std::vector<int>{blocks[0], blocks[1], blocks[2]})) {
    int block = 0, occ = 0;
    int32_t cap = 0;
    if (choose_smem_config(c->sms, limit, n_max, n_max, label16, b, &block, &occ, &cap) != GSOFA_OK) continue;
    const int32_t caps[2] = {cap, n_max < 1024 ? n_max : 1024};
    for (int ci = 0; ci < 2; ci++) {
      if (ci == 1 && caps[1] >= cap) continue;
      for (int chunk : {1, 4}) {
        LaunchShape sh;
        sh.block = block; sh.occ = occ; sh.list_cap = caps[ci]; sh.work_chunk = chunk;
        out.push_back(sh);
        if (chunk == 1) {  // the same shape with the fill-first check
          sh.fill_first = 1;
          out.push_back(sh);
        }
      }
    }
  }
  for (int per_sm : (order == 1 ? std::vector<int>{} : std::vector<int>{16, 32, 40})) {
    LaunchShape sh;
    sh.kernel = 1;
    sh.occ = per_sm;  // warps per SM (above 32: the 48-register build)
    sh.slots = class_slots(c, n_max, per_sm);
    if (sh.slots > 0) out.push_back(sh);
  }
  return out;
}

// Enqueue the first phase (counters, validation, traversal, supernodes, size read-back).
cudaError_t enqueue_phase1(const BatchPlan& p, const gsofa_options& o, cudaStream_t st, cudaEvent_t t0,
                           cudaEvent_t t1) {
  cudaError_t e;
  if ((e = launch_init_counters(p.ctr(), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(p.d_ctr + 256, 0, p.ctr_bytes - 256, st)) != cudaSuccess) return e;
  if (o.validate != 2 && (e = launch_validate_batch(p.d_mats, p.B, p.N, p.ctr(), st)) != cudaSuccess) return e;
  TravArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = p.n_max;
  a.S = p.n_max;
  a.nsrc = (int32_t)p.N;
  a.list_cap = p.shape.list_cap;
  a.spill = p.spill;
  a.spill_cap = p.spill_cap;
  a.pool = p.pool;
  a.pool_cap = p.pool_cap;
  a.row_off = p.row_off;
  a.row_nL = p.row_nL;
  a.row_nU = p.row_nU;
  a.fill_count = p.fill;
  a.ctr = p.ctr();
  a.fill_first = (o.fill_first || p.shape.fill_first) ? 1 : 0;
  a.collect_stats = o.collect_stats == 1;  // work counters (2: times only)
  a.mats = p.d_mats;
  a.item_start = p.d_item_start;
  a.mat_order = p.d_mat_order;
  a.nmats = p.B;
  a.chunk = p.shape.work_chunk;
  a.mat_tot = p.mat_tot();
  a.expand_mode = (o.expand_mode == 0 || o.expand_mode == 3) ? 3 : o.expand_mode;
  if (a.expand_mode == 3) {
    // adjacency records of every member (both traversal kernels read them)
    if ((e = launch_build_ell_batch(p.d_mats, p.B, p.N, p.ell, p.ctr(), st)) != cudaSuccess) return e;
    a.ell = p.ell;
  }
  // while capturing, external records become event nodes of the graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  const unsigned rf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (t0 && (e = cudaEventRecordWithFlags(t0, st, rf)) != cudaSuccess) return e;
  if (p.shape.kernel == 1) {
    a.g_V = p.c_V;
    a.g_VS = p.c_VS;
    a.g_log = p.c_log;
    a.g_cap = p.c_cap;
    a.g_slots = p.shape.slots;
    a.ct_qw = p.c_cfg.qw;
    a.ct_vwords = p.c_cfg.vwords;
    a.ct_nbig = 0;
    a.ct_heads = clean_heads_mode(o.clean_heads, p.c_cfg.vm);
    if ((e = launch_trav_class(a, (p.shape.slots + CLASS_WARPS_PER_CTA - 1) / CLASS_WARPS_PER_CTA, p.c_cfg.vm,
                               p.c_cfg.warps_per_sm, st)) != cudaSuccess)
      return e;
  } else if ((e = launch_trav_smem(a, p.grid, p.shape.block, p.label16, st)) != cudaSuccess) {
    return e;
  }
  if (t1 && (e = cudaEventRecordWithFlags(t1, st, rf)) != cudaSuccess) return e;
  if ((e = launch_supernode_batch(p.d_mats, p.B, p.chunks, o.chunk_size, p.pool, p.row_off, p.row_nL, p.row_nU,
                                  p.flags, p.mat_nsuper(), p.ctr(), st)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(p.h_ctr, p.d_ctr, p.ctr_bytes, cudaMemcpyDeviceToHost, st);
}

int set_shape(Ctx* c, BatchPlan* p, const LaunchShape& sh) {
  p->shape = sh;
  p->grid = c->sms * sh.occ;
  if (p->max_ctas > 0 && p->max_ctas < p->grid) p->grid = p->max_ctas;
  if (sh.kernel == 1) {
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    const int64_t cap = ((int64_t)p->n_max + 1023) / 1024 * 1024;
    p->c_cfg = class_config(c, p->n_max, sh.occ);
    if (p->c_V && p->c_cap >= cap && p->c_slots >= sh.slots) return GSOFA_OK;
    cudaStream_t ast = p->transient ? p->stream : p->cap_stream;
    free_slot_arrays(p->c_V, p->c_VS, p->c_log, p->transient, ast);
    const int rc = alloc_slot_arrays(c, cap, sh.slots, &p->c_V, &p->c_VS, &p->c_log, p->transient, ast);
    if (rc) return rc;
    if (!p->transient) cudaStreamSynchronize(ast);
    p->c_cap = cap;
    p->c_slots = sh.slots;
    return GSOFA_OK;
  }
  // per CTA two overflow lists of (n_max - list capacity) entries
  p->spill_cap = p->n_max > sh.list_cap ? (int64_t)p->n_max - sh.list_cap : 1;
  const int64_t need = (int64_t)p->grid * 2 * p->spill_cap;
  if (!p->spill || need > p->spill_alloc) {
    if (p->transient) cudaFreeAsync(p->spill, p->stream); else cudaFree(p->spill);
    p->spill = nullptr;
    p->spill_alloc = 0;
    const cudaError_t ea = p->transient
        ? cudaMallocFromPoolAsync((void**)&p->spill, sizeof(int32_t) * (size_t)need, c->mpool, p->stream)
        : cudaMalloc(&p->spill, sizeof(int32_t) * (size_t)need);
    if (ea != cudaSuccess) {
      cudaGetLastError();
      p->spill = nullptr;
      return GSOFA_E_NOMEM;
    }
    p->spill_alloc = need;
  }
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return GSOFA_OK;
}

// Pinned host scratch of the calling thread (descriptor uploads, size read-backs
// of transient batches); reused once the previous call on this thread waited.
void* thread_pinned(size_t bytes, int slot) {
  thread_local void* buf[2] = {nullptr, nullptr};
  thread_local size_t cap[2] = {0, 0};
  if (cap[slot] < bytes) {
    if (buf[slot]) cudaFreeHost(buf[slot]);
    buf[slot] = nullptr;
    cap[slot] = 0;
    const size_t want = bytes + (bytes >> 1) + 4096;
    if (cudaMallocHost(&buf[slot], want) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cap[slot] = want;
  }
  return buf[slot];
}

int build_plan(Ctx* c, const std::vector<int32_t>& members, const int32_t* n, const int32_t* const* rp,
               const int32_t* const* ci, const gsofa_options& o, uint64_t sig, BatchPlan** out,
               bool transient, cudaStream_t st, int64_t pool_entries = 0) {
  BatchPlan* p = new BatchPlan();
  p->transient = transient;
  p->stream = st;
  p->ctx = c;
  p->max_ctas = o.max_ctas;
  p->sig = sig;
  if (o.collect_stats) {
    cudaEventCreate(&p->ev0);
    cudaEventCreate(&p->ev1);
  }
  p->members = members;
  p->B = (int32_t)members.size();
  std::vector<MatDesc> mats(p->B);
  int64_t rbase = 0, cbase = 0;
  for (int32_t k = 0; k < p->B; k++) {
    const int32_t nk = n[members[k]];
    mats[k].rowptr = rp[members[k]];
    mats[k].colidx = ci[members[k]];
    mats[k].n = nk;
    mats[k].row_base = rbase;
    mats[k].chunk_base = cbase;
    p->row_base.push_back(rbase);
    rbase += nk;
    cbase += (nk + o.chunk_size - 1) / o.chunk_size;
    if (nk > p->n_max) p->n_max = nk;
  }
  p->N = rbase;
  p->chunks = cbase;
  p->label16 = p->n_max <= 65533 ? 1 : 0;
  // work order: source index descending, then matrices by decreasing order
  std::vector<int32_t> order(p->B);
  for (int32_t k = 0; k < p->B; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return mats[x].n > mats[y].n; });
  std::vector<int32_t> item_start(p->n_max > 0 ? p->n_max : 1, 0);
  {
    // cnt(s) = #{m : n_m > s}; item_start[s] = sum_{s' > s} cnt(s')
    std::vector<int32_t> cnt(p->n_max + 1, 0);
    for (int32_t k = 0; k < p->B; k++) cnt[mats[k].n]++;  // count by n, then suffix sums
    int32_t above = 0;
    std::vector<int32_t> c_s(p->n_max, 0);
    for (int32_t s = p->n_max - 1; s >= 0; s--) {
      above += cnt[s + 1];
      c_s[s] = above;  // matrices with n > s
    }
    int64_t acc = 0;
    for (int32_t s = p->n_max - 1; s >= 0; s--) {
      item_start[s] = (int32_t)acc;
      acc += c_s[s];
    }
  }
  p->ctr_bytes = 256 + 16 * (size_t)p->B + 4 * (size_t)p->B;
  {
    std::lock_guard<std::mutex> lk(c->hmu);
    auto it = c->pool_hint.find(-(int32_t)(sig & 0x7FFFFFFF) - 1);
    p->pool_cap = it != c->pool_hint.end() ? it->second : 0;
  }
  if (p->pool_cap == 0 && pool_entries > 0) p->pool_cap = pool_entries + (1 << 16);
  if (p->pool_cap == 0) p->pool_cap = pool_estimate(c, p->N, 64, 0);
  if (transient) {
    const size_t b_mats = sizeof(MatDesc) * (size_t)(p->B > 0 ? p->B : 1);
    const size_t b_is = sizeof(int32_t) * item_start.size();
    const size_t b_ord = sizeof(int32_t) * (size_t)(p->B > 0 ? p->B : 1);
    unsigned char* stage = (unsigned char*)thread_pinned(b_mats + b_is + b_ord, 0);
    p->h_ctr = (unsigned char*)thread_pinned(p->ctr_bytes, 1);
    bool ok = stage && p->h_ctr &&
              palloc(c, &p->d_mats, (size_t)(p->B > 0 ? p->B : 1), st) == cudaSuccess &&
              palloc(c, &p->d_item_start, item_start.size(), st) == cudaSuccess &&
              palloc(c, &p->d_mat_order, (size_t)(p->B > 0 ? p->B : 1), st) == cudaSuccess &&
              palloc(c, &p->d_ctr, p->ctr_bytes, st) == cudaSuccess &&
              palloc(c, &p->row_off, (size_t)p->N, st) == cudaSuccess &&
              palloc(c, &p->row_nL, (size_t)p->N, st) == cudaSuccess &&
              palloc(c, &p->row_nU, (size_t)p->N, st) == cudaSuccess &&
              palloc(c, &p->flags, (size_t)p->N, st) == cudaSuccess &&
              palloc(c, &p->fill, (size_t)p->N, st) == cudaSuccess &&
              palloc(c, &p->pool, (size_t)p->pool_cap, st) == cudaSuccess &&
              palloc(c, &p->ell, (size_t)(p->N > 0 ? p->N : 1), st) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      p->h_ctr = nullptr;
      free_plan(p);
      return GSOFA_E_NOMEM;
    }
    std::memcpy(stage, mats.data(), sizeof(MatDesc) * (size_t)p->B);
    std::memcpy(stage + b_mats, item_start.data(), b_is);
    std::memcpy(stage + b_mats + b_is, order.data(), sizeof(int32_t) * (size_t)p->B);
    if (cudaMemcpyAsync(p->d_mats, stage, b_mats, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(p->d_item_start, stage + b_mats, b_is, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(p->d_mat_order, stage + b_mats + b_is, b_ord, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      p->h_ctr = nullptr;
      free_plan(p);
      return GSOFA_E_CUDA;
    }
    *out = p;
    return GSOFA_OK;
  }
  bool ok = cudaMalloc(&p->d_mats, sizeof(MatDesc) * (size_t)(p->B > 0 ? p->B : 1)) == cudaSuccess &&
            cudaMalloc(&p->d_item_start, sizeof(int32_t) * item_start.size()) == cudaSuccess &&
            cudaMalloc(&p->d_mat_order, sizeof(int32_t) * (size_t)(p->B > 0 ? p->B : 1)) == cudaSuccess &&
            cudaMalloc(&p->d_ctr, p->ctr_bytes) == cudaSuccess &&
            cudaMallocHost(&p->h_ctr, p->ctr_bytes) == cudaSuccess &&
            cudaMalloc(&p->row_off, sizeof(int64_t) * (size_t)p->N) == cudaSuccess &&
            cudaMalloc(&p->row_nL, sizeof(int32_t) * (size_t)p->N) == cudaSuccess &&
            cudaMalloc(&p->row_nU, sizeof(int32_t) * (size_t)p->N) == cudaSuccess &&
            cudaMalloc(&p->flags, sizeof(int32_t) * (size_t)p->N) == cudaSuccess &&
            cudaMalloc(&p->fill, sizeof(int32_t) * (size_t)p->N) == cudaSuccess &&
            cudaMalloc(&p->pool, sizeof(uint32_t) * (size_t)p->pool_cap) == cudaSuccess &&
            cudaMalloc(&p->ell, sizeof(int4) * (size_t)(p->N > 0 ? p->N : 1)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_plan(p);
    return GSOFA_E_NOMEM;
  }
  if (cudaMemcpy(p->d_mats, mats.data(), sizeof(MatDesc) * (size_t)p->B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_item_start, item_start.data(), sizeof(int32_t) * item_start.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_mat_order, order.data(), sizeof(int32_t) * (size_t)p->B, cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    free_plan(p);
    return GSOFA_E_CUDA;
  }
  *out = p;
  return GSOFA_OK;
}

// Time every candidate launch shape once on this batch and keep the fastest.
int autotune_plan(Ctx* c, BatchPlan* p, const gsofa_options& o, cudaStream_t st, size_t limit) {
  std::vector<LaunchShape> cands = candidate_shapes(c, p->n_max, p->label16, limit, o.frontier_order);
  if (cands.empty()) return GSOFA_E_CUDA;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  LaunchShape best_sh = cands[0];
  for (const LaunchShape& sh : cands) {
    int rc = set_shape(c, p, sh);
    if (rc) { cudaEventDestroy(t0); cudaEventDestroy(t1); return rc; }
    if (enqueue_phase1(*p, o, st, t0, t1) != cudaSuccess) { cudaEventDestroy(t0); cudaEventDestroy(t1); return GSOFA_E_CUDA; }
    rc = wait_stream(st);
    if (rc) { cudaEventDestroy(t0); cudaEventDestroy(t1); return rc; }
    if (p->hctr()->err & (ERR_INPUT | ERR_NOCONV)) break;  // reported by the real run
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best) { best = ms; best_sh = sh; }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return set_shape(c, p, best_sh);
}

int capture_plan(BatchPlan* p, const gsofa_options& o) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return GSOFA_E_CUDA;
  const cudaError_t e1 = enqueue_phase1(*p, o, p->cap_stream, p->ev0, p->ev1);
  const cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return GSOFA_E_CUDA;
  }
  const cudaError_t e3 = cudaGraphInstantiate(&p->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    cudaGetLastError();
    p->gexec = nullptr;
    return GSOFA_E_CUDA;
  }
  return GSOFA_OK;
}

// Phase 1 (counters, validation, traversal, supernodes, size read-back),
// rerun with an exact pool when the row pool overflowed.
int batch_phase1(Ctx* c, BatchPlan* p, const gsofa_options& o, cudaStream_t st, bool use_graph, int* launches) {
  for (int attempt = 0; attempt < 3; attempt++) {
    if (use_graph && !p->gexec && capture_plan(p, o) != GSOFA_OK) use_graph = false;
    if (use_graph) {
      if (cudaGraphLaunch(p->gexec, st) != cudaSuccess) return GSOFA_E_CUDA;
    } else if (enqueue_phase1(*p, o, st, p->ev0, p->ev1) != cudaSuccess) {
      return GSOFA_E_CUDA;
    }
    *launches += 4 + (o.validate != 2 ? 1 : 0);
    int rc = wait_stream(st);
    if (rc) return rc;
    const DevCounters* h = p->hctr();
    if (h->err & ERR_INPUT) return GSOFA_E_INVAL;
    if (h->err & ERR_NOCONV) return GSOFA_E_NOCONVERGE;
    note_pool_use(c, h->pool_cursor, p->N);
    if (!(h->err & ERR_OVERFLOW)) return GSOFA_OK;
    // the row pool was too small; the totals are exact now
    const long long need = (long long)h->pool_cursor + ((long long)h->pool_cursor >> 4) + 1024;
    cudaError_t ea;
    if (p->transient) {
      cudaFreeAsync(p->pool, st);
      p->pool = nullptr;
      ea = palloc(c, &p->pool, (size_t)need, st);
    } else {
      cudaFree(p->pool);
      p->pool = nullptr;
      ea = cudaMalloc(&p->pool, sizeof(uint32_t) * (size_t)need);
    }
    if (ea != cudaSuccess) {
      cudaGetLastError();
      p->pool_cap = 0;
      return GSOFA_E_NOMEM;
    }
    p->pool_cap = need;
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
  }
  return GSOFA_E_NOMEM;
}

// Phase 2: exact outputs for every member in one shared allocation.
int batch_phase2(Ctx* c, BatchPlan* p, const int32_t* n, cudaStream_t st, gsofa_result* outs, int* launches) {
  const DevCounters* h = p->hctr();
  const int64_t total_L = (int64_t)h->total_L, total_U = (int64_t)h->total_U;
  const int64_t total_super = h->n_super;
  SharedBlock* blk = new SharedBlock();
  blk->stream = st;
  blk->device = c->device;
  int64_t *Lrp = nullptr, *Urp = nullptr, *GL = nullptr, *GU = nullptr, *P = nullptr;
  int32_t *Lci = nullptr, *Uci = nullptr, *sup = nullptr, *fill = nullptr;
  void* tmp = nullptr;
  bool ok = palloc(c, &Lrp, (size_t)(p->N + p->B), st) == cudaSuccess &&
            palloc(c, &Urp, (size_t)(p->N + p->B), st) == cudaSuccess &&
            palloc(c, &Lci, (size_t)total_L, st) == cudaSuccess && palloc(c, &Uci, (size_t)total_U, st) == cudaSuccess &&
            palloc(c, &sup, (size_t)(total_super + p->B), st) == cudaSuccess &&
            palloc(c, &fill, (size_t)p->N, st) == cudaSuccess && palloc(c, &GL, (size_t)p->N + 1, st) == cudaSuccess &&
            palloc(c, &GU, (size_t)p->N + 1, st) == cudaSuccess && palloc(c, &P, (size_t)p->N + 1, st) == cudaSuccess &&
            cudaMallocFromPoolAsync(&tmp, scan_tmp_bytes_long(p->N), c->mpool, st) == cudaSuccess;
  for (void* q : {(void*)Lrp, (void*)Urp, (void*)Lci, (void*)Uci, (void*)sup, (void*)fill})
    if (q) blk->ptrs.push_back(q);
  cudaError_t e = ok ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = launch_scan_i32_i64_long(p->row_nL, GL, p->N, tmp, st);
  if (e == cudaSuccess) e = launch_scan_i32_i64_long(p->row_nU, GU, p->N, tmp, st);
  if (e == cudaSuccess) e = launch_rebase_rowptr(p->d_mats, p->B, p->N, GL, Lrp, st);
  if (e == cudaSuccess) e = launch_rebase_rowptr(p->d_mats, p->B, p->N, GU, Urp, st);
  if (e == cudaSuccess) e = launch_compact_long(p->N, p->pool, p->row_off, p->row_nL, p->row_nU, GL, GU, Lci, Uci, st);
  if (e == cudaSuccess) e = launch_scan_i32_i64_long(p->flags, P, p->N, tmp, st);
  if (e == cudaSuccess) e = launch_scatter_starts_batch(p->d_mats, p->B, p->N, p->flags, P, sup, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(fill, p->fill, sizeof(int32_t) * (size_t)p->N, cudaMemcpyDeviceToDevice, st);
  *launches += 3 * 3 + 4;
  pfree(GL, st);
  pfree(GU, st);
  pfree(P, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (void* q : blk->ptrs) cudaFreeAsync(q, st);
    delete blk;
    return ok ? GSOFA_E_CUDA : GSOFA_E_NOMEM;
  }
  // views into the block (host-side prefix sums of the per-matrix totals)
  const unsigned long long* tot = p->h_tot();
  const int32_t* ns = p->h_nsuper();
  int64_t offL = 0, offU = 0, offS = 0;
  blk->refs.store(p->B);
  for (int32_t k = 0; k < p->B; k++) {
    gsofa_result* r = &outs[p->members[k]];
    zero_result(r);
    Priv* pv = new Priv();
    pv->stream = st;
    pv->device = c->device;
    pv->shared = blk;
    r->_priv = pv;
    r->n = n[p->members[k]];
    r->on_device = 1;
    r->err_detail = -1;
    r->nnz_L = (int64_t)tot[2 * k];
    r->nnz_U = (int64_t)tot[2 * k + 1];
    r->n_super = ns[k];
    r->L_rowptr = Lrp + p->row_base[k] + k;
    r->U_rowptr = Urp + p->row_base[k] + k;
    r->L_colidx = Lci + offL;
    r->U_colidx = Uci + offU;
    r->fill_count = fill + p->row_base[k];
    r->super_start = sup + offS + k;
    offL += r->nnz_L;
    offU += r->nnz_U;
    offS += ns[k];
  }
  if (p->B == 0) delete blk;
  if (p->ev0 && p->B > 0) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess) {
      outs[p->members[0]].stats.ms_traverse = ms;
      if (p->shape.kernel == 1) outs[p->members[0]].stats.ms_traverse_global = ms;
      else outs[p->members[0]].stats.ms_traverse_smem = ms;
    }
    cudaGetLastError();
  }
  if (p->B > 0) {  // counters of the batched launch (collect_stats)
    const DevCounters* h = p->hctr();
    gsofa_stats& sm = outs[p->members[0]].stats;
    sm.vertices_expanded = (int64_t)h->expansions;
    sm.edges_scanned = (int64_t)h->edges;
    sm.levels = (int64_t)h->levels;
    sm.cycles_traverse = (int64_t)h->cyc_trav;
    sm.cycles_emit = (int64_t)h->cyc_emit;
  }
  return GSOFA_OK;
}

LaunchShape default_shape(Ctx* c, BatchCache& bc, const BatchPlan* p, const gsofa_options& o, size_t limit, int* rc) {
  LaunchShape sh;
  const uint64_t key = bucket_key(p->n_max, p->N, p->label16) ^ ((uint64_t)o.threads_per_source << 48);
  auto tt = bc.tuned.find(key);
  if (tt != bc.tuned.end() && o.list_capacity == 0 && o.work_chunk == 0) return tt->second;
  if (o.threads_per_source == 0 && o.list_capacity == 0 && o.work_chunk == 0 && o.frontier_order != 1) {
    // untuned default: the class-ordered warp tier (fewest expansions), 40 warps per SM
    sh.kernel = 1;
    sh.occ = 40;
    sh.slots = class_slots(c, p->n_max, 40);
    if (o.max_ctas > 0 && sh.slots > o.max_ctas * CLASS_WARPS_PER_CTA) sh.slots = o.max_ctas * CLASS_WARPS_PER_CTA;
    if (sh.slots > 0) { *rc = GSOFA_OK; return sh; }
    sh.kernel = 0;
  }
  int32_t cap = 0;
  *rc = choose_smem_config(c->sms, limit, p->n_max, p->n_max, p->label16, o.threads_per_source, &sh.block, &sh.occ,
                           &cap);
  if (o.list_capacity > 0 && o.list_capacity < cap) cap = o.list_capacity < 32 ? 32 : o.list_capacity;
  sh.list_cap = cap;
  sh.work_chunk = o.work_chunk > 0 ? o.work_chunk : 1;
  return sh;
}

// Batched path for the members that fit the shared-memory tier.  transient:
// one-off composition (served batches): pooled workspace, no graph, no cache.
int run_batch_members(Ctx* c, const std::vector<int32_t>& members, const int32_t* n, const int32_t* const* rp,
                      const int32_t* const* ci, const gsofa_options& o, cudaStream_t st, gsofa_result* outs,
                      int* launches, bool transient, const int64_t* pool_entries) {
  BatchCache& bc = g_batch[c->device];
  const int stat = trav_smem_static_bytes();
  const size_t limit = (size_t)c->smem_optin - (size_t)stat - 64;
  if (transient) {
    BatchPlan* p = nullptr;
    int64_t pe = 0;
    if (pool_entries)
      for (int32_t k : members) pe += pool_entries[k];
    int rc = build_plan(c, members, n, rp, ci, o, 0, &p, true, st, pe);
    if (rc) return rc;
    {
      std::lock_guard<std::mutex> lk(bc.mu);
      load_tune_file(bc);
      LaunchShape sh = default_shape(c, bc, p, o, limit, &rc);
      // a caller's cap on sources in flight (a server's memory share) bounds the slots
      if (sh.kernel == 1 && o.max_concurrent > 0 && sh.slots > o.max_concurrent) sh.slots = o.max_concurrent;
      if (rc == GSOFA_OK) rc = set_shape(c, p, sh);
    }
    if (rc == GSOFA_OK) rc = batch_phase1(c, p, o, st, false, launches);
    if (rc == GSOFA_OK) rc = batch_phase2(c, p, n, st, outs, launches);
    free_plan(p);
    return rc;
  }
  uint64_t sig = 0x5EED;
  for (int32_t k : members) {
    sig = mix64(sig, (uint64_t)k);  // position in the caller's arrays
    sig = mix64(sig, (uint64_t)n[k]);
    sig = mix64(sig, (uint64_t)(uintptr_t)rp[k]);
    sig = mix64(sig, (uint64_t)(uintptr_t)ci[k]);
  }
  sig = mix64(sig, ((uint64_t)o.chunk_size << 32) ^ ((uint64_t)o.fill_first << 8) ^ (uint64_t)o.validate);
  sig = mix64(sig, ((uint64_t)o.work_chunk << 32) ^ ((uint64_t)o.list_capacity << 4) ^ (uint64_t)o.threads_per_source);
  sig = mix64(sig, ((uint64_t)o.collect_stats << 32) ^ (uint64_t)o.max_ctas);
  sig = mix64(sig, ((uint64_t)o.frontier_order << 48) ^ ((uint64_t)o.expand_mode << 32) ^
                       ((uint64_t)o.label_bits << 16) ^ (uint64_t)o.autotune);
  sig = mix64(sig, ((uint64_t)(uint32_t)o.clean_heads << 32) ^ (uint64_t)(uint32_t)o.team_sources);
  std::unique_lock<std::mutex> lk(bc.mu);  // cached plans are used by one call at a time
  load_tune_file(bc);
  BatchPlan* p = nullptr;
  auto it = bc.plans.find(sig);
  if (it != bc.plans.end()) {
    p = it->second;
  } else {
    int rc = build_plan(c, members, n, rp, ci, o, sig, &p, false, st);
    if (rc) return rc;
    const uint64_t key = bucket_key(p->n_max, p->N, p->label16) ^ ((uint64_t)o.threads_per_source << 48);
    if (o.autotune && o.threads_per_source == 0 && o.list_capacity == 0 && o.work_chunk == 0 &&
        bc.tuned.find(key) == bc.tuned.end()) {
      rc = autotune_plan(c, p, o, st, limit);
      if (rc) { free_plan(p); return rc; }
      bc.tuned[key] = p->shape;
      save_tune_entry(key, p->shape);
    } else {
      const LaunchShape sh = default_shape(c, bc, p, o, limit, &rc);
      if (rc == GSOFA_OK) rc = set_shape(c, p, sh);
      if (rc) { free_plan(p); return rc; }
    }
    if (bc.plans.size() >= 8) {  // keep at most 8 plans: drop the least recently used
      auto victim = bc.plans.begin();
      for (auto jt = bc.plans.begin(); jt != bc.plans.end(); ++jt)
        if (jt->second->last_use < victim->second->last_use) victim = jt;
      cudaDeviceSynchronize();
      free_plan(victim->second);
      bc.plans.erase(victim);
    }
    bc.plans[sig] = p;
  }
  p->last_use = ++bc.clock;
  int rc = batch_phase1(c, p, o, st, true, launches);
  if (rc == GSOFA_E_NOMEM) {
    bc.plans.erase(p->sig);
    free_plan(p);
    return rc;
  }
  if (rc) return rc;
  return batch_phase2(c, p, n, st, outs, launches);
}

int run_batch(Ctx* c, int32_t count, const int32_t* n, const int32_t* const* rp, const int32_t* const* ci,
              const gsofa_options& o, cudaStream_t st, gsofa_result* outs, bool transient,
              const int64_t* pool_entries = nullptr) {
  for (int32_t k = 0; k < count; k++) zero_result(&outs[k]);
  // members: matrices whose every source fits the shared-memory tier together
  const int stat = trav_smem_static_bytes();
  const size_t limit = (size_t)c->smem_optin - (size_t)stat - 64;
  std::vector<int32_t> idx(count);
  for (int32_t k = 0; k < count; k++) {
    if (n[k] < 0 || !rp[k] || (n[k] > 0 && !ci[k])) return GSOFA_E_INVAL;
    idx[k] = k;
  }
  std::vector<int32_t> members, singles;
  for (int32_t k = 0; k < count; k++) {
    const int32_t nk = n[k];
    if (nk == 0) { singles.push_back(k); continue; }
    const int l16 = nk <= 65533 ? 1 : 0;
    if (o.smem_max_source == 0 && trav_smem_max_S(nk, limit, l16) >= nk) members.push_back(k);
    else singles.push_back(k);
  }
  int launches = 0;
  int rc = GSOFA_OK;
  if (!members.empty())
    rc = run_batch_members(c, members, n, rp, ci, o, st, outs, &launches, transient, pool_entries);
  for (size_t j = 0; rc == GSOFA_OK && j < singles.size(); j++) {
    const int32_t k = singles[j];
    rc = run_device(c, n[k], rp[k], ci[k], o, st, &outs[k], pool_entries ? pool_entries[k] : 0);
    if (rc == GSOFA_OK) launches += outs[k].stats.kernel_launches;
  }
  if (rc != GSOFA_OK) {
    for (int32_t k = 0; k < count; k++) gsofa_free(&outs[k]);
    return rc;
  }
  if (count > 0) outs[0].stats.kernel_launches = launches;
  return GSOFA_OK;
}

}  // namespace

// Served batches: one-off composition, pooled workspace, no graph (serve.cu).
int batch_transient(int32_t count, const int32_t* n, const int32_t* const* rp, const int32_t* const* ci,
                    const gsofa_options* opt, cudaStream_t st, gsofa_result* outs, const int64_t* pool_entries) {
  gsofa_options o;
  if (check_options(opt, &o) != GSOFA_OK) return GSOFA_E_INVAL;
  if (count <= 0) return count == 0 ? GSOFA_OK : GSOFA_E_INVAL;
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return err;
  return run_batch(c, count, n, rp, ci, o, st, outs, true, pool_entries);
}

int64_t global_slot_bytes(int32_t n) { return slot_bytes(((int64_t)n + 1023) / 1024 * 1024); }

int64_t global_device_slot_bytes(int32_t n) { return device_slot_bytes(((int64_t)n + 1023) / 1024 * 1024); }

int32_t batch_class_slots(int32_t n_max) {
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  return c ? class_slots(c, n_max, 40) : 0;
}

int64_t library_pool_bytes(int high, int reset_high) {
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return 0;
  uint64_t v = 0;
  if (cudaMemPoolGetAttribute(c->mpool, high ? cudaMemPoolAttrUsedMemHigh : cudaMemPoolAttrUsedMemCurrent, &v) !=
      cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  if (reset_high) {
    uint64_t z = 0;
    cudaMemPoolSetAttribute(c->mpool, cudaMemPoolAttrUsedMemHigh, &z);
  }
  return (int64_t)v;
}

int64_t library_slot_bytes() {
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return 0;
  std::lock_guard<std::mutex> lk(c->gmu);
  return c->g_V ? (int64_t)c->g_slots * slot_bytes(c->g_cap) : 0;
}

int64_t global_tier_bytes(int32_t n, const gsofa_options* opts) {
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return 0;
  gsofa_options o;
  if (check_options(opts, &o) != GSOFA_OK) gsofa_default_options(&o);
  const int64_t cap = ((int64_t)n + 1023) / 1024 * 1024;
  return global_slots(c, n, o) * slot_bytes(cap);
}

int device_sms() {
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  return c ? c->sms : 0;
}

int32_t smem_tier_max_order() {
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return 0;
  const size_t limit = (size_t)c->smem_optin - (size_t)trav_smem_static_bytes() - 64;
  // largest n whose every source fits the shared-memory tier (16-bit labels)
  int32_t lo = 0, hi = 65533;
  while (lo < hi) {
    const int32_t mid = (int32_t)(((int64_t)lo + hi + 1) / 2);
    if (trav_smem_max_S(mid, limit, 1) >= mid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

namespace {
}  // namespace

// A completed result whose producing stream may go away: free it unordered.
void detach_result_stream(gsofa_result* r) {
  Priv* pv = (Priv*)r->_priv;
  if (!pv) return;
  pv->stream = nullptr;
  if (pv->shared) pv->shared->stream = nullptr;
}

namespace {
}  // namespace
}  // namespace gsofa

using namespace gsofa;

extern "C" {

int gsofa_version(void) { return 10000; }

const char* gsofa_strerror(int code) {
  switch (code) {
    case GSOFA_OK: return "ok";
    case GSOFA_E_INVAL: return "invalid argument or malformed CSR";
    case GSOFA_E_NOMEM: return "out of memory or memory budget too small";
    case GSOFA_E_CUDA: return "CUDA runtime error";
    case GSOFA_E_NOCONVERGE: return "traversal iteration cap reached";
    case GSOFA_E_TIMEOUT: return "bounded wait timed out";
    case GSOFA_E_BUSY: return "admission queue full";
    case GSOFA_E_NOTFOUND: return "unknown ticket";
    case GSOFA_E_PENDING: return "request still pending";
    default: return "unknown error";
  }
}

int gsofa_default_options(gsofa_options* opt) {
  if (!opt) return GSOFA_E_INVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->chunk_size = 128;
  opt->validate = 1;
  return GSOFA_OK;
}

void gsofa_free(gsofa_result* res) {
  if (!res) return;
  Priv* pv = (Priv*)res->_priv;
  if (res->on_device && pv && pv->shared) {
    SharedBlock* b = pv->shared;
    if (b->refs.fetch_sub(1) == 1) {
      int cur = -1;
      cudaGetDevice(&cur);
      if (cur != b->device) cudaSetDevice(b->device);
      for (void* q : b->ptrs) cudaFreeAsync(q, b->stream);
      if (cur != b->device && cur >= 0) cudaSetDevice(cur);
      delete b;
    }
  } else if (res->on_device) {
    cudaStream_t st = pv ? pv->stream : nullptr;
    int cur = -1;
    cudaGetDevice(&cur);
    if (pv && cur != pv->device) cudaSetDevice(pv->device);
    pfree(res->L_rowptr, st);
    pfree(res->L_colidx, st);
    pfree(res->U_rowptr, st);
    pfree(res->U_colidx, st);
    pfree(res->fill_count, st);
    pfree(res->super_start, st);
    if (pv && cur != pv->device && cur >= 0) cudaSetDevice(cur);
  } else if (pv) {
    pinned_put(pv->host_block, pv->host_cap);
  }
  delete pv;
  std::memset(res, 0, sizeof(*res));
}

namespace {

// One matrix: pick the frontier order (class order unless autotuned), then run.
// Autotune reads nnz (device input: one read) and keeps its choice per (n, nnz).
int run_single(Ctx* c, int32_t n, const int32_t* d_rowptr, const int32_t* d_colidx, gsofa_options o,
               cudaStream_t st, gsofa_result* out, int64_t nnz_known) {
  const bool tune = o.autotune && o.frontier_order == 0 && n > 0;
  if (o.frontier_order == 0 && !tune) {
    // class order for every source (the fewest expansions and the fastest on
    // every workload measured); an explicit smem_max_source keeps the sources
    // below it in the breadth-first shared-memory tier
    o.frontier_order = o.smem_max_source > 0 ? 1 : 2;
  }
  int64_t nnz = nnz_known;
  if (tune && nnz < 0) {
    int32_t v = 0;
    if (cudaMemcpyAsync(&v, d_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        wait_stream(st) != GSOFA_OK)
      return GSOFA_E_CUDA;
    nnz = v;
  }
  if (tune) {
    // time once per shape: breadth-first without and with the fill-first check
    // (Section 4, "line 9.5"), and class order; keep the fastest
    const std::pair<int32_t, int64_t> key(n, nnz);
    int best = 0;
    {
      std::lock_guard<std::mutex> lk(c->hmu);
      auto it = c->order_tuned.find(key);
      if (it != c->order_tuned.end()) best = it->second;
    }
    if (best == 0) {
      float ms[4] = {0.f, 0.f, 0.f, 0.f};
      for (int cand = 1; cand <= 3; cand++) {  // 1 breadth-first, 2 class order, 3 breadth-first + fill-first
        gsofa_options t = o;
        t.frontier_order = cand == 2 ? 2 : 1;
        t.fill_first = cand == 3 ? 1 : o.fill_first;
        t.collect_stats = 2;  // phase times without the work counters
        t.autotune = 0;
        for (int rep = 0; rep < 2; rep++) {  // the first run also sizes the row pool
          gsofa_result r;
          const int rc = run_device(c, n, d_rowptr, d_colidx, t, st, &r);
          if (rc) return rc;
          ms[cand] = r.stats.ms_traverse;
          gsofa_free(&r);
        }
      }
      best = 1;
      for (int cand = 2; cand <= 3; cand++)
        if (ms[cand] < ms[best]) best = cand;
      std::lock_guard<std::mutex> lk(c->hmu);
      c->order_tuned[key] = best;
    }
    o.frontier_order = best == 2 ? 2 : 1;
    if (best == 3) o.fill_first = 1;
  }
  return run_device(c, n, d_rowptr, d_colidx, o, st, out);
}

}  // namespace

int gsofa_symbolic_device(int32_t n, const int32_t* d_rowptr, const int32_t* d_colidx,
                          const gsofa_options* opt, void* stream, gsofa_result* out) {
  if (!out) return GSOFA_E_INVAL;
  zero_result(out);
  out->err_detail = -1;
  gsofa_options o;
  if (check_options(opt, &o) != GSOFA_OK) return GSOFA_E_INVAL;
  if (n < 0 || !d_rowptr || (n > 0 && !d_colidx)) return GSOFA_E_INVAL;
  if (n > INT32_MAX - 2) return GSOFA_E_INVAL;
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return err;
  cudaStream_t st = (cudaStream_t)stream;
  return run_single(c, n, d_rowptr, d_colidx, o, st, out, -1);
}

int gsofa_symbolic(int32_t n, const int32_t* rowptr, const int32_t* colidx, const gsofa_options* opt,
                   gsofa_result* out) {
  if (!out) return GSOFA_E_INVAL;
  zero_result(out);
  out->err_detail = -1;
  if (n < 0 || !rowptr || (n > 0 && !colidx)) return GSOFA_E_INVAL;
  if (rowptr[0] != 0 || rowptr[n] < 0) { out->err_detail = 0; return GSOFA_E_INVAL; }
  gsofa_options o;
  if (check_options(opt, &o) != GSOFA_OK) return GSOFA_E_INVAL;
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return err;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return GSOFA_E_CUDA;
  const int64_t nnz = rowptr[n];
  int32_t *d_rp = nullptr, *d_ci = nullptr;
  gsofa_result dres;
  zero_result(&dres);
  int rc = GSOFA_OK;
  if (palloc(c, &d_rp, (size_t)n + 1, st) != cudaSuccess || palloc(c, &d_ci, (size_t)nnz, st) != cudaSuccess) {
    rc = GSOFA_E_NOMEM;
  } else if (cudaMemcpyAsync(d_rp, rowptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess ||
             (nnz > 0 && cudaMemcpyAsync(d_ci, colidx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice,
                                         st) != cudaSuccess)) {
    rc = GSOFA_E_CUDA;
  } else {
    rc = run_single(c, n, d_rp, d_ci, o, st, &dres, nnz);
  }
  if (rc == GSOFA_OK) {
    out->n = n;
    out->n_super = dres.n_super;
    out->nnz_L = dres.nnz_L;
    out->nnz_U = dres.nnz_U;
    out->stats = dres.stats;
    out->on_device = 0;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_rp = al(8 * ((size_t)n + 1)), b_lc = al(4 * (size_t)dres.nnz_L + 4),
                 b_uc = al(4 * (size_t)dres.nnz_U + 4), b_fc = al(4 * (size_t)n + 4),
                 b_ss = al(4 * ((size_t)dres.n_super + 1));
    Priv* hp = new Priv();
    hp->device = c->device;
    out->_priv = hp;
    char* blk = (char*)pinned_get(2 * b_rp + b_lc + b_uc + b_fc + b_ss, &hp->host_cap);
    hp->host_block = blk;
    if (!blk) {
      rc = GSOFA_E_NOMEM;
    } else {
      out->L_rowptr = (int64_t*)blk;
      out->U_rowptr = (int64_t*)(blk + b_rp);
      out->L_colidx = (int32_t*)(blk + 2 * b_rp);
      out->U_colidx = (int32_t*)(blk + 2 * b_rp + b_lc);
      out->fill_count = (int32_t*)(blk + 2 * b_rp + b_lc + b_uc);
      out->super_start = (int32_t*)(blk + 2 * b_rp + b_lc + b_uc + b_fc);
      cudaError_t e = cudaSuccess;
      e = e ? e : cudaMemcpyAsync(out->L_rowptr, dres.L_rowptr, 8 * ((size_t)n + 1), cudaMemcpyDeviceToHost, st);
      e = e ? e : cudaMemcpyAsync(out->U_rowptr, dres.U_rowptr, 8 * ((size_t)n + 1), cudaMemcpyDeviceToHost, st);
      if (dres.nnz_L > 0)
        e = e ? e : cudaMemcpyAsync(out->L_colidx, dres.L_colidx, 4 * (size_t)dres.nnz_L, cudaMemcpyDeviceToHost, st);
      if (dres.nnz_U > 0)
        e = e ? e : cudaMemcpyAsync(out->U_colidx, dres.U_colidx, 4 * (size_t)dres.nnz_U, cudaMemcpyDeviceToHost, st);
      if (n > 0)
        e = e ? e : cudaMemcpyAsync(out->fill_count, dres.fill_count, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
      e = e ? e : cudaMemcpyAsync(out->super_start, dres.super_start, 4 * ((size_t)dres.n_super + 1),
                                  cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) rc = GSOFA_E_CUDA;
      const int w = wait_stream(st);
      if (rc == GSOFA_OK) rc = w;
    }
  } else {
    out->err_detail = dres.err_detail;
  }
  gsofa_free(&dres);
  pfree(d_rp, st);
  pfree(d_ci, st);
  wait_stream(st);
  cudaStreamDestroy(st);
  if (rc != GSOFA_OK) {
    const int32_t det = out->err_detail;
    gsofa_free(out);
    out->err_detail = det;
  }
  return rc;
}

int gsofa_batch(int32_t count, const int32_t* n, const int32_t* const* d_rowptr, const int32_t* const* d_colidx,
                const gsofa_options* opt, void* stream, gsofa_result* outs) {
  if (count < 0 || (count > 0 && (!n || !d_rowptr || !d_colidx || !outs))) return GSOFA_E_INVAL;
  gsofa_options o;
  if (check_options(opt, &o) != GSOFA_OK) return GSOFA_E_INVAL;
  if (count == 0) return GSOFA_OK;
  int err = GSOFA_OK;
  Ctx* c = get_ctx(&err);
  if (!c) return err;
  return run_batch(c, count, n, d_rowptr, d_colidx, o, (cudaStream_t)stream, outs, false);
}

}  // extern "C"
