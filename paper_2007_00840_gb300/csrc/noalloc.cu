// gsofa_row_counts_noalloc: per-row L/U sizes and fill counts without any
// device allocation.
//
// Some callers cannot allocate device memory when they need the sizes of the
// factors: a solver that reserved all free device memory for itself at start-up
// and hands out sub-buffers, a latency-critical loop in which cudaMalloc or
// cudaFree would synchronise the device, or a host process that forbids
// allocation after initialisation.  They pass their own input and output
// buffers; everything else the kernels need (the counters block and the
// overflow area of the frontier lists) lives in the fixed array below, which
// every GPU that loads this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "gsofa.h"
#include "internal.cuh"

namespace gsofa {
namespace {

static_assert(GSOFA_NOALLOC_SCRATCH_BYTES >= 4096, "scratch too small");
static_assert(sizeof(DevCounters) <= 256, "the counters block must fit ahead of the overflow lists");

// Scratch of this entry point: [0, 256) counters, then frontier overflow lists.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GSOFA_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_dev_addr[128] = {nullptr};
int g_sms[128] = {0};
int g_optin[128] = {0};

// Device address of the scratch array on the current device (the name is only
// a host-side stand-in in host code).  Resolved once per device.
int scratch_address(int dev, void** out, int* sms, int* optin) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GSOFA_E_CUDA;
    }
    if (cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_optin[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return GSOFA_E_CUDA;
    }
    g_dev_addr[dev] = p;
  }
  *out = g_dev_addr[dev];
  *sms = g_sms[dev];
  *optin = g_optin[dev];
  return GSOFA_OK;
}

}  // namespace
}  // namespace gsofa

using namespace gsofa;

extern "C" int gsofa_row_counts_noalloc(int32_t n, const int32_t* d_rowptr, const int32_t* d_colidx,
                                        int32_t* d_nnzL, int32_t* d_nnzU, int32_t* d_fill_count, void* stream) {
  if (n < 0 || n > GSOFA_NOALLOC_MAX_N || !d_rowptr) return GSOFA_E_INVAL;
  if (n > 0 && (!d_colidx || !d_nnzL || !d_nnzU || !d_fill_count)) return GSOFA_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return GSOFA_E_CUDA;
  void* base = nullptr;
  int sms = 0, optin = 0;
  int rc = scratch_address(dev, &base, &sms, &optin);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DevCounters* ctr = (DevCounters*)base;
  int32_t* spill = (int32_t*)((unsigned char*)base + 256);
  const size_t spill_bytes = GSOFA_NOALLOC_SCRATCH_BYTES - 256;

  // every source in the shared-memory tier with 16-bit maxId labels
  const int label16 = 1;
  const int stat = trav_smem_static_bytes();
  const size_t limit = (size_t)optin - (size_t)stat - 64;
  int block = 0, occ = 0;
  int32_t cap = 0;
  if (n > 0) {
    if (trav_smem_max_S(n, limit, label16) < n) return GSOFA_E_INVAL;
    rc = choose_smem_config(sms, limit, n, n, label16, 0, &block, &occ, &cap);
    if (rc) return rc;
  }
  const int64_t spill_cap = n > cap ? (int64_t)n - cap : 1;
  long long grid = (long long)sms * occ;
  const long long fit = (long long)(spill_bytes / (2 * sizeof(int32_t) * (size_t)spill_cap));
  if (grid > fit) grid = fit;  // fewer CTAs when the overflow lists would not fit the scratch
  if (n > 0 && grid < 1) return GSOFA_E_NOMEM;

  // the counters must start at zero on every call; the overflow lists need no reset
  if (launch_init_counters(ctr, st) != cudaSuccess) return GSOFA_E_CUDA;
  if (launch_validate(n, d_rowptr, d_colidx, ctr, st) != cudaSuccess) return GSOFA_E_CUDA;
  if (n > 0) {
    TravArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.rowptr = d_rowptr;
    a.colidx = d_colidx;
    a.order = nullptr;  // sources n-1 .. 0
    a.nsrc = n;
    a.S = n;
    a.list_cap = cap;
    a.spill = spill;
    a.spill_cap = spill_cap;
    a.row_nL = d_nnzL;
    a.row_nU = d_nnzU;
    a.fill_count = d_fill_count;
    a.ctr = ctr;
    a.counts_only = 1;
    a.expand_mode = 1;
    if (launch_trav_smem(a, (int)grid, block, label16, st) != cudaSuccess) return GSOFA_E_CUDA;
  }
  DevCounters h;
  if (cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GSOFA_E_CUDA;
  rc = wait_stream(st);
  if (rc) return rc;
  if (h.err & ERR_INPUT) return GSOFA_E_INVAL;
  if (h.err & ERR_NOCONV) return GSOFA_E_NOCONVERGE;
  return GSOFA_OK;
}
