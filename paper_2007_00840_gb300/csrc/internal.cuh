// Internal declarations shared by the CUDA translation units of libgsofa.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gsofa.h"

namespace gsofa {

// ---- device error word bits (err[0]); err[1] keeps the first offending row
enum : int32_t {
  ERR_COL_RANGE = 1,   // a column index outside [0, n)
  ERR_ROWPTR = 2,      // rowptr[0] != 0, decreasing rowptr, or rowptr[n] inconsistent
  ERR_UNSORTED = 4,    // columns not strictly increasing inside a row
  ERR_NOCONV = 8,      // traversal iteration cap reached
  ERR_OVERFLOW = 16,   // row pool too small (the host grows it and reruns)
  ERR_INPUT = ERR_COL_RANGE | ERR_ROWPTR | ERR_UNSORTED,
};


constexpr unsigned FULL = 0xFFFFFFFFu;

// Counters in one small device block so one copy brings them back.
struct DevCounters {
  unsigned long long pool_cursor;   // entries requested from the row pool
  unsigned long long total_L;       // sum of nnz(L(i,:))
  unsigned long long total_U;       // sum of nnz(U(i,:)) (diagonal included)
  unsigned long long expansions;    // frontier expansions (stats)
  unsigned long long edges;         // adjacency entries read (stats)
  int32_t err;                      // ERR_* bits
  int32_t err_row;                  // first offending row (atomicMin), INT32_MAX if none
  int32_t n_super;                  // supernodes found
  int32_t work_smem;                // work counter of the shared-memory tier
  int32_t work_global;              // work counter of the global tier (class kernel: warp items)
  int32_t work_team;                // class kernel: work counter of the CTA-team items
  int32_t pad[2];
  unsigned long long levels;        // frontier levels over all sources (stats)
  unsigned long long cyc_trav;      // SM cycles in frontier levels (stats, thread 0 of each CTA)
  unsigned long long cyc_emit;      // SM cycles in row emission (stats)
};

// Input errors found so far (read through L2, not a cached copy).
__device__ __forceinline__ int input_error(const DevCounters* c) {
  return *(const volatile int32_t*)&c->err & ERR_INPUT;
}

// One matrix of a batch: its CSR and where its rows sit in the concatenated
// per-row arrays (row_base) and in the concatenated supernode chunks.
struct MatDesc {
  const int32_t* rowptr;
  const int32_t* colidx;
  int32_t n;
  int32_t pad;
  int64_t row_base;
  int64_t chunk_base;
};

// Arguments of the traversal kernels (Section 4, Fig. 5).
struct TravArgs {
  int32_t n;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colidx;
  const int32_t* __restrict__ order;  // source rows to process, in order of issue (null: nsrc-1 .. 0)
  int32_t nsrc;
  int32_t S;                          // shared tier: label capacity (all sources < S)
  int32_t list_cap;                   // shared tier: frontier list capacity in shared memory
  int32_t* spill;                     // shared tier: per CTA 2 x spill_cap overflow entries
  int64_t spill_cap;
  uint32_t* pool;                     // row pool: per source [L cols | s | U cols]
  int64_t pool_cap;                   // entries
  int64_t* row_off;                   // per row: pool offset (-1 if it did not fit)
  int32_t* row_nL;
  int32_t* row_nU;
  int32_t* fill_count;
  DevCounters* ctr;
  int32_t fill_first;                 // optional "line 9.5" of Section 4
  int32_t collect_stats;
  int32_t counts_only;                // 1: write per-row counts only (no pool, no row_off)
  int32_t expand_mode;                // shared tier: 1 row slots, 2 edge-balanced
  const int4* ell;                    // shared tier: 16-bit offset copy of A (null: CSR only)
  // batch mode (mats != nullptr): item k -> source s (descending) and matrix m;
  // item_start[s] = number of items with a larger source index, mat_order lists
  // matrices by decreasing order n; n above is the largest order in the batch
  const MatDesc* mats;
  const int32_t* item_start;
  const int32_t* mat_order;
  int32_t nmats;
  int32_t chunk;                      // work items taken per fetch (>= 1)
  unsigned long long* mat_tot;        // per matrix: [sum nnz(L(i,:)), sum nnz(U(i,:))]
  int64_t g_cap;                      // class kernel: per-slot capacity in vertices (>= n, multiple of 1024)
  int32_t g_slots;                    // class kernel: number of slots (warps) of the launch
  int32_t async_sched;                // shared-memory tier: worklist without level barriers (16-bit, S >= n)
  // class-ordered kernel (trav_class_kernel): per-slot visited bitmaps and
  // logs; slot = warp of the launch, each g_cap vertices
  uint32_t* g_V;                      // slots x g_cap/32 (global V only)
  uint32_t* g_VS;                     // slots x g_cap/1024 (summary of g_V)
  int32_t* g_log;                     // slots x g_cap (level overflow from the bottom, L row from the top)
  int32_t ct_qw;                      // shared queue entries per warp and level parity
  int32_t ct_vwords;                  // shared V: words per warp (>= ceil(n/32))
  int32_t ct_nbig;                    // leading work items processed by four-warp CTA teams
  int32_t ct_heads;                   // clean-head gathers: -1 off, 0 adaptive, 1 before every class
  const int4* ellw;                   // class kernel: 32-bit column records, row v at ellw[2v..2v+1] (null: ell)
};

// ---- launchers (return cudaGetLastError())
size_t trav_smem_bytes(int32_t n, int32_t S, int32_t cap, int label16);
int32_t trav_smem_max_S(int32_t n, size_t smem_limit, int label16);
cudaError_t launch_trav_smem(const TravArgs& a, int grid, int block, int label16, cudaStream_t st);
int trav_smem_static_bytes();
int trav_smem_occupancy(int block, size_t dyn_bytes, int label16);
// Class-ordered kernel with a visited bitmap (four-warp CTAs).  vm: where the
// bitmaps live (0 shared memory, ct_vwords words per warp; 1 global slots);
// warps_per_sm above 32: 48-register build.
cudaError_t launch_trav_class(const TravArgs& a, int grid, int vm, int warps_per_sm, cudaStream_t st);
int trav_class_occupancy(int vm, int warps_per_sm, int vwords, int qw);
size_t trav_class_smem(int vm, int vwords, int qw);
constexpr int CLASS_WARPS_PER_CTA = 4;

cudaError_t launch_validate(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                            DevCounters* ctr, cudaStream_t st);
cudaError_t launch_validate_batch(const MatDesc* mats, int32_t nmats, int64_t total_rows, DevCounters* ctr,
                                  cudaStream_t st);
cudaError_t launch_supernode_batch(const MatDesc* mats, int32_t nmats, int64_t total_chunks, int32_t chunk,
                                   const uint32_t* pool, const int64_t* row_off, const int32_t* row_nL,
                                   const int32_t* row_nU, int32_t* flags, int32_t* mat_nsuper, DevCounters* ctr,
                                   cudaStream_t st);
cudaError_t launch_rebase_rowptr(const MatDesc* mats, int32_t nmats, int64_t total_rows, const int64_t* G,
                                 int64_t* out, cudaStream_t st);
cudaError_t launch_scatter_starts_batch(const MatDesc* mats, int32_t nmats, int64_t total_rows,
                                        const int32_t* flags, const int64_t* pos, int32_t* super_start,
                                        cudaStream_t st);
cudaError_t launch_scan_i32_i64_long(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t st);
size_t scan_tmp_bytes_long(int64_t n);
cudaError_t launch_compact_long(int64_t nrows, const uint32_t* pool, const int64_t* row_off, const int32_t* row_nL,
                                const int32_t* row_nU, const int64_t* L_off, const int64_t* U_off,
                                int32_t* L_colidx, int32_t* U_colidx, cudaStream_t st);

// exclusive scan of int32 counts into int64 offsets (out has n+1 entries)
size_t scan_tmp_bytes(int32_t n);
cudaError_t launch_scan_i32_i64(const int32_t* in, int64_t* out, int32_t n, void* tmp,
                                cudaStream_t st);
cudaError_t launch_compact(int32_t n, const uint32_t* pool, const int64_t* row_off,
                           const int32_t* row_nL, const int32_t* row_nU,
                           const int64_t* L_rowptr, const int64_t* U_rowptr,
                           int32_t* L_colidx, int32_t* U_colidx, cudaStream_t st);
cudaError_t launch_supernode_flags(int32_t n, int32_t chunk, const uint32_t* pool,
                                   const int64_t* row_off, const int32_t* row_nL,
                                   const int32_t* row_nU, int32_t* flags, DevCounters* ctr,
                                   cudaStream_t st);
cudaError_t launch_scatter_starts(int32_t n, const int32_t* flags, const int64_t* pos,
                                  int32_t* super_start, cudaStream_t st);
cudaError_t launch_fill_i32(int32_t* p, int64_t count, int32_t v, cudaStream_t st);
cudaError_t launch_init_counters(DevCounters* c, cudaStream_t st);
// Wide records for the class kernel: the (at most 8) off-diagonal columns of
// row v as int32 in ellw[2v], ellw[2v+1], empty slots holding v itself; rows
// with more entries (or a column out of range) have -1 in slot 0.
cudaError_t launch_build_ellw(int32_t n, const int32_t* rowptr, const int32_t* colidx, int4* ellw, DevCounters* ctr,
                              cudaStream_t st);
cudaError_t launch_build_ell(int32_t n, const int32_t* rowptr, const int32_t* colidx, int4* ell, DevCounters* ctr,
                             cudaStream_t st);
cudaError_t launch_build_ell_batch(const MatDesc* mats, int32_t nmats, int64_t total_rows, int4* ell,
                                   DevCounters* ctr, cudaStream_t st);
cudaError_t launch_iota_desc(int32_t* out, int32_t hi, int32_t count, cudaStream_t st);

// host helpers (api.cu)
// Served batches: one-off composition, pooled workspace, no graph.  pool_entries
// (per matrix, or null): the first row-pool size the caller charged for it.
int batch_transient(int32_t count, const int32_t* n, const int32_t* const* rp, const int32_t* const* ci,
                    const gsofa_options* opt, cudaStream_t st, gsofa_result* outs, const int64_t* pool_entries);
int device_sms();
// Bytes of the global-tier slots a single-matrix call of order n would hold.
int64_t global_tier_bytes(int32_t n, const gsofa_options* opts);
// Bytes of one global-tier slot for order n.
int64_t global_slot_bytes(int32_t n);
// Device bytes of one slot whose log lives in host memory (bitmaps only).
int64_t global_device_slot_bytes(int32_t n);
void detach_result_stream(gsofa_result* r);
int32_t smem_tier_max_order();
// Class-kernel slots an untuned batch of largest order n_max would use.
int32_t batch_class_slots(int32_t n_max);
// Bytes of the library's stream-ordered pool in use now (high 0) or at its
// high-water mark (high 1; reset_high 1 restarts the mark).
int64_t library_pool_bytes(int high, int reset_high);
// Bytes held by the single-matrix class-kernel slots (kept between calls).
int64_t library_slot_bytes();
int wait_stream(cudaStream_t st);  // bounded wait; GSOFA_OK / GSOFA_E_TIMEOUT / GSOFA_E_CUDA
int choose_smem_config(int sms, size_t limit, int32_t n, int32_t S, int label16, int threads_req, int* block,
                       int* occ, int32_t* cap);

}  // namespace gsofa
