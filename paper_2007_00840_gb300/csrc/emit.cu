// CSR validation, prefix sums, row compaction and supernode detection.
#include <climits>

#include "internal.cuh"

namespace gsofa {

namespace {
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__device__ __forceinline__ void flag_row(DevCounters* c, int bit, int row) {
  atomicOr(&c->err, bit);
  atomicMin(&c->err_row, row);
}
}  // namespace

// ---------------------------------------------------------------- validate
// One warp per row: rowptr[0] == 0, rowptr non-decreasing, 0 <= col < n and
// columns strictly increasing inside every row (Section 2.4 uses CSR input).
__global__ void validate_kernel(int32_t n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colidx, DevCounters* ctr) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  if (gw == 0 && lane == 0 && rowptr[0] != 0) flag_row(ctr, ERR_ROWPTR, 0);
  for (int i = gw; i < n; i += nw) {
    const int rb = rowptr[i], re = rowptr[i + 1];
    if (re < rb || rb < 0) {
      if (lane == 0) flag_row(ctr, ERR_ROWPTR, i);
      continue;
    }
    bool bad_range = false, bad_order = false;
    for (int e = rb + lane; e < re; e += 32) {
      const int c = colidx[e];
      if ((unsigned)c >= (unsigned)n) bad_range = true;
      if (e > rb && colidx[e - 1] >= c) bad_order = true;
    }
    if (__any_sync(FULL, bad_range) && lane == 0) flag_row(ctr, ERR_COL_RANGE, i);
    if (__any_sync(FULL, bad_order) && lane == 0) flag_row(ctr, ERR_UNSORTED, i);
  }
}

__global__ void init_counters_kernel(DevCounters* c) {
  if (threadIdx.x == 0) {
    c->pool_cursor = 0ull;
    c->total_L = 0ull;
    c->total_U = 0ull;
    c->expansions = 0ull;
    c->edges = 0ull;
    c->err = 0;
    c->err_row = INT_MAX;
    c->n_super = 0;
    c->work_smem = 0;
    c->work_global = 0;
    c->work_team = 0;
    c->levels = 0ull;
    c->cyc_trav = 0ull;
    c->cyc_emit = 0ull;
  }
}

cudaError_t launch_validate(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                            DevCounters* ctr, cudaStream_t st) {
  const int block = 256;
  long long warps = n > 0 ? n : 1;
  long long grid = (warps * 32 + block - 1) / block;
  if (grid > 4096) grid = 4096;
  validate_kernel<<<(int)grid, block, 0, st>>>(n, rowptr, colidx, ctr);
  return cudaGetLastError();
}

cudaError_t launch_init_counters(DevCounters* c, cudaStream_t st) {
  init_counters_kernel<<<1, 32, 0, st>>>(c);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- scan
// out[0] = 0, out[i+1] = in[0] + ... + in[i]  (int32 in, int64 out)
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sh, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long y = lane < nw ? sh[lane] : 0;
    long long z = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(FULL, z, o);
      if (lane >= o) z += t;
    }
    if (lane < nw) sh[lane] = z - y;
    if (lane == 31) sh[32] = z;
  }
  __syncthreads();
  const long long r = sh[warp] + x - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

__global__ void scan_reduce_kernel(const int32_t* __restrict__ in, int32_t n, long long* part) {
  __shared__ long long sh[33];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  long long s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; k++) {
    const long long i = base + (long long)threadIdx.x * SCAN_PER_THREAD + k;
    if (i < n) s += in[i];
  }
  long long tot;
  block_excl_scan(s, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void scan_parts_kernel(long long* part, int32_t nparts) {
  __shared__ long long sh[33];
  long long carry = 0;
  for (int b0 = 0; b0 < nparts; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const long long v = b < nparts ? part[b] : 0;
    long long tot;
    const long long ex = block_excl_scan(v, sh, &tot);
    if (b < nparts) part[b] = carry + ex;
    carry += tot;
  }
}

__global__ void scan_down_kernel(const int32_t* __restrict__ in, int32_t n, const long long* part,
                                 int64_t* out) {
  __shared__ long long sh[33];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int32_t v[SCAN_PER_THREAD];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; k++) {
    const long long i = base + (long long)threadIdx.x * SCAN_PER_THREAD + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  long long tot;
  long long ex = block_excl_scan(s, sh, &tot) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; k++) {
    const long long i = base + (long long)threadIdx.x * SCAN_PER_THREAD + k;
    if (i < n) out[i] = ex;
    ex += v[k];
    if (i == (long long)n - 1) out[n] = ex;
  }
}

size_t scan_tmp_bytes(int32_t n) {
  const long long parts = ((long long)n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(parts > 0 ? parts : 1) * sizeof(long long);
}

cudaError_t launch_scan_i32_i64(const int32_t* in, int64_t* out, int32_t n, void* tmp, cudaStream_t st) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
  }
  const int parts = (int)(((long long)n + SCAN_TILE - 1) / SCAN_TILE);
  long long* part = (long long*)tmp;
  scan_reduce_kernel<<<parts, SCAN_THREADS, 0, st>>>(in, n, part);
  scan_parts_kernel<<<1, SCAN_THREADS, 0, st>>>(part, parts);
  scan_down_kernel<<<parts, SCAN_THREADS, 0, st>>>(in, n, part, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- compact
// Move every row from the pool ([L cols | s | U cols] at row_off) to its CSR slot.
__global__ void compact_kernel(int32_t n, const uint32_t* __restrict__ pool,
                               const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_nL,
                               const int32_t* __restrict__ row_nU, const int64_t* __restrict__ L_rowptr,
                               const int64_t* __restrict__ U_rowptr, int32_t* __restrict__ L_colidx,
                               int32_t* __restrict__ U_colidx) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < n; i += nw) {
    const int64_t off = row_off[i];
    const int nL = row_nL[i], nU = row_nU[i];
    const uint32_t* src = pool + off;
    int32_t* dL = L_colidx + L_rowptr[i];
    int32_t* dU = U_colidx + U_rowptr[i];
    for (int k = lane; k < nL; k += 32) dL[k] = (int32_t)__ldcs(src + k);
    for (int k = lane; k < nU; k += 32) dU[k] = (int32_t)__ldcs(src + nL + k);
  }
}

cudaError_t launch_compact(int32_t n, const uint32_t* pool, const int64_t* row_off,
                           const int32_t* row_nL, const int32_t* row_nU, const int64_t* L_rowptr,
                           const int64_t* U_rowptr, int32_t* L_colidx, int32_t* U_colidx,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  long long grid = ((long long)n * 32 + block - 1) / block;
  const long long cap = 16LL * device_sms();  // 16 resident CTAs of 256 threads per SM
  if (cap > 0 && grid > cap) grid = cap;
  compact_kernel<<<(int)grid, block, 0, st>>>(n, pool, row_off, row_nL, row_nU, L_rowptr, U_rowptr,
                                              L_colidx, U_colidx);
  return cudaGetLastError();
}

// -------------------------------------------------------------- supernodes
// Two-phase T3 detection (Section 5, Fig. 7), one CTA per aligned chunk.
// Phase I : thread t tests nnz(U(s,:)) == nnz(U(s-1,:)) - 1 for row s = chunk
//           start + t into a shared bitmap; rows that fail lead a run.
// Phase II: every leading row walks its run: row s stays in the supernode
//           that starts at r while its bit is set and L(s, r) != 0 (binary
//           search in the sorted L row); otherwise s starts a new supernode.
// flags[s] = 1 iff s is the first row of a supernode.
__global__ void supernode_kernel(int32_t n, int32_t chunk, const uint32_t* __restrict__ pool,
                                 const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_nL,
                                 const int32_t* __restrict__ row_nU, int32_t* __restrict__ flags,
                                 DevCounters* ctr) {
  extern __shared__ uint32_t bits[];  // ceil(chunk/32) words
  __shared__ int s_count;
  // rejected input: the traversal wrote no rows, so there is nothing to read
  if (input_error(ctr)) return;
  const int c0 = blockIdx.x * chunk;
  const int cend = min(n, c0 + chunk);
  const int nwords = (chunk + 31) >> 5;
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) bits[i] = 0u;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  for (int t = threadIdx.x; c0 + t < cend; t += blockDim.x) {
    const int s = c0 + t;
    if (t > 0 && row_nU[s] == row_nU[s - 1] - 1) atomicOr(&bits[t >> 5], 1u << (t & 31));
  }
  __syncthreads();
  int local = 0;
  for (int t = threadIdx.x; c0 + t < cend; t += blockDim.x) {
    if (bits[t >> 5] & (1u << (t & 31))) continue;  // not a leading row
    int r = c0 + t;
    flags[r] = 1;
    local++;
    for (int u = t + 1; c0 + u < cend && (bits[u >> 5] & (1u << (u & 31))); u++) {
      const int s = c0 + u;
      const int64_t off = row_off[s];
      bool has = false;
      if (off >= 0) {
        int lo = 0, hi = row_nL[s];
        const uint32_t key = (uint32_t)r;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const uint32_t x = pool[off + mid];
          if (x < key) lo = mid + 1; else hi = mid;
        }
        has = lo < row_nL[s] && pool[off + lo] == key;
      }
      if (has) {
        flags[s] = 0;
      } else {
        flags[s] = 1;
        r = s;
        local++;
      }
    }
  }
  if (local) atomicAdd(&s_count, local);
  __syncthreads();
  if (threadIdx.x == 0 && s_count) atomicAdd(&ctr->n_super, s_count);
}

cudaError_t launch_supernode_flags(int32_t n, int32_t chunk, const uint32_t* pool, const int64_t* row_off,
                                   const int32_t* row_nL, const int32_t* row_nU, int32_t* flags,
                                   DevCounters* ctr, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nchunks = (int)(((long long)n + chunk - 1) / chunk);
  const int block = chunk >= 1024 ? 1024 : ((chunk + 31) / 32) * 32;
  const size_t sm = (size_t)((chunk + 31) / 32) * 4;
  supernode_kernel<<<nchunks, block, sm, st>>>(n, chunk, pool, row_off, row_nL, row_nU, flags, ctr);
  return cudaGetLastError();
}

__global__ void scatter_starts_kernel(int32_t n, const int32_t* __restrict__ flags,
                                      const int64_t* __restrict__ pos, int32_t* __restrict__ super_start) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (flags[i]) super_start[pos[i]] = (int32_t)i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) super_start[pos[n]] = n;
}

cudaError_t launch_scatter_starts(int32_t n, const int32_t* flags, const int64_t* pos,
                                  int32_t* super_start, cudaStream_t st) {
  const int block = 256;
  long long grid = ((long long)(n > 0 ? n : 1) + block - 1) / block;
  if (grid > 4096) grid = 4096;
  scatter_starts_kernel<<<(int)grid, block, 0, st>>>(n, flags, pos, super_start);
  return cudaGetLastError();
}

__global__ void fill_i32_kernel(int32_t* p, int64_t count, int32_t v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t launch_fill_i32(int32_t* p, int64_t count, int32_t v, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int block = 256;
  long long grid = (count + block - 1) / block;
  if (grid > 4096) grid = 4096;
  fill_i32_kernel<<<(int)grid, block, 0, st>>>(p, count, v);
  return cudaGetLastError();
}

__global__ void iota_desc_kernel(int32_t* out, int32_t hi, int32_t count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = hi - 1 - (int32_t)i;
}

cudaError_t launch_iota_desc(int32_t* out, int32_t hi, int32_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int block = 256;
  long long grid = ((long long)count + block - 1) / block;
  if (grid > 4096) grid = 4096;
  iota_desc_kernel<<<(int)grid, block, 0, st>>>(out, hi, count);
  return cudaGetLastError();
}

}  // namespace gsofa

// ------------------------------------------------------------ batch helpers
namespace gsofa {
namespace {
// matrix of a global row: the last descriptor whose row_base <= r
__device__ __forceinline__ int mat_of_row(const MatDesc* mats, int nmats, long long r) {
  int lo = 0, hi = nmats - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mats[mid].row_base <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int mat_of_chunk(const MatDesc* mats, int nmats, long long c) {
  int lo = 0, hi = nmats - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mats[mid].chunk_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}
}  // namespace

// validation of every matrix of a batch, one warp per (global) row
__global__ void validate_batch_kernel(const MatDesc* __restrict__ mats, int32_t nmats, long long total_rows,
                                      DevCounters* ctr) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (gw < nmats && lane == 0 && mats[gw].rowptr[0] != 0) flag_row(ctr, ERR_ROWPTR, (int)mats[gw].row_base);
  for (long long r = gw; r < total_rows; r += nw) {
    const int m = mat_of_row(mats, nmats, r);
    const MatDesc d = mats[m];
    const int i = (int)(r - d.row_base);
    const int rb = d.rowptr[i], re = d.rowptr[i + 1];
    if (re < rb || rb < 0) {
      if (lane == 0) flag_row(ctr, ERR_ROWPTR, (int)r);
      continue;
    }
    bool bad_range = false, bad_order = false;
    for (int e = rb + lane; e < re; e += 32) {
      const int c = d.colidx[e];
      if ((unsigned)c >= (unsigned)d.n) bad_range = true;
      if (e > rb && d.colidx[e - 1] >= c) bad_order = true;
    }
    if (__any_sync(FULL, bad_range) && lane == 0) flag_row(ctr, ERR_COL_RANGE, (int)r);
    if (__any_sync(FULL, bad_order) && lane == 0) flag_row(ctr, ERR_UNSORTED, (int)r);
  }
}

cudaError_t launch_validate_batch(const MatDesc* mats, int32_t nmats, int64_t total_rows, DevCounters* ctr,
                                  cudaStream_t st) {
  const int block = 256;
  long long w = total_rows > nmats ? total_rows : nmats;
  long long grid = (w * 32 + block - 1) / block;
  if (grid > 8192) grid = 8192;
  if (grid < 1) grid = 1;
  validate_batch_kernel<<<(int)grid, block, 0, st>>>(mats, nmats, total_rows, ctr);
  return cudaGetLastError();
}

// two-phase T3 detection (Section 5, Fig. 7) over the chunks of every matrix
__global__ void supernode_batch_kernel(const MatDesc* __restrict__ mats, int32_t nmats, int32_t chunk,
                                       const uint32_t* __restrict__ pool, const int64_t* __restrict__ row_off,
                                       const int32_t* __restrict__ row_nL, const int32_t* __restrict__ row_nU,
                                       int32_t* __restrict__ flags, int32_t* __restrict__ mat_nsuper,
                                       DevCounters* ctr) {
  extern __shared__ uint32_t bits[];
  __shared__ int s_count;
  if (input_error(ctr)) return;
  const int m = mat_of_chunk(mats, nmats, blockIdx.x);
  const MatDesc d = mats[m];
  const long long rb = d.row_base;
  const int c0 = (int)((long long)blockIdx.x - d.chunk_base) * chunk;
  const int cend = min(d.n, c0 + chunk);
  const int nwords = (chunk + 31) >> 5;
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) bits[i] = 0u;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  for (int t = threadIdx.x; c0 + t < cend; t += blockDim.x) {
    const long long g = rb + c0 + t;
    if (t > 0 && row_nU[g] == row_nU[g - 1] - 1) atomicOr(&bits[t >> 5], 1u << (t & 31));
  }
  __syncthreads();
  int local = 0;
  for (int t = threadIdx.x; c0 + t < cend; t += blockDim.x) {
    if (bits[t >> 5] & (1u << (t & 31))) continue;
    int r = c0 + t;
    flags[rb + r] = 1;
    local++;
    for (int u = t + 1; c0 + u < cend && (bits[u >> 5] & (1u << (u & 31))); u++) {
      const long long g = rb + c0 + u;
      const int64_t off = row_off[g];
      bool has = false;
      if (off >= 0) {
        int lo = 0, hi = row_nL[g];
        const uint32_t key = (uint32_t)r;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (pool[off + mid] < key) lo = mid + 1; else hi = mid;
        }
        has = lo < row_nL[g] && pool[off + lo] == key;
      }
      if (has) {
        flags[g] = 0;
      } else {
        flags[g] = 1;
        r = c0 + u;
        local++;
      }
    }
  }
  if (local) atomicAdd(&s_count, local);
  __syncthreads();
  if (threadIdx.x == 0 && s_count) {
    atomicAdd(&mat_nsuper[m], s_count);
    atomicAdd(&ctr->n_super, s_count);
  }
}

cudaError_t launch_supernode_batch(const MatDesc* mats, int32_t nmats, int64_t total_chunks, int32_t chunk,
                                   const uint32_t* pool, const int64_t* row_off, const int32_t* row_nL,
                                   const int32_t* row_nU, int32_t* flags, int32_t* mat_nsuper, DevCounters* ctr,
                                   cudaStream_t st) {
  if (total_chunks <= 0) return cudaSuccess;
  const int block = chunk >= 1024 ? 1024 : ((chunk + 31) / 32) * 32;
  const size_t sm = (size_t)((chunk + 31) / 32) * 4;
  supernode_batch_kernel<<<(unsigned)total_chunks, block, sm, st>>>(mats, nmats, chunk, pool, row_off, row_nL,
                                                                   row_nU, flags, mat_nsuper, ctr);
  return cudaGetLastError();
}

// per-matrix row pointers from the global exclusive scan G (length total+1):
// matrix m's rowptr occupies out[row_base + m .. row_base + m + n] and starts at 0
__global__ void rebase_rowptr_kernel(const MatDesc* __restrict__ mats, int32_t nmats, long long total_rows,
                                     const int64_t* __restrict__ G, int64_t* __restrict__ out) {
  const long long total = total_rows + nmats;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    // x = row_base[m] + m + i with 0 <= i <= n_m
    int lo = 0, hi = nmats - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (mats[mid].row_base + mid <= x) lo = mid; else hi = mid - 1;
    }
    const long long rb = mats[lo].row_base;
    const long long i = x - rb - lo;
    out[x] = G[rb + i] - G[rb];
  }
}

cudaError_t launch_rebase_rowptr(const MatDesc* mats, int32_t nmats, int64_t total_rows, const int64_t* G,
                                 int64_t* out, cudaStream_t st) {
  const int block = 256;
  long long grid = (total_rows + nmats + block - 1) / block;
  if (grid > 8192) grid = 8192;
  if (grid < 1) grid = 1;
  rebase_rowptr_kernel<<<(int)grid, block, 0, st>>>(mats, nmats, total_rows, G, out);
  return cudaGetLastError();
}

// super_start of matrix m lives at P[row_base_m] + m; its last entry is n_m
__global__ void scatter_starts_batch_kernel(const MatDesc* __restrict__ mats, int32_t nmats, long long total_rows,
                                            const int32_t* __restrict__ flags, const int64_t* __restrict__ P,
                                            int32_t* __restrict__ super_start) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < total_rows;
       r += (long long)gridDim.x * blockDim.x) {
    if (!flags[r]) continue;
    const int m = mat_of_row(mats, nmats, r);
    super_start[P[r] + m] = (int32_t)(r - mats[m].row_base);
  }
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < nmats;
       m += (long long)gridDim.x * blockDim.x) {
    const long long end = mats[m].row_base + mats[m].n;
    super_start[P[end] + m] = mats[m].n;
  }
}

cudaError_t launch_scatter_starts_batch(const MatDesc* mats, int32_t nmats, int64_t total_rows,
                                        const int32_t* flags, const int64_t* pos, int32_t* super_start,
                                        cudaStream_t st) {
  const int block = 256;
  long long w = total_rows > nmats ? total_rows : nmats;
  long long grid = (w + block - 1) / block;
  if (grid > 8192) grid = 8192;
  if (grid < 1) grid = 1;
  scatter_starts_batch_kernel<<<(int)grid, block, 0, st>>>(mats, nmats, total_rows, flags, pos, super_start);
  return cudaGetLastError();
}

size_t scan_tmp_bytes_long(int64_t n) {
  const long long parts = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(parts > 0 ? parts : 1) * sizeof(long long);
}

cudaError_t launch_scan_i32_i64_long(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t st) {
  if (n > INT32_MAX - SCAN_TILE) return cudaErrorInvalidValue;
  return launch_scan_i32_i64(in, out, (int32_t)n, tmp, st);
}

cudaError_t launch_compact_long(int64_t nrows, const uint32_t* pool, const int64_t* row_off, const int32_t* row_nL,
                                const int32_t* row_nU, const int64_t* L_off, const int64_t* U_off,
                                int32_t* L_colidx, int32_t* U_colidx, cudaStream_t st) {
  if (nrows > INT32_MAX) return cudaErrorInvalidValue;
  return launch_compact((int32_t)nrows, pool, row_off, row_nL, row_nU, L_off, U_off, L_colidx, U_colidx, st);
}

}  // namespace gsofa

// ------------------------------------------------------------- ELL copy
// Row v of A without its diagonal as up to 8 signed 16-bit offsets w - v in one
// 16-byte record, padded with 0 (an offset of 0 names v itself, which the
// traversal skips).  Rows with more entries or offsets beyond +-32767 get the
// marker -32768 in slot 0 and are read from the CSR instead.
namespace gsofa {
// ELL record of row v: up to 8 off-diagonal neighbours as 16-bit offsets w - v,
// zero-padded; rows that do not fit (more than 8 neighbours, an offset beyond
// +-32767, or a column out of range, possible only when validation is skipped)
// get the sentinel -32768 in slot 0 and are read from the CSR, which checks them.
__device__ int4 ell_record(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int32_t n,
                           long long v) {
  const int rb = rowptr[v], re = rowptr[v + 1];
  short off[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int k = 0;
  bool fits = true;
  for (int e = rb; e < re; e++) {
    const int w = colidx[e];
    const long long d = (long long)w - v;
    if (d == 0) continue;
    if (k == 8 || d > 32767 || d < -32767 || w < 0 || w >= n) { fits = false; break; }
    off[k++] = (short)d;
  }
  if (!fits) {
    off[0] = (short)-32768;
    for (int q = 1; q < 8; q++) off[q] = 0;
  }
  int4 r;
  r.x = (int)(((unsigned)(unsigned short)off[1] << 16) | (unsigned short)off[0]);
  r.y = (int)(((unsigned)(unsigned short)off[3] << 16) | (unsigned short)off[2]);
  r.z = (int)(((unsigned)(unsigned short)off[5] << 16) | (unsigned short)off[4]);
  r.w = (int)(((unsigned)(unsigned short)off[7] << 16) | (unsigned short)off[6]);
  return r;
}

__global__ void build_ell_kernel(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                 int4* __restrict__ ell, DevCounters* ctr) {
  if (input_error(ctr)) return;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    ell[v] = ell_record(rowptr, colidx, n, v);
}

// Wide record of row v: up to 8 off-diagonal columns as int32 (unused slots v).
__device__ void ellw_record(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int32_t n,
                            int32_t v, int4* __restrict__ out) {
  const int rb = rowptr[v], re = rowptr[v + 1];
  int c[8] = {v, v, v, v, v, v, v, v};
  int k = 0;
  bool fits = true;
  for (int e = rb; e < re; e++) {
    const int w = colidx[e];
    if (w == v) continue;
    if (k == 8 || w < 0 || w >= n) { fits = false; break; }
    c[k++] = w;
  }
  if (!fits) {
    c[0] = -1;
    for (int q = 1; q < 8; q++) c[q] = v;
  }
  out[0] = make_int4(c[0], c[1], c[2], c[3]);
  out[1] = make_int4(c[4], c[5], c[6], c[7]);
}

__global__ void build_ellw_kernel(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                  int4* __restrict__ ellw, DevCounters* ctr) {
  if (input_error(ctr)) return;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    ellw_record(rowptr, colidx, n, (int32_t)v, ellw + 2 * v);
}

// Records of every row of a batch, indexed by the row's global index (row_base + v).
__global__ void build_ell_batch_kernel(const MatDesc* __restrict__ mats, int32_t nmats, long long total_rows,
                                       int4* __restrict__ ell, DevCounters* ctr) {
  if (input_error(ctr)) return;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < total_rows;
       r += (long long)gridDim.x * blockDim.x) {
    const MatDesc d = mats[mat_of_row(mats, nmats, r)];
    ell[r] = ell_record(d.rowptr, d.colidx, d.n, r - d.row_base);
  }
}

cudaError_t launch_build_ell_batch(const MatDesc* mats, int32_t nmats, int64_t total_rows, int4* ell,
                                   DevCounters* ctr, cudaStream_t st) {
  if (total_rows <= 0) return cudaSuccess;
  const int block = 256;
  long long grid = (total_rows + block - 1) / block;
  if (grid > 8192) grid = 8192;
  build_ell_batch_kernel<<<(int)grid, block, 0, st>>>(mats, nmats, total_rows, ell, ctr);
  return cudaGetLastError();
}

cudaError_t launch_build_ell(int32_t n, const int32_t* rowptr, const int32_t* colidx, int4* ell, DevCounters* ctr,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  long long grid = ((long long)n + block - 1) / block;
  if (grid > 8192) grid = 8192;
  build_ell_kernel<<<(int)grid, block, 0, st>>>(n, rowptr, colidx, ell, ctr);
  return cudaGetLastError();
}
cudaError_t launch_build_ellw(int32_t n, const int32_t* rowptr, const int32_t* colidx, int4* ellw, DevCounters* ctr,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  long long grid = ((long long)n + block - 1) / block;
  if (grid > 8192) grid = 8192;
  build_ellw_kernel<<<(int)grid, block, 0, st>>>(n, rowptr, colidx, ellw, ctr);
  return cudaGetLastError();
}
}  // namespace gsofa
