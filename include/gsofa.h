/*
 * gsofa.h - C ABI of the GB300 symbolic LU library (gSoFa, arXiv 2007.00840).
 *
 * The library computes the static symbolic LU factorisation of a square
 * nonsymmetric sparsity pattern A (no pivoting, nonzero pivots):
 *
 *   - the L and U patterns of L+U (Theorem 1, Section 2.1: entry (i, j) is
 *     nonzero iff A(i, j) != 0, i == j, or G(A) has a path i -> j whose
 *     intermediate vertices are all numbered below min(i, j));
 *   - the number of fill-ins of every row;
 *   - the T3 supernode partition (Definition 1, Section 2.2), limited to
 *     aligned chunks of `chunk_size` rows (Section 5, Eq. 1).
 *
 * The fill pattern is found by the multi-source maxId traversal of Section 4
 * (Fig. 5): many source rows are traversed concurrently, every frontier vertex
 * of every source is expanded in parallel, and a vertex is revisited whenever
 * its maxId (the smallest largest-intermediate over the paths found so far)
 * drops.  Supernodes use the two-phase detection of Section 5 (Fig. 7).
 *
 * Conventions shared by every entry point
 *   - Input: CSR with int32 row pointers (n+1, rowptr[0] == 0, non-decreasing)
 *     and int32 column indices (rowptr[n] entries, 0 <= col < n, strictly
 *     increasing inside each row).  Inputs are borrowed and never modified.
 *     The diagonal may be absent; U(i,i) is emitted regardless.
 *   - Output: L holds the strictly lower part (unit diagonal implied, not
 *     stored); U holds the upper part including the diagonal.  Column indices
 *     are sorted ascending inside every row.  Row pointers are int64.
 *   - Errors: every function returns GSOFA_OK (0) or a negative GSOFA_E_*
 *     code; on error the result struct is left zeroed and nothing needs to be
 *     freed.  gsofa_strerror() names a code.
 *   - Threads: calls on different streams may run concurrently from different
 *     host threads; one result must not be used from two threads at once.
 */
#ifndef GSOFA_H
#define GSOFA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSOFA_OK             0
#define GSOFA_E_INVAL       -1  /* bad argument or malformed CSR (see gsofa_result.err_detail) */
#define GSOFA_E_NOMEM       -2  /* device or host allocation failed / budget too small */
#define GSOFA_E_CUDA        -3  /* a CUDA runtime call failed */
#define GSOFA_E_NOCONVERGE  -4  /* a traversal hit its iteration cap (never expected) */
#define GSOFA_E_TIMEOUT     -5  /* a bounded host-side wait ran out */
#define GSOFA_E_BUSY        -6  /* server admission queue is full */
#define GSOFA_E_NOTFOUND    -7  /* unknown ticket */
#define GSOFA_E_PENDING     -8  /* request not finished yet (gsofa_server_poll) */

/* Tuning knobs.  Zero in any field selects the default. */
typedef struct gsofa_options {
    int32_t chunk_size;          /* rows per supernode chunk = maximum supernode size (default 128, Section 5) */
    int32_t threads_per_source;  /* CTA size of the shared-memory traversal (default: the size with the most
                                    resident threads, 512 x 2 per SM for n = 32,768; 64..1024, multiple of 32) */
    int32_t smem_max_source;     /* sources below this use shared-memory labels (default 0: as many as fit;
                                    -1: none, every source uses the global-memory tier) */
    int32_t max_concurrent;      /* global-label tier: concurrent source slots, one warp each (default: 32 per SM
                                    within the memory budget) */
    int64_t mem_budget_bytes;    /* global-label tier: half of it bounds the slots' memory (default: half of
                                    the device memory free at first use, at most 96 GiB) */
    int32_t fill_first;          /* 1: skip lowering the maxId of a vertex already known to be a fill
                                    (the optional "line 9.5" of Section 4); same result */
    int32_t collect_stats;       /* 1: record per-phase CUDA-event times and work counters (expanded vertices,
                                    scanned entries: extra loads in the traversal), 2: the times only */
    int32_t validate;            /* 0 or 1: check the CSR on the device first (default 1); 2: skip */
    int32_t autotune;            /* 1 = time candidates once and keep the fastest: gsofa_batch per batch shape
                                    (kernel, block size, CTAs or warps per SM, frontier list capacity,
                                    work items per fetch, the fill-first check); single matrices per
                                    (n, nnz) (frontier order, and the fill-first check for breadth-first).
                                    0 = heuristic choices */
    int32_t work_chunk;          /* work items a CTA takes per fetch (default 1) */
    int32_t list_capacity;       /* frontier list entries kept in shared memory, the rest spilling to global
                                    memory: breadth-first kernel, per CTA (default 2,048, fewer if the
                                    occupancy needs it); class-ordered kernel on one matrix, per warp and
                                    level parity (default 512 with visited bitmaps in global memory,
                                    else 128; 32-1024) */
    int32_t max_ctas;            /* cap on traversal CTAs per launch, so concurrent launches share the GPU
                                    (default 0: one full wave) */
    int32_t frontier_order;      /* 0: automatic: class order for every source (sources below an explicit
                                    smem_max_source stay breadth-first in shared memory); with
                                    autotune = 1 both orders are timed once per (n, nnz) and the faster
                                    kept.  1: breadth-first levels (shared-memory tier wherever the
                                    maxId array fits on chip, class order above).  2: by increasing
                                    maxId class for every source (visited bitmaps, one warp per
                                    source).  Same result */
    int32_t label_bits;          /* shared-memory tier maxId width: 0 automatic (16 when n <= 65533), 16 or 32 */
    int32_t expand_mode;         /* shared-memory tier row access: 0 automatic, 1 CSR row slots per lane,
                                    2 CSR edge-balanced (a warp flattens its rows' entries), 3 16-byte
                                    records of 16-bit column offsets built from the CSR (rows that do
                                    not fit fall back to the CSR) */
    int32_t schedule;            /* shared-memory tier: 0 automatic, 1 breadth-first levels with one
                                    barrier each, 2 a worklist without level barriers (warps take
                                    queued vertices as they come; 16-bit labels and every vertex on
                                    chip only, else levels).  Same result */
    int32_t team_sources;        /* class-ordered kernel: how many of the largest sources a whole CTA of four
                                    warps expands together (the rest: one warp each).  0 or -1: none (the
                                    default: one warp per source was faster on every workload measured),
                                    > 0: that many.  Same result */
    int32_t warps_per_sm;        /* class-ordered kernel on one matrix: resident warps (sources in flight)
                                    per SM, 0 automatic (32; 40 selects a 48-register build).  Batches
                                    choose theirs with autotune */
    int32_t host_spill;          /* class-ordered kernel: keep each slot's log (level overflow and L row,
                                    4 bytes per vertex) in pinned host memory the GPU reads directly,
                                    and only the visited bitmaps (n/8 bytes per slot) in device memory:
                                    the external frontier management of Section 6.  0 automatic (when
                                    the slot budget cannot hold one whole slot in device memory), 1
                                    always, -1 never (GSOFA_E_NOMEM instead).  Same result */
    int32_t clean_heads;         /* class-ordered kernel: retire runs of pending classes whose heads reach
                                    nothing new (every neighbour already reached) together, up to 32 per
                                    warp-wide check, instead of one class at a time.  0 automatic (on
                                    where the visited bitmaps are in global memory, off where they are
                                    in shared memory), 1 on (after a check that retires nothing, the next
                                    1, 3, 7, 15 or 31 classes go one at a time), 2 a check before every
                                    class, -1 off.  Same result */
    int32_t reserved;
} gsofa_options;

/* Per-call statistics.  Times are filled when options.collect_stats is 1 or 2,
 * cycles, edges_scanned and the class-ordered kernel's vertices_expanded when
 * it is 1; kernel_launches, pool_retries, levels and the shared-memory tier's
 * vertices_expanded always. */
typedef struct gsofa_stats {
    float ms_validate, ms_traverse, ms_emit, ms_supernode, ms_total;
    float ms_traverse_smem;      /* breadth-first shared-memory kernel (sources below smem_max_source) */
    float ms_traverse_global;    /* class-ordered kernel (every other source; all of them by default) */
    int32_t traverse_launches;
    int32_t kernel_launches;     /* every kernel this call launched */
    int64_t vertices_expanded;   /* frontier expansions, revisits included */
    int64_t edges_scanned;       /* adjacency entries read by expansions */
    int64_t pool_retries;        /* times the row pool had to grow and the traversal rerun */
    int64_t levels;              /* frontier levels summed over sources (both kernels) */
    int64_t cycles_traverse;     /* shared-memory tier: SM cycles in frontier levels, summed over sources */
    int64_t cycles_emit;         /* shared-memory tier: SM cycles emitting rows, summed over sources */
} gsofa_stats;

/* Result.  Arrays are owned by the library and released by gsofa_free().
 * on_device == 1: arrays are device pointers (same device as the call);
 * on_device == 0: host pointers. */
typedef struct gsofa_result {
    int32_t n;
    int32_t n_super;             /* number of supernodes */
    int64_t nnz_L, nnz_U;        /* U counts the diagonal */
    int64_t *L_rowptr;           /* n+1 */
    int32_t *L_colidx;           /* nnz_L */
    int64_t *U_rowptr;           /* n+1 */
    int32_t *U_colidx;           /* nnz_U */
    int32_t *fill_count;         /* n: entries of row i of L+U not in A (diagonal counted as present) */
    int32_t *super_start;        /* n_super+1: first row of each supernode, then n */
    int32_t on_device;
    int32_t err_detail;          /* for GSOFA_E_INVAL: first offending row (or -1) */
    gsofa_stats stats;
    void *_priv;                 /* library bookkeeping */
} gsofa_result;

/* Fill *opt with the defaults. */
int gsofa_default_options(gsofa_options *opt);

/*
 * gsofa_symbolic - host CSR in, host result out (Sections 4 and 5).
 *   n        order of A (n >= 0)
 *   rowptr   host int32[n+1]; colidx host int32[rowptr[n]]
 *   opt      NULL for defaults
 *   out      zeroed by the call, then filled; release with gsofa_free().
 * Copies A to the current CUDA device, runs gsofa_symbolic_device on an
 * internal stream, copies the result back and waits.  Blocking.
 */
int gsofa_symbolic(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                   const gsofa_options *opt, gsofa_result *out);

/*
 * gsofa_symbolic_device - device CSR in, device result out.
 *   d_rowptr, d_colidx  device pointers on the current device (borrowed)
 *   stream              cudaStream_t (NULL = legacy default stream)
 * All kernels run on `stream`.  The call reads back the output sizes once
 * (a stream synchronisation) and returns after the result is complete.
 */
int gsofa_symbolic_device(int32_t n, const int32_t *d_rowptr, const int32_t *d_colidx,
                          const gsofa_options *opt, void *stream, gsofa_result *out);

/*
 * gsofa_batch - many independent matrices in one pass: the Section 4 traversal
 * and Section 5 supernode detection of every matrix, with the source rows of
 * all matrices scheduled together.  Matrix k is (n[k], d_rowptr[k],
 * d_colidx[k]) on the current device (borrowed).  Matrices whose maxId arrays
 * fit in shared memory run in ONE persistent traversal launch whose work items
 * are (matrix, source row) pairs, largest source row first across the batch;
 * the launch sequence up to the size read-back is captured once per batch
 * signature (matrix count, orders, input pointers, options) into a CUDA graph
 * and replayed on later calls with the same signature.  Larger matrices run
 * one after another through the single-matrix path.  outs[k] receives matrix
 * k's device result; batch members share one allocation that is released when
 * the last of them is passed to gsofa_free().  On error every out is zeroed.
 */
int gsofa_batch(int32_t count, const int32_t *n, const int32_t *const *d_rowptr,
                const int32_t *const *d_colidx, const gsofa_options *opt, void *stream,
                gsofa_result *outs);

/*
 * gsofa_row_counts_noalloc - per-row sizes of L and U and fill counts, without
 * allocating any device memory.  The paper has no counterpart: this entry point
 * is for callers that cannot allocate at the time they need the sizes (a
 * solver that reserved the device's free memory for itself and hands out
 * sub-buffers, a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device, a host that forbids allocation after start-up).
 *   n                  order of A, 0 <= n <= GSOFA_NOALLOC_MAX_N (else GSOFA_E_INVAL)
 *   d_rowptr, d_colidx device CSR of A (borrowed, validated on the device)
 *   d_nnzL, d_nnzU     device int32[n]: nnz(L(i,:)) and nnz(U(i,:)) (diagonal included)
 *   d_fill_count       device int32[n]: fill-ins of row i (as gsofa_result.fill_count)
 *   stream             cudaStream_t.  Every call copies its counters to the host
 *                      and waits until all work queued on `stream` has finished
 *                      before it returns (a bounded wait, GSOFA_E_TIMEOUT).
 * Scratch: a fixed array of GSOFA_NOALLOC_SCRATCH_BYTES in device memory, held
 * by every GPU that loads the library until the process exits.  The first call
 * on a device looks up that array's device address (once per device); make the
 * first call before any stream capture.  Near GSOFA_NOALLOC_MAX_N the frontier
 * overflow lists of fewer CTAs fit the array, so the launch uses fewer CTAs;
 * GSOFA_E_NOMEM if not even one fits.  All calls share the array, so calls
 * that overlap on the GPU (concurrent streams or host threads) race; serialise
 * them.  No cudaMalloc, cudaFree or other allocating routine is called.
 */
#define GSOFA_NOALLOC_MAX_N 65533
#define GSOFA_NOALLOC_SCRATCH_BYTES (16u << 20)
int gsofa_row_counts_noalloc(int32_t n, const int32_t *d_rowptr, const int32_t *d_colidx,
                             int32_t *d_nnzL, int32_t *d_nnzU, int32_t *d_fill_count, void *stream);

/*
 * Serving (an extension built on the Section 4/5 method): a request loop
 * that factors incoming sparsity patterns with continuous batching.
 * Requests are admitted in arrival order while the server's device memory fits
 * under mem_cap_bytes: each admitted request is charged its projected bytes
 * (CSR copy, per-row workspace, row pool and outputs), each running batch or
 * large request the class-kernel slots it uses while it runs (fewer slots when
 * the cap leaves less room), and each completed result its size until the
 * caller collects it (a batch's results share one block, released with the
 * last of them; uncollected results therefore hold admission back).
 * Admitted requests wait in two queues, batchable orders (visited bitmaps on
 * chip) and large ones; a free slot of `streams` takes whichever holds the
 * oldest request: all waiting batchable requests (up to max_batch) as one
 * multi-matrix batch, or one large request alone (one at a time: they share
 * the library's class slots), so a large request never holds up the small
 * ones.  Slots launch as soon as they are free, so their
 * work overlaps on the GPU (opts.max_ctas can split the GPU between slots
 * instead).  A request whose slots alone would exceed the cap runs alone with
 * as many slots as the cap leaves room for (space-budget mode: fewer sources in
 * flight, same result); one that does not fit even with one slot runs with
 * the slots' logs in host memory and only their visited bitmaps on the device
 * (opts.host_spill >= 0), and is refused with GSOFA_E_NOMEM only when not even
 * that fits.
 */
typedef struct gsofa_server gsofa_server;

typedef struct gsofa_server_config {
    int64_t mem_cap_bytes;       /* admission cap on projected device memory (default 150 GiB) */
    int32_t max_inflight;        /* admitted, unfinished requests at most (default 8192) */
    int32_t streams;             /* concurrent batch slots (default 2, at most 16) */
    int32_t max_batch;           /* requests per batch launch (default 512) */
    int32_t queue_capacity;      /* pending requests before submit returns GSOFA_E_BUSY (default 2^20) */
    gsofa_options opts;          /* options of every batch */
} gsofa_server_config;

typedef struct gsofa_server_stats {
    int64_t completed, failed, batches, pending;
    int32_t inflight;
    int32_t kernel_launches;     /* library kernels launched for completed batches (saturates) */
    int64_t total_nnz;           /* nnz(L+U) of completed requests */
    int64_t total_rows;          /* rows of completed requests */
    int64_t mem_in_use, peak_mem_in_use;   /* projected bytes of admitted requests and running batches */
    float p50_ms, p99_ms, max_ms;          /* latency, submission to completed result */
    float pad2;
    double span_s;               /* first submission to last completion */
    int64_t peak_device_bytes;   /* device memory the server's work held at its peak, beyond what the
                                    library held when the server started: stream-ordered pool high-water
                                    mark (uncollected results included), class-kernel slots it made the
                                    library keep, and copies of host inputs */
} gsofa_server_stats;

int gsofa_server_default_config(gsofa_server_config *cfg);
/* Start the dispatcher threads on the current device. */
int gsofa_server_create(const gsofa_server_config *cfg, gsofa_server **server);
/* Queue one pattern.  on_device = 1: rowptr/colidx are device pointers; 0: host
 * pointers (copied at dispatch).  Either way the buffers must stay valid and
 * unchanged until the request completes.  GSOFA_E_BUSY when the queue is full,
 * GSOFA_E_NOMEM when the request alone exceeds the cap. */
int gsofa_server_submit(gsofa_server *server, int32_t n, const int32_t *rowptr, const int32_t *colidx,
                        int32_t on_device, uint64_t *ticket);
/* Non-blocking: GSOFA_OK moves the device result to *out (release with gsofa_free;
 * out may be NULL to discard it), GSOFA_E_PENDING if not finished, GSOFA_E_NOTFOUND. */
int gsofa_server_poll(gsofa_server *server, uint64_t ticket, gsofa_result *out, double *latency_ms);
/* Blocking variant of poll with a timeout in seconds (GSOFA_E_TIMEOUT). */
int gsofa_server_wait(gsofa_server *server, uint64_t ticket, double timeout_s, gsofa_result *out,
                      double *latency_ms);
int gsofa_server_get_stats(gsofa_server *server, gsofa_server_stats *stats);
/* Finish admitted requests, drop pending ones, free unclaimed results. */
void gsofa_server_destroy(gsofa_server *server);

/* Release every array of *res (device or host) and zero it.  NULL-safe.
 * Device arrays are freed stream-ordered on the stream of the call that made
 * them; the caller must not use them afterwards. */
void gsofa_free(gsofa_result *res);

/* Human-readable name of an error code. */
const char *gsofa_strerror(int code);

/* Library version as an integer (major*10000 + minor*100 + patch). */
int gsofa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSOFA_H */
