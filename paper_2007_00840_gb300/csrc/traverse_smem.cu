// Multi-source maxId traversal, shared-memory tier (Section 4, Fig. 5).
//
// One CTA owns one source row s at a time and loops over sources from a global
// work counter (persistent CTAs).  Per source it keeps, in shared memory:
//   lab[0..S)   maxId of every vertex below the source (bubble removal,
//               Section 6: vertices above s never need one), stored with the
//               value-range windows of Section 4 ("Optimizing the initialization
//               of maxId"): source number k of this CTA uses the window
//               [base_k, base_k + n + 1] with base_k decreasing, so anything
//               above the window reads as "not reached" and lab[] is never
//               cleared between sources;
//   fA/fB       the current / next frontier as bitmaps over [0, s);
//   ub          the U part of the row as a bitmap over [0, n).
// maxId of a vertex is the smallest "largest intermediate vertex" over the
// paths found so far; a direct neighbour of s has no intermediate (-1).
//
// Level loop: every frontier vertex f proposes nm = max(maxId(f), f) to each
// neighbour w (atomicMin).  If the proposal lowers maxId(w) and w was not
// already a fill (old > w), w's own proposal changed, so w joins the next
// frontier; w is a fill of L(s,:) iff its final maxId < w (Theorem 1).
// Neighbours above s are U entries.  The frontier of a level is expanded by all
// warps in parallel; a warp turns 32 bitmap words into a compact list of
// vertices with ballot/shuffle and expands them one vertex per lane, with
// rows longer than 32 entries expanded by the whole warp.
//
// Emission writes the sorted row [L cols | s | U cols] to the row pool at an
// offset taken with one atomicAdd, plus the row's counts and fill count.
#include "internal.cuh"

namespace gsofa {

namespace {

constexpr int BIG_DEG = 32;

__device__ __forceinline__ int nth_set_bit(uint32_t x, int k) {
  // position of the k-th (0-based) set bit of x, by halving
  int pos = 0;
  int c = __popc(x & 0xFFFFu);
  if (k >= c) { k -= c; x >>= 16; pos += 16; }
  c = __popc(x & 0xFFu);
  if (k >= c) { k -= c; x >>= 8; pos += 8; }
  c = __popc(x & 0xFu);
  if (k >= c) { k -= c; x >>= 4; pos += 4; }
  c = __popc(x & 0x3u);
  if (k >= c) { k -= c; x >>= 2; pos += 2; }
  c = (int)(x & 1u);
  if (k >= c) { pos += 1; }
  return pos;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

struct SmemState {
  uint32_t* lab;
  uint32_t* ub;
  uint32_t base;
  int32_t s;
  int32_t n;
  int32_t fill_first;
};

// Relax edge (f -> w) with encoded proposal nmE.  Returns 1 if w was enqueued.
__device__ __forceinline__ int relax_smem(const SmemState& st, uint32_t* nxt, int w, uint32_t nmE,
                                          int* bad) {
  if ((unsigned)w >= (unsigned)st.n) { *bad = 1; return 0; }
  if (w < st.s) {
    const uint32_t wE = st.base + 1u + (uint32_t)w;   // encoded value of label == w
    if (st.fill_first && st.lab[w] < wE) return 0;   // already a fill: proposal stays w
    const uint32_t old = atomicMin(&st.lab[w], nmE);
    if (nmE < old && old > wE) {
      const uint32_t bit = 1u << (w & 31);
      if (!(nxt[w >> 5] & bit)) atomicOr(&nxt[w >> 5], bit);
      return 1;
    }
  } else if (w > st.s) {
    const uint32_t bit = 1u << (w & 31);
    if (!(st.ub[w >> 5] & bit)) atomicOr(&st.ub[w >> 5], bit);
  }
  return 0;
}

}  // namespace

size_t trav_smem_bytes(int32_t n, int32_t S) {
  const size_t SW = ((size_t)S + 31) / 32, NW = ((size_t)n + 31) / 32;
  return 4 * ((size_t)S + 2 * SW + NW);
}

int32_t trav_smem_max_S(int32_t n, size_t smem_limit) {
  const size_t NW = ((size_t)n + 31) / 32;
  if (4 * NW + 64 >= smem_limit) return 0;
  size_t S = (smem_limit - 4 * NW - 16) * 32 / (4 * 32 + 8);  // 4 bytes label + 2 frontier bits
  S &= ~(size_t)31;
  while (S > 0 && trav_smem_bytes(n, (int32_t)S) > smem_limit) S -= 32;
  if (S > (size_t)n) S = (size_t)n;
  return (int32_t)S;
}

__global__ void __launch_bounds__(1024, 1) trav_smem_kernel(TravArgs a) {
  extern __shared__ uint32_t sm[];
  const int n = a.n, S = a.S;
  const int SW = (S + 31) >> 5, NW = (n + 31) >> 5;
  uint32_t* lab = sm;
  uint32_t* fA = lab + S;
  uint32_t* fB = fA + SW;
  uint32_t* ub = fB + SW;

  __shared__ int s_src, s_diag;
  __shared__ int s_wcL[32], s_wcU[32];
  __shared__ long long s_off;
  __shared__ int s_nL;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarps = nthr >> 5;

  for (int i = tid; i < S; i += nthr) lab[i] = 0xFFFFFFFFu;
  for (int i = tid; i < SW; i += nthr) { fA[i] = 0u; fB[i] = 0u; }
  for (int i = tid; i < NW; i += nthr) ub[i] = 0u;

  const uint32_t span = (uint32_t)n + 2u;
  uint32_t base = 0xFFFFFFFFu - span;
  bool first = true;
  unsigned long long n_exp = 0, n_edge = 0;
  int bad = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const int k = atomicAdd(&a.ctr->work_smem, 1);
      s_src = (k < a.nsrc && !input_error(a.ctr)) ? a.order[k] : -1;
      s_diag = 0;
    }
    __syncthreads();
    const int s = s_src;
    if (s < 0) break;

    // next maxId window (Section 4); refill lab[] only when the range is used up
    if (!first) {
      if (base >= span) {
        base -= span;
      } else {
        for (int i = tid; i < S; i += nthr) lab[i] = 0xFFFFFFFFu;
        base = 0xFFFFFFFFu - span;
        __syncthreads();
      }
    }
    first = false;

    SmemState st{lab, ub, base, s, n, a.fill_first};

    // seed: neighbours of s; those below s start the frontier with maxId -1
    const int rb = a.rowptr[s], re = a.rowptr[s + 1];
    for (int e = rb + tid; e < re; e += nthr) {
      const int w = a.colidx[e];
      if ((unsigned)w >= (unsigned)n) { bad = 1; continue; }
      if (w < s) {
        lab[w] = base;  // encoded -1
        atomicOr(&fA[w >> 5], 1u << (w & 31));
      } else if (w > s) {
        atomicOr(&ub[w >> 5], 1u << (w & 31));
      } else {
        s_diag = 1;
      }
    }
    __syncthreads();

    uint32_t* cur = fA;
    uint32_t* nxt = fB;
    const int SWs = (s + 31) >> 5;
    // After k levels every maxId is at most the best value over paths of <= k
    // hops (each changed vertex is expanded again); simple paths through
    // vertices below s have at most s hops, so level s+2 changes nothing.
    const long long cap = (long long)s + 3;
    long long level = 0;
    for (;;) {
      int any = 0;
      for (int b = warp * 32; b < SWs; b += nwarps * 32) {
        const int wi = b + lane;
        uint32_t word = 0u;
        if (wi < SWs) {
          word = cur[wi];
          if (word) cur[wi] = 0u;
        }
        const int cnt = __popc(word);
        const int incl = warp_incl_scan(cnt, lane);
        const int total = __shfl_sync(FULL, incl, 31);
        for (int r0 = 0; r0 < total; r0 += 32) {
          const int rank = r0 + lane;
          int sl = 0;  // number of lanes whose inclusive count is <= rank
#pragma unroll
          for (int bb = 16; bb >= 1; bb >>= 1) {
            const int t = __shfl_sync(FULL, incl, sl + bb - 1);
            if (t <= rank) sl += bb;
          }
          const int slc = sl < 31 ? sl : 31;
          const uint32_t wsrc = __shfl_sync(FULL, word, slc);
          const int exsrc = __shfl_sync(FULL, incl, slc) - __popc(wsrc);
          int v = -1;
          if (rank < total) v = ((b + slc) << 5) + nth_set_bit(wsrc, rank - exsrc);

          int eb = 0, ee = 0;
          uint32_t nmE = 0u;
          if (v >= 0) {
            eb = a.rowptr[v];
            ee = a.rowptr[v + 1];
            const uint32_t lv = lab[v];
            const uint32_t vE = base + 1u + (uint32_t)v;
            nmE = lv > vE ? lv : vE;  // encoded max(maxId(v), v)
            n_exp++;
            if (ee - eb <= BIG_DEG) {
              n_edge += (unsigned long long)(ee - eb);
              for (int e = eb; e < ee; e++) any |= relax_smem(st, nxt, a.colidx[e], nmE, &bad);
            }
          }
          unsigned bigm = __ballot_sync(FULL, v >= 0 && (ee - eb) > BIG_DEG);
          while (bigm) {
            const int l = __ffs(bigm) - 1;
            bigm &= bigm - 1;
            const int beb = __shfl_sync(FULL, eb, l), bee = __shfl_sync(FULL, ee, l);
            const uint32_t bnm = __shfl_sync(FULL, nmE, l);
            if (lane == 0) n_edge += (unsigned long long)(bee - beb);
            for (int e = beb + lane; e < bee; e += 32) any |= relax_smem(st, nxt, a.colidx[e], bnm, &bad);
          }
        }
      }
      level++;
      any = __syncthreads_or(any);
      uint32_t* t = cur;
      cur = nxt;
      nxt = t;
      if (!any) break;
      if (level >= cap) {
        if (tid == 0) atomicOr(&a.ctr->err, ERR_NOCONV);
        for (int i = tid; i < SWs; i += nthr) cur[i] = 0u;
        __syncthreads();
        break;
      }
    }

    // ---- emission: counts, pool offset, sorted row
    const int perL = (((s + nwarps - 1) / nwarps) + 31) & ~31;
    const int loL = warp * perL, hiL = min(s, loL + perL);
    int cL = 0;
    for (int i0 = loL; i0 < hiL; i0 += 32) {
      const int i = i0 + lane;
      const bool f = i < hiL && lab[i] < base + 1u + (uint32_t)i;
      cL += __popc(__ballot_sync(FULL, f));
    }
    const int ws = (s + 1) >> 5;  // first word that can hold a column > s
    const int nUW = NW - ws;
    const int perU = (((nUW + nwarps - 1) / nwarps) + 31) & ~31;
    const int loU = ws + warp * perU, hiU = min(NW, loU + perU);
    int cU = 0;
    for (int j = loU + lane; j < hiU; j += 32) cU += __popc(ub[j]);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cU += __shfl_xor_sync(FULL, cU, o);
    if (lane == 0) { s_wcL[warp] = cL; s_wcU[warp] = cU; }
    __syncthreads();
    if (tid == 0) {
      int tl = 0, tu = 0;
      for (int w = 0; w < nwarps; w++) {
        const int x = s_wcL[w]; s_wcL[w] = tl; tl += x;
        const int y = s_wcU[w]; s_wcU[w] = tu; tu += y;
      }
      const int nL = tl, nU = tu + 1;
      const unsigned long long off = atomicAdd(&a.ctr->pool_cursor, (unsigned long long)(nL + nU));
      const bool ok = off + (unsigned long long)(nL + nU) <= (unsigned long long)a.pool_cap;
      s_off = ok ? (long long)off : -1LL;
      s_nL = nL;
      a.row_off[s] = ok ? (int64_t)off : -1;
      a.row_nL[s] = nL;
      a.row_nU[s] = nU;
      a.fill_count[s] = nL + nU - ((re - rb) + (s_diag ? 0 : 1));
      atomicAdd(&a.ctr->total_L, (unsigned long long)nL);
      atomicAdd(&a.ctr->total_U, (unsigned long long)nU);
      if (ok) a.pool[off + nL] = (uint32_t)s;
      else atomicOr(&a.ctr->err, ERR_OVERFLOW);
    }
    __syncthreads();
    const long long off = s_off;
    const int nL = s_nL;
    if (off >= 0) {
      int pos = s_wcL[warp];
      for (int i0 = loL; i0 < hiL; i0 += 32) {
        const int i = i0 + lane;
        const bool f = i < hiL && lab[i] < base + 1u + (uint32_t)i;
        const unsigned m = __ballot_sync(FULL, f);
        if (f) a.pool[off + pos + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
        pos += __popc(m);
      }
    }
    {
      int pos = s_wcU[warp];
      for (int j0 = loU; j0 < hiU; j0 += 32) {
        const int j = j0 + lane;
        uint32_t word = 0u;
        if (j < hiU) { word = ub[j]; if (word) ub[j] = 0u; }
        const int c = __popc(word);
        const int inc = warp_incl_scan(c, lane);
        if (off >= 0 && word) {
          long long p = off + nL + 1 + pos + (inc - c);
          while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1;
            a.pool[p++] = (uint32_t)((j << 5) + bit);
          }
        }
        pos += __shfl_sync(FULL, inc, 31);
      }
    }
  }

  if (bad) {
    atomicOr(&a.ctr->err, ERR_COL_RANGE);
  }
  if (a.collect_stats) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      n_exp += __shfl_xor_sync(FULL, n_exp, o);
      n_edge += __shfl_xor_sync(FULL, n_edge, o);
    }
    if (lane == 0) {
      atomicAdd(&a.ctr->expansions, n_exp);
      atomicAdd(&a.ctr->edges, n_edge);
    }
  }
}

cudaError_t launch_trav_smem(const TravArgs& a, int grid, int block, cudaStream_t st) {
  const size_t bytes = trav_smem_bytes(a.n, a.S);
  cudaError_t e = cudaFuncSetAttribute(trav_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  trav_smem_kernel<<<grid, block, bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace gsofa

namespace gsofa {

int trav_smem_static_bytes() {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, trav_smem_kernel) != cudaSuccess) {
    cudaGetLastError();
    return 1024;
  }
  return (int)fa.sharedSizeBytes;
}

int trav_smem_occupancy(int block, size_t dyn_bytes) {
  if (cudaFuncSetAttribute(trav_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trav_smem_kernel, block, dyn_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace gsofa
