// Multi-source maxId traversal, global-memory tier (Section 4, Fig. 5).
//
// Used for sources whose maxId array does not fit in shared memory.  The rule
// is the same as in traverse_smem.cu; the data placement differs:
//   g_lab      per-slot maxId array in HBM (slot = CTA), encoded with the
//              value-range windows of Section 4; the window base persists per
//              slot across sources and launches (g_base), so the array is only
//              refilled when the 32-bit range is used up;
//   g_queue    current / next frontier as compact queues (a frontier holds at
//              most s distinct vertices), deduplicated with the g_inq bitmap;
//   g_rowbits  the columns of row s found so far (L fills and U entries) as a
//              bitmap over [0, n), with a one-bit-per-word summary in shared
//              memory so emission visits only nonzero words, in order.
// Bubble removal (Section 6): vertices above the source keep no maxId.
#include "internal.cuh"

namespace gsofa {

namespace {

constexpr int BIG_DEG = 32;
constexpr int BATCH = 8;  // column loads issued together per frontier vertex

struct GState {
  uint32_t* lab;
  uint32_t* inq;
  uint32_t* rowbits;
  uint32_t* summ;
  int32_t* qnext;
  int* qn;         // shared counter of qnext
  uint32_t base;
  int32_t s;
  int32_t n;
  int32_t fill_first;
};

__device__ __forceinline__ void set_rowbit(const GState& g, int w) {
  const uint32_t bit = 1u << (w & 31);
  uint32_t* p = &g.rowbits[w >> 5];
  if (*(volatile uint32_t*)p & bit) return;
  const uint32_t old = atomicOr(p, bit);
  if (old == 0u) atomicOr(&g.summ[w >> 10], 1u << ((w >> 5) & 31));
}

__device__ __forceinline__ void enqueue(const GState& g, int w) {
  const uint32_t bit = 1u << (w & 31);
  const uint32_t old = atomicOr(&g.inq[w >> 5], bit);
  if (!(old & bit)) {
    const int pos = atomicAdd(g.qn, 1);
    g.qnext[pos] = w;
  }
}

__device__ __forceinline__ void relax_g(const GState& g, int w, uint32_t nmE, int* bad) {
  if ((unsigned)w >= (unsigned)g.n) { *bad = 1; return; }
  if (w < g.s) {
    const uint32_t wE = g.base + 1u + (uint32_t)w;
    if (g.fill_first && *(volatile uint32_t*)&g.lab[w] < wE) return;
    const uint32_t old = atomicMin(&g.lab[w], nmE);
    if (nmE < old) {
      if (nmE < wE && old >= wE) set_rowbit(g, w);   // w just became a fill of L(s,:)
      if (old > wE) enqueue(g, w);                   // w's own proposal changed
    }
  } else if (w > g.s) {
    set_rowbit(g, w);
  }
}

}  // namespace

size_t trav_global_smem_bytes(int32_t n) {
  const size_t NW = ((size_t)n + 31) / 32;
  return 4 * ((NW + 31) / 32);
}

__global__ void __launch_bounds__(1024, 1) trav_global_kernel(TravArgs a) {
  extern __shared__ uint32_t summ[];
  const int n = a.n;
  const int NW = (n + 31) >> 5, NSW = (NW + 31) >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarps = nthr >> 5;
  const size_t slot = blockIdx.x;
  const size_t cap = (size_t)a.g_cap, capW = (cap + 31) / 32;
  uint32_t* lab = a.g_lab + slot * cap;
  int32_t* qA = a.g_queue + slot * 2 * cap;
  int32_t* qB = qA + cap;
  uint32_t* inq = a.g_inq + slot * capW;
  uint32_t* rowbits = a.g_rowbits + slot * capW;

  __shared__ int s_src, s_diag;
  __shared__ int s_q[3];
  __shared__ int s_wc[32][2];
  __shared__ long long s_off;
  __shared__ int s_nL;
  __shared__ uint32_t s_base;

  for (int i = tid; i < NSW; i += nthr) summ[i] = 0u;
  const uint32_t span = (uint32_t)n + 2u;
  if (tid == 0) s_base = a.g_base[slot];
  unsigned long long n_exp = 0, n_edge = 0;
  int bad = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const int k = atomicAdd(&a.ctr->work_global, 1);
      s_src = (k < a.nsrc && !input_error(a.ctr)) ? a.order[k] : -1;
      s_diag = 0;
      s_q[0] = s_q[1] = s_q[2] = 0;
    }
    __syncthreads();
    const int s = s_src;
    if (s < 0) break;

    // next maxId window; refill the slot when the 32-bit range is used up
    uint32_t base = s_base;
    if (base >= span) {
      base -= span;
    } else {
      for (size_t i = tid; i < cap; i += nthr) lab[i] = 0xFFFFFFFFu;
      base = 0xFFFFFFFFu - span;
    }
    __syncthreads();  // everyone has read s_base (and the refill is done)
    if (tid == 0) s_base = base;

    GState g{lab, inq, rowbits, summ, qA, &s_q[0], base, s, n, a.fill_first};

    const int rb = a.rowptr[s], re = a.rowptr[s + 1];
    for (int e = rb + tid; e < re; e += nthr) {
      const int w = a.colidx[e];
      if ((unsigned)w >= (unsigned)n) { bad = 1; continue; }
      if (w < s) {
        lab[w] = base;          // encoded -1: no intermediate vertex
        set_rowbit(g, w);
        enqueue(g, w);
      } else if (w > s) {
        set_rowbit(g, w);
      } else {
        s_diag = 1;
      }
    }
    __syncthreads();

    int32_t* qcur = qA;
    int32_t* qnxt = qB;
    int qlen = s_q[0];
    // same bound as the shared tier: labels are final after s+1 levels
    const long long cap_lv = (long long)s + 3;
    long long level = 0;
    while (qlen > 0) {
      level++;
      const int li = (int)(level % 3);
      if (tid == 0) s_q[(li + 1) % 3] = 0;
      g.qnext = qnxt;
      g.qn = &s_q[li];
      // From here on a dedup bit means "already in the next frontier": clear the
      // bits of the current frontier before any expansion of this level, so a
      // vertex whose maxId drops while it is being expanded is queued again.
      for (int i = tid; i < qlen; i += nthr) {
        const int v = qcur[i];
        atomicAnd(&inq[v >> 5], ~(1u << (v & 31)));
      }
      __syncthreads();
      for (int i0 = warp * 32; i0 < qlen; i0 += nthr) {
        const int i = i0 + lane;
        int v = -1, eb = 0, ee = 0;
        uint32_t nmE = 0u;
        if (i < qlen) {
          v = qcur[i];
          eb = __ldg(a.rowptr + v);
          ee = __ldg(a.rowptr + v + 1);
          const uint32_t lv = *(volatile uint32_t*)&lab[v];
          const uint32_t vE = base + 1u + (uint32_t)v;
          nmE = lv > vE ? lv : vE;
          n_exp++;
          if (ee - eb <= BIG_DEG) {
            n_edge += (unsigned long long)(ee - eb);
            for (int e0 = eb; e0 < ee; e0 += BATCH) {
              int wv[BATCH];  // independent loads first, then the relaxations
#pragma unroll
              for (int q = 0; q < BATCH; q++) wv[q] = (e0 + q < ee) ? __ldg(a.colidx + e0 + q) : 0;
#pragma unroll
              for (int q = 0; q < BATCH; q++)
                if (e0 + q < ee) relax_g(g, wv[q], nmE, &bad);
            }
          }
        }
        unsigned bigm = __ballot_sync(FULL, v >= 0 && (ee - eb) > BIG_DEG);
        while (bigm) {
          const int l = __ffs(bigm) - 1;
          bigm &= bigm - 1;
          const int beb = __shfl_sync(FULL, eb, l), bee = __shfl_sync(FULL, ee, l);
          const uint32_t bnm = __shfl_sync(FULL, nmE, l);
          if (lane == 0) n_edge += (unsigned long long)(bee - beb);
          for (int e = beb + lane; e < bee; e += 32) relax_g(g, __ldg(a.colidx + e), bnm, &bad);
        }
      }
      __syncthreads();
      qlen = s_q[li];
      int32_t* t = qcur;
      qcur = qnxt;
      qnxt = t;
      if (level >= cap_lv && qlen > 0) {
        // never expected: drop the frontier, leave the slot clean, flag it
        for (int i = tid; i < qlen; i += nthr) {
          const int v = qcur[i];
          atomicAnd(&inq[v >> 5], ~(1u << (v & 31)));
        }
        if (tid == 0) atomicOr(&a.ctr->err, ERR_NOCONV);
        __syncthreads();
        break;
      }
    }

    // ---- emission: walk the summary in order; thread t owns a contiguous range
    const int per = (NSW + nthr - 1) / nthr;
    const int lo = tid * per, hi = min(NSW, lo + per);
    int cL = 0, cU = 0;
    for (int sw = lo; sw < hi; sw++) {
      uint32_t m = summ[sw];
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        const int fw = (sw << 5) + j;
        const uint32_t word = rowbits[fw];
        const int wb = fw << 5;
        if (wb + 31 < s) cL += __popc(word);
        else if (wb > s) cU += __popc(word);
        else {
          const int k = s - wb;  // bit of s inside this word (never set)
          const uint32_t lowm = (k == 0) ? 0u : (0xFFFFFFFFu >> (32 - k));
          cL += __popc(word & lowm);
          cU += __popc(word & ~lowm);
        }
      }
    }
    // block-wide exclusive scan of (cL, cU) in thread order
    int iL = cL, iU = cU;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int tL = __shfl_up_sync(FULL, iL, o), tU = __shfl_up_sync(FULL, iU, o);
      if (lane >= o) { iL += tL; iU += tU; }
    }
    if (lane == 31) { s_wc[warp][0] = iL; s_wc[warp][1] = iU; }
    __syncthreads();
    if (tid == 0) {
      int tl = 0, tu = 0;
      for (int w = 0; w < nwarps; w++) {
        const int x = s_wc[w][0]; s_wc[w][0] = tl; tl += x;
        const int y = s_wc[w][1]; s_wc[w][1] = tu; tu += y;
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
    long long pL = off + s_wc[warp][0] + (iL - cL);
    long long pU = off + nL + 1 + s_wc[warp][1] + (iU - cU);
    for (int sw = lo; sw < hi; sw++) {
      uint32_t m = summ[sw];
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        const int fw = (sw << 5) + j;
        uint32_t word = rowbits[fw];
        rowbits[fw] = 0u;
        if (off >= 0) {
          while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int col = (fw << 5) + b;
            if (col < s) a.pool[pL++] = (uint32_t)col;
            else a.pool[pU++] = (uint32_t)col;
          }
        }
      }
      summ[sw] = 0u;
    }
  }

  __syncthreads();
  if (tid == 0) a.g_base[slot] = s_base;
  if (bad) atomicOr(&a.ctr->err, ERR_COL_RANGE);
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

cudaError_t launch_trav_global(const TravArgs& a, int grid, int block, cudaStream_t st) {
  const size_t bytes = trav_global_smem_bytes(a.n);
  cudaError_t e = cudaFuncSetAttribute(trav_global_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(bytes > 0 ? bytes : 4));
  if (e != cudaSuccess) return e;
  trav_global_kernel<<<grid, block, bytes > 0 ? bytes : 4, st>>>(a);
  return cudaGetLastError();
}

}  // namespace gsofa
