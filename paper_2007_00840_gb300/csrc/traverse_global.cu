// Multi-source maxId traversal, global-memory tier (Section 4, Fig. 5), with
// the frontier processed in maxId-class order.
//
// Used when a source's maxId array does not fit in shared memory.  One warp
// owns one source at a time (persistent warps, work counter in global memory);
// each warp has a slot of global memory with
//   lab      the maxId array, encoded with the value-range windows of Section 4
//            (the window base persists per slot across sources and launches);
//   P, PS    pending frontier vertices as a bitmap over [0, s) plus a summary
//            with one bit per nonzero P word;
//   U, US    the U part of the row as a bitmap plus its summary;
//   queue    the frontier of the class being expanded; list: the L columns.
//
// Frontier order.  A frontier vertex f proposes nm = max(maxId(f), f) to its
// neighbours (the relaxation of Section 4).  On large graphs with long paths
// (nested-dissection orderings, whose separators carry consecutive ids)
// breadth-first order lowers the same maxId many times (tens of expansions per
// vertex).  Here the frontier is expanded by increasing proposal, one class of
// equal proposals at a time (label-bucketed frontier processing with bucket
// width 1, cf. the comparison with Dijkstra's algorithm in Section 8).  In that
// order a maxId is set once, when a vertex is first reached, and a vertex
// reached from class p with id w > p is a fill whose proposal is its own id w;
// so the deferred part of the frontier is exactly the set of pending fills,
// kept as the bitmap P and taken in increasing order.  Class p is the pending
// fill p together with the vertices below p it reaches through unreached
// vertices below p, all expanded in parallel breadth-first levels.  The L row
// is the sequence of classes (sorted by construction); the U row comes from
// the U bitmap.
#include "internal.cuh"

namespace gsofa {

namespace {

struct Slot {
  uint32_t* lab;
  int32_t* qa;
  int32_t* qb;
  int32_t* list;
  uint32_t* P;
  uint32_t* PS;
  uint32_t* U;
  uint32_t* US;
};

__device__ __forceinline__ void set_bit2(uint32_t* W, uint32_t* S, int v) {
  const uint32_t bit = 1u << (v & 31);
  uint32_t* p = &W[v >> 5];
  if (*(volatile uint32_t*)p & bit) return;
  const uint32_t old = atomicOr(p, bit);
  if (old == 0u) atomicOr(&S[v >> 10], 1u << ((v >> 5) & 31));
}

// Fire-and-forget variant of set_bit2 (reductions, no return): the word and its
// summary bit are both set; a summary bit over a word that already had bits is
// harmless.  Visible to the warp's later reads after __syncwarp.
__device__ __forceinline__ void red_bit2(uint32_t* W, uint32_t* S, int v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(W + (v >> 5)), "r"(1u << (v & 31)) : "memory");
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(S + (v >> 10)), "r"(1u << ((v >> 5) & 31)) : "memory");
}

// Global atomic minimum issued under a predicate; 0xFFFFFFFF when not issued.
// Written as a predicated instruction so that the 8 slots of a record are in
// flight together instead of one after another behind branches.
__device__ __forceinline__ uint32_t gmin_if(uint32_t* p, uint32_t v, bool pred) {
  uint32_t r = 0xFFFFFFFFu;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.global.min.u32 %0, [%1], %2;\n\t}"
               : "+r"(r)
               : "l"(p), "r"(v), "r"((uint32_t)pred)
               : "memory");
  return r;
}

// Smallest set bit of P at a position in [from, s); -1 if none.  Warp-wide.
__device__ int next_pending(const Slot& sl, int from, int s, int lane) {
  if (from >= s) return -1;
  const int w0 = from >> 5;
  const uint32_t first = *(volatile uint32_t*)&sl.P[w0] & (0xFFFFFFFFu << (from & 31));
  if (first) {
    const int v = (w0 << 5) + __ffs(first) - 1;
    return v < s ? v : -1;
  }
  // summary search from P word w0 + 1
  const int wstart = w0 + 1;
  const int nw = (s + 31) >> 5;
  for (int sw0 = wstart >> 5; (sw0 << 5) < nw; sw0 += 32) {
    const int sw = sw0 + lane;
    uint32_t m = 0u;
    if ((sw << 5) < nw) {
      m = *(volatile uint32_t*)&sl.PS[sw];
      if (sw == (wstart >> 5)) m &= 0xFFFFFFFFu << (wstart & 31);
    }
    const unsigned any = __ballot_sync(FULL, m != 0u);
    if (any) {
      const int l = __ffs(any) - 1;
      const uint32_t ml = __shfl_sync(FULL, m, l);
      const int pw = ((sw0 + l) << 5) + __ffs(ml) - 1;  // P word index
      const uint32_t word = *(volatile uint32_t*)&sl.P[pw];
      const int v = (pw << 5) + __ffs(word) - 1;
      return (word != 0u && v < s) ? v : -1;
    }
  }
  return -1;
}

// Relax edge (. -> w) for class t of source s with encoded proposal pE.
// Returns 1 when w joins class t.
__device__ __forceinline__ int relax_class(const Slot& sl, int w, int s, int t, uint32_t pE, int n, int* bad) {
  if ((unsigned)w >= (unsigned)n) { *bad = 1; return 0; }
  if (w > s) { set_bit2(sl.U, sl.US, w); return 0; }
  if (w == s) return 0;
  const uint32_t old = atomicMin(&sl.lab[w], pE);
  if (old > pE) {                       // first reached, now with maxId t
    if (w < t) return 1;                // same class
    set_bit2(sl.P, sl.PS, w);           // a fill of L(s,:); its own class later
  }
  return 0;
}

// Relax neighbours Q0 .. Q0+K-1 of one vertex read from its ELL record for
// class t: w = v + offset, in [0, n) by construction of the records, empty
// slots hold w == v.  The label updates are issued together; vertices above s
// are U entries, lowered vertices above t are pending fills (their own class
// later).  Returns the slots whose vertex joins class t.
template <int Q0, int K>
__device__ __forceinline__ unsigned relax_slots_class(const Slot& sl, const int (&wv)[8], int v, int s, int t,
                                                      uint32_t pE) {
  uint32_t old[K];
#pragma unroll
  for (int q = 0; q < K; q++)
    old[q] = gmin_if(&sl.lab[wv[Q0 + q] < 0 ? 0 : wv[Q0 + q]], pE, wv[Q0 + q] != v && wv[Q0 + q] < s);
  unsigned em = 0u;
#pragma unroll
  for (int q = 0; q < K; q++) {
    const int w = wv[Q0 + q];
    if (w == v) continue;
    if (w > s) {
      red_bit2(sl.U, sl.US, w);
    } else if (w < s && old[q] > pE) {  // first reached, now with maxId t
      if (w < t) em |= 1u << (Q0 + q);   // same class
      else red_bit2(sl.P, sl.PS, w);     // a fill of L(s,:)
    }
  }
  return em;
}

// All 8 slots in one group, or (when registers are scarce, MINB > 8) in two
// groups of 4.
template <int MINB>
__device__ __forceinline__ unsigned relax8_class(const Slot& sl, const int (&wv)[8], int v, int s, int t,
                                                 uint32_t pE) {
  if constexpr (MINB > 8)
    return relax_slots_class<0, 4>(sl, wv, v, s, t, pE) | relax_slots_class<4, 4>(sl, wv, v, s, t, pE);
  else
    return relax_slots_class<0, 8>(sl, wv, v, s, t, pE);
}

}  // namespace

// MINB: CTAs of 4 warps per SM the register budget is sized for (8: 32 warps
// per SM with up to 64 registers; 10: 40 warps with up to 48).
template <int MINB>
__global__ void __launch_bounds__(32 * GLOBAL_WARPS_PER_CTA, MINB) trav_global_kernel(TravArgs a) {
  const int lane = threadIdx.x & 31;
  const int slot = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (slot >= a.g_slots) return;
  const size_t cap = (size_t)a.g_cap, capW = cap / 32, capS = capW / 32;
  Slot sl;
  sl.lab = a.g_lab + (size_t)slot * cap;
  sl.qa = a.g_queue + (size_t)slot * 2 * cap;
  sl.qb = sl.qa + cap;
  sl.list = a.g_list + (size_t)slot * cap;
  sl.P = a.g_P + (size_t)slot * capW;
  sl.PS = a.g_PS + (size_t)slot * capS;
  sl.U = a.g_U + (size_t)slot * capW;
  sl.US = a.g_US + (size_t)slot * capS;
  const unsigned lt = (1u << lane) - 1u;

  uint32_t base = a.g_base[slot];
  unsigned long long n_exp = 0, n_edge = 0;
  int bad = 0;

  for (;;) {
    int s = -1, mi = 0;
    if (lane == 0) {
      const int k = atomicAdd(&a.ctr->work_global, 1);
      if (k < a.nsrc && !input_error(a.ctr)) {
        if (a.mats) {  // batch: smallest source index s with item_start[s] <= k
          int lo = 0, hi = a.n - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.item_start[mid] <= k) hi = mid; else lo = mid + 1;
          }
          s = lo;
          mi = a.mat_order[k - a.item_start[lo]];
        } else {
          s = a.order ? a.order[k] : a.nsrc - 1 - k;
        }
      }
    }
    s = __shfl_sync(FULL, s, 0);
    if (s < 0) break;
    mi = __shfl_sync(FULL, mi, 0);
    int n = a.n;
    const int32_t* __restrict__ rowptr = a.rowptr;
    const int32_t* __restrict__ colidx = a.colidx;
    long long rowb = 0;
    if (a.mats) {
      const MatDesc d = a.mats[mi];
      n = d.n;
      rowptr = d.rowptr;
      colidx = d.colidx;
      rowb = d.row_base;
    }

    // maxId window of this source (values base+1+l for l in [-1, s))
    const uint32_t span = (uint32_t)s + 1u;
    if (base >= span) {
      base -= span;
    } else {
      for (size_t i = lane; i < cap; i += 32) sl.lab[i] = 0xFFFFFFFFu;
      base = 0xFFFFFFFFu - span;
      __syncwarp();
    }

    // seed: neighbours below s are pending fills with maxId -1; above s, U entries
    const int rb = __ldg(rowptr + s), re = __ldg(rowptr + s + 1);
    int diag = 0;
    for (int e = rb + lane; e < re; e += 32) {
      const int w = __ldg(colidx + e);
      if ((unsigned)w >= (unsigned)n) { bad = 1; continue; }
      if (w < s) {
        sl.lab[w] = base;
        set_bit2(sl.P, sl.PS, w);
      } else if (w > s) {
        set_bit2(sl.U, sl.US, w);
      } else {
        diag = 1;
      }
    }
    diag = __any_sync(FULL, diag);
    __syncwarp();

    // sweep the pending fills in increasing order; each starts one class
    int nL = 0;
    int cursor = 0;
    for (;;) {
      const int t = next_pending(sl, cursor, s, lane);
      if (t < 0) break;
      cursor = t + 1;
      if (lane == 0) {
        const uint32_t bit = 1u << (t & 31);
        const uint32_t old = atomicAnd(&sl.P[t >> 5], ~bit);
        if ((old & ~bit) == 0u) atomicAnd(&sl.PS[t >> 10], ~(1u << ((t >> 5) & 31)));
        sl.list[nL] = t;  // t is a fill of L(s,:)
      }
      nL++;
      const uint32_t pE = base + 1u + (uint32_t)t;  // encoded class value (proposal) t
      // class t: breadth-first over unreached vertices below t; the first level is t alone
      int32_t* qc = sl.qa;
      int32_t* qn = sl.qb;
      int qlen = 1;
      bool single = true;
      while (qlen > 0) {
        int nq = 0;
        if (a.ell) {
          // one vertex per lane from its ELL record; rows without a record
          // (sentinel) are walked from the CSR, one lane per row, afterwards
          for (int i0 = 0; i0 < qlen; i0 += 32) {
            const int i = i0 + lane;
            int v = -1;
            if (i < qlen) v = single ? t : qc[i];
            uint32_t h0 = 0u, h1 = 0u, h2 = 0u, h3 = 0u;
            bool fb = false;
            if (v >= 0) {
              const int4 r4 = __ldg(a.ell + rowb + v);
              h0 = (uint32_t)r4.x; h1 = (uint32_t)r4.y; h2 = (uint32_t)r4.z; h3 = (uint32_t)r4.w;
              fb = (h0 & 0xFFFFu) == 0x8000u;
              if (fb) h0 = 0u;
              if (a.collect_stats) {
                n_exp++;
                n_edge += (unsigned long long)(__ldg(rowptr + v + 1) - __ldg(rowptr + v));
              }
            }
            int wv[8];
            wv[0] = v + (int)(short)(h0 & 0xFFFFu); wv[1] = v + (int)(short)(h0 >> 16);
            wv[2] = v + (int)(short)(h1 & 0xFFFFu); wv[3] = v + (int)(short)(h1 >> 16);
            wv[4] = v + (int)(short)(h2 & 0xFFFFu); wv[5] = v + (int)(short)(h2 >> 16);
            wv[6] = v + (int)(short)(h3 & 0xFFFFu); wv[7] = v + (int)(short)(h3 >> 16);
            const unsigned em = v >= 0 ? relax8_class<MINB>(sl, wv, v, s, t, pE) : 0u;
            const int cnt = __popc(em);
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int tt = __shfl_up_sync(FULL, inc, o);
              if (lane >= o) inc += tt;
            }
            int pos = nq + inc - cnt;
#pragma unroll
            for (int q = 0; q < 8; q++)
              if ((em >> q) & 1u) qn[pos++] = wv[q];
            nq += __shfl_sync(FULL, inc, 31);
            // rows that did not fit a record
            unsigned fm = __ballot_sync(FULL, fb);
            while (fm) {
              const int l = __ffs(fm) - 1;
              fm &= fm - 1;
              const int u = __shfl_sync(FULL, v, l);
              const int eb = __ldg(rowptr + u), ee = __ldg(rowptr + u + 1);
              for (int e0 = eb; e0 < ee; e0 += 32) {
                const int e = e0 + lane;
                int w = 0, enq = 0;
                if (e < ee) {
                  w = __ldg(colidx + e);
                  if (w != u) enq = relax_class(sl, w, s, t, pE, n, &bad);
                }
                const unsigned m = __ballot_sync(FULL, enq);
                if (enq) qn[nq + __popc(m & lt)] = w;
                nq += __popc(m);
              }
            }
          }
          single = false;
        } else if (single) {  // one vertex: the lanes share its row
          const int eb = __ldg(rowptr + t), ee = __ldg(rowptr + t + 1);
          if (lane == 0) { n_exp++; n_edge += (unsigned long long)(ee - eb); }
          for (int e0 = eb; e0 < ee; e0 += 32) {
            const int e = e0 + lane;
            int w = 0, enq = 0;
            if (e < ee) {
              w = __ldg(colidx + e);
              enq = relax_class(sl, w, s, t, pE, n, &bad);
            }
            const unsigned m = __ballot_sync(FULL, enq);
            if (enq) qn[nq + __popc(m & lt)] = w;
            nq += __popc(m);
          }
          single = false;
        } else {  // several: one vertex per lane
          for (int i0 = 0; i0 < qlen; i0 += 32) {
            const int i = i0 + lane;
            int eb = 0, ee = 0;
            if (i < qlen) {
              const int v = qc[i];
              eb = __ldg(rowptr + v);
              ee = __ldg(rowptr + v + 1);
              n_exp++;
              n_edge += (unsigned long long)(ee - eb);
            }
            const int maxdeg = __reduce_max_sync(FULL, ee - eb);
            for (int k = 0; k < maxdeg; k++) {
              int w = 0, enq = 0;
              if (eb + k < ee) {
                w = __ldg(colidx + eb + k);
                enq = relax_class(sl, w, s, t, pE, n, &bad);
              }
              const unsigned m = __ballot_sync(FULL, enq);
              if (enq) qn[nq + __popc(m & lt)] = w;
              nq += __popc(m);
            }
          }
        }
        __syncwarp();
        int32_t* tq = qc;
        qc = qn;
        qn = tq;
        qlen = nq;
      }
    }

    // ---- emission: count U through its summary, take a pool offset, write the row
    const int nw = (n + 31) >> 5;
    const int ns = (nw + 31) >> 5;
    const int s_lo = (s + 1) >> 10;  // first summary word that can hold a column > s
    int nU = 1;
    for (int sw0 = s_lo; sw0 < ns; sw0 += 32) {
      const int sw = sw0 + lane;
      const uint32_t m = sw < ns ? *(volatile uint32_t*)&sl.US[sw] : 0u;
      unsigned any = __ballot_sync(FULL, m != 0u);
      while (any) {
        const int l = __ffs(any) - 1;
        any &= any - 1;
        const uint32_t ml = __shfl_sync(FULL, m, l);
        const int pw = ((sw0 + l) << 5) + lane;
        const uint32_t word = ((ml >> lane) & 1u) ? *(volatile uint32_t*)&sl.U[pw] : 0u;
        int c = __popc(word);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        nU += c;
      }
    }
    unsigned long long off = 0ull;
    int ok = 0;
    if (lane == 0) {
      off = atomicAdd(&a.ctr->pool_cursor, (unsigned long long)(nL + nU));
      ok = off + (unsigned long long)(nL + nU) <= (unsigned long long)a.pool_cap;
      a.row_off[rowb + s] = ok ? (int64_t)off : -1;
      a.row_nL[rowb + s] = nL;
      a.row_nU[rowb + s] = nU;
      a.fill_count[rowb + s] = nL + nU - ((re - rb) + (diag ? 0 : 1));
      atomicAdd(&a.ctr->total_L, (unsigned long long)nL);
      atomicAdd(&a.ctr->total_U, (unsigned long long)nU);
      if (a.mat_tot) {
        atomicAdd(&a.mat_tot[2 * mi], (unsigned long long)nL);
        atomicAdd(&a.mat_tot[2 * mi + 1], (unsigned long long)nU);
      }
      if (ok) a.pool[off + nL] = (uint32_t)s;
      else atomicOr(&a.ctr->err, ERR_OVERFLOW);
    }
    off = __shfl_sync(FULL, off, 0);
    ok = __shfl_sync(FULL, ok, 0);
    if (ok)
      for (int i = lane; i < nL; i += 32) a.pool[off + i] = (uint32_t)sl.list[i];
    long long pos = (long long)off + nL + 1;
    for (int sw0 = s_lo; sw0 < ns; sw0 += 32) {
      const int sw = sw0 + lane;
      const uint32_t m = sw < ns ? *(volatile uint32_t*)&sl.US[sw] : 0u;
      unsigned any = __ballot_sync(FULL, m != 0u);
      while (any) {
        const int l = __ffs(any) - 1;
        any &= any - 1;
        const uint32_t ml = __shfl_sync(FULL, m, l);
        const int pw = ((sw0 + l) << 5) + lane;
        uint32_t word = 0u;
        if ((ml >> lane) & 1u) {
          word = *(volatile uint32_t*)&sl.U[pw];
          sl.U[pw] = 0u;
        }
        const int c = __popc(word);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int tt = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += tt;
        }
        if (ok) {
          long long p = pos + (inc - c);
          while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            a.pool[p++] = (uint32_t)((pw << 5) + b);
          }
        }
        pos += __shfl_sync(FULL, inc, 31);
      }
      if (sw < ns && m) sl.US[sw] = 0u;
    }
    __syncwarp();
  }

  if (lane == 0) a.g_base[slot] = base;
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

cudaError_t launch_trav_global(const TravArgs& a, int grid, int block, cudaStream_t st, int warps_per_sm) {
  if (block != 32 * GLOBAL_WARPS_PER_CTA) return cudaErrorInvalidConfiguration;
  if (warps_per_sm > 32) trav_global_kernel<10><<<grid, block, 0, st>>>(a);
  else trav_global_kernel<8><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace gsofa
