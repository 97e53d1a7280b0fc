// Multi-source maxId traversal, shared-memory tier (Section 4, Fig. 5).
//
// One CTA owns one source row s at a time and loops over sources from a global
// work counter (persistent CTAs, largest source first).  Per source it keeps
// in shared memory:
//   lab[0..S)   maxId of every vertex below the source (bubble removal,
//               Section 6: vertices above s never need one), or of every
//               vertex of the matrix when S >= n (then also used for U, see
//               below).  16-bit when the matrix order allows it, else 32-bit.
//               Values use the value-range windows of Section 4 ("Optimizing
//               the initialization of maxId"): the k-th source of this CTA
//               uses the window [base_k, base_k + s_k] with base_k decreasing,
//               so any value above the window reads as "not reached" and lab[]
//               is refilled only when the range is used up;
//   list0/list1 the current and next frontier as compact lists; entries past
//               the list capacity spill to a per-CTA area in global memory (the
//               external frontier management of Section 6, one level down);
//   D0/D1       dedup bitmaps: bit v of D[b] is set iff v is in list b;
//   ub          the U part of the row as a bitmap over [0, n) (when S < n).
// maxId of a vertex is the smallest "largest intermediate vertex" over the
// paths found so far; a direct neighbour of s has no intermediate (-1).
//
// Level loop: every frontier vertex f proposes nm = max(maxId(f), f) to each
// neighbour w (atomic min).  If the proposal lowers maxId(w) and w was not
// already a fill (old > w), w's own proposal changed, so w joins the next
// frontier; w is a fill of L(s,:) iff its final maxId < w (Theorem 1).
// Neighbours above s are U entries: with a label slot for every vertex they
// are recorded by lowering their label into the window ("U by labels"), else
// in ub.  Neighbours come from 16-byte ELL records of 16-bit offsets (one load
// per vertex; rows that do not fit are read from the CSR) or from the CSR.
// Lanes of a warp take consecutive list entries (on small frontiers 2, 4 or 8
// lanes share a vertex and split its record), and newly queued vertices are
// appended with one shared-memory atomic per warp.  One barrier per level.
// A worklist schedule without level barriers is an option (async_source).
//
// Emission writes the sorted row [L cols | s | U cols] to the row pool at an
// offset taken with one atomicAdd, plus the row's counts and fill count.
#include "internal.cuh"

namespace gsofa {

namespace {

constexpr int BIG_DEG = 32;
constexpr int BATCH = 8;      // column loads issued together per frontier vertex (row slots)
constexpr int EB_UNROLL = 4;  // flattened chunks of 32 entries loaded together (edge-balanced)


__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename LabT>
struct LabOps;

template <>
struct LabOps<uint32_t> {
  static constexpr uint32_t MAXV = 0xFFFFFFFFu;
  // lab[w] = min(lab[w], v); *old = the previous value; true iff it decreased
  static __device__ __forceinline__ bool lower(uint32_t* lab, int w, uint32_t v, uint32_t* old) {
    *old = atomicMin(lab + w, v);
    return v < *old;
  }
};

template <>
struct LabOps<uint16_t> {
  static constexpr uint32_t MAXV = 0xFFFFu;
  // lab[w] = min(lab[w], v) by compare-and-swap on the aligned 32-bit word that
  // holds lab[w] and its neighbour; *old = the previous value; true iff it decreased
  static __device__ __forceinline__ bool lower(uint16_t* lab, int w, uint32_t v, uint32_t* old) {
    uint32_t* wp = reinterpret_cast<uint32_t*>(lab) + (w >> 1);
    const int sh = (w & 1) << 4;
    uint32_t word = *(volatile uint32_t*)wp;
    uint32_t cur = (word >> sh) & 0xFFFFu;
    while (v < cur) {
      const uint32_t prev = atomicCAS(wp, word, (word & ~(0xFFFFu << sh)) | (v << sh));
      if (prev == word) { *old = cur; return true; }
      word = prev;
      cur = (word >> sh) & 0xFFFFu;
    }
    *old = cur;
    return false;
  }
};

template <typename LabT>
struct Src {
  LabT* lab;
  uint32_t* ub;
  uint32_t* Dn;      // dedup bitmap of the list being built
  LabT* Ln;          // list being built (shared part)
  int32_t* Sn;       // list being built (spilled part)
  int* qn;           // its length counter
  uint32_t base;
  int32_t s, n, cap;
};

// relax() for a neighbour w < s (no range check: callers guarantee w in [0, s)).
template <typename LabT, bool FF>
__device__ __forceinline__ int relax_low(const Src<LabT>& c, int w, uint32_t nmE) {
  const uint32_t wE = c.base + 1u + (uint32_t)w;
  if (FF && (uint32_t)c.lab[w] < wE) return 0;
  uint32_t old;
  if (!LabOps<LabT>::lower(c.lab, w, nmE, &old) || old <= wE) return 0;
  // nearly every lowering that reaches here is a vertex's first entry into the
  // list, so a read of the bit before the atomic would rarely save it
  const uint32_t bit = 1u << (w & 31);
  return (atomicOr(&c.Dn[w >> 5], bit) & bit) ? 0 : 1;
}

// relax() when every vertex of the matrix has a label slot ("U by labels"):
// a neighbour w > s is recorded as a U entry by lowering its label into the
// current window, like any other vertex, so there is no U branch; only w < s
// can join the frontier.  w in [0, n) is the caller's guarantee; w == s and
// w == f are harmless (s is never read back, f's own proposal never lowers it).
template <typename LabT, bool FF>
__device__ __forceinline__ int relax_ul(const Src<LabT>& c, int w, uint32_t nmE) {
  const uint32_t wE = c.base + 1u + (uint32_t)w;
  if (FF && w < c.s && (uint32_t)c.lab[w] < wE) return 0;
  uint32_t old;
  if (!LabOps<LabT>::lower(c.lab, w, nmE, &old) || w >= c.s || old <= wE) return 0;
  // nearly every lowering that reaches here is a vertex's first entry into the
  // list, so a read of the bit before the atomic would rarely save it
  const uint32_t bit = 1u << (w & 31);
  return (atomicOr(&c.Dn[w >> 5], bit) & bit) ? 0 : 1;
}

// relax() for a neighbour read from an ELL record: w is in [0, n) and w != f
// by construction of the records, so neither is checked here.
template <typename LabT, bool FF, bool UL>
__device__ __forceinline__ int relax_rec(const Src<LabT>& c, int w, uint32_t nmE) {
  if (UL) return relax_ul<LabT, FF>(c, w, nmE);
  if (w < c.s) return relax_low<LabT, FF>(c, w, nmE);
  if (w > c.s) atomicOr(&c.ub[w >> 5], 1u << (w & 31));
  return 0;
}

// Decide edge (f -> w) with encoded proposal nmE.  Returns 1 if w must be
// appended to the next frontier (its dedup bit was set here).
template <typename LabT, bool FF, bool UL>
__device__ __forceinline__ int relax(const Src<LabT>& c, int w, uint32_t nmE, int* bad) {
  if ((unsigned)w >= (unsigned)c.n) { *bad = 1; return 0; }
  if (UL) return relax_ul<LabT, FF>(c, w, nmE);
  if (w < c.s) return relax_low<LabT, FF>(c, w, nmE);
  if (w > c.s) {
    const uint32_t bit = 1u << (w & 31);
    if (!(c.ub[w >> 5] & bit)) atomicOr(&c.ub[w >> 5], bit);
  }
  return 0;
}

// Append w (if enq) with one shared atomic per warp; all 32 lanes call this.
template <typename LabT>
__device__ __forceinline__ void append(const Src<LabT>& c, int enq, int w, int lane) {
  const unsigned m = __ballot_sync(FULL, enq);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(c.qn, __popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (enq) {
    const int pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < c.cap) c.Ln[pos] = (LabT)w;
    else c.Sn[pos - c.cap] = w;
  }
}

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// One level of the ELL path when the frontier is small: LPV lanes share a
// frontier vertex and each relaxes 8 / LPV of its record's slots, so the chain
// of dependent slot updates a warp walks is LPV times shorter (the level is
// latency-bound: every warp has at most one round).  Rows without a record are
// walked from the CSR by the whole warp.
template <typename LabT, bool FF, bool UL, int LPV>
__device__ __forceinline__ void small_level(const Src<LabT>& c, const TravArgs& a, const LabT* Lc, const int32_t* Sc,
                                            uint32_t* Dc, int qc, int CAP, long long rowb, uint32_t base,
                                            const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                            int warp, int nwarps, int lane, unsigned long long& n_exp,
                                            unsigned long long& n_edge, int* bad) {
  constexpr int SPL = 8 / LPV, VPW = 32 / LPV;
  const int sub = lane & (LPV - 1);
  const unsigned lt = (1u << lane) - 1u;
  for (int r0 = warp * VPW; r0 < qc; r0 += nwarps * VPW) {
    const int r = r0 + lane / LPV;
    int v = -1;
    uint32_t nmE = 0u;
    if (r < qc) {
      v = r < CAP ? (int)Lc[r] : Sc[r - CAP];
      Dc[v >> 5] = 0u;  // as in the main loop: nothing sets bits of Dc during the level
      const uint32_t lv = (uint32_t)c.lab[v];
      const uint32_t vE = base + 1u + (uint32_t)v;
      nmE = lv > vE ? lv : vE;
      if (sub == 0) {
        n_exp++;
        if (a.collect_stats) n_edge += (unsigned long long)(__ldg(rowptr + v + 1) - __ldg(rowptr + v));
      }
    }
    bool fb = false;
    uint32_t x0 = 0u, x1 = 0u;  // this lane's record words (SPL = 4: two words; 2: one; 1: half of one)
    if (v >= 0) {
      const int4 r4 = __ldg(a.ell + rowb + v);
      fb = ((uint32_t)r4.x & 0xFFFFu) == 0x8000u;
      if (!fb) {
        if (SPL == 4) {
          x0 = sub ? (uint32_t)r4.z : (uint32_t)r4.x;
          x1 = sub ? (uint32_t)r4.w : (uint32_t)r4.y;
        } else {
          const int wi = SPL == 2 ? sub : (sub >> 1);
          x0 = wi == 0 ? (uint32_t)r4.x : wi == 1 ? (uint32_t)r4.y : wi == 2 ? (uint32_t)r4.z : (uint32_t)r4.w;
          if (SPL == 1) x0 = (sub & 1) ? (x0 >> 16) : (x0 & 0xFFFFu);
        }
      }
    }
    int wv[SPL];
#pragma unroll
    for (int q = 0; q < SPL; q++) {
      const uint32_t x = q < 2 ? x0 : x1;
      wv[q] = v + (int)(short)((q & 1) ? (x >> 16) : (x & 0xFFFFu));
    }
    unsigned em = 0u;
#pragma unroll
    for (int q = 0; q < SPL; q++)
      if (wv[q] != v && relax_rec<LabT, FF, UL>(c, wv[q], nmE)) em |= 1u << q;
    const int cnt = __popc(em);
    const int incl = warp_incl_scan(cnt, lane);
    const int tot = __shfl_sync(FULL, incl, 31);
    if (tot) {
      int basep = 0;
      if (lane == 31) basep = atomicAdd(c.qn, tot);
      basep = __shfl_sync(FULL, basep, 31);
      int pos = basep + incl - cnt;
#pragma unroll
      for (int q = 0; q < SPL; q++) {
        if ((em >> q) & 1u) {
          if (pos < CAP) c.Ln[pos] = (LabT)wv[q]; else c.Sn[pos - CAP] = wv[q];
          pos++;
        }
      }
    }
    unsigned fm = __ballot_sync(FULL, fb && sub == 0);
    while (fm) {
      const int l = __ffs(fm) - 1;
      fm &= fm - 1u;
      const int u = __shfl_sync(FULL, v, l);
      const uint32_t unm = __shfl_sync(FULL, nmE, l);
      const int eb = __ldg(rowptr + u), ee = __ldg(rowptr + u + 1);
      for (int e0 = eb; e0 < ee; e0 += 32) {
        const int e = e0 + lane;
        int w = u, enq = 0;
        if (e < ee) {
          w = __ldg(colidx + e);
          if (w != u) enq = relax<LabT, FF, UL>(c, w, unm, bad);
        }
        const unsigned m = __ballot_sync(FULL, enq);
        if (m) {
          const int leader = __ffs(m) - 1;
          int b2 = 0;
          if (lane == leader) b2 = atomicAdd(c.qn, __popc(m));
          b2 = __shfl_sync(FULL, b2, leader);
          if (enq) {
            const int p2 = b2 + __popc(m & lt);
            if (p2 < CAP) c.Ln[p2] = (LabT)w; else c.Sn[p2 - CAP] = w;
          }
        }
      }
    }
  }
}



}  // namespace

template <typename LabT>
size_t trav_smem_bytes_t(int32_t n, int32_t S, int32_t cap) {
  const size_t SW = ((size_t)S + 31) / 32, NW = ((size_t)n + 31) / 32;
  return align16(sizeof(LabT) * (size_t)S) + 4 * (2 * SW + NW) + align16(2 * sizeof(LabT) * (size_t)cap);
}

size_t trav_smem_bytes(int32_t n, int32_t S, int32_t cap, int label16) {
  return label16 ? trav_smem_bytes_t<uint16_t>(n, S, cap) : trav_smem_bytes_t<uint32_t>(n, S, cap);
}

// Emission of the 16-bit labels, 8 per lane (one 16-byte load): bit q of the
// result is set iff i + q lies in (lo_excl, hi) and its label marks it: L
// (below the source) when label < base + 1 + (i + q), i.e. maxId < i + q, U
// (above it) when label <= top, i.e. reached in this window.  i is a multiple
// of 8 inside the label array.
template <bool U>
__device__ __forceinline__ unsigned label_mask8(const uint16_t* lab, int i, int lo_excl, int hi, uint32_t base,
                                                uint32_t top) {
  if (i >= hi) return 0u;
  const uint4 r = *reinterpret_cast<const uint4*>(lab + i);
  const uint32_t wd[4] = {r.x, r.y, r.z, r.w};
  unsigned m = 0u;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const uint32_t l = (wd[q >> 1] >> ((q & 1) << 4)) & 0xFFFFu;
    const int j = i + q;
    const bool f = U ? (j > lo_excl && j < hi && l <= top) : (j < hi && l < base + 1u + (uint32_t)j);
    m |= (unsigned)f << q;
  }
  return m;
}

constexpr uint16_t RING_EMPTY = 0xFFFFu;  // vertex ids of the 16-bit tier are <= 65532
constexpr long long ASYNC_WAIT_CYCLES = 2000000000LL;  // bound of every wait (about 1 s)

// A wait gives up when its bound passes or another wait already gave up.
__device__ __forceinline__ bool wait_expired(long long t0, DevCounters* ctr) {
  if (*(volatile int32_t*)&ctr->err & ERR_NOCONV) return true;
  if (clock64() - t0 > ASYNC_WAIT_CYCLES) {
    atomicOr(&ctr->err, ERR_NOCONV);
    return true;
  }
  return false;
}

__device__ __forceinline__ void fence_sc_cta() { asm volatile("fence.sc.cta;" ::: "memory"); }

// relax_ul for the asynchronous schedule: the in-queue bit is examined by an
// atomic after a sequentially consistent fence, so that either this lane sees
// a popper's clearing of the bit (and queues w again) or the popper, which
// fences between clearing the bit and reading the label, sees the new label.
__device__ __forceinline__ int relax_async(const Src<uint16_t>& c, int w, uint32_t nmE) {
  const uint32_t wE = c.base + 1u + (uint32_t)w;
  uint32_t old;
  if (!LabOps<uint16_t>::lower(c.lab, w, nmE, &old) || w >= c.s || old <= wE) return 0;
  fence_sc_cta();
  const uint32_t bit = 1u << (w & 31);
  return (atomicOr(&c.Dn[w >> 5], bit) & bit) ? 0 : 1;
}

// Ring slot of position p (positions grow without bound within a source).
__device__ __forceinline__ int ring_slot(int p, int qs) { return p % qs; }

// Push `cnt` vertices of this lane (in w[0..7] where bit q of em is set) to
// the ring; all 32 lanes call this.  pending is raised before the positions
// are taken, so a warp that sees pending == 0 knows nothing is queued or being
// processed.  A slot from the previous lap may still be in a popper's hands
// (reserved, not yet read): wait for it, bounded.
__device__ __forceinline__ void ring_push8(uint16_t* ring, int qs, int* head_tail_pend, const int (&wv)[8],
                                           unsigned em, int lane, DevCounters* ctr) {
  const int cnt = __popc(em);
  const int incl = warp_incl_scan(cnt, lane);
  const int tot = __shfl_sync(FULL, incl, 31);
  if (!tot) return;
  int basep = 0;
  if (lane == 31) {
    atomicAdd(&head_tail_pend[2], tot);
    basep = atomicAdd(&head_tail_pend[1], tot);
  }
  basep = __shfl_sync(FULL, basep, 31);
  int pos = basep + incl - cnt;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    if ((em >> q) & 1u) {
      volatile uint16_t* sl = ring + ring_slot(pos, qs);
      const long long t0 = clock64();
      while (*sl != RING_EMPTY)
        if (wait_expired(t0, ctr)) break;
      *sl = (uint16_t)wv[q];
      pos++;
    }
  }
}

// The asynchronous schedule of one source (16-bit labels, every vertex with a
// label slot, ELL records): instead of breadth-first levels separated by
// barriers, warps take up to 32 queued vertices at a time from a ring in
// shared memory and queue what they lower.  Dn is the in-queue bitmap (one bit
// per vertex: queued and not yet taken), so the ring never holds more than S
// entries.  Ends when nothing is queued and no warp holds taken work.
__device__ void async_source(const Src<uint16_t>& c, const TravArgs& a, uint16_t* ring, int qs, int* htp,
                             long long rowb, uint32_t base, const int32_t* __restrict__ rowptr,
                             const int32_t* __restrict__ colidx, int lane, unsigned long long& n_exp,
                             unsigned long long& n_edge, int* bad) {
  const unsigned lt = (1u << lane) - 1u;
  long long idle0 = -1;
  for (;;) {
    int h = 0, take = 0;
    if (lane == 0) {
      int hh = *(volatile int*)&htp[0];
      for (;;) {
        const int avail = *(volatile int*)&htp[1] - hh;
        take = avail < 32 ? avail : 32;
        if (take <= 0) break;
        const int prev = atomicCAS(&htp[0], hh, hh + take);
        if (prev == hh) break;
        hh = prev;
      }
      h = hh;
      if (take <= 0) {
        if (*(volatile int*)&htp[2] == 0) {
          take = -1;  // finished
        } else {
          if (idle0 < 0) idle0 = clock64();
          else if (wait_expired(idle0, a.ctr)) take = -1;
        }
      } else {
        idle0 = -1;
      }
    }
    take = __shfl_sync(FULL, take, 0);
    if (take < 0) break;
    if (take == 0) {
      __nanosleep(64);
      continue;
    }
    h = __shfl_sync(FULL, h, 0);
    int v = -1;
    uint32_t nmE = 0u;
    if (lane < take) {
      volatile uint16_t* sl = ring + ring_slot(h + lane, qs);
      uint16_t x;
      const long long t0 = clock64();
      while ((x = *sl) == RING_EMPTY)
        if (wait_expired(t0, a.ctr)) break;
      *sl = RING_EMPTY;
      v = x == RING_EMPTY ? -1 : (int)x;
      if (v >= 0) {
        atomicAnd(&c.Dn[v >> 5], ~(1u << (v & 31)));  // v leaves the queue before its label is read
        fence_sc_cta();
        const uint32_t lv = (uint32_t)((volatile uint16_t*)c.lab)[v];
        const uint32_t vE = base + 1u + (uint32_t)v;
        nmE = lv > vE ? lv : vE;
        n_exp++;
        if (a.collect_stats) n_edge += (unsigned long long)(__ldg(rowptr + v + 1) - __ldg(rowptr + v));
      }
    }
    bool fb = false;
    uint32_t h0 = 0u, h1 = 0u, h2 = 0u, h3 = 0u;
    if (v >= 0) {
      const int4 r4 = __ldg(a.ell + rowb + v);
      h0 = (uint32_t)r4.x; h1 = (uint32_t)r4.y; h2 = (uint32_t)r4.z; h3 = (uint32_t)r4.w;
      fb = (h0 & 0xFFFFu) == 0x8000u;
      if (fb) h0 = 0u;
    }
    int wv[8];
    wv[0] = v + (int)(short)(h0 & 0xFFFFu); wv[1] = v + (int)(short)(h0 >> 16);
    wv[2] = v + (int)(short)(h1 & 0xFFFFu); wv[3] = v + (int)(short)(h1 >> 16);
    wv[4] = v + (int)(short)(h2 & 0xFFFFu); wv[5] = v + (int)(short)(h2 >> 16);
    wv[6] = v + (int)(short)(h3 & 0xFFFFu); wv[7] = v + (int)(short)(h3 >> 16);
    unsigned em = 0u;
#pragma unroll
    for (int q = 0; q < 8; q++)
      if (wv[q] != v && relax_async(c, wv[q], nmE)) em |= 1u << q;
    ring_push8(ring, qs, htp, wv, em, lane, a.ctr);
    // rows without a record: the whole warp walks each from the CSR
    unsigned fm = __ballot_sync(FULL, fb);
    while (fm) {
      const int l = __ffs(fm) - 1;
      fm &= fm - 1u;
      const int u = __shfl_sync(FULL, v, l);
      const uint32_t unm = __shfl_sync(FULL, nmE, l);
      const int eb = __ldg(rowptr + u), ee = __ldg(rowptr + u + 1);
      for (int e0 = eb; e0 < ee; e0 += 32) {
        const int e = e0 + lane;
        int w[8] = {u, u, u, u, u, u, u, u};
        unsigned en = 0u;
        if (e < ee) {
          w[0] = __ldg(colidx + e);
          if ((unsigned)w[0] >= (unsigned)c.n) { *bad = 1; w[0] = u; }
          if (w[0] != u && relax_async(c, w[0], unm)) en = 1u;
        }
        ring_push8(ring, qs, htp, w, en, lane, a.ctr);
      }
    }
    __syncwarp();
    if (lane == 0) atomicSub(&htp[2], take);  // the taken entries are done (their pushes are in)
  }
}

// EB: edge-balanced expansion (the warp flattens the rows of its 32 frontier
// vertices so every lane works on an entry) instead of lock-step row slots.
// FF: the optional fill-first check of Section 4.
// ELL: read rows from the 16-bit offset records (CSR only for rows that do not fit).
template <typename LabT, bool EB, bool FF, bool ELL, bool UL, bool ASYNC>
__global__ void __launch_bounds__(1024, 1) trav_smem_kernel(TravArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n_max = a.n, S = a.S, CAP = a.list_cap;
  const int SW = (S + 31) >> 5, NWmax = (n_max + 31) >> 5;
  LabT* lab = (LabT*)smraw;
  uint32_t* D0 = (uint32_t*)(smraw + align16(sizeof(LabT) * (size_t)S));
  uint32_t* D1 = D0 + SW;
  uint32_t* ub = D1 + SW;
  LabT* L0 = (LabT*)(ub + NWmax);
  LabT* L1 = L0 + CAP;
  int32_t* S0 = a.spill + (size_t)blockIdx.x * 2 * (size_t)a.spill_cap;
  int32_t* S1 = S0 + a.spill_cap;

  __shared__ int s_src, s_diag, s_n;
  __shared__ const int32_t* s_rp;
  __shared__ const int32_t* s_ci;
  __shared__ long long s_rowb;
  __shared__ int s_mat;
  __shared__ int s_q[3];
  __shared__ int s_wcL[32], s_wcU[32];
  __shared__ long long s_off;
  __shared__ int s_nL;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarps = nthr >> 5;
  const unsigned lt = (1u << lane) - 1u;

  for (int i = tid; i < S; i += nthr) lab[i] = (LabT)LabOps<LabT>::MAXV;
  for (int i = tid; i < SW; i += nthr) { D0[i] = 0u; D1[i] = 0u; }
  for (int i = tid; i < NWmax; i += nthr) ub[i] = 0u;
  // asynchronous schedule: the two lists form one ring of 2 x CAP >= S entries
  const int QS = 2 * CAP;
  if (ASYNC)
    for (int i = tid; i < QS; i += nthr) L0[i] = (LabT)RING_EMPTY;

  // window base of the previous source; MAXV stands for the fill value
  uint32_t base = LabOps<LabT>::MAXV;
  unsigned long long n_exp = 0, n_edge = 0;
  int my_k = 0, my_left = 0;  // thread 0's current chunk of work items
  int bad = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      if (my_left == 0) {  // take the next chunk of work items
        const int chunk = a.chunk > 0 ? a.chunk : 1;
        my_k = atomicAdd(&a.ctr->work_smem, chunk);
        my_left = chunk;
      }
      const int k = my_k++;
      my_left--;
      int src = -1;
      if (k < a.nsrc && !input_error(a.ctr)) {
        if (a.mats) {
          // source index: smallest s with item_start[s] <= k (item_start decreases in s)
          int lo = 0, hi = n_max - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.item_start[mid] <= k) hi = mid; else lo = mid + 1;
          }
          src = lo;
          const int m = a.mat_order[k - a.item_start[lo]];
          const MatDesc d = a.mats[m];
          s_rp = d.rowptr;
          s_ci = d.colidx;
          s_n = d.n;
          s_rowb = d.row_base;
          s_mat = m;
        } else {
          src = a.order ? a.order[k] : a.nsrc - 1 - k;
          s_rp = a.rowptr;
          s_ci = a.colidx;
          s_n = a.n;
          s_rowb = 0;
          s_mat = 0;
        }
      }
      s_src = src;
      s_diag = 0;
      s_q[0] = s_q[1] = s_q[2] = 0;
    }
    __syncthreads();
    const int s = s_src;
    if (s < 0) break;
    const int n = s_n;
    const int NW = (n + 31) >> 5;
    const int32_t* __restrict__ rowptr = s_rp;
    const int32_t* __restrict__ colidx = s_ci;
    const long long rowb = s_rowb;

    // maxId window of this source: encoded values base+1+l for l in [-1, s),
    // strictly below every value an earlier source left behind
    const uint32_t span = (uint32_t)s + 1u;
    if (base >= span) {
      base -= span;
    } else {
      for (int i = tid; i < S; i += nthr) lab[i] = (LabT)LabOps<LabT>::MAXV;
      base = LabOps<LabT>::MAXV - span;
      __syncthreads();
    }

    // seed: neighbours of s; those below s form frontier 0 with maxId -1
    const int rb = __ldg(rowptr + s), re = __ldg(rowptr + s + 1);
    for (int e = rb + tid; e < re; e += nthr) {
      const int w = __ldg(colidx + e);
      if ((unsigned)w >= (unsigned)n) { bad = 1; continue; }
      if (w < s) {
        lab[w] = (LabT)base;  // encoded -1
        const uint32_t bit = 1u << (w & 31);
        if (!(atomicOr(&D0[w >> 5], bit) & bit)) {  // once per vertex: the list holds < s entries
          if (ASYNC) {  // queue it: s_q = {head, tail, pending}
            atomicAdd(&s_q[2], 1);
            L0[atomicAdd(&s_q[1], 1)] = (LabT)w;  // the ring is empty and deg(s) < QS
          } else {
            const int pos = atomicAdd(&s_q[0], 1);
            if (pos < CAP) L0[pos] = (LabT)w; else S0[pos - CAP] = w;
          }
        }
      } else if (w > s) {
        if (UL) lab[w] = (LabT)base;  // any value of the window marks a U entry
        else atomicOr(&ub[w >> 5], 1u << (w & 31));
      } else {
        s_diag = 1;
      }
    }
    __syncthreads();

    // After k levels every maxId is at most the best value over paths of <= k
    // hops (each changed vertex is expanded again); simple paths through
    // vertices below s have at most s hops, so level s+2 changes nothing.
    const int cap_lv = s + 3;
    int qc = ASYNC ? 0 : s_q[0];
    long long t_start = 0;
    if (a.collect_stats && tid == 0) t_start = clock64();
    int L = 1;
    if constexpr (ASYNC) {
      if constexpr (sizeof(LabT) == 2) {
        Src<uint16_t> c{lab, ub, D0, L0, S0, &s_q[1], base, s, n, CAP};
        async_source(c, a, (uint16_t*)L0, QS, s_q, rowb, base, rowptr, colidx, lane, n_exp, n_edge, &bad);
      }
      __syncthreads();
    }
    for (; qc > 0; L++) {
      const int cb = (L - 1) & 1, nb = L & 1;
      LabT* Lc = cb ? L1 : L0;
      int32_t* Sc = cb ? S1 : S0;
      uint32_t* Dc = cb ? D1 : D0;
      Src<LabT> c{lab, ub, nb ? D1 : D0, nb ? L1 : L0, nb ? S1 : S0, &s_q[L % 3], base, s, n, CAP};
      if (tid == 0) s_q[(L + 1) % 3] = 0;
      // small frontier: several lanes per vertex (one round per warp)
      const int lpv = !ELL ? 1 : qc * 8 <= nthr ? 8 : qc * 4 <= nthr ? 4 : qc * 2 <= nthr ? 2 : 1;
      if (ELL && lpv == 8)
        small_level<LabT, FF, UL, 8>(c, a, Lc, Sc, Dc, qc, CAP, rowb, base, rowptr, colidx, warp, nwarps, lane, n_exp,
                                     n_edge, &bad);
      else if (ELL && lpv == 4)
        small_level<LabT, FF, UL, 4>(c, a, Lc, Sc, Dc, qc, CAP, rowb, base, rowptr, colidx, warp, nwarps, lane, n_exp,
                                     n_edge, &bad);
      else if (ELL && lpv == 2)
        small_level<LabT, FF, UL, 2>(c, a, Lc, Sc, Dc, qc, CAP, rowb, base, rowptr, colidx, warp, nwarps, lane, n_exp,
                                     n_edge, &bad);
      for (int r0 = warp * 32; lpv == 1 && r0 < qc; r0 += nthr) {
        const int r = r0 + lane;
        int v = -1, eb = 0, ee = 0;
        uint32_t nmE = 0u;
        if (r < qc) {
          v = r < CAP ? (int)Lc[r] : Sc[r - CAP];
          // v leaves the current list.  Nothing sets bits of Dc during this level
          // and every vertex with a bit in Dc is dequeued in it, so the word can
          // simply be zeroed.
          Dc[v >> 5] = 0u;
          if (!ELL || a.collect_stats) {
            eb = __ldg(rowptr + v);
            ee = __ldg(rowptr + v + 1);
          }
          const uint32_t lv = (uint32_t)lab[v];
          const uint32_t vE = base + 1u + (uint32_t)v;
          nmE = lv > vE ? lv : vE;  // encoded max(maxId(v), v)
          n_exp++;
          n_edge += (unsigned long long)(ee - eb);
        }
        if (EB && !ELL) {
          // flattened entries of the warp's rows; entry e belongs to the lane
          // whose inclusive degree sum first exceeds e
          const int deg = v >= 0 ? ee - eb : 0;
          const int incl = warp_incl_scan(deg, lane);
          const int total = __shfl_sync(FULL, incl, 31);
          for (int c0 = 0; c0 < total; c0 += 32 * EB_UNROLL) {
            int wv[EB_UNROLL], ov[EB_UNROLL];
            uint32_t onm[EB_UNROLL];
#pragma unroll
            for (int u = 0; u < EB_UNROLL; u++) {
              const int e = c0 + 32 * u + lane;
              int o = 0;
#pragma unroll
              for (int b = 16; b >= 1; b >>= 1) {
                const int t = __shfl_sync(FULL, incl, o + b - 1);
                if (t <= e) o += b;
              }
              const int oc = o < 31 ? o : 31;
              const int o_excl = __shfl_sync(FULL, incl - deg, oc);
              const int o_eb = __shfl_sync(FULL, eb, oc);
              ov[u] = __shfl_sync(FULL, v, oc);
              onm[u] = __shfl_sync(FULL, nmE, oc);
              wv[u] = e < total ? __ldg(colidx + o_eb + (e - o_excl)) : ov[u];
            }
            unsigned em = 0u;
#pragma unroll
            for (int u = 0; u < EB_UNROLL; u++)
              if (wv[u] != ov[u] && relax<LabT, FF, UL>(c, wv[u], onm[u], &bad)) em |= 1u << u;  // diagonal skipped
            const int cnt = __popc(em);
            const int inc2 = warp_incl_scan(cnt, lane);
            const int tot = __shfl_sync(FULL, inc2, 31);
            if (tot) {
              int basep = 0;
              if (lane == 31) basep = atomicAdd(c.qn, tot);
              basep = __shfl_sync(FULL, basep, 31);
              int pos = basep + inc2 - cnt;
#pragma unroll
              for (int u = 0; u < EB_UNROLL; u++) {
                if ((em >> u) & 1u) {
                  if (pos < CAP) c.Ln[pos] = (LabT)wv[u]; else c.Sn[pos - CAP] = wv[u];
                  pos++;
                }
              }
            }
          }
          continue;
        }
        if (ELL) {
          // one 16-byte record per row: up to 8 offsets w - v (0 = empty)
          bool fb = false;
          int wv[8];
          if (v >= 0) {
            const int4 r4 = __ldg(a.ell + rowb + v);
            const uint32_t h[4] = {(uint32_t)r4.x, (uint32_t)r4.y, (uint32_t)r4.z, (uint32_t)r4.w};
            fb = (h[0] & 0xFFFFu) == 0x8000u;
#pragma unroll
            for (int q = 0; q < 4; q++) {
              wv[2 * q] = v + (int)(short)(h[q] & 0xFFFFu);
              wv[2 * q + 1] = v + (int)(short)(h[q] >> 16);
            }
            if (fb) {
#pragma unroll
              for (int q = 0; q < 8; q++) wv[q] = v;
            }
          } else {
#pragma unroll
            for (int q = 0; q < 8; q++) wv[q] = v;
          }
          unsigned em = 0u;
#pragma unroll
          for (int q = 0; q < 8; q++)
            if (wv[q] != v && relax_rec<LabT, FF, UL>(c, wv[q], nmE)) em |= 1u << q;
          const int cnt = __popc(em);
          const int incl = warp_incl_scan(cnt, lane);
          const int tot = __shfl_sync(FULL, incl, 31);
          if (tot) {
            int basep = 0;
            if (lane == 31) basep = atomicAdd(c.qn, tot);
            basep = __shfl_sync(FULL, basep, 31);
            int pos = basep + incl - cnt;
#pragma unroll
            for (int q = 0; q < 8; q++) {
              if ((em >> q) & 1u) {
                if (pos < CAP) c.Ln[pos] = (LabT)wv[q]; else c.Sn[pos - CAP] = wv[q];
                pos++;
              }
            }
          }
          if (!__any_sync(FULL, fb)) continue;
          if (!fb) v = -1;  // rows that did not fit the record continue below from the CSR
          if (v >= 0) {
            eb = __ldg(rowptr + v);
            ee = __ldg(rowptr + v + 1);
          }
        }
        const int deg = (v >= 0 && ee - eb <= BIG_DEG) ? ee - eb : 0;
        const int maxdeg = __reduce_max_sync(FULL, deg);
        for (int k0 = 0; k0 < maxdeg; k0 += BATCH) {
          int wv[BATCH];  // independent loads first, then the relaxations
#pragma unroll
          for (int q = 0; q < BATCH; q++) wv[q] = (k0 + q < deg) ? __ldg(colidx + eb + k0 + q) : v;
          unsigned em = 0u;  // slots whose vertex joins the next frontier
#pragma unroll
          for (int q = 0; q < BATCH; q++)
            if (wv[q] != v && relax<LabT, FF, UL>(c, wv[q], nmE, &bad)) em |= 1u << q;  // the diagonal entry is skipped
          // one shared atomic per warp for the whole batch
          const int cnt = __popc(em);
          const int incl = warp_incl_scan(cnt, lane);
          const int tot = __shfl_sync(FULL, incl, 31);
          if (tot) {
            int basep = 0;
            if (lane == 31) basep = atomicAdd(c.qn, tot);
            basep = __shfl_sync(FULL, basep, 31);
            int pos = basep + incl - cnt;
#pragma unroll
            for (int q = 0; q < BATCH; q++) {
              if ((em >> q) & 1u) {
                if (pos < CAP) c.Ln[pos] = (LabT)wv[q]; else c.Sn[pos - CAP] = wv[q];
                pos++;
              }
            }
          }
        }
        unsigned bigm = __ballot_sync(FULL, v >= 0 && (ee - eb) > BIG_DEG);
        while (bigm) {  // long rows: the whole warp walks one row
          const int l = __ffs(bigm) - 1;
          bigm &= bigm - 1;
          const int beb = __shfl_sync(FULL, eb, l), bee = __shfl_sync(FULL, ee, l);
          const uint32_t bnm = __shfl_sync(FULL, nmE, l);
          const int bv = __shfl_sync(FULL, v, l);
          for (int e0 = beb; e0 < bee; e0 += 32) {
            const int e = e0 + lane;
            const int w = e < bee ? __ldg(colidx + e) : bv;
            const int enq = w != bv ? relax<LabT, FF, UL>(c, w, bnm, &bad) : 0;
            append(c, enq, w, lane);
          }
        }
      }
      __syncthreads();
      qc = s_q[L % 3];
      if (qc > 0 && L >= cap_lv) {
        // never expected: drop the frontier (clearing its dedup bits) and flag it
        LabT* Ln = nb ? L1 : L0;
        int32_t* Sn = nb ? S1 : S0;
        uint32_t* Dn = nb ? D1 : D0;
        for (int r = tid; r < qc; r += nthr) {
          const int v = r < CAP ? (int)Ln[r] : Sn[r - CAP];
          atomicAnd(&Dn[v >> 5], ~(1u << (v & 31)));
        }
        if (tid == 0) atomicOr(&a.ctr->err, ERR_NOCONV);
        __syncthreads();
        break;
      }
    }

    long long t_mid = 0;
    // levels and expansions are always counted (the library uses their ratio,
    // the mean frontier size, to pick the frontier order of later calls)
    if (tid == 0) atomicAdd(&a.ctr->levels, (unsigned long long)(L - 1));
    if (a.collect_stats && tid == 0) {
      t_mid = clock64();
      atomicAdd(&a.ctr->cyc_trav, (unsigned long long)(t_mid - t_start));
    }
    // ---- emission: counts, pool offset, sorted row
    // (16-bit labels with U by labels: 8 labels per lane, see label_mask8)
    constexpr bool VEC = UL && sizeof(LabT) == 2;
    const int perL = (((s + nwarps - 1) / nwarps) + 31) & ~31;
    const int loL = warp * perL, hiL = min(s, loL + perL);
    const uint32_t top = base + (uint32_t)s;  // largest value of this window
    int cL = 0;
    if constexpr (VEC) {
      for (int i0 = loL; i0 < hiL; i0 += 256)
        cL += __popc(label_mask8<false>((const uint16_t*)lab, i0 + 8 * lane, -1, hiL, base, top));
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) cL += __shfl_xor_sync(FULL, cL, o);
    } else {
      for (int i0 = loL; i0 < hiL; i0 += 32) {
        const int i = i0 + lane;
        const bool f = i < hiL && (uint32_t)lab[i] < base + 1u + (uint32_t)i;
        cL += __popc(__ballot_sync(FULL, f));
      }
    }
    // U part: labelled vertices above s (UL), else words of the ub bitmap
    const int ws = (s + 1) >> 5;  // first word that can hold a column > s
    const int us = (s + 1) & ~7;  // vector scan: first aligned label block that can hold a column > s
    const int nUW = VEC ? n - us : UL ? n - (s + 1) : NW - ws;
    const int perU = VEC ? (((nUW + nwarps - 1) / nwarps) + 7) & ~7 : (((nUW + nwarps - 1) / nwarps) + 31) & ~31;
    const int loU = (VEC ? us : UL ? s + 1 : ws) + warp * perU, hiU = min(UL ? n : NW, loU + perU);
    int cU = 0;
    if constexpr (VEC) {
      for (int i0 = loU; i0 < hiU; i0 += 256)
        cU += __popc(label_mask8<true>((const uint16_t*)lab, i0 + 8 * lane, s, hiU, base, top));
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) cU += __shfl_xor_sync(FULL, cU, o);
    } else if (UL) {
      for (int i0 = loU; i0 < hiU; i0 += 32) {
        const int i = i0 + lane;
        cU += __popc(__ballot_sync(FULL, i < hiU && (uint32_t)lab[i] <= top));
      }
    } else {
      for (int j = loU + lane; j < hiU; j += 32) cU += __popc(ub[j]);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) cU += __shfl_xor_sync(FULL, cU, o);
    }
    if (lane == 0) { s_wcL[warp] = cL; s_wcU[warp] = cU; }
    __syncthreads();
    if (tid == 0) {
      int tl = 0, tu = 0;
      for (int w = 0; w < nwarps; w++) {
        const int x = s_wcL[w]; s_wcL[w] = tl; tl += x;
        const int y = s_wcU[w]; s_wcU[w] = tu; tu += y;
      }
      const int nL = tl, nU = tu + 1;
      bool ok = false;
      unsigned long long off = 0ull;
      if (!a.counts_only) {
        off = atomicAdd(&a.ctr->pool_cursor, (unsigned long long)(nL + nU));
        ok = off + (unsigned long long)(nL + nU) <= (unsigned long long)a.pool_cap;
        a.row_off[rowb + s] = ok ? (int64_t)off : -1;
        if (ok) a.pool[off + nL] = (uint32_t)s;
        else atomicOr(&a.ctr->err, ERR_OVERFLOW);
      }
      s_off = ok ? (long long)off : -1LL;
      s_nL = nL;
      a.row_nL[rowb + s] = nL;
      a.row_nU[rowb + s] = nU;
      a.fill_count[rowb + s] = nL + nU - ((re - rb) + (s_diag ? 0 : 1));
      atomicAdd(&a.ctr->total_L, (unsigned long long)nL);
      atomicAdd(&a.ctr->total_U, (unsigned long long)nU);
      if (a.mat_tot) {
        atomicAdd(&a.mat_tot[2 * s_mat], (unsigned long long)nL);
        atomicAdd(&a.mat_tot[2 * s_mat + 1], (unsigned long long)nU);
      }
    }
    __syncthreads();
    const long long off = s_off;
    const int nL = s_nL;
    if (VEC && off >= 0) {
      // 8 labels per lane; lanes hold consecutive blocks, so a warp scan of the
      // per-lane counts keeps the row sorted
      int pos = s_wcL[warp];
      for (int i0 = loL; i0 < hiL; i0 += 256) {
        const int i = i0 + 8 * lane;
        unsigned m = label_mask8<false>((const uint16_t*)lab, i, -1, hiL, base, top);
        const int c = __popc(m);
        const int inc = warp_incl_scan(c, lane);
        long long p = off + pos + (inc - c);
        while (m) {
          const int q = __ffs(m) - 1;
          m &= m - 1u;
          a.pool[p++] = (uint32_t)(i + q);
        }
        pos += __shfl_sync(FULL, inc, 31);
      }
      pos = s_wcU[warp];
      for (int i0 = loU; i0 < hiU; i0 += 256) {
        const int i = i0 + 8 * lane;
        unsigned m = label_mask8<true>((const uint16_t*)lab, i, s, hiU, base, top);
        const int c = __popc(m);
        const int inc = warp_incl_scan(c, lane);
        long long p = off + nL + 1 + pos + (inc - c);
        while (m) {
          const int q = __ffs(m) - 1;
          m &= m - 1u;
          a.pool[p++] = (uint32_t)(i + q);
        }
        pos += __shfl_sync(FULL, inc, 31);
      }
    } else if (!VEC && off >= 0) {
      int pos = s_wcL[warp];
      for (int i0 = loL; i0 < hiL; i0 += 32) {
        const int i = i0 + lane;
        const bool f = i < hiL && (uint32_t)lab[i] < base + 1u + (uint32_t)i;
        const unsigned m = __ballot_sync(FULL, f);
        if (f) a.pool[off + pos + __popc(m & lt)] = (uint32_t)i;
        pos += __popc(m);
      }
    }
    if (VEC) {
      // written above
    } else if (UL) {
      if (off >= 0) {
        int pos = s_wcU[warp];
        for (int i0 = loU; i0 < hiU; i0 += 32) {
          const int i = i0 + lane;
          const bool f = i < hiU && (uint32_t)lab[i] <= top;
          const unsigned m = __ballot_sync(FULL, f);
          if (f) a.pool[off + nL + 1 + pos + __popc(m & lt)] = (uint32_t)i;
          pos += __popc(m);
        }
      }
    } else {
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
    if (a.collect_stats && tid == 0) atomicAdd(&a.ctr->cyc_emit, (unsigned long long)(clock64() - t_mid));
  }

  if (bad) atomicOr(&a.ctr->err, ERR_COL_RANGE);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    n_exp += __shfl_xor_sync(FULL, n_exp, o);
    n_edge += __shfl_xor_sync(FULL, n_edge, o);
  }
  if (lane == 0) {
    atomicAdd(&a.ctr->expansions, n_exp);
    if (a.collect_stats) atomicAdd(&a.ctr->edges, n_edge);
  }
}

template <typename LabT>
static int32_t max_S_t(int32_t n, size_t limit, int32_t min_cap) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {  // largest S whose layout (with a list of min_cap entries) fits
    const int32_t mid = (int32_t)(((int64_t)lo + hi + 1) / 2);
    const int32_t cap = mid < min_cap ? mid : min_cap;
    if (trav_smem_bytes_t<LabT>(n, mid, cap) <= limit) lo = mid; else hi = mid - 1;
  }
  return lo;
}

int32_t trav_smem_max_S(int32_t n, size_t smem_limit, int label16) {
  return label16 ? max_S_t<uint16_t>(n, smem_limit, 1024) : max_S_t<uint32_t>(n, smem_limit, 1024);
}

template <typename LabT, bool EB, bool FF, bool ELL, bool UL, bool ASYNC = false>
static cudaError_t launch_t(const TravArgs& a, int grid, int block, size_t bytes, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(trav_smem_kernel<LabT, EB, FF, ELL, UL, ASYNC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  trav_smem_kernel<LabT, EB, FF, ELL, UL, ASYNC><<<grid, block, bytes, st>>>(a);
  return cudaGetLastError();
}

template <typename LabT>
static cudaError_t launch_l(const TravArgs& a, int grid, int block, size_t bytes, cudaStream_t st) {
  const bool ff = a.fill_first != 0;
  if (a.ell) {
    // U entries by labels when every vertex has a label slot
    if (a.S >= a.n) {
      if constexpr (sizeof(LabT) == 2) {
        // asynchronous schedule (the ring of 2 x list_cap entries must hold S)
        if (a.async_sched && !ff && 2 * a.list_cap >= a.S && 2 * a.list_cap >= 64)
          return launch_t<LabT, false, false, true, true, true>(a, grid, block, bytes, st);
      }
      return ff ? launch_t<LabT, false, true, true, true>(a, grid, block, bytes, st)
                : launch_t<LabT, false, false, true, true>(a, grid, block, bytes, st);
    }
    return ff ? launch_t<LabT, false, true, true, false>(a, grid, block, bytes, st)
              : launch_t<LabT, false, false, true, false>(a, grid, block, bytes, st);
  }
  if (a.expand_mode == 2) return ff ? launch_t<LabT, true, true, false, false>(a, grid, block, bytes, st)
                                    : launch_t<LabT, true, false, false, false>(a, grid, block, bytes, st);
  return ff ? launch_t<LabT, false, true, false, false>(a, grid, block, bytes, st)
            : launch_t<LabT, false, false, false, false>(a, grid, block, bytes, st);
}

cudaError_t launch_trav_smem(const TravArgs& a, int grid, int block, int label16, cudaStream_t st) {
  const size_t bytes = trav_smem_bytes(a.n, a.S, a.list_cap, label16);
  return label16 ? launch_l<uint16_t>(a, grid, block, bytes, st) : launch_l<uint32_t>(a, grid, block, bytes, st);
}

int trav_smem_static_bytes() {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, trav_smem_kernel<uint32_t, false, false, false, false, false>) != cudaSuccess) {
    cudaGetLastError();
    return 1024;
  }
  return (int)fa.sharedSizeBytes;
}

int trav_smem_occupancy(int block, size_t dyn_bytes, int label16) {
  const void* f = label16 ? (const void*)trav_smem_kernel<uint16_t, false, false, true, true, false>
                          : (const void*)trav_smem_kernel<uint32_t, false, false, true, true, false>;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, block, dyn_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace gsofa
