// Multi-source maxId traversal in maxId-class order with a visited bitmap
// (Section 4, Fig. 5; class order as in the comparison with Dijkstra's
// algorithm in Section 8).
//
// For source row s, maxId(w) is the smallest largest-intermediate over the
// paths s -> w through vertices below s (Theorem 1).  A frontier vertex f
// proposes max(maxId(f), f) to its neighbours.  Expanding the frontier by
// increasing proposal, one class of equal proposals at a time, sets every
// maxId exactly once, when its vertex is first reached:
//   * the direct neighbours w < s of s (maxId -1) and every vertex w > t first
//     reached from class t are fills of L(s,:); a fill w opens its own class w
//     (its proposal is w itself);
//   * class t is the fill t together with the vertices below t that it reaches
//     through unreached vertices below t (they all get maxId t > w, so they
//     are not fills and propose t again);
//   * every reached w > s is an entry of U(s,:).
// So the only state a source needs is the set V of reached vertices: when the
// classes are taken in increasing order with a cursor just above the last
// class, the pending classes are exactly V ∩ [cursor, s), members of class t
// are the first-reached vertices below t, and U(s,:) is V ∩ (s, n).  The
// relaxation of an edge is one atomic OR of the neighbour's bit; the returned
// word says whether this edge reached it first.
//
// Teams.  A team owns one source at a time: a warp, or for the first `nbig`
// sources of the issue order (the largest ones) the whole CTA of four warps,
// whose levels of a class are split over 128 threads with one barrier per
// level.  Persistent CTAs take team sources from one counter until they run
// out, then each warp takes single sources from another.
//
// Storage.  V is n bits per team: in shared memory (SV) when that leaves
// enough CTAs per SM, else in a global-memory slot per warp with a summary
// bitmap (one bit per nonzero V word) that bounds the searches and the
// clearing.  Frontier levels live in shared-memory queues of `qw` entries per
// warp; longer levels overflow into the slot's log array from its bottom, each
// level after the previous one of the same class, while the L row grows down
// from its top one class at a time (sorted by construction).  A vertex below s
// is a class member or a fill, never both, and joins at most one level, so the
// two ends never meet in s entries.  Each source clears the bits it set.
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace gsofa {

namespace {

constexpr int CT_WARPS = 4;  // warps per CTA (one team in team mode)
constexpr int CT_THREADS = 32 * CT_WARPS;

// Per-team control block in shared memory.
struct CtCtl {
  int src;        // team mode: the current source (-1: no more team sources)
  int mi;         // its matrix (batch mode)
  int t;          // the class being expanded (-1: no pending class)
  int qcnt[3];    // rotating level lengths
  int smin, smax; // summary words touched (global V)
};

// ---- bit operations on V, in shared (SV) or global memory
// Atomic OR issued under a predicate; returns `bit` (= already set) when not issued.
template <bool SV>
__device__ __forceinline__ uint32_t v_or_if(uint32_t* V, int word, uint32_t bit, bool pred) {
  uint32_t r = bit;
  if constexpr (SV) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(V + word);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.shared.or.b32 %0, [%1], %2;\n\t}"
                 : "+r"(r)
                 : "r"(a), "r"(bit), "r"((uint32_t)pred)
                 : "memory");
  } else {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.global.or.b32 %0, [%1], %2;\n\t}"
                 : "+r"(r)
                 : "l"(V + word), "r"(bit), "r"((uint32_t)pred)
                 : "memory");
  }
  return r;
}

__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <bool SV>
__device__ __forceinline__ uint32_t v_load(const uint32_t* V, int word) {
  if constexpr (SV) return V[word];
  else return *(const volatile uint32_t*)(V + word);
}

// Set bit w of V (one lane).  Returns true when this call set it.  Global V:
// a word that was empty gets its summary bit and widens [smin, smax].
template <bool SV>
__device__ __forceinline__ bool v_set(uint32_t* V, uint32_t* VS, int w, int& smin, int& smax) {
  const uint32_t bit = 1u << (w & 31);
  const uint32_t old = v_or_if<SV>(V, w >> 5, bit, true);
  if (old & bit) return false;
  if constexpr (!SV) {
    if (old == 0u) {
      red_or(VS + (w >> 10), 1u << ((w >> 5) & 31));
      smin = min(smin, w >> 10);
      smax = max(smax, w >> 10);
    }
  }
  return true;
}

// The team's view of one source: where V, the queues and the list live.
struct Team {
  uint32_t* V;        // n bits
  uint32_t* VS;       // summary (global V only)
  int32_t* qa;        // shared queue, even levels
  int32_t* qb;        // shared queue, odd levels
  int qcap;           // shared queue capacity (entries per level)
  int32_t* log;       // level overflow from the bottom, L(s,:) from the top
  int64_t cap;        // entries of log (>= n)
};

// Entry idx of the level with parity `level` whose overflow starts at log[base].
__device__ __forceinline__ int32_t* q_slot(const Team& tm, int level, int64_t base, int idx) {
  if (idx < tm.qcap) return ((level & 1) ? tm.qb : tm.qa) + idx;
  return tm.log + base + (idx - tm.qcap);
}

// k-th entry of L(s,:) (top of the log, growing down).
__device__ __forceinline__ int32_t* l_slot(const Team& tm, int k) { return tm.log + (tm.cap - 1 - k); }

// Log position of the level after one of length qlen that starts at base.
__device__ __forceinline__ int64_t next_base(const Team& tm, int64_t base, int qlen) {
  return base + (qlen > tm.qcap ? qlen - tm.qcap : 0);
}

// Smallest vertex of V in [from, s), or -1: the next pending class.
// Warp-wide; every lane returns the same value.
template <bool SV>
__device__ int next_class(const Team& tm, int from, int s, int lane) {
  if (from >= s) return -1;
  const int wfirst = from >> 5;
  const int wend = (s + 31) >> 5;  // words holding positions below s
  if constexpr (SV) {
    for (int w0 = wfirst; w0 < wend; w0 += 32) {
      const int j = w0 + lane;
      uint32_t m = 0u;
      if (j < wend) {
        m = v_load<SV>(tm.V, j);
        if (j == wfirst) m &= 0xFFFFFFFFu << (from & 31);
        const int hi = s - (j << 5);
        if (hi < 32) m &= (1u << hi) - 1u;
      }
      const unsigned b = __ballot_sync(FULL, m != 0u);
      if (b) {
        const int l = __ffs(b) - 1;
        m = __shfl_sync(FULL, m, l);
        return ((w0 + l) << 5) + __ffs(m) - 1;
      }
    }
    return -1;
  } else {
    // the cursor's own word first
    uint32_t m = v_load<SV>(tm.V, wfirst) & (0xFFFFFFFFu << (from & 31));
    if (m) {
      const int v = (wfirst << 5) + __ffs(m) - 1;
      return v < s ? v : -1;
    }
    // then the summary from the next word on
    const int wstart = wfirst + 1;
    if (wstart >= wend) return -1;
    const int send = (wend + 31) >> 5;
    for (int sw0 = wstart >> 5; sw0 < send; sw0 += 32) {
      const int sw = sw0 + lane;
      uint32_t sm = 0u;
      if (sw < send) {
        sm = v_load<SV>(tm.VS, sw);
        if (sw == (wstart >> 5)) sm &= 0xFFFFFFFFu << (wstart & 31);
      }
      const unsigned b = __ballot_sync(FULL, sm != 0u);
      if (b) {
        const int l = __ffs(b) - 1;
        sm = __shfl_sync(FULL, sm, l);
        const int pw = ((sw0 + l) << 5) + __ffs(sm) - 1;  // first nonzero V word at or after wstart
        const uint32_t word = v_load<SV>(tm.V, pw);
        const int v = (pw << 5) + __ffs(word) - 1;
        return (word != 0u && v < s) ? v : -1;
      }
    }
    return -1;
  }
}

// Relax the 8 record slots of vertex v for class t of source s.  The OR
// operations are issued together (predicated), then the first-reached
// vertices below t are returned as a slot mask (members of class t).
template <bool SV>
__device__ __forceinline__ unsigned relax8(const Team& tm, const int (&wv)[8], int v, int s, int t, int& smin,
                                           int& smax) {
  uint32_t old[8];
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int w = wv[q];
    old[q] = v_or_if<SV>(tm.V, (w < 0 ? 0 : w) >> 5, 1u << (w & 31), w != v && w != s);
  }
  unsigned em = 0u;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int w = wv[q];
    const uint32_t bit = 1u << (w & 31);
    if (!(old[q] & bit)) {  // first reach (not issued: old == bit)
      if constexpr (!SV) {
        if (old[q] == 0u) {
          red_or(tm.VS + (w >> 10), 1u << ((w >> 5) & 31));
          smin = min(smin, w >> 10);
          smax = max(smax, w >> 10);
        }
      }
      if (w < t) em |= 1u << q;
    }
  }
  return em;
}

// Decode an ELL record of v into its neighbours (empty slots hold v itself).
__device__ __forceinline__ void decode(const int4 r4, int v, int (&wv)[8], bool& fallback) {
  uint32_t h0 = (uint32_t)r4.x;
  fallback = (h0 & 0xFFFFu) == 0x8000u;
  if (fallback) h0 = 0u;
  const uint32_t h1 = (uint32_t)r4.y, h2 = (uint32_t)r4.z, h3 = (uint32_t)r4.w;
  wv[0] = v + (int)(short)(h0 & 0xFFFFu); wv[1] = v + (int)(short)(h0 >> 16);
  wv[2] = v + (int)(short)(h1 & 0xFFFFu); wv[3] = v + (int)(short)(h1 >> 16);
  wv[4] = v + (int)(short)(h2 & 0xFFFFu); wv[5] = v + (int)(short)(h2 >> 16);
  wv[6] = v + (int)(short)(h3 & 0xFFFFu); wv[7] = v + (int)(short)(h3 >> 16);
}

// Source-independent inputs of one source.
struct Src {
  int s;
  int n;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colidx;
  const int4* __restrict__ ell;  // records of this matrix (row v at ell[v]) or null
  long long rowb;                // row offset in the per-row arrays (batch)
  int mi;
};

}  // namespace

namespace {

// Walk row u from the CSR (rows without an ELL record, or no records at all):
// the warp takes 32 entries at a time; first-reached vertices below t join the
// next level.  Columns are range-checked here.
template <bool SV, bool TEAM>
__device__ void walk_row(const Src& sc, const Team& tm, CtCtl* ctl, int u, int t, int level, int64_t nb, int& nq,
                         int& smin, int& smax, int& bad) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int eb = __ldg(sc.rowptr + u), ee = __ldg(sc.rowptr + u + 1);
  for (int e0 = eb; e0 < ee; e0 += 32) {
    const int e = e0 + lane;
    int w = -1;
    bool enq = false;
    if (e < ee) {
      w = __ldg(sc.colidx + e);
      if ((unsigned)w >= (unsigned)sc.n) {
        bad = 1;
      } else if (w != u && w != sc.s) {
        enq = v_set<SV>(tm.V, tm.VS, w, smin, smax) && w < t;
      }
    }
    const unsigned m = __ballot_sync(FULL, enq);
    if (!m) continue;
    int base;
    if constexpr (TEAM) {
      if (lane == 0) base = atomicAdd(&ctl->qcnt[(level + 1) % 3], __popc(m));
      base = __shfl_sync(FULL, base, 0);
    } else {
      base = nq;
      nq += __popc(m);
    }
    if (enq) *q_slot(tm, level + 1, nb, base + __popc(m & lt)) = w;
  }
}

// Expand one level of class t: the calling warp (TEAM false) or the whole CTA
// (TEAM true) takes the level's vertices, relaxes their neighbours and appends
// the first-reached vertices below t to the next level.  head: the class's
// first level, t alone (qlen 1).  `level` indexes the queues and counters.
// Warp mode returns the next level's length in nq; team mode counts it in
// ctl->qcnt[(level + 1) % 3].
template <bool SV, bool TEAM>
__device__ void expand_level(const TravArgs& a, const Src& sc, const Team& tm, CtCtl* ctl, int t, int level,
                             int64_t cb, int64_t nb, bool head, int qlen, int& nq, int& smin, int& smax,
                             unsigned long long& n_exp, unsigned long long& n_edge, int& bad) {
  const int lane = threadIdx.x & 31;
  const int nthr = TEAM ? CT_THREADS : 32;
  const int tid = TEAM ? (int)threadIdx.x : lane;
  for (int i0 = 0; i0 < qlen; i0 += nthr) {
    const int i = i0 + tid;
    int v = -1;
    if (i < qlen) v = head ? t : *q_slot(tm, level, cb, i);
    int wv[8];
    bool fb = false;
    unsigned em = 0u;
    if (v >= 0) {
      if (sc.ell) {
        decode(__ldg(sc.ell + v), v, wv, fb);
        if (!fb) em = relax8<SV>(tm, wv, v, sc.s, t, smin, smax);
      } else {
        fb = true;
      }
      if (a.collect_stats) {
        n_exp++;
        n_edge += (unsigned long long)(__ldg(sc.rowptr + v + 1) - __ldg(sc.rowptr + v));
      }
    }
    // append the members found through records
    const int cnt = __popc(em);
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += x;
    }
    const int tot = __shfl_sync(FULL, inc, 31);
    if (tot) {
      int base;
      if constexpr (TEAM) {
        if (lane == 0) base = atomicAdd(&ctl->qcnt[(level + 1) % 3], tot);
        base = __shfl_sync(FULL, base, 0);
      } else {
        base = nq;
        nq += tot;
      }
      int pos = base + inc - cnt;
#pragma unroll
      for (int q = 0; q < 8; q++)
        if ((em >> q) & 1u) *q_slot(tm, level + 1, nb, pos++) = wv[q];
    }
    // rows read from the CSR
    unsigned fm = __ballot_sync(FULL, fb);
    while (fm) {
      const int l = __ffs(fm) - 1;
      fm &= fm - 1;
      walk_row<SV, TEAM>(sc, tm, ctl, __shfl_sync(FULL, v, l), t, level, nb, nq, smin, smax, bad);
    }
  }
}

// Relax slots [Q0, Q0 + G) of the lane's K-slot group (their OR operations
// issued together); first-reached vertices below t set their bit in em.
template <bool SV, int K, int Q0, int G>
__device__ __forceinline__ void relax_group(const Team& tm, const int (&wv)[K], int v, int s, int t, unsigned& em,
                                            int& smin, int& smax) {
  uint32_t old[G];
#pragma unroll
  for (int q = 0; q < G; q++) {
    const int w = wv[Q0 + q];
    old[q] = v_or_if<SV>(tm.V, w >> 5, 1u << (w & 31), w != v && w != s);
  }
#pragma unroll
  for (int q = 0; q < G; q++) {
    const int w = wv[Q0 + q];
    if (!(old[q] & (1u << (w & 31)))) {  // first reach (an OR not issued returns the bit)
      if constexpr (!SV) {
        if (old[q] == 0u) {
          red_or(tm.VS + (w >> 10), 1u << ((w >> 5) & 31));
          smin = min(smin, w >> 10);
          smax = max(smax, w >> 10);
        }
      }
      if (w < t) em |= 1u << (Q0 + q);
    }
  }
}

// Warp mode: one level with LPV lanes per vertex, each lane relaxing K = 8/LPV
// consecutive record slots of its vertex (small levels keep most lanes busy:
// a class head alone takes one round of 8 lanes instead of one lane doing 8
// slots).  Appends members to the next level (length in nq).
template <bool SV, int LPV>
__device__ void expand_level_warp(const TravArgs& a, const Src& sc, const Team& tm, int t, int level, int64_t cb,
                                  int64_t nb, bool head, int qlen, int& nq, int& smin, int& smax,
                                  unsigned long long& n_exp, unsigned long long& n_edge, int& bad) {
  constexpr int K = 8 / LPV;
  constexpr int PER = 32 / LPV;  // vertices per round
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int sub = lane % LPV;    // which K slots of the vertex
  const int vi = lane / LPV;
  for (int i0 = 0; i0 < qlen; i0 += PER) {
    const int i = i0 + vi;
    int v = -1;
    if (i < qlen) v = head ? t : *q_slot(tm, level, cb, i);
    int wv[K];
    bool fb = false;
    unsigned em = 0u;
    uint32_t h[(K + 1) / 2];
#pragma unroll
    for (int q = 0; q < (K + 1) / 2; q++) h[q] = 0u;
    if (v >= 0) {
      if (sc.ell) {
        if constexpr (K == 8) {
          const int4 r = __ldg(sc.ell + v);
          h[0] = (uint32_t)r.x; h[1] = (uint32_t)r.y; h[2] = (uint32_t)r.z; h[3] = (uint32_t)r.w;
        } else if constexpr (K == 4) {
          const int2 r = __ldg((const int2*)(sc.ell + v) + sub);
          h[0] = (uint32_t)r.x; h[1] = (uint32_t)r.y;
        } else if constexpr (K == 2) {
          h[0] = (uint32_t)__ldg((const int*)(sc.ell + v) + sub);
        } else {
          h[0] = (uint32_t)(unsigned short)__ldg((const short*)(sc.ell + v) + sub);
        }
        fb = sub == 0 && (h[0] & 0xFFFFu) == 0x8000u;  // sentinel: the row is read from the CSR
        if (fb) h[0] = 0u;
      } else {
        fb = sub == 0;
      }
      if (a.collect_stats && sub == 0) {
        n_exp++;
        n_edge += (unsigned long long)(__ldg(sc.rowptr + v + 1) - __ldg(sc.rowptr + v));
      }
    }
    // empty slots (offset 0) and lanes without a vertex give w == v: skipped
    const int vv = v < 0 ? 0 : v;
#pragma unroll
    for (int q = 0; q < K; q++) {
      const uint32_t half = (q & 1) ? (h[q >> 1] >> 16) : (h[q >> 1] & 0xFFFFu);
      wv[q] = vv + (int)(short)half;
    }
    if constexpr (K == 8) {
      // records are packed, so slots 4-7 are empty for rows of up to 4 neighbours
      relax_group<SV, 8, 0, 4>(tm, wv, vv, sc.s, t, em, smin, smax);
      if (__any_sync(FULL, (h[2] | h[3]) != 0u)) relax_group<SV, 8, 4, 4>(tm, wv, vv, sc.s, t, em, smin, smax);
    } else {
      relax_group<SV, K, 0, K>(tm, wv, vv, sc.s, t, em, smin, smax);
    }
    // append the members: ballots for one or two slots per lane, else a scan
    if constexpr (K <= 2) {
      const unsigned b0 = __ballot_sync(FULL, em & 1u);
      unsigned b1 = 0u;
      if constexpr (K == 2) b1 = __ballot_sync(FULL, em & 2u);
      if (em & 1u) *q_slot(tm, level + 1, nb, nq + __popc(b0 & lt)) = wv[0];
      if constexpr (K == 2)
        if (em & 2u) *q_slot(tm, level + 1, nb, nq + __popc(b0) + __popc(b1 & lt)) = wv[1];
      nq += __popc(b0) + __popc(b1);
    } else {
      const int cnt = __popc(em);
      int inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += x;
      }
      const int tot = __shfl_sync(FULL, inc, 31);
      if (tot) {
        int pos = nq + inc - cnt;
#pragma unroll
        for (int q = 0; q < K; q++)
          if ((em >> q) & 1u) *q_slot(tm, level + 1, nb, pos++) = wv[q];
        nq += tot;
      }
    }
    unsigned fm = __ballot_sync(FULL, fb);
    while (fm) {
      const int l = __ffs(fm) - 1;
      fm &= fm - 1;
      walk_row<SV, false>(sc, tm, nullptr, __shfl_sync(FULL, v, l), t, level, nb, nq, smin, smax, bad);
    }
  }
}

// Warp mode: pick the lanes per vertex from the level's length.
template <bool SV>
__device__ __forceinline__ void expand_warp(const TravArgs& a, const Src& sc, const Team& tm, int t, int level,
                                            int64_t cb, int64_t nb, bool head, int qlen, int& nq, int& smin,
                                            int& smax, unsigned long long& n_exp, unsigned long long& n_edge,
                                            int& bad) {
  if (qlen <= 4)
    expand_level_warp<SV, 8>(a, sc, tm, t, level, cb, nb, head, qlen, nq, smin, smax, n_exp, n_edge, bad);
  else if (qlen <= 8)
    expand_level_warp<SV, 4>(a, sc, tm, t, level, cb, nb, head, qlen, nq, smin, smax, n_exp, n_edge, bad);
  else if (qlen <= 16)
    expand_level_warp<SV, 2>(a, sc, tm, t, level, cb, nb, head, qlen, nq, smin, smax, n_exp, n_edge, bad);
  else
    expand_level_warp<SV, 1>(a, sc, tm, t, level, cb, nb, head, qlen, nq, smin, smax, n_exp, n_edge, bad);
}

// Emit the row of source s (one warp): [L cols | s | U cols] into the row pool
// at an atomically taken offset, plus the per-row counts.  swmax: the last
// summary word that may be nonzero (global V).
template <bool SV>
__device__ void emit_row(const TravArgs& a, const Src& sc, const Team& tm, int nL, int diag, int rb, int re,
                         int swmax) {
  const int lane = threadIdx.x & 31;
  const int s = sc.s;
  const int ws = s >> 5;                                  // word holding s
  const uint32_t first_mask = (s & 31) == 31 ? 0u : (0xFFFFFFFEu << (s & 31));  // bits above s in word ws
  const int vwords = (sc.n + 31) >> 5;
  // count U(s,:)
  int nU = 1;
  if constexpr (SV) {
    for (int j0 = ws; j0 < vwords; j0 += 32) {
      const int j = j0 + lane;
      uint32_t m = j < vwords ? tm.V[j] : 0u;
      if (j == ws) m &= first_mask;
      int c = __popc(m);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
      nU += c;
    }
  } else {
    for (int sw0 = ws >> 5; sw0 <= swmax; sw0 += 32) {
      const int sw = sw0 + lane;
      uint32_t sm = sw <= swmax ? v_load<SV>(tm.VS, sw) : 0u;
      if (sw == (ws >> 5)) sm &= 0xFFFFFFFFu << (ws & 31);
      unsigned any = __ballot_sync(FULL, sm != 0u);
      while (any) {
        const int l = __ffs(any) - 1;
        any &= any - 1;
        const uint32_t ml = __shfl_sync(FULL, sm, l);
        const int pw = ((sw0 + l) << 5) + lane;
        uint32_t word = ((ml >> lane) & 1u) ? v_load<SV>(tm.V, pw) : 0u;
        if (pw == ws) word &= first_mask;
        int c = __popc(word);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        nU += c;
      }
    }
  }
  unsigned long long off = 0ull;
  int ok = 0;
  if (lane == 0) {
    const long long r = sc.rowb + s;
    const int total = nL + nU;
    if (a.counts_only) {
      ok = 0;
    } else {
      off = atomicAdd(&a.ctr->pool_cursor, (unsigned long long)total);
      ok = off + (unsigned long long)total <= (unsigned long long)a.pool_cap;
      a.row_off[r] = ok ? (int64_t)off : -1;
      if (ok) a.pool[off + nL] = (uint32_t)s;
      else atomicOr(&a.ctr->err, ERR_OVERFLOW);
    }
    a.row_nL[r] = nL;
    a.row_nU[r] = nU;
    a.fill_count[r] = total - ((re - rb) + (diag ? 0 : 1));
    atomicAdd(&a.ctr->total_L, (unsigned long long)nL);
    atomicAdd(&a.ctr->total_U, (unsigned long long)nU);
    if (a.mat_tot) {
      atomicAdd(&a.mat_tot[2 * sc.mi], (unsigned long long)nL);
      atomicAdd(&a.mat_tot[2 * sc.mi + 1], (unsigned long long)nU);
    }
  }
  off = __shfl_sync(FULL, off, 0);
  ok = __shfl_sync(FULL, ok, 0);
  if (!ok) return;
  for (int i = lane; i < nL; i += 32) a.pool[off + i] = (uint32_t)*l_slot(tm, i);
  // write U(s,:) above the diagonal, in increasing order
  long long pos = (long long)off + nL + 1;
  if constexpr (SV) {
    for (int j0 = ws; j0 < vwords; j0 += 32) {
      const int j = j0 + lane;
      uint32_t word = j < vwords ? tm.V[j] : 0u;
      if (j == ws) word &= first_mask;
      const int c = __popc(word);
      int inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += x;
      }
      long long p = pos + (inc - c);
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        a.pool[p++] = (uint32_t)((j << 5) + b);
      }
      pos += __shfl_sync(FULL, inc, 31);
    }
  } else {
    for (int sw0 = ws >> 5; sw0 <= swmax; sw0 += 32) {
      const int sw = sw0 + lane;
      uint32_t sm = sw <= swmax ? v_load<SV>(tm.VS, sw) : 0u;
      if (sw == (ws >> 5)) sm &= 0xFFFFFFFFu << (ws & 31);
      unsigned any = __ballot_sync(FULL, sm != 0u);
      while (any) {
        const int l = __ffs(any) - 1;
        any &= any - 1;
        const uint32_t ml = __shfl_sync(FULL, sm, l);
        const int pw = ((sw0 + l) << 5) + lane;
        uint32_t word = ((ml >> lane) & 1u) ? v_load<SV>(tm.V, pw) : 0u;
        if (pw == ws) word &= first_mask;
        const int c = __popc(word);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int x = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += x;
        }
        long long p = pos + (inc - c);
        while (word) {
          const int b = __ffs(word) - 1;
          word &= word - 1;
          a.pool[p++] = (uint32_t)((pw << 5) + b);
        }
        pos += __shfl_sync(FULL, inc, 31);
      }
    }
  }
}

// Clear the bits the source set (threads tid, tid + nthr, ...).  Global V:
// the summary words in [swmin, swmax] say which V words hold bits.
template <bool SV>
__device__ __forceinline__ void clear_v(const Team& tm, int vwords, int swmin, int swmax, int tid, int nthr) {
  if constexpr (SV) {
    for (int j = tid; j < vwords; j += nthr) tm.V[j] = 0u;
  } else {
    if (swmin > swmax) return;  // the source set no bit (no off-diagonal neighbour)
    for (int sw = swmin + tid; sw <= swmax; sw += nthr) {
      uint32_t m = tm.VS[sw];
      if (!m) continue;
      tm.VS[sw] = 0u;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        tm.V[(sw << 5) + b] = 0u;
      }
    }
  }
}

__device__ __forceinline__ int warp_min(int x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x = min(x, __shfl_xor_sync(FULL, x, o));
  return x;
}
__device__ __forceinline__ int warp_max(int x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x = max(x, __shfl_xor_sync(FULL, x, o));
  return x;
}

}  // namespace

namespace {

// Source of work item k (items in issue order, largest source first).
__device__ __forceinline__ Src source_of(const TravArgs& a, int k) {
  Src sc;
  sc.n = a.n;
  sc.rowptr = a.rowptr;
  sc.colidx = a.colidx;
  sc.ell = a.ell;
  sc.rowb = 0;
  sc.mi = 0;
  if (a.mats) {  // batch: smallest source index s with item_start[s] <= k, then the matrix
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a.item_start[mid] <= k) hi = mid; else lo = mid + 1;
    }
    sc.s = lo;
    sc.mi = a.mat_order[k - a.item_start[lo]];
    const MatDesc d = a.mats[sc.mi];
    sc.n = d.n;
    sc.rowptr = d.rowptr;
    sc.colidx = d.colidx;
    sc.rowb = d.row_base;
    if (a.ell) sc.ell = a.ell + d.row_base;
  } else {
    sc.s = a.order ? a.order[k] : a.nsrc - 1 - k;
  }
  return sc;
}

// One source from seeds to a cleared V.  TEAM: the whole CTA (warp 0 searches
// classes and emits), else the calling warp.
template <bool SV, bool TEAM>
__device__ void run_source(const TravArgs& a, const Src& sc, const Team& tm, CtCtl* ctl, unsigned long long& n_exp,
                           unsigned long long& n_edge, unsigned long long& n_lev, int& bad) {
  const int lane = threadIdx.x & 31;
  const int nthr = TEAM ? CT_THREADS : 32;
  const int tid = TEAM ? (int)threadIdx.x : lane;
  const bool leader = !TEAM || threadIdx.x < 32;
  const int s = sc.s;
  int smin = 0x7FFFFFFF, smax = -1;

  // seeds: neighbours below s are classes with maxId -1; above s, U entries
  const int rb = __ldg(sc.rowptr + s), re = __ldg(sc.rowptr + s + 1);
  int diag = 0;
  for (int e = rb + tid; e < re; e += nthr) {
    const int w = __ldg(sc.colidx + e);
    if ((unsigned)w >= (unsigned)sc.n) { bad = 1; continue; }
    if (w == s) { diag = 1; continue; }
    v_set<SV>(tm.V, tm.VS, w, smin, smax);
  }
  if constexpr (TEAM) diag = __syncthreads_or(diag);
  else diag = __any_sync(FULL, diag);

  if constexpr (!TEAM) __syncwarp();

  int cursor = 0, nL = 0;
  int level = 0;  // team mode: running level index (queues and counters rotate with it)
  for (;;) {
    int t;
    if constexpr (TEAM) {
      // warp 0 finds the class and expands its head (t alone) into the next
      // level; the counter it fills and the one it zeroes are not the one the
      // other warps may still be reading (the last level's zero length)
      if (leader) {
        t = next_class<SV>(tm, cursor, s, lane);
        int nq = 0;
        if (t >= 0) {
          if (lane == 0) *l_slot(tm, nL) = t;
          // the class's levels overflow into the log from its bottom
          expand_warp<SV>(a, sc, tm, t, level, 0, 0, true, 1, nq, smin, smax, n_exp, n_edge, bad);
          n_lev++;
        }
        if (lane == 0) {
          ctl->t = t;
          ctl->qcnt[(level + 1) % 3] = nq;
          ctl->qcnt[(level + 2) % 3] = 0;
        }
      }
      __syncthreads();
      t = ctl->t;
      if (t < 0) break;
      cursor = t + 1;
      nL++;
      int64_t cb = 0;
      for (level++;; level++) {
        const int qlen = ctl->qcnt[level % 3];
        if (qlen == 0) break;
        if (leader) n_lev++;
        if (threadIdx.x == 0) ctl->qcnt[(level + 2) % 3] = 0;
        int nq_unused = 0;
        const int64_t nb = next_base(tm, cb, qlen);
        expand_level<SV, true>(a, sc, tm, ctl, t, level, cb, nb, false, qlen, nq_unused, smin, smax, n_exp, n_edge,
                               bad);
        cb = nb;
        __syncthreads();
      }
    } else {
      t = next_class<SV>(tm, cursor, s, lane);
      if (t < 0) break;
      cursor = t + 1;
      if (lane == 0) *l_slot(tm, nL) = t;
      nL++;
      int qlen = 1;
      int64_t cb = 0;  // the class's levels overflow into the log from its bottom
      for (int lv = 0; qlen > 0; lv++) {
        int nq = 0;
        n_lev++;
        const int64_t nb = lv == 0 ? 0 : next_base(tm, cb, qlen);
        expand_warp<SV>(a, sc, tm, t, lv, cb, nb, lv == 0, qlen, nq, smin, smax, n_exp, n_edge, bad);
        __syncwarp();
        cb = nb;
        qlen = nq;
      }
    }
  }

  // the summary words this source touched
  int swmin = smin, swmax = smax;
  if constexpr (!SV) {
    swmin = warp_min(smin);
    swmax = warp_max(smax);
    if constexpr (TEAM) {
      if (threadIdx.x == 0) { ctl->smin = 0x7FFFFFFF; ctl->smax = -1; }
      __syncthreads();
      if (lane == 0) { atomicMin(&ctl->smin, swmin); atomicMax(&ctl->smax, swmax); }
      __syncthreads();
      swmin = ctl->smin;
      swmax = ctl->smax;
    }
  }
  if (leader) emit_row<SV>(a, sc, tm, nL, diag, rb, re, swmax);
  if constexpr (TEAM) __syncthreads();
  else __syncwarp();
  clear_v<SV>(tm, (sc.n + 31) >> 5, swmin, swmax, tid, nthr);
  if constexpr (TEAM) __syncthreads();
  else __syncwarp();
}

// Shared memory: control blocks (one per warp; team mode uses warp 0's), two
// queues of qw entries per warp, then (SV) one V of vwords words per warp.
__host__ __device__ __forceinline__ size_t ct_smem_bytes(int sv, int vwords, int qw) {
  return (size_t)CT_WARPS * 64 + (size_t)2 * CT_WARPS * qw * 4 + (sv ? (size_t)CT_WARPS * vwords * 4 : 0);
}

}  // namespace

// MINB: CTAs of four warps per SM the register budget is sized for.
template <bool SV, int MINB>
__global__ void __launch_bounds__(CT_THREADS, MINB) trav_class_kernel(TravArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qw = a.ct_qw;
  const int vwords = a.ct_vwords;
  CtCtl* ctls = (CtCtl*)smem;
  int32_t* q0 = (int32_t*)(smem + CT_WARPS * 64);
  int32_t* q1 = q0 + CT_WARPS * qw;
  uint32_t* vsh = (uint32_t*)(q1 + CT_WARPS * qw);
  const size_t gcap = (size_t)a.g_cap;

  if constexpr (SV) {
    for (int j = threadIdx.x; j < CT_WARPS * vwords; j += CT_THREADS) vsh[j] = 0u;
    __syncthreads();
  }
  unsigned long long n_exp = 0, n_edge = 0, n_lev = 0;
  int bad = 0;

  // ---- team phase: the first nbig items, one CTA per source
  if (a.ct_nbig > 0) {
    const size_t slot = (size_t)blockIdx.x * CT_WARPS;
    Team tm;
    tm.V = SV ? vsh : a.g_V + slot * (gcap / 32);
    tm.VS = SV ? nullptr : a.g_VS + slot * (gcap / 1024);
    tm.qa = q0;
    tm.qb = q1;
    tm.qcap = CT_WARPS * qw;
    tm.log = a.g_log + slot * gcap;
    tm.cap = (int64_t)gcap;
    CtCtl* ctl = &ctls[0];
    for (;;) {
      if (threadIdx.x == 0) {
        const int k = atomicAdd(&a.ctr->work_team, 1);
        ctl->src = (k < a.ct_nbig && !input_error(a.ctr)) ? k : -1;
      }
      __syncthreads();
      const int k = ctl->src;
      if (k < 0) break;
      const Src sc = source_of(a, k);
      run_source<SV, true>(a, sc, tm, ctl, n_exp, n_edge, n_lev, bad);
    }
    __syncthreads();
  }

  // ---- warp phase: every other item, one warp per source
  if ((long long)blockIdx.x * CT_WARPS + warp < a.g_slots) {
    const size_t slot = (size_t)blockIdx.x * CT_WARPS + warp;
    Team tm;
    tm.V = SV ? vsh + (size_t)warp * vwords : a.g_V + slot * (gcap / 32);
    tm.VS = SV ? nullptr : a.g_VS + slot * (gcap / 1024);
    tm.qa = q0 + warp * qw;
    tm.qb = q1 + warp * qw;
    tm.qcap = qw;
    tm.log = a.g_log + slot * gcap;
    tm.cap = (int64_t)gcap;
    CtCtl* ctl = &ctls[warp];
    for (;;) {
      int k = -1;
      if (lane == 0) {
        k = a.ct_nbig + atomicAdd(&a.ctr->work_global, 1);
        if (k >= a.nsrc || input_error(a.ctr)) k = -1;
      }
      k = __shfl_sync(FULL, k, 0);
      if (k < 0) break;
      const Src sc = source_of(a, k);
      run_source<SV, false>(a, sc, tm, ctl, n_exp, n_edge, n_lev, bad);
    }
  }

  if (bad) atomicOr(&a.ctr->err, ERR_COL_RANGE);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    n_exp += __shfl_xor_sync(FULL, n_exp, o);
    n_edge += __shfl_xor_sync(FULL, n_edge, o);
  }
  if (lane == 0) {
    if (a.collect_stats) {
      atomicAdd(&a.ctr->expansions, n_exp);
      atomicAdd(&a.ctr->edges, n_edge);
    }
    atomicAdd(&a.ctr->levels, n_lev);
  }
}

size_t trav_class_smem(int sv, int vwords, int qw) { return ct_smem_bytes(sv, vwords, qw); }

namespace {
template <bool SV, int MINB>
cudaError_t launch_one(const TravArgs& a, int grid, size_t smem, cudaStream_t st) {
  static int attr_set[128] = {0};  // per device: the dynamic shared-memory limit was raised
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 128 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(trav_class_kernel<SV, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[dev] = 1;
  }
  trav_class_kernel<SV, MINB><<<grid, CT_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <bool SV, int MINB>
int occupancy_one(size_t smem) {
  // answers are cached per (device, build, shared-memory size): the query is
  // made on every plan and every server admission
  static std::mutex mu;
  static std::map<std::tuple<int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, smem});
    if (it != cache.end()) return it->second;
  }
  cudaFuncSetAttribute(trav_class_kernel<SV, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trav_class_kernel<SV, MINB>, CT_THREADS, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[{dev, smem}] = occ;
  return occ;
}
}  // namespace

// CTAs of four warps per SM the class kernel reaches with this shared memory;
// warps_per_sm above 32 selects the 48-register build.
int trav_class_occupancy(int sv, int warps_per_sm, int vwords, int qw) {
  const size_t smem = ct_smem_bytes(sv, vwords, qw);
  if (smem > 227 * 1024) return 0;
  if (warps_per_sm > 32) return sv ? occupancy_one<true, 10>(smem) : occupancy_one<false, 10>(smem);
  return sv ? occupancy_one<true, 8>(smem) : occupancy_one<false, 8>(smem);
}

cudaError_t launch_trav_class(const TravArgs& a, int grid, int sv, int warps_per_sm, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  const size_t smem = ct_smem_bytes(sv, a.ct_vwords, a.ct_qw);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (warps_per_sm > 32) return sv ? launch_one<true, 10>(a, grid, smem, st) : launch_one<false, 10>(a, grid, smem, st);
  return sv ? launch_one<true, 8>(a, grid, smem, st) : launch_one<false, 8>(a, grid, smem, st);
}

}  // namespace gsofa
