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
// out, then each warp takes single sources from another.  A level of q
// vertices is expanded with 8, 4, 2 or 1 lanes per vertex (each lane relaxing
// 1, 2, 4 or 8 of the vertex's record slots), chosen by q, so small levels
// (class heads are single vertices) keep most lanes busy.
//
// Where V lives (template parameter VM): VM_SMEM, all n bits in shared memory,
// one bitmap per warp (orders whose bitmaps leave at least 16 warps per SM);
// VM_GLOBAL, a global-memory slot per warp with a summary bitmap (one bit per
// nonzero V word) that bounds the searches and the clearing.
// Frontier levels live in shared-memory queues of `qw` entries per warp;
// longer levels overflow into the slot's log array from its bottom, each level
// after the previous one of the same class, while the L row grows down from
// its top one class at a time (sorted by construction).  A vertex below s is a
// class member or a fill, never both, and joins at most one level, so the two
// ends never meet in s entries.  Each source clears the bits it set.
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace gsofa {

namespace {

constexpr int CT_WARPS = 4;  // warps per CTA (one team in team mode)
constexpr int CT_THREADS = 32 * CT_WARPS;
constexpr int VM_SMEM = 0, VM_GLOBAL = 1;

// Per-team control block in shared memory.
struct CtCtl {
  int src;        // team mode: the current work item (-1: no more team items)
  int t;          // the class being expanded (-1: no pending class)
  int qcnt[3];    // rotating level lengths
  int smin, smax; // summary words touched (global V)
  int cmin;       // team mode: the smallest seed below the source
};

// ---- primitive bit operations
// Atomic OR issued under a predicate; returns `bit` (= already set) when not issued.
__device__ __forceinline__ uint32_t or_shared_if(uint32_t* p, uint32_t bit, bool pred) {
  uint32_t r = bit;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.shared.or.b32 %0, [%1], %2;\n\t}"
               : "+r"(r)
               : "r"(a), "r"(bit), "r"((uint32_t)pred)
               : "memory");
  return r;
}

__device__ __forceinline__ uint32_t or_global_if(uint32_t* p, uint32_t bit, bool pred) {
  uint32_t r = bit;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.global.or.b32 %0, [%1], %2;\n\t}"
               : "+r"(r)
               : "l"(p), "r"(bit), "r"((uint32_t)pred)
               : "memory");
  return r;
}

__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return *(const volatile uint32_t*)p; }

// The team's view of one source: where V, the queues and the log live.
struct Team {
  uint32_t* V;        // VM_SMEM: n bits in shared memory; else the global slot (n bits)
  uint32_t* VS;       // summary of the global slot
  int32_t* qa;        // shared queue, even levels
  int32_t* qb;        // shared queue, odd levels
  int qcap;           // shared queue capacity (entries per level)
  int32_t* log;       // level overflow from the bottom, L(s,:) from the top
  int64_t cap;        // entries of log (>= n)
};

// Per-lane bookkeeping of the global slot: the summary words touched.
struct VState {
  int smin, smax;
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

// Issue the OR of w's bit under pred.
template <int VM>
__device__ __forceinline__ uint32_t v_or_if(const Team& tm, int w, bool pred) {
  const uint32_t bit = 1u << (w & 31);
  if constexpr (VM == VM_SMEM) return or_shared_if(tm.V + (w >> 5), bit, pred);
  else return or_global_if(tm.V + (w >> 5), bit, pred);
}

// Book-keeping after this lane's OR set w's bit first: a global word that was
// empty gets its summary bit.
template <int VM>
__device__ __forceinline__ void v_first(const Team& tm, int w, uint32_t old, VState& st) {
  if constexpr (VM == VM_GLOBAL) {
    if (old == 0u) {
      red_or(tm.VS + (w >> 10), 1u << ((w >> 5) & 31));
      st.smin = min(st.smin, w >> 10);
      st.smax = max(st.smax, w >> 10);
    }
  }
}

// Set bit w (one lane).  Returns true when this call set it.
template <int VM>
__device__ __forceinline__ bool v_set(const Team& tm, int w, VState& st) {
  const uint32_t old = v_or_if<VM>(tm, w, true);
  if (old & (1u << (w & 31))) return false;
  v_first<VM>(tm, w, old, st);
  return true;
}

// Smallest set bit at a vertex p in [from, lim) of a shared bitmap W whose
// bit 0 is vertex `base` (base a multiple of 32); -1 if none.  Warp-wide.
__device__ int scan_smem(const uint32_t* W, int base, int from, int lim, int lane) {
  if (from >= lim) return -1;
  const int wfirst = (from - base) >> 5;
  const int wend = (lim - base + 31) >> 5;
  {  // the word holding `from` first (every lane reads it): the next class is usually there
    const uint32_t m = W[wfirst] & (0xFFFFFFFFu << ((from - base) & 31));
    if (m) {
      const int v = base + (wfirst << 5) + __ffs(m) - 1;
      return v < lim ? v : -1;
    }
  }
  for (int w0 = wfirst + 1; w0 < wend; w0 += 32) {
    const int j = w0 + lane;
    uint32_t m = 0u;
    if (j < wend) {
      m = W[j];
      const int hi = lim - base - (j << 5);
      if (hi < 32) m &= (1u << hi) - 1u;
    }
    const unsigned b = __ballot_sync(FULL, m != 0u);
    if (b) {
      const int l = __ffs(b) - 1;
      m = __shfl_sync(FULL, m, l);
      return base + ((w0 + l) << 5) + __ffs(m) - 1;
    }
  }
  return -1;
}

// Smallest set bit in [from, lim) of the global slot, through its summary; -1
// if none.  Warp-wide.
__device__ int scan_global(const Team& tm, int from, int lim, int lane) {
  if (from >= lim) return -1;
  const int wfirst = from >> 5;
  const int wend = (lim + 31) >> 5;
  // the cursor's own word first
  const uint32_t m = ld_cg(tm.V + wfirst) & (0xFFFFFFFFu << (from & 31));
  if (m) {
    const int v = (wfirst << 5) + __ffs(m) - 1;
    return v < lim ? v : -1;
  }
  // then the summary from the next word on
  const int wstart = wfirst + 1;
  if (wstart >= wend) return -1;
  const int send = (wend + 31) >> 5;
  for (int sw0 = wstart >> 5; sw0 < send; sw0 += 32) {
    const int sw = sw0 + lane;
    uint32_t sm = 0u;
    if (sw < send) {
      sm = ld_cg(tm.VS + sw);
      if (sw == (wstart >> 5)) sm &= 0xFFFFFFFFu << (wstart & 31);
    }
    const unsigned b = __ballot_sync(FULL, sm != 0u);
    if (b) {
      const int l = __ffs(b) - 1;
      sm = __shfl_sync(FULL, sm, l);
      const int pw = ((sw0 + l) << 5) + __ffs(sm) - 1;  // first nonzero word at or after wstart
      const uint32_t word = ld_cg(tm.V + pw);
      const int v = (pw << 5) + __ffs(word) - 1;
      return (word != 0u && v < lim) ? v : -1;
    }
  }
  return -1;
}

// Smallest vertex of V in [from, s): the next pending class, or -1.
template <int VM>
__device__ int next_class(const Team& tm, int from, int s, int lane) {
  if constexpr (VM == VM_SMEM) return scan_smem(tm.V, 0, from, s, lane);
  else return scan_global(tm, from, s, lane);
}

// Relax slots [Q0, Q0 + G) of the lane's record group (their OR operations
// issued together); first-reached vertices below t set their bit in em.
template <int VM, int K, int Q0, int G>
__device__ __forceinline__ void relax_group(const Team& tm, const int (&wv)[K], int v, int s, int t, unsigned& em,
                                            VState& st) {
  uint32_t old[G];
#pragma unroll
  for (int q = 0; q < G; q++) {
    const int w = wv[Q0 + q];
    old[q] = v_or_if<VM>(tm, w, w != v && w != s);
  }
#pragma unroll
  for (int q = 0; q < G; q++) {
    const int w = wv[Q0 + q];
    if (!(old[q] & (1u << (w & 31)))) {  // first reach (an OR not issued returns the bit)
      v_first<VM>(tm, w, old[q], st);
      if (w < t) em |= 1u << (Q0 + q);
    }
  }
}

// Source-independent inputs of one source.
struct Src {
  int s;
  int n;
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ colidx;
  const int4* __restrict__ ell;  // records of this matrix (row v at ell[v]) or null
  const int4* __restrict__ ellw; // wide records (row v at ellw[2v], ellw[2v+1]) or null
  long long rowb;                // row offset in the per-row arrays (batch)
  int mi;
};

// Clean class heads.  A pending class t whose head has every neighbour
// (other than s) in V already changes nothing when expanded: no member, no
// new fill, no new U entry.  Taken in increasing order, each such class
// leaves V as it found it, so a run of them can be decided together: the
// warp gathers the (up to 32) smallest pending classes t_0 < t_1 < ... from
// t0 on, reads their heads' neighbours' bits, and retires the longest prefix
// of clean heads at once (appended to L(s,:)).  The first class that is not
// clean, if any, is returned in tnext and expanded as usual; the classes
// after it stay pending.  Returns the number retired; last = the largest
// class gathered (when every gathered class was clean, the search resumes
// above it).  Warp-wide; the scratch is the team's even-level queue, free
// between classes.
template <int VM>
__device__ int retire_clean(const TravArgs& a, const Src& sc, const Team& tm, int t0, int nL, int lane, int& tnext,
                            int& last, unsigned long long& n_exp, unsigned long long& n_edge) {
  const int s = sc.s;
  const int K = tm.qcap < 32 ? tm.qcap : 32;
  // gather: lane l reads word (t0 >> 5) + l; set bits in [t0, s) ranked by a warp scan
  const int wl = (t0 >> 5) + lane;
  uint32_t m = 0u;
  if ((wl << 5) < s) {
    if constexpr (VM == VM_SMEM) m = tm.V[wl];
    else m = ld_cg(tm.V + wl);
    if (lane == 0) m &= 0xFFFFFFFFu << (t0 & 31);
    const int hi = s - (wl << 5);
    if (hi < 32) m &= (1u << hi) - 1u;
  }
  const int c = __popc(m);
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += x;
  }
  const int total = __shfl_sync(FULL, inc, 31);
  int pos = inc - c;
  while (m && pos < K) {
    const int b = __ffs(m) - 1;
    m &= m - 1;
    tm.qa[pos++] = (wl << 5) + b;
  }
  __syncwarp();
  const int cnt = total < K ? total : K;  // >= 1: t0 is pending
  const int tj = lane < cnt ? tm.qa[lane] : -1;
  __syncwarp();
  // check: every neighbour of t_j (CSR rows of more than 8 entries count as not clean)
  bool clean = false;
  int deg = 0;
  if (tj >= 0) {
    int wv[8];
    int nw = 0;
    bool csr = (VM != VM_SMEM || sc.ell == nullptr) && sc.ellw == nullptr;
    if (sc.ellw) {
      const int4 r0 = __ldg(sc.ellw + 2 * (size_t)tj), r1 = __ldg(sc.ellw + 2 * (size_t)tj + 1);
      wv[0] = r0.x; wv[1] = r0.y; wv[2] = r0.z; wv[3] = r0.w;
      wv[4] = r1.x; wv[5] = r1.y; wv[6] = r1.z; wv[7] = r1.w;
      if (wv[0] < 0) csr = true;  // sentinel
      else nw = 8;                // empty slots hold t_j itself
    } else if (VM == VM_SMEM && !csr) {
      const int4 r = __ldg(sc.ell + tj);
      const uint32_t h[4] = {(uint32_t)r.x, (uint32_t)r.y, (uint32_t)r.z, (uint32_t)r.w};
      if ((h[0] & 0xFFFFu) == 0x8000u) {
        csr = true;
      } else {
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int off = (int)(short)((q & 1) ? (h[q >> 1] >> 16) : (h[q >> 1] & 0xFFFFu));
          wv[q] = tj + off;  // offset 0 (empty slot): w == t_j, skipped below
        }
        nw = 8;
      }
    }
    clean = true;
    if (csr) {
      const int rb = __ldg(sc.rowptr + tj), re = __ldg(sc.rowptr + tj + 1);
      if (re - rb > 8) {
        clean = false;
      } else {
#pragma unroll
        for (int q = 0; q < 8; q++) wv[q] = q < re - rb ? __ldg(sc.colidx + rb + q) : tj;
        nw = 8;
      }
    }
    if (clean) {
      uint32_t wd[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int w = wv[q];
        wd[q] = 0xFFFFFFFFu;
        if (q < nw && w != tj && w != s) {
          if ((unsigned)w >= (unsigned)sc.n) wd[q] = 0u;  // left to the expansion, which flags it
          else if constexpr (VM == VM_SMEM) wd[q] = tm.V[w >> 5];
          else wd[q] = ld_cg(tm.V + (w >> 5));
        }
      }
#pragma unroll
      for (int q = 0; q < 8; q++)
        if (!((wd[q] >> (wv[q] & 31)) & 1u)) clean = false;
    }
    if (a.collect_stats) deg = __ldg(sc.rowptr + tj + 1) - __ldg(sc.rowptr + tj);
  }
  const unsigned dirty = __ballot_sync(FULL, tj >= 0 && !clean);
  const int k = dirty ? __ffs(dirty) - 1 : cnt;
  if (lane < k) {
    *l_slot(tm, nL + lane) = tj;
    if (a.collect_stats) {
      n_exp++;
      n_edge += (unsigned long long)deg;
    }
  }
  tnext = k < cnt ? __shfl_sync(FULL, tj, k & 31) : -1;
  last = __shfl_sync(FULL, tj, (cnt - 1) & 31);
  return k;
}

}  // namespace

namespace {

// Append this warp's `cnt` new entries (in lane order) to the next level:
// warp mode bumps nq, team mode takes room from the shared counter.  Returns
// the level index of the warp's first entry.
template <bool TEAM>
__device__ __forceinline__ int append_base(CtCtl* ctl, int level, int tot, int& nq) {
  if constexpr (TEAM) {
    int base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(&ctl->qcnt[(level + 1) % 3], tot);
    return __shfl_sync(FULL, base, 0);
  } else {
    const int base = nq;
    nq += tot;
    return base;
  }
}

// Walk row u from the CSR (rows without an ELL record, or no records at all):
// the warp takes 32 entries at a time; first-reached vertices below t join the
// next level.  Columns are range-checked here.
template <int VM, bool TEAM>
__device__ void walk_row(const Src& sc, const Team& tm, CtCtl* ctl, int u, int t, int level, int64_t nb, int& nq,
                         VState& st, int& bad) {
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
        enq = v_set<VM>(tm, w, st) && w < t;
      }
    }
    const unsigned m = __ballot_sync(FULL, enq);
    if (!m) continue;
    const int base = append_base<TEAM>(ctl, level, __popc(m), nq);
    if (enq) *q_slot(tm, level + 1, nb, base + __popc(m & lt)) = w;
  }
}

// One level of class t with LPV lanes per vertex: the calling warp (TEAM
// false) or the CTA (TEAM true) takes the level's vertices, each lane relaxing
// K = 8/LPV consecutive record slots of its vertex, and appends the
// first-reached vertices below t to the next level.  head: the class's first
// level, t alone.  `level` indexes the queues (parity) and team counters; the
// level's overflow starts at log[cb], the next level's at log[nb].
template <int VM, bool TEAM, int LPV>
__device__ void expand_level(const TravArgs& a, const Src& sc, const Team& tm, CtCtl* ctl, int t, int level,
                             int64_t cb, int64_t nb, bool head, int qlen, int& nq, VState& st,
                             unsigned long long& n_exp, unsigned long long& n_edge, int& bad) {
  constexpr int K = 8 / LPV;
  constexpr int PER = (TEAM ? CT_THREADS : 32) / LPV;  // vertices per round
  const int lane = threadIdx.x & 31;
  const int rank = TEAM ? (int)threadIdx.x : lane;
  const unsigned lt = (1u << lane) - 1u;
  const int sub = lane % LPV;  // which K slots of the vertex
  const int vi = rank / LPV;
  for (int i0 = 0; i0 < qlen; i0 += PER) {
    const int i = i0 + vi;
    int v = -1;
    if (i < qlen) v = head ? t : *q_slot(tm, level, cb, i);
    int wv[K];
    bool fb = false;
    unsigned em = 0u;
    bool hi4 = false;  // K == 8: slots 4-7 hold neighbours (records are packed)
    // empty slots and lanes without a vertex give w == v (0 for no vertex): skipped
    const int vv = v < 0 ? 0 : v;
    if (sc.ellw) {
#pragma unroll
      for (int q = 0; q < K; q++) wv[q] = vv;
      if (v >= 0) {
        const int4* rec = sc.ellw + 2 * (size_t)v;
        if constexpr (K == 8) {
          const int4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
          wv[0] = r0.x; wv[1] = r0.y; wv[2] = r0.z; wv[3] = r0.w;
          wv[4] = r1.x; wv[5] = r1.y; wv[6] = r1.z; wv[7] = r1.w;
        } else if constexpr (K == 4) {
          const int4 r = __ldg(rec + sub);
          wv[0] = r.x; wv[1] = r.y; wv[2] = r.z; wv[3] = r.w;
        } else if constexpr (K == 2) {
          const int2 r = __ldg((const int2*)rec + sub);
          wv[0] = r.x; wv[1] = r.y;
        } else {
          wv[0] = __ldg((const int*)rec + sub);
        }
        fb = sub == 0 && wv[0] < 0;  // sentinel: the row is read from the CSR
        if (fb) wv[0] = vv;
        if constexpr (K == 8) hi4 = wv[4] != vv;
        if (a.collect_stats && sub == 0) {
          n_exp++;
          n_edge += (unsigned long long)(__ldg(sc.rowptr + v + 1) - __ldg(sc.rowptr + v));
        }
      }
    } else {
      // 16-bit records exist only for orders up to 32,768, i.e. with shared
      // bitmaps; the global-bitmap build reads rows without wide records from the CSR
      uint32_t h[(K + 1) / 2];
#pragma unroll
      for (int q = 0; q < (K + 1) / 2; q++) h[q] = 0u;
      if (v >= 0) {
        if (VM == VM_SMEM && sc.ell) {
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
#pragma unroll
      for (int q = 0; q < K; q++) {
        const uint32_t half = (q & 1) ? (h[q >> 1] >> 16) : (h[q >> 1] & 0xFFFFu);
        wv[q] = vv + (int)(short)half;
      }
      if constexpr (K == 8) hi4 = (h[2] | h[3]) != 0u;
    }
    if constexpr (K == 8) {
      relax_group<VM, 8, 0, 4>(tm, wv, vv, sc.s, t, em, st);
      if (__any_sync(FULL, hi4)) relax_group<VM, 8, 4, 4>(tm, wv, vv, sc.s, t, em, st);
    } else {
      relax_group<VM, K, 0, K>(tm, wv, vv, sc.s, t, em, st);
    }
    // append the members: ballots for one or two slots per lane, else a scan
    if constexpr (K <= 2) {
      const unsigned b0 = __ballot_sync(FULL, em & 1u);
      unsigned b1 = 0u;
      if constexpr (K == 2) b1 = __ballot_sync(FULL, em & 2u);
      const int tot = __popc(b0) + __popc(b1);
      if (tot) {
        const int base = append_base<TEAM>(ctl, level, tot, nq);
        if (em & 1u) *q_slot(tm, level + 1, nb, base + __popc(b0 & lt)) = wv[0];
        if constexpr (K == 2)
          if (em & 2u) *q_slot(tm, level + 1, nb, base + __popc(b0) + __popc(b1 & lt)) = wv[1];
      }
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
        int pos = append_base<TEAM>(ctl, level, tot, nq) + inc - cnt;
#pragma unroll
        for (int q = 0; q < K; q++)
          if ((em >> q) & 1u) *q_slot(tm, level + 1, nb, pos++) = wv[q];
      }
    }
    unsigned fm = __ballot_sync(FULL, fb);
    while (fm) {
      const int l = __ffs(fm) - 1;
      fm &= fm - 1;
      walk_row<VM, TEAM>(sc, tm, ctl, __shfl_sync(FULL, v, l), t, level, nb, nq, st, bad);
    }
  }
}

// The head level of class t (one warp): lane q < 8 relaxes slot q of t's
// record; first-reached vertices below t become the class's level 1, at the
// start of the odd-level queue (at most 8 entries).  Returns their number, or
// -1 when t has no record (its row is walked from the CSR by expand).
template <int VM>
__device__ __forceinline__ int expand_head(const TravArgs& a, const Src& sc, const Team& tm, int t, VState& st,
                                           unsigned long long& n_exp, unsigned long long& n_edge) {
  const int lane = threadIdx.x & 31;
  int w = t;
  bool none = sc.ell == nullptr && sc.ellw == nullptr;
  if (sc.ellw) {
    if (lane < 8) w = __ldg((const int*)(sc.ellw + 2 * (size_t)t) + lane);
    none = __shfl_sync(FULL, w, 0) < 0;  // sentinel
  } else if (sc.ell) {
    int off = 0;
    if (lane < 8) off = (int)__ldg((const short*)(sc.ell + t) + lane);
    none = __shfl_sync(FULL, off, 0) == -32768;  // sentinel
    w = t + off;                                 // offset 0 (empty slot): w == t
  }
  if (none) return -1;
  if (a.collect_stats && lane == 0) {
    n_exp++;
    n_edge += (unsigned long long)(__ldg(sc.rowptr + t + 1) - __ldg(sc.rowptr + t));
  }
  const bool pred = lane < 8 && w != t && w != sc.s;
  const uint32_t bit = 1u << (w & 31);
  const uint32_t old = v_or_if<VM>(tm, w, pred);
  bool member = false;
  if (!(old & bit)) {  // first reach (an OR not issued returns the bit)
    v_first<VM>(tm, w, old, st);
    member = w < t;
  }
  const unsigned m = __ballot_sync(FULL, member);
  if (member) tm.qb[__popc(m & ((1u << lane) - 1u))] = w;
  return __popc(m);
}

// Lanes per vertex from the level's length: a warp covers 32/LPV vertices per
// round (a team four times as many).
template <int VM, bool TEAM>
__device__ __forceinline__ void expand(const TravArgs& a, const Src& sc, const Team& tm, CtCtl* ctl, int t,
                                       int level, int64_t cb, int64_t nb, bool head, int qlen, int& nq, VState& st,
                                       unsigned long long& n_exp, unsigned long long& n_edge, int& bad) {
  constexpr int R = TEAM ? CT_WARPS : 1;
  if (qlen <= 4 * R)
    expand_level<VM, TEAM, 8>(a, sc, tm, ctl, t, level, cb, nb, head, qlen, nq, st, n_exp, n_edge, bad);
  else if (qlen <= 8 * R)
    expand_level<VM, TEAM, 4>(a, sc, tm, ctl, t, level, cb, nb, head, qlen, nq, st, n_exp, n_edge, bad);
  else if (qlen <= 16 * R)
    expand_level<VM, TEAM, 2>(a, sc, tm, ctl, t, level, cb, nb, head, qlen, nq, st, n_exp, n_edge, bad);
  else
    expand_level<VM, TEAM, 1>(a, sc, tm, ctl, t, level, cb, nb, head, qlen, nq, st, n_exp, n_edge, bad);
}

}  // namespace

namespace {

__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}
__device__ __forceinline__ int warp_min(int x) { return __reduce_min_sync(FULL, x); }
__device__ __forceinline__ int warp_max(int x) { return __reduce_max_sync(FULL, x); }

// Set bits of shared words [j0, j1) (word j0 masked by m0).  Warp-wide count.
__device__ int count_smem(const uint32_t* W, int j0, int j1, uint32_t m0, int lane) {
  int c = 0;
  for (int jb = j0; jb < j1; jb += 32) {
    const int j = jb + lane;
    uint32_t m = j < j1 ? W[j] : 0u;
    if (j == j0) m &= m0;
    c += __popc(m);
  }
  return warp_sum(c);
}

// Write, in increasing order from pool[pos], the vertices of the set bits of
// shared words [j0, j1) (word j0 masked by m0; word 0 is vertex base).
__device__ long long write_smem(const uint32_t* W, int base, int j0, int j1, uint32_t m0, uint32_t* pool,
                                long long pos, int lane) {
  for (int jb = j0; jb < j1; jb += 32) {
    const int j = jb + lane;
    uint32_t word = j < j1 ? W[j] : 0u;
    if (j == j0) word &= m0;
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
      pool[p++] = (uint32_t)(base + (j << 5) + b);
    }
    pos += __shfl_sync(FULL, inc, 31);
  }
  return pos;
}

// Set bits of the global slot from word ws on (ws masked by m0), through the
// summary up to summary word swmax.  count: returns the number; else writes
// them in increasing order from pool[pos] and returns the end position.
template <bool COUNT>
__device__ long long scan_global_words(const Team& tm, int ws, uint32_t m0, int swmax, uint32_t* pool,
                                       long long pos, int lane) {
  long long c = 0;
  for (int sw0 = ws >> 5; sw0 <= swmax; sw0 += 32) {
    const int sw = sw0 + lane;
    uint32_t sm = sw <= swmax ? ld_cg(tm.VS + sw) : 0u;
    if (sw == (ws >> 5)) sm &= 0xFFFFFFFFu << (ws & 31);
    unsigned any = __ballot_sync(FULL, sm != 0u);
    while (any) {
      const int l = __ffs(any) - 1;
      any &= any - 1;
      const uint32_t ml = __shfl_sync(FULL, sm, l);
      const int pw = ((sw0 + l) << 5) + lane;
      uint32_t word = ((ml >> lane) & 1u) ? ld_cg(tm.V + pw) : 0u;
      if (pw == ws) word &= m0;
      const int cw = __popc(word);
      if constexpr (COUNT) {
        c += warp_sum(cw);
      } else {
        int inc = cw;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int x = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += x;
        }
        long long p = pos + (inc - cw);
        while (word) {
          const int b = __ffs(word) - 1;
          word &= word - 1;
          pool[p++] = (uint32_t)((pw << 5) + b);
        }
        pos += __shfl_sync(FULL, inc, 31);
      }
    }
  }
  return COUNT ? c : pos;
}

// Emit the row of source s (one warp): [L cols | s | U cols] into the row pool
// at an atomically taken offset, plus the per-row counts.  swmax: the last
// summary word that may be nonzero (VM_GLOBAL).
template <int VM>
__device__ void emit_row(const TravArgs& a, const Src& sc, const Team& tm, int nL, int diag, int rb, int re,
                         int swmax) {
  const int lane = threadIdx.x & 31;
  const int s = sc.s;
  const uint32_t above = (s & 31) == 31 ? 0u : (0xFFFFFFFEu << (s & 31));  // bits above s in its word
  // count U(s,:)
  int nU = 1;
  if constexpr (VM == VM_SMEM) nU += count_smem(tm.V, s >> 5, (sc.n + 31) >> 5, above, lane);
  else nU += (int)scan_global_words<true>(tm, s >> 5, above, swmax, nullptr, 0, lane);
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
  // U(s,:) above the diagonal, in increasing order
  const long long pos = (long long)off + nL + 1;
  if constexpr (VM == VM_SMEM) write_smem(tm.V, 0, s >> 5, (sc.n + 31) >> 5, above, a.pool, pos, lane);
  else scan_global_words<false>(tm, s >> 5, above, swmax, a.pool, pos, lane);
}

// Clear the bits the source set (threads tid, tid + nthr, ...): shared words
// all, global words through the summary words in [swmin, swmax].
template <int VM>
__device__ __forceinline__ void clear_v(const Team& tm, int n, int swmin, int swmax, int tid, int nthr) {
  if constexpr (VM == VM_SMEM) {
    for (int j = tid; j < ((n + 31) >> 5); j += nthr) tm.V[j] = 0u;
  } else {
    if (swmin > swmax) return;  // no global bit was set
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

}  // namespace

namespace {

// Source of work item k (items in issue order, largest source first).
__device__ __forceinline__ Src source_of(const TravArgs& a, int k) {
  Src sc;
  sc.n = a.n;
  sc.rowptr = a.rowptr;
  sc.colidx = a.colidx;
  sc.ell = a.ell;
  sc.ellw = a.mats ? nullptr : a.ellw;
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

struct Counts {
  unsigned long long n_exp = 0, n_edge = 0, n_lev = 0;
  int bad = 0;
};

// The next class to expand from cursor on, retiring runs of clean heads on
// the way (ct_heads >= 0); -1 when no class is pending.  Adaptive mode
// (ct_heads == 0): after a gather whose first class was not clean, the next
// 1, 3, 7, 15 or 31 classes are taken one by one before the next gather.
template <int VM>
__device__ int next_expand(const TravArgs& a, const Src& sc, const Team& tm, int& cursor, int& nL, int& skip,
                           int& fails, int lane, Counts& cn) {
  for (;;) {
    const int t = next_class<VM>(tm, cursor, sc.s, lane);
    if (t < 0 || a.ct_heads < 0) return t;
    if (skip > 0) {
      skip--;
      return t;
    }
    int tn = -1, last = t;
    const int k = retire_clean<VM>(a, sc, tm, t, nL, lane, tn, last, cn.n_exp, cn.n_edge);
    nL += k;
    if (k == 0 && a.ct_heads == 0) {
      fails = fails < 5 ? fails + 1 : 5;
      skip = (1 << fails) - 1;
    } else if (k > 0) {
      fails = 0;
    }
    if (tn >= 0) return tn;
    cursor = last + 1;
  }
}

// One source from seeds to a cleared V.  TEAM: the whole CTA (warp 0 searches
// classes, expands their heads and emits), else the calling warp.
template <int VM, bool TEAM>
__device__ void run_source(const TravArgs& a, const Src& sc, const Team& tm, CtCtl* ctl, Counts& cn) {
  const int lane = threadIdx.x & 31;
  const int nthr = TEAM ? CT_THREADS : 32;
  const int tid = TEAM ? (int)threadIdx.x : lane;
  const bool leader = !TEAM || threadIdx.x < 32;
  const int s = sc.s;
  VState st;
  st.smin = 0x7FFFFFFF;
  st.smax = -1;

  // seeds: neighbours below s are classes with maxId -1; above s, U entries
  const int rb = __ldg(sc.rowptr + s), re = __ldg(sc.rowptr + s + 1);
  int diag = 0;
  int wmin = 0x7FFFFFFF;  // the first class: no vertex below it is reached yet
  for (int e = rb + tid; e < re; e += nthr) {
    const int w = __ldg(sc.colidx + e);
    if ((unsigned)w >= (unsigned)sc.n) { cn.bad = 1; continue; }
    if (w == s) { diag = 1; continue; }
    if (w < s) wmin = min(wmin, w);
    v_set<VM>(tm, w, st);
  }
  wmin = __reduce_min_sync(FULL, wmin);
  if constexpr (TEAM) {
    if (lane == 0) atomicMin(&ctl->cmin, wmin);
    diag = __syncthreads_or(diag);
    wmin = ctl->cmin;
  } else {
    diag = __any_sync(FULL, diag);
    __syncwarp();
  }

  int cursor = wmin < s ? wmin : s, nL = 0;
  int skip = 0, fails = 0;  // clean-head gathers (leader only)
  int level = 0;  // team mode: running level index (queues and counters rotate with it)
  for (;;) {
    int t;
    if constexpr (TEAM) {
      // warp 0 finds the class and expands its head (t alone) into the next
      // level; the counter it fills and the one it zeroes are not the one the
      // other warps may still be reading (the last level's zero length)
      if (leader) {
        t = next_expand<VM>(a, sc, tm, cursor, nL, skip, fails, lane, cn);
        int nq = 0;
        if (t >= 0) {
          if (lane == 0) *l_slot(tm, nL) = t;
          // the class's levels overflow into the log from its bottom
          expand<VM, false>(a, sc, tm, ctl, t, level, 0, 0, true, 1, nq, st, cn.n_exp, cn.n_edge, cn.bad);
          cn.n_lev++;
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
        if (leader) cn.n_lev++;
        if (threadIdx.x == 0) ctl->qcnt[(level + 2) % 3] = 0;
        int nq_unused = 0;
        const int64_t nb = next_base(tm, cb, qlen);
        expand<VM, true>(a, sc, tm, ctl, t, level, cb, nb, false, qlen, nq_unused, st, cn.n_exp, cn.n_edge, cn.bad);
        cb = nb;
        __syncthreads();
      }
    } else {
      t = next_expand<VM>(a, sc, tm, cursor, nL, skip, fails, lane, cn);
      if (t < 0) break;
      cursor = t + 1;
      if (lane == 0) *l_slot(tm, nL) = t;
      nL++;
      // shared bitmaps: the head level (t alone) by its record's eight lanes,
      // where most classes end; otherwise (or without a record) the general
      // level code takes the head too (one call site keeps the kernel small)
      int qlen = -1;
      if constexpr (VM == VM_SMEM) {
        qlen = expand_head<VM>(a, sc, tm, t, st, cn.n_exp, cn.n_edge);
        if (qlen >= 0) cn.n_lev++;
        __syncwarp();
      }
      const bool head = qlen < 0;
      if (head) qlen = 1;
      int64_t cb = 0;  // the class's levels overflow into the log from its bottom
      for (int lv = head ? 0 : 1; qlen > 0; lv++) {
        int nq = 0;
        cn.n_lev++;
        const int64_t nb = lv == 0 ? 0 : next_base(tm, cb, qlen);
        expand<VM, false>(a, sc, tm, ctl, t, lv, cb, nb, lv == 0, qlen, nq, st, cn.n_exp, cn.n_edge, cn.bad);
        __syncwarp();
        cb = nb;
        qlen = nq;
      }
    }
  }

  // the summary words this source touched
  int swmin = st.smin, swmax = st.smax;
  if constexpr (VM == VM_GLOBAL) {
    swmin = warp_min(st.smin);
    swmax = warp_max(st.smax);
    if constexpr (TEAM) {
      if (threadIdx.x == 0) { ctl->smin = 0x7FFFFFFF; ctl->smax = -1; }
      __syncthreads();
      if (lane == 0) { atomicMin(&ctl->smin, swmin); atomicMax(&ctl->smax, swmax); }
      __syncthreads();
      swmin = ctl->smin;
      swmax = ctl->smax;
    }
  }
  if (leader) emit_row<VM>(a, sc, tm, nL, diag, rb, re, swmax);
  if constexpr (TEAM) __syncthreads();
  else __syncwarp();
  clear_v<VM>(tm, sc.n, swmin, swmax, tid, nthr);
  if constexpr (TEAM) __syncthreads();
  else __syncwarp();
}

// Shared memory: control blocks (one per warp; team mode uses warp 0's), two
// queues of qw entries per warp, then (VM_SMEM) vwords bitmap words per warp.
__host__ __device__ __forceinline__ size_t ct_smem_bytes(int vm, int vwords, int qw) {
  return (size_t)CT_WARPS * 64 + (size_t)2 * CT_WARPS * qw * 4 +
         (vm != VM_GLOBAL ? (size_t)CT_WARPS * vwords * 4 : 0);
}

}  // namespace

// MINB: CTAs of four warps per SM the register budget is sized for.  TEAMS:
// the build with the CTA-team phase (only launched when ct_nbig > 0, so the
// default build carries no team code).
template <int VM, int MINB, bool TEAMS>
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

  if constexpr (VM != VM_GLOBAL) {
    for (int j = threadIdx.x; j < CT_WARPS * vwords; j += CT_THREADS) vsh[j] = 0u;
    __syncthreads();
  }
  Counts cn;

  // ---- team phase: the first nbig items, one CTA per source
  if (TEAMS && a.ct_nbig > 0) {
    const size_t slot = (size_t)blockIdx.x * CT_WARPS;
    Team tm;
    tm.V = VM == VM_SMEM ? vsh : a.g_V + slot * (gcap / 32);
    tm.VS = a.g_VS + slot * (gcap / 1024);
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
        ctl->cmin = 0x7FFFFFFF;
      }
      __syncthreads();
      const int k = ctl->src;
      if (k < 0) break;
      run_source<VM, true>(a, source_of(a, k), tm, ctl, cn);
    }
    __syncthreads();
  }

  // ---- warp phase: every other item, one warp per source
  if ((long long)blockIdx.x * CT_WARPS + warp < a.g_slots) {
    const size_t slot = (size_t)blockIdx.x * CT_WARPS + warp;
    Team tm;
    tm.V = VM == VM_SMEM ? vsh + (size_t)warp * vwords : a.g_V + slot * (gcap / 32);
    tm.VS = a.g_VS + slot * (gcap / 1024);
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
      run_source<VM, false>(a, source_of(a, k), tm, ctl, cn);
    }
  }

  if (cn.bad) atomicOr(&a.ctr->err, ERR_COL_RANGE);
  unsigned long long n_exp = cn.n_exp, n_edge = cn.n_edge;
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
    atomicAdd(&a.ctr->levels, cn.n_lev);
  }
}

size_t trav_class_smem(int vm, int vwords, int qw) { return ct_smem_bytes(vm, vwords, qw); }

namespace {
template <int VM, int MINB, bool TEAMS>
cudaError_t launch_one(const TravArgs& a, int grid, size_t smem, cudaStream_t st) {
  static int attr_set[128] = {0};  // per device: the dynamic shared-memory limit was raised
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 128 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(trav_class_kernel<VM, MINB, TEAMS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[dev] = 1;
  }
  trav_class_kernel<VM, MINB, TEAMS><<<grid, CT_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

template <int VM, int MINB>
int occupancy_one(size_t smem) {
  // answers are cached per (device, shared-memory size): the query is made on
  // every plan and every server admission
  static std::mutex mu;
  static std::map<std::tuple<int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, smem});
    if (it != cache.end()) return it->second;
  }
  cudaFuncSetAttribute(trav_class_kernel<VM, MINB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trav_class_kernel<VM, MINB, false>, CT_THREADS, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[{dev, smem}] = occ;
  return occ;
}

template <int VM>
int occupancy_vm(int warps_per_sm, size_t smem) {
  return warps_per_sm > 32 ? occupancy_one<VM, 10>(smem) : occupancy_one<VM, 8>(smem);
}

template <int VM>
cudaError_t launch_vm(const TravArgs& a, int grid, int warps_per_sm, size_t smem, cudaStream_t st) {
  if (a.ct_nbig > 0) return launch_one<VM, 8, true>(a, grid, smem, st);  // teams: the 64-register build
  return warps_per_sm > 32 ? launch_one<VM, 10, false>(a, grid, smem, st) : launch_one<VM, 8, false>(a, grid, smem, st);
}
}  // namespace

// CTAs of four warps per SM the class kernel reaches with this shared memory;
// warps_per_sm above 32 selects the 48-register build.
int trav_class_occupancy(int vm, int warps_per_sm, int vwords, int qw) {
  const size_t smem = ct_smem_bytes(vm, vwords, qw);
  if (smem > 227 * 1024) return 0;
  if (vm == VM_SMEM) return occupancy_vm<VM_SMEM>(warps_per_sm, smem);
  return occupancy_vm<VM_GLOBAL>(warps_per_sm, smem);
}

cudaError_t launch_trav_class(const TravArgs& a, int grid, int vm, int warps_per_sm, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  const size_t smem = ct_smem_bytes(vm, a.ct_vwords, a.ct_qw);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (vm == VM_SMEM) return launch_vm<VM_SMEM>(a, grid, warps_per_sm, smem, st);
  return launch_vm<VM_GLOBAL>(a, grid, warps_per_sm, smem, st);
}

}  // namespace gsofa
