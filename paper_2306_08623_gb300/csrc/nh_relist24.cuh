// nh_relist24.cuh -- re-listing of (2,4) over the per-edge triangle lists (part of nh_peel.cuh).
//
// The 4-cliques containing edge R = (a,b) are the adjacent pairs {w, x} of R's triangle list
// T(R) (the common neighbours of a and b; Alg. 3's re-listing step for s - r = 2).  Each pair is
// found once through the orientation: x in N+(w).  With the round stamps (peel) or core numbers
// (two-phase hierarchy) of the edges {a,y}, {b,y} of every candidate y known, most candidates can
// be dropped before any pair is formed:
//   - peel (core numbers only, or the approximate peel): an s-clique with a member peeled in an
//     earlier round is already dead, and one whose member of least id in the frontier is not R
//     belongs to that member; R needs neither, so a candidate y whose edge {a,y} or {b,y} was
//     peeled earlier or is in the frontier with a smaller id takes part in no s-clique R handles;
//   - two-phase hierarchy at level c (core of R): an s-clique joins its members at level c only
//     when every member has core >= c, and only its member of least id among those of core c
//     performs the unions; the label hierarchy also needs to know whether R lies in any s-clique
//     at its own level, so it keeps candidates that only fail the least-id test (flag kSpoil).
// The remaining (live) candidates are staged in shared memory in list order -- flags, out-list
// start and length, and an open-addressing hash of vertex ids to positions -- in one pass that
// keeps several loads in flight per thread.  Every live w then scans its out-list N+(w) and
// tests each entry x against the hash; the scans of all staged w's form one index space (a
// prefix sum of the out-list lengths over the positions), which the warps cut into steps of 32
// entries.  The decrements (or unions) of the members {a,y}, {b,y} are summed per staged
// candidate, over both of its roles (as w and as x), and applied once per candidate; only the
// member {w,x} is decremented per s-clique.
//
// Work split: the r-cliques of a frontier (or level) are cut into sub-tasks.  A sub-task stages
// the whole live candidate set of its r-clique and takes one range of the scan index space
// (positions are in list order, so every sub-task of an r-clique stages the same positions and
// the same index space); the number of sub-tasks per r-clique grows with its precomputed scan
// bound (list length plus the sum of d+(w) over the list) relative to the round's total and to the
// warps of the grid, so a round that peels a few dense edges spreads their scans over the grid
// and a round of many short lists keeps one task per r-clique.  Warps take sub-tasks from a
// shared counter; a sub-task whose list is longer than a warp's staging area goes to a queue
// that whole blocks then take.  A block stages up to kC24BlockCap live candidates; when an
// r-clique has more, it falls back to slabs of consecutive list entries, each staged in turn
// while every w of the sub-task's list range scans against it.  Every wait is bounded.
#pragma once

namespace nhp {

constexpr int kC24WarpHS = 512;   // hash slots of a warp's staging area
constexpr int kC24WarpCap = 256;  // longest list a warp takes (and live candidates it stages)
constexpr int kC24BlockHS = 4096;
constexpr int kC24BlockCap = 2048;  // live candidates a block stages at once
// area layout: key i32[HS], ob u32[cap] (out-list start of a position's w), meta u32[cap],
// epre u32[cap] (inclusive prefix of the out-list lengths), pos u16[HS]
constexpr int c24_area_bytes(int hs, int cap) { return hs * 4 + cap * 12 + hs * 2; }
constexpr int kC24WarpBytes = c24_area_bytes(kC24WarpHS, kC24WarpCap);
constexpr int kC24BlockBytes = c24_area_bytes(kC24BlockHS, kC24BlockCap);
static_assert(kC24WarpBytes * (kThreads / 32) == kC24BlockBytes, "warp areas tile the block area");
constexpr int kC24U = 4;              // list entries per thread in one staging step
constexpr int kC24MaxSplit = 0xffff;  // sub-tasks per r-clique (16 bits of a queue entry)
constexpr int64_t kC24MaxRel = 0xffff;  // list positions kept in meta (16 bits)
constexpr uint32_t kC24AccMax = 0x1fff;  // s-cliques summed per staged candidate (13 bits)
// dynamic shared memory of a kernel running this re-listing: the staging area, the sub-task
// prefix sums of a frontier of at most kTaskItems r-cliques, per warp 32 w-side accumulators (slab
// mode), then the small words: 16 reduction words, 9 compaction counters, per-warp compaction
// counts of one staging step, a broadcast word
constexpr int kC24Pref = kC24BlockBytes;
constexpr int kC24Wacc = kC24Pref + kTaskItems * 4;
constexpr int kC24Cnt = kC24Wacc + (kThreads / 32) * 32 * 4;
constexpr int kC24Red = kC24Cnt;                                  // u64[16]
constexpr int kC24Tcnt = kC24Red + 16 * 8;                        // int[16]
constexpr int kC24Wcnt = kC24Tcnt + 16 * 4;                       // int[kC24U * 8]
constexpr int kC24Bcast = kC24Wcnt + kC24U * (kThreads / 32) * 4;  // u64
constexpr int kC24SmemBytes = kC24Bcast + 8;

// meta word of a staged candidate: list position (bits 16..31; in slab mode relative to the
// slab), flags (13..15), count of s-cliques handled through it (0..12)
constexpr uint32_t kDecA = 1u << 13;   // decrement {a,y} (it is live and outside the frontier)
constexpr uint32_t kDecB = 1u << 14;   // decrement {b,y}
constexpr uint32_t kSpoil = 1u << 15;  // y's s-cliques are not R's to unite (label hierarchy only)

struct C24Area {
  int32_t* key;
  uint32_t* ob;
  uint32_t* meta;
  uint32_t* epre;
  uint16_t* pos;
  int hs, lg, cap;
};

__device__ __forceinline__ C24Area c24_area(unsigned char* base, int hs, int lg, int cap) {
  C24Area G;
  G.key = reinterpret_cast<int32_t*>(base);
  G.ob = reinterpret_cast<uint32_t*>(base + 4 * hs);
  G.meta = reinterpret_cast<uint32_t*>(base + 4 * hs + 4 * cap);
  G.epre = reinterpret_cast<uint32_t*>(base + 4 * hs + 8 * cap);
  G.pos = reinterpret_cast<uint16_t*>(base + 4 * hs + 12 * cap);
  G.hs = hs;
  G.lg = lg;
  G.cap = cap;
  return G;
}

__device__ __forceinline__ uint32_t c24_slot(int32_t y, int lg) {
  return ((uint32_t)y * 0x9E3779B1u) >> (32 - lg);  // Fibonacci hashing of the vertex id
}

// position of vertex x among the staged candidates, or -1
__device__ __forceinline__ int c24_find(const C24Area& G, int32_t x) {
  uint32_t h = c24_slot(x, G.lg);
  for (int it = 0; it < G.hs; ++it) {
    const int32_t k = G.key[h];
    if (k == x) return G.pos[h];
    if (k == -1) return -1;
    h = (h + 1) & (uint32_t)(G.hs - 1);
  }
  return -1;
}

// Classification of a candidate from the values of its edges {a,y} (ea, va) and {b,y} (eb, vb):
// round stamps (peel) or core numbers / labels (hierarchy), see the file comment; false drops it.
__device__ __forceinline__ bool c24_keep(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr, int32_t ea,
                                         int32_t eb, uint32_t va, uint32_t vb, uint32_t& fl) {
  fl = 0;
  if (A.union_mode) {
    if (va < thr || vb < thr) return false;
    if ((va == thr && ea < Rid) || (vb == thr && eb < Rid)) {
      if (!A.mark) return false;
      fl = kSpoil;
    }
    return true;
  }
  if ((va != 0u && va < t) || (vb != 0u && vb < t)) return false;  // dead
  if ((va == t && ea < Rid) || (vb == t && eb < Rid)) return false;  // another member's
  fl = ((va == 0u || va > t) ? kDecA : 0u) | ((vb == 0u || vb > t) ? kDecB : 0u);
  return true;
}

__device__ __forceinline__ const uint32_t* c24_vals(const PeelArgs& A) { return A.union_mode ? A.val : A.round; }

// count decrement by n (exact: Alg. 3; approximate: Alg. 2); true when the count crossed to <= thr,
// after which the caller appends x to the next frontier
template <bool EXACT>
__device__ __forceinline__ bool c24_dec(const PeelArgs& A, int32_t x, uint32_t n, uint32_t t, uint32_t thr,
                                        LocalStats& ls) {
  const uint32_t old = atomicSub(A.cnt + x, n);
  ls.dec++;
  if (old > thr && (unsigned long long)old <= (unsigned long long)thr + n) {
    __stcg(A.round + x, t + 1u);
    __stcg(A.val + x, EXACT ? thr : min(thr, __ldg(A.cnt0 + x)));
    return true;
  }
  return false;
}

__device__ __forceinline__ void c24_unite(const PeelArgs& A, int32_t a, int32_t b, LocalStats& ls) {
  const int32_t child = uf_unite(A.lk.uf, a, b, A.lk.ctl);
  if (child >= 0) {
    ls.unite++;
    const unsigned long long pos = atomicAdd(A.touched_n, 2ull);
    if (pos + 1 < A.touched_cap) {
      A.touched[pos] = child;
      A.touched[pos + 1] = uf_find(A.lk.uf, child);
    } else {
      atomicCAS(&A.lk.ctl->err, 0, NH_ERR_OVERFLOW);
    }
  }
}

// applies the n s-cliques counted through the candidate at list entry j (its edges {a,y}, {b,y}):
// decrements (peel) or unions (hierarchy); warp-collective (appends crossings)
template <bool EXACT>
__device__ __forceinline__ void c24_apply(const PeelArgs& A, int64_t j, uint32_t fl, uint32_t n, int32_t Rid,
                                          uint32_t t, uint32_t thr, int32_t* nf, int lane, LocalStats& ls) {
  int32_t ea = 0, eb = 0;
  bool ca = false, cb = false;
  if (n > 0) {
    ea = __ldg(A.g.t2ea + j);
    eb = __ldg(A.g.t2eb + j);
    ls.scan += 2;
    if (A.union_mode) {
      c24_unite(A, Rid, ea, ls);
      c24_unite(A, Rid, eb, ls);
    } else {
      if (fl & kDecA) ca = c24_dec<EXACT>(A, ea, n, t, thr, ls);
      if (fl & kDecB) cb = c24_dec<EXACT>(A, eb, n, t, thr, ls);
    }
  }
  if (!A.union_mode) {
    unsigned long long p = warp_append(&A.lk.ctl->nf_count, ca, lane);
    if (ca) nf[p] = ea;
    p = warp_append(&A.lk.ctl->nf_count, cb, lane);
    if (cb) nf[p] = eb;
  }
}

template <bool BLOCK>
__device__ __forceinline__ void c24_sync() {
  if (BLOCK) __syncthreads(); else __syncwarp();
}

// Stages the live candidates among list entries [j0, j0 + cnt) of the list at lo, at the next
// positions, in list order; meta position = entry index - rel0.  Positions at or beyond the
// area's capacity are counted but not written (the caller sees the overflow in *tcnt).  The
// team's hash keys must be cleared and *tcnt set before the first call.  Team-collective; wcnt
// (block teams) holds kC24U * 8 counts.
template <bool BLOCK>
__device__ __forceinline__ void c24_stage(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr, int64_t lo,
                                          int64_t j0, int64_t cnt, int64_t rel0, const C24Area& G, int* tcnt,
                                          int* wcnt, LocalStats& ls) {
  constexpr int TEAM = BLOCK ? kThreads : 32;
  const int tid = BLOCK ? (int)threadIdx.x : (int)(threadIdx.x & 31);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const uint32_t* vals = c24_vals(A);
  for (int64_t s0 = 0; s0 < cnt; s0 += (int64_t)TEAM * kC24U) {
    int32_t ea[kC24U], eb[kC24U];
    uint32_t va[kC24U], vb[kC24U];
#pragma unroll
    for (int u = 0; u < kC24U; u++) {
      const int64_t i = s0 + (int64_t)u * TEAM + tid;
      ea[u] = eb[u] = 0;
      if (i < cnt) {
        ea[u] = __ldg(A.g.t2ea + lo + j0 + i);
        eb[u] = __ldg(A.g.t2eb + lo + j0 + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kC24U; u++) {
      const int64_t i = s0 + (int64_t)u * TEAM + tid;
      va[u] = vb[u] = 0;
      if (i < cnt) {
        va[u] = __ldcg(vals + ea[u]);
        vb[u] = __ldcg(vals + eb[u]);
      }
    }
    uint32_t fl[kC24U];
    unsigned mk[kC24U];
    int32_t wv[kC24U];
#pragma unroll
    for (int u = 0; u < kC24U; u++) {
      const int64_t i = s0 + (int64_t)u * TEAM + tid;
      const bool keep = i < cnt && c24_keep(A, Rid, t, thr, ea[u], eb[u], va[u], vb[u], fl[u]);
      mk[u] = __ballot_sync(NH_FULL, keep);
      wv[u] = keep ? __ldg(A.g.t2w + lo + j0 + i) : 0;
      if (i < cnt) {
        ls.scan += 2;
        ls.stamp += 2;
      }
    }
    // positions in list order: step entry i = u * TEAM + tid, so (u, warp, lane) lexicographically
    int base[kC24U];
    if (BLOCK) {
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < kC24U; u++) wcnt[u * (kThreads / 32) + wib] = __popc(mk[u]);
      }
      __syncthreads();
      int run = *tcnt;
#pragma unroll
      for (int u = 0; u < kC24U; u++) {
        int b = run;
        for (int w = 0; w < kThreads / 32; w++) {
          const int c = wcnt[u * (kThreads / 32) + w];
          if (w < wib) b += c;
          run += c;
        }
        base[u] = b;
      }
      __syncthreads();  // every thread has read *tcnt and wcnt
      if (threadIdx.x == 0) *tcnt = run;
    } else {
      int run = *tcnt;
#pragma unroll
      for (int u = 0; u < kC24U; u++) {
        base[u] = run;
        run += __popc(mk[u]);
      }
      __syncwarp();
      if (lane == 0) *tcnt = run;
    }
    int64_t o0[kC24U], o1[kC24U];
#pragma unroll
    for (int u = 0; u < kC24U; u++) {
      o0[u] = o1[u] = 0;
      if ((mk[u] >> lane) & 1u) {
        o0[u] = __ldg(A.g.ooff + wv[u]);
        o1[u] = __ldg(A.g.ooff + wv[u] + 1);
        ls.scan += 4;
      }
    }
#pragma unroll
    for (int u = 0; u < kC24U; u++) {
      if (!((mk[u] >> lane) & 1u)) continue;
      const int p = base[u] + __popc(mk[u] & ((1u << lane) - 1u));
      if (p >= G.cap) continue;
      const int64_t i = s0 + (int64_t)u * TEAM + tid;
      G.meta[p] = ((uint32_t)(j0 + i - rel0) << 16) | fl[u];
      G.ob[p] = (uint32_t)o0[u];
      G.epre[p] = (uint32_t)(o1[u] - o0[u]);
      uint32_t h = c24_slot(wv[u], G.lg);
      for (int it = 0; it < G.hs && atomicCAS(&G.key[h], -1, wv[u]) != -1; ++it) h = (h + 1) & (uint32_t)(G.hs - 1);
      G.pos[h] = (uint16_t)p;
    }
    c24_sync<BLOCK>();
  }
}

// The s-clique {a, b, w, x} of a scan entry whose x is staged at position px, given its edge e =
// {w, x} and e's round stamp (peel) or core number (hierarchy) v.  Peel: if it is live and R's, it
// is counted on x's staged position and on *wslot (w's position, or a w-side accumulator), and e
// is decremented at once (cross: a crossing to append); with xdirect the x side is decremented at
// once as well (cxa / xa, cxb / xb).  Hierarchy: unions with e and marks on the positions.
template <bool EXACT>
__device__ __forceinline__ void c24_pair_apply(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr,
                                               const C24Area& G, int px, int32_t e, uint32_t v, uint32_t wfl,
                                               uint32_t* wslot, bool xdirect, int64_t xrel_base, bool& in_level,
                                               bool& cross, bool& cxa, int32_t& xa, bool& cxb, int32_t& xb,
                                               LocalStats& ls) {
  if (A.union_mode) {
    if (v >= thr) {
      in_level = true;
      if (!(wfl & kSpoil) && !(G.meta[px] & kSpoil) && !(v == thr && e < Rid)) {
        ls.listed++;
        atomicOr(wslot, 1u);
        atomicOr(&G.meta[px], 1u);
        c24_unite(A, Rid, e, ls);
      }
    }
    return;
  }
  if ((v != 0u && v < t) || (v == t && e < Rid)) return;
  ls.listed++;
  atomicAdd(wslot, 1u);
  if (!xdirect) {
    atomicAdd(&G.meta[px], 1u);
  } else {  // the x side per s-clique (its sums could exceed the meta field)
    const uint32_t mx = G.meta[px];
    const int64_t jx = xrel_base + (mx >> 16);
    xa = __ldg(A.g.t2ea + jx);
    xb = __ldg(A.g.t2eb + jx);
    if (mx & kDecA) cxa = c24_dec<EXACT>(A, xa, 1u, t, thr, ls);
    if (mx & kDecB) cxb = c24_dec<EXACT>(A, xb, 1u, t, thr, ls);
  }
  if (v == 0u || v > t) cross = c24_dec<EXACT>(A, e, 1u, t, thr, ls);
}

// One scan entry q of the out-list of a w (flags wfl), see c24_pair_apply.
template <bool EXACT>
__device__ __forceinline__ void c24_pair(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr, const C24Area& G,
                                         int64_t q, uint32_t wfl, uint32_t* wslot, bool xdirect, int64_t xrel_base,
                                         bool& in_level, bool& cross, int32_t& e, bool& cxa, int32_t& xa, bool& cxb,
                                         int32_t& xb, LocalStats& ls) {
  const int32_t x = __ldg(A.g.oadj + q);
  const int32_t eq = __ldg(A.g.oeid + q);
  ls.scan += 2;
  ls.expand++;
  const int px = c24_find(G, x);
  if (px < 0) return;
  e = eq;
  ls.stamp++;
  const uint32_t v = __ldcg(c24_vals(A) + e);
  c24_pair_apply<EXACT>(A, Rid, t, thr, G, px, e, v, wfl, wslot, xdirect, xrel_base, in_level, cross, cxa, xa, cxb,
                        xb, ls);
}

// appends this step's crossings to the next frontier (warp-collective)
__device__ __forceinline__ void c24_append(const PeelArgs& A, int32_t* nf, bool xdirect, bool cross, int32_t e,
                                           bool cxa, int32_t xa, bool cxb, int32_t xb) {
  if (A.union_mode) return;
  const int lane = threadIdx.x & 31;
  unsigned long long p = warp_append(&A.lk.ctl->nf_count, cross, lane);
  if (cross) nf[p] = e;
  if (xdirect) {
    p = warp_append(&A.lk.ctl->nf_count, cxa, lane);
    if (cxa) nf[p] = xa;
    p = warp_append(&A.lk.ctl->nf_count, cxb, lane);
    if (cxb) nf[p] = xb;
  }
}

// One step of 32 scan entries of the out-lists of up to 32 w's (one per lane: out-list start ob,
// length dlen, flags wfl, inclusive prefix incl of the lengths), the w-side sums in wacc[lane]
// (slab mode).  Warp-collective.
template <bool EXACT>
__device__ __forceinline__ void c24_pairs(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr, int32_t* nf,
                                          const C24Area& G, uint32_t idx, uint32_t total, uint32_t incl,
                                          uint32_t dlen, int64_t ob, uint32_t wfl, uint32_t* wacc, bool xdirect,
                                          int64_t xrel_base, bool& in_level, LocalStats& ls) {
  int own = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t v = __shfl_sync(NH_FULL, incl, own + step - 1);
    if (v <= idx) own += step;
  }
  const int64_t oob = __shfl_sync(NH_FULL, ob, own);
  const uint32_t oincl = __shfl_sync(NH_FULL, incl, own);
  const uint32_t olen = __shfl_sync(NH_FULL, dlen, own);
  const uint32_t ofl = __shfl_sync(NH_FULL, wfl, own);
  bool cross = false, cxa = false, cxb = false;
  int32_t e = 0, xa = 0, xb = 0;
  if (idx < total)
    c24_pair<EXACT>(A, Rid, t, thr, G, oob + (int64_t)(idx - (oincl - olen)), ofl, &wacc[own], xdirect, xrel_base,
                    in_level, cross, e, cxa, xa, cxb, xb, ls);
  c24_append(A, nf, xdirect, cross, e, cxa, xa, cxb, xb);
}

// inclusive prefix of 32 lanes' values and its total (warp-collective)
__device__ __forceinline__ uint32_t c24_scan(uint32_t v, uint32_t& total) {
  const int lane = threadIdx.x & 31;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(NH_FULL, incl, d);
    if (lane >= d) incl += o;
  }
  total = __shfl_sync(NH_FULL, incl, 31);
  return incl;
}

// epre[0, nc) <- inclusive prefix sums of its entries (nc <= 8 * TEAM); returns the total.
// Team-collective; red: 8 words (block teams).
template <bool BLOCK>
__device__ __forceinline__ uint32_t c24_team_scan(uint32_t* epre, int nc, unsigned long long* red) {
  constexpr int TEAM = BLOCK ? kThreads : 32;
  const int tid = BLOCK ? (int)threadIdx.x : (int)(threadIdx.x & 31);
  const int lane = threadIdx.x & 31;
  static_assert(8 * kThreads >= kC24BlockCap && 8 * 32 >= kC24WarpCap, "8 positions per thread");
  const int b = tid * 8;
  uint32_t v[8];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    v[j] = (b + j < nc) ? epre[b + j] : 0u;
    sum += v[j];
  }
  uint32_t tot;
  uint32_t incl = c24_scan(sum, tot);
  uint32_t base = incl - sum;
  if (BLOCK) {
    if (lane == 31) red[threadIdx.x >> 5] = incl;
    __syncthreads();
    tot = 0;
    for (int w = 0; w < kThreads / 32; w++) {
      const uint32_t x = (uint32_t)red[w];
      if (w < (int)(threadIdx.x >> 5)) base += x;
      tot += x;
    }
  }
#pragma unroll
  for (int j = 0; j < 8; j++) {
    base += v[j];
    if (b + j < nc) epre[b + j] = base;
  }
  c24_sync<BLOCK>();
  return tot;
}

// flushes the sums of staged positions [0, nc) (list entry of position p: jbase + its meta
// position); skip: positions hold no sums.  Team-collective.
template <bool EXACT, bool BLOCK>
__device__ __forceinline__ void c24_flush(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr, int32_t* nf,
                                          const C24Area& G, int nc, int64_t jbase, bool skip, LocalStats& ls) {
  constexpr int TEAM = BLOCK ? kThreads : 32;
  const int tid = BLOCK ? (int)threadIdx.x : (int)(threadIdx.x & 31);
  const int lane = threadIdx.x & 31;
  for (int p0 = 0; p0 < nc; p0 += TEAM) {
    const int p = p0 + tid;
    const uint32_t mt = p < nc ? G.meta[p] : 0u;
    const uint32_t n = skip ? 0u : (mt & kC24AccMax);
    c24_apply<EXACT>(A, jbase + (mt >> 16), mt, n, Rid, t, thr, nf, lane, ls);
  }
}

// Re-lists sub-task `sub` of `nsub` of R's 4-cliques with one team: a warp (BLOCK = false, list
// length <= kC24WarpCap) or the whole block.  All threads of the team call it with the same
// arguments.
template <bool EXACT, bool BLOCK>
__device__ void c24_item(const PeelArgs& A, int32_t Rid, int sub, int nsub, uint32_t t, uint32_t thr, int32_t* nf,
                         const C24Area& G, uint32_t* wacc, int* tcnt, int* wcnt, unsigned long long* red,
                         LocalStats& ls) {
  constexpr int TEAM = BLOCK ? kThreads : 32;
  const int tid = BLOCK ? (int)threadIdx.x : (int)(threadIdx.x & 31);
  const int lane = threadIdx.x & 31;
  const int wit = BLOCK ? (int)(threadIdx.x >> 5) : 0;
  const GView& g = A.g;
  const int64_t lo = __ldg(g.t2off + Rid);
  const int64_t len = __ldg(g.t2off + Rid + 1) - lo;
  bool in_level = false;  // label hierarchy: R lies in an s-clique whose members all reach its label
  // stage every live candidate of the list when they fit the area
  int nc = G.cap + 1;
  if (len <= kC24MaxRel) {
    for (int i = tid; i < G.hs; i += TEAM) G.key[i] = -1;
    if (tid == 0) *tcnt = 0;
    c24_sync<BLOCK>();
    c24_stage<BLOCK>(A, Rid, t, thr, lo, 0, len, 0, G, tcnt, wcnt, ls);
    nc = *tcnt;
  }
  if (nc <= G.cap) {
    // the scan index space of the staged w's; this sub-task's range [x0, x1) (multiples of 32)
    const uint32_t E = c24_team_scan<BLOCK>(G.epre, nc, red);
    const uint32_t xstep = (uint32_t)((((unsigned long long)E + nsub - 1) / nsub + 31) & ~31ull);
    const unsigned long long xa0 = (unsigned long long)sub * xstep;
    const uint32_t x0 = xa0 < E ? (uint32_t)xa0 : E;
    const uint32_t x1 = x0 + xstep < E ? x0 + xstep : E;
    // two scan entries per lane and step, their loads issued together
    const uint32_t* vals = c24_vals(A);
    for (uint32_t cb = x0 + (uint32_t)wit * 64; cb < x1; cb += 2 * TEAM) {
      int pw[2], px[2];
      int32_t e[2];
      uint32_t v[2];
      int64_t q[2];
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const uint32_t idx = cb + 32 * k + lane;
        pw[k] = -1;
        q[k] = 0;
        if (idx < x1) {
          int plo = 0, phi = nc;  // first position whose inclusive prefix exceeds idx
          while (plo < phi) {
            const int mid = (plo + phi) >> 1;
            if (G.epre[mid] <= idx) plo = mid + 1; else phi = mid;
          }
          pw[k] = plo;
          q[k] = (int64_t)G.ob[plo] + (idx - (plo ? G.epre[plo - 1] : 0u));
        }
      }
      int32_t xv[2];
#pragma unroll
      for (int k = 0; k < 2; k++) {
        xv[k] = 0;
        e[k] = 0;
        if (pw[k] >= 0) {
          xv[k] = __ldg(A.g.oadj + q[k]);
          e[k] = __ldg(A.g.oeid + q[k]);
          ls.scan += 2;
          ls.expand++;
        }
      }
#pragma unroll
      for (int k = 0; k < 2; k++) {
        px[k] = pw[k] >= 0 ? c24_find(G, xv[k]) : -1;
        v[k] = 0;
        if (px[k] >= 0) {
          v[k] = __ldcg(vals + e[k]);
          ls.stamp++;
        }
      }
      bool cross[2] = {false, false};
#pragma unroll
      for (int k = 0; k < 2; k++) {
        bool cxa = false, cxb = false;
        int32_t xa = 0, xb = 0;
        if (px[k] >= 0)
          c24_pair_apply<EXACT>(A, Rid, t, thr, G, px[k], e[k], v[k], G.meta[pw[k]], &G.meta[pw[k]], false, 0,
                                in_level, cross[k], cxa, xa, cxb, xb, ls);
      }
#pragma unroll
      for (int k = 0; k < 2; k++) c24_append(A, nf, false, cross[k], e[k], false, 0, false, 0);
    }
    c24_sync<BLOCK>();
    c24_flush<EXACT, BLOCK>(A, Rid, t, thr, nf, G, nc, lo, false, ls);
    c24_sync<BLOCK>();
  } else {
    // slabs of consecutive list entries; the w's of this sub-task: list entries [w0, w1)
    const int64_t wstep = ((len + nsub - 1) / nsub + 31) & ~(int64_t)31;
    const int64_t w0 = (int64_t)sub * wstep;
    const int64_t w1 = w0 + wstep < len ? w0 + wstep : len;
    const bool xdirect = (w1 > w0 ? w1 - w0 : 0) > (int64_t)kC24AccMax && !A.union_mode;
    const uint32_t* vals = c24_vals(A);
    for (int64_t s0 = 0; s0 < len; s0 += G.cap) {
      const int64_t slen = len - s0 < G.cap ? len - s0 : G.cap;
      c24_sync<BLOCK>();
      for (int i = tid; i < G.hs; i += TEAM) G.key[i] = -1;
      if (tid == 0) *tcnt = 0;
      c24_sync<BLOCK>();
      c24_stage<BLOCK>(A, Rid, t, thr, lo, s0, slen, s0, G, tcnt, wcnt, ls);
      const int ns = *tcnt;  // <= slen <= cap
      for (int64_t wb = w0 + (int64_t)wit * 32; wb < w1; wb += TEAM) {
        const int64_t i = wb + lane;
        uint32_t wfl = 0, dlen = 0;
        int64_t ob = 0;
        bool live = false;
        if (i < w1) {
          const int32_t ea = __ldg(g.t2ea + lo + i), eb = __ldg(g.t2eb + lo + i);
          live = c24_keep(A, Rid, t, thr, ea, eb, __ldcg(vals + ea), __ldcg(vals + eb), wfl);
          ls.scan += 2;
          ls.stamp += 2;
          if (live) {
            const int32_t w = __ldg(g.t2w + lo + i);
            ob = __ldg(g.ooff + w);
            dlen = (uint32_t)(__ldg(g.ooff + w + 1) - ob);
            ls.scan += 5;
          }
        }
        wacc[lane] = 0;
        __syncwarp();
        uint32_t total;
        const uint32_t incl = c24_scan(dlen, total);
        for (uint32_t pbx = 0; pbx < total; pbx += 32)
          c24_pairs<EXACT>(A, Rid, t, thr, nf, G, pbx + lane, total, incl, dlen, ob, wfl, wacc, xdirect, lo + s0,
                           in_level, ls);
        __syncwarp();
        c24_apply<EXACT>(A, lo + i, wfl, live ? wacc[lane] : 0u, Rid, t, thr, nf, lane, ls);
        __syncwarp();
      }
      c24_sync<BLOCK>();
      c24_flush<EXACT, BLOCK>(A, Rid, t, thr, nf, G, ns, lo + s0, xdirect, ls);
    }
    c24_sync<BLOCK>();
  }
  if (A.mark && in_level && !__ldcg(A.mark + Rid)) __stcg(A.mark + Rid, 1u);
}

// next entry of the block queue (r-clique << 32 | sub-task << 16 | sub-tasks), or ~0 when it is
// empty for good (thread 0 of a block).  Every claim takes a ticket (one atomic add, no retries); a
// ticket below the number of entries pushed so far names its entry, which the pusher may still be
// writing (wait for it); a higher ticket waits until either an entry arrives for it or every
// block has finished its warp phase (no more pushes: the queue is closed).  Every wait is bounded.
__device__ __forceinline__ unsigned long long c24_claim(const PeelArgs& A) {
  PeelCtl* ctl = A.lk.ctl;
  volatile PeelCtl* vc = ctl;
  const unsigned long long k = atomicAdd(&ctl->c24_hk, 1ull);
  for (int it = 0; it < (1 << 24); ++it) {
    if (vc->err) return ~0ull;
    if (k < vc->c24_hn) {
      volatile unsigned long long* slot = A.c24_queue + k;
      for (int sp = 0; sp < (1 << 24); ++sp) {
        const unsigned long long v = *slot;
        if (v != ~0ull) {
          *slot = ~0ull;  // the queue is all ~0 again once every entry is taken (end of the round)
          return v;
        }
        __nanosleep(32);
      }
      break;
    }
    if (vc->c24_done == gridDim.x) {
      __threadfence();
      if (k >= vc->c24_hn) return ~0ull;  // closed, and nothing left for this ticket
      continue;
    }
    __nanosleep(64);
  }
  atomicCAS(&ctl->err, 0, NH_ERR_TIMEOUT);
  return ~0ull;
}

// Sub-tasks of the n r-cliques of items (block-collective; every block computes the same
// result).  With n <= kTaskItems, r-clique i gets K_i sub-tasks, K_i growing with its scan bound
// (list length + t2cost) over the round's total (about c24_per_warp warp sub-tasks per warp of the
// grid, or as many block sub-tasks per block for lists too long for a warp), with a scan bound of
// at least c24_wgrain per warp sub-task and c24_bgrain per block sub-task, and at least
// c24_len_mult times the list length (each sub-task stages the whole list); s_pref[i] = K_0 + ... + K_i.  Returns the number of sub-tasks; n > kTaskItems:
// one per r-clique (s_pref unused).
__device__ __forceinline__ unsigned long long c24_prefix(const PeelArgs& A, const int32_t* items, unsigned long long n,
                                                         long long nwarps, uint32_t* s_pref, unsigned long long* s_red,
                                                         int* any_long) {
  if (n > (unsigned long long)kTaskItems) {
    *any_long = 1;  // not looked at: the block queue phase runs
    return n;
  }
  constexpr int kPer = kTaskItems / kThreads;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned int b = threadIdx.x * kPer;
  uint32_t len[kPer], est[kPer];
  unsigned long long sum = 0;
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    len[j] = est[j] = 0;
    if (b + j < n) {
      const int32_t R = __ldcg(items + b + j);
      const int64_t l = __ldg(A.g.t2off + R + 1) - __ldg(A.g.t2off + R);
      len[j] = l > 0x7fffffffll ? 0x7fffffffu : (uint32_t)l;
      const unsigned long long c = (unsigned long long)len[j] + __ldg(A.g.t2cost + R);
      est[j] = c > 0xffffffffull ? 0xffffffffu : (uint32_t)c;
    }
    sum += est[j];
  }
  bool lng = false;
#pragma unroll
  for (int j = 0; j < kPer; j++) lng = lng || len[j] > (uint32_t)kC24WarpCap;
  sum = warp_sum_u64(sum);
  lng = __any_sync(NH_FULL, lng);
  __syncthreads();  // the previous round's readers of s_pref / s_red / any_long are done
  if (threadIdx.x == 0) *any_long = 0;
  __syncthreads();
  if (lane == 0) s_red[wib] = sum;
  if (lane == 0 && lng) *any_long = 1;
  __syncthreads();
  unsigned long long W = 0;
  for (int w = 0; w < kThreads / 32; w++) W += s_red[w];
  if (W == 0) W = 1;
  // single precision on purpose: this runs every round in every block, and only the schedule
  // depends on it
  const float q = A.c24_per_warp * (float)nwarps / (float)W;  // warp sub-tasks per unit of scan bound
  const float qb = q * (1.0f / (kThreads / 32));
  const float rw = 1.0f / (float)A.c24_wgrain, rb = 1.0f / (float)A.c24_bgrain;
  uint32_t k[kPer];
  unsigned long long ks = 0;
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    k[j] = 0;
    if (b + j < n) {
      const bool blk = len[j] > (uint32_t)kC24WarpCap;
      const float e = (float)est[j];
      const float want = (blk ? qb : q) * e;
      float most = e * (blk ? rb : rw) + 1.0f;
      if (A.c24_len_mult > 0) {
        const float m2 = __fdividef(e, (float)A.c24_len_mult * (float)len[j]) + 1.0f;
        most = m2 < most ? m2 : most;
      }
      float kk = want < most ? want : most;
      kk = kk < (float)kC24MaxSplit ? kk : (float)kC24MaxSplit;
      k[j] = kk < 1.0f ? 1u : (uint32_t)kk;
    }
    ks += k[j];
  }
  unsigned long long incl = ks;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(NH_FULL, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_red[8 + wib] = incl;
  __syncthreads();
  unsigned long long base = incl - ks, total = 0;
  for (int w = 0; w < kThreads / 32; w++) {
    const unsigned long long x = s_red[8 + w];
    if (w < wib) base += x;
    total += x;
  }
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    base += k[j];
    if (b + j < n) s_pref[b + j] = (uint32_t)base;
  }
  __syncthreads();
  return total;  // <= 4096 * 65535 < 2^32
}

// Re-lists the n r-cliques of items (frontier or level), block-collective.  smem: kC24SmemBytes.
template <bool EXACT>
__device__ void c24_list(const PeelArgs& A, const int32_t* items, unsigned long long n, uint32_t t, uint32_t thr,
                         int32_t* nf, long long gwarp, long long nwarps, unsigned char* smem, LocalStats& ls) {
  PeelCtl* ctl = A.lk.ctl;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t* s_pref = reinterpret_cast<uint32_t*>(smem + kC24Pref);
  uint32_t* wacc = reinterpret_cast<uint32_t*>(smem + kC24Wacc) + 32 * wib;
  unsigned long long* s_red = reinterpret_cast<unsigned long long*>(smem + kC24Red);
  int* tcnt = reinterpret_cast<int*>(smem + kC24Tcnt);
  int* wcnt = reinterpret_cast<int*>(smem + kC24Wcnt);
  volatile unsigned long long* bcast = reinterpret_cast<volatile unsigned long long*>(smem + kC24Bcast);
  const C24Area Gw = c24_area(smem + (size_t)kC24WarpBytes * wib, kC24WarpHS, 9, kC24WarpCap);
  const C24Area Gb = c24_area(smem, kC24BlockHS, 12, kC24BlockCap);
  const bool split = n <= (unsigned long long)kTaskItems;
  const unsigned long long ntask = c24_prefix(A, items, n, nwarps, s_pref, s_red, tcnt + 9);
  const bool any_long = tcnt[9] != 0;  // every block computed the same
  const bool trace = A.round_log && !A.union_mode && blockIdx.x == 0 && threadIdx.x == 0 && t >= 1 &&
                     t <= A.round_log_cap;  // block 0's phase times of the round
  if (trace) A.round_log[8 * (t - 1) + 5] = nh_globaltimer();
  const unsigned long long expand0 = ls.expand;
  if (A.round_log && blockIdx.x == 0 && threadIdx.x == 0) ctl->c24_tasks = ntask;
  // warps: sub-task gwarp first (no counter traffic when a round has fewer sub-tasks than warps),
  // then the rest, from nwarps on, in batches from a shared counter
  const unsigned long long NW = (unsigned long long)nwarps;
  const unsigned long long rest = ntask > NW ? ntask - NW : 0ull;
  const unsigned long long per = rest / (NW * 8ull);
  const unsigned long long bt = per > 0 ? per : 1ull;
  bool first = true;
  for (;;) {
    unsigned long long k0 = 0, k1 = 0;
    if (first) {
      first = false;
      k0 = (unsigned long long)gwarp;
      k1 = k0 + 1;
    } else {
      if (rest == 0) break;
      if (lane == 0) k0 = atomicAdd(&ctl->c24_next, bt);
      k0 = NW + __shfl_sync(NH_FULL, k0, 0);
      k1 = k0 + bt;
    }
    if (k0 >= ntask) break;
    if (k1 > ntask) k1 = ntask;
    for (unsigned long long k = k0; k < k1; ++k) {
      unsigned int i = (unsigned int)k;
      int sub = 0, nsub = 1;
      if (split) {
        unsigned int lo = 0, hi = (unsigned int)n;  // first r-clique whose inclusive prefix exceeds k
        while (lo < hi) {
          const unsigned int mid = (lo + hi) >> 1;
          if ((unsigned long long)s_pref[mid] <= k) lo = mid + 1; else hi = mid;
        }
        i = lo;
        const uint32_t before = i ? s_pref[i - 1] : 0u;
        sub = (int)(k - before);
        nsub = (int)(s_pref[i] - before);
      }
      const int32_t Rid = __ldcg(items + i);
      const int64_t len = __ldg(A.g.t2off + Rid + 1) - __ldg(A.g.t2off + Rid);
      if (len > kC24WarpCap) {
        if (lane == 0) {
          const unsigned long long q = atomicAdd(&ctl->c24_hn, 1ull);
          const unsigned long long e =
              ((unsigned long long)(uint32_t)Rid << 32) | ((unsigned long long)sub << 16) | (unsigned long long)nsub;
          if (q < A.c24_qcap) {
            *(volatile unsigned long long*)(A.c24_queue + q) = e;
            __threadfence();
          } else {
            atomicCAS(&ctl->err, 0, NH_ERR_OVERFLOW);  // the claim loop then gives up at once
          }
        }
        continue;
      }
      if (len > 0) c24_item<EXACT, false>(A, Rid, sub, nsub, t, thr, nf, Gw, wacc, tcnt + wib, nullptr, nullptr, ls);
    }
  }
  if (trace) A.round_log[8 * (t - 1) + 6] = nh_globaltimer();
  // blocks: the long lists (none in this round: skip the queue)
  if (any_long) {
    __syncthreads();  // this block's warps have pushed everything they will push this round
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&ctl->c24_done, 1u);
    }
  }
  while (any_long) {
    if (threadIdx.x == 0) *bcast = c24_claim(A);
    __syncthreads();
    const unsigned long long e = *bcast;
    __syncthreads();
    if (e == ~0ull) break;
    c24_item<EXACT, true>(A, (int32_t)(e >> 32), (int)((e >> 16) & 0xffffu), (int)(e & 0xffffu), t, thr, nf, Gb,
                          wacc, tcnt + 8, wcnt, s_red, ls);
  }
  if (trace) A.round_log[8 * (t - 1) + 7] = nh_globaltimer();
  if (A.round_log) {
    const unsigned long long d = warp_sum_u64(ls.expand - expand0);
    if (lane == 0 && d) atomicAdd(&ctl->dbg_work, d);
  }
}

}  // namespace nhp
