// nh_peel.cuh -- device code of the peel (Alg. 3 / Alg. 5 exact, Alg. 2 approximate) and of the
// two-phase hierarchy (§7.4), shared by nh_peel.cu (drivers and entry points) and the per-(r,s)
// translation units nh_peel_rs*.cu, which instantiate the kernel templates (so that the five
// pairs compile in parallel).  Every wait is bounded; see nh_peel.cu for the round structure.
#pragma once
#include <cstdint>

#include "nh_internal.cuh"

namespace nhp {

constexpr int kThreads = 256;
constexpr int kTaskItems = 4096;  // largest frontier re-listed in work-proportional tasks
constexpr int kMinBlocks = 4;     // resident blocks per SM the persistent kernels are compiled for
constexpr int kLinkStack = 16;
constexpr int64_t kC24QueueSlack = 1 << 16;  // block sub-tasks of a round beyond one per r-clique
constexpr uint32_t kNone = 0xffffffffu;

struct PeelCtl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int err;
  int done;
  unsigned int t;
  unsigned int thr;
  unsigned int bucket;
  unsigned int rounds_in_bucket;
  unsigned int need_scan;
  unsigned int cur;
  unsigned int alive_cur;
  unsigned int gmin;
  unsigned int draining;
  unsigned int drain_buf;
  unsigned int ovf_cur;
  unsigned int kmax;
  unsigned long long finished;
  unsigned long long fsize;
  unsigned long long nf_count;
  unsigned long long alive_n;
  unsigned long long alive2_count;
  unsigned long long f_count;
  unsigned long long drain_n;
  unsigned long long ovf_count[2];
  unsigned long long task_next;     // next re-listing task of the round (work-proportional mode)
  unsigned long long c24_next;      // (2,4) triangle-list re-listing: next list item for warps,
  unsigned long long c24_hn;        // entries pushed to the block queue,
  unsigned long long c24_hk;        // tickets taken for it
  unsigned int c24_done;            // blocks whose warps finished pushing to it this round
  unsigned int c24_pad;
  unsigned long long c24_tasks;     // sub-tasks of the round (round trace)
  unsigned long long dbg_work;      // list entries expanded in the round (round trace)
  // statistics
  unsigned long long st_rounds, st_levels, st_listed, st_dec, st_link, st_unite, st_scan, st_probe, st_front,
      st_ovf, st_stamp;
};

struct LinkEnv {
  int32_t* uf;
  int32_t* L;
  const uint32_t* core;
  int32_t* J;                       // jump pointers (may be null)
  unsigned long long* cache;        // lossy set of linked root pairs (may be null)
  unsigned long long cache_mask;
  int2* ovf[2];
  unsigned long long ovf_cap;
  PeelCtl* ctl;
};

struct PeelArgs {
  GView g;
  int64_t n_r;
  uint32_t* cnt;          // working counts
  const uint32_t* cnt0;   // s-clique-degrees
  uint32_t* val;          // core (exact) or approximate value
  uint32_t* round;
  int32_t* alive[2];
  int32_t* front[2];
  const uint32_t* thresholds;
  int n_thr;
  uint32_t T;
  int link_mode;          // 0 definitional, 1 pairwise, -1 none
  int union_mode;         // two-phase hierarchy: re-listing unites instead of peeling
  int gmax;               // largest number of warps per frontier r-clique (power of two)
  const uint32_t* cost;   // chunks of 32 list entries per r-clique (work-proportional re-listing)
  uint32_t* mark;         // label hierarchy: 1 for an r-clique in an s-clique at its own level
  unsigned int task_items;  // largest list re-listed in work-proportional tasks (<= kTaskItems)
  int32_t* touched;       // two-phase: roots joined at the current level
  unsigned long long* touched_n;
  unsigned long long touched_cap;
  int stats;
  unsigned long long timeout_ns;
  int use24;              // (2,4) without links: re-list over the per-edge triangle lists
  int4* et3;              // (3,4): per-edge triangle lists with mirrored state, {w, triangle, stamp, value}
  int32_t* tpos;          //        the three list positions of every triangle (or null: plain lists)
  const ulonglong2* eh;   // (3,4): {edge id << 32 | w, list position} of every list entry (or null:
  unsigned long long eh_mask;  //   binary searches), open addressing at load <= 0.5
  unsigned long long* round_log;  // optional trace: per round (frontier << 32 | levels, end time)
  unsigned long long round_log_cap;
  unsigned long long* c24_queue;  // block queue of that re-listing (all ~0 between rounds)
  unsigned long long c24_qcap;    // its entries: n_r + kC24QueueSlack (sub-tasks of a round)
  float c24_per_warp;             // sub-tasks per warp of the grid a round aims at
  int c24_wgrain, c24_bgrain;     // least scan bound per warp / block sub-task
  int c24_len_mult;               // and at least this many times the list length (0: off)
  LinkEnv lk;
};

struct LocalStats {
  unsigned long long listed, dec, link, unite, scan, probe, ovf, stamp, expand;
};

// ---------------------------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t warp_min_u32(uint32_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = min(v, __shfl_xor_sync(NH_FULL, v, d));
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(NH_FULL, v, d);
  return v;
}

// warp-aggregated append; every lane of the warp must call it
__device__ __forceinline__ unsigned long long warp_append(unsigned long long* counter, bool pred, int lane) {
  const unsigned m = __ballot_sync(NH_FULL, pred);
  if (!m) return 0;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(NH_FULL, base, leader);
  return base + __popc(m & ((1u << lane) - 1u));
}

// Grid barrier with a bounded wait.  The last block to arrive runs `leader` (thread 0) before
// releasing the others.  Returns false once any block has recorded an error.
template <class F>
__device__ __forceinline__ bool grid_sync(PeelCtl* ctl, unsigned long long timeout_ns, F leader) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile PeelCtl* vc = ctl;
    const unsigned int gen = vc->bar_gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      __threadfence();
      leader();
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = nh_globaltimer();
      while (vc->bar_gen == gen) {
        __nanosleep(64);
        if (nh_globaltimer() - t0 > timeout_ns) {
          atomicCAS(&ctl->err, 0, NH_ERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    s_ok = (vc->err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// The control words a round needs, copied to shared memory by one thread after each grid barrier:
// independent loads from L2 instead of one dependent volatile read per field and thread.
struct RoundView {
  unsigned int done, err, need_scan, t, thr, cur, alive_cur, draining, drain_buf;
  unsigned long long fsize, alive_n, drain_n;
};

__device__ __forceinline__ void round_view_load(PeelCtl* c, RoundView* v) {
  RoundView x;
  x.done = __ldcg(reinterpret_cast<const unsigned int*>(&c->done));
  x.err = __ldcg(reinterpret_cast<const unsigned int*>(&c->err));
  x.need_scan = __ldcg(&c->need_scan);
  x.t = __ldcg(&c->t);
  x.thr = __ldcg(&c->thr);
  x.cur = __ldcg(&c->cur);
  x.alive_cur = __ldcg(&c->alive_cur);
  x.draining = __ldcg(&c->draining);
  x.drain_buf = __ldcg(&c->drain_buf);
  x.fsize = __ldcg(&c->fsize);
  x.alive_n = __ldcg(&c->alive_n);
  x.drain_n = __ldcg(&c->drain_n);
  *v = x;
}

// grid_sync, then the round view refreshed in shared memory (block-collective)
template <class F>
__device__ __forceinline__ bool grid_sync_view(PeelCtl* ctl, unsigned long long timeout_ns, RoundView* v, F leader) {
  const bool ok = grid_sync(ctl, timeout_ns, leader);
  if (threadIdx.x == 0) round_view_load(ctl, v);
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------------------------
// concurrent union-find (CAS, path halving) and link-efficient (Alg. 5)
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ int32_t uf_find(int32_t* uf, int32_t x) {
  // parent ids strictly decrease along a path, so this ends; the cap is only a guard
  for (int it = 0; it < (1 << 24); ++it) {
    const int32_t p = __ldcg(uf + x);
    if (p == x) return x;
    const int32_t gp = __ldcg(uf + p);
    if (gp != p) atomicCAS(uf + x, p, gp);
    x = gp;
  }
  return x;
}

// unite the sets of a and b: the root of larger id is hung under the root of smaller id.
// Returns the root that was hung (it is this caller's job to pass on its L entry), or -1 when
// a and b were already in one set.
__device__ __forceinline__ int32_t uf_unite(int32_t* uf, int32_t a, int32_t b, PeelCtl* ctl) {
  for (int it = 0; it < (1 << 20); ++it) {
    a = uf_find(uf, a);
    b = uf_find(uf, b);
    if (a == b) return -1;
    if (a < b) { const int32_t t = a; a = b; b = t; }
    if (atomicCAS(uf + a, a, b) == a) {
      __threadfence();
      return a;
    }
  }
  atomicCAS(&ctl->err, 0, NH_ERR_TIMEOUT);
  return -1;
}

__device__ __forceinline__ void ovf_push(const LinkEnv& E, int32_t a, int32_t b, LocalStats& ls) {
  const unsigned int cur = *(volatile unsigned int*)&E.ctl->ovf_cur;
  const unsigned long long pos = atomicAdd(&E.ctl->ovf_count[cur], 1ull);
  if (pos < E.ovf_cap) E.ovf[cur][pos] = make_int2(a, b);
  else atomicCAS(&E.ctl->err, 0, NH_ERR_OVERFLOW);
  ls.ovf++;
}

// link-efficient(R0, Q0) of Alg. 5 with the recursion replaced by a small per-thread stack; calls
// that do not fit go to the overflow queue, drained after the round.
static __device__ void link_run(const LinkEnv& E, int32_t R0, int32_t Q0, LocalStats& ls) {
  int32_t sR[kLinkStack], sQ[kLinkStack];
  int sp = 0;
  sR[0] = R0; sQ[0] = Q0; sp = 1;
  auto push = [&](int32_t a, int32_t b) {
    if (a < 0 || b < 0) return;
    if (sp < kLinkStack) { sR[sp] = a; sQ[sp] = b; ++sp; }
    else ovf_push(E, a, b, ls);
  };
  unsigned int guard = 0;
  while (sp > 0) {
    if (++guard > (1u << 22)) { atomicCAS(&E.ctl->err, 0, NH_ERR_TIMEOUT); return; }
    --sp;
    int32_t R = sR[sp], Q = sQ[sp];
    if (R < 0 || Q < 0) continue;
    ls.link++;
    uint32_t nR = __ldcg(E.core + R), nQ = __ldcg(E.core + Q);
    if (nQ < nR) {
      const int32_t t = R; R = Q; Q = t;
      const uint32_t u = nR; nR = nQ; nQ = u;
    }
    R = uf_find(E.uf, R);
    Q = uf_find(E.uf, Q);
    if (R == Q) continue;
    if (E.cache) {
      // a pair of roots already linked states nothing new (components only grow)
      const unsigned long long key = ((unsigned long long)(uint32_t)R << 32) | (uint32_t)Q;
      unsigned long long* slot = E.cache + (nh_mix64(key) & E.cache_mask);
      if (__ldcg(slot) == key) continue;
      *slot = key;
    }
    if (nR == nQ) {
      // Alg. 5 passes on L of whichever of R, Q stopped being a root.  Concurrently the roots
      // actually joined may be others (R or Q may have been hung meanwhile), so the thread whose
      // CAS hung a root passes on that root's L -- every hung root is handled exactly by the
      // thread that hung it.
      const int32_t child = uf_unite(E.uf, R, Q, E.ctl);
      if (child >= 0) {
        ls.unite++;
        push(__ldcg(E.L + child), uf_find(E.uf, child));
      }
      continue;
    }
    // nR < nQ.  L[Q] is read only after Q is re-found as a root, and the value that was tested is
    // the one passed on: with concurrent unites, a value read from a component that has just
    // stopped being a root (or re-read after the test) could drop the fact "R meets Q at level
    // nR" -- the sequential order of the paper's loop does not survive concurrency otherwise.
    //
    // The walk down Q's chain (Alg. 5's call link(R, L[Q]) when ND[L[Q]] > ND[R]) continues in
    // place.  Jump pointers shorten it: J[C] is a component known to meet C at level core(J[C]) <
    // core(C) (every component on C's chain qualifies, and the relation only ever grows), so for
    // core(J[C]) >= nR the call link(R, C) states exactly what link(R, J[C]) states, and no
    // component between C and J[C] (all of core > core(J[C])) is where R belongs.  Each walk
    // records the deepest component it passed above level nR as the jump pointer of its start.
    const int32_t Q0 = Q;
    int32_t deepest = -1;
    uint32_t c_deepest = 0;
    for (unsigned int spin = 0;; ++spin) {
      if (spin > (1u << 20)) { atomicCAS(&E.ctl->err, 0, NH_ERR_TIMEOUT); return; }
      Q = uf_find(E.uf, Q);
      if (E.J) {
        const int32_t jq = __ldcg(E.J + Q);
        if (jq >= 0) {
          const uint32_t cj = __ldcg(E.core + jq);
          if (cj > nR) {
            deepest = jq;
            c_deepest = cj;
            Q = jq;
            ++ls.link;
            continue;
          }
          if (cj == nR) {
            push(R, jq);
            break;
          }
        }
      }
      const int32_t LQ = __ldcg(E.L + Q);
      if (LQ < 0) {
        if (atomicCAS(E.L + Q, -1, R) == -1) {
          __threadfence();
          const int32_t pQ = uf_find(E.uf, Q);
          if (pQ != Q) push(R, pQ);
          break;
        }
        continue;  // L[Q] was set meanwhile: retry with its value
      }
      const uint32_t cL = __ldcg(E.core + LQ);
      if (cL < nR) {
        if (atomicCAS(E.L + Q, LQ, R) == LQ) {
          __threadfence();
          const int32_t pQ = uf_find(E.uf, Q);
          if (pQ != Q) push(R, pQ);
          push(R, LQ);
          break;
        }
        continue;
      }
      if (cL == nR) {
        push(R, LQ);
        break;
      }
      deepest = LQ;  // ND[L[Q]] > ND[R]: continue the walk from L[Q]
      c_deepest = cL;
      Q = LQ;
      ++ls.link;
    }
    if (E.J && deepest >= 0) {
      const int32_t j0 = __ldcg(E.J + Q0);
      if (j0 < 0 || c_deepest < __ldcg(E.core + j0)) E.J[Q0] = deepest;
    }
  }
}

// host: one drain step of the overflow queue of deferred link calls (nh_peel.cu)
int link_drain_round(const LinkEnv& E, cudaStream_t st);

// one out-of-line copy for the rarely taken call sites (keeps the kernels' code size down)
// link-efficient counters of a link_run done out of line
struct LinkDelta {
  unsigned long long link, unite, ovf;
};

__device__ __forceinline__ void add_delta(LocalStats& ls, const LinkDelta& d) {
  ls.link += d.link;
  ls.unite += d.unite;
  ls.ovf += d.ovf;
}

static __device__ __noinline__ LinkDelta link_run_call(const LinkEnv E, int32_t R0, int32_t Q0) {
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  link_run(E, R0, Q0, ls);
  return LinkDelta{ls.link, ls.unite, ls.ovf};
}

// ---------------------------------------------------------------------------------------------
// per (R, S) step
// ---------------------------------------------------------------------------------------------

// (3,4) with mirrored lists: triangle x's round stamp and value, copied into its three list
// entries (8-byte stores: a reader of an entry sees the pair before or after, never half of it)
__device__ __forceinline__ void mirror_set(const PeelArgs& A, int32_t x, uint32_t rd, uint32_t v) {
  const int32_t* tp = A.tpos + 3 * (int64_t)x;
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const int64_t k = __ldg(tp + j);
    __stcg(reinterpret_cast<uint2*>(reinterpret_cast<char*>(A.et3 + k) + 8), make_uint2(rd, v));
  }
}

template <bool EXACT>
__device__ __forceinline__ void dec(const PeelArgs& A, int32_t x, uint32_t t, uint32_t thr, int32_t* nf,
                                    LocalStats& ls) {
  const uint32_t old = atomicSub(A.cnt + x, 1u);
  ls.dec++;
  if (old == thr + 1u) {
    const unsigned long long pos = atomicAdd(&A.lk.ctl->nf_count, 1ull);
    nf[pos] = x;
    const uint32_t v = EXACT ? thr : min(thr, __ldg(A.cnt0 + x));
    __stcg(A.round + x, t + 1u);
    __stcg(A.val + x, v);
    if (A.et3) mirror_set(A, x, t + 1u, v);
  }
}

__device__ __forceinline__ int32_t tri_id(const PeelArgs& A, unsigned long long key, LocalStats& ls) {
  ls.probe++;
  const int64_t id = nh_tri_lookup(A.g.table, A.g.mask, key);
  if (id < 0) {
    atomicCAS(&A.lk.ctl->err, 0, NH_ERR_INTERNAL);
    return 0;
  }
  return (int32_t)id;
}

// ---------------------------------------------------------------------------------------------
// per-warp link buffer: the link targets of one frontier r-clique R are collected, replaced by
// their union-find roots, sorted by decreasing core and de-duplicated, then linked as a chain
// R - t1 - t2 - ... (t_i = targets in that order).  Since R meets t_i at level core(t_i) and
// core(t_{i-1}) >= core(t_i), "t_{i-1} meets t_i at level core(t_i)" states the same
// connectivity as "R meets t_i at core(t_i)", while link-efficient walks only between adjacent
// levels instead of from R's level down to each target's level.
// ---------------------------------------------------------------------------------------------

constexpr int kLinkBuf = 256;

struct WarpLinks {
  unsigned long long* buf;
  int* cnt;
  int32_t* seen;  // kSeen roots this warp has already chained from the current R (direct-mapped)
};

constexpr int kSeen = 64;

// dynamic shared memory of the persistent kernels on the adjacency / chunk-task path: per warp a
// link buffer and a seen-roots filter, the task prefix sums, per-warp sums, per-warp buffer counts
constexpr int kSmLinks = 0;
constexpr int kSmPref = kSmLinks + (kThreads / 32) * kLinkBuf * 8;
constexpr int kSmSeen = kSmPref + kTaskItems * 4;
constexpr int kSmWsum = kSmSeen + (kThreads / 32) * kSeen * 4;
constexpr int kSmLcnt = kSmWsum + (kThreads / 32) * 8;
constexpr int kSmOldBytes = kSmLcnt + (kThreads / 32) * 4;

// warp-collective: forget the roots seen for the previous frontier r-clique
__device__ __forceinline__ void wl_begin(const WarpLinks& W, int lane) {
  __syncwarp();
  for (int i = lane; i < kSeen; i += 32) W.seen[i] = -1;
  __syncwarp();
}

__device__ __forceinline__ void wl_add(const WarpLinks& W, const PeelArgs& A, int32_t Rid, int32_t m,
                                       LocalStats& ls) {
  // a target whose component this warp has already chained from R adds nothing: R meets that
  // whole component at its level already (a root that changed since only misses the filter)
  const int32_t rt = uf_find(A.lk.uf, m);
  if (W.seen[rt & (kSeen - 1)] == rt) return;
  const int pos = atomicAdd(W.cnt, 1);
  if (pos < kLinkBuf) W.buf[pos] = (unsigned long long)(uint32_t)m;
  else add_delta(ls, link_run_call(A.lk, Rid, m));  // buffer full (cannot happen with the flush policy)
}

// warp-collective
// out of line (one copy per kernel); arguments by value so that the callers' state stays in
// registers
static __device__ __noinline__ LinkDelta wl_flush_impl(const WarpLinks W, const LinkEnv E, const uint32_t* val,
                                                       int32_t Rid, int lane) {
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  __syncwarp();
  const int n = min(*(volatile int*)W.cnt, kLinkBuf);
  if (n == 0) return LinkDelta{0, 0, 0};
  int P = 2;  // sort only the smallest power of two holding the n entries
  while (P < n) P <<= 1;
  for (int i = lane; i < P; i += 32) {
    unsigned long long key = ~0ull;
    if (i < n) {
      const int32_t rt = uf_find(E.uf, (int32_t)W.buf[i]);
      const uint32_t c = __ldcg(val + rt);
      key = ((unsigned long long)(~c) << 32) | (uint32_t)rt;
    }
    W.buf[i] = key;
  }
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = W.buf[i], b = W.buf[ixj];
          if ((a > b) == ((i & k) == 0)) {
            W.buf[i] = b;
            W.buf[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < n; i += 32) {
    const int32_t cur = (int32_t)(W.buf[i] & 0xffffffffull);
    const int32_t prev = (i == 0) ? Rid : (int32_t)(W.buf[i - 1] & 0xffffffffull);
    if (i > 0 && prev == cur) continue;
    link_run(E, prev, cur, ls);
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {  // record after every link of the chain has completed
    const int32_t cur = (int32_t)(W.buf[i] & 0xffffffffull);
    W.seen[cur & (kSeen - 1)] = cur;
  }
  __syncwarp();
  if (lane == 0) *W.cnt = 0;
  __syncwarp();
  return LinkDelta{ls.link, ls.unite, ls.ovf};
}

__device__ __forceinline__ void wl_flush(const WarpLinks& W, const PeelArgs& A, int32_t Rid, int lane, LocalStats& ls) {
  add_delta(ls, wl_flush_impl(W, A.lk, A.val, Rid, lane));
}

// flush when another step of 32 lanes could overflow the buffer (warp-collective)
__device__ __forceinline__ void wl_maybe_flush(const WarpLinks& W, const PeelArgs& A, int32_t Rid, int lane,
                                               int per_lane, LocalStats& ls) {
  __syncwarp();
  if (*(volatile int*)W.cnt > kLinkBuf - 32 * per_lane) wl_flush(W, A, Rid, lane, ls);
}

template <int CM, bool EXACT>
__device__ __forceinline__ void process_S(const PeelArgs& A, int32_t Rid, const int32_t (&mem)[CM], uint32_t t,
                                          uint32_t thr, int32_t* nf, const WarpLinks& W, LocalStats& ls) {
  ls.stamp += CM;
  if (A.union_mode) {
    // two-phase hierarchy at level thr (= core of Rid): an s-clique whose least member core is
    // thr joins all its members; its member of least id among those of core thr does it
    int32_t attr = Rid;
#pragma unroll
    for (int j = 0; j < CM; j++) {
      const uint32_t c = __ldcg(A.val + mem[j]);
      if (c < thr) return;
      if (c == thr && mem[j] < attr) attr = mem[j];
    }
    ls.listed++;
    if (A.mark && !__ldcg(A.mark + Rid)) __stcg(A.mark + Rid, 1u);  // least label over S is Rid's
    if (attr != Rid) return;
#pragma unroll
    for (int j = 0; j < CM; j++) {
      const int32_t child = uf_unite(A.lk.uf, Rid, mem[j], A.lk.ctl);
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
    return;
  }
  uint32_t rd[CM];
  bool dead = false;
  int32_t attr = Rid;
#pragma unroll
  for (int j = 0; j < CM; j++) {
    rd[j] = __ldcg(A.round + mem[j]);
    if (rd[j] != 0u && rd[j] < t) dead = true;
    else if (rd[j] == t && mem[j] < attr) attr = mem[j];
  }
  ls.listed++;
  if (dead) {
    if (EXACT && A.link_mode == 0) {
      int32_t best = -1;
      uint32_t bc = kNone;
#pragma unroll
      for (int j = 0; j < CM; j++) {
        if (rd[j] != 0u && rd[j] < t) {
          const uint32_t c = __ldcg(A.val + mem[j]);
          if (c < bc) { bc = c; best = mem[j]; }
        }
      }
      wl_add(W, A, Rid, best, ls);
    }
  } else if (attr == Rid) {
#pragma unroll
    for (int j = 0; j < CM; j++)
      if (rd[j] == 0u || rd[j] > t) dec<EXACT>(A, mem[j], t, thr, nf, ls);
    if (EXACT && A.link_mode == 0) {
#pragma unroll
      for (int j = 0; j < CM; j++)
        if (rd[j] == t) wl_add(W, A, Rid, mem[j], ls);
    }
  }
  if (EXACT && A.link_mode == 1) {
#pragma unroll
    for (int j = 0; j < CM; j++)
      if (rd[j] != 0u && rd[j] <= t) wl_add(W, A, Rid, mem[j], ls);
  }
}

// process_S with the members' round stamps rdv (peel) and values cv (core or approximate value)
// already loaded (the (3,4) mirrored lists); the same decisions as process_S
template <int CM, bool EXACT>
__device__ __forceinline__ void process_S_pre(const PeelArgs& A, int32_t Rid, const int32_t (&mem)[CM],
                                              const uint32_t (&rdv)[CM], const uint32_t (&cv)[CM], uint32_t t,
                                              uint32_t thr, int32_t* nf, const WarpLinks& W, LocalStats& ls) {
  ls.stamp += CM;
  if (A.union_mode) {
    int32_t attr = Rid;
#pragma unroll
    for (int j = 0; j < CM; j++) {
      if (cv[j] < thr) return;
      if (cv[j] == thr && mem[j] < attr) attr = mem[j];
    }
    ls.listed++;
    if (A.mark && !__ldcg(A.mark + Rid)) __stcg(A.mark + Rid, 1u);
    if (attr != Rid) return;
#pragma unroll
    for (int j = 0; j < CM; j++) {
      const int32_t child = uf_unite(A.lk.uf, Rid, mem[j], A.lk.ctl);
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
    return;
  }
  bool dead = false;
  int32_t attr = Rid;
#pragma unroll
  for (int j = 0; j < CM; j++) {
    if (rdv[j] != 0u && rdv[j] < t) dead = true;
    else if (rdv[j] == t && mem[j] < attr) attr = mem[j];
  }
  ls.listed++;
  if (dead) {
    if (EXACT && A.link_mode == 0) {
      int32_t best = -1;
      uint32_t bc = kNone;
#pragma unroll
      for (int j = 0; j < CM; j++)
        if (rdv[j] != 0u && rdv[j] < t && cv[j] < bc) { bc = cv[j]; best = mem[j]; }
      wl_add(W, A, Rid, best, ls);
    }
  } else if (attr == Rid) {
#pragma unroll
    for (int j = 0; j < CM; j++)
      if (rdv[j] == 0u || rdv[j] > t) dec<EXACT>(A, mem[j], t, thr, nf, ls);
    if (EXACT && A.link_mode == 0) {
#pragma unroll
      for (int j = 0; j < CM; j++)
        if (rdv[j] == t) wl_add(W, A, Rid, mem[j], ls);
    }
  }
  if (EXACT && A.link_mode == 1) {
#pragma unroll
    for (int j = 0; j < CM; j++)
      if (rdv[j] != 0u && rdv[j] <= t) wl_add(W, A, Rid, mem[j], ls);
  }
}

// ---------------------------------------------------------------------------------------------
// re-listing of one frontier r-clique by one warp
// ---------------------------------------------------------------------------------------------

// Whether an s-clique with member x (besides R) can still be one R handles: always for the
// linking peels (a dead s-clique is linked too); otherwise not when x was peeled in an earlier
// round or is in the frontier with a smaller id (peel), or when x lies below the level or is of
// the level with a smaller id (two-phase hierarchy; the label hierarchy keeps the latter, whose
// s-cliques still mark R).  process_S decides exactly; this only saves the searches for the rest.
__device__ __forceinline__ bool member_may_count_v(const PeelArgs& A, int32_t Rid, int32_t x, uint32_t rd, uint32_t c,
                                                   uint32_t t, uint32_t thr) {
  if (A.union_mode) return c >= thr && (A.mark || c > thr || x > Rid);
  if (A.link_mode == 0 || A.link_mode == 1) return true;
  return !((rd != 0u && rd < t) || (rd == t && x < Rid));
}

__device__ __forceinline__ bool member_may_count(const PeelArgs& A, int32_t Rid, int32_t x, uint32_t t, uint32_t thr,
                                                 LocalStats& ls) {
  if (A.union_mode) {
    const uint32_t c = __ldcg(A.val + x);
    ls.stamp++;
    return c >= thr && (A.mark || c > thr || x > Rid);
  }
  if (A.link_mode == 0 || A.link_mode == 1) return true;
  const uint32_t rd = __ldcg(A.round + x);
  ls.stamp++;
  return !((rd != 0u && rd < t) || (rd == t && x < Rid));
}

// Length of the list whose 32-entry chunks the re-listing of r-clique Rid walks: the adjacency
// list of its vertex of least degree, for (2,3) with per-edge triangle lists the edge's own list,
// or for (3,4) the shortest triangle list of its three edges.
template <int R, int S>
__device__ __forceinline__ int64_t relist_len(const GView& g, int32_t Rid) {
  if constexpr (R == 1) {
    return __ldg(g.off + Rid + 1) - __ldg(g.off + Rid);
  } else if constexpr (R == 2) {
    if (S == 3 && g.t2off) return __ldg(g.t2off + Rid + 1) - __ldg(g.t2off + Rid);
    const int32_t u = __ldg(g.eu + Rid), v = __ldg(g.ev + Rid);
    const int64_t du = __ldg(g.off + u + 1) - __ldg(g.off + u), dv = __ldg(g.off + v + 1) - __ldg(g.off + v);
    return du < dv ? du : dv;
  } else {
    const int32_t v0 = __ldg(g.tri + 3 * (int64_t)Rid), v1 = __ldg(g.tri + 3 * (int64_t)Rid + 1),
                  v2 = __ldg(g.tri + 3 * (int64_t)Rid + 2);
    if constexpr (S == 4) {
      const int64_t e[3] = {nh_edge_id(g, v0, v1), nh_edge_id(g, v0, v2), nh_edge_id(g, v1, v2)};
      int64_t m = INT64_MAX;
#pragma unroll
      for (int i = 0; i < 3; i++) {
        const int64_t len = e[i] < 0 ? 0 : __ldg(g.etoff + e[i] + 1) - __ldg(g.etoff + e[i]);
        m = len < m ? len : m;
      }
      return m;
    } else {
      int64_t m = INT64_MAX;
      const int32_t vv[3] = {v0, v1, v2};
#pragma unroll
      for (int i = 0; i < 3; i++) {
        const int64_t len = __ldg(g.off + vv[i] + 1) - __ldg(g.off + vv[i]);
        m = len < m ? len : m;
      }
      return m;
    }
  }
}

// chunks of 32 list entries per r-clique, the unit of work-proportional re-listing
template <int R, int S>
__global__ void k_chunk_cost(GView g, int64_t n_r, uint32_t* __restrict__ cost) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = (relist_len<R, S>(g, (int32_t)i) + 31) >> 5;
    cost[i] = c > 0xffffffffll ? 0xffffffffu : (uint32_t)c;
  }
}

// Re-lists the s-cliques of r-clique Rid found from chunks c0, c0 + cstep, ... (< cend) of its
// list (chunk c = entries [32c, 32c + 32)).  For s - r = 2 the out-lists of the candidates found
// in a chunk are split over Ge callers: this one expands candidates of lane index = se mod Ge.
// The caller brackets the calls for one Rid with wl_begin / wl_flush (exact peel).
template <int R, int S, bool EXACT>
__device__ __forceinline__ void relist_item(const PeelArgs& A, int32_t Rid, uint32_t t, uint32_t thr, int32_t* nf, int lane,
                            int64_t c0, int64_t cstep, int64_t cend, int Ge, int se, const WarpLinks& W,
                            LocalStats& ls) {
  constexpr int kPerLane = (S - R == 1) ? R : 5;  // link targets one lane can add per converged step
  const GView& g = A.g;
  int32_t vx[3] = {0, 0, 0};
  int32_t eR[3] = {0, 0, 0};  // r = 3: edges (v0,v1), (v0,v2), (v1,v2)
  if (R == 1) {
    vx[0] = Rid;
  } else if (R == 2) {
    vx[0] = __ldg(g.eu + Rid);
    vx[1] = __ldg(g.ev + Rid);
  } else {
    vx[0] = __ldg(g.tri + 3 * (int64_t)Rid);
    vx[1] = __ldg(g.tri + 3 * (int64_t)Rid + 1);
    vx[2] = __ldg(g.tri + 3 * (int64_t)Rid + 2);
    int32_t mine = 0;
    if (lane < 3) {
      if (g.tedge) {
        mine = __ldg(g.tedge + 3 * (int64_t)Rid + lane);
      } else {
        const int32_t x = (lane == 2) ? vx[1] : vx[0];
        const int32_t y = (lane == 0) ? vx[1] : vx[2];
        const int64_t p = nh_find(g.adj, __ldg(g.off + x), __ldg(g.off + x + 1), y);
        mine = (p >= 0) ? __ldg(g.eid + p) : 0;
      }
    }
    eR[0] = __shfl_sync(NH_FULL, mine, 0);
    eR[1] = __shfl_sync(NH_FULL, mine, 1);
    eR[2] = __shfl_sync(NH_FULL, mine, 2);
  }
  if constexpr (R == 3 && S == 4) {
    // the 4-cliques on triangle R = {v0,v1,v2} are the w common to the triangle lists of its
    // three edges; the ids of {v0,v1,w}, {v0,v2,w}, {v1,v2,w} are read from the list positions
    int64_t tl[3], th[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
      tl[i] = __ldg(g.etoff + eR[i]);
      th[i] = __ldg(g.etoff + eR[i] + 1);
    }
    int bt = 0;
    if (th[1] - tl[1] < th[bt] - tl[bt]) bt = 1;
    if (th[2] - tl[2] < th[bt] - tl[bt]) bt = 2;
    if (A.et3) {
      // mirrored lists: an entry holds its triangle's round stamp and value, so a search hit
      // brings everything the s-clique needs in one sector.  The scanned list (edge bt) and the
      // other two (i0 < i1) are taken apart into scalars so that nothing is indexed at run time.
      const int64_t lb = (bt == 0) ? tl[0] : (bt == 1) ? tl[1] : tl[2];
      const int64_t hb = (bt == 0) ? th[0] : (bt == 1) ? th[1] : th[2];
      const int64_t l0 = (bt == 0) ? tl[1] : tl[0], h0 = (bt == 0) ? th[1] : th[0];
      const int64_t l1 = (bt == 2) ? tl[1] : tl[2], h1 = (bt == 2) ? th[1] : th[2];
      const int32_t e0 = (bt == 0) ? eR[1] : eR[0], e1 = (bt == 2) ? eR[1] : eR[2];
      if (lane == 0 && c0 == 0 && se == 0) ls.scan += (unsigned long long)(4 * (hb - lb));
      for (int64_t c = c0; c < cend && lb + 32 * c < hb; c += cstep) {
        const int64_t j = lb + 32 * c + lane;
        bool ok = j < hb;
        int4 en = make_int4(0, 0, 0, 0), f0 = en, f1 = en;
        if (ok) {
          en = __ldcg(A.et3 + j);
          const int32_t w = en.x;
          ok = member_may_count_v(A, Rid, en.y, (uint32_t)en.z, (uint32_t)en.w, t, thr);
          if (ok) {
            // w's entries in the other two lists: both lookups advance in the same loop, so that
            // each lane has two independent loads in flight and the chain of dependent loads is
            // that of one lookup, not two
            int64_t p0 = -1, p1 = -1;
            if (A.eh) {
              const unsigned long long k0 = ((unsigned long long)(uint32_t)e0 << 32) | (uint32_t)w;
              const unsigned long long k1 = ((unsigned long long)(uint32_t)e1 << 32) | (uint32_t)w;
              unsigned long long q0 = nh_mix64(k0) & A.eh_mask, q1 = nh_mix64(k1) & A.eh_mask;
              bool d0 = false, d1 = false;
              for (unsigned long long q = 0; q <= A.eh_mask && !(d0 && d1); ++q) {
                const ulonglong2 s0 = d0 ? make_ulonglong2(0ull, 0ull) : __ldg(A.eh + q0);
                const ulonglong2 s1 = d1 ? make_ulonglong2(0ull, 0ull) : __ldg(A.eh + q1);
                if (!d0) {
                  ++ls.probe;
                  if (s0.x == k0) { p0 = (int64_t)s0.y; d0 = true; }
                  else if (s0.x == NH_EMPTY_KEY) d0 = true;
                  else q0 = (q0 + 1) & A.eh_mask;
                }
                if (!d1) {
                  ++ls.probe;
                  if (s1.x == k1) { p1 = (int64_t)s1.y; d1 = true; }
                  else if (s1.x == NH_EMPTY_KEY) d1 = true;
                  else q1 = (q1 + 1) & A.eh_mask;
                }
              }
            } else {
              // first entries with w' >= w in both lists, searched in lockstep over the compact
              // third-vertex array (4-byte entries: the last five steps of a search stay within
              // one 128-byte line) rather than the 16-byte mirrored entries
              int64_t a0 = l0, b0 = h0, a1 = l1, b1 = h1;
              ls.scan += (65 - __clzll((unsigned long long)(h0 - l0))) + (65 - __clzll((unsigned long long)(h1 - l1)));
              while (a0 < b0 || a1 < b1) {
                const int64_t m0 = (a0 + b0) >> 1, m1 = (a1 + b1) >> 1;
                const int32_t x0 = (a0 < b0) ? __ldg(g.etw + m0) : 0;
                const int32_t x1 = (a1 < b1) ? __ldg(g.etw + m1) : 0;
                if (a0 < b0) { if (x0 < w) a0 = m0 + 1; else b0 = m0; }
                if (a1 < b1) { if (x1 < w) a1 = m1 + 1; else b1 = m1; }
              }
              p0 = a0;
              p1 = a1;
            }
            ok = p0 >= 0 && p1 >= 0 && p0 < h0 && p1 < h1;
            if (ok) {
              f0 = __ldcg(A.et3 + p0);
              f1 = __ldcg(A.et3 + p1);
              ok = f0.x == w && f1.x == w;
              if (ok) ls.scan += 6;
            }
          }
        }
        if (ok) {
          // members in edge order: the scanned list's triangle at bt, the others at i0 < i1
          const int32_t mem[3] = {bt == 0 ? en.y : f0.y, bt == 1 ? en.y : (bt == 0 ? f0.y : f1.y),
                                  bt == 2 ? en.y : f1.y};
          const uint32_t rdv[3] = {(uint32_t)(bt == 0 ? en.z : f0.z), (uint32_t)(bt == 1 ? en.z : (bt == 0 ? f0.z : f1.z)),
                                   (uint32_t)(bt == 2 ? en.z : f1.z)};
          const uint32_t cv[3] = {(uint32_t)(bt == 0 ? en.w : f0.w), (uint32_t)(bt == 1 ? en.w : (bt == 0 ? f0.w : f1.w)),
                                  (uint32_t)(bt == 2 ? en.w : f1.w)};
          process_S_pre<3, EXACT>(A, Rid, mem, rdv, cv, t, thr, nf, W, ls);
        }
        if constexpr (EXACT) wl_maybe_flush(W, A, Rid, lane, kPerLane, ls);
      }
      return;
    }
    if (lane == 0 && c0 == 0 && se == 0) ls.scan += (unsigned long long)(th[bt] - tl[bt]);
    for (int64_t c = c0; c < cend && tl[bt] + 32 * c < th[bt]; c += cstep) {
      const int64_t j = tl[bt] + 32 * c + lane;
      bool ok = j < th[bt];
      int32_t mem[3] = {0, 0, 0};
      if (ok) {
        const int32_t w = __ldg(g.etw + j);
        mem[bt] = __ldg(g.ettid + j);
        // without links, an s-clique whose member from the scanned list is dead, below the level
        // or another frontier member's is none of R's business: skip the two searches
        ok = member_may_count(A, Rid, mem[bt], t, thr, ls);
#pragma unroll
        for (int i = 0; i < 3; i++) {
          if (i != bt && ok) {
            const int64_t p = nh_find(g.etw, tl[i], th[i], w);
            ls.scan += 65 - __clzll((unsigned long long)(th[i] - tl[i]));  // search steps and the id
            if (p < 0) ok = false;
            else mem[i] = __ldg(g.ettid + p);
          }
        }
      }
      if (ok) process_S<3, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
      if constexpr (EXACT) wl_maybe_flush(W, A, Rid, lane, kPerLane, ls);
    }
    return;
  }
  if constexpr (R == 2 && S == 3) {
    if (g.t2off) {
      // the triangles of edge Rid are its triangle list: members {a,w} and {b,w} read directly
      const int64_t b0 = __ldg(g.t2off + Rid), b1 = __ldg(g.t2off + Rid + 1);
      if (lane == 0 && c0 == 0 && se == 0) ls.scan += (unsigned long long)(2 * (b1 - b0));
      for (int64_t c = c0; c < cend && b0 + 32 * c < b1; c += cstep) {
        const int64_t j = b0 + 32 * c + lane;
        if (j < b1) {
          const int32_t mem[2] = {__ldg(g.t2ea + j), __ldg(g.t2eb + j)};
          process_S<2, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
        }
        if constexpr (EXACT) wl_maybe_flush(W, A, Rid, lane, kPerLane, ls);
      }
      return;
    }
  }
  int64_t lo[3], hi[3];
#pragma unroll
  for (int i = 0; i < R; i++) {
    lo[i] = __ldg(g.off + vx[i]);
    hi[i] = __ldg(g.off + vx[i] + 1);
  }
  int best = 0;
#pragma unroll
  for (int i = 1; i < R; i++)
    if (hi[i] - lo[i] < hi[best] - lo[best]) best = i;
  const int64_t b0 = lo[best], b1 = hi[best];
  if (lane == 0 && c0 == 0 && se == 0) ls.scan += (unsigned long long)(b1 - b0);
  for (int64_t c = c0; c < cend && b0 + 32 * c < b1; c += cstep) {
    const int64_t j = b0 + 32 * c + lane;
    bool ok = j < b1;
    int32_t w = 0;
    int32_t ew[3] = {0, 0, 0};
    if (ok) {
      w = __ldg(g.adj + j);
#pragma unroll
      for (int i = 0; i < R; i++) {
        if (i == best) {
          ew[i] = __ldg(g.eid + j);
        } else if (ok) {
          const int64_t id = nh_edge_id(g, vx[i], w);  // one probe instead of a binary search
          ls.scan += 3;                               // an 8-byte key and a 4-byte id
          if (id < 0) ok = false;
          else ew[i] = (int32_t)id;
        }
      }
    }
    if constexpr (S - R == 1) {
      if (ok) {
        if constexpr (R == 1) {
          const int32_t mem[1] = {w};
          process_S<1, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
        } else if constexpr (R == 2) {
          const int32_t mem[2] = {ew[0], ew[1]};
          process_S<2, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
        } else {
          const int32_t mem[3] = {
              tri_id(A, nh_tri_key(vx[0], vx[1], w, eR[0], ew[0], ew[1]), ls),
              tri_id(A, nh_tri_key(vx[0], vx[2], w, eR[1], ew[0], ew[2]), ls),
              tri_id(A, nh_tri_key(vx[1], vx[2], w, eR[2], ew[1], ew[2]), ls)};
          process_S<3, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
        }
      }
    } else {
      // s - r = 2: pairs (w, x), x in N+(w) adjacent to every vertex of R, expanded across the
      // warp so that lanes share the out-lists of the candidates found in this chunk
      const uint32_t len =
          (ok && (lane % Ge) == se) ? (uint32_t)(__ldg(g.ooff + w + 1) - __ldg(g.ooff + w)) : 0u;
      uint32_t incl = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(NH_FULL, incl, d);
        if (lane >= d) incl += o;
      }
      const uint32_t total = __shfl_sync(NH_FULL, incl, 31);
      for (uint32_t pb = 0; pb < total; pb += 32) {
        const uint32_t idx = pb + lane;
        int own = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const uint32_t v = __shfl_sync(NH_FULL, incl, own + step - 1);
          if (v <= idx) own += step;
        }
        const int32_t ow = __shfl_sync(NH_FULL, w, own);
        const uint32_t oincl = __shfl_sync(NH_FULL, incl, own);
        const uint32_t olen = __shfl_sync(NH_FULL, len, own);
        const int32_t oe0 = __shfl_sync(NH_FULL, ew[0], own);
        const int32_t oe1 = __shfl_sync(NH_FULL, ew[1], own);
        if (idx < total) {
          const int64_t q = __ldg(g.ooff + ow) + (int64_t)(idx - (oincl - olen));
          const int32_t x = __ldg(g.oadj + q);
          const int32_t e_wx = __ldg(g.oeid + q);
          ls.scan += 2;
          bool okx = true;
          int32_t ex[2] = {0, 0};
#pragma unroll
          for (int i = 0; i < R; i++) {
            if (!okx) break;
            const int64_t id = nh_edge_id(g, vx[i], x);
            ls.scan += 3;
            if (id < 0) okx = false;
            else ex[i] = (int32_t)id;
          }
          if (okx) {
            if constexpr (R == 1) {
              const int32_t mem[2] = {ow, x};
              process_S<2, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
            } else if constexpr (R == 2) {
              const int32_t mem[5] = {oe0, oe1, ex[0], ex[1], e_wx};
              process_S<5, EXACT>(A, Rid, mem, t, thr, nf, W, ls);
            }
          }
        }
        if constexpr (EXACT) wl_maybe_flush(W, A, Rid, lane, kPerLane, ls);
      }
    }
    if constexpr (EXACT && S - R == 1) wl_maybe_flush(W, A, Rid, lane, kPerLane, ls);
  }
}

// Work-proportional form: a list of at most kTaskItems r-cliques is cut into tasks of one
// 32-entry chunk each (for s - r = 2: one Ge-th of a chunk's out-list expansions), which warps
// take from a shared counter, so that a round lasts about its total work over the grid rather
// than its heaviest r-clique.  Every block builds the inclusive prefix sums of the chunk counts
// in shared memory itself (block-collective); false when the total does not fit 31 bits.
template <int R, int S>
__device__ __forceinline__ bool relist_prefix(const PeelArgs& A, const int32_t* items, unsigned int n, int lane,
                                              uint32_t* s_pref, unsigned long long* s_wsum,
                                              unsigned long long& total) {
  constexpr int kPer = kTaskItems / kThreads;
  const unsigned int b = threadIdx.x * kPer;
  uint32_t v[kPer];
  unsigned long long sum = 0;
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    v[j] = (b + j < n) ? __ldg(A.cost + __ldcg(items + b + j)) : 0u;
    sum += v[j];
  }
  unsigned long long incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(NH_FULL, incl, d);
    if (lane >= d) incl += o;
  }
  __syncthreads();  // the previous round's readers of s_pref / s_wsum are done
  if (lane == 31) s_wsum[threadIdx.x >> 5] = incl;
  __syncthreads();
  unsigned long long base = incl - sum;
  total = 0;
  for (int w = 0; w < kThreads / 32; w++) {
    const unsigned long long x = s_wsum[w];
    if (w < (int)(threadIdx.x >> 5)) base += x;
    total += x;
  }
  if (total >= (1ull << 31)) return false;
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    base += v[j];
    if (b + j < n) s_pref[b + j] = (uint32_t)base;
  }
  __syncthreads();
  return true;
}

// Re-lists the n r-cliques of items: in tasks (see relist_prefix) when `tasks`, else with G warps
// per r-clique (G, a power of two up to gmax, as many as the grid has for the list; G = 1: warps
// take r-cliques in batches from a shared counter; for s - r = 2
// the G warps form G / Ge chunk-groups of Ge warps, the Ge warps of one chunk-group scanning the
// same 32 candidates and each expanding the out-lists of every Ge-th of them).  One call site of
// relist_item per kernel.
template <int R, int S, bool EXACT>
__device__ __forceinline__ void relist_list(const PeelArgs& A, const int32_t* items, unsigned long long n, bool tasks,
                                            unsigned long long total, uint32_t t, uint32_t thr, int32_t* nf,
                                            int lane, long long gwarp, long long nwarps, const WarpLinks& W,
                                            LocalStats& ls, const uint32_t* s_pref, unsigned long long* task_next) {
  // task form
  int Ge_t = 1;
  if constexpr (S - R == 2)
    while (Ge_t < 32 && total * (unsigned long long)(2 * Ge_t) <= 4ull * (unsigned long long)nwarps) Ge_t *= 2;
  const unsigned long long ntask = total * (unsigned long long)Ge_t;
  const unsigned long long per = ntask / ((unsigned long long)nwarps * 8ull);
  const unsigned long long bt = per > 0 ? per : 1ull;
  unsigned long long k = 0, k1 = 0;
  // group form
  int G = 1;
  while (G < A.gmax && (unsigned long long)(2 * G) * n <= (unsigned long long)nwarps) G *= 2;
  const int Ge = (S - R == 2) ? (G < 32 ? G : 32) : 1;
  const long long ngroups = nwarps / G, grp = gwarp / G;
  const int sub = (int)(gwarp % G), Gc = G / Ge, sc = sub / Ge, se_g = sub % Ge;
  unsigned long long it = (unsigned long long)grp;
  // one warp per r-clique: r-cliques in batches from the shared counter (per-r-clique work is
  // heavy-tailed, so a fixed stride would leave the round to its unluckiest warp)
  const unsigned long long dNW = (unsigned long long)nwarps;
  const unsigned long long drest = n > dNW ? n - dNW : 0ull;
  const unsigned long long dper = drest / (dNW * 16ull);
  const unsigned long long dbt = dper > 0 ? dper : 1ull;
  unsigned long long dk = (unsigned long long)gwarp, dk1 = dk + 1;  // r-clique gwarp first
  int32_t curR = -1;
  for (;;) {
    int32_t Rid;
    int64_t c0, cstep, cend;
    int ge, se;
    if (tasks) {
      if (k >= k1) {
        unsigned long long k0 = 0;
        if (lane == 0) k0 = atomicAdd(task_next, bt);
        k0 = __shfl_sync(NH_FULL, k0, 0);
        if (k0 >= ntask) break;
        k = k0;
        k1 = k0 + bt < ntask ? k0 + bt : ntask;
      }
      const uint32_t kc = (uint32_t)(k / (unsigned long long)Ge_t);
      unsigned int lo = 0, hi = (unsigned int)n;  // first item whose inclusive prefix exceeds kc
      while (lo < hi) {
        const unsigned int mid = (lo + hi) >> 1;
        if (s_pref[mid] <= kc) lo = mid + 1; else hi = mid;
      }
      const uint32_t cl = kc - (lo ? s_pref[lo - 1] : 0u);
      // with whole chunks (Ge = 1) the run of this batch's chunks within one item is one call
      const unsigned long long run =
          Ge_t == 1 ? ((unsigned long long)s_pref[lo] < k1 ? (unsigned long long)s_pref[lo] : k1) - k : 1ull;
      Rid = __ldcg(items + lo);
      c0 = cl;
      cstep = 1;
      cend = (int64_t)cl + (int64_t)run;
      ge = Ge_t;
      se = (int)(k % (unsigned long long)Ge_t);
      k += run;
    } else if (G == 1) {
      if (dk >= dk1) {
        if (drest == 0) break;
        unsigned long long k0 = 0;
        if (lane == 0) k0 = atomicAdd(task_next, dbt);
        k0 = dNW + __shfl_sync(NH_FULL, k0, 0);
        dk = k0;
        dk1 = k0 + dbt < n ? k0 + dbt : n;
      }
      if (dk >= n) break;
      Rid = __ldcg(items + dk);
      ++dk;
      c0 = 0;
      cstep = 1;
      cend = INT64_MAX;
      ge = 1;
      se = 0;
    } else {
      if (grp >= ngroups || it >= n) break;
      Rid = __ldcg(items + it);
      it += (unsigned long long)ngroups;
      c0 = sc;
      cstep = Gc;
      cend = INT64_MAX;
      ge = Ge;
      se = se_g;
    }
    if (Rid != curR) {
      if constexpr (EXACT) {
        if (curR >= 0) wl_flush(W, A, curR, lane, ls);
        wl_begin(W, lane);
      }
      curR = Rid;
    }
    relist_item<R, S, EXACT>(A, Rid, t, thr, nf, lane, c0, cstep, cend, ge, se, W, ls);
  }
  if constexpr (EXACT) {
    if (curR >= 0) wl_flush(W, A, curR, lane, ls);
  }
}

}  // namespace nhp

#include "nh_relist24.cuh"

namespace nhp {

// ---------------------------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------------------------

// The leaders run in the last block to reach a grid barrier, while every other block waits: they
// read every control word they need at once (independent loads from L2), then write the next
// round's words.
template <bool EXACT>
__device__ void leader_after_scan(const PeelArgs& A) {
  PeelCtl* c = A.lk.ctl;
  const unsigned int gm = __ldcg(&c->gmin), ac = __ldcg(&c->alive_cur), thr0 = __ldcg(&c->thr);
  const unsigned int bucket0 = __ldcg(&c->bucket);
  const unsigned long long a2 = __ldcg(&c->alive2_count), lv = __ldcg(&c->st_levels);
  c->gmin = kNone;
  c->alive_cur = ac ^ 1u;
  c->alive_n = a2;
  c->alive2_count = 0;
  c->f_count = 0;
  if (EXACT) {
    if (gm != kNone && gm > thr0) c->thr = gm;
  } else {
    unsigned int b = bucket0;
    while ((int)b + 1 < A.n_thr && A.thresholds[b] < gm) b++;
    if (b != bucket0) {
      c->bucket = b;
      c->rounds_in_bucket = 0;
    }
    c->thr = A.thresholds[b];
  }
  c->st_levels = lv + 1;
}

template <bool EXACT>
__device__ void leader_end_of_round(const PeelArgs& A) {
  PeelCtl* c = A.lk.ctl;
  const unsigned int oc = __ldcg(&c->ovf_cur), thr = __ldcg(&c->thr), kmax = __ldcg(&c->kmax);
  const unsigned int t = __ldcg(&c->t), cur = __ldcg(&c->cur), rib = __ldcg(&c->rounds_in_bucket);
  const unsigned int bucket = __ldcg(&c->bucket);
  const unsigned long long ov0 = __ldcg(&c->ovf_count[0]), ov1 = __ldcg(&c->ovf_count[1]);
  const unsigned long long finished = __ldcg(&c->finished), fsize = __ldcg(&c->fsize);
  const unsigned long long rounds = __ldcg(&c->st_rounds), front = __ldcg(&c->st_front);
  const unsigned long long nfc = __ldcg(&c->nf_count), hn = __ldcg(&c->c24_hn);
  c->task_next = 0;
  c->c24_next = 0;
  c->c24_hn = 0;
  c->c24_hk = 0;
  c->c24_done = 0;
  const unsigned long long ovc = oc ? ov1 : ov0;
  if (ovc > 0) {
    c->draining = 1;
    c->drain_buf = oc;
    c->drain_n = ovc < A.lk.ovf_cap ? ovc : A.lk.ovf_cap;
    c->ovf_count[oc] = 0;
    c->ovf_cur = oc ^ 1u;
    return;
  }
  c->draining = 0;
  c->finished = finished + fsize;
  if (A.round_log && rounds < A.round_log_cap) {
    unsigned long long* L = A.round_log + 8 * rounds;
    L[0] = (fsize << 32) | (__ldcg(&c->st_levels) & 0xffffffffull);
    L[1] = nh_globaltimer();
    L[2] = __ldcg(&c->dbg_work);
    L[3] = (__ldcg(&c->c24_tasks) << 32) | (hn & 0xffffffffull);
    c->dbg_work = 0;
  }
  c->st_rounds = rounds + 1;
  c->st_front = front + fsize;
  if (thr > kmax && fsize > 0) c->kmax = thr;
  c->t = t + 1;
  if (finished + fsize >= (unsigned long long)A.n_r) {
    c->done = 1;
    return;
  }
  if (!EXACT) {
    if (rib + 1 >= A.T) {
      const unsigned int b = ((int)bucket + 1 < A.n_thr) ? bucket + 1 : bucket;
      c->bucket = b;
      c->rounds_in_bucket = 0;
      c->thr = A.thresholds[b];
      c->need_scan = 1;
      c->nf_count = 0;
      return;
    }
    c->rounds_in_bucket = rib + 1;
  }
  if (nfc > 0) {
    c->cur = cur ^ 1u;
    c->fsize = nfc;
    c->nf_count = 0;
    c->need_scan = 0;
  } else {
    c->need_scan = 1;
  }
}

// resident blocks per SM a kernel is compiled for: (2,4) stages candidates in about 50 KB of
// shared memory per block and gets the registers of three blocks per SM
template <int R, int S>
constexpr int min_blocks() { return (R == 2 && S == 4) ? 3 : kMinBlocks; }

// C24: the (2,4) triangle-list re-listing (nh_relist24.cuh) in place of the adjacency / chunk-task
// path, as its own instantiation so that neither carries the other's registers
template <int R, int S, bool EXACT, bool C24>
__global__ void __launch_bounds__(kThreads, min_blocks<R, S>()) k_peel(PeelArgs A) {
  PeelCtl* ctl = A.lk.ctl;
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  extern __shared__ __align__(16) unsigned char s_dyn[];
  unsigned long long* s_links = reinterpret_cast<unsigned long long*>(s_dyn + kSmLinks);
  uint32_t* s_pref = reinterpret_cast<uint32_t*>(s_dyn + kSmPref);
  int32_t* s_seen = reinterpret_cast<int32_t*>(s_dyn + kSmSeen);
  unsigned long long* s_wsum = reinterpret_cast<unsigned long long*>(s_dyn + kSmWsum);
  int* s_lcnt = reinterpret_cast<int*>(s_dyn + kSmLcnt);
  constexpr bool use24 = C24;
  if (!use24 && lane == 0) s_lcnt[threadIdx.x >> 5] = 0;
  __syncwarp();
  const WarpLinks W{s_links + (threadIdx.x >> 5) * kLinkBuf, &s_lcnt[threadIdx.x >> 5], s_seen + (threadIdx.x >> 5) * kSeen};
  __shared__ RoundView s_rv;
  if (threadIdx.x == 0) round_view_load(ctl, &s_rv);
  __syncthreads();
  const RoundView& rv = s_rv;
  for (;;) {
    if (rv.done || rv.err) break;
    if (rv.need_scan) {
      // compact the live list and take the minimum count over it
      {
        const unsigned int ac = rv.alive_cur;
        const int32_t* ain = A.alive[ac];
        int32_t* aout = A.alive[ac ^ 1u];
        const unsigned long long na = rv.alive_n;
        const unsigned int t = rv.t;
        uint32_t lmin = kNone;
        for (unsigned long long base = (unsigned long long)gwarp * 32; base < na;
             base += (unsigned long long)nwarps * 32) {
          const unsigned long long i = base + lane;
          bool live = false;
          int32_t x = 0;
          if (i < na) {
            x = __ldcg(ain + i);
            const uint32_t rd = __ldcg(A.round + x);
            live = (rd == 0u || rd >= t);
            if (live) lmin = min(lmin, __ldcg(A.cnt + x));
          }
          const unsigned long long pos = warp_append(&ctl->alive2_count, live, lane);
          if (live) aout[pos] = x;
        }
        lmin = warp_min_u32(lmin);
        if (lane == 0 && lmin != kNone) atomicMin(&ctl->gmin, lmin);
      }
      if (!grid_sync_view(ctl, A.timeout_ns, &s_rv, [&] { leader_after_scan<EXACT>(A); })) break;
      // frontier = live with count <= threshold
      {
        const int32_t* al = A.alive[rv.alive_cur];
        const unsigned long long na = rv.alive_n;
        const unsigned int thr = rv.thr, t = rv.t;
        int32_t* fr = A.front[rv.cur];
        for (unsigned long long base = (unsigned long long)gwarp * 32; base < na;
             base += (unsigned long long)nwarps * 32) {
          const unsigned long long i = base + lane;
          bool take = false;
          int32_t x = 0;
          if (i < na) {
            x = __ldcg(al + i);
            take = __ldcg(A.cnt + x) <= thr;
          }
          const unsigned long long pos = warp_append(&ctl->f_count, take, lane);
          if (take) {
            fr[pos] = x;
            const uint32_t v = EXACT ? thr : min(thr, __ldg(A.cnt0 + x));
            __stcg(A.round + x, t);
            __stcg(A.val + x, v);
            if constexpr (R == 3 && S == 4) {
              if (A.et3) mirror_set(A, x, t, v);
            }
          }
        }
      }
      if (!grid_sync_view(ctl, A.timeout_ns, &s_rv, [&] {
            ctl->fsize = __ldcg(&ctl->f_count);
            ctl->f_count = 0;
          }))
        break;
    }
    // re-list the frontier
    {
      const unsigned int t = rv.t, thr = rv.thr, cur = rv.cur;
      const unsigned long long fs = rv.fsize;
      const int32_t* fr = A.front[cur];
      int32_t* nf = A.front[cur ^ 1u];
      if constexpr (use24) {
        if (A.round_log && blockIdx.x == 0 && threadIdx.x == 0 && t >= 1 && t <= A.round_log_cap)
          A.round_log[8 * (t - 1) + 4] = nh_globaltimer();
        c24_list<EXACT>(A, fr, fs, t, thr, nf, gwarp, nwarps, s_dyn, ls);
      } else {
        unsigned long long total = 0;
        const bool tasks = fs <= (unsigned long long)A.task_items &&
                           relist_prefix<R, S>(A, fr, (unsigned int)fs, lane, s_pref, s_wsum, total);
        relist_list<R, S, EXACT>(A, fr, fs, tasks, total, t, thr, nf, lane, gwarp, nwarps, W, ls, s_pref,
                                 &ctl->task_next);
      }
    }
    // end of round: drain deferred link calls, then advance
    bool ok = true;
    for (;;) {
      if (!grid_sync_view(ctl, A.timeout_ns, &s_rv, [&] { leader_end_of_round<EXACT>(A); })) { ok = false; break; }
      if (!rv.draining) break;
      if constexpr (!C24) {  // the triangle-list re-listing never links, so never defers a call
        const int2* q = A.lk.ovf[rv.drain_buf];
        const unsigned long long nq = rv.drain_n;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
             i += (unsigned long long)gridDim.x * blockDim.x) {
          const int2 p = __ldcg(q + i);
          add_delta(ls, link_run_call(A.lk, p.x, p.y));
        }
      }
    }
    if (!ok) break;
  }
  if (A.stats) {
    const unsigned long long v0 = warp_sum_u64(ls.listed), v1 = warp_sum_u64(ls.dec), v2 = warp_sum_u64(ls.link),
                             v3 = warp_sum_u64(ls.unite), v4 = warp_sum_u64(ls.scan), v5 = warp_sum_u64(ls.probe),
                             v6 = warp_sum_u64(ls.ovf), v7 = warp_sum_u64(ls.stamp);
    if (lane == 0) {
      atomicAdd(&ctl->st_stamp, v7);
      atomicAdd(&ctl->st_listed, v0);
      atomicAdd(&ctl->st_dec, v1);
      atomicAdd(&ctl->st_link, v2);
      atomicAdd(&ctl->st_unite, v3);
      atomicAdd(&ctl->st_scan, v4);
      atomicAdd(&ctl->st_probe, v5);
      atomicAdd(&ctl->st_ovf, v6);
    }
  }
}

template <int R, int S, bool EXACT>
int launch_peel(PeelArgs& A, cudaStream_t st) {
  const void* fn = (const void*)k_peel<R, S, EXACT, false>;
  if constexpr (R == 2 && S == 4) {
    if (A.use24) fn = (const void*)k_peel<R, S, EXACT, true>;
  }
  int dev = 0, sms = 0, per = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return NH_ERR_UNSUPPORTED;
  const int smem = A.use24 ? kC24SmemBytes : kSmOldBytes;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return NH_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, smem) != cudaSuccess || per < 1)
    return NH_ERR_CUDA;
  dim3 grid((unsigned)(sms * per)), block(kThreads);
  void* args[] = {&A};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, grid, block, args, (size_t)smem, st);
  nh_note_launch();
  return e == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------------
// §7.4 practical two-phase hierarchy (anh-te): with the core numbers known, levels are processed
// from the largest core down to 1 with one union-find: at level c every r-clique of core c
// re-lists its s-cliques and joins the members of those whose least core is c; then every
// component holding an r-clique of core c gets a node at level c, which adopts the previous top
// nodes of the components it absorbed.  One persistent cooperative kernel, four grid barriers
// per level.
// ---------------------------------------------------------------------------------------------


struct TreeOut {
  const int32_t* order;    // r-cliques sorted by core (any order within a level)
  const int64_t* lvl_off;  // [kmax + 2]
  uint32_t kmax;
  uint32_t* lvl;           // per root: last level it got a node
  int32_t* nid;            // per root: that node
  int32_t* top;            // per root: current top node of its component
  int32_t* parent;         // [n_r + nodes]
  uint32_t* label;
  unsigned long long* node_count;
};

template <int R, int S, bool C24>
__global__ void __launch_bounds__(kThreads, min_blocks<R, S>()) k_two_phase(PeelArgs A, TreeOut T) {
  PeelCtl* ctl = A.lk.ctl;
  volatile PeelCtl* vc = ctl;
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  extern __shared__ __align__(16) unsigned char s_dyn[];
  unsigned long long* s_links = reinterpret_cast<unsigned long long*>(s_dyn + kSmLinks);
  uint32_t* s_pref = reinterpret_cast<uint32_t*>(s_dyn + kSmPref);
  int32_t* s_seen = reinterpret_cast<int32_t*>(s_dyn + kSmSeen);
  unsigned long long* s_wsum = reinterpret_cast<unsigned long long*>(s_dyn + kSmWsum);
  int* s_lcnt = reinterpret_cast<int*>(s_dyn + kSmLcnt);
  constexpr bool use24 = C24;
  if (!use24 && lane == 0) s_lcnt[threadIdx.x >> 5] = 0;
  __syncwarp();
  const WarpLinks W{s_links + (threadIdx.x >> 5) * kLinkBuf, &s_lcnt[threadIdx.x >> 5], s_seen + (threadIdx.x >> 5) * kSeen};
  const int64_t n_r = A.n_r;
  for (uint32_t level = T.kmax; level >= 1; --level) {
    const int64_t lo = T.lvl_off[level], hi = T.lvl_off[level + 1];
    const unsigned long long cnt = (unsigned long long)(hi - lo);
    if (cnt == 0) continue;
    // unions at this level
    if constexpr (use24) {
      c24_list<true>(A, T.order + lo, cnt, 0u, level, nullptr, gwarp, nwarps, s_dyn, ls);
    } else {
      unsigned long long total = 0;
      const bool tasks = cnt <= (unsigned long long)A.task_items &&
                         relist_prefix<R, S>(A, T.order + lo, (unsigned int)cnt, lane, s_pref, s_wsum, total);
      relist_list<R, S, true>(A, T.order + lo, cnt, tasks, total, 0u, level, nullptr, lane, gwarp, nwarps, W, ls,
                              s_pref, &ctl->task_next);
    }
    if (!grid_sync(ctl, A.timeout_ns, [&] {
          ctl->task_next = 0;
          ctl->c24_next = 0;
          ctl->c24_hn = 0;
          ctl->c24_hk = 0;
          ctl->c24_done = 0;
        }))
      break;
    // a node for every component holding an r-clique of this level (with labels that are not
    // core numbers, an r-clique in no s-clique at its own level is alone there: no node; it
    // becomes a leaf of the first node its component gets at a lower level, through the touched
    // list below)
    for (long long i = gtid; i < (long long)cnt; i += nthreads) {
      const int32_t R0 = T.order[lo + i];
      if (A.mark && !__ldcg(A.mark + R0)) continue;
      const int32_t y = uf_find(A.lk.uf, R0);
      uint32_t cur = __ldcg(T.lvl + y);
      while (cur != level) {
        const uint32_t prev = atomicCAS(T.lvl + y, cur, level);
        if (prev == cur) {
          const int32_t id = (int32_t)atomicAdd(T.node_count, 1ull);
          T.nid[y] = id;
          T.label[id] = level;
          T.parent[n_r + id] = -1;
          break;
        }
        cur = prev;
      }
    }
    if (!grid_sync(ctl, A.timeout_ns, [] {})) break;
    // leaves of this level, and previous top nodes of every joined component
    for (long long i = gtid; i < (long long)cnt; i += nthreads) {
      const int32_t R0 = T.order[lo + i];
      if (A.mark && !__ldcg(A.mark + R0)) continue;
      T.parent[R0] = __ldcg(T.nid + uf_find(A.lk.uf, R0));
    }
    {
      const unsigned long long nt = *(volatile unsigned long long*)A.touched_n;
      for (unsigned long long i = (unsigned long long)gtid; i < nt; i += (unsigned long long)nthreads) {
        const int32_t x = __ldcg(A.touched + i);
        const int32_t tp = __ldcg(T.top + x);
        if (tp >= 0) T.parent[n_r + tp] = __ldcg(T.nid + uf_find(A.lk.uf, x));
        else if (A.mark) T.parent[x] = __ldcg(T.nid + uf_find(A.lk.uf, x));  // x was alone until now
      }
    }
    if (!grid_sync(ctl, A.timeout_ns, [&] { *A.touched_n = 0; })) break;
    for (long long i = gtid; i < (long long)cnt; i += nthreads) {
      const int32_t R0 = T.order[lo + i];
      if (A.mark && !__ldcg(A.mark + R0)) continue;
      const int32_t y = uf_find(A.lk.uf, R0);
      T.top[y] = __ldcg(T.nid + y);
    }
    if (!grid_sync(ctl, A.timeout_ns, [] {})) break;
  }
  if (A.stats) {
    const unsigned long long v0 = warp_sum_u64(ls.listed), v3 = warp_sum_u64(ls.unite);
    if (lane == 0) {
      atomicAdd(&ctl->st_listed, v0);
      atomicAdd(&ctl->st_unite, v3);
    }
  }
}

template <int R, int S>
int launch_two_phase(PeelArgs& A, TreeOut& T, cudaStream_t st) {
  const void* fn = (const void*)k_two_phase<R, S, false>;
  if constexpr (R == 2 && S == 4) {
    if (A.use24) fn = (const void*)k_two_phase<R, S, true>;
  }
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = A.use24 ? kC24SmemBytes : kSmOldBytes;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return NH_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, smem) != cudaSuccess || per < 1) return NH_ERR_CUDA;
  void* args[] = {&A, &T};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)(sms * per)), dim3(kThreads), args, (size_t)smem, st);
  nh_note_launch();
  return e == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

// per-(r,s) entry points, one translation unit each
int peel_launch_pair(int r, int s, bool exact, PeelArgs& A, cudaStream_t st);
int two_phase_launch_pair(int r, int s, PeelArgs& A, TreeOut& T, cudaStream_t st);
int chunk_cost_pair(int r, int s, const GView& g, int64_t n_r, uint32_t* cost, cudaStream_t st);

#define NH_PEEL_PAIR(R, S)                                                                          \
  int peel_launch_##R##S(bool exact, PeelArgs& A, cudaStream_t st) {                                \
    return exact ? launch_peel<R, S, true>(A, st) : launch_peel<R, S, false>(A, st);                \
  }                                                                                                 \
  int two_phase_launch_##R##S(PeelArgs& A, TreeOut& T, cudaStream_t st) {                          \
    return launch_two_phase<R, S>(A, T, st);                                                        \
  }                                                                                                 \
  int chunk_cost_##R##S(const GView& g, int64_t n_r, uint32_t* cost, cudaStream_t st) {             \
    k_chunk_cost<R, S><<<nh_blocks_for(n_r, 256, 152 * 16), 256, 0, st>>>(g, n_r, cost);            \
    nh_note_launch();                                                                               \
    return NH_OK;                                                                                   \
  }

#define NH_PEEL_PAIR_DECL(R, S)                                                 \
  int peel_launch_##R##S(bool exact, PeelArgs& A, cudaStream_t st);            \
  int two_phase_launch_##R##S(PeelArgs& A, TreeOut& T, cudaStream_t st);       \
  int chunk_cost_##R##S(const GView& g, int64_t n_r, uint32_t* cost, cudaStream_t st);
NH_PEEL_PAIR_DECL(1, 2)
NH_PEEL_PAIR_DECL(1, 3)
NH_PEEL_PAIR_DECL(2, 3)
NH_PEEL_PAIR_DECL(2, 4)
NH_PEEL_PAIR_DECL(3, 4)

}  // namespace nhp
