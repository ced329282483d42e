// nh_generic.cu -- the pairs 1 <= r < s <= 7 beyond the specialised ones (§1 and §8 run r < s <= 7),
// and link-basic (Alg. 4) for every pair.
//
//   index      r = 4..6: a chain of hash tables; the r-cliques are listed per (r-1)-clique P in
//              lexicographic order of P as the common neighbours above P's largest vertex, so ids
//              are lexicographic; the key of (p_0 < ... < p_{r-2} < c) is id(P) << 32 | c (the r = 3
//              table keys triangles the same way on the edge id of their two smaller vertices).
//   counting   rec-list-cliques (Alg. 3, count step): one warp per out-edge (v -> a) stages
//              B = N+(v) n N+(a) and lists the (s-2)-cliques inside B (lanes split the first
//              vertex, each lane searches on); every s-clique is listed once, and each of its
//              C(s,r) r-subsets is looked up in the chain and counted.
//   peel       Alg. 3's rounds (exact) or Alg. 2's buckets (approximate), one host round trip per
//              round: the frontier A = {alive : count <= threshold} is compacted from the alive
//              list, stamped, and re-listed one warp per r-clique (common neighbours of its
//              vertices, then (s-r)-cliques among them); an s-clique with a member peeled in an
//              earlier round is dead, otherwise its frontier member of least id decrements the
//              others once (each s-clique dies once).
//   hierarchy  link-efficient (Alg. 5) over every s-clique after the peel: the definitional
//              reading links the member of least value with every other member (level c_S), the
//              pair rule links the member of largest value with every other member; then
//              construct-tree (nh_tree.cu).  The same calls on arbitrary labels give the label
//              hierarchy.
//   link-basic Alg. 4: one union-find per level 1..kmax; an s-clique unites its members in every
//              level up to c_S; construct-tree-basic builds the tree level by level from the top,
//              one node per component that is not already a component one level up.
#include <cmath>
#include <vector>

#include "nh_peel.cuh"

namespace {

using nhp::LinkEnv;
using nhp::LocalStats;
using nhp::PeelCtl;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxS = 7;
constexpr int kMaxC = 35;     // C(7,3) = C(7,4)
constexpr int kMaxDepth = 6;  // (s - r) or (s - 2) vertices chosen inside a candidate set

// r-subsets of an s-set as bit masks; with the s vertices sorted ascending, the vertices of a mask
// taken in bit order are sorted too
struct Subsets {
  int s, r, C;
  unsigned char mask[kMaxC];
};

Subsets make_subsets(int s, int r) {
  Subsets q{};
  q.s = s;
  q.r = r;
  for (int m = 0; m < (1 << s); m++)
    if (__builtin_popcount(m) == r) q.mask[q.C++] = (unsigned char)m;
  return q;
}

// the lookups that turn a sorted r-tuple into its id
struct RChain {
  int r;
  const unsigned long long* ekey;
  const uint32_t* eval;
  unsigned long long emask;
  const nh_slot* tab[4];  // levels 3..6
  unsigned long long mask[4];
};

RChain make_chain(const nh_oriented* o, const nh_rindex* ri) {
  RChain c{};
  c.r = ri->r;
  c.ekey = o->ekey;
  c.eval = o->eval;
  c.emask = o->emask;
  for (const nh_rindex* x = ri; x && x->r >= 3; x = x->prev) {
    c.tab[x->r - 3] = x->table;
    c.mask[x->r - 3] = x->mask;
  }
  return c;
}

__device__ __forceinline__ int64_t edge_lookup(const RChain& c, int32_t x, int32_t y) {
  const unsigned long long key = (x < y) ? (((unsigned long long)(uint32_t)x << 32) | (uint32_t)y)
                                         : (((unsigned long long)(uint32_t)y << 32) | (uint32_t)x);
  unsigned long long h = nh_mix64(key) & c.emask;
  for (unsigned long long p = 0; p <= c.emask; ++p) {
    const unsigned long long k = __ldg(c.ekey + h);
    if (k == key) return (int64_t)__ldg(c.eval + h);
    if (k == NH_EMPTY_KEY) return -1;
    h = (h + 1) & c.emask;
  }
  return -1;
}

// id of the r-clique with sorted vertices v[0..r-1], or -1 when absent
__device__ __forceinline__ int64_t chain_id(const RChain& c, const int32_t* v, int r) {
  if (r == 1) return v[0];
  int64_t id = edge_lookup(c, v[0], v[1]);
  for (int l = 3; l <= r && id >= 0; ++l)
    id = nh_tri_lookup(c.tab[l - 3], c.mask[l - 3], ((unsigned long long)id << 32) | (uint32_t)v[l - 1]);
  return id;
}

__device__ __forceinline__ bool adjacent(const RChain& c, int32_t x, int32_t y) { return edge_lookup(c, x, y) >= 0; }

// ---------------------------------------------------------------------------------------------
// index r = 4..6 from the index of the (r-1)-cliques (tuples ptup, r-1 per clique)
// ---------------------------------------------------------------------------------------------

// common neighbours c > p_{q-1} of all q members of P: the member whose upper adjacency part is
// shortest is scanned, the others are binary-searched.  emit(k, c): the k-th extension (order kept).
template <class F>
__device__ __forceinline__ uint32_t extensions(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                               const int32_t* p, int q, int lane, F emit) {
  const int32_t top = p[q - 1];
  int best = 0;
  int64_t bb = 0, be = 0, blen = -1;
  for (int j = 0; j < q; j++) {
    const int64_t lo = nh_lower_bound(adj, off[p[j]], off[p[j] + 1], top + 1), hi = off[p[j] + 1];
    if (blen < 0 || hi - lo < blen) { blen = hi - lo; bb = lo; be = hi; best = j; }
  }
  uint32_t found = 0;
  for (int64_t base = bb; base < be; base += 32) {
    const int64_t k = base + lane;
    int32_t c = 0;
    bool ok = false;
    if (k < be) {
      c = adj[k];
      ok = true;
      for (int j = 0; j < q && ok; j++)
        if (j != best) ok = nh_find(adj, off[p[j]], off[p[j] + 1], c) >= 0;
    }
    const unsigned msk = __ballot_sync(NH_FULL, ok);
    if (ok) emit(found + __popc(msk & ((1u << lane) - 1u)), c);
    found += __popc(msk);
  }
  return found;
}

__global__ void k_gidx_count(int64_t np, int q, const int32_t* __restrict__ ptup, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ adj, uint32_t* __restrict__ ext) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t p[kMaxS];
  for (int64_t P = warp; P < np; P += nwarps) {
    for (int j = 0; j < q; j++) p[j] = ptup[P * q + j];
    const uint32_t n = extensions(off, adj, p, q, lane, [](uint32_t, int32_t) {});
    if (lane == 0) ext[P] = n;
  }
}

__device__ __forceinline__ bool slot_insert(nh_slot* t, unsigned long long mask, unsigned long long key, uint32_t id) {
  unsigned long long h = nh_mix64(key) & mask;
  for (unsigned long long p = 0; p <= mask; ++p) {
    const unsigned long long old = atomicCAS(&t[h].key, NH_EMPTY_KEY, key);
    if (old == NH_EMPTY_KEY || old == key) {
      t[h].val = id;
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

__global__ void k_gidx_fill(int64_t np, int q, const int32_t* __restrict__ ptup, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ adj, const int64_t* __restrict__ eoff, int32_t* __restrict__ tup,
                            nh_slot* __restrict__ table, unsigned long long mask, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t p[kMaxS];
  for (int64_t P = warp; P < np; P += nwarps) {
    for (int j = 0; j < q; j++) p[j] = ptup[P * q + j];
    const int64_t base = eoff[P];
    extensions(off, adj, p, q, lane, [&](uint32_t k, int32_t c) {
      const int64_t id = base + k;
      for (int j = 0; j < q; j++) tup[id * (q + 1) + j] = p[j];
      tup[id * (q + 1) + q] = c;
      if (!slot_insert(table, mask, ((unsigned long long)P << 32) | (uint32_t)c, (uint32_t)id))
        atomicCAS(status, 0, NH_ERR_TABLE_FULL);
    });
  }
}

__global__ void k_fill_slots(nh_slot* t, unsigned long long cap) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    t[i].key = NH_EMPTY_KEY;
    t[i].val = 0xffffffffu;
    t[i].pad = 0;
  }
}

unsigned warp_blocks(int64_t items, int64_t cap = 152 * 32) {
  int64_t b = (items + kWarps - 1) / kWarps;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------------------------
// s-clique listing with a per-clique action (counting, linking, link-basic)
// ---------------------------------------------------------------------------------------------

enum { kCount = 0, kLinkMin = 1, kLinkMax = 2, kBasic = 3 };

struct ListArgs {
  GView g;
  RChain ch;
  Subsets sub;
  int s;
  int64_t n_r;
  int32_t* buf;              // per-warp candidate buffers, cap entries each
  int64_t cap;
  uint32_t* cnt;             // kCount
  unsigned long long* n_s;   // kCount: s-cliques listed
  const uint32_t* val;       // linking: core numbers or labels
  LinkEnv lk;                // kLinkMin / kLinkMax
  int32_t* ufb;              // kBasic: kmax union-finds of n_r entries, level i at (i-1) n_r
  unsigned long long* unites;
  int* status;
};

// sorts w[0..n-1] ascending (n <= 7)
__device__ __forceinline__ void sort_small(int32_t* w, int n) {
  for (int i = 1; i < n; i++) {
    const int32_t x = w[i];
    int j = i - 1;
    while (j >= 0 && w[j] > x) { w[j + 1] = w[j]; --j; }
    w[j + 1] = x;
  }
}

// ids of the C r-subsets of the sorted s-set w; false when one is missing (status set)
__device__ __forceinline__ bool member_ids(const RChain& ch, const Subsets& sub, const int32_t* w, int32_t* mem,
                                           int* status) {
  int32_t v[kMaxS];
  for (int j = 0; j < sub.C; j++) {
    int k = 0;
    for (int b = 0; b < sub.s; b++)
      if (sub.mask[j] >> b & 1) v[k++] = w[b];
    const int64_t id = chain_id(ch, v, sub.r);
    if (id < 0) {
      atomicCAS(status, 0, NH_ERR_INTERNAL);
      return false;
    }
    mem[j] = (int32_t)id;
  }
  return true;
}

template <int MODE>
__device__ __forceinline__ void clique_action(const ListArgs& A, const int32_t* w0, LocalStats& ls,
                                              unsigned long long& found, unsigned long long& unites) {
  int32_t w[kMaxS];
  for (int j = 0; j < A.s; j++) w[j] = w0[j];
  sort_small(w, A.s);
  int32_t mem[kMaxC];
  if (!member_ids(A.ch, A.sub, w, mem, A.status)) return;
  ++found;
  const int C = A.sub.C;
  if (MODE == kCount) {
    for (int j = 0; j < C; j++) atomicAdd(A.cnt + mem[j], 1u);
    return;
  }
  // the member of least value (definitional reading; ties: least id) or of largest value (pair rule)
  int32_t m = mem[0];
  uint32_t mv = __ldg(A.val + m);
  for (int j = 1; j < C; j++) {
    const uint32_t x = __ldg(A.val + mem[j]);
    const bool better = (MODE == kLinkMax) ? (x > mv || (x == mv && mem[j] < m)) : (x < mv || (x == mv && mem[j] < m));
    if (better) { m = mem[j]; mv = x; }
  }
  if (MODE == kLinkMin || MODE == kLinkMax) {
    uint32_t lo = mv;
    if (MODE == kLinkMax)
      for (int j = 0; j < C; j++) lo = min(lo, __ldg(A.val + mem[j]));
    if (lo == 0) return;  // level 0 joins nothing
    for (int j = 0; j < C; j++)
      if (mem[j] != m) nhp::link_run(A.lk, m, mem[j], ls);
    return;
  }
  // kBasic: unite in every level 1..c_S
  for (uint32_t i = 1; i <= mv; i++) {
    int32_t* uf = A.ufb + (int64_t)(i - 1) * A.n_r;
    for (int j = 0; j < C; j++)
      if (mem[j] != m && nhp::uf_unite(uf, m, mem[j], A.lk.ctl) >= 0) ++unites;
  }
}

// one warp per out-edge (v -> a): B = N+(v) n N+(a) in the warp's buffer (ascending ids), then the
// (s-2)-subsets of B that are cliques
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_list(ListArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* B = A.buf + warp * A.cap;
  const GView& g = A.g;
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long found = 0, unites = 0;
  const int D = A.s - 2;
  for (int64_t p = warp; p < g.m; p += nwarps) {
    const int32_t v = g.osrc[p], a = g.oadj[p];
    int64_t sb = g.ooff[v], se = g.ooff[v + 1], lb = g.ooff[a], le = g.ooff[a + 1];
    if (se - sb > le - lb) {
      int64_t t0 = sb, t1 = se;
      sb = lb; se = le; lb = t0; le = t1;
    }
    uint32_t nb = 0;
    for (int64_t base = sb; base < se; base += 32) {
      const int64_t j = base + lane;
      int32_t x = 0;
      bool ok = false;
      if (j < se) {
        x = g.oadj[j];
        ok = nh_find(g.oadj, lb, le, x) >= 0;
      }
      const unsigned msk = __ballot_sync(NH_FULL, ok);
      if (ok) B[nb + __popc(msk & ((1u << lane) - 1u))] = x;
      nb += __popc(msk);
    }
    __syncwarp();
    if (D == 0) {
      if (lane == 0) {
        int32_t w[kMaxS] = {v, a};
        clique_action<MODE>(A, w, ls, found, unites);
      }
      __syncwarp();
      continue;
    }
    // lane-parallel first choice, then a depth-first search over later candidates
    for (uint32_t i0 = lane; i0 < nb; i0 += 32) {
      uint32_t idx[kMaxDepth];
      int32_t w[kMaxS];
      w[0] = v; w[1] = a;
      idx[0] = i0;
      int d = 1;
      uint32_t next = i0 + 1;
      if (D == 1) {
        w[2] = B[i0];
        clique_action<MODE>(A, w, ls, found, unites);
        continue;
      }
      while (d > 0) {
        bool pushed = false;
        while (next < nb) {
          const int32_t x = B[next];
          bool ok = true;
          for (int k = 0; k < d && ok; k++) ok = adjacent(A.ch, B[idx[k]], x);
          if (ok) {
            idx[d] = next;
            if (d + 1 == D) {
              for (int k = 0; k < D; k++) w[2 + k] = B[idx[k]];
              clique_action<MODE>(A, w, ls, found, unites);
              ++next;
              continue;
            }
            ++d;
            ++next;
            pushed = true;
            break;
          }
          ++next;
        }
        if (pushed) continue;
        --d;  // exhausted this depth: resume after the index chosen at the level above
        if (d > 0) next = idx[d] + 1;
      }
    }
    __syncwarp();
  }
  if (MODE == kCount) {
    found = nhp::warp_sum_u64(found);
    if (lane == 0 && found) atomicAdd(A.n_s, found);
  }
  if (MODE == kBasic) {
    unites = nhp::warp_sum_u64(unites);
    if (lane == 0 && unites) atomicAdd(A.unites, unites);
  }
  if (MODE == kLinkMin || MODE == kLinkMax) {
    const unsigned long long l = nhp::warp_sum_u64(ls.link), u = nhp::warp_sum_u64(ls.unite);
    if (lane == 0) {
      if (l) atomicAdd(&A.lk.ctl->st_link, l);
      if (u) atomicAdd(&A.lk.ctl->st_unite, u);
    }
  }
}

int list_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (sms > 0 ? sms : 152) * 4;
}

template <int MODE>
int launch_list(ListArgs& A, cudaStream_t st) {
  const int grid = list_grid();
  A.cap = A.g.m > 0 ? A.cap : 1;
  int rc = nh_alloc(&A.buf, (int64_t)grid * kWarps * (A.cap > 0 ? A.cap : 1), st);
  if (rc) return rc;
  k_list<MODE><<<grid, kThreads, 0, st>>>(A);
  nh_note_launch();
  nh_free(A.buf, st);
  A.buf = nullptr;
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

ListArgs list_args(const nh_oriented* o, const nh_rindex* ri, int s) {
  ListArgs A{};
  A.g = make_view(o, ri);
  A.ch = make_chain(o, ri);
  A.sub = make_subsets(s, ri->r);
  A.s = s;
  A.n_r = ri->n_r;
  A.cap = o->max_out > 0 ? o->max_out : 1;
  return A;
}

// ---------------------------------------------------------------------------------------------
// peel (exact and approximate): host-driven rounds
// ---------------------------------------------------------------------------------------------

struct GenCtl {
  unsigned long long n_front, n_alive, min_rest;
  unsigned long long listed, dec, scan, stamp;
};

// frontier A = {x in alive : cnt[x] <= thr}; the rest goes to alive_out, and their least count
__global__ void k_select(const int32_t* __restrict__ alive, unsigned long long n_alive, const uint32_t* __restrict__ cnt,
                         uint32_t thr, int32_t* __restrict__ front, int32_t* __restrict__ alive_out,
                         GenCtl* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  uint32_t mn = 0xffffffffu;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n_alive; base += stride) {
    const unsigned long long i = base + threadIdx.x;
    const bool in = i < n_alive;
    const int32_t x = in ? alive[i] : 0;
    const uint32_t v = in ? cnt[x] : 0xffffffffu;
    const bool f = in && v <= thr;
    const bool rest = in && !f;
    const unsigned long long pf = nhp::warp_append(&c->n_front, f, lane);
    const unsigned long long pa = nhp::warp_append(&c->n_alive, rest, lane);
    if (f) front[pf] = x;
    if (rest) {
      alive_out[pa] = x;
      mn = min(mn, v);
    }
  }
  mn = nhp::warp_min_u32(mn);
  if (lane == 0 && mn != 0xffffffffu) atomicMin(&c->min_rest, (unsigned long long)mn);
}

// stamp the frontier: round t, value (exact: the level; approximate: min(t_i, s-clique-degree))
__global__ void k_commit(const int32_t* __restrict__ front, unsigned long long n, uint32_t t, uint32_t v, int exact,
                         const uint32_t* __restrict__ cnt0, uint32_t* __restrict__ round, uint32_t* __restrict__ val) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int32_t x = front[i];
    round[x] = t;
    val[x] = exact ? v : min(v, cnt0[x]);
  }
}

struct RelistArgs {
  GView g;
  RChain ch;
  Subsets sub;
  int r, s;
  const int32_t* tup;  // r >= 3 vertex tuples (r per r-clique)
  const int32_t* front;
  unsigned long long n_front;
  uint32_t t;
  uint32_t* cnt;
  const uint32_t* round;
  int32_t* buf;
  int64_t cap;
  GenCtl* ctl;
  int* status;
};

// per (R, S): S is dead when a member was peeled in an earlier round; otherwise the frontier member
// of least id decrements every member not peeled yet
__device__ __forceinline__ void relist_action(const RelistArgs& A, int32_t Rid, const int32_t* w0,
                                              unsigned long long& listed, unsigned long long& dec) {
  int32_t w[kMaxS];
  for (int j = 0; j < A.s; j++) w[j] = w0[j];
  sort_small(w, A.s);
  int32_t mem[kMaxC];
  if (!member_ids(A.ch, A.sub, w, mem, A.status)) return;
  ++listed;
  const int C = A.sub.C;
  int32_t attr = Rid;
  for (int j = 0; j < C; j++) {
    const uint32_t rd = __ldcg(A.round + mem[j]);
    if (rd != 0u && rd < A.t) return;  // dead: removed in an earlier round
    if (rd == A.t && mem[j] < attr) attr = mem[j];
  }
  if (attr != Rid) return;
  for (int j = 0; j < C; j++)
    if (__ldcg(A.round + mem[j]) == 0u) {
      atomicSub(A.cnt + mem[j], 1u);
      ++dec;
    }
}

__global__ void __launch_bounds__(kThreads) k_relist(RelistArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* B = A.buf + warp * A.cap;
  const GView& g = A.g;
  unsigned long long listed = 0, dec = 0, scan = 0;
  const int D = A.s - A.r;
  for (unsigned long long i = warp; i < A.n_front; i += nwarps) {
    const int32_t Rid = A.front[i];
    int32_t u[kMaxS];
    if (A.r == 1) u[0] = Rid;
    else if (A.r == 2) { u[0] = g.eu[Rid]; u[1] = g.ev[Rid]; }
    else for (int j = 0; j < A.r; j++) u[j] = A.tup[(int64_t)Rid * A.r + j];
    // candidates: the common neighbours of R's vertices (the vertex of least degree is scanned)
    int best = 0;
    for (int j = 1; j < A.r; j++)
      if (g.off[u[j] + 1] - g.off[u[j]] < g.off[u[best] + 1] - g.off[u[best]]) best = j;
    const int64_t sb = g.off[u[best]], se = g.off[u[best] + 1];
    uint32_t nb = 0;
    for (int64_t base = sb; base < se; base += 32) {
      const int64_t j = base + lane;
      int32_t x = 0;
      bool ok = false;
      if (j < se) {
        x = g.adj[j];
        ok = true;
        for (int k = 0; k < A.r && ok; k++)
          if (k != best) ok = nh_find(g.adj, g.off[u[k]], g.off[u[k] + 1], x) >= 0;
      }
      const unsigned msk = __ballot_sync(NH_FULL, ok);
      if (ok) B[nb + __popc(msk & ((1u << lane) - 1u))] = x;
      nb += __popc(msk);
    }
    scan += (unsigned long long)(se - sb);
    __syncwarp();
    for (uint32_t i0 = lane; i0 < nb; i0 += 32) {
      uint32_t idx[kMaxDepth];
      int32_t w[kMaxS];
      for (int j = 0; j < A.r; j++) w[j] = u[j];
      if (D == 1) {
        w[A.r] = B[i0];
        relist_action(A, Rid, w, listed, dec);
        continue;
      }
      idx[0] = i0;
      int d = 1;
      uint32_t next = i0 + 1;
      while (d > 0) {
        bool pushed = false;
        while (next < nb) {
          const int32_t x = B[next];
          bool ok = true;
          for (int k = 0; k < d && ok; k++) ok = adjacent(A.ch, B[idx[k]], x);
          if (ok) {
            idx[d] = next;
            if (d + 1 == D) {
              for (int k = 0; k < D; k++) w[A.r + k] = B[idx[k]];
              relist_action(A, Rid, w, listed, dec);
              ++next;
              continue;
            }
            ++d;
            ++next;
            pushed = true;
            break;
          }
          ++next;
        }
        if (pushed) continue;
        --d;
        if (d > 0) next = idx[d] + 1;
      }
    }
    __syncwarp();
  }
  listed = nhp::warp_sum_u64(listed);
  dec = nhp::warp_sum_u64(dec);
  if (lane == 0) {
    if (listed) atomicAdd(&A.ctl->listed, listed);
    if (dec) atomicAdd(&A.ctl->dec, dec);
    if (scan) atomicAdd(&A.ctl->scan, scan);
  }
}

__global__ void k_gen_init(int64_t n_r, const uint32_t* __restrict__ cnt0, uint32_t* __restrict__ cnt,
                           uint32_t* __restrict__ round, uint32_t* __restrict__ val, int32_t* __restrict__ alive) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    cnt[i] = cnt0[i];
    round[i] = 0;
    val[i] = 0;
    alive[i] = (int32_t)i;
  }
}

__global__ void k_uf_init(int64_t n, int32_t* __restrict__ uf, int32_t* __restrict__ L) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uf[i] = (int32_t)i;
    L[i] = -1;
  }
}

__global__ void k_max_val(int64_t n, const uint32_t* __restrict__ v, unsigned int* __restrict__ out) {
  uint32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, v[i]);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(NH_FULL, m, d));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// link-efficient over every s-clique (definitional: least-value member; pair rule: largest), then
// the deferred calls of the overflow queue until none is left
int link_all(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* val, int32_t* uf, int32_t* L,
             int pair_rule, nh_peel_stats* stats, cudaStream_t st) {
  const int64_t n_r = ri->n_r;
  ListArgs A = list_args(o, ri, s);
  A.val = val;
  A.lk.uf = uf;
  A.lk.L = L;
  A.lk.core = val;
  A.lk.ovf_cap = (unsigned long long)(n_r > (1 << 20) ? n_r : (1 << 20));
  int* status = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&A.lk.ctl, 1, st)) || (rc = nh_alloc(&A.lk.ovf[0], (int64_t)A.lk.ovf_cap, st)) ||
      (rc = nh_alloc(&A.lk.ovf[1], (int64_t)A.lk.ovf_cap, st)) || (rc = nh_alloc(&status, 1, st))) {
    nh_free(A.lk.ctl, st); nh_free(A.lk.ovf[0], st); nh_free(A.lk.ovf[1], st); nh_free(status, st);
    return rc;
  }
  A.status = status;
  cudaMemsetAsync(A.lk.ctl, 0, sizeof(PeelCtl), st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  rc = pair_rule ? launch_list<kLinkMax>(A, st) : launch_list<kLinkMin>(A, st);
  PeelCtl h{};
  int hs = 0;
  for (int iter = 0; iter < 1000 && !rc; iter++) {
    cudaMemcpyAsync(&h, A.lk.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
    if (h.err) { rc = h.err; break; }
    if (hs) { rc = hs; break; }
    if (h.ovf_count[h.ovf_cur] == 0) break;
    if ((rc = nhp::link_drain_round(A.lk, st))) break;
  }
  if (!rc && stats) {
    stats->link_calls += h.st_link;
    stats->unites += h.st_unite;
  }
  nh_free(A.lk.ctl, st); nh_free(A.lk.ovf[0], st); nh_free(A.lk.ovf[1], st); nh_free(status, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// entry points used by nh_orient.cu, nh_count.cu, nh_peel.cu
// ---------------------------------------------------------------------------------------------

int nh_index_generic(const nh_oriented* o, nh_rindex* prev, int r, nh_rindex* ri, cudaStream_t st) {
  if (!o || !prev || !ri || r < 4 || r > 6 || prev->r != r - 1) return NH_ERR_INVALID;
  const int q = r - 1;
  const int64_t np = prev->n_r;
  int32_t* ptup = prev->tri;  // r - 1 >= 4: the previous level's tuples; r - 1 = 3: the triangles
  uint32_t* ext = nullptr;
  int64_t* eoff = nullptr;
  int* status = nullptr;
  int rc = NH_OK;
  ri->n_r = 0;
  if (np == 0) {  // no (r-1)-cliques: no r-cliques either (a one-slot empty table)
    ri->mask = 0;
    if (nh_alloc(&ri->table, 1, st) || nh_alloc(&ri->tri, 1, st)) return NH_ERR_OOM;
    k_fill_slots<<<1, 32, 0, st>>>(ri->table, 1);
    nh_note_launch();
    return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
  }
  if ((rc = nh_alloc(&ext, np, st)) || (rc = nh_alloc(&eoff, np + 1, st)) || (rc = nh_alloc(&status, 1, st))) {
    nh_free(ext, st); nh_free(eoff, st); nh_free(status, st);
    return rc;
  }
  k_gidx_count<<<warp_blocks(np), kThreads, 0, st>>>(np, q, ptup, o->off, o->adj, ext);
  nh_note_launch();
  rc = nh_exclusive_scan_u32(ext, eoff, np, st);
  int64_t tot = 0;
  if (!rc) {
    cudaMemcpyAsync(&tot, eoff + np, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
  }
  if (!rc && (tot >= (1ll << 31) || np >= (1ll << 32))) rc = NH_ERR_UNSUPPORTED;  // ids are int32 on the path
  unsigned long long cap = 1024;
  while (!rc && cap < 2ull * (unsigned long long)tot) cap <<= 1;
  if (!rc) rc = nh_alloc(&ri->tri, (int64_t)r * (tot > 0 ? tot : 1), st);
  if (!rc) rc = nh_alloc(&ri->table, (int64_t)cap, st);
  if (!rc) {
    ri->mask = cap - 1;
    ri->n_r = tot;
    cudaMemsetAsync(status, 0, sizeof(int), st);
    k_fill_slots<<<nh_blocks_for((int64_t)cap, 256, 152 * 32), 256, 0, st>>>(ri->table, cap);
    k_gidx_fill<<<warp_blocks(np), kThreads, 0, st>>>(np, q, ptup, o->off, o->adj, eoff, ri->tri, ri->table,
                                                       ri->mask, status);
    nh_note_launch(2);
    int hs = 0;
    cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    if (!rc && hs) rc = hs;
  }
  nh_free(ext, st); nh_free(eoff, st); nh_free(status, st);
  return rc;
}

int nh_count_generic(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, unsigned long long* dcount,
                     int* status, cudaStream_t st) {
  ListArgs A = list_args(o, ri, s);
  A.cnt = cnt;
  A.n_s = dcount;
  A.status = status;
  return launch_list<kCount>(A, st);
}

int nh_peel_generic(bool exact, const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* cnt0, uint32_t* val,
                    uint32_t* round, int32_t* uf, int32_t* L, int link_mode, double delta, nh_peel_stats* stats,
                    cudaStream_t st) {
  const int r = ri->r;
  const int64_t n_r = ri->n_r;
  if (stats) *stats = nh_peel_stats{};
  if (n_r == 0) return NH_OK;
  const int C = nh_binom(s, r);
  uint32_t* cnt = nullptr;
  int32_t *alive[2] = {nullptr, nullptr}, *front = nullptr, *buf = nullptr;
  GenCtl* ctl = nullptr;
  int* status = nullptr;
  int rc = NH_OK;
  const int grid = list_grid();
  const int64_t cap = o->max_deg > 0 ? o->max_deg : 1;
  if ((rc = nh_alloc(&cnt, n_r, st)) || (rc = nh_alloc(&alive[0], n_r, st)) || (rc = nh_alloc(&alive[1], n_r, st)) ||
      (rc = nh_alloc(&front, n_r, st)) || (rc = nh_alloc(&ctl, 1, st)) || (rc = nh_alloc(&status, 1, st)) ||
      (rc = nh_alloc(&buf, (int64_t)grid * kWarps * cap, st))) {
    nh_free(cnt, st); nh_free(alive[0], st); nh_free(alive[1], st); nh_free(front, st); nh_free(ctl, st);
    nh_free(status, st); nh_free(buf, st);
    return rc;
  }
  k_gen_init<<<nh_blocks_for(n_r, 256, 152 * 32), 256, 0, st>>>(n_r, cnt0, cnt, round, val, alive[0]);
  nh_note_launch();
  cudaMemsetAsync(status, 0, sizeof(int), st);
  // Alg. 2's bucket ends and round cap per bucket (nh_approx_table / nh_approx_cap, nh_peel.cu)
  std::vector<uint32_t> thr;
  uint32_t T = 0;
  if (!exact) {
    unsigned int* dmax = nullptr;
    if ((rc = nh_alloc(&dmax, 1, st))) goto done;
    cudaMemsetAsync(dmax, 0, sizeof(unsigned int), st);
    k_max_val<<<nh_blocks_for(n_r, 256, 152 * 8), 256, 0, st>>>(n_r, cnt0, dmax);
    nh_note_launch();
    unsigned int hmax = 0;
    cudaMemcpyAsync(&hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st);
    nh_free(dmax, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; goto done; }
    thr.resize(1 << 16);
    thr.resize((size_t)nh_approx_table(C, delta, hmax, thr.data(), 1 << 16));
    T = nh_approx_cap(C, delta, n_r);
  }
  {
    RelistArgs R{};
    R.g = make_view(o, ri);
    R.ch = make_chain(o, ri);
    R.sub = make_subsets(s, r);
    R.r = r;
    R.s = s;
    R.tup = ri->tri;
    R.front = front;
    R.cnt = cnt;
    R.round = round;
    R.buf = buf;
    R.cap = cap;
    R.ctl = ctl;
    R.status = status;
    unsigned long long n_alive = (unsigned long long)n_r;
    int cur = 0;
    uint32_t k = 0, t = 0, kmax = 0;
    size_t bucket = 0;
    uint32_t in_bucket = 0;
    unsigned long long levels = 0, ftot = 0;
    GenCtl h{};
    for (unsigned long long guard = 0; n_alive > 0; ++guard) {
      if (guard > 4ull * (unsigned long long)n_r + 1000000ull) { rc = NH_ERR_TIMEOUT; break; }
      const uint32_t th = exact ? k : thr[bucket < thr.size() ? bucket : thr.size() - 1];
      cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned long long), st);
      cudaMemsetAsync(&ctl->min_rest, 0xff, sizeof(unsigned long long), st);
      k_select<<<nh_blocks_for((int64_t)n_alive, 256, 152 * 16), 256, 0, st>>>(alive[cur], n_alive, cnt, th, front,
                                                                               alive[cur ^ 1], ctl);
      nh_note_launch();
      cudaMemcpyAsync(&h, ctl, sizeof(GenCtl), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
      cur ^= 1;
      n_alive = h.n_alive;
      if (h.n_front == 0) {
        if (exact) {
          k = (uint32_t)h.min_rest;  // > k: every alive count is above the old level
          ++levels;
        } else {
          ++bucket;
          in_bucket = 0;
          if (bucket >= thr.size()) { rc = NH_ERR_INTERNAL; break; }  // the last end covers every count
        }
        continue;
      }
      ++t;
      ftot += h.n_front;
      if (exact) kmax = k;
      k_commit<<<nh_blocks_for((int64_t)h.n_front, 256, 152 * 16), 256, 0, st>>>(front, h.n_front, t, th,
                                                                                exact ? 1 : 0, cnt0, round, val);
      nh_note_launch();
      R.n_front = h.n_front;
      R.t = t;
      k_relist<<<grid, kThreads, 0, st>>>(R);
      nh_note_launch();
      if (!exact && ++in_bucket >= T) {
        ++bucket;
        in_bucket = 0;
      }
    }
    int hs = 0;
    cudaMemcpyAsync(&h, ctl, sizeof(GenCtl), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
    if (!rc && hs) rc = hs;
    if (stats) {  // the select clears only its own words: the re-listing counters span all rounds
      stats->rounds = t;
      stats->levels = levels;
      stats->kmax = kmax;
      stats->frontier_total = ftot;
      stats->s_cliques_listed = h.listed;
      stats->decrements = h.dec;
      stats->scan_elements = h.scan;
    }
  }
  if (!rc && exact && link_mode < 2) {
    k_uf_init<<<nh_blocks_for(n_r, 256, 152 * 32), 256, 0, st>>>(n_r, uf, L);
    nh_note_launch();
    rc = link_all(o, ri, s, val, uf, L, link_mode == 1, stats, st);
  }
done:
  nh_free(cnt, st); nh_free(alive[0], st); nh_free(alive[1], st); nh_free(front, st); nh_free(ctl, st);
  nh_free(status, st); nh_free(buf, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

int nh_label_hierarchy_generic(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* labels,
                               int32_t* parent, uint32_t* label, int64_t* n_nodes, cudaStream_t st) {
  const int64_t n_r = ri->n_r;
  int32_t *uf = nullptr, *L = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&uf, n_r, st)) || (rc = nh_alloc(&L, n_r, st))) {
    nh_free(uf, st); nh_free(L, st);
    return rc;
  }
  k_uf_init<<<nh_blocks_for(n_r, 256, 152 * 32), 256, 0, st>>>(n_r, uf, L);
  nh_note_launch();
  rc = link_all(o, ri, s, labels, uf, L, 0, nullptr, st);
  if (!rc) rc = nh_construct_tree(n_r, labels, uf, L, parent, label, n_nodes, st);
  nh_free(uf, st); nh_free(L, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

// ---------------------------------------------------------------------------------------------
// link-basic (Alg. 4) and construct-tree-basic
// ---------------------------------------------------------------------------------------------

namespace {

__global__ void k_bl_init(int64_t n_r, int64_t total, int32_t* __restrict__ ufb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    ufb[i] = (int32_t)(i % n_r);
}

// level i: every r-clique's root (stored back: full compression) and the size of every component
__global__ void k_bl_roots(int64_t n_r, int32_t* __restrict__ uf, uint32_t* __restrict__ size) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_r; x += (int64_t)gridDim.x * blockDim.x) {
    int32_t y = (int32_t)x;
    for (int64_t it = 0; it < n_r; ++it) {
      const int32_t p = __ldcg(uf + y);
      if (p == y) break;
      y = p;
    }
    atomicAdd(size + y, 1u);
    __stcg(uf + x, y);
  }
}

// a component of at least two r-cliques gets a node at level i unless it is, as a set, the
// component of its root one level up (same size as the node that holds its root)
__global__ void k_bl_nodes(int64_t n_r, const int32_t* __restrict__ uf, const uint32_t* __restrict__ size,
                           const int32_t* __restrict__ top, uint32_t* __restrict__ tsize, uint32_t level,
                           int32_t* __restrict__ newnode, uint32_t* __restrict__ label,
                           unsigned long long* __restrict__ n_nodes) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_r; x += (int64_t)gridDim.x * blockDim.x) {
    if (uf[x] != (int32_t)x) continue;
    const uint32_t sz = size[x];
    const int32_t T = top[x];
    int32_t N = -1;
    if (sz >= 2 && !(T >= 0 && tsize[T] == sz)) {
      N = (int32_t)atomicAdd(n_nodes, 1ull);
      label[N] = level;
      tsize[N] = sz;
    }
    newnode[x] = N;
  }
}

// every member of a new node hangs its current top node (or itself) from it
__global__ void k_bl_attach(int64_t n_r, const int32_t* __restrict__ uf, const int32_t* __restrict__ newnode,
                            int32_t* __restrict__ top, int32_t* __restrict__ parent) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_r; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t N = newnode[uf[x]];
    if (N < 0) continue;
    const int32_t T = top[x];
    if (T < 0) parent[x] = N;
    else parent[n_r + T] = N;
    top[x] = N;
  }
}

__global__ void k_fill_i32(int64_t n, int32_t* __restrict__ a, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

}  // namespace

extern "C" int nh_hierarchy_basic(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* core,
                                  int32_t* parent, uint32_t* label, int64_t* n_nodes, uint64_t* unites, void* stream) {
  if (!o || !ri || ri->o != o || !n_nodes) return NH_ERR_INVALID;
  const int r = ri->r;
  if (!(nh_supported(r, s) || nh_generic_pair(r, s))) return NH_ERR_UNSUPPORTED;
  const int64_t n_r = ri->n_r;
  if (n_r > 0 && (!core || !parent || !label)) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  *n_nodes = 0;
  if (unites) *unites = 0;
  if (n_r == 0) return NH_OK;
  int rc = NH_OK;
  unsigned int* dmax = nullptr;
  if ((rc = nh_alloc(&dmax, 1, st))) return rc;
  cudaMemsetAsync(dmax, 0, sizeof(unsigned int), st);
  k_max_val<<<nh_blocks_for(n_r, 256, 152 * 8), 256, 0, st>>>(n_r, core, dmax);
  nh_note_launch();
  unsigned int kmax = 0;
  cudaMemcpyAsync(&kmax, dmax, sizeof(kmax), cudaMemcpyDeviceToHost, st);
  nh_free(dmax, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return NH_ERR_CUDA;
  k_fill_i32<<<nh_blocks_for(2 * n_r, 256, 152 * 32), 256, 0, st>>>(2 * n_r, parent, -1);
  nh_note_launch();
  if (kmax == 0) return cudaStreamSynchronize(st) == cudaSuccess ? NH_OK : NH_ERR_CUDA;
  // one union-find per level: kmax * n_r entries (the space cost Alg. 4 is known for)
  const int64_t total = (int64_t)kmax * n_r;
  size_t free_b = 0, tot_b = 0;
  if (cudaMemGetInfo(&free_b, &tot_b) != cudaSuccess) return NH_ERR_CUDA;
  if ((double)total * 4.0 > 0.8 * (double)free_b) return NH_ERR_OOM;
  int32_t *ufb = nullptr, *top = nullptr, *newnode = nullptr;
  uint32_t *size = nullptr, *tsize = nullptr;
  unsigned long long *counters = nullptr;  // {unites, nodes}
  int* status = nullptr;
  PeelCtl* ctl = nullptr;
  if ((rc = nh_alloc(&ufb, total, st)) || (rc = nh_alloc(&top, n_r, st)) || (rc = nh_alloc(&newnode, n_r, st)) ||
      (rc = nh_alloc(&size, n_r, st)) || (rc = nh_alloc(&tsize, n_r, st)) || (rc = nh_alloc(&counters, 2, st)) ||
      (rc = nh_alloc(&status, 1, st)) || (rc = nh_alloc(&ctl, 1, st)))
    goto done;
  k_bl_init<<<nh_blocks_for(total, 256, 152 * 64), 256, 0, st>>>(n_r, total, ufb);
  k_fill_i32<<<nh_blocks_for(n_r, 256, 152 * 32), 256, 0, st>>>(n_r, top, -1);
  nh_note_launch(2);
  cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), st);
  {
    // link-basic for the definitional calls of every s-clique: its least-core member with each other
    // member, in every level up to c_S
    ListArgs A = list_args(o, ri, s);
    A.val = core;
    A.ufb = ufb;
    A.unites = counters;
    A.status = status;
    A.lk.ctl = ctl;
    if ((rc = launch_list<kBasic>(A, st))) goto done;
  }
  for (uint32_t i = kmax; i >= 1 && !rc; i--) {
    int32_t* uf = ufb + (int64_t)(i - 1) * n_r;
    const unsigned b = nh_blocks_for(n_r, 256, 152 * 32);
    cudaMemsetAsync(size, 0, sizeof(uint32_t) * n_r, st);
    k_bl_roots<<<b, 256, 0, st>>>(n_r, uf, size);
    k_bl_nodes<<<b, 256, 0, st>>>(n_r, uf, size, top, tsize, i, newnode, label, counters + 1);
    k_bl_attach<<<b, 256, 0, st>>>(n_r, uf, newnode, top, parent);
    nh_note_launch(3);
    if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
  }
  if (!rc) {
    unsigned long long hc[2] = {0, 0};
    int hs = 0, herr = 0;
    cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&herr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    if (!rc && hs) rc = hs;
    if (!rc && herr) rc = herr;
    if (!rc) {
      *n_nodes = (int64_t)hc[1];
      if (unites) *unites = hc[0];
    }
  }
done:
  nh_free(ufb, st); nh_free(top, st); nh_free(newnode, st); nh_free(size, st); nh_free(tsize, st);
  nh_free(counters, st); nh_free(status, st); nh_free(ctl, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}
