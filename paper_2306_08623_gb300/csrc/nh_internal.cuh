// nh_internal.cuh -- shared internals of libnucleus (device helpers, handle layouts).
//
// Data layout in HBM (all int32 unless noted):
//   CSR             off[n+1] (int64), adj[2m]                         caller-owned
//   eid[2m]         canonical (lexicographic) edge id of every adjacency entry
//   ooff[n+1] (i64), oadj[m], oeid[m], osrc[m]   out-CSR of the degree orientation, the edge id and
//                   the source vertex of every out-entry
//   uoff[n+1] (i64) first lexicographic edge id of each vertex (edges (u,v), u<v)
//   eu[m], ev[m]    endpoints of edge id e (eu < ev)
//   tri[3 n_r]      vertices of triangle id t (r = 3), toff[m+1] (i64) first triangle id per edge
//   tedge[3 n_r]    ids of the edges {a,b}, {a,c}, {b,c} of triangle t = {a < b < c}
//   table[cap]      16-byte slots {key u64, id u32, pad}: key = (edge id of (a,b)) << 32 | c
//   ekey[cap] (u64), eval[cap]   open-addressing edge table (load <= 0.5): key (u << 32 | v), u < v,
//                   and the edge id in the parallel value array (a miss reads the 8-byte keys only,
//                   so the key array of a few-million-edge graph stays resident in L2)
//   etoff[m+1] (i64), etw[3 n_r], ettid[3 n_r]   r = 3: for every edge (p,q), the third vertices w
//                   of all triangles {p,q,w} in ascending order, with the triangle ids
//   t2off[m+1] (i64), t2w, t2ea, t2eb [3 T]   r = 2 (T = number of triangles): for every edge
//                   (a,b), a < b, the third vertices w of its triangles in ascending order with the
//                   ids of the edges {a,w} and {b,w} -- the s-cliques of (2,3) and the candidate sets
//                   of (2,4) without any adjacency probe; t2cost[m] (u32, saturating): per edge the
//                   sum over its list of the out-degrees d+(w), the (2,4) re-listing's work bound
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nucleus.h"

#define NH_FULL 0xffffffffu
#define NH_EMPTY_KEY 0xffffffffffffffffull

struct nh_slot {
  unsigned long long key;
  uint32_t val;
  uint32_t pad;
};

struct nh_oriented {
  int64_t n, m;
  const int64_t* off;
  const int32_t* adj;
  int32_t* eid;
  int64_t* ooff;
  int32_t* oadj;
  int32_t* oeid;
  int32_t* osrc;
  int64_t* uoff;
  int32_t* eu;
  int32_t* ev;
  int64_t max_out, max_deg;
  unsigned long long* ekey;
  uint32_t* eval;
  unsigned long long emask;
  cudaStream_t stream;  // stream the handle was built on (frees are ordered on it)
};

struct nh_rindex {
  int r;
  int64_t n_r;
  const nh_oriented* o;
  int32_t* tri;
  int32_t* tedge;
  int64_t* toff;
  nh_slot* table;
  unsigned long long mask;
  int64_t* etoff;
  int32_t* etw;
  int32_t* ettid;
  int64_t* t2off;
  int32_t* t2w;
  int32_t* t2ea;
  int32_t* t2eb;
  uint32_t* t2cost;
  nh_rindex* prev;  // r >= 4: the index of the (r-1)-cliques this one extends (owned)
  cudaStream_t stream;
};

// Read-only view of the graph, passed to kernels by value.
struct GView {
  const int64_t* off;
  const int32_t* adj;
  const int32_t* eid;
  const int64_t* ooff;
  const int32_t* oadj;
  const int32_t* oeid;
  const int32_t* osrc;
  const int32_t* eu;
  const int32_t* ev;
  const unsigned long long* ekey;
  const uint32_t* eval;
  unsigned long long emask;
  const int32_t* tri;
  const int32_t* tedge;
  const nh_slot* table;
  unsigned long long mask;
  const int64_t* etoff;
  const int32_t* etw;
  const int32_t* ettid;
  const int64_t* t2off;
  const int32_t* t2w;
  const int32_t* t2ea;
  const int32_t* t2eb;
  const uint32_t* t2cost;
  int64_t n, m;
};

static inline GView make_view(const nh_oriented* o, const nh_rindex* ri) {
  GView g;
  g.off = o->off; g.adj = o->adj; g.eid = o->eid;
  g.ooff = o->ooff; g.oadj = o->oadj; g.oeid = o->oeid; g.osrc = o->osrc;
  g.eu = o->eu; g.ev = o->ev;
  g.ekey = o->ekey; g.eval = o->eval; g.emask = o->emask;
  g.tri = ri ? ri->tri : nullptr;
  g.tedge = ri ? ri->tedge : nullptr;
  g.table = ri ? ri->table : nullptr;
  g.mask = ri ? ri->mask : 0ull;
  g.etoff = ri ? ri->etoff : nullptr;
  g.etw = ri ? ri->etw : nullptr;
  g.ettid = ri ? ri->ettid : nullptr;
  g.t2off = ri ? ri->t2off : nullptr;
  g.t2w = ri ? ri->t2w : nullptr;
  g.t2ea = ri ? ri->t2ea : nullptr;
  g.t2eb = ri ? ri->t2eb : nullptr;
  g.t2cost = ri ? ri->t2cost : nullptr;
  g.n = o->n; g.m = o->m;
  return g;
}

// ---------------------------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------------------------

// first index p in [lo, hi) with a[p] >= x (a sorted ascending)
__device__ __forceinline__ int64_t nh_lower_bound(const int32_t* __restrict__ a, int64_t lo, int64_t hi,
                                                  int32_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// position of x in a[lo, hi) or -1
__device__ __forceinline__ int64_t nh_find(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t x) {
  int64_t p = nh_lower_bound(a, lo, hi, x);
  return (p < hi && __ldg(a + p) == x) ? p : -1;
}

// SplitMix64 finalizer (Steele, Lea, Flood 2014) as the hash of a 64-bit key.
__device__ __forceinline__ unsigned long long nh_mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// Key of triangle {x, y, z} given the edge ids of its three pairs: the edge id of the two
// smaller vertices, shifted up, and the largest vertex.
__device__ __forceinline__ unsigned long long nh_tri_key(int32_t x, int32_t y, int32_t z, int32_t exy,
                                                         int32_t exz, int32_t eyz) {
  if (x > y && x > z) return ((unsigned long long)(uint32_t)eyz << 32) | (uint32_t)x;
  if (y > z) return ((unsigned long long)(uint32_t)exz << 32) | (uint32_t)y;
  return ((unsigned long long)(uint32_t)exy << 32) | (uint32_t)z;
}

// Triangle id for a key, or -1 when absent.  Linear probing with a probe cap of the table size.
__device__ __forceinline__ int64_t nh_tri_lookup(const nh_slot* __restrict__ t, unsigned long long mask,
                                                 unsigned long long key) {
  unsigned long long h = nh_mix64(key) & mask;
  for (unsigned long long p = 0; p <= mask; ++p) {
    ulonglong2 s = __ldg(reinterpret_cast<const ulonglong2*>(t + h));
    if (s.x == key) return (int64_t)(uint32_t)s.y;
    if (s.x == NH_EMPTY_KEY) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// id of edge {x, y} or -1 when x and y are not adjacent
__device__ __forceinline__ int64_t nh_edge_id(const GView& g, int32_t x, int32_t y) {
  const unsigned long long key = (x < y) ? (((unsigned long long)(uint32_t)x << 32) | (uint32_t)y)
                                         : (((unsigned long long)(uint32_t)y << 32) | (uint32_t)x);
  unsigned long long h = nh_mix64(key) & g.emask;
  for (unsigned long long p = 0; p <= g.emask; ++p) {
    const unsigned long long k = __ldg(g.ekey + h);
    if (k == key) return (int64_t)__ldg(g.eval + h);
    if (k == NH_EMPTY_KEY) return -1;
    h = (h + 1) & g.emask;
  }
  return -1;
}

__device__ __forceinline__ unsigned long long nh_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int32_t nh_ld_volatile(const int32_t* p) { return *(const volatile int32_t*)p; }
__device__ __forceinline__ uint32_t nh_ld_volatile(const uint32_t* p) { return *(const volatile uint32_t*)p; }

// host-side launch helpers
#define NH_CUDA_TRY(x)                      \
  do {                                      \
    cudaError_t _e = (x);                   \
    if (_e != cudaSuccess) {                \
      (void)cudaGetLastError();             \
      return (_e == cudaErrorMemoryAllocation) ? NH_ERR_OOM : NH_ERR_CUDA; \
    }                                       \
  } while (0)

static inline unsigned nh_blocks_for(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// count one kernel launch made by the library (reported by nh_kernel_launches)
void nh_note_launch(int64_t k = 1);

// counting driver shared by the plain and the partitioned entry points (nh_count.cu); vertex_cost
// (optional) selects the cost-balanced partition, measure (optional) receives per-vertex cost
int nh_count_impl(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, uint64_t* n_s,
                  const float* vertex_cost, float* measure, cudaStream_t st);
// out-edge items in decreasing estimated cost (log2 buckets) and a zeroed shared work counter for
// dynamic scheduling (nh_mlp.cu); the caller frees both
int nh_schedule_items(const nh_oriented* o, const float* vertex_cost, int32_t** order, unsigned long long** next,
                      cudaStream_t st);

// tile of the device-wide scan (threads per block x items per thread); a scan of n entries uses
// ceil(n / kNhScanTile) block sums
constexpr int kNhScanThreads = 256;
constexpr int kNhScanItems = 8;
constexpr int kNhScanTile = kNhScanThreads * kNhScanItems;
// exclusive prefix sum of 32-bit (or 64-bit) counts into int64 offsets, out[n] = total
int nh_exclusive_scan_u32(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t st);
int nh_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
// block sums a scan of n entries needs, and the scan with caller-provided block-sum storage
int nh_scan_u32_blocks(int64_t n);
int nh_exclusive_scan_u32_into(const uint32_t* in, int64_t* out, int64_t n, int64_t* bsum, cudaStream_t st);

// stream-ordered pieces of the path (no host synchronisation; results stay in device words)
int nh_count_enqueue(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, const float* vertex_cost,
                     float* measure, unsigned long long* dcount, int* status, cudaStream_t st);
// status_dev (int64, may be null): set to NH_ERR_INVALID when a union-find walk finds a cycle
int nh_tree_enqueue(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L, int32_t* parent,
                    uint32_t* label, int64_t* n_nodes_dev, int64_t* status_dev, cudaStream_t st);

// allocation helpers (stream ordered)
template <typename T>
static inline int nh_alloc(T** p, int64_t count, cudaStream_t st) {
  *p = nullptr;
  size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  cudaError_t e = cudaMallocAsync((void**)p, bytes, st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return NH_ERR_OOM;
  }
  return NH_OK;
}
template <typename T>
static inline void nh_free(T* p, cudaStream_t st) {
  if (p) (void)cudaFreeAsync((void*)p, st);
}

static inline int nh_binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  int b = 1;
  for (int i = 1; i <= k; i++) b = b * (n - k + i) / i;
  return b;
}

static inline bool nh_supported(int r, int s) {
  return (r == 1 && (s == 2 || s == 3)) || (r == 2 && (s == 3 || s == 4)) || (r == 3 && s == 4);
}
// Alg. 2's bucket ends (at most cap, returns how many) and round cap (nh_peel.cu; host only)
int nh_approx_table(int C, double delta, uint32_t max_count, uint32_t* out, int cap);
uint32_t nh_approx_cap(int C, double delta, int64_t n_r);
// pairs served by the generic path (nh_generic.cu): every other 1 <= r < s <= 7
static inline bool nh_generic_pair(int r, int s) { return r >= 1 && s > r && s <= 7 && !nh_supported(r, s); }
// generic path entry points (nh_generic.cu)
int nh_index_generic(const nh_oriented* o, nh_rindex* prev, int r, nh_rindex* out, cudaStream_t st);
int nh_count_generic(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, unsigned long long* dcount,
                     int* status, cudaStream_t st);
int nh_peel_generic(bool exact, const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* cnt, uint32_t* val,
                    uint32_t* round, int32_t* uf, int32_t* L, int link_mode, double delta, nh_peel_stats* stats,
                    cudaStream_t st);
int nh_label_hierarchy_generic(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* labels,
                               int32_t* parent, uint32_t* label, int64_t* n_nodes, cudaStream_t st);
