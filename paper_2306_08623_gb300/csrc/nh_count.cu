// nh_count.cu -- a3: rec-list-cliques.  Every s-clique is listed once, from its lowest-ranked
// vertex v and its out-neighbour a (one warp per out-edge (v -> a)), by intersecting sorted
// out-lists; the s-clique-degree of each of its binom(s,r) r-subsets is incremented.
#include "nh_internal.cuh"

extern long long g_nh_inject_count_base;  // fault injection (nh_api.cu): initial count value

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(NH_FULL, v, d);
  return v;
}

// cnt[x] += inc (a reduction: the old value is not needed).  A count that passes 2^32 - 1 wraps
// and loses exactly 2^32, which the check after the count (k_count_check) sees in the sum of all
// counts; status is unused here.
__device__ __forceinline__ void cnt_add(uint32_t* cnt, int64_t x, uint32_t inc, int* status) {
  (void)status;
  atomicAdd(&cnt[x], inc);
}

__device__ __forceinline__ void tri_add(const GView& g, unsigned long long key, uint32_t inc, uint32_t* cnt,
                                        int* status) {
  int64_t id = nh_tri_lookup(g.table, g.mask, key);
  if (id < 0) { atomicExch(status, NH_ERR_INTERNAL); return; }
  cnt_add(cnt, id, inc, status);
}

// Three independent triangle-id look-ups advanced in lockstep (linear probing, each capped at the
// table size): every probe round issues up to three independent loads, so the chain of dependent
// loads is that of one look-up, not three.  A key that is absent sets NH_ERR_INTERNAL.
__device__ __forceinline__ void tri_add3(const GView& g, unsigned long long k0, unsigned long long k1,
                                         unsigned long long k2, uint32_t* cnt, int* status) {
  const unsigned long long m = g.mask;
  unsigned long long h0 = nh_mix64(k0) & m, h1 = nh_mix64(k1) & m, h2 = nh_mix64(k2) & m;
  int64_t i0 = -1, i1 = -1, i2 = -1;
  bool d0 = false, d1 = false, d2 = false;
  for (unsigned long long q = 0; q <= m && !(d0 && d1 && d2); ++q) {
    const ulonglong2 s0 = d0 ? make_ulonglong2(0ull, 0ull) : __ldg(reinterpret_cast<const ulonglong2*>(g.table + h0));
    const ulonglong2 s1 = d1 ? make_ulonglong2(0ull, 0ull) : __ldg(reinterpret_cast<const ulonglong2*>(g.table + h1));
    const ulonglong2 s2 = d2 ? make_ulonglong2(0ull, 0ull) : __ldg(reinterpret_cast<const ulonglong2*>(g.table + h2));
    if (!d0) {
      if (s0.x == k0) { i0 = (int64_t)(uint32_t)s0.y; d0 = true; }
      else if (s0.x == NH_EMPTY_KEY) d0 = true;
      else h0 = (h0 + 1) & m;
    }
    if (!d1) {
      if (s1.x == k1) { i1 = (int64_t)(uint32_t)s1.y; d1 = true; }
      else if (s1.x == NH_EMPTY_KEY) d1 = true;
      else h1 = (h1 + 1) & m;
    }
    if (!d2) {
      if (s2.x == k2) { i2 = (int64_t)(uint32_t)s2.y; d2 = true; }
      else if (s2.x == NH_EMPTY_KEY) d2 = true;
      else h2 = (h2 + 1) & m;
    }
  }
  if (i0 < 0 || i1 < 0 || i2 < 0) { atomicExch(status, NH_ERR_INTERNAL); return; }
  cnt_add(cnt, i0, 1u, status);
  cnt_add(cnt, i1, 1u, status);
  cnt_add(cnt, i2, 1u, status);
}

// (1,2): the s-clique-degree of a vertex is its degree
__global__ void k_count_12(int64_t n, const int64_t* __restrict__ off, uint32_t* __restrict__ cnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    cnt[v] = (uint32_t)(off[v + 1] - off[v]);
}

// s = 3: triangles (v, a, b) with a, b in N+(v), b in N+(a)
// Work items are out-edges (v -> a).  With order == null the warps stride over all items;
// otherwise the warps take chunks of kChunk items of `order` (items sorted by decreasing
// estimated cost) from the shared counter *next: the heaviest items start first and every warp
// keeps taking work until none is left (largest-first dynamic scheduling).  When cost != null
// the work of each item (list entries touched, binary-search steps included) is added to
// cost[v]: the measured listing cost the work estimator learns.
__device__ __forceinline__ float log2p1(int64_t x) { return log2f((float)x + 1.0f); }

constexpr unsigned long long kChunk = 8;

// next work item of this warp, or -1 when there is none left (warp-uniform).  Dynamic chunks grow
// with the position in the order: the items come heaviest first, so the first grabs take kChunk
// items and later ones about (position / (16 * warps)) of the lighter items, which keeps the
// shared counter to a few dozen grabs per warp.
struct ItemCursor {
  const int32_t* order;
  unsigned long long* next;
  int64_t m, nwarps, p;        // plain stride
  unsigned long long cur, end; // dynamic chunk
  __device__ __forceinline__ int64_t get(int lane) {
    if (!order) {
      const int64_t q = p;
      p += nwarps;
      return q < m ? q : -1;
    }
    if (cur >= end) {
      unsigned long long want = end / (16ull * (unsigned long long)nwarps);
      if (want < kChunk) want = kChunk;
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(next, want);
      b = __shfl_sync(NH_FULL, b, 0);
      if (b >= (unsigned long long)m) return -1;
      cur = b;
      end = min(b + want, (unsigned long long)m);
    }
    return order[cur++];
  }
};

template <int R>
__global__ void k_count_s3(GView g, uint32_t* __restrict__ cnt, unsigned long long* __restrict__ n_s,
                           const int32_t* __restrict__ order, unsigned long long* __restrict__ next,
                           float* __restrict__ cost, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long found = 0;
  ItemCursor it{order, next, g.m, nwarps, warp, 0, 0};
  for (int64_t p = it.get(lane); p >= 0; p = it.get(lane)) {
    const int32_t v = g.osrc[p], a = g.oadj[p], e_va = g.oeid[p];
    int64_t sb = g.ooff[v], se = g.ooff[v + 1];  // scanned list
    int64_t lb = g.ooff[a], le = g.ooff[a + 1];  // searched list
    const bool scan_v = (se - sb) <= (le - lb);
    if (!scan_v) {
      int64_t t0 = sb, t1 = se;
      sb = lb; se = le; lb = t0; le = t1;
    }
    uint32_t tot = 0;
    for (int64_t j = sb + lane; j < se; j += 32) {
      const int32_t b = g.oadj[j];
      const int64_t q = nh_find(g.oadj, lb, le, b);
      if (q < 0) continue;
      tot++;
      const int32_t e_vb = g.oeid[scan_v ? j : q], e_ab = g.oeid[scan_v ? q : j];
      if (R == 1) cnt_add(cnt, b, 1u, status);
      if (R == 2) { cnt_add(cnt, e_vb, 1u, status); cnt_add(cnt, e_ab, 1u, status); }
    }
    tot = warp_sum(tot);
    if (lane == 0 && tot) {
      if (R == 1) { cnt_add(cnt, v, tot, status); cnt_add(cnt, a, tot, status); }
      if (R == 2) cnt_add(cnt, e_va, tot, status);
      found += tot;
    }
    if (cost && lane == 0) atomicAdd(&cost[v], (float)(se - sb) * (1.0f + log2p1(le - lb)) + 1.0f);
  }
  if (lane == 0 && found) atomicAdd(n_s, found);
}

// s = 4: 4-cliques (v, a, b, c): C2 = N+(v) n N+(a) is staged per warp (in shared memory when it
// fits, else in a global per-warp slice); c runs over N+(b) and is searched in C2.
template <int R>
__global__ void k_count_s4(GView g, uint32_t* __restrict__ cnt, unsigned long long* __restrict__ n_s,
                           int32_t* __restrict__ gscratch, int cap, int use_smem, int* __restrict__ status,
                           const int32_t* __restrict__ order, unsigned long long* __restrict__ next,
                           float* __restrict__ cost) {
  extern __shared__ int32_t smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* base = use_smem ? smem + (size_t)wib * 3 * cap : gscratch + (size_t)warp * 3 * cap;
  int32_t* c2v = base;
  int32_t* c2e1 = base + cap;  // edge (v, b)
  int32_t* c2e2 = base + 2 * cap;  // edge (a, b)
  unsigned long long found = 0;
  ItemCursor it{order, next, g.m, nwarps, warp, 0, 0};
  for (int64_t p = it.get(lane); p >= 0; p = it.get(lane)) {
    const int32_t v = g.osrc[p], a = g.oadj[p], e_va = g.oeid[p];
    int64_t sb = g.ooff[v], se = g.ooff[v + 1];
    int64_t lb = g.ooff[a], le = g.ooff[a + 1];
    const bool scan_v = (se - sb) <= (le - lb);
    if (!scan_v) {
      int64_t t0 = sb, t1 = se;
      sb = lb; se = le; lb = t0; le = t1;
    }
    float work = (float)(se - sb) * (1.0f + log2p1(le - lb)) + 1.0f;
    int n2 = 0;
    for (int64_t base_j = sb; base_j < se; base_j += 32) {
      const int64_t j = base_j + lane;
      int64_t q = -1;
      int32_t b = 0;
      if (j < se) {
        b = g.oadj[j];
        q = nh_find(g.oadj, lb, le, b);
      }
      const unsigned msk = __ballot_sync(NH_FULL, q >= 0);
      if (q >= 0) {
        const int k = n2 + __popc(msk & ((1u << lane) - 1u));
        c2v[k] = b;
        c2e1[k] = g.oeid[scan_v ? j : q];
        c2e2[k] = g.oeid[scan_v ? q : j];
      }
      n2 += __popc(msk);
    }
    __syncwarp();
    uint32_t tot_item = 0;
    for (int i = 0; i < n2; i++) {
      const int32_t b = c2v[i], e_vb = c2e1[i], e_ab = c2e2[i];
      const int64_t bb = g.ooff[b], be = g.ooff[b + 1];
      work += (float)(be - bb) * (1.0f + log2p1(n2));
      uint32_t n3 = 0;
      for (int64_t j = bb + lane; j < be; j += 32) {
        const int32_t c = g.oadj[j];
        // c is an out-neighbour of v and a exactly when it is in C2 (sorted by id)
        int lo = 0, hi = n2;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (c2v[mid] < c) lo = mid + 1; else hi = mid;
        }
        const int k = (lo < n2 && c2v[lo] == c) ? lo : -1;
        if (k < 0) continue;
        n3++;
        const int32_t e_vc = c2e1[k], e_ac = c2e2[k], e_bc = g.oeid[j];
        if (R == 1) cnt_add(cnt, c, 1u, status);
        if (R == 2) { cnt_add(cnt, e_vc, 1u, status); cnt_add(cnt, e_ac, 1u, status); cnt_add(cnt, e_bc, 1u, status); }
        if (R == 3)
          tri_add3(g, nh_tri_key(v, a, c, e_va, e_vc, e_ac), nh_tri_key(v, b, c, e_vb, e_vc, e_bc),
                   nh_tri_key(a, b, c, e_ab, e_ac, e_bc), cnt, status);
      }
      n3 = warp_sum(n3);
      if (lane == 0 && n3) {
        if (R == 1) cnt_add(cnt, b, n3, status);
        if (R == 2) { cnt_add(cnt, e_vb, n3, status); cnt_add(cnt, e_ab, n3, status); }
        if (R == 3) tri_add(g, nh_tri_key(v, a, b, e_va, e_vb, e_ab), n3, cnt, status);
      }
      tot_item += n3;
    }
    if (lane == 0 && tot_item) {
      if (R == 1) { cnt_add(cnt, v, tot_item, status); cnt_add(cnt, a, tot_item, status); }
      if (R == 2) cnt_add(cnt, e_va, tot_item, status);
      found += tot_item;
    }
    if (cost && lane == 0) atomicAdd(&cost[v], work);
    __syncwarp();
  }
  if (lane == 0 && found) atomicAdd(n_s, found);
}

int grid_for(const void* fn, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (per < 1) per = 1;
  return sms * per;
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// Overflow check after counting: every s-clique adds 1 to each of its C r-subsets, so the counts
// sum to base * n_r + C * n_s (base: their initial value).  A count that wrapped lost a multiple
// of 2^32, which the 64-bit sum of the stored counts shows.  sums[0] accumulates the sum.
__global__ void k_count_sum(int64_t n, const uint32_t* __restrict__ cnt, unsigned long long* __restrict__ sums) {
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += cnt[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(NH_FULL, s, d);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(sums, s);
}

__global__ void k_count_check(const unsigned long long* __restrict__ sums, const unsigned long long* __restrict__ n_s,
                              int64_t n_r, unsigned long long C, unsigned long long base, int* __restrict__ status) {
  if (sums[0] != base * (unsigned long long)n_r + C * n_s[0]) atomicCAS(status, 0, NH_ERR_COUNT_OVERFLOW);
}

__global__ void k_fill_u32(int64_t n, uint32_t* __restrict__ a, uint32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

}  // namespace

// Stream-ordered counting: launches only (no host synchronisation), the s-clique total into
// dcount and an error code into status (both device words the caller provides and zeroes).
int nh_count_enqueue(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, const float* vertex_cost,
                     float* measure, unsigned long long* dcount, int* status, cudaStream_t st) {
  if (!o || !ri || ri->o != o) return NH_ERR_INVALID;
  const int r = ri->r;
  const bool special = nh_supported(r, s) || (r == 1 && s == 4);
  if (!special && !nh_generic_pair(r, s)) return NH_ERR_UNSUPPORTED;
  if (!cnt && ri->n_r > 0) return NH_ERR_INVALID;
  GView g = make_view(o, ri);
  if (r == 1 && s == 2) {
    k_count_12<<<nh_blocks_for(o->n, 256, 152 * 32), 256, 0, st>>>(o->n, o->off, cnt);
    nh_note_launch();
    k_set_u64<<<1, 1, 0, st>>>(dcount, (unsigned long long)o->m);
    nh_note_launch();
    return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
  }
  int32_t* scratch = nullptr;
  int32_t* order = nullptr;
  unsigned long long* next = nullptr;
  int rc = NH_OK;
  if (measure) cudaMemsetAsync(measure, 0, sizeof(float) * (size_t)o->n, st);
  if (g_nh_inject_count_base == 0) {
    cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)ri->n_r, st);
  } else {  // fault injection: counts start near 2^32 (tests of the overflow check)
    k_fill_u32<<<nh_blocks_for(ri->n_r, 256, 152 * 32), 256, 0, st>>>(ri->n_r, cnt, (uint32_t)g_nh_inject_count_base);
    nh_note_launch();
  }
  if (!special) {
    rc = nh_count_generic(o, ri, s, cnt, dcount, status, st);  // every other pair: recursive listing
  } else if (s == 3) {
    const void* fn = (r == 1) ? (const void*)k_count_s3<1> : (const void*)k_count_s3<2>;
    int grid = grid_for(fn, kThreads, 0);
    if (vertex_cost && (rc = nh_schedule_items(o, vertex_cost, &order, &next, st))) return rc;
    if (r == 1) k_count_s3<1><<<grid, kThreads, 0, st>>>(g, cnt, dcount, order, next, measure, status);
    else k_count_s3<2><<<grid, kThreads, 0, st>>>(g, cnt, dcount, order, next, measure, status);
    nh_note_launch();
  } else {
    const int cap = (int)(o->max_out > 0 ? o->max_out : 1);
    const size_t smem = (size_t)kWarpsPerBlock * 3 * cap * sizeof(int32_t);
    const int use_smem = smem <= 200 * 1024;
    const void* fn = (r == 1) ? (const void*)k_count_s4<1> : (r == 2) ? (const void*)k_count_s4<2> : (const void*)k_count_s4<3>;
    if (use_smem) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = grid_for(fn, kThreads, use_smem ? smem : 0);
    if (!use_smem && (rc = nh_alloc(&scratch, (int64_t)grid * kWarpsPerBlock * 3 * cap, st))) return rc;
    const size_t dyn = use_smem ? smem : 0;
    if (vertex_cost && (rc = nh_schedule_items(o, vertex_cost, &order, &next, st))) {
      nh_free(scratch, st);
      return rc;
    }
    if (r == 1) k_count_s4<1><<<grid, kThreads, dyn, st>>>(g, cnt, dcount, scratch, cap, use_smem, status, order, next, measure);
    else if (r == 2) k_count_s4<2><<<grid, kThreads, dyn, st>>>(g, cnt, dcount, scratch, cap, use_smem, status, order, next, measure);
    else k_count_s4<3><<<grid, kThreads, dyn, st>>>(g, cnt, dcount, scratch, cap, use_smem, status, order, next, measure);
    nh_note_launch();
  }
  if (!rc && ri->n_r > 0) {
    unsigned long long* sums = nullptr;
    if (!(rc = nh_alloc(&sums, 1, st))) {
      cudaMemsetAsync(sums, 0, sizeof(unsigned long long), st);
      k_count_sum<<<nh_blocks_for(ri->n_r, 256, 152 * 8), 256, 0, st>>>(ri->n_r, cnt, sums);
      k_count_check<<<1, 1, 0, st>>>(sums, dcount, ri->n_r, (unsigned long long)nh_binom(s, r),
                                     (unsigned long long)g_nh_inject_count_base, status);
      nh_note_launch(2);
      nh_free(sums, st);
    }
  }
  if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
  nh_free(scratch, st); nh_free(order, st); nh_free(next, st);
  return rc;
}

int nh_count_impl(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, uint64_t* n_s,
                  const float* vertex_cost, float* measure, cudaStream_t st) {
  unsigned long long* dcount = nullptr;
  int* status = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&dcount, 1, st)) || (rc = nh_alloc(&status, 1, st))) {
    nh_free(dcount, st); nh_free(status, st);
    return rc;
  }
  cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  rc = nh_count_enqueue(o, ri, s, cnt, vertex_cost, measure, dcount, status, st);
  unsigned long long hcount = 0;
  int hs = 0;
  if (!rc) {
    cudaMemcpyAsync(&hcount, dcount, sizeof(hcount), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  }
  nh_free(dcount, st); nh_free(status, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  if (!rc && hs) rc = hs;
  if (!rc && n_s) *n_s = hcount;
  return rc;
}

extern "C" int nh_count_s_cliques(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, uint64_t* n_s,
                                  void* stream) {
  return nh_count_impl(o, ri, s, cnt, n_s, nullptr, nullptr, (cudaStream_t)stream);
}
