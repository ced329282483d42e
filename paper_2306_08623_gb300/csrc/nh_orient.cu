// nh_orient.cu -- a1 (Arb-Orient: degree orientation + canonical edge ids) and a2 (r-clique index).
#include "nh_internal.cuh"

extern long long g_nh_inject_table_cap;  // fault injection (nh_api.cu): forced table capacity

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

__device__ __forceinline__ bool rank_less(int64_t du, int32_t u, int64_t dv, int32_t v) {
  return du < dv || (du == dv && u < v);
}

// CSR checks before anything indexes through it: offsets start at 0, never decrease and end at
// nnz (first kernel); neighbour ids in range, strictly increasing, no self-loop (second kernel)
__global__ void k_check_off(int64_t n, int64_t nnz, const int64_t* __restrict__ off, int* __restrict__ bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = off[v];
    if (o < 0 || o > nnz || (v == 0 && o != 0) || (v == n && o != nnz) || (v < n && off[v + 1] < o)) atomicExch(bad, 1);
  }
}

__global__ void k_check_adj(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            int* __restrict__ bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t prev = -1;
    for (int64_t j = off[v]; j < off[v + 1]; j++) {
      const int32_t w = adj[j];
      if (w < 0 || w >= n || w == (int32_t)v || w <= prev) { atomicExch(bad, 1); break; }
      prev = w;
    }
  }
}

// per vertex: out-degree under the degree order, number of neighbours above the vertex id
__global__ void k_orient_count(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                               uint32_t* __restrict__ outdeg, uint32_t* __restrict__ updeg,
                               unsigned long long* __restrict__ maxes) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int64_t b = off[v], e = off[v + 1], dv = e - b;
    uint32_t cnt = 0;
    for (int64_t j = b + lane; j < e; j += 32) {
      int32_t w = adj[j];
      int64_t dw = off[w + 1] - off[w];
      cnt += rank_less(dv, (int32_t)v, dw, w) ? 1u : 0u;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(NH_FULL, cnt, d);
    if (lane == 0) {
      int64_t up = e - nh_lower_bound(adj, b, e, (int32_t)v + 1);
      outdeg[v] = cnt;
      updeg[v] = (uint32_t)up;
      atomicMax(&maxes[0], (unsigned long long)cnt);
      atomicMax(&maxes[1], (unsigned long long)dv);
    }
  }
}

// per adjacency entry: canonical edge id; per upper entry: edge endpoints; per out entry: the
// out-CSR (order of the adjacency list is kept, so out-lists stay sorted by vertex id)
__global__ void k_orient_fill(int64_t n, int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                              const int64_t* __restrict__ uoff, const int64_t* __restrict__ ooff,
                              int32_t* __restrict__ eid, int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                              int32_t* __restrict__ oadj, int32_t* __restrict__ oeid, int32_t* __restrict__ osrc,
                              int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int64_t b = off[v], e = off[v + 1], dv = e - b;
    const int64_t upos = nh_lower_bound(adj, b, e, (int32_t)v + 1);
    int64_t opos = ooff[v];
    for (int64_t base = b; base < e; base += 32) {
      const int64_t j = base + lane;
      bool out = false;
      int32_t w = 0, id = 0;
      if (j < e) {
        w = adj[j];
        const int64_t bw = off[w], ew = off[w + 1];
        if (w > (int32_t)v) {
          id = (int32_t)(uoff[v] + (j - upos));
          if (id < m) {  // false only for a non-symmetric input, which is then rejected
            eu[id] = (int32_t)v;
            ev[id] = w;
          }
        } else {
          const int64_t p = nh_lower_bound(adj, bw, ew, (int32_t)v);
          const int64_t upw = nh_lower_bound(adj, bw, ew, w + 1);
          id = (int32_t)(uoff[w] + (p - upw));
          if (p >= ew || adj[p] != (int32_t)v) atomicExch(bad, 1);  // the mirror entry is missing
        }
        eid[j] = id;
        out = rank_less(dv, (int32_t)v, ew - bw, w);
      }
      const unsigned mask = __ballot_sync(NH_FULL, out);
      const int64_t q = opos + __popc(mask & ((1u << lane) - 1u));
      if (out && q < m) {  // q >= m only for a non-symmetric input, which is then rejected
        oadj[q] = w;
        oeid[q] = id;
        osrc[q] = (int32_t)v;
      }
      opos += __popc(mask);
    }
  }
}

// triangles per lexicographic edge (a,b): common neighbours c > b
__global__ void k_tri_count(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                            uint32_t* __restrict__ tcount) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    const int32_t a = eu[e], b = ev[e];
    int64_t ab = nh_lower_bound(adj, off[a], off[a + 1], b + 1), ae = off[a + 1];
    int64_t bb = nh_lower_bound(adj, off[b], off[b + 1], b + 1), be = off[b + 1];
    // scan the shorter upper part, search the longer
    if (ae - ab > be - bb) {
      int64_t t0 = ab, t1 = ae;
      ab = bb; ae = be; bb = t0; be = t1;
    }
    uint32_t cnt = 0;
    for (int64_t j = ab + lane; j < ae; j += 32) cnt += (nh_find(adj, bb, be, adj[j]) >= 0) ? 1u : 0u;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(NH_FULL, cnt, d);
    if (lane == 0) tcount[e] = cnt;
  }
}

__global__ void k_tri_fill(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ eid, const int32_t* __restrict__ eu,
                           const int32_t* __restrict__ ev, const int64_t* __restrict__ toff, int32_t* __restrict__ tri,
                           int32_t* __restrict__ tedge, nh_slot* __restrict__ table, unsigned long long mask,
                           int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    const int32_t a = eu[e], b = ev[e];
    int64_t ab = nh_lower_bound(adj, off[a], off[a + 1], b + 1), ae = off[a + 1];
    int64_t bb = nh_lower_bound(adj, off[b], off[b + 1], b + 1), be = off[b + 1];
    const bool scan_a = ae - ab <= be - bb;
    if (!scan_a) {
      int64_t t0 = ab, t1 = ae;
      ab = bb; ae = be; bb = t0; be = t1;
    }
    int64_t pos = toff[e];
    for (int64_t base = ab; base < ae; base += 32) {
      const int64_t j = base + lane;
      int32_t c = 0;
      int64_t q = -1;
      if (j < ae) {
        c = adj[j];
        q = nh_find(adj, bb, be, c);
      }
      const bool hit = q >= 0;
      const unsigned msk = __ballot_sync(NH_FULL, hit);
      if (hit) {
        const int64_t id = pos + __popc(msk & ((1u << lane) - 1u));
        tri[3 * id + 0] = a;
        tri[3 * id + 1] = b;
        tri[3 * id + 2] = c;
        tedge[3 * id + 0] = (int32_t)e;                 // {a, b}
        tedge[3 * id + 1] = eid[scan_a ? j : q];         // {a, c}
        tedge[3 * id + 2] = eid[scan_a ? q : j];         // {b, c}
        const unsigned long long key = ((unsigned long long)(uint32_t)e << 32) | (uint32_t)c;
        unsigned long long h = nh_mix64(key) & mask;
        bool done = false;
        for (unsigned long long p = 0; p <= mask; ++p) {
          unsigned long long old = atomicCAS(&table[h].key, NH_EMPTY_KEY, key);
          if (old == NH_EMPTY_KEY || old == key) {
            table[h].val = (uint32_t)id;
            done = true;
            break;
          }
          h = (h + 1) & mask;
        }
        if (!done) atomicExch(status, NH_ERR_TABLE_FULL);
      }
      pos += __popc(msk);
    }
  }
}

// all triangles per edge (a,b): |N(a) n N(b)|
__global__ void k_et_count(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                           uint32_t* __restrict__ etcount) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    const int32_t a = eu[e], b = ev[e];
    int64_t sb = off[a], se = off[a + 1], lb = off[b], le = off[b + 1];
    if (se - sb > le - lb) {
      int64_t t0 = sb, t1 = se;
      sb = lb; se = le; lb = t0; le = t1;
    }
    uint32_t cnt = 0;
    for (int64_t j = sb + lane; j < se; j += 32) cnt += (nh_find(adj, lb, le, adj[j]) >= 0) ? 1u : 0u;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(NH_FULL, cnt, d);
    if (lane == 0) etcount[e] = cnt;
  }
}

// per edge (a,b): the third vertices w of its triangles, ascending, and each triangle's id
__global__ void k_et_fill(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                          const int32_t* __restrict__ eid, const int32_t* __restrict__ eu,
                          const int32_t* __restrict__ ev, const int64_t* __restrict__ etoff,
                          const nh_slot* __restrict__ table, unsigned long long mask, int32_t* __restrict__ etw,
                          int32_t* __restrict__ ettid, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    const int32_t a = eu[e], b = ev[e];
    int64_t sb = off[a], se = off[a + 1], lb = off[b], le = off[b + 1];
    const bool scan_a = (se - sb) <= (le - lb);
    if (!scan_a) {
      int64_t t0 = sb, t1 = se;
      sb = lb; se = le; lb = t0; le = t1;
    }
    int64_t pos = etoff[e];
    for (int64_t base = sb; base < se; base += 32) {
      const int64_t j = base + lane;
      int32_t w = 0;
      int64_t q = -1;
      if (j < se) {
        w = adj[j];
        q = nh_find(adj, lb, le, w);
      }
      const unsigned msk = __ballot_sync(NH_FULL, q >= 0);
      if (q >= 0) {
        const int64_t k = pos + __popc(msk & ((1u << lane) - 1u));
        const int32_t e_aw = eid[scan_a ? j : q], e_bw = eid[scan_a ? q : j];
        const int64_t id = nh_tri_lookup(table, mask, nh_tri_key(a, b, w, (int32_t)e, e_aw, e_bw));
        if (id < 0) atomicExch(status, NH_ERR_INTERNAL);
        etw[k] = w;
        ettid[k] = (int32_t)id;
      }
      pos += __popc(msk);
    }
  }
}

// r = 2: per edge (a,b), the third vertices w of its triangles in ascending order with the ids of
// the edges {a,w} and {b,w} (read from the adjacency positions of the intersection, no probe)
__global__ void k_et2_fill(int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ eid, const int32_t* __restrict__ eu,
                           const int32_t* __restrict__ ev, const int64_t* __restrict__ t2off,
                           int32_t* __restrict__ t2w, int32_t* __restrict__ t2ea, int32_t* __restrict__ t2eb) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    const int32_t a = eu[e], b = ev[e];
    int64_t sb = off[a], se = off[a + 1], lb = off[b], le = off[b + 1];
    const bool scan_a = (se - sb) <= (le - lb);
    if (!scan_a) {
      int64_t t0 = sb, t1 = se;
      sb = lb; se = le; lb = t0; le = t1;
    }
    int64_t pos = t2off[e];
    for (int64_t base = sb; base < se; base += 32) {
      const int64_t j = base + lane;
      int32_t w = 0;
      int64_t q = -1;
      if (j < se) {
        w = adj[j];
        q = nh_find(adj, lb, le, w);
      }
      const unsigned msk = __ballot_sync(NH_FULL, q >= 0);
      if (q >= 0) {
        const int64_t k = pos + __popc(msk & ((1u << lane) - 1u));
        t2w[k] = w;
        t2ea[k] = eid[scan_a ? j : q];
        t2eb[k] = eid[scan_a ? q : j];
      }
      pos += __popc(msk);
    }
  }
}

// per edge: the sum of d+(w) over its triangle list (saturating at 2^32 - 1)
__global__ void k_et2_cost(int64_t m, const int64_t* __restrict__ ooff, const int64_t* __restrict__ t2off,
                           const int32_t* __restrict__ t2w, uint32_t* __restrict__ t2cost) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < m; e += nwarps) {
    unsigned long long sum = 0;
    for (int64_t j = t2off[e] + lane; j < t2off[e + 1]; j += 32) {
      const int32_t w = t2w[j];
      sum += (unsigned long long)(ooff[w + 1] - ooff[w]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(NH_FULL, sum, d);
    if (lane == 0) t2cost[e] = sum > 0xffffffffull ? 0xffffffffu : (uint32_t)sum;
  }
}

__global__ void k_edge_insert(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                              unsigned long long* __restrict__ ekey, uint32_t* __restrict__ eval,
                              unsigned long long mask, int* __restrict__ status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = ((unsigned long long)(uint32_t)eu[e] << 32) | (uint32_t)ev[e];
    unsigned long long h = nh_mix64(key) & mask;
    bool done = false;
    for (unsigned long long p = 0; p <= mask; ++p) {
      const unsigned long long old = atomicCAS(ekey + h, NH_EMPTY_KEY, key);
      if (old == NH_EMPTY_KEY || old == key) {
        eval[h] = (uint32_t)e;
        done = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (!done) atomicExch(status, NH_ERR_TABLE_FULL);
  }
}

__global__ void k_fill_empty_keys(unsigned long long* k, unsigned long long cap) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x)
    k[i] = NH_EMPTY_KEY;
}

__global__ void k_fill_empty(nh_slot* t, unsigned long long cap) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    t[i].key = NH_EMPTY_KEY;
    t[i].val = 0xffffffffu;
    t[i].pad = 0;
  }
}

__global__ void k_tuples(int r, int64_t n_r, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                         const int32_t* __restrict__ tri, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    if (r == 1) out[i] = (int32_t)i;
    else if (r == 2) { out[2 * i] = eu[i]; out[2 * i + 1] = ev[i]; }
    else { out[3 * i] = tri[3 * i]; out[3 * i + 1] = tri[3 * i + 1]; out[3 * i + 2] = tri[3 * i + 2]; }
  }
}

unsigned warp_grid(int64_t items) {
  int64_t blocks = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 64) blocks = 152 * 64;
  return (unsigned)blocks;
}

void free_oriented(nh_oriented* o) {
  if (!o) return;
  cudaFree(o->eid); cudaFree(o->ooff); cudaFree(o->oadj); cudaFree(o->oeid); cudaFree(o->osrc);
  cudaFree(o->uoff); cudaFree(o->eu); cudaFree(o->ev); cudaFree(o->ekey); cudaFree(o->eval);
  delete o;
}

void free_rindex(nh_rindex* ri) {
  if (!ri) return;
  cudaFree(ri->tri); cudaFree(ri->tedge); cudaFree(ri->toff); cudaFree(ri->table);
  cudaFree(ri->etoff); cudaFree(ri->etw); cudaFree(ri->ettid);
  cudaFree(ri->t2off); cudaFree(ri->t2w); cudaFree(ri->t2ea); cudaFree(ri->t2eb); cudaFree(ri->t2cost);
  if (ri->prev) free_rindex(ri->prev);
  delete ri;
}

}  // namespace

extern "C" int nh_build_orientation(int64_t n, int64_t nnz, const int64_t* off, const int32_t* adj,
                                    nh_oriented** out, void* stream) {
  if (!out) return NH_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || nnz < 0 || (nnz & 1) || !off || (nnz > 0 && !adj) || n >= (1ll << 31) || nnz / 2 >= (1ll << 31))
    return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  nh_oriented* o = new nh_oriented();
  o->n = n; o->m = nnz / 2; o->off = off; o->adj = adj; o->stream = st;
  const int64_t m = o->m;
  uint32_t *outdeg = nullptr, *updeg = nullptr;
  unsigned long long* maxes = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&o->eid, nnz, st)) || (rc = nh_alloc(&o->ooff, n + 1, st)) || (rc = nh_alloc(&o->oadj, m, st)) ||
      (rc = nh_alloc(&o->oeid, m, st)) || (rc = nh_alloc(&o->osrc, m, st)) || (rc = nh_alloc(&o->uoff, n + 1, st)) ||
      (rc = nh_alloc(&o->eu, m, st)) || (rc = nh_alloc(&o->ev, m, st)) || (rc = nh_alloc(&outdeg, n, st)) ||
      (rc = nh_alloc(&updeg, n, st)) || (rc = nh_alloc(&maxes, 3, st))) {
    nh_free(outdeg, st); nh_free(updeg, st); nh_free(maxes, st);
    cudaStreamSynchronize(st);
    free_oriented(o);
    return rc;
  }
  unsigned long long hmax[3] = {0, 0, 0};
  int64_t m_check = -1;
  {
    // validate the CSR before any kernel indexes through it
    int* bad = (int*)(maxes + 2);
    int hbad = 0;
    cudaMemsetAsync(maxes, 0, 3 * sizeof(unsigned long long), st);
    k_check_off<<<nh_blocks_for(n + 1, 256, 152 * 16), 256, 0, st>>>(n, nnz, off, bad);
    nh_note_launch();
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    if (!rc && !hbad && nnz > 0) {
      k_check_adj<<<nh_blocks_for(n, 256, 152 * 16), 256, 0, st>>>(n, off, adj, bad);
      nh_note_launch();
      cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    }
    if (!rc && hbad) rc = NH_ERR_INVALID;
    if (rc) {
      nh_free(outdeg, st); nh_free(updeg, st); nh_free(maxes, st);
      cudaStreamSynchronize(st);
      free_oriented(o);
      return rc;
    }
  }
  cudaMemsetAsync(maxes, 0, 3 * sizeof(unsigned long long), st);
  k_orient_count<<<warp_grid(n), kThreads, 0, st>>>(n, off, adj, outdeg, updeg, maxes);
  nh_note_launch();
  if (!rc) rc = nh_exclusive_scan_u32(outdeg, o->ooff, n, st);
  if (!rc) rc = nh_exclusive_scan_u32(updeg, o->uoff, n, st);
  if (!rc) {
    k_orient_fill<<<warp_grid(n), kThreads, 0, st>>>(n, m, off, adj, o->uoff, o->ooff, o->eid, o->eu, o->ev, o->oadj,
                                                     o->oeid, o->osrc, (int*)(maxes + 2));
    nh_note_launch();
    cudaMemcpyAsync(hmax, maxes, sizeof(hmax), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&m_check, o->uoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  }
  nh_free(outdeg, st); nh_free(updeg, st); nh_free(maxes, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (!rc && e != cudaSuccess) rc = NH_ERR_CUDA;
  if (!rc && cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
  if (!rc && (m_check != m || hmax[2] != 0)) rc = NH_ERR_INVALID;  // not symmetric
  if (rc) {
    free_oriented(o);
    return rc;
  }
  o->max_out = (int64_t)hmax[0];
  o->max_deg = (int64_t)hmax[1];
  // edge table: (u, v) -> edge id, for one-probe adjacency tests
  {
    unsigned long long cap = 1024;
    while (cap < 2ull * (unsigned long long)m) cap <<= 1;
    if (g_nh_inject_table_cap > 0) cap = (unsigned long long)g_nh_inject_table_cap;
    int* status = nullptr;
    if ((rc = nh_alloc(&o->ekey, (int64_t)cap, st)) || (rc = nh_alloc(&o->eval, (int64_t)cap, st)) ||
        (rc = nh_alloc(&status, 1, st))) {
      nh_free(status, st);
      cudaStreamSynchronize(st);
      free_oriented(o);
      return rc;
    }
    o->emask = cap - 1;
    cudaMemsetAsync(status, 0, sizeof(int), st);
    k_fill_empty_keys<<<nh_blocks_for((int64_t)cap, 256, 152 * 32), 256, 0, st>>>(o->ekey, cap);
    nh_note_launch();
    k_edge_insert<<<nh_blocks_for(m, 256, 152 * 32), 256, 0, st>>>(m, o->eu, o->ev, o->ekey, o->eval, o->emask,
                                                                    status);
    nh_note_launch();
    int hs = 0;
    cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    nh_free(status, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    if (!rc && hs) rc = hs;
    if (rc) {
      free_oriented(o);
      return rc;
    }
  }
  *out = o;
  return NH_OK;
}

extern "C" int nh_oriented_info(const nh_oriented* o, int64_t* n, int64_t* m, int64_t* max_out, int64_t* max_deg) {
  if (!o) return NH_ERR_INVALID;
  if (n) *n = o->n;
  if (m) *m = o->m;
  if (max_out) *max_out = o->max_out;
  if (max_deg) *max_deg = o->max_deg;
  return NH_OK;
}

extern "C" void nh_oriented_free(nh_oriented* o) { free_oriented(o); }

extern "C" int nh_index_r_cliques(const nh_oriented* o, int r, nh_rindex** out, int64_t* n_r, void* stream) {
  if (!out || !o || r < 1 || r > 6) return NH_ERR_INVALID;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  if (r >= 4) {
    // r = 4..6: a chain of tables, each r-clique keyed by the id of its first r-1 vertices
    nh_rindex* prev = nullptr;
    int rc = nh_index_r_cliques(o, r - 1, &prev, nullptr, stream);
    if (rc) return rc;
    nh_rindex* ri = new nh_rindex();
    ri->r = r; ri->o = o; ri->stream = st; ri->prev = prev;
    rc = nh_index_generic(o, prev, r, ri, st);
    if (rc) {
      cudaStreamSynchronize(st);
      free_rindex(ri);
      return rc;
    }
    if (n_r) *n_r = ri->n_r;
    *out = ri;
    return NH_OK;
  }
  nh_rindex* ri = new nh_rindex();
  ri->r = r; ri->o = o; ri->stream = st;
  if (r == 1) ri->n_r = o->n;
  if (r == 2) {
    ri->n_r = o->m;
    // per-edge triangle lists with the ids of the two other edges: the (2,3) s-cliques and the
    // (2,4) candidate sets of every edge.  Optional: without device memory for them (36 bytes per
    // triangle) the peels fall back to adjacency scans with edge-table probes.
    const int64_t m = o->m;
    if (m > 0) {
      uint32_t* tcount = nullptr;
      int rc = nh_alloc(&tcount, m, st);
      if (!rc) rc = nh_alloc(&ri->t2off, m + 1, st);
      if (!rc) {
        k_et_count<<<warp_grid(m), kThreads, 0, st>>>(m, o->off, o->adj, o->eu, o->ev, tcount);
        nh_note_launch();
        rc = nh_exclusive_scan_u32(tcount, ri->t2off, m, st);
      }
      int64_t tot = 0;
      if (!rc) {
        cudaMemcpyAsync(&tot, ri->t2off + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
      }
      nh_free(tcount, st);
      if (!rc && tot >= (1ll << 31)) rc = NH_ERR_UNSUPPORTED;  // positions are int32 in the peel
      if (!rc) rc = nh_alloc(&ri->t2w, tot, st);
      if (!rc) rc = nh_alloc(&ri->t2ea, tot, st);
      if (!rc) rc = nh_alloc(&ri->t2eb, tot, st);
      if (!rc) rc = nh_alloc(&ri->t2cost, m, st);
      if (!rc) {
        k_et2_fill<<<warp_grid(m), kThreads, 0, st>>>(m, o->off, o->adj, o->eid, o->eu, o->ev, ri->t2off, ri->t2w,
                                                       ri->t2ea, ri->t2eb);
        k_et2_cost<<<warp_grid(m), kThreads, 0, st>>>(m, o->ooff, ri->t2off, ri->t2w, ri->t2cost);
        nh_note_launch(2);
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
      }
      if (rc == NH_ERR_CUDA) {
        free_rindex(ri);
        return rc;
      }
      if (rc) {  // no room (or too many triangles): run without the lists
        (void)cudaGetLastError();
        cudaFree(ri->t2off); cudaFree(ri->t2w); cudaFree(ri->t2ea); cudaFree(ri->t2eb); cudaFree(ri->t2cost);
        ri->t2off = nullptr; ri->t2w = ri->t2ea = ri->t2eb = nullptr;
        ri->t2cost = nullptr;
      }
    }
  }
  if (r == 3) {
    const int64_t m = o->m;
    uint32_t* tcount = nullptr;
    int* status = nullptr;
    int rc = NH_OK;
    if ((rc = nh_alloc(&tcount, m, st)) || (rc = nh_alloc(&ri->toff, m + 1, st)) || (rc = nh_alloc(&status, 1, st))) {
      nh_free(tcount, st); nh_free(status, st);
      cudaStreamSynchronize(st);
      free_rindex(ri);
      return rc;
    }
    k_tri_count<<<warp_grid(m), kThreads, 0, st>>>(m, o->off, o->adj, o->eu, o->ev, tcount);
    nh_note_launch();
    rc = nh_exclusive_scan_u32(tcount, ri->toff, m, st);
    int64_t ntri = 0;
    if (!rc) cudaMemcpyAsync(&ntri, ri->toff + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    if (!rc && ntri >= (1ll << 32) - 1) rc = NH_ERR_UNSUPPORTED;
    unsigned long long cap = 1024;
    while (cap < 2ull * (unsigned long long)ntri) cap <<= 1;
    if (g_nh_inject_table_cap > 0) cap = (unsigned long long)g_nh_inject_table_cap;
    if (!rc) rc = nh_alloc(&ri->tri, 3 * ntri, st);
    if (!rc) rc = nh_alloc(&ri->tedge, 3 * ntri, st);
    if (!rc) rc = nh_alloc(&ri->table, (int64_t)cap, st);
    if (!rc) {
      ri->mask = cap - 1;
      ri->n_r = ntri;
      cudaMemsetAsync(status, 0, sizeof(int), st);
      k_fill_empty<<<nh_blocks_for((int64_t)cap, 256, 152 * 32), 256, 0, st>>>(ri->table, cap);
      nh_note_launch();
      k_tri_fill<<<warp_grid(m), kThreads, 0, st>>>(m, o->off, o->adj, o->eid, o->eu, o->ev, ri->toff, ri->tri,
                                                     ri->tedge, ri->table, ri->mask, status);
    nh_note_launch();
      int hs = 0;
      cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
      if (!rc && hs) rc = hs;
    }
    // per-edge triangle lists (every triangle appears in the lists of its three edges)
    if (!rc) rc = nh_alloc(&ri->etoff, m + 1, st);
    if (!rc) {
      k_et_count<<<warp_grid(m), kThreads, 0, st>>>(m, o->off, o->adj, o->eu, o->ev, tcount);
      nh_note_launch();
      rc = nh_exclusive_scan_u32(tcount, ri->etoff, m, st);
    }
    if (!rc) rc = nh_alloc(&ri->etw, 3 * ntri, st);
    if (!rc) rc = nh_alloc(&ri->ettid, 3 * ntri, st);
    if (!rc) {
      cudaMemsetAsync(status, 0, sizeof(int), st);
      k_et_fill<<<warp_grid(m), kThreads, 0, st>>>(m, o->off, o->adj, o->eid, o->eu, o->ev, ri->etoff, ri->table,
                                                    ri->mask, ri->etw, ri->ettid, status);
      nh_note_launch();
      int hs = 0;
      int64_t tot = -1;
      cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(&tot, ri->etoff + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
      if (!rc && hs) rc = hs;
      if (!rc && tot != 3 * ntri) rc = NH_ERR_INTERNAL;
    }
    nh_free(tcount, st); nh_free(status, st);
    if (rc) {
      cudaStreamSynchronize(st);
      free_rindex(ri);
      return rc;
    }
  }
  if (n_r) *n_r = ri->n_r;
  *out = ri;
  return NH_OK;
}

extern "C" int nh_rindex_tuples(const nh_rindex* ri, int32_t* tuples, void* stream) {
  if (!ri || (!tuples && ri->n_r > 0)) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (ri->n_r == 0) return NH_OK;
  if (ri->r >= 4)
    return cudaMemcpyAsync(tuples, ri->tri, sizeof(int32_t) * (size_t)ri->r * (size_t)ri->n_r, cudaMemcpyDeviceToDevice,
                           st) == cudaSuccess ? NH_OK : NH_ERR_CUDA;
  k_tuples<<<nh_blocks_for(ri->n_r, 256, 152 * 32), 256, 0, st>>>(ri->r, ri->n_r, ri->o->eu, ri->o->ev, ri->tri, tuples);
  nh_note_launch();
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

extern "C" void nh_rindex_free(nh_rindex* ri) { free_rindex(ri); }
