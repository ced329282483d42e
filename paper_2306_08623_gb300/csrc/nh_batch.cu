// nh_batch.cu -- a batch of graphs as one disjoint union, so that one persistent peel launch
// serves every graph of the batch (frontiers of all graphs share each round).  s-cliques never
// cross graphs, so every core number and every hierarchy node is that of its own graph; the
// union's lexicographic r-clique order lists graph 0's r-cliques first, then graph 1's, and so on.
#include <vector>

#include "nh_internal.cuh"

namespace {

struct UnionDesc {
  const int64_t* off;
  const int32_t* adj;
  int64_t n, nnz, vbase, ebase;
};

// blockIdx.y = graph; threads stride over that graph's offsets and adjacency entries
__global__ void k_union(const UnionDesc* __restrict__ d, int64_t* __restrict__ off_out, int32_t* __restrict__ adj_out) {
  const UnionDesc g = d[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride)
    off_out[g.vbase + i] = g.ebase + g.off[i];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.nnz; j += stride)
    adj_out[g.ebase + j] = (int32_t)(g.vbase + g.adj[j]);
}

__global__ void k_union_tail(int64_t* off_out, int64_t N, int64_t NNZ) { off_out[N] = NNZ; }

// first r-clique id of each graph: r = 2 -> uoff[vbase]; r = 3 -> toff[uoff[vbase]]
__global__ void k_rbases(const int64_t* __restrict__ vb, int ng, const int64_t* __restrict__ uoff,
                         const int64_t* __restrict__ toff, int r, int64_t* __restrict__ out) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= ng; g += gridDim.x * blockDim.x) {
    const int64_t e = uoff[vb[g]];
    out[g] = (r == 2) ? e : toff[e];
  }
}

}  // namespace

extern "C" int nh_batch_union(const nh_graph_desc* graphs, int n_graphs, int64_t* off_out, int32_t* adj_out,
                              int64_t* vbase, void* stream) {
  if (!graphs || n_graphs < 1 || !off_out || !vbase) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<UnionDesc> h(n_graphs);
  int64_t N = 0, NNZ = 0, maxlen = 0;
  for (int g = 0; g < n_graphs; g++) {
    const nh_graph_desc& x = graphs[g];
    if (x.n < 0 || x.nnz < 0 || (x.n > 0 && !x.off) || (x.nnz > 0 && !x.adj)) return NH_ERR_INVALID;
    h[g] = UnionDesc{x.off, x.adj, x.n, x.nnz, N, NNZ};
    vbase[g] = N;
    N += x.n;
    NNZ += x.nnz;
    maxlen = x.n > maxlen ? x.n : maxlen;
    maxlen = x.nnz > maxlen ? x.nnz : maxlen;
  }
  vbase[n_graphs] = N;
  if (N >= (1ll << 31) || (NNZ > 0 && !adj_out)) return NH_ERR_INVALID;
  UnionDesc* d = nullptr;
  int rc = nh_alloc(&d, n_graphs, st);
  if (rc) return rc;
  if (cudaMemcpyAsync(d, h.data(), sizeof(UnionDesc) * n_graphs, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = NH_ERR_CUDA;
  if (!rc) {
    const unsigned bx = nh_blocks_for(maxlen, 256, 64);
    k_union<<<dim3(bx, (unsigned)n_graphs), 256, 0, st>>>(d, off_out, adj_out);
    k_union_tail<<<1, 1, 0, st>>>(off_out, N, NNZ);
    nh_note_launch(2);
    if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
  }
  nh_free(d, st);
  // the host descriptor table is read by the copy above: wait for it before returning
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

extern "C" int nh_rindex_bases(const nh_rindex* ri, const int64_t* vbase, int n_graphs, int64_t* rbase, void* stream) {
  if (!ri || !vbase || !rbase || n_graphs < 1) return NH_ERR_INVALID;
  if (ri->r > 3) return NH_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  if (ri->r == 1) {
    for (int g = 0; g <= n_graphs; g++) rbase[g] = vbase[g];
    return NH_OK;
  }
  int64_t *dv = nullptr, *dout = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&dv, n_graphs + 1, st)) || (rc = nh_alloc(&dout, n_graphs + 1, st))) {
    nh_free(dv, st); nh_free(dout, st);
    return rc;
  }
  cudaMemcpyAsync(dv, vbase, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice, st);
  k_rbases<<<nh_blocks_for(n_graphs + 1, 256, 64), 256, 0, st>>>(dv, n_graphs, ri->o->uoff, ri->toff, ri->r, dout);
  nh_note_launch();
  cudaMemcpyAsync(rbase, dout, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyDeviceToHost, st);
  nh_free(dv, st); nh_free(dout, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
  return rc;
}

// ---------------------------------------------------------------------------------------------
// nh_batch_*: a batch as one object -- the union CSR, its orientation and its r-clique index are
// built once (nh_batch_prepare); nh_batch_run then enqueues counts, the persistent peel and
// construct-tree for one s on the whole union with no host synchronisation (capturable).
// ---------------------------------------------------------------------------------------------

struct nh_batch {
  int n_graphs = 0, r = 0;
  int64_t N = 0, NNZ = 0;
  int64_t* off = nullptr;  // union CSR (device, owned)
  int32_t* adj = nullptr;
  int64_t* rbase_dev = nullptr;  // first r-clique id of every graph, n_graphs + 1 entries (device)
  std::vector<int64_t> vbase, rbase;
  nh_oriented* o = nullptr;
  nh_rindex* ri = nullptr;
  cudaStream_t stream = nullptr;
};

namespace {

// nbase[g] = least node id that a leaf of graph g hangs from (construct-tree numbers nodes in the
// order of their root r-cliques, and every node's root r-clique hangs from it, so this is the
// first node of graph g); graphs without nodes keep INT64_MAX
__global__ void k_node_bases(int64_t n_r, const int32_t* __restrict__ parent, const int64_t* __restrict__ rbase,
                             int ng, unsigned long long* __restrict__ nbase) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent[i];
    if (p < 0) continue;
    int lo = 0, hi = ng;  // graph g with rbase[g] <= i < rbase[g+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (rbase[mid] <= i) lo = mid; else hi = mid;
    }
    atomicMin(nbase + lo, (unsigned long long)p);
  }
}

}  // namespace

extern "C" void nh_batch_free(nh_batch* b) {
  if (!b) return;
  cudaStream_t st = b->stream;
  if (b->ri) nh_rindex_free(b->ri);
  if (b->o) nh_oriented_free(b->o);
  cudaStreamSynchronize(st);  // the handles above are freed in stream order before the CSR they read
  nh_free(b->off, st);
  nh_free(b->adj, st);
  nh_free(b->rbase_dev, st);
  cudaStreamSynchronize(st);
  delete b;
}

extern "C" int nh_batch_prepare(const nh_graph_desc* graphs, int n_graphs, int r, nh_batch** out, int64_t* n_r,
                                void* stream) {
  if (!out) return NH_ERR_INVALID;
  *out = nullptr;
  if (!graphs || n_graphs < 1 || r < 1 || r > 3) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  nh_batch* b = new nh_batch();
  b->n_graphs = n_graphs;
  b->r = r;
  b->stream = st;
  for (int g = 0; g < n_graphs; g++) {
    if (graphs[g].n < 0 || graphs[g].nnz < 0) { delete b; return NH_ERR_INVALID; }
    b->N += graphs[g].n;
    b->NNZ += graphs[g].nnz;
  }
  if (b->N < 1 || b->N >= (1ll << 31)) { delete b; return NH_ERR_INVALID; }
  b->vbase.assign(n_graphs + 1, 0);
  b->rbase.assign(n_graphs + 1, 0);
  int rc = NH_OK;
  if ((rc = nh_alloc(&b->off, b->N + 1, st)) || (rc = nh_alloc(&b->adj, b->NNZ, st)) ||
      (rc = nh_alloc(&b->rbase_dev, n_graphs + 1, st))) {
    nh_batch_free(b);
    return rc;
  }
  int64_t nr = 0;
  if (!rc) rc = nh_batch_union(graphs, n_graphs, b->off, b->adj, b->vbase.data(), stream);
  if (!rc) rc = nh_build_orientation(b->N, b->NNZ, b->off, b->adj, &b->o, stream);
  if (!rc) rc = nh_index_r_cliques(b->o, r, &b->ri, &nr, stream);
  if (!rc) rc = nh_rindex_bases(b->ri, b->vbase.data(), n_graphs, b->rbase.data(), stream);
  if (!rc && cudaMemcpyAsync(b->rbase_dev, b->rbase.data(), sizeof(int64_t) * (n_graphs + 1),
                             cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = NH_ERR_CUDA;
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
  if (rc) {
    nh_batch_free(b);
    return rc;
  }
  *out = b;
  if (n_r) *n_r = nr;
  return NH_OK;
}

extern "C" int nh_batch_bases(const nh_batch* b, int64_t* vbase, int64_t* rbase) {
  if (!b) return NH_ERR_INVALID;
  for (int g = 0; g <= b->n_graphs; g++) {
    if (vbase) vbase[g] = b->vbase[g];
    if (rbase) rbase[g] = b->rbase[g];
  }
  return NH_OK;
}

extern "C" int nh_batch_run(nh_batch* b, int s, uint32_t* cnt, uint32_t* core, uint32_t* round, int32_t* uf,
                            int32_t* L, int32_t* parent, uint32_t* label, int64_t* res, void* stream) {
  if (!b) return NH_ERR_INVALID;
  return nh_hierarchy_enqueue(b->o, b->ri, s, cnt, core, round, uf, L, parent, label, res, stream);
}

extern "C" int nh_batch_node_bases(const nh_batch* b, const int32_t* parent, int64_t n_nodes, int64_t* nbase,
                                   void* stream) {
  if (!b || !nbase || n_nodes < 0 || (b->ri->n_r > 0 && !parent)) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const int ng = b->n_graphs;
  unsigned long long* d = nullptr;
  int rc = nh_alloc(&d, ng, st);
  if (rc) return rc;
  cudaMemsetAsync(d, 0xff, sizeof(unsigned long long) * ng, st);
  if (b->ri->n_r > 0) {
    k_node_bases<<<nh_blocks_for(b->ri->n_r, 256, 152 * 16), 256, 0, st>>>(b->ri->n_r, parent, b->rbase_dev, ng, d);
    nh_note_launch();
  }
  std::vector<unsigned long long> h(ng);
  if (cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * ng, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = NH_ERR_CUDA;
  nh_free(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  if (rc) return rc;
  nbase[ng] = n_nodes;
  for (int g = ng - 1; g >= 0; g--) {
    const unsigned long long v = h[g];
    nbase[g] = (v == ~0ull || (int64_t)v > nbase[g + 1]) ? nbase[g + 1] : (int64_t)v;
  }
  return NH_OK;
}
