// nh_batch.cu -- a12: a batch of graphs as one disjoint union, so that one persistent peel launch
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
