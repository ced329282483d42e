// nh_tree.cu -- a9: construct-tree-efficient (Alg. 5).  One node per union-find component; the
// parent of node C is the node of find(L[C]); a node whose subtree holds one r-clique (one
// member, no child node) is dropped and that r-clique hangs from the dropped node's parent.
#include "nh_internal.cuh"

namespace {

// full path compression: uf[i] = root of i (parents only ever point to ancestors)
__global__ void k_tree_roots(int64_t n_r, int32_t* __restrict__ uf, uint32_t* __restrict__ own) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = (int32_t)i;
    for (int it = 0; it < (1 << 24); ++it) {
      const int32_t p = __ldcg(uf + x);
      if (p == x) break;
      x = p;
    }
    __stcg(uf + i, x);
    atomicAdd(own + x, 1u);
  }
}

__global__ void k_tree_children(int64_t n_r, const int32_t* __restrict__ uf, const int32_t* __restrict__ L,
                                uint32_t* __restrict__ nch) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    if (__ldcg(uf + i) == (int32_t)i && L[i] >= 0) atomicAdd(nch + __ldcg(uf + L[i]), 1u);
  }
}

__global__ void k_tree_flags(int64_t n_r, const int32_t* __restrict__ uf, const uint32_t* __restrict__ own,
                             const uint32_t* __restrict__ nch, uint32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (uf[i] == (int32_t)i && !(own[i] == 1u && nch[i] == 0u)) ? 1u : 0u;
}

__global__ void k_tree_write(int64_t n_r, const int32_t* __restrict__ uf, const int32_t* __restrict__ L,
                             const uint32_t* __restrict__ core, const uint32_t* __restrict__ flag,
                             const int64_t* __restrict__ nid, int32_t* __restrict__ parent,
                             uint32_t* __restrict__ label) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t C = uf[i];
    const int32_t up = (L[C] >= 0) ? (int32_t)nid[uf[L[C]]] : -1;
    parent[i] = flag[C] ? (int32_t)nid[C] : up;
    if (C == (int32_t)i && flag[i]) {
      const int64_t j = nid[i];
      label[j] = core[i];
      parent[n_r + j] = up;
    }
  }
}

}  // namespace

extern "C" int nh_construct_tree(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L, int32_t* parent,
                                 uint32_t* label, int64_t* n_nodes, void* stream) {
  if (n_r < 0 || (n_r > 0 && (!core || !uf || !L || !parent || !label)) || n_r >= (1ll << 31)) return NH_ERR_INVALID;
  if (n_r == 0) {
    if (n_nodes) *n_nodes = 0;
    return NH_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *own = nullptr, *nch = nullptr, *flag = nullptr;
  int64_t* nid = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&own, n_r, st)) || (rc = nh_alloc(&nch, n_r, st)) || (rc = nh_alloc(&flag, n_r, st)) ||
      (rc = nh_alloc(&nid, n_r + 1, st))) {
    nh_free(own, st); nh_free(nch, st); nh_free(flag, st); nh_free(nid, st);
    return rc;
  }
  const unsigned blocks = nh_blocks_for(n_r, 256, 152 * 32);
  cudaMemsetAsync(own, 0, sizeof(uint32_t) * n_r, st);
  cudaMemsetAsync(nch, 0, sizeof(uint32_t) * n_r, st);
  k_tree_roots<<<blocks, 256, 0, st>>>(n_r, uf, own);
  nh_note_launch();
  k_tree_children<<<blocks, 256, 0, st>>>(n_r, uf, L, nch);
  nh_note_launch();
  k_tree_flags<<<blocks, 256, 0, st>>>(n_r, uf, own, nch, flag);
  nh_note_launch();
  rc = nh_exclusive_scan_u32(flag, nid, n_r, st);
  int64_t nn = 0;
  if (!rc) {
    k_tree_write<<<blocks, 256, 0, st>>>(n_r, uf, L, core, flag, nid, parent, label);
    nh_note_launch();
    cudaMemcpyAsync(&nn, nid + n_r, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  }
  if (cudaGetLastError() != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  nh_free(own, st); nh_free(nch, st); nh_free(flag, st); nh_free(nid, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  if (!rc && n_nodes) *n_nodes = nn;
  return rc;
}
