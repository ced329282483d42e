// nh_tree.cu -- a9: construct-tree-efficient (Alg. 5).  One node per union-find component; the
// parent of node C is the node of find(L[C]); a node whose subtree holds one r-clique (one
// member, no child node) is dropped and that r-clique hangs from the dropped node's parent.
#include <mutex>

#include "nh_internal.cuh"

namespace {

// full path compression: uf[i] = root of i (parents only ever point to ancestors).  A path in a
// forest of n_r entries has fewer than n_r steps; a walk that takes n_r steps has met a cycle (a
// corrupt uf), records NH_ERR_INVALID in *status (first error wins) and leaves uf[i] as it was.
__global__ void k_tree_roots(int64_t n_r, int32_t* __restrict__ uf, uint32_t* __restrict__ own,
                             int64_t* __restrict__ status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = (int32_t)i;
    int64_t it = 0;
    for (; it < n_r; ++it) {
      const int32_t p = __ldcg(uf + x);
      if (p == x) break;
      x = p;
    }
    if (it == n_r) {
      atomicCAS(reinterpret_cast<unsigned long long*>(status), 0ull, (unsigned long long)(int64_t)NH_ERR_INVALID);
      continue;
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

// Stream-ordered construct-tree: launches only; the node count lands in the device word
// n_nodes_dev.  n_r >= 1, arguments checked by the caller.
int nh_tree_enqueue(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L, int32_t* parent,
                    uint32_t* label, int64_t* n_nodes_dev, int64_t* status_dev, cudaStream_t st) {
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
  k_tree_roots<<<blocks, 256, 0, st>>>(n_r, uf, own, status_dev);
  nh_note_launch();
  k_tree_children<<<blocks, 256, 0, st>>>(n_r, uf, L, nch);
  nh_note_launch();
  k_tree_flags<<<blocks, 256, 0, st>>>(n_r, uf, own, nch, flag);
  nh_note_launch();
  rc = nh_exclusive_scan_u32(flag, nid, n_r, st);
  if (!rc) {
    k_tree_write<<<blocks, 256, 0, st>>>(n_r, uf, L, core, flag, nid, parent, label);
    nh_note_launch();
    cudaMemcpyAsync(n_nodes_dev, nid + n_r, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  }
  if (cudaGetLastError() != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  nh_free(own, st); nh_free(nch, st); nh_free(flag, st); nh_free(nid, st);
  return rc;
}

extern "C" int nh_construct_tree(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L, int32_t* parent,
                                 uint32_t* label, int64_t* n_nodes, void* stream) {
  if (n_r < 0 || (n_r > 0 && (!core || !uf || !L || !parent || !label)) || n_r >= (1ll << 31)) return NH_ERR_INVALID;
  if (n_r == 0) {
    if (n_nodes) *n_nodes = 0;
    return NH_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int64_t* nn_dev = nullptr;  // {n_nodes, status}
  int rc = nh_alloc(&nn_dev, 2, st);
  if (rc) return rc;
  cudaMemsetAsync(nn_dev, 0, 2 * sizeof(int64_t), st);
  rc = nh_tree_enqueue(n_r, core, uf, L, parent, label, nn_dev, nn_dev + 1, st);
  int64_t nn[2] = {0, 0};
  if (!rc) cudaMemcpyAsync(nn, nn_dev, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  nh_free(nn_dev, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  if (!rc && nn[1]) rc = (int)nn[1];
  if (!rc && n_nodes) *n_nodes = nn[0];
  return rc;
}

// ---------------------------------------------------------------------------------------------
// nh_construct_tree_noalloc: the same tree construction with its working memory in a fixed
// device array instead of stream-ordered allocations.
//
// Working memory for up to NH_TREE_NOALLOC_MAX r-cliques: three uint32 counters/flags per
// r-clique, one int64 node id per r-clique (+1), and the scan's block sums.  The array lives in
// every device that loads this library, for the life of the process (about 5.3 MB).  Host code
// cannot use the array's name as a device address, so the address is looked up once per device
// with cudaGetSymbolAddress (on that device) and kept.
// ---------------------------------------------------------------------------------------------

namespace {

constexpr int64_t kNoAllocMax = NH_TREE_NOALLOC_MAX;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOwnOff = 0;
constexpr size_t kNchOff = kOwnOff + align_up(sizeof(uint32_t) * kNoAllocMax);
constexpr size_t kFlagOff = kNchOff + align_up(sizeof(uint32_t) * kNoAllocMax);
constexpr size_t kNidOff = kFlagOff + align_up(sizeof(uint32_t) * kNoAllocMax);
constexpr int64_t kBsumSlots = (kNoAllocMax + kNhScanTile - 1) / kNhScanTile;  // scan block sums
constexpr size_t kBsumOff = kNidOff + align_up(sizeof(int64_t) * (kNoAllocMax + 1));
constexpr size_t kStatusOff = kBsumOff + align_up(sizeof(int64_t) * kBsumSlots);
constexpr size_t kScratchBytes = kStatusOff + align_up(sizeof(int64_t));

}  // namespace

static __device__ __align__(256) unsigned char g_tree_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
void* g_tree_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_tree_scratch_mu;

// device address of g_tree_scratch on the current device (looked up on first use per device)
int tree_scratch(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NH_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NH_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_tree_scratch_mu);
  if (!g_tree_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tree_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return NH_ERR_CUDA;
    }
    g_tree_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_tree_scratch_addr[dev]);
  return NH_OK;
}

}  // namespace

extern "C" int nh_construct_tree_noalloc(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L,
                                         int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream) {
  if (n_r < 0 || n_r > kNoAllocMax) return NH_ERR_INVALID;
  if (n_r > 0 && (!core || !uf || !L || !parent || !label)) return NH_ERR_INVALID;
  if (n_r == 0) {
    if (n_nodes) *n_nodes = 0;
    return NH_OK;
  }
  unsigned char* base = nullptr;
  int rc = tree_scratch(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* own = reinterpret_cast<uint32_t*>(base + kOwnOff);
  uint32_t* nch = reinterpret_cast<uint32_t*>(base + kNchOff);
  uint32_t* flag = reinterpret_cast<uint32_t*>(base + kFlagOff);
  int64_t* nid = reinterpret_cast<int64_t*>(base + kNidOff);
  int64_t* bsum = reinterpret_cast<int64_t*>(base + kBsumOff);
  int64_t* status = reinterpret_cast<int64_t*>(base + kStatusOff);
  if (nh_scan_u32_blocks(n_r) > kBsumSlots) return NH_ERR_INTERNAL;
  // the array keeps the previous call's contents: the counters and the status must start at zero
  if (cudaMemsetAsync(own, 0, sizeof(uint32_t) * n_r, st) != cudaSuccess ||
      cudaMemsetAsync(nch, 0, sizeof(uint32_t) * n_r, st) != cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(int64_t), st) != cudaSuccess)
    return NH_ERR_CUDA;
  const unsigned blocks = nh_blocks_for(n_r, 256, 152 * 32);
  k_tree_roots<<<blocks, 256, 0, st>>>(n_r, uf, own, status);
  k_tree_children<<<blocks, 256, 0, st>>>(n_r, uf, L, nch);
  k_tree_flags<<<blocks, 256, 0, st>>>(n_r, uf, own, nch, flag);
  nh_note_launch(3);
  rc = nh_exclusive_scan_u32_into(flag, nid, n_r, bsum, st);
  int64_t nn = 0, bad = 0;
  if (!rc) {
    k_tree_write<<<blocks, 256, 0, st>>>(n_r, uf, L, core, flag, nid, parent, label);
    nh_note_launch();
    if (cudaMemcpyAsync(&nn, nid + n_r, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&bad, status, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = NH_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  if (!rc && bad) rc = (int)bad;
  if (!rc && n_nodes) *n_nodes = nn;
  return rc;
}

// ---------------------------------------------------------------------------------------------
// nh_cut_hierarchy: the c-(r,s) nuclei read off a hierarchy (§8, dense subgraphs).  Removing every
// node of level < c leaves a forest whose trees are the c-nuclei; each r-clique maps to the top
// node of the tree that holds its smallest node.  Node-level pointer jumping: up[N] starts at N's
// parent when that parent keeps level >= c (else N itself), and up[N] = up[up[N]] is repeated
// ceil(log2 n_nodes) + 1 times, which reaches the top of any path of at most n_nodes nodes.
// ---------------------------------------------------------------------------------------------

namespace {

__global__ void k_cut_init(int64_t n_r, int64_t n_nodes, const int32_t* __restrict__ parent,
                           const uint32_t* __restrict__ label, uint32_t c, int32_t* __restrict__ up,
                           unsigned long long* __restrict__ n_top) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_nodes; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent[n_r + j];
    const bool keep_up = p >= 0 && p < n_nodes && label[p] >= c;
    up[j] = keep_up ? p : (int32_t)j;
    if (!keep_up && label[j] >= c) atomicAdd(n_top, 1ull);
  }
}

__global__ void k_cut_jump(int64_t n_nodes, const int32_t* __restrict__ up_in, int32_t* __restrict__ up_out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_nodes; j += (int64_t)gridDim.x * blockDim.x)
    up_out[j] = up_in[up_in[j]];
}

__global__ void k_cut_leaves(int64_t n_r, int64_t n_nodes, const int32_t* __restrict__ parent,
                             const uint32_t* __restrict__ label, uint32_t c, const int32_t* __restrict__ up,
                             int32_t* __restrict__ nucleus) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t N = parent[i];
    nucleus[i] = (N >= 0 && N < n_nodes && label[N] >= c) ? up[N] : -1;
  }
}

}  // namespace

extern "C" int nh_cut_hierarchy(int64_t n_r, int64_t n_nodes, const int32_t* parent, const uint32_t* label,
                                uint32_t c, int32_t* nucleus, int64_t* n_nuclei, void* stream) {
  if (n_r < 0 || n_nodes < 0 || n_nodes > n_r || n_r >= (1ll << 31) || (n_r > 0 && (!parent || !nucleus)) ||
      (n_nodes > 0 && !label))
    return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_r == 0) {
    if (n_nuclei) *n_nuclei = 0;
    return NH_OK;
  }
  int32_t *up0 = nullptr, *up1 = nullptr;
  unsigned long long* cnt = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&up0, n_nodes, st)) || (rc = nh_alloc(&up1, n_nodes, st)) || (rc = nh_alloc(&cnt, 1, st))) {
    nh_free(up0, st); nh_free(up1, st); nh_free(cnt, st);
    return rc;
  }
  cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
  const unsigned bn = nh_blocks_for(n_nodes, 256, 152 * 16), br = nh_blocks_for(n_r, 256, 152 * 16);
  if (n_nodes > 0) {
    k_cut_init<<<bn, 256, 0, st>>>(n_r, n_nodes, parent, label, c, up0, cnt);
    nh_note_launch();
    int rounds = 1;
    while ((1ll << (rounds - 1)) < n_nodes) rounds++;
    for (int k = 0; k < rounds; k++) {
      k_cut_jump<<<bn, 256, 0, st>>>(n_nodes, up0, up1);
      nh_note_launch();
      int32_t* t = up0; up0 = up1; up1 = t;
    }
  }
  k_cut_leaves<<<br, 256, 0, st>>>(n_r, n_nodes, parent, label, c, up0, nucleus);
  nh_note_launch();
  unsigned long long h = 0;
  if (n_nuclei) cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
  nh_free(up0, st); nh_free(up1, st); nh_free(cnt, st);
  if (n_nuclei) {
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
    if (!rc) *n_nuclei = (int64_t)h;
  }
  return rc;
}
