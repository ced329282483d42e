// nh_util.cu -- device-wide exclusive prefix sum (reduce, scan block sums, scan tiles).
#include "nh_internal.cuh"

namespace {

constexpr int kScanThreads = kNhScanThreads;
constexpr int kScanItems = kNhScanItems;
constexpr int kScanTile = kNhScanTile;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t o = __shfl_up_sync(NH_FULL, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// exclusive scan of one value per thread across the block; returns the block total in *total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  constexpr int kWarps = kScanThreads / 32;
  __shared__ int64_t warp_tot[kWarps];
  __shared__ int64_t s_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t w = (lane < kWarps) ? warp_tot[lane] : 0;
    int64_t wi = warp_incl_scan(w);
    if (lane < kWarps) warp_tot[lane] = wi - w;
    if (lane == kWarps - 1) s_total = wi;
  }
  __syncthreads();
  int64_t res = warp_tot[wid] + inc - v;
  *total = s_total;
  __syncthreads();
  return res;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, int64_t* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t j = base + i;
    if (j < n) s += (int64_t)in[j];
  }
  int64_t total;
  (void)block_excl_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// one block: exclusive scan of nb block sums in place; writes the grand total to *total_out
__global__ void k_scan_bsums(int64_t* bsum, int64_t nb, int64_t* total_out) {
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t j = base + threadIdx.x;
    int64_t v = (j < nb) ? bsum[j] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan(v, &tot);
    if (j < nb) bsum[j] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <typename T>
__global__ void k_scan_final(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ bsum,
                             int64_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t j = base + i;
    v[i] = (j < n) ? (int64_t)in[j] : 0;
    s += v[i];
  }
  int64_t tot;
  int64_t ex = block_excl_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t j = base + i;
    if (j < n) out[j] = ex;
    ex += v[i];
  }
}

template <typename T>
int scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t st) {
  if (n < 0 || !out) return NH_ERR_INVALID;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    NH_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return NH_OK;
  }
  int64_t* bsum = nullptr;
  int rc = nh_alloc(&bsum, nb, st);
  if (rc) return rc;
  k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum);
  nh_note_launch();
  k_scan_bsums<<<1, kScanThreads, 0, st>>>(bsum, nb, out + n);
  nh_note_launch();
  k_scan_final<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum, out);
  nh_note_launch();
  cudaError_t e = cudaGetLastError();
  nh_free(bsum, st);
  return e == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

}  // namespace

int nh_exclusive_scan_u32(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t st) {
  return scan_impl<uint32_t>(in, out, n, st);
}
int nh_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
  return scan_impl<int64_t>(in, out, n, st);
}

int nh_scan_u32_blocks(int64_t n) { return (int)((n + kScanTile - 1) / kScanTile); }

// the same scan with caller-provided block-sum storage (nh_scan_u32_blocks(n) entries); no allocation
int nh_exclusive_scan_u32_into(const uint32_t* in, int64_t* out, int64_t n, int64_t* bsum, cudaStream_t st) {
  if (n < 0 || !out || !bsum) return NH_ERR_INVALID;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), st) == cudaSuccess ? NH_OK : NH_ERR_CUDA;
  k_scan_reduce<uint32_t><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum);
  k_scan_bsums<<<1, kScanThreads, 0, st>>>(bsum, nb, out + n);
  k_scan_final<uint32_t><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum, out);
  nh_note_launch(3);
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}
