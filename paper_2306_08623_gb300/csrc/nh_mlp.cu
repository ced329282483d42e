// nh_mlp.cu -- the learned work estimator and the cost-driven schedule of the s-clique
// listing work.  A small MLP (8 features -> 64 -> 64 -> 1, ReLU; BF16 weights, FP32
// accumulation) is trained on per-vertex listing costs that the counting kernel measures, and
// predicts cost per vertex; the out-edge work items are then ordered by decreasing predicted cost
// (log2 buckets) and handed out to warps in chunks from a shared counter, largest first.
// Counting results do not depend on the schedule; the degree cost d+(v)^(s-1) is the baseline.
#include <cuda_bf16.h>

#include <cmath>

#include "nh_internal.cuh"

namespace {

constexpr int F = NH_MLP_FEATURES;
constexpr int H = NH_MLP_HIDDEN;
// parameter layout (flat): W1[H][F], b1[H], W2[H][H], b2[H], W3[H], b3
constexpr int OW1 = 0, OB1 = OW1 + H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
static_assert(OB3 + 1 == NH_MLP_PARAMS, "parameter count");

// ---------------------------------------------------------------------------------------------
// features and costs
// ---------------------------------------------------------------------------------------------

// per vertex v: log1p of deg, out-degree, sum of out-neighbours' out-degrees, sum of neighbours'
// degrees, largest out-neighbour out-degree, sum over out-neighbours of min(out-degrees), the
// squared log out-degree / 8, and a constant 1
__global__ void k_features(GView g, float* __restrict__ feats) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps) {
    const int64_t ob = g.ooff[v], oe = g.ooff[v + 1], dout = oe - ob;
    const int64_t b = g.off[v], e = g.off[v + 1];
    double s2 = 0.0, sdeg = 0.0, smin = 0.0, mx = 0.0;
    for (int64_t j = ob + lane; j < oe; j += 32) {
      const int32_t a = g.oadj[j];
      const double da = (double)(g.ooff[a + 1] - g.ooff[a]);
      s2 += da;
      smin += fmin(da, (double)dout);
      mx = fmax(mx, da);
    }
    for (int64_t j = b + lane; j < e; j += 32) {
      const int32_t u = g.adj[j];
      sdeg += (double)(g.off[u + 1] - g.off[u]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      s2 += __shfl_xor_sync(NH_FULL, s2, d);
      sdeg += __shfl_xor_sync(NH_FULL, sdeg, d);
      smin += __shfl_xor_sync(NH_FULL, smin, d);
      mx = fmax(mx, __shfl_xor_sync(NH_FULL, mx, d));
    }
    if (lane == 0) {
      const float lo = log1pf((float)dout);
      float* f = feats + v * F;
      f[0] = log1pf((float)(e - b));
      f[1] = lo;
      f[2] = (float)log1p(s2);
      f[3] = (float)log1p(sdeg);
      f[4] = (float)log1p(mx);
      f[5] = (float)log1p(smin);
      f[6] = lo * lo * 0.125f;
      f[7] = 1.0f;
    }
  }
}

__global__ void k_degree_cost(GView g, int s, float* __restrict__ cost) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const float d = (float)(g.ooff[v + 1] - g.ooff[v]);
    cost[v] = powf(d, (float)(s - 1));
  }
}

// per out-edge item: its source vertex's cost spread evenly over the vertex's out-edges; the item's
// bucket is 31 - floor(log2(cost + 1)), so bucket 0 holds the heaviest items
// per item: its cost bucket (31 - floor(log2(cost per out-entry + 1))); per-bucket counts are
// summed in shared memory and added once per block
__global__ void k_item_bucket(GView g, const float* __restrict__ vcost, uint8_t* __restrict__ bucket,
                              uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[32];
  if (threadIdx.x < 32) sh[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.m; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = g.osrc[p];
    const float d = (float)(g.ooff[v + 1] - g.ooff[v]);
    const float c = fmaxf(vcost[v], 0.0f) / fmaxf(d, 1.0f);
    const int lg = (int)fminf(floorf(log2f(c + 1.0f)), 31.0f);
    const uint8_t bk = (uint8_t)(31 - lg);
    bucket[p] = bk;
    atomicAdd(sh + bk, 1u);
  }
  __syncthreads();
  if (threadIdx.x < 32 && sh[threadIdx.x]) atomicAdd(hist + threadIdx.x, sh[threadIdx.x]);
}

// items in bucket order: every block takes one contiguous range of items, counts it per bucket
// in shared memory, reserves each bucket's share with one atomic per bucket and writes its items
// there (the order inside a bucket does not matter)
__global__ void k_item_scatter(int64_t m, const uint8_t* __restrict__ bucket, const int64_t* __restrict__ off,
                               unsigned long long* __restrict__ cursor, int32_t* __restrict__ order) {
  __shared__ uint32_t cnt[32];
  __shared__ unsigned long long base[32];
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per;
  const int64_t b1 = b0 + per < m ? b0 + per : m;
  if (threadIdx.x < 32) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) atomicAdd(cnt + bucket[p], 1u);
  __syncthreads();
  if (threadIdx.x < 32) {
    base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(cursor + threadIdx.x, (unsigned long long)cnt[threadIdx.x]) : 0ull;
    cnt[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int64_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) {
    const uint8_t bk = bucket[p];
    order[off[bk] + (int64_t)(base[bk] + atomicAdd(cnt + bk, 1u))] = (int32_t)p;
  }
}

// ---------------------------------------------------------------------------------------------
// MLP: forward with BF16 weights (FP32 accumulation), full-batch Adam on an FP32 master copy
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// one thread per training sample: activations h1, h2 and the output's loss gradient
__global__ void k_mlp_forward_train(const float* __restrict__ X, const float* __restrict__ T,
                                    const int64_t* __restrict__ idx, int64_t n, const __nv_bfloat16* __restrict__ W,
                                    float* __restrict__ h1, float* __restrict__ h2, float* __restrict__ dy,
                                    float* __restrict__ loss) {
  __shared__ float sW[NH_MLP_PARAMS];
  for (int i = threadIdx.x; i < NH_MLP_PARAMS; i += blockDim.x) sW[i] = bf(W, i);
  __syncthreads();
  float lsum = 0.0f;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float* x = X + idx[k] * F;
    float xin[F];
#pragma unroll
    for (int f = 0; f < F; f++) xin[f] = x[f];
    float a1[H];
#pragma unroll 4
    for (int j = 0; j < H; j++) {
      float acc = sW[OB1 + j];
#pragma unroll
      for (int f = 0; f < F; f++) acc = fmaf(sW[OW1 + j * F + f], xin[f], acc);
      a1[j] = fmaxf(acc, 0.0f);
      h1[k * H + j] = a1[j];
    }
    float y = sW[OB3];
    for (int j = 0; j < H; j++) {
      float acc = sW[OB2 + j];
#pragma unroll 8
      for (int i = 0; i < H; i++) acc = fmaf(sW[OW2 + j * H + i], a1[i], acc);
      acc = fmaxf(acc, 0.0f);
      h2[k * H + j] = acc;
      y = fmaf(sW[OW3 + j], acc, y);
    }
    const float err = y - T[idx[k]];
    dy[k] = 2.0f * err / (float)n;
    lsum += err * err;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) lsum += __shfl_xor_sync(NH_FULL, lsum, d);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum / (float)n);
}

// one thread per sample: back-propagated deltas of layer 2 and layer 1
__global__ void k_mlp_backward_delta(int64_t n, const __nv_bfloat16* __restrict__ W, const float* __restrict__ h1,
                                     const float* __restrict__ h2, const float* __restrict__ dy,
                                     float* __restrict__ d2, float* __restrict__ d1) {
  __shared__ float sW[NH_MLP_PARAMS];
  for (int i = threadIdx.x; i < NH_MLP_PARAMS; i += blockDim.x) sW[i] = bf(W, i);
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    float dd2[H];
#pragma unroll 8
    for (int j = 0; j < H; j++) {
      dd2[j] = (h2[k * H + j] > 0.0f) ? dy[k] * sW[OW3 + j] : 0.0f;
      d2[k * H + j] = dd2[j];
    }
    for (int i = 0; i < H; i++) {
      float acc = 0.0f;
#pragma unroll 8
      for (int j = 0; j < H; j++) acc = fmaf(sW[OW2 + j * H + i], dd2[j], acc);
      d1[k * H + i] = (h1[k * H + i] > 0.0f) ? acc : 0.0f;
    }
  }
}

// parameter gradients: one block per output row, summing over a slice of the samples
// grad[row][col] += sum_k A[k][row] * B[k][col]  (B == null means B = 1, i.e. a bias)
__global__ void k_mlp_outer(int64_t n, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                            int cols, const int64_t* __restrict__ idx, float* __restrict__ grad) {
  const int row = blockIdx.x;
  const int64_t chunk = (n + gridDim.y - 1) / gridDim.y;
  const int64_t k0 = blockIdx.y * chunk, k1 = min(n, k0 + chunk);
  for (int col = threadIdx.x; col < cols; col += blockDim.x) {
    float acc = 0.0f;
    for (int64_t k = k0; k < k1; k++) {
      const float a = A[k * lda + row];
      const float b = B ? B[(idx ? idx[k] : k) * ldb + col] : 1.0f;
      acc = fmaf(a, b, acc);
    }
    atomicAdd(&grad[row * cols + col], acc);
  }
}

__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ m1, float* __restrict__ m2,
                           const float* __restrict__ grad, __nv_bfloat16* __restrict__ W, float lr, int step) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH_MLP_PARAMS; i += gridDim.x * blockDim.x) {
    const float gr = grad[i];
    m1[i] = b1 * m1[i] + (1.0f - b1) * gr;
    m2[i] = b2 * m2[i] + (1.0f - b2) * gr * gr;
    master[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
    W[i] = __float2bfloat16(master[i]);
  }
}

// Kaiming-style initialisation from a counter-based hash (SplitMix64 of seed and index)
__global__ void k_mlp_init(float* __restrict__ master, __nv_bfloat16* __restrict__ W, unsigned long long seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH_MLP_PARAMS; i += gridDim.x * blockDim.x) {
    const unsigned long long h = nh_mix64(seed * 0x9e3779b97f4a7c15ull + (unsigned long long)i);
    const float u = ((float)(h >> 40) / (float)(1ull << 24)) * 2.0f - 1.0f;  // uniform [-1, 1)
    float v = 0.0f;
    if (i < OB1) v = u * sqrtf(6.0f / F);
    else if (i >= OW2 && i < OB2) v = u * sqrtf(6.0f / H);
    else if (i >= OW3 && i < OB3) v = u * sqrtf(3.0f / H);
    master[i] = v;
    W[i] = __float2bfloat16(v);
  }
}

__global__ void k_sample_idx(int64_t n_all, int64_t n, unsigned long long seed, int64_t* __restrict__ idx) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    idx[k] = (int64_t)(nh_mix64(seed ^ (0x632be59bd9b4e019ull * (unsigned long long)(k + 1))) % (unsigned long long)n_all);
}

__global__ void k_log_target(int64_t n, const float* __restrict__ cost, float* __restrict__ t) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    t[v] = log1pf(fmaxf(cost[v], 0.0f));
}

// inference: one thread per vertex, predicted cost = expm1(output)
__global__ void k_mlp_predict(const float* __restrict__ X, int64_t n, const __nv_bfloat16* __restrict__ W,
                              float* __restrict__ out) {
  __shared__ float sW[NH_MLP_PARAMS];
  for (int i = threadIdx.x; i < NH_MLP_PARAMS; i += blockDim.x) sW[i] = bf(W, i);
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    float xin[F];
#pragma unroll
    for (int f = 0; f < F; f++) xin[f] = X[v * F + f];
    float a1[H];
#pragma unroll 4
    for (int j = 0; j < H; j++) {
      float acc = sW[OB1 + j];
#pragma unroll
      for (int f = 0; f < F; f++) acc = fmaf(sW[OW1 + j * F + f], xin[f], acc);
      a1[j] = fmaxf(acc, 0.0f);
    }
    float y = sW[OB3];
    for (int j = 0; j < H; j++) {
      float acc = sW[OB2 + j];
#pragma unroll 8
      for (int i = 0; i < H; i++) acc = fmaf(sW[OW2 + j * H + i], a1[i], acc);
      y = fmaf(sW[OW3 + j], fmaxf(acc, 0.0f), y);
    }
    out[v] = expm1f(fminf(fmaxf(y, 0.0f), 30.0f));
  }
}

}  // namespace

// items in decreasing estimated cost, for largest-first dynamic scheduling
int nh_schedule_items(const nh_oriented* o, const float* vertex_cost, int32_t** order_out,
                      unsigned long long** next_out, cudaStream_t st) {
  *order_out = nullptr;
  *next_out = nullptr;
  GView g = make_view(o, nullptr);
  uint8_t* bucket = nullptr;
  uint32_t* hist = nullptr;
  int64_t* off = nullptr;
  unsigned long long* cursor = nullptr;
  int32_t* order = nullptr;
  unsigned long long* next = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&bucket, o->m, st)) || (rc = nh_alloc(&hist, 32, st)) || (rc = nh_alloc(&off, 33, st)) ||
      (rc = nh_alloc(&cursor, 32, st)) || (rc = nh_alloc(&order, o->m, st)) || (rc = nh_alloc(&next, 1, st))) {
    nh_free(bucket, st); nh_free(hist, st); nh_free(off, st); nh_free(cursor, st); nh_free(order, st); nh_free(next, st);
    return rc;
  }
  cudaMemsetAsync(hist, 0, 32 * sizeof(uint32_t), st);
  cudaMemsetAsync(cursor, 0, 32 * sizeof(unsigned long long), st);
  cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
  k_item_bucket<<<nh_blocks_for(o->m, 256, 152 * 32), 256, 0, st>>>(g, vertex_cost, bucket, hist);
  nh_note_launch();
  rc = nh_exclusive_scan_u32(hist, off, 32, st);
  if (!rc) {
    k_item_scatter<<<nh_blocks_for(o->m, 256, 152 * 32), 256, 0, st>>>(o->m, bucket, off, cursor, order);
    nh_note_launch();
  }
  nh_free(bucket, st); nh_free(hist, st); nh_free(off, st); nh_free(cursor, st);
  if (rc) {
    nh_free(order, st); nh_free(next, st);
    return rc;
  }
  *order_out = order;
  *next_out = next;
  return NH_OK;
}

extern "C" int nh_vertex_features(const nh_oriented* o, float* feats, void* stream) {
  if (!o || !feats) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  k_features<<<nh_blocks_for(o->n * 32, 256, 152 * 32), 256, 0, st>>>(make_view(o, nullptr), feats);
  nh_note_launch();
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

extern "C" int nh_listing_cost(const nh_oriented* o, const nh_rindex* ri, int s, float* cost, void* stream) {
  if (!o || !ri || !cost) return NH_ERR_INVALID;
  if (ri->r == 1 && s == 2) return NH_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* cnt = nullptr;
  int rc = nh_alloc(&cnt, ri->n_r, st);
  if (rc) return rc;
  rc = nh_count_impl(o, ri, s, cnt, nullptr, nullptr, cost, st);
  nh_free(cnt, st);
  return rc;
}

extern "C" int nh_degree_cost(const nh_oriented* o, int s, float* cost, void* stream) {
  if (!o || !cost || s < 2) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  k_degree_cost<<<nh_blocks_for(o->n, 256, 152 * 32), 256, 0, st>>>(make_view(o, nullptr), s, cost);
  nh_note_launch();
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

extern "C" int nh_mlp_train(const float* feats, const float* cost, int64_t n, int64_t n_train, int steps, float lr,
                            uint64_t seed, uint16_t* weights, float* final_loss, void* stream) {
  if (!feats || !cost || !weights || n < 1 || n_train < 1 || steps < 1 || !(lr > 0.0f)) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(weights);
  float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr, *target = nullptr, *h1 = nullptr,
        *h2 = nullptr, *d1 = nullptr, *d2 = nullptr, *dy = nullptr, *loss = nullptr;
  int64_t* idx = nullptr;
  int rc = NH_OK;
  if ((rc = nh_alloc(&master, NH_MLP_PARAMS, st)) || (rc = nh_alloc(&m1, NH_MLP_PARAMS, st)) ||
      (rc = nh_alloc(&m2, NH_MLP_PARAMS, st)) || (rc = nh_alloc(&grad, NH_MLP_PARAMS, st)) ||
      (rc = nh_alloc(&target, n, st)) || (rc = nh_alloc(&h1, n_train * H, st)) || (rc = nh_alloc(&h2, n_train * H, st)) ||
      (rc = nh_alloc(&d1, n_train * H, st)) || (rc = nh_alloc(&d2, n_train * H, st)) || (rc = nh_alloc(&dy, n_train, st)) ||
      (rc = nh_alloc(&loss, 1, st)) || (rc = nh_alloc(&idx, n_train, st))) {
    goto done;
  }
  cudaMemsetAsync(m1, 0, sizeof(float) * NH_MLP_PARAMS, st);
  cudaMemsetAsync(m2, 0, sizeof(float) * NH_MLP_PARAMS, st);
  k_mlp_init<<<(NH_MLP_PARAMS + 255) / 256, 256, 0, st>>>(master, W, seed);
  k_sample_idx<<<nh_blocks_for(n_train, 256, 152 * 8), 256, 0, st>>>(n, n_train, seed, idx);
  k_log_target<<<nh_blocks_for(n, 256, 152 * 32), 256, 0, st>>>(n, cost, target);
  nh_note_launch(3);
  {
    const unsigned fb = nh_blocks_for(n_train, 128, 152 * 4);
    const dim3 go(H, 32), gb(H, 32);
    for (int step = 1; step <= steps; step++) {
      cudaMemsetAsync(grad, 0, sizeof(float) * NH_MLP_PARAMS, st);
      cudaMemsetAsync(loss, 0, sizeof(float), st);
      k_mlp_forward_train<<<fb, 128, 0, st>>>(feats, target, idx, n_train, W, h1, h2, dy, loss);
      k_mlp_backward_delta<<<fb, 128, 0, st>>>(n_train, W, h1, h2, dy, d2, d1);
      // dW3[j] = sum dy h2[j]; db3 = sum dy
      k_mlp_outer<<<dim3(1, 32), 64, 0, st>>>(n_train, dy, 1, h2, H, H, nullptr, grad + OW3);
      k_mlp_outer<<<dim3(1, 32), 32, 0, st>>>(n_train, dy, 1, nullptr, 0, 1, nullptr, grad + OB3);
      // dW2[j][i] = sum d2[j] h1[i]; db2 = sum d2
      k_mlp_outer<<<go, 64, 0, st>>>(n_train, d2, H, h1, H, H, nullptr, grad + OW2);
      k_mlp_outer<<<gb, 32, 0, st>>>(n_train, d2, H, nullptr, 0, 1, nullptr, grad + OB2);
      // dW1[i][f] = sum d1[i] x[f]; db1 = sum d1
      k_mlp_outer<<<go, 32, 0, st>>>(n_train, d1, H, feats, F, F, idx, grad + OW1);
      k_mlp_outer<<<gb, 32, 0, st>>>(n_train, d1, H, nullptr, 0, 1, nullptr, grad + OB1);
      k_mlp_adam<<<(NH_MLP_PARAMS + 255) / 256, 256, 0, st>>>(master, m1, m2, grad, W, lr, step);
      nh_note_launch(9);
    }
  }
  if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
  if (!rc && final_loss) {
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    k_mlp_forward_train<<<nh_blocks_for(n_train, 128, 152 * 4), 128, 0, st>>>(feats, target, idx, n_train, W, h1, h2,
                                                                              dy, loss);
    nh_note_launch();
    cudaMemcpyAsync(final_loss, loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  }
done:
  nh_free(master, st); nh_free(m1, st); nh_free(m2, st); nh_free(grad, st); nh_free(target, st);
  nh_free(h1, st); nh_free(h2, st); nh_free(d1, st); nh_free(d2, st); nh_free(dy, st); nh_free(loss, st);
  nh_free(idx, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

extern "C" int nh_mlp_predict(const float* feats, int64_t n, const uint16_t* weights, float* pred, void* stream) {
  if (!feats || !weights || !pred || n < 0) return NH_ERR_INVALID;
  if (n == 0) return NH_OK;
  cudaStream_t st = (cudaStream_t)stream;
  k_mlp_predict<<<nh_blocks_for(n, 128, 152 * 16), 128, 0, st>>>(feats, n, reinterpret_cast<const __nv_bfloat16*>(weights),
                                                                 pred);
  nh_note_launch();
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

extern "C" int nh_count_s_cliques_partitioned(const nh_oriented* o, const nh_rindex* ri, int s,
                                              const float* vertex_cost, uint32_t* cnt, uint64_t* n_s, void* stream) {
  if (!o || !ri || !vertex_cost) return NH_ERR_INVALID;
  return nh_count_impl(o, ri, s, cnt, n_s, vertex_cost, nullptr, (cudaStream_t)stream);
}
