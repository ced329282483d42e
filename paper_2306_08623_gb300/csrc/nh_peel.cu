// nh_peel.cu -- the peeling loop of Alg. 3 (exact, interleaved with
// link-efficient of Alg. 5) and of Alg. 2 (approximate), as one persistent cooperative kernel
// per call; plus link-efficient on a batch of calls (nh_link_pairs).
//
// Round t of the loop (all blocks run it in lockstep, separated by a bounded grid barrier whose
// last arriving block updates the shared control block):
//   frontier A  -- either the r-cliques whose count crossed to <= threshold during round t-1
//                  (kept exactly: a decrement that takes a count from thr+1 to thr appends it),
//                  or, when that set is empty (new level) or the approximate bucket changes, a
//                  scan of the compacted live list: threshold = max(k, min count) (exact) or the
//                  first bucket end >= min count (approx), A = live with count <= threshold.
//   re-listing  -- one warp per R in A: candidates are the common neighbours of R's vertices
//                  (the shortest adjacency list is scanned, the others binary-searched), then
//                  (s-r)-cliques among them through the orientation; for each s-clique S the
//                  other members' ids come from the adjacency positions (edge ids) or the
//                  triangle hash table.
//   per (R, S)  -- S is dead if a member was peeled in an earlier round (round stamp in [1,t));
//                  otherwise the member of least id among S n A decrements the live members once
//                  (each s-clique dies exactly once) and links S n A; a dead S links R with an
//                  earlier-peeled member of least core (that member's core is min core over S).
// round[] stamps: 0 = never peeled, t = peeled in round t; an r-clique that crosses during round
// t is stamped t+1 at once, which every reader of round t treats as live.
#include <cmath>
#include <vector>

#include "nh_peel.cuh"

extern long long g_nh_inject_wait_ns;  // fault injection (nh_api.cu): grid-barrier wait limit
extern uint64_t* g_nh_round_log;       // round trace (nh_api.cu)
extern long long g_nh_round_log_cap;
static int g_peel_max_group = 1024;   // set by nh_set_peel_max_group
static int g_peel_task_items = -1;    // set by nh_set_peel_task_items (-1: automatic)
static int g_peel_relist24 = 1;       // set by nh_set_peel_relist24
static int g_peel_list_hash = 0;      // set by nh_set_peel_list_hash (0 off, 1 automatic, 2 always)
static float g_split_per_warp = 1.0f;  // set by nh_set_relist_split
static int g_split_wgrain = 128, g_split_bgrain = 1024, g_split_len_mult = 0;

// Alg. 2's schedule (readings R9, R10): bucket upper ends t_i = floor(x_i) with x_0 = (C+delta)(1+delta)
// and x_{i+1} = x_i (1+delta) in IEEE double, up to the first end >= max_count (at most cap ends);
// the round cap T = ceil(ln(max(n_r, 2)) / log1p(delta / C)) + 1.  Shared by both peels.
int nh_approx_table(int C, double delta, uint32_t max_count, uint32_t* out, int cap) {
  double x = ((double)C + delta) * (1.0 + delta);
  int k = 0;
  while (k < cap) {
    const double f = std::floor(x);
    const uint32_t tv = (f >= 4294967295.0) ? 4294967295u : (uint32_t)f;
    out[k++] = tv;
    if (tv >= max_count) break;
    x = x * (1.0 + delta);
  }
  return k;
}

uint32_t nh_approx_cap(int C, double delta, int64_t n_r) {
  const double nn = (double)(n_r > 2 ? n_r : 2);
  return (uint32_t)std::ceil(std::log(nn) / std::log1p(delta / (double)C)) + 1u;
}

extern "C" int nh_approx_thresholds(int C, double delta, uint32_t max_count, uint32_t* out, int cap, int* n) {
  if (C < 1 || !(delta > 0.0) || !out || cap < 1 || !n) return NH_ERR_INVALID;
  *n = nh_approx_table(C, delta, max_count, out, cap);
  return NH_OK;
}

extern "C" int nh_approx_round_cap(int C, double delta, int64_t n_r, uint32_t* T) {
  if (C < 1 || !(delta > 0.0) || n_r < 0 || !T) return NH_ERR_INVALID;
  *T = nh_approx_cap(C, delta, n_r);
  return NH_OK;
}

namespace nhp {

__global__ void k_peel_init(int64_t n_r, const uint32_t* __restrict__ cnt0, uint32_t* __restrict__ cnt,
                            uint32_t* __restrict__ round, uint32_t* __restrict__ val, int32_t* __restrict__ alive,
                            int32_t* __restrict__ uf, int32_t* __restrict__ L) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    cnt[i] = cnt0[i];
    round[i] = 0;
    val[i] = 0;
    alive[i] = (int32_t)i;
    if (uf) uf[i] = (int32_t)i;
    if (L) L[i] = -1;
  }
}

// (3,4) mirrored lists: entry k of edge e's triangle list = {w, triangle, stamp, value} with
// stamp = value = init (the value array's entry when init is given, else 0), and the list
// position of every triangle's three entries (slot = which of its edges the list belongs to)
__global__ void k_et3_fill(GView g, int4* __restrict__ et3, int32_t* __restrict__ tpos,
                           const uint32_t* __restrict__ init) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < g.m; e += nwarps) {
    for (int64_t k = g.etoff[e] + lane; k < g.etoff[e + 1]; k += 32) {
      const int32_t tid = g.ettid[k];
      const int32_t* te = g.tedge + 3 * (int64_t)tid;
      const int slot = (te[0] == (int32_t)e) ? 0 : (te[1] == (int32_t)e) ? 1 : 2;
      tpos[3 * (int64_t)tid + slot] = (int32_t)k;
      const int32_t v = init ? (int32_t)init[tid] : 0;
      et3[k] = make_int4(g.etw[k], tid, v, v);
    }
  }
}

__global__ void k_peel_result(const PeelCtl* c, int64_t* res) {
  if (res[0] == 0) res[0] = c->err ? c->err : (c->done ? NH_OK : NH_ERR_INTERNAL);
  res[3] = (int64_t)c->st_rounds;
}

__global__ void k_status_into(const int* status, int64_t* res) {
  if (res[0] == 0 && *status) res[0] = *status;
}

__global__ void k_ctl_init(PeelCtl* c, int64_t n_r, unsigned int thr0) {
  c->t = 1;
  c->thr = thr0;
  c->need_scan = 1;
  c->gmin = kNone;
  c->alive_n = (unsigned long long)n_r;
  c->done = (n_r == 0);
}

__global__ void k_max_u32(int64_t n, const uint32_t* __restrict__ a, unsigned int* __restrict__ out) {
  unsigned int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, a[i]);
  m = warp_min_u32(~m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, ~m);
}

// nh_link_pairs: one thread per call
// (3,4): the (edge id, third vertex) -> list position table of the per-edge triangle lists
__global__ void k_eh_fill(GView g, ulonglong2* __restrict__ eh, unsigned long long mask, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < g.m; e += nwarps) {
    for (int64_t k = g.etoff[e] + lane; k < g.etoff[e + 1]; k += 32) {
      const unsigned long long key = ((unsigned long long)(uint32_t)e << 32) | (uint32_t)g.etw[k];
      unsigned long long h = nh_mix64(key) & mask;
      bool done = false;
      for (unsigned long long q = 0; q <= mask && !done; ++q) {
        const unsigned long long old = atomicCAS(&eh[h].x, NH_EMPTY_KEY, key);
        if (old == NH_EMPTY_KEY || old == key) {
          eh[h].y = (unsigned long long)k;
          done = true;
        }
        h = (h + 1) & mask;
      }
      if (!done) atomicCAS(status, 0, NH_ERR_TABLE_FULL);
    }
  }
}

__global__ void k_eh_empty(ulonglong2* eh, unsigned long long cap) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x)
    eh[i] = make_ulonglong2(NH_EMPTY_KEY, 0ull);
}

// Builds A.eh over the 3 n_r list entries when the knob asks for it and the table fits;
// otherwise leaves A.eh null (binary searches).  Automatic (knob 1): only for the peels that
// prune candidates before the lookups (cores only, approximate).  Measured on R-MAT 18 (3,4) with
// the searches over the compact third-vertex array: cores-only peel 1100 ms searching, 1098 ms
// with the table; linking peel 1992 vs 2301 ms; two-phase hierarchy 897 vs 927 ms (the list
// searches stay in cache, the table's slots do not), so the default (knob 0) searches.
// status: device word for a full table.
void build_list_hash(PeelArgs& A, int64_t n_r, bool pruned, int* status, ulonglong2** table, cudaStream_t st) {
  *table = nullptr;
  A.eh = nullptr;
  if (!A.et3 || g_peel_list_hash == 0 || (g_peel_list_hash == 1 && !pruned)) return;
  unsigned long long cap = 1024;
  while (cap < 5ull * (unsigned long long)n_r) cap <<= 1;  // 3 n_r entries at load <= 0.6
  if (nh_alloc(table, (int64_t)cap, st) != NH_OK) {
    (void)cudaGetLastError();
    *table = nullptr;
    return;
  }
  k_eh_empty<<<nh_blocks_for((int64_t)cap, 256, 152 * 32), 256, 0, st>>>(*table, cap);
  k_eh_fill<<<nh_blocks_for(A.g.m * 32, 256, 152 * 16), 256, 0, st>>>(A.g, *table, cap - 1, status);
  nh_note_launch(2);
  A.eh = *table;
  A.eh_mask = cap - 1;
}

__global__ void k_link_pairs(LinkEnv E, const int2* __restrict__ pairs, unsigned long long n) {
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int2 p = pairs[i];
    link_run(E, p.x, p.y, ls);
  }
}

__global__ void k_link_swap(PeelCtl* c, unsigned long long cap) {
  const unsigned int oc = c->ovf_cur;
  c->drain_buf = oc;
  c->drain_n = c->ovf_count[oc] < cap ? c->ovf_count[oc] : cap;
  c->ovf_count[oc] = 0;
  c->ovf_cur = oc ^ 1u;
}

__global__ void k_link_drain(LinkEnv E) {
  LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const unsigned int b = E.ctl->drain_buf;
  const unsigned long long n = E.ctl->drain_n;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int2 p = __ldcg(E.ovf[b] + i);
    link_run(E, p.x, p.y, ls);
  }
}

// one drain step of link-efficient's overflow queue: swap the queues, re-run the deferred calls
int link_drain_round(const LinkEnv& E, cudaStream_t st) {
  k_link_swap<<<1, 1, 0, st>>>(E.ctl, E.ovf_cap);
  k_link_drain<<<152 * 8, 128, 0, st>>>(E);
  nh_note_launch(2);
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

int peel_launch_pair(int r, int s, bool exact, PeelArgs& A, cudaStream_t st) {
  if (r == 1 && s == 2) return peel_launch_12(exact, A, st);
  if (r == 1 && s == 3) return peel_launch_13(exact, A, st);
  if (r == 2 && s == 3) return peel_launch_23(exact, A, st);
  if (r == 2 && s == 4) return peel_launch_24(exact, A, st);
  if (r == 3 && s == 4) return peel_launch_34(exact, A, st);
  return NH_ERR_UNSUPPORTED;
}

int two_phase_launch_pair(int r, int s, PeelArgs& A, TreeOut& T, cudaStream_t st) {
  if (r == 1 && s == 2) return two_phase_launch_12(A, T, st);
  if (r == 1 && s == 3) return two_phase_launch_13(A, T, st);
  if (r == 2 && s == 3) return two_phase_launch_23(A, T, st);
  if (r == 2 && s == 4) return two_phase_launch_24(A, T, st);
  if (r == 3 && s == 4) return two_phase_launch_34(A, T, st);
  return NH_ERR_UNSUPPORTED;
}

// chunk counts of the re-listed lists (they depend on r, and for r = 3 on s)
int chunk_cost_pair(int r, int s, const GView& g, int64_t n_r, uint32_t* cost, cudaStream_t st) {
  if (r == 1) return chunk_cost_12(g, n_r, cost, st);
  if (r == 2 && s == 3) return chunk_cost_23(g, n_r, cost, st);
  if (r == 2 && s == 4) return chunk_cost_24(g, n_r, cost, st);
  if (r == 3 && s == 4) return chunk_cost_34(g, n_r, cost, st);
  return NH_ERR_UNSUPPORTED;
}

// shared driver for the exact and the approximate peel
// res_dev == nullptr: synchronous (status returned, stats read back).  Otherwise exact only and
// stream ordered: nothing is read back; the status goes to res_dev[0] (unless it already holds
// one) and the round count to res_dev[3].
int run_peel(bool exact, const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* cnt, uint32_t* val,
             uint32_t* round, int32_t* uf, int32_t* L, int link_mode, double delta, nh_peel_stats* stats,
             int64_t* res_dev, cudaStream_t st) {
  if (res_dev && !exact) return NH_ERR_INVALID;
  if (!o || !ri || ri->o != o) return NH_ERR_INVALID;
  const int r = ri->r;
  if (nh_generic_pair(r, s)) {
    // other pairs: Alg. 3 / Alg. 2 rounds with one host round trip each (not stream-ordered)
    if (res_dev) return NH_ERR_UNSUPPORTED;
    if (ri->n_r > 0 && (!cnt || !val || !round)) return NH_ERR_INVALID;
    if (exact && (link_mode < 0 || link_mode > 2 || (link_mode < 2 && ri->n_r > 0 && (!uf || !L))))
      return NH_ERR_INVALID;
    if (!exact && !(delta > 0.0)) return NH_ERR_INVALID;
    return nh_peel_generic(exact, o, ri, s, cnt, val, round, uf, L, exact ? link_mode : -1, delta, stats, st);
  }
  if (stats) *stats = nh_peel_stats{};
  if (ri->n_r == 0 && nh_supported(r, s)) return NH_OK;  // arrays may be empty (null)
  if (!cnt || !val || !round) return NH_ERR_INVALID;
  if (!nh_supported(r, s)) return NH_ERR_UNSUPPORTED;
  if (exact && (link_mode < 0 || link_mode > 2 || (link_mode < 2 && (!uf || !L)))) return NH_ERR_INVALID;
  if (!exact && !(delta > 0.0)) return NH_ERR_INVALID;
  const int64_t n_r = ri->n_r;
  if (stats) *stats = nh_peel_stats{};
  if (n_r == 0) return NH_OK;
  const int C = nh_binom(s, r);
  PeelArgs A{};
  A.g = make_view(o, ri);
  A.n_r = n_r;
  A.cnt0 = cnt;
  A.val = val;
  A.round = round;
  A.link_mode = exact ? link_mode : -1;
  A.stats = stats != nullptr;
  A.gmax = g_peel_max_group;
  // automatic: link-efficient chains the targets of one r-clique per warp, so spreading its chunks
  // over many warps repeats walks; for s - r = 1 that costs more than the balance gains
  A.task_items = (unsigned int)(g_peel_task_items >= 0 ? g_peel_task_items
                                : (exact && link_mode < 2 && s - r == 1) ? 0 : kTaskItems);
  A.timeout_ns = g_nh_inject_wait_ns > 0 ? (unsigned long long)g_nh_inject_wait_ns : 60ull * 1000000000ull;
  A.lk.uf = uf;
  A.lk.L = L;
  A.lk.core = val;
  A.lk.ovf_cap = (unsigned long long)(n_r / 4 > (1 << 20) ? n_r / 4 : (1 << 20));
  A.use24 = (r == 2 && s == 4 && ri->t2off && g_peel_relist24 && (!exact || link_mode == 2)) ? 1 : 0;
  A.c24_per_warp = g_split_per_warp;
  A.c24_wgrain = g_split_wgrain;
  A.c24_bgrain = g_split_bgrain;
  A.c24_len_mult = g_split_len_mult;
  A.round_log = reinterpret_cast<unsigned long long*>(g_nh_round_log);
  A.round_log_cap = (unsigned long long)g_nh_round_log_cap;
  int rc = NH_OK;
  uint32_t* thr_dev = nullptr;
  unsigned int* dmax = nullptr;
  uint32_t* cost = nullptr;
  ulonglong2* eh_table = nullptr;
  std::vector<uint32_t> thr_host;
  if ((rc = nh_alloc(&A.cnt, n_r, st)) || (rc = nh_alloc(&A.alive[0], n_r, st)) ||
      (rc = nh_alloc(&A.alive[1], n_r, st)) || (rc = nh_alloc(&A.front[0], n_r, st)) ||
      (rc = nh_alloc(&A.front[1], n_r, st)) || (rc = nh_alloc(&A.lk.ctl, 1, st)) ||
      (rc = nh_alloc(&cost, n_r, st))) {
    goto cleanup;
  }
  if (A.use24) {
    A.c24_qcap = (unsigned long long)(n_r + kC24QueueSlack);
    if ((rc = nh_alloc(&A.c24_queue, (int64_t)A.c24_qcap, st))) goto cleanup;
    cudaMemsetAsync(A.c24_queue, 0xff, sizeof(unsigned long long) * A.c24_qcap, st);
  }
  if ((rc = chunk_cost_pair(r, s, A.g, n_r, cost, st))) goto cleanup;
  A.cost = cost;
  if (r == 3 && s == 4 && g_peel_relist24 && A.g.tedge && 3 * n_r < (1ll << 31)) {
    if (nh_alloc(&A.et3, 3 * n_r, st) == NH_OK && nh_alloc(&A.tpos, 3 * n_r, st) == NH_OK) {
      k_et3_fill<<<nh_blocks_for(A.g.m * 32, 256, 152 * 16), 256, 0, st>>>(A.g, A.et3, A.tpos, nullptr);
      nh_note_launch();
    } else {  // no room: the plain lists
      (void)cudaGetLastError();
      nh_free(A.et3, st); nh_free(A.tpos, st);
      A.et3 = nullptr; A.tpos = nullptr;
    }
  }
  if (exact) {
    if ((rc = nh_alloc(&A.lk.ovf[0], (int64_t)A.lk.ovf_cap, st)) || (rc = nh_alloc(&A.lk.ovf[1], (int64_t)A.lk.ovf_cap, st)))
      goto cleanup;
    unsigned long long cap = link_mode == 2 ? 1 : 4096;
    while (link_mode != 2 && cap < 2ull * (unsigned long long)n_r && cap < (1ull << 24)) cap <<= 1;
    if ((rc = nh_alloc(&A.lk.cache, (int64_t)cap, st))) goto cleanup;
    A.lk.cache_mask = cap - 1;
    cudaMemsetAsync(A.lk.cache, 0xff, sizeof(unsigned long long) * cap, st);
    if ((rc = nh_alloc(&A.lk.J, n_r, st))) goto cleanup;
    cudaMemsetAsync(A.lk.J, 0xff, sizeof(int32_t) * n_r, st);
  }
  if (!exact) {
    // bucket upper ends t_i = floor(x_i), x_0 = (C+delta)(1+delta), x_{i+1} = x_i (1+delta), up to
    // the largest count
    if ((rc = nh_alloc(&dmax, 1, st))) goto cleanup;
    cudaMemsetAsync(dmax, 0, sizeof(unsigned int), st);
    k_max_u32<<<nh_blocks_for(n_r, 256, 152 * 8), 256, 0, st>>>(n_r, cnt, dmax);
    nh_note_launch();
    unsigned int hmax = 0;
    cudaMemcpyAsync(&hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; goto cleanup; }
    thr_host.resize(1 << 16);
    thr_host.resize((size_t)nh_approx_table(C, delta, hmax, thr_host.data(), 1 << 16));
    A.T = nh_approx_cap(C, delta, n_r);
    A.n_thr = (int)thr_host.size();
    if ((rc = nh_alloc(&thr_dev, A.n_thr, st))) goto cleanup;
    if (cudaMemcpyAsync(thr_dev, thr_host.data(), sizeof(uint32_t) * thr_host.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) { rc = NH_ERR_CUDA; goto cleanup; }
    A.thresholds = thr_dev;
  }
  cudaMemsetAsync(A.lk.ctl, 0, sizeof(PeelCtl), st);
  k_ctl_init<<<1, 1, 0, st>>>(A.lk.ctl, n_r, exact ? 0u : thr_host[0]);
  nh_note_launch();
  k_peel_init<<<nh_blocks_for(n_r, 256, 152 * 32), 256, 0, st>>>(n_r, cnt, A.cnt, round, val, A.alive[0],
                                                                  exact ? uf : nullptr, exact ? L : nullptr);
  nh_note_launch();
  build_list_hash(A, n_r, !exact || link_mode == 2, &A.lk.ctl->err, &eh_table, st);
  if (cudaGetLastError() != cudaSuccess) { rc = NH_ERR_CUDA; goto cleanup; }
  rc = peel_launch_pair(r, s, exact, A, st);
  if (!rc && res_dev) {
    k_peel_result<<<1, 1, 0, st>>>(A.lk.ctl, res_dev);
    nh_note_launch();
  } else if (!rc) {
    PeelCtl h{};
    cudaMemcpyAsync(&h, A.lk.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    else if (h.err) rc = h.err;
    else if (!h.done) rc = NH_ERR_INTERNAL;
    if (!rc && stats) {
      stats->rounds = h.st_rounds;
      stats->levels = h.st_levels;
      stats->kmax = h.kmax;
      stats->s_cliques_listed = h.st_listed;
      stats->decrements = h.st_dec;
      stats->link_calls = h.st_link;
      stats->unites = h.st_unite;
      stats->scan_elements = h.st_scan;
      stats->hash_probes = h.st_probe;
      stats->frontier_total = h.st_front;
      stats->overflow_links = h.st_ovf;
      stats->stamp_reads = h.st_stamp;
    }
  }
cleanup:
  nh_free(A.cnt, st); nh_free(A.alive[0], st); nh_free(A.alive[1], st); nh_free(A.front[0], st);
  nh_free(A.front[1], st); nh_free(A.lk.ctl, st); nh_free(A.lk.ovf[0], st); nh_free(A.lk.ovf[1], st);
  nh_free(A.lk.cache, st); nh_free(A.lk.J, st);
  nh_free(thr_dev, st); nh_free(dmax, st); nh_free(cost, st); nh_free(A.c24_queue, st);
  nh_free(A.et3, st); nh_free(A.tpos, st); nh_free(eh_table, st);
  if (res_dev) return (cudaGetLastError() != cudaSuccess && !rc) ? NH_ERR_CUDA : rc;
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

}  // namespace nhp

using namespace nhp;

extern "C" int nh_peel_and_link(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* cnt, uint32_t* core,
                                uint32_t* round, int32_t* uf, int32_t* L, int link_mode, nh_peel_stats* stats,
                                void* stream) {
  return run_peel(true, o, ri, s, cnt, core, round, uf, L, link_mode, 0.0, stats, nullptr, (cudaStream_t)stream);
}

extern "C" int nh_approx_nucleus(const nh_oriented* o, const nh_rindex* ri, int s, double delta, const uint32_t* cnt,
                                 uint32_t* approx, uint32_t* round, nh_peel_stats* stats, void* stream) {
  return run_peel(false, o, ri, s, cnt, approx, round, nullptr, nullptr, -1, delta, stats, nullptr,
                  (cudaStream_t)stream);
}

extern "C" int nh_hierarchy_enqueue(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, uint32_t* core,
                                    uint32_t* round, int32_t* uf, int32_t* L, int32_t* parent, uint32_t* label,
                                    int64_t* res, void* stream) {
  if (!o || !ri || ri->o != o || !res) return NH_ERR_INVALID;
  if (!nh_supported(ri->r, s)) return NH_ERR_UNSUPPORTED;
  const int64_t n_r = ri->n_r;
  if (n_r > 0 && (!cnt || !core || !round || !uf || !L || !parent || !label)) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(res, 0, 4 * sizeof(int64_t), st) != cudaSuccess) return NH_ERR_CUDA;
  if (n_r == 0) return NH_OK;
  int* cstat = nullptr;
  int rc = nh_alloc(&cstat, 1, st);
  if (rc) return rc;
  cudaMemsetAsync(cstat, 0, sizeof(int), st);
  rc = nh_count_enqueue(o, ri, s, cnt, nullptr, nullptr, reinterpret_cast<unsigned long long*>(res + 1), cstat, st);
  if (!rc) {
    k_status_into<<<1, 1, 0, st>>>(cstat, res);
    nh_note_launch();
  }
  nh_free(cstat, st);
  if (!rc) rc = run_peel(true, o, ri, s, cnt, core, round, uf, L, 0, 0.0, nullptr, res, st);
  if (!rc) rc = nh_tree_enqueue(n_r, core, uf, L, parent, label, res + 2, res, st);
  return rc;
}

extern "C" int nh_link_pairs(int64_t n_r, const uint32_t* core, int32_t* uf, int32_t* L, const int32_t* pairs,
                             int64_t n_pairs, void* stream) {
  if (n_r < 0 || n_pairs < 0 || (n_r > 0 && (!core || !uf || !L)) || (n_pairs > 0 && !pairs)) return NH_ERR_INVALID;
  if (n_pairs == 0) return NH_OK;
  cudaStream_t st = (cudaStream_t)stream;
  LinkEnv E{};
  E.uf = uf;
  E.L = L;
  E.core = core;
  E.ovf_cap = (unsigned long long)(n_pairs > (1 << 16) ? n_pairs : (1 << 16));
  int rc = NH_OK;
  if ((rc = nh_alloc(&E.ctl, 1, st)) || (rc = nh_alloc(&E.ovf[0], (int64_t)E.ovf_cap, st)) ||
      (rc = nh_alloc(&E.ovf[1], (int64_t)E.ovf_cap, st))) {
    nh_free(E.ctl, st); nh_free(E.ovf[0], st); nh_free(E.ovf[1], st);
    return rc;
  }
  cudaMemsetAsync(E.ctl, 0, sizeof(PeelCtl), st);
  k_link_pairs<<<nh_blocks_for(n_pairs, 128, 152 * 16), 128, 0, st>>>(E, (const int2*)pairs,
                                                                    (unsigned long long)n_pairs);
  nh_note_launch();
  PeelCtl h{};
  for (int iter = 0; iter < 1000 && !rc; iter++) {
    cudaMemcpyAsync(&h, E.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
    if (h.err) { rc = h.err; break; }
    if (h.ovf_count[h.ovf_cur] == 0) break;
    k_link_swap<<<1, 1, 0, st>>>(E.ctl, E.ovf_cap);
    nh_note_launch();
    k_link_drain<<<152 * 8, 128, 0, st>>>(E);
    nh_note_launch();
  }
  nh_free(E.ctl, st); nh_free(E.ovf[0], st); nh_free(E.ovf[1], st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

// ---------------------------------------------------------------------------------------------
// §7.4 practical two-phase hierarchy (anh-te): with the core numbers known, levels are processed
// from the largest core down to 1 with one union-find: at level c every r-clique of core c
// re-lists its s-cliques and joins the members of those whose least core is c; then every
// component holding an r-clique of core c gets a node at level c, which adopts the previous top
// nodes of the components it absorbed.  One persistent cooperative kernel, four grid barriers
// per level.
// ---------------------------------------------------------------------------------------------

namespace nhp {

__global__ void k_core_hist(int64_t n_r, const uint32_t* __restrict__ core, uint32_t* __restrict__ hist) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(hist + core[i], 1u);
}

__global__ void k_core_scatter(int64_t n_r, const uint32_t* __restrict__ core, const int64_t* __restrict__ off,
                               unsigned long long* __restrict__ cursor, int32_t* __restrict__ order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = core[i];
    order[off[c] + (int64_t)atomicAdd(cursor + c, 1ull)] = (int32_t)i;
  }
}

__global__ void k_two_phase_init(int64_t n_r, int32_t* __restrict__ uf, uint32_t* __restrict__ lvl,
                                 int32_t* __restrict__ top, int32_t* __restrict__ parent) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += (int64_t)gridDim.x * blockDim.x) {
    uf[i] = (int32_t)i;
    lvl[i] = 0;
    top[i] = -1;
    parent[i] = -1;
  }
}

}  // namespace nhp

// label_mode: `core` holds arbitrary labels; r-cliques alone at their own level are handled
static int two_phase_impl(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* core, int32_t* parent,
                          uint32_t* label, int64_t* n_nodes, bool label_mode, void* stream) {
  if (!o || !ri || ri->o != o) return NH_ERR_INVALID;
  const int r = ri->r;
  if (!nh_supported(r, s) && !nh_generic_pair(r, s)) return NH_ERR_UNSUPPORTED;
  const int64_t n_r = ri->n_r;
  if (n_r == 0) {
    if (n_nodes) *n_nodes = 0;
    return NH_OK;
  }
  if (!core || !parent || !label) return NH_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (!nh_supported(r, s)) {
    // other pairs: link-efficient over every s-clique at the level of its least member value,
    // then construct-tree (the definitional hierarchy of those values; core numbers included)
    int64_t nn = 0;
    const int rc = nh_label_hierarchy_generic(o, ri, s, core, parent, label, &nn, st);
    if (!rc && n_nodes) *n_nodes = nn;
    return rc;
  }
  PeelArgs A{};
  TreeOut T{};
  A.g = make_view(o, ri);
  A.n_r = n_r;
  A.val = const_cast<uint32_t*>(core);
  A.union_mode = 1;
  A.gmax = g_peel_max_group;
  A.task_items = (unsigned int)(g_peel_task_items >= 0 ? g_peel_task_items : kTaskItems);
  A.link_mode = -1;
  A.stats = 0;
  A.timeout_ns = g_nh_inject_wait_ns > 0 ? (unsigned long long)g_nh_inject_wait_ns : 60ull * 1000000000ull;
  A.touched_cap = 2ull * (unsigned long long)n_r + 64;
  A.use24 = (r == 2 && s == 4 && ri->t2off && g_peel_relist24) ? 1 : 0;
  A.c24_per_warp = g_split_per_warp;
  A.c24_wgrain = g_split_wgrain;
  A.c24_bgrain = g_split_bgrain;
  A.c24_len_mult = g_split_len_mult;
  unsigned int* dmax = nullptr;
  uint32_t* hist = nullptr;
  int64_t* off = nullptr;
  unsigned long long* cursor = nullptr;
  int32_t* order = nullptr;
  uint32_t* cost = nullptr;
  uint32_t* mark = nullptr;
  ulonglong2* eh_table = nullptr;
  int rc = NH_OK;
  unsigned int kmax = 0;
  if (label_mode) {
    if ((rc = nh_alloc(&mark, n_r, st))) return rc;
    cudaMemsetAsync(mark, 0, sizeof(uint32_t) * (size_t)n_r, st);
    A.mark = mark;
  }
  if ((rc = nh_alloc(&A.lk.uf, n_r, st)) || (rc = nh_alloc(&A.lk.ctl, 1, st)) || (rc = nh_alloc(&A.touched, (int64_t)A.touched_cap, st)) ||
      (rc = nh_alloc(&A.touched_n, 1, st)) || (rc = nh_alloc(&T.lvl, n_r, st)) || (rc = nh_alloc(&T.nid, n_r, st)) ||
      (rc = nh_alloc(&T.top, n_r, st)) || (rc = nh_alloc(&T.node_count, 1, st)) || (rc = nh_alloc(&dmax, 1, st)) ||
      (rc = nh_alloc(&order, n_r, st)) || (rc = nh_alloc(&cost, n_r, st)) ||
      (A.use24 && (rc = nh_alloc(&A.c24_queue, n_r + kC24QueueSlack, st))))
    goto cleanup;
  A.c24_qcap = (unsigned long long)(n_r + kC24QueueSlack);
  if (A.use24) cudaMemsetAsync(A.c24_queue, 0xff, sizeof(unsigned long long) * A.c24_qcap, st);
  if ((rc = chunk_cost_pair(r, s, A.g, n_r, cost, st))) goto cleanup;
  A.cost = cost;
  if (r == 3 && s == 4 && g_peel_relist24 && A.g.tedge && 3 * n_r < (1ll << 31)) {
    if (nh_alloc(&A.et3, 3 * n_r, st) == NH_OK && nh_alloc(&A.tpos, 3 * n_r, st) == NH_OK) {
      k_et3_fill<<<nh_blocks_for(A.g.m * 32, 256, 152 * 16), 256, 0, st>>>(A.g, A.et3, A.tpos, core);
      nh_note_launch();
    } else {
      (void)cudaGetLastError();
      nh_free(A.et3, st); nh_free(A.tpos, st);
      A.et3 = nullptr; A.tpos = nullptr;
    }
  }
  cudaMemsetAsync(dmax, 0, sizeof(unsigned int), st);
  k_max_u32<<<nh_blocks_for(n_r, 256, 152 * 8), 256, 0, st>>>(n_r, core, dmax);
  nh_note_launch();
  cudaMemcpyAsync(&kmax, dmax, sizeof(kmax), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; goto cleanup; }
  if (kmax > (1u << 30)) { rc = NH_ERR_INVALID; goto cleanup; }  // one histogram entry per level
  if ((rc = nh_alloc(&hist, (int64_t)kmax + 2, st)) || (rc = nh_alloc(&off, (int64_t)kmax + 3, st)) ||
      (rc = nh_alloc(&cursor, (int64_t)kmax + 2, st)))
    goto cleanup;
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (kmax + 2), st);
  cudaMemsetAsync(cursor, 0, sizeof(unsigned long long) * (kmax + 2), st);
  k_core_hist<<<nh_blocks_for(n_r, 256, 152 * 16), 256, 0, st>>>(n_r, core, hist);
  nh_note_launch();
  if ((rc = nh_exclusive_scan_u32(hist, off, (int64_t)kmax + 2, st))) goto cleanup;
  k_core_scatter<<<nh_blocks_for(n_r, 256, 152 * 16), 256, 0, st>>>(n_r, core, off, cursor, order);
  k_two_phase_init<<<nh_blocks_for(n_r, 256, 152 * 32), 256, 0, st>>>(n_r, A.lk.uf, T.lvl, T.top, parent);
  nh_note_launch(2);
  cudaMemsetAsync(A.lk.ctl, 0, sizeof(PeelCtl), st);
  cudaMemsetAsync(A.touched_n, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(T.node_count, 0, sizeof(unsigned long long), st);
  build_list_hash(A, n_r, false, &A.lk.ctl->err, &eh_table, st);
  T.order = order;
  T.lvl_off = off;
  T.kmax = kmax;
  T.parent = parent;
  T.label = label;
  if (kmax >= 1) {
    rc = two_phase_launch_pair(r, s, A, T, st);
  }
  if (!rc) {
    PeelCtl h{};
    unsigned long long nn = 0;
    cudaMemcpyAsync(&h, A.lk.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&nn, T.node_count, sizeof(nn), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    else if (h.err) rc = h.err;
    if (!rc && n_nodes) *n_nodes = (int64_t)nn;
  }
cleanup:
  nh_free(A.lk.uf, st); nh_free(A.lk.ctl, st); nh_free(A.touched, st); nh_free(A.touched_n, st);
  nh_free(T.lvl, st); nh_free(T.nid, st); nh_free(T.top, st); nh_free(T.node_count, st); nh_free(dmax, st);
  nh_free(order, st); nh_free(hist, st); nh_free(off, st); nh_free(cursor, st); nh_free(cost, st);
  nh_free(mark, st); nh_free(A.c24_queue, st); nh_free(A.et3, st); nh_free(A.tpos, st); nh_free(eh_table, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = NH_ERR_CUDA;
  return rc;
}

extern "C" int nh_hierarchy_two_phase(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* core,
                                      int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream) {
  return two_phase_impl(o, ri, s, core, parent, label, n_nodes, false, stream);
}

extern "C" int nh_label_hierarchy(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* labels,
                                  int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream) {
  return two_phase_impl(o, ri, s, labels, parent, label, n_nodes, true, stream);
}

extern "C" int nh_set_peel_max_group(int g) {
  if (g < 1 || g > 1024 || (g & (g - 1))) return NH_ERR_INVALID;
  g_peel_max_group = g;
  return NH_OK;
}

extern "C" int nh_set_peel_list_hash(int mode) {
  if (mode < 0 || mode > 2) return NH_ERR_INVALID;
  g_peel_list_hash = mode;
  return NH_OK;
}

extern "C" int nh_set_peel_relist24(int on) {
  if (on != 0 && on != 1) return NH_ERR_INVALID;
  g_peel_relist24 = on;
  return NH_OK;
}

extern "C" int nh_set_relist_split(float per_warp, int warp_grain, int block_grain, int len_mult) {
  if (!(per_warp >= 0.125f && per_warp <= 64.0f) || warp_grain < 32 || block_grain < 256 || len_mult < 0 ||
      len_mult > 1024)
    return NH_ERR_INVALID;
  g_split_per_warp = per_warp;
  g_split_wgrain = warp_grain;
  g_split_bgrain = block_grain;
  g_split_len_mult = len_mult;
  return NH_OK;
}

extern "C" int nh_set_peel_task_items(int n) {
  if (n < -1 || n > kTaskItems) return NH_ERR_INVALID;
  g_peel_task_items = n;
  return NH_OK;
}
