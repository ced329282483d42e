/*
 * nucleus.h -- C-ABI of libnucleus, a GB300 (sm_103a) implementation of exact and approximate
 * hierarchical (r,s) nucleus decomposition.
 *
 * Paper: J. Shi, L. Dhulipala, J. Shun, "Parallel Algorithms for Hierarchical Nucleus
 * Decomposition" (arXiv 2306.08623).  The path is the interleaved framework of Alg. 3 with
 * link-efficient / construct-tree-efficient (Alg. 5), and the approximate peel of Alg. 2.
 *
 * Conventions for every entry point
 *  - Graph input: an undirected simple graph in CSR form in DEVICE memory: off[n+1] (int64,
 *    off[0] = 0, off[n] = 2m) and adj[2m] (int32); every neighbour list sorted ascending, no
 *    self-loops, no duplicate edges.  The caller owns these buffers and must keep them alive and
 *    unchanged while any handle built from them exists.
 *  - Every other array argument is a DEVICE pointer owned by the caller, unless it is marked
 *    "host".  Handles (nh_oriented, nh_rindex) are opaque, allocated by the library with
 *    stream-ordered device allocations and released by the matching *_free call.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  Work is enqueued on
 *    it; an entry point that returns a host value (counts, statistics) synchronises the stream
 *    before returning.  No entry point aborts, traps or prints.
 *  - r-clique ids: the canonical order is lexicographic by the sorted vertex tuple, so id i of
 *    (r=1) is vertex i, of (r=2) the i-th edge (u<v) in lexicographic order, of (r=3) the i-th
 *    triangle (a<b<c) in lexicographic order, and so on for r up to 6.
 *  - Supported (r,s): every 1 <= r < s <= 7.  (1,2), (1,3), (2,3), (2,4), (3,4) run specialised
 *    kernels (persistent peel, no host round trip per round); the other pairs run the generic
 *    path (see "Pairs" below).  Others return NH_ERR_UNSUPPORTED.
 *  - Counts and core numbers are uint32.  Counting checks every increment and returns
 *    NH_ERR_COUNT_OVERFLOW when an s-clique-degree would exceed 2^32 - 1 (core numbers and
 *    approximate values never exceed the s-clique-degree).
 *  - Return value: NH_OK (0) or one of the NH_ERR_* codes below.  A code returned by a device-side
 *    check (table full, bounded wait expired, bad index) leaves the context usable.
 */
#ifndef NUCLEUS_H
#define NUCLEUS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NH_OK 0
#define NH_ERR_INVALID 1      /* bad argument, null pointer, unsupported graph layout         */
#define NH_ERR_OOM 2          /* a device allocation failed                                   */
#define NH_ERR_TABLE_FULL 3   /* the r-clique hash table ran out of slots                      */
#define NH_ERR_OVERFLOW 4     /* an internal work queue overflowed                            */
#define NH_ERR_TIMEOUT 5      /* a bounded device wait (grid barrier, CAS retry) expired       */
#define NH_ERR_UNSUPPORTED 6  /* (r,s) outside the supported set                              */
#define NH_ERR_CUDA 7         /* a CUDA runtime call failed                                   */
#define NH_ERR_INTERNAL 8     /* a device-side consistency check failed (lookup miss)          */
#define NH_ERR_COUNT_OVERFLOW 9 /* an s-clique-degree exceeds 2^32 - 1 (counts are uint32)     */

typedef struct nh_oriented nh_oriented;
typedef struct nh_rindex nh_rindex;

/* Peel statistics, written to host memory when the pointer is not NULL. */
typedef struct nh_peel_stats {
  uint64_t rounds;             /* peeling rounds (rho of §5 for the exact peel)                */
  uint64_t levels;             /* rounds that opened a new level / bucket by a full scan       */
  uint32_t kmax;               /* largest core number (exact) or largest value (approx)        */
  uint32_t reserved;
  uint64_t s_cliques_listed;   /* (R, S) pairs re-listed over the whole peel                   */
  uint64_t decrements;         /* count decrements applied                                     */
  uint64_t link_calls;         /* link-efficient invocations including cascades               */
  uint64_t unites;             /* successful union-find unions                                 */
  uint64_t scan_elements;      /* adjacency entries scanned while re-listing                   */
  uint64_t hash_probes;        /* r-clique hash look-ups (r = 3)                               */
  uint64_t frontier_total;     /* sum of frontier sizes                                        */
  uint64_t overflow_links;     /* link calls deferred to the device overflow queue             */
  uint64_t stamp_reads;        /* round stamps (or core numbers) of members read while re-listing */
} nh_peel_stats;

/* Orientation -- Arb-Orient (Alg. 3, first step; §3 on O(alpha)-orientations).
 * Builds the low out-degree orientation: u -> v iff (deg u, u) < (deg v, v) lexicographically;
 * out-lists keep ascending vertex order.  Also builds, per adjacency entry, the canonical id of
 * its edge, and the lexicographic edge list.  n >= 1; nnz = off[n] = 2m (read from the host
 * copy of off[n] the caller passes as nnz).  Errors: NH_ERR_INVALID, NH_ERR_OOM, NH_ERR_CUDA. */
int nh_build_orientation(int64_t n, int64_t nnz, const int64_t* off, const int32_t* adj,
                         nh_oriented** out, void* stream);
/* host outputs: vertices, undirected edges, largest out-degree, largest degree */
int nh_oriented_info(const nh_oriented* o, int64_t* n, int64_t* m, int64_t* max_out, int64_t* max_deg);
void nh_oriented_free(nh_oriented* o);

/* r-clique index -- the r-cliques (the keys of table U in Alg. 3).  r = 1: vertices; r = 2: edges;
 * r = 3: triangles, enumerated per lexicographic edge (a,b) as the common neighbours c > b, and
 * inserted into a device open-addressing hash table keyed by (edge id of (a,b), c); r = 4..6: the
 * same one level up -- per (r-1)-clique P in lexicographic order, the common neighbours c above
 * P's largest vertex, keyed by (id of P, c) -- a chain of tables ending at the triangles.  Ids
 * are lexicographic in every case.
 * *n_r (host) receives the number of r-cliques.
 * Errors: NH_ERR_INVALID, NH_ERR_OOM, NH_ERR_TABLE_FULL, NH_ERR_CUDA. */
int nh_index_r_cliques(const nh_oriented* o, int r, nh_rindex** out, int64_t* n_r, void* stream);
/* write the vertex tuples of all r-cliques, tuples[i*r + j] (int32, device, n_r*r entries) */
int nh_rindex_tuples(const nh_rindex* ri, int32_t* tuples, void* stream);
void nh_rindex_free(nh_rindex* ri);

/* Pairs.  Every entry point that takes (r,s) accepts 1 <= r < s <= 7 (§1: r < s <= 7).  (1,2),
 * (1,3), (2,3), (2,4) and (3,4) run the specialised kernels described below; every other pair runs
 * the generic path: counting by recursive listing, the peel (exact or approximate) with one host
 * round trip per round, and the hierarchy by link-efficient (Alg. 5) over every s-clique after the
 * peel followed by construct-tree.  nh_hierarchy_enqueue takes the specialised pairs only. */

/* Counting -- rec-list-cliques (Alg. 3, count step): cnt[R] = number of s-cliques containing R
 * (s-clique-degree, §3), for every r-clique R, found by recursive intersection of out-lists of
 * the orientation so that each s-clique is listed once.  cnt: uint32[n_r] (overwritten).
 * *n_s (host, may be NULL) receives the number of s-cliques.
 * Errors: NH_ERR_INVALID, NH_ERR_UNSUPPORTED, NH_ERR_OOM, NH_ERR_INTERNAL, NH_ERR_COUNT_OVERFLOW,
 * NH_ERR_CUDA. */
int nh_count_s_cliques(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt,
                       uint64_t* n_s, void* stream);

/* Peel -- the peeling loop of Alg. 3 interleaved with link-efficient (Alg. 5), in one
 * persistent cooperative kernel.  Round t: k = max(k, min count over live r-cliques); the
 * frontier A is every live r-clique with count <= k; each R in A re-lists its s-cliques; an
 * s-clique whose members were all live at the start of the round dies now: its member of least
 * id in A decrements the other live members once and links the members of A in it; an
 * s-clique that died in an earlier round is linked from R to one of its earlier-peeled members
 * of least core (link_mode 0, the definition of §3) -- link_mode 1 instead links R with every
 * member peeled no later than R (the literal pair rule of Alg. 3); link_mode 2 computes the core
 * numbers only (uf and L may be NULL), for nh_hierarchy_two_phase (§7.4).
 * Inputs: cnt uint32[n_r] (s-clique-degrees, not modified).
 * Outputs: core uint32[n_r] (exact (r,s)-clique core numbers), round uint32[n_r] (1-based peel
 * round), uf int32[n_r] and L int32[n_r] (the union-find and nearest-lower-core table of
 * Alg. 5; -1 = empty).  round and uf/L are required.
 * Errors: NH_ERR_INVALID, NH_ERR_UNSUPPORTED, NH_ERR_OOM, NH_ERR_TIMEOUT, NH_ERR_OVERFLOW,
 * NH_ERR_INTERNAL, NH_ERR_CUDA. */
int nh_peel_and_link(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* cnt,
                     uint32_t* core, uint32_t* round, int32_t* uf, int32_t* L, int link_mode,
                     nh_peel_stats* stats, void* stream);

/* Tree -- construct-tree-efficient (Alg. 5): one node per union-find component, its parent the
 * node of find(L[root]); a node whose subtree holds a single r-clique is dropped and that
 * r-clique hangs from the dropped node's parent (§7.3 remark on single-child parents).
 * uf is compressed in place.  Outputs: parent int32[n_r + n_nodes] (entries 0..n_r-1: node of
 * each r-clique or -1; entries n_r + j: parent node of node j or -1) -- the caller passes room
 * for 2*n_r entries; label uint32[n_r] (label[j] = level of node j); *n_nodes (host).
 * Errors: NH_ERR_INVALID (also: uf holds a cycle, so it is no union-find forest), NH_ERR_OOM,
 * NH_ERR_CUDA. */
int nh_construct_tree(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L,
                      int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream);

/* nh_construct_tree without any device allocation.  Some callers cannot allocate device memory
 * while they run: a process whose device memory is already claimed by its own pooling allocator
 * (a cudaMalloc would fail or fragment that pool), or a latency-bound caller for which the
 * device-wide synchronisation that cudaMalloc / cudaFree may cause is not acceptable.  This entry
 * point gives them the same tree as nh_construct_tree (same arguments, outputs and errors) while
 * calling no cudaMalloc, cudaFree or other allocating routine.  The paper has no counterpart.
 *  - Working memory is a fixed array in device memory, sized for n_r <= NH_TREE_NOALLOC_MAX
 *    r-cliques (about 5.3 MB); every device that loads the library holds it until the process
 *    exits.  Larger n_r returns NH_ERR_INVALID before any device work.
 *  - The first call on a device looks up the array's device address (once per device, with that
 *    device current); make that first call before any stream capture begins on that device.
 *  - All calls share the one array: calls whose device work overlaps (on different streams, or
 *    from different host threads) race and corrupt each other's results -- serialise them.
 *  - The call synchronises `stream` before returning (it returns *n_nodes on the host). */
#define NH_TREE_NOALLOC_MAX (1 << 18)
int nh_construct_tree_noalloc(int64_t n_r, const uint32_t* core, int32_t* uf, const int32_t* L,
                              int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream);

/* Basic link (§7.2) -- link-basic and construct-tree-basic (Alg. 4), the ablation the paper measures
 * against link-efficient: one union-find per level 1..kmax (kmax * n_r int32 of device memory:
 * NH_ERR_OOM when that exceeds 80 % of the free memory); every s-clique unites its member of least
 * core with each other member in every level up to c_S (the definitional reading of §3, the same
 * connections the interleaved peel makes); then, from level kmax down to 1, every component of at
 * least two r-cliques that is not already, as a set, a component one level up becomes a node of
 * that level adopting its members' current top nodes.  Inputs: the core numbers of the exact peel.
 * Outputs as nh_construct_tree (parent int32[2 n_r], label uint32[n_r], *n_nodes host); *unites
 * (host, may be NULL) = successful unions over all levels.  Synchronises `stream`.
 * Errors: NH_ERR_INVALID, NH_ERR_UNSUPPORTED, NH_ERR_OOM, NH_ERR_INTERNAL, NH_ERR_TIMEOUT, NH_ERR_CUDA. */
int nh_hierarchy_basic(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* core, int32_t* parent,
                       uint32_t* label, int64_t* n_nodes, uint64_t* unites, void* stream);

/* c-(r,s) nuclei from a hierarchy (§8's use of the hierarchy for dense subgraphs; §3: the
 * c-(r,s) nuclei are the connected components of the r-cliques of core >= c).  Removing every node
 * of level < c from the tree of nh_construct_tree / nh_hierarchy_two_phase leaves a forest whose
 * trees are exactly the c-nuclei.  Inputs (device): parent int32[n_r + n_nodes] and label
 * uint32[n_nodes] in that layout.  Output (device, caller-owned): nucleus int32[n_r] = the node id
 * of the top of the c-nucleus holding r-clique i, or -1 when i's core is below c (or i is in no
 * node).  *n_nuclei (host, may be NULL; when given the call synchronises `stream`) = the number of
 * c-nuclei.  Entries out of range in parent are treated as absent.
 * Errors: NH_ERR_INVALID, NH_ERR_OOM, NH_ERR_CUDA. */
int nh_cut_hierarchy(int64_t n_r, int64_t n_nodes, const int32_t* parent, const uint32_t* label, uint32_t c,
                     int32_t* nucleus, int64_t* n_nuclei, void* stream);

/* §7.4 practical two-phase hierarchy (anh-te), from final core numbers: levels c = kmax .. 1 are
 * processed with one union-find; at level c every r-clique of core c re-lists its s-cliques and
 * joins the members of those whose least member core is c (the definition of §3); each component
 * holding an r-clique of core c then gets a node at level c that adopts the top nodes of the
 * components it absorbed.  Same output layout as nh_construct_tree (parent int32[2*n_r], label
 * uint32[n_r], *n_nodes host); single-leaf nodes never arise.
 * Errors: NH_ERR_INVALID, NH_ERR_UNSUPPORTED, NH_ERR_OOM, NH_ERR_TIMEOUT, NH_ERR_OVERFLOW, NH_ERR_CUDA. */
int nh_hierarchy_two_phase(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* core,
                           int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream);

/* The definitional hierarchy (§3) of arbitrary labels in place of core numbers, by the same
 * two-phase procedure: at level c the r-cliques of label >= c are joined through every s-clique
 * whose members all have label >= c; a node is a component of at least two r-cliques, labelled
 * with its least member label.  With the approximate values of nh_approx_nucleus as labels this
 * is the approximate hierarchy of §6 (Alg. 1 applied to approximate values, read
 * definitionally).  An r-clique in no s-clique whose members all reach its own label is alone at
 * that level and becomes a leaf of the first node its component gets at a lower level (parent
 * -1 if none).  labels: device uint32[n_r], every label <= 2^30 (NH_ERR_INVALID otherwise);
 * parent / label / n_nodes as nh_construct_tree.  Synchronises the stream. */
int nh_label_hierarchy(const nh_oriented* o, const nh_rindex* ri, int s, const uint32_t* labels,
                       int32_t* parent, uint32_t* label, int64_t* n_nodes, void* stream);

/* Approximate peel -- approx-arb-nucleus (Alg. 2): buckets with upper ends t_i = floor(x_i),
 * x_0 = (C+delta)(1+delta), x_{i+1} = x_i (1+delta) (IEEE double, C = binom(s,r)); round t peels
 * every live r-clique with count <= t_i; after T = ceil(ln(max(n_r,2)) / log1p(delta/C)) + 1
 * rounds in one bucket, or when it is empty, the next bucket opens.  approx[R] = min(t_i,
 * cnt[R]) for the bucket it is peeled in.  Outputs approx uint32[n_r], round uint32[n_r].
 * delta > 0.  Errors as nh_peel_and_link. */
int nh_approx_nucleus(const nh_oriented* o, const nh_rindex* ri, int s, double delta,
                      const uint32_t* cnt, uint32_t* approx, uint32_t* round,
                      nh_peel_stats* stats, void* stream);

/* The schedule both approximate peels use (host only, no device work): Alg. 2's bucket upper ends
 * t_i = floor(x_i), x_0 = (C + delta)(1 + delta), x_{i+1} = x_i (1 + delta) in IEEE double
 * (saturating at 2^32 - 1), written to out (host uint32[cap]) up to and including the first end
 * >= max_count, *n = how many (at most cap); and the round cap per bucket
 * T = ceil(ln(max(n_r, 2)) / log1p(delta / C)) + 1 (the constant Alg. 2 leaves open).  C = C(s,r).
 * Errors: NH_ERR_INVALID (C < 1, delta <= 0, null pointers, cap < 1, n_r < 0). */
int nh_approx_thresholds(int C, double delta, uint32_t max_count, uint32_t* out, int cap, int* n);
int nh_approx_round_cap(int C, double delta, int64_t n_r, uint32_t* T);

/* link-efficient (Alg. 5) applied to a batch of calls, one device thread per call, all
 * concurrent: pairs int32[2*n_pairs] (R, Q), core uint32[n_r] (ND), uf / L int32[n_r] updated
 * in place.  The building block of nh_peel_and_link, exported for direct use and testing.
 * Errors: NH_ERR_INVALID, NH_ERR_OOM, NH_ERR_TIMEOUT, NH_ERR_OVERFLOW, NH_ERR_CUDA. */
int nh_link_pairs(int64_t n_r, const uint32_t* core, int32_t* uf, int32_t* L,
                  const int32_t* pairs, int64_t n_pairs, void* stream);

/* Work estimator -- a learned estimator for the s-clique listing (rec-list-cliques) work.
 * Work items are the out-edges (v -> a) of the orientation; a cost estimate per vertex orders the
 * items by decreasing cost, and the warps of the counting kernel take them in chunks from a shared
 * counter (largest first).  Counts do not depend on the schedule.  The estimator is an MLP NH_MLP_FEATURES -> 64 -> 64 -> 1 (ReLU),
 * BF16 weights, FP32 accumulation, trained (Adam, full batch, MSE on log1p(cost)) on the
 * per-vertex costs that the counting kernel itself measures.  The paper has no counterpart: it
 * schedules this work with a work-stealing scheduler (§3).
 * Weight layout (bf16, NH_MLP_PARAMS entries): W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3. */
#define NH_MLP_FEATURES 8
#define NH_MLP_HIDDEN 64
#define NH_MLP_PARAMS 4801
/* feats float[n * NH_MLP_FEATURES]: log1p of degree, out-degree, 2-hop out-degree sum, 2-hop
 * degree sum, largest out-neighbour out-degree, sum of min out-degrees; (log out-degree)^2 / 8; 1 */
int nh_vertex_features(const nh_oriented* o, float* feats, void* stream);
/* cost float[n]: measured listing work per vertex (list entries touched incl. binary-search
 * steps) of one counting pass for (r,s); NH_ERR_UNSUPPORTED for (1,2) */
int nh_listing_cost(const nh_oriented* o, const nh_rindex* ri, int s, float* cost, void* stream);
/* cost float[n] = d+(v)^(s-1): the degree-based baseline estimate */
int nh_degree_cost(const nh_oriented* o, int s, float* cost, void* stream);
/* train on n_train vertices sampled (counter-based hash of seed) from feats/cost (n rows);
 * weights uint16[NH_MLP_PARAMS] (bf16 bit patterns, written); *final_loss (host, may be NULL) */
int nh_mlp_train(const float* feats, const float* cost, int64_t n, int64_t n_train, int steps, float lr,
                 uint64_t seed, uint16_t* weights, float* final_loss, void* stream);
/* pred float[n] = predicted listing cost per vertex */
int nh_mlp_predict(const float* feats, int64_t n, const uint16_t* weights, float* pred, void* stream);
/* nh_count_s_cliques with the items scheduled largest-first by vertex_cost (float[n], any estimate) */
int nh_count_s_cliques_partitioned(const nh_oriented* o, const nh_rindex* ri, int s, const float* vertex_cost,
                                   uint32_t* cnt, uint64_t* n_s, void* stream);

/* Batches of graphs.  A batch is run as the disjoint union of its graphs (vertex ids of
 * graph g shifted by vbase[g]), so one persistent peel launch serves all of them; s-cliques never
 * cross graphs, so every core number and hierarchy node equals that of its own graph, and the
 * r-cliques of graph g are the union's ids [rbase[g], rbase[g+1]).  The paper has no counterpart.
 * graphs: host array of device CSRs; off_out int64[N+1], adj_out int32[NNZ] (device, caller-
 * allocated, N = sum of n, NNZ = sum of nnz); vbase int64[n_graphs+1] (host, written). */
typedef struct nh_graph_desc {
  int64_t n, nnz;
  const int64_t* off;
  const int32_t* adj;
} nh_graph_desc;
int nh_batch_union(const nh_graph_desc* graphs, int n_graphs, int64_t* off_out, int32_t* adj_out, int64_t* vbase,
                   void* stream);
/* rbase int64[n_graphs+1] (host): first r-clique id of each graph of a union built from vbase */
int nh_rindex_bases(const nh_rindex* ri, const int64_t* vbase, int n_graphs, int64_t* rbase, void* stream);

/* A batch as one library object.  nh_batch_prepare copies the graphs into their disjoint
 * union (owned by the handle), builds its orientation and its r-clique index (r = 1, 2, 3), and
 * returns *n_r (host) = the union's r-cliques; it synchronises `stream` (sizes come back to the
 * host).  nh_batch_run then enqueues, for one s, exactly what nh_hierarchy_enqueue does on the
 * union -- counts, the persistent peel with link-efficient (one launch for every graph of the
 * batch) and construct-tree -- with no host synchronisation, so the caller can capture it into a
 * CUDA graph and replay it; outputs and res as nh_hierarchy_enqueue (n_r-sized arrays of the
 * union).  The r-cliques of graph g are [rbase[g], rbase[g+1]) (nh_batch_bases, host arrays of
 * n_graphs + 1 entries; vbase likewise for vertices); core numbers and hierarchy nodes never mix
 * graphs.  nh_batch_node_bases (after a run, synchronises `stream`) writes nbase (host,
 * n_graphs + 1): the nodes of graph g are [nbase[g], nbase[g+1]), n_nodes = res[2].
 * The paper has no counterpart (it runs one graph at a time).  The graphs' CSRs are only read
 * by nh_batch_prepare.  Errors: NH_ERR_INVALID (bad descriptor, r outside 1..3, more than 2^31
 * vertices in all), NH_ERR_UNSUPPORTED (pair), NH_ERR_OOM, NH_ERR_TABLE_FULL, NH_ERR_CUDA. */
typedef struct nh_batch nh_batch;
int nh_batch_prepare(const nh_graph_desc* graphs, int n_graphs, int r, nh_batch** out, int64_t* n_r, void* stream);
int nh_batch_bases(const nh_batch* b, int64_t* vbase, int64_t* rbase);
int nh_batch_run(nh_batch* b, int s, uint32_t* cnt, uint32_t* core, uint32_t* round, int32_t* uf, int32_t* L,
                 int32_t* parent, uint32_t* label, int64_t* res, void* stream);
int nh_batch_node_bases(const nh_batch* b, const int32_t* parent, int64_t n_nodes, int64_t* nbase, void* stream);
void nh_batch_free(nh_batch* b);

/* The whole exact path for one (r,s) on an existing r-clique index -- s-clique counts (as
 * nh_count_s_cliques), the peel with link-efficient in link mode 0 (as nh_peel_and_link) and
 * construct-tree (as nh_construct_tree) -- in stream order with no host synchronisation and no
 * read-back, so that a caller can capture the sequence into a CUDA graph (stream capture) and
 * replay it.  Working memory is taken and returned with cudaMallocAsync / cudaFreeAsync on the
 * stream.  Outputs (device, caller-owned): cnt, core, round, uf, L [n_r]; parent [2 n_r];
 * label [n_r]; res (int64 [4]) = {status, n_s, n_nodes, rounds}, valid once the stream reaches
 * the end of the sequence; status is 0 or the first NH_ERR_* a step recorded (a step after a
 * failed one still runs, on whatever its inputs hold, and cannot change a recorded status).
 * Return value: argument / launch errors found while enqueuing (NH_ERR_INVALID, NH_ERR_OOM,
 * NH_ERR_UNSUPPORTED, NH_ERR_CUDA). */
int nh_hierarchy_enqueue(const nh_oriented* o, const nh_rindex* ri, int s, uint32_t* cnt, uint32_t* core,
                         uint32_t* round, int32_t* uf, int32_t* L, int32_t* parent, uint32_t* label,
                         int64_t* res, void* stream);

/* Tuning knob of the peel and two-phase kernels (process-wide, default 1024): the largest number
 * of warps that share one frontier r-clique when the frontier is small.  More warps shorten a
 * round's critical path; with link-efficient each warp chains its own link targets, so more
 * warps also repeat walks.  g: power of two in [1, 1024].  Results never depend on it. */
int nh_set_peel_max_group(int g);

/* Tuning knob of the peel and two-phase kernels (process-wide): a frontier (or level) of at most
 * n r-clique ids is cut into tasks of one 32-entry chunk of a re-listed list each, which warps
 * take from a shared counter; larger ones get warp groups as above.  0 turns the task form off;
 * -1 (the default) is automatic: 4096, except 0 for the linking peel (link modes 0, 1) with
 * s - r = 1, where one r-clique's link targets spread over many warps repeat walks.
 * n in [-1, 4096]; NH_ERR_INVALID otherwise.  Results never depend on it. */
int nh_set_peel_task_items(int n);

/* Tuning knob (process-wide, default 1): with on = 1
 *  - the (2,4) peel without links (link mode 2, the approximate peel) and the (2,4) two-phase /
 *    label hierarchies re-list each edge from its triangle list (built by nh_index_r_cliques for
 *    r = 2): candidates whose edges to the frontier edge were peeled earlier (or, in the
 *    hierarchy, lie below the level) are dropped before any pair is formed, the rest are staged
 *    in shared memory, and the decrements of one candidate's two edges are summed;
 *  - every (3,4) peel and hierarchy re-lists over a copy of the per-edge triangle lists whose
 *    entries also carry their triangle's round stamp and value (16 bytes per entry, 48 bytes per
 *    triangle of working memory for the call), so that a list search returns all a 4-clique's
 *    member needs in one read.
 * on = 0 uses the plain re-listing of every other pair.  Results never depend on it.
 * NH_ERR_INVALID for other values. */
int nh_set_peel_relist24(int on);

/* Tuning knob (process-wide, default 0) of the (3,4) re-listing over the mirrored triangle lists:
 * how a candidate's entries in its other two triangle lists are found.  mode = 0: binary searches
 * of the lists (both lists searched in lockstep); 2: a table keyed by (edge id, third vertex)
 * built for the call (16-byte slots, at most 60 % full: 48 to 128 bytes per triangle of extra
 * working memory; skipped when it cannot be allocated); 1 (automatic): the table for the
 * cores-only and the approximate peel, whose candidates are pruned before the lookups, binary
 * searches for the linking peel and the two-phase hierarchy.  On R-MAT 18 (3,4) the searches are
 * as fast as the table for the cores-only peel and faster elsewhere, hence the default 0.
 * Results never depend on it.  NH_ERR_INVALID for other values. */
int nh_set_peel_list_hash(int mode);

/* Tuning knob of that (2,4) re-listing (process-wide): a frontier (or level) of at most 4096
 * r-cliques is cut into sub-tasks, each staging its r-clique's whole candidate set and taking one
 * share of its out-list scans; the sub-tasks of a round number about per_warp per warp of the
 * grid, shared out by scan bound (list length plus the sum of the candidates' out-degrees), with
 * a bound of at least warp_grain (block_grain for lists staged by a whole block) and at least
 * len_mult times the list length per sub-task (0: no such floor).  Defaults (1, 128, 1024, 0).
 * per_warp in [0.125, 64], warp_grain >= 32, block_grain >= 256, len_mult in [0, 1024];
 * NH_ERR_INVALID otherwise.  Results never depend on it. */
int nh_set_relist_split(float per_warp, int warp_grain, int block_grain, int len_mult);

/* number of CUDA kernels this library has launched in the process so far (host counter) */
int64_t nh_kernel_launches(void);

/* static description of a status code (never NULL) */
const char* nh_status_string(int status);
/* library version: major*10000 + minor*100 + patch */
int nh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NUCLEUS_H */
