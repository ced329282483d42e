/*
 * nucleus_oracle.c -- plain, sequential CPU oracle for (r,s) nucleus decomposition.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the GPU path is
 * checked against.  Only the test suite, __graft_entry__.smoke() and the CPU-baseline /
 * reference leg of bench.py may load it.  It shares no code, header, table or helper with
 * the CUDA library in paper_2306_08623_gb300/; the two are written separately from the paper.
 *
 * Paper: J. Shi, L. Dhulipala, J. Shun, "Parallel Algorithms for Hierarchical Nucleus
 * Decomposition" (arXiv 2306.08623).  What each part follows:
 *
 *  - Definitions (§3, Preliminaries): an r-clique R lies in an s-clique S when R is a subset of S;
 *    the s-clique-degree of R is the number of s-cliques containing R; the (r,s)-clique core
 *    number of R is the largest c such that R belongs to a c-(r,s) nucleus; two r-cliques are
 *    s-clique-adjacent when one s-clique contains both.
 *  - Core numbers: the sequential peel that §6 (proof of Lemma 1) attributes to Sariyuce et al.:
 *    repeatedly remove an r-clique of minimum current s-clique-degree and decrement the other
 *    members of every s-clique it destroys; the core number is the running maximum of the
 *    removal degrees.  The bucket queue is the Batagelj-Zaversnik O(1) bucket order
 *    (published k-core algorithm) generalised from edges to s-cliques.
 *  - Hierarchy: the definition (§3): at level c the r-cliques of core >= c are joined through
 *    every s-clique all of whose r-subsets have core >= c; a node is a connected set of at
 *    least two r-cliques, labelled by the highest level at which it exists.  A second,
 *    "pairwise" reading joins two r-cliques of one s-clique at min(core, core) whatever the
 *    other members are; that is the literal pair rule of Alg. 1 and Alg. 3 and is kept as a
 *    flagged variant.
 *  - Alg. 3 + Alg. 5 (link-efficient, construct-tree-efficient), run sequentially, as a second
 *    derivation of the same hierarchy and as the subject of the worked trace in §7.3.
 *  - Alg. 2 (approximate core numbers) with its round semantics; thresholds and round cap are
 *    read as: t_i = floor(x_i) with x_0 = (C+delta)(1+delta), x_{i+1} = x_i (1+delta) in IEEE
 *    double; T = ceil(ln(max(n_r,2)) / log1p(delta/C)) + 1.
 *
 * Nothing here is optimised beyond the plain algorithms: binary-search adjacency, lexicographic
 * clique enumeration by ascending extension, explicit s-clique member lists.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAX_K 8
#define ORC_EMPTY (-1)

enum {
  ORC_OK = 0,
  ORC_ERR_ARGS = 1,
  ORC_ERR_NOMEM = 2,
  ORC_ERR_DEPTH = 3,
};

typedef struct {
  int64_t n;
  const int64_t* off;
  const int32_t* adj;
} orc_graph;

/* ------------------------------------------------------------------------------------------ */
/* basic graph helpers                                                                         */
/* ------------------------------------------------------------------------------------------ */

static int64_t lower_bound32(const int32_t* a, int64_t lo, int64_t hi, int32_t x) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* is v a neighbour of u? (adjacency lists are sorted) */
static int adjacent(const orc_graph* g, int32_t u, int32_t v) {
  int64_t e = g->off[u + 1];
  int64_t p = lower_bound32(g->adj, g->off[u], e, v);
  return p < e && g->adj[p] == v;
}

static int64_t binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  int64_t b = 1;
  for (int i = 1; i <= k; i++) b = b * (n - k + i) / i;
  return b;
}

/* ------------------------------------------------------------------------------------------ */
/* k-clique enumeration in lexicographic order (ascending extension)                           */
/* ------------------------------------------------------------------------------------------ */

typedef void (*clique_visit)(const int32_t* cl, void* ctx);

/* cl[0..depth) is a clique in increasing vertex order; extend it by every larger vertex that is
 * adjacent to all of it.  Candidates are the neighbours of the last (largest) vertex. */
static void enum_rec(const orc_graph* g, int32_t* cl, int depth, int k, clique_visit visit, void* ctx) {
  if (depth == k) { visit(cl, ctx); return; }
  int32_t last = cl[depth - 1];
  int64_t e = g->off[last + 1];
  for (int64_t j = lower_bound32(g->adj, g->off[last], e, last + 1); j < e; j++) {
    int32_t w = g->adj[j];
    int ok = 1;
    for (int i = 0; i < depth - 1 && ok; i++) ok = adjacent(g, cl[i], w);
    if (!ok) continue;
    cl[depth] = w;
    enum_rec(g, cl, depth + 1, k, visit, ctx);
  }
}

static void enum_cliques(const orc_graph* g, int k, clique_visit visit, void* ctx) {
  int32_t cl[ORC_MAX_K];
  for (int64_t v = 0; v < g->n; v++) {
    cl[0] = (int32_t)v;
    if (k == 1) visit(cl, ctx); else enum_rec(g, cl, 1, k, visit, ctx);
  }
}

typedef struct { int64_t count; int32_t* out; int k; } collect_ctx;

static void visit_count(const int32_t* cl, void* c) { (void)cl; ((collect_ctx*)c)->count++; }
static void visit_store(const int32_t* cl, void* c) {
  collect_ctx* cc = (collect_ctx*)c;
  memcpy(cc->out + cc->count * cc->k, cl, sizeof(int32_t) * cc->k);
  cc->count++;
}

int64_t orc_count_cliques(int64_t n, const int64_t* off, const int32_t* adj, int k) {
  if (k < 1 || k > ORC_MAX_K) return -1;
  orc_graph g = {n, off, adj};
  collect_ctx c = {0, NULL, k};
  enum_cliques(&g, k, visit_count, &c);
  return c.count;
}

/* all k-cliques, each as k increasing vertex ids, in lexicographic order; out has room for
 * count*k entries (count from orc_count_cliques) */
int64_t orc_list_cliques(int64_t n, const int64_t* off, const int32_t* adj, int k, int32_t* out) {
  if (k < 1 || k > ORC_MAX_K) return -1;
  orc_graph g = {n, off, adj};
  collect_ctx c = {0, out, k};
  enum_cliques(&g, k, visit_store, &c);
  return c.count;
}

/* id of a sorted r-tuple in the lexicographically sorted table, or -1 */
static int64_t tuple_id(const int32_t* tab, int64_t n_r, int r, const int32_t* key) {
  int64_t lo = 0, hi = n_r;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    const int32_t* t = tab + mid * r;
    int cmp = 0;
    for (int i = 0; i < r && cmp == 0; i++) cmp = (t[i] < key[i]) ? -1 : (t[i] > key[i]) ? 1 : 0;
    if (cmp < 0) lo = mid + 1; else hi = mid;
  }
  if (lo < n_r) {
    const int32_t* t = tab + lo * r;
    for (int i = 0; i < r; i++) if (t[i] != key[i]) return -1;
    return lo;
  }
  return -1;
}

/* index combinations of r out of s, lexicographic: combos[j*r + i] */
static int make_combos(int s, int r, int* combos) {
  int idx[ORC_MAX_K];
  for (int i = 0; i < r; i++) idx[i] = i;
  int c = 0;
  for (;;) {
    for (int i = 0; i < r; i++) combos[c * r + i] = idx[i];
    c++;
    int i = r - 1;
    while (i >= 0 && idx[i] == s - r + i) i--;
    if (i < 0) break;
    idx[i]++;
    for (int j = i + 1; j < r; j++) idx[j] = idx[j - 1] + 1;
  }
  return c;
}

/* ------------------------------------------------------------------------------------------ */
/* s-clique member lists                                                                       */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  const int32_t* rtab; int64_t n_r; int r; int s; int C;
  const int* combos;
  int32_t* members; /* [n_s * C] r-clique ids of every s-clique, in combo order */
  int64_t count;
  int err;
} member_ctx;

static void visit_members(const int32_t* cl, void* c) {
  member_ctx* mc = (member_ctx*)c;
  int32_t key[ORC_MAX_K];
  for (int j = 0; j < mc->C; j++) {
    for (int i = 0; i < mc->r; i++) key[i] = cl[mc->combos[j * mc->r + i]];
    int64_t id = tuple_id(mc->rtab, mc->n_r, mc->r, key);
    if (id < 0) mc->err = 1;
    mc->members[mc->count * mc->C + j] = (int32_t)id;
  }
  mc->count++;
}

/* ------------------------------------------------------------------------------------------ */
/* result object                                                                               */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int32_t r, s, C, status;
  int64_t n_r, n_s;
  int32_t* tuples;        /* [n_r*r] lexicographic r-cliques                              */
  uint32_t* cnt;          /* [n_r] s-clique-degree                                        */
  uint32_t* core;         /* [n_r] exact (r,s)-clique core number, or NULL                 */
  uint32_t kmax;
  int64_t n_nodes;
  int32_t* leaf_node;     /* [n_r] smallest hierarchy node containing the r-clique, or -1  */
  int32_t* node_parent;   /* [n_nodes] parent node or -1                                   */
  uint32_t* node_label;   /* [n_nodes] level (core number) of the node                     */
  int64_t n_link_calls;   /* link-efficient statistics (hier modes 3, 4)                   */
  int64_t n_unite_calls;
  uint32_t* approx;       /* [n_r] approximate core number, or NULL                        */
  int64_t approx_rounds;
  uint32_t approx_T;
  int32_t n_thresholds;
  uint32_t* thresholds;   /* [n_thresholds]                                                */
  uint32_t* removal;      /* [n_r] 1-based position in the exact peel's removal order, or NULL */
} orc_result;

void orc_free(orc_result* res) {
  if (!res) return;
  free(res->tuples); free(res->cnt); free(res->core);
  free(res->leaf_node); free(res->node_parent); free(res->node_label);
  free(res->approx); free(res->thresholds); free(res->removal);
  free(res);
}

/* ------------------------------------------------------------------------------------------ */
/* exact peel (core numbers)                                                                   */
/* ------------------------------------------------------------------------------------------ */

/* Batagelj-Zaversnik bucket order over r-cliques.  At every step the unprocessed r-clique with
 * the smallest current degree is removed; every s-clique it still belongs to dies and each
 * other member whose degree is above the removed one's loses 1 (a member already at that level
 * stays there: the running maximum makes its core that level anyway). */
static int exact_peel(int64_t n_r, const uint32_t* cnt0, const int64_t* inc_off, const int64_t* inc,
                      const int32_t* members, int C, int64_t n_s, uint32_t* core, uint32_t* kmax_out,
                      uint32_t* removal) {
  uint32_t md = 0;
  for (int64_t i = 0; i < n_r; i++) if (cnt0[i] > md) md = cnt0[i];
  uint32_t* d = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
  int64_t* bin = calloc((size_t)md + 2, sizeof(int64_t));
  int64_t* pos = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* vert = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  unsigned char* dead = calloc((size_t)(n_s ? n_s : 1), 1);
  if (!d || !bin || !pos || !vert || !dead) {
    free(d); free(bin); free(pos); free(vert); free(dead); return ORC_ERR_NOMEM;
  }
  memcpy(d, cnt0, sizeof(uint32_t) * n_r);
  for (int64_t v = 0; v < n_r; v++) bin[d[v]]++;
  int64_t start = 0;
  for (uint32_t x = 0; x <= md; x++) { int64_t num = bin[x]; bin[x] = start; start += num; }
  for (int64_t v = 0; v < n_r; v++) { pos[v] = bin[d[v]]; vert[pos[v]] = v; bin[d[v]]++; }
  for (uint32_t x = md; x >= 1; x--) bin[x] = bin[x - 1];
  bin[0] = 0;
  uint32_t kmax = 0;
  for (int64_t i = 0; i < n_r; i++) {
    int64_t R = vert[i];
    core[R] = d[R];
    if (removal) removal[R] = (uint32_t)(i + 1);
    if (d[R] > kmax) kmax = d[R];
    for (int64_t q = inc_off[R]; q < inc_off[R + 1]; q++) {
      int64_t S = inc[q];
      if (dead[S]) continue;
      dead[S] = 1;
      for (int j = 0; j < C; j++) {
        int64_t u = members[S * C + j];
        if (u == R || d[u] <= d[R]) continue;
        uint32_t du = d[u];
        int64_t pu = pos[u], pw = bin[du], w = vert[pw];
        if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
        bin[du]++;
        d[u]--;
      }
    }
  }
  *kmax_out = kmax;
  free(d); free(bin); free(pos); free(vert); free(dead);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* hierarchy by levels (definitional and pairwise readings)                                    */
/* ------------------------------------------------------------------------------------------ */

static int64_t uf_find(int64_t* p, int64_t x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}

/* Union edges (a,b,level): a and b are joined at every level <= level.  Processes levels from
 * kmax down to 1 with one union-find; at level c a new node is made for every component of at
 * least two r-cliques that holds an r-clique of label exactly c (components made only of
 * higher-label r-cliques are unchanged from level c+1).  The new node adopts the current top
 * nodes of the components it absorbed.  An r-clique still alone at its own level (possible for
 * labels that are not core numbers, never for core numbers, since an r-clique of core c >= 1
 * lies in an s-clique of the c-nucleus) waits in its component's pending list and becomes a leaf
 * of the first node its component gets at a lower level (or of none). */
static int hierarchy_by_levels(int64_t n_r, const uint32_t* core, uint32_t kmax,
                               const int64_t* lvl_off, const int32_t* ea, const int32_t* eb,
                               orc_result* res) {
  int64_t* par = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* sz = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* head = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* tail = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* stamp_node = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  uint32_t* stamp_lvl = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
  int64_t* pnext = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* by_core_off = calloc((size_t)kmax + 2, sizeof(int64_t));
  int64_t* by_core = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* ph = malloc(sizeof(int64_t) * (n_r ? n_r : 1));   /* pending list head / tail per root */
  int64_t* pt = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int64_t* pn = malloc(sizeof(int64_t) * (n_r ? n_r : 1));   /* next pending r-clique */
  res->leaf_node = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  res->node_parent = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  res->node_label = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
  if (!par || !sz || !head || !tail || !stamp_node || !stamp_lvl || !pnext || !by_core_off || !by_core ||
      !ph || !pt || !pn || !res->leaf_node || !res->node_parent || !res->node_label) {
    free(par); free(sz); free(head); free(tail); free(stamp_node); free(stamp_lvl); free(pnext);
    free(by_core_off); free(by_core); free(ph); free(pt); free(pn);
    return ORC_ERR_NOMEM;
  }
  for (int64_t i = 0; i < n_r; i++) {
    par[i] = i; sz[i] = 1; head[i] = tail[i] = -1; stamp_lvl[i] = 0; stamp_node[i] = -1;
    ph[i] = pt[i] = pn[i] = -1;
    res->leaf_node[i] = -1;
  }
  for (int64_t i = 0; i < n_r; i++) by_core_off[core[i] + 1]++;
  for (uint32_t c = 0; c <= kmax; c++) by_core_off[c + 1] += by_core_off[c];
  {
    int64_t* fill = malloc(sizeof(int64_t) * ((size_t)kmax + 1));
    if (!fill) return ORC_ERR_NOMEM;
    for (uint32_t c = 0; c <= kmax; c++) fill[c] = by_core_off[c];
    for (int64_t i = 0; i < n_r; i++) by_core[fill[core[i]]++] = i;
    free(fill);
  }
  int64_t nn = 0;
  for (uint32_t c = kmax; c >= 1; c--) {
    for (int64_t q = lvl_off[c]; q < lvl_off[c + 1]; q++) {
      int64_t a = uf_find(par, ea[q]), b = uf_find(par, eb[q]);
      if (a == b) continue;
      if (sz[a] < sz[b]) { int64_t t = a; a = b; b = t; }
      par[b] = a; sz[a] += sz[b];
      if (head[b] >= 0) {
        if (head[a] < 0) { head[a] = head[b]; tail[a] = tail[b]; }
        else { pnext[tail[a]] = head[b]; tail[a] = tail[b]; }
        head[b] = tail[b] = -1;
      }
      if (ph[b] >= 0) {
        if (ph[a] < 0) { ph[a] = ph[b]; pt[a] = pt[b]; }
        else { pn[pt[a]] = ph[b]; pt[a] = pt[b]; }
        ph[b] = pt[b] = -1;
      }
    }
    for (int64_t q = by_core_off[c]; q < by_core_off[c + 1]; q++) {
      int64_t R = by_core[q];
      int64_t root = uf_find(par, R);
      if (sz[root] == 1) {  /* alone at its own level: pending */
        if (ph[root] < 0) { ph[root] = R; pt[root] = R; }
        else { pn[pt[root]] = R; pt[root] = R; }
        continue;
      }
      if (stamp_lvl[root] != c || stamp_node[root] < 0) {
        int64_t N = nn++;
        res->node_label[N] = c;
        res->node_parent[N] = -1;
        for (int64_t x = head[root]; x >= 0; x = pnext[x]) res->node_parent[x] = (int32_t)N;
        head[root] = tail[root] = N;
        pnext[N] = -1;
        stamp_lvl[root] = c;
        stamp_node[root] = N;
      }
      res->leaf_node[R] = (int32_t)stamp_node[root];
      for (int64_t x = ph[root]; x >= 0; x = pn[x]) res->leaf_node[x] = (int32_t)stamp_node[root];
      ph[root] = pt[root] = -1;
    }
    if (c == 1) break;
  }
  res->n_nodes = nn;
  free(par); free(sz); free(head); free(tail); free(stamp_node); free(stamp_lvl); free(pnext);
  free(by_core_off); free(by_core); free(ph); free(pt); free(pn);
  return ORC_OK;
}

/* Union edges of every s-clique.
 *  definitional (mode 0): all members of S join at c_S = min core over S; edges form a star
 *                         from the first member of minimum core.
 *  pairwise     (mode 1): members R, R' of S join at min(core R, core R'); a chain through the
 *                         members sorted by decreasing core realises all these pairs. */
static int build_level_edges(int64_t n_s, int C, const int32_t* members, const uint32_t* core,
                             uint32_t kmax, int mode, int64_t** lvl_off_out, int32_t** ea_out,
                             int32_t** eb_out) {
  int64_t ne = n_s * (C - 1);
  int64_t* lvl_off = calloc((size_t)kmax + 2, sizeof(int64_t));
  int32_t* ea = malloc(sizeof(int32_t) * (ne ? ne : 1));
  int32_t* eb = malloc(sizeof(int32_t) * (ne ? ne : 1));
  int64_t* fill = malloc(sizeof(int64_t) * ((size_t)kmax + 2));
  if (!lvl_off || !ea || !eb || !fill) { free(lvl_off); free(ea); free(eb); free(fill); return ORC_ERR_NOMEM; }
  int32_t m[64];
  for (int pass = 0; pass < 2; pass++) {
    if (pass == 1) {
      for (uint32_t c = 0; c <= kmax; c++) lvl_off[c + 1] += lvl_off[c];
      for (uint32_t c = 0; c <= kmax + 1; c++) fill[c] = lvl_off[c];
    }
    for (int64_t S = 0; S < n_s; S++) {
      const int32_t* mem = members + S * C;
      if (mode == 0) {
        int jmin = 0;
        for (int j = 1; j < C; j++) if (core[mem[j]] < core[mem[jmin]]) jmin = j;
        uint32_t cs = core[mem[jmin]];
        for (int j = 0; j < C; j++) {
          if (j == jmin) continue;
          if (pass == 0) lvl_off[cs + 1]++;
          else { int64_t q = fill[cs]++; ea[q] = mem[jmin]; eb[q] = mem[j]; }
        }
      } else {
        for (int j = 0; j < C; j++) m[j] = mem[j];
        for (int j = 1; j < C; j++) { /* insertion sort by decreasing core */
          int32_t x = m[j]; int i = j - 1;
          while (i >= 0 && core[m[i]] < core[x]) { m[i + 1] = m[i]; i--; }
          m[i + 1] = x;
        }
        for (int j = 1; j < C; j++) {
          uint32_t lv = core[m[j]];
          if (pass == 0) lvl_off[lv + 1]++;
          else { int64_t q = fill[lv]++; ea[q] = m[j - 1]; eb[q] = m[j]; }
        }
      }
    }
  }
  free(fill);
  *lvl_off_out = lvl_off; *ea_out = ea; *eb_out = eb;
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Alg. 5: link-efficient and construct-tree-efficient, sequential                             */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int32_t* uf;           /* union-find parent over r-cliques                                  */
  int32_t* L;            /* nearest lower-core component, ORC_EMPTY if none                   */
  const uint32_t* ND;    /* core numbers                                                      */
  int64_t n_link, n_unite;
  int err;
} lk_state;

static int32_t lk_find(lk_state* st, int32_t x) {
  while (st->uf[x] != x) { st->uf[x] = st->uf[st->uf[x]]; x = st->uf[x]; }
  return x;
}

/* unite two roots; the smaller id becomes the root */
static void lk_unite(lk_state* st, int32_t a, int32_t b) {
  a = lk_find(st, a); b = lk_find(st, b);
  if (a == b) return;
  if (a < b) st->uf[b] = a; else st->uf[a] = b;
  st->n_unite++;
}

/* Alg. 5, link-efficient(R, Q, ND), written as recursion like the paper. */
static void lk_link(lk_state* st, int32_t R, int32_t Q, int depth) {
  if (R == ORC_EMPTY || Q == ORC_EMPTY) return;
  if (depth > 100000) { st->err = ORC_ERR_DEPTH; return; }
  st->n_link++;
  if (st->ND[Q] < st->ND[R]) { int32_t t = R; R = Q; Q = t; }
  R = lk_find(st, R);
  Q = lk_find(st, Q);
  if (st->ND[R] == st->ND[Q]) {
    lk_unite(st, R, Q);
    if (lk_find(st, R) != R) lk_link(st, st->L[R], lk_find(st, R), depth + 1);
    if (lk_find(st, Q) != Q) lk_link(st, st->L[Q], lk_find(st, Q), depth + 1);
    return;
  }
  /* ND[R] < ND[Q] */
  for (;;) {
    int32_t LQ = st->L[Q];
    Q = lk_find(st, Q);
    if (st->L[Q] == ORC_EMPTY) {                          /* CAS(L[Q], empty, R) succeeds */
      st->L[Q] = R;
      if (lk_find(st, Q) != Q) lk_link(st, R, lk_find(st, Q), depth + 1);
      return;
    } else if (LQ != ORC_EMPTY && st->ND[LQ] < st->ND[R]) {
      if (st->L[Q] == LQ) {                               /* CAS(L[Q], LQ, R) succeeds */
        st->L[Q] = R;
        if (lk_find(st, Q) != Q) lk_link(st, R, lk_find(st, Q), depth + 1);
        lk_link(st, R, LQ, depth + 1);
        return;
      }
      /* CAS failed: retry with the current L[Q] */
    } else {
      lk_link(st, R, st->L[Q], depth + 1);
      return;
    }
  }
}

/* Apply a sequence of link calls to given uf / L arrays (used for the §7.3 worked example). */
int orc_link_apply(int64_t n_r, const uint32_t* ND, int32_t* uf, int32_t* L,
                   const int32_t* calls /* pairs R,Q */, int64_t n_calls) {
  lk_state st = {uf, L, ND, 0, 0, 0};
  (void)n_r;
  for (int64_t i = 0; i < n_calls; i++) lk_link(&st, calls[2 * i], calls[2 * i + 1], 0);
  return st.err;
}

int32_t orc_uf_find(int32_t* uf, int32_t x) {
  while (uf[x] != x) { uf[x] = uf[uf[x]]; x = uf[x]; }
  return x;
}

/* construct-tree-efficient: one node per uf component, its parent the node of find(L[root]);
 * nodes whose subtree holds a single r-clique are dropped (§7.3 note on single-child parents),
 * that r-clique then hangs from the dropped node's parent. */
static int construct_tree_efficient(int64_t n_r, int32_t* uf, const int32_t* L, const uint32_t* ND,
                                    orc_result* res) {
  int64_t* own = calloc((size_t)(n_r ? n_r : 1), sizeof(int64_t));
  int64_t* nch = calloc((size_t)(n_r ? n_r : 1), sizeof(int64_t));
  int64_t* nid = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  int32_t* root = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  res->leaf_node = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  res->node_parent = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  res->node_label = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
  if (!own || !nch || !nid || !root || !res->leaf_node || !res->node_parent || !res->node_label) {
    free(own); free(nch); free(nid); free(root); return ORC_ERR_NOMEM;
  }
  for (int64_t R = 0; R < n_r; R++) { root[R] = orc_uf_find(uf, (int32_t)R); own[root[R]]++; }
  for (int64_t C = 0; C < n_r; C++)
    if (root[C] == C && L[C] != ORC_EMPTY) nch[root[L[C]]]++;
  int64_t nn = 0;
  for (int64_t C = 0; C < n_r; C++) {
    nid[C] = -1;
    if (root[C] == C && !(own[C] == 1 && nch[C] == 0)) nid[C] = nn++;
  }
  for (int64_t C = 0; C < n_r; C++) {
    if (nid[C] < 0) continue;
    res->node_label[nid[C]] = ND[C];
    res->node_parent[nid[C]] = (L[C] != ORC_EMPTY) ? (int32_t)nid[root[L[C]]] : -1;
  }
  for (int64_t R = 0; R < n_r; R++) {
    int32_t C = root[R];
    if (nid[C] >= 0) res->leaf_node[R] = (int32_t)nid[C];
    else res->leaf_node[R] = (L[C] != ORC_EMPTY) ? (int32_t)nid[root[L[C]]] : -1;
  }
  res->n_nodes = nn;
  free(own); free(nch); free(nid); free(root);
  return ORC_OK;
}

/* construct-tree-efficient on given uf / L / core arrays (used for the §7.3 tree example) */
orc_result* orc_tree_from_uf(int64_t n_r, const int32_t* uf_in, const int32_t* L, const uint32_t* ND) {
  orc_result* res = calloc(1, sizeof(orc_result));
  if (!res) return NULL;
  int32_t* uf = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  if (!uf) { res->status = ORC_ERR_NOMEM; return res; }
  memcpy(uf, uf_in, sizeof(int32_t) * n_r);
  res->n_r = n_r;
  res->status = construct_tree_efficient(n_r, uf, L, ND, res);
  free(uf);
  return res;
}

/* Alg. 3 run sequentially: r-cliques are taken in order of (core, id), which is an order the
 * peel can produce up to ties, and every s-clique of the current r-clique is examined.
 *  mode 0 (definitional): link the r-clique with one already-processed member of S of minimum
 *                         core (that member's core is c_S).
 *  mode 1 (pairwise, the literal Alg. 3 test ND[R'] <= ND[R]): link with every already
 *                         processed member. */
static int hierarchy_link_efficient(int64_t n_r, const uint32_t* core, uint32_t kmax,
                                    const int64_t* inc_off, const int64_t* inc, const int32_t* members,
                                    int C, int mode, orc_result* res) {
  int32_t* uf = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  int32_t* L = malloc(sizeof(int32_t) * (n_r ? n_r : 1));
  unsigned char* done = calloc((size_t)(n_r ? n_r : 1), 1);
  int64_t* off = calloc((size_t)kmax + 2, sizeof(int64_t));
  int64_t* order = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  if (!uf || !L || !done || !off || !order) { free(uf); free(L); free(done); free(off); free(order); return ORC_ERR_NOMEM; }
  for (int64_t i = 0; i < n_r; i++) { uf[i] = (int32_t)i; L[i] = ORC_EMPTY; off[core[i] + 1]++; }
  for (uint32_t c = 0; c <= kmax; c++) off[c + 1] += off[c];
  for (int64_t i = 0; i < n_r; i++) order[off[core[i]]++] = i; /* stable: ids ascending per core */
  lk_state st = {uf, L, core, 0, 0, 0};
  for (int64_t q = 0; q < n_r; q++) {
    int64_t R = order[q];
    for (int64_t p = inc_off[R]; p < inc_off[R + 1]; p++) {
      const int32_t* mem = members + inc[p] * C;
      if (mode == 0) {
        int32_t best = ORC_EMPTY;
        for (int j = 0; j < C; j++) {
          int32_t x = mem[j];
          if (x == R || !done[x]) continue;
          if (best == ORC_EMPTY || core[x] < core[best]) best = x;
        }
        if (best != ORC_EMPTY) lk_link(&st, best, (int32_t)R, 0);
      } else {
        for (int j = 0; j < C; j++) {
          int32_t x = mem[j];
          if (x != R && done[x]) lk_link(&st, x, (int32_t)R, 0);
        }
      }
    }
    done[R] = 1;
  }
  int rc = st.err ? st.err : construct_tree_efficient(n_r, uf, L, core, res);
  res->n_link_calls = st.n_link;
  res->n_unite_calls = st.n_unite;
  free(uf); free(L); free(done); free(off); free(order);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Alg. 2: approximate core numbers                                                            */
/* ------------------------------------------------------------------------------------------ */

/* bucket upper ends t_i = floor((C+delta)(1+delta)^(i+1)), by repeated multiplication */
int orc_approx_thresholds(int C, double delta, uint32_t max_cnt, uint32_t* out, int cap) {
  double x = ((double)C + delta) * (1.0 + delta);
  int k = 0;
  while (k < cap) {
    double f = floor(x);
    uint32_t t = (f >= 4294967295.0) ? 4294967295u : (uint32_t)f;
    out[k++] = t;
    if (t >= max_cnt) break;
    x = x * (1.0 + delta);
  }
  return k;
}

uint32_t orc_approx_round_cap(int C, double delta, int64_t n_r) {
  double nn = (double)(n_r > 2 ? n_r : 2);
  return (uint32_t)ceil(log(nn) / log1p(delta / (double)C)) + 1u;
}

static int approx_peel(int64_t n_r, const uint32_t* cnt0, const int64_t* inc_off, const int64_t* inc,
                       const int32_t* members, int C, int64_t n_s, double delta, orc_result* res) {
  uint32_t md = 0;
  for (int64_t i = 0; i < n_r; i++) if (cnt0[i] > md) md = cnt0[i];
  int cap = 1 << 16;
  res->thresholds = malloc(sizeof(uint32_t) * cap);
  res->approx = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
  uint32_t* cnt = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
  unsigned char* alive = malloc((size_t)(n_r ? n_r : 1));
  unsigned char* dead = calloc((size_t)(n_s ? n_s : 1), 1);
  int64_t* A = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
  if (!res->thresholds || !res->approx || !cnt || !alive || !dead || !A) {
    free(cnt); free(alive); free(dead); free(A); return ORC_ERR_NOMEM;
  }
  res->n_thresholds = orc_approx_thresholds(C, delta, md, res->thresholds, cap);
  res->approx_T = orc_approx_round_cap(C, delta, n_r);
  memcpy(cnt, cnt0, sizeof(uint32_t) * n_r);
  memset(alive, 1, (size_t)n_r);
  int64_t finished = 0, total_rounds = 0;
  int i = 0;
  uint32_t rounds = 0;
  while (finished < n_r) {
    uint32_t ti = res->thresholds[i < res->n_thresholds ? i : res->n_thresholds - 1];
    int64_t na = 0;
    for (int64_t R = 0; R < n_r; R++) if (alive[R] && cnt[R] <= ti) A[na++] = R;
    if (na == 0) { i++; rounds = 0; continue; }
    for (int64_t q = 0; q < na; q++) {
      int64_t R = A[q];
      alive[R] = 0;
      res->approx[R] = ti < cnt0[R] ? ti : cnt0[R];
    }
    for (int64_t q = 0; q < na; q++) {
      int64_t R = A[q];
      for (int64_t p = inc_off[R]; p < inc_off[R + 1]; p++) {
        int64_t S = inc[p];
        if (dead[S]) continue;
        dead[S] = 1;
        for (int j = 0; j < C; j++) {
          int32_t x = members[S * C + j];
          if (alive[x]) cnt[x]--;
        }
      }
    }
    finished += na;
    rounds++;
    total_rounds++;
    if (rounds >= res->approx_T) { i++; rounds = 0; }
  }
  res->approx_rounds = total_rounds;
  free(cnt); free(alive); free(dead); free(A);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* driver                                                                                      */
/* ------------------------------------------------------------------------------------------ */

enum { ORC_WANT_CORE = 1, ORC_WANT_APPROX = 2 };
enum { ORC_HIER_NONE = 0, ORC_HIER_DEF = 1, ORC_HIER_PAIR = 2, ORC_HIER_LINK_DEF = 3, ORC_HIER_LINK_PAIR = 4 };

/* Full sequential run on an undirected simple graph in CSR form (sorted lists, no loops or
 * duplicates).  flags: ORC_WANT_CORE | ORC_WANT_APPROX; hier_mode selects the hierarchy. */
static orc_result* nucleus_impl(int64_t n, const int64_t* off, const int32_t* adj, int r, int s, int flags,
                                int hier_mode, double delta, const uint32_t* labels) {
  orc_result* res = calloc(1, sizeof(orc_result));
  if (!res) return NULL;
  res->r = r; res->s = s;
  if (r < 1 || s <= r || s > ORC_MAX_K || binom(s, r) > 64) { res->status = ORC_ERR_ARGS; return res; }
  orc_graph g = {n, off, adj};
  int C = (int)binom(s, r);
  res->C = C;
  int* combos = malloc(sizeof(int) * C * r);
  if (!combos) { res->status = ORC_ERR_NOMEM; return res; }
  make_combos(s, r, combos);

  /* r-cliques, lexicographic */
  res->n_r = orc_count_cliques(n, off, adj, r);
  res->tuples = malloc(sizeof(int32_t) * (res->n_r ? res->n_r : 1) * r);
  res->cnt = calloc((size_t)(res->n_r ? res->n_r : 1), sizeof(uint32_t));
  if (!res->tuples || !res->cnt) { free(combos); res->status = ORC_ERR_NOMEM; return res; }
  orc_list_cliques(n, off, adj, r, res->tuples);

  /* s-cliques with their member r-clique ids */
  res->n_s = orc_count_cliques(n, off, adj, s);
  int64_t n_r = res->n_r, n_s = res->n_s;
  member_ctx mc = {res->tuples, n_r, r, s, C, combos, NULL, 0, 0};
  mc.members = malloc(sizeof(int32_t) * (n_s ? n_s : 1) * C);
  if (!mc.members) { free(combos); res->status = ORC_ERR_NOMEM; return res; }
  enum_cliques(&g, s, visit_members, &mc);
  free(combos);
  if (mc.err) { free(mc.members); res->status = ORC_ERR_ARGS; return res; }

  /* s-clique-degree and incidence lists */
  for (int64_t q = 0; q < n_s * C; q++) res->cnt[mc.members[q]]++;
  int64_t* inc_off = calloc((size_t)n_r + 1, sizeof(int64_t));
  int64_t* inc = malloc(sizeof(int64_t) * (n_s ? n_s : 1) * C);
  if (!inc_off || !inc) { free(mc.members); free(inc_off); free(inc); res->status = ORC_ERR_NOMEM; return res; }
  for (int64_t R = 0; R < n_r; R++) inc_off[R + 1] = inc_off[R] + res->cnt[R];
  {
    int64_t* fill = malloc(sizeof(int64_t) * (n_r ? n_r : 1));
    if (!fill) { res->status = ORC_ERR_NOMEM; goto done; }
    for (int64_t R = 0; R < n_r; R++) fill[R] = inc_off[R];
    for (int64_t S = 0; S < n_s; S++)
      for (int j = 0; j < C; j++) inc[fill[mc.members[S * C + j]]++] = S;
    free(fill);
  }

  if (labels) {  /* the hierarchy of given labels in place of core numbers */
    res->core = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
    if (!res->core) { res->status = ORC_ERR_NOMEM; goto done; }
    res->kmax = 0;
    for (int64_t R = 0; R < n_r; R++) {
      res->core[R] = labels[R];
      if (labels[R] > res->kmax) res->kmax = labels[R];
    }
  } else if ((flags & ORC_WANT_CORE) || hier_mode != ORC_HIER_NONE) {
    res->core = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
    if (!res->core) { res->status = ORC_ERR_NOMEM; goto done; }
    res->removal = malloc(sizeof(uint32_t) * (n_r ? n_r : 1));
    if (!res->removal) { res->status = ORC_ERR_NOMEM; goto done; }
    res->status = exact_peel(n_r, res->cnt, inc_off, inc, mc.members, C, n_s, res->core, &res->kmax,
                             res->removal);
    if (res->status) goto done;
  }
  if (hier_mode == ORC_HIER_DEF || hier_mode == ORC_HIER_PAIR) {
    int64_t* lvl_off; int32_t* ea; int32_t* eb;
    res->status = build_level_edges(n_s, C, mc.members, res->core, res->kmax,
                                    hier_mode == ORC_HIER_DEF ? 0 : 1, &lvl_off, &ea, &eb);
    if (res->status) goto done;
    res->status = hierarchy_by_levels(n_r, res->core, res->kmax, lvl_off, ea, eb, res);
    free(lvl_off); free(ea); free(eb);
    if (res->status) goto done;
  } else if (hier_mode == ORC_HIER_LINK_DEF || hier_mode == ORC_HIER_LINK_PAIR) {
    res->status = hierarchy_link_efficient(n_r, res->core, res->kmax, inc_off, inc, mc.members, C,
                                           hier_mode == ORC_HIER_LINK_DEF ? 0 : 1, res);
    if (res->status) goto done;
  }
  if (flags & ORC_WANT_APPROX) {
    res->status = approx_peel(n_r, res->cnt, inc_off, inc, mc.members, C, n_s, delta, res);
  }
done:
  free(mc.members); free(inc_off); free(inc);
  return res;
}

orc_result* orc_nucleus(int64_t n, const int64_t* off, const int32_t* adj, int r, int s, int flags,
                        int hier_mode, double delta) {
  return nucleus_impl(n, off, adj, r, s, flags, hier_mode, delta, NULL);
}

/* The definitional hierarchy (§3) of arbitrary per-r-clique labels (lexicographic r-clique ids)
 * instead of core numbers: at level c the r-cliques of label >= c are joined through every
 * s-clique whose members all have label >= c; nodes are the components of at least two
 * r-cliques, labelled by the highest level at which they exist (= their least member label).
 * With core numbers as labels this is the core hierarchy; with the approximate values of
 * Alg. 2 it is the approximate hierarchy of §6 (which applies Alg. 1 to approximate values). */
orc_result* orc_label_hierarchy(int64_t n, const int64_t* off, const int32_t* adj, int r, int s,
                                const uint32_t* labels) {
  return nucleus_impl(n, off, adj, r, s, 0, ORC_HIER_DEF, 0.0, labels);
}

/* ------------------------------------------------------------------------------------------ */
/* local certificate on sampled r-cliques (for graphs too large for the full oracle)           */
/* ------------------------------------------------------------------------------------------ */

/* For each sampled r-clique R (ids in lexicographic order, the r-clique table given) enumerate
 * the s-cliques containing R directly from the definition and check a claimed result:
 *   bad[0] += cnt[R] differs from the number of s-cliques containing R
 *   bad[1] += fewer than core[R] s-cliques containing R have all members of core >= core[R]
 *             (then the set {core >= core[R]} would not be a core[R]-nucleus witness)
 *   bad[2] += more than core[R] s-cliques containing R have all members peeled no earlier than
 *             R (round[] = peel round); then R could not have been removed at level core[R]
 *   bad[3] += for an s-clique S containing R, the members' hierarchy nodes at level
 *             c_S = min core over S differ (parent[] over n_r leaves then nodes, label[] over nodes)
 * Arrays may be NULL to skip a check. */
int orc_check_sample(int64_t n, const int64_t* off, const int32_t* adj, int r, int s,
                     const int32_t* rtab, int64_t n_r, const int64_t* sample, int64_t n_sample,
                     const uint32_t* cnt, const uint32_t* core, const uint32_t* round,
                     const int32_t* parent, const uint32_t* label, int64_t* bad) {
  orc_graph g = {n, off, adj};
  int C = (int)binom(s, r);
  int combos[64 * ORC_MAX_K];
  if (r < 1 || s <= r || s > ORC_MAX_K || C > 64) return ORC_ERR_ARGS;
  make_combos(s, r, combos);
  int d = s - r;
  int32_t* W = NULL;
  int64_t wcap = 0;
  for (int q = 0; q < 4; q++) bad[q] = 0;
  for (int64_t si = 0; si < n_sample; si++) {
    int64_t R = sample[si];
    const int32_t* rv = rtab + R * r;
    /* candidates: common neighbours of R's vertices, scanning the shortest list */
    int best = 0;
    for (int i = 1; i < r; i++)
      if (off[rv[i] + 1] - off[rv[i]] < off[rv[best] + 1] - off[rv[best]]) best = i;
    int64_t deg = off[rv[best] + 1] - off[rv[best]];
    if (deg > wcap) { free(W); wcap = deg; W = malloc(sizeof(int32_t) * wcap); if (!W) return ORC_ERR_NOMEM; }
    int64_t nw = 0;
    for (int64_t j = off[rv[best]]; j < off[rv[best] + 1]; j++) {
      int32_t w = adj[j];
      int ok = 1;
      for (int i = 0; i < r && ok; i++) if (i != best) ok = adjacent(&g, rv[i], w);
      if (ok) W[nw++] = w;
    }
    /* d-cliques inside W, ascending index tuples */
    int64_t ix[ORC_MAX_K];
    int64_t n_found = 0, n_valid = 0, n_late = 0;
    int depth = 0;
    ix[0] = -1;
    while (depth >= 0) {
      ix[depth]++;
      if (ix[depth] >= nw) { depth--; continue; }
      int ok = 1;
      for (int i = 0; i < depth && ok; i++) ok = adjacent(&g, W[ix[i]], W[ix[depth]]);
      if (!ok) continue;
      if (depth + 1 < d) { depth++; ix[depth] = ix[depth - 1]; continue; }
      /* S = R plus W[ix[0..d)] */
      int32_t S[ORC_MAX_K];
      int ns = 0;
      for (int i = 0; i < r; i++) S[ns++] = rv[i];
      for (int i = 0; i < d; i++) S[ns++] = W[ix[i]];
      for (int i = 1; i < s; i++) { int32_t x = S[i]; int j = i - 1; while (j >= 0 && S[j] > x) { S[j + 1] = S[j]; j--; } S[j + 1] = x; }
      int64_t mid[64];
      for (int j = 0; j < C; j++) {
        int32_t key[ORC_MAX_K];
        for (int i = 0; i < r; i++) key[i] = S[combos[j * r + i]];
        mid[j] = tuple_id(rtab, n_r, r, key);
        if (mid[j] < 0) return ORC_ERR_ARGS;
      }
      n_found++;
      if (core) {
        int all_ge = 1;
        uint32_t cs = core[mid[0]];
        for (int j = 0; j < C; j++) { if (core[mid[j]] < core[R]) all_ge = 0; if (core[mid[j]] < cs) cs = core[mid[j]]; }
        n_valid += all_ge;
        if (parent && label) {
          int64_t node0 = -2;
          for (int j = 0; j < C; j++) {
            int64_t N = parent[mid[j]];
            while (N >= 0 && parent[n_r + N] >= 0 && label[parent[n_r + N]] >= cs) N = parent[n_r + N];
            if (N < 0 || label[N] < cs) { bad[3]++; break; }
            if (node0 == -2) node0 = N; else if (N != node0) { bad[3]++; break; }
          }
        }
      }
      if (round) {
        int late = 1;
        for (int j = 0; j < C; j++) if (round[mid[j]] < round[R]) late = 0;
        n_late += late;
      }
    }
    if (cnt && (int64_t)cnt[R] != n_found) bad[0]++;
    if (core && n_valid < (int64_t)core[R]) bad[1]++;
    if (core && round && n_late > (int64_t)core[R]) bad[2]++;
  }
  free(W);
  return ORC_OK;
}
