/*
 * certify.c -- local certificate of an exact (r,s) nucleus decomposition, for full-size checks.
 *
 * TEST INFRASTRUCTURE ONLY, like nucleus_oracle.c: loaded by the test suite, never by the CUDA
 * library, with which it shares no code, header, table or helper.
 *
 * The sequential oracle cannot enumerate the 2.3e9 4-cliques of the benchmark graph in test time.
 * This checker computes no decomposition; it verifies a claimed one (counts, core numbers, peel
 * rounds, hierarchy) against conditions that together determine it exactly.  With the paper's
 * definitions (§3: s-clique-degree, c-(r,s) nucleus, core number; the hierarchy of nuclei):
 *   C0 count:        cnt[R] = the number of s-cliques containing R.
 *   C1 validity:     every R with core[R] = c >= 1 lies in at least c s-cliques whose r-subsets
 *                    all have core >= c.  Then every member of X_c = {core >= c} lies in >= c
 *                    s-cliques inside X_c, so X_c is inside the union of the c-nuclei: the true
 *                    core is at least the claimed one.
 *   C2 peel order:   at most core[R] s-cliques containing R have all their members peeled no
 *                    earlier than R (round >= round[R]): the s-cliques still alive when R was
 *                    removed.  With core non-decreasing in round order (checked by the caller),
 *                    this removal order is a peel whose running maximum of removal degrees is the
 *                    claimed core (§6, Lemma 1's sequential peel): the true core is at most it.
 *   H1 under-merge:  for every s-clique S with c_S = min core over S >= 1, the leaf nodes of its
 *                    members have a common ancestor of label exactly c_S (they meet at level c_S).
 *   H2 over-merge:   every node X of label c is connected by the s-cliques of level exactly c:
 *                    its parts -- each child node, and each r-clique hanging directly from X --
 *                    end up in one set when every s-clique S with c_S = c unites the parts of X
 *                    that hold its members; and X has at least two parts.
 * C1 and C2 for every r-clique prove the core numbers.  H1 gives every level-c component (the
 * r-cliques of core >= c joined through the s-cliques of level >= c) inside one node, H2 gives
 * every node inside one component: together the tree is the definitional hierarchy.
 *
 * Enumeration: every s-clique once, from its vertex of least (degree, id) rank, by intersecting
 * sorted out-lists of that orientation (§3's low out-degree orientation); the members' ids come
 * from the lexicographic edge ids of the list positions (r = 2) or from a lookup in the
 * lexicographic triangle table (r = 3).  Threads (POSIX) take vertices in chunks, add to shared
 * counters with relaxed atomic adds and unite into their own union-finds, merged in one thread at
 * the end.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { CRT_OK = 0, CRT_ERR_ARGS = 1, CRT_ERR_NOMEM = 2 };

#define CRT_TREE_MAX 16384 /* largest node count whose LCA / child tables (nodes^2 ints) are built */

typedef struct {
  /* input */
  int64_t n;
  const int64_t* off;
  const int32_t* adj;
  int r, s, C;
  int64_t n_r;
  const uint32_t* cnt;
  const uint32_t* core;
  const uint32_t* round;
  const int32_t* parent; /* [n_r + nn]: leaf node of each r-clique, then parent of each node */
  const uint32_t* label; /* [nn] */
  int64_t nn;
  int tree;              /* hierarchy checks on */
  /* derived */
  int64_t* uoff;   /* first lexicographic edge id of each vertex */
  int32_t* eid;    /* lexicographic edge id of every adjacency entry */
  int64_t* ooff;   /* out-lists of the (degree, id) orientation, ascending vertex id */
  int32_t* oadj;
  int32_t* oeid;
  int64_t* tbase;  /* r = 3: per lexicographic edge (x,y), first id of the triangles {x,y,z}, z > y */
  int32_t* tz;     /*        and their z, ascending */
  int32_t* lca;    /* [nn * nn] lowest common ancestor of two nodes, or -1 */
  int32_t* child;  /* [nn * nn] child[X * nn + N]: the child of X on the path up from N, or -1 */
  /* output */
  uint32_t* count;
  uint32_t* valid;
  uint32_t* late;
  int64_t next_v;  /* work counter (atomic) */
  int64_t n_s;     /* s-cliques enumerated (atomic) */
  int64_t bad_h1;  /* (atomic) */
} crt_ctx;

/* ------------------------------------------------------------------------------------------ */

static int64_t crt_lower(const int32_t* a, int64_t lo, int64_t hi, int32_t x) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static int crt_rank_less(const crt_ctx* c, int32_t u, int32_t v) {
  int64_t du = c->off[u + 1] - c->off[u], dv = c->off[v + 1] - c->off[v];
  return du < dv || (du == dv && u < v);
}

static int32_t uf_find32(int32_t* p, int32_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

static void uf_unite32(int32_t* p, int32_t a, int32_t b) {
  a = uf_find32(p, a);
  b = uf_find32(p, b);
  if (a == b) return;
  if (a < b) p[b] = a; else p[a] = b;
}

/* lexicographic id of edge {x, y} (x != y, adjacent) */
static int64_t crt_edge(const crt_ctx* c, int32_t x, int32_t y) {
  if (x > y) { int32_t t = x; x = y; y = t; }
  int64_t p = crt_lower(c->adj, c->off[x], c->off[x + 1], y);
  return c->eid[p];
}

/* lexicographic id of triangle {x, y, z} given the id of the edge of its two smallest vertices */
static int64_t crt_tri(const crt_ctx* c, int64_t exy, int32_t z) {
  int64_t p = crt_lower(c->tz, c->tbase[exy], c->tbase[exy + 1], z);
  return (p < c->tbase[exy + 1] && c->tz[p] == z) ? p : -1;
}

static void crt_sort3(int32_t* a) {
  int32_t t;
  if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
  if (a[1] > a[2]) { t = a[1]; a[1] = a[2]; a[2] = t; }
  if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
}

/* the checks of one s-clique with member ids m[0..C) */
static void crt_visit(crt_ctx* c, const int64_t* m, int32_t* uf) {
  const int C = c->C;
  uint32_t cs = 0xffffffffu, rs = 0xffffffffu;
  for (int j = 0; j < C; j++) {
    __atomic_fetch_add(&c->count[m[j]], 1u, __ATOMIC_RELAXED);
    if (c->core && c->core[m[j]] < cs) cs = c->core[m[j]];
    if (c->round && c->round[m[j]] < rs) rs = c->round[m[j]];
  }
  for (int j = 0; j < C; j++) {
    if (c->core && c->core[m[j]] == cs) __atomic_fetch_add(&c->valid[m[j]], 1u, __ATOMIC_RELAXED);
    if (c->round && c->round[m[j]] == rs) __atomic_fetch_add(&c->late[m[j]], 1u, __ATOMIC_RELAXED);
  }
  if (!c->tree || !c->core || cs == 0) return;
  const int64_t nn = c->nn;
  int64_t X = c->parent[m[0]];
  for (int j = 1; j < C && X >= 0; j++) {
    const int64_t N = c->parent[m[j]];
    X = (N >= 0) ? c->lca[X * nn + N] : -1;
  }
  if (X < 0 || c->label[X] != cs) {
    __atomic_fetch_add(&c->bad_h1, 1, __ATOMIC_RELAXED);
    return;
  }
  int32_t p0 = -1;
  for (int j = 0; j < C; j++) {
    const int64_t N = c->parent[m[j]];
    const int32_t part = (N == X) ? (int32_t)m[j] : (int32_t)(c->n_r + c->child[X * nn + N]);
    if (j == 0) p0 = part; else uf_unite32(uf, p0, part);
  }
}

typedef struct {
  crt_ctx* c;
  int32_t* uf;
  int err;
} crt_thread;

static void* crt_worker(void* arg) {
  crt_thread* th = (crt_thread*)arg;
  crt_ctx* c = th->c;
  const int64_t chunk = 64;
  int64_t cap = 0;
  int32_t *c2v = NULL, *c2ev = NULL, *c2ea = NULL;
  for (;;) {
    const int64_t v0 = __atomic_fetch_add(&c->next_v, chunk, __ATOMIC_RELAXED);
    if (v0 >= c->n) break;
    const int64_t v1 = v0 + chunk < c->n ? v0 + chunk : c->n;
    for (int64_t vv = v0; vv < v1; vv++) {
      const int32_t v = (int32_t)vv;
      const int64_t vb = c->ooff[v], ve = c->ooff[v + 1];
      if (ve - vb > cap) {
        cap = ve - vb;
        free(c2v); free(c2ev); free(c2ea);
        c2v = malloc(sizeof(int32_t) * cap);
        c2ev = malloc(sizeof(int32_t) * cap);
        c2ea = malloc(sizeof(int32_t) * cap);
        if (!c2v || !c2ev || !c2ea) { th->err = CRT_ERR_NOMEM; goto done; }
      }
      for (int64_t ia = vb; ia < ve; ia++) {
        const int32_t a = c->oadj[ia], e_va = c->oeid[ia];
        int64_t m[6];
        if (c->s == 2) {
          if (c->r == 1) { m[0] = v; m[1] = a; }
          crt_visit(c, m, th->uf);
          __atomic_fetch_add(&c->n_s, 1, __ATOMIC_RELAXED);
          continue;
        }
        /* C2 = N+(v) n N+(a), with the edge ids to v and to a */
        int64_t k2 = 0;
        {
          int64_t i = vb, j = c->ooff[a];
          const int64_t je = c->ooff[a + 1];
          while (i < ve && j < je) {
            if (c->oadj[i] < c->oadj[j]) i++;
            else if (c->oadj[i] > c->oadj[j]) j++;
            else { c2v[k2] = c->oadj[i]; c2ev[k2] = c->oeid[i]; c2ea[k2] = c->oeid[j]; k2++; i++; j++; }
          }
        }
        int64_t found = 0;
        for (int64_t k = 0; k < k2; k++) {
          const int32_t b = c2v[k];
          const int32_t e_vb = c2ev[k], e_ab = c2ea[k];
          if (c->s == 3) {
            if (c->r == 1) { m[0] = v; m[1] = a; m[2] = b; }
            else { m[0] = e_va; m[1] = e_vb; m[2] = e_ab; }
            crt_visit(c, m, th->uf);
            found++;
            continue;
          }
          /* s = 4: c in C2 n N+(b) */
          int64_t i = 0, j = c->ooff[b];
          const int64_t je = c->ooff[b + 1];
          while (i < k2 && j < je) {
            if (c2v[i] < c->oadj[j]) i++;
            else if (c2v[i] > c->oadj[j]) j++;
            else {
              const int32_t x = c2v[i];
              const int32_t e_vx = c2ev[i], e_ax = c2ea[i], e_bx = c->oeid[j];
              if (c->r == 1) {
                m[0] = v; m[1] = a; m[2] = b; m[3] = x;
              } else if (c->r == 2) {
                m[0] = e_va; m[1] = e_vb; m[2] = e_vx; m[3] = e_ab; m[4] = e_ax; m[5] = e_bx;
              } else {
                /* the four triangles; each keyed by the edge of its two smallest vertices */
                const int32_t tv[4][3] = {{v, a, b}, {v, a, x}, {v, b, x}, {a, b, x}};
                for (int q = 0; q < 4; q++) {
                  int32_t t3[3] = {tv[q][0], tv[q][1], tv[q][2]};
                  crt_sort3(t3);
                  m[q] = crt_tri(c, crt_edge(c, t3[0], t3[1]), t3[2]);
                  if (m[q] < 0) { th->err = CRT_ERR_ARGS; goto done; }
                }
              }
              crt_visit(c, m, th->uf);
              found++;
              i++;
              j++;
            }
          }
        }
        __atomic_fetch_add(&c->n_s, found, __ATOMIC_RELAXED);
      }
    }
  }
done:
  free(c2v); free(c2ev); free(c2ea);
  return NULL;
}

/* r = 3 triangle table: per lexicographic edge (x,y) the z > y adjacent to both, ascending */
typedef struct {
  crt_ctx* c;
  int64_t e0, e1;
  int64_t* cntz;
  int fill;
} crt_tri_job;

static void* crt_tri_worker(void* arg) {
  crt_tri_job* jb = (crt_tri_job*)arg;
  crt_ctx* c = jb->c;
  for (int64_t x = 0; x < c->n; x++) {
    const int64_t ub = crt_lower(c->adj, c->off[x], c->off[x + 1], (int32_t)x + 1);
    for (int64_t q = ub; q < c->off[x + 1]; q++) {
      const int64_t e = c->eid[q];
      if (e < jb->e0 || e >= jb->e1) continue;
      const int32_t y = c->adj[q];
      const int64_t yb = crt_lower(c->adj, c->off[y], c->off[y + 1], y + 1);
      const int64_t xb = crt_lower(c->adj, c->off[x], c->off[x + 1], y + 1);
      int64_t k = 0, i = xb, j = yb;
      while (i < c->off[x + 1] && j < c->off[y + 1]) {
        if (c->adj[i] < c->adj[j]) i++;
        else if (c->adj[i] > c->adj[j]) j++;
        else {
          if (jb->fill) c->tz[c->tbase[e] + k] = c->adj[i];
          k++; i++; j++;
        }
      }
      if (!jb->fill) jb->cntz[e] = k;
    }
  }
  return NULL;
}

static int crt_run_threads(void* (*fn)(void*), void* jobs, size_t job_size, int threads) {
  pthread_t* t = malloc(sizeof(pthread_t) * (size_t)threads);
  if (!t) return CRT_ERR_NOMEM;
  int started = 0;
  for (int i = 0; i < threads; i++) {
    if (pthread_create(&t[i], NULL, fn, (char*)jobs + job_size * (size_t)i) != 0) break;
    started++;
  }
  for (int i = 0; i < started; i++) pthread_join(t[i], NULL);
  free(t);
  if (started == 0) return CRT_ERR_NOMEM;
  /* jobs that did not get a thread run here */
  for (int i = started; i < threads; i++) fn((char*)jobs + job_size * (size_t)i);
  return CRT_OK;
}

/* out[0..7]: C0 violations, C1 violations, C2 violations, H1 violations, H2 violations,
 * hierarchy checked (0/1), s-cliques enumerated, nodes with fewer than two parts (counted in H2
 * too).  cnt / core / round / parent+label may be NULL to skip their checks. */
int crt_certify(int64_t n, const int64_t* off, const int32_t* adj, int r, int s, int64_t n_r,
                const uint32_t* cnt, const uint32_t* core, const uint32_t* round, const int32_t* parent,
                const uint32_t* label, int64_t nn, int threads, int64_t* out) {
  if (n < 1 || r < 1 || r > 3 || s <= r || s > 4 || threads < 1) return CRT_ERR_ARGS;
  crt_ctx cx;
  memset(&cx, 0, sizeof(cx));
  crt_ctx* c = &cx;
  c->n = n; c->off = off; c->adj = adj; c->r = r; c->s = s;
  c->C = (r == 1) ? s : (r == 2) ? (s == 3 ? 3 : 6) : 4;
  c->n_r = n_r; c->cnt = cnt; c->core = core; c->round = round;
  c->parent = parent; c->label = label; c->nn = nn;
  c->tree = (parent && label && core && nn >= 0 && nn <= CRT_TREE_MAX) ? 1 : 0;
  for (int q = 0; q < 8; q++) out[q] = 0;
  int rc = CRT_OK;
  const int64_t nnz = off[n];
  crt_thread* th = NULL;
  crt_tri_job* jobs = NULL;
  /* lexicographic edge ids of every adjacency entry */
  c->uoff = malloc(sizeof(int64_t) * (size_t)(n + 1));
  c->eid = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  c->ooff = malloc(sizeof(int64_t) * (size_t)(n + 1));
  c->oadj = malloc(sizeof(int32_t) * (size_t)(nnz / 2 + 1));
  c->oeid = malloc(sizeof(int32_t) * (size_t)(nnz / 2 + 1));
  c->count = calloc((size_t)(n_r > 0 ? n_r : 1), sizeof(uint32_t));
  c->valid = calloc((size_t)(n_r > 0 ? n_r : 1), sizeof(uint32_t));
  c->late = calloc((size_t)(n_r > 0 ? n_r : 1), sizeof(uint32_t));
  if (!c->uoff || !c->eid || !c->ooff || !c->oadj || !c->oeid || !c->count || !c->valid || !c->late) {
    rc = CRT_ERR_NOMEM;
    goto out;
  }
  c->uoff[0] = 0;
  for (int64_t u = 0; u < n; u++) {
    const int64_t ub = crt_lower(adj, off[u], off[u + 1], (int32_t)u + 1);
    c->uoff[u + 1] = c->uoff[u] + (off[u + 1] - ub);
  }
  for (int64_t u = 0; u < n; u++) {
    const int64_t ub = crt_lower(adj, off[u], off[u + 1], (int32_t)u + 1);
    for (int64_t q = off[u]; q < off[u + 1]; q++) {
      const int32_t w = adj[q];
      if (q >= ub) c->eid[q] = (int32_t)(c->uoff[u] + (q - ub));
      else {
        const int64_t p = crt_lower(adj, off[w], off[w + 1], (int32_t)u);
        const int64_t wb = crt_lower(adj, off[w], off[w + 1], w + 1);
        c->eid[q] = (int32_t)(c->uoff[w] + (p - wb));
      }
    }
  }
  if (r == 2 && n_r != c->uoff[n]) { rc = CRT_ERR_ARGS; goto out; }
  if (r == 1 && n_r != n) { rc = CRT_ERR_ARGS; goto out; }
  /* orientation */
  c->ooff[0] = 0;
  for (int64_t u = 0; u < n; u++) {
    int64_t k = 0;
    for (int64_t q = off[u]; q < off[u + 1]; q++) k += crt_rank_less(c, (int32_t)u, adj[q]);
    c->ooff[u + 1] = c->ooff[u] + k;
  }
  for (int64_t u = 0; u < n; u++) {
    int64_t k = c->ooff[u];
    for (int64_t q = off[u]; q < off[u + 1]; q++)
      if (crt_rank_less(c, (int32_t)u, adj[q])) { c->oadj[k] = adj[q]; c->oeid[k] = c->eid[q]; k++; }
  }
  /* r = 3: lexicographic triangle table */
  if (r == 3) {
    const int64_t m = c->uoff[n];
    int64_t* cz = calloc((size_t)(m > 0 ? m : 1), sizeof(int64_t));
    c->tbase = malloc(sizeof(int64_t) * (size_t)(m + 1));
    jobs = malloc(sizeof(crt_tri_job) * (size_t)threads);
    if (!cz || !c->tbase || !jobs) { free(cz); rc = CRT_ERR_NOMEM; goto out; }
    for (int pass = 0; pass < 2; pass++) {
      for (int i = 0; i < threads; i++) {
        jobs[i].c = c; jobs[i].cntz = cz; jobs[i].fill = pass;
        jobs[i].e0 = m * i / threads; jobs[i].e1 = m * (i + 1) / threads;
      }
      if ((rc = crt_run_threads(crt_tri_worker, jobs, sizeof(crt_tri_job), threads))) { free(cz); goto out; }
      if (pass == 0) {
        c->tbase[0] = 0;
        for (int64_t e = 0; e < m; e++) c->tbase[e + 1] = c->tbase[e] + cz[e];
        if (c->tbase[m] != n_r) { free(cz); rc = CRT_ERR_ARGS; goto out; }
        c->tz = malloc(sizeof(int32_t) * (size_t)(n_r > 0 ? n_r : 1));
        if (!c->tz) { free(cz); rc = CRT_ERR_NOMEM; goto out; }
      }
    }
    free(cz);
  }
  /* hierarchy tables: nodes in ascending label order (a parent's label is below its child's) */
  if (c->tree && nn > 0) {
    for (int64_t x = 0; x < nn; x++) {
      const int32_t p = parent[n_r + x];
      if (p >= nn || (p >= 0 && label[p] >= label[x])) { c->tree = 0; out[3] = -1; break; }
    }
  }
  if (c->tree && nn > 0) {
    c->lca = malloc(sizeof(int32_t) * (size_t)(nn * nn));
    c->child = malloc(sizeof(int32_t) * (size_t)(nn * nn));
    int32_t* order = malloc(sizeof(int32_t) * (size_t)nn);
    uint8_t* anc = calloc((size_t)nn, 1);
    if (!c->lca || !c->child || !order || !anc) { free(order); free(anc); rc = CRT_ERR_NOMEM; goto out; }
    for (int64_t x = 0; x < nn; x++) order[x] = (int32_t)x;
    /* insertion-free ordering: counting sort by label */
    {
      uint32_t lmax = 0;
      for (int64_t x = 0; x < nn; x++) if (label[x] > lmax) lmax = label[x];
      int64_t* b = calloc((size_t)lmax + 2, sizeof(int64_t));
      if (!b) { free(order); free(anc); rc = CRT_ERR_NOMEM; goto out; }
      for (int64_t x = 0; x < nn; x++) b[label[x] + 1]++;
      for (uint32_t l = 0; l <= lmax; l++) b[l + 1] += b[l];
      for (int64_t x = 0; x < nn; x++) order[b[label[x]]++] = (int32_t)x;
      free(b);
    }
    for (int64_t a = 0; a < nn; a++) {
      for (int64_t y = a; y >= 0; y = parent[n_r + y]) anc[y] = 1;
      int32_t* row = c->lca + a * nn;
      for (int64_t i = 0; i < nn; i++) {
        const int32_t b = order[i];
        const int32_t pb = parent[n_r + b];
        row[b] = anc[b] ? b : (pb >= 0 ? row[pb] : -1);
      }
      for (int64_t y = a; y >= 0; y = parent[n_r + y]) anc[y] = 0;
    }
    for (int64_t i = 0; i < nn * nn; i++) c->child[i] = -1;
    for (int64_t N = 0; N < nn; N++) {
      int64_t prev = N;
      for (int64_t y = parent[n_r + N]; y >= 0; y = parent[n_r + y]) {
        c->child[y * nn + N] = (int32_t)prev;
        prev = y;
      }
    }
    free(order);
    free(anc);
  }
  /* enumeration */
  th = calloc((size_t)threads, sizeof(crt_thread));
  if (!th) { rc = CRT_ERR_NOMEM; goto out; }
  const int64_t nparts = n_r + (nn > 0 ? nn : 0);
  for (int i = 0; i < threads; i++) {
    th[i].c = c;
    if (c->tree) {
      th[i].uf = malloc(sizeof(int32_t) * (size_t)(nparts > 0 ? nparts : 1));
      if (!th[i].uf) { rc = CRT_ERR_NOMEM; goto out; }
      for (int64_t x = 0; x < nparts; x++) th[i].uf[x] = (int32_t)x;
    }
  }
  if ((rc = crt_run_threads(crt_worker, th, sizeof(crt_thread), threads))) goto out;
  for (int i = 0; i < threads; i++) if (th[i].err) { rc = th[i].err; goto out; }
  out[6] = c->n_s;
  for (int64_t R = 0; R < n_r; R++) {
    if (cnt && c->count[R] != cnt[R]) out[0]++;
    if (core && c->valid[R] < core[R]) out[1]++;
    if (core && round && c->late[R] > core[R]) out[2]++;
  }
  if (c->tree) {
    out[5] = 1;
    out[3] += c->bad_h1;
    /* one union-find: thread 0's, with every other thread's sets added */
    int32_t* g = th[0].uf;
    for (int i = 1; i < threads; i++)
      for (int64_t x = 0; x < nparts; x++)
        if (th[i].uf[x] != x) uf_unite32(g, (int32_t)x, uf_find32(th[i].uf, (int32_t)x));
    int32_t* rep = malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    int64_t* parts = calloc((size_t)(nn > 0 ? nn : 1), sizeof(int64_t));
    if (!rep || !parts) { free(rep); free(parts); rc = CRT_ERR_NOMEM; goto out; }
    for (int64_t x = 0; x < nn; x++) rep[x] = -1;
    for (int64_t p = 0; p < nparts; p++) {
      /* part p belongs to node X: an r-clique to its leaf node, a node to its parent */
      const int64_t X = (p < n_r) ? parent[p] : parent[p];
      if (X < 0) continue;
      parts[X]++;
      const int32_t rt = uf_find32(g, (int32_t)p);
      if (rep[X] < 0) rep[X] = rt;
      else if (rep[X] != rt) out[4]++;
    }
    for (int64_t x = 0; x < nn; x++)
      if (parts[x] < 2) { out[4]++; out[7]++; }
    free(rep);
    free(parts);
  }
out:
  if (th) {
    for (int i = 0; i < threads; i++) free(th[i].uf);
    free(th);
  }
  free(jobs);
  free(c->uoff); free(c->eid); free(c->ooff); free(c->oadj); free(c->oeid);
  free(c->tbase); free(c->tz); free(c->lca); free(c->child);
  free(c->count); free(c->valid); free(c->late);
  return rc;
}
