/*
 * oracle/oracle.c -- CPU oracle for k-clique and k-motif counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against an
 * independent, obviously correct computation.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * What is computed (Sec. 2.1 "Graph Pattern Mining", Sec. 2.2): the method
 * of the paper is exact, so the oracle computes the plain definitions:
 *   - k-clique count: the number of k-vertex subsets whose vertices are
 *     pairwise adjacent (Sec. 2.2, footnote on complete subgraphs).
 *   - k-motif counts: for each isomorphism class of connected k-vertex
 *     graphs, the number of k-vertex subsets S whose vertex-induced
 *     subgraph G[S] is connected and in that class, each subset counted
 *     once (vertex-induced embeddings, Sec. 2.1; canonical/duplicate-free
 *     counting, Sec. 2.1 and Sec. 3.2; support = count, Listing 4).
 * Motif output order (fixed here, since the paper's motif figure is not
 * available): k=3 -> [wedge, triangle]; k=4 -> [3-star, 4-path,
 * tailed-triangle, 4-cycle, diamond, 4-clique]; k=5 -> the 21 connected
 * graphs on 5 vertices ordered by edge count, then by the degree sequence
 * (sorted non-increasing, compared lexicographically, smaller first), then
 * by the canonical code (the smallest 10-bit adjacency code over the 120
 * relabellings; bit i = pair i of (0,1),(0,2),(0,3),(0,4),(1,2),(1,3),
 * (1,4),(2,3),(2,4),(3,4)).
 *
 * Tiers (all single-threaded unless `nthreads` > 1, in which case roots
 * are split across OpenMP threads and the integer partial sums added):
 *   orc_bf_*        brute force over all k-subsets of a graph with n <= 64.
 *   orc_clique_*    plain depth-first clique enumerator; candidates of the
 *                   next depth = current candidates intersected with the
 *                   later neighbours of the chosen vertex (two-pointer
 *                   merge).  Order either by vertex ID or by (degree, ID).
 *   orc_esu_motifs  ESU enumeration (Wernicke, "Efficient detection of
 *                   network motifs", 2006): every connected k-set is
 *                   generated exactly once from its minimum vertex.
 *   orc_fsm         frequent subgraph mining (edge-induced, vertex labels,
 *                   MNI support, 1..3 edges): every connected edge set
 *                   enumerated once by its shape; orc_fsm_bf_support is the
 *                   matching-based MNI definition for tiny graphs.
 *   orc_formula_motifs  count special patterns directly, derive the rest
 *                   from the relationships among patterns (the "eliding
 *                   isomorphism test" idea of Sec. 2.2, PGD-style):
 *                   non-induced counts from degrees, per-edge triangle
 *                   counts, 4-cycles (Chiba-Nishizeki rank-ordered wedges)
 *                   and 4-cliques, then the induced counts by inverting the
 *                   containment matrix.  Intermediates are 128-bit.
 *
 * Input format (Sec. 6.1): CSR of a simple undirected graph, int64 row
 * pointers, int32 neighbour IDs sorted ascending, symmetric, no loops.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-3)
#define ORC_EOVERFLOW (-6)

/* ------------------------------------------------------------ helpers */
static int adjacent(const int64_t *rp, const int32_t *col, int32_t u, int32_t v) {
  int64_t lo = rp[u], hi = rp[u + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo < rp[u + 1] && col[lo] == v;
}

static int popcount64(uint64_t x) { return __builtin_popcountll(x); }

/* Classify a connected 3- or 4-vertex induced subgraph from its edge count
 * and maximum degree.  3 vertices: 2 edges -> wedge, 3 -> triangle.
 * 4 vertices: 3 edges -> star (max degree 3) or path; 4 edges -> tailed
 * triangle (max degree 3) or 4-cycle; 5 -> diamond; 6 -> clique. */
static int classify(int k, int edges, int maxdeg) {
  if (k == 3) return edges == 3 ? 1 : 0;
  switch (edges) {
    case 3: return maxdeg == 3 ? 0 : 1;
    case 4: return maxdeg == 3 ? 2 : 3;
    case 5: return 4;
    case 6: return 5;
  }
  return -1;
}

/* Exclusive prefix sum, the allocation step of inspection-execution
 * (Sec. 5.3): out[i] = sum of cnt[0..i-1]; out[len] = total. */
/* --------------------------------------------- 5-vertex isomorphism classes */
static const int P5[10][2] = {{0, 1}, {0, 2}, {0, 3}, {0, 4}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}};
static int16_t g_p5_class[1024]; /* adjacency code -> class (-1: disconnected) */
static int g_p5_ready = 0;

static int p5_adj(int code, int a, int b) {
  for (int i = 0; i < 10; i++)
    if ((P5[i][0] == a && P5[i][1] == b) || (P5[i][0] == b && P5[i][1] == a)) return (code >> i) & 1;
  return 0;
}

static int p5_connected(int code) {
  int seen = 1, grew = 1;
  while (grew) {
    grew = 0;
    for (int a = 0; a < 5; a++)
      if (seen & (1 << a))
        for (int b = 0; b < 5; b++)
          if (!(seen & (1 << b)) && p5_adj(code, a, b)) {
            seen |= 1 << b;
            grew = 1;
          }
  }
  return seen == 31;
}

/* smallest code over all 120 relabellings (perm[v] = new label of v) */
static int p5_canon(int code) {
  int best = 1 << 10, perm[5] = {0, 1, 2, 3, 4};
  /* iterate permutations in lexicographic order */
  for (;;) {
    int c = 0;
    for (int i = 0; i < 10; i++)
      if (p5_adj(code, P5[i][0], P5[i][1])) {
        int a = perm[P5[i][0]], b = perm[P5[i][1]];
        for (int j = 0; j < 10; j++)
          if ((P5[j][0] == a && P5[j][1] == b) || (P5[j][0] == b && P5[j][1] == a)) c |= 1 << j;
      }
    if (c < best) best = c;
    int i = 3;
    while (i >= 0 && perm[i] > perm[i + 1]) i--;
    if (i < 0) break;
    int j = 4;
    while (perm[j] < perm[i]) j--;
    int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    for (int a = i + 1, b = 4; a < b; a++, b--) { t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
  }
  return best;
}

/* sort key of a class: edges, then the degree sequence (non-increasing)
 * lexicographically, then the canonical code */
static void p5_key(int code, int key[7]) {
  int deg[5] = {0, 0, 0, 0, 0}, e = 0;
  for (int i = 0; i < 10; i++)
    if ((code >> i) & 1) { deg[P5[i][0]]++; deg[P5[i][1]]++; e++; }
  for (int a = 0; a < 5; a++)
    for (int b = a + 1; b < 5; b++)
      if (deg[b] > deg[a]) { int t = deg[a]; deg[a] = deg[b]; deg[b] = t; }
  key[0] = e;
  for (int a = 0; a < 5; a++) key[1 + a] = deg[a];
  key[6] = code;
}

static int p5_key_cmp(const void *x, const void *y) {
  int kx[7], ky[7];
  p5_key(*(const int *)x, kx);
  p5_key(*(const int *)y, ky);
  for (int i = 0; i < 7; i++)
    if (kx[i] != ky[i]) return kx[i] < ky[i] ? -1 : 1;
  return 0;
}

static void p5_init(void) {
  if (g_p5_ready) return;
  int canon[1024], classes[64], nc = 0;
  for (int c = 0; c < 1024; c++) {
    canon[c] = p5_connected(c) ? p5_canon(c) : -1;
    if (canon[c] >= 0 && canon[c] == c) classes[nc++] = c; /* a canonical code is its own class's minimum */
  }
  qsort(classes, (size_t)nc, sizeof(int), p5_key_cmp);
  for (int c = 0; c < 1024; c++) {
    g_p5_class[c] = -1;
    for (int i = 0; i < nc; i++)
      if (canon[c] == classes[i]) g_p5_class[c] = (int16_t)i;
  }
  g_p5_ready = 1;
}

/* number of classes and their canonical codes, in output order (tests) */
int orc_p5_classes(int32_t *codes) {
  p5_init();
  int n = 0;
  for (int c = 0; c < 1024; c++)
    if (g_p5_class[c] >= 0 && p5_canon(c) == c) codes[g_p5_class[c]] = c, n++;
  return n;
}

void orc_exclusive_scan(int64_t len, const int64_t *cnt, int64_t *out) {
  int64_t s = 0;
  for (int64_t i = 0; i < len; i++) {
    out[i] = s;
    s += cnt[i];
  }
  out[len] = s;
}

/* Connectivity of candidate u to each vertex of an embedding (Sec. 5.4,
 * binary-search connectivity check): bit j set iff emb[j] is in N(u). */
uint32_t orc_connectivity_mask(const int64_t *rp, const int32_t *col, int32_t k,
                               const int32_t *emb, int32_t u) {
  uint32_t m = 0;
  for (int32_t j = 0; j < k; j++)
    if (adjacent(rp, col, u, emb[j])) m |= 1u << j;
  return m;
}

/* ------------------------------------------------------ brute force */
/* Adjacency bit rows of a graph with n <= 64. */
static int bits_from_csr(int32_t n, const int64_t *rp, const int32_t *col, uint64_t *adj) {
  if (n < 0 || n > 64) return ORC_EINVAL;
  for (int32_t v = 0; v < n; v++) {
    adj[v] = 0;
    for (int64_t a = rp[v]; a < rp[v + 1]; a++) adj[v] |= 1ULL << col[a];
  }
  return ORC_OK;
}

static int connected_bits(const uint64_t *adj, uint64_t set) {
  if (!set) return 0;
  uint64_t seen = set & (~set + 1); /* lowest vertex */
  for (;;) {
    uint64_t grow = seen;
    for (uint64_t s = seen; s; s &= s - 1) grow |= adj[__builtin_ctzll(s)] & set;
    if (grow == seen) break;
    seen = grow;
  }
  return seen == set;
}

/* visit every k-subset of [0, n) in lexicographic order */
typedef void (*subset_fn)(const uint64_t *adj, uint64_t set, void *ctx);
static void for_subsets(int32_t n, int32_t k, int32_t start, uint64_t set, int32_t left,
                        const uint64_t *adj, subset_fn fn, void *ctx) {
  if (left == 0) { fn(adj, set, ctx); return; }
  for (int32_t v = start; v <= n - left; v++)
    for_subsets(n, k, v + 1, set | (1ULL << v), left - 1, adj, fn, ctx);
}

static void bf_clique_visit(const uint64_t *adj, uint64_t set, void *ctx) {
  for (uint64_t s = set; s; s &= s - 1) {
    int v = __builtin_ctzll(s);
    if ((adj[v] & set) != (set & ~(1ULL << v))) return;
  }
  (*(uint64_t *)ctx)++;
}

typedef struct { int k; uint64_t cnt[21]; } bf_motif_ctx;
static void bf_motif_visit(const uint64_t *adj, uint64_t set, void *vctx) {
  bf_motif_ctx *c = (bf_motif_ctx *)vctx;
  if (!connected_bits(adj, set)) return;
  if (c->k == 5) {
    int v[5], nv = 0, code = 0;
    for (uint64_t s = set; s; s &= s - 1) v[nv++] = __builtin_ctzll(s);
    for (int i = 0; i < 10; i++)
      if ((adj[v[P5[i][0]]] >> v[P5[i][1]]) & 1) code |= 1 << i;
    c->cnt[g_p5_class[code]]++;
    return;
  }
  int deg_sum = 0, maxdeg = 0;
  for (uint64_t s = set; s; s &= s - 1) {
    int d = popcount64(adj[__builtin_ctzll(s)] & set);
    deg_sum += d;
    if (d > maxdeg) maxdeg = d;
  }
  int p = classify(c->k, deg_sum / 2, maxdeg);
  if (p >= 0) c->cnt[p]++;
}

/* Number of k-cliques by checking every k-subset (n <= 64, 1 <= k <= 8). */
int orc_bf_cliques(int32_t n, const int64_t *rp, const int32_t *col, int32_t k, uint64_t *out) {
  uint64_t adj[64];
  if (k < 1 || k > 8 || bits_from_csr(n, rp, col, adj)) return ORC_EINVAL;
  uint64_t c = 0;
  if (k <= n) for_subsets(n, k, 0, 0, k, adj, bf_clique_visit, &c);
  *out = c;
  return ORC_OK;
}

/* Motif counts by checking every k-subset (n <= 64, k in {3, 4, 5}). */
int orc_bf_motifs(int32_t n, const int64_t *rp, const int32_t *col, int32_t k, uint64_t *out) {
  uint64_t adj[64];
  if ((k < 3 || k > 5) || bits_from_csr(n, rp, col, adj)) return ORC_EINVAL;
  p5_init();
  bf_motif_ctx c;
  memset(&c, 0, sizeof(c));
  c.k = k;
  if (k <= n) for_subsets(n, k, 0, 0, k, adj, bf_motif_visit, &c);
  memcpy(out, c.cnt, sizeof(uint64_t) * (k == 3 ? 2 : k == 4 ? 6 : 21));
  return ORC_OK;
}

/* ---------------------------------------------- clique enumerator */
/* Later neighbours of v under a total order given by key[] (ascending),
 * each list kept in ascending ID order so that lists merge directly. */
typedef struct {
  int64_t *rp;
  int32_t *col;
} later_lists;

static int build_later(int32_t n, const int64_t *rp, const int32_t *col, const int64_t *key,
                       later_lists *L) {
  L->rp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  int64_t na = rp[n];
  L->col = (int32_t *)malloc((size_t)(na ? na : 1) * sizeof(int32_t));
  if (!L->rp || !L->col) return ORC_ENOMEM;
  int64_t w = 0;
  for (int32_t v = 0; v < n; v++) {
    L->rp[v] = w;
    for (int64_t a = rp[v]; a < rp[v + 1]; a++) {
      int32_t u = col[a];
      if (key[u] > key[v]) L->col[w++] = u;
    }
  }
  L->rp[n] = w;
  return ORC_OK;
}

/* sorted two-pointer intersection; returns the output length */
static int64_t merge_intersect(const int32_t *a, int64_t na, const int32_t *b, int64_t nb,
                               int32_t *out) {
  int64_t i = 0, j = 0, w = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else { out[w++] = a[i]; i++; j++; }
  }
  return w;
}

/* depth-first extension: cand holds the common later neighbours of the
 * current clique of size `depth`; each of them extends it to a
 * (depth+1)-clique.  scratch holds one list per remaining depth. */
static void clique_dfs(const later_lists *L, int32_t k, int32_t depth, const int32_t *cand,
                       int64_t nc, int32_t *scratch, int64_t scratch_stride, u128 *per_level) {
  per_level[depth + 1] += (u128)nc;
  if (depth + 1 >= k) return;
  for (int64_t i = 0; i < nc; i++) {
    int32_t u = cand[i];
    int64_t nn = merge_intersect(cand, nc, L->col + L->rp[u], L->rp[u + 1] - L->rp[u], scratch);
    clique_dfs(L, k, depth + 1, scratch, nn, scratch + scratch_stride, scratch_stride, per_level);
  }
}

/* Count l-cliques for l = 1..k whose first vertex (in the chosen order)
 * is in [root_lo, root_hi).  order = 0: by vertex ID; order = 1: by
 * (degree, ID).  per_level must hold k+1 entries (index 0 unused). */
int orc_clique_count(int32_t n, const int64_t *rp, const int32_t *col, int32_t k, int32_t order,
                     int32_t root_lo, int32_t root_hi, int32_t nthreads, uint64_t *per_level) {
  if (k < 1 || k > 16 || n < 0 || root_lo < 0 || root_hi > n || root_lo > root_hi)
    return ORC_EINVAL;
  int64_t *key = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!key) return ORC_ENOMEM;
  for (int32_t v = 0; v < n; v++)
    key[v] = order ? (((rp[v + 1] - rp[v]) << 32) | (int64_t)v) : (int64_t)v;
  later_lists L;
  int rc = build_later(n, rp, col, key, &L);
  free(key);
  if (rc) { free(L.rp); free(L.col); return rc; }
  int64_t dmax = 0;
  for (int32_t v = 0; v < n; v++)
    if (L.rp[v + 1] - L.rp[v] > dmax) dmax = L.rp[v + 1] - L.rp[v];
  u128 total[17];
  memset(total, 0, sizeof(total));
  if (nthreads < 1) nthreads = 1;
  int failed = 0;
#pragma omp parallel num_threads(nthreads)
  {
    u128 mine[17];
    memset(mine, 0, sizeof(mine));
    int32_t *scratch = (int32_t *)malloc((size_t)(dmax + 1) * (size_t)(k + 1) * sizeof(int32_t));
    if (!scratch) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int32_t v = root_lo; v < root_hi; v++) {
        mine[1] += 1;
        if (k >= 2)
          clique_dfs(&L, k, 1, L.col + L.rp[v], L.rp[v + 1] - L.rp[v], scratch, dmax + 1, mine);
      }
      free(scratch);
    }
#pragma omp critical
    for (int l = 0; l <= k; l++) total[l] += mine[l];
  }
  free(L.rp);
  free(L.col);
  if (failed) return ORC_ENOMEM;
  for (int l = 0; l <= k; l++) {
    if (total[l] > (u128)UINT64_MAX) return ORC_EOVERFLOW;
    per_level[l] = (uint64_t)total[l];
  }
  return ORC_OK;
}

/* --------------------------------------------------------------- ESU */
typedef struct {
  const int64_t *rp;
  const int32_t *col;
  int32_t k;
  int32_t root;
  int32_t sub[8];
  int32_t nsub;
  u128 cnt[21];
} esu_ctx;

static int in_list(const int32_t *a, int32_t len, int32_t x) {
  for (int32_t i = 0; i < len; i++)
    if (a[i] == x) return 1;
  return 0;
}

static void esu_leaf(esu_ctx *c) {
  if (c->k == 5) {
    int code = 0;
    for (int i = 0; i < 10; i++)
      if (adjacent(c->rp, c->col, c->sub[P5[i][0]], c->sub[P5[i][1]])) code |= 1 << i;
    c->cnt[g_p5_class[code]] += 1;
    return;
  }
  int deg[8] = {0}, edges = 0, maxdeg = 0;
  for (int i = 0; i < c->k; i++)
    for (int j = i + 1; j < c->k; j++)
      if (adjacent(c->rp, c->col, c->sub[i], c->sub[j])) {
        deg[i]++; deg[j]++; edges++;
      }
  for (int i = 0; i < c->k; i++)
    if (deg[i] > maxdeg) maxdeg = deg[i];
  int p = classify(c->k, edges, maxdeg);
  if (p >= 0) c->cnt[p] += 1;
}

/* ExtendSubgraph(V_sub, V_ext, root) of ESU: pick w out of V_ext in turn;
 * the new extension set is the rest of V_ext plus the exclusive
 * neighbours of w (greater than the root, not in V_sub, and not adjacent
 * to any vertex of V_sub). */
static void esu_extend(esu_ctx *c, const int32_t *ext, int64_t next) {
  if (c->nsub == c->k) { esu_leaf(c); return; }
  int64_t cap = next;
  for (int64_t i = 0; i < next; i++) {
    int32_t w = ext[i];
    cap += c->rp[w + 1] - c->rp[w];
  }
  int32_t *ext2 = (int32_t *)malloc((size_t)(cap ? cap : 1) * sizeof(int32_t));
  if (!ext2) abort();
  for (int64_t i = 0; i < next; i++) {
    int32_t w = ext[i];
    /* V_ext' = remaining V_ext (those after w) + N_excl(w, V_sub) */
    int64_t n2 = 0;
    for (int64_t j = i + 1; j < next; j++) ext2[n2++] = ext[j];
    for (int64_t a = c->rp[w]; a < c->rp[w + 1]; a++) {
      int32_t u = c->col[a];
      if (u <= c->root) continue;
      if (in_list(c->sub, c->nsub, u)) continue;
      int near = 0;
      for (int32_t s = 0; s < c->nsub && !near; s++)
        if (adjacent(c->rp, c->col, c->sub[s], u)) near = 1;
      if (near) continue;
      /* u cannot already be in the remaining V_ext: those vertices all
       * neighbour V_sub, and u does not */
      ext2[n2++] = u;
    }
    c->sub[c->nsub++] = w;
    esu_extend(c, ext2, n2);
    c->nsub--;
  }
  free(ext2);
}

/* Motif counts (k in {3, 4, 5}) of the connected k-sets whose minimum vertex
 * lies in [root_lo, root_hi). */
int orc_esu_motifs(int32_t n, const int64_t *rp, const int32_t *col, int32_t k, int32_t root_lo,
                   int32_t root_hi, int32_t nthreads, uint64_t *out) {
  if ((k < 3 || k > 5) || root_lo < 0 || root_hi > n || root_lo > root_hi) return ORC_EINVAL;
  const int np = k == 3 ? 2 : k == 4 ? 6 : 21;
  p5_init();
  u128 total[21];
  memset(total, 0, sizeof(total));
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
  {
    esu_ctx c;
    memset(&c, 0, sizeof(c));
    c.rp = rp;
    c.col = col;
    c.k = k;
#pragma omp for schedule(dynamic, 16)
    for (int32_t v = root_lo; v < root_hi; v++) {
      int64_t d = rp[v + 1] - rp[v];
      int32_t *ext = (int32_t *)malloc((size_t)(d ? d : 1) * sizeof(int32_t));
      if (!ext) abort();
      int64_t ne = 0;
      for (int64_t a = rp[v]; a < rp[v + 1]; a++)
        if (col[a] > v) ext[ne++] = col[a];
      c.root = v;
      c.nsub = 1;
      c.sub[0] = v;
      esu_extend(&c, ext, ne);
      free(ext);
    }
#pragma omp critical
    for (int p = 0; p < np; p++) total[p] += c.cnt[p];
  }
  for (int p = 0; p < np; p++) {
    if (total[p] > (u128)UINT64_MAX) return ORC_EOVERFLOW;
    out[p] = (uint64_t)total[p];
  }
  return ORC_OK;
}

/* ---------------------------------------------------- formula counter */
/* Motif counts of the graph induced on vertex range [lo, hi), which must
 * be a union of connected components (no arc leaves the range).
 *
 * Definitions used (all counts of subgraphs that need not be induced):
 *   S' = sum_v C(d_v, 3)                                  3-stars
 *   P' = sum_{uv in E} (d_u - 1)(d_v - 1) - 3 T           3-edge paths
 *   T' = sum_v t_v (d_v - 2)                              tailed triangles
 *   C' = 4-cycles (each once, Chiba-Nishizeki rank order)
 *   D' = sum_{e in E} C(t_e, 2)                           diamonds
 *   K' = 4-cliques
 * with t_e the triangles on edge e, t_v the triangles on vertex v, T the
 * triangle count.  A copy of pattern X lies inside an induced pattern Y a
 * fixed number of times: S in {S:1, T:1, D:2, K:4}; P in {P:1, T:2, C:4,
 * D:6, K:12}; T in {T:1, D:4, K:12}; C in {C:1, D:1, K:3}; D in {D:1,
 * K:6}; K in {K:1}.  Inverting that triangular system gives the induced
 * counts.  3-motifs: triangles = T, wedges = sum_v C(d_v, 2) - 3 T. */
int orc_formula_motifs_range(int32_t n, const int64_t *rp, const int32_t *col, int32_t lo,
                             int32_t hi, int32_t k, int32_t nthreads, uint64_t *out) {
  if ((k != 3 && k != 4) || lo < 0 || hi > n || lo > hi) return ORC_EINVAL;
  for (int32_t v = lo; v < hi; v++)
    for (int64_t a = rp[v]; a < rp[v + 1]; a++)
      if (col[a] < lo || col[a] >= hi) return ORC_EINVAL;
  if (nthreads < 1) nthreads = 1;
  const int64_t a0 = rp[lo], na = rp[hi] - rp[lo];
  /* t_e per arc (both directions get the same value) */
  int64_t *te = (int64_t *)calloc((size_t)(na ? na : 1), sizeof(int64_t));
  int64_t *tv = (int64_t *)calloc((size_t)(hi - lo + 1), sizeof(int64_t));
  if (!te || !tv) { free(te); free(tv); return ORC_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int32_t u = lo; u < hi; u++) {
    for (int64_t a = rp[u]; a < rp[u + 1]; a++) {
      int32_t v = col[a];
      /* |N(u) & N(v)| by two-pointer merge */
      int64_t i = rp[u], j = rp[v], c = 0;
      while (i < rp[u + 1] && j < rp[v + 1]) {
        if (col[i] < col[j]) i++;
        else if (col[i] > col[j]) j++;
        else { c++; i++; j++; }
      }
      te[a - a0] = c;
    }
  }
  i128 T3 = 0, W2 = 0, Sp = 0, Pp = 0, Tp = 0, Dp = 0;
  for (int32_t u = lo; u < hi; u++) {
    int64_t d = rp[u + 1] - rp[u];
    int64_t s = 0;
    for (int64_t a = rp[u]; a < rp[u + 1]; a++) s += te[a - a0];
    tv[u - lo] = s / 2; /* each triangle at u is seen on its two edges at u */
    T3 += s;            /* every triangle seen 6 times over all arcs */
    W2 += (i128)d * (d - 1) / 2;
    Sp += (i128)d * (d - 1) * (d - 2) / 6;
    Tp += (i128)tv[u - lo] * (d - 2 > 0 ? d - 2 : 0);
    for (int64_t a = rp[u]; a < rp[u + 1]; a++) {
      int32_t v = col[a];
      if (v < u) continue; /* each undirected edge once */
      int64_t dv = rp[v + 1] - rp[v];
      Pp += (i128)(d - 1) * (dv - 1);
      Dp += (i128)te[a - a0] * (te[a - a0] - 1) / 2;
    }
  }
  T3 /= 6;
  Pp -= 3 * T3;
  free(te);
  free(tv);
  if (k == 3) {
    i128 tri = T3, wedge = W2 - 3 * T3;
    if (wedge < 0 || tri < 0 || wedge > (i128)UINT64_MAX || tri > (i128)UINT64_MAX)
      return ORC_EOVERFLOW;
    out[0] = (uint64_t)wedge;
    out[1] = (uint64_t)tri;
    return ORC_OK;
  }
  /* 4-cycles: rank = (degree, ID); for each u, count for every w of lower
   * rank the wedges u-v-w with v of lower rank than u; pairs of such
   * wedges close a 4-cycle whose highest-ranked vertex is u, counted once. */
  i128 Cp = 0;
#pragma omp parallel num_threads(nthreads)
  {
    i128 mine = 0;
    int64_t *cnt = (int64_t *)calloc((size_t)(hi - lo + 1), sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc((size_t)(hi - lo + 1) * sizeof(int32_t));
    if (!cnt || !touched) abort();
#pragma omp for schedule(dynamic, 64)
    for (int32_t u = lo; u < hi; u++) {
      int64_t du = rp[u + 1] - rp[u];
      int64_t nt = 0;
      for (int64_t a = rp[u]; a < rp[u + 1]; a++) {
        int32_t v = col[a];
        int64_t dv = rp[v + 1] - rp[v];
        if (dv > du || (dv == du && v > u)) continue; /* need rank(v) < rank(u) */
        for (int64_t b = rp[v]; b < rp[v + 1]; b++) {
          int32_t w = col[b];
          int64_t dw = rp[w + 1] - rp[w];
          if (dw > du || (dw == du && w >= u)) continue; /* need rank(w) < rank(u) */
          if (cnt[w - lo]++ == 0) touched[nt++] = w;
        }
      }
      for (int64_t i = 0; i < nt; i++) {
        int64_t c = cnt[touched[i] - lo];
        mine += (i128)c * (c - 1) / 2;
        cnt[touched[i] - lo] = 0;
      }
    }
    free(cnt);
    free(touched);
#pragma omp critical
    Cp += mine;
  }
  /* 4-cliques with the degree-ordered enumerator over this range */
  uint64_t lv[5];
  int64_t *rp_local = (int64_t *)malloc(((size_t)(hi - lo) + 1) * sizeof(int64_t));
  int32_t *col_local = (int32_t *)malloc((size_t)(na ? na : 1) * sizeof(int32_t));
  if (!rp_local || !col_local) { free(rp_local); free(col_local); return ORC_ENOMEM; }
  for (int32_t v = lo; v <= hi; v++) rp_local[v - lo] = rp[v] - a0;
  for (int64_t a = 0; a < na; a++) col_local[a] = col[a0 + a] - lo;
  int rc = orc_clique_count(hi - lo, rp_local, col_local, 4, 1, 0, hi - lo, nthreads, lv);
  free(rp_local);
  free(col_local);
  if (rc) return rc;
  i128 Kp = lv[4];
  /* invert the containment relations */
  i128 K = Kp;
  i128 D = Dp - 6 * K;
  i128 C = Cp - D - 3 * K;
  i128 T = Tp - 4 * D - 12 * K;
  i128 P = Pp - 2 * T - 4 * C - 6 * D - 12 * K;
  i128 S = Sp - T - 2 * D - 4 * K;
  i128 res[6] = {S, P, T, C, D, K};
  for (int p = 0; p < 6; p++) {
    if (res[p] < 0 || res[p] > (i128)UINT64_MAX) return ORC_EOVERFLOW;
    out[p] = (uint64_t)res[p];
  }
  return ORC_OK;
}

int orc_formula_motifs(int32_t n, const int64_t *rp, const int32_t *col, int32_t k,
                       int32_t nthreads, uint64_t *out) {
  return orc_formula_motifs_range(n, rp, col, 0, n, k, nthreads, out);
}

/* Per-graph motif counts of a batch: graph g owns [vtx_off[g], vtx_off[g+1]). */
int orc_formula_motifs_batch(int32_t n, const int64_t *rp, const int32_t *col, int32_t G,
                             const int64_t *vtx_off, int32_t k, uint64_t *out) {
  int np = (k == 3) ? 2 : 6;
  for (int32_t g = 0; g < G; g++) {
    int rc = orc_formula_motifs_range(n, rp, col, (int32_t)vtx_off[g], (int32_t)vtx_off[g + 1], k,
                                      1, out + (int64_t)g * np);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* Summary statistics used by identities in tests: sum_v C(d_v, 2) and
 * sum_v C(d_v, 3) (as 128-bit values split in two words), max degree. */
void orc_degree_sums(int32_t n, const int64_t *rp, uint64_t *c2_lo_hi, uint64_t *c3_lo_hi,
                     int64_t *dmax) {
  u128 s2 = 0, s3 = 0;
  int64_t m = 0;
  for (int32_t v = 0; v < n; v++) {
    u128 d = (u128)(rp[v + 1] - rp[v]);
    if ((int64_t)d > m) m = (int64_t)d;
    if (d >= 2) s2 += d * (d - 1) / 2;
    if (d >= 3) s3 += d * (d - 1) * (d - 2) / 6;
  }
  c2_lo_hi[0] = (uint64_t)s2;
  c2_lo_hi[1] = (uint64_t)(s2 >> 64);
  c3_lo_hi[0] = (uint64_t)s3;
  c3_lo_hi[1] = (uint64_t)(s3 >> 64);
  *dmax = m;
}

/* ------------------------------------------------ frequent subgraph mining
 * Frequent subgraph mining (Sec. 2.1 "FSM"; Sec. 3.3 Listing 5).  In a
 * vertex-labelled graph, an edge-induced embedding is a connected set of l
 * edges; its pattern is the labelled graph formed by those edges and their
 * endpoints (Sec. 2.1, edge-induced embeddings), up to label-preserving
 * isomorphism.  The support of a pattern is its MNI (domain) support
 * (Sec. 2.1): for every vertex of the pattern, the number of distinct graph
 * vertices mapped to it over all embeddings of the pattern -- every
 * matching, so an embedding contributes its vertices at every position an
 * automorphism of the pattern can move them to -- and the support is the
 * minimum over the pattern's vertices.  A pattern is frequent if its
 * support is at least `min_support`.
 *
 * The oracle enumerates every connected edge set of 1 .. max_edges (<= 3)
 * edges exactly once by its shape (a connected graph with at most 3 edges
 * is an edge, a 2-edge path, a triangle, a 3-edge path or a 3-star) and
 * computes the support of every pattern without filtering: the Filter
 * phase of the method drops only embeddings of infrequent patterns, whose
 * super-patterns are infrequent by the anti-monotonicity of MNI support,
 * so the set of frequent patterns and their supports do not depend on it.
 *
 * Pattern format of this file's output: nv vertices (2..4), labels
 * lab[0..nv) and adjacency bits over the pairs (0,1), (0,2), (0,3), (1,2),
 * (1,3), (2,3) (bit index in that order), all in the canonical vertex
 * order: the order that makes the tuple (lab[0], .., lab[nv-1], adjacency
 * bits) lexicographically smallest.  Labels must be below 2^12.
 */
typedef struct {
  int nv;
  int lab[4];
  unsigned adj;
} fsm_pat;

static int fsm_pb(int i, int j) { /* bit of the pair (i, j), i < j <= 3 */
  return i == 0 ? j - 1 : (i == 1 ? j + 1 : 5);
}
static int fsm_adjacent(unsigned adj, int a, int b) {
  if (a == b) return 0;
  return a < b ? (adj >> fsm_pb(a, b)) & 1u : (adj >> fsm_pb(b, a)) & 1u;
}

static int fsm_perm[5][24][4];
static int fsm_nperm[5];
static int fsm_perm_ready = 0;

static void fsm_perm_gen(int nv, int depth, int *cur, int used) {
  if (depth == nv) {
    memcpy(fsm_perm[nv][fsm_nperm[nv]++], cur, sizeof(int) * 4);
    return;
  }
  for (int v = 0; v < nv; v++)
    if (!(used & (1 << v))) {
      cur[depth] = v;
      fsm_perm_gen(nv, depth + 1, cur, used | (1 << v));
    }
}

static void fsm_perm_init(void) {
  if (fsm_perm_ready) return;
  for (int nv = 1; nv <= 4; nv++) {
    int cur[4] = {0, 0, 0, 0};
    fsm_nperm[nv] = 0;
    fsm_perm_gen(nv, 0, cur, 0);
  }
  fsm_perm_ready = 1;
}

/* the pattern seen through the vertex order p (position i = vertex p[i]) */
static void fsm_reorder(const fsm_pat *in, const int *p, fsm_pat *out) {
  out->nv = in->nv;
  out->adj = 0;
  for (int i = 0; i < 4; i++) out->lab[i] = i < in->nv ? in->lab[p[i]] : 0;
  for (int i = 0; i < in->nv; i++)
    for (int j = i + 1; j < in->nv; j++)
      if (fsm_adjacent(in->adj, p[i], p[j])) out->adj |= 1u << fsm_pb(i, j);
}

static int fsm_cmp(const fsm_pat *x, const fsm_pat *y) {
  if (x->nv != y->nv) return x->nv < y->nv ? -1 : 1;
  for (int i = 0; i < x->nv; i++)
    if (x->lab[i] != y->lab[i]) return x->lab[i] < y->lab[i] ? -1 : 1;
  if (x->adj != y->adj) return x->adj < y->adj ? -1 : 1;
  return 0;
}

/* canonical form of `in` and the order that produces it */
static void fsm_canon(const fsm_pat *in, fsm_pat *out, int *best) {
  fsm_pat cand;
  for (int q = 0; q < fsm_nperm[in->nv]; q++) {
    const int *p = fsm_perm[in->nv][q];
    fsm_reorder(in, p, &cand);
    if (q == 0 || fsm_cmp(&cand, out) < 0) {
      *out = cand;
      memcpy(best, p, sizeof(int) * 4);
    }
  }
}

/* orbit of every position of a canonical pattern under its automorphisms
 * (orders that reproduce the same labels and adjacency): the smallest
 * position an automorphism maps it to */
static void fsm_orbits(const fsm_pat *c, int *orb) {
  for (int i = 0; i < c->nv; i++) orb[i] = i;
  fsm_pat img;
  for (int q = 0; q < fsm_nperm[c->nv]; q++) {
    const int *p = fsm_perm[c->nv][q];
    fsm_reorder(c, p, &img);
    if (fsm_cmp(&img, c) != 0) continue;
    for (int i = 0; i < c->nv; i++)
      if (p[i] < orb[i]) orb[i] = p[i];
  }
}

typedef struct {
  /* pattern table (open addressing on a packed key) */
  uint64_t *keys;  /* packed key + 1, 0 = empty */
  int32_t *slot;
  int cap_log2;
  fsm_pat *pats;
  int *orb;        /* 4 per pattern */
  uint64_t *count;
  int npat, pat_cap;
  /* (pattern, orbit, vertex) triples of every embedding and position */
  uint64_t *tri;
  int64_t ntri, tri_cap;
  int err;
} fsm_ctx;

static uint64_t fsm_pack(const fsm_pat *c, int edges) {
  uint64_t k = (uint64_t)edges | ((uint64_t)c->nv << 2) | ((uint64_t)c->adj << 5);
  for (int i = 0; i < 4; i++) k |= (uint64_t)(i < c->nv ? c->lab[i] : 0) << (11 + 12 * i);
  return k;
}

static int fsm_lookup(fsm_ctx *x, const fsm_pat *c, int edges) {
  const uint64_t key = fsm_pack(c, edges) + 1;
  const uint64_t mask = ((uint64_t)1 << x->cap_log2) - 1;
  uint64_t h = (key * 0x9E3779B97F4A7C15ull) >> (64 - x->cap_log2);
  for (;;) {
    if (x->keys[h] == key) return x->slot[h];
    if (x->keys[h] == 0) break;
    h = (h + 1) & mask;
  }
  if (x->npat >= x->pat_cap) {
    x->err = ORC_ENOMEM;
    return -1;
  }
  const int id = x->npat++;
  x->keys[h] = key;
  x->slot[h] = id;
  x->pats[id] = *c;
  x->count[id] = 0;
  fsm_orbits(c, x->orb + 4 * id);
  return id;
}

/* one embedding: vertices v[0..nv) and adjacency over them */
static void fsm_embedding(fsm_ctx *x, int nv, const int32_t *v, unsigned adj, const int32_t *lab) {
  if (x->err) return;
  fsm_pat e, c;
  int best[4];
  e.nv = nv;
  e.adj = adj;
  for (int i = 0; i < 4; i++) e.lab[i] = i < nv ? lab[v[i]] : 0;
  fsm_canon(&e, &c, best);
  int edges = 0;
  for (int b = 0; b < 6; b++) edges += (adj >> b) & 1u;
  const int id = fsm_lookup(x, &c, edges);
  if (id < 0) return;
  x->count[id]++;
  if (x->ntri + nv > x->tri_cap) {
    int64_t nc = x->tri_cap * 2 + 1024;
    uint64_t *t = (uint64_t *)realloc(x->tri, (size_t)nc * sizeof(uint64_t));
    if (!t) {
      x->err = ORC_ENOMEM;
      return;
    }
    x->tri = t;
    x->tri_cap = nc;
  }
  for (int i = 0; i < nv; i++)  /* canonical position i holds vertex v[best[i]] */
    x->tri[x->ntri++] = ((uint64_t)id << 36) | ((uint64_t)x->orb[4 * id + i] << 32) | (uint32_t)v[best[i]];
}

typedef struct {
  int edges;
  fsm_pat pat;
  uint64_t support, count;
} fsm_out;

static int fsm_out_cmp(const void *a, const void *b) {
  const fsm_out *x = (const fsm_out *)a, *y = (const fsm_out *)b;
  if (x->edges != y->edges) return x->edges < y->edges ? -1 : 1;
  return fsm_cmp(&x->pat, &y->pat);
}

static int cmp_u64(const void *a, const void *b) {
  const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Frequent patterns of 1 .. max_edges edges (max_edges in 1..3) with MNI
 * support >= min_support (0 lists every pattern that occurs), ordered by
 * (edges, nv, labels, adjacency).  Per pattern: meta[7] = (edges, nv, lab0,
 * lab1, lab2, lab3, adjacency bits) and val[2] = (support, embeddings).
 * *n_out receives the number of such patterns; at most `cap` are written. */
int orc_fsm(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *lab, int32_t max_edges,
            int64_t min_support, int32_t *meta, uint64_t *val, int32_t cap, int32_t *n_out) {
  if (n < 0 || max_edges < 1 || max_edges > 3 || !n_out) return ORC_EINVAL;
  for (int32_t v = 0; v < n; v++)
    if (lab[v] < 0 || lab[v] >= 4096) return ORC_EINVAL;
  fsm_perm_init();
  fsm_ctx x;
  memset(&x, 0, sizeof(x));
  x.cap_log2 = 18;
  x.pat_cap = 1 << 17;
  x.keys = (uint64_t *)calloc((size_t)1 << x.cap_log2, sizeof(uint64_t));
  x.slot = (int32_t *)calloc((size_t)1 << x.cap_log2, sizeof(int32_t));
  x.pats = (fsm_pat *)calloc((size_t)x.pat_cap, sizeof(fsm_pat));
  x.orb = (int *)calloc((size_t)x.pat_cap * 4, sizeof(int));
  x.count = (uint64_t *)calloc((size_t)x.pat_cap, sizeof(uint64_t));
  int rc = ORC_OK;
  if (!x.keys || !x.slot || !x.pats || !x.orb || !x.count) {
    rc = ORC_ENOMEM;
    goto done;
  }
  for (int32_t u = 0; u < n; u++) {
    const int32_t *N = col + rp[u];
    const int64_t d = rp[u + 1] - rp[u];
    for (int64_t i = 0; i < d; i++) {
      /* 1 edge: (u, N[i]) once, from its smaller end */
      if (N[i] > u) {
        int32_t v[4] = {u, N[i], 0, 0};
        fsm_embedding(&x, 2, v, 1u << fsm_pb(0, 1), lab);
      }
      if (max_edges < 2) continue;
      for (int64_t j = i + 1; j < d; j++) {
        /* 2 edges: the pair at its shared vertex u */
        int32_t v[4] = {u, N[i], N[j], 0};
        fsm_embedding(&x, 3, v, (1u << fsm_pb(0, 1)) | (1u << fsm_pb(0, 2)), lab);
        if (max_edges < 3) continue;
        /* 3 edges, star: the triple at its centre u */
        for (int64_t l = j + 1; l < d; l++) {
          int32_t w[4] = {u, N[i], N[j], N[l]};
          fsm_embedding(&x, 4, w, (1u << fsm_pb(0, 1)) | (1u << fsm_pb(0, 2)) | (1u << fsm_pb(0, 3)), lab);
        }
        /* 3 edges, triangle: once, from its smallest vertex */
        if (N[i] > u && adjacent(rp, col, N[i], N[j])) {
          int32_t w[4] = {u, N[i], N[j], 0};
          fsm_embedding(&x, 3, w, (1u << fsm_pb(0, 1)) | (1u << fsm_pb(0, 2)) | (1u << fsm_pb(1, 2)), lab);
        }
      }
      /* 3 edges, path a - u - c - b: once, from its middle edge (u, c), u < c */
      const int32_t c = N[i];
      if (max_edges < 3 || c < u) continue;
      for (int64_t j = 0; j < d; j++) {
        const int32_t a = N[j];
        if (a == c) continue;
        for (int64_t l = rp[c]; l < rp[c + 1]; l++) {
          const int32_t b = col[l];
          if (b == u || b == a) continue;
          int32_t w[4] = {a, u, c, b};
          fsm_embedding(&x, 4, w, (1u << fsm_pb(0, 1)) | (1u << fsm_pb(1, 2)) | (1u << fsm_pb(2, 3)), lab);
        }
      }
    }
    if (x.err) break;
  }
  if (x.err) {
    rc = x.err;
    goto done;
  }
  /* domains: the distinct (pattern, orbit, vertex) triples, counted per (pattern, orbit) */
  qsort(x.tri, (size_t)x.ntri, sizeof(uint64_t), cmp_u64);
  {
    uint64_t *dom = (uint64_t *)calloc((size_t)x.npat * 4 + 1, sizeof(uint64_t));
    fsm_out *res = (fsm_out *)malloc(sizeof(fsm_out) * (size_t)(x.npat + 1));
    if (!dom || !res) {
      free(dom);
      free(res);
      rc = ORC_ENOMEM;
      goto done;
    }
    for (int64_t t = 0; t < x.ntri; t++)
      if (t == 0 || x.tri[t] != x.tri[t - 1]) dom[(x.tri[t] >> 36) * 4 + ((x.tri[t] >> 32) & 15)]++;
    int32_t nr = 0;
    for (int32_t q = 0; q < x.npat; q++) {
      uint64_t sup = UINT64_MAX; /* the smallest domain over the pattern's vertices */
      for (int i = 0; i < x.pats[q].nv; i++) {
        const uint64_t d = dom[(uint64_t)q * 4 + (uint64_t)x.orb[4 * q + i]];
        if (d < sup) sup = d;
      }
      if ((int64_t)sup < min_support) continue;
      int edges = 0;
      for (int bit = 0; bit < 6; bit++) edges += (x.pats[q].adj >> bit) & 1u;
      res[nr].edges = edges;
      res[nr].pat = x.pats[q];
      res[nr].support = sup;
      res[nr].count = x.count[q];
      nr++;
    }
    qsort(res, (size_t)nr, sizeof(fsm_out), fsm_out_cmp);
    for (int32_t r = 0; r < nr && r < cap; r++) {
      int32_t *m = meta + 7 * (int64_t)r;
      m[0] = res[r].edges;
      m[1] = res[r].pat.nv;
      for (int i = 0; i < 4; i++) m[2 + i] = i < res[r].pat.nv ? res[r].pat.lab[i] : 0;
      m[6] = (int32_t)res[r].pat.adj;
      val[2 * (int64_t)r] = res[r].support;
      val[2 * (int64_t)r + 1] = res[r].count;
    }
    *n_out = nr;
    free(res);
    free(dom);
  }
done:
  free(x.keys);
  free(x.slot);
  free(x.pats);
  free(x.orb);
  free(x.count);
  free(x.tri);
  return rc;
}

/* MNI support by its textbook definition, for pins on tiny graphs (n <= 64):
 * every injective map f of the pattern's vertices (nv <= 4, labels plab,
 * adjacency bits padj in the pair order above) into the graph that keeps
 * labels and maps every pattern edge onto a graph edge (edge-induced: other
 * graph edges among the images are allowed); the domain of pattern vertex i
 * is the set of f(i); support = the smallest domain.  *matchings receives
 * the number of such maps (= embeddings x automorphisms). */
int orc_fsm_bf_support(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *lab, int32_t nv,
                       const int32_t *plab, int32_t padj, uint64_t *support, uint64_t *matchings) {
  if (n < 0 || n > 64 || nv < 1 || nv > 4 || !support || !matchings) return ORC_EINVAL;
  if (n == 0) {
    *support = 0;
    *matchings = 0;
    return ORC_OK;
  }
  uint64_t adj[64];
  bits_from_csr(n, rp, col, adj);
  uint64_t dom[4] = {0, 0, 0, 0};
  uint64_t cnt = 0;
  int32_t f[4] = {0, 0, 0, 0};
  /* odometer over all nv-tuples of vertices */
  for (;;) {
    int ok = 1;
    for (int i = 0; i < nv && ok; i++) {
      if (lab[f[i]] != plab[i]) ok = 0;
      for (int j = 0; j < i && ok; j++) {
        if (f[i] == f[j]) ok = 0;
        else if (fsm_adjacent((unsigned)padj, j, i) && !((adj[f[i]] >> f[j]) & 1u)) ok = 0;
      }
    }
    if (ok) {
      cnt++;
      for (int i = 0; i < nv; i++) dom[i] |= 1ull << f[i];
    }
    int p = 0;
    while (p < nv && ++f[p] == n) f[p++] = 0;
    if (p == nv) break;
  }
  uint64_t s = UINT64_MAX;
  for (int i = 0; i < nv; i++) {
    const uint64_t d = (uint64_t)popcount64(dom[i]);
    if (d < s) s = d;
  }
  *support = s;
  *matchings = cnt;
  return ORC_OK;
}
