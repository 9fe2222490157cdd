/*
 * graphgen/gen.c -- seeded synthetic graph generators.
 *
 * Inputs only: this file builds simple undirected graphs in CSR form
 * (symmetric, sorted neighbour lists, no self-loops, no duplicate edges,
 * the input format the paper assumes in Sec. 6.1) and nothing else.  It
 * holds no pattern-mining arithmetic; both the oracle and the CUDA path
 * consume its output.
 *
 * Random numbers: xoshiro256** seeded through splitmix64 (Blackman & Vigna,
 * "Scrambled linear pseudorandom number generators", 2018), written from
 * the published definition.  Every generator takes (seed, stream) so that
 * sub-graphs of a batch get independent, reproducible streams.
 *
 * Generators (each from its published description):
 *   - Erdos-Renyi G(n,p) by geometric skipping (Batagelj & Brandes,
 *     "Efficient generation of large random networks", 2005).
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, 2004) sampled until an exact
 *     number of unique undirected non-loop edges exists, then a random
 *     vertex relabelling.
 *   - Chung-Lu expected-degree graphs by the exact O(n+m) skipping
 *     sampler of Miller & Hagberg ("Efficient generation of networks with
 *     given expected degrees", 2011), then a random relabelling.
 *   - Barabasi-Albert preferential attachment from a seed clique K_{m+1},
 *     degree-proportional choice via the list of arc endpoints.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */
typedef struct {
  uint64_t s[4];
} gg_rng;

static uint64_t splitmix64_next(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ULL);
  /* mix the stream id in through one extra splitmix round */
  x = splitmix64_next(&x) ^ stream;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng *r) {
  uint64_t *s = r->s;
  const uint64_t result = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_u01(gg_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound) by rejection (no modulo bias) */
static inline uint64_t rng_below(gg_rng *r, uint64_t bound) {
  if (bound <= 1) return 0;
  uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
  uint64_t x;
  do {
    x = rng_next(r);
  } while (x >= lim);
  return x % bound;
}

/* ------------------------------------------------------------ edge list */
typedef struct {
  uint32_t *u, *v;
  int64_t len, cap;
} edge_list;

static int el_push(edge_list *e, uint32_t a, uint32_t b) {
  if (e->len == e->cap) {
    int64_t nc = e->cap ? e->cap * 2 : 1024;
    uint32_t *nu = (uint32_t *)realloc(e->u, (size_t)nc * sizeof(uint32_t));
    if (!nu) return -1;
    e->u = nu;
    uint32_t *nv = (uint32_t *)realloc(e->v, (size_t)nc * sizeof(uint32_t));
    if (!nv) return -1;
    e->v = nv;
    e->cap = nc;
  }
  e->u[e->len] = a;
  e->v[e->len] = b;
  e->len++;
  return 0;
}

static void el_free(edge_list *e) {
  free(e->u);
  free(e->v);
  memset(e, 0, sizeof(*e));
}

/* -------------------------------------------------------------- CSR out */
typedef struct {
  int64_t n;
  int64_t narcs;
  int64_t *rowptr; /* n+1 */
  int32_t *col;    /* narcs */
} gg_graph;

/* Build a simple symmetric CSR from an undirected edge list: both arc
 * directions, self-loops dropped, rows sorted ascending, duplicates
 * removed.  Two stable counting-sort passes (by target, then by source). */
static gg_graph *csr_from_edges(int64_t n, const edge_list *e) {
  gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
  if (!g) return NULL;
  g->n = n;
  int64_t na = 0;
  for (int64_t i = 0; i < e->len; i++)
    if (e->u[i] != e->v[i]) na += 2;
  uint32_t *src = (uint32_t *)malloc((size_t)(na ? na : 1) * sizeof(uint32_t));
  uint32_t *dst = (uint32_t *)malloc((size_t)(na ? na : 1) * sizeof(uint32_t));
  uint32_t *tsrc = (uint32_t *)malloc((size_t)(na ? na : 1) * sizeof(uint32_t));
  uint32_t *tdst = (uint32_t *)malloc((size_t)(na ? na : 1) * sizeof(uint32_t));
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!src || !dst || !tsrc || !tdst || !cnt) goto fail;
  int64_t k = 0;
  for (int64_t i = 0; i < e->len; i++) {
    uint32_t a = e->u[i], b = e->v[i];
    if (a == b) continue;
    src[k] = a; dst[k] = b; k++;
    src[k] = b; dst[k] = a; k++;
  }
  /* pass 1: stable by dst */
  memset(cnt, 0, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < na; i++) cnt[dst[i] + 1]++;
  for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
  for (int64_t i = 0; i < na; i++) {
    int64_t p = cnt[dst[i]]++;
    tsrc[p] = src[i];
    tdst[p] = dst[i];
  }
  /* pass 2: stable by src */
  memset(cnt, 0, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < na; i++) cnt[tsrc[i] + 1]++;
  for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
  for (int64_t i = 0; i < na; i++) {
    int64_t p = cnt[tsrc[i]]++;
    src[p] = tsrc[i];
    dst[p] = tdst[i];
  }
  free(tsrc); tsrc = NULL;
  free(tdst); tdst = NULL;
  /* dedupe (arcs are now sorted by (src, dst)) */
  g->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  g->col = (int32_t *)malloc((size_t)(na ? na : 1) * sizeof(int32_t));
  if (!g->rowptr || !g->col) goto fail;
  int64_t w = 0;
  for (int64_t i = 0; i < na; i++) {
    if (i > 0 && src[i] == src[i - 1] && dst[i] == dst[i - 1]) continue;
    g->col[w++] = (int32_t)dst[i];
    g->rowptr[src[i] + 1]++;
  }
  for (int64_t i = 0; i < n; i++) g->rowptr[i + 1] += g->rowptr[i];
  g->narcs = w;
  free(src);
  free(dst);
  free(cnt);
  return g;
fail:
  free(src); free(dst); free(tsrc); free(tdst); free(cnt);
  if (g) { free(g->rowptr); free(g->col); free(g); }
  return NULL;
}

/* Fisher-Yates permutation of [0, n) */
static uint32_t *random_perm(int64_t n, gg_rng *r) {
  uint32_t *p = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; i++) p[i] = (uint32_t)i;
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)rng_below(r, (uint64_t)i + 1);
    uint32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
  return p;
}

static int relabel(edge_list *e, int64_t n, gg_rng *r) {
  uint32_t *p = random_perm(n, r);
  if (!p) return -1;
  for (int64_t i = 0; i < e->len; i++) {
    e->u[i] = p[e->u[i]];
    e->v[i] = p[e->v[i]];
  }
  free(p);
  return 0;
}

/* ------------------------------------------------------------ exported */
int64_t gg_graph_n(const gg_graph *g) { return g->n; }
int64_t gg_graph_narcs(const gg_graph *g) { return g->narcs; }
void gg_graph_copy(const gg_graph *g, int64_t *rowptr, int32_t *col) {
  memcpy(rowptr, g->rowptr, ((size_t)g->n + 1) * sizeof(int64_t));
  if (g->narcs) memcpy(col, g->col, (size_t)g->narcs * sizeof(int32_t));
}
void gg_graph_free(gg_graph *g) {
  if (!g) return;
  free(g->rowptr);
  free(g->col);
  free(g);
}

/* simple graph from an explicit undirected edge list (loops/dups removed) */
gg_graph *gg_from_edges(int64_t n, int64_t ne, const int64_t *us, const int64_t *vs) {
  edge_list e = {0};
  for (int64_t i = 0; i < ne; i++) {
    if (us[i] < 0 || vs[i] < 0 || us[i] >= n || vs[i] >= n) { el_free(&e); return NULL; }
    if (el_push(&e, (uint32_t)us[i], (uint32_t)vs[i])) { el_free(&e); return NULL; }
  }
  gg_graph *g = csr_from_edges(n, &e);
  el_free(&e);
  return g;
}

/* Erdos-Renyi G(n, p): Batagelj-Brandes geometric skipping over the pairs
 * (v, w) with w < v in row-major order. */
static int er_edges(int64_t n, double p, gg_rng *r, edge_list *e) {
  if (n < 2 || p <= 0.0) return 0;
  if (p >= 1.0) {
    for (int64_t v = 1; v < n; v++)
      for (int64_t w = 0; w < v; w++)
        if (el_push(e, (uint32_t)v, (uint32_t)w)) return -1;
    return 0;
  }
  const double lq = log(1.0 - p);
  int64_t v = 1, w = -1;
  while (v < n) {
    double u = rng_u01(r);
    /* 1 - u is in (0, 1], so the logarithm is finite */
    w = w + 1 + (int64_t)floor(log(1.0 - u) / lq);
    while (w >= v && v < n) {
      w -= v;
      v++;
    }
    if (v < n)
      if (el_push(e, (uint32_t)v, (uint32_t)w)) return -1;
  }
  return 0;
}

gg_graph *gg_er(int64_t n, double p, uint64_t seed, uint64_t stream) {
  gg_rng r;
  rng_seed(&r, seed, stream);
  edge_list e = {0};
  if (er_edges(n, p, &r, &e)) { el_free(&e); return NULL; }
  gg_graph *g = csr_from_edges(n, &e);
  el_free(&e);
  return g;
}

/* open-addressing set of undirected edges keyed (min << 32 | max) */
typedef struct {
  uint64_t *slot;
  uint64_t mask;
} edge_set;

static inline uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xFF51AFD7ED558CCDULL;
  x ^= x >> 33;
  x *= 0xC4CEB9FE1A85EC53ULL;
  x ^= x >> 33;
  return x;
}

/* returns 1 if inserted, 0 if already present */
static inline int es_insert(edge_set *s, uint64_t key) {
  uint64_t h = mix64(key) & s->mask;
  for (;;) {
    uint64_t cur = s->slot[h];
    if (cur == UINT64_MAX) {
      s->slot[h] = key;
      return 1;
    }
    if (cur == key) return 0;
    h = (h + 1) & s->mask;
  }
}

/* R-MAT edges on [0, n) with 2^scale >= n: each sample descends `scale`
 * quadrant levels with probabilities (a, b, c, 1-a-b-c); samples that are
 * loops, fall outside [0, n), or repeat an existing undirected edge are
 * discarded, until exactly m unique edges exist.  Returns -2 when the
 * attempt budget (64 m + 2^20 samples) runs out. */
static int rmat_edges(int scale, int64_t n, int64_t m, double a, double b, double c,
                      gg_rng *r, edge_list *e) {
  if (m <= 0) return 0;
  uint64_t cap = 1;
  while (cap < (uint64_t)m * 2 + 16) cap <<= 1;
  edge_set s;
  s.slot = (uint64_t *)malloc(cap * sizeof(uint64_t));
  if (!s.slot) return -1;
  memset(s.slot, 0xFF, cap * sizeof(uint64_t));
  s.mask = cap - 1;
  const double ab = a + b, abc = a + b + c;
  int64_t have = 0;
  uint64_t budget = (uint64_t)m * 64 + (1u << 20);
  while (have < m) {
    if (budget-- == 0) { free(s.slot); return -2; }
    uint64_t u = 0, v = 0;
    for (int l = 0; l < scale; l++) {
      double x = rng_u01(r);
      uint64_t bu, bv;
      if (x < a) { bu = 0; bv = 0; }
      else if (x < ab) { bu = 0; bv = 1; }
      else if (x < abc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    if (u == v || u >= (uint64_t)n || v >= (uint64_t)n) continue;
    uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
    if (es_insert(&s, (lo << 32) | hi)) {
      if (el_push(e, (uint32_t)lo, (uint32_t)hi)) { free(s.slot); return -1; }
      have++;
    }
  }
  free(s.slot);
  return 0;
}

gg_graph *gg_rmat(int64_t n, int64_t m, double a, double b, double c, uint64_t seed,
                  uint64_t stream) {
  int scale = 0;
  while (((int64_t)1 << scale) < n) scale++;
  gg_rng r;
  rng_seed(&r, seed, stream);
  edge_list e = {0};
  if (rmat_edges(scale, n, m, a, b, c, &r, &e)) { el_free(&e); return NULL; }
  if (relabel(&e, n, &r)) { el_free(&e); return NULL; }
  gg_graph *g = csr_from_edges(n, &e);
  el_free(&e);
  return g;
}

/* Chung-Lu weights w_i = min(wmax, C (i+1)^(-1/(gamma-1))), C chosen by
 * bisection so that mean(w) = mean_deg.  Non-increasing in i. */
static double *chung_lu_weights(int64_t n, double gamma, double mean_deg, double wmax) {
  double *w = (double *)malloc((size_t)n * sizeof(double));
  if (!w) return NULL;
  const double ex = -1.0 / (gamma - 1.0);
  double lo = 0.0, hi = mean_deg * (double)n + 1.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi), s = 0.0;
    for (int64_t i = 0; i < n; i++) {
      double x = mid * pow((double)(i + 1), ex);
      s += x < wmax ? x : wmax;
    }
    if (s / (double)n < mean_deg) lo = mid; else hi = mid;
  }
  const double C = 0.5 * (lo + hi);
  for (int64_t i = 0; i < n; i++) {
    double x = C * pow((double)(i + 1), ex);
    w[i] = x < wmax ? x : wmax;
  }
  return w;
}

/* Miller-Hagberg: for each u, walk v > u with geometric skips under the
 * running upper bound p, accept with probability q/p where q is the true
 * pair probability min(1, w_u w_v / S).  Weights must be non-increasing. */
static int chung_lu_edges(int64_t n, const double *w, gg_rng *r, edge_list *e) {
  double S = 0.0;
  for (int64_t i = 0; i < n; i++) S += w[i];
  if (S <= 0.0) return 0;
  for (int64_t u = 0; u + 1 < n; u++) {
    int64_t v = u + 1;
    double p = w[u] * w[v] / S;
    if (p > 1.0) p = 1.0;
    while (v < n && p > 0.0) {
      if (p != 1.0) {
        double x = 1.0 - rng_u01(r); /* (0, 1] */
        v += (int64_t)floor(log(x) / log(1.0 - p));
      }
      if (v < n) {
        double q = w[u] * w[v] / S;
        if (q > 1.0) q = 1.0;
        double x = rng_u01(r);
        if (x < q / p)
          if (el_push(e, (uint32_t)u, (uint32_t)v)) return -1;
        p = q;
        v++;
      }
    }
  }
  return 0;
}

gg_graph *gg_chung_lu(int64_t n, double gamma, double mean_deg, double wmax, uint64_t seed,
                      uint64_t stream) {
  gg_rng r;
  rng_seed(&r, seed, stream);
  double *w = chung_lu_weights(n, gamma, mean_deg, wmax);
  if (!w) return NULL;
  edge_list e = {0};
  int rc = chung_lu_edges(n, w, &r, &e);
  free(w);
  if (rc || relabel(&e, n, &r)) { el_free(&e); return NULL; }
  gg_graph *g = csr_from_edges(n, &e);
  el_free(&e);
  return g;
}

/* Barabasi-Albert: seed clique on vertices 0..m, then each new vertex
 * attaches to m distinct existing vertices drawn in proportion to degree
 * (uniform draws from the list of all arc endpoints so far). */
static int ba_edges(int64_t n, int64_t m, gg_rng *r, edge_list *e) {
  if (n <= 0) return 0;
  if (m < 1) m = 1;
  int64_t k0 = m + 1 < n ? m + 1 : n;
  for (int64_t i = 0; i < k0; i++)
    for (int64_t j = 0; j < i; j++)
      if (el_push(e, (uint32_t)i, (uint32_t)j)) return -1;
  if (n <= k0) return 0;
  int64_t cap = 2 * (k0 * (k0 - 1) / 2 + (n - k0) * m) + 16;
  uint32_t *ends = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
  uint32_t *pick = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
  if (!ends || !pick) { free(ends); free(pick); return -1; }
  int64_t ne = 0;
  for (int64_t i = 0; i < e->len; i++) {
    ends[ne++] = e->u[i];
    ends[ne++] = e->v[i];
  }
  for (int64_t v = k0; v < n; v++) {
    int64_t got = 0;
    while (got < m) {
      uint32_t t = ends[rng_below(r, (uint64_t)ne)];
      int dup = 0;
      for (int64_t j = 0; j < got; j++)
        if (pick[j] == t) { dup = 1; break; }
      if (!dup) pick[got++] = t;
    }
    for (int64_t j = 0; j < m; j++) {
      if (el_push(e, (uint32_t)v, pick[j])) { free(ends); free(pick); return -1; }
      ends[ne++] = (uint32_t)v;
      ends[ne++] = pick[j];
    }
  }
  free(ends);
  free(pick);
  return 0;
}

gg_graph *gg_ba(int64_t n, int64_t m, uint64_t seed, uint64_t stream) {
  gg_rng r;
  rng_seed(&r, seed, stream);
  edge_list e = {0};
  if (ba_edges(n, m, &r, &e)) { el_free(&e); return NULL; }
  gg_graph *g = csr_from_edges(n, &e);
  el_free(&e);
  return g;
}

/* ------------------------------------------------------------- batches */
/* A batch is the disjoint union of G graphs, graph i owning the vertex
 * range [vtx_off[i], vtx_off[i+1]) and global vertex IDs in col. */
typedef struct {
  int64_t G;
  int64_t *vtx_off; /* G+1 */
  int32_t *kind;    /* G: 0 = ER, 1 = BA, 2 = R-MAT */
  double *param;    /* G: average degree (ER), m (BA), average degree (R-MAT) */
  gg_graph *g;      /* union CSR */
} gg_batch;

static gg_batch *batch_from_parts(int64_t G, gg_graph **parts, int32_t *kind, double *param) {
  gg_batch *b = (gg_batch *)calloc(1, sizeof(gg_batch));
  if (!b) return NULL;
  b->G = G;
  b->kind = kind;
  b->param = param;
  b->vtx_off = (int64_t *)calloc((size_t)G + 1, sizeof(int64_t));
  b->g = (gg_graph *)calloc(1, sizeof(gg_graph));
  if (!b->vtx_off || !b->g) return NULL;
  int64_t N = 0, A = 0;
  for (int64_t i = 0; i < G; i++) {
    b->vtx_off[i] = N;
    N += parts[i]->n;
    A += parts[i]->narcs;
  }
  b->vtx_off[G] = N;
  b->g->n = N;
  b->g->narcs = A;
  b->g->rowptr = (int64_t *)malloc(((size_t)N + 1) * sizeof(int64_t));
  b->g->col = (int32_t *)malloc((size_t)(A ? A : 1) * sizeof(int32_t));
  if (!b->g->rowptr || !b->g->col) return NULL;
  int64_t ao = 0;
  for (int64_t i = 0; i < G; i++) {
    gg_graph *p = parts[i];
    int64_t vo = b->vtx_off[i];
    for (int64_t v = 0; v < p->n; v++) b->g->rowptr[vo + v] = ao + p->rowptr[v];
    for (int64_t a = 0; a < p->narcs; a++) b->g->col[ao + a] = (int32_t)(vo + p->col[a]);
    ao += p->narcs;
    gg_graph_free(p);
    parts[i] = NULL;
  }
  b->g->rowptr[N] = ao;
  return b;
}

/* Many small graphs of uneven size: n_i uniform in [nmin, nmax]; even i
 * Erdos-Renyi with average degree uniform in [dmin, dmax] and
 * p = min(1, d / (n - 1)); odd i Barabasi-Albert with m uniform in
 * [mmin, mmax].  Graph i uses random stream i of the seed. */
gg_batch *gg_batch_small(int64_t G, int64_t nmin, int64_t nmax, double dmin, double dmax,
                         int64_t mmin, int64_t mmax, uint64_t seed) {
  gg_graph **parts = (gg_graph **)calloc((size_t)(G ? G : 1), sizeof(gg_graph *));
  int32_t *kind = (int32_t *)calloc((size_t)(G ? G : 1), sizeof(int32_t));
  double *param = (double *)calloc((size_t)(G ? G : 1), sizeof(double));
  if (!parts || !kind || !param) return NULL;
  for (int64_t i = 0; i < G; i++) {
    gg_rng r;
    rng_seed(&r, seed, (uint64_t)i + 1);
    int64_t n = nmin + (int64_t)rng_below(&r, (uint64_t)(nmax - nmin + 1));
    edge_list e = {0};
    int rc;
    if ((i & 1) == 0) {
      double d = dmin + (dmax - dmin) * rng_u01(&r);
      double p = n > 1 ? d / (double)(n - 1) : 0.0;
      if (p > 1.0) p = 1.0;
      kind[i] = 0;
      param[i] = d;
      rc = er_edges(n, p, &r, &e);
    } else {
      int64_t m = mmin + (int64_t)rng_below(&r, (uint64_t)(mmax - mmin + 1));
      kind[i] = 1;
      param[i] = (double)m;
      rc = ba_edges(n, m, &r, &e);
    }
    if (rc) { el_free(&e); return NULL; }
    parts[i] = csr_from_edges(n, &e);
    el_free(&e);
    if (!parts[i]) return NULL;
  }
  gg_batch *b = batch_from_parts(G, parts, kind, param);
  free(parts);
  return b;
}

/* Resident graphs for a query stream: G graphs, the first half R-MAT with
 * (a, b, c), the second half Barabasi-Albert; n log-uniform on
 * [nmin, nmax], average degree uniform on [dmin, dmax] (BA: m = round(d/2)). */
gg_batch *gg_batch_mixed(int64_t G, int64_t nmin, int64_t nmax, double dmin, double dmax,
                         double a, double b, double c, uint64_t seed) {
  gg_graph **parts = (gg_graph **)calloc((size_t)(G ? G : 1), sizeof(gg_graph *));
  int32_t *kind = (int32_t *)calloc((size_t)(G ? G : 1), sizeof(int32_t));
  double *param = (double *)calloc((size_t)(G ? G : 1), sizeof(double));
  if (!parts || !kind || !param) return NULL;
  for (int64_t i = 0; i < G; i++) {
    gg_rng r;
    rng_seed(&r, seed, (uint64_t)i + 1);
    double ln = log((double)nmin) + (log((double)nmax) - log((double)nmin)) * rng_u01(&r);
    int64_t n = (int64_t)llround(exp(ln));
    if (n < nmin) n = nmin;
    if (n > nmax) n = nmax;
    double d = dmin + (dmax - dmin) * rng_u01(&r);
    edge_list e = {0};
    int rc;
    if (i < G / 2) {
      int scale = 0;
      while (((int64_t)1 << scale) < n) scale++;
      int64_t m = (int64_t)llround(d * (double)n / 2.0);
      kind[i] = 2;
      param[i] = d;
      rc = rmat_edges(scale, n, m, a, b, c, &r, &e);
      if (!rc) rc = relabel(&e, n, &r);
    } else {
      int64_t m = (int64_t)llround(d / 2.0);
      if (m < 1) m = 1;
      kind[i] = 1;
      param[i] = (double)m;
      rc = ba_edges(n, m, &r, &e);
    }
    if (rc) { el_free(&e); return NULL; }
    parts[i] = csr_from_edges(n, &e);
    el_free(&e);
    if (!parts[i]) return NULL;
  }
  gg_batch *bt = batch_from_parts(G, parts, kind, param);
  free(parts);
  return bt;
}

int64_t gg_batch_G(const gg_batch *b) { return b->G; }
const gg_graph *gg_batch_graph(const gg_batch *b) { return b->g; }
void gg_batch_copy_meta(const gg_batch *b, int64_t *vtx_off, int32_t *kind, double *param) {
  memcpy(vtx_off, b->vtx_off, ((size_t)b->G + 1) * sizeof(int64_t));
  memcpy(kind, b->kind, (size_t)b->G * sizeof(int32_t));
  memcpy(param, b->param, (size_t)b->G * sizeof(double));
}
void gg_batch_free(gg_batch *b) {
  if (!b) return;
  free(b->vtx_off);
  free(b->kind);
  free(b->param);
  gg_graph_free(b->g);
  free(b);
}

/* Draw `count` exponential inter-arrival gaps (rate lam) and uniform
 * integers below `bound` (query type / target choice) from one stream. */
void gg_poisson_stream(int64_t count, double lam, int64_t ntypes, int64_t ngraphs,
                       uint64_t seed, double *t_arrive, int32_t *qtype, int32_t *graph) {
  gg_rng r;
  rng_seed(&r, seed, 0x5e7e);
  double t = 0.0;
  for (int64_t i = 0; i < count; i++) {
    double x = 1.0 - rng_u01(&r);
    t += -log(x) / lam;
    t_arrive[i] = t;
    qtype[i] = (int32_t)rng_below(&r, (uint64_t)ntypes);
    graph[i] = (int32_t)rng_below(&r, (uint64_t)ngraphs);
  }
}
