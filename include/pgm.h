/*
 * pgm.h -- C ABI of libpgm: exact k-clique and k-motif counting on one
 * NVIDIA B300 (sm_103a) with Pangolin's extend-reduce model.
 *
 * The calls follow the paper's statement of the problem (Sec. 2.1): given
 * an input graph G and a pattern (a k-clique, or every connected k-vertex
 * pattern for motif counting), return its support, which for these
 * applications is the number of embeddings (Sec. 3.3, Listings 3-4).  The
 * input is a simple undirected graph in CSR form with sorted neighbour
 * lists (Sec. 6.1).
 *
 * Conventions shared by every call:
 *   - Every call returns a pgm_status; no C++ exception crosses the ABI.
 *   - Output arguments are written only when the call returns PGM_OK.
 *   - Host buffers belong to the caller; the library copies what it needs.
 *     Device memory allocated by the library belongs to the library and is
 *     released by the matching destroy call.  "_dev" entry points read
 *     caller-owned device buffers and never free them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return counts synchronise that stream before
 *     returning.
 *   - A graph handle is immutable once oriented; counting calls on
 *     different handles may run concurrently on different streams.  Calls
 *     on the same handle must not overlap (they share its workspace).
 *   - pgm_last_error() returns a thread-local message for the last failure.
 *   - There is no CPU fallback: without a usable CUDA device every
 *     counting call fails with PGM_ECUDA.
 */
#ifndef PGM_H
#define PGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PGM_OK = 0,
  PGM_EINVAL = -1,       /* malformed argument or input graph             */
  PGM_EUNSUPPORTED = -2, /* k or size outside what this build supports    */
  PGM_ENOMEM = -3,       /* device allocation failed or budget too small  */
  PGM_ECUDA = -4,        /* CUDA runtime error (message in last_error)    */
  PGM_ETIMEOUT = -5,     /* a bounded wait ran out                        */
  PGM_EOVERFLOW = -6,    /* a count does not fit in uint64                */
  PGM_EBUSY = -7         /* resource in use (server queue full, ...)      */
} pgm_status;

/* flags of pgm_graph_create_csr */
#define PGM_VALIDATE 1u /* reject loops, duplicates, unsorted or asymmetric lists */
#define PGM_SANITIZE 2u /* drop loops and duplicates, sort, symmetrise (host side) */

typedef struct pgm_graph pgm_graph;   /* opaque: device CSR + oriented DAG */
typedef struct pgm_batch pgm_batch;   /* opaque: disjoint union of many graphs */
typedef struct pgm_server pgm_server; /* opaque: request loop over resident graphs */

/* Summary of a graph (exact integers). */
typedef struct {
  int64_t n;            /* vertices                                  */
  int64_t m;            /* undirected edges                          */
  int64_t dmax;         /* maximum degree                            */
  int64_t dag_dmax;     /* maximum out-degree of the oriented DAG (0 before orientation) */
  uint64_t sum_c2[2];   /* sum_v C(d_v, 2) as a 128-bit value (low, high) */
  uint64_t sum_c3[2];   /* sum_v C(d_v, 3) as a 128-bit value (low, high) */
} pgm_graph_stats;

/* Tunables (pgm_set_options / pgm_get_options).  A zero field keeps the
 * current value, except `profile`, `clique_engine`, `motif_order`,
 * `count_headroom_log2` and `fsm_domain_order`, which every call sets
 * (0 = off / auto). */
typedef struct {
  int32_t block_threads;   /* threads per block of the warp-per-parent kernels, 64..512 (default 256) */
  int32_t warp_stage_cap;  /* per-warp shared-memory staging capacity, ints (default 512)     */
  int32_t hub_threshold;   /* segment length that moves a parent to the block-per-parent kernel (default = warp_stage_cap) */
  int32_t blocks_per_sm;   /* persistent-grid blocks per SM (default 0 = occupancy-derived)   */
  int64_t level_budget;    /* max entries of one materialised level chunk (edge blocking, default 1<<31) */
  int32_t profile;         /* 1 = record per-launch CUDA-event times (pgm_last_profile)       */
  int32_t reverse_ratio;   /* intersect in reverse (scan the shorter list, search the longer)
                              when the longer is this many times longer (default 2)          */
  int32_t clique_engine;   /* 0 = auto (bitset levels for k = 3..10, level lists if they do not fit),
                              1 = level lists (vid arrays + inspection-execution),
                              2 = bitset levels where supported                               */
  int32_t bitset_forward_ratio;  /* bitset rows: build row i by scanning N+(P[i]) when it is at most
                                    this many times longer than P, else by testing P in it (default 4) */
  int32_t bitset_smem_degree;    /* bitset rows: largest out-degree whose rows live in shared memory;
                                    64, 256, 512 or 1024 (default 1024); larger ones use global scratch */
  int32_t motif_order;           /* full-range motif counts: 0 = on a copy relabelled by degree
                                    (ascending for k = 3, descending for k = 4; counts are unchanged),
                                    1 = on the input IDs (every call sets this field)              */
  int32_t count_headroom_log2;   /* test hook for PGM_EOVERFLOW, 0 = off (every call sets this field):
                                    with x in [1, 63], the count accumulators of pgm_count_kcliques(_range)
                                    and pgm_count_motifs(_range) start at 2^64 - 2^x and that start is
                                    subtracted again on readback, so a count below 2^x is returned
                                    unchanged and a count of 2^x or more fails with PGM_EOVERFLOW    */
  int32_t motif_b_side_min;      /* 4-motif last level: a level-2 edge (v0, v1) with at least this many
                                    children adjacent to v0 is counted whole by extending the members
                                    of N(v1) above v0 (one scan of each member's list; none of its
                                    children is stored in the level-3 list); an edge with fewer stores
                                    its children and scans their lists (default 8; 1 = always, 2^30 =
                                    never)                                                          */
  int32_t fsm_domain_order;      /* pgm_fsm, domain passes of 2-edge patterns (every call sets this field):
                                    0 = auto (by centre vertex in label order when at least half the
                                    arcs are frequent and the pass's bitmaps exceed half of L2, else by
                                    first edge), 1 = by first edge, 2 = by centre; results are the same */
} pgm_options;

/* Per-call profile (when options.profile = 1): one record per kernel phase. */
#define PGM_PROFILE_MAX 64
typedef struct {
  char name[32];          /* kernel / phase name                                   */
  int32_t level;          /* embedding level the phase works on                    */
  int32_t launches;       /* launches merged into this record                      */
  double ms;              /* summed CUDA-event time of those launches              */
  double entries;         /* embeddings read by the phase                          */
  double alg_bytes;       /* algorithmic bytes (adjacency lists + records) moved   */
} pgm_phase;

typedef struct {
  int32_t nphases;
  pgm_phase phase[PGM_PROFILE_MAX];
  uint64_t level_size[16]; /* |L_l| for l = 1..k (index l) of the last count call */
  int32_t chunks;          /* edge-blocking chunks used                            */
} pgm_profile;

/* ---------------------------------------------------------------- graphs */

/* Create a graph from a host CSR (Sec. 6.1 input format: symmetric, no
 * self-loops, no duplicate edges, neighbour lists sorted ascending).
 *   n       vertices, 0 <= n < 2^31
 *   rowptr  host int64[n+1], rowptr[0] = 0, non-decreasing; total arcs
 *           rowptr[n] < 2^31
 *   col     host int32[rowptr[n]] neighbour IDs
 *   flags   PGM_VALIDATE checks the format on the device and fails with
 *           PGM_EINVAL on a violation; PGM_SANITIZE repairs it on the host
 *           first (the two may be combined).  0 trusts the input.
 *   stream  stream used for the upload and every later call on the handle
 *   out     receives the handle (library-owned; free with pgm_graph_destroy)
 * The host arrays are copied; the caller keeps ownership. */
pgm_status pgm_graph_create_csr(int32_t n, const int64_t *rowptr, const int32_t *col,
                                uint32_t flags, void *stream, pgm_graph **out);

/* Same, from caller-owned DEVICE arrays (int64 rowptr, int32 col); the
 * library copies them into its own buffers.  PGM_SANITIZE is not accepted. */
pgm_status pgm_graph_create_csr_dev(int32_t n, const int64_t *rowptr_dev, const int32_t *col_dev,
                                    int64_t narcs, uint32_t flags, void *stream, pgm_graph **out);

/* Orient the graph into a DAG (Sec. 4.1, "Directed Acyclic Graph"): arc
 * u->v is kept iff (d(u), u) < (d(v), v), i.e. edges point to the vertex of
 * higher degree and ties to the larger ID.  Out-lists stay ID-sorted.
 * Idempotent.  Needed by pgm_count_kcliques (called implicitly there). */
pgm_status pgm_graph_orient_by_degree(pgm_graph *g);

/* Exact summary statistics (degrees from the CSR). */
pgm_status pgm_graph_stats_get(const pgm_graph *g, pgm_graph_stats *out);

void pgm_graph_destroy(pgm_graph *g);

/* --------------------------------------------------------------- counting */

/* Number of k-cliques (Sec. 2.2; Sec. 3.3 Listing 3 "clique finding"):
 * k-vertex subsets whose vertices are pairwise adjacent.  k = 1 gives n,
 * k = 2 gives m; k in [3, 10] runs the level-wise engine on the oriented
 * DAG: extension of the last vertex only (eager pruning, Sec. 4.1), a
 * connectivity check of each candidate against the embedding, and a fused
 * count at the last level (Sec. 3.1, reduce only at the last level).  The
 * default engine keeps the level-3 children of each vertex as bit rows
 * over its out-list, so deeper levels are ANDs of rows (k >= 6 walks the
 * chains depth-first); the level-list engine (options.clique_engine = 1)
 * materialises the levels with inspection-execution (Sec. 5.3), sorted
 * intersection and edge blocking (Sec. 5.2).
 * Orients the graph first if needed.  Returns PGM_EUNSUPPORTED outside
 * [1, 10]. */
pgm_status pgm_count_kcliques(pgm_graph *g, int32_t k, uint64_t *out_count);

/* The part of the k-clique count whose first DAG vertex lies in
 * [v_lo, v_hi): the edge-blocking unit (Sec. 5.2) used to shard one count
 * across devices or processes; the parts over a partition of [0, n) add up
 * to pgm_count_kcliques. */
pgm_status pgm_count_kcliques_range(pgm_graph *g, int32_t k, int32_t v_lo, int32_t v_hi,
                                    uint64_t *out_count);

/* List the k-cliques (1 <= k <= 10; Sec. 3.3 Listing 3 with the last level
 * written instead of reduced, as the embedding lists of Sec. 5.1 allow).
 * Writes one row of k vertex IDs per clique into the caller's DEVICE buffer
 * out_dev (int32, cap_rows * k entries, row-major), the vertices of each row
 * in the orientation order of the DAG (Sec. 4.1); rows appear in no
 * particular order.  *n_rows receives the number of cliques.  out_dev = NULL
 * is a size query (returns PGM_OK with *n_rows set).  PGM_EOVERFLOW (with
 * *n_rows set) if the cliques exceed cap_rows; nothing is written then. */
pgm_status pgm_list_kcliques(pgm_graph* g, int32_t k, int32_t* out_dev, int64_t cap_rows, int64_t* n_rows);

/* pgm_list_kcliques with the rows written to a HOST buffer out_host
 * (cap_rows * k int32), for listings larger than device memory (the
 * edge-blocking of Sec. 5.2 carried to the output).  The last level of each
 * chunk is emitted into one of two device staging buffers of
 * max(min(level_budget, 2^26), d+_max) rows and copied out while the other
 * fills, so device memory beyond the graph stays bounded.  Page-locked host
 * memory lets the copies overlap the listing; pageable memory works,
 * slower.  Rows are in chunk order; same size query, overflow and k rules
 * as pgm_list_kcliques. */
pgm_status pgm_list_kcliques_host(pgm_graph* g, int32_t k, int32_t* out_host, int64_t cap_rows, int64_t* n_rows);

/* Vertex-induced motif counts (Sec. 2.2; Sec. 3.3 Listing 4 "motif
 * counting"; customised classification Sec. 4.2, Listing 6): for each
 * connected k-vertex pattern, the number of vertex sets whose induced
 * subgraph is that pattern, each set counted once (canonical test,
 * Sec. 3.2).  Output order:
 *   k = 3: [wedge, triangle]                                   (cap >= 2)
 *   k = 4: [3-star, 4-path, tailed-triangle, 4-cycle, diamond, 4-clique] (cap >= 6)
 *   k = 5: the 21 connected 5-vertex graphs (cap >= 21), generic
 *          classification by adjacency code, ordered by edge count, then
 *          degree sequence (non-increasing, lexicographically smaller first),
 *          then canonical code (the smallest 10-bit adjacency code over the
 *          120 relabellings, bit i = pair i of (0,1),(0,2),(0,3),(0,4),(1,2),
 *          (1,3),(1,4),(2,3),(2,4),(3,4)); index 0 = 5-path, 2 = 4-star,
 *          3 = 5-cycle, 20 = 5-clique.  Levels 3 and 4 are materialised as
 *          vertex tuples, in chunks of at most level_budget / 8 entries.
 * Other k: PGM_EUNSUPPORTED.  Requires n < 2^30. */
pgm_status pgm_count_motifs(pgm_graph *g, int32_t k, uint64_t *out_counts, int32_t cap);

/* Motif counts of the embeddings whose first vertex (the minimum ID)
 * lies in [v_lo, v_hi); additive over a partition of [0, n). */
pgm_status pgm_count_motifs_range(pgm_graph *g, int32_t k, int32_t v_lo, int32_t v_hi,
                                  uint64_t *out_counts, int32_t cap);

/* List the connected k-vertex sets (k = 3, 4, 5; Sec. 3.3 Listing 4 with
 * the last level written instead of reduced, Sec. 5.1).  Writes one row of
 * k + 1 int32 per set into the caller's DEVICE buffer out_dev (cap_rows *
 * (k + 1) entries, row-major): the k vertex IDs in the breadth-first
 * canonical order of the set (first the minimum ID, then each next vertex
 * the unused one adjacent to the prefix with the smallest (index of its
 * first neighbour in the prefix, ID)), then the pattern index in the order
 * of pgm_count_motifs.  Rows appear in no particular order.  *n_rows
 * receives the number of sets (the sum of the motif counts).  out_dev =
 * NULL is a size query; PGM_EOVERFLOW (with *n_rows set) if the sets
 * exceed cap_rows, nothing written then.  Other k: PGM_EUNSUPPORTED.
 * Requires n < 2^30. */
pgm_status pgm_list_motifs(pgm_graph *g, int32_t k, int32_t *out_dev, int64_t cap_rows, int64_t *n_rows);

/* pgm_list_motifs with the rows written to a HOST buffer out_host
 * (cap_rows * (k + 1) int32), for listings larger than device memory.  The
 * last level is inspected (rows per entry), cut into entry ranges whose
 * rows fit a device staging buffer of max(min(level_budget, 2^26),
 * (k - 1) * d_max) rows, emitted there and copied out on a copy stream
 * while the other of two staging buffers fills.  Rows are in chunk order;
 * same size query, overflow and k rules as pgm_list_motifs. */
pgm_status pgm_list_motifs_host(pgm_graph *g, int32_t k, int32_t *out_host, int64_t cap_rows, int64_t *n_rows);

/* --------------------------------------------------------------- batches */

/* A batch is the disjoint union of G graphs in one concatenated CSR: graph
 * i owns the vertices [vtx_off[i], vtx_off[i+1]) and its arcs use those
 * global IDs (no arc may leave its graph; PGM_EINVAL otherwise).  Host
 * arrays:
 *   vtx_off     int64[G+1], vtx_off[0] = 0, non-decreasing
 *   rowptr_cat  int64[vtx_off[G]+1]
 *   col_cat     int32[rowptr_cat[vtx_off[G]]]
 * A NULL stream makes the batch create (and own) a non-blocking stream,
 * since CUDA-graph capture needs a stream other than the legacy default.
 * (not in the paper: many-small-graphs batching). */
pgm_status pgm_batch_create(int32_t G, const int64_t *vtx_off, const int64_t *rowptr_cat,
                            const int32_t *col_cat, uint32_t flags, void *stream, pgm_batch **out);

/* Tunables of the batched path, chosen by pgm_batch_autotune or by hand.
 * Zero fields keep the library defaults. */
typedef struct {
  int32_t block_threads;  /* threads per block, 64..512           */
  int32_t warp_stage_cap; /* per-warp staging capacity (ints)     */
  int32_t hub_threshold;  /* block-per-parent threshold           */
  int32_t blocks_per_sm;  /* persistent grid size per SM          */
  int32_t use_graph;      /* 1 = replay a captured CUDA graph     */
  int32_t motif_b_side_min;     /* intersection variant of the 4-motif last level (options field) */
  int32_t reverse_ratio;        /* level-list intersection direction (options field)              */
  int32_t bitset_forward_ratio; /* bitset row-building direction (options field)                  */
} pgm_tune;

/* Per-graph motif counts of every graph of the batch in one pass of the
 * level engine over the union (persistent kernels pulling parents from a
 * device queue, counts attributed per graph), optionally replayed as a
 * captured CUDA graph.  k = 3, 4, 5; out: host uint64[G * (2, 6 or 21)],
 * row i = graph i in pgm_count_motifs order.  t may be NULL (defaults). */
pgm_status pgm_batch_count_motifs(pgm_batch *b, int32_t k, uint64_t *out, const pgm_tune *t);

/* Per-graph k-clique counts (out: host uint64[G]). */
pgm_status pgm_batch_count_kcliques(pgm_batch *b, int32_t k, uint64_t *out, const pgm_tune *t);

/* The baseline the batched path is measured against: the same counts by
 * one plain pgm_count_motifs-style launch sequence per graph, in a host
 * loop on one stream (same device data, natural per-level syncs). */
pgm_status pgm_batch_count_motifs_loop(pgm_batch *b, int32_t k, uint64_t *out);

/* Time candidate pgm_tune settings on this batch and return the fastest
 * (exact counts are identical for every setting; a mismatch is reported
 * as PGM_EINVAL). */
pgm_status pgm_batch_autotune(pgm_batch *b, int32_t k, pgm_tune *best, double *best_ms);

/* One timed candidate of pgm_batch_autotune_ex. */
typedef struct {
  pgm_tune tune;
  double ms; /* mean CUDA-event time of two timed runs after a warm-up */
} pgm_tune_trial;

/* pgm_batch_autotune (k = 3, 4) with its trials and a cache.  The search
 * walks the knobs one at a time from the defaults -- block_threads {128,
 * 256, 512}, warp_stage_cap {128, 256, 512, 1024}, blocks_per_sm {0, 2, 4},
 * motif_b_side_min {8, 32, 128, 2^30} -- keeping each knob's fastest value.
 *   trials, cap   every timed candidate in order, up to cap (NULL, 0: none);
 *                 *n_trials receives the number written (may be NULL)
 *   cache_path    a JSON file of earlier winners keyed by k and the batch's
 *                 features (graphs, vertices, arcs, largest degree, each
 *                 rounded down to a power of two), or NULL.  A hit returns
 *                 the stored setting and time without timing anything
 *                 (*from_cache = 1); a miss searches and adds the winner.
 * Not safe against concurrent writers of the same cache file. */
pgm_status pgm_batch_autotune_ex(pgm_batch *b, int32_t k, const char *cache_path, pgm_tune *best,
                                 double *best_ms, pgm_tune_trial *trials, int32_t cap, int32_t *n_trials,
                                 int32_t *from_cache);

int32_t pgm_batch_size(const pgm_batch *b);
void pgm_batch_destroy(pgm_batch *b);

/* ---------------------------------------------------------------- server */

typedef enum { PGM_Q_TRIANGLE = 0, PGM_Q_KCLIQUE = 1, PGM_Q_MOTIF = 2 } pgm_query_kind;

typedef struct {
  int32_t kind;   /* pgm_query_kind                                   */
  int32_t k;      /* clique size (KCLIQUE) or motif size (MOTIF)      */
  int32_t graph;  /* resident graph id returned by pgm_server_add_graph */
  int32_t pad;
} pgm_query;

typedef struct {
  int32_t done;       /* 1 when the result is final                      */
  int32_t status;     /* pgm_status of the query                          */
  uint64_t counts[6]; /* clique count in [0], or motif counts             */
  double submit_s;    /* host clock (s) at submission                     */
  double start_s;     /* host clock when admitted to the device           */
  double finish_s;    /* host clock when the result was seen on the host  */
  int64_t mem_bytes;  /* predicted embedding-list bytes used for admission */
} pgm_result;

/* Request loop over device-resident graphs (not in the paper: serving).
 * budget_bytes bounds the predicted embedding-list memory of the queries
 * in flight; max_inflight bounds the concurrent queries (one CUDA stream
 * and one workspace each).  Worker threads admit queued queries as memory
 * and slots free up, so queries on different graphs overlap on the GPU. */
pgm_status pgm_server_create(int64_t budget_bytes, int32_t max_inflight, pgm_server **out);
/* Upload a graph (host CSR as in pgm_graph_create_csr) and orient it. */
pgm_status pgm_server_add_graph(pgm_server *s, int32_t n, const int64_t *rowptr,
                                const int32_t *col, int32_t *graph_id);
/* Queue a query; *ticket identifies it in pgm_server_poll. */
pgm_status pgm_server_submit(pgm_server *s, const pgm_query *q, int64_t *ticket);
/* Non-blocking: copies the current state of the ticket's result. */
pgm_status pgm_server_poll(pgm_server *s, int64_t ticket, pgm_result *out);
/* Block until every submitted query is done (PGM_ETIMEOUT after timeout_s). */
pgm_status pgm_server_drain(pgm_server *s, double timeout_s);
void pgm_server_destroy(pgm_server *s);

/* ------------------------------------------------------- no allocation */

/* Triangle count of an oriented graph that the caller already holds on the
 * device, for callers that cannot call cudaMalloc (e.g. code running under
 * an application or framework allocator that owns all device memory, or a
 * latency-critical caller that cannot take the device-wide synchronisation
 * of an allocation).  No counterpart in the paper.
 *   n, m            vertices and arcs of the DAG (m = dag_rowptr[n] < 2^31)
 *   dag_rowptr_dev  device int32[n+1]; dag_col_dev device int32[m]: any
 *                   acyclic orientation (each undirected edge once) with
 *                   out-lists sorted by ascending ID, e.g. the degree
 *                   orientation of pgm_graph_orient_by_degree
 *   count_dev       device uint64 that receives the count
 * Nothing is allocated: the kernels' scratch (512 B of counters and 8 MiB
 * of hub-parent slots) is a fixed file-scope device array that every GPU
 * loading the library holds until the process exits.  Graphs that could
 * need more hub slots than that fail with PGM_EUNSUPPORTED before any
 * device work: m / (h + 1) + 2 > 2^20, where h = min(options.hub_threshold,
 * options.warp_stage_cap) (h = warp_stage_cap while hub_threshold is
 * unset), the out-degree above which a parent is a hub.  The first call on a device looks up the array's device
 * address (make that first call before any stream capture).  All calls
 * share the one array and clear its counters on entry: calls that overlap
 * on the GPU race and must be serialised by the caller.  Synchronises
 * `stream` before returning. */
pgm_status pgm_count_triangles_noalloc(int32_t n, const int32_t *dag_rowptr_dev,
                                       const int32_t *dag_col_dev, int64_t m,
                                       unsigned long long *count_dev, void *stream);

/* ------------------------------------------- frequent subgraph mining */

/* Vertex labels for pgm_fsm: labels is a HOST array int32[n], each label in
 * [0, 2^15); copied to the device (the caller keeps ownership).  Replaces
 * earlier labels.  PGM_EINVAL on a null array (n > 0) or a label out of
 * range (nothing changed then). */
pgm_status pgm_graph_set_labels(pgm_graph *g, const int32_t *labels);

/* One frequent pattern: its vertices in canonical order -- the order that
 * makes (labels[0..nv-1], adj) lexicographically smallest, adj bit i set
 * when pair i of (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) is an edge -- its MNI
 * support and its number of edge-induced embeddings (distinct edge sets). */
typedef struct pgm_fsm_pattern {
  int32_t edges;       /* 1, 2 or 3 */
  int32_t nv;          /* vertices: 2, 3 or 4 */
  int32_t labels[4];   /* labels[nv..3] = 0 */
  uint32_t adj;
  uint32_t pad;
  uint64_t support;    /* smallest domain over the pattern's vertices */
  uint64_t embeddings;
} pgm_fsm_pattern;

/* Frequent subgraph mining (Sec. 2.1 "FSM"; Sec. 3.3 Listing 5): the
 * connected labelled patterns of 1..max_edges edges (max_edges = 1, 2 or 3)
 * whose minimum-image-based support -- over the orbits of the pattern, the
 * smallest number of distinct graph vertices that play that orbit in some
 * edge-induced embedding -- is at least min_support (>= 1).  Embeddings are
 * extended one edge at a time, only from frequent patterns (Filter).
 * Labels come from pgm_graph_set_labels (PGM_EINVAL without).  out is a
 * HOST array of cap patterns, written in the order (edges, nv, labels, adj);
 * out = NULL (cap 0) is a size query, which runs the whole mining (a
 * caller can pass a generous cap instead and retry on PGM_EOVERFLOW);
 * *n_out receives the number of frequent patterns, and PGM_EOVERFLOW
 * (nothing written) when it exceeds cap.  Device memory: a 2^22-slot
 * pattern table per level (PGM_ENOMEM when the distinct patterns of one
 * size overfill it) and, per pattern whose embedding count leaves it a
 * chance to be frequent, one bitmap per orbit over the vertices of the
 * orbit's label, in passes over the level of at most 64 GB of bitmaps (or
 * 60% of the free device memory); the bitmaps stay with the handle for the
 * next call.  Other max_edges: PGM_EUNSUPPORTED. */
pgm_status pgm_fsm(pgm_graph *g, int32_t max_edges, int64_t min_support, pgm_fsm_pattern *out, int32_t cap,
                   int32_t *n_out);

/* ---------------------------------------------------------------- misc */

pgm_status pgm_set_options(const pgm_options *o);
pgm_status pgm_get_options(pgm_options *o);
/* Profile of the last counting call made by this thread (options.profile). */
pgm_status pgm_last_profile(pgm_profile *out);
/* Exclusive prefix sum on the device (inspection-execution's allocation
 * step, Sec. 5.3): out[i] = sum of cnt[0..i-1], out[len] = total.  Device
 * pointers: cnt uint32[len], out int64[len+1].  Synchronises the stream. */
pgm_status pgm_exclusive_scan_dev(const uint32_t *cnt_dev, int64_t len, int64_t *out_dev,
                                  void *stream);
const char *pgm_last_error(void);
const char *pgm_version(void);
/* Number of CUDA kernels this library has launched in the process (all
 * threads; a CUDA-graph replay adds the kernel nodes of the graph). */
uint64_t pgm_kernel_launches(void);

/* Bounds-checked build (libpgm_debug.so, compiled with PGM_DEBUG): the
 * number of out-of-range indices met at the checked global-memory sites
 * since the last reset (each such access is skipped, nothing traps); when
 * non-zero, pgm_last_error() names the first site and index.  reset != 0
 * clears the counters.  Always 0 in the regular build. */
uint64_t pgm_debug_errors(int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* PGM_H */
