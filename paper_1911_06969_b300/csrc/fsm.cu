// fsm.cu -- frequent subgraph mining (Sec. 2.1 "FSM"; Sec. 3.3 Listing 5):
// edge-induced embeddings of a vertex-labelled graph, MNI (domain) support,
// and the Filter phase between levels (Algorithm 1: Extend, Reduce, Filter).
//
// Level l holds the embeddings of l edges (l = 1..3), extended one edge at a
// time (edge-induced extension: a candidate is an edge incident to the
// embedding).  Every connected edge set is generated once by the canonical
// rule for edge sequences (first the smallest edge ID, then the smallest edge
// adjacent to it, then the rest): a 2-edge embedding (e_a, e_b) has e_a < e_b;
// a 3-edge one extends it by e_c > e_a, and by e_c > e_b when e_c shares a
// vertex with e_a (Sec. 3.2, automorphism-canonical test, edge form).  Edge ID
// = index of the arc from the smaller endpoint.
//
// Reduce: the pattern of an embedding is identified by a key that is an
// isomorphism invariant of its labelled shape (edge, 2-edge path, triangle,
// 3-edge path, 3-star, plus labels in a shape-specific canonical order), so
// no per-embedding isomorphism test is needed; the key also fixes which
// automorphism orbit of the pattern each embedding vertex sits in.  MNI
// support (Sec. 2.1): the domain of an orbit is the set of distinct vertices
// seen there, kept as a bitmap per (pattern, orbit); support = the smallest
// domain.  Filter: only embeddings whose pattern is frequent (support >=
// min_support) are extended -- by anti-monotonicity the dropped ones have no
// frequent super-pattern.  Each level runs its enumeration at least twice:
// first the pattern keys go into a device hash table with their embedding
// counts (then compact IDs go to the patterns with nv * count >= min_support,
// the only ones that can reach it); then every embedding marks its domains
// (pre-sized bitmaps instead of dynamic allocation, as the paper's GPU
// version does -- but in passes over ID ranges that fit the memory budget,
// so the bitmaps do not bound the input size).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace pgm {
namespace {

constexpr int kFsmTableLog2 = 22;   // pattern-table slots per level
constexpr uint32_t kFsmMaxProbe = 512;  // linear-probe limit (then the table counts as full)
constexpr int kFsmGrab = 4;
constexpr int64_t kFsmDomainBytes = (int64_t)64 << 30;  // domain bitmaps held at once, at most

enum FsmType : int { fEdge = 1, fWedge = 2, fTriangle = 3, fStar = 4, fPath = 5 };

// The pattern table of a level, open addressing on the key.  Per slot: the
// key, the compact ID of a pattern that may be frequent (else -1), its
// Filter flag (set once the level's supports are known) and, during a
// domain pass, the first word of each orbit's domain row (off.x = -1: the
// pattern is not in this pass) -- one 16-byte load after the probe.
struct FsmTable {
  unsigned long long* keys;  // 0 = empty
  int32_t* id;
  uint8_t* frequent;
  int4* off;
  unsigned long long* cnt;  // embeddings per slot (first pass)
  uint32_t mask;
};

__device__ __forceinline__ unsigned long long fsm_key(int type, int l0, int l1, int l2, int l3) {
  return (unsigned long long)type | ((unsigned long long)l0 << 3) | ((unsigned long long)l1 << 18) |
         ((unsigned long long)l2 << 33) | ((unsigned long long)l3 << 48);
}

__device__ __forceinline__ int fsm_key_nv(unsigned long long k) {
  const int t = (int)(k & 7);
  return t == fEdge ? 2 : (t == fWedge || t == fTriangle ? 3 : 4);
}

__device__ __forceinline__ uint32_t fsm_hash(unsigned long long k, uint32_t mask) {
  return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> 40) & mask;
}

// slot of a key, inserted if absent; -1 if the table is full
__device__ __forceinline__ int fsm_insert(const FsmTable& T, unsigned long long k) {
  uint32_t h = fsm_hash(k, T.mask);
  for (uint32_t probe = 0; probe < kFsmMaxProbe; probe++) {
    const unsigned long long cur = T.keys[h];
    if (cur == k) return (int)h;
    if (cur == 0ull) {
      const unsigned long long old = atomicCAS(T.keys + h, 0ull, k);
      if (old == 0ull || old == k) return (int)h;
    }
    h = (h + 1) & T.mask;
  }
  return -1;
}

// slot of a key, -1 if absent
__device__ __forceinline__ int fsm_slot(const FsmTable& T, unsigned long long k) {
  uint32_t h = fsm_hash(k, T.mask);
  for (uint32_t probe = 0; probe < kFsmMaxProbe; probe++) {
    const unsigned long long cur = T.keys[h];
    if (cur == k) return (int)h;
    if (cur == 0ull) return -1;
    h = (h + 1) & T.mask;
  }
  return -1;
}

// the pattern of a key is known to be frequent
__device__ __forceinline__ bool fsm_frequent(const FsmTable& T, unsigned long long k) {
  const int h = fsm_slot(T, k);
  return h >= 0 && T.frequent[h] != 0;
}

struct FsmArgs {
  const int32_t* rp;   // undirected CSR
  const int32_t* col;
  const int32_t* src;  // arc -> source vertex
  const int32_t* rev;  // arc -> reverse arc
  const int32_t* lab;  // vertex labels
  const int32_t* rank; // vertex -> index among the vertices of its label (bit of a domain row)
  const int32_t* centres;   // level 2: vertices of degree >= 2 in (label, ID) order
  const int64_t* wprefix;   // level 2: exclusive prefix of C(d, 2) over centres
  int64_t ncentres, nwedges;
  int64_t narcs;
  int mode;            // 0: insert and count pattern keys, 1: mark domains
  FsmTable T;          // this level's patterns
  FsmTable T2;         // level 3: the 2-edge patterns (frequent flags set)
  const uint8_t* freq_arc;  // levels 2, 3: the arc's 1-edge pattern is frequent
  uint32_t* dom;            // mode 1: domain bitmaps of this pass (rows at the slots' off[])
  unsigned long long* queue;  // work queue
  unsigned long long* err;    // [0] table full, [1] pattern missing in mode 1
  unsigned long long* stat;   // candidates examined
};

// One embedding per lane (valid lanes only).  Mode 0: insert its key and
// count it (one atomic per distinct pattern of the warp).  Mode 1: set its
// vertices' bits in the domain bitmaps of their orbits, for the patterns
// with rows in this pass; the bit positions (label ranks) are loaded before
// the probe, so that they do not wait behind it.
__device__ __forceinline__ void fsm_emit(const FsmArgs& A, bool valid, unsigned long long key, int nv,
                                         const int32_t (&v)[4], const int (&orb)[4], bool centre_first) {
  if (A.mode == 0) {
    const int h = valid ? fsm_insert(A.T, key) : -1;
    if (valid && h < 0) atomicAdd(A.err, 1ull);
    const unsigned grp = __match_any_sync(kFull, h);
    if (h >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(A.T.cnt + h, (unsigned long long)__popc(grp));
    return;
  }
  int32_t r[4] = {0, 0, 0, 0};  // bit positions, loaded before the probe (independent of it)
#pragma unroll
  for (int i = 0; i < 4; i++)
    if (valid && i < nv) r[i] = A.rank[v[i]];
  const int h = valid ? fsm_slot(A.T, key) : -1;
  if (valid && h < 0) atomicAdd(A.err + 1, 1ull);
  const int4 e1 = h >= 0 ? A.T.off[h] : make_int4(-1, 0, 0, 0);
  if (e1.x >= 0) {  // the pattern has rows in this pass
#pragma unroll
    for (int i = 0; i < 4; i++)
      if (i < nv) {
        const int o = orb[i];
        const int32_t row = o == 0 ? e1.x : (o == 1 ? e1.y : (o == 2 ? e1.z : e1.w));
        uint32_t* word = A.dom + row + (r[i] >> 5);
        const uint32_t bit = 1u << (r[i] & 31);
        // v[0] is a centre shared by the warp's lanes and by the warps on the
        // same hub: after its first set, a cached read (stale only towards 0)
        // spares the same-word atomics (checking the other shared vertex as
        // well, or every vertex, measured slower)
        if (i == 0 && centre_first && (*word & bit)) continue;
        atomicOr(word, bit);
      }
  }
}

// ---------------------------------------------------- pattern descriptions
// Each sets the key and the orbit of every vertex (v[i] -> orb[i]).

__device__ __forceinline__ unsigned long long fsm_edge(const int32_t* lab, int32_t a, int32_t b, int32_t (&v)[4],
                                                      int (&orb)[4]) {
  const int la = lab[a], lb = lab[b];
  v[0] = la <= lb ? a : b;
  v[1] = la <= lb ? b : a;
  orb[0] = 0;
  orb[1] = la == lb ? 0 : 1;
  return fsm_key(fEdge, min(la, lb), max(la, lb), 0, 0);
}

// 2-edge path with centre c and ends x, y
__device__ __forceinline__ unsigned long long fsm_wedge(const int32_t* lab, int32_t c, int32_t x, int32_t y,
                                                       int32_t (&v)[4], int (&orb)[4]) {
  const int lc = lab[c], lx = lab[x], ly = lab[y];
  v[0] = c;
  v[1] = lx <= ly ? x : y;
  v[2] = lx <= ly ? y : x;
  orb[0] = 0;
  orb[1] = 1;
  orb[2] = lx == ly ? 1 : 2;
  return fsm_key(fWedge, lc, min(lx, ly), max(lx, ly), 0);
}

// sort three (label, vertex) pairs by label
__device__ __forceinline__ void fsm_sort3(int (&l)[3], int32_t (&w)[3]) {
#pragma unroll
  for (int p = 0; p < 2; p++)
#pragma unroll
    for (int q = 0; q < 2 - p; q++)
      if (l[q] > l[q + 1]) {
        const int tl = l[q];
        l[q] = l[q + 1];
        l[q + 1] = tl;
        const int32_t tw = w[q];
        w[q] = w[q + 1];
        w[q + 1] = tw;
      }
}

__device__ __forceinline__ unsigned long long fsm_triangle(const int32_t* lab, int32_t a, int32_t b, int32_t c,
                                                          int32_t (&v)[4], int (&orb)[4]) {
  int l[3] = {lab[a], lab[b], lab[c]};
  int32_t w[3] = {a, b, c};
  fsm_sort3(l, w);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    v[i] = w[i];
    orb[i] = l[i] == l[0] ? 0 : (l[i] == l[1] ? 1 : 2);  // first position of its label
  }
  return fsm_key(fTriangle, l[0], l[1], l[2], 0);
}

__device__ __forceinline__ unsigned long long fsm_star(const int32_t* lab, int32_t c, int32_t x, int32_t y, int32_t z,
                                                      int32_t (&v)[4], int (&orb)[4]) {
  int l[3] = {lab[x], lab[y], lab[z]};
  int32_t w[3] = {x, y, z};
  fsm_sort3(l, w);
  v[0] = c;
  orb[0] = 0;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    v[1 + i] = w[i];
    orb[1 + i] = 1 + (l[i] == l[0] ? 0 : (l[i] == l[1] ? 1 : 2));
  }
  return fsm_key(fStar, lab[c], l[0], l[1], l[2]);
}

// 3-edge path a - b - c - d, read from the end that gives the smaller labels
__device__ __forceinline__ unsigned long long fsm_path(const int32_t* lab, int32_t a, int32_t b, int32_t c,
                                                      int32_t d, int32_t (&v)[4], int (&orb)[4]) {
  const int la = lab[a], lb = lab[b], lc = lab[c], ld = lab[d];
  const bool fwd = la < ld || (la == ld && lb <= lc);
  v[0] = fwd ? a : d;
  v[1] = fwd ? b : c;
  v[2] = fwd ? c : b;
  v[3] = fwd ? d : a;
  const bool pal = la == ld && lb == lc;  // the reversal is an automorphism
  orb[0] = 0;
  orb[1] = 1;
  orb[2] = pal ? 1 : 2;
  orb[3] = pal ? 0 : 3;
  return fwd ? fsm_key(fPath, la, lb, lc, ld) : fsm_key(fPath, ld, lc, lb, la);
}

__device__ __forceinline__ int64_t fsm_eid(const FsmArgs& A, int32_t p, int32_t q, int64_t arc) {
  return p < q ? arc : (int64_t)A.rev[arc];  // the arc from the smaller endpoint
}

// ------------------------------------------------------------- level 1
// every arc from its smaller endpoint is a 1-edge embedding
__global__ void __launch_bounds__(256) fsm_level1(FsmArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t lim = (A.narcs + 31) / 32 * 32;  // whole warps in every iteration
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < lim; a += stride) {
    bool valid = false;
    int32_t v[4] = {0, 0, 0, 0};
    int orb[4] = {0, 0, 0, 0};
    unsigned long long key = 0;
    if (a < A.narcs) {
      const int32_t u = A.src[a], w = A.col[a];
      valid = u < w;
      if (valid) key = fsm_edge(A.lab, u, w, v, orb);
    }
    fsm_emit(A, valid, key, 2, v, orb, false);
  }
}

// level-2 candidates of the 1-edge embedding e_a = (u, w), u < w: slot t of
// N(u) then N(w); the candidate edge e_b shares the slot's list owner p
// (the wedge centre) with e_a.  Canonical: e_b > e_a; Filter: e_b frequent.
struct FsmPair {
  bool ok;
  int32_t centre, x, y;  // wedge: centre, end on e_a, end on e_b
  int64_t eb;
};

__device__ __forceinline__ FsmPair fsm_pair(const FsmArgs& A, int64_t ea, int32_t u, int32_t w, int du, int dw,
                                            int t) {
  FsmPair r;
  r.ok = false;
  r.centre = r.x = r.y = 0;
  r.eb = 0;
  if (t >= du + dw) return r;
  const bool at_u = t < du;
  const int32_t p = at_u ? u : w, o = at_u ? w : u;
  const int64_t arc = (int64_t)A.rp[p] + (at_u ? t : t - du);
  const int32_t q = A.col[arc];
  if (q == o || !A.freq_arc[arc]) return r;
  const int64_t eb = fsm_eid(A, p, q, arc);
  if (eb <= ea) return r;
  r.ok = true;
  r.centre = p;
  r.x = o;
  r.y = q;
  r.eb = eb;
  return r;
}

// Level 2 by centre.  A 2-edge embedding is a pair of frequent edges at a
// common vertex, its centre; taking each pair {i < j} of a centre's list
// once gives each embedding once.  The pairs of all centres form one index
// space (wprefix), cut into chunks of 32 * kFsmPairIters pairs that warps
// take from a queue, so hubs spread over many warps.  Centres come in
// (label, ID) order: at any time the warps touch the patterns -- and the
// domain rows -- of one centre label, few enough to stay in L2, and the
// centres' own bits are set in rank order.
constexpr int kFsmPairIters = 8;

__global__ void __launch_bounds__(256, 4) fsm_level2_centres(FsmArgs A) {
  const int lane = threadIdx.x & 31;
  unsigned long long seen = 0;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(A.queue, 32ull * kFsmPairIters);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= A.nwedges) break;
    // centre of the chunk's first pair: the largest q with wprefix[q] <= p0
    int64_t q = 0;
    if (lane == 0) {
      int64_t lo = 0, hi = A.ncentres - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (A.wprefix[mid] <= (int64_t)p0) lo = mid; else hi = mid - 1;
      }
      q = lo;
    }
    q = __shfl_sync(kFull, q, 0);
    for (int it = 0; it < kFsmPairIters; it++) {
      const int64_t t = (int64_t)p0 + it * 32 + lane;
      bool ok = false;
      int32_t v[4] = {0, 0, 0, 0};
      int orb[4] = {0, 0, 0, 0};
      unsigned long long key = 0;
      if (t < A.nwedges) {
        while (A.wprefix[q + 1] <= t) q++;  // later centres of the chunk (every centre has a pair)
        const int32_t c = A.centres[q];
        const int64_t r0 = A.rp[c];
        const int64_t d = A.rp[c + 1] - r0;
        const int64_t tl = t - A.wprefix[q];
        // pair tl in the order (0,1), (0,2), ..., (1,2), ...: row i starts at
        // i (2d - i - 1) / 2; a root estimate (single precision below 2^20
        // neighbours, double above, where float would be thousands of rows
        // off), then exact correction
        int64_t i;
        if (d < (1 << 20)) {
          const float b = (float)(2 * d - 1);
          i = (int64_t)((b - sqrtf(fmaxf(b * b - 8.0f * (float)tl, 0.0f))) * 0.5f);
        } else {
          const double b = (double)(2 * d - 1);
          i = (int64_t)((b - sqrt(fmax(b * b - 8.0 * (double)tl, 0.0))) * 0.5);
        }
        i = max((int64_t)0, min(i, d - 2));
        while (i > 0 && i * (2 * d - i - 1) / 2 > tl) i--;
        while (i + 1 <= d - 2 && (i + 1) * (2 * d - i - 2) / 2 <= tl) i++;
        const int64_t j = i + 1 + (tl - i * (2 * d - i - 1) / 2);
        seen++;
        ok = A.freq_arc[r0 + i] && A.freq_arc[r0 + j];
        if (ok) key = fsm_wedge(A.lab, c, A.col[r0 + i], A.col[r0 + j], v, orb);
      }
      fsm_emit(A, ok, key, 3, v, orb, true);  // v[0] = the centre
    }
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(A.stat, seen);
}

// Level 2 by first edge: one warp per frequent 1-edge embedding e_a (a
// queue over arcs), lanes over N(u) then N(w) for the second edge e_b > e_a.
// Cost ~ the frequent arcs' d(u) + d(w): the cheaper order when the Filter
// has dropped many edges.
__global__ void __launch_bounds__(256) fsm_level2_arcs(FsmArgs A) {
  const int lane = threadIdx.x & 31;
  unsigned long long seen = 0;
  for (;;) {
    unsigned long long g0 = 0;
    if (lane == 0) g0 = atomicAdd(A.queue, (unsigned long long)kFsmGrab);
    g0 = __shfl_sync(kFull, g0, 0);
    if ((int64_t)g0 >= A.narcs) break;
    for (int64_t ea = (int64_t)g0; ea < min((int64_t)g0 + kFsmGrab, A.narcs); ea++) {
      const int32_t u = A.src[ea], w = A.col[ea];
      if (u > w || !A.freq_arc[ea]) continue;
      const int du = A.rp[u + 1] - A.rp[u], dw = A.rp[w + 1] - A.rp[w];
      for (int t0 = 0; t0 < du + dw; t0 += 32) {
        const FsmPair pr = fsm_pair(A, ea, u, w, du, dw, t0 + lane);
        int32_t v[4] = {0, 0, 0, 0};
        int orb[4] = {0, 0, 0, 0};
        const unsigned long long key = pr.ok ? fsm_wedge(A.lab, pr.centre, pr.x, pr.y, v, orb) : 0ull;
        fsm_emit(A, pr.ok, key, 3, v, orb, false);
      }
      if (lane == 0) seen += (unsigned long long)(du + dw);
    }
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(A.stat, seen);
}

// one warp per frequent 1-edge embedding e_a: its frequent canonical 2-edge
// extensions (e_a, e_b), 32 candidates at a time, then for each of them the
// third edge e_c from the lists of the wedge's three vertices:
//   list of the centre c:  3-star (c; x, y, q),            needs e_c > e_b
//   list of x (end of e_a): triangle x-c-y if q = y, else
//                           3-path q - x - c - y,          needs e_c > e_b
//   list of y (end of e_b): 3-path x - c - y - q,          needs e_c > e_a
// (e_c sharing a vertex with e_a must exceed e_b; the closing edge (x, y) of
// a triangle is taken from x's list only).
__global__ void __launch_bounds__(256, 6) fsm_level3(FsmArgs A) {
  const int lane = threadIdx.x & 31;
  unsigned long long seen = 0;
  for (;;) {
    unsigned long long g0 = 0;
    if (lane == 0) g0 = atomicAdd(A.queue, (unsigned long long)kFsmGrab);
    g0 = __shfl_sync(kFull, g0, 0);
    if ((int64_t)g0 >= A.narcs) break;
    for (int64_t ea = (int64_t)g0; ea < min((int64_t)g0 + kFsmGrab, A.narcs); ea++) {
      const int32_t u = A.src[ea], w = A.col[ea];
      if (u > w || !A.freq_arc[ea]) continue;
      const int du = A.rp[u + 1] - A.rp[u], dw = A.rp[w + 1] - A.rp[w];
      for (int t0 = 0; t0 < du + dw; t0 += 32) {
        FsmPair pr = fsm_pair(A, ea, u, w, du, dw, t0 + lane);
        if (pr.ok) {  // Filter: the 2-edge pattern must be frequent
          int32_t v[4];
          int orb[4];
          pr.ok = fsm_frequent(A.T2, fsm_wedge(A.lab, pr.centre, pr.x, pr.y, v, orb));
        }
        for (unsigned todo = __ballot_sync(kFull, pr.ok); todo; todo &= todo - 1) {
          const int q = __ffs(todo) - 1;
          const int32_t c = __shfl_sync(kFull, pr.centre, q);
          const int32_t x = __shfl_sync(kFull, pr.x, q);
          const int32_t y = __shfl_sync(kFull, pr.y, q);
          const int64_t eb = __shfl_sync(kFull, pr.eb, q);
          const int64_t bx = A.rp[x], bc = A.rp[c], by = A.rp[y];
          const int dx = A.rp[x + 1] - (int32_t)bx, dc = A.rp[c + 1] - (int32_t)bc, dy = A.rp[y + 1] - (int32_t)by;
          const int total = dx + dc + dy;
          if (lane == 0) seen += (unsigned long long)total;
          for (int s0 = 0; s0 < total; s0 += 32) {
            const int s = s0 + lane;
            bool ok = false;
            int32_t v[4] = {0, 0, 0, 0};
            int orb[4] = {0, 0, 0, 0};
            unsigned long long key = 0;
            int nv = 4;
            if (s < total) {
              const int which = s < dx ? 0 : (s < dx + dc ? 1 : 2);  // 0: x, 1: c, 2: y
              const int32_t p = which == 0 ? x : (which == 1 ? c : y);
              const int64_t arc = which == 0 ? bx + s : (which == 1 ? bc + (s - dx) : by + (s - dx - dc));
              const int32_t r = A.col[arc];
              if (A.freq_arc[arc]) {
                const int64_t ec = fsm_eid(A, p, r, arc);
                if (which == 1) {
                  ok = r != x && r != y && ec > eb;
                  if (ok) key = fsm_star(A.lab, c, x, y, r, v, orb);
                } else if (which == 0) {
                  ok = r != c && ec > eb;
                  if (ok && r == y) {
                    key = fsm_triangle(A.lab, x, c, y, v, orb);
                    nv = 3;
                  } else if (ok) {
                    key = fsm_path(A.lab, r, x, c, y, v, orb);
                  }
                } else {
                  ok = r != c && r != x && ec > ea;
                  if (ok) key = fsm_path(A.lab, x, c, y, r, v, orb);
                }
              }
            }
            fsm_emit(A, ok, key, nv, v, orb, false);  // a triangle has 3 vertices, the others 4
          }
        }
      }
    }
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(A.stat, seen);
}

// Compact IDs for the occupied slots whose pattern may be frequent: an orbit
// of r pattern vertices has a domain of at most r * count vertices, so a
// pattern with nv * count < min_support cannot reach it and gets ID -1 (no
// domain bitmaps).
__global__ void fsm_assign(FsmTable T, int64_t min_support, unsigned long long* keys_by_id,
                           unsigned long long* cnt_by_id, unsigned long long* nid) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h <= (int64_t)T.mask;
       h += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = T.keys[h];
    if (!k) continue;
    const unsigned long long c = T.cnt[h];
    T.frequent[h] = 0;
    T.off[h] = make_int4(-1, 0, 0, 0);
    if ((double)c * fsm_key_nv(k) >= (double)min_support) {
      const unsigned long long i = atomicAdd(nid, 1ull);
      T.id[h] = (int32_t)i;
      keys_by_id[i] = k;
      cnt_by_id[i] = c;
    } else {
      T.id[h] = -1;
    }
  }
}

// Row offsets of one domain pass: the slots of IDs [id_lo, id_lo + id_n)
// get the first word of each orbit's row (rowoff, relative to the pass's
// bitmap buffer); the others are marked out of the pass.
__global__ void fsm_pass_rows(FsmTable T, const int64_t* rowoff, int32_t id_lo, int32_t id_n) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h <= (int64_t)T.mask;
       h += (int64_t)gridDim.x * blockDim.x) {
    if (!T.keys[h]) continue;
    const int32_t id = T.id[h], j = id - id_lo;
    if (id >= 0 && j < id_n) {
      const int64_t* r = rowoff + (int64_t)j * 4;
      T.off[h] = make_int4((int32_t)r[0], (int32_t)r[1], (int32_t)r[2], (int32_t)r[3]);
    } else {
      T.off[h] = make_int4(-1, 0, 0, 0);
    }
  }
}

// Filter flags of a level once its supports are known (freq by compact ID)
__global__ void fsm_set_frequent(FsmTable T, const uint8_t* freq) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h <= (int64_t)T.mask;
       h += (int64_t)gridDim.x * blockDim.x) {
    if (T.keys[h] && T.id[h] >= 0) T.frequent[h] = freq[T.id[h]];
  }
}

// domain sizes: popcount of the words [rowoff[r], rowoff[r + 1]) of each
// row r, one block per row
__global__ void __launch_bounds__(256) fsm_popcount(const uint32_t* dom, const int64_t* rowoff, int64_t rows,
                                                     unsigned long long* out) {
  __shared__ unsigned long long part[8];
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t w0 = rowoff[r], w1 = rowoff[r + 1];
    unsigned long long c = 0;
    for (int64_t i = w0 + threadIdx.x; i < w1; i += blockDim.x) c += (unsigned long long)__popc(dom[i]);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += part[i];
      out[r] = t;
    }
    __syncthreads();
  }
}

// level-1 Filter flags per arc: the arc's 1-edge pattern is frequent
__global__ void fsm_arc_flags(FsmArgs A, uint8_t* out) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A.narcs;
       a += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    int orb[4];
    out[a] = fsm_frequent(A.T, fsm_edge(A.lab, A.src[a], A.col[a], v, orb)) ? 1 : 0;
  }
}

// --------------------------------------------------------------- host side
// The documented pattern form: nv vertices in the order that makes (labels,
// adjacency bits over the pairs (0,1), (0,2), (0,3), (1,2), (1,3), (2,3))
// lexicographically smallest, found by trying every order.
int pair_bit(int i, int j) { return i == 0 ? j - 1 : (i == 1 ? j + 1 : 5); }

void canonical_form(int nv, const int* lab, const int (*edges)[2], int ne, pgm_fsm_pattern* out) {
  int order[4] = {0, 1, 2, 3};
  bool first = true;
  int best_lab[4] = {0, 0, 0, 0};
  uint32_t best_adj = 0;
  do {
    int pos[4];
    for (int i = 0; i < nv; i++) pos[order[i]] = i;
    int l[4] = {0, 0, 0, 0};
    for (int i = 0; i < nv; i++) l[i] = lab[order[i]];
    uint32_t adj = 0;
    for (int e = 0; e < ne; e++) {
      const int a = pos[edges[e][0]], b = pos[edges[e][1]];
      adj |= 1u << pair_bit(std::min(a, b), std::max(a, b));
    }
    const bool better = first || std::lexicographical_compare(l, l + nv, best_lab, best_lab + nv) ||
                        (std::equal(l, l + nv, best_lab) && adj < best_adj);
    if (better) {
      std::copy(l, l + 4, best_lab);
      best_adj = adj;
      first = false;
    }
  } while (std::next_permutation(order, order + nv));
  out->edges = ne;
  out->nv = nv;
  for (int i = 0; i < 4; i++) out->labels[i] = i < nv ? best_lab[i] : 0;
  out->adj = best_adj;
}

// the pattern a key describes, in canonical form
void key_pattern(unsigned long long key, pgm_fsm_pattern* out) {
  const int type = (int)(key & 7);
  const int l[4] = {(int)((key >> 3) & 0x7fff), (int)((key >> 18) & 0x7fff), (int)((key >> 33) & 0x7fff),
                    (int)((key >> 48) & 0x7fff)};
  static const int e_edge[1][2] = {{0, 1}};
  static const int e_wedge[2][2] = {{0, 1}, {0, 2}};
  static const int e_tri[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  static const int e_star[3][2] = {{0, 1}, {0, 2}, {0, 3}};
  static const int e_path[3][2] = {{0, 1}, {1, 2}, {2, 3}};
  switch (type) {
    case fEdge: canonical_form(2, l, e_edge, 1, out); break;
    case fWedge: canonical_form(3, l, e_wedge, 2, out); break;
    case fTriangle: canonical_form(3, l, e_tri, 3, out); break;
    case fStar: canonical_form(4, l, e_star, 3, out); break;
    default: canonical_form(4, l, e_path, 3, out); break;
  }
}

bool pattern_less(const pgm_fsm_pattern& a, const pgm_fsm_pattern& b) {
  if (a.edges != b.edges) return a.edges < b.edges;
  if (a.nv != b.nv) return a.nv < b.nv;
  for (int i = 0; i < a.nv; i++)
    if (a.labels[i] != b.labels[i]) return a.labels[i] < b.labels[i];
  return a.adj < b.adj;
}

// Domain-row words of orbit o of a pattern key: an orbit's domain holds
// vertices of one label only (label field o of the key), so its bitmap spans
// the vertices of that label; orbits the pattern does not use get none.
int64_t orbit_words(unsigned long long key, int o, const std::vector<int64_t>& per_label) {
  const int type = (int)(key & 7);
  int f[4];
  for (int i = 0; i < 4; i++) f[i] = (int)((key >> (3 + 15 * i)) & 0x7fff);
  bool used;
  switch (type) {
    case fEdge: used = o == 0 || (o == 1 && f[1] != f[0]); break;
    case fWedge: used = o <= 1 || (o == 2 && f[2] != f[1]); break;
    case fTriangle: used = o == 0 || (o <= 2 && f[o] != f[o - 1]); break;
    case fStar: used = o <= 1 || f[o] != f[o - 1]; break;
    default: used = o <= 1 || !(f[0] == f[3] && f[1] == f[2]); break;  // a palindrome uses orbits 0, 1
  }
  if (!used || f[o] >= (int)per_label.size()) return 0;
  return (per_label[(size_t)f[o]] + 31) / 32;
}

// device buffers of one mining call, released on every return path
struct FsmBuffers {
  DevArr<unsigned long long> keys[3], slot_cnt, kbi, cbi, ctr, pop;
  DevArr<int32_t> ids[3];
  DevArr<uint8_t> frequent[3], freq_arc, freq;
  DevArr<int4> off;
  DevArr<int64_t> rowoff;
  ~FsmBuffers() {
    for (int i = 0; i < 3; i++) {
      keys[i].release();
      ids[i].release();
      frequent[i].release();
    }
    off.release();
    freq.release();
    slot_cnt.release();
    kbi.release();
    cbi.release();
    ctr.release();
    pop.release();
    freq_arc.release();
    rowoff.release();
  }
};

constexpr int kCtrQueue = 0, kCtrErr = 1, kCtrStat = 3, kCtrNid = 4, kCtrSlots = 8;

pgm_status fsm_run(Graph& g, int max_edges, int64_t min_support, std::vector<pgm_fsm_pattern>& res,
                   uint64_t* examined) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);  // labels and the cached bitmaps
  PGM_TRY(graph_prepare_motifs(g));  // arc sources and reverse arcs
  cudaStream_t s = g.stream;
  DevArr<uint32_t>& dom = g.ws.dom;
  const uint32_t slots = 1u << kFsmTableLog2;
  FsmBuffers B;
  PGM_TRY(B.ctr.reserve(kCtrSlots));
  PGM_TRY(B.slot_cnt.reserve(slots));
  PGM_TRY(B.kbi.reserve(slots));
  PGM_TRY(B.cbi.reserve(slots));
  PGM_TRY(B.freq_arc.reserve((size_t)std::max<int64_t>(g.narcs, 1)));
  const int threads = 256;
  const int g1 = std::max(1, std::min(num_sms() * 8, (int)((g.narcs + threads - 1) / threads)));
  const int gq2c = grid_for((const void*)fsm_level2_centres, threads, 0);
  const int gq2a = grid_for((const void*)fsm_level2_arcs, threads, 0);
  // Level 2 by centre enumerates every pair of edges at a vertex (about
  // sum d^2 / 2 candidates), by first edge the lists of the frequent arcs
  // (about f sum d^2 for a fraction f of frequent arcs).  The key pass goes
  // by first edge (hub centres would make many warps count into the same
  // slots); a domain pass goes by centre when at least half the arcs are
  // frequent and its bitmaps exceed half of L2 (below that they stay cached
  // in either order).
  bool centre_ok = false, by_centre = false;
  int l2_bytes = 0;
  PGM_TRY_CUDA(cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, device_id()));
  const int gq3 = grid_for((const void*)fsm_level3, threads, 0);
  Profiler& prof = profiler();
  *examined = 0;
  for (int l = 1; l <= max_edges; l++) {
    PGM_NVTX(kNvtxLevel[l]);
    PGM_TRY(B.keys[l - 1].reserve(slots));
    PGM_TRY(B.ids[l - 1].reserve(slots));
    PGM_TRY(B.frequent[l - 1].reserve(slots));
    PGM_TRY(B.off.reserve(slots));  // only the current level has domain passes
    PGM_TRY_CUDA(cudaMemsetAsync(B.keys[l - 1].p, 0, slots * sizeof(unsigned long long), s));
    PGM_TRY_CUDA(cudaMemsetAsync(B.slot_cnt.p, 0, slots * sizeof(unsigned long long), s));
    PGM_TRY_CUDA(cudaMemsetAsync(B.ctr.p, 0, kCtrSlots * sizeof(unsigned long long), s));
    FsmArgs A;
    memset(&A, 0, sizeof(A));
    A.rp = g.rp;
    A.col = g.col;
    A.src = g.src;
    A.rev = g.rev;
    A.lab = g.labels;
    A.rank = g.label_rank;
    A.centres = g.wedge_centres;
    A.wprefix = g.wedge_prefix;
    A.ncentres = g.n_wedge_centres;
    A.nwedges = g.n_wedges;
    A.narcs = g.narcs;
    A.T = FsmTable{B.keys[l - 1].p, B.ids[l - 1].p, B.frequent[l - 1].p, B.off.p, B.slot_cnt.p, slots - 1};
    if (l == 3) A.T2 = FsmTable{B.keys[1].p, B.ids[1].p, B.frequent[1].p, nullptr, nullptr, slots - 1};
    A.freq_arc = B.freq_arc.p;
    A.queue = B.ctr.p + kCtrQueue;
    A.err = B.ctr.p + kCtrErr;
    A.stat = B.ctr.p + kCtrStat;
    auto launch = [&](int mode) -> pgm_status {
      A.mode = mode;
      PGM_TRY_CUDA(cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s));
      const char* names[2][3] = {{"fsm_level1_keys", "fsm_level2_keys", "fsm_level3_keys"},
                                 {"fsm_level1_domains", "fsm_level2_domains", "fsm_level3_domains"}};
      const int id = prof.begin(names[mode][l - 1], l);
      if (l == 1 || g.narcs == 0)
        fsm_level1<<<g1, threads, 0, s>>>(A);
      else if (l == 2)
        if (mode == 1 && by_centre)
          fsm_level2_centres<<<gq2c, threads, 0, s>>>(A);
        else
          fsm_level2_arcs<<<gq2a, threads, 0, s>>>(A);
      else
        fsm_level3<<<gq3, threads, 0, s>>>(A);
      PGM_CHECK_LAUNCH();
      prof.end(id, 0.0, 0.0);
      return PGM_OK;
    };
    // Extend, first pass: the level's pattern keys and their embedding
    // counts; then IDs for the patterns that may be frequent
    if (l > 1 || g.narcs > 0) PGM_TRY(launch(0));
    fsm_assign<<<num_sms() * 4, 256, 0, s>>>(A.T, min_support, B.kbi.p, B.cbi.p, B.ctr.p + kCtrNid);
    PGM_CHECK_LAUNCH();
    unsigned long long h[kCtrSlots];
    PGM_TRY_CUDA(cudaMemcpyAsync(h, B.ctr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    PGM_TRY_CUDA(cudaStreamSynchronize(s));
    if (h[kCtrErr]) {
      set_error("pgm_fsm: the table of %d-edge patterns is full (%u slots)", l, slots);
      return PGM_ENOMEM;
    }
    const int64_t nid = (int64_t)h[kCtrNid];
    std::vector<unsigned long long> keys((size_t)nid), cnt((size_t)nid), pop((size_t)std::max<int64_t>(nid * 4, 1), 0);
    if (nid > 0) {
      PGM_TRY_CUDA(cudaMemcpyAsync(keys.data(), B.kbi.p, nid * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      PGM_TRY_CUDA(cudaMemcpyAsync(cnt.data(), B.cbi.p, nid * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      PGM_TRY_CUDA(cudaStreamSynchronize(s));
      // Extend, second pass: domains (Reduce by MNI support), for as many
      // patterns at a time as the bitmap budget holds
      std::vector<int64_t> words((size_t)nid * 4);
      for (int64_t i = 0; i < nid; i++)
        for (int o = 0; o < 4; o++) words[(size_t)(i * 4 + o)] = orbit_words(keys[(size_t)i], o, g.h_label_count);
      size_t free_b = 0, total_b = 0;
      PGM_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
      const double budget = std::min((double)kFsmDomainBytes, 0.6 * (double)free_b + (double)dom.cap * 4.0);
      // row offsets are int32 words in the slots: at most 2^31 - 1 words per pass
      const int64_t budget_words = std::max<int64_t>(std::min<int64_t>((int64_t)(budget / 4.0), INT32_MAX), 1);
      std::vector<int64_t> off;
      for (int64_t lo = 0; lo < nid;) {
        int64_t hi = lo, tot = 0;
        off.assign(1, 0);
        while (hi < nid) {  // at least one pattern per pass
          int64_t pw = 0;
          for (int o = 0; o < 4; o++) pw += words[(size_t)(hi * 4 + o)];
          if (hi > lo && tot + pw > budget_words) break;
          for (int o = 0; o < 4; o++) off.push_back(off.back() + words[(size_t)(hi * 4 + o)]);
          tot += pw;
          hi++;
        }
        const int64_t cn = hi - lo;
        PGM_TRY(dom.reserve((size_t)std::max<int64_t>(tot, 1)));
        PGM_TRY(B.rowoff.reserve(off.size()));
        PGM_TRY(B.pop.reserve((size_t)(cn * 4)));
        PGM_TRY_CUDA(cudaMemcpyAsync(B.rowoff.p, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        PGM_TRY_CUDA(cudaMemsetAsync(dom.p, 0, (size_t)tot * sizeof(uint32_t), s));
        const int order = options().fsm_domain_order;
        by_centre = g.n_wedges > 0 &&
                    (order == 2 || (order == 0 && centre_ok && 4.0 * (double)tot > 0.5 * (double)l2_bytes));
        fsm_pass_rows<<<num_sms() * 4, 256, 0, s>>>(A.T, B.rowoff.p, (int32_t)lo, (int32_t)cn);
        PGM_CHECK_LAUNCH();
        A.dom = dom.p;
        PGM_TRY(launch(1));
        fsm_popcount<<<(int)std::min<int64_t>(cn * 4, (int64_t)num_sms() * 16), 256, 0, s>>>(dom.p, B.rowoff.p,
                                                                                             cn * 4, B.pop.p);
        PGM_CHECK_LAUNCH();
        PGM_TRY_CUDA(cudaMemcpyAsync(pop.data() + lo * 4, B.pop.p, cn * 4 * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
        PGM_TRY_CUDA(cudaStreamSynchronize(s));  // off is reused by the next pass
        lo = hi;
      }
      PGM_TRY_CUDA(cudaMemcpyAsync(h, B.ctr.p, sizeof(h), cudaMemcpyDeviceToHost, s));
      PGM_TRY_CUDA(cudaStreamSynchronize(s));
      if (h[kCtrErr + 1]) {
        set_error("pgm_fsm: internal error, %llu embeddings of unknown patterns", h[kCtrErr + 1]);
        return PGM_ECUDA;
      }
    }
    *examined += h[kCtrStat];
    // support = the smallest domain over the orbits in use; Filter flags
    std::vector<uint8_t> fr((size_t)std::max<int64_t>(nid, 1), 0);
    int64_t nfreq = 0;
    for (int64_t i = 0; i < nid; i++) {
      uint64_t sup = UINT64_MAX;
      for (int o = 0; o < 4; o++) {
        const uint64_t d = pop[(size_t)(i * 4 + o)];
        if (d && d < sup) sup = d;
      }
      if (sup == UINT64_MAX || (int64_t)sup < min_support) continue;
      fr[(size_t)i] = 1;
      nfreq++;
      pgm_fsm_pattern p;
      memset(&p, 0, sizeof(p));
      key_pattern(keys[(size_t)i], &p);
      p.support = sup;
      p.embeddings = cnt[(size_t)i];
      res.push_back(p);
    }
    if (nfreq == 0) break;  // nothing to extend
    if (l == 1) {
      unsigned long long freq_edges = 0;
      for (int64_t i = 0; i < nid; i++)
        if (fr[(size_t)i]) freq_edges += cnt[(size_t)i];
      centre_ok = 4.0 * (double)freq_edges >= (double)g.narcs && g.n_wedges > 0;  // 2 arcs per edge
    }
    if (l < max_edges) {
      PGM_TRY(B.freq.reserve(fr.size()));
      PGM_TRY_CUDA(cudaMemcpyAsync(B.freq.p, fr.data(), fr.size(), cudaMemcpyHostToDevice, s));
      fsm_set_frequent<<<num_sms() * 4, 256, 0, s>>>(A.T, B.freq.p);
      PGM_CHECK_LAUNCH();
      if (l == 1) {
        fsm_arc_flags<<<g1, threads, 0, s>>>(A, B.freq_arc.p);
        PGM_CHECK_LAUNCH();
      }
      PGM_TRY_CUDA(cudaStreamSynchronize(s));  // fr is a host buffer of this iteration
    }
  }
  std::sort(res.begin(), res.end(), pattern_less);
  return PGM_OK;
}

}  // namespace

static pgm_status graph_set_labels(Graph& g, const int32_t* labels) {
  for (int32_t v = 0; v < g.n; v++)
    if (labels[v] < 0 || labels[v] >= (1 << 15)) {
      set_error("pgm_graph_set_labels: label %d of vertex %d outside [0, 2^15)", labels[v], v);
      return PGM_EINVAL;
    }
  // rank of each vertex among the vertices of its label: its bit in a domain row
  std::vector<int64_t> count;
  std::vector<int32_t> rank((size_t)g.n);
  for (int32_t v = 0; v < g.n; v++) {
    if ((size_t)labels[v] >= count.size()) count.resize((size_t)labels[v] + 1, 0);
    rank[(size_t)v] = (int32_t)count[(size_t)labels[v]]++;
  }
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  // wedge centres (degree >= 2) in (label, ID) order and the prefix of their pair counts
  PGM_TRY(graph_host_rp(g));
  std::vector<int64_t> start(count.size() + 1, 0);
  for (size_t l = 0; l < count.size(); l++) start[l + 1] = start[l] + count[l];
  std::vector<int32_t> order((size_t)g.n);
  for (int32_t v = 0; v < g.n; v++) order[(size_t)(start[(size_t)labels[v]] + rank[(size_t)v])] = v;
  std::vector<int32_t> centres;
  std::vector<int64_t> wprefix(1, 0);
  for (int32_t v : order) {
    const int64_t d = g.h_rp[(size_t)v + 1] - g.h_rp[(size_t)v];
    if (d < 2) continue;
    centres.push_back(v);
    wprefix.push_back(wprefix.back() + d * (d - 1) / 2);
  }
  if (g.wedge_centres) pgm::dev_free(g.wedge_centres);
  if (g.wedge_prefix) pgm::dev_free(g.wedge_prefix);
  g.wedge_centres = nullptr;
  g.wedge_prefix = nullptr;
  PGM_TRY_CUDA(pgm::dev_malloc(&g.wedge_centres, std::max<size_t>(centres.size(), 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(pgm::dev_malloc(&g.wedge_prefix, wprefix.size() * sizeof(int64_t)));
  if (!centres.empty())
    PGM_TRY_CUDA(cudaMemcpyAsync(g.wedge_centres, centres.data(), centres.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, g.stream));
  PGM_TRY_CUDA(cudaMemcpyAsync(g.wedge_prefix, wprefix.data(), wprefix.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, g.stream));
  g.n_wedge_centres = (int64_t)centres.size();
  g.n_wedges = wprefix.back();
  const size_t bytes = (size_t)std::max<int32_t>(g.n, 1) * sizeof(int32_t);
  if (!g.labels) PGM_TRY_CUDA(pgm::dev_malloc(&g.labels, bytes));
  if (!g.label_rank) PGM_TRY_CUDA(pgm::dev_malloc(&g.label_rank, bytes));
  if (g.n > 0) {
    PGM_TRY_CUDA(cudaMemcpyAsync(g.labels, labels, (size_t)g.n * sizeof(int32_t), cudaMemcpyHostToDevice, g.stream));
    PGM_TRY_CUDA(cudaMemcpyAsync(g.label_rank, rank.data(), (size_t)g.n * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 g.stream));
  }
  PGM_TRY_CUDA(cudaStreamSynchronize(g.stream));
  g.h_label_count.swap(count);
  return PGM_OK;
}

}  // namespace pgm

extern "C" {

pgm_status pgm_graph_set_labels(pgm_graph* g, const int32_t* labels) {
  PGM_NVTX("pgm_graph_set_labels");
  if (!g || (!labels && g->g.n > 0)) {
    pgm::set_error("pgm_graph_set_labels: null argument");
    return PGM_EINVAL;
  }
  return pgm::graph_set_labels(g->g, labels);
}

pgm_status pgm_fsm(pgm_graph* g, int32_t max_edges, int64_t min_support, pgm_fsm_pattern* out, int32_t cap,
                   int32_t* n_out) {
  PGM_NVTX("pgm_fsm");
  if (!g || !n_out || cap < 0 || (cap > 0 && !out)) {
    pgm::set_error("pgm_fsm: bad arguments");
    return PGM_EINVAL;
  }
  if (max_edges < 1 || max_edges > 3) {
    pgm::set_error("pgm_fsm: max_edges=%d unsupported (1, 2 or 3)", max_edges);
    return PGM_EUNSUPPORTED;
  }
  if (min_support < 1) {
    pgm::set_error("pgm_fsm: min_support must be >= 1");
    return PGM_EINVAL;
  }
  if (!g->g.labels) {
    pgm::set_error("pgm_fsm: the graph has no vertex labels (pgm_graph_set_labels)");
    return PGM_EINVAL;
  }
  pgm::profiler().start(g->g.stream);
  std::vector<pgm_fsm_pattern> res;
  uint64_t examined = 0;
  PGM_TRY(pgm::fsm_run(g->g, max_edges, min_support, res, &examined));
  *n_out = (int32_t)res.size();
  if (out && (int64_t)res.size() > cap) {
    pgm::set_error("pgm_fsm: %zu frequent patterns exceed the capacity %d", res.size(), cap);
    return PGM_EOVERFLOW;
  }
  if (out && !res.empty()) memcpy(out, res.data(), res.size() * sizeof(pgm_fsm_pattern));
  pgm::Profiler& prof = pgm::profiler();
  if (prof.on) PGM_TRY(prof.finish(&pgm::last_profile()));
  return PGM_OK;
}

}  // extern "C"
