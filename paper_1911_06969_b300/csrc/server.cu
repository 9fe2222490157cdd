// server.cu -- request loop over device-resident graphs (not in the paper:
// the serving pattern).
//
// Graphs are uploaded, oriented and prepared once.  Queries (triangle count,
// k-clique count, 3-/4-motif count) are queued by pgm_server_submit and
// picked up by `max_inflight` worker threads, each with its own CUDA stream
// and workspace, so queries on the same or different graphs overlap on the
// GPU.  Admission is by predicted embedding-list memory: a queued query
// starts only when the bytes it may materialise, added to those of the
// queries in flight, fit the budget (continuous batching: the first queued
// query that fits is taken, so a large query does not block smaller ones
// behind it).  A query predicted above the whole budget fails with
// PGM_ENOMEM instead of waiting forever.
//
// Prediction (an upper bound from degree statistics, capped by the edge
// blocking budget that bounds any one materialised chunk):
//   k-clique, k >= 4: 12 B per DAG arc (counts + offsets of level 2) +
//     16 B per level-3 entry, level 3 <= sum_v C(d+(v), 2);
//   4-motif: 12 B per arc + 4 B per level-3 entry, level 3 <= sum_v C(d(v), 2),
//     plus the hub kernel's scratch (blocks x 16 warps x dmax ints);
//   triangles and 3-motifs materialise no level: 8 B per vertex (hub lists).
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

#include "common.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct SGraph {
  pgm::Graph g;
  double c2_dag = 0;   // sum_v C(d+(v), 2)
  double c2 = 0;       // sum_v C(d(v), 2)
};

struct Req {
  pgm_query q;
  pgm_result r;
};

}  // namespace

struct pgm_server {
  int64_t budget = 0;
  int32_t max_inflight = 1;
  int device = 0;
  std::vector<std::unique_ptr<SGraph>> graphs;
  std::deque<Req> reqs;            // indexed by ticket (deque keeps references valid)
  std::deque<int64_t> queue;       // queued tickets, arrival order
  int64_t mem_in_use = 0;
  int64_t pending = 0;             // submitted and not finished
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
  cudaStream_t upload_stream = nullptr;
};

namespace {

int64_t predict_bytes(const pgm_server* s, const SGraph& sg, const pgm_query& q) {
  const double budget_entries = (double)pgm::options().level_budget;
  const pgm::Graph& g = sg.g;
  const double arcs = (double)g.narcs, n = (double)g.n;
  const bool clique = q.kind == PGM_Q_TRIANGLE || q.kind == PGM_Q_KCLIQUE;
  const int k = q.kind == PGM_Q_TRIANGLE ? 3 : q.k;
  double b = 8.0 * n + 4096.0;
  const int engine = pgm::options().clique_engine;
  if (clique && engine != 1) {
    // bitset levels: bucket lists, plus row scratch (rows and the warps' C
    // buffers, k - 4 of them for k >= 6) when out-lists exceed the shared-memory rows
    b += 4.0 * n + (double)pgm::bitset_scratch_bytes(g, k);
  } else if (clique && k >= 4) {
    b += 12.0 * (arcs / 2) + 16.0 * std::min(sg.c2_dag, budget_entries);
    if (k >= 5) b += 16.0 * budget_entries;  // deeper levels: at most one budget chunk each
  } else if (!clique && k == 4) {
    const double scratch = (double)pgm::num_sms() * 16.0 * (double)std::max<int64_t>(g.dmax, 1) * 4.0;
    b += 12.0 * arcs + 4.0 * std::min(sg.c2, budget_entries) + scratch;
  }
  (void)s;
  return (int64_t)b;
}

void worker_main(pgm_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  pgm::Workspace ws;
  for (;;) {
    int64_t ticket = -1;
    Req* req = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) break;
        // the first queued request whose predicted memory fits
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
          Req& r = s->reqs[*it];
          if (s->mem_in_use + r.r.mem_bytes <= s->budget) {
            ticket = *it;
            s->queue.erase(it);
            break;
          }
        }
        if (ticket >= 0) break;
        s->cv_work.wait(lk);
      }
      if (ticket < 0) break;
      req = &s->reqs[ticket];
      s->mem_in_use += req->r.mem_bytes;
      req->r.start_s = now_s();
    }
    SGraph& sg = *s->graphs[req->q.graph];
    uint64_t c[6] = {0, 0, 0, 0, 0, 0};
    pgm_status rc;
    pgm::profiler().start(st);
    pgm::profiler().on = false;
    if (req->q.kind == PGM_Q_MOTIF)
      rc = pgm::count_motifs(sg.g, ws, st, req->q.k, 0, sg.g.n, c, nullptr);
    else
      rc = pgm::count_kcliques(sg.g, ws, st, req->q.kind == PGM_Q_TRIANGLE ? 3 : req->q.k, 0, sg.g.n,
                               c, nullptr);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      req->r.status = rc;
      if (rc == PGM_OK) memcpy(req->r.counts, c, sizeof(c));
      req->r.finish_s = now_s();
      req->r.done = 1;
      s->mem_in_use -= req->r.mem_bytes;
      s->pending--;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  cudaStreamSynchronize(st);
  ws.release_all();
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

pgm_status pgm_server_create(int64_t budget_bytes, int32_t max_inflight, pgm_server** out) {
  if (!out || budget_bytes <= 0 || max_inflight < 1 || max_inflight > 64) {
    pgm::set_error("pgm_server_create: bad arguments (budget %lld, max_inflight %d)",
                   (long long)budget_bytes, max_inflight);
    return PGM_EINVAL;
  }
  pgm_server* s = new (std::nothrow) pgm_server();
  if (!s) return PGM_ENOMEM;
  s->budget = budget_bytes;
  s->max_inflight = max_inflight;
  s->device = pgm::device_id();
  if (cudaStreamCreateWithFlags(&s->upload_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    pgm::set_error("pgm_server_create: stream creation failed");
    return PGM_ECUDA;
  }
  for (int i = 0; i < max_inflight; i++) s->workers.emplace_back(worker_main, s);
  *out = s;
  return PGM_OK;
}

pgm_status pgm_server_add_graph(pgm_server* s, int32_t n, const int64_t* rowptr, const int32_t* col,
                                int32_t* graph_id) {
  PGM_NVTX("pgm_server_add_graph");
  if (!s || !graph_id) {
    pgm::set_error("pgm_server_add_graph: null argument");
    return PGM_EINVAL;
  }
  auto sg = std::make_unique<SGraph>();
  pgm::profiler().start(s->upload_stream);
  pgm_status st = pgm::graph_upload(sg->g, n, rowptr, col, false, 0, 0, s->upload_stream);
  if (st == PGM_OK) st = pgm::graph_orient(sg->g);
  if (st == PGM_OK) st = pgm::graph_prepare_motifs(sg->g);
  if (st == PGM_OK) st = pgm::graph_host_dag_rp(sg->g);  // before any worker uses the graph
  // the relabelled copies the motif queries count on, prepared before any worker uses them
  for (int order = 0; order < 2 && st == PGM_OK; order++) {
    pgm::Graph* r = nullptr;
    st = pgm::graph_relabeled(sg->g, order, &r);
    if (st == PGM_OK) st = pgm::graph_prepare_motifs(*r);
  }
  if (st != PGM_OK) {
    pgm::graph_free(sg->g);
    return st;
  }
  for (int32_t v = 0; v < n; v++) {
    const double d = (double)(sg->g.h_rp[v + 1] - sg->g.h_rp[v]);
    const double dd = (double)(sg->g.h_dag_rp[v + 1] - sg->g.h_dag_rp[v]);
    sg->c2 += d * (d - 1) / 2;
    sg->c2_dag += dd * (dd - 1) / 2;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *graph_id = (int32_t)s->graphs.size();
  s->graphs.push_back(std::move(sg));
  return PGM_OK;
}

pgm_status pgm_server_submit(pgm_server* s, const pgm_query* q, int64_t* ticket) {
  if (!s || !q || !ticket) {
    pgm::set_error("pgm_server_submit: null argument");
    return PGM_EINVAL;
  }
  Req r;
  memset(&r, 0, sizeof(r));
  r.q = *q;
  r.r.submit_s = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->graph < 0 || q->graph >= (int32_t)s->graphs.size()) {
      pgm::set_error("pgm_server_submit: unknown graph %d", q->graph);
      return PGM_EINVAL;
    }
    const bool ok = (q->kind == PGM_Q_TRIANGLE) || (q->kind == PGM_Q_KCLIQUE && q->k >= 1 && q->k <= 10) ||
                    (q->kind == PGM_Q_MOTIF && (q->k == 3 || q->k == 4));
    if (!ok) {
      pgm::set_error("pgm_server_submit: unsupported query (kind %d, k %d)", q->kind, q->k);
      return PGM_EUNSUPPORTED;
    }
    if (s->stop) {
      pgm::set_error("pgm_server_submit: server is shutting down");
      return PGM_EBUSY;
    }
    r.r.mem_bytes = predict_bytes(s, *s->graphs[q->graph], *q);
    const int64_t t = (int64_t)s->reqs.size();
    if (r.r.mem_bytes > s->budget) {
      r.r.done = 1;
      r.r.status = PGM_ENOMEM;
      r.r.start_s = r.r.finish_s = r.r.submit_s;
      s->reqs.push_back(r);
      *ticket = t;
      return PGM_OK;
    }
    s->reqs.push_back(r);
    s->queue.push_back(t);
    s->pending++;
    *ticket = t;
  }
  s->cv_work.notify_one();
  return PGM_OK;
}

pgm_status pgm_server_poll(pgm_server* s, int64_t ticket, pgm_result* out) {
  if (!s || !out) {
    pgm::set_error("pgm_server_poll: null argument");
    return PGM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) {
    pgm::set_error("pgm_server_poll: unknown ticket %lld", (long long)ticket);
    return PGM_EINVAL;
  }
  *out = s->reqs[ticket].r;
  return PGM_OK;
}

pgm_status pgm_server_drain(pgm_server* s, double timeout_s) {
  if (!s) {
    pgm::set_error("pgm_server_drain: null server");
    return PGM_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(std::max(timeout_s, 0.0)));
  while (s->pending > 0) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->pending > 0) {
      pgm::set_error("pgm_server_drain: %lld queries still pending", (long long)s->pending);
      return PGM_ETIMEOUT;
    }
  }
  return PGM_OK;
}

void pgm_server_destroy(pgm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // queued queries are cancelled
    for (int64_t t : s->queue) {
      s->reqs[t].r.done = 1;
      s->reqs[t].r.status = PGM_EBUSY;
      s->pending--;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& w : s->workers) w.join();
  for (auto& g : s->graphs) pgm::graph_free(g->g);
  if (s->upload_stream) cudaStreamDestroy(s->upload_stream);
  delete s;
}

}  // extern "C"
