// Serving runtime: many tracked graphs resident on one GPU, update requests
// arriving at any time, worked on concurrently.
//
// Each admitted graph owns a handle (CSR with slack, membership, K, Sigma,
// Delta Sigma on the device) and a CUDA stream of its own.  A pool of worker
// threads ("slots") takes work as soon as a slot is free:
//   * admission: the oldest waiting graph whose footprint
//     (leiden_footprint_bytes) fits in the remaining device budget is
//     created and gets its static Leiden; the budget also keeps room for
//     the aggregation buffers that `slots` concurrent calls draw from the
//     stream-ordered pool (slots times the largest admitted graph's);
//   * requests: among admitted graphs that are not busy, the one whose next
//     request is oldest runs that request (leiden_update on its stream).
// Requests of one graph run one at a time in submission order, so each
// result is the one the graph would get alone; requests of different graphs
// overlap on the device.  Host code only: no kernels live here.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct ServerGraph {
  enum State { PENDING, ADMITTING, READY, FAILED, REMOVED };
  int64_t n = 0;
  std::vector<int64_t> off;  // host copy until admitted
  std::vector<int32_t> col, w;
  int64_t bytes = 0;
  int64_t agg_bytes = 0;  // aggregation buffers a call on it draws from the pool
  leiden_handle *h = nullptr;
  cudaStream_t stream = nullptr;
  State state = PENDING;
  bool busy = false;
  std::deque<int64_t> queue;  // tickets in submission order
  std::string err;
};

struct ServerRequest {
  int32_t graph = 0;
  std::vector<leiden_edge> del, ins;
  leiden_mode mode = LEIDEN_DF;
  bool keep = false;
  std::vector<int32_t> membership;
  leiden_status status = LEIDEN_OK;
  bool done = false;
  std::string err;
  clock_type::time_point t_submit, t_start, t_done;
};

}  // namespace

struct leiden_server {
  leiden_params p{};
  int device = 0;
  int64_t budget = 0, used = 0;
  int64_t max_agg = 0;  // largest agg_bytes of the graphs admitted so far
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<ServerGraph *> graphs;
  std::map<int64_t, ServerRequest *> reqs;
  int64_t next_ticket = 1;
  int64_t completed = 0, running = 0;
  bool stop = false;
  std::string err;
};

namespace {

// Admission of one graph (run by a worker, lock not held).
void admit(leiden_server *S, ServerGraph *g) {
  cudaSetDevice(S->device);
  leiden_status st = LEIDEN_OK;
  std::string err;
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = LEIDEN_ERR_CUDA;
    err = "stream creation failed";
  }
  if (st == LEIDEN_OK) {
    st = leiden_create(&S->p, g->n, g->off.data(), g->col.data(), g->w.data(), g->stream, &g->h);
    if (st != LEIDEN_OK) err = leiden_last_error(nullptr);
  }
  if (st == LEIDEN_OK) {
    st = leiden_static(g->h, nullptr);
    if (st != LEIDEN_OK) err = leiden_last_error(g->h);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (st == LEIDEN_OK) {
    g->state = ServerGraph::READY;
    std::vector<int64_t>().swap(g->off);  // the device copy is the graph now
    std::vector<int32_t>().swap(g->col);
    std::vector<int32_t>().swap(g->w);
  } else {
    g->state = ServerGraph::FAILED;
    g->err = err;
    if (g->h) { leiden_destroy(g->h); g->h = nullptr; }
    if (g->stream) { cudaStreamDestroy(g->stream); g->stream = nullptr; }
    S->used -= g->bytes;
  }
}

// One request of graph g (lock not held; g is marked busy).
void serve(leiden_server *S, ServerGraph *g, ServerRequest *r) {
  cudaSetDevice(S->device);
  r->t_start = clock_type::now();
  if (r->keep) r->membership.resize((size_t)g->n);
  leiden_status st = leiden_update(g->h, r->del.data(), (int64_t)r->del.size(), r->ins.data(), (int64_t)r->ins.size(),
                                   r->mode, r->keep ? r->membership.data() : nullptr);
  r->status = st;
  if (st != LEIDEN_OK) r->err = leiden_last_error(g->h);
  r->t_done = clock_type::now();
}

void fail_queue(leiden_server *S, ServerGraph *g, leiden_status st, const std::string &why) {
  for (int64_t t : g->queue) {
    auto it = S->reqs.find(t);
    if (it == S->reqs.end()) continue;
    it->second->status = st;
    it->second->err = why;
    it->second->done = true;
    it->second->t_done = clock_type::now();
  }
  g->queue.clear();
}

void worker_loop(leiden_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    if (S->stop) return;
    // failed graphs answer their queued requests at once
    for (ServerGraph *g : S->graphs)
      if (g->state == ServerGraph::FAILED && !g->queue.empty()) {
        fail_queue(S, g, LEIDEN_ERR_OOM, "graph could not be admitted: " + g->err);
        S->cv_done.notify_all();
      }
    // admission by footprint, oldest graph first among those that fit
    ServerGraph *adm = nullptr;
    int64_t nslots = (int64_t)S->workers.size();
    for (ServerGraph *g : S->graphs)
      if (g->state == ServerGraph::PENDING &&
          S->used + g->bytes + nslots * std::max(S->max_agg, g->agg_bytes) <= S->budget) {
        adm = g;
        break;
      }
    if (adm) {
      adm->state = ServerGraph::ADMITTING;
      S->used += adm->bytes;
      S->max_agg = std::max(S->max_agg, adm->agg_bytes);
      S->running++;
      lk.unlock();
      admit(S, adm);
      lk.lock();
      S->running--;
      S->cv_work.notify_all();
      S->cv_done.notify_all();
      continue;
    }
    // the oldest request of a graph that is ready and not busy
    ServerGraph *pick = nullptr;
    int64_t best = 0;
    for (ServerGraph *g : S->graphs)
      if (g->state == ServerGraph::READY && !g->busy && !g->queue.empty() && (!pick || g->queue.front() < best)) {
        pick = g;
        best = g->queue.front();
      }
    if (pick) {
      int64_t t = pick->queue.front();
      pick->queue.pop_front();
      pick->busy = true;
      ServerRequest *r = S->reqs[t];
      S->running++;
      lk.unlock();
      serve(S, pick, r);
      lk.lock();
      S->running--;
      pick->busy = false;
      r->done = true;
      S->completed++;
      S->cv_done.notify_all();
      S->cv_work.notify_all();
      continue;
    }
    S->cv_work.wait(lk);
  }
}

thread_local std::string g_server_error;

}  // namespace

extern "C" {

leiden_status leiden_server_create(const leiden_params *params, int64_t device_bytes, int32_t slots,
                                   leiden_server **out) {
  g_server_error.clear();
  if (!out || device_bytes <= 0 || slots < 1 || slots > 256) {
    g_server_error = "invalid arguments (device_bytes > 0, 1 <= slots <= 256)";
    return LEIDEN_ERR_ARG;
  }
  leiden_server *S = new leiden_server();
  leiden_default_params(&S->p);
  if (params) S->p = *params;
  cudaGetDevice(&S->device);
  S->budget = device_bytes;
  for (int k = 0; k < slots; k++) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return LEIDEN_OK;
}

leiden_status leiden_server_add_graph(leiden_server *S, int64_t n, const int64_t *offsets, const int32_t *cols,
                                      const int32_t *weights, int32_t *graph_out) {
  if (!S || !graph_out || n < 1 || !offsets || (offsets[n] > 0 && !cols)) return LEIDEN_ERR_ARG;
  ServerGraph *g = new ServerGraph();
  g->n = n;
  g->off.assign(offsets, offsets + n + 1);
  g->col.assign(cols, cols + offsets[n]);
  if (weights) g->w.assign(weights, weights + offsets[n]);
  else g->w.assign((size_t)offsets[n], 1);
  g->bytes = leiden_footprint_bytes(&S->p, n, offsets);
  g->agg_bytes = leiden_transient_bytes(n, offsets);
  std::lock_guard<std::mutex> lk(S->mu);
  if (g->bytes + (int64_t)S->workers.size() * g->agg_bytes > S->budget) {
    delete g;
    S->err = "graph footprint exceeds the server's device budget";
    return LEIDEN_ERR_OOM;
  }
  *graph_out = (int32_t)S->graphs.size();
  S->graphs.push_back(g);
  S->cv_work.notify_all();
  return LEIDEN_OK;
}

leiden_status leiden_server_submit(leiden_server *S, int32_t graph, const leiden_edge *del, int64_t n_del,
                                   const leiden_edge *ins, int64_t n_ins, leiden_mode mode, int32_t keep_membership,
                                   int64_t *ticket_out) {
  if (!S || !ticket_out || n_del < 0 || n_ins < 0 || (n_del && !del) || (n_ins && !ins) || mode < LEIDEN_ND ||
      mode > LEIDEN_DF)
    return LEIDEN_ERR_ARG;
  ServerRequest *r = new ServerRequest();
  r->graph = graph;
  r->del.assign(del, del + n_del);
  r->ins.assign(ins, ins + n_ins);
  r->mode = mode;
  r->keep = keep_membership != 0;
  r->t_submit = clock_type::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (graph < 0 || graph >= (int32_t)S->graphs.size() || S->graphs[graph]->state == ServerGraph::REMOVED) {
    delete r;
    S->err = "unknown or removed graph";
    return LEIDEN_ERR_ARG;
  }
  int64_t t = S->next_ticket++;
  S->reqs[t] = r;
  S->graphs[graph]->queue.push_back(t);
  *ticket_out = t;
  S->cv_work.notify_one();
  return LEIDEN_OK;
}

leiden_status leiden_server_wait_for(leiden_server *S, int64_t ticket, double timeout_ms, int32_t *membership_out,
                                     double *latency_ms, double *service_ms) {
  if (!S) return LEIDEN_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) { S->err = "unknown ticket"; return LEIDEN_ERR_ARG; }
  ServerRequest *r = it->second;
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, [&] { return r->done; });
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] { return r->done; })) {
    S->err = "request not done within the time limit (the ticket stays valid)";
    return LEIDEN_ERR_TIMEOUT;
  }
  S->reqs.erase(it);
  lk.unlock();
  if (membership_out && r->keep && !r->membership.empty())
    memcpy(membership_out, r->membership.data(), r->membership.size() * sizeof(int32_t));
  using ms = std::chrono::duration<double, std::milli>;
  if (latency_ms) *latency_ms = ms(r->t_done - r->t_submit).count();
  if (service_ms) *service_ms = r->status == LEIDEN_OK ? ms(r->t_done - r->t_start).count() : 0.0;
  leiden_status st = r->status;
  if (st != LEIDEN_OK) {
    lk.lock();
    S->err = r->err;
  }
  delete r;
  return st;
}

leiden_status leiden_server_wait(leiden_server *S, int64_t ticket, int32_t *membership_out, double *latency_ms,
                                 double *service_ms) {
  return leiden_server_wait_for(S, ticket, -1.0, membership_out, latency_ms, service_ms);
}

leiden_status leiden_server_remove_graph(leiden_server *S, int32_t graph) {
  if (!S) return LEIDEN_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (graph < 0 || graph >= (int32_t)S->graphs.size()) return LEIDEN_ERR_ARG;
  ServerGraph *g = S->graphs[graph];
  // let its queued requests finish (a pending graph is admitted first)
  S->cv_done.wait(lk, [&] {
    return g->state == ServerGraph::FAILED || g->state == ServerGraph::REMOVED ||
           (g->state == ServerGraph::READY && !g->busy && g->queue.empty()) ||
           (g->state == ServerGraph::PENDING && g->queue.empty());
  });
  if (g->state == ServerGraph::REMOVED) return LEIDEN_OK;
  bool held = g->state == ServerGraph::READY;
  g->state = ServerGraph::REMOVED;
  leiden_handle *h = g->h;
  cudaStream_t st = g->stream;
  g->h = nullptr;
  g->stream = nullptr;
  lk.unlock();
  if (h) leiden_destroy(h);
  if (st) cudaStreamDestroy(st);
  lk.lock();
  if (held) S->used -= g->bytes;
  S->cv_work.notify_all();
  return LEIDEN_OK;
}

leiden_status leiden_server_membership(leiden_server *S, int32_t graph, int32_t *membership_out) {
  if (!S || !membership_out) return LEIDEN_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (graph < 0 || graph >= (int32_t)S->graphs.size()) return LEIDEN_ERR_ARG;
  ServerGraph *g = S->graphs[graph];
  S->cv_done.wait(lk, [&] {
    return g->state != ServerGraph::PENDING && g->state != ServerGraph::ADMITTING && !g->busy && g->queue.empty();
  });
  if (g->state != ServerGraph::READY) { S->err = "graph is not resident"; return LEIDEN_ERR_STATE; }
  g->busy = true;  // keep workers off it while it is read
  lk.unlock();
  cudaSetDevice(S->device);
  const int32_t *dC = nullptr;
  leiden_status st = leiden_membership_device(g->h, (const int32_t **)&dC);
  if (st == LEIDEN_OK && cudaMemcpyAsync(membership_out, dC, (size_t)g->n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                         g->stream) != cudaSuccess)
    st = LEIDEN_ERR_CUDA;
  if (st == LEIDEN_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) st = LEIDEN_ERR_CUDA;
  lk.lock();
  g->busy = false;
  S->cv_work.notify_all();
  return st;
}

leiden_status leiden_server_get_stats(leiden_server *S, leiden_server_stats *out) {
  if (!S || !out) return LEIDEN_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  for (ServerGraph *g : S->graphs) {
    if (g->state == ServerGraph::READY) out->graphs_resident++;
    if (g->state == ServerGraph::PENDING || g->state == ServerGraph::ADMITTING) out->graphs_waiting++;
    out->requests_queued += (int64_t)g->queue.size();
  }
  out->requests_done = S->completed;
  out->requests_running = S->running;
  out->bytes_used = S->used;
  out->bytes_budget = S->budget;
  return LEIDEN_OK;
}

const char *leiden_server_last_error(leiden_server *S) {
  if (!S) return g_server_error.c_str();
  std::lock_guard<std::mutex> lk(S->mu);
  thread_local std::string copy;
  copy = S->err;
  return copy.c_str();
}

void leiden_server_destroy(leiden_server *S) {
  if (!S) return;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->running == 0; });
    S->stop = true;
    S->cv_work.notify_all();
  }
  for (auto &t : S->workers) t.join();
  cudaSetDevice(S->device);
  for (ServerGraph *g : S->graphs) {
    if (g->h) leiden_destroy(g->h);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
  }
  for (auto &kv : S->reqs) delete kv.second;
  delete S;
}

}  // extern "C"
