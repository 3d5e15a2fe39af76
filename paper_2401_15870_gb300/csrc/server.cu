// server.cu -- a request loop over resident graphs: update batches arrive at
// any time for any graph, and one worker thread turns them into DF / DF-P
// updates.
//
// Grouped mode (continuous batching).  Each graph is IDLE, READY (its batch
// applied, its update not yet launched) or IN_FLIGHT (part of the running
// group update).  The worker repeats:
//   1. take the pending requests of every IDLE graph, admitted by free device
//      memory (the estimated scratch of each graph's batch must leave the
//      reserve free; the first graph is always admitted) and by a cap on the
//      edges of one round;
//   2. merge each graph's requests in arrival order into one batch (per edge
//      the last operation wins: applying the merged batch gives the same edge
//      set as applying the requests one after another, Sec. 3.2) and apply it
//      on the graphs' stream -- this overlaps with the group update already
//      running on the group stream;
//   3. hand the READY graphs to the device: a large graph (at least
//      PR_DEVICE_LOOP_SLOTS in-CSR slots) goes to the solo thread, which runs
//      pr_update on such graphs one after another (its host loop picks the
//      push or pull form per iteration, much cheaper than the pull-only group
//      form when a batch's frontier starts small on a large graph; large
//      updates run side by side would each take about as long as both in
//      turn, which only lengthens the first one's latency); the small graphs
//      -- those pr_update itself runs as a one-graph group -- go, when no
//      group update is running, into one group update (pr_group machinery)
//      together;
//   4. when the running group update has finished, complete its requests.
// Every graph has its own stream while the server runs, so a solo update, the
// group update and the batch edits of other graphs overlap on the device; the
// worker never waits for a solo update.  A request that arrives for a READY or
// IN_FLIGHT graph waits for the next round of that graph, so the batches of a
// graph are applied in arrival order.
//
// Plain mode: one pr_apply_batch + pr_update per request, in arrival order --
// the baseline the grouped mode is measured against.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>
#include "dfpr.h"
#include "group.cuh"
#include "handle.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t ticket;
  int32_t graph;
  double t_submit;
  std::vector<int32_t> ds, dd, is, id;
};

enum GraphState { IDLE = 0, READY = 1, IN_FLIGHT = 2 };

// device scratch a batch of e edges may need while it is applied (keys,
// sort buffers, flags, row staging), for admission
constexpr int64_t BYTES_PER_BATCH_EDGE = 160;
constexpr int64_t BYTES_PER_BATCH = 4 << 20;
// a graph with at least this many in-CSR slots is updated by the solo thread
// (pr_update), the others by group updates
bool large_graph(const pr_graph* g) { return g->g.in.cap >= PR_DEVICE_LOOP_SLOTS; }

}  // namespace

struct pr_server {
  pr_server_options opt;
  int32_t G = 0;
  std::vector<pr_graph*> graphs;
  std::vector<void*> old_streams;
  std::vector<cudaStream_t> streams;   // one per graph while the server runs
  cudaStream_t group_stream = nullptr;
  pr_group* group = nullptr;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> pending;
  std::unordered_map<int64_t, pr_request_info> results;
  int64_t next_ticket = 0;
  int64_t outstanding = 0;
  bool stop = false;
  std::thread worker;
  // solo updates: large graphs queued by the worker, run by the solo thread
  std::vector<std::thread> solo;
  std::condition_variable cv_solo;
  std::deque<std::pair<int32_t, int64_t>> solo_q;   // (graph, round)
  int solo_busy = 0;                                 // queued or running
  bool solo_stop = false;

  // worker-only state
  std::vector<int> state;
  std::vector<std::vector<Request>> ready_reqs;   // per graph, requests of its READY / IN_FLIGHT batch
  std::vector<double> t_start;
  std::vector<int32_t> members;
  std::vector<pr_stats> stats;
  int64_t round = 0;
  int64_t ready_bytes = 0, ready_edges = 0;   // admitted into the next round so far
};

namespace {

void finish_requests(pr_server* S, std::vector<Request>& reqs, int32_t status, int64_t round, double t0,
                     const pr_stats* st) {
  const double t = now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  for (Request& r : reqs) {
    pr_request_info info;
    memset(&info, 0, sizeof(info));
    info.ticket = r.ticket;
    info.graph = r.graph;
    info.status = status;
    info.round = round;
    info.merged = (int32_t)reqs.size();
    info.t_submit = r.t_submit;
    info.t_start = t0;
    info.t_done = t;
    if (st) info.stats = *st;
    S->results[r.ticket] = info;
    S->outstanding--;
  }
  reqs.clear();
  S->cv_done.notify_all();
}

// the requests of one graph merged in arrival order: per edge the last
// operation wins (deletions of a request before its insertions).  The
// requests' edge lists are not needed afterwards; a lone request's are moved.
void merge_requests(std::vector<Request>& reqs, std::vector<int32_t>* ds, std::vector<int32_t>* dd,
                    std::vector<int32_t>* is, std::vector<int32_t>* id) {
  if (reqs.size() == 1) {
    *ds = std::move(reqs[0].ds);
    *dd = std::move(reqs[0].dd);
    *is = std::move(reqs[0].is);
    *id = std::move(reqs[0].id);
    return;
  }
  size_t total = 0;
  for (const Request& r : reqs) total += r.ds.size() + r.is.size();
  std::unordered_map<uint64_t, char> last;
  last.reserve(total * 2);
  std::vector<uint64_t> order;
  order.reserve(total);
  auto put = [&](int32_t u, int32_t v, char op) {
    const uint64_t k = ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
    auto it = last.find(k);
    if (it == last.end()) {
      last.emplace(k, op);
      order.push_back(k);
    } else {
      it->second = op;
    }
  };
  for (const Request& r : reqs) {
    for (size_t i = 0; i < r.ds.size(); i++) put(r.ds[i], r.dd[i], 0);
    for (size_t i = 0; i < r.is.size(); i++) put(r.is[i], r.id[i], 1);
  }
  for (uint64_t k : order) {
    const int32_t u = (int32_t)(k >> 32), v = (int32_t)(uint32_t)k;
    if (last[k]) {
      is->push_back(u);
      id->push_back(v);
    } else {
      ds->push_back(u);
      dd->push_back(v);
    }
  }
}

int64_t free_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
  return (int64_t)fr;
}

void run_plain(pr_server* S) {
  for (;;) {
    Request r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->pending.empty()) return;   // stop with nothing left
      r = std::move(S->pending.front());
      S->pending.pop_front();
    }
    const double t0 = now_s();
    pr_graph* g = S->graphs[r.graph];
    pr_stats st;
    memset(&st, 0, sizeof(st));
    pr_status rc = pr_apply_batch(g, r.ds.data(), r.dd.data(), (int64_t)r.ds.size(), r.is.data(), r.id.data(),
                                  (int64_t)r.is.size());
    if (rc == PR_OK) rc = pr_update(g, (pr_method)S->opt.method, S->opt.alpha, S->opt.tau, &S->opt.opts, &st);
    std::vector<Request> one;
    one.push_back(std::move(r));
    finish_requests(S, one, rc, S->round++, t0, &st);
  }
}

// the solo thread: one pr_update per queued graph, in turn, each on the
// graph's own stream
void run_solo(pr_server* S) {
  for (;;) {
    std::pair<int32_t, int64_t> job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_solo.wait(lk, [&] { return S->solo_stop || !S->solo_q.empty(); });
      if (S->solo_q.empty()) return;
      job = S->solo_q.front();
      S->solo_q.pop_front();
    }
    const int32_t gi = job.first;
    pr_stats st;
    memset(&st, 0, sizeof(st));
    pr_status rc = pr_update(S->graphs[gi], (pr_method)S->opt.method, S->opt.alpha, S->opt.tau, &S->opt.opts, &st);
    finish_requests(S, S->ready_reqs[gi], rc, job.second, S->t_start[gi], &st);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->state[gi] = IDLE;
      S->solo_busy--;
    }
    S->cv_work.notify_all();
  }
}

void run_grouped(pr_server* S) {
  const int G = S->G;
  bool in_flight = false;
  int64_t flight_round = 0;
  for (;;) {
    // 1. admit the pending requests of idle graphs
    std::vector<std::vector<Request>> take(G);
    std::vector<int32_t> order;   // graphs in order of their first pending request
    {
      std::unique_lock<std::mutex> lk(S->mu);
      auto has_work = [&] {
        for (const Request& r : S->pending)
          if (S->state[r.graph] == IDLE) return true;
        return false;
      };
      // READY graphs that step 4 would hand to the device now
      auto can_launch = [&] {
        for (int i = 0; i < G; i++)
          if (S->state[i] == READY && (large_graph(S->graphs[i]) || !in_flight)) return true;
        return false;
      };
      if (!has_work() && !can_launch()) {
        if (in_flight) {
          S->cv_work.wait_for(lk, std::chrono::microseconds(50));   // poll the group update
        } else if (S->stop) {
          bool busy = S->solo_busy > 0 || !S->pending.empty();
          for (int i = 0; i < G; i++) busy = busy || S->state[i] != IDLE;
          if (!busy) return;                                          // every request is done
          S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
        } else {
          S->cv_work.wait(lk, [&] { return S->stop || has_work() || can_launch(); });
        }
      }
      // the next round holds the READY graphs and those admitted now; the
      // free device memory is asked for (a driver call) only when a request
      // after the round's first one is weighed
      bool have_free = false;
      int64_t free_b = 0;
      int64_t edges = S->ready_edges;
      bool any_ready = false;
      for (int i = 0; i < G; i++) any_ready = any_ready || S->state[i] == READY;
      std::vector<char> refused(G, 0);
      std::deque<Request> keep;
      for (Request& r : S->pending) {
        const int32_t gi = r.graph;
        if (S->state[gi] != IDLE || refused[gi]) {
          keep.push_back(std::move(r));
          continue;
        }
        const int64_t e = (int64_t)(r.ds.size() + r.is.size());
        const bool first = order.empty() && !any_ready;
        const bool new_graph = take[gi].empty();
        const int64_t need = (new_graph ? BYTES_PER_BATCH : 0) + BYTES_PER_BATCH_EDGE * e;
        if (!first && !have_free) {
          free_b = free_device_bytes() - S->opt.hbm_reserve - S->ready_bytes;
          have_free = true;
        }
        const bool fits_mem = first || need <= free_b;
        const bool fits_edges = S->opt.max_round_edges <= 0 || edges + e <= S->opt.max_round_edges;
        if (!first && (!fits_mem || !fits_edges)) {
          refused[gi] = 1;   // later requests of this graph wait too: arrival order
          keep.push_back(std::move(r));
          continue;
        }
        if (new_graph) order.push_back(gi);
        if (have_free) free_b -= need;
        edges += e;
        S->ready_bytes += need;
        S->ready_edges += e;
        take[gi].push_back(std::move(r));
      }
      S->pending.swap(keep);
    }
    // 2. merge and apply on each graph's stream, overlapping the running updates
    for (int32_t gi : order) {
      std::vector<int32_t> ds, dd, is, id;
      merge_requests(take[gi], &ds, &dd, &is, &id);
      const double t0 = now_s();
      pr_status rc = pr_apply_batch(S->graphs[gi], ds.data(), dd.data(), (int64_t)ds.size(), is.data(), id.data(),
                                    (int64_t)is.size());
      if (rc != PR_OK) {
        finish_requests(S, take[gi], rc, -1, t0, nullptr);
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->state[gi] = READY;
      }
      S->t_start[gi] = t0;
      S->ready_reqs[gi] = std::move(take[gi]);
    }
    // 3. complete the running group update
    if (in_flight && group_done(S->group)) {
      pr_status rc = group_complete(S->group, S->stats.data());
      for (int32_t gi : S->members) {
        finish_requests(S, S->ready_reqs[gi], rc, flight_round, S->t_start[gi], &S->stats[gi]);
        std::lock_guard<std::mutex> lk(S->mu);
        S->state[gi] = IDLE;
      }
      in_flight = false;
      S->cv_work.notify_all();
    }
    // 4. hand the READY graphs to the solo thread (large) or to one group
    //    update (small)
    std::vector<int32_t> big, small;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (int i = 0; i < G; i++)
        if (S->state[i] == READY) (large_graph(S->graphs[i]) ? big : small).push_back(i);
      for (int32_t gi : big) {
        S->state[gi] = IN_FLIGHT;
        S->solo_q.emplace_back(gi, S->round++);
        S->solo_busy++;
      }
    }
    if (!big.empty()) S->cv_solo.notify_all();
    if (big.empty() && small.empty()) continue;
    if (small.empty() || !in_flight) {
      S->ready_bytes = 0;
      S->ready_edges = 0;
    }
    if (!small.empty() && !in_flight) {
      S->members = small;
      pr_status rc = group_launch(S->group, (pr_method)S->opt.method, S->opt.alpha, S->opt.tau, &S->opt.opts,
                                  S->members.data(), (int32_t)S->members.size());
      if (rc != PR_OK) {
        for (int32_t gi : S->members) {
          finish_requests(S, S->ready_reqs[gi], rc, -1, S->t_start[gi], nullptr);
          std::lock_guard<std::mutex> lk(S->mu);
          S->state[gi] = IDLE;
        }
      } else {
        std::lock_guard<std::mutex> lk(S->mu);
        for (int32_t gi : S->members) S->state[gi] = IN_FLIGHT;
        in_flight = true;
        flight_round = S->round++;
      }
    }
  }
}

void server_free(pr_server* S) {
  if (!S) return;
  if (S->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    S->worker.join();
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->solo_stop = true;
  }
  S->cv_solo.notify_all();
  for (std::thread& t : S->solo)
    if (t.joinable()) t.join();
  if (S->group) pr_group_destroy(S->group);
  for (size_t i = 0; i < S->old_streams.size(); i++) pr_set_stream(S->graphs[i], S->old_streams[i]);
  for (cudaStream_t st : S->streams)
    if (st) cudaStreamDestroy(st);
  if (S->group_stream) cudaStreamDestroy(S->group_stream);
  delete S;
}

}  // namespace

extern "C" {

double pr_server_clock(void) { return now_s(); }

pr_status pr_server_create(int32_t count, pr_graph* const* graphs, const pr_server_options* opts,
                           pr_server** out) {
  if (!out || !opts) return PR_EINVAL;
  *out = nullptr;
  if (count < 1 || count > PR_GROUP_MAX || !graphs) return PR_EINVAL;
  if (opts->mode != PR_SERVE_GROUPED && opts->mode != PR_SERVE_PLAIN) return PR_EINVAL;
  if (opts->method != PR_DF && opts->method != PR_DFP) return PR_EINVAL;
  if (!(opts->alpha >= 0.0 && opts->alpha < 1.0) || !(opts->tau >= 0.0) || opts->hbm_reserve < 0) return PR_EINVAL;
  for (int32_t i = 0; i < count; i++)
    if (!graphs[i] || !graphs[i]->g.has_ranks) return graphs[i] ? PR_ENORANKS : PR_EINVAL;
  pr_server* S = new (std::nothrow) pr_server();
  if (!S) return PR_ENOMEM;
  S->opt = *opts;
  S->G = count;
  S->graphs.assign(graphs, graphs + count);
  S->state.assign(count, IDLE);
  S->ready_reqs.resize(count);
  S->t_start.assign(count, 0.0);
  S->stats.resize(count);
  if (cudaStreamCreateWithFlags(&S->group_stream, cudaStreamNonBlocking) != cudaSuccess) {
    server_free(S);
    return PR_ECUDA;
  }
  // every graph works on a stream of its own while the server runs
  // (pr_set_stream finishes the work queued on its old stream first)
  S->streams.assign(count, nullptr);
  for (int32_t i = 0; i < count; i++) {
    if (cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      server_free(S);
      return PR_ECUDA;
    }
    S->old_streams.push_back((void*)graphs[i]->g.stream);
    pr_status rc = pr_set_stream(graphs[i], S->streams[i]);
    if (rc != PR_OK) {
      server_free(S);
      return rc;
    }
  }
  if (opts->mode == PR_SERVE_GROUPED) {
    pr_status rc = pr_group_create(count, graphs, S->group_stream, &S->group);
    if (rc != PR_OK) {
      server_free(S);
      return rc;
    }
  }
  int dev = 0;
  cudaGetDevice(&dev);
  S->worker = std::thread([S, dev] {
    cudaSetDevice(dev);
    if (S->opt.mode == PR_SERVE_PLAIN) run_plain(S);
    else run_grouped(S);
  });
  if (opts->mode == PR_SERVE_GROUPED)
    S->solo.emplace_back([S, dev] {
      cudaSetDevice(dev);
      run_solo(S);
    });
  *out = S;
  return PR_OK;
}

pr_status pr_server_submit(pr_server* S, int32_t graph, const int32_t* del_src, const int32_t* del_dst,
                           int64_t n_del, const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                           int64_t* ticket) {
  if (!S || !ticket || graph < 0 || graph >= S->G || n_del < 0 || n_ins < 0) return PR_EINVAL;
  if ((n_del > 0 && (!del_src || !del_dst)) || (n_ins > 0 && (!ins_src || !ins_dst))) return PR_EINVAL;
  const int32_t n = S->graphs[graph]->g.n;
  for (int64_t i = 0; i < n_del; i++)
    if (del_src[i] < 0 || del_src[i] >= n || del_dst[i] < 0 || del_dst[i] >= n) return PR_ERANGE;
  for (int64_t i = 0; i < n_ins; i++)
    if (ins_src[i] < 0 || ins_src[i] >= n || ins_dst[i] < 0 || ins_dst[i] >= n) return PR_ERANGE;
  Request r;
  r.graph = graph;
  r.ds.assign(del_src, del_src + n_del);
  r.dd.assign(del_dst, del_dst + n_del);
  r.is.assign(ins_src, ins_src + n_ins);
  r.id.assign(ins_dst, ins_dst + n_ins);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return PR_EINVAL;
    r.ticket = S->next_ticket++;
    r.t_submit = now_s();
    *ticket = r.ticket;
    S->outstanding++;
    S->pending.push_back(std::move(r));
  }
  S->cv_work.notify_all();
  return PR_OK;
}

pr_status pr_server_wait(pr_server* S, int64_t ticket, double timeout_s, pr_request_info* info) {
  if (!S || ticket < 0) return PR_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket >= S->next_ticket) return PR_EINVAL;
  auto ready = [&] { return S->results.count(ticket) > 0; };
  if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return PR_ETIMEOUT;
  if (info) *info = S->results[ticket];
  return PR_OK;
}

pr_status pr_server_drain(pr_server* S, double timeout_s) {
  if (!S) return PR_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return S->outstanding == 0; }))
    return PR_ETIMEOUT;
  return PR_OK;
}

void pr_server_destroy(pr_server* S) { server_free(S); }

}  // extern "C"
