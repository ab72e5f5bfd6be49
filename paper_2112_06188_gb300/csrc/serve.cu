// serve.cu -- a request server around one resident forest: continuous
// batching of insert / erase / k-NN requests as they arrive, admission by a
// device-memory budget for the requests' own buffers, and per-request
// timestamps for latency percentiles.
//
// Semantics: requests take effect in submission order, exactly as if each
// had been issued alone by the plain calls (bdl_insert / bdl_erase /
// bdl_knn) in that order.  Batching only changes how they are launched:
//  * a run of consecutive k-NN requests reads one state of the forest, so the
//    run goes to the device as one k-NN launch (one job per request); a run
//    with one k may be as large as max_group_queries, a run of small requests
//    may mix k (up to kMixQueries queries in all): it is launched with the
//    largest k and each request's rows are cut to its own k on the way out --
//    the k nearest by (d2, id) are the first k of the kmax nearest, padding
//    included;
//  * a run of consecutive inserts is one Insert_L of the concatenated points:
//    the ids are the same consecutive ids and the live set afterwards is the
//    same, so every later answer is the same (k-NN results are exact and
//    unique under (d2, id));
//  * a run of consecutive erases is one Erase_L of all their ids, whose
//    marking pass takes the requests' lists in order, so that an id counts for
//    the first request that names it: each request's count is the one it gets
//    when the erases run one after another, and the live set afterwards is
//    the same.
//
// Three host threads move requests through three CUDA streams:
//   admission  -- takes submitted requests in order while the number in flight
//                 and their device bytes stay within the limits, allocates
//                 their device buffers and copies their inputs (copy-in
//                 stream);
//   execution  -- forms groups from the admitted requests and runs them on the
//                 compute stream after their inputs have arrived, then queues
//                 the copies of their outputs (copy-out stream);
//   completion -- waits for each group's outputs, stamps the requests done,
//                 frees their buffers and wakes admission and waiters.
// So the inputs of later requests and the outputs of earlier ones move while
// the current group computes, and requests that arrive meanwhile join the
// next group.  With `serial` set, every request is its own group and the
// next one is admitted only after the previous one completed: the plain
// one-request-at-a-time path, for comparison.
#include "bdl_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace bdl {

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  bdl_request r{};
  size_t in_bytes = 0, out_bytes = 0;
  void *d_in = nullptr;             // device copy of the input
  void *d_out = nullptr;            // device outputs (k-NN: ids then d2)
  cudaEvent_t ev_in = nullptr;      // input copy done
  bdl_result res{};
};

struct Group {
  std::vector<Req *> reqs;
  cudaEvent_t ev_out = nullptr;     // outputs copied back
  void *merged = nullptr;           // merged insert input, or a mixed-k k-NN run's outputs
  size_t merged_bytes = 0;
};

constexpr int64_t kMixQueries = 1 << 15;   // a k-NN run that mixes k stays this small

}  // namespace
}  // namespace bdl

struct bdl_server {
  bdl_forest *f = nullptr;
  bdl_server_config cfg{};
  cudaMemPool_t pool = nullptr;
  cudaStream_t s_in = nullptr, s_exec = nullptr, s_out = nullptr;
  bdl::Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit, cv_exec, cv_done, cv_wait;
  std::deque<bdl::Req *> submitted, admitted;
  std::deque<bdl::Group *> finishing;
  std::unordered_map<uint64_t, bdl::Req *> live;      // tickets not yet collected
  uint64_t next_ticket = 1;
  int inflight = 0;                 // admitted, not completed
  int64_t staged = 0;               // device bytes of admitted requests
  int64_t groups = 0;
  bool stop = false;
  std::thread th_admit, th_exec, th_done;
  std::vector<cudaEvent_t> spare_events;
};

namespace bdl {
namespace {

double ms_since(const bdl_server *S) {
  return std::chrono::duration<double, std::milli>(Clock::now() - S->t0).count();
}

cudaEvent_t get_event(bdl_server *S) {   // caller holds S->mu
  if (!S->spare_events.empty()) {
    cudaEvent_t e = S->spare_events.back();
    S->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

void request_bytes(const bdl_forest *f, Req *q) {
  const int64_t n = q->r.n;
  switch (q->r.kind) {
    case BDL_REQ_INSERT: q->in_bytes = (size_t)n * f->dim * 4; q->out_bytes = 0; break;
    case BDL_REQ_ERASE: q->in_bytes = (size_t)n * 4; q->out_bytes = 0; break;
    default:
      q->in_bytes = (size_t)n * f->dim * 4;
      q->out_bytes = (size_t)n * q->r.k * 12;
      break;
  }
}

void admission_loop(bdl_server *S) {
  cudaSetDevice(S->f->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    S->cv_admit.wait(lk, [&] {
      if (S->stop && S->submitted.empty()) return true;
      if (S->submitted.empty()) return false;
      const Req *q = S->submitted.front();
      const int64_t b = (int64_t)(q->in_bytes + q->out_bytes);
      if (S->cfg.serial) return S->inflight == 0;
      if (S->inflight >= S->cfg.max_inflight) return false;
      // a request larger than the whole budget goes alone
      return S->inflight == 0 || S->staged + b <= S->cfg.staging_budget_bytes;
    });
    if (S->submitted.empty()) return;   // stopping
    Req *q = S->submitted.front();
    S->submitted.pop_front();
    S->inflight++;
    S->staged += (int64_t)(q->in_bytes + q->out_bytes);
    q->ev_in = get_event(S);
    lk.unlock();
    int st = BDL_OK;
    if (q->in_bytes) {
      st = cuda_check(cudaMallocFromPoolAsync(&q->d_in, q->in_bytes, S->pool, S->s_in), "staging");
      if (!st) st = cuda_check(cudaMemcpyAsync(q->d_in, q->r.in_host, q->in_bytes, cudaMemcpyHostToDevice,
                                               S->s_in), "request input copy");
    }
    if (!st && q->out_bytes)
      st = cuda_check(cudaMallocFromPoolAsync(&q->d_out, q->out_bytes, S->pool, S->s_in), "staging");
    if (st) {
      if (q->d_in) cudaFreeAsync(q->d_in, S->s_in);
      if (q->d_out) cudaFreeAsync(q->d_out, S->s_in);
      q->d_in = q->d_out = nullptr;
    }
    cudaEventRecord(q->ev_in, S->s_in);
    q->res.status = st;
    lk.lock();
    S->admitted.push_back(q);
    S->cv_exec.notify_one();
  }
}

// Take the next group off the admitted queue (caller holds S->mu).
Group *form_group(bdl_server *S) {
  Group *g = new Group();
  Req *first = S->admitted.front();
  S->admitted.pop_front();
  g->reqs.push_back(first);
  if (S->cfg.serial || first->res.status) return g;
  const int kind = first->r.kind;
  int64_t total = first->r.n;
  const int64_t cap = kind == BDL_REQ_KNN ? S->cfg.max_group_queries : S->cfg.max_group_points;
  bool mixed = false;
  while (!S->admitted.empty()) {
    Req *q = S->admitted.front();
    if (q->res.status || q->r.kind != kind) break;
    if (total + q->r.n > cap) break;
    if (kind == BDL_REQ_KNN) {
      const bool mx = mixed || q->r.k != first->r.k;
      if (mx && total + q->r.n > kMixQueries) break;
      mixed = mx;
    }
    total += q->r.n;
    g->reqs.push_back(q);
    S->admitted.pop_front();
  }
  return g;
}

int run_insert(bdl_server *S, Group *g) {
  bdl_forest *f = S->f;
  int64_t n = 0;
  for (Req *q : g->reqs) n += q->r.n;
  const int32_t *pts = (const int32_t *)g->reqs[0]->d_in;
  bool one_by_one = false;
  if (g->reqs.size() > 1 && n > 0) {       // concatenate the inputs
    g->merged_bytes = (size_t)n * f->dim * 4;
    if (cudaMallocFromPoolAsync(&g->merged, g->merged_bytes, S->pool, S->s_exec) != cudaSuccess) {
      cudaGetLastError();
      g->merged = nullptr;
      one_by_one = true;                   // no room to merge: same results, one call each
    }
  }
  if (g->merged) {
    size_t off = 0;
    for (Req *q : g->reqs) {
      if (q->in_bytes)
        cudaMemcpyAsync((char *)g->merged + off, q->d_in, q->in_bytes, cudaMemcpyDeviceToDevice, S->s_exec);
      off += q->in_bytes;
    }
    pts = (const int32_t *)g->merged;
  }
  const int64_t first_id = f->next_id;
  int st = one_by_one ? BDL_EINVAL : bdl_insert(f, pts, n, nullptr, S->s_exec);
  if (st == BDL_EINVAL && g->reqs.size() > 1) {
    // one of them is bad: run them one by one so each gets its own status
    for (Req *q : g->reqs) {
      const int64_t fid = f->next_id;
      q->res.status = bdl_insert(f, (const int32_t *)q->d_in, q->r.n, nullptr, S->s_exec);
      if (!q->res.status && q->r.out_ids_host)
        for (int64_t j = 0; j < q->r.n; ++j) q->r.out_ids_host[j] = (int32_t)(fid + j);
      q->res.n_done = q->res.status ? 0 : q->r.n;
    }
    return BDL_OK;
  }
  int64_t id = first_id;
  for (Req *q : g->reqs) {
    q->res.status = st;
    q->res.n_done = st ? 0 : q->r.n;
    if (!st && q->r.out_ids_host)
      for (int64_t j = 0; j < q->r.n; ++j) q->r.out_ids_host[j] = (int32_t)(id + j);
    id += q->r.n;
  }
  return BDL_OK;
}

// A run of erases: one Erase_L over the requests' lists in order.
void run_erase(bdl_server *S, Group *g) {
  std::vector<const int32_t *> ids;
  std::vector<int64_t> n, cnt(g->reqs.size(), 0);
  for (Req *q : g->reqs) {
    ids.push_back((const int32_t *)q->d_in);
    n.push_back(q->r.n);
  }
  const int st = erase_lists(S->f, ids, n, cnt.data(), S->s_exec);
  for (size_t j = 0; j < g->reqs.size(); ++j) {
    g->reqs[j]->res.status = st;
    g->reqs[j]->res.n_done = cnt[j];
  }
}

// A run of k-NN requests: one launch.  Same k: each request's rows go to its
// own device buffer.  Mixed k: one launch with the largest k into a group
// buffer, each request's rows cut to its k by 2-D copies; without room for
// that buffer, each request runs by itself (same rows).
void run_knn(bdl_server *S, Group *g) {
  const size_t nr = g->reqs.size();
  int kmax = 0;
  int64_t rows = 0;
  bool mixed = false;
  for (Req *q : g->reqs) {
    kmax = std::max(kmax, (int)q->r.k);
    mixed = mixed || q->r.k != g->reqs[0]->r.k;
    rows += q->r.n;
  }
  std::vector<bdl_forest *> F(nr, S->f);
  std::vector<const int32_t *> qv(nr);
  std::vector<int64_t> mv(nr);
  std::vector<int32_t *> oi(nr);
  std::vector<int64_t *> od(nr);
  if (mixed && rows > 0) {
    g->merged_bytes = (size_t)rows * kmax * 12;
    if (cudaMallocFromPoolAsync(&g->merged, g->merged_bytes, S->pool, S->s_exec) != cudaSuccess) {
      cudaGetLastError();
      g->merged = nullptr;
    }
  }
  int64_t row = 0;
  for (size_t j = 0; j < nr; ++j) {
    Req *q = g->reqs[j];
    qv[j] = (const int32_t *)q->d_in;
    mv[j] = q->r.n;
    if (g->merged) {     // [rows][kmax] d2, then [rows][kmax] ids
      od[j] = (int64_t *)g->merged + row * kmax;
      oi[j] = (int32_t *)((int64_t *)g->merged + rows * kmax) + row * kmax;
    } else {
      od[j] = (int64_t *)q->d_out;
      oi[j] = (int32_t *)((char *)q->d_out + (size_t)q->r.n * q->r.k * 8);
    }
    row += q->r.n;
  }
  std::vector<int> st(nr, BDL_OK);
  if (!mixed || g->merged) {
    const int s1 = bdl_knn_batch(F.data(), (int)nr, qv.data(), mv.data(), kmax, oi.data(), od.data(), S->s_exec);
    std::fill(st.begin(), st.end(), s1);
  } else {
    for (size_t j = 0; j < nr; ++j)
      st[j] = bdl_knn(S->f, qv[j], mv[j], g->reqs[j]->r.k, oi[j], od[j], S->s_exec);
  }
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ev = get_event(S);
  }
  cudaEventRecord(ev, S->s_exec);
  cudaStreamWaitEvent(S->s_out, ev, 0);
  for (size_t j = 0; j < nr; ++j) {
    Req *q = g->reqs[j];
    q->res.status = st[j];
    q->res.n_done = st[j] ? 0 : q->r.n;
    if (st[j] || q->r.n == 0) continue;
    const int k = q->r.k;
    const int w = g->merged ? kmax : k;     // row width on the device
    if (q->r.out_d2_host)
      cudaMemcpy2DAsync(q->r.out_d2_host, (size_t)k * 8, od[j], (size_t)w * 8, (size_t)k * 8, (size_t)q->r.n,
                        cudaMemcpyDeviceToHost, S->s_out);
    if (q->r.out_ids_host)
      cudaMemcpy2DAsync(q->r.out_ids_host, (size_t)k * 4, oi[j], (size_t)w * 4, (size_t)k * 4, (size_t)q->r.n,
                        cudaMemcpyDeviceToHost, S->s_out);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->spare_events.push_back(ev);   // recorded already; reuse after the group completes is safe
}

void run_group(bdl_server *S, Group *g) {
  for (Req *q : g->reqs) cudaStreamWaitEvent(S->s_exec, q->ev_in, 0);
  const double t = ms_since(S);
  for (Req *q : g->reqs) {
    q->res.t_start_ms = t;
    q->res.group = S->groups;
  }
  S->groups++;
  Req *first = g->reqs[0];
  if (first->res.status) {
    // admission failed (no memory for its buffers): nothing to run
  } else if (first->r.kind == BDL_REQ_INSERT) {
    run_insert(S, g);
  } else if (first->r.kind == BDL_REQ_ERASE) {
    run_erase(S, g);
  } else {
    run_knn(S, g);
  }
  // buffers are released on the copy-out stream after everything that reads them
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ev = get_event(S);
  }
  cudaEventRecord(ev, S->s_exec);
  cudaStreamWaitEvent(S->s_out, ev, 0);
  for (Req *q : g->reqs) {
    if (q->d_in) cudaFreeAsync(q->d_in, S->s_out);
    if (q->d_out) cudaFreeAsync(q->d_out, S->s_out);
    q->d_in = q->d_out = nullptr;
  }
  if (g->merged) cudaFreeAsync(g->merged, S->s_out);
  g->merged = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->spare_events.push_back(ev);
    g->ev_out = get_event(S);
  }
  cudaEventRecord(g->ev_out, S->s_out);
}

void exec_loop(bdl_server *S) {
  cudaSetDevice(S->f->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    S->cv_exec.wait(lk, [&] { return !S->admitted.empty() || (S->stop && S->submitted.empty() &&
                                                              S->inflight == 0); });
    if (S->admitted.empty()) return;
    Group *g = form_group(S);
    lk.unlock();
    run_group(S, g);
    lk.lock();
    S->finishing.push_back(g);
    S->cv_done.notify_one();
  }
}

void done_loop(bdl_server *S) {
  cudaSetDevice(S->f->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    S->cv_done.wait(lk, [&] { return !S->finishing.empty() || (S->stop && S->inflight == 0); });
    if (S->finishing.empty()) return;
    Group *g = S->finishing.front();
    S->finishing.pop_front();
    lk.unlock();
    const cudaError_t e = cudaEventSynchronize(g->ev_out);
    const double t = ms_since(S);
    lk.lock();
    for (Req *q : g->reqs) {
      if (e != cudaSuccess && !q->res.status) q->res.status = BDL_ECUDA;
      q->res.t_done_ms = t;
      S->spare_events.push_back(q->ev_in);
      q->ev_in = nullptr;
      S->staged -= (int64_t)(q->in_bytes + q->out_bytes);
      S->inflight--;
      q->res.kind = q->r.kind;
      q->res.ticket = q->ticket;
      q->res.done = 1;
    }
    S->spare_events.push_back(g->ev_out);
    delete g;
    S->cv_admit.notify_one();
    S->cv_exec.notify_one();
    S->cv_wait.notify_all();
  }
}

}  // namespace
}  // namespace bdl

using namespace bdl;

extern "C" {

void bdl_server_default_config(bdl_server_config *cfg) {
  if (!cfg) return;
  cfg->max_inflight = 64;
  cfg->serial = 0;
  cfg->staging_budget_bytes = (int64_t)1 << 30;
  cfg->max_group_queries = (int64_t)1 << 20;
  cfg->max_group_points = (int64_t)1 << 21;
}

int bdl_server_create(bdl_forest *f, const bdl_server_config *cfg, bdl_server **out) {
  if (!out) return set_error(BDL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  bdl_server_config c;
  bdl_server_default_config(&c);
  if (cfg) c = *cfg;
  if (c.max_inflight < 1 || c.staging_budget_bytes < 0 || c.max_group_queries < 1 || c.max_group_points < 1)
    return set_error(BDL_EINVAL, "bad server config");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != f->device) cudaSetDevice(f->device);
  bdl_server *S = new bdl_server();
  S->f = f;
  S->cfg = c;
  S->pool = f->pool;
  S->t0 = Clock::now();
  int st = cuda_check(cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!st) st = cuda_check(cudaStreamCreateWithFlags(&S->s_exec, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!st) st = cuda_check(cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking), "cudaStreamCreate");
  if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
  if (st) {
    if (S->s_in) cudaStreamDestroy(S->s_in);
    if (S->s_exec) cudaStreamDestroy(S->s_exec);
    if (S->s_out) cudaStreamDestroy(S->s_out);
    delete S;
    return st;
  }
  S->th_admit = std::thread(admission_loop, S);
  S->th_exec = std::thread(exec_loop, S);
  S->th_done = std::thread(done_loop, S);
  *out = S;
  return BDL_OK;
}

int bdl_server_submit(bdl_server *S, const bdl_request *req, uint64_t *out_ticket) {
  if (!S || !req) return set_error(BDL_EINVAL, "NULL pointer");
  if (req->kind != BDL_REQ_INSERT && req->kind != BDL_REQ_ERASE && req->kind != BDL_REQ_KNN)
    return set_error(BDL_EINVAL, "unknown request kind");
  if (req->n < 0) return set_error(BDL_EINVAL, "n < 0");
  if (req->n > 0 && !req->in_host) return set_error(BDL_EINVAL, "in_host is NULL");
  if (req->kind == BDL_REQ_KNN) {
    if (req->k < 1 || req->k > kMaxK) return set_error(BDL_EINVAL, "k must be in 1..32");
    if (req->n > 0 && (!req->out_ids_host || !req->out_d2_host))
      return set_error(BDL_EINVAL, "k-NN outputs are NULL");
  }
  Req *q = new Req();
  q->r = *req;
  request_bytes(S->f, q);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    delete q;
    return set_error(BDL_EINVAL, "server is stopping");
  }
  q->ticket = S->next_ticket++;
  q->res.t_submit_ms = ms_since(S);
  S->live[q->ticket] = q;
  S->submitted.push_back(q);
  if (out_ticket) *out_ticket = q->ticket;
  S->cv_admit.notify_one();
  return BDL_OK;
}

int bdl_server_wait(bdl_server *S, uint64_t ticket, bdl_result *out) {
  if (!S) return set_error(BDL_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) return set_error(BDL_EINVAL, "unknown or already collected ticket");
  Req *q = it->second;
  S->cv_wait.wait(lk, [&] { return q->res.done != 0; });
  if (out) *out = q->res;
  S->live.erase(it);
  delete q;
  return BDL_OK;
}

int bdl_server_drain(bdl_server *S) {
  if (!S) return set_error(BDL_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_wait.wait(lk, [&] { return S->submitted.empty() && S->inflight == 0; });
  return BDL_OK;
}

double bdl_server_now_ms(const bdl_server *S) { return S ? ms_since(S) : 0.0; }

int bdl_server_stats(const bdl_server *S, int64_t *out_groups) {
  if (!S) return set_error(BDL_EINVAL, "server is NULL");
  if (out_groups) *out_groups = S->groups;
  return BDL_OK;
}

int bdl_server_destroy(bdl_server *S) {
  if (!S) return BDL_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_admit.notify_all();
  S->cv_exec.notify_all();
  S->cv_done.notify_all();
  S->th_admit.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
  }
  S->cv_exec.notify_all();
  S->th_exec.join();
  S->cv_done.notify_all();
  S->th_done.join();
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != S->f->device) cudaSetDevice(S->f->device);
  cudaStreamSynchronize(S->s_out);
  for (auto &kv : S->live) delete kv.second;
  for (cudaEvent_t e : S->spare_events) cudaEventDestroy(e);
  cudaStreamDestroy(S->s_in);
  cudaStreamDestroy(S->s_exec);
  cudaStreamDestroy(S->s_out);
  if (prev >= 0 && prev != S->f->device) cudaSetDevice(prev);
  delete S;
  return BDL_OK;
}

}  // extern "C"
