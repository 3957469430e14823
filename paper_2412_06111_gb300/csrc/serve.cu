// Serving loop: many resident sketch streams on one GPU, updated by a
// continuous stream of requests (the streaming use of Sec. 4: sketches are
// linear in the tensor, so every update is folded in as it arrives, and
// recovery runs whenever a caller asks for the current approximation).
//
// Worker threads own the device work, each with its own CUDA stream and
// request queue (server stream k goes to worker k % workers).  A worker takes
// batches from its queue -- at most one request per stream per batch, so
// every stream sees its requests in submission order -- launches the
// first-level pass of every update in the batch, then runs the tree walks of
// all of them as one merged program (each dependency level of every walk in
// one launch), then the recoveries; the box side blocks of the whole batch
// are cut from the cached blocks in one gather launch first.  Completion is
// tracked by CUDA events, so a worker records the next batch while the device
// runs the previous ones.  Streams are admitted while the device memory of
// all open streams stays within the server's budget.  Every wait of a
// caller is bounded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "plan.cuh"

namespace ttnn {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int kind;             // 0 update, 1 recover
  int stream;
  uint64_t ticket;
  const void* data;
  Box box;
  const float* scale;
  double lambda;
  double* cores;
  int64_t bytes;        // tensor bytes of an update
  Clock::time_point t0;
};

struct Done {
  ttnn_status status;
  std::string msg;
};

struct Slot {
  ttnn_plan_t plan = nullptr;
  ttnn_state_t state = nullptr;
  int64_t bytes = 0;
  int pending = 0;
};

}  // namespace
}  // namespace ttnn

using namespace ttnn;

// One worker: its own CUDA stream and request queue; stream k of the server
// is served by worker k % (number of workers), so each stream's requests
// stay in order on one CUDA stream while workers record in parallel.
struct Worker {
  cudaStream_t st = nullptr;
  std::deque<Request> queue;
  std::condition_variable cv_work;
  std::thread thread;
};

struct ttnn_server_s {
  int device = 0;
  cudaStream_t st_admin = nullptr;  // plan creation
  int64_t budget = 0, used = 0;
  int max_batch = 64;
  size_t capacity = 65536;
  int stream_capacity = 0;   // outstanding requests per stream (0: unbounded)
  size_t queued = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::vector<Worker> workers;
  std::map<int, Slot> slots;
  std::map<uint64_t, Done> done;
  std::set<uint64_t> inflight;
  int next_stream = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  // statistics since the last reset
  std::vector<double> lat_us;
  int64_t n_updates = 0, n_recovers = 0, n_batches = 0, n_failed = 0, bytes = 0;
  double host_s = 0;   // worker time spent recording and launching batches
  Clock::time_point since = Clock::now();
};

namespace ttnn {
namespace {

int store_bytes_of(const ttnn_plan_s& P) {
  return P.pass_store == 0 ? 8 : P.pass_store == 1 ? 4 : P.pass_store == 2 ? 2 : 1;
}

void finish(ttnn_server_s& S, const Request& r, ttnn_status s, const std::string& msg,
            Clock::time_point t1) {
  S.done[r.ticket] = Done{s, msg};
  S.inflight.erase(r.ticket);
  auto it = S.slots.find(r.stream);
  if (it != S.slots.end()) --it->second.pending;
  S.lat_us.push_back(std::chrono::duration<double, std::micro>(t1 - r.t0).count());
  if (s != TTNN_OK) ++S.n_failed;
  if (r.kind == 0) {
    ++S.n_updates;
    S.bytes += r.bytes;
  } else {
    ++S.n_recovers;
  }
}

// A batch whose device work has been enqueued; done when its event is.
struct InFlight {
  cudaEvent_t ev = nullptr;
  std::vector<Request> reqs;
  std::vector<ttnn_status> st;
  std::vector<std::string> msg;
};

constexpr int kMaxInFlight = 4;

void complete(ttnn_server_s* S, InFlight& f, ttnn_status ev_status, const std::string& ev_msg) {
  const Clock::time_point t1 = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < f.reqs.size(); ++i) {
      ttnn_status s = f.st[i];
      std::string m = f.msg[i];
      if (s == TTNN_OK && ev_status != TTNN_OK) {
        s = ev_status;
        m = ev_msg;
      }
      finish(*S, f.reqs[i], s, m, t1);
    }
    ++S->n_batches;
  }
  S->cv_done.notify_all();
}

// Completes the oldest in-flight batch, waiting for it if `block`.
bool retire(ttnn_server_s* S, std::deque<InFlight>& q, std::vector<cudaEvent_t>& pool, bool block) {
  if (q.empty()) return false;
  InFlight& f = q.front();
  cudaError_t e = block ? cudaEventSynchronize(f.ev) : cudaEventQuery(f.ev);
  if (e == cudaErrorNotReady) return false;
  ttnn_status es = TTNN_OK;
  std::string em;
  if (e != cudaSuccess) {
    cudaGetLastError();
    es = TTNN_ECUDA;
    em = std::string("serving batch: ") + cudaGetErrorString(e);
  }
  complete(S, f, es, em);
  pool.push_back(f.ev);
  q.pop_front();
  return true;
}

void worker_main(ttnn_server_s* S, int k) {
  cudaSetDevice(S->device);
  Worker& W = S->workers[k];
  std::deque<InFlight> inflight;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<ttnn_plan_s*, ttnn_state_s*>> who;
  while (true) {
    while (retire(S, inflight, pool, false)) {
    }
    InFlight f;
    who.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (inflight.empty())
        W.cv_work.wait_for(lk, std::chrono::milliseconds(50),
                           [&] { return S->stop || !W.queue.empty(); });
      if (S->stop && W.queue.empty() && inflight.empty()) break;
      // one request per stream per batch, in queue order; a stream whose
      // earlier request was deferred defers all its later ones too
      std::set<int> in_batch, blocked;
      for (auto it = W.queue.begin();
           it != W.queue.end() && (int)f.reqs.size() < S->max_batch;) {
        if (blocked.count(it->stream) || in_batch.count(it->stream)) {
          blocked.insert(it->stream);
          ++it;
          continue;
        }
        in_batch.insert(it->stream);
        f.reqs.push_back(*it);
        auto& sl = S->slots.at(it->stream);
        who.emplace_back(sl.plan, sl.state);
        it = W.queue.erase(it);
        --S->queued;
      }
    }
    if (f.reqs.empty()) {
      // nothing new: wait for the oldest batch on the device
      retire(S, inflight, pool, true);
      continue;
    }
    const Clock::time_point th0 = Clock::now();
    const size_t nb = f.reqs.size();
    f.st.assign(nb, TTNN_OK);
    f.msg.assign(nb, std::string());
    // updates: the batch's box side blocks in one gather, then every
    // first-level pass, then the walks as one merged program
    UpdateBatch ub;
    for (size_t i = 0; i < nb; ++i) {
      const Request& r = f.reqs[i];
      if (r.kind != 0) continue;
      f.st[i] = run_dense_update(*who[i].first, who[i].second->acc, r.data, r.box, r.scale,
                                 r.lambda, W.st, false, nullptr, &ub);
      if (f.st[i] != TTNN_OK) f.msg[i] = last_error();
    }
    const ttnn_status ms = ub.launch(W.st);
    if (ms != TTNN_OK) {
      const std::string m = last_error();
      for (size_t i = 0; i < nb; ++i)
        if (f.reqs[i].kind == 0 && f.st[i] == TTNN_OK) {
          f.st[i] = ms;
          f.msg[i] = m;
        }
    }
    // recoveries (each waits for the stream's earlier work: it reads the
    // kept ranks back)
    for (size_t i = 0; i < nb; ++i) {
      const Request& r = f.reqs[i];
      if (r.kind != 1) continue;
      f.st[i] = run_recover(*who[i].first, who[i].second->acc, r.cores, W.st, false, nullptr);
      if (f.st[i] != TTNN_OK) f.msg[i] = last_error();
    }
    if (pool.empty()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(W.st);
        while (retire(S, inflight, pool, true)) {
        }
        complete(S, f, TTNN_OK, "");
        continue;
      }
      pool.push_back(e);
    }
    f.ev = pool.back();
    pool.pop_back();
    cudaEventRecord(f.ev, W.st);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->host_s += std::chrono::duration<double>(Clock::now() - th0).count();
    }
    inflight.push_back(std::move(f));
    if ((int)inflight.size() > kMaxInFlight) retire(S, inflight, pool, true);
  }
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace
}  // namespace ttnn

extern "C" {

ttnn_status ttnn_server_create(const ttnn_server_opts* opts, ttnn_server_t* out) {
  TTNN_CHECK_ARG(opts && out, "null argument");
  TTNN_CHECK_ARG(opts->hbm_budget_bytes > static_scratch_resident_bytes(),
                 "hbm_budget_bytes must exceed the library's %lld-byte static scratch block",
                 (long long)static_scratch_resident_bytes());
  *out = nullptr;
  ttnn_server_s* S = new (std::nothrow) ttnn_server_s();
  if (!S) {
    set_error("host allocation failed");
    return TTNN_ENOMEM;
  }
  // the library's static scratch block is resident beside the streams
  S->budget = opts->hbm_budget_bytes - static_scratch_resident_bytes();
  S->max_batch = opts->max_batch > 0 ? opts->max_batch : 64;
  S->capacity = opts->queue_capacity > 0 ? (size_t)opts->queue_capacity : 65536;
  S->stream_capacity = opts->stream_queue_capacity > 0 ? opts->stream_queue_capacity : 0;
  const int nw = opts->workers > 0 ? std::min(opts->workers, 64) : 4;
  S->workers = std::vector<Worker>(nw);
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st_admin, cudaStreamNonBlocking);
  for (int k = 0; k < nw && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithFlags(&S->workers[k].st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("server streams: %s", cudaGetErrorString(e));
    for (auto& w : S->workers)
      if (w.st) cudaStreamDestroy(w.st);
    if (S->st_admin) cudaStreamDestroy(S->st_admin);
    delete S;
    return TTNN_ECUDA;
  }
  try {
    for (int k = 0; k < nw; ++k) S->workers[k].thread = std::thread(worker_main, S, k);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    for (auto& w : S->workers) {
      w.cv_work.notify_all();
      if (w.thread.joinable()) w.thread.join();
      cudaStreamDestroy(w.st);
    }
    cudaStreamDestroy(S->st_admin);
    delete S;
    set_error("cannot start the server threads");
    return TTNN_ENOMEM;
  }
  *out = S;
  return TTNN_OK;
}

void ttnn_server_destroy(ttnn_server_t S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  for (auto& w : S->workers) {
    w.cv_work.notify_all();
    if (w.thread.joinable()) w.thread.join();
  }
  for (auto& kv : S->slots) {
    ttnn_state_destroy(kv.second.state);
    ttnn_plan_destroy(kv.second.plan);
  }
  for (auto& w : S->workers) cudaStreamDestroy(w.st);
  cudaStreamDestroy(S->st_admin);
  delete S;
}

ttnn_status ttnn_server_open(ttnn_server_t S, const ttnn_tree* tree, int32_t d, const int64_t* dims,
                             const int32_t* ranks, const int32_t* oversample, uint64_t seed,
                             const ttnn_opts* opts, int32_t* stream_id) {
  TTNN_CHECK_ARG(S && stream_id, "null argument");
  ttnn_plan_t plan = nullptr;
  TTNN_TRY(ttnn_plan_create(tree, d, dims, ranks, oversample, seed, opts, S->st_admin, &plan));
  ttnn_state_t state = nullptr;
  ttnn_status s = ttnn_state_create(plan, S->st_admin, &state);
  if (s == TTNN_OK && cudaStreamSynchronize(S->st_admin) != cudaSuccess) {
    cudaGetLastError();
    set_error("server open: stream synchronisation failed");
    s = TTNN_ECUDA;
  }
  if (s != TTNN_OK) {
    ttnn_plan_destroy(plan);
    return s;
  }
  const int64_t bytes = plan->dev_bytes + state->elems * (plan->walk_f64 ? 8 : 4);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->used + bytes > S->budget) {
    ttnn_state_destroy(state);
    ttnn_plan_destroy(plan);
    set_error("admission: stream needs %lld bytes, %lld of %lld in use", (long long)bytes,
              (long long)S->used, (long long)S->budget);
    return TTNN_EBUSY;
  }
  S->used += bytes;
  const int id = S->next_stream++;
  Slot& sl = S->slots[id];
  sl.plan = plan;
  sl.state = state;
  sl.bytes = bytes;
  *stream_id = id;
  return TTNN_OK;
}

ttnn_status ttnn_server_close(ttnn_server_t S, int32_t stream_id, int64_t timeout_us) {
  TTNN_CHECK_ARG(S, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->slots.find(stream_id);
  TTNN_CHECK_ARG(it != S->slots.end(), "no open stream %d", stream_id);
  if (!S->cv_done.wait_for(lk, std::chrono::microseconds(std::max<int64_t>(timeout_us, 0)),
                           [&] { return S->slots.at(stream_id).pending == 0; })) {
    set_error("stream %d still has pending requests", stream_id);
    return TTNN_ETIMEOUT;
  }
  Slot sl = it->second;
  S->slots.erase(it);
  S->used -= sl.bytes;
  lk.unlock();
  ttnn_state_destroy(sl.state);
  ttnn_plan_destroy(sl.plan);
  return TTNN_OK;
}

static ttnn_status enqueue(ttnn_server_s* S, Request&& r, uint64_t* ticket) {
  Worker& W = S->workers[r.stream % (int)S->workers.size()];
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->slots.find(r.stream);
    TTNN_CHECK_ARG(it != S->slots.end(), "no open stream %d", r.stream);
    // back-pressure: requests outstanding (queued or on the device) are
    // bounded, so a request's wait is bounded by the work ahead of it
    if (S->inflight.size() >= S->capacity) {
      set_error("request queue full (%zu outstanding)", S->capacity);
      return TTNN_EBUSY;
    }
    if (S->stream_capacity > 0 && it->second.pending >= S->stream_capacity) {
      set_error("stream %d has %d requests outstanding", r.stream, it->second.pending);
      return TTNN_EBUSY;
    }
    r.ticket = S->next_ticket++;
    r.t0 = Clock::now();
    ++it->second.pending;
    S->inflight.insert(r.ticket);
    *ticket = r.ticket;
    W.queue.push_back(std::move(r));
    ++S->queued;
  }
  W.cv_work.notify_one();
  return TTNN_OK;
}

ttnn_status ttnn_server_submit(ttnn_server_t S, int32_t stream_id, const void* data,
                               const int64_t* offset, const int64_t* extent,
                               const float* tile_scale, double lambda, uint64_t* ticket) {
  TTNN_CHECK_ARG(S && data && ticket, "null argument");
  ttnn_plan_s* P = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->slots.find(stream_id);
    TTNN_CHECK_ARG(it != S->slots.end(), "no open stream %d", stream_id);
    P = it->second.plan;
  }
  Request r{};
  r.kind = 0;
  r.stream = stream_id;
  r.data = data;
  r.scale = tile_scale;
  r.lambda = lambda;
  r.box.off.assign(P->d, 0);
  r.box.ext = P->dims;
  r.box.full = true;
  int64_t n = 1;
  for (int m = 0; m < P->d; ++m) {
    if (offset) r.box.off[m] = offset[m];
    if (extent) r.box.ext[m] = extent[m];
    TTNN_CHECK_ARG(r.box.ext[m] >= 1 && r.box.off[m] >= 0 && r.box.off[m] + r.box.ext[m] <= P->dims[m],
                   "box outside the tensor on mode %d", m);
    if (r.box.off[m] != 0 || r.box.ext[m] != P->dims[m]) r.box.full = false;
    n *= r.box.ext[m];
  }
  TTNN_CHECK_ARG(P->pass_store != 3 || tile_scale, "E4M3 updates need tile scales");
  TTNN_CHECK_ARG(!(P->flags & TTNN_FLAG_STRUCTURED_ONLY), "stream plan takes no dense updates");
  r.bytes = n * store_bytes_of(*P);
  return enqueue(S, std::move(r), ticket);
}

ttnn_status ttnn_server_recover(ttnn_server_t S, int32_t stream_id, double* cores,
                                uint64_t* ticket) {
  TTNN_CHECK_ARG(S && cores && ticket, "null argument");
  Request r{};
  r.kind = 1;
  r.stream = stream_id;
  r.cores = cores;
  return enqueue(S, std::move(r), ticket);
}

ttnn_status ttnn_server_wait(ttnn_server_t S, uint64_t ticket, int64_t timeout_us,
                             ttnn_status* result) {
  TTNN_CHECK_ARG(S && result, "null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  TTNN_CHECK_ARG(S->done.count(ticket) || S->inflight.count(ticket), "unknown ticket %llu",
                 (unsigned long long)ticket);
  if (!S->cv_done.wait_for(lk, std::chrono::microseconds(std::max<int64_t>(timeout_us, 0)),
                           [&] { return S->done.count(ticket) > 0; })) {
    set_error("ticket %llu not finished", (unsigned long long)ticket);
    return TTNN_ETIMEOUT;
  }
  const Done d = S->done.at(ticket);
  S->done.erase(ticket);
  *result = d.status;
  if (d.status != TTNN_OK) set_error("%s", d.msg.c_str());
  return TTNN_OK;
}

ttnn_status ttnn_server_stream_state(ttnn_server_t S, int32_t stream_id, ttnn_state_t* state) {
  TTNN_CHECK_ARG(S && state, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->slots.find(stream_id);
  TTNN_CHECK_ARG(it != S->slots.end(), "no open stream %d", stream_id);
  *state = it->second.state;
  return TTNN_OK;
}

ttnn_status ttnn_server_stats(ttnn_server_t S, int32_t reset, ttnn_server_report* out) {
  TTNN_CHECK_ARG(S && out, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  std::vector<double> v = S->lat_us;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(q * (double)v.size()))];
  };
  out->completed_updates = S->n_updates;
  out->completed_recoveries = S->n_recovers;
  out->failed = S->n_failed;
  out->batches = S->n_batches;
  out->update_bytes = S->bytes;
  out->p50_us = pct(0.50);
  out->p99_us = pct(0.99);
  out->max_us = v.empty() ? 0.0 : v.back();
  out->seconds = std::chrono::duration<double>(Clock::now() - S->since).count();
  out->device_bytes = S->used;
  out->open_streams = (int32_t)S->slots.size();
  out->queued = (int64_t)S->queued;
  out->worker_host_s = S->host_s;
  if (reset) {
    S->host_s = 0;
    S->lat_us.clear();
    S->n_updates = S->n_recovers = S->n_batches = S->n_failed = S->bytes = 0;
    S->since = Clock::now();
  }
  return TTNN_OK;
}

}  // extern "C"
