// Continuous-batching query server over a resident index (no counterpart in
// the paper; it serves Alg. 7 queries arriving one at a time).
//
// Requests are admitted into a fixed pool of slots (admission fails with
// DETLSH_EADMIT when the pool is full: its size bounds the host memory and,
// through the per-batch capacity, the device memory in use). A worker thread
// forms batches from the arrival queue and runs each through one of several
// pipelines; a pipeline owns a query plan (preallocated device buffers, one
// CUDA graph launch per batch), a stream, pinned staging buffers and an event.
// While one pipeline's batch runs, the next batch is formed and launched on
// another, so host work, copies and kernels of consecutive batches overlap.
// A batch starts when it is full, when no batch is running, or when its
// oldest request has waited max_delay_us. Completion is detected by polling
// the pipeline's event, never by a blocking wait.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { R_FREE = 0, R_QUEUED, R_RUNNING, R_DONE };

struct Req {
  uint32_t gen = 0;
  int state = R_FREE;
  int status = DETLSH_OK;
  int32_t k = 0;
  float c = 0.f, r = 0.f;
  int32_t stats[4] = {0, 0, 0, 0};
  Clock::time_point t_sub, t_done;
};

struct Pipe {
  detlsh_plan* plan = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  void* Qh = nullptr;
  int32_t* kh = nullptr;
  float* ch = nullptr;
  float* rh = nullptr;
  int64_t* idsh = nullptr;
  float* disth = nullptr;
  int32_t* statsh = nullptr;
  std::vector<uint32_t> batch;
  bool busy = false;
  int fail = DETLSH_OK;
};

}  // namespace

struct detlsh_server {
  const detlsh_index* idx = nullptr;
  detlsh_server_config cfg{};
  int dev = 0;
  size_t qrow = 0;
  int64_t slots = 0, cap = 0;
  std::vector<Req> reqs;
  std::vector<unsigned char> qpool;   // [cap][qrow]
  std::vector<int64_t> idpool;        // [cap][k_max]
  std::vector<float> dpool;           // [cap][k_max]
  std::vector<uint32_t> free_slots;
  std::deque<uint32_t> queue;
  std::vector<Pipe> pipes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int64_t n_submitted = 0, n_completed = 0, n_rejected = 0, n_batches = 0, n_batched = 0, max_batch = 0,
          n_errors = 0;
};

namespace detlsh {
namespace {

void free_pipe(Pipe& P) {
  if (P.plan) detlsh_plan_destroy(P.plan);
  if (P.ev) cudaEventDestroy(P.ev);
  if (P.s) cudaStreamDestroy(P.s);
  void* hs[] = {P.Qh, P.kh, P.ch, P.rh, P.idsh, P.disth, P.statsh};
  for (void* h : hs)
    if (h) cudaFreeHost(h);
  P = Pipe{};
}

int make_pipe(detlsh_server* S, const detlsh_query_params& qp, Pipe* P) {
  DL_CUDA(cudaStreamCreateWithFlags(&P->s, cudaStreamNonBlocking));
  DL_CUDA(cudaEventCreateWithFlags(&P->ev, cudaEventDisableTiming));
  DL_TRY(detlsh_plan_create(S->idx, S->slots, S->cfg.k_max, &qp, DETLSH_PLAN_GRAPH, P->s, &P->plan));
  const int64_t B = S->slots, km = S->cfg.k_max;
  DL_CUDA(cudaHostAlloc(&P->Qh, S->qrow * B, cudaHostAllocDefault));
  DL_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->kh), sizeof(int32_t) * B, cudaHostAllocDefault));
  DL_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->ch), sizeof(float) * B, cudaHostAllocDefault));
  DL_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->rh), sizeof(float) * B, cudaHostAllocDefault));
  DL_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->idsh), sizeof(int64_t) * B * km, cudaHostAllocDefault));
  DL_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->disth), sizeof(float) * B * km, cudaHostAllocDefault));
  DL_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->statsh), sizeof(int32_t) * B * 4, cudaHostAllocDefault));
  return DETLSH_OK;
}

// the finished batch of P: results and status into its requests (lock held)
void complete(detlsh_server* S, Pipe& P, int st) {
  const int km = S->cfg.k_max;
  const auto now = Clock::now();
  for (size_t i = 0; i < P.batch.size(); ++i) {
    const uint32_t slot = P.batch[i];
    Req& R = S->reqs[slot];
    if (st == DETLSH_OK) {
      std::memcpy(&S->idpool[(size_t)slot * km], P.idsh + i * km, sizeof(int64_t) * km);
      std::memcpy(&S->dpool[(size_t)slot * km], P.disth + i * km, sizeof(float) * km);
      std::memcpy(R.stats, P.statsh + i * 4, sizeof(R.stats));
    } else {
      ++S->n_errors;
    }
    R.status = st;
    R.state = R_DONE;
    R.t_done = now;
    ++S->n_completed;
  }
  P.batch.clear();
  P.busy = false;
  P.fail = DETLSH_OK;
}

void worker_loop(detlsh_server* S) {
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  const auto max_delay = std::chrono::microseconds(S->cfg.max_delay_us);
  while (true) {
    bool progressed = false, any_busy = false;
    for (Pipe& P : S->pipes) {
      if (!P.busy) continue;
      const cudaError_t e = cudaEventQuery(P.ev);
      if (e == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      int st = P.fail;
      if (st == DETLSH_OK && e != cudaSuccess) {
        set_error("batch failed: %s", cudaGetErrorString(e));
        st = DETLSH_ECUDA;
      }
      if (st == DETLSH_OK) st = detlsh_plan_status(P.plan, P.s);   // the stream is idle here
      complete(S, P, st);
      progressed = true;
      S->cv_done.notify_all();
    }
    Pipe* freep = nullptr;
    for (Pipe& P : S->pipes)
      if (!P.busy) {
        freep = &P;
        break;
      }
    if (S->stop && S->queue.empty() && !any_busy && freep && !progressed) {
      bool idle = true;
      for (Pipe& P : S->pipes) idle = idle && !P.busy;
      if (idle) break;
    }
    if (freep && !S->queue.empty()) {
      const auto now = Clock::now();
      const bool full = (int64_t)S->queue.size() >= S->slots;
      const bool waited = now - S->reqs[S->queue.front()].t_sub >= max_delay;
      if (full || !any_busy || waited || S->stop) {
        Pipe& P = *freep;
        const int64_t m = std::min<int64_t>(S->slots, (int64_t)S->queue.size());
        P.batch.assign(S->queue.begin(), S->queue.begin() + m);
        S->queue.erase(S->queue.begin(), S->queue.begin() + m);
        for (uint32_t slot : P.batch) S->reqs[slot].state = R_RUNNING;
        P.busy = true;
        ++S->n_batches;
        S->n_batched += m;
        S->max_batch = std::max<int64_t>(S->max_batch, m);
        const bool inject = S->cfg.test_fail_batch > 0 && S->n_batches == S->cfg.test_fail_batch;
        // running requests are not touched by submitters: stage them unlocked
        lk.unlock();
        for (int64_t i = 0; i < m; ++i) {
          const Req& R = S->reqs[P.batch[i]];
          std::memcpy(static_cast<char*>(P.Qh) + i * S->qrow, &S->qpool[(size_t)P.batch[i] * S->qrow], S->qrow);
          P.kh[i] = R.k;
          P.ch[i] = R.c;
          P.rh[i] = R.r;
        }
        int st = DETLSH_OK;
        if (inject) {
          set_error("batch %lld failed by request (test_fail_batch)", (long long)S->cfg.test_fail_batch);
          st = DETLSH_ECUDA;
        } else {
          st = plan_enqueue(P.plan, P.Qh, m, P.kh, P.ch, P.rh, P.idsh, P.disth, P.statsh, cudaMemcpyDefault,
                            cudaMemcpyDefault, P.s);
        }
        if (cudaEventRecord(P.ev, P.s) != cudaSuccess && st == DETLSH_OK) st = DETLSH_ECUDA;
        lk.lock();
        P.fail = st;
        progressed = true;
      }
    }
    if (!progressed) {
      // wake on a submit, else poll the running batches every 20 us
      const auto wait = any_busy ? std::chrono::microseconds(20)
                                 : (S->queue.empty() ? std::chrono::microseconds(2000) : max_delay / 4 + std::chrono::microseconds(1));
      S->cv_work.wait_for(lk, wait);
    }
  }
}

int poll_impl(detlsh_server* S, uint64_t ticket, int32_t wait_us, int64_t* ids, float* dist, int32_t* stats,
              double* latency_us, Clock::time_point* t_done) {
  const uint32_t slot = (uint32_t)(ticket & 0xffffffffu), gen = (uint32_t)(ticket >> 32);
  std::unique_lock<std::mutex> lk(S->mu);
  if ((int64_t)slot >= S->cap || S->reqs[slot].gen != gen || S->reqs[slot].state == R_FREE) {
    set_error("unknown or already collected ticket");
    return DETLSH_EINVAL;
  }
  Req& R = S->reqs[slot];
  if (R.state != R_DONE && wait_us > 0)
    S->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return R.state == R_DONE; });
  if (R.state != R_DONE) return DETLSH_PENDING;
  const int km = S->cfg.k_max;
  if (R.status == DETLSH_OK) {
    if (ids) std::memcpy(ids, &S->idpool[(size_t)slot * km], sizeof(int64_t) * km);
    if (dist) std::memcpy(dist, &S->dpool[(size_t)slot * km], sizeof(float) * km);
    if (stats) std::memcpy(stats, R.stats, sizeof(R.stats));
  }
  if (latency_us) latency_us[0] = std::chrono::duration<double, std::micro>(R.t_done - R.t_sub).count();
  if (t_done) *t_done = R.t_done;
  const int st = R.status;
  R.state = R_FREE;
  S->free_slots.push_back(slot);
  return st;
}

}  // namespace
}  // namespace detlsh

using namespace detlsh;

extern "C" {

int detlsh_server_create(const detlsh_index* idx, const detlsh_server_config* cfg, detlsh_server** out) {
  DL_REQUIRE(idx && cfg && out, "NULL argument");
  *out = nullptr;
  detlsh_server_config c = *cfg;
  DL_REQUIRE(c.k_max >= 1 && c.k_max <= kMaxTopK, "k_max must be in [1, %d]", kMaxTopK);
  if (c.pipelines == 0) c.pipelines = 2;
  DL_REQUIRE(c.pipelines >= 1 && c.pipelines <= 4, "pipelines must be in [1, 4]");
  DL_REQUIRE(c.slots >= 0 && c.queue_cap >= 0 && c.max_delay_us >= 0 && c.mem_budget >= 0,
             "slots, queue_cap, max_delay_us and mem_budget must be >= 0");
  if (c.max_delay_us == 0) c.max_delay_us = 200;
  if (c.mem_budget == 0) c.mem_budget = (int64_t)8 << 30;
  detlsh_query_params qp{};
  qp.eps = c.eps;
  qp.beta = c.beta;
  qp.shortlist = c.shortlist;
  qp.tuning = c.tuning;
  QueryTuning tu;
  DL_TRY(tuning_from_params(&qp, &tu));
  double beta = c.beta;
  // batch capacity: the requested one, else the largest power of two (at
  // most 4096) whose buffers for all pipelines fit the memory budget
  int64_t B = c.slots;
  if (B == 0) {
    for (B = 4096; B > 1; B /= 2) {
      tu.batch = B;
      QueryShape sh;
      DL_TRY(query_shape(idx, B, c.k_max, beta, c.shortlist, tu, &sh));
      if ((int64_t)sh.bytes * c.pipelines <= c.mem_budget) break;
    }
  }
  {
    tu.batch = B;
    QueryShape sh;
    DL_TRY(query_shape(idx, B, c.k_max, beta, c.shortlist, tu, &sh));
    if ((int64_t)sh.bytes * c.pipelines > c.mem_budget) {
      set_error("batches of %lld queries need %zu bytes per pipeline, over the memory budget", (long long)B,
                sh.bytes);
      return DETLSH_EADMIT;
    }
  }
  if (c.queue_cap == 0) c.queue_cap = (int32_t)std::min<int64_t>((int64_t)1 << 20, 4 * B * c.pipelines);
  DL_REQUIRE(c.queue_cap >= 1, "queue_cap must be >= 1");
  detlsh_server* S = new (std::nothrow) detlsh_server();
  if (!S) {
    set_error("host allocation failed");
    return DETLSH_ENOMEM;
  }
  S->idx = idx;
  S->cfg = c;
  S->slots = B;
  S->cap = c.queue_cap;
  S->qrow = (size_t)idx->d * (idx->dtype == DETLSH_U8 ? 1 : 4);
  int st = DETLSH_OK;
  try {
    S->reqs.resize(S->cap);
    S->qpool.resize((size_t)S->cap * S->qrow);
    S->idpool.resize((size_t)S->cap * c.k_max);
    S->dpool.resize((size_t)S->cap * c.k_max);
    S->free_slots.reserve(S->cap);
    for (int64_t i = S->cap - 1; i >= 0; --i) S->free_slots.push_back((uint32_t)i);
  } catch (...) {
    st = DETLSH_ENOMEM;
    set_error("host allocation failed");
  }
  if (st == DETLSH_OK && cudaGetDevice(&S->dev) != cudaSuccess) st = DETLSH_ECUDA;
  S->pipes.resize(c.pipelines);
  for (int i = 0; i < c.pipelines && st == DETLSH_OK; ++i) st = make_pipe(S, qp, &S->pipes[i]);
  if (st != DETLSH_OK) {
    for (Pipe& P : S->pipes) free_pipe(P);
    delete S;
    return st;
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return DETLSH_OK;
}

int detlsh_server_submit(detlsh_server* S, const void* q, int32_t k, float c, float r_min, uint64_t* ticket) {
  DL_REQUIRE(S && q && ticket, "NULL argument");
  DL_REQUIRE(k >= 1 && k <= S->cfg.k_max, "k must be in [1, k_max]");
  DL_REQUIRE(std::isfinite(c) && c > 1.0f, "c must be finite and > 1");
  DL_REQUIRE(std::isfinite(r_min), "r_min must be finite");
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->stop) {
    set_error("the server is shutting down");
    return DETLSH_EINVAL;
  }
  if (S->free_slots.empty()) {
    ++S->n_rejected;
    set_error("all %lld request slots are in use", (long long)S->cap);
    return DETLSH_EADMIT;
  }
  const uint32_t slot = S->free_slots.back();
  S->free_slots.pop_back();
  Req& R = S->reqs[slot];
  ++R.gen;
  R.state = R_QUEUED;
  R.status = DETLSH_OK;
  R.k = k;
  R.c = c;
  R.r = r_min;
  R.t_sub = Clock::now();
  std::memcpy(&S->qpool[(size_t)slot * S->qrow], q, S->qrow);
  S->queue.push_back(slot);
  ++S->n_submitted;
  *ticket = ((uint64_t)R.gen << 32) | slot;
  lk.unlock();
  S->cv_work.notify_one();
  return DETLSH_OK;
}

int detlsh_server_poll(detlsh_server* S, uint64_t ticket, int32_t wait_us, int64_t* ids, float* dist,
                       int32_t* stats, double* latency_us) {
  DL_REQUIRE(S != nullptr, "server is NULL");
  return poll_impl(S, ticket, wait_us, ids, dist, stats, latency_us, nullptr);
}

int detlsh_server_replay(detlsh_server* S, const void* Q, int64_t nq, const int32_t* k, const float* c,
                         const float* r_min, const double* arrival_us, int64_t* out_ids, float* out_dist,
                         int32_t* out_stats, double* latency_us) {
  DL_REQUIRE(S && (nq == 0 || (Q && k && c && r_min && arrival_us && latency_us)), "NULL argument");
  DL_REQUIRE(nq >= 0, "nq must be >= 0");
  for (int64_t i = 0; i < nq; ++i) {
    DL_REQUIRE(k[i] >= 1 && k[i] <= S->cfg.k_max, "k[%lld] must be in [1, k_max]", (long long)i);
    DL_REQUIRE(std::isfinite(c[i]) && c[i] > 1.0f, "c[%lld] must be finite and > 1", (long long)i);
    DL_REQUIRE(std::isfinite(r_min[i]), "r_min[%lld] must be finite", (long long)i);
    DL_REQUIRE(i == 0 || arrival_us[i] >= arrival_us[i - 1], "arrival times must not decrease");
  }
  if (nq == 0) return DETLSH_OK;
  std::vector<uint64_t> tickets(nq);
  std::atomic<int64_t> issued(0);
  std::atomic<int> first_err(DETLSH_OK);
  const auto t0 = Clock::now();
  const int km = S->cfg.k_max;
  // collector: results in submission order; latency from the scheduled arrival
  std::thread collector([&] {
    for (int64_t i = 0; i < nq; ++i) {
      while (issued.load(std::memory_order_acquire) <= i) std::this_thread::yield();
      Clock::time_point td;
      int st;
      while ((st = poll_impl(S, tickets[i], 1000, out_ids ? out_ids + i * km : nullptr,
                             out_dist ? out_dist + i * km : nullptr, out_stats ? out_stats + i * 4 : nullptr,
                             nullptr, &td)) == DETLSH_PENDING) {
      }
      if (st != DETLSH_OK) {
        int expect = DETLSH_OK;
        first_err.compare_exchange_strong(expect, st);
        latency_us[i] = -1.0;
      } else {
        const auto arrive = t0 + std::chrono::duration_cast<Clock::duration>(
                                     std::chrono::duration<double, std::micro>(arrival_us[i]));
        latency_us[i] = std::chrono::duration<double, std::micro>(td - arrive).count();
      }
    }
  });
  const size_t qrow = S->qrow;
  for (int64_t i = 0; i < nq; ++i) {
    const auto arrive = t0 + std::chrono::duration_cast<Clock::duration>(
                                 std::chrono::duration<double, std::micro>(arrival_us[i]));
    while (Clock::now() < arrive) {
      const auto left = arrive - Clock::now();
      if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
      else std::this_thread::yield();
    }
    int st;
    // open loop with back-pressure: a full pool delays the submission (the
    // wait counts in the latency, measured from the scheduled arrival)
    while ((st = detlsh_server_submit(S, static_cast<const char*>(Q) + i * qrow, k[i], c[i], r_min[i],
                                      &tickets[i])) == DETLSH_EADMIT)
      std::this_thread::sleep_for(std::chrono::microseconds(5));
    if (st != DETLSH_OK) {
      // cannot happen after the checks above; stop issuing
      first_err.store(st);
      for (int64_t j = i; j < nq; ++j) latency_us[j] = -1.0;
      issued.store(i, std::memory_order_release);
      collector.join();
      return st;
    }
    issued.store(i + 1, std::memory_order_release);
  }
  collector.join();
  return first_err.load();
}

int detlsh_server_stats(detlsh_server* S, int64_t* out8) {
  DL_REQUIRE(S && out8, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out8[0] = S->n_submitted;
  out8[1] = S->n_completed;
  out8[2] = S->n_rejected;
  out8[3] = S->n_batches;
  out8[4] = S->n_batched;
  out8[5] = S->max_batch;
  out8[6] = S->n_errors;
  out8[7] = S->slots;
  return DETLSH_OK;
}

void detlsh_server_destroy(detlsh_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Pipe& P : S->pipes) {
    if (P.s) cudaStreamSynchronize(P.s);
    free_pipe(P);
  }
  delete S;
}

}  // extern "C"
