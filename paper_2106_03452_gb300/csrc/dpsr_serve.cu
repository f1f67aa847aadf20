// Serving: a request loop that admits DPSR solves by device-memory budget and
// runs them concurrently (continuous batching). Each admitted request takes a
// slot (its own CUDA stream) and a pooled plan of its grid size; its host-to-
// device copies, kernels and device-to-host copies are queued on the slot's
// stream, so requests that arrive while others are running start as soon as
// a slot and enough budget are free, and their work overlaps on the GPU.
// A worker thread owns every CUDA call of the server; callers only enqueue
// requests and wait for tickets.
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dpsr.h"

extern "C" int dpsr_internal_io(dpsr_plan p, int64_t N, float** pts, float** nrm, float** chi,
                                float** dchi, float** dpts, float** dnrm);

namespace {

struct Request {
  int64_t ticket = 0;
  int r = 0;
  int64_t N = 0;
  const float* points = nullptr;
  const float* normals = nullptr;
  const float* dchi = nullptr;
  float* chi = nullptr;
  float* dpoints = nullptr;
  float* dnormals = nullptr;
  size_t bytes = 0;
  int status = DPSR_OK;
  bool done = false;
};

struct PooledPlan {
  dpsr_plan plan = nullptr;
  int r = 0;
  int64_t cap = 0;
  bool busy = false;
  size_t bytes = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int64_t ticket = -1;   // -1: free
  int pooled = -1;       // index into the plan pool
  bool claimed = false;  // admitted, its work being queued
};

}  // namespace

struct dpsr_server_s {
  size_t budget = 0;
  float sigma = 2.f;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::map<int64_t, Request> reqs;
  std::vector<Slot> slots;
  std::vector<PooledPlan> pool;
  size_t used = 0;  // bytes held by admitted requests
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  int64_t completed = 0, admitted = 0, max_active = 0;
};

namespace {

size_t request_bytes(int r, int64_t N, bool bwd) {
  const size_t grid = (size_t)r * r * r * sizeof(float);
  return dpsr_plan_workspace_bytes(r, N, bwd) + 2 * grid + 4 * (size_t)N * 3 * sizeof(float);
}

// Find or create an idle plan of grid size r holding N points. Called from
// the worker thread only (the pool belongs to it).
int get_plan(dpsr_server s, int r, int64_t N) {
  int best = -1;
  for (size_t i = 0; i < s->pool.size(); ++i) {
    const PooledPlan& p = s->pool[i];
    if (!p.busy && p.r == r && p.cap >= N && (best < 0 || p.cap < s->pool[best].cap)) best = (int)i;
  }
  if (best >= 0) return best;
  // Grow an idle plan of the right size, or make a new one.
  for (size_t i = 0; i < s->pool.size(); ++i) {
    PooledPlan& p = s->pool[i];
    if (!p.busy && p.r == r) {
      if (dpsr_plan_reserve(p.plan, N) != DPSR_OK) return -1;
      p.cap = N;
      return (int)i;
    }
  }
  PooledPlan p;
  p.r = r;
  if (dpsr_plan_create(r, s->sigma, &p.plan) != DPSR_OK) return -1;
  if (dpsr_plan_reserve(p.plan, N) != DPSR_OK) {
    dpsr_plan_destroy(p.plan);
    return -1;
  }
  p.cap = N;
  s->pool.push_back(p);
  return (int)s->pool.size() - 1;
}

// Queue one request on a slot's stream.
int launch(dpsr_server s, Slot& sl, Request& q) {
  const int pi = get_plan(s, q.r, q.N);
  if (pi < 0) return DPSR_ENOMEM;
  PooledPlan& pp = s->pool[pi];
  dpsr_plan p = pp.plan;
  dpsr_plan_set_stream(p, sl.stream);
  float *pts, *nrm, *chi, *dchi, *dpts, *dnrm;
  int rc = dpsr_internal_io(p, q.N, &pts, &nrm, &chi, &dchi, &dpts, &dnrm);
  if (rc != DPSR_OK) return rc;
  const size_t nb = sizeof(float) * 3 * q.N, gb = sizeof(float) * q.r * q.r * q.r;
  if (cudaMemcpyAsync(pts, q.points, nb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
      cudaMemcpyAsync(nrm, q.normals, nb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
    return DPSR_ECUDA;
  rc = dpsr_forward(p, pts, nrm, q.N, chi);
  if (rc != DPSR_OK) return rc;
  if (q.dchi) {
    if (cudaMemcpyAsync(dchi, q.dchi, gb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
      return DPSR_ECUDA;
    rc = dpsr_backward(p, dchi, dpts, dnrm);
    if (rc != DPSR_OK) return rc;
    if (cudaMemcpyAsync(q.dpoints, dpts, nb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaMemcpyAsync(q.dnormals, dnrm, nb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      return DPSR_ECUDA;
  }
  if (cudaMemcpyAsync(q.chi, chi, gb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
      cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
    return DPSR_ECUDA;
  pp.busy = true;
  sl.pooled = pi;
  sl.ticket = q.ticket;
  return DPSR_OK;
}

void worker_main(dpsr_server s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    int active = 0;
    // completions
    for (Slot& sl : s->slots) {
      if (sl.ticket < 0) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) {
        ++active;
        continue;
      }
      Request& rq = s->reqs[sl.ticket];
      PooledPlan& pp = s->pool[sl.pooled];
      rq.status = q == cudaSuccess ? dpsr_sync(pp.plan) : DPSR_ECUDA;
      if (q != cudaSuccess) cudaGetLastError();
      rq.done = true;
      pp.busy = false;
      dpsr_plan_set_stream(pp.plan, nullptr);
      s->used -= rq.bytes;
      sl.ticket = -1;
      sl.pooled = -1;
      ++s->completed;
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // admissions (FIFO): a request enters when a slot is free and its bytes
    // fit the budget next to the running ones; one too large for the whole
    // budget is rejected. The CUDA work of the admitted requests is queued
    // with the lock released (submit, poll and wait only need the lock for
    // the queue and the request table; slots and plans belong to this thread).
    std::vector<std::pair<Slot*, Request*>> admit;
    while (!s->queue.empty()) {
      Request& q = s->reqs[s->queue.front()];
      if (q.bytes > s->budget) {
        q.status = DPSR_EBUSY;
        q.done = true;
        s->queue.pop_front();
        s->cv_done.notify_all();
        continue;
      }
      if (s->used + q.bytes > s->budget) break;
      Slot* free_slot = nullptr;
      for (Slot& sl : s->slots)
        if (sl.ticket < 0 && !sl.claimed) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      s->queue.pop_front();
      free_slot->claimed = true;
      s->used += q.bytes;
      admit.emplace_back(free_slot, &q);  // the table never moves its entries
    }
    if (!admit.empty()) {
      lk.unlock();
      std::vector<int> rcs;
      for (auto& a : admit) rcs.push_back(launch(s, *a.first, *a.second));
      lk.lock();
      for (size_t i = 0; i < admit.size(); ++i) {
        Slot& sl = *admit[i].first;
        Request& q = *admit[i].second;
        sl.claimed = false;
        if (rcs[i] != DPSR_OK) {
          q.status = rcs[i];
          q.done = true;
          s->used -= q.bytes;
          s->cv_done.notify_all();
          continue;
        }
        ++s->admitted;
        ++active;
      }
      progress = true;
    }
    if (active > s->max_active) s->max_active = active;
    if (!progress) {
      // poll running work every 20 us; sleep until a submission otherwise
      if (active > 0)
        s->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    }
  }
}

}  // namespace

extern "C" {

int dpsr_server_create(size_t hbm_budget_bytes, int slots, float sigma, dpsr_server* out) {
  if (!out || hbm_budget_bytes == 0 || slots < 1 || slots > 64 || !(sigma >= 0.f)) return DPSR_EINVAL;
  *out = nullptr;
  dpsr_server s = new (std::nothrow) dpsr_server_s();
  if (!s) return DPSR_ENOMEM;
  s->budget = hbm_budget_bytes;
  s->sigma = sigma;
  cudaGetDevice(&s->device);
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      dpsr_server_destroy(s);
      return DPSR_ECUDA;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return DPSR_OK;
}

int dpsr_server_destroy(dpsr_server s) {
  if (!s) return DPSR_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Slot& sl : s->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  // Plans first: a pooled plan still refers to the stream of the last slot
  // that ran it, and destroying a plan synchronises that stream.
  for (PooledPlan& p : s->pool) {
    dpsr_plan_set_stream(p.plan, nullptr);
    dpsr_plan_destroy(p.plan);
  }
  for (Slot& sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
  return DPSR_OK;
}

int dpsr_server_submit(dpsr_server s, int r, const float* points, const float* normals, int64_t N,
                       const float* dchi, float* chi_out, float* dpoints, float* dnormals,
                       int64_t* ticket) {
  if (!s || !points || !normals || !chi_out || !ticket || N < 1) return DPSR_EINVAL;
  if (dchi && (!dpoints || !dnormals)) return DPSR_EINVAL;
  if (dpsr_plan_workspace_bytes(r, N, 1) == 0) return DPSR_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Request q;
    q.ticket = s->next_ticket++;
    q.r = r;
    q.N = N;
    q.points = points;
    q.normals = normals;
    q.dchi = dchi;
    q.chi = chi_out;
    q.dpoints = dpoints;
    q.dnormals = dnormals;
    q.bytes = request_bytes(r, N, dchi != nullptr);
    s->reqs[q.ticket] = q;
    s->queue.push_back(q.ticket);
    *ticket = q.ticket;
  }
  s->cv_work.notify_all();
  return DPSR_OK;
}

int dpsr_server_poll(dpsr_server s, int64_t ticket, int* done) {
  if (!s || !done) return DPSR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return DPSR_EINVAL;
  *done = it->second.done ? 1 : 0;
  if (!it->second.done) return DPSR_OK;
  const int st = it->second.status;
  s->reqs.erase(it);
  return st;
}

int dpsr_server_wait(dpsr_server s, int64_t ticket, double timeout_s) {
  if (!s) return DPSR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return DPSR_EINVAL;
  const bool ok = s->cv_done.wait_for(
      lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
      [&] { return s->reqs[ticket].done; });
  if (!ok) return DPSR_ETIMEOUT;
  const int st = s->reqs[ticket].status;
  s->reqs.erase(ticket);
  return st;
}

int dpsr_server_stats(dpsr_server s, int64_t* out4) {
  if (!s || !out4) return DPSR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out4[0] = s->admitted;
  out4[1] = s->completed;
  out4[2] = s->max_active;
  out4[3] = (int64_t)s->used;
  return DPSR_OK;
}

}  // extern "C"
