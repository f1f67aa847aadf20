// Serving: a request loop that admits DPSR solves by device-memory budget and
// runs them concurrently (continuous batching). An admitted request takes a
// slot (its own CUDA stream); its host-to-device copies, kernels and
// device-to-host copies are queued on the slot's stream, so requests that
// arrive while others are running start as soon as a slot and enough budget
// are free, and their work overlaps on the GPU. Requests of grid size up to
// kCoalesceMaxR that wait in the queue with the same grid size and mode
// (forward only, or forward + backward) are admitted together, up to
// max_group of them, and run as one batched launch per kernel (a pooled
// dpsr_batch of that grid size) on one slot; larger grids, which fill the GPU
// on their own, run as solo solves on pooled plans.
// A worker thread owns every CUDA call of the server; callers only enqueue
// requests and wait for tickets.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dpsr.h"
#include "nvtx.h"

extern "C" int dpsr_internal_io(dpsr_plan p, int64_t N, float** pts, float** nrm, float** chi,
                                float** dchi, float** dpts, float** dnrm);
extern "C" dpsr_plan dpsr_internal_batch_plan(dpsr_batch b, int i);
extern "C" int dpsr_internal_batch_run(dpsr_batch b, int k, int with_bwd);

namespace {

constexpr int kCoalesceMaxR = 128;  // grid sizes whose solves are coalesced
constexpr int kMaxGroup = 8;        // instances of a pooled batch
constexpr int64_t kPoolN = 200000;  // point capacity of pooled plans and batches

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

struct PooledBatch {
  dpsr_batch batch = nullptr;
  int r = 0;
  bool busy = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int64_t ticket = -1;         // -1: free; else the (first) request running here
  std::vector<int64_t> group;  // a coalesced group: its tickets, instance order
  int pooled = -1;             // index into the plan pool (solo request)
  int pbatch = -1;             // index into the batch pool (coalesced group)
  bool claimed = false;        // admitted, its work being queued
};

}  // namespace

struct dpsr_server_s {
  size_t budget = 0;
  float sigma = 2.f;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::deque<int64_t> done_q;  // completed tickets in completion order (dpsr_server_wait_any)
  std::map<int64_t, Request> reqs;
  std::vector<Slot> slots;
  std::vector<PooledPlan> pool;
  std::vector<PooledBatch> bpool;
  int max_group = kMaxGroup;
  size_t used = 0;  // bytes held by admitted requests
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  int64_t completed = 0, admitted = 0, max_active = 0;
  int64_t groups = 0, grouped = 0;  // coalesced launches and the requests they ran
};

namespace {

// A request's result is final (caller holds s->mu).
void finish(dpsr_server s, Request& rq, int status) {
  rq.status = status;
  rq.done = true;
  s->done_q.push_back(rq.ticket);
  // tickets retired by poll or wait stay in the queue until wait_any passes
  // them: drop them once they outnumber the live requests (amortised O(1))
  if (s->done_q.size() > 4096 && s->done_q.size() > 2 * s->reqs.size()) {
    std::deque<int64_t> keep;
    for (int64_t t : s->done_q)
      if (s->reqs.find(t) != s->reqs.end()) keep.push_back(t);
    s->done_q.swap(keep);
  }
}

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

// Find or create an idle pooled batch of grid size r (kMaxGroup instances of
// kPoolN points). A new batch is warmed once on `st`: every instance bound to
// a small valid cloud (256 points on a sphere, zero dchi) in its plan's
// staging, one forward and backward of all instances (which tunes the
// batch's plane paths on them), and a sync that clears their status words.
// Worker thread only.
int get_batch(dpsr_server s, int r, cudaStream_t st) {
  for (size_t i = 0; i < s->bpool.size(); ++i)
    if (!s->bpool[i].busy && s->bpool[i].r == r) return (int)i;
  int rs[kMaxGroup];
  float sig[kMaxGroup];
  int64_t nm[kMaxGroup];
  for (int i = 0; i < kMaxGroup; ++i) {
    rs[i] = r;
    sig[i] = s->sigma;
    nm[i] = kPoolN;
  }
  PooledBatch pb;
  pb.r = r;
  if (dpsr_batch_create(kMaxGroup, rs, sig, nm, &pb.batch) != DPSR_OK) return -1;
  constexpr int n0 = 256;
  std::vector<float> hp(3 * n0), hn(3 * n0);
  for (int j = 0; j < n0; ++j) {  // a spiral of directions over the sphere
    const double z = 1.0 - (2.0 * j + 1.0) / n0, rho = sqrt(1.0 - z * z), phi = 2.399963229728653 * j;
    const double d[3] = {rho * cos(phi), rho * sin(phi), z};
    for (int a = 0; a < 3; ++a) {
      hp[3 * j + a] = (float)(0.5 + 0.3 * d[a]);
      hn[3 * j + a] = (float)d[a];
    }
  }
  int rc = dpsr_batch_set_stream(pb.batch, st);
  for (int i = 0; i < kMaxGroup && rc == DPSR_OK; ++i) {
    float *pts, *nrm, *chi, *dchi, *dpts, *dnrm;
    dpsr_plan p = dpsr_internal_batch_plan(pb.batch, i);
    rc = dpsr_internal_io(p, kPoolN, &pts, &nrm, &chi, &dchi, &dpts, &dnrm);
    if (rc != DPSR_OK) break;
    rc = dpsr_internal_io(p, n0, &pts, &nrm, &chi, &dchi, &dpts, &dnrm);
    if (rc != DPSR_OK) break;
    if (cudaMemcpyAsync(pts, hp.data(), sizeof(float) * 3 * n0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(nrm, hn.data(), sizeof(float) * 3 * n0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(dchi, 0, sizeof(float) * r * r * r, st) != cudaSuccess) {
      rc = DPSR_ECUDA;
      break;
    }
    rc = dpsr_batch_bind(pb.batch, i, pts, nrm, n0, chi, dchi, dpts, dnrm);
  }
  if (rc == DPSR_OK) rc = dpsr_internal_batch_run(pb.batch, kMaxGroup, 1);
  if (rc == DPSR_OK) rc = dpsr_batch_sync(pb.batch);
  if (rc != DPSR_OK) {
    cudaGetLastError();
    dpsr_batch_destroy(pb.batch);
    return -1;
  }
  s->bpool.push_back(pb);
  return (int)s->bpool.size() - 1;
}

// Queue a coalesced group (same r and mode, 2..kMaxGroup requests) on a
// slot's stream as one batched launch of its first g.size() instances.
int launch_group(dpsr_server s, Slot& sl, std::vector<Request*>& g) {
  dpsr::NvtxRange nvtx_call("dpsr_server.group");
  const int r = g[0]->r;
  const bool bwd = g[0]->dchi != nullptr;
  const int bi = get_batch(s, r, sl.stream);
  if (bi < 0) return DPSR_ENOMEM;
  dpsr_batch b = s->bpool[bi].batch;
  if (dpsr_batch_set_stream(b, sl.stream) != DPSR_OK) return DPSR_ECUDA;
  const size_t gb = sizeof(float) * r * r * r;
  std::vector<float*> out(3 * g.size());
  for (size_t i = 0; i < g.size(); ++i) {
    Request& q = *g[i];
    float *pts, *nrm, *chi, *dchi, *dpts, *dnrm;
    int rc = dpsr_internal_io(dpsr_internal_batch_plan(b, (int)i), q.N, &pts, &nrm, &chi, &dchi, &dpts, &dnrm);
    if (rc != DPSR_OK) return rc;
    const size_t nb = sizeof(float) * 3 * q.N;
    if (cudaMemcpyAsync(pts, q.points, nb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
        cudaMemcpyAsync(nrm, q.normals, nb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
        (bwd && cudaMemcpyAsync(dchi, q.dchi, gb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess))
      return DPSR_ECUDA;
    rc = dpsr_batch_bind(b, (int)i, pts, nrm, q.N, chi, bwd ? dchi : nullptr, dpts, dnrm);
    if (rc != DPSR_OK) return rc;
    out[3 * i] = chi;
    out[3 * i + 1] = dpts;
    out[3 * i + 2] = dnrm;
  }
  int rc = dpsr_internal_batch_run(b, (int)g.size(), bwd ? 1 : 0);
  if (rc != DPSR_OK) return rc;
  for (size_t i = 0; i < g.size(); ++i) {
    Request& q = *g[i];
    const size_t nb = sizeof(float) * 3 * q.N;
    if (cudaMemcpyAsync(q.chi, out[3 * i], gb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        (bwd && (cudaMemcpyAsync(q.dpoints, out[3 * i + 1], nb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
                 cudaMemcpyAsync(q.dnormals, out[3 * i + 2], nb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)))
      return DPSR_ECUDA;
  }
  if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return DPSR_ECUDA;
  s->bpool[bi].busy = true;
  sl.pbatch = bi;
  sl.ticket = g[0]->ticket;
  sl.group.clear();
  for (Request* q : g) sl.group.push_back(q->ticket);
  return DPSR_OK;
}

// Queue one request on a slot's stream.
int launch(dpsr_server s, Slot& sl, Request& q) {
  dpsr::NvtxRange nvtx_call("dpsr_server.request");
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
      if (q != cudaSuccess) cudaGetLastError();
      if (sl.pbatch >= 0) {  // a coalesced group: instance i is request group[i]
        PooledBatch& pb = s->bpool[sl.pbatch];
        for (size_t i = 0; i < sl.group.size(); ++i) {
          Request& rq = s->reqs[sl.group[i]];
          finish(s, rq, q == cudaSuccess ? dpsr_sync(dpsr_internal_batch_plan(pb.batch, (int)i)) : DPSR_ECUDA);
          s->used -= rq.bytes;
          ++s->completed;
        }
        pb.busy = false;
        dpsr_batch_set_stream(pb.batch, nullptr);
        sl.group.clear();
        sl.pbatch = -1;
      } else {
        Request& rq = s->reqs[sl.ticket];
        PooledPlan& pp = s->pool[sl.pooled];
        finish(s, rq, q == cudaSuccess ? dpsr_sync(pp.plan) : DPSR_ECUDA);
        pp.busy = false;
        dpsr_plan_set_stream(pp.plan, nullptr);
        s->used -= rq.bytes;
        ++s->completed;
      }
      sl.ticket = -1;
      sl.pooled = -1;
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // admissions (FIFO): a request enters when a slot is free and its bytes
    // fit the budget next to the running ones; one too large for the whole
    // budget is rejected. The CUDA work of the admitted requests is queued
    // with the lock released (submit, poll and wait only need the lock for
    // the queue and the request table; slots and plans belong to this thread).
    // Each admission takes the head of the queue and, for a coalescible grid
    // size, the queued requests behind it with the same grid size and mode
    // that fit the budget (up to max_group, in queue order).
    std::vector<std::pair<Slot*, std::vector<Request*>>> admit;
    while (!s->queue.empty()) {
      Request& q = s->reqs[s->queue.front()];
      if (q.bytes > s->budget) {
        finish(s, q, DPSR_EBUSY);
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
      std::vector<Request*> grp{&q};  // the table never moves its entries
      size_t bytes = q.bytes;
      if (q.r <= kCoalesceMaxR && s->max_group > 1) {
        for (auto it = s->queue.begin(); it != s->queue.end() && (int)grp.size() < s->max_group;) {
          Request& o = s->reqs[*it];
          if (o.r == q.r && (o.dchi != nullptr) == (q.dchi != nullptr) && o.bytes <= s->budget &&
              s->used + bytes + o.bytes <= s->budget) {
            grp.push_back(&o);
            bytes += o.bytes;
            it = s->queue.erase(it);
          } else {
            ++it;
          }
        }
      }
      free_slot->claimed = true;
      s->used += bytes;
      admit.emplace_back(free_slot, std::move(grp));
    }
    if (!admit.empty()) {
      lk.unlock();
      std::vector<int> rcs;
      for (auto& a : admit)
        rcs.push_back(a.second.size() > 1 ? launch_group(s, *a.first, a.second)
                                          : launch(s, *a.first, *a.second[0]));
      lk.lock();
      for (size_t i = 0; i < admit.size(); ++i) {
        Slot& sl = *admit[i].first;
        sl.claimed = false;
        if (rcs[i] != DPSR_OK) {
          for (Request* q : admit[i].second) {
            finish(s, *q, rcs[i]);
            s->used -= q->bytes;
          }
          s->cv_done.notify_all();
          continue;
        }
        s->admitted += (int64_t)admit[i].second.size();
        if (admit[i].second.size() > 1) {
          ++s->groups;
          s->grouped += (int64_t)admit[i].second.size();
        }
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
  // Plans and batches first: a pooled plan still refers to the stream of the
  // last slot that ran it, and destroying a plan synchronises that stream.
  for (PooledPlan& p : s->pool) {
    dpsr_plan_set_stream(p.plan, nullptr);
    dpsr_plan_destroy(p.plan);
  }
  for (PooledBatch& b : s->bpool) {
    dpsr_batch_set_stream(b.batch, nullptr);
    dpsr_batch_destroy(b.batch);
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
  // find, never operator[]: another thread may retire the ticket meanwhile
  // (poll), and operator[] would insert a fresh request that never completes
  auto done = [&] {
    auto f = s->reqs.find(ticket);
    return f == s->reqs.end() || f->second.done;
  };
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9), done);
  if (!ok) return DPSR_ETIMEOUT;
  auto f = s->reqs.find(ticket);
  if (f == s->reqs.end()) return DPSR_EINVAL;  // retired by another caller
  const int st = f->second.status;
  s->reqs.erase(f);
  return st;
}

int dpsr_server_wait_any(dpsr_server s, int64_t* tickets, int* statuses, int max, double timeout_s,
                         int* count) {
  if (!s || !tickets || !statuses || !count || max < 1) return DPSR_EINVAL;
  *count = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  // tickets retired meanwhile by poll or wait are skipped
  auto ready = [&] {
    while (!s->done_q.empty() && s->reqs.find(s->done_q.front()) == s->reqs.end()) s->done_q.pop_front();
    return !s->done_q.empty();
  };
  if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9), ready))
    return DPSR_ETIMEOUT;
  int n = 0;
  while (n < max && !s->done_q.empty()) {
    const int64_t t = s->done_q.front();
    s->done_q.pop_front();
    auto it = s->reqs.find(t);
    if (it == s->reqs.end()) continue;
    tickets[n] = t;
    statuses[n] = it->second.status;
    s->reqs.erase(it);
    ++n;
  }
  *count = n;
  return DPSR_OK;
}

int dpsr_server_cancel(dpsr_server s, int64_t ticket) {
  if (!s) return DPSR_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return DPSR_EINVAL;
    // admission takes requests out of the queue under this lock: a ticket
    // still queued here has no work on the GPU and none will be queued
    auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
    if (it->second.done || q == s->queue.end()) return DPSR_EBUSY;
    s->queue.erase(q);
    finish(s, it->second, DPSR_ECANCELED);
  }
  s->cv_done.notify_all();
  return DPSR_OK;
}

int dpsr_server_set_max_group(dpsr_server s, int max_group) {
  if (!s || max_group < 1 || max_group > kMaxGroup) return DPSR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_group = max_group;
  return DPSR_OK;
}

int dpsr_server_group_stats(dpsr_server s, int64_t* out2) {
  if (!s || !out2) return DPSR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out2[0] = s->groups;
  out2[1] = s->grouped;
  return DPSR_OK;
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
