// Batched solves: many point clouds of uneven N and mixed r, each kernel of
// the forward / backward sequence launched once per grid size for all
// instances of that size (the instance is blockIdx.z of every kernel, its
// descriptor read from a device table), the whole sequence capturable into
// one CUDA graph and replayed with a single launch.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dpsr.h"
#include "dpsr_dev.cuh"
#include "launch.h"
#include "nvtx.h"

using dpsr::Solve;

// Internal hooks of dpsr_api.cu (same library).
extern "C" const void* dpsr_internal_solve(dpsr_plan p);
extern "C" int dpsr_internal_cluster(dpsr_plan p, int kind);
extern "C" int dpsr_internal_forced(int kind, int r);
extern "C" int dpsr_internal_tc_lookup(int kind, int r, int batch);
extern "C" void dpsr_internal_tc_store(int kind, int r, int batch, int path, float ms);

struct BatchClass {
  int r = 0;
  std::vector<int> members;  // instance indices
  Solve* dtab = nullptr;     // device table, one descriptor per member
  int nmax = 0;
  int C[4] = {1, 1, 1, 1};
  bool tuned[4] = {false, false, false, false};
  // Classes run side by side: each on its own stream, forked from and
  // joined back into the batch stream (also inside a captured graph).
  cudaStream_t st = nullptr;
  cudaEvent_t join = nullptr;
};

struct dpsr_batch_s {
  int count = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<dpsr_plan> plans;
  std::vector<Solve> host;  // per instance, bound pointers
  std::vector<int64_t> nmax;
  std::vector<BatchClass> classes;
  Solve* hstage = nullptr;  // pinned staging of the tables
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_bwd = -1;  // what the graph holds: 0 forward, 1 forward + backward, 2 training step
  bool have_fwd = false;
};

namespace {

int upload(dpsr_batch b) {
  size_t off = 0;
  for (auto& c : b->classes) {
    for (size_t k = 0; k < c.members.size(); ++k) b->hstage[off + k] = b->host[c.members[k]];
    if (cudaMemcpyAsync(c.dtab, b->hstage + off, sizeof(Solve) * c.members.size(),
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return DPSR_ECUDA;
    off += c.members.size();
  }
  return DPSR_OK;
}

// Launch `body(class, stream)` for every class on the class's stream, after
// everything queued on the batch stream, and make the batch stream wait for
// all of them.
template <class F>
cudaError_t per_class(dpsr_batch b, F body) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (auto& c : b->classes) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.st, b->fork, 0);
    if (e == cudaSuccess) e = body(c, c.st);
    if (e == cudaSuccess) e = cudaEventRecord(c.join, c.st);
  }
  for (auto& c : b->classes)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, c.join, 0);
  return e;
}

cudaError_t launch_fwd(dpsr_batch b) {
  const Solve dummy = {};
  return per_class(b, [&](BatchClass& c, cudaStream_t st) {
    const int n = (int)c.members.size();
    cudaError_t e = dpsr::launch_bin(dummy, c.dtab, n, c.nmax, c.r, st);
    if (e == cudaSuccess) e = dpsr::launch_plane(0, c.r, c.C[0], dummy, c.dtab, n, st);
    if (e == cudaSuccess) e = dpsr::launch_xpass(false, c.r, dummy, c.dtab, n, st);
    if (e == cudaSuccess) e = dpsr::launch_plane(1, c.r, c.C[1], dummy, c.dtab, n, st);
    return e;
  });
}

// L_DPSR of every instance against its bound target (Eq. 9), gradient into
// the instance's dchi buffer.
cudaError_t launch_mse(dpsr_batch b) {
  const Solve dummy = {};
  return per_class(b, [&](BatchClass& c, cudaStream_t st) {
    return dpsr::launch_mse_grad(dummy, c.dtab, (int)c.members.size(), c.r, st);
  });
}

cudaError_t launch_bwd(dpsr_batch b) {
  const Solve dummy = {};
  return per_class(b, [&](BatchClass& c, cudaStream_t st) {
    const int n = (int)c.members.size();
    cudaError_t e = dpsr::launch_plane(2, c.r, c.C[2], dummy, c.dtab, n, st);
    if (e == cudaSuccess) e = dpsr::launch_xpass(true, c.r, dummy, c.dtab, n, st);
    if (e == cudaSuccess) e = dpsr::launch_plane(3, c.r, c.C[3], dummy, c.dtab, n, st);
    if (e == cudaSuccess) e = dpsr::launch_combine(dummy, c.dtab, n, c.nmax, c.C[3] == dpsr::kPathSplit, st);
    return e;
  });
}

// Batch autotuner. A class launch covers all of its instances, so it is
// bound by throughput where a solo solve is bound by latency, and the best
// plane path can differ from the solo choice. On the first eager run of a
// batch, each plane kind of each class is timed over every path that fits
// (the pencil passes and each cluster size; fastest of three timed runs after
// an untimed one) on the class's own instances, in the order of the solve, so
// that every kind runs on its real inputs; the last run leaves the chosen
// path's results. The environment's fixed paths (DPSR_PLANE_PATH[S_<r>]) and
// DPSR_TUNE=0 take precedence; a choice persisted in the DPSR_TUNE_CACHE file
// for this class size is used without timing.
cudaError_t tune_kind(BatchClass& c, int kind, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  const Solve dummy = {};
  const int n = (int)c.members.size();
  const int forced = dpsr_internal_forced(kind, c.r);
  if (forced != -1) {
    if (forced >= 0) c.C[kind] = forced;
    c.tuned[kind] = true;
    return dpsr::launch_plane(kind, c.r, c.C[kind], dummy, c.dtab, n, st);
  }
  {  // a choice persisted by an earlier process (DPSR_TUNE_CACHE)
    const int cached = dpsr_internal_tc_lookup(kind, c.r, n);
    const size_t sm = cached >= 0 ? dpsr::plane_smem_bytes(kind, c.r, cached) : 0;
    if (sm != 0 && sm <= 227 * 1024 - 1024) {
      c.C[kind] = cached;
      c.tuned[kind] = true;
      return dpsr::launch_plane(kind, c.r, cached, dummy, c.dtab, n, st);
    }
  }
  const int cands[6] = {0, 1, 2, 4, 8, dpsr::kPathSplit};
  float best = 1e30f;
  int bestC = c.C[kind];
  for (int C : cands) {
    const size_t sm = dpsr::plane_smem_bytes(kind, c.r, C);
    if (sm == 0 || sm > 227 * 1024 - 1024) continue;
    cudaError_t e = dpsr::launch_plane(kind, c.r, C, dummy, c.dtab, n, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      float m = 0.f;
      e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = dpsr::launch_plane(kind, c.r, C, dummy, c.dtab, n, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&m, e0, e1);
      if (e == cudaSuccess && m < ms) ms = m;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (ms < best) {
      best = ms;
      bestC = C;
    }
  }
  c.C[kind] = bestC;
  c.tuned[kind] = true;
  cudaError_t e = dpsr::launch_plane(kind, c.r, bestC, dummy, c.dtab, n, st);
  if (e == cudaSuccess && best < 1e30f) dpsr_internal_tc_store(kind, c.r, n, bestC, best);
  return e;
}

// One eager forward (and backward) of every class on the batch stream, tuning
// the plane kinds not tuned yet. Not capturable (it synchronises on events).
cudaError_t tune_batch(dpsr_batch b, bool with_bwd) {
  const Solve dummy = {};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  cudaStream_t st = b->stream;
  for (auto& c : b->classes) {
    const int n = (int)c.members.size();
    auto plane = [&](int kind) {
      return c.tuned[kind] ? dpsr::launch_plane(kind, c.r, c.C[kind], dummy, c.dtab, n, st)
                           : tune_kind(c, kind, st, e0, e1);
    };
    if (e == cudaSuccess) e = dpsr::launch_bin(dummy, c.dtab, n, c.nmax, c.r, st);
    if (e == cudaSuccess) e = plane(0);
    if (e == cudaSuccess) e = dpsr::launch_xpass(false, c.r, dummy, c.dtab, n, st);
    if (e == cudaSuccess) e = plane(1);
    if (with_bwd) {
      if (e == cudaSuccess) e = plane(2);
      if (e == cudaSuccess) e = dpsr::launch_xpass(true, c.r, dummy, c.dtab, n, st);
      if (e == cudaSuccess) e = plane(3);
      if (e == cudaSuccess) e = dpsr::launch_combine(dummy, c.dtab, n, c.nmax, c.C[3] == dpsr::kPathSplit, st);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

bool needs_tuning(dpsr_batch b, bool with_bwd) {
  for (auto& c : b->classes)
    for (int k = 0; k < (with_bwd ? 4 : 2); ++k)
      if (!c.tuned[k]) return true;
  return false;
}

void drop_graph(dpsr_batch b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_bwd = -1;
}

}  // namespace

extern "C" {

int dpsr_batch_create(int count, const int* r, const float* sigma, const int64_t* n_max,
                      dpsr_batch* out) {
  return dpsr_batch_create_box(count, r, sigma, nullptr, n_max, out);
}

int dpsr_batch_create_box(int count, const int* r, const float* sigma, const double* box,
                          const int64_t* n_max, dpsr_batch* out) {
  if (!out || count < 1 || !r || !sigma || !n_max) return DPSR_EINVAL;
  *out = nullptr;
  dpsr_batch b = new (std::nothrow) dpsr_batch_s();
  if (!b) return DPSR_ENOMEM;
  b->count = count;
  cudaGetDevice(&b->device);
  b->plans.assign(count, nullptr);
  b->host.resize(count);
  b->nmax.assign(n_max, n_max + count);
  int rc = DPSR_OK;
  for (int i = 0; i < count && rc == DPSR_OK; ++i) {
    rc = dpsr_plan_create_box(r[i], sigma[i], box ? box + 3 * i : nullptr, &b->plans[i]);
    if (rc == DPSR_OK) rc = dpsr_plan_reserve(b->plans[i], n_max[i]);
    if (rc == DPSR_OK) memcpy(&b->host[i], dpsr_internal_solve(b->plans[i]), sizeof(Solve));
  }
  if (rc == DPSR_OK) {
    std::vector<int> rs(r, r + count);
    std::sort(rs.begin(), rs.end());
    rs.erase(std::unique(rs.begin(), rs.end()), rs.end());
    for (int rr : rs) {
      BatchClass c;
      c.r = rr;
      for (int i = 0; i < count; ++i)
        if (r[i] == rr) {
          c.members.push_back(i);
          c.nmax = std::max<int>(c.nmax, (int)n_max[i]);
        }
      for (int k = 0; k < 4; ++k) c.C[k] = dpsr_internal_cluster(b->plans[c.members[0]], k);
      if (cudaMalloc(&c.dtab, sizeof(Solve) * c.members.size()) != cudaSuccess ||
          cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rc = DPSR_ENOMEM;
      }
      b->classes.push_back(c);
    }
  }
  if (rc == DPSR_OK && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rc = DPSR_ENOMEM;
  }
  if (rc == DPSR_OK && cudaMallocHost(&b->hstage, sizeof(Solve) * count) != cudaSuccess) {
    cudaGetLastError();
    rc = DPSR_ENOMEM;
  }
  if (rc != DPSR_OK) {
    dpsr_batch_destroy(b);
    return rc;
  }
  *out = b;
  return DPSR_OK;
}

int dpsr_batch_destroy(dpsr_batch b) {
  if (!b) return DPSR_EINVAL;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& c : b->classes) {
    if (c.st) cudaStreamSynchronize(c.st);
    if (c.join) cudaEventDestroy(c.join);
    if (c.st) cudaStreamDestroy(c.st);
    if (c.dtab) cudaFree(c.dtab);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  for (dpsr_plan p : b->plans)
    if (p) dpsr_plan_destroy(p);
  if (b->hstage) cudaFreeHost(b->hstage);
  delete b;
  return DPSR_OK;
}

int dpsr_batch_set_stream(dpsr_batch b, void* stream) {
  if (!b) return DPSR_EINVAL;
  b->stream = (cudaStream_t)stream;
  for (dpsr_plan p : b->plans) dpsr_plan_set_stream(p, stream);
  drop_graph(b);
  return DPSR_OK;
}

int dpsr_batch_bind(dpsr_batch b, int i, const float* points, const float* normals, int64_t N,
                    float* chi, const float* dchi, float* dpoints, float* dnormals) {
  if (!b || i < 0 || i >= b->count || !points || !normals || !chi) return DPSR_EINVAL;
  if (N < 1 || N > b->nmax[i]) return DPSR_ESTATE;
  if (((uintptr_t)chi & 15) || ((uintptr_t)dchi & 15)) return DPSR_EINVAL;
  Solve& s = b->host[i];
  s.points = points;
  s.normals = normals;
  dpsr::set_count(s, N);
  s.chi = chi;
  s.dchi = dchi;
  s.dchi_rw = const_cast<float*>(dchi);  // written by the training step's loss pass
  s.dpoints = dpoints;
  s.dnormals = dnormals;
  return DPSR_OK;
}

int dpsr_batch_forward(dpsr_batch b) {
  dpsr::NvtxRange nvtx_call("dpsr_batch_forward");
  if (!b) return DPSR_EINVAL;
  int rc = upload(b);
  if (rc != DPSR_OK) return rc;
  const bool tune = needs_tuning(b, false);
  if ((tune ? tune_batch(b, false) : launch_fwd(b)) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  b->have_fwd = true;
  return DPSR_OK;
}

int dpsr_batch_backward(dpsr_batch b) {
  dpsr::NvtxRange nvtx_call("dpsr_batch_backward");
  if (!b) return DPSR_EINVAL;
  if (!b->have_fwd) return DPSR_ESTATE;
  for (int i = 0; i < b->count; ++i)
    if (!b->host[i].dchi || !b->host[i].dpoints || !b->host[i].dnormals) return DPSR_EINVAL;
  int rc = upload(b);
  if (rc != DPSR_OK) return rc;
  // tuning the backward kinds runs the forward again first (it is idempotent)
  const bool tune = needs_tuning(b, true);
  if ((tune ? tune_batch(b, true) : launch_bwd(b)) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  return DPSR_OK;
}

// mode: 0 forward, 1 forward + backward, 2 training step (forward, L_DPSR
// against the bound targets, backward).
static int graph_launch(dpsr_batch b, int mode) {
  if (!b) return DPSR_EINVAL;
  const bool with_bwd = mode != 0;
  if (with_bwd)
    for (int i = 0; i < b->count; ++i)
      if (!b->host[i].dchi || !b->host[i].dpoints || !b->host[i].dnormals) return DPSR_EINVAL;
  if (mode == 2)
    for (int i = 0; i < b->count; ++i)
      if (!b->host[i].target) return DPSR_EINVAL;
  int rc = upload(b);
  if (rc != DPSR_OK) return rc;
  if (!b->graph || b->graph_bwd != mode) {
    drop_graph(b);
    if (b->stream == nullptr) return DPSR_EINVAL;  // capture needs a non-default stream
    if (needs_tuning(b, with_bwd)) {  // picks the paths the graph will hold
      if (tune_batch(b, with_bwd) != cudaSuccess) {
        cudaGetLastError();
        return DPSR_ECUDA;
      }
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return DPSR_ECUDA;
    cudaError_t e = launch_fwd(b);
    if (e == cudaSuccess && mode == 2) e = launch_mse(b);
    if (e == cudaSuccess && with_bwd) e = launch_bwd(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return DPSR_ECUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->graph = nullptr;
      return DPSR_ECUDA;
    }
    b->graph_bwd = mode;
  }
  if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  b->have_fwd = true;
  return DPSR_OK;
}

int dpsr_batch_graph_launch(dpsr_batch b, int with_bwd) {
  dpsr::NvtxRange nvtx_call("dpsr_batch_graph_launch");
  return graph_launch(b, with_bwd ? 1 : 0);
}

int dpsr_batch_bind_target(dpsr_batch b, int i, const float* target) {
  if (!b || i < 0 || i >= b->count || !target) return DPSR_EINVAL;
  if (((uintptr_t)target) & 15) return DPSR_EINVAL;
  b->host[i].target = target;
  return DPSR_OK;
}

int dpsr_batch_train_step(dpsr_batch b) {
  dpsr::NvtxRange nvtx_call("dpsr_batch_train_step");
  if (!b) return DPSR_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (((uintptr_t)b->host[i].dchi_rw) & 15) return DPSR_EINVAL;
  return graph_launch(b, 2);
}

int dpsr_batch_losses(dpsr_batch b, double* out) {
  if (!b || !out) return DPSR_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  for (int i = 0; i < b->count; ++i)
    if (cudaMemcpy(&out[i], &b->host[i].sc->loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return DPSR_ECUDA;
  return DPSR_OK;
}

int dpsr_batch_sync(dpsr_batch b) {
  if (!b) return DPSR_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  // worst first: a failed CUDA call, then a timed-out wait, then a degenerate input
  auto rank = [](int st) {
    return st == DPSR_ECUDA ? 3 : (st == DPSR_ETIMEOUT ? 2 : (st == DPSR_OK ? 0 : 1));
  };
  int worst = DPSR_OK;
  for (dpsr_plan p : b->plans) {
    const int st = dpsr_sync(p);
    if (rank(st) > rank(worst)) worst = st;
  }
  return worst;
}

// Internal hooks for the server (same library, not exported): the plan of
// instance i (its staging buffers hold a request's inputs and outputs), and a
// run of the forward (and backward) of the first k instances only. The first
// k instances of a batch of one grid size are the first k members of its
// class, so a launch with k instances instead of all of them runs exactly
// those (the paths were tuned on the whole class).
dpsr_plan dpsr_internal_batch_plan(dpsr_batch b, int i) {
  return (b && i >= 0 && i < b->count) ? b->plans[i] : nullptr;
}

int dpsr_internal_batch_run(dpsr_batch b, int k, int with_bwd) {
  if (!b || b->classes.size() != 1 || k < 1 || k > b->count) return DPSR_EINVAL;
  BatchClass& c = b->classes[0];
  const Solve dummy = {};
  int rc = upload(b);
  if (rc != DPSR_OK) return rc;
  if (needs_tuning(b, with_bwd != 0)) {  // once, on the whole class (all bound)
    if (tune_batch(b, with_bwd != 0) != cudaSuccess) {
      cudaGetLastError();
      return DPSR_ECUDA;
    }
    return DPSR_OK;
  }
  cudaStream_t st = b->stream;
  cudaError_t e = dpsr::launch_bin(dummy, c.dtab, k, c.nmax, c.r, st);
  if (e == cudaSuccess) e = dpsr::launch_plane(0, c.r, c.C[0], dummy, c.dtab, k, st);
  if (e == cudaSuccess) e = dpsr::launch_xpass(false, c.r, dummy, c.dtab, k, st);
  if (e == cudaSuccess) e = dpsr::launch_plane(1, c.r, c.C[1], dummy, c.dtab, k, st);
  if (with_bwd) {
    if (e == cudaSuccess) e = dpsr::launch_plane(2, c.r, c.C[2], dummy, c.dtab, k, st);
    if (e == cudaSuccess) e = dpsr::launch_xpass(true, c.r, dummy, c.dtab, k, st);
    if (e == cudaSuccess) e = dpsr::launch_plane(3, c.r, c.C[3], dummy, c.dtab, k, st);
    if (e == cudaSuccess) e = dpsr::launch_combine(dummy, c.dtab, k, c.nmax, c.C[3] == dpsr::kPathSplit, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  b->have_fwd = true;
  return DPSR_OK;
}

int dpsr_batch_paths(dpsr_batch b, int r, int* C4) {
  if (!b || !C4) return DPSR_EINVAL;
  for (const auto& c : b->classes)
    if (c.r == r) {
      for (int k = 0; k < 4; ++k) C4[k] = c.C[k];
      return DPSR_OK;
    }
  return DPSR_EINVAL;
}

int dpsr_batch_launches(dpsr_batch b, int with_bwd) {
  if (!b) return -1;
  int n = 0;
  for (const auto& c : b->classes) {
    n += 3 + dpsr::plane_launches(c.C[0]) + dpsr::plane_launches(c.C[1]);
    if (with_bwd) n += 2 + dpsr::plane_launches(c.C[2]) + dpsr::plane_launches(c.C[3]);
  }
  return n;
}

}  // extern "C"
