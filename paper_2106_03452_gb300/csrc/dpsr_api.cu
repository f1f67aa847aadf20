// C ABI of libdpsr: plans, workspace, and the launch sequences of the forward
// and backward passes of the spectral DPSR layer.
//
// Forward (Sec. 3.1, Eq. A1-A9):
//   bin    counting sort of the points by the x-cell of their stencil
//   plane  per x-plane cluster: splat (Eq. A2), R2C along z, FFT along y
//   xpass  FFT along x, spectral solve (Eq. 3), inverse FFT along x, and the
//          spectral sums giving mu and chi'(0) (Eq. 4)
//   final  scalars mu, s, m/|s|
//   inv    per x-plane cluster: IFFT along y, C2R along z, chi = m/|s| (chi'-mu)
// Backward (adjoint of the above):
//   bfwd   R2C/y-FFT of dchi with sum(dchi) and sum(dchi chi)
//   final  s_bar, mu_bar and the coefficients of the adjoint spectrum
//   xpass  adjoint spectral solve, Q1 = IFFT_x(F), Q2 = IFFT_x(-i u_x F)
//   binv   IFFT along y, C2R along z of V_bar_{x,y,z}, gather + weight
//          derivatives at the points
//   combine  the two plane sides of each point, in the caller's order
#include <cstdio>
#include <cstdlib>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "dpsr.h"
#include "dpsr_dev.cuh"
#include "launch.h"
#include "nvtx.h"

using dpsr::Solve;

struct dpsr_plan_s {
  int r = 0;
  float sigma = 0.f;
  double box[3] = {1.0, 1.0, 1.0};  // side lengths of the periodic domain
  int device = 0;
  cudaStream_t stream = nullptr;
  int C[4] = {1, 1, 1, 1};
  // grid workspace
  void* grid_ws = nullptr;
  size_t grid_bytes = 0;
  // point workspace
  void* pts_ws = nullptr;
  int64_t n_cap = 0;
  Solve s = {};
  bool have_fwd = false;
  int spectra = 0;  // what the spectral buffers hold: 1 the forward's, 2 the backward's
  int last_launches = 0;
  // device staging for the host-buffer variants
  void* host_io = nullptr;
  size_t host_io_bytes = 0;
  int64_t host_n = 0;
  // recorded after the work of every forward / backward call: destroy waits on
  // it, so it never touches a stream the caller may have destroyed since
  cudaEvent_t done_ev = nullptr;
  // pinned host copy of the status word, filled on the plan's stream by
  // dpsr_sync so that one stream synchronisation returns it
  unsigned* status_host = nullptr;
  // dpsr_solve_host: a second stream for the copies that overlap the
  // kernels, and the events that order the two streams (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_dchi = nullptr, ev_fwd = nullptr, ev_chi = nullptr;
  // optional per-kernel timing: an event before and after each launch
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;  // kind of each recorded pair
  size_t ev_used = 0;        // events recorded (2 per launch)
};

namespace {

// Per-kernel event timing (plan profiling) launches without programmatic
// dependent launch, for the scope of one API call.
struct PdlScope {
  explicit PdlScope(bool off) { dpsr::pdl_suspend(off); }
  ~PdlScope() { dpsr::pdl_suspend(false); }
};

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool valid_r(int r) { return r >= 8 && r <= 512 && (r & (r - 1)) == 0; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t spec_bytes(int r) { return (size_t)r * r * dpsr::kpitch(r) * sizeof(float2); }

int part_count(int r) {
  const int a = dpsr::xpass_blocks(r), b = r * 16;
  return a > b ? a : b;
}

size_t grid_ws_bytes(int r) {
  size_t b = dpsr::kNSpec * align256(spec_bytes(r));
  b += align256(sizeof(float2) * r) + align256(sizeof(float) * 7 * r);
  b += align256(sizeof(dpsr::Scalars)) + align256(sizeof(unsigned));
  b += align256(sizeof(float4) * part_count(r));
  b += align256(sizeof(int) * dpsr::bins_ints(r));
  return b;
}

size_t pts_ws_bytes(int64_t n) {
  size_t b = align256(sizeof(float4) * 2 * n);  // sorted
  b += align256(sizeof(int) * n);              // cellx
  b += align256(sizeof(float4) * 2 * n);       // gfwd
  b += align256(sizeof(float) * 24 * n);       // slots ([2][3][n] float4 on the split adjoint path)
  return b;
}

// Cluster size of a plane kernel: the smallest whose CTAs fit two per SM
// (<= 113 KB of shared memory), else the smallest that fits at all, else 0:
// the pencil passes (r = 512, where no cluster kernel is built).
int pick_cluster(int kind, int r) {
  const int cands[4] = {1, 2, 4, 8};
  for (int C : cands) {
    const size_t sm = dpsr::plane_smem_bytes(kind, r, C);
    if (sm > 0 && sm <= 113 * 1024) return C;
  }
  for (int C : cands) {
    const size_t sm = dpsr::plane_smem_bytes(kind, r, C);
    if (sm > 0 && sm <= 227 * 1024 - 1024) return C;
  }
  return 0;
}

// Record an event (profiling mode only); pairs bracket one launch.
cudaError_t prof_mark(dpsr_plan p, int kind, bool begin) {
  if (!p->profile) return cudaSuccess;
  if (p->ev_used == p->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    p->ev_pool.push_back(e);
  }
  if (begin) p->ev_kind.push_back(kind);
  return cudaEventRecord(p->ev_pool[p->ev_used++], p->stream);
}

int cuda_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? DPSR_ENOMEM : DPSR_ECUDA; }

// ---------------------------------------------------------------------------
// Autotuner: the cluster size C of each plane kernel (CTAs per x-plane) is
// picked by timing every candidate that fits on the first solve of a given r
// in this process. The plane kernels are idempotent (they rewrite the same
// outputs from the same inputs), so the candidates run in place, one after
// the other; the last run leaves the correct results. Results are cached per
// (kernel, r) for the process, and with DPSR_TUNE_CACHE=<file> persisted
// across processes (tune_cache.cu): a choice found there is used without
// timing. DPSR_TUNE=0 in the environment switches the tuner off (the static
// choice of pick_cluster is used).
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
int g_tuned[4][10] = {};  // [kind][log2 r]: 1 + chosen C (0 = pencil path), 0 = not tuned yet

}  // namespace
extern "C" int dpsr_internal_tc_lookup(int kind, int r, int batch);
extern "C" void dpsr_internal_tc_store(int kind, int r, int batch, int path, float ms);
namespace {

int log2i(int r) {
  int l = 0;
  while ((1 << l) < r) ++l;
  return l;
}

bool tuning_enabled() {
  const char* e = getenv("DPSR_TUNE");
  return !(e && e[0] == '0');
}

// Plane paths fixed from the environment (tests and measurements):
// DPSR_PLANE_PATHS_<r> = "a,b,c,d" fixes the four kinds at grid size r (for
// instance the choices an autotuned run reported, to profile the same
// kernels), else DPSR_PLANE_PATH fixes every kind at every r; 0 = pencil
// passes, 1/2/4/8 = cluster size, 3 = the adjoint kind split by channel
// (kind 3 only). Returns -1 when neither applies.
int forced_path(int kind, int r) {
  auto valid = [](int c) { return dpsr::valid_path(c); };
  char name[32];
  snprintf(name, sizeof(name), "DPSR_PLANE_PATHS_%d", r);
  if (const char* e = getenv(name)) {
    int c[4];
    if (sscanf(e, "%d,%d,%d,%d", &c[0], &c[1], &c[2], &c[3]) == 4 && kind >= 0 && kind < 4 &&
        valid(c[kind]))
      return c[kind];
  }
  const char* e = getenv("DPSR_PLANE_PATH");
  if (!e || !*e) return -1;
  const int c = atoi(e);
  return valid(c) && c != dpsr::kPathSplit ? c : -1;  // the split path exists for one kind only
}

// Launch plane kernel `kind` for every candidate C, time each with events
// (the fastest of three timed runs after one untimed, so that one disturbed
// run does not decide), record the fastest. Returns the last launch error.
cudaError_t tune_plane(dpsr_plan p, int kind, const Solve& s, cudaStream_t st) {
  const int r = p->r;
  const int cands[6] = {0, 1, 2, 4, 8, dpsr::kPathSplit};  // 0: the z/y pencil passes
  float best = 1e30f;
  int bestC = p->C[kind];
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cudaGetLastError();
  }
  for (int C : cands) {
    const size_t sm = dpsr::plane_smem_bytes(kind, r, C);
    if (sm == 0 || sm > 227 * 1024 - 1024) continue;
    cudaError_t e = dpsr::launch_plane(kind, r, C, s, nullptr, 1, st);
    if (e != cudaSuccess) {  // e.g. a cluster shape this GPU cannot schedule
      cudaGetLastError();
      continue;
    }
    float ms = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, st);
      e = dpsr::launch_plane(kind, r, C, s, nullptr, 1, st);
      cudaEventRecord(e1, st);
      float m = 0.f;
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&m, e0, e1) != cudaSuccess) {
        e = cudaErrorUnknown;
        break;
      }
      ms = m < ms ? m : ms;
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
  // leave the outputs of the chosen configuration in place
  cudaError_t e = dpsr::launch_plane(kind, r, bestC, s, nullptr, 1, st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[kind][log2i(r)] = bestC + 1;
      p->C[kind] = bestC;
    }
    dpsr_internal_tc_store(kind, r, 0, bestC, best);
  }
  return e;
}

// Launch plane kernel `kind`, tuning it first if it has not been tuned for
// this r (and the stream is not being captured).
cudaError_t run_plane(dpsr_plan p, int kind, const Solve& s, cudaStream_t st) {
  const int forced = forced_path(kind, p->r);
  if (forced >= 0) {
    p->C[kind] = forced;
    return dpsr::launch_plane(kind, p->r, forced, s, nullptr, 1, st);
  }
  if (tuning_enabled() && p->r >= 64) {
    int tuned;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tuned = g_tuned[kind][log2i(p->r)];
    }
    if (!tuned) {  // a choice persisted by an earlier process (DPSR_TUNE_CACHE)
      const int c = dpsr_internal_tc_lookup(kind, p->r, 0);
      const size_t sm = c >= 0 ? dpsr::plane_smem_bytes(kind, p->r, c) : 0;
      if (sm != 0 && sm <= 227 * 1024 - 1024) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[kind][log2i(p->r)] = c + 1;
        tuned = c + 1;
      }
    }
    if (tuned) {
      p->C[kind] = tuned - 1;
    } else {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone && !p->profile)
        return tune_plane(p, kind, s, st);
    }
  }
  return dpsr::launch_plane(kind, p->r, p->C[kind], s, nullptr, 1, st);
}

int grow_points(dpsr_plan p, int64_t n) {
  if (n <= p->n_cap) return DPSR_OK;
  int64_t cap = p->n_cap ? p->n_cap : 1024;
  while (cap < n) cap *= 2;
  if (p->pts_ws) {
    if (p->done_ev) cudaEventSynchronize(p->done_ev);
    cudaFree(p->pts_ws);
    p->pts_ws = nullptr;
    p->n_cap = 0;
  }
  void* w = nullptr;
  cudaError_t e = cudaMalloc(&w, pts_ws_bytes(cap));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ENOMEM;
  }
  p->pts_ws = w;
  p->n_cap = cap;
  char* q = (char*)w;
  p->s.sorted = (float4*)q;
  q += align256(sizeof(float4) * 2 * cap);
  p->s.cellx = (int*)q;
  q += align256(sizeof(int) * cap);
  p->s.gfwd = (float4*)q;
  q += align256(sizeof(float4) * 2 * cap);
  p->s.slots = (float*)q;
  p->have_fwd = false;
  return DPSR_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

namespace dpsr {
static thread_local bool t_pdl_off = false;

int status_code(unsigned st) {
  if (st & kStTimeout) return DPSR_ETIMEOUT;  // a wait gave up: the outputs are incomplete
  if (st & kStBounds) return DPSR_EBOUNDS;    // a debug-build index check failed
  if (st) return DPSR_EDEGENERATE;
  return DPSR_OK;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("DPSR_PDL");
    return !(v && v[0] == '0');
  }();
  return on && !t_pdl_off;
}

void pdl_suspend(bool off) { t_pdl_off = off; }

// Spectral buffer k: complex (8-byte) elements [x][ky][kz], kz < r/2+1 valid
// out of a row pitch of r/2+2. tmx: boxes of 16 kz x 1 ky x r x; tmy: boxes
// of 16 kz x r ky x 1 x. Out-of-range kz reads as zero and is not written.
int make_tensor_maps(Solve& s, int r) {
  auto enc = tensor_map_encoder();
  if (!enc) return DPSR_ECUDA;
  const cuuint64_t dims[3] = {(cuuint64_t)(r / 2 + 1), (cuuint64_t)r, (cuuint64_t)r};
  const cuuint64_t strides[2] = {(cuuint64_t)kpitch(r) * 8, (cuuint64_t)r * kpitch(r) * 8};
  const cuuint32_t boxx[3] = {16, 1, (cuuint32_t)tma_rows(r)}, boxy[3] = {16, (cuuint32_t)tma_rows(r), 1};
  const cuuint32_t es[3] = {1, 1, 1};
  for (int k = 0; k < kNSpec; ++k) {
    for (int w = 0; w < 2; ++w) {
      CUresult rc = enc(w == 0 ? &s.tmx[k] : &s.tmy[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                        (void*)s.spec[k], dims, strides, w == 0 ? boxx : boxy, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (rc != CUDA_SUCCESS) return DPSR_ECUDA;
    }
  }
  return DPSR_OK;
}
}  // namespace dpsr

extern "C" {

const char* dpsr_strerror(int st) {
  switch (st) {
    case DPSR_OK: return "ok";
    case DPSR_EINVAL: return "invalid argument";
    case DPSR_ENOMEM: return "device out of memory";
    case DPSR_ECUDA: return "CUDA runtime error";
    case DPSR_EDEGENERATE: return "degenerate input (non-finite value or vanishing scale chi'(0) - mu)";
    case DPSR_ESTATE: return "invalid call order (backward without forward)";
    case DPSR_ETIMEOUT: return "bounded device wait timed out";
    case DPSR_EBUSY: return "resource busy";
    case DPSR_ECANCELED: return "request cancelled";
    case DPSR_EBOUNDS: return "debug index check failed";
    default: return "unknown status";
  }
}

int dpsr_check_bounded_wait(double limit_s) {
  if (!(limit_s > 0.0 && limit_s <= 10.0)) return DPSR_EINVAL;
  unsigned* d = nullptr;
  cudaStream_t st = nullptr;
  unsigned h = 0;
  int rc = DPSR_ECUDA;
  if (cudaMalloc(&d, sizeof(unsigned)) == cudaSuccess &&
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
      cudaMemsetAsync(d, 0, sizeof(unsigned), st) == cudaSuccess &&
      dpsr::launch_wait_probe(d, limit_s, st) == cudaSuccess &&
      cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
      cudaStreamSynchronize(st) == cudaSuccess)
    rc = (h & dpsr::kStTimeout) ? DPSR_ETIMEOUT : DPSR_OK;
  if (rc == DPSR_ECUDA) cudaGetLastError();
  if (st) cudaStreamDestroy(st);
  if (d) cudaFree(d);
  return rc;
}

size_t dpsr_plan_workspace_bytes(int r, int64_t n_max, int with_bwd) {
  (void)with_bwd;  // the backward reuses the forward's buffers
  if (!valid_r(r) || n_max < 0) return 0;
  return grid_ws_bytes(r) + pts_ws_bytes(n_max > 0 ? n_max : 1);
}

static bool valid_box(const double* box) {
  if (!box) return true;
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0.0) || !isfinite(box[d])) return false;
  return true;
}

int dpsr_plan_create(int r, float sigma, dpsr_plan* out) { return dpsr_plan_create_box(r, sigma, nullptr, out); }

int dpsr_plan_create_box(int r, float sigma, const double* box, dpsr_plan* out) {
  if (!out || !valid_r(r) || !(sigma >= 0.f) || !isfinite(sigma) || !valid_box(box)) return DPSR_EINVAL;
  *out = nullptr;
  dpsr_plan p = new (std::nothrow) dpsr_plan_s();
  if (!p) return DPSR_ENOMEM;
  p->r = r;
  p->sigma = sigma;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return DPSR_ECUDA;
  }
  for (int k = 0; k < 4; ++k) p->C[k] = pick_cluster(k, r);
  p->grid_bytes = grid_ws_bytes(r);
  if (cudaMalloc(&p->grid_ws, p->grid_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return DPSR_ENOMEM;
  }
  Solve& s = p->s;
  for (int d = 0; d < 3; ++d) {
    p->box[d] = box ? box[d] : 1.0;
    s.inv_box[d] = box ? (float)(1.0 / box[d]) : 1.f;
    s.box[d] = box ? box[d] : 1.0;
  }
  dpsr::set_grid(s, r);
  char* q = (char*)p->grid_ws;
  for (int k = 0; k < dpsr::kNSpec; ++k) {
    s.spec[k] = (float2*)q;
    q += align256(spec_bytes(r));
  }
  float2* tw = (float2*)q;
  q += align256(sizeof(float2) * r);
  float* tab = (float*)q;
  q += align256(sizeof(float) * 7 * r);
  s.sc = (dpsr::Scalars*)q;
  q += align256(sizeof(dpsr::Scalars));
  s.status = (unsigned*)q;
  q += align256(sizeof(unsigned));
  s.part = (float4*)q;
  q += align256(sizeof(float4) * part_count(r));
  s.bins = (int*)q;
  s.tw = tw;
  s.g1 = tab;
  s.u2 = tab + r;
  s.iu = tab + 4 * r;
  float2* htw = (float2*)malloc(sizeof(float2) * r);
  float* htab = (float*)malloc(sizeof(float) * 7 * r);
  int rc = DPSR_OK;
  if (!htw || !htab) {
    rc = DPSR_ENOMEM;
  } else {
    dpsr::spectral_tables(r, (double)sigma, box, htw, htab);
    if (cudaMemcpy(tw, htw, sizeof(float2) * r, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tab, htab, sizeof(float) * 7 * r, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s.bins, 0, sizeof(int) * dpsr::bins_ints(r)) != cudaSuccess ||
        cudaMemset(s.status, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(s.sc, 0, sizeof(dpsr::Scalars)) != cudaSuccess)
      rc = DPSR_ECUDA;
  }
  free(htw);
  free(htab);
  if (rc == DPSR_OK) rc = dpsr::make_tensor_maps(s, r);
  if (rc == DPSR_OK && cudaHostAlloc((void**)&p->status_host, sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    p->status_host = nullptr;
    rc = DPSR_ENOMEM;
  }
  if (rc == DPSR_OK && cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess)
    rc = DPSR_ECUDA;
  if (rc == DPSR_OK) rc = grow_points(p, 1024);
  if (rc != DPSR_OK) {
    cudaFree(p->grid_ws);
    if (p->pts_ws) cudaFree(p->pts_ws);
    if (p->status_host) cudaFreeHost(p->status_host);
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    delete p;
    return rc;
  }
  *out = p;
  return DPSR_OK;
}

int dpsr_plan_destroy(dpsr_plan p) {
  if (!p) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (p->done_ev) {
    cudaEventSynchronize(p->done_ev);
    cudaEventDestroy(p->done_ev);
  }
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  if (p->copy_stream) {
    cudaStreamSynchronize(p->copy_stream);
    cudaStreamDestroy(p->copy_stream);
  }
  for (cudaEvent_t e : {p->ev_dchi, p->ev_fwd, p->ev_chi})
    if (e) cudaEventDestroy(e);
  cudaFree(p->grid_ws);
  if (p->pts_ws) cudaFree(p->pts_ws);
  if (p->host_io) cudaFree(p->host_io);
  if (p->status_host) cudaFreeHost(p->status_host);
  delete p;
  return DPSR_OK;
}

int dpsr_plan_set_stream(dpsr_plan p, void* stream) {
  if (!p) return DPSR_EINVAL;
  p->stream = (cudaStream_t)stream;
  return DPSR_OK;
}

int dpsr_plan_reserve(dpsr_plan p, int64_t n_max) {
  if (!p || n_max < 1 || n_max > INT32_MAX / 2) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  return grow_points(p, n_max);
}

int dpsr_plan_last_launches(dpsr_plan p) { return p ? p->last_launches : -1; }

int dpsr_grid_sample(const float* grid, int r, const float* q, int64_t M, float* out,
                     void* stream) {
  if (!valid_r(r) || !grid || !q || !out || M < 0) return DPSR_EINVAL;
  if (M == 0) return DPSR_OK;
  return dpsr::launch_grid_sample(grid, r, q, M, out, (cudaStream_t)stream) == cudaSuccess
             ? DPSR_OK
             : DPSR_ECUDA;
}

int dpsr_grid_splat(float* grid, int r, const float* q, const float* vals, int64_t M,
                    int accumulate, void* stream) {
  if (!valid_r(r) || !grid || !q || !vals || M < 0) return DPSR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!accumulate &&
      cudaMemsetAsync(grid, 0, sizeof(float) * (size_t)r * r * r, st) != cudaSuccess)
    return DPSR_ECUDA;
  if (M == 0) return DPSR_OK;
  return dpsr::launch_grid_splat(grid, r, q, vals, M, st) == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

// Internal hooks for the batch driver (same library, not exported).
const void* dpsr_internal_solve(dpsr_plan p) { return p ? (const void*)&p->s : nullptr; }
int dpsr_internal_cluster(dpsr_plan p, int kind) {
  if (!p || kind < 0 || kind > 3) return 1;
  const int forced = forced_path(kind, p->r);
  if (forced >= 0) return forced;
  if (tuning_enabled()) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int t = g_tuned[kind][log2i(p->r)];
    if (t) return t - 1;
  }
  return p->C[kind];
}

// The path of plane kind `kind` at grid size r fixed by the environment, or
// -1 (tune), or -2 (tuning switched off: keep the plan's choice).
int dpsr_internal_forced(int kind, int r) {
  const int forced = forced_path(kind, r);
  if (forced >= 0) return forced;
  return tuning_enabled() ? -1 : -2;
}

int dpsr_plan_clusters(dpsr_plan p, int* C4) {
  if (!p || !C4) return DPSR_EINVAL;
  for (int k = 0; k < 4; ++k) C4[k] = p->C[k];
  return DPSR_OK;
}

int dpsr_plan_profile(dpsr_plan p, int enable) {
  if (!p) return DPSR_EINVAL;
  p->profile = enable != 0;
  p->ev_used = 0;
  p->ev_kind.clear();
  return DPSR_OK;
}

int dpsr_plan_profile_read(dpsr_plan p, double* ms, int* launches) {
  if (!p || !ms || !launches) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return DPSR_ECUDA;
  for (int k = 0; k < DPSR_K_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < p->ev_kind.size(); ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev_pool[2 * i], p->ev_pool[2 * i + 1]) != cudaSuccess)
      return DPSR_ECUDA;
    ms[p->ev_kind[i]] += t;
    launches[p->ev_kind[i]] += 1;
  }
  p->ev_used = 0;
  p->ev_kind.clear();
  return DPSR_OK;
}

int dpsr_forward(dpsr_plan p, const float* points, const float* normals, int64_t N,
                 float* chi_out) {
  dpsr::NvtxRange nvtx_call("dpsr_forward");
  if (!p || !points || !normals || !chi_out || N < 1 || N > INT32_MAX / 2) return DPSR_EINVAL;
  if (((uintptr_t)chi_out & 15) != 0) return DPSR_EINVAL;  // read back by vector loads
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  p->spectra = 0;
  int rc = grow_points(p, N);
  if (rc != DPSR_OK) return rc;
  PdlScope pdl(p->profile);
  Solve s = p->s;
  dpsr::set_count(s, N);
  s.points = points;
  s.normals = normals;
  s.chi = chi_out;
  const int r = p->r;
  cudaStream_t st = p->stream;
  cudaError_t e = cudaSuccess;
  auto run = [&](int kind, auto&& fn) {
    dpsr::NvtxRange nr(dpsr::stage_name(kind));
    if (e == cudaSuccess) e = prof_mark(p, kind, true);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = prof_mark(p, kind, false);
  };
  run(DPSR_K_BIN, [&] { return dpsr::launch_bin(s, nullptr, 1, (int)N, r, st); });
  run(DPSR_K_PLANE_FWD, [&] { return run_plane(p, 0, s, st); });
  run(DPSR_K_XPASS_FWD, [&] { return dpsr::launch_xpass(false, r, s, nullptr, 1, st); });
  run(DPSR_K_PLANE_INV, [&] { return run_plane(p, 1, s, st); });
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->have_fwd = false;
    // the x-pass may not have cleared the bin counters: the next forward needs them at zero
    cudaMemsetAsync(s.bins, 0, sizeof(int) * dpsr::bins_ints(r), st);
    return cuda_err(e);
  }
  // bin: count and scatter (+ scan), plane pass(es), x-pass (+ scalars), inverse plane pass(es)
  p->last_launches = 3 + dpsr::plane_launches(p->C[0]) + dpsr::plane_launches(p->C[1]);
  cudaEventRecord(p->done_ev, st);
  p->s.N = s.N;
  p->s.inv_N = s.inv_N;
  p->s.points = points;
  p->s.normals = normals;
  p->s.chi = chi_out;
  p->have_fwd = true;
  p->spectra = 1;
  return DPSR_OK;
}

int dpsr_backward(dpsr_plan p, const float* dchi, float* dpoints, float* dnormals) {
  dpsr::NvtxRange nvtx_call("dpsr_backward");
  if (!p || !dchi || !dpoints || !dnormals) return DPSR_EINVAL;
  if (((uintptr_t)dchi & 15) != 0) return DPSR_EINVAL;  // rows move by bulk copies
  if (!p->have_fwd) return DPSR_ESTATE;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  p->spectra = 0;  // the backward reuses the forward's spectral buffers
  PdlScope pdl(p->profile);
  Solve s = p->s;
  s.dchi = dchi;
  s.dpoints = dpoints;
  s.dnormals = dnormals;
  const int r = p->r;
  cudaStream_t st = p->stream;
  cudaError_t e = cudaSuccess;
  auto run = [&](int kind, auto&& fn) {
    dpsr::NvtxRange nr(dpsr::stage_name(kind));
    if (e == cudaSuccess) e = prof_mark(p, kind, true);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = prof_mark(p, kind, false);
  };
  run(DPSR_K_PLANE_BFWD, [&] { return run_plane(p, 2, s, st); });
  run(DPSR_K_XPASS_BWD, [&] { return dpsr::launch_xpass(true, r, s, nullptr, 1, st); });
  run(DPSR_K_PLANE_BINV, [&] { return run_plane(p, 3, s, st); });
  run(DPSR_K_COMBINE, [&] { return dpsr::launch_combine(s, nullptr, 1, s.N, p->C[3] == dpsr::kPathSplit, st); });
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_err(e);
  }
  // plane pass(es) (+ scalars), x-pass, inverse plane pass(es), combine
  p->last_launches = 2 + dpsr::plane_launches(p->C[2]) + dpsr::plane_launches(p->C[3]);
  p->spectra = 2;
  cudaEventRecord(p->done_ev, st);
  return DPSR_OK;
}

int dpsr_sync(dpsr_plan p) {
  if (!p) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  // the status word comes back on the plan's stream, behind its work: one
  // host round trip
  if (cudaMemcpyAsync(p->status_host, p->s.status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                      p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  const unsigned st = *p->status_host;
  if (st) cudaMemset(p->s.status, 0, sizeof(unsigned));
  return dpsr::status_code(st);
}

int dpsr_plan_check_bounded_wait(dpsr_plan p, double limit_s) {
  if (!p || !(limit_s > 0.0 && limit_s <= 10.0)) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  if (dpsr::launch_wait_probe(p->s.status, limit_s, p->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  cudaEventRecord(p->done_ev, p->stream);
  return DPSR_OK;
}

int dpsr_mse_grad(dpsr_plan p, const float* target, float* dchi) {
  if (!p || !target || !dchi) return DPSR_EINVAL;
  if ((((uintptr_t)target) | ((uintptr_t)dchi)) & 15) return DPSR_EINVAL;  // float4 accesses
  if (!p->have_fwd) return DPSR_ESTATE;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  PdlScope pdl(p->profile);
  Solve s = p->s;
  s.target = target;
  s.dchi_rw = dchi;
  if (dpsr::launch_mse_grad(s, nullptr, 1, p->r, p->stream) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  cudaEventRecord(p->done_ev, p->stream);
  return DPSR_OK;
}

int dpsr_get_loss(dpsr_plan p, double* loss) {
  if (!p || !loss) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return DPSR_ECUDA;
  if (cudaMemcpy(loss, &p->s.sc->loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DPSR_ECUDA;
  return DPSR_OK;
}

int dpsr_debug_read_spectrum(dpsr_plan p, int which, void* out_host) {
  if (!p || !out_host || which < 0 || which > 5) return DPSR_EINVAL;
  if (p->spectra != (which < 4 ? 1 : 2)) return DPSR_ESTATE;
  DeviceGuard dg(p->device);
  if (!dg.ok || cudaStreamSynchronize(p->stream) != cudaSuccess) return DPSR_ECUDA;
  static const int buf[6] = {dpsr::kSpD, dpsr::kSpC, dpsr::kSpW, dpsr::kSpChi, dpsr::kSpD, dpsr::kSpChi};
  const int r = p->r;
  const size_t w = sizeof(float2) * (size_t)(r / 2 + 1);
  if (cudaMemcpy2D(out_host, w, p->s.spec[buf[which]], sizeof(float2) * (size_t)dpsr::kpitch(r), w,
                   (size_t)r * r, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  return DPSR_OK;
}

int dpsr_get_scalars(dpsr_plan p, double out[3]) {
  if (!p || !out) return DPSR_EINVAL;
  if (!p->have_fwd) return DPSR_ESTATE;
  DeviceGuard dg(p->device);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return DPSR_ECUDA;
  dpsr::Scalars sc;
  if (cudaMemcpy(&sc, p->s.sc, sizeof(sc), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DPSR_ECUDA;
  out[0] = sc.mu;
  out[1] = sc.s;
  out[2] = sc.alpha;
  return DPSR_OK;
}

// Host-buffer variants: device staging owned by the plan.
static int host_io_reserve(dpsr_plan p, int64_t N) {
  const size_t need = align256(sizeof(float) * 3 * N) * 4 + align256(sizeof(float) * p->r * p->r * p->r) * 2;
  if (need <= p->host_io_bytes) return DPSR_OK;
  if (p->host_io) {
    if (p->done_ev) cudaEventSynchronize(p->done_ev);
    cudaFree(p->host_io);
    p->host_io = nullptr;
    p->host_io_bytes = 0;
  }
  if (cudaMalloc(&p->host_io, need) != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ENOMEM;
  }
  p->host_io_bytes = need;
  return DPSR_OK;
}

struct HostIo {
  float *pts, *nrm, *dpts, *dnrm, *chi, *dchi;
};
static HostIo host_io_view(dpsr_plan p, int64_t N) {
  HostIo v;
  char* q = (char*)p->host_io;
  const size_t a = align256(sizeof(float) * 3 * N), g = align256(sizeof(float) * p->r * p->r * p->r);
  v.pts = (float*)q;
  v.nrm = (float*)(q + a);
  v.dpts = (float*)(q + 2 * a);
  v.dnrm = (float*)(q + 3 * a);
  v.chi = (float*)(q + 4 * a);
  v.dchi = (float*)(q + 4 * a + g);
  return v;
}

// Internal hook for the server (same library): the plan's device staging
// buffers for N points.
int dpsr_internal_io(dpsr_plan p, int64_t N, float** pts, float** nrm, float** chi, float** dchi,
                     float** dpts, float** dnrm) {
  if (!p || N < 1) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  const int rc = host_io_reserve(p, N);
  if (rc != DPSR_OK) return rc;
  HostIo v = host_io_view(p, N);
  *pts = v.pts;
  *nrm = v.nrm;
  *chi = v.chi;
  *dchi = v.dchi;
  *dpts = v.dpts;
  *dnrm = v.dnrm;
  return DPSR_OK;
}

int dpsr_forward_host(dpsr_plan p, const float* points, const float* normals, int64_t N,
                      float* chi_out) {
  dpsr::NvtxRange nvtx_call("dpsr_forward_host");
  if (!p || !points || !normals || !chi_out || N < 1 || N > INT32_MAX / 2) return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  int rc = host_io_reserve(p, N);
  if (rc != DPSR_OK) return rc;
  HostIo v = host_io_view(p, N);
  const size_t nb = sizeof(float) * 3 * N, gb = sizeof(float) * p->r * p->r * p->r;
  if (cudaMemcpyAsync(v.pts, points, nb, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaMemcpyAsync(v.nrm, normals, nb, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
    return DPSR_ECUDA;
  rc = dpsr_forward(p, v.pts, v.nrm, N, v.chi);
  if (rc != DPSR_OK) return rc;
  if (cudaMemcpyAsync(chi_out, v.chi, gb, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
    return DPSR_ECUDA;
  p->host_n = N;
  return dpsr_sync(p);
}

int dpsr_solve_host(dpsr_plan p, const float* points, const float* normals, int64_t N, const float* dchi,
                    float* chi_out, float* dpoints, float* dnormals) {
  dpsr::NvtxRange nvtx_call("dpsr_solve_host");
  if (!p || !points || !normals || !dchi || !chi_out || !dpoints || !dnormals || N < 1 || N > INT32_MAX / 2)
    return DPSR_EINVAL;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  int rc = host_io_reserve(p, N);
  if (rc != DPSR_OK) return rc;
  if (!p->copy_stream) {
    if (cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_dchi, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fwd, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_chi, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return DPSR_ECUDA;
    }
  }
  HostIo v = host_io_view(p, N);
  const size_t nb = sizeof(float) * 3 * N, gb = sizeof(float) * p->r * p->r * p->r;
  cudaStream_t st = p->stream, cs = p->copy_stream;
  // copy stream: the upstream gradient goes up while the forward pass runs;
  // the plan's stream (and the staging it reuses) is free of earlier work first
  if (cudaEventRecord(p->ev_fwd, st) != cudaSuccess || cudaStreamWaitEvent(cs, p->ev_fwd, 0) != cudaSuccess ||
      cudaMemcpyAsync(v.dchi, dchi, gb, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
      cudaEventRecord(p->ev_dchi, cs) != cudaSuccess)
    return DPSR_ECUDA;
  if (cudaMemcpyAsync(v.pts, points, nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(v.nrm, normals, nb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return DPSR_ECUDA;
  rc = dpsr_forward(p, v.pts, v.nrm, N, v.chi);
  if (rc != DPSR_OK) return rc;
  // chi comes down while the backward pass runs (it reads chi, never writes it)
  if (cudaEventRecord(p->ev_fwd, st) != cudaSuccess || cudaStreamWaitEvent(cs, p->ev_fwd, 0) != cudaSuccess ||
      cudaMemcpyAsync(chi_out, v.chi, gb, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaEventRecord(p->ev_chi, cs) != cudaSuccess || cudaStreamWaitEvent(st, p->ev_dchi, 0) != cudaSuccess)
    return DPSR_ECUDA;
  p->host_n = N;
  rc = dpsr_backward(p, v.dchi, v.dpts, v.dnrm);
  if (rc != DPSR_OK) return rc;
  if (cudaMemcpyAsync(dpoints, v.dpts, nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(dnormals, v.dnrm, nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamWaitEvent(st, p->ev_chi, 0) != cudaSuccess)
    return DPSR_ECUDA;
  return dpsr_sync(p);
}

int dpsr_backward_host(dpsr_plan p, const float* dchi, float* dpoints, float* dnormals) {
  dpsr::NvtxRange nvtx_call("dpsr_backward_host");
  if (!p || !dchi || !dpoints || !dnormals) return DPSR_EINVAL;
  if (!p->have_fwd || p->s.points != (const float*)host_io_view(p, p->host_n).pts)
    return DPSR_ESTATE;
  DeviceGuard dg(p->device);
  if (!dg.ok) return DPSR_ECUDA;
  const int64_t N = p->host_n;
  HostIo v = host_io_view(p, N);
  const size_t nb = sizeof(float) * 3 * N, gb = sizeof(float) * p->r * p->r * p->r;
  if (cudaMemcpyAsync(v.dchi, dchi, gb, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
    return DPSR_ECUDA;
  int rc = dpsr_backward(p, v.dchi, v.dpts, v.dnrm);
  if (rc != DPSR_OK) return rc;
  if (cudaMemcpyAsync(dpoints, v.dpts, nb, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaMemcpyAsync(dnormals, v.dnrm, nb, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
    return DPSR_ECUDA;
  return dpsr_sync(p);
}

}  // extern "C"
