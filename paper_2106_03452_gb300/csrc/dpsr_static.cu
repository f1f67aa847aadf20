// dpsr_forward_static: the DPSR forward pass for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host callback
// or a driver layer where allocation would deadlock or is forbidden, plugins
// handed a fixed memory budget by a host application, and real-time loops
// that must not hit the allocator's latency. For them this entry point runs
// the same kernels as dpsr_forward, but all of its scratch memory lives in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits. It calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// Limits: r <= 64 and N <= 65536 (the array is sized for exactly that).
// Larger sizes are rejected with DPSR_EINVAL.
//
// Sharing: every call, on every stream, uses the same array, and the array
// keeps what the last call left in it. Calls that overlap on the GPU race on
// it and corrupt each other's results; this entry point therefore waits for
// its own work to finish before it returns. Calls from several host threads
// at once overlap on the GPU whatever streams they use, so they are not
// supported. What must start at zero (the bin counters and the status word)
// is cleared at the start of each call.
//
// Set-up: the first call in a CUDA context of a device looks up the device
// address of the array (cudaGetSymbolAddress, with that device current) and
// keeps it with the context's unique id; a device reset makes a new context,
// and the next call looks the address up again. The call synchronises its
// stream and reads the status word back, so it refuses to run (DPSR_ESTATE)
// while a stream capture is active.
#include <math.h>
#include <mutex>

#include <cudaTypedefs.h>

#include "dpsr.h"
#include "dpsr_dev.cuh"
#include "launch.h"

namespace {

constexpr int kMaxR = 64;
constexpr int kMaxN = 65536;
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the static scratch, for r = kMaxR and N = kMaxN.
constexpr size_t kSpec = al((size_t)kMaxR * kMaxR * dpsr::kpitch(kMaxR) * sizeof(float2));
constexpr size_t kOffSpec = 0;
constexpr size_t kOffTw = kOffSpec + dpsr::kNSpec * kSpec;
constexpr size_t kOffTab = kOffTw + al(sizeof(float2) * kMaxR);
constexpr size_t kOffSc = kOffTab + al(sizeof(float) * 7 * kMaxR);
constexpr size_t kOffStatus = kOffSc + al(sizeof(dpsr::Scalars));
constexpr size_t kParts = ((kMaxR / 2 + 1 + 15) / 16) * kMaxR > kMaxR * 8
                              ? ((kMaxR / 2 + 1 + 15) / 16) * kMaxR : kMaxR * 8;
constexpr size_t kOffPart = kOffStatus + al(sizeof(unsigned));
constexpr size_t kOffBins = kOffPart + al(sizeof(float4) * kParts);
constexpr size_t kOffSorted = kOffBins + al(sizeof(int) * dpsr::bins_ints(kMaxR));
constexpr size_t kOffCell = kOffSorted + al(sizeof(float4) * 2 * kMaxN);
constexpr size_t kOffGfwd = kOffCell + al(sizeof(int) * kMaxN);
constexpr size_t kScratchBytes = kOffGfwd + al(sizeof(float4) * 2 * kMaxN);  // ~14 MB

}  // namespace

static __device__ __align__(256) unsigned char g_dpsr_static_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void* g_addr[64] = {};                 // device address of the array, per device ordinal
unsigned long long g_ctx_id[64] = {};  // unique id of the context it was looked up in

// Unique id (never reused within the process) of the device's current
// context, through the driver entry points the runtime hands out; 0 if it
// cannot be read.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = (PFN_cuCtxGetCurrent_v4000)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (PFN_cuCtxGetId_v12000)p;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Look up (once per device and context, with that device current) the device
// address of the static array. The array's name in host code is only a
// stand-in: a kernel given it would fault or, where the GPU can reach host
// memory, silently use the wrong memory.
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return DPSR_EINVAL;
  const unsigned long long id = current_context_id();  // 0: unknown, look up again
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dpsr_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return DPSR_ECUDA;
    }
    g_addr[dev] = p;
    g_ctx_id[dev] = id;
  }
  *out = (unsigned char*)g_addr[dev];
  return DPSR_OK;
}

// Whether work queued on `st` now would be captured: its own capture, or a
// global-mode capture on another stream (which makes the query on the legacy
// stream fail). Either way this entry point must not run.
bool capture_active(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

extern "C" DPSR_API int dpsr_forward_static(int r, float sigma, const float* points,
                                            const float* normals, int64_t N, float* chi_out,
                                            void* stream) {
  if (r < 8 || r > kMaxR || (r & (r - 1)) != 0) return DPSR_EINVAL;
  if (N < 1 || N > kMaxN) return DPSR_EINVAL;
  if (!points || !normals || !chi_out || !(sigma >= 0.f) || !isfinite(sigma)) return DPSR_EINVAL;
  if (((uintptr_t)chi_out & 15) != 0) return DPSR_EINVAL;  // written by bulk and vector stores
  cudaStream_t st = (cudaStream_t)stream;
  if (capture_active(st)) return DPSR_ESTATE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DPSR_ECUDA;
  unsigned char* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != DPSR_OK) return rc;

  // Per-call tables (unit cube): twiddles, Gaussian factor, u^2, derivative u.
  float2 htw[kMaxR];
  float htab[7 * kMaxR];
  dpsr::spectral_tables(r, (double)sigma, nullptr, htw, htab);
  dpsr::Solve s = {};
  dpsr::set_grid(s, r);
  dpsr::set_count(s, N);
  s.points = points;
  s.normals = normals;
  s.chi = chi_out;
  for (int k = 0; k < dpsr::kNSpec; ++k) s.spec[k] = (float2*)(base + kOffSpec + k * kSpec);
  float2* tw = (float2*)(base + kOffTw);
  float* tab = (float*)(base + kOffTab);
  s.tw = tw;
  s.g1 = tab;
  s.u2 = tab + r;
  s.iu = tab + 4 * r;
  s.sc = (dpsr::Scalars*)(base + kOffSc);
  s.status = (unsigned*)(base + kOffStatus);
  s.part = (float4*)(base + kOffPart);
  s.bins = (int*)(base + kOffBins);
  s.sorted = (float4*)(base + kOffSorted);
  s.cellx = (int*)(base + kOffCell);
  s.gfwd = (float4*)(base + kOffGfwd);
  if (dpsr::make_tensor_maps(s, r) != DPSR_OK) return DPSR_ECUDA;

  cudaError_t e = cudaMemcpyAsync(tw, htw, sizeof(float2) * r, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab, htab, sizeof(float) * 7 * r, cudaMemcpyHostToDevice, st);
  // the bin counters and the status word must start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(s.bins, 0, sizeof(int) * dpsr::bins_ints(r), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = dpsr::launch_bin(s, nullptr, 1, (int)N, r, st);
  if (e == cudaSuccess) e = dpsr::launch_plane(0, r, 1, s, nullptr, 1, st);
  if (e == cudaSuccess) e = dpsr::launch_xpass(false, r, s, nullptr, 1, st);
  if (e == cudaSuccess) e = dpsr::launch_plane(1, r, 1, s, nullptr, 1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DPSR_ECUDA;
  }
  unsigned status = 0;
  if (cudaMemcpy(&status, s.status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DPSR_ECUDA;
  return dpsr::status_code(status);
}
