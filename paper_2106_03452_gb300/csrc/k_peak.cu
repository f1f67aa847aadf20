// FP32 FMA throughput of this GPU, measured: the ceiling of the group FFT's
// butterflies, which run on the FP32 pipe next to the shared-memory exchange.
// Every thread runs 8 independent dependent-FMA chains (enough in flight to
// cover the pipe latency at full occupancy) for `iters` steps; the grid is
// 8 CTAs of 256 threads per SM. The inputs come from the caller so that no
// chain folds to a constant, and the results feed one guarded store so that
// none is dropped.
#include <cuda_runtime.h>

#include "dpsr.h"

namespace {

__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (float)threadIdx.x * 1e-7f + (float)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == -1.f) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" DPSR_API int dpsr_fp32_fma_peak(int iters, double* flops_per_s) {
  if (!flops_per_s || iters < 1) return DPSR_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DPSR_ECUDA;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DPSR_ECUDA;
  const int blocks = sms * 8, threads = 256;
  if (cudaMalloc(&out, sizeof(float) * blocks) == cudaSuccess &&
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    k_fma_peak<<<blocks, threads, 0, st>>>(out, iters < 64 ? iters : 64, 0.9999f, 1e-6f);  // warm-up
    float best = 1e30f;
    bool ok = cudaGetLastError() == cudaSuccess;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      float ms = 0.f;
      ok = cudaEventRecord(e0, st) == cudaSuccess;
      k_fma_peak<<<blocks, threads, 0, st>>>(out, iters, 0.9999f, 1e-6f);
      ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
           cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (ok && ms < best) best = ms;
    }
    if (ok && best > 0.f) {
      const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
      *flops_per_s = flops / (best * 1e-3);
      rc = DPSR_OK;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return rc;
}

// ---------------------------------------------------------------------------
// Debug-build check of the index checks themselves: one access whose index
// (40) lies outside its logical range [0, 32) but inside its 64-float
// allocation, so that a build without the checks writes harmlessly and a
// build with them skips the write and raises the status bit.
// ---------------------------------------------------------------------------
#include "dpsr_dev.cuh"

namespace {

__global__ void k_dbg_selftest(float* buf, unsigned* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int i = 40;
    if (dpsr::dbg_in_range(status, i, 32)) buf[i] = 1.f;
  }
}

}  // namespace

namespace dpsr {
int status_code(unsigned st);
}

extern "C" DPSR_API int dpsr_debug_checks(void) {
#ifdef DPSR_DEBUG_CHECKS
  return 1;
#else
  return 0;
#endif
}

extern "C" DPSR_API int dpsr_debug_check_selftest(void) {
  float* buf = nullptr;
  unsigned* st = nullptr;
  int rc = DPSR_ECUDA;
  if (cudaMalloc(&buf, sizeof(float) * 64) == cudaSuccess && cudaMalloc(&st, sizeof(unsigned)) == cudaSuccess &&
      cudaMemset(st, 0, sizeof(unsigned)) == cudaSuccess) {
    k_dbg_selftest<<<1, 32>>>(buf, st);
    unsigned h = 0;
    if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(&h, st, sizeof(unsigned), cudaMemcpyDeviceToHost) == cudaSuccess)
      rc = dpsr::status_code(h);
  }
  cudaGetLastError();
  if (buf) cudaFree(buf);
  if (st) cudaFree(st);
  return rc;
}
