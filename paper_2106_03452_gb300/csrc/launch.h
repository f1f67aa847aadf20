// Internal launchers of libdpsr (host side). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "dpsr_dev.cuh"

namespace dpsr {

// Whether solve kernels are launched with programmatic stream serialization
// (on unless the environment sets DPSR_PDL=0, or the calling thread has
// suspended it: per-kernel event timing wants each kernel to start after the
// previous one has completed).
bool pdl_enabled();
void pdl_suspend(bool off);

// cudaLaunchKernelEx with an optional cluster size (x) and the programmatic
// launch attribute.
template <class... KArgs, class... Args>
cudaError_t launch_k(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     int cluster, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int n = 0;
  if (cluster > 0) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = cluster;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  if (pdl_enabled()) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  cfg.attrs = attr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

// Plane kernels: kind 0 = forward splat/z/y, 1 = forward inverse y/z + lookup
// gradient, 2 = backward z/y of dchi, 3 = backward inverse y/z + point adjoint.
cudaError_t launch_plane(int kind, int r, int C, const Solve& s, const Solve* tab, int count,
                         cudaStream_t st);
size_t plane_smem_bytes(int kind, int r, int C);
// The same four kinds as z and y passes of independent CTAs (two launches
// each; "cluster size 0" to the tuner).
cudaError_t launch_pencil(int kind, int r, const Solve& s, const Solve* tab, int count,
                          cudaStream_t st);
size_t pencil_smem_bytes(int kind, int r);
// Persistent CTAs: the number of CTAs that fit the GPU at once (at most
// `tiles`), for a kernel that loops over tiles with a stride of gridDim.x.
template <class K>
inline int persistent_ctas(K fn, int nthreads, size_t smem, int tiles, int count) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nthreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return tiles;
  }
  const int n = (sms * (occ > 0 ? occ : 1)) / (count > 0 ? count : 1);
  return n < 1 ? 1 : (n < tiles ? n : tiles);
}

// Plane path codes: 0 the two pencil passes, 1/2/4/8 the cluster size of the
// plane kernels, kPathSplit the adjoint kind as one CTA per plane and
// channel (k_plane_binv_ch; r = 64 and 128).
constexpr int kPathSplit = 3;
inline bool valid_path(int C) { return C == 0 || C == 1 || C == 2 || C == kPathSplit || C == 4 || C == 8; }
// Kernel launches of one plane kind with path C (0: two pencil passes).
inline int plane_launches(int C) { return C == 0 ? 2 : 1; }
cudaError_t launch_xpass(bool bwd, int r, const Solve& s, const Solve* tab, int count,
                         cudaStream_t st);
int xpass_blocks(int r);

// TMA descriptors of the four spectral buffers of `s` (s.spec must be set).
// Returns 0 on success.
int make_tensor_maps(Solve& s, int r);
// Points: x-plane bucketing (count, scan, scatter) and the backward combine.
cudaError_t launch_bin(const Solve& s, const Solve* tab, int count, int nmax, int r, cudaStream_t st);
// split: the adjoint kind ran on path kPathSplit (per-channel slots).
cudaError_t launch_combine(const Solve& s, const Solve* tab, int count, int nmax, bool split,
                           cudaStream_t st);

// Trilinear lookup of a grid at query points and its adjoint (atomic adds).
cudaError_t launch_grid_sample(const float* grid, int r, const float* q, int64_t M, float* out,
                               cudaStream_t st);
cudaError_t launch_grid_splat(float* grid, int r, const float* q, const float* vals, int64_t M,
                              cudaStream_t st);
// L_DPSR (Eq. 9) against S.target: loss into S.sc->loss, gradient into
// S.dchi_rw. r: the grid size of every instance of the launch.
cudaError_t launch_mse_grad(const Solve& s, const Solve* tab, int count, int r, cudaStream_t st);
// Public status of a device status word: DPSR_ETIMEOUT when a bounded wait
// gave up (ahead of everything else), DPSR_EDEGENERATE for any other bit.
int status_code(unsigned st);
// One CTA waiting (bounded) on a barrier that nothing completes.
cudaError_t launch_wait_probe(unsigned* status, double limit_s, cudaStream_t st);

}  // namespace dpsr
