// Point kernels: bucketing of the points by the x-cell of their trilinear
// stencil (a counting sort, so that each x-plane cluster reads only the points
// that touch its plane), and the final combine of the backward pass.
#include <algorithm>

#include "dpsr_dev.cuh"
#include "finalize.cuh"
#include "launch.h"
#include "tma.cuh"

namespace dpsr {

__device__ __forceinline__ bool coord_ok(float c, int r) {
  return isfinite(c) && fabsf(c * (float)r) < 1073741824.f;  // |c r| < 2^30
}

// Bin key of a point from its x and y cells (see nbins).
__device__ __forceinline__ int bin_key(int ix, int iy, int r) { return ix * nybins(r) + iy / ybin(r); }

// count[key]++ per point (see nbins for the key); validates the inputs
// (non-finite or huge values raise kStBadInput and are replaced by 0 so that
// indexing stays in range). Per-block histogram in shared memory, then one
// global add per touched bin. The counts must be zero on entry: the forward
// x-pass clears them (and the scatter cursors) once the scatter is done.
// Dynamic shared memory: the histogram, nbins(r) ints.
__global__ void __launch_bounds__(256) k_bin_count(const __grid_constant__ Solve s0,
                                                   const Solve* __restrict__ tab) {
  extern __shared__ int h[];
  pdl_trigger();
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int r = S.r, nb = nbins(r);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
  pdl_wait();
  __syncthreads();
  bool bad = false;
  // r / L_d per axis (FP64 cell arithmetic only off the unit cube)
  const double sx = S.gscale[0], sy = S.gscale[1];
  const bool unit[2] = {S.box[0] == 1.0, S.box[1] == 1.0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S.N; p += gridDim.x * blockDim.x) {
    // box coordinates; the check uses their unit-cube size
    float x = S.points[3 * p], y = S.points[3 * p + 1];
    const float z = S.points[3 * p + 2];
    const float nx = S.normals[3 * p], ny = S.normals[3 * p + 1], nz = S.normals[3 * p + 2];
    const bool okx = coord_ok(x * S.inv_box[0], r), oky = coord_ok(y * S.inv_box[1], r);
    if (!(okx && oky && coord_ok(z * S.inv_box[2], r) && isfinite(nx) && isfinite(ny) && isfinite(nz))) {
      bad = true;
      if (!okx) x = 0.f;
      if (!oky) y = 0.f;
    }
    const int key = bin_key(axis_in_box(x, sx, unit[0], r).i0, axis_in_box(y, sy, unit[1], r).i0, r);
    S.cellx[p] = key;
    if (!dbg_in_range(S.status, key, nb)) continue;
    atomicAdd(&h[key], 1);
  }
  if (bad) atomicOr(S.status, kStBadInput);
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (h[i]) atomicAdd(&S.bins[i], h[i]);
}

// Shared-memory slot of bin i in the scatter's scan: one pad word per 32
// bins, so that threads scanning 16 consecutive bins each hit distinct banks.
__host__ __device__ constexpr int scan_slot(int i) { return i + (i >> 5); }

// Counting-sort scatter. Every block first turns the (L2-resident) bin counts
// into exclusive prefix sums in its own shared memory: each thread sums a
// run of consecutive bins, a block scan offsets the runs. No block waits for
// another, so there is no serial last-block step. Block 0 also publishes the
// offsets off[0..nbins] (read by the plane passes) and resets the arrival
// counters of the solve's last-block reductions. A point's slot is its bin's
// offset plus a ticket from that bin's cursor (zero on entry; cleared again
// by the forward x-pass). Dynamic shared memory: scan_slot(nbins(r)) ints.
__global__ void __launch_bounds__(256) k_bin_scatter(const __grid_constant__ Solve s0,
                                                     const Solve* __restrict__ tab) {
  constexpr int NT = 256;
  extern __shared__ int h[];
  __shared__ int wsum[NT / 32];
  pdl_trigger();
  pdl_wait();
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int r = S.r, nb = nbins(r), tid = threadIdx.x;
  int* off = S.bins + nb;
  int* cur = off + nb + 1;
  for (int i = tid; i < nb; i += NT) h[scan_slot(i)] = __ldcg(S.bins + i);
  __syncthreads();
  const int C = (nb + NT - 1) / NT;  // consecutive bins per thread
  const int b0 = tid * C;
  int run = 0;
  for (int j = 0; j < C; ++j)
    if (b0 + j < nb) run += h[scan_slot(b0 + j)];
  // block-wide exclusive scan of the runs: lanes, then warps in order
  const int lane = tid & 31, w = tid >> 5;
  int incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int wbase = 0, total = 0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) {
    wbase += k < w ? wsum[k] : 0;
    total += wsum[k];
  }
  int acc = wbase + incl - run;
  for (int j = 0; j < C; ++j) {
    if (b0 + j < nb) {
      const int c = h[scan_slot(b0 + j)];
      h[scan_slot(b0 + j)] = acc;
      acc += c;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int i = tid; i < nb; i += NT) off[i] = h[scan_slot(i)];
    if (tid == 0) {
      off[nb] = total;
      S.sc->ticket[0] = 0;
      S.sc->ticket[1] = 0;
      S.sc->ticket[2] = 0;
    }
  }
  const double sx = S.gscale[0], sy = S.gscale[1], sz = S.gscale[2];
  const bool unit[3] = {S.box[0] == 1.0, S.box[1] == 1.0, S.box[2] == 1.0};
  for (int p = blockIdx.x * NT + tid; p < S.N; p += gridDim.x * NT) {
    // box coordinates; the records hold each point's cells and in-cell
    // fractions (the same FP64 arithmetic as the count's key)
    float x = S.points[3 * p], y = S.points[3 * p + 1], z = S.points[3 * p + 2];
    float nx = S.normals[3 * p], ny = S.normals[3 * p + 1], nz = S.normals[3 * p + 2];
    if (!coord_ok(x * S.inv_box[0], r)) x = 0.f;
    if (!coord_ok(y * S.inv_box[1], r)) y = 0.f;
    if (!coord_ok(z * S.inv_box[2], r)) z = 0.f;
    if (!isfinite(nx)) nx = 0.f;
    if (!isfinite(ny)) ny = 0.f;
    if (!isfinite(nz)) nz = 0.f;
    const int key = S.cellx[p];  // key of k_bin_count
    if (!dbg_in_range(S.status, key, nb)) continue;
    const int pos = h[scan_slot(key)] + atomicAdd(&cur[key], 1);
    if (!dbg_in_range(S.status, pos, S.N)) continue;
    const Axis ax = axis_in_box(x, sx, unit[0], r), ay = axis_in_box(y, sy, unit[1], r),
               az = axis_in_box(z, sz, unit[2], r);
    S.sorted[2 * pos] = make_float4(ax.t, ay.t, az.t, nx);
    S.sorted[2 * pos + 1] = make_float4(ny, nz, __int_as_float(p), __uint_as_float(pack_cells(ax.i0, ay.i0, az.i0)));
  }
}

cudaError_t launch_bin(const Solve& s, const Solve* tab, int count, int nmax, int r, cudaStream_t st) {
  const int blocks = min(max((nmax + 255) / 256, 1), 1184);
  const size_t hc = sizeof(int) * nbins(r), hs = sizeof(int) * scan_slot(nbins(r));
  static bool attr_set = false;  // 16384 bins at r = 512 need more than the default 48 KB
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(int) * nbins(512)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(int) * scan_slot(nbins(512))));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = launch_k(k_bin_count, dim3(blocks, 1, count), dim3(256), hc, st, 0, s, tab);
  if (e == cudaSuccess) e = launch_k(k_bin_scatter, dim3(blocks, 1, count), dim3(256), hs, st, 0, s, tab);
  return e;
}

// dpoints = (sum of the two plane sides of the weight-derivative terms
//            + (mu_bar / (N n)) * gradient of the lookup of y (Eq. 4 adjoint)) / L_d;
// dnormals = sum of the two plane sides of the gather. Written in the
// caller's point order. SPLIT: the adjoint kind left [side][channel][point]
// float4 slots (gather, three derivative terms), summed over the channels in
// the order the one-CTA adjoint accumulates them; else [side][point][6].
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_combine(const __grid_constant__ Solve s0,
                                                 const Solve* __restrict__ tab) {
  pdl_trigger();
  pdl_wait();
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const float c_mu = S.sc->c_mu;
  const size_t N = S.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.N; i += gridDim.x * blockDim.x) {
    const int orig = __float_as_int(S.sorted[2 * i + 1].z);
    if (!dbg_in_range(S.status, orig, S.N)) continue;
    float a[6], b[6];
    if constexpr (SPLIT) {
      const float4* q = reinterpret_cast<const float4*>(S.slots);
      float4 u[3], w[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        u[ch] = q[(size_t)ch * N + i];
        w[ch] = q[(size_t)(3 + ch) * N + i];
      }
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        a[ch] = u[ch].x;
        b[ch] = w[ch].x;
      }
      a[3] = (u[0].y + u[1].y) + u[2].y;
      a[4] = (u[0].z + u[1].z) + u[2].z;
      a[5] = (u[0].w + u[1].w) + u[2].w;
      b[3] = (w[0].y + w[1].y) + w[2].y;
      b[4] = (w[0].z + w[1].z) + w[2].z;
      b[5] = (w[0].w + w[1].w) + w[2].w;
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        a[k] = S.slots[(size_t)i * 6 + k];
        b[k] = S.slots[(N + i) * 6 + k];
      }
    }
    const float4 ga = S.gfwd[i], gb = S.gfwd[N + i];
    S.dnormals[3 * orig] = a[0] + b[0];
    S.dnormals[3 * orig + 1] = a[1] + b[1];
    S.dnormals[3 * orig + 2] = a[2] + b[2];
    // derivatives in unit-cube coordinates, times dx_d / dc_d = 1 / L_d
    S.dpoints[3 * orig] = ((a[3] + b[3]) + c_mu * (ga.x + gb.x)) * S.inv_box[0];
    S.dpoints[3 * orig + 1] = ((a[4] + b[4]) + c_mu * (ga.y + gb.y)) * S.inv_box[1];
    S.dpoints[3 * orig + 2] = ((a[5] + b[5]) + c_mu * (ga.z + gb.z)) * S.inv_box[2];
  }
}

cudaError_t launch_combine(const Solve& s, const Solve* tab, int count, int nmax, bool split,
                           cudaStream_t st) {
  const int blocks = min(max((nmax + 255) / 256, 1), 1184);
  return split ? launch_k(k_combine<true>, dim3(blocks, 1, count), dim3(256), 0, st, 0, s, tab)
               : launch_k(k_combine<false>, dim3(blocks, 1, count), dim3(256), 0, st, 0, s, tab);
}

// ---------------------------------------------------------------------------
// Trilinear lookup of a grid at query points and its adjoint (the same
// periodic stencil as the rasterization of Eq. A1): used by losses defined on
// chi at target points, e.g. mean_k chi(q_k)^2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_grid_sample(const float* __restrict__ grid, int r,
                                                     const float* __restrict__ q, int64_t M,
                                                     float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Axis ax = axis_of(q[3 * i], r), ay = axis_of(q[3 * i + 1], r), az = axis_of(q[3 * i + 2], r);
    float acc = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int dx = d >> 2, dy = (d >> 1) & 1, dz = d & 1;
      const float w = (dx ? ax.t : 1.f - ax.t) * (dy ? ay.t : 1.f - ay.t) * (dz ? az.t : 1.f - az.t);
      const size_t j = ((size_t)(dx ? ax.i1 : ax.i0) * r + (dy ? ay.i1 : ay.i0)) * r + (dz ? az.i1 : az.i0);
      acc += w * grid[j];
    }
    out[i] = acc;
  }
}

__global__ void __launch_bounds__(256) k_grid_splat(float* __restrict__ grid, int r,
                                                    const float* __restrict__ q,
                                                    const float* __restrict__ vals, int64_t M) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Axis ax = axis_of(q[3 * i], r), ay = axis_of(q[3 * i + 1], r), az = axis_of(q[3 * i + 2], r);
    const float v = vals[i];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int dx = d >> 2, dy = (d >> 1) & 1, dz = d & 1;
      const float w = (dx ? ax.t : 1.f - ax.t) * (dy ? ay.t : 1.f - ay.t) * (dz ? az.t : 1.f - az.t);
      const size_t j = ((size_t)(dx ? ax.i1 : ax.i0) * r + (dy ? ay.i1 : ay.i0)) * r + (dz ? az.i1 : az.i0);
      atomicAdd(&grid[j], w * v);
    }
  }
}

// ---------------------------------------------------------------------------
// L_DPSR of Eq. 9, the training loss of the learning setting (Sec. 3.3): the
// mean squared error between the solved indicator grid chi and a target grid
// (the solve of a dense ground-truth sampling), and its gradient, in one pass:
//   loss = (1/n) sum_j (chi_j - target_j)^2,   dchi_j = (2/n) (chi_j - target_j).
// Per-thread FP32 sums, float-float block and grid sums (the last block to
// arrive writes sc->loss), deterministic. n = r^3 is a power of two, so 2/n
// and 1/n are exact.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mse_grad(const __grid_constant__ Solve s0,
                                                  const Solve* __restrict__ tab) {
  constexpr int NT = 256;
  pdl_trigger();
  pdl_wait();
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int64_t n4 = (int64_t)S.r * S.r * S.r / 4;
  const float two_n = 2.f / ((float)S.r * (float)S.r * (float)S.r);
  const float4* chi = reinterpret_cast<const float4*>(S.chi);
  const float4* tg = reinterpret_cast<const float4*>(S.target);
  float4* g = reinterpret_cast<float4*>(S.dchi_rw);
  // this instance's blocks (a batch launch sizes the grid for its largest r)
  const int nblk = (int)min((int64_t)gridDim.x, max(n4 / (2 * NT), (int64_t)1));
  if ((int)blockIdx.x >= nblk) return;
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n4; i += (int64_t)nblk * NT) {
    const float4 a = __ldcs(chi + i), b = __ldcs(tg + i);
    const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    __stcs(g + i, make_float4(two_n * d.x, two_n * d.y, two_n * d.z, two_n * d.w));
    acc += (d.x * d.x + d.y * d.y) + (d.z * d.z + d.w * d.w);
  }
  FF a = {acc, 0.f}, z = {0.f, 0.f};
  block_sum_ff<NT>(a, z);
  __shared__ unsigned last;
  if (threadIdx.x == 0) {
    S.part[blockIdx.x] = make_float4(a.hi, a.lo, 0.f, 0.f);
    __threadfence();
    last = atomicAdd(&S.sc->ticket[2], 1u) == (unsigned)nblk - 1u ? 1u : 0u;
    if (last) __threadfence();
  }
  __syncthreads();
  if (!last) return;
  FF x = {0.f, 0.f}, y = {0.f, 0.f};
  for (int i = threadIdx.x; i < nblk; i += NT) {
    const float4 p = __ldcg(S.part + i);
    x = ff_add(x, FF{p.x, p.y});
  }
  block_sum_ff<NT>(x, y);
  if (threadIdx.x == 0) {
    S.sc->loss = ff_to_double(x) / ((double)S.r * S.r * S.r);
    S.sc->ticket[2] = 0;
  }
}

// Blocks of the loss pass for grid size r: two float4 per thread, at most
// the r * 16 block partials the workspace holds.
int mse_blocks(int r) {
  const int64_t n4 = (int64_t)r * r * r / 4;
  const int64_t b = n4 / (2 * 256);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)r * 16));
}

cudaError_t launch_mse_grad(const Solve& s, const Solve* tab, int count, int r, cudaStream_t st) {
  return launch_k(k_mse_grad, dim3(mse_blocks(r), 1, count), dim3(256), 0, st, 0, s, tab);
}

// A bounded wait on a barrier that nothing completes (see
// dpsr_check_bounded_wait): it must give up after limit_ns and say so.
__global__ void k_wait_probe(unsigned* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = __syncthreads_and(mbar_wait(&bar, 0, limit_ns));
  if (!ok && threadIdx.x == 0) atomicOr(status, kStTimeout);
}

cudaError_t launch_wait_probe(unsigned* status, double limit_s, cudaStream_t st) {
  k_wait_probe<<<1, 64, 0, st>>>(status, (unsigned long long)(limit_s * 1e9));
  return cudaGetLastError();
}

cudaError_t launch_grid_sample(const float* grid, int r, const float* q, int64_t M, float* out,
                               cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((M + 255) / 256, 4736);
  k_grid_sample<<<std::max(blocks, 1), 256, 0, st>>>(grid, r, q, M, out);
  return cudaGetLastError();
}

cudaError_t launch_grid_splat(float* grid, int r, const float* q, const float* vals, int64_t M,
                              cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((M + 255) / 256, 4736);
  k_grid_splat<<<std::max(blocks, 1), 256, 0, st>>>(grid, r, q, vals, M);
  return cudaGetLastError();
}

}  // namespace dpsr
