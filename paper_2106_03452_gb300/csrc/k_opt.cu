// Kernels of the optimisation setting (Sec. 3.2; supplementary Sec. B)
// around the DPSR layer: the bi-directional L2 Chamfer distance between
// points sampled on the mesh and the input cloud (with its gradient with
// respect to the mesh points), the largest component of the mesh for the
// resampling step, and area-weighted sampling of points on the mesh.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "dpsr.h"
#include "dpsr_dev.cuh"
#include "finalize.cuh"
#include "launch.h"

namespace dpsr {

// ---------------------------------------------------------------------------
// Nearest neighbour by brute force: for every query q_i, the index of the
// closest target (ties: the lowest index) and the squared distance. Targets
// pass through shared memory in tiles of 1024.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_nearest(const float* __restrict__ q, int64_t nq,
                                                 const float* __restrict__ t, int64_t nt,
                                                 int* __restrict__ idx, float* __restrict__ d2) {
  constexpr int TILE = 1024;
  __shared__ float4 sh[TILE];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float qx = 0.f, qy = 0.f, qz = 0.f;
  if (i < nq) {
    qx = q[3 * i];
    qy = q[3 * i + 1];
    qz = q[3 * i + 2];
  }
  float best = INFINITY;
  int bi = -1;
  for (int64_t base = 0; base < nt; base += TILE) {
    const int n = (int)std::min<int64_t>(TILE, nt - base);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int64_t j = base + k;
      sh[k] = make_float4(t[3 * j], t[3 * j + 1], t[3 * j + 2], 0.f);
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const float4 p = sh[k];
      const float dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
      const float d = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d < best) {
        best = d;
        bi = (int)(base + k);
      }
    }
  }
  if (i < nq) {
    idx[i] = bi;
    d2[i] = best;
  }
}

// dL/da for L = mean_a min_b |a-b|^2 + mean_b min_a |a-b|^2 with respect to
// the points a (the second term scatters: each b pulls its nearest a).
__global__ void __launch_bounds__(256) k_chamfer_grad(const float* __restrict__ a, int64_t na,
                                                      const float* __restrict__ b, int64_t nb,
                                                      const int* __restrict__ ab, const int* __restrict__ ba,
                                                      float* __restrict__ ga) {
  const float ca = 2.f / (float)na, cb = 2.f / (float)nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < na + nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < na) {
      const int j = ab[i];
#pragma unroll
      for (int d = 0; d < 3; ++d) atomicAdd(&ga[3 * i + d], ca * (a[3 * i + d] - b[3 * (int64_t)j + d]));
    } else {
      const int64_t k = i - na;
      const int j = ba[k];
#pragma unroll
      for (int d = 0; d < 3; ++d) atomicAdd(&ga[3 * (int64_t)j + d], cb * (a[3 * (int64_t)j + d] - b[3 * k + d]));
    }
  }
}

// Sum of n values in float-float, in one block (a small reduction per call).
__global__ void __launch_bounds__(256) k_sum2(const float* __restrict__ x, int64_t nx, const float* __restrict__ y,
                                              int64_t ny, double* __restrict__ out) {
  FF sx = {0.f, 0.f}, sy = {0.f, 0.f};
  for (int64_t i = threadIdx.x; i < nx; i += blockDim.x) sx = ff_add(sx, x[i]);
  for (int64_t i = threadIdx.x; i < ny; i += blockDim.x) sy = ff_add(sy, y[i]);
  block_sum_ff<256>(sx, sy);
  if (threadIdx.x == 0) *out = ff_to_double(sx) / (double)nx + ff_to_double(sy) / (double)ny;
}

// ---------------------------------------------------------------------------
// Components of the inside region {chi < level} of the periodic grid, with
// voxels joined along the edge directions of the mesh's tetrahedra (x, y, z,
// x+y, x+z, y+z, x+y+z), so that the negative corners of a tetrahedron are
// always in one component and every mesh triangle belongs to exactly one.
// Lock-free union-find: parent[v] = v for inside voxels, -1 outside; a union
// hangs the larger root under the smaller one with compare-and-swap. Every
// loop is bounded (a count far above any path length); running out sets
// *err.
// ---------------------------------------------------------------------------
constexpr int kFindLimit = 1 << 22;

// Parents are read at L2 (another SM may have just changed them through an
// atomic; a stale L1 copy would only make the CAS below fail again).
__device__ __forceinline__ int uf_find(int* parent, int v, unsigned* err) {
  for (int it = 0; it < kFindLimit; ++it) {
    const int p = __ldcg(parent + v);
    if (p == v) return v;
    const int gp = __ldcg(parent + p);
    if (gp != p) atomicCAS(&parent[v], p, gp);  // path halving
    v = gp;
  }
  atomicOr(err, 1u);
  return v;
}

__global__ void k_cc_init(const float* __restrict__ chi, int64_t n, float level, int* __restrict__ parent) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    parent[v] = chi[v] < level ? (int)v : -1;
}

__global__ void k_cc_union(int r, int* __restrict__ parent, unsigned* __restrict__ err) {
  const int64_t n = (int64_t)r * r * r;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (__ldcg(parent + v) < 0) continue;
    const int i = (int)(v / ((int64_t)r * r)), j = (int)((v / r) % r), k = (int)(v % r);
#pragma unroll
    for (int d = 1; d < 8; ++d) {  // the seven monotone offsets (dx, dy, dz) in {0,1}^3 \ 0
      const int64_t w = ((int64_t)((i + (d & 1)) & (r - 1)) * r + ((j + ((d >> 1) & 1)) & (r - 1))) * r +
                        ((k + ((d >> 2) & 1)) & (r - 1));
      if (__ldcg(parent + w) < 0) continue;
      int a = (int)v, b = (int)w;
      for (int it = 0; it < kFindLimit; ++it) {
        a = uf_find(parent, a, err);
        b = uf_find(parent, b, err);
        if (a == b) break;
        if (a < b) {
          const int s = a;
          a = b;
          b = s;
        }
        if (atomicCAS(&parent[a], a, b) == a) break;
        if (it == kFindLimit - 1) atomicOr(err, 1u);
      }
    }
  }
}

// Flatten to roots and count voxels per root.
__global__ void k_cc_flatten(int64_t n, int* __restrict__ parent, int* __restrict__ size, unsigned* __restrict__ err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (__ldcg(parent + v) < 0) continue;
    const int root = uf_find(parent, (int)v, err);
    atomicAdd(&size[root], 1);
  }
}
__global__ void k_cc_relabel(int64_t n, int* __restrict__ parent, unsigned* __restrict__ err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (__ldcg(parent + v) >= 0) parent[v] = uf_find(parent, (int)v, err);
}

// The root with the most voxels (ties: the lowest root), as
// (size << 32) | (0xffffffff - root) maxima.
__global__ void k_cc_largest(int64_t n, const int* __restrict__ size, unsigned long long* __restrict__ best) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int s = size[v];
    if (s > 0) atomicMax(best, ((unsigned long long)s << 32) | (0xffffffffull - (unsigned long long)v));
  }
}

// ---------------------------------------------------------------------------
// Area-weighted sampling of points on a triangle soup: areas, their prefix
// sums (per block, then the block totals by one block, then the offsets), a
// counter-based uniform per sample (a 64-bit integer hash of seed and index,
// SplitMix64's finaliser), a binary search, and uniform barycentric
// coordinates (the reflection of the unit square onto the triangle).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t seed, uint64_t i) {
  return (double)(mix64(seed + 0x9e3779b97f4a7c15ull * (i + 1)) >> 11) * (1.0 / 9007199254740992.0);
}

constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(kScanBlock) k_area_scan(const float* __restrict__ tris, int64_t T,
                                                          double* __restrict__ cum, double* __restrict__ block_tot) {
  __shared__ double s[kScanBlock];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  double a = 0.0;
  if (i < T) {
    const float* t = tris + 9 * i;
    const double ux = t[3] - t[0], uy = t[4] - t[1], uz = t[5] - t[2];
    const double vx = t[6] - t[0], vy = t[7] - t[1], vz = t[8] - t[2];
    const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
    a = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int d = 1; d < kScanBlock; d <<= 1) {  // inclusive Hillis-Steele scan
    const double x = threadIdx.x >= d ? s[threadIdx.x - d] : 0.0;
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  if (i < T) cum[i] = s[threadIdx.x];
  if (threadIdx.x == kScanBlock - 1) block_tot[blockIdx.x] = s[threadIdx.x];
}

// One block: exclusive prefix of the block totals (serial per thread chunk).
__global__ void __launch_bounds__(256) k_block_offsets(double* __restrict__ tot, int nblocks) {
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      const double v = tot[b];
      tot[b] = acc;
      acc += v;
    }
    tot[nblocks] = acc;
  }
}

__global__ void k_add_offsets(double* __restrict__ cum, int64_t T, const double* __restrict__ off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x)
    cum[i] += off[i / kScanBlock];
}

__global__ void __launch_bounds__(256) k_sample(const float* __restrict__ tris, const float* __restrict__ nrm,
                                                int64_t T, const double* __restrict__ cum,
                                                const double* __restrict__ total, int64_t M, uint64_t seed,
                                                float* __restrict__ p, float* __restrict__ n) {
  const double A = *total;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < M; s += (int64_t)gridDim.x * blockDim.x) {
    const double x = u01(seed, 3 * s) * A;
    int64_t lo = 0, hi = T - 1;  // first triangle whose cumulative area exceeds x
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cum[mid] > x) hi = mid;
      else lo = mid + 1;
    }
    double u = u01(seed, 3 * s + 1), v = u01(seed, 3 * s + 2);
    if (u + v > 1.0) {
      u = 1.0 - u;
      v = 1.0 - v;
    }
    const float* t = tris + 9 * lo;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      p[3 * s + d] = (float)(t[d] + u * (t[3 + d] - t[d]) + v * (t[6 + d] - t[d]));
      n[3 * s + d] = nrm[3 * lo + d];
    }
  }
}

}  // namespace dpsr

extern "C" {

int dpsr_chamfer(const float* a, int64_t na, const float* b, int64_t nb, int* ws_idx, float* ws_d2, float* grad_a,
                 double* loss, void* stream) {
  if (!a || !b || !ws_idx || !ws_d2 || !grad_a || !loss || na < 1 || nb < 1 || na > INT32_MAX || nb > INT32_MAX)
    return DPSR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int* ab = ws_idx;
  int* ba = ws_idx + na;
  float* dab = ws_d2;
  float* dba = ws_d2 + na;
  if (cudaMemsetAsync(grad_a, 0, sizeof(float) * 3 * na, st) != cudaSuccess) return DPSR_ECUDA;
  dpsr::k_nearest<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(a, na, b, nb, ab, dab);
  dpsr::k_nearest<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(b, nb, a, na, ba, dba);
  const int blocks = (int)std::min<int64_t>((na + nb + 255) / 256, 4736);
  dpsr::k_chamfer_grad<<<blocks, 256, 0, st>>>(a, na, b, nb, ab, ba, grad_a);
  dpsr::k_sum2<<<1, 256, 0, st>>>(dab, na, dba, nb, loss);
  return cudaGetLastError() == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

int dpsr_largest_region(const float* chi, int r, float level, int* labels, int* ws, unsigned long long* best,
                        unsigned* err, void* stream) {
  if (!chi || !labels || !ws || !best || !err || r < 2 || r > 512 || (r & (r - 1))) return DPSR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = (int64_t)r * r * r;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
  if (cudaMemsetAsync(ws, 0, sizeof(int) * n, st) != cudaSuccess ||
      cudaMemsetAsync(best, 0, sizeof(unsigned long long), st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess)
    return DPSR_ECUDA;
  dpsr::k_cc_init<<<blocks, 256, 0, st>>>(chi, n, level, labels);
  dpsr::k_cc_union<<<blocks, 256, 0, st>>>(r, labels, err);
  dpsr::k_cc_flatten<<<blocks, 256, 0, st>>>(n, labels, ws, err);
  dpsr::k_cc_relabel<<<blocks, 256, 0, st>>>(n, labels, err);
  dpsr::k_cc_largest<<<blocks, 256, 0, st>>>(n, ws, best);
  return cudaGetLastError() == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

int dpsr_mesh_sample(const float* tris, const float* normals, int64_t T, int64_t M, uint64_t seed, double* ws,
                     float* points, float* pnormals, void* stream) {
  if (!tris || !normals || !ws || !points || !pnormals || T < 1 || M < 0) return DPSR_EINVAL;
  if (M == 0) return DPSR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int nblk = (int)((T + dpsr::kScanBlock - 1) / dpsr::kScanBlock);
  double* cum = ws;
  double* tot = ws + T;  // nblk + 1 entries
  dpsr::k_area_scan<<<nblk, dpsr::kScanBlock, 0, st>>>(tris, T, cum, tot);
  dpsr::k_block_offsets<<<1, 256, 0, st>>>(tot, nblk);
  dpsr::k_add_offsets<<<(unsigned)std::min<int64_t>((T + 255) / 256, 4736), 256, 0, st>>>(cum, T, tot);
  dpsr::k_sample<<<(unsigned)std::min<int64_t>((M + 255) / 256, 4736), 256, 0, st>>>(
      tris, normals, T, cum, tot + nblk, M, seed, points, pnormals);
  return cudaGetLastError() == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

}  // extern "C"
