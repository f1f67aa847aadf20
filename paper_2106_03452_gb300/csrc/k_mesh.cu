// Mesh extraction on the indicator grid and the surrogate gradient through
// it: the optimisation setting of Sec. 3.2 turns chi into a mesh at level 0
// and back-propagates a loss on points of that mesh through the inverse
// surface normal (Eq. 6: d p_mesh / d chi = -n_mesh).
//
// Extraction: a marching-cubes variant without case tables. Each cube of the
// periodic grid is split into Kuhn's six tetrahedra (the monotone paths from
// corner (0,0,0) to (1,1,1) along the three axes in every order); the level
// set is linear inside each tetrahedron: one triangle where one corner's sign
// differs from the other three, two (a quad) where two and two differ. The
// split puts on every face of a cube the diagonal from its lowest to its
// highest corner, the same diagonal the neighbouring cube puts there, and a
// vertex on an edge is computed from the edge's lower endpoint in both cubes,
// so neighbouring cubes produce bit-identical shared vertices: the surface is
// closed (watertight) wherever it stays away from the wrap-around of the
// periodic domain. Output: a triangle soup in unit-cube coordinates
// (unwrapped: a cube at index r - 1 reaches 1.0), each triangle with its unit
// normal pointing towards increasing chi (outwards for outward point
// normals, reading 8), its corners wound counter-clockwise about it.
#include <math.h>

#include <algorithm>

#include "dpsr.h"
#include "dpsr_dev.cuh"
#include "launch.h"

namespace dpsr {

// Corner c of a cube (bits x, y, z) and the six Kuhn tetrahedra as corner ids.
__device__ __constant__ unsigned char kTet[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                                    {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

__device__ __forceinline__ int tet_tris(unsigned m) {  // triangles of a sign mask of 4 corners
  const int n = __popc(m);
  return n == 0 || n == 4 ? 0 : (n == 2 ? 2 : 1);
}

struct Cube {
  float f[8];   // chi - level at the corners
  float3 o;     // unwrapped grid coordinates of corner 0
};

// Vertex on the tetrahedron edge from corner u to corner v (u's coordinates
// below v's on every axis where they differ): from the lower endpoint, in
// unit-cube coordinates.
__device__ __forceinline__ float3 edge_vertex(const Cube& c, int u, int v, float inv_r) {
  const float fu = c.f[u], fv = c.f[v];
  const float t = fu / (fu - fv);
  const float ux = c.o.x + (u & 1), uy = c.o.y + ((u >> 1) & 1), uz = c.o.z + ((u >> 2) & 1);
  const float dx = (float)((v & 1) - (u & 1)), dy = (float)(((v >> 1) & 1) - ((u >> 1) & 1)),
              dz = (float)(((v >> 2) & 1) - ((u >> 2) & 1));
  return make_float3((ux + t * dx) * inv_r, (uy + t * dy) * inv_r, (uz + t * dz) * inv_r);
}

__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 f3cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Emit triangle (p0, p1, p2) oriented towards `up` (a vector from the
// tetrahedron's negative corners to its positive ones).
__device__ __forceinline__ void emit(float* tris, float* nrm, unsigned long long k, unsigned long long cap,
                                     float3 p0, float3 p1, float3 p2, float3 up) {
  if (k >= cap) return;
  float3 n = f3cross(f3sub(p1, p0), f3sub(p2, p0));
  if (f3dot(n, up) < 0.f) {
    const float3 q = p1;
    p1 = p2;
    p2 = q;
    n = make_float3(-n.x, -n.y, -n.z);
  }
  const float len = sqrtf(f3dot(n, n));
  const float s = len > 0.f ? 1.f / len : 0.f;
  float* t = tris + 9 * k;
  t[0] = p0.x; t[1] = p0.y; t[2] = p0.z;
  t[3] = p1.x; t[4] = p1.y; t[5] = p1.z;
  t[6] = p2.x; t[7] = p2.y; t[8] = p2.z;
  nrm[3 * k] = n.x * s;
  nrm[3 * k + 1] = n.y * s;
  nrm[3 * k + 2] = n.z * s;
}

// labels (optional): a component label per voxel (dpsr_largest_region);
// then only the tetrahedra whose negative corners carry label `keep` emit
// (their negative corners are always in one component).
__global__ void __launch_bounds__(256) k_mesh_extract(const float* __restrict__ chi, int r, float level,
                                                      float* __restrict__ tris, float* __restrict__ nrm,
                                                      unsigned long long* __restrict__ count,
                                                      unsigned long long cap, const int* __restrict__ labels,
                                                      int keep) {
  const int64_t n = (int64_t)r * r * r;
  const float inv_r = 1.f / (float)r;  // r is a power of two: exact
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < n;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(cell / ((int64_t)r * r)), j = (int)((cell / r) % r), k = (int)(cell % r);
    Cube c;
    unsigned neg = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int ii = (i + (q & 1)) & (r - 1), jj = (j + ((q >> 1) & 1)) & (r - 1), kk = (k + ((q >> 2) & 1)) & (r - 1);
      c.f[q] = __ldg(chi + ((int64_t)ii * r + jj) * r + kk) - level;
      neg |= (c.f[q] < 0.f ? 1u : 0u) << q;
    }
    if (neg == 0u || neg == 255u) continue;
    if (labels) {  // keep the negative corners of component `keep` only
      unsigned kept = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!((neg >> q) & 1u)) continue;
        const int ii = (i + (q & 1)) & (r - 1), jj = (j + ((q >> 1) & 1)) & (r - 1), kk = (k + ((q >> 2) & 1)) & (r - 1);
        if (__ldg(labels + ((int64_t)ii * r + jj) * r + kk) == keep) kept |= 1u << q;
      }
      if (!kept) continue;
      // a tetrahedron emits when its negative corners are kept ones
      neg |= (~kept & neg) << 8;  // bits 8..15: negative corners of other components
    }
    c.o = make_float3((float)i, (float)j, (float)k);
    // count first, reserve once per cube, then write
    const unsigned other = neg >> 8;
    neg &= 255u;
    auto skip = [&](int t) {  // a tetrahedron whose negative corners lie in another component
      unsigned o = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) o |= (other >> kTet[t][a]) & 1u;
      return o != 0u;
    };
    int nt = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      unsigned m = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) m |= ((neg >> kTet[t][a]) & 1u) << a;
      if (!skip(t)) nt += tet_tris(m);
    }
    unsigned long long base = atomicAdd(count, (unsigned long long)nt);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      int q[4];
      unsigned m = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        q[a] = kTet[t][a];
        m |= ((neg >> q[a]) & 1u) << a;
      }
      const int cnt = __popc(m);
      if (cnt == 0 || cnt == 4 || skip(t)) continue;
      // up: from the centroid of the negative corners to that of the positive ones
      float3 pn = make_float3(0.f, 0.f, 0.f), pp = pn;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float3 g = make_float3((float)(q[a] & 1), (float)((q[a] >> 1) & 1), (float)((q[a] >> 2) & 1));
        if ((m >> a) & 1u) pn = make_float3(pn.x + g.x, pn.y + g.y, pn.z + g.z);
        else pp = make_float3(pp.x + g.x, pp.y + g.y, pp.z + g.z);
      }
      const float wn = 1.f / (float)cnt, wp = 1.f / (float)(4 - cnt);
      const float3 up = make_float3(pp.x * wp - pn.x * wn, pp.y * wp - pn.y * wn, pp.z * wp - pn.z * wn);
      // edges keep the tetrahedron's vertex order (corner ids increase along it)
      auto ev = [&](int a, int b) { return a < b ? edge_vertex(c, q[a], q[b], inv_r) : edge_vertex(c, q[b], q[a], inv_r); };
      if (cnt == 1 || cnt == 3) {
        int odd = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if ((((m >> a) & 1u) != 0u) == (cnt == 1)) odd = a;
        int o[3], w = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (a != odd) o[w++] = a;
        emit(tris, nrm, base++, cap, ev(odd, o[0]), ev(odd, o[1]), ev(odd, o[2]), up);
      } else {
        int ng[2], ps[2], a0 = 0, a1 = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if ((m >> a) & 1u) ng[a0++] = a;
          else ps[a1++] = a;
        }
        // the quad ng0-ps0, ng0-ps1, ng1-ps1, ng1-ps0 in cyclic order
        const float3 v0 = ev(ng[0], ps[0]), v1 = ev(ng[0], ps[1]), v2 = ev(ng[1], ps[1]), v3 = ev(ng[1], ps[0]);
        emit(tris, nrm, base++, cap, v0, v1, v2, up);
        emit(tris, nrm, base++, cap, v0, v2, v3, up);
      }
    }
  }
}

// Surrogate gradient of Eq. 6 at M mesh points: the loss gradient dL/dp_i
// reaches chi as dL/dchi(p_i) = dL/dp_i . (-n_i), and that value goes onto
// the grid by the adjoint of the trilinear lookup at p_i (the rasterization
// of Eq. A2 with scalar values).
__global__ void __launch_bounds__(256) k_mesh_surrogate(float* __restrict__ grid, int r,
                                                        const float* __restrict__ p, const float* __restrict__ n,
                                                        const float* __restrict__ g, int64_t M) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = -(g[3 * i] * n[3 * i] + g[3 * i + 1] * n[3 * i + 1] + g[3 * i + 2] * n[3 * i + 2]);
    const Axis ax = axis_of(p[3 * i], r), ay = axis_of(p[3 * i + 1], r), az = axis_of(p[3 * i + 2], r);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int dx = d >> 2, dy = (d >> 1) & 1, dz = d & 1;
      const float w = (dx ? ax.t : 1.f - ax.t) * (dy ? ay.t : 1.f - ay.t) * (dz ? az.t : 1.f - az.t);
      const size_t j = ((size_t)(dx ? ax.i1 : ax.i0) * r + (dy ? ay.i1 : ay.i0)) * r + (dz ? az.i1 : az.i0);
      atomicAdd(&grid[j], w * v);
    }
  }
}

}  // namespace dpsr

extern "C" {

int dpsr_mesh_extract(const float* chi, int r, float level, float* tris, float* normals, int64_t max_tris,
                      unsigned long long* count, void* stream) {
  if (!chi || !count || r < 2 || r > 512 || (r & (r - 1)) || max_tris < 0 || !isfinite(level))
    return DPSR_EINVAL;
  if (max_tris > 0 && (!tris || !normals)) return DPSR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return DPSR_ECUDA;
  const int64_t n = (int64_t)r * r * r;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 64);
  dpsr::k_mesh_extract<<<blocks, 256, 0, st>>>(chi, r, level, tris, normals, count,
                                                (unsigned long long)max_tris, nullptr, 0);
  return cudaGetLastError() == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

int dpsr_mesh_extract_region(const float* chi, int r, float level, const int* labels, int keep, float* tris,
                             float* normals, int64_t max_tris, unsigned long long* count, void* stream) {
  if (!chi || !labels || !count || r < 2 || r > 512 || (r & (r - 1)) || max_tris < 0 || !isfinite(level))
    return DPSR_EINVAL;
  if (max_tris > 0 && (!tris || !normals)) return DPSR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return DPSR_ECUDA;
  const int64_t n = (int64_t)r * r * r;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 64);
  dpsr::k_mesh_extract<<<blocks, 256, 0, st>>>(chi, r, level, tris, normals, count,
                                                (unsigned long long)max_tris, labels, keep);
  return cudaGetLastError() == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

int dpsr_mesh_surrogate_splat(float* dchi, int r, const float* points, const float* normals, const float* dldp,
                              int64_t M, int accumulate, void* stream) {
  if (!dchi || r < 2 || r > 512 || (r & (r - 1)) || M < 0) return DPSR_EINVAL;
  if (M > 0 && (!points || !normals || !dldp)) return DPSR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!accumulate && cudaMemsetAsync(dchi, 0, sizeof(float) * (size_t)r * r * r, st) != cudaSuccess)
    return DPSR_ECUDA;
  if (M == 0) return DPSR_OK;
  const int blocks = (int)std::min<int64_t>((M + 255) / 256, 4736);
  dpsr::k_mesh_surrogate<<<blocks, 256, 0, st>>>(dchi, r, points, normals, dldp, M);
  return cudaGetLastError() == cudaSuccess ? DPSR_OK : DPSR_ECUDA;
}

}  // extern "C"
