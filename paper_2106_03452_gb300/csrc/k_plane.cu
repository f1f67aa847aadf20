// Plane kernels: one thread-block cluster per x-plane of the r^3 grid. The C
// CTAs of a cluster each own r/C consecutive y-rows of the plane in shared
// memory; the transform along y reads the whole plane through distributed
// shared memory (DSMEM), so a plane never round-trips through HBM between the
// z and y passes.
//
//   k_plane_fwd  (forward)  splat (Eq. A2) -> R2C along z -> FFT along y;
//                           writes D = i u_z v~_z + i u_y v~_y (partially
//                           transformed), C = v~_x and W~ (transform of the
//                           weight field, for the mean of Eq. 4).
//   k_plane_inv  (forward)  IFFT along y -> C2R along z -> chi = a y + b
//                           (Eq. 4); stores the gradient of the trilinear
//                           lookup of chi' at the points for the backward.
//   k_plane_bfwd (backward) R2C along z and FFT along y of dchi, with the sums
//                           S = sum dchi and sum dchi * chi.
//   k_plane_binv (backward) IFFT along y -> C2R along z of the three adjoint
//                           fields V_bar_a, then the adjoint of the splat
//                           (gather and weight derivatives) at the points.
#include "dpsr_dev.cuh"
#include "launch.h"

namespace dpsr {

template <int L, int C>
struct PlaneGeo {
  static constexpr int R1 = Shape<L>::R1, T = Shape<L>::T, G = kNT / T;
  static constexpr int R = L / C;        // rows per CTA
  static constexpr int H = L / 2;        // packed half-spectrum slots per channel
  static constexpr int SPC = H / C;      // slots per CTA per channel (y pass)
  static constexpr int SP = L + 1;       // staging column pitch (float2)
  static constexpr int KP = L / 2 + 2;   // row pitch of the spectral buffers in HBM
  static constexpr int SWM = (H < 16 ? H : 16) - 1;
  static_assert(R >= 2 && R % 2 == 0, "at least one row pair per CTA");
};

// XOR swizzle inside aligned 16-slot blocks: a column read across 16 rows and
// a row read across 16 columns both touch 16 distinct bank pairs.
template <int RP, int SWM>
__device__ __forceinline__ int sw(int row, int col) {
  return row * RP + (col ^ (row & SWM));
}

// Points whose trilinear stencil touches x-plane X: cells X (delta_x = 0) and
// X - 1 (delta_x = 1), from the bin offsets of the x-sort.
struct PlanePoints {
  int b0, n0, b1, n1;
  __device__ PlanePoints(const Solve& S, int X) {
    const int* off = S.bins + S.r;
    const int Xm = (X - 1) & (S.r - 1);
    b0 = off[X];
    n0 = off[X + 1] - b0;
    b1 = off[Xm];
    n1 = off[Xm + 1] - b1;
  }
  __device__ int total() const { return n0 + n1; }
  __device__ int index(int i, int& dx) const {
    dx = i < n0 ? 0 : 1;
    return i < n0 ? b0 + i : b1 + (i - n0);
  }
};

__device__ __forceinline__ float wsel(int d, float t) { return d ? t : 1.f - t; }

// Write a chunk of y-transformed columns (staging [group][ky]) to the spectral
// buffer dst[X][ky][kz]. Slot 0 carries the packed DC and Nyquist columns and
// is separated into kz = 0 and kz = L/2.
template <int L, int C>
__device__ __forceinline__ void store_cols(float2* __restrict__ dst, int X, int s_first,
                                           int nvalid, const float2* scr) {
  using P = PlaneGeo<L, C>;
  for (int i = threadIdx.x; i < P::G * L; i += kNT) {
    const int gi = i % P::G, ky = i / P::G;
    if (gi >= nvalid) continue;
    const int s = s_first + gi;
    const float2* col = scr + gi * P::SP;
    const float2 v = col[ky];
    const size_t base = ((size_t)X * L + ky) * P::KP;
    if (s != 0) {
      dst[base + s] = v;
    } else {
      float2 x0, xn;
      unpack_dc_nyq(v, col[(L - ky) & (L - 1)], x0, xn);
      dst[base] = x0;
      dst[base + P::H] = xn;
    }
  }
}

// Load a chunk of columns src[X][ky][kz] into staging [group][ky]; slot 0 is
// packed as X0 + i Xn from kz = 0 and kz = L/2 (both transform to real rows).
// mul(ky, s, v) may scale the value on the way in.
template <int L, int C, class Mul>
__device__ __forceinline__ void load_cols(const float2* __restrict__ src, int X, int s_first,
                                          int nvalid, float2* scr, Mul mul) {
  using P = PlaneGeo<L, C>;
  for (int i = threadIdx.x; i < P::G * L; i += kNT) {
    const int gi = i % P::G, ky = i / P::G;
    if (gi >= nvalid) continue;
    const int s = s_first + gi;
    const size_t base = ((size_t)X * L + ky) * P::KP;
    float2 v;
    if (s != 0) {
      v = src[base + s];
    } else {
      const float2 a = src[base], b = src[base + P::H];
      v = make_float2(a.x - b.y, a.y + b.x);
    }
    scr[gi * P::SP + ky] = mul(ky, s, v);
  }
}

// Push a chunk of y-domain columns (staging [group][y]) into the rows of their
// owner CTAs: row y, slot `choff + s`.
template <int L, int C, int RP>
__device__ __forceinline__ void push_cols(float2* const* rb, int s_first, int nvalid, int choff,
                                          const float2* scr) {
  using P = PlaneGeo<L, C>;
  for (int i = threadIdx.x; i < P::G * L; i += kNT) {
    const int gi = i % P::G, y = i / P::G;
    if (gi >= nvalid) continue;
    const int q = y / P::R, lr = y % P::R;
    rb[q][sw<RP, P::SWM>(lr, choff + s_first + gi)] = scr[gi * P::SP + y];
  }
}

// ===========================================================================
// Forward plane kernel: splat + R2C(z) + FFT(y).
// ===========================================================================
template <int L, int C>
__global__ void __launch_bounds__(kNT, 1)
    k_plane_fwd(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = L;  // two channels of H packed slots (or L complex in real space)
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ float4 smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = rows + P::R * RP;
  float* iu = reinterpret_cast<float*>(tw + L);
  float2* scr = tw + L + L / 2;
  float2* stg = scr + g * P::SP;
  float2* rb[C];
#pragma unroll
  for (int q = 0; q < C; ++q) rb[q] = cl.map_shared_rank(rows, q);
  for (int i = tid; i < L; i += kNT) {
    tw[i] = S.tw[i];
    iu[i] = S.iu[i];
  }
  const PlanePoints pp(S, X);
  const int y_lo = c * P::R;

  for (int round = 0; round < 2; ++round) {
    for (int i = tid; i < P::R * RP; i += kNT) rows[i] = czero();
    __syncthreads();
    // Rasterization (Eq. A2): round 0 splats (n_y, n_z), round 1 (n_x, 1).
    for (int i = tid; i < pp.total(); i += kNT) {
      int dx;
      const int idx = pp.index(i, dx);
      const float4 a = S.sorted[2 * idx], b = S.sorted[2 * idx + 1];
      const Axis ax = axis_of(a.x, L), ay = axis_of(a.y, L), az = axis_of(a.z, L);
      const float fx = wsel(dx, ax.t);
      const float va = round == 0 ? b.x : a.w;
      const float vb = round == 0 ? b.y : 1.f;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int ly = (dy ? ay.i1 : ay.i0) - y_lo;
        if ((unsigned)ly >= (unsigned)P::R) continue;
        const float fxy = fx * wsel(dy, ay.t);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int z = dz ? az.i1 : az.i0;
          const float w = fxy * wsel(dz, az.t);
          float2* cell = &rows[sw<RP, P::SWM>(ly, z)];
          atomicAdd(&cell->x, w * va);
          atomicAdd(&cell->y, w * vb);
        }
      }
    }
    __syncthreads();
    // R2C along z of each row; channel B of round 0 takes the factor i u_z.
    for (int r0 = 0; r0 < P::R; r0 += P::G) {
      const int row = r0 + g;
      const bool ok = row < P::R;
      const int rr = ok ? row : 0;
      r2c_pair<L>(
          t, stg, tw, [&](int z) { return rows[sw<RP, P::SWM>(rr, z)]; },
          [&](int s, float2 v) {
            if (ok) rows[sw<RP, P::SWM>(rr, s)] = v;
          },
          [&](int s, float2 v) {
            if (!ok) return;
            if (round == 0) v = s == 0 ? czero() : cmul_iu(v, iu[s]);
            rows[sw<RP, P::SWM>(rr, P::H + s)] = v;
          });
    }
    cl.sync();
    // FFT along y of this CTA's slots, reading all rows of the plane.
    for (int cb = 0; cb < P::SPC; cb += P::G) {
      const int nvalid = min(P::G, P::SPC - cb);
      const int s_first = c * P::SPC + cb;
      const int s = s_first + min(g, nvalid - 1);
      float2 va[P::R1];
      auto load = [&](float2(&v)[P::R1], int choff) {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) {
          const int y = t + P::T * j;
          v[j] = rb[y / P::R][sw<RP, P::SWM>(y % P::R, choff + s)];
        }
      };
      load(va, 0);
      fft<L, -1>(va, t, stg, tw);
      if (round == 0) {
        float2 vb[P::R1];
        load(vb, P::H);
        fft<L, -1>(vb, t, stg, tw);
#pragma unroll
        for (int j = 0; j < P::R1; ++j) {
          const int ky = t + P::T * j;
          stg[ky] = cadd(vb[j], cmul_iu(va[j], iu[ky]));
        }
        __syncthreads();
        store_cols<L, C>(S.spec[0], X, s_first, nvalid, scr);
        __syncthreads();
      } else {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = va[j];
        __syncthreads();
        store_cols<L, C>(S.spec[1], X, s_first, nvalid, scr);
        __syncthreads();
        load(va, P::H);
        fft<L, -1>(va, t, stg, tw);
#pragma unroll
        for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = va[j];
        __syncthreads();
        store_cols<L, C>(S.spec[2], X, s_first, nvalid, scr);
        __syncthreads();
      }
    }
    cl.sync();
  }
}

// ===========================================================================
// Forward inverse plane kernel: IFFT(y) + C2R(z) + normalisation + lookup
// gradient of chi' at the points.
// ===========================================================================
template <int L, int C>
__global__ void __launch_bounds__(kNT, 1)
    k_plane_inv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = P::H;  // one channel
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ float4 smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = rows + P::R * RP;
  float2* scr = tw + L;
  float2* stg = scr + g * P::SP;
  float2* rb[C];
#pragma unroll
  for (int q = 0; q < C; ++q) rb[q] = cl.map_shared_rank(rows, q);
  for (int i = tid; i < L; i += kNT) tw[i] = S.tw[i];
  const float a_chi = S.sc->a_chi, b_chi = S.sc->b_chi;

  for (int cb = 0; cb < P::SPC; cb += P::G) {
    const int nvalid = min(P::G, P::SPC - cb);
    const int s_first = c * P::SPC + cb;
    load_cols<L, C>(S.spec[3], X, s_first, nvalid, scr, [](int, int, float2 v) { return v; });
    __syncthreads();
    float2 v[P::R1];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) v[j] = stg[t + P::T * j];
    fft<L, +1>(v, t, stg, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = v[j];
    __syncthreads();
    push_cols<L, C, RP>(rb, s_first, nvalid, 0, scr);
    __syncthreads();
  }
  cl.sync();
  // C2R along z of row pairs (2p, 2p+1); output written in place as pairs
  // (y_2p[z], y_2p+1[z]) at logical slot z of the pair.
  float* chi = S.chi;
  for (int p0 = 0; p0 < P::R / 2; p0 += P::G) {
    const int p = p0 + g;
    const bool ok = p < P::R / 2;
    const int pr = ok ? p : 0;
    const int ya = c * P::R + 2 * pr;
    c2r_pair<L>(
        t, stg, tw, [&](int k) { return rows[sw<RP, P::SWM>(2 * pr, k)]; },
        [&](int k) { return rows[sw<RP, P::SWM>(2 * pr + 1, k)]; },
        [&](int z, float2 v) {
          if (!ok) return;
          const size_t o = ((size_t)X * L + ya) * L + z;
          chi[o] = fmaf(a_chi, v.x, b_chi);
          chi[o + L] = fmaf(a_chi, v.y, b_chi);
          rows[sw<RP, P::SWM>(2 * pr + z / P::H, z % P::H)] = v;
        });
  }
  cl.sync();
  // Gradient of the trilinear lookup of y = n chi' at the points, this plane's
  // share (delta_x fixed by the plane).
  {
    const PlanePoints pp(S, X);
    const int y_lo = c * P::R;
    auto yval = [&](int y, int z) {
      const int q = y / P::R, lr = y % P::R, p2 = lr & ~1;
      const float2 f = rb[q][sw<RP, P::SWM>(p2 + z / P::H, z % P::H)];
      return (lr & 1) ? f.y : f.x;
    };
    for (int i = tid; i < pp.total(); i += kNT) {
      int dx;
      const int idx = pp.index(i, dx);
      const float4 a = S.sorted[2 * idx];
      const Axis ax = axis_of(a.x, L), ay = axis_of(a.y, L), az = axis_of(a.z, L);
      if (ay.i0 - y_lo < 0 || ay.i0 - y_lo >= P::R) continue;
      const float fx = wsel(dx, ax.t), dfx = dx ? (float)L : -(float)L;
      float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int y = dy ? ay.i1 : ay.i0;
        const float fy = wsel(dy, ay.t), dfy = dy ? (float)L : -(float)L;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int z = dz ? az.i1 : az.i0;
          const float fz = wsel(dz, az.t), dfz = dz ? (float)L : -(float)L;
          const float val = yval(y, z);
          gx += dfx * fy * fz * val;
          gy += fx * dfy * fz * val;
          gz += fx * fy * dfz * val;
        }
      }
      S.gfwd[(size_t)dx * S.N + idx] = make_float4(gx, gy, gz, 0.f);
    }
  }
  cl.sync();
}

// ===========================================================================
// Backward plane kernel: R2C(z) + FFT(y) of dchi, and the sums of dchi and
// dchi * chi needed by the adjoint of Eq. 4.
// ===========================================================================
template <int L, int C>
__global__ void __launch_bounds__(kNT, 1)
    k_plane_bfwd(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = P::H;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ float4 smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = rows + P::R * RP;
  float2* scr = tw + L;
  float2* stg = scr + g * P::SP;
  __shared__ double red[2][kNT / 32];
  float2* rb[C];
#pragma unroll
  for (int q = 0; q < C; ++q) rb[q] = cl.map_shared_rank(rows, q);
  for (int i = tid; i < L; i += kNT) tw[i] = S.tw[i];
  __syncthreads();
  const float* gin = S.dchi;
  const float* chi = S.chi;
  float accS = 0.f, accD = 0.f;
  for (int p0 = 0; p0 < P::R / 2; p0 += P::G) {
    const int p = p0 + g;
    const bool ok = p < P::R / 2;
    const int pr = ok ? p : 0;
    const size_t o = ((size_t)X * L + c * P::R + 2 * pr) * L;
    r2c_pair<L>(
        t, stg, tw,
        [&](int z) {
          const float a = gin[o + z], b = gin[o + L + z];
          if (ok) {
            accS += a + b;
            accD += a * chi[o + z] + b * chi[o + L + z];
          }
          return make_float2(a, b);
        },
        [&](int s, float2 v) {
          if (ok) rows[sw<RP, P::SWM>(2 * pr, s)] = v;
        },
        [&](int s, float2 v) {
          if (ok) rows[sw<RP, P::SWM>(2 * pr + 1, s)] = v;
        });
  }
  cl.sync();
  for (int cb = 0; cb < P::SPC; cb += P::G) {
    const int nvalid = min(P::G, P::SPC - cb);
    const int s_first = c * P::SPC + cb;
    const int s = s_first + min(g, nvalid - 1);
    float2 v[P::R1];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      const int y = t + P::T * j;
      v[j] = rb[y / P::R][sw<RP, P::SWM>(y % P::R, s)];
    }
    fft<L, -1>(v, t, stg, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = v[j];
    __syncthreads();
    store_cols<L, C>(S.spec[3], X, s_first, nvalid, scr);
    __syncthreads();
  }
  // block partial sums in FP64, fixed order
  {
    double dS = accS, dD = accD;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      dS += __shfl_xor_sync(0xffffffffu, dS, m);
      dD += __shfl_xor_sync(0xffffffffu, dD, m);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = dS;
      red[1][tid >> 5] = dD;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0, b = 0;
      for (int w = 0; w < kNT / 32; ++w) {
        a += red[0][w];
        b += red[1][w];
      }
      S.part[2 * blockIdx.x] = a;
      S.part[2 * blockIdx.x + 1] = b;
    }
  }
  cl.sync();
}

// ===========================================================================
// Backward inverse plane kernel: IFFT(y) + C2R(z) of the three adjoint fields
// V_bar_x, V_bar_y, V_bar_z, then dnormals = gather and the weight-derivative
// part of dpoints, per plane side.
// ===========================================================================
template <int L, int C>
__global__ void __launch_bounds__(kNT, 1)
    k_plane_binv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = 3 * P::H;  // channels X | Y | Z
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ float4 smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = rows + P::R * RP;
  float* iu = reinterpret_cast<float*>(tw + L);
  float2* scr = tw + L + L / 2;
  float2* stg = scr + g * P::SP;
  float2* rb[C];
#pragma unroll
  for (int q = 0; q < C; ++q) rb[q] = cl.map_shared_rank(rows, q);
  for (int i = tid; i < L; i += kNT) {
    tw[i] = S.tw[i];
    iu[i] = S.iu[i];
  }
  __syncthreads();

  for (int cb = 0; cb < P::SPC; cb += P::G) {
    const int nvalid = min(P::G, P::SPC - cb);
    const int s_first = c * P::SPC + cb;
    const int s = s_first + min(g, nvalid - 1);
    float2 v[P::R1];
    // X channel: Q2 = IFFT_x(-i u_x F), y-inverse as is.
    load_cols<L, C>(S.spec[1], X, s_first, nvalid, scr, [](int, int, float2 w) { return w; });
    __syncthreads();
#pragma unroll
    for (int j = 0; j < P::R1; ++j) v[j] = stg[t + P::T * j];
    fft<L, +1>(v, t, stg, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = v[j];
    __syncthreads();
    push_cols<L, C, RP>(rb, s_first, nvalid, 0, scr);
    __syncthreads();
    // Y and Z channels from Q1 = IFFT_x(F): -i u_y before the y-inverse,
    // -i u_z (a constant per column) for Z.
    load_cols<L, C>(S.spec[0], X, s_first, nvalid, scr, [](int, int, float2 w) { return w; });
    __syncthreads();
    float2 q1[P::R1];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      const int ky = t + P::T * j;
      q1[j] = stg[ky];
      v[j] = cmul_iu(q1[j], -iu[ky]);
    }
    fft<L, +1>(v, t, stg, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = v[j];
    __syncthreads();
    push_cols<L, C, RP>(rb, s_first, nvalid, P::H, scr);
    __syncthreads();
    const float ez = s == 0 ? 0.f : -iu[s];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) v[j] = cmul_iu(q1[j], ez);
    fft<L, +1>(v, t, stg, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) stg[t + P::T * j] = v[j];
    __syncthreads();
    push_cols<L, C, RP>(rb, s_first, nvalid, 2 * P::H, scr);
    __syncthreads();
  }
  cl.sync();
  // C2R along z: rows of (X, Y) pairs in place as (Vx[z], Vy[z]); Z channel
  // by row pairs, in place as (Vz_2p[z], Vz_2p+1[z]) over the Z slots of the
  // two rows.
  for (int r0 = 0; r0 < P::R; r0 += P::G) {
    const int row = r0 + g;
    const bool ok = row < P::R;
    const int rr = ok ? row : 0;
    c2r_pair<L>(
        t, stg, tw, [&](int k) { return rows[sw<RP, P::SWM>(rr, k)]; },
        [&](int k) { return rows[sw<RP, P::SWM>(rr, P::H + k)]; },
        [&](int z, float2 w) {
          if (ok) rows[sw<RP, P::SWM>(rr, z)] = w;
        });
  }
  for (int p0 = 0; p0 < P::R / 2; p0 += P::G) {
    const int p = p0 + g;
    const bool ok = p < P::R / 2;
    const int pr = ok ? p : 0;
    c2r_pair<L>(
        t, stg, tw, [&](int k) { return rows[sw<RP, P::SWM>(2 * pr, 2 * P::H + k)]; },
        [&](int k) { return rows[sw<RP, P::SWM>(2 * pr + 1, 2 * P::H + k)]; },
        [&](int z, float2 w) {
          if (ok) rows[sw<RP, P::SWM>(2 * pr + z / P::H, 2 * P::H + z % P::H)] = w;
        });
  }
  cl.sync();
  {
    const PlanePoints pp(S, X);
    const int y_lo = c * P::R;
    for (int i = tid; i < pp.total(); i += kNT) {
      int dx;
      const int idx = pp.index(i, dx);
      const float4 a = S.sorted[2 * idx], b = S.sorted[2 * idx + 1];
      const Axis ax = axis_of(a.x, L), ay = axis_of(a.y, L), az = axis_of(a.z, L);
      if (ay.i0 - y_lo < 0 || ay.i0 - y_lo >= P::R) continue;
      const float n0 = a.w, n1 = b.x, n2 = b.y;
      const float fx = wsel(dx, ax.t), dfx = dx ? (float)L : -(float)L;
      float nb0 = 0.f, nb1 = 0.f, nb2 = 0.f, cb0 = 0.f, cb1 = 0.f, cb2 = 0.f;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int y = dy ? ay.i1 : ay.i0;
        const int q = y / P::R, lr = y % P::R, p2 = lr & ~1;
        const float fy = wsel(dy, ay.t), dfy = dy ? (float)L : -(float)L;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          const int z = dz ? az.i1 : az.i0;
          const float fz = wsel(dz, az.t), dfz = dz ? (float)L : -(float)L;
          const float2 xy = rb[q][sw<RP, P::SWM>(lr, z)];
          const float2 zz = rb[q][sw<RP, P::SWM>(p2 + z / P::H, 2 * P::H + z % P::H)];
          const float vz = (lr & 1) ? zz.y : zz.x;
          const float w = fx * fy * fz;
          nb0 += w * xy.x;
          nb1 += w * xy.y;
          nb2 += w * vz;
          const float sdot = n0 * xy.x + n1 * xy.y + n2 * vz;
          cb0 += dfx * fy * fz * sdot;
          cb1 += fx * dfy * fz * sdot;
          cb2 += fx * fy * dfz * sdot;
        }
      }
      float* o = S.slots + ((size_t)dx * S.N + idx) * 6;
      o[0] = nb0;
      o[1] = nb1;
      o[2] = nb2;
      o[3] = cb0;
      o[4] = cb1;
      o[5] = cb2;
    }
  }
  cl.sync();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int L, int C>
constexpr size_t plane_smem(int kind) {
  using P = PlaneGeo<L, C>;
  const int rp = kind == 0 ? L : (kind == 3 ? 3 * P::H : P::H);
  const int extra = (kind == 0 || kind == 3) ? L / 2 : 0;  // iu table
  return sizeof(float2) * ((size_t)P::R * rp + L + extra + (size_t)P::G * P::SP);
}

template <int L, int C>
static cudaError_t launch_plane_t(int kind, const Solve& s, const Solve* tab, int count,
                                  cudaStream_t st) {
  void (*fn)(Solve, const Solve*) = nullptr;
  switch (kind) {
    case 0: fn = k_plane_fwd<L, C>; break;
    case 1: fn = k_plane_inv<L, C>; break;
    case 2: fn = k_plane_bfwd<L, C>; break;
    default: fn = k_plane_binv<L, C>; break;
  }
  const size_t smem = plane_smem<L, C>(kind);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set[4] = {false, false, false, false};  // per instantiation and kind
  if (!attr_set[kind]) {
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[kind] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L * C, 1, count);
  cfg.blockDim = dim3(kNT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, s, tab);
}

// Cluster sizes instantiated per grid size: one CTA per plane up to r = 64,
// 1/2/4 CTAs at r = 128, 2/4/8 CTAs at r = 256 (r^2 complex values of one
// plane do not fit one SM's shared memory there).
template <int L, int C>
constexpr bool plane_inst() {
  return L <= 64 ? C == 1 : (L == 128 ? (C == 1 || C == 2 || C == 4) : (C == 2 || C == 4 || C == 8));
}

template <int L>
static cudaError_t launch_plane_L(int kind, int C, const Solve& s, const Solve* tab, int count,
                                  cudaStream_t st) {
  switch (C) {
    case 1: if constexpr (plane_inst<L, 1>()) return launch_plane_t<L, 1>(kind, s, tab, count, st); break;
    case 2: if constexpr (plane_inst<L, 2>()) return launch_plane_t<L, 2>(kind, s, tab, count, st); break;
    case 4: if constexpr (plane_inst<L, 4>()) return launch_plane_t<L, 4>(kind, s, tab, count, st); break;
    case 8: if constexpr (plane_inst<L, 8>()) return launch_plane_t<L, 8>(kind, s, tab, count, st); break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_plane(int kind, int r, int C, const Solve& s, const Solve* tab, int count,
                         cudaStream_t st) {
  switch (r) {
    case 8: return launch_plane_L<8>(kind, C, s, tab, count, st);
    case 16: return launch_plane_L<16>(kind, C, s, tab, count, st);
    case 32: return launch_plane_L<32>(kind, C, s, tab, count, st);
    case 64: return launch_plane_L<64>(kind, C, s, tab, count, st);
    case 128: return launch_plane_L<128>(kind, C, s, tab, count, st);
    case 256: return launch_plane_L<256>(kind, C, s, tab, count, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t plane_smem_bytes(int kind, int r, int C) {
  auto pick = [&](auto Lc) -> size_t {
    constexpr int L = decltype(Lc)::value;
    switch (C) {
      case 1: if constexpr (plane_inst<L, 1>()) return plane_smem<L, 1>(kind); return 0;
      case 2: if constexpr (plane_inst<L, 2>()) return plane_smem<L, 2>(kind); return 0;
      case 4: if constexpr (plane_inst<L, 4>()) return plane_smem<L, 4>(kind); return 0;
      case 8: if constexpr (plane_inst<L, 8>()) return plane_smem<L, 8>(kind); return 0;
      default: return 0;
    }
  };
  switch (r) {
    case 8: return pick(std::integral_constant<int, 8>{});
    case 16: return pick(std::integral_constant<int, 16>{});
    case 32: return pick(std::integral_constant<int, 32>{});
    case 64: return pick(std::integral_constant<int, 64>{});
    case 128: return pick(std::integral_constant<int, 128>{});
    case 256: return pick(std::integral_constant<int, 256>{});
    default: return 0;
  }
}

}  // namespace dpsr
