// Pencil kernels: the (y, z) transforms of a plane split into a z pass over
// blocks of YB y-rows and a y pass over chunks of 16 kz columns, with the
// intermediate spectra in the spectral buffers (L2-resident up to r = 128).
// Each CTA is independent (no cluster, no DSMEM), so thousands of small CTAs
// keep every SM busy; the plane kernels of k_plane.cu instead keep a plane in
// the shared memory of a cluster. The autotuner picks between the two per
// kernel kind (cluster size 0 = this path).
//
//   forward   k_zfwd  splat (Eq. A2) of v_y, v_z, v_x, w into YB rows, R2C
//                     along z (v_z times i u_z)   -> buffers 0..3 (y, kz)
//             k_yfwd  FFT along y: D = FFT(i u_z v_z) + i u_y FFT(v_y) -> kSpD,
//                     C -> kSpC, W~ -> kSpW         (ky, kz)
//   inverse   k_yinv  IFFT along y of chi~ (kSpChi) -> kSpYa (y, kz)
//             k_zinv<1> C2R along z, chi = a y + b (Eq. 4), lookup gradient
//   backward  k_zbfwd sums of Eq. 4's adjoint, R2C along z of dchi -> kSpD
//             k_yfwd  FFT along y of kSpD in place
//   adjoint   k_yinv  IFFT along y of Q2, -i u_y Q1, -i u_z Q1 -> kSpC, kSpYa,
//                     kSpYb
//             k_zinv<3> C2R along z of the three fields, adjoint of the splat
// The buffer roles are listed with kNSpec.
//
// Half spectra along z are stored "packed" between the passes: slot 0 holds
// the DC and Nyquist terms of a real row as one complex number.
#include "dpsr_dev.cuh"
#include "finalize.cuh"
#include "launch.h"
#include "tma.cuh"

namespace dpsr {

template <int L>
struct Pen {
  static constexpr int T = Shape<L>::T, R1 = Shape<L>::R1;
  static constexpr int H = L / 2, KP = kpitch(L);
  static constexpr int YB = L < 16 ? L : 16;  // y-rows per z-pass CTA
  static constexpr int NYB = L / YB;
  static constexpr int NCOL = H < 16 ? H : 16;  // kz columns per y-pass CTA
  static constexpr int NKC = H / NCOL;          // y-pass CTAs per plane
  static constexpr int BOX = L * 16;            // float2 per TMA box [ky][16 kz]
  static constexpr int ZNT = 256;               // threads of the z-pass kernels
  static constexpr int ZG = ZNT / T;
  static_assert(YB == ybin(L) && NYB == nybins(L), "one point bin per z-pass CTA");
};

// Row pairs of the pair transforms in shared memory: pair p (rows 2p and
// 2p + 1, L floats each, contiguous) starts pair_off(p) floats in. The pitch
// 2L + 16 and 8 more floats for p = 2, 3 (mod 4) put the pairs that the
// groups of one warp transform on distinct banks (T = 8: offsets 0, 16, 8,
// 24 mod 32 banks; T = 16: 0, 16) for the 32-bit row loads and the 64-bit
// FFT exchange alike; with a plain 2L pitch every group of a warp hits the
// same banks. Offsets are multiples of 8 floats (bulk copies need 16 bytes).
// SP = false keeps the plain pitch: where a pass only makes 64-bit accesses
// and a group fills a half-warp (T = 16), the spread buys nothing and its
// shared memory would cost occupancy.
template <int L, bool SP = true>
__host__ __device__ constexpr int pair_off(int p) {
  return SP ? p * (2 * L + 16) + ((p & 2) ? 8 : 0) : p * 2 * L;
}
template <int L, bool SP = true>
__host__ __device__ constexpr int row_off(int q) {
  return pair_off<L, SP>(q >> 1) + (q & 1) * L;
}
template <int L, bool SP = true>
constexpr int pairs_floats(int np) {  // floats spanned by np pairs
  return pair_off<L, SP>(np - 1) + 2 * L;
}

// 1D weight of the trilinear stencil (Eq. A1): corner d of the cell, offset t.
__device__ __forceinline__ float tri_w(int d, float t) { return d ? t : 1.f - t; }

// Column 0 of a box holds P = X0 + i Xn, the transforms of the DC and Nyquist
// columns packed together. Split them in place (column 0 <- X0) and hand Xn
// to nyq(ky, value). Run by the T threads of one group.
template <int L, bool IL = false, class Nyq>
__device__ __forceinline__ void split_dc_nyq(float2* b, int t, Nyq nyq) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  float2 x0[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    const int ky = t + T * j;
    float2 xn;
    unpack_dc_nyq(b[bx(ky, 0)], b[bx((L - ky) & (L - 1), 0)], x0[j], xn);
    nyq(ky, xn);  // never column 0
  }
  group_sync<T, IL>();
#pragma unroll
  for (int j = 0; j < R1; ++j) b[bx(t + T * j, 0)] = x0[j];
}

// Sorted-point index range of point bin (x-cell xc, y-block yb): the points
// whose stencil origin lies in rows [yb * YB, yb * YB + YB) of x-cell xc.
__device__ __forceinline__ int2 bin_range(const Solve& S, int xc, int yb) {
  const int* off = S.bins + nbins(S.r);
  const int k = xc * nybins(S.r) + yb;
  return make_int2(off[k], off[k + 1]);
}

// R2C of two real rows a = p[0..L), b = p[L..2L): A's and B's packed half
// spectra (H slots each; slot 0 holds the real DC and Nyquist values) end in
// registers, A[j] and B[j] at slot t + T j. The rows' storage is the FFT
// exchange area. The group's lanes are contiguous (see Lanes).
//
// Z = FFT(a + i b) leaves Z[t + T j] in v[j] of thread t; the separation
// A[k] = (Z[k] + conj Z[L-k]) / 2, B[k] = -i (Z[k] - conj Z[L-k]) / 2 needs
// Z[L - k], k = t + T j, which is v[R1 - 1 - j] of thread T - t (t > 0) or
// v[R1 - j] of thread 0 itself (t = 0, j > 0): one shuffle per value instead
// of a round trip through shared memory. With iu given, both spectra leave
// multiplied by i u(k) (slot 0, DC and Nyquist, becomes 0): the spectral
// derivative of the forward's v_z rows, folded into the stores.
template <int L, class Tw>
__device__ __forceinline__ void r2c_pair_ab(int t, const Tw& tw, float* p, const float* iu,
                                            float2 (&A)[Shape<L>::R1 / 2], float2 (&B)[Shape<L>::R1 / 2]) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = make_float2(p[t + T * j], p[L + t + T * j]);
  group_sync<T>();
  float2* x = reinterpret_cast<float2*>(p);
  fft_r<L, -1>(v, t, [x](int i) -> float2& { return x[i]; }, tw);  // ends with a group sync
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gmask = T >= 32 ? 0xffffffffu : (((1u << (T & 31)) - 1u) << (lane & ~(unsigned)(T - 1)));
  const int src = (int)(lane & ~(unsigned)(T - 1)) | ((T - t) & (T - 1));
#pragma unroll
  for (int j = 0; j < R1 / 2; ++j) {
    float2 zm = v[(R1 - j) & (R1 - 1)];  // thread 0's own mirror (j > 0)
    if constexpr (T > 1) {
      const float2 s = v[R1 - 1 - j];
      const float mx = __shfl_sync(gmask, s.x, src), my = __shfl_sync(gmask, s.y, src);
      if (t != 0) zm = make_float2(mx, my);
    }
    const float2 zk = v[j];
    if (t == 0 && j == 0) {  // k = 0: Z[0] and Z[H] (v[R1 / 2] of thread 0)
      const float2 zn = v[R1 / 2];
      A[j] = make_float2(zk.x, zn.x);
      B[j] = make_float2(zk.y, zn.y);
    } else {
      zm = cconj(zm);
      A[j] = cscale(cadd(zk, zm), 0.5f);
      const float2 d = csub(zk, zm);  // B = -i d / 2
      B[j] = make_float2(0.5f * d.y, -0.5f * d.x);
    }
  }
  if (iu) {
#pragma unroll
    for (int j = 0; j < R1 / 2; ++j) {
      const int k = t + T * j;
      const float u = k == 0 ? 0.f : iu[k];
      A[j] = cmul_iu(A[j], u);
      B[j] = cmul_iu(B[j], u);
    }
  }
}

// Straight to global memory: the packed spectra of rows a and b go to the
// rows ga and gb of a spectral buffer from registers (a group's lanes write
// consecutive slots: whole 128-byte lines), with no shared-memory write and
// no bulk copy reading them back. `p` is left as FFT exchange scratch.
template <int L, class Tw>
__device__ __forceinline__ void r2c_pair_st(int t, const Tw& tw, float* p, const float* iu, float2* ga,
                                            float2* gb) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  float2 A[R1 / 2], B[R1 / 2];
  r2c_pair_ab<L>(t, tw, p, iu, A, B);
#pragma unroll
  for (int j = 0; j < R1 / 2; ++j) {
    ga[t + T * j] = A[j];
    gb[t + T * j] = B[j];
  }
}

// C2R of two packed half spectra A, B in place, through an accessor: x(i),
// i < L, addresses the pair's storage (A's slots for i < H, B's for
// i >= H); it is also the FFT exchange area and receives (a[z], b[z]) at
// x(z), unnormalised.
template <int L, class Tw, class Acc>
__device__ __forceinline__ void c2r_acc(int t, const Tw& tw, Acc x) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T, H = L / 2;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    const int k = t + T * j;
    if (k == 0 || k == H) {
      const float2 a = x(0), b = x(H);
      v[j] = (k == 0) ? make_float2(a.x, b.x) : make_float2(a.y, b.y);
    } else if (k < H) {
      const float2 a = x(k), b = x(H + k);
      v[j] = make_float2(a.x - b.y, a.y + b.x);
    } else {
      const float2 a = x(L - k), b = x(H + L - k);
      v[j] = make_float2(a.x + b.y, b.x - a.y);
    }
  }
  group_sync<T>();
  fft_r<L, +1>(v, t, x, tw);
#pragma unroll
  for (int j = 0; j < R1; ++j) x(t + T * j) = v[j];
}

// ===========================================================================
// Forward z pass: splat of the four channels into YB rows of plane X, R2C.
// ===========================================================================
template <int L>
constexpr size_t zfwd_smem() {
  using P = Pen<L>;
  return sizeof(float) * (pairs_floats<L>(2 * P::YB) + L) + sizeof(float2) * L;
}

// One z-pass tile (plane X, rows y0 .. y0 + YB - 1) on zeroed `rows`:
// splat, R2C, bulk stores of the packed rows.
template <int L>
__device__ __forceinline__ void zfwd_tile(const Solve& S, int X, int y0, float* rows,
                                          const float2* twt, const float* iu) {
  using P = Pen<L>;
  constexpr int YB = P::YB, H = P::H;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  // Rasterization (Eq. A2): points of x-cells X (dx = 0) and X - 1 (dx = 1)
  // whose stencil rows i0 or i1 fall in [y0, y0 + YB), i.e. i0 in
  // [y0 - 1, y0 + YB - 1] (mod L): per side the CTA's own bin and the
  // previous y-block's bin (its last row only). The four ranges are read up
  // front and visited as one sequence, so that their loads overlap.
  const int yb = y0 / YB, ylast = (y0 - 1) & (L - 1);
  int q0, q1, q2, q3, c1, c2, c3, c4;  // range starts, cumulative counts
  {
    const int* off = S.bins + nbins(L);
    auto key = [&](int k) {
      return ((X - (k >> 1)) & (L - 1)) * P::NYB + ((k & 1) ? (yb + P::NYB - 1) % P::NYB : yb);
    };
    const bool prev = YB < L;  // with YB == L one bin holds the whole plane
    const int k0 = key(0), k1 = key(1), k2 = key(2), k3 = key(3);
    q0 = off[k0];
    q1 = prev ? off[k1] : 0;
    q2 = off[k2];
    q3 = prev ? off[k3] : 0;
    const int e0 = off[k0 + 1], e1 = prev ? off[k1 + 1] : 0, e2 = off[k2 + 1], e3 = prev ? off[k3 + 1] : 0;
    c1 = e0 - q0;
    c2 = c1 + (e1 - q1);
    c3 = c2 + (e2 - q2);
    c4 = c3 + (e3 - q3);
  }
  for (int v = tid; v < c4; v += P::ZNT) {
    const int k = v < c1 ? 0 : (v < c2 ? 1 : (v < c3 ? 2 : 3));
    const int i = k == 0 ? q0 + v : (k == 1 ? q1 + (v - c1) : (k == 2 ? q2 + (v - c2) : q3 + (v - c3)));
    const int side = k >> 1, part = k & 1;
    if (!dbg_in_range(S.status, i, S.N)) continue;
    const float4 a = S.sorted[2 * i], b = S.sorted[2 * i + 1];
    const Axis ay = axis_rec(a.y, b.w, 1, L);
    if (part == 1 && ay.i0 != ylast) continue;
    const Axis ax = axis_rec(a.x, b.w, 0, L), az = axis_rec(a.z, b.w, 2, L);
    const float wx = tri_w(side, ax.t);
    const float val[4] = {b.x, b.y, a.w, 1.f};
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int ly = (dy ? ay.i1 : ay.i0) - y0;
      if ((unsigned)ly >= (unsigned)YB) continue;
      const float f = wx * tri_w(dy, ay.t);
      const float f0 = f * (1.f - az.t), f1 = f * az.t;
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        float* row = rows + row_off<L>(ch * YB + ly);
        atomicAdd(row + az.i0, f0 * val[ch]);
        atomicAdd(row + az.i1, f1 * val[ch]);
      }
    }
  }
  __syncthreads();
  TwTab<L> twr{twt, t};
  constexpr int NP = 4 * YB / 2;
  for (int p0 = 0; p0 < NP; p0 += P::ZG) {
    const int pi = p0 + g;
    if (pi < NP) {  // whole groups
      // the v_z rows (pairs YB/2 .. YB-1) take i u_z (zero at DC and Nyquist)
      const bool vz = pi >= YB / 2 && pi < YB;
      const int ch = (2 * pi) / YB, ly = (2 * pi) % YB;  // rows ly, ly + 1 of channel ch
      float2* ga = S.spec[ch] + ((size_t)X * L + y0 + ly) * P::KP;
      r2c_pair_st<L>(t, twr, rows + pair_off<L>(pi), vz ? iu : nullptr, ga, ga + P::KP);
    }
  }
}

template <int L>
__global__ void __launch_bounds__(Pen<L>::ZNT, L >= 512 ? 1 : (L >= 256 ? 3 : 4)) k_zfwd(const __grid_constant__ Solve s0,
                                                      const Solve* __restrict__ tab) {
  using P = Pen<L>;
  constexpr int YB = P::YB;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int X = blockIdx.x / P::NYB, y0 = (blockIdx.x % P::NYB) * YB;
  const int tid = threadIdx.x;
  extern __shared__ float4 smem4[];
  constexpr int RF = pairs_floats<L>(2 * YB);
  float* rows = reinterpret_cast<float*>(smem4);  // rows ch * YB + ly (row_off): v_y, v_z, v_x, w
  float2* twt = reinterpret_cast<float2*>(rows + RF);
  float* iu = reinterpret_cast<float*>(twt + L);
  pdl_trigger();
  for (int i = tid; i < L; i += P::ZNT) {
    twt[i] = S.tw[i];
    iu[i] = S.iu[2 * L + i];  // z axis
  }
  for (int i = tid; i < RF / 4; i += P::ZNT) smem4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  pdl_wait();
  __syncthreads();
  zfwd_tile<L>(S, X, y0, rows, twt, iu);
}

// ===========================================================================
// Forward y pass over 16 kz columns of plane X, by CTA kind (blockIdx.y):
// 0: D = FFT(i u_z v_z) + i u_y FFT(v_y) from buffers 0 and 1 into kSpD;
// 1: C = FFT(v_x) in place in kSpC, and from r = 256 on (yfwd_merge) also
// W~ = FFT(w) in place in kSpW; 2 (below r = 256): W~. BWD: FFT of the
// z-transformed dchi in place in kSpD. Merging C and W~ halves the CTAs of
// the bandwidth-bound r = 256 pass; below, where the pass is bound by the
// latency of each CTA, more and shorter CTAs win.
// ===========================================================================
template <int L>
constexpr int ynt() {
  return 16 * Shape<L>::T >= 32 ? 16 * Shape<L>::T : 32;  // one group per column
}

template <int L>
constexpr bool yfwd_merge() {
  return L >= 256;
}

template <int L, bool BWD>
constexpr size_t yfwd_smem() {
  return 1024 + sizeof(float2) * ((size_t)(BWD ? 1 : 2) * Pen<L>::BOX + L) + sizeof(float) * L;
}

// Input buffers of a y-pass tile of kind `kind` (see k_yfwd): box 0 holds
// buf0 (input and output), box 1 (kinds 0 and merged 1) buf1.
struct YfwdBufs {
  int buf0, buf1;
  bool two;
};
template <int L, bool BWD>
__device__ __forceinline__ YfwdBufs yfwd_bufs(int kind) {
  YfwdBufs b;
  b.buf0 = kind == 1 ? kSpC : (kind == 2 ? kSpW : kSpD);
  b.buf1 = kind == 1 ? kSpW : 1;
  b.two = !BWD && (kind == 0 || (kind == 1 && yfwd_merge<L>()));
  return b;
}

// Thread 0: the TMA tile loads of a y-pass tile, completion on `bar`.
template <int L, bool BWD>
__device__ __forceinline__ void yfwd_issue(const Solve& S, int X, int kz0, int kind, float2* box,
                                           uint64_t* bar) {
  using P = Pen<L>;
  const YfwdBufs b = yfwd_bufs<L, BWD>(kind);
  mbar_expect_tx(bar, (b.two ? 2 : 1) * P::BOX * (uint32_t)sizeof(float2));
  for (int y = 0; y < L; y += tma_rows(L)) {
    tma_load_3d(box + y * 16, &S.tmy[b.buf0], kz0, y, X, bar);
    if (b.two) tma_load_3d(box + P::BOX + y * 16, &S.tmy[b.buf1], kz0, y, X, bar);
  }
}

// All threads: wait for the tile (phase `phase` of `bar`), transform, store
// (thread 0 waits until the stores have read shared memory). False if the
// bounded wait gave up (status set; the caller leaves).
template <int L, bool BWD>
__device__ __forceinline__ bool yfwd_tile(const Solve& S, int X, int kz0, int kind, float2* box,
                                          const float2* twt, const float* iu, uint64_t* bar,
                                          uint32_t phase) {
  using P = Pen<L>;
  constexpr int H = P::H;
  const YfwdBufs bb = yfwd_bufs<L, BWD>(kind);
  const int buf0 = bb.buf0, buf1 = bb.buf1;
  const bool two = bb.two;
  constexpr bool IL = P::T == 16;  // interleaved groups: conflict-free column accesses
  using LN = Lanes<P::T, IL>;
  const int tid = threadIdx.x, g = LN::group(tid), t = LN::lane(tid);
  const bool landed = __syncthreads_and(mbar_wait(bar, phase));
  if (!landed) {
    if (tid == 0) atomicOr(S.status, kStTimeout);
    mbar_wait(bar, phase);  // a last bounded chance for copies in flight
    return false;
  }
  TwTab<L> twr{twt, t};
  if (g < P::NCOL) {  // whole groups; one column array live at a time
    float2* b0 = box;
    auto c0 = [b0, g](int e) -> float2& { return b0[bx(e, g)]; };
    float2 a[P::R1];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) a[j] = c0(t + P::T * j);
    fft_r<L, -1, IL>(a, t, c0, twr);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) c0(t + P::T * j) = a[j];
    if (two) {
      float2* b1 = box + P::BOX;
      auto c1 = [b1, g](int e) -> float2& { return b1[bx(e, g)]; };
#pragma unroll
      for (int j = 0; j < P::R1; ++j) a[j] = c1(t + P::T * j);
      fft_r<L, -1, IL>(a, t, c1, twr);
      if (kind == 0) {  // D = FFT(i u_z v_z) + i u_y FFT(v_y); this lane wrote c0 above
#pragma unroll
        for (int j = 0; j < P::R1; ++j) {
          const int ky = t + P::T * j;
          c0(ky) = cadd(a[j], cmul_iu(c0(ky), iu[ky]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) c1(t + P::T * j) = a[j];
      }
    }
  }
  __syncthreads();
  const int nsplit = kind == 1 && two ? 2 : 1;  // tiles whose column 0 packs DC and Nyquist
  if (kz0 == 0 && g < nsplit) {
    // column 0 holds X0 + i Xn of the DC and Nyquist columns: split them
    float2* bq = box + g * P::BOX;
    float2* dst = S.spec[g == 0 ? buf0 : buf1];
    split_dc_nyq<L, IL>(bq, t, [&](int ky, float2 w) {
      if (H < 16) bq[bx(ky, H)] = w;
      else dst[((size_t)X * L + ky) * P::KP + H] = w;
    });
  }
  fence_async_smem();
  __syncthreads();
  if (tid == 0) {
    for (int y = 0; y < L; y += tma_rows(L)) {
      tma_store_3d(&S.tmy[buf0], kz0, y, X, box + y * 16);
      if (kind == 1 && two) tma_store_3d(&S.tmy[buf1], kz0, y, X, box + P::BOX + y * 16);
    }
    tma_store_commit();
    tma_store_wait_read();
  }
  return true;
}

template <int L, bool BWD>
__global__ void __launch_bounds__(ynt<L>(), L >= 512 ? 1 : (BWD ? 4 : (L >= 256 ? 3 : 5))) k_yfwd(const __grid_constant__ Solve s0,
                                                   const Solve* __restrict__ tab) {
  using P = Pen<L>;
  constexpr int NT = ynt<L>();
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int X = blockIdx.x / P::NKC, kz0 = (blockIdx.x % P::NKC) * P::NCOL;
  const int kind = BWD ? 3 : (int)blockIdx.y;
  const int tid = threadIdx.x;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  float2* box = reinterpret_cast<float2*>(smem_raw + pad);  // 1 or 2 boxes
  float2* twt = box + (BWD ? 1 : 2) * P::BOX;
  float* iu = reinterpret_cast<float*>(twt + L);
  __shared__ uint64_t bar;
  pdl_trigger();
  // thread 0 issues the tile loads first; the tables load while they fly
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_wait();
  if (tid == 0) yfwd_issue<L, BWD>(S, X, kz0, kind, box, &bar);
  for (int i = tid; i < L; i += NT) {
    twt[i] = S.tw[i];
    iu[i] = S.iu[L + i];  // y axis
  }
  __syncthreads();
  yfwd_tile<L, BWD>(S, X, kz0, kind, box, twt, iu, &bar, 0);
}

// ===========================================================================
// Inverse y pass over 16 kz columns of plane X, out of place (the pass can
// run again on the same inputs). NCH = 1: chi~ (kSpChi) -> kSpYa. NCH = 3:
// the adjoint fields V_bar_x = IFFT_y(Q2) -> kSpC, V_bar_y = IFFT_y(-i u_y
// Q1) -> kSpYa, V_bar_z = -i u_z IFFT_y(Q1) -> kSpYb, with Q1 in kSpD and
// Q2 in kSpChi. Below r = 256 (yinv_split) the adjoint fields take two CTA
// kinds (blockIdx.y): 0: V_bar_x from Q2; 1: V_bar_y and V_bar_z from Q1.
// There the pass is bound by each CTA's latency and shorter CTAs win; at
// r = 256, bound by bandwidth, one CTA does all three.
// ===========================================================================
template <int L, int NCH>
constexpr bool yinv_split() {
  return NCH == 3 && L < 256;
}

template <int L, int NCH>
constexpr size_t yinv_smem() {
  return 1024 + sizeof(float2) * ((size_t)NCH * Pen<L>::BOX + L) + sizeof(float) * L;
}

// Thread 0: the TMA tile loads of an inverse y-pass tile (part: -1 all
// fields, else the CTA kind of yinv_split), completion on `bar`.
template <int L, int NCH>
__device__ __forceinline__ void yinv_issue(const Solve& S, int X, int kz0, int part, float2* box,
                                           uint64_t* bar) {
  using P = Pen<L>;
  // NCH = 1: box 0 <- chi~; NCH = 3: box 0 <- Q2, box 1 <- Q1 (split: only
  // the kind's own input)
  const bool do0 = part != 1, do1 = NCH == 3 && part != 0;
  mbar_expect_tx(bar, ((do0 ? 1 : 0) + (do1 ? 1 : 0)) * P::BOX * (uint32_t)sizeof(float2));
  for (int y = 0; y < L; y += tma_rows(L)) {
    if (do0) tma_load_3d(box + y * 16, &S.tmy[kSpChi], kz0, y, X, bar);
    if (do1) tma_load_3d(box + P::BOX + y * 16, &S.tmy[kSpD], kz0, y, X, bar);
  }
}

// All threads: wait, transform, TMA stores (thread 0 waits until they have
// read shared memory). False if the bounded wait gave up.
template <int L, int NCH>
__device__ __forceinline__ bool yinv_tile(const Solve& S, int X, int kz0, int part, float2* box,
                                          const float2* twt, const float* iu, uint64_t* bar,
                                          uint32_t phase) {
  using P = Pen<L>;
  constexpr int H = P::H;
  constexpr bool IL = P::T == 16;  // interleaved groups: conflict-free column accesses
  using LN = Lanes<P::T, IL>;
  const int tid = threadIdx.x, g = LN::group(tid), t = LN::lane(tid);
  constexpr int NIN = NCH == 1 ? 1 : 2;
  const bool do0 = part != 1, do1 = NCH == 3 && part != 0;
  const bool landed = __syncthreads_and(mbar_wait(bar, phase));
  if (!landed) {
    if (tid == 0) atomicOr(S.status, kStTimeout);
    mbar_wait(bar, phase);
    return false;
  }
  TwTab<L> twr{twt, t};
  if (kz0 == 0 && g < NIN && (g == 0 ? do0 : do1)) {
    // column 0 becomes X0 + i Xn (Xn: the Nyquist column); the same lanes
    // read these elements again below
    float2* b = box + g * P::BOX;
    const float2* nq = S.spec[g == 0 ? kSpChi : kSpD] + (size_t)X * L * P::KP + H;
    for (int j = 0; j < P::R1; ++j) {
      const int ky = t + P::T * j;
      const float2 n = H >= 16 ? nq[(size_t)ky * P::KP] : b[bx(ky, H)];
      const float2 x0 = b[bx(ky, 0)];
      b[bx(ky, 0)] = make_float2(x0.x - n.y, x0.y + n.x);
    }
  }
  __syncthreads();
  if (g < P::NCOL) {
    const int sz = kz0 + g;
    auto cref = [&](int k) {
      float2* b = box + k * P::BOX;
      return [b, g](int e) -> float2& { return b[bx(e, g)]; };
    };
    float2 v[P::R1];
    auto c0 = cref(0);
    if (do0) {
#pragma unroll
      for (int j = 0; j < P::R1; ++j) v[j] = c0(t + P::T * j);
      fft_r<L, +1, IL>(v, t, c0, twr);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) c0(t + P::T * j) = v[j];
    }
    if (do1) {
      auto c1 = cref(1);
      auto c2 = cref(2);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) {
        v[j] = c1(t + P::T * j);
        c2(t + P::T * j) = v[j];
        v[j] = cmul_iu(v[j], -iu[t + P::T * j]);
      }
      fft_r<L, +1, IL>(v, t, c1, twr);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) c1(t + P::T * j) = v[j];
      group_sync<P::T, IL>();
#pragma unroll
      for (int j = 0; j < P::R1; ++j) v[j] = c2(t + P::T * j);
      fft_r<L, +1, IL>(v, t, c2, twr);
      const float ez = sz == 0 ? 0.f : -__ldg(S.iu + 2 * L + sz);  // z axis
#pragma unroll
      for (int j = 0; j < P::R1; ++j) c2(t + P::T * j) = cmul_iu(v[j], ez);
    }
  }
  fence_async_smem();
  __syncthreads();
  if (tid == 0) {
    for (int y = 0; y < L; y += tma_rows(L)) {
      if constexpr (NCH == 1) {
        tma_store_3d(&S.tmy[kSpYa], kz0, y, X, box + y * 16);
      } else {
        if (do0) tma_store_3d(&S.tmy[kSpC], kz0, y, X, box + y * 16);
        if (do1) {
          tma_store_3d(&S.tmy[kSpYa], kz0, y, X, box + P::BOX + y * 16);
          tma_store_3d(&S.tmy[kSpYb], kz0, y, X, box + 2 * P::BOX + y * 16);
        }
      }
    }
    tma_store_commit();
    tma_store_wait_read();
  }
  return true;
}

template <int L, int NCH>
__global__ void __launch_bounds__(16 * Shape<L>::T >= 32 ? 16 * Shape<L>::T : 32,
                                  L >= 512 ? 1 : (NCH == 1 || yinv_split<L, NCH>() ? 4 : 2))
    k_yinv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = Pen<L>;
  constexpr int NT = 16 * P::T >= 32 ? 16 * P::T : 32;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int X = blockIdx.x / P::NKC, kz0 = (blockIdx.x % P::NKC) * P::NCOL;
  const int tid = threadIdx.x;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  float2* box = reinterpret_cast<float2*>(smem_raw + pad);
  float2* twt = box + NCH * P::BOX;
  float* iu = reinterpret_cast<float*>(twt + L);
  __shared__ uint64_t bar;
  pdl_trigger();
  // thread 0 issues the tile loads first; the tables load while they fly
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_wait();
  const int part = yinv_split<L, NCH>() ? (int)blockIdx.y : -1;  // -1: all fields
  if (tid == 0) yinv_issue<L, NCH>(S, X, kz0, part, box, &bar);
  for (int i = tid; i < L; i += NT) {
    twt[i] = S.tw[i];
    iu[i] = S.iu[L + i];  // y axis
  }
  __syncthreads();
  yinv_tile<L, NCH>(S, X, kz0, part, box, twt, iu, &bar, 0);
}

// ===========================================================================
// Inverse z passes over tiles of YB rows of plane X (+ 2 halo rows for the
// stencil's row i0 + 1): persistent CTAs, each loading tile i + 1 by bulk
// copies (two stages) while it transforms tile i. Per tile: C2R of row pairs
// in place, then
//   NCH = 1 (forward): chi = a_chi y + b_chi for the YB rows, and the
//     gradient of the trilinear lookup of y at the points whose stencil row
//     i0 is one of them (this plane's share, delta_x fixed by the plane);
//   NCH = 3 (adjoint): C2R of V_bar_x (kSpC), V_bar_y (kSpYa), V_bar_z
//     (kSpYb); at those points the gather of the three fields (dnormals
//     share) and the weight derivatives times n . V (dpoints share).
// ===========================================================================
template <int L, int NCH>
struct ZiGeo {
  static constexpr int NR = Pen<L>::YB + 2;              // rows per tile
  // float2 per stage: NCH * NR / 2 row pairs at pair_off (rows of H float2);
  // the C2R makes 64-bit accesses only, spread needed below T = 16
  static constexpr bool SP = Shape<L>::T < 16;
  static constexpr int STAGE = pairs_floats<L, SP>(NCH * NR / 2) / 2;
  static constexpr int NT = 256;
};

template <int L, int NCH>
constexpr size_t zinv_smem() {
  return sizeof(float2) * ((size_t)2 * ZiGeo<L, NCH>::STAGE + L);
}

// Thread 0: bulk loads of a z-pass tile's rows (H slots each, YB + 2 rows
// per field) into the stage at `sb`, completion on `bar`.
template <int L, int NCH>
__device__ __forceinline__ void zinv_issue(const Solve& S, int tile, float2* sb, uint64_t* bar) {
  using P = Pen<L>;
  using Z = ZiGeo<L, NCH>;
  constexpr int YB = P::YB, H = P::H, NR = Z::NR, KP = P::KP;
  const int X = tile / P::NYB, y0 = (tile % P::NYB) * YB;
  mbar_expect_tx(bar, NCH * NR * H * (uint32_t)sizeof(float2));
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = NCH == 1 ? kSpYa : (ch == 0 ? kSpC : (ch == 1 ? kSpYa : kSpYb));
    const float2* base = S.spec[buf] + (size_t)X * L * KP;
    for (int ly = 0; ly < NR; ++ly)  // row y0 + ly, wrapping to rows 0, 1
      bulk_load(sb + row_off<L, Z::SP>(ch * NR + ly) / 2, base + (size_t)((y0 + ly) & (L - 1)) * KP,
                H * (uint32_t)sizeof(float2), bar);
  }
}

// All threads: one z-pass tile whose rows land in the stage at `sb`. The
// tile's point bins and this thread's first point record are read before
// wait_stage() (which waits for the rows, block-uniformly, and returns false
// on a timeout), so that their latencies overlap it; then C2R of the row
// pairs in place and the per-point outputs.
template <int L, int NCH, class Wait>
__device__ __forceinline__ bool zinv_tile(const Solve& S, int tile, float2* sb, const float2* twt,
                                          float a_chi, float b_chi, Wait wait_stage) {
  using P = Pen<L>;
  using Z = ZiGeo<L, NCH>;
  constexpr int YB = P::YB, NR = Z::NR, NT = Z::NT, G = NT / P::T;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  const int X = tile / P::NYB, y0 = (tile % P::NYB) * YB;
  // The tile's point bins (both plane sides, one sequence) and this
  // thread's first point record, read before the stage wait and the C2R so
  // that their dependent latencies overlap them.
  const int2 r0 = bin_range(S, X, y0 / YB), r1 = bin_range(S, (X - 1) & (L - 1), y0 / YB);
  const int n0 = r0.y - r0.x, nv = n0 + (r1.y - r1.x);
  float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
  if (tid < nv) {
    const int i = tid < n0 ? r0.x + tid : r1.x + (tid - n0);
    if (dbg_in_range(S.status, i, S.N)) {
      pa = S.sorted[2 * i];
      pb = S.sorted[2 * i + 1];  // normals (adjoint) and the packed cells
    }
  }
  if (!wait_stage()) return false;
  TwTab<L> twr{twt, t};
  // pair p of channel ch: rows 2p (A) and 2p + 1 (B) of the stage, L float2
  auto pair = [&](int ch, int p) {
    float2* ra = sb + pair_off<L, Z::SP>(ch * (NR / 2) + p) / 2;
    return [ra](int i) -> float2& { return ra[i]; };
  };
  constexpr int NP = NCH * NR / 2;
  for (int p0 = 0; p0 < NP; p0 += G) {
    const int pi = p0 + g;
    if (pi < NP) c2r_acc<L>(t, twr, pair(pi / (NR / 2), pi % (NR / 2)));  // whole groups
  }
  __syncthreads();
  // value of channel ch, tile row ly, column z
  auto val = [&](int ch, int ly, int z) {
    const float2 f = pair(ch, ly >> 1)(z);
    return (ly & 1) ? f.y : f.x;
  };
  if constexpr (NCH == 1) {
    float* chi = S.chi;
    for (int i = tid; i < YB * L / 4; i += NT) {
      const int ly = i / (L / 4), z4 = (i % (L / 4)) * 4;
      float4 o;
      o.x = fmaf(a_chi, val(0, ly, z4), b_chi);
      o.y = fmaf(a_chi, val(0, ly, z4 + 1), b_chi);
      o.z = fmaf(a_chi, val(0, ly, z4 + 2), b_chi);
      o.w = fmaf(a_chi, val(0, ly, z4 + 3), b_chi);
      reinterpret_cast<float4*>(chi + ((size_t)X * L + y0 + ly) * L)[z4 / 4] = o;
    }
  }
  for (int v = tid; v < nv; v += NT) {
    const int side = v < n0 ? 0 : 1;
    const int i = side ? r1.x + (v - n0) : r0.x + v;
    if (!dbg_in_range(S.status, i, S.N)) continue;
    {
      const float4 a = v == tid ? pa : S.sorted[2 * i];
      const float4 b = v == tid ? pb : S.sorted[2 * i + 1];
      const Axis ax = axis_rec(a.x, b.w, 0, L), ay = axis_rec(a.y, b.w, 1, L), az = axis_rec(a.z, b.w, 2, L);
      const int ly0 = ay.i0 - y0;  // in [0, YB); row i1 is ly0 + 1 (a halo row at most)
      const float fx = tri_w(side, ax.t), dfx = side ? (float)L : -(float)L;
      if constexpr (NCH == 1) {
        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const float fy = tri_w(dy, ay.t), dfy = dy ? (float)L : -(float)L;
#pragma unroll
          for (int dz = 0; dz < 2; ++dz) {
            const int z = dz ? az.i1 : az.i0;
            const float fz = tri_w(dz, az.t), dfz = dz ? (float)L : -(float)L;
            const float vv = val(0, ly0 + dy, z);
            gx += dfx * fy * fz * vv;
            gy += fx * dfy * fz * vv;
            gz += fx * fy * dfz * vv;
          }
        }
        S.gfwd[(size_t)side * S.N + i] = make_float4(gx, gy, gz, 0.f);
      } else {
        const float n0_ = a.w, n1 = b.x, n2 = b.y;
        float nb0 = 0.f, nb1 = 0.f, nb2 = 0.f, cb0 = 0.f, cb1 = 0.f, cb2 = 0.f;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const float fy = tri_w(dy, ay.t), dfy = dy ? (float)L : -(float)L;
#pragma unroll
          for (int dz = 0; dz < 2; ++dz) {
            const int z = dz ? az.i1 : az.i0;
            const float fz = tri_w(dz, az.t), dfz = dz ? (float)L : -(float)L;
            const float vx = val(0, ly0 + dy, z), vy = val(1, ly0 + dy, z), vz = val(2, ly0 + dy, z);
            const float w = fx * fy * fz;
            nb0 += w * vx;
            nb1 += w * vy;
            nb2 += w * vz;
            const float sdot = n0_ * vx + n1 * vy + n2 * vz;
            cb0 += dfx * fy * fz * sdot;
            cb1 += fx * dfy * fz * sdot;
            cb2 += fx * fy * dfz * sdot;
          }
        }
        float* o = S.slots + ((size_t)side * S.N + i) * 6;
        o[0] = nb0;
        o[1] = nb1;
        o[2] = nb2;
        o[3] = cb0;
        o[4] = cb1;
        o[5] = cb2;
      }
    }
  }
  fence_async_smem();  // this stage is refilled by a bulk copy later
  __syncthreads();
  return true;
}

template <int L, int NCH>
__global__ void __launch_bounds__(ZiGeo<L, NCH>::NT, L >= 512 ? 1 : (NCH == 1 ? 4 : (L >= 256 ? 2 : 3)))
    k_zinv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = Pen<L>;
  using Z = ZiGeo<L, NCH>;
  constexpr int NT = Z::NT;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int tid = threadIdx.x;
  extern __shared__ float4 smem4[];
  float2* stg = reinterpret_cast<float2*>(smem4);  // 2 stages, row (ch, ly) at row_off(ch NR + ly)
  float2* twt = stg + 2 * Z::STAGE;
  __shared__ uint64_t bar[2];
  pdl_trigger();
  for (int i = tid; i < L; i += NT) twt[i] = S.tw[i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_wait();
  __syncthreads();
  constexpr int ntiles = L * P::NYB;
  float a_chi = 0.f, b_chi = 0.f;
  if constexpr (NCH == 1) {
    a_chi = S.sc->a_chi;
    b_chi = S.sc->b_chi;
  }
  uint32_t ph = 0u;  // bit st: parity of stage st's next completion
  int tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) zinv_issue<L, NCH>(S, tile, stg, &bar[0]);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int st = it & 1;
    const int next = tile + gridDim.x;
    // released at the end of the last iteration
    if (tid == 0 && next < ntiles) zinv_issue<L, NCH>(S, next, stg + (st ^ 1) * Z::STAGE, &bar[st ^ 1]);
    bool ok = zinv_tile<L, NCH>(S, tile, stg + st * Z::STAGE, twt, a_chi, b_chi, [&]() {
      const bool landed = __syncthreads_and(mbar_wait(&bar[st], (ph >> st) & 1u));
      ph ^= 1u << st;
      return landed;
    });
    if (!ok) {
      if (tid == 0) {
        atomicOr(S.status, kStTimeout);
        if (next < ntiles) mbar_wait(&bar[st ^ 1], (ph >> (st ^ 1)) & 1u);  // the prefetch, bounded
      }
      break;
    }
  }
}

// ===========================================================================
// Backward z pass over tiles of ZB rows: the sums S = sum dchi and
// sum dchi * chi (per-CTA partials, reduced by the last CTA into the adjoint
// scalars) and the R2C along z of dchi -> kSpD. Persistent CTAs, each loading
// the next tile's dchi and chi rows by bulk copies while it transforms the
// current one. The pass reads no points, so its tile height is free: two
// rows per FFT group, every group busy.
// ===========================================================================
template <int L>
struct ZbGeo {
  static constexpr int NT = 128, G = NT / Shape<L>::T;
  static constexpr int ZB = 2 * G < L ? 2 * G : L;  // rows per tile
};

template <int L>
constexpr size_t zbfwd_smem() {
  return sizeof(float) * 2 * (pairs_floats<L>(ZbGeo<L>::ZB / 2) + ZbGeo<L>::ZB * L) + sizeof(float2) * L;
}

template <int L>
__global__ void __launch_bounds__(ZbGeo<L>::NT, L >= 512 ? 1 : 3) k_zbfwd(const __grid_constant__ Solve s0,
                                                          const Solve* __restrict__ tab) {
  using P = Pen<L>;
  constexpr int YB = ZbGeo<L>::ZB, H = P::H, NT = ZbGeo<L>::NT, ZG = ZbGeo<L>::G;
  constexpr int DF = pairs_floats<L>(YB / 2);
  constexpr int STAGE = DF + YB * L;  // floats: dchi (row pairs, pair_off), chi
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ float4 smem4[];
  float* stg = reinterpret_cast<float*>(smem4);
  float2* twt = reinterpret_cast<float2*>(stg + 2 * STAGE);
  __shared__ uint64_t bar[2];
  pdl_trigger();
  for (int i = tid; i < L; i += NT) twt[i] = S.tw[i];
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_wait();
  __syncthreads();
  constexpr int ntiles = L * (L / YB);
  constexpr uint32_t kRowBytes = YB * L * sizeof(float);
  auto issue = [&](int tile, int st) {  // thread 0: dchi and chi rows of the tile
    const size_t row0 = (size_t)tile * YB * L;  // tiles are consecutive blocks of rows
    mbar_expect_tx(&bar[st], 2 * kRowBytes);
    for (int q = 0; q < YB / 2; ++q)
      bulk_load(stg + st * STAGE + pair_off<L>(q), S.dchi + row0 + 2 * q * L,
                2 * L * (uint32_t)sizeof(float), &bar[st]);
    bulk_load(stg + st * STAGE + DF, S.chi + row0, kRowBytes, &bar[st]);
  };
  TwTab<L> twr{twt, t};
  FF dS = {0.f, 0.f}, dD = {0.f, 0.f};  // float-float over the CTA's tiles
  uint32_t ph = 0u;
  int tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue(tile, 0);
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int st = it & 1;
    const int next = tile + gridDim.x;
    if (tid == 0 && next < ntiles) issue(next, st ^ 1);  // stage st ^ 1 was released last tile
    const bool ok = __syncthreads_and(mbar_wait(&bar[st], (ph >> st) & 1u));
    ph ^= 1u << st;
    if (!ok) {
      if (tid == 0) {
        atomicOr(S.status, kStTimeout);
        if (next < ntiles) mbar_wait(&bar[st ^ 1], (ph >> (st ^ 1)) & 1u);
      }
      break;
    }
    float* rows = stg + st * STAGE;  // dchi row pairs, then chi rows
    const float4* c4 = reinterpret_cast<const float4*>(rows + DF);
    float accS = 0.f, accD = 0.f;
    for (int i = tid; i < YB * L / 4; i += NT) {
      const int q = i / (L / 2), w = i % (L / 2);  // pair, float4 within the pair
      const float4 a = *reinterpret_cast<const float4*>(rows + pair_off<L>(q) + 4 * w), b = c4[i];
      accS += (a.x + a.y) + (a.z + a.w);
      accD += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    }
    dS = ff_add(dS, accS);
    dD = ff_add(dD, accD);
    __syncthreads();  // the sums have read the rows before the R2C rewrites them
    {
      const int X = tile / (L / YB), y0 = (tile % (L / YB)) * YB;
      for (int p0 = 0; p0 < YB / 2; p0 += ZG) {
        const int pi = p0 + g;
        if (pi < YB / 2) {  // whole groups; the packed rows go straight to global memory
          float2* ga = S.spec[kSpD] + ((size_t)X * L + y0 + 2 * pi) * P::KP;
          r2c_pair_st<L>(t, twr, rows + pair_off<L>(pi), nullptr, ga, ga + P::KP);
        }
      }
    }
    // every thread is done with this stage before a bulk copy refills it
    fence_async_smem();
    __syncthreads();
  }
  // this CTA's partial sums, fixed order; the last CTA finalises
  block_sum_ff<NT>(dS, dD);
  last_block_finalize<NT>(S, 1, (int)gridDim.x, (int)blockIdx.x, dS, dD, true);
}

// ---------------------------------------------------------------------------
// Launchers: kind 0 forward (z, y), 1 inverse (y, z), 2 backward (z, y),
// 3 adjoint (y, z).
// ---------------------------------------------------------------------------
template <class K>
static cudaError_t set_smem(K fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int L>
static cudaError_t launch_pencil_t(int kind, const Solve& s, const Solve* tab, int count,
                                   cudaStream_t st) {
  using P = Pen<L>;
  const dim3 gz(L * P::NYB, 1, count), gy(L * P::NKC, 1, count);
  static bool attr_set[4] = {false, false, false, false};
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case 0: {
      constexpr size_t a = zfwd_smem<L>(), b = yfwd_smem<L, false>();
      if (!attr_set[0]) {
        e = set_smem(k_zfwd<L>, a);
        if (e == cudaSuccess) e = set_smem(k_yfwd<L, false>, b);
        if (e != cudaSuccess) return e;
        attr_set[0] = true;
      }
      e = launch_k(k_zfwd<L>, gz, dim3(P::ZNT), a, st, 0, s, tab);
      if (e == cudaSuccess)
        e = launch_k(k_yfwd<L, false>, dim3(L * P::NKC, yfwd_merge<L>() ? 2 : 3, count), dim3(ynt<L>()),
                     b, st, 0, s, tab);
      return e;
    }
    case 1: {
      constexpr size_t a = yinv_smem<L, 1>(), b = zinv_smem<L, 1>();
      constexpr int nt = 16 * P::T >= 32 ? 16 * P::T : 32;
      static int nz = 0;
      if (!attr_set[1]) {
        e = set_smem(k_yinv<L, 1>, a);
        if (e == cudaSuccess) e = set_smem(k_zinv<L, 1>, b);
        if (e != cudaSuccess) return e;
        nz = persistent_ctas(k_zinv<L, 1>, ZiGeo<L, 1>::NT, b, L * P::NYB, 1);
        attr_set[1] = true;
      }
      e = launch_k(k_yinv<L, 1>, gy, dim3(nt), a, st, 0, s, tab);
      if (e == cudaSuccess)
        e = launch_k(k_zinv<L, 1>, dim3(nz, 1, count), dim3(ZiGeo<L, 1>::NT), b, st, 0, s, tab);
      return e;
    }
    case 2: {
      constexpr size_t a = zbfwd_smem<L>(), b = yfwd_smem<L, true>();
      static int nz = 0;
      if (!attr_set[2]) {
        e = set_smem(k_zbfwd<L>, a);
        if (e == cudaSuccess) e = set_smem(k_yfwd<L, true>, b);
        if (e != cudaSuccess) return e;
        nz = persistent_ctas(k_zbfwd<L>, ZbGeo<L>::NT, a, L * (L / ZbGeo<L>::ZB), 1);
        attr_set[2] = true;
      }
      e = launch_k(k_zbfwd<L>, dim3(nz, 1, count), dim3(ZbGeo<L>::NT), a, st, 0, s, tab);
      if (e == cudaSuccess) e = launch_k(k_yfwd<L, true>, gy, dim3(ynt<L>()), b, st, 0, s, tab);
      return e;
    }
    default: {
      constexpr size_t a = yinv_smem<L, 3>(), b = zinv_smem<L, 3>();
      constexpr int nt = 16 * P::T >= 32 ? 16 * P::T : 32;
      static int nz = 0;
      if (!attr_set[3]) {
        e = set_smem(k_yinv<L, 3>, a);
        if (e == cudaSuccess) e = set_smem(k_zinv<L, 3>, b);
        if (e != cudaSuccess) return e;
        nz = persistent_ctas(k_zinv<L, 3>, ZiGeo<L, 3>::NT, b, L * P::NYB, 1);
        attr_set[3] = true;
      }
      e = launch_k(k_yinv<L, 3>, dim3(L * P::NKC, yinv_split<L, 3>() ? 2 : 1, count), dim3(nt), a, st, 0,
                   s, tab);
      if (e == cudaSuccess)
        e = launch_k(k_zinv<L, 3>, dim3(nz, 1, count), dim3(ZiGeo<L, 3>::NT), b, st, 0, s, tab);
      return e;
    }
  }
}

cudaError_t launch_pencil(int kind, int r, const Solve& s, const Solve* tab, int count,
                          cudaStream_t st) {
  switch (r) {
    case 8: return launch_pencil_t<8>(kind, s, tab, count, st);
    case 16: return launch_pencil_t<16>(kind, s, tab, count, st);
    case 32: return launch_pencil_t<32>(kind, s, tab, count, st);
    case 64: return launch_pencil_t<64>(kind, s, tab, count, st);
    case 128: return launch_pencil_t<128>(kind, s, tab, count, st);
    case 256: return launch_pencil_t<256>(kind, s, tab, count, st);
    case 512: return launch_pencil_t<512>(kind, s, tab, count, st);
    default: return cudaErrorInvalidValue;
  }
}

// Largest dynamic shared memory of the two kernels of a kind (for the tuner).
size_t pencil_smem_bytes(int kind, int r) {
  auto pick = [&](auto Lc) -> size_t {
    constexpr int L = decltype(Lc)::value;
    size_t a = 0, b = 0;
    switch (kind) {
      case 0: a = zfwd_smem<L>(); b = yfwd_smem<L, false>(); break;
      case 1: a = yinv_smem<L, 1>(); b = zinv_smem<L, 1>(); break;
      case 2: a = zbfwd_smem<L>(); b = yfwd_smem<L, true>(); break;
      default: a = yinv_smem<L, 3>(); b = zinv_smem<L, 3>(); break;
    }
    return a > b ? a : b;
  };
  switch (r) {
    case 8: return pick(std::integral_constant<int, 8>{});
    case 16: return pick(std::integral_constant<int, 16>{});
    case 32: return pick(std::integral_constant<int, 32>{});
    case 64: return pick(std::integral_constant<int, 64>{});
    case 128: return pick(std::integral_constant<int, 128>{});
    case 256: return pick(std::integral_constant<int, 256>{});
    case 512: return pick(std::integral_constant<int, 512>{});
    default: return 0;
  }
}

}  // namespace dpsr
