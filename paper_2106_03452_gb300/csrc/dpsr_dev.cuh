// Device-side building blocks of libdpsr: complex arithmetic, small DFTs in
// registers, the group FFT used by every pass, the per-solve descriptor and
// the trilinear stencil of the point rasterization (Eq. A1).
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dpsr {
namespace cg = cooperative_groups;

constexpr int kNT = 256;  // threads of the plane kernels
constexpr float kM = 0.5f;  // m of Eq. 2

// ---------------------------------------------------------------------------
// Programmatic dependent launch. Every kernel of a solve lets the next kernel
// of its stream be scheduled once all of its own CTAs are resident
// (pdl_trigger, first thing), and waits for the previous kernel to complete
// and its memory to be visible (pdl_wait) before it reads or writes anything
// that kernel produced or consumed; only plan-constant tables (twiddles,
// frequencies) and shared memory are touched before. Both are no-ops for a
// kernel launched without the programmatic attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (i u) for real u
__device__ __forceinline__ float2 cmul_iu(float2 a, float u) { return make_float2(-a.y * u, a.x * u); }
__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// ---------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------
template <int I, int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor<I + 1, N>(f);
  }
}

// cos / sin of 2*pi*q/16: the sixteenth roots of unity.
__host__ __device__ constexpr float cos16(int q) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f,
                  h = 0.70710678118654752440f;
  switch (q & 15) {
    case 0: return 1.f;   case 1: return c1;  case 2: return h;   case 3: return s1;
    case 4: return 0.f;   case 5: return -s1; case 6: return -h;  case 7: return -c1;
    case 8: return -1.f;  case 9: return -c1; case 10: return -h; case 11: return -s1;
    case 12: return 0.f;  case 13: return s1; case 14: return h;  default: return c1;
  }
}
__host__ __device__ constexpr float sin16(int q) { return cos16(q - 4); }

// a * exp(DIR * 2 pi i q / 16), with the trivial factors folded at compile time.
template <int Q, int DIR>
__device__ __forceinline__ float2 twc(float2 a) {
  constexpr int q = ((Q % 16) + 16) % 16;
  if constexpr (q == 0) {
    return a;
  } else if constexpr (q == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (q == 4 || q == 12) {
    constexpr float s = DIR * sin16(q);  // +-1
    return make_float2(-a.y * s, a.x * s);
  } else if constexpr ((q & 3) == 2) {
    constexpr float c = cos16(q), s = DIR * sin16(q);  // |c| == |s|
    const float p = (c == s) ? (a.x - a.y) : (a.x + a.y);
    const float m = (c == s) ? (a.x + a.y) : (a.y - a.x);
    return make_float2(p * c, m * c);
  } else {
    constexpr float c = cos16(q), s = DIR * sin16(q);
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// cos / sin of 2*pi*q/32 for odd q: cos(k pi / 16), k = 1, 3, 5, 7 and
// their reflections (the even q are the sixteenth roots above).
__host__ __device__ constexpr float cos32_odd(int q) {
  constexpr float c1 = 0.98078528040323044913f, c3 = 0.83146961230254523708f,
                  c5 = 0.55557023301960222474f, c7 = 0.19509032201612826785f;
  switch (q & 31) {
    case 1: return c1;   case 3: return c3;   case 5: return c5;   case 7: return c7;
    case 9: return -c7;  case 11: return -c5; case 13: return -c3; case 15: return -c1;
    case 17: return -c1; case 19: return -c3; case 21: return -c5; case 23: return -c7;
    case 25: return c7;  case 27: return c5;  case 29: return c3;  default: return c1;  // 31
  }
}
__host__ __device__ constexpr float sin32_odd(int q) { return cos32_odd((q - 8) & 31); }

// a * exp(DIR * 2 pi i q / 32).
template <int Q, int DIR>
__device__ __forceinline__ float2 twc32(float2 a) {
  constexpr int q = ((Q % 32) + 32) % 32;
  if constexpr ((q & 1) == 0) {
    return twc<q / 2, DIR>(a);
  } else {
    constexpr float c = cos32_odd(q), s = DIR * sin32_odd(q);
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// In-register DFT of E points (E = 1, 2, 4, 8, 16, 32), natural order in and
// out, exponent sign DIR (-1 forward, +1 inverse), unnormalised. Radix-2
// decimation in time, fully unrolled.
template <int E, int DIR>
struct Dft {
  static __device__ __forceinline__ void run(float2* v) {
    float2 ev[E / 2], od[E / 2];
    sfor<0, E / 2>([&](auto i) {
      ev[i] = v[2 * i];
      od[i] = v[2 * i + 1];
    });
    Dft<E / 2, DIR>::run(ev);
    Dft<E / 2, DIR>::run(od);
    sfor<0, E / 2>([&](auto k) {
      constexpr int q = decltype(k)::value * (32 / E);
      const float2 t = twc32<q, DIR>(od[k]);
      v[k] = cadd(ev[k], t);
      v[k + E / 2] = csub(ev[k], t);
    });
  }
};
template <int DIR>
struct Dft<1, DIR> {
  static __device__ __forceinline__ void run(float2*) {}
};

// Synchronise the T lanes of this thread's group (aligned groups of T lanes
// within a warp); a one-thread group needs no synchronisation. Groups may
// therefore call the FFT helpers independently of the rest of their warp.
//
// Interleaved lanes (IL, used with T = 16 only): the two groups of a warp
// share both half-warps, 8 lanes each (see Lanes), and synchronise on their
// own 16 lanes.
template <int T, bool IL = false>
__device__ __forceinline__ void group_sync() {
  if constexpr (IL && T == 16) {
    __syncwarp(0x00FF00FFu << (threadIdx.x & 8u));
  } else if constexpr (T >= 32) {
    __syncwarp();
  } else if constexpr (T > 1) {
    const unsigned lane = threadIdx.x & 31u;
    __syncwarp(((1u << T) - 1u) << (lane & ~(unsigned)(T - 1)));
  }
}

// ---------------------------------------------------------------------------
// Group FFT of length L by T threads, each holding R1 = L / T values.
// Distribution (in and out): thread t holds element t + T*j in v[j].
// Two Cooley-Tukey stages L = R1 * T: an R1-point DFT per thread over the
// stride-T subsequence, a twiddle W_L^(t*k1), an exchange through shared
// memory (XOR-swizzled so neither side conflicts), and T-point DFTs.
// tw[m] = exp(-2 pi i m / L), m < L (FP64-computed, rounded to FP32).
// xch: L float2 of shared memory owned by the group. Every lane of the warp
// must call this together (they synchronise through group_sync).
// ---------------------------------------------------------------------------
// Group and lane-in-group of thread tid. Contiguous: group g holds lanes
// [g T, g T + T) of its warp. Interleaved (T = 16): group 2w + h of warp w
// holds lanes 8h..8h+7 and 16+8h..16+8h+7, thread t = (lane & 7) | (lane >> 4) << 3.
// A group that reads one column of a 128-byte-swizzled box (rows of 16
// float2) reaches only 16 of the 32 banks, so a half-warp of one group needs
// two wavefronts per access; with the lanes interleaved each half-warp holds
// 8 rows of two adjacent columns (groups 2w, 2w + 1), all 32 banks.
template <int T, bool IL>
struct Lanes {
  static constexpr bool kIL = IL && T == 16;
  static __device__ __forceinline__ int group(int tid) {
    if constexpr (kIL) return 2 * (tid >> 5) + ((tid >> 3) & 1);
    else return tid / T;
  }
  static __device__ __forceinline__ int lane(int tid) {
    if constexpr (kIL) return (tid & 7) | (((tid >> 4) & 1) << 3);
    else return tid % T;
  }
};

template <int L> struct Shape;
template <> struct Shape<8>   { static constexpr int R1 = 8,  T = 1; };
template <> struct Shape<16>  { static constexpr int R1 = 16, T = 1; };
template <> struct Shape<32>  { static constexpr int R1 = 8,  T = 4; };
template <> struct Shape<64>  { static constexpr int R1 = 8,  T = 8; };
template <> struct Shape<128> { static constexpr int R1 = 16, T = 8; };
template <> struct Shape<256> { static constexpr int R1 = 16, T = 16; };
template <> struct Shape<512> { static constexpr int R1 = 32, T = 16; };

// Rows of a TMA box along a transform axis: the whole axis up to r = 256;
// at r = 512 (above the 256-element limit of a box dimension) two boxes of
// 256 rows, placed one after the other in shared memory (both start on a
// 1024-byte boundary, so the 128-byte swizzle runs on unchanged).
__host__ __device__ constexpr int tma_rows(int r) { return r < 256 ? r : 256; }

template <int L, int DIR, class XA>
__device__ __forceinline__ void fft_x(float2 (&v)[Shape<L>::R1], int t, XA xa, const float2* tw) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  if constexpr (T == 1) {
    Dft<L, DIR>::run(v);
  } else {
    Dft<R1, DIR>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      float2 w = tw[t * k1];
      if (DIR > 0) w.y = -w.y;
      v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) xa(k1 * T + (t ^ (k1 % T))) = v[k1];
    group_sync<T>();
    constexpr int M = R1 / T;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float2 u[T];
      const int k1 = t + T * m;
#pragma unroll
      for (int n2 = 0; n2 < T; ++n2) u[n2] = xa(k1 * T + (n2 ^ t));
      Dft<T, DIR>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < T; ++k2) v[m + M * k2] = u[k2];
    }
    group_sync<T>();
  }
}

template <int L, int DIR>
__device__ __forceinline__ void fft(float2 (&v)[Shape<L>::R1], int t, float2* xch,
                                    const float2* tw) {
  fft_x<L, DIR>(v, t, [xch](int i) -> float2& { return xch[i]; }, tw);
}

// The stage twiddles W_L^(t*k1), k1 = 1..R1-1, of thread t held in registers
// (the same for every transform the thread performs).
template <int L>
struct Twid {
  float2 w[Shape<L>::R1];
  __device__ __forceinline__ void load(int t, const float2* tw) {
#pragma unroll
    for (int k1 = 0; k1 < Shape<L>::R1; ++k1)
      w[k1] = Shape<L>::T == 1 ? make_float2(1.f, 0.f) : tw[(t * k1) & (L - 1)];
  }
  __device__ __forceinline__ float2 operator()(int k1) const { return w[k1]; }
};

// The same stage twiddles read from a shared-memory table at each use
// (fewer live registers than Twid).
template <int L>
struct TwTab {
  const float2* tab;  // exp(-2 pi i m / L), m < L, in shared memory
  int t;
  __device__ __forceinline__ float2 operator()(int k1) const { return tab[(t * k1) & (L - 1)]; }
};

// Group FFT with register twiddles (see fft_x).
template <int L, int DIR, bool IL = false, class XA, class TW>
__device__ __forceinline__ void fft_r(float2 (&v)[Shape<L>::R1], int t, XA xa, const TW& tw) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  if constexpr (T == 1) {
    Dft<L, DIR>::run(v);
  } else {
    Dft<R1, DIR>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      float2 w = tw(k1);
      if (DIR > 0) w.y = -w.y;
      v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) xa(k1 * T + (t ^ (k1 % T))) = v[k1];
    group_sync<T, IL>();
    constexpr int M = R1 / T;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float2 u[T];
      const int k1 = t + T * m;
#pragma unroll
      for (int n2 = 0; n2 < T; ++n2) u[n2] = xa(k1 * T + (n2 ^ t));
      Dft<T, DIR>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < T; ++k2) v[m + M * k2] = u[k2];
    }
    group_sync<T, IL>();
  }
}

// ---------------------------------------------------------------------------
// Real <-> half-complex pairs. Two real rows a, b of length L are packed as
// z = a + i b and transformed together. Half spectra are stored "packed":
// slot 0 holds (A[0], A[L/2]) (both real for a real row), slots 1..L/2-1 hold
// A[1..L/2-1].
// ---------------------------------------------------------------------------
// Forward: ld(k) -> z[k]; sa(slot, A), sb(slot, B).
template <int L, class Tw, class Ld, class StA, class StB>
__device__ __forceinline__ void r2c_pair(int t, float2* xch, const Tw& tw, Ld ld, StA sa,
                                         StB sb) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T, H = L / 2;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = ld(t + T * j);
  fft_r<L, -1>(v, t, [xch](int i) -> float2& { return xch[i]; }, tw);
#pragma unroll
  for (int j = 0; j < R1; ++j) xch[t + T * j] = v[j];
  group_sync<T>();
  float2 A[R1 / 2], B[R1 / 2];
#pragma unroll
  for (int j = 0; j < R1 / 2; ++j) {
    const int k = t + T * j;
    if (k == 0) {
      const float2 z0 = xch[0], zn = xch[H];
      A[j] = make_float2(z0.x, zn.x);
      B[j] = make_float2(z0.y, zn.y);
    } else {
      const float2 zk = xch[k], zm = cconj(xch[L - k]);
      A[j] = cscale(cadd(zk, zm), 0.5f);
      const float2 d = csub(zk, zm);  // B = -i d / 2
      B[j] = make_float2(0.5f * d.y, -0.5f * d.x);
    }
  }
  group_sync<T>();
#pragma unroll
  for (int j = 0; j < R1 / 2; ++j) {
    sa(t + T * j, A[j]);
    sb(t + T * j, B[j]);
  }
}

// Inverse: la(slot) -> packed A, lb(slot) -> packed B; st(z, (a[z], b[z]))
// with the unnormalised inverse transform (values times L).
template <int L, class Tw, class LdA, class LdB, class St>
__device__ __forceinline__ void c2r_pair(int t, float2* xch, const Tw& tw, LdA la, LdB lb,
                                         St st) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T, H = L / 2;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    const int k = t + T * j;
    if (k == 0 || k == H) {
      const float2 a = la(0), b = lb(0);
      v[j] = (k == 0) ? make_float2(a.x, b.x) : make_float2(a.y, b.y);
    } else if (k < H) {
      const float2 a = la(k), b = lb(k);
      v[j] = make_float2(a.x - b.y, a.y + b.x);
    } else {
      const float2 a = la(L - k), b = lb(L - k);
      v[j] = make_float2(a.x + b.y, b.x - a.y);
    }
  }
  fft_r<L, +1>(v, t, [xch](int i) -> float2& { return xch[i]; }, tw);
#pragma unroll
  for (int j = 0; j < R1; ++j) st(t + T * j, v[j]);
}

// Separate a packed column P = X0 + i Xn of two spectra whose inverse is real:
// X0[k] = (P[k] + conj(P[-k])) / 2, Xn[k] = -i (P[k] - conj(P[-k])) / 2.
__device__ __forceinline__ void unpack_dc_nyq(float2 pk, float2 pm, float2& x0, float2& xn) {
  const float2 cm = cconj(pm);
  x0 = cscale(cadd(pk, cm), 0.5f);
  const float2 d = csub(pk, cm);
  xn = make_float2(0.5f * d.y, -0.5f * d.x);
}

// ---------------------------------------------------------------------------
// Per-solve descriptor. All pointers are device pointers.
// ---------------------------------------------------------------------------
struct Scalars {
  double acc_mu, acc_s0;  // spectral sums of the forward pass
  double mu, s, alpha;    // Eq. 4
  double S, D, s_bar, mu_bar;
  float a_chi, b_chi;     // chi = a_chi * y + b_chi, y = unnormalised inverse FFT
  float g_a, g_s, g_w;    // backward: G^ = g_a * FFT(dchi) + g_s + g_w * W^
  float c_mu;             // backward: weight of the stored lookup gradient
  double loss;            // L_DPSR of Eq. 9 (mean squared error against a target grid)
  // arrival counters of the last-block reductions: [0] forward x-pass,
  // [1] backward plane pass, [2] the L_DPSR loss (all reset by the binning's
  // scatter of every forward, and each by its own last block)
  unsigned ticket[3];
};

// Spectral buffers of a solve (Solve::spec) and what they hold between the
// passes (complex [x][ky][kz], kz pitch r/2 + 2):
//   kSpD   forward D; backward FFT_zy(dchi), then Q1 = IFFT_x(F)
//   kSpChi forward chi~ after the x-pass; backward Q2 = IFFT_x(-i u_x F)
//   kSpC   forward C; adjoint (pencil) V_bar_x
//   kSpW   W~, kept from the forward for every backward
//   kSpYa  pencil: y-domain chi~; adjoint V_bar_y
//   kSpYb  pencil: adjoint V_bar_z
// The pencil forward holds v_y, i u_z v_z, v_x, w (y-domain) in buffers
// 0..3 before its y pass.
constexpr int kSpD = 0, kSpChi = 1, kSpC = 2, kSpW = 3, kSpYa = 4, kSpYb = 5;
constexpr int kNSpec = 6;

struct Solve {
  // TMA descriptors of the spectral buffers (dims kz = r/2+1, ky, x): tmx
  // boxes are 16 kz x 1 ky x r x (x-pass tiles), tmy boxes 16 kz x r ky x
  // 1 x (plane tiles). 128-byte swizzle.
  CUtensorMap tmx[kNSpec];
  CUtensorMap tmy[kNSpec];
  int r;
  int N;
  double inv_N;  // 1 / N (set with N by set_count)
  // A periodic box of side lengths L (voxel size L_d / r along axis d, Eq.
  // A1 with a per-axis s): the binning finds each point's cell and in-cell
  // fraction from c r / L_d in FP64 (box), the combine turns unit-cube
  // gradients into box ones (times 1 / L_d, inv_box).
  float inv_box[3] = {1.f, 1.f, 1.f};
  double box[3] = {1.0, 1.0, 1.0};
  double gscale[3] = {0.0, 0.0, 0.0};  // r / L_d, set with r (set_grid)
  // per call (caller-owned)
  const float* points;
  const float* normals;
  float* chi;
  const float* dchi;
  float* dpoints;
  float* dnormals;
  const float* target;  // L_DPSR target grid (r^3), and where its gradient goes
  float* dchi_rw;
  // plan workspace
  float4* sorted;   // 2 records per point: (tx, ty, tz, nx), (ny, nz, orig, cells) (see axis_rec)
  int* cellx;       // N
  int* bins;        // count[r*r], off[r*r + 1], cursor[r*r] (see nbins)
  float2* spec[kNSpec];  // r * r * (r/2 + 2) complex each
  float4* gfwd;     // [2][N]: gradient of the lookup of y, per plane side
  float* slots;     // [2][N][6]: backward partials per plane side
  float4* part;     // per-block partial sums, float-float pairs (a.hi, a.lo, b.hi, b.lo)
  Scalars* sc;
  unsigned* status;
  const float2* tw;  // r
  // Spectral tables, indexed by the integer frequency index k of an axis
  // (f = k below r/2, k - r above, |f| = r/2 at Nyquist):
  const float* g1;   // r: exp(-2 sigma^2 f^2 / r^2), the same on every axis
  const float* u2;   // 3 x r, axis-major: (f / L_d)^2
  const float* iu;   // 3 x r, axis-major: f / L_d, 0 at Nyquist (spectral derivative)
};

// Host side: the spectral tables of one plan, computed in FP64 and rounded
// to FP32. tw[r]: twiddles exp(-2 pi i m / r); tab[7r]: g1 (r), u2 (3r) and
// iu (3r) as laid out in Solve. box: side lengths L_d (nullptr: unit cube).
inline void spectral_tables(int r, double sigma, const double* box, float2* tw, float* tab) {
  const double pi = 3.14159265358979323846264338327950288;
  for (int m = 0; m < r; ++m) {
    const double ang = -2.0 * pi * (double)m / (double)r;
    tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    const double f = m < r / 2 ? (double)m : (m == r / 2 ? (double)(r / 2) : (double)(m - r));
    tab[m] = (float)exp(-2.0 * sigma * sigma * f * f / ((double)r * r));
    for (int d = 0; d < 3; ++d) {
      const double u = f / (box ? box[d] : 1.0);
      tab[(1 + d) * r + m] = (float)(u * u);
      tab[(4 + d) * r + m] = m == r / 2 ? 0.f : (float)u;
    }
  }
}

enum : unsigned { kStBadInput = 1u, kStDegenerate = 2u, kStTimeout = 4u, kStBounds = 8u };

// Debug builds (-DDPSR_DEBUG_CHECKS) check each data-dependent index of the
// point kernels (bin keys, sorted positions, point indices read from the
// bins) before it is used: an index outside [0, n) sets kStBounds in the
// status word (reported as DPSR_EBOUNDS) and its access is skipped, so a
// broken invariant shows up as a status instead of a stray access. Release
// builds compile the checks away.
#ifdef DPSR_DEBUG_CHECKS
__device__ __forceinline__ bool dbg_in_range(unsigned* status, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(status, kStBounds);
  return false;
}
#else
__device__ __forceinline__ bool dbg_in_range(unsigned*, long long, long long) { return true; }
#endif

// The grid size of a solve and its per-axis scales r / L_d (host side).
inline void set_grid(Solve& s, int r) {
  s.r = r;
  for (int d = 0; d < 3; ++d) s.gscale[d] = (double)r / s.box[d];
}

// The point count of a solve and its reciprocal (used by the scalar pass).
inline void set_count(Solve& s, int64_t N) {
  s.N = (int)N;
  s.inv_N = 1.0 / (double)N;
}

// Row pitch (complex values) of the spectral buffers along kz: the r/2 + 1
// valid slots padded so that, from r = 32 on, every row starts on a 128-byte
// line (the 16-slot tiles of the plane and x passes are then one line each).
__host__ __device__ constexpr int kpitch(int r) { return r / 2 < 16 ? r / 2 + 2 : r / 2 + 16; }

// Trilinear stencil along one axis (Eq. A1, floor cell, periodic wrap):
// x~ = c r (exact for r a power of two), i0 = floor(x~) mod r, t = x~ - floor(x~).
// Point bins: a counting sort of the points by the x-cell of their stencil
// origin and the block of ybin(r) y-rows its y-cell falls in, key
// x * nybins(r) + y / ybin(r), so that the points of an x-plane, and of a
// block of y-rows within it, are contiguous. S.bins holds count[nbins],
// off[nbins + 1] (exclusive prefix sums) and cur[nbins] (scatter cursors).
__host__ __device__ constexpr int ybin(int r) { return r < 16 ? r : 16; }
__host__ __device__ constexpr int nybins(int r) { return r / ybin(r); }
__host__ __device__ constexpr int nbins(int r) { return r * nybins(r); }
__host__ __device__ constexpr size_t bins_ints(int r) { return 3 * (size_t)nbins(r) + 1; }

// Clear the bin counts and scatter cursors of a solve for its next forward
// pass, spread over the calling grid (block bid of nblocks). Run by a kernel
// that follows the scatter in stream order and reads neither array: the
// forward x-pass.
__device__ __forceinline__ void clear_bin_counters(const Solve& S, int bid, int nblocks) {
  const int nb = nbins(S.r);
  int* count = S.bins;
  int* cur = S.bins + 2 * nb + 1;
  for (int i = bid * (int)blockDim.x + (int)threadIdx.x; i < nb; i += nblocks * (int)blockDim.x) {
    count[i] = 0;
    cur[i] = 0;
  }
}

struct Axis {
  int i0, i1;
  float t;
};
__device__ __forceinline__ Axis axis_of(float c, int r) {
  const float x = c * (float)r;
  const float f = floorf(x);
  Axis a;
  a.t = x - f;
  const int i = (int)f;
  a.i0 = i & (r - 1);
  a.i1 = (i + 1) & (r - 1);
  return a;
}

// The cell of a point along axis d from its coordinate c in the periodic
// box [0, L_d), given scale = r / L_d (FP64): on the unit cube (L_d = 1)
// exactly axis_of (c r is exact in FP32); in a box the grid coordinate
// c r / L_d in FP64, its floor (wrapped to the grid) and the fraction in
// [0, 1) rounded once to FP32, which avoids the extra rounding of an FP32
// c / L_d (up to r 2^-24 voxel). One FP64 multiply per coordinate.
__device__ __forceinline__ Axis axis_in_box(float c, double scale, bool unit, int r) {
  if (unit) return axis_of(c, r);
  const double g = (double)c * scale;
  double f = floor(g);
  float t = (float)(g - f);
  if (t >= 1.f) {  // g - f within half an FP32 ulp of 1
    t = 0.f;
    f += 1.0;
  }
  Axis a;
  a.t = t;
  const long long i = (long long)f;
  a.i0 = (int)(i & (long long)(r - 1));
  a.i1 = (a.i0 + 1) & (r - 1);
  return a;
}

// Sorted point records (the binning's output): (tx, ty, tz, nx) and
// (ny, nz, original index, cells), t the fraction within the cell along each
// axis and cells = i0x | i0y << 10 | i0z << 20 (r <= 512).
__device__ __forceinline__ unsigned pack_cells(int ix, int iy, int iz) {
  return (unsigned)ix | ((unsigned)iy << 10) | ((unsigned)iz << 20);
}
__device__ __forceinline__ Axis axis_rec(float t, float cells_bits, int d, int r) {
  Axis a;
  a.t = t;
  a.i0 = (int)((__float_as_uint(cells_bits) >> (10 * d)) & 1023u);
  a.i1 = (a.i0 + 1) & (r - 1);
  return a;
}

}  // namespace dpsr
