// x-axis pass: FFT along x of the partially transformed fields, the spectral
// solve of Eq. 3 (forward) or its adjoint (backward), and the inverse FFT
// along x, for a tile of 16 consecutive kz columns at one ky.
//
// Forward:  chi~ = G(k) (D + i u_x C),  G = g(u) / (-2 pi |u|^2),
//           g = exp(-2 sigma^2 |u|^2 / r^2)                        (Eq. 3, A7)
//           with the spectral sums for the mean and the value at x = 0 of
//           Eq. 4 (Parseval over the half spectrum).
// Backward: F = G(k) (g_a FFT(dchi) + g_s + g_w W~);  Q1 = IFFT_x(F),
//           Q2 = IFFT_x(-i u_x F)  (the adjoint of Eq. 3, conj(H_a) = -H_a).
#include "dpsr_dev.cuh"
#include "launch.h"

namespace dpsr {

template <int L>
struct XGeo {
  static constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  static constexpr int KC = 16 * T >= 32 ? 16 : 32 / T;  // kz columns per CTA (>= 1 warp)
  static constexpr int NT = KC * T;      // threads
  static constexpr int SP = L + 1;       // smem column pitch
  static constexpr int H = L / 2;
  static constexpr int KP = L / 2 + 2;
  static constexpr int NCHUNK = (H + 1 + KC - 1) / KC;
};

__device__ __forceinline__ float spectral_G(int kx, int ky, int kz, const float* g1,
                                            const float* u2) {
  const float s = u2[kx] + u2[ky] + u2[kz];
  if (s == 0.f) return 0.f;
  return g1[kx] * g1[ky] * g1[kz] / (-6.28318530717958647692f * s);
}

template <int L, bool BWD>
__global__ void __launch_bounds__(XGeo<L>::NT)
    k_xpass(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = XGeo<L>;
  constexpr int NCH = BWD ? 2 : 3;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int kz0 = blockIdx.x * P::KC, ky = blockIdx.y;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ float4 smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);  // [NCH][KC][SP]
  float2* tw = buf + NCH * P::KC * P::SP;
  float* g1 = reinterpret_cast<float*>(tw + L);
  float* u2 = g1 + L;
  float* iu = u2 + L;
  __shared__ double red[2][P::NT / 32 + 1];
  for (int i = tid; i < L; i += P::NT) {
    tw[i] = S.tw[i];
    g1[i] = S.g1[i];
    u2[i] = S.u2[i];
    iu[i] = S.iu[i];
  }
  const float2* src[NCH];
  if constexpr (BWD) {
    src[0] = S.spec[3];  // FFT_zy(dchi)
    src[1] = S.spec[2];  // W~ (zy)
  } else {
    src[0] = S.spec[0];  // D
    src[1] = S.spec[1];  // C
    src[2] = S.spec[2];  // W~
  }
  for (int i = tid; i < NCH * P::KC * L; i += P::NT) {
    const int ch = i / (P::KC * L), rem = i % (P::KC * L);
    const int x = rem / P::KC, kzl = rem % P::KC, kz = kz0 + kzl;
    float2 v = czero();
    if (kz <= P::H) v = src[ch][((size_t)x * L + ky) * P::KP + kz];
    buf[(ch * P::KC + kzl) * P::SP + x] = v;
  }
  __syncthreads();
  const int kz = min(kz0 + g, P::H);
  const bool valid = kz0 + g <= P::H;
  float2* c0 = buf + (0 * P::KC + g) * P::SP;
  float2* c1 = buf + (1 * P::KC + g) * P::SP;
  float2 a[P::R1], b[P::R1];
#pragma unroll
  for (int j = 0; j < P::R1; ++j) a[j] = c0[t + P::T * j];
  fft<L, -1>(a, t, c0, tw);
#pragma unroll
  for (int j = 0; j < P::R1; ++j) b[j] = c1[t + P::T * j];
  fft<L, -1>(b, t, c1, tw);
  if constexpr (!BWD) {
    float2* c2 = buf + (2 * P::KC + g) * P::SP;
    float2 w[P::R1];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) w[j] = c2[t + P::T * j];
    fft<L, -1>(w, t, c2, tw);
    const float wz = (kz == 0 || kz == P::H) ? 1.f : 2.f;
    float am = 0.f, as = 0.f;
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      const int kx = t + P::T * j;
      const float G = spectral_G(kx, ky, kz, g1, u2);
      const float2 chi = cscale(cadd(a[j], cmul_iu(b[j], iu[kx])), G);
      am += w[j].x * chi.x + w[j].y * chi.y;  // Re(conj(W~) chi~)
      as += chi.x;
      a[j] = chi;
    }
    if (!valid) am = as = 0.f;
    fft<L, +1>(a, t, c0, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) c0[t + P::T * j] = a[j];
    // block partial sums (FP64, fixed order)
    double dm = (double)am * wz, ds = (double)as * wz;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      dm += __shfl_xor_sync(0xffffffffu, dm, m);
      ds += __shfl_xor_sync(0xffffffffu, ds, m);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = dm;
      red[1][tid >> 5] = ds;
    }
    __syncthreads();
    if (tid == 0) {
      double sm = 0, ss = 0;
      for (int q = 0; q < P::NT / 32; ++q) {
        sm += red[0][q];
        ss += red[1][q];
      }
      const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
      S.part[2 * bid] = sm;
      S.part[2 * bid + 1] = ss;
    }
    for (int i = tid; i < P::KC * L; i += P::NT) {
      const int x = i / P::KC, kzl = i % P::KC, kzz = kz0 + kzl;
      if (kzz <= P::H) S.spec[3][((size_t)x * L + ky) * P::KP + kzz] = buf[kzl * P::SP + x];
    }
  } else {
    const Scalars* sc = S.sc;
    const float ga = sc->g_a, gs = sc->g_s, gw = sc->g_w;
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      const int kx = t + P::T * j;
      const float G = spectral_G(kx, ky, kz, g1, u2);
      float2 f = cadd(cscale(a[j], ga), cscale(b[j], gw));
      f.x += gs;
      f = cscale(f, G);
      a[j] = f;
      b[j] = cmul_iu(f, -iu[kx]);
    }
    fft<L, +1>(a, t, c0, tw);
    fft<L, +1>(b, t, c1, tw);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      c0[t + P::T * j] = a[j];
      c1[t + P::T * j] = b[j];
    }
    __syncthreads();
    for (int i = tid; i < 2 * P::KC * L; i += P::NT) {
      const int ch = i / (P::KC * L), rem = i % (P::KC * L);
      const int x = rem / P::KC, kzl = rem % P::KC, kzz = kz0 + kzl;
      if (kzz <= P::H)
        S.spec[ch][((size_t)x * L + ky) * P::KP + kzz] = buf[(ch * P::KC + kzl) * P::SP + x];
    }
  }
}

template <int L, bool BWD>
static cudaError_t launch_xpass_t(const Solve& s, const Solve* tab, int count, cudaStream_t st) {
  using P = XGeo<L>;
  constexpr int NCH = BWD ? 2 : 3;
  const size_t smem = sizeof(float2) * ((size_t)NCH * P::KC * P::SP + L) + 3 * sizeof(float) * L;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_xpass<L, BWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_xpass<L, BWD><<<dim3(P::NCHUNK, L, count), P::NT, smem, st>>>(s, tab);
  return cudaGetLastError();
}

cudaError_t launch_xpass(bool bwd, int r, const Solve& s, const Solve* tab, int count,
                         cudaStream_t st) {
  switch (r) {
    case 8: return bwd ? launch_xpass_t<8, true>(s, tab, count, st) : launch_xpass_t<8, false>(s, tab, count, st);
    case 16: return bwd ? launch_xpass_t<16, true>(s, tab, count, st) : launch_xpass_t<16, false>(s, tab, count, st);
    case 32: return bwd ? launch_xpass_t<32, true>(s, tab, count, st) : launch_xpass_t<32, false>(s, tab, count, st);
    case 64: return bwd ? launch_xpass_t<64, true>(s, tab, count, st) : launch_xpass_t<64, false>(s, tab, count, st);
    case 128: return bwd ? launch_xpass_t<128, true>(s, tab, count, st) : launch_xpass_t<128, false>(s, tab, count, st);
    case 256: return bwd ? launch_xpass_t<256, true>(s, tab, count, st) : launch_xpass_t<256, false>(s, tab, count, st);
    default: return cudaErrorInvalidValue;
  }
}

int xpass_blocks(int r) {
  switch (r) {
    case 8: return XGeo<8>::NCHUNK * 8;
    case 16: return XGeo<16>::NCHUNK * 16;
    case 32: return XGeo<32>::NCHUNK * 32;
    case 64: return XGeo<64>::NCHUNK * 64;
    case 128: return XGeo<128>::NCHUNK * 128;
    case 256: return XGeo<256>::NCHUNK * 256;
    default: return 0;
  }
}

// ---------------------------------------------------------------------------
// Scalar finalisation (one block): fixed-order FP64 reduction of the block
// partials, then the scalars of Eq. 4 (forward) or of its adjoint (backward).
// ---------------------------------------------------------------------------
__device__ void reduce_parts(const double* part, int n, double& a, double& b) {
  __shared__ double ra[256], rb[256];
  double x = 0, y = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  ra[threadIdx.x] = x;
  rb[threadIdx.x] = y;
  __syncthreads();
  for (int m = blockDim.x / 2; m > 0; m >>= 1) {
    if ((int)threadIdx.x < m) {
      ra[threadIdx.x] += ra[threadIdx.x + m];
      rb[threadIdx.x] += rb[threadIdx.x + m];
    }
    __syncthreads();
  }
  a = ra[0];
  b = rb[0];
}

__global__ void __launch_bounds__(256) k_finalize(const __grid_constant__ Solve s0,
                                                  const Solve* __restrict__ tab, int nparts,
                                                  int bwd) {
  const Solve& S = tab ? tab[blockIdx.x] : s0;
  double a, b;
  reduce_parts(S.part, nparts, a, b);
  if (threadIdx.x != 0) return;
  Scalars* sc = S.sc;
  const double n = (double)S.r * S.r * S.r;
  if (!bwd) {
    // mu = <W, chi'> / N, chi'(0) = sum_k chi~ / n, s = chi'(0) - mu (Eq. 4)
    const double mu = a / ((double)S.N * n);
    const double chi0 = b / n;
    const double s = chi0 - mu;
    sc->acc_mu = a;
    sc->acc_s0 = b;
    sc->mu = mu;
    sc->s = s;
    const bool bad = !isfinite(s) || !(fabs(s) > 1e-7 * (fabs(chi0) + fabs(mu)) + 1e-37);
    if (bad) {
      atomicOr(S.status, kStDegenerate);
      sc->alpha = 0;
      sc->a_chi = 0.f;
      sc->b_chi = 0.f;
    } else {
      const double alpha = (double)kM / fabs(s);
      sc->alpha = alpha;
      sc->a_chi = (float)(alpha / n);
      sc->b_chi = (float)(-alpha * mu);
    }
  } else {
    // a = sum dchi, b = sum dchi * chi = alpha * sum dchi (chi' - mu)
    const double alpha = sc->alpha, s = sc->s;
    const double Ssum = a;
    const double D = alpha > 0 ? b / alpha : 0.0;
    const double s_bar = -(double)kM * (s > 0 ? 1.0 : -1.0) * D / (s * s);
    const double mu_bar = -alpha * Ssum - s_bar;
    sc->S = Ssum;
    sc->D = D;
    sc->s_bar = s_bar;
    sc->mu_bar = mu_bar;
    sc->g_a = (float)(alpha / n);
    sc->g_s = (float)(s_bar / n);
    sc->g_w = (float)(mu_bar / ((double)S.N * n));
    sc->c_mu = (float)(mu_bar / ((double)S.N * n));
  }
}

cudaError_t launch_finalize(bool bwd, int nparts, const Solve& s, const Solve* tab, int count,
                            cudaStream_t st) {
  k_finalize<<<count, 256, 0, st>>>(s, tab, nparts, bwd ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace dpsr
