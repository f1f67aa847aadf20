// x-axis pass: FFT along x of the partially transformed fields, the spectral
// solve of Eq. 3 (forward) or its adjoint (backward), and the inverse FFT
// along x, for a tile of 16 consecutive kz columns at one ky, moved between
// HBM and shared memory by TMA.
//
// Forward:  chi~ = G(k) (D + i u_x C),  G = g(u) / (-2 pi |u|^2),
//           g = exp(-2 sigma^2 |u|^2 / r^2)                        (Eq. 3, A7)
//           with the spectral sums for the mean and the value at x = 0 of
//           Eq. 4 (Parseval over the half spectrum, and along x).
// Backward: F = G(k) (g_a FFT(dchi) + g_s + g_w W~);  Q1 = IFFT_x(F),
//           Q2 = IFFT_x(-i u_x F)  (the adjoint of Eq. 3, conj(H_a) = -H_a).
// Three FFTs of length r per column in each direction.
#include "dpsr_dev.cuh"
#include "launch.h"
#include "finalize.cuh"
#include "tma.cuh"

namespace dpsr {

template <int L>
struct XGeo {
  static constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  static constexpr int KC = 16;                             // kz columns per CTA (one TMA box row)
  static constexpr int NG = KC * T >= 32 ? KC : 32 / T;     // groups (at least one warp)
  static constexpr int NT = NG * T;                         // threads
  static constexpr int H = L / 2;
  static constexpr int NCHUNK = (H + 1 + KC - 1) / KC;
  static constexpr int BOX = L * KC;                        // float2 per box
  static constexpr int KP = kpitch(L);                      // row pitch of the spectral buffers
  // Two tiles per CTA in both directions. The forward needs W~ only for its
  // spectral sums, after the transforms of C: up to r = 128 it reads W~'s
  // column straight from L2 (the spectra stay resident there); at r = 256 a
  // TMA load brings W~'s tile into C's box once every group is done with C,
  // overlapping the inverse transform.
  static constexpr bool WL2 = L <= 128;
  template <bool BWD>
  static constexpr int nch() { return 2; }
};

// G(k) = g(k) / (-2 pi |u|^2) with g separable: g1[kx] * (g1[ky] g1[kz]);
// gyz and u2yz are the per-thread (ky, kz) factors. Zero at k = 0.
__device__ __forceinline__ float spectral_G(int kx, float gyz, float u2yz, const float* g1,
                                            const float* u2) {
  const float s = u2[kx] + u2yz;
  if (s == 0.f) return 0.f;
  return __fdividef(g1[kx] * gyz, -6.28318530717958647692f * s);
}

// Stage twiddles of the thread (see Twid / TwTab).
template <int L, class Tw>
__device__ __forceinline__ Tw make_tw(const float2* tw, int t) {
  if constexpr (std::is_same<Tw, Twid<L>>::value) {
    Tw w;
    w.load(t, tw);
    return w;
  } else {
    return Tw{tw, t};
  }
}

template <int L, bool BWD>
constexpr size_t xpass_smem() {
  using P = XGeo<L>;
  constexpr int NCH = P::template nch<BWD>();
  return 1024 + sizeof(float2) * ((size_t)NCH * P::BOX + L) + 3 * sizeof(float) * L;
}

// One CTA per (kz tile of 16, ky): TMA loads the tiles [x][16 kz] of the
// input channels (128B-swizzled boxes), each group of T threads transforms
// one kz column along x in registers (the box column doubles as its exchange
// buffer), and TMA stores the results.
template <int L, bool BWD>
__global__ void __launch_bounds__(XGeo<L>::NT, L >= 512 ? 1 : (L >= 256 ? (BWD ? 2 : 3) : 5))
    k_xpass(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = XGeo<L>;
  constexpr int NCH = P::template nch<BWD>();
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int kz0 = blockIdx.x * P::KC, ky = blockIdx.y;
  constexpr bool IL = P::T == 16;  // interleaved groups: conflict-free column accesses
  using LN = Lanes<P::T, IL>;
  const int tid = threadIdx.x, g = LN::group(tid), t = LN::lane(tid);
  extern __shared__ unsigned char smem_raw[];
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  float2* box = reinterpret_cast<float2*>(smem_raw + pad);  // NCH boxes, 1024-aligned
  float2* tw = box + NCH * P::BOX;
  float* g1 = reinterpret_cast<float*>(tw + L);
  float* u2 = g1 + L;
  float* iu = u2 + L;
  // One barrier per box: the forward transforms D while C and W~ still land.
  __shared__ uint64_t bar[NCH];
  // inputs: forward D, C, W~; backward FFT_zy(dchi), W~
  const int src0 = kSpD, src1 = BWD ? kSpW : kSpC;
  pdl_trigger();
  pdl_wait();
  // the binning of this forward pass is done: its counters start the next one at zero
  if constexpr (!BWD) clear_bin_counters(S, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
  if (tid == 0) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) mbar_init(&bar[c], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      mbar_expect_tx(&bar[c], P::BOX * (uint32_t)sizeof(float2));
      for (int x = 0; x < L; x += tma_rows(L))
        tma_load_3d(box + c * P::BOX + x * P::KC, &S.tmx[c == 0 ? src0 : (c == 1 ? src1 : kSpW)], kz0, ky,
                    x, &bar[c]);
    }
  }
  for (int i = tid; i < L; i += P::NT) {
    tw[i] = S.tw[i];
    g1[i] = S.g1[i];
    u2[i] = S.u2[i];  // x axis
    iu[i] = S.iu[i];
  }
  __syncthreads();
  // Each thread records its own bounded waits; the block votes before any
  // store, so that a timeout leaves uniformly (the transforms of a lane whose
  // wait ran out compute on stale data, which is never stored).
  bool ok = true;
  auto box_wait = [&](int c, uint32_t phase = 0u) {
    if (ok) ok = mbar_wait(&bar[c], phase);
  };
  bool w_reload = false;  // r = 256 forward: W~ went into box 1 (its second phase)
  auto leave = [&]() {  // after a failed vote
    if (tid == 0) {
      atomicOr(S.status, kStTimeout);
#pragma unroll
      for (int c = 0; c < NCH; ++c) mbar_wait(&bar[c], 0);  // copies in flight: a last bounded chance
      if (w_reload) mbar_wait(&bar[1], 1);
    }
  };
  const int gc = g < P::KC ? g : P::KC - 1;  // extra groups (tiny r) shadow the last column
  const bool own = g < P::KC;
  const int kz = min(kz0 + gc, P::H);
  const bool valid = own && kz0 + g <= P::H;
  // shared-memory twiddles and one live column array: at r = 256 three CTAs
  // per SM forward (two backward, where three would spill), five below
  using Tw = TwTab<L>;
  Tw twr = make_tw<L, Tw>(tw, t);
  // u2 in shared memory is the x axis' table; the y and z axes' come from global memory
  const float gyz = g1[ky] * g1[kz], u2yz = __ldg(S.u2 + L + ky) + __ldg(S.u2 + 2 * L + kz);
  auto colref = [&](int ch) {
    float2* b = box + ch * P::BOX;
    return [b, gc](int e) -> float2& { return b[bx(e, gc)]; };
  };
  auto c0 = colref(0);
  auto c1 = colref(1);
  float2 a[P::R1];
  if constexpr (!BWD) {
    // Columns past Nyquist (the last kz tile) hold zeros and are not stored:
    // their groups skip the transforms.
    float am = 0.f, as = 0.f, wz = 0.f;
    if (valid) {
      // chi~ = G (FFT_x(D) + i u_x FFT_x(C)); one column array live at a time:
      // FFT_x(D) goes back to its column, FFT_x(C) meets it there.
      box_wait(0);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) a[j] = c0(t + P::T * j);
      fft_r<L, -1, IL>(a, t, c0, twr);
      if (own) {  // groups past the last column (tiny r) only shadow it
#pragma unroll
        for (int j = 0; j < P::R1; ++j) c0(t + P::T * j) = a[j];
      }
      box_wait(1);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) a[j] = c1(t + P::T * j);
      fft_r<L, -1, IL>(a, t, c1, twr);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) {
        const int kx = t + P::T * j;  // this lane wrote c0(kx) above
        const float G = spectral_G(kx, gyz, u2yz, g1, u2);
        a[j] = cscale(cadd(c0(kx), cmul_iu(a[j], iu[kx])), G);
      }
    }
    if constexpr (!P::WL2) {
      // every group is done with box 1 (C and its exchange): W~'s tile goes
      // there (the fence orders this thread's writes to it before the copy's)
      fence_async_smem();
      __syncthreads();
      if (tid == 0 && ok) {
        mbar_expect_tx(&bar[1], P::BOX * (uint32_t)sizeof(float2));
        for (int x = 0; x < L; x += tma_rows(L))
          tma_load_3d(box + P::BOX + x * P::KC, &S.tmx[kSpW], kz0, ky, x, &bar[1]);
      }
      w_reload = true;
    }
    if (valid) {
      fft_r<L, +1, IL>(a, t, c0, twr);  // P = unnormalised IFFT_x(chi~)
      // Spectral sums of Eq. 4, by Parseval along x against the x-domain W~
      // (its tile, or up to r = 128 its column straight from L2):
      // sum_kx conj(W~(kx)) chi~(kx) = sum_x conj(W~_x(x)) P(x),
      // sum_kx chi~(kx) = P(x = 0).
      if constexpr (!P::WL2) {
        box_wait(1, 1u);
#pragma unroll
        for (int j = 0; j < P::R1; ++j) {
          const float2 w = c1(t + P::T * j);
          am += w.x * a[j].x + w.y * a[j].y;
        }
      } else {
        const float2* wc = S.spec[kSpW] + (size_t)ky * P::KP + kz;
#pragma unroll
        for (int j = 0; j < P::R1; ++j) {
          const float2 w = __ldcg(wc + (size_t)(t + P::T * j) * L * P::KP);
          am += w.x * a[j].x + w.y * a[j].y;
        }
      }
      if (t == 0) as = a[0].x;
      wz = (kz == 0 || kz == P::H) ? 1.f : 2.f;
      if (own) {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) c0(t + P::T * j) = a[j];
      }
    }
    FF fm = {am * wz, 0.f}, fs = {as * wz, 0.f};  // wz in {1, 2}: exact
    if (!__syncthreads_and(ok)) {
      leave();
      return;
    }
    fence_async_smem();
    block_sum_ff<P::NT>(fm, fs);  // synchronises the block: the tile is complete
    if (tid == 0) {
      for (int x = 0; x < L; x += tma_rows(L)) tma_store_3d(&S.tmx[kSpChi], kz0, ky, x, box + x * P::KC);
      tma_store_commit();
    }
    last_block_finalize<P::NT>(S, 0, (int)(gridDim.x * gridDim.y),
                               (int)(blockIdx.y * gridDim.x + blockIdx.x), fm, fs, false);
    if (tid == 0) tma_store_wait_read();
  } else {
    // FFT_x of (g_a FFT_zy(dchi) + g_w W~ + g_s delta_{x=0}): the three terms
    // of the adjoint spectrum combined before the transform (it is linear).
    const Scalars* sc = S.sc;
    const float ga = sc->g_a, gs = sc->g_s, gw = sc->g_w;
    box_wait(0);
    box_wait(1);
    if (!__syncthreads_and(ok)) {  // both tiles are needed from the start
      leave();
      return;
    }
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      const int x = t + P::T * j;
      a[j] = cadd(cscale(c0(x), ga), cscale(c1(x), gw));
      if (x == 0) a[j].x += gs;
    }
    fft_r<L, -1, IL>(a, t, c0, twr);
    {
      // F = G (.); Q2's input -i u_x F goes to the column of W~ (read above by
      // this group), Q1 = IFFT_x(F) is transformed from registers first
#pragma unroll
      for (int j = 0; j < P::R1; ++j) {
        const int kx = t + P::T * j;
        a[j] = cscale(a[j], spectral_G(kx, gyz, u2yz, g1, u2));
        if (own) c1(kx) = cmul_iu(a[j], -iu[kx]);
      }
      fft_r<L, +1, IL>(a, t, c0, twr);
      if (own) {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) c0(t + P::T * j) = a[j];
      }
      group_sync<P::T, IL>();
#pragma unroll
      for (int j = 0; j < P::R1; ++j) a[j] = c1(t + P::T * j);
      fft_r<L, +1, IL>(a, t, c1, twr);
      if (own) {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) c1(t + P::T * j) = a[j];
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      for (int x = 0; x < L; x += tma_rows(L)) {
        tma_store_3d(&S.tmx[kSpD], kz0, ky, x, box + x * P::KC);             // Q1
        tma_store_3d(&S.tmx[kSpChi], kz0, ky, x, box + P::BOX + x * P::KC);  // Q2
      }
      tma_store_commit();
      tma_store_wait_read();
    }
  }
}

template <int L, bool BWD>
static cudaError_t launch_xpass_t(const Solve& s, const Solve* tab, int count, cudaStream_t st) {
  using P = XGeo<L>;
  constexpr size_t smem = xpass_smem<L, BWD>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_xpass<L, BWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return launch_k(k_xpass<L, BWD>, dim3(P::NCHUNK, L, count), dim3(P::NT), smem, st, 0, s, tab);
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
    case 512: return bwd ? launch_xpass_t<512, true>(s, tab, count, st) : launch_xpass_t<512, false>(s, tab, count, st);
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
    case 512: return XGeo<512>::NCHUNK * 512;
    default: return 0;
  }
}

}  // namespace dpsr
