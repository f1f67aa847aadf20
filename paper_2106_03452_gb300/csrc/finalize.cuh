// Scalar finalisation of a solve, run by the last block to finish of the pass
// that produces the block partials (forward x-pass, backward plane pass).
//
// The sums run in float-float arithmetic: a value is an FP32 pair (hi, lo)
// whose exact sum carries it, combined with error-free transformations
// (Knuth's TwoSum, Dekker's Fast2Sum), about 44 significant bits. This
// GPU's FP64 pipe issues roughly one warp instruction per ~18 SM cycles, so
// FP64 shuffle trees and long FP64 reductions on the critical path cost
// several microseconds; FP32 pairs do the same job on the FP32 pipe, in a
// fixed order (deterministic run to run). Only the few scalar formulas of
// Eq. 4, once per solve in one thread, stay in FP64.
#pragma once

#include "dpsr_dev.cuh"

namespace dpsr {

struct FF {
  float hi, lo;
};

// a + b = s + e exactly (TwoSum; no ordering condition on a and b).
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  const float e = s.lo + (x.lo + y.lo);
  const float hi = s.hi + e;  // Fast2Sum: |s.hi| >= |e|
  return {hi, e - (hi - s.hi)};
}

__device__ __forceinline__ FF ff_add(FF x, float y) {
  const FF s = ff_two_sum(x.hi, y);
  const float e = s.lo + x.lo;
  const float hi = s.hi + e;
  return {hi, e - (hi - s.hi)};
}

__device__ __forceinline__ FF ff_shfl_xor(FF x, int m) {
  return {__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)};
}

__device__ __forceinline__ double ff_to_double(FF x) { return (double)x.hi + (double)x.lo; }

// Block sums of two per-thread values in a fixed order (lane butterfly, then
// the warps in index order); the result is valid in thread 0. Every thread
// of the block calls it (it synchronises the block).
template <int NT>
__device__ __forceinline__ void block_sum_ff(FF& a, FF& b) {
  static_assert(NT % 32 == 0, "whole warps");
  __shared__ FF red[2][NT / 32];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    a = ff_add(a, ff_shfl_xor(a, m));
    b = ff_add(b, ff_shfl_xor(b, m));
  }
  const int tid = threadIdx.x;
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = a;
    red[1][tid >> 5] = b;
  }
  __syncthreads();
  if (tid == 0) {
    a = red[0][0];
    b = red[1][0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      a = ff_add(a, red[0][w]);
      b = ff_add(b, red[1][w]);
    }
  }
}

// Thread 0: the scalars from the reduced sums.
__device__ inline void finalize_scalars(const Solve& S, double a, double b, bool bwd) {
  Scalars* sc = S.sc;
  // r^3 is a power of two: its reciprocal is exact in FP32
  const double inv_n = (double)__frcp_rn((float)S.r * (float)S.r * (float)S.r);
  if (!bwd) {
    // mu = <W, chi'> / N, chi'(0) = sum_k chi~ / n, s = chi'(0) - mu (Eq. 4)
    const double mu = a * inv_n * S.inv_N;
    const double chi0 = b * inv_n;
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
      sc->a_chi = (float)(alpha * inv_n);
      sc->b_chi = (float)(-alpha * mu);
    }
  } else {
    // a = sum dchi, b = sum dchi * chi = alpha * sum dchi (chi' - mu);
    // with alpha = m / |s|: D = b / alpha = b |s| / m and
    // s_bar = -m sign(s) D / s^2 = -sign(s) D alpha^2 / m
    const double alpha = sc->alpha, s = sc->s;
    const double Ssum = a;
    const double D = alpha > 0 ? b * fabs(s) * (1.0 / (double)kM) : 0.0;
    const double s_bar = -(s > 0 ? 1.0 : -1.0) * D * alpha * alpha * (1.0 / (double)kM);
    const double mu_bar = -alpha * Ssum - s_bar;
    sc->S = Ssum;
    sc->D = D;
    sc->s_bar = s_bar;
    sc->mu_bar = mu_bar;
    sc->g_a = (float)(alpha * inv_n);
    sc->g_s = (float)(s_bar * inv_n);
    sc->g_w = (float)(mu_bar * inv_n * S.inv_N);
    sc->c_mu = sc->g_w;
  }
}

// Every thread of the block calls this after the block sums (a, b) are in
// thread 0 (block_sum_ff). Thread 0 publishes them as the block's partial
// S.part[bid]; the last of the `nblocks` blocks of the solve to arrive sums
// all partials (each thread a strided subset, loads in flight together, then
// the block tree: a fixed order) and writes the scalars. Only thread 0
// fences, on both sides of its ticket; the block barrier orders the other
// threads' accesses around it (the pattern of a cooperative grid barrier).
template <int NT>
__device__ inline void last_block_finalize(const Solve& S, int ticket, int nblocks, int bid, FF a,
                                           FF b, bool bwd) {
  __shared__ unsigned last;
  const int tid = threadIdx.x;
  if (tid == 0) {
    S.part[bid] = make_float4(a.hi, a.lo, b.hi, b.lo);
    __threadfence();  // this block's partials before its arrival
    last = atomicAdd(&S.sc->ticket[ticket], 1u) == (unsigned)nblocks - 1u ? 1u : 0u;
    if (last) __threadfence();  // every arrival before the reads below
  }
  __syncthreads();
  if (!last) return;
  FF x = {0.f, 0.f}, y = {0.f, 0.f};
#pragma unroll 4
  for (int i = tid; i < nblocks; i += NT) {
    const float4 p = __ldcg(S.part + i);
    x = ff_add(x, FF{p.x, p.y});
    y = ff_add(y, FF{p.z, p.w});
  }
  block_sum_ff<NT>(x, y);
  if (tid == 0) {
    finalize_scalars(S, ff_to_double(x), ff_to_double(y), bwd);
    S.sc->ticket[ticket] = 0;
  }
}

}  // namespace dpsr
