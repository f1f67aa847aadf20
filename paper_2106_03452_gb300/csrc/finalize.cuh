// Scalar finalisation of a solve, run by the last block to finish of the pass
// that produces the block partials (forward x-pass, backward plane pass).
#pragma once

#include "dpsr_dev.cuh"

namespace dpsr {

// ---------------------------------------------------------------------------
// Scalar finalisation, by the last block to finish of the pass that produces
// the block partials: a fixed-order FP64 reduction of the partials, then the
// scalars of Eq. 4 (forward) or of its adjoint (backward).
// ---------------------------------------------------------------------------
// Sums of the n partial pairs by one warp: lane-strided sums (the loads of a
// lane issued together), then a butterfly over the lanes, the same order on
// every run; the result is valid in every lane. The partials come from other
// blocks of this grid, so they are read past L1.
__device__ inline void reduce_parts_warp(const double* part, int n, double& a, double& b) {
  const int lane = threadIdx.x & 31;
  double x = 0, y = 0;
  int i = lane;
  for (; i + 96 < n; i += 128) {
    const double x0 = __ldcg(part + 2 * i), y0 = __ldcg(part + 2 * i + 1);
    const double x1 = __ldcg(part + 2 * i + 64), y1 = __ldcg(part + 2 * i + 65);
    const double x2 = __ldcg(part + 2 * i + 128), y2 = __ldcg(part + 2 * i + 129);
    const double x3 = __ldcg(part + 2 * i + 192), y3 = __ldcg(part + 2 * i + 193);
    x += ((x0 + x1) + (x2 + x3));
    y += ((y0 + y1) + (y2 + y3));
  }
  for (; i < n; i += 32) {
    x += __ldcg(part + 2 * i);
    y += __ldcg(part + 2 * i + 1);
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, m);
    y += __shfl_xor_sync(0xffffffffu, y, m);
  }
  a = x;
  b = y;
}

// Thread 0: the scalars from the reduced sums.
__device__ inline void finalize_scalars(const Solve& S, double a, double b, bool bwd) {
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

// Warp 0 of every block calls this after its lane 0 has written the block's
// partials to S.part[2 * bid, 2 * bid + 1]; the last of the `nblocks` blocks
// of the solve to arrive reduces them and writes the scalars. The other
// warps of the block need not wait.
__device__ inline void last_block_finalize(const Solve& S, int ticket, int nblocks, bool bwd) {
  unsigned last = 0;
  if ((threadIdx.x & 31) == 0) {
    __threadfence();  // this block's partials before its arrival
    last = atomicAdd(&S.sc->ticket[ticket], 1u) == (unsigned)nblocks - 1u ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  double a, b;
  reduce_parts_warp(S.part, nblocks, a, b);
  if ((threadIdx.x & 31) == 0) {
    finalize_scalars(S, a, b, bwd);
    S.sc->ticket[ticket] = 0;
  }
}

}  // namespace dpsr
