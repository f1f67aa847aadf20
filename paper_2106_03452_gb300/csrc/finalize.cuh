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
// Sums of the n partial pairs: thread-strided sums, a warp tree, then the
// warps in order (the same order on every run). Every thread of the block
// calls it; the result is valid in thread 0. The partials come from other
// blocks of this grid, so they are read past L1.
__device__ inline void reduce_parts(const double* part, int n, double& a, double& b) {
  __shared__ double wa[32], wb[32];
  double x = 0, y = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x += __ldcg(part + 2 * i);
    y += __ldcg(part + 2 * i + 1);
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, m);
    y += __shfl_xor_sync(0xffffffffu, y, m);
  }
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x >> 5] = x;
    wb[threadIdx.x >> 5] = y;
  }
  __syncthreads();
  a = 0;
  b = 0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
      a += wa[w];
      b += wb[w];
    }
  }
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

// Every thread of a block calls this after its thread 0 has written the
// block's partials to S.part[2 * bid, 2 * bid + 1]; the last of the
// `nblocks` blocks of the solve reduces them and writes the scalars.
__device__ inline void last_block_finalize(const Solve& S, int ticket, int nblocks, bool bwd) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partials before its arrival
    last = atomicAdd(&S.sc->ticket[ticket], 1u) == (unsigned)nblocks - 1u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a, b;
  reduce_parts(S.part, nblocks, a, b);
  if (threadIdx.x == 0) {
    finalize_scalars(S, a, b, bwd);
    S.sc->ticket[ticket] = 0;
  }
}

}  // namespace dpsr
