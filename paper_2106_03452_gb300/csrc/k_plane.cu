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
#include "tma.cuh"

namespace dpsr {

template <int L, int C>
struct PlaneGeo {
  static constexpr int R1 = Shape<L>::R1, T = Shape<L>::T, G = kNT / T;
  static constexpr int R = L / C;        // rows per CTA
  static constexpr int H = L / 2;        // packed half-spectrum slots per channel
  static constexpr int SPC = H / C;      // slots per CTA per channel (y pass)
  static constexpr int CHK = G < SPC ? G : SPC;  // slots per chunk (one group each)
  static constexpr int NB = (CHK + 15) / 16;     // TMA boxes per chunk
  static constexpr int BOX = L * 16;             // float2 per box [ky][16 kz]
  static constexpr int XP = L + 1;               // per-group exchange pitch (z pass)
  static constexpr int SCR0 = NB * BOX > G * XP ? NB * BOX : G * XP;
  static constexpr int SCR = (SCR0 + 127) / 128 * 128;  // scratch float2, whole KiB
  static constexpr int KP = L / 2 + 2;   // row pitch of the spectral buffers in HBM
  static constexpr int SWM = (H < 16 ? H : 16) - 1;
  static_assert(R >= 2 && R % 2 == 0, "at least one row pair per CTA");
  static_assert(SPC >= 16 || C == 1, "a CTA owns whole 16-slot TMA boxes");
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

// Column `g` of the chunk boxes (box g/16, complex g%16), element row e.
template <int L>
__device__ __forceinline__ float2& boxcol(float2* sbox, int g, int e) {
  return sbox[(g >> 4) * (L * 16) + bx(e, g & 15)];
}

// Dynamic shared memory: 1024-aligned scratch (TMA boxes / exchange areas),
// then the rows of the plane, then an optional table.
__device__ __forceinline__ float2* aligned_smem(unsigned char* raw) {
  const uint32_t pad = (1024u - (smem_u32(raw) & 1023u)) & 1023u;
  return reinterpret_cast<float2*>(raw + pad);
}

// The slot-0 column of a chunk holds the packed DC and Nyquist columns
// P = X0 + i Xn. Separate them in place (column 0 <- X0) and hand Xn to
// `nyq(ky, value)`. Run by the T threads of group 0.
template <int L, class Nyq>
__device__ __forceinline__ void separate_dc_nyq(float2* sbox, int t, Nyq nyq) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T;
  float2 x0[R1], xn[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    const int ky = t + T * j;
    unpack_dc_nyq(boxcol<L>(sbox, 0, ky), boxcol<L>(sbox, 0, (L - ky) & (L - 1)), x0[j], xn[j]);
  }
  group_sync<T>();
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    boxcol<L>(sbox, 0, t + T * j) = x0[j];
    nyq(t + T * j, xn[j]);
  }
}

// Issue (one thread) the TMA loads / stores of a chunk's boxes.
template <int L, int C>
__device__ __forceinline__ void chunk_load(const CUtensorMap* tm, float2* sbox, int s_first, int X,
                                           uint64_t* bar) {
  using P = PlaneGeo<L, C>;
  mbar_expect_tx(bar, P::NB * P::BOX * (uint32_t)sizeof(float2));
  for (int b = 0; b < P::NB; ++b) tma_load_3d(sbox + b * P::BOX, tm, s_first + 16 * b, 0, X, bar);
}
template <int L, int C>
__device__ __forceinline__ void chunk_store(const CUtensorMap* tm, const float2* sbox, int s_first,
                                            int X) {
  using P = PlaneGeo<L, C>;
  for (int b = 0; b < P::NB; ++b) tma_store_3d(tm, s_first + 16 * b, 0, X, sbox + b * P::BOX);
  tma_store_commit();
}

// Push a chunk of y-domain columns (boxes) into the rows of their owner CTAs:
// row y, slot `choff + s_first + gi`.
template <int L, int C, int RP>
__device__ __forceinline__ void push_cols(cg::cluster_group& cl, float2* rows, int s_first,
                                          int choff, float2* sbox) {
  using P = PlaneGeo<L, C>;
  for (int i = threadIdx.x; i < P::CHK * L; i += kNT) {
    const int gi = i % P::CHK, y = i / P::CHK;
    const int q = y / P::R, lr = y % P::R;
    dsmem_st(dsmem_map(rows, q) + 8u * sw<RP, P::SWM>(lr, choff + s_first + gi), boxcol<L>(sbox, gi, y));
  }
}

// Bounded wait on a TMA barrier, block-uniform outcome.
__device__ __forceinline__ bool chunk_wait(uint64_t* bar, uint32_t phase, unsigned* status) {
  const bool ok = __syncthreads_and(mbar_wait(bar, phase));
  if (!ok && threadIdx.x == 0) atomicOr(status, kStTimeout);
  return ok;
}

// kind: 0 forward plane (2 channels per row + derivative table), 1 inverse
// (1 channel), 2 backward forward-transform (1 channel), 3 backward inverse
// (3 channels + table).
template <int L, int C>
constexpr size_t plane_smem(int kind) {
  using P = PlaneGeo<L, C>;
  const int rp = kind == 0 ? L : (kind == 3 ? 3 * P::H : P::H);
  const int table = (kind == 0 || kind == 3) ? L / 2 : 0;  // iu, as float2 units
  return 1024 + sizeof(float2) * ((size_t)P::SCR + (size_t)P::R * rp + table + L);
}

// Two CTAs per SM where their shared memory fits (<= 113 KB each).
template <int L, int C>
constexpr int plane_minb(int kind) {
  return plane_smem<L, C>(kind) <= 113 * 1024 ? 2 : 1;
}


// ===========================================================================
// Forward plane kernel: splat + R2C(z) + FFT(y), one channel per round
// (v_y, v_z, v_x, W). Rows of a CTA are half-spectrum rows in 16-slot blocks
// swizzled like TMA box rows (rsw); after the z pass every CTA pushes, with
// bulk copies into the other CTAs' shared memory, the slot segments each of
// them transforms along y, so the y pass reads only local shared memory.
// D = FFT_y(i u_z v~_z) + i u_y FFT_y(v~_y) accumulates in the output boxes
// over the v_y and v_z rounds.
// ===========================================================================
// Threads of the forward plane kernel: 512 (one CTA per SM) up to 4-CTA
// clusters; 256 for larger clusters, whose CTAs then fit two per SM.
template <int C>
constexpr int fwd_threads() {
  return C >= 8 ? 256 : 512;
}

template <int H>
__device__ __forceinline__ int rsw(int y, int s) {
  if constexpr (H < 16) {
    return s;
  } else {
    return (s & ~15) | (((((s >> 1) ^ y) & 7)) << 1) | (s & 1);
  }
}

template <int L, int C>
struct FwdGeo {
  static constexpr int NT = fwd_threads<C>();
  static constexpr int T = Shape<L>::T, R1 = Shape<L>::R1, G = NT / T;
  static constexpr int R = L / C, H = L / 2, SPC = H / C;
  static constexpr int NB = (SPC + 15) / 16;  // output boxes (16 slots each)
  static constexpr int BOX = L * 16;
  static constexpr int ZG = R / 2 < G ? R / 2 : G;  // groups of the z pass
  // The boxes keep D between the v_y and v_z rounds, so the z-pass exchange
  // areas (L per group) cannot share them: with C > 1 they live in the
  // receive buffer (free during the z pass, exactly R/2 * L), else apart.
  static constexpr int SCR = (NB * BOX + 127) / 128 * 128;
  static constexpr int ROWS = R * H;               // float2 (R real rows of L floats)
  static constexpr int RECV = C > 1 ? L * SPC : ZG * L;  // float2
  static_assert(G >= SPC, "one y pass per round (D accumulates in the boxes)");
  static_assert(T == 1 || SPC % (32 / T) == 0 || SPC >= G, "idle y groups must fill whole warps");
};

template <int L, int C>
constexpr size_t fwd_smem() {
  using F = FwdGeo<L, C>;
  return 1024 + sizeof(float2) * ((size_t)F::SCR + F::ROWS + F::RECV + L) + sizeof(float) * L;
}

template <int L, int C>
__global__ void __launch_bounds__(fwd_threads<C>(), 512 / fwd_threads<C>())
    k_plane_fwd(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  using F = FwdGeo<L, C>;
  constexpr int H = F::H, SPC = F::SPC;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / F::T, t = tid % F::T;
  extern __shared__ unsigned char smem_raw[];
  float2* sbox = aligned_smem(smem_raw);
  float2* rows = sbox + F::SCR;
  float* rows_f = reinterpret_cast<float*>(rows);
  float2* recv = rows + F::ROWS;
  float2* twt = recv + F::RECV;
  float* iu = reinterpret_cast<float*>(twt + L);
  __shared__ uint64_t bar;
  for (int i = tid; i < L; i += F::NT) {
    iu[i] = S.iu[i];
    twt[i] = S.tw[i];
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  TwTab<L> twr{twt, t};
  const PlanePoints pp(S, X);
  const int y_lo = c * F::R;
  const float2* ysrc = C > 1 ? recv : rows;  // [y][SPC] in the y pass
  uint32_t phase = 0;
  bool alive = true;
  // y pass: group g -> slot sl = g of this CTA; its box column is g
  const bool yact = g < SPC;
  auto xa = [&](int e) -> float2& { return boxcol<L>(sbox, yact ? g : 0, e); };
  float2* xz = recv + g * L;  // z-pass exchange (groups < ZG)

  for (int rd = 0; rd < 4; ++rd) {
    const int ch = rd == 0 ? 1 : (rd == 1 ? 2 : (rd == 2 ? 0 : 3));  // v_y, v_z, v_x, W
    for (int i = tid; i < F::ROWS / 2; i += F::NT)
      reinterpret_cast<float4*>(rows)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    // Rasterization (Eq. A2) of one channel into real rows.
    for (int i = tid; i < pp.total(); i += F::NT) {
      int dx;
      const int idx = pp.index(i, dx);
      const float4 a = S.sorted[2 * idx], b = S.sorted[2 * idx + 1];
      const float val = ch == 0 ? a.w : (ch == 1 ? b.x : (ch == 2 ? b.y : 1.f));
      const Axis ax = axis_of(a.x, L), ay = axis_of(a.y, L), az = axis_of(a.z, L);
      const float fx = wsel(dx, ax.t) * val;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int ly = (dy ? ay.i1 : ay.i0) - y_lo;
        if ((unsigned)ly >= (unsigned)F::R) continue;
        const float fxy = fx * wsel(dy, ay.t);
        atomicAdd(&rows_f[ly * L + az.i0], fxy * (1.f - az.t));
        atomicAdd(&rows_f[ly * L + az.i1], fxy * az.t);
      }
    }
    __syncthreads();
    // R2C along z of row pairs, in place; the v_z channel takes i u_z.
    for (int p0 = 0; p0 < F::R / 2; p0 += F::ZG) {
      const int p = p0 + g;
      if (g < F::ZG) {  // whole warps (ZG a multiple of 32/T, or T = 1)
        const bool ok = p < F::R / 2;
        const int pr = ok ? p : 0;
        const int ya = y_lo + 2 * pr;
        auto put = [&](int row, int yy, int s, float2 v) {
          if (!ok) return;
          if (ch == 2) v = s == 0 ? czero() : cmul_iu(v, iu[s]);
          rows[row * H + rsw<H>(yy, s)] = v;
        };
        r2c_pair<L>(
            t, xz, twr,
            [&](int z) { return make_float2(rows_f[2 * pr * L + z], rows_f[(2 * pr + 1) * L + z]); },
            [&](int s, float2 v) { put(2 * pr, ya, s, v); },
            [&](int s, float2 v) { put(2 * pr + 1, ya + 1, s, v); });
      }
    }
    if constexpr (C > 1) {
      // Exchange: row lr's segment of CTA q's slots goes to q's receive
      // buffer, row y_lo + lr. Arm, sync (all armed, receive buffers free),
      // push, wait for this CTA's own segments.
      if (tid == 0) mbar_expect_tx(&bar, L * SPC * (uint32_t)sizeof(float2));
      fence_async_smem();
      cl.sync();
      for (int i = tid; i < F::R * C; i += F::NT) {
        const int lr = i % F::R, q = i / F::R;
        const uint32_t dst = dsmem_map(recv, q) + 8u * (uint32_t)((y_lo + lr) * SPC);
        bulk_push(dst, rows + lr * H + q * SPC, SPC * (uint32_t)sizeof(float2), dsmem_map(&bar, q));
      }
      alive = chunk_wait(&bar, phase, S.status) && alive;
      phase ^= 1;
    } else {
      __syncthreads();
    }
    // FFT along y of this CTA's SPC slots.
    if (yact) {
      float2 v[F::R1], part[F::R1];
#pragma unroll
      for (int j = 0; j < F::R1; ++j) {
        const int y = t + F::T * j;
        v[j] = ysrc[y * SPC + rsw<H>(y, g)];
        // the FFT below uses the box column as its exchange buffer: take the
        // v_y partial of D out of it first
        if (rd == 1) part[j] = xa(y);
      }
      fft_r<L, -1>(v, t, xa, twr);
#pragma unroll
      for (int j = 0; j < F::R1; ++j) {
        const int ky = t + F::T * j;
        if (rd == 0) xa(ky) = cmul_iu(v[j], iu[ky]);
        else if (rd == 1) xa(ky) = cadd(part[j], v[j]);
        else xa(ky) = v[j];
      }
    }
    __syncthreads();
    if (rd >= 1) {
      const int buf = rd == 1 ? 0 : (rd == 2 ? 1 : 2);  // D, C, W~
      if (c == 0 && g == 0) {
        float2* dst = S.spec[buf];
        separate_dc_nyq<L>(sbox, t, [&](int ky, float2 w) {
          if (H < 16) boxcol<L>(sbox, H, ky) = w;
          else dst[((size_t)X * L + ky) * P::KP + H] = w;
        });
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        for (int b = 0; b < F::NB; ++b)
          tma_store_3d(&S.tmy[buf], c * SPC + 16 * b, 0, X, sbox + b * F::BOX);
        tma_store_commit();
        tma_store_wait_read();
      }
      __syncthreads();
    }
    if constexpr (C > 1) cl.sync();  // receive buffers and rows are reused next round
  }
  (void)alive;
}

// ===========================================================================
// Forward inverse plane kernel: IFFT(y) + C2R(z) + normalisation + lookup
// gradient of chi' at the points.
// ===========================================================================
template <int L, int C>
__global__ void __launch_bounds__(kNT, plane_minb<L, C>(1))
    k_plane_inv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = P::H;  // one channel
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ unsigned char smem_raw[];
  float2* sbox = aligned_smem(smem_raw);
  float2* rows = sbox + P::SCR;
  float2* twt = rows + P::R * RP;
  __shared__ uint64_t bar;
  for (int i = tid; i < L; i += kNT) twt[i] = S.tw[i];
  TwTab<L> twr{twt, t};
  const float a_chi = S.sc->a_chi, b_chi = S.sc->b_chi;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  bool alive = true;
  for (int cb = 0; cb < P::SPC && alive; cb += P::CHK) {
    const int s_first = c * P::SPC + cb;
    if (tid == 0) chunk_load<L, C>(&S.tmy[3], sbox, s_first, X, &bar);
    const bool head = (c == 0 && cb == 0);
    float2 nyq[P::R1];
    if (head && g == 0 && P::H >= 16) {
#pragma unroll
      for (int j = 0; j < P::R1; ++j)
        nyq[j] = S.spec[3][((size_t)X * L + t + P::T * j) * P::KP + P::H];
    }
    alive = chunk_wait(&bar, phase, S.status);
    phase ^= 1;
    if (!alive) break;
    auto xa = [&](int e) -> float2& { return boxcol<L>(sbox, g, e); };
    float2 v[P::R1];
#pragma unroll
    for (int j = 0; j < P::R1; ++j) {
      const int ky = t + P::T * j;
      v[j] = xa(ky);
      if (head && g == 0) {  // pack X0 + i Xn
        const float2 n = P::H >= 16 ? nyq[j] : boxcol<L>(sbox, P::H, ky);
        v[j] = make_float2(v[j].x - n.y, v[j].y + n.x);
      }
    }
    fft_r<L, +1>(v, t, xa, twr);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) xa(t + P::T * j) = v[j];
    __syncthreads();
    push_cols<L, C, RP>(cl, rows, s_first, 0, sbox);
    __syncthreads();
  }
  cl.sync();
  if (!alive) return;
  // C2R along z of row pairs (2p, 2p+1); output written in place as pairs
  // (y_2p[z], y_2p+1[z]) at logical slot z of the pair.
  float* chi = S.chi;
  float2* xz = sbox + g * P::XP;
  for (int p0 = 0; p0 < P::R / 2; p0 += P::G) {
    const int p = p0 + g;
    const bool ok = p < P::R / 2;
    const int pr = ok ? p : 0;
    const int ya = c * P::R + 2 * pr;
    c2r_pair<L>(
        t, xz, twr, [&](int k) { return rows[sw<RP, P::SWM>(2 * pr, k)]; },
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
      const float2 f = dsmem_ld(dsmem_map(rows, q) + 8u * sw<RP, P::SWM>(p2 + z / P::H, z % P::H));
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
__global__ void __launch_bounds__(kNT, plane_minb<L, C>(2))
    k_plane_bfwd(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = P::H;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ unsigned char smem_raw[];
  float2* sbox = aligned_smem(smem_raw);
  float2* rows = sbox + P::SCR;
  float2* twt = rows + P::R * RP;
  float2* xz = sbox + g * P::XP;
  for (int i = tid; i < L; i += kNT) twt[i] = S.tw[i];
  __shared__ double red[2][kNT / 32];
  uint32_t rb[C];  // shared::cluster address of each CTA's rows
#pragma unroll
  for (int q = 0; q < C; ++q) rb[q] = dsmem_map(rows, q);
  TwTab<L> twr{twt, t};
  __shared__ uint64_t bar;
  // The CTA's R rows of dchi are contiguous in HBM: one bulk copy into the
  // rows buffer (R real rows of L floats fill exactly R packed half-spectrum
  // rows), then the sums of Eq. 4's adjoint against chi with vector loads.
  const size_t row0 = ((size_t)X * L + c * P::R) * L;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, P::R * L * (uint32_t)sizeof(float));
    bulk_load(rows, S.dchi + row0, P::R * L * (uint32_t)sizeof(float), &bar);
  }
  const float4* chi4 = reinterpret_cast<const float4*>(S.chi + row0);
  __syncthreads();
  const bool landed = chunk_wait(&bar, 0, S.status);
  float accS = 0.f, accD = 0.f;
  if (landed) {
    const float4* g4 = reinterpret_cast<const float4*>(rows);
#pragma unroll 4
    for (int i = tid; i < P::R * L / 4; i += kNT) {
      const float4 a = g4[i], b = chi4[i];
      accS += (a.x + a.y) + (a.z + a.w);
      accD += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    }
  }
  __syncthreads();
  const float* rf = reinterpret_cast<const float*>(rows);
  for (int p0 = 0; p0 < P::R / 2 && landed; p0 += P::G) {
    const int p = p0 + g;
    const bool ok = p < P::R / 2;
    const int pr = ok ? p : 0;
    r2c_pair<L>(
        t, xz, twr, [&](int z) { return make_float2(rf[2 * pr * L + z], rf[(2 * pr + 1) * L + z]); },
        [&](int s, float2 v) {
          if (ok) rows[sw<RP, P::SWM>(2 * pr, s)] = v;
        },
        [&](int s, float2 v) {
          if (ok) rows[sw<RP, P::SWM>(2 * pr + 1, s)] = v;
        });
  }
  cl.sync();
  for (int cb = 0; cb < P::SPC; cb += P::CHK) {
    const int s_first = c * P::SPC + cb;
    const int s = s_first + min(g, P::CHK - 1);
    auto xa = [&](int e) -> float2& { return boxcol<L>(sbox, g, e); };
    float2 v[P::R1];
    constexpr int RT = P::R / P::T;  // row y = t + T j lives in CTA j / RT
#pragma unroll
    for (int j = 0; j < P::R1; ++j) v[j] = dsmem_ld(rb[j / RT] + 8u * sw<RP, P::SWM>(t + P::T * (j % RT), s));
    fft_r<L, -1>(v, t, xa, twr);
#pragma unroll
    for (int j = 0; j < P::R1; ++j) xa(t + P::T * j) = v[j];
    __syncthreads();
    if (c == 0 && cb == 0 && g == 0) {
      separate_dc_nyq<L>(sbox, t, [&](int ky, float2 w) {
        if (P::H < 16) boxcol<L>(sbox, P::H, ky) = w;
        else S.spec[3][((size_t)X * L + ky) * P::KP + P::H] = w;
      });
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      chunk_store<L, C>(&S.tmy[3], sbox, s_first, X);
      tma_store_wait_read();
    }
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
__global__ void __launch_bounds__(kNT, plane_minb<L, C>(3))
    k_plane_binv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using P = PlaneGeo<L, C>;
  constexpr int RP = 3 * P::H;  // channels X | Y | Z
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / P::T, t = tid % P::T;
  extern __shared__ unsigned char smem_raw[];
  float2* sbox = aligned_smem(smem_raw);
  float2* rows = sbox + P::SCR;
  float* iu = reinterpret_cast<float*>(rows + P::R * RP);
  float2* twt = reinterpret_cast<float2*>(iu + L);
  __shared__ uint64_t bar;
  for (int i = tid; i < L; i += kNT) {
    iu[i] = S.iu[i];
    twt[i] = S.tw[i];
  }
  TwTab<L> twr{twt, t};
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  bool alive = true;
  for (int cb = 0; cb < P::SPC && alive; cb += P::CHK) {
    const int s_first = c * P::SPC + cb;
    const int s = s_first + min(g, P::CHK - 1);
    const bool head = (c == 0 && cb == 0);
    auto xa = [&](int e) -> float2& { return boxcol<L>(sbox, g, e); };
    float2 v[P::R1];
    // X channel: Q2 = IFFT_x(-i u_x F), y-inverse as is. Y and Z channels from
    // Q1 = IFFT_x(F): -i u_y before the y-inverse, -i u_z (a constant per
    // column) for Z.
    for (int src = 0; src < 3 && alive; ++src) {
      // src 0: X from Q2; src 1: Y = -i u_y Q1; src 2: Z = -i u_z Q1 (Q1 is
      // loaded again rather than kept in registers; the second load hits L2)
      const int buf = src == 0 ? 1 : 0;
      if (tid == 0) chunk_load<L, C>(&S.tmy[buf], sbox, s_first, X, &bar);
      float2 nyq[P::R1];
      if (head && g == 0 && P::H >= 16) {
#pragma unroll
        for (int j = 0; j < P::R1; ++j)
          nyq[j] = S.spec[buf][((size_t)X * L + t + P::T * j) * P::KP + P::H];
      }
      alive = chunk_wait(&bar, phase, S.status);
      phase ^= 1;
      if (!alive) break;
#pragma unroll
      for (int j = 0; j < P::R1; ++j) {
        const int ky = t + P::T * j;
        v[j] = xa(ky);
        if (head && g == 0) {
          const float2 n = P::H >= 16 ? nyq[j] : boxcol<L>(sbox, P::H, ky);
          v[j] = make_float2(v[j].x - n.y, v[j].y + n.x);
        }
      }
      if (src == 1) {
#pragma unroll
        for (int j = 0; j < P::R1; ++j) v[j] = cmul_iu(v[j], -iu[t + P::T * j]);
      } else if (src == 2) {
        const float ez = s == 0 ? 0.f : -iu[s];
#pragma unroll
        for (int j = 0; j < P::R1; ++j) v[j] = cmul_iu(v[j], ez);
      }
      fft_r<L, +1>(v, t, xa, twr);
#pragma unroll
      for (int j = 0; j < P::R1; ++j) xa(t + P::T * j) = v[j];
      __syncthreads();
      push_cols<L, C, RP>(cl, rows, s_first, src * P::H, sbox);
      __syncthreads();
    }
  }
  cl.sync();
  if (!alive) return;
  // C2R along z: rows of (X, Y) pairs in place as (Vx[z], Vy[z]); Z channel
  // by row pairs, in place as (Vz_2p[z], Vz_2p+1[z]) over the Z slots of the
  // two rows.
  float2* xz = sbox + g * P::XP;
  for (int r0 = 0; r0 < P::R; r0 += P::G) {
    const int row = r0 + g;
    const bool ok = row < P::R;
    const int rr = ok ? row : 0;
    c2r_pair<L>(
        t, xz, twr, [&](int k) { return rows[sw<RP, P::SWM>(rr, k)]; },
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
        t, xz, twr, [&](int k) { return rows[sw<RP, P::SWM>(2 * pr, 2 * P::H + k)]; },
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
          const uint32_t rq = dsmem_map(rows, q);
          const float2 xy = dsmem_ld(rq + 8u * sw<RP, P::SWM>(lr, z));
          const float2 zz = dsmem_ld(rq + 8u * sw<RP, P::SWM>(p2 + z / P::H, 2 * P::H + z % P::H));
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
// Cluster sizes instantiated per grid size: one CTA per plane up to r = 64,
// 1/2/4 CTAs at r = 128, 2/4/8 CTAs at r = 256 (r^2 complex values of one
// plane do not fit one SM's shared memory there).
template <int L, int C>
constexpr bool plane_inst() {
  // every CTA must own at least 16 slots (one TMA box of kz) so that box
  // stores never cover a neighbour's slots
  return L <= 64 ? C == 1 : (L == 128 ? (C == 1 || C == 2 || C == 4) : (C == 2 || C == 4 || C == 8));
}

// The forward plane kernel transforms all slots of a CTA in one y pass, which
// needs at least as many groups as slots (r = 256: C >= 4).
template <int L, int C>
constexpr bool fwd_inst() {
  return plane_inst<L, C>() && (fwd_threads<C>() / Shape<L>::T) >= (L / 2) / C;
}

template <int L, int C>
static cudaError_t launch_plane_t(int kind, const Solve& s, const Solve* tab, int count,
                                  cudaStream_t st) {
  void (*fn)(Solve, const Solve*) = nullptr;
  switch (kind) {
    case 0:
      if constexpr (fwd_inst<L, C>()) fn = k_plane_fwd<L, C>;
      else return cudaErrorInvalidValue;
      break;
    case 1: fn = k_plane_inv<L, C>; break;
    case 2: fn = k_plane_bfwd<L, C>; break;
    default: fn = k_plane_binv<L, C>; break;
  }
  size_t smem = plane_smem<L, C>(kind);
  if constexpr (fwd_inst<L, C>()) {
    if (kind == 0) smem = fwd_smem<L, C>();
  }
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set[4] = {false, false, false, false};  // per instantiation and kind
  if (!attr_set[kind]) {
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr_set[kind] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L * C, 1, count);
  cfg.blockDim = dim3(kind == 0 ? fwd_threads<C>() : kNT, 1, 1);
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

template <int L>
static cudaError_t launch_plane_L(int kind, int C, const Solve& s, const Solve* tab, int count,
                                  cudaStream_t st) {
  switch (C) {
    case 1: if constexpr (plane_inst<L, 1>()) return launch_plane_t<L, 1>(kind, s, tab, count, st); break;
    case 2: if constexpr (plane_inst<L, 2>()) return launch_plane_t<L, 2>(kind, s, tab, count, st); break;
    case 4: if constexpr (plane_inst<L, 4>()) return launch_plane_t<L, 4>(kind, s, tab, count, st); break;
    case 8: if constexpr (plane_inst<L, 8>()) return launch_plane_t<L, 8>(kind, s, tab, count, st); break;
    case 16: if constexpr (plane_inst<L, 16>()) return launch_plane_t<L, 16>(kind, s, tab, count, st); break;
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
      case 1: if constexpr (plane_inst<L, 1>()) { if (kind == 0) { if constexpr (fwd_inst<L, 1>()) return fwd_smem<L, 1>(); return 0; } return plane_smem<L, 1>(kind); } return 0;
      case 2: if constexpr (plane_inst<L, 2>()) { if (kind == 0) { if constexpr (fwd_inst<L, 2>()) return fwd_smem<L, 2>(); return 0; } return plane_smem<L, 2>(kind); } return 0;
      case 4: if constexpr (plane_inst<L, 4>()) { if (kind == 0) { if constexpr (fwd_inst<L, 4>()) return fwd_smem<L, 4>(); return 0; } return plane_smem<L, 4>(kind); } return 0;
      case 8: if constexpr (plane_inst<L, 8>()) { if (kind == 0) { if constexpr (fwd_inst<L, 8>()) return fwd_smem<L, 8>(); return 0; } return plane_smem<L, 8>(kind); } return 0;
      case 16: if constexpr (plane_inst<L, 16>()) { if (kind == 0) { if constexpr (fwd_inst<L, 16>()) return fwd_smem<L, 16>(); return 0; } return plane_smem<L, 16>(kind); } return 0;
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
