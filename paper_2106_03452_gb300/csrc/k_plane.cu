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
#include "finalize.cuh"
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
  static constexpr int KP = kpitch(L);   // row pitch of the spectral buffers in HBM
  static constexpr int SWM = (H < 16 ? H : 16) - 1;
  static_assert(R >= 2 && R % 2 == 0, "at least one row pair per CTA");
  static_assert(SPC >= 16 || C == 1, "a CTA owns whole 16-slot TMA boxes");
};

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
  return plane_inst<L, C>() && (512 / Shape<L>::T) >= (L / 2) / C;
}

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
    const int* off = S.bins + nbins(S.r);
    const int Xm = (X - 1) & (S.r - 1);
    const int ny = nybins(S.r);
    b0 = off[X * ny];
    n0 = off[(X + 1) * ny] - b0;
    b1 = off[Xm * ny];
    n1 = off[(Xm + 1) * ny] - b1;
  }
  __device__ int total() const { return n0 + n1; }
  __device__ int index(int i, int& dx) const {
    dx = i < n0 ? 0 : 1;
    return i < n0 ? b0 + i : b1 + (i - n0);
  }
};

__device__ __forceinline__ float wsel(int d, float t) { return d ? t : 1.f - t; }

// Points of the plane whose stencil touches the rows [y_lo, y_lo + R) of a
// CTA (row i0 only, or i0 or i1 with `both`), as entries idx | dx << 31 in
// `list` (capacity kListCap), so that the per-channel passes over the points
// visit only those. Returns the count, or -1 when it exceeds the capacity
// (the caller then visits all of the plane's points). Called by all NT
// threads of the CTA (NT a multiple of 32); the order of the entries is
// irrelevant: every entry is processed independently of the others.
constexpr int kListCap = 2048;

template <int NT>
__device__ int plane_list(const Solve& S, const PlanePoints& pp, int L, int y_lo, int R, bool both,
                          unsigned* list, int* cnt) {
  if (threadIdx.x == 0) *cnt = 0;
  __syncthreads();
  const float* pf = reinterpret_cast<const float*>(S.sorted);
  const int n = pp.total();
  const unsigned lane = threadIdx.x & 31u;
  for (int i0 = 0; i0 < n; i0 += NT) {
    const int i = i0 + (int)threadIdx.x;
    bool in = false;
    int idx = 0, dx = 0;
    if (i < n) idx = pp.index(i, dx);
    if (i < n && dbg_in_range(S.status, idx, S.N)) {
      const Axis ay = axis_rec(pf[8 * (size_t)idx + 1], pf[8 * (size_t)idx + 7], 1, L);
      in = (unsigned)(ay.i0 - y_lo) < (unsigned)R || (both && (unsigned)(ay.i1 - y_lo) < (unsigned)R);
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int pos = base + __popc(m & ((1u << lane) - 1u));
    if (in && pos < kListCap) list[pos] = (unsigned)idx | ((unsigned)dx << 31);
  }
  __syncthreads();
  const int c = *cnt;
  return c <= kListCap ? c : -1;
}

// Entry i of the visit: from the list, or the plane's i-th point.
__device__ __forceinline__ int visit_point(const unsigned* list, int nlist, const PlanePoints& pp,
                                           int i, int& dx) {
  if (nlist >= 0) {
    const unsigned e = list[i];
    dx = (int)(e >> 31);
    return (int)(e & 0x7fffffffu);
  }
  return pp.index(i, dx);
}



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

// Shared memory of the inverse (kind 1) and backward forward-transform
// (kind 2) plane kernels: scratch, one channel of R rows, twiddles. The
// forward (kind 0) and backward inverse (kind 3) kernels have their own
// layouts (fwd_smem, binv_smem).
template <int L, int C>
constexpr size_t plane_smem(int kind) {
  using P = PlaneGeo<L, C>;
  const int rp = P::H;
  const int table = 0;
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
// Threads of the forward plane kernel: 256 where the configuration fits two
// CTAs per SM (a CTA's shared memory <= 113 KB and 256 threads still cover
// all slots of the CTA in one y pass), 512 (one CTA per SM) otherwise.
template <int L, int C>
constexpr size_t fwd_smem_nt(int nt);

template <int L, int C>
constexpr int fwd_threads() {
  constexpr int spc = (L / 2) / C;
  return (fwd_smem_nt<L, C>(256) <= 113 * 1024 && 256 / Shape<L>::T >= spc) ? 256 : 512;
}

template <int H>
__device__ __forceinline__ int rsw(int y, int s) {
  if constexpr (H < 16) {
    return s;
  } else {
    return (s & ~15) | (((((s >> 1) ^ y) & 7)) << 1) | (s & 1);
  }
}

template <int L, int C, int NTT>
struct FwdGeoT {
  static constexpr int NT = NTT;
  static constexpr int T = Shape<L>::T, R1 = Shape<L>::R1, G = NT / T;
  static constexpr int R = L / C, H = L / 2, SPC = H / C;
  static constexpr int NB = (SPC + 15) / 16;  // output boxes (16 slots each)
  static constexpr int BOX = L * 16;
  static constexpr int ZG = R / 2 < G ? R / 2 : G;  // groups of the z pass
  // The boxes keep D between the v_y and v_z rounds, so the z-pass exchange
  // areas (L per group) cannot share them: with C > 1 they live in the
  // receive buffer (free during the z pass, exactly R/2 * L), else apart.
  static constexpr int SCR = (NB * BOX + 127) / 128 * 128;
  static constexpr int ROWS = R * H;                     // float2 (R real rows of L floats)
  static constexpr int RECV = C > 1 ? L * SPC : ZG * L;  // float2
};

template <int L, int C>
constexpr size_t fwd_smem_nt(int nt) {
  // the footprint does not depend on the thread count except through the
  // z-pass exchange of C = 1 (one area per z group)
  using A = FwdGeoT<L, C, 256>;
  using B = FwdGeoT<L, C, 512>;
  const int recv = nt == 256 ? A::RECV : B::RECV;
  return 1024 + sizeof(float2) * ((size_t)A::SCR + A::ROWS + recv + L) + sizeof(float) * L +
         sizeof(unsigned) * kListCap;
}

template <int L, int C>
struct FwdGeo : FwdGeoT<L, C, fwd_threads<L, C>()> {
  using B = FwdGeoT<L, C, fwd_threads<L, C>()>;
  static_assert(B::G >= B::SPC, "one y pass per round (D accumulates in the boxes)");
  static_assert(B::T == 1 || B::SPC % (32 / B::T) == 0 || B::SPC >= B::G,
                "idle y groups must fill whole warps");
};

template <int L, int C>
constexpr size_t fwd_smem() {
  return fwd_smem_nt<L, C>(fwd_threads<L, C>());
}

template <int L, int C>
__global__ void __launch_bounds__(fwd_threads<L, C>(), 512 / fwd_threads<L, C>())
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
  unsigned* list = reinterpret_cast<unsigned*>(iu + L);
  __shared__ uint64_t bar;
  __shared__ int list_n;
  pdl_trigger();
  for (int i = tid; i < L; i += F::NT) {
    iu[i] = S.iu[L + i];  // y axis; the z axis is read from global memory
    twt[i] = S.tw[i];
  }
  const float* __restrict__ iuz = S.iu + 2 * L;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_wait();
  __syncthreads();
  TwTab<L> twr{twt, t};
  const PlanePoints pp(S, X);
  const int y_lo = c * F::R;
  const int nlist = C > 1 ? plane_list<F::NT>(S, pp, L, y_lo, F::R, true, list, &list_n) : -1;
  const int nvisit = nlist >= 0 ? nlist : pp.total();
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
    for (int i = tid; i < nvisit; i += F::NT) {
      int dx;
      const int idx = visit_point(list, nlist, pp, i, dx);
      if (!dbg_in_range(S.status, idx, S.N)) continue;
      const float4 a = S.sorted[2 * idx], b = S.sorted[2 * idx + 1];
      const float val = ch == 0 ? a.w : (ch == 1 ? b.x : (ch == 2 ? b.y : 1.f));
      const Axis ax = axis_rec(a.x, b.w, 0, L), ay = axis_rec(a.y, b.w, 1, L), az = axis_rec(a.z, b.w, 2, L);
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
          if (ch == 2) v = s == 0 ? czero() : cmul_iu(v, __ldg(iuz + s));
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
      const int buf = rd == 1 ? kSpD : (rd == 2 ? kSpC : kSpW);
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
  pdl_trigger();
  for (int i = tid; i < L; i += kNT) twt[i] = S.tw[i];
  TwTab<L> twr{twt, t};
  pdl_wait();
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
    if (tid == 0) chunk_load<L, C>(&S.tmy[kSpChi], sbox, s_first, X, &bar);
    const bool head = (c == 0 && cb == 0);
    float2 nyq[P::R1];
    if (head && g == 0 && P::H >= 16) {
#pragma unroll
      for (int j = 0; j < P::R1; ++j)
        nyq[j] = S.spec[kSpChi][((size_t)X * L + t + P::T * j) * P::KP + P::H];
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
      if (!dbg_in_range(S.status, idx, S.N)) continue;
      const float4 a = S.sorted[2 * idx];
      const float cells = S.sorted[2 * idx + 1].w;
      const Axis ax = axis_rec(a.x, cells, 0, L), ay = axis_rec(a.y, cells, 1, L), az = axis_rec(a.z, cells, 2, L);
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
  pdl_trigger();
  for (int i = tid; i < L; i += kNT) twt[i] = S.tw[i];
  pdl_wait();
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
        else S.spec[kSpD][((size_t)X * L + ky) * P::KP + P::H] = w;
      });
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      chunk_store<L, C>(&S.tmy[kSpD], sbox, s_first, X);
      tma_store_wait_read();
    }
    __syncthreads();
  }
  // block partial sums (float-float, fixed order); the last CTA of the solve
  // turns them into the adjoint scalars
  FF dS = {accS, 0.f}, dD = {accD, 0.f};
  block_sum_ff<kNT>(dS, dD);
  last_block_finalize<kNT>(S, 1, (int)gridDim.x, (int)blockIdx.x, dS, dD, true);
  cl.sync();
}

// ===========================================================================
// Backward inverse plane kernel: IFFT(y) + C2R(z) of the three adjoint fields
// V_bar_x, V_bar_y, V_bar_z, then dnormals = gather and the weight-derivative
// part of dpoints, per plane side. One channel per round:
//   y pass  : IFFT along y of this CTA's SPC columns, in their TMA boxes;
//   push    : rows [q R, q R + R) of every box go to CTA q with one bulk copy
//             per (box, q) (a contiguous R x 128 B run of the box);
//   z pass  : C2R of row pairs, in place in the receive buffer (the pair's
//             own storage is also the FFT exchange area);
//   gather  : the channel's share of the point adjoint, read through DSMEM.
// Both source boxes (Q2 for X, Q1 for Y and Z) are fetched by TMA at the
// start; the Z channel's y-inverse is computed from the Q1 box in the Y
// round (u_z is constant along a column, so it commutes with the y-inverse).
// ===========================================================================
// Threads of the adjoint plane kernel: with one CTA per plane (C = 1) the
// CTA is alone on its SM (its two box buffers fill the shared memory), so it
// runs 512 threads (16 warps, at most 128 registers each; from r = 64 on) to hide the
// latency of its serial rounds; cluster CTAs keep 256.
template <int L, int C>
constexpr int binv_threads() { return C == 1 && L >= 64 ? 512 : kNT; }

template <int L, int C>
struct BinvGeo {
  static constexpr int NT = binv_threads<L, C>();
  static constexpr int T = Shape<L>::T, R1 = Shape<L>::R1, G = NT / T;
  static constexpr int R = L / C, H = L / 2, SPC = H / C;
  static constexpr int NB = (SPC + 15) / 16;
  static constexpr int BOX = L * 16;  // float2 per box [ky][16 kz]
  static constexpr int BUF = NB * BOX;
  // receive buffer: R rows x H slots in blocks of 16 slots ([block][row][16],
  // rows swizzled like box rows); with C = 1 the box buffer itself
  static constexpr int RECV = C > 1 ? R * H : 0;
  static constexpr int BLK = (C > 1 ? R : L) * 16;  // float2 per slot block
  static_assert(C == 1 || (SPC % 16 == 0 && R % 8 == 0), "whole boxes, swizzle-aligned runs");
};

template <int L, int C>
constexpr size_t binv_smem() {
  using B = BinvGeo<L, C>;
  return 1024 + sizeof(float2) * ((size_t)2 * B::BUF + B::RECV + L) + sizeof(float) * L +
         sizeof(unsigned) * kListCap;
}

template <int L, int C>
constexpr bool binv_inst() {
  return plane_inst<L, C>() && binv_smem<L, C>() <= 227 * 1024;
}

// float2 index of (row, slot) in a block-of-16-slots buffer.
template <int BLK>
__device__ __forceinline__ int rb(int row, int slot) {
  return (slot >> 4) * BLK + bx(row, slot & 15);
}

// C2R of a row pair whose storage (L float2 through `acc`: A's slots, then
// B's) is also the exchange area and receives the output (a[z], b[z]) at z.
template <int L, class Tw, class Acc>
__device__ __forceinline__ void c2r_pair_ip(int t, const Tw& tw, Acc acc) {
  constexpr int R1 = Shape<L>::R1, T = Shape<L>::T, H = L / 2;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    const int k = t + T * j;
    if (k == 0 || k == H) {
      const float2 a = acc(0), b = acc(H);
      v[j] = (k == 0) ? make_float2(a.x, b.x) : make_float2(a.y, b.y);
    } else if (k < H) {
      const float2 a = acc(k), b = acc(H + k);
      v[j] = make_float2(a.x - b.y, a.y + b.x);
    } else {
      const float2 a = acc(L - k), b = acc(H + L - k);
      v[j] = make_float2(a.x + b.y, b.x - a.y);
    }
  }
  group_sync<T>();  // every lane has read the pair before it becomes exchange
  fft_r<L, +1>(v, t, acc, tw);
#pragma unroll
  for (int j = 0; j < R1; ++j) acc(t + T * j) = v[j];
}

template <int L, int C>
__global__ void __launch_bounds__(binv_threads<L, C>(), binv_smem<L, C>() <= 113 * 1024 ? 2 : 1)
    k_plane_binv(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using B = BinvGeo<L, C>;
  constexpr int NT = B::NT;
  constexpr int H = B::H, R = B::R, SPC = B::SPC, T = B::T, R1 = B::R1, G = B::G;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int X = blockIdx.x / C;
  const int tid = threadIdx.x, g = tid / T, t = tid % T;
  extern __shared__ unsigned char smem_raw[];
  float2* buf0 = aligned_smem(smem_raw);
  float2* buf1 = buf0 + B::BUF;
  float2* recv = buf1 + B::BUF;
  float2* twt = recv + B::RECV;
  float* iu = reinterpret_cast<float*>(twt + L);
  unsigned* list = reinterpret_cast<unsigned*>(iu + L);
  __shared__ uint64_t barL[2], barR;
  __shared__ int list_n;
  pdl_trigger();
  for (int i = tid; i < L; i += NT) {
    iu[i] = S.iu[L + i];  // y axis; the z axis is read from global memory
    twt[i] = S.tw[i];
  }
  pdl_wait();
  const int s_first = c * SPC;
  if (tid == 0) {
    mbar_init(&barL[0], 1);
    mbar_init(&barL[1], 1);
    mbar_init(&barR, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // X channel from Q2 = IFFT_x(-i u_x F), Y and Z from Q1 = IFFT_x(F):
    // the NB boxes of this CTA's SPC slots (x coordinate even: 16-B aligned)
    for (int k = 0; k < 2; ++k) {
      mbar_expect_tx(&barL[k], B::NB * B::BOX * (uint32_t)sizeof(float2));
      for (int b = 0; b < B::NB; ++b)
        tma_load_3d((k ? buf1 : buf0) + b * B::BOX, &S.tmy[k ? kSpD : kSpChi], s_first + 16 * b, 0, X, &barL[k]);
    }
  }
  __syncthreads();
  TwTab<L> twr{twt, t};
  const PlanePoints pp(S, X);
  const int y_lo = c * R;
  // (overlaps the box loads in flight)
  const int nlist = C > 1 ? plane_list<NT>(S, pp, L, y_lo, R, false, list, &list_n) : -1;
  const int nvisit = nlist >= 0 ? nlist : pp.total();
  uint32_t phR = 0;
  bool alive = true;
  // y-domain column `sl` of a box buffer
  auto col = [](float2* bf, int sl, int e) -> float2& { return bf[(sl >> 4) * B::BOX + bx(e, sl & 15)]; };

#pragma unroll 1
  for (int ch = 0; ch < 3; ++ch) {
    float2* src = ch == 1 ? buf1 : buf0;  // y-inverse of channel ch (push source)
    float2* dst = C > 1 ? recv : src;     // this CTA's rows of channel ch
    if (ch < 2) {
      if constexpr (C == 1) __syncthreads();  // buf0 was read by the last gather
      alive = chunk_wait(&barL[ch], 0, S.status) && alive;
      if (alive && c == 0 && g == 0) {
        // column kz = 0 becomes P = X0 + i Xn (Xn: the Nyquist column); the
        // same lanes read these elements again in the y pass below
        const float2* nq = S.spec[ch == 0 ? kSpChi : kSpD] + (size_t)X * L * kpitch(L) + H;
        for (int j = 0; j < R1; ++j) {
          const int ky = t + T * j;
          const float2 n = H >= 16 ? nq[(size_t)ky * kpitch(L)] : col(src, H, ky);
          const float2 x0 = col(src, 0, ky);
          col(src, 0, ky) = make_float2(x0.x - n.y, x0.y + n.x);
        }
      }
      if (alive) {
        for (int sl0 = 0; sl0 < SPC; sl0 += G) {
          const int sl = sl0 + g;
          if (sl < SPC) {  // whole groups; T-lane syncs only
            const int s = s_first + sl;
            float2 v[R1];
#pragma unroll
            for (int j = 0; j < R1; ++j) v[j] = col(src, sl, t + T * j);
            if (ch == 1) {
#pragma unroll
              for (int j = 0; j < R1; ++j) col(buf0, sl, t + T * j) = v[j];  // Q1 for Z
#pragma unroll
              for (int j = 0; j < R1; ++j) v[j] = cmul_iu(v[j], -iu[t + T * j]);
            }
            fft_r<L, +1>(v, t, [&](int e) -> float2& { return col(src, sl, e); }, twr);
#pragma unroll
            for (int j = 0; j < R1; ++j) col(src, sl, t + T * j) = v[j];
            if (ch == 1) {
              group_sync<T>();
#pragma unroll
              for (int j = 0; j < R1; ++j) v[j] = col(buf0, sl, t + T * j);
              fft_r<L, +1>(v, t, [&](int e) -> float2& { return col(buf0, sl, e); }, twr);
              const float ez = s == 0 ? 0.f : -__ldg(S.iu + 2 * L + s);  // z axis
#pragma unroll
              for (int j = 0; j < R1; ++j) col(buf0, sl, t + T * j) = cmul_iu(v[j], ez);
            }
          }
        }
      }
    }
    if constexpr (C > 1) {
      // Arm, make the boxes visible to the async proxy, sync (every receive
      // buffer is free and armed), push, wait for this CTA's rows.
      if (tid == 0) mbar_expect_tx(&barR, R * H * (uint32_t)sizeof(float2));
      fence_async_smem();
      cl.sync();
      if (tid < C * B::NB) {
        const int q = tid / B::NB, b = tid % B::NB;
        const int blk = s_first / 16 + b;  // slot block of the receiver
        bulk_push(dsmem_map(recv + blk * B::BLK, q), src + b * B::BOX + q * R * 16,
                  R * 16 * (uint32_t)sizeof(float2), dsmem_map(&barR, q));
      }
      alive = chunk_wait(&barR, phR, S.status) && alive;
      phR ^= 1;
    } else {
      __syncthreads();
    }
    // C2R along z of row pairs, in place.
    if (alive) {
      for (int p0 = 0; p0 < R / 2; p0 += G) {
        const int p = p0 + g;
        if (p < R / 2) {
          c2r_pair_ip<L>(t, twr, [&](int i) -> float2& { return dst[rb<B::BLK>(2 * p + i / H, i % H)]; });
        }
      }
    }
    if constexpr (C > 1) cl.sync(); else __syncthreads();
    // This channel's share of the point adjoint: dnormals_ch = gather of
    // V_ch, and d/dp of the weights times n_ch V_ch.
    if (alive) {
      for (int i = tid; i < nvisit; i += NT) {
        int dx;
        const int idx = visit_point(list, nlist, pp, i, dx);
        if (!dbg_in_range(S.status, idx, S.N)) continue;
        const float4 a = S.sorted[2 * idx], b = S.sorted[2 * idx + 1];
        const Axis ay = axis_rec(a.y, b.w, 1, L);
        if ((unsigned)(ay.i0 - y_lo) >= (unsigned)R) continue;
        const Axis ax = axis_rec(a.x, b.w, 0, L), az = axis_rec(a.z, b.w, 2, L);
        const float nch = ch == 0 ? a.w : (ch == 1 ? b.x : b.y);
        const float fx = wsel(dx, ax.t), dfx = dx ? (float)L : -(float)L;
        float nb = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int y = dy ? ay.i1 : ay.i0;
          const int q = y / R, lr = y % R, p2 = lr & ~1;
          const float fy = wsel(dy, ay.t), dfy = dy ? (float)L : -(float)L;
          const uint32_t base = dsmem_map(dst, q);
#pragma unroll
          for (int dz = 0; dz < 2; ++dz) {
            const int z = dz ? az.i1 : az.i0;
            const float fz = wsel(dz, az.t), dfz = dz ? (float)L : -(float)L;
            const float2 f = dsmem_ld(base + 8u * rb<B::BLK>(p2 + z / H, z % H));
            const float V = (lr & 1) ? f.y : f.x;
            const float sv = nch * V;
            nb += fx * fy * fz * V;
            c0 += dfx * fy * fz * sv;
            c1 += fx * dfy * fz * sv;
            c2 += fx * fy * dfz * sv;
          }
        }
        float* o = S.slots + ((size_t)dx * S.N + idx) * 6;
        o[ch] = nb;
        if (ch == 0) {
          o[3] = c0;
          o[4] = c1;
          o[5] = c2;
        } else {
          o[3] += c0;
          o[4] += c1;
          o[5] += c2;
        }
      }
    }
  }
  if constexpr (C > 1) cl.sync();  // peers may still read this CTA's rows
}

// ===========================================================================
// The adjoint plane kind split by channel (path code 3): one CTA per (plane
// X, channel) instead of one per plane. A CTA holds one channel's boxes, a
// third of k_plane_binv<L, 1>'s shared memory, so three CTAs share an SM and
// 3r CTAs fill the GPU where the r CTAs of the one-CTA kernel leave SMs idle
// and run their three channels back to back. A channel's arithmetic is that
// of k_plane_binv<L, 1> (the same transforms in the same order: the same
// bits). Its per-point results go to slots of their own, [side][channel]
// [point] as float4 (gather, three weight-derivative terms), which k_combine
// adds in the one-CTA kernel's order.
// ===========================================================================
template <int L>
struct BinvChGeo {
  static constexpr int NT = kNT;
  static constexpr int T = Shape<L>::T, R1 = Shape<L>::R1, G = NT / T;
  static constexpr int H = L / 2;
  static constexpr int NB = (H + 15) / 16;  // boxes of 16 slots
  static constexpr int BOX = L * 16;        // float2 per box [ky][16 kz]
  static constexpr int BUF = NB * BOX;
};

template <int L>
constexpr bool binv_ch_inst() { return L == 64 || L == 128; }

template <int L>
constexpr size_t binv_ch_smem() {
  using B = BinvChGeo<L>;
  return 1024 + sizeof(float2) * ((size_t)B::BUF + L) + sizeof(float) * L;
}

template <int L>
__global__ void __launch_bounds__(BinvChGeo<L>::NT, 3)
    k_plane_binv_ch(const __grid_constant__ Solve s0, const Solve* __restrict__ tab) {
  using B = BinvChGeo<L>;
  constexpr int NT = B::NT, H = B::H, T = B::T, R1 = B::R1, G = B::G;
  const Solve& S = tab ? tab[blockIdx.z] : s0;
  const int X = blockIdx.x, ch = blockIdx.y;
  const int tid = threadIdx.x, g = tid / T, t = tid % T;
  extern __shared__ unsigned char smem_raw[];
  float2* buf = aligned_smem(smem_raw);
  float2* twt = buf + B::BUF;
  float* iu = reinterpret_cast<float*>(twt + L);
  __shared__ uint64_t bar;
  pdl_trigger();
  for (int i = tid; i < L; i += NT) {
    iu[i] = S.iu[L + i];  // y axis; the z axis is read from global memory
    twt[i] = S.tw[i];
  }
  pdl_wait();
  // X channel from Q2 = IFFT_x(-i u_x F), Y and Z from Q1 = IFFT_x(F)
  const int sp = ch == 0 ? kSpChi : kSpD;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, B::NB * B::BOX * (uint32_t)sizeof(float2));
    for (int b = 0; b < B::NB; ++b) tma_load_3d(buf + b * B::BOX, &S.tmy[sp], 16 * b, 0, X, &bar);
  }
  __syncthreads();
  TwTab<L> twr{twt, t};
  const PlanePoints pp(S, X);
  auto col = [&](int sl, int e) -> float2& { return buf[(sl >> 4) * B::BOX + bx(e, sl & 15)]; };
  const bool alive = chunk_wait(&bar, 0, S.status);
  if (alive) {
    if (g == 0) {
      // column kz = 0 becomes P = X0 + i Xn (Xn: the Nyquist column); the
      // same lanes read these elements again in the y pass below
      const float2* nq = S.spec[sp] + (size_t)X * L * kpitch(L) + H;
      for (int j = 0; j < R1; ++j) {
        const int ky = t + T * j;
        const float2 n = nq[(size_t)ky * kpitch(L)];
        const float2 x0 = col(0, ky);
        col(0, ky) = make_float2(x0.x - n.y, x0.y + n.x);
      }
    }
    // IFFT along y of the H columns (Y: times -i u_y first; Z: times -i u_z
    // after, which commutes with the y transform; zero at DC and Nyquist)
    for (int sl0 = 0; sl0 < H; sl0 += G) {
      const int sl = sl0 + g;
      if (sl < H) {  // whole groups; T-lane syncs only
        float2 v[R1];
#pragma unroll
        for (int j = 0; j < R1; ++j) v[j] = col(sl, t + T * j);
        if (ch == 1) {
#pragma unroll
          for (int j = 0; j < R1; ++j) v[j] = cmul_iu(v[j], -iu[t + T * j]);
        }
        fft_r<L, +1>(v, t, [&](int e) -> float2& { return col(sl, e); }, twr);
        if (ch == 2) {
          const float ez = sl == 0 ? 0.f : -__ldg(S.iu + 2 * L + sl);  // z axis
#pragma unroll
          for (int j = 0; j < R1; ++j) v[j] = cmul_iu(v[j], ez);
        }
#pragma unroll
        for (int j = 0; j < R1; ++j) col(sl, t + T * j) = v[j];
      }
    }
  }
  __syncthreads();
  // C2R along z of row pairs, in place.
  if (alive) {
    for (int p0 = 0; p0 < L / 2; p0 += G) {
      const int p = p0 + g;
      if (p < L / 2) {
        c2r_pair_ip<L>(t, twr, [&](int i) -> float2& { return buf[rb<B::BOX>(2 * p + i / H, i % H)]; });
      }
    }
  }
  __syncthreads();
  // This channel's share of the point adjoint: the gather of V_ch, and d/dp
  // of the weights times n_ch V_ch.
  if (!alive) return;
  float4* out = reinterpret_cast<float4*>(S.slots);
  const int nvisit = pp.total();
  for (int i = tid; i < nvisit; i += NT) {
    int dx;
    const int idx = pp.index(i, dx);
    if (!dbg_in_range(S.status, idx, S.N)) continue;
    const float4 a = S.sorted[2 * idx], b = S.sorted[2 * idx + 1];
    const Axis ay = axis_rec(a.y, b.w, 1, L);
    const Axis ax = axis_rec(a.x, b.w, 0, L), az = axis_rec(a.z, b.w, 2, L);
    const float nch = ch == 0 ? a.w : (ch == 1 ? b.x : b.y);
    const float fx = wsel(dx, ax.t), dfx = dx ? (float)L : -(float)L;
    float nb = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int y = dy ? ay.i1 : ay.i0;
      const int p2 = y & ~1;
      const float fy = wsel(dy, ay.t), dfy = dy ? (float)L : -(float)L;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const int z = dz ? az.i1 : az.i0;
        const float fz = wsel(dz, az.t), dfz = dz ? (float)L : -(float)L;
        const float2 f = buf[rb<B::BOX>(p2 + z / H, z % H)];
        const float V = (y & 1) ? f.y : f.x;
        const float sv = nch * V;
        nb += fx * fy * fz * V;
        c0 += dfx * fy * fz * sv;
        c1 += fx * dfy * fz * sv;
        c2 += fx * fy * dfz * sv;
      }
    }
    out[((size_t)dx * 3 + ch) * S.N + idx] = make_float4(nb, c0, c1, c2);
  }
}

template <int L>
static cudaError_t launch_binv_ch_t(const Solve& s, const Solve* tab, int count, cudaStream_t st) {
  if constexpr (!binv_ch_inst<L>()) {
    return cudaErrorInvalidValue;
  } else {
    constexpr size_t smem = binv_ch_smem<L>();
    static bool attr_set = false;
    if (!attr_set) {
      const cudaError_t e =
          cudaFuncSetAttribute(k_plane_binv_ch<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    return launch_k(k_plane_binv_ch<L>, dim3(L, 3, count), dim3(BinvChGeo<L>::NT), smem, st, 1, s, tab);
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
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
    default:
      if constexpr (binv_inst<L, C>()) fn = k_plane_binv<L, C>;
      else return cudaErrorInvalidValue;
      break;
  }
  size_t smem = plane_smem<L, C>(kind);
  if constexpr (fwd_inst<L, C>()) {
    if (kind == 0) smem = fwd_smem<L, C>();
  }
  if (kind == 3) smem = binv_smem<L, C>();
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
  dim3 block(kNT);
  if constexpr (fwd_inst<L, C>()) {
    if (kind == 0) block = dim3(fwd_threads<L, C>());
  }
  if (kind == 3) block = dim3(binv_threads<L, C>());
  return launch_k(fn, dim3(L * C, 1, count), block, smem, st, C, s, tab);
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
  if (C == 0) return launch_pencil(kind, r, s, tab, count, st);
  if (C == kPathSplit) {
    if (kind != 3) return cudaErrorInvalidValue;
    if (r == 64) return launch_binv_ch_t<64>(s, tab, count, st);
    if (r == 128) return launch_binv_ch_t<128>(s, tab, count, st);
    return cudaErrorInvalidValue;
  }
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

template <int L, int C>
static size_t kind_smem(int kind) {
  if constexpr (!plane_inst<L, C>()) {
    return 0;
  } else {
    if (kind == 0) {
      if constexpr (fwd_inst<L, C>()) return fwd_smem<L, C>();
      return 0;
    }
    if (kind == 3) {
      if constexpr (binv_inst<L, C>()) return binv_smem<L, C>();
      return 0;
    }
    return plane_smem<L, C>(kind);
  }
}

size_t plane_smem_bytes(int kind, int r, int C) {
  if (C == 0) return pencil_smem_bytes(kind, r);
  if (C == kPathSplit) {
    if (kind != 3) return 0;
    if (r == 64) return binv_ch_smem<64>();
    if (r == 128) return binv_ch_smem<128>();
    return 0;
  }
  auto pick = [&](auto Lc) -> size_t {
    constexpr int L = decltype(Lc)::value;
    switch (C) {
      case 1: return kind_smem<L, 1>(kind);
      case 2: return kind_smem<L, 2>(kind);
      case 4: return kind_smem<L, 4>(kind);
      case 8: return kind_smem<L, 8>(kind);
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
