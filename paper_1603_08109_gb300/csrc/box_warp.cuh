// Warp-strip streaming forward for the box spatial kernel at small order
// (N <= 8) and small radius (W <= 8): the memory-bound regime of Algorithm 2.
//
// Each warp owns a strip of 32 C region columns, C = 8 or 4 consecutive
// columns per lane (the ceil(W / C) lanes at each end carry the W-column
// halos, the others produce the strip's output columns: 240 for C = 8, 120
// or 112 for C = 4 and W = 3 or 5), and a band of output rows.  Four columns
// per lane halve the per-warp ring and the registers, so about twice as many
// warps are resident per SM, for twice the halo shuffles per pixel and more
// halo lanes.  It streams down the
// band two rows at a time with no block barrier and no value passed through
// shared memory from one thread to another:
//   * input rows are copied with cp.async into a per-lane ring in shared
//     memory DP row pairs ahead of use; every lane reads back only the bytes
//     it copied itself;
//   * per column and channel n the running vertical window sum
//     V_n = sum of u_n over the 2W + 1 rows of the window stays in registers,
//     u_n = e^{-H^2/2} H^n being the power image F_n of Algorithm 2 (unscaled:
//     |u_n| <= (n/e)^{n/2} <= 75 for n <= 8).  A row leaving the window is
//     regenerated from its ring entry by the same instructions that produced
//     it on entry, so what is subtracted is bitwise what was added;
//   * horizontal window sums S_n take the W halo columns from the lanes one
//     (or, for C = 4 and W > 4, two) positions away by warp shuffles;
//   * Algorithm 2's sums at the centre pixel are P = sum_{n<N} H^n S_{n+1}/n!
//     and Q = sum_{n<N} H^n S_n/n! (Horner form); the centre's factor
//     e^{-H^2/2} of Q' and P' cancels in f_GPA = t_c + sigma_r P/Q and is
//     computed only when Q' = e^{-H^2/2} Q w(0) is requested.
// Column pairs go through the packed two-lane FP32 instructions (fma / add /
// mul on float2, each lane rounded exactly as the scalar operation).
// Out-of-image columns of the ring hold a sentinel intensity whose u_n are
// exactly 0 (zero extension of the power images); out-of-image rows are
// skipped by warp-uniform branches.  Strips and bands that touch no image
// edge run a loop without any of these checks.
#pragma once

#include "gpa_fixed.cuh"
#include "gpa_tile.cuh"

namespace bfk {

struct WarpStripArgs {
  TileIO io;
  float tc, sr;
  float kg, kg0;    // g = f kg + kg0 = (f - t_c) sqrt(log2(e)/2) / sigma_r; u_0 = 2^(-g^2)
  float hs, hs0;    // H = f hs + hs0 = (f - t_c) / sigma_r
  float qscale;     // w(0) = 1 / (2W + 1)^2: normalised Q'
  float sentinel;   // intensity with u_n = 0 exactly (t_c + 1e4 sigma_r)
  float inv_n[12];  // 1 / n (entry 0 unused)
  int band;         // output rows per warp (even)
  int nstrips, nbands;
  int nimg;               // images of the same size and parameters
  long long img_stride;   // elements from one image (in, out, Q') to the next
  int vec_in;       // input rows 16-byte aligned: 16-byte copies
  int vec_out;      // out (and Q') rows 16-byte aligned: 16-byte stores
};

template <int R, int DP = 1, int C = 8>
struct WarpStripGeom {
  static_assert(C == 4 || C == 8, "4 or 8 columns per lane");
  static constexpr int SW = 32 * C;             // region columns of a strip
  static constexpr int HL = (R + C - 1) / C;    // halo lanes on each side
  static constexpr int TW = SW - 2 * HL * C;    // output columns of a strip
  static constexpr int NCH = C / 4;             // 16-byte chunks per lane and row
  static constexpr int L = 2 * R + 1;
  // ring rows: the L + 2 rows a row pair reads (two leave, two enter) plus
  // the DP pairs in flight
  static constexpr int RS = L + 2 + 2 * DP;
  static constexpr size_t warp_floats = (size_t)RS * SW;
};

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ float ws_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ws_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Per-warp constants as packed pairs.
struct WsConst {
  float2 kg, kg0, hs, hs0;
};

// u_0 of two intensities: 2^(-g^2) by the hardware base-2 exponential (<= 2 ulp
// relative).  The same instruction sequence serves a row entering and leaving,
// so the two results are bitwise equal.
__device__ __forceinline__ float2 ws_u0(const WsConst &K, float2 f) {
  const float2 g = __ffma2_rn(f, K.kg, K.kg0);
  const float2 t = __fmul2_rn(g, g);
  return make_float2(ws_ex2(-t.x), ws_ex2(-t.y));
}

// The lane's C intensities of one ring row (chunk j at slot + 128 j).
template <int C>
__device__ __forceinline__ void ws_load(const float *slot, float2 (&f)[C / 2]) {
#pragma unroll
  for (int j = 0; j < C / 4; ++j) {
    const float4 v = *reinterpret_cast<const float4 *>(slot + 128 * j);
    f[2 * j] = make_float2(v.x, v.y);
    f[2 * j + 1] = make_float2(v.z, v.w);
  }
}

// V_n += u_n (ADD) or V_n -= u_n for the lane's intensities of one row.  The
// subtraction is fma(u_n, -1, V_n), rounded as V_n + (-u_n), with u_n from
// the same instructions as on entry.
template <int NN, int NP, bool ADD>
__device__ __forceinline__ void ws_update(const WsConst &K, float2 (&V)[NN][NP],
                                          const float2 (&f)[NP]) {
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float2 u = ws_u0(K, f[p]);
    const float2 h = __ffma2_rn(f[p], K.hs, K.hs0);
#pragma unroll
    for (int n = 0; n < NN; ++n) {
      if (n > 0) u = __fmul2_rn(u, h);
      V[n][p] = ADD ? __fadd2_rn(V[n][p], u) : __ffma2_rn(u, f2(-1.f), V[n][p]);
    }
  }
}

template <int M>
__device__ __forceinline__ float ws_tree_sum(const float *e) {
  if constexpr (M == 1) {
    return e[0];
  } else {
    return ws_tree_sum<M / 2>(e) + ws_tree_sum<M - M / 2>(e + M / 2);
  }
}

// Box sums over 2W + 1 columns of v at the lane's C columns; the W columns on
// each side come from the neighbouring lanes (one or two lanes away).
template <int R, int C>
__device__ __forceinline__ void ws_hsum(const float2 (&v2)[C / 2], float2 (&S2)[C / 2]) {
  constexpr unsigned FULL = 0xffffffffu;
  float v[C];
#pragma unroll
  for (int p = 0; p < C / 2; ++p) {
    v[2 * p] = v2[p].x;
    v[2 * p + 1] = v2[p].y;
  }
  float e[C + 2 * R];
#pragma unroll
  for (int k = 0; k < C; ++k) e[R + k] = v[k];
#pragma unroll
  for (int d = 1; d <= R; ++d) {  // column d to the left / right of the lane's columns
    const int m = (d + C - 1) / C;  // lanes away (compile-time after unrolling)
    e[R - d] = __shfl_up_sync(FULL, v[C * m - d], m);
    e[R + C - 1 + d] = __shfl_down_sync(FULL, v[d - 1 - C * (m - 1)], m);
  }
  float S[C];
  float s = ws_tree_sum<2 * R + 1>(e);
  S[0] = s;
#pragma unroll
  for (int k = 1; k < C; ++k) {
    s += e[k + 2 * R] - e[k - 1];
    S[k] = s;
  }
#pragma unroll
  for (int p = 0; p < C / 2; ++p) S2[p] = make_float2(S[2 * p], S[2 * p + 1]);
}

// f_GPA (and optionally Q') of one output row from the window sums V and the
// centre intensities fc.
template <int R, int NN, int C, bool FULL>
__device__ __forceinline__ void ws_row_out(const WarpStripArgs &A, const WsConst &K,
                                           const float2 (&V)[NN][C / 2],
                                           const float2 (&fc)[C / 2], int yo, int x0,
                                           bool store, long long off) {
  constexpr int N = NN - 1, NP = C / 2;
  float2 H[NP], Pa[NP], Qa[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) H[p] = __ffma2_rn(fc[p], K.hs, K.hs0);
#pragma unroll
  for (int m = NN - 1; m >= 0; --m) {
    float2 S[NP];
    ws_hsum<R, C>(V[m], S);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      if (m == N) {
        Pa[p] = S[p];
      } else {
        if (m >= 1) Pa[p] = __ffma2_rn(__fmul2_rn(H[p], f2(A.inv_n[m])), Pa[p], S[p]);
        Qa[p] = m == N - 1 ? S[p]
                           : __ffma2_rn(__fmul2_rn(H[p], f2(A.inv_n[m + 1])), Qa[p], S[p]);
      }
    }
  }
  if (!store) return;
  const TileIO &io = A.io;
  float2 o[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    // P/Q by the approximate reciprocal (<= 2 ulp, as __fdividef)
    const float2 r = __fmul2_rn(Pa[p], make_float2(ws_rcp(Qa[p].x), ws_rcp(Qa[p].y)));
    o[p] = __ffma2_rn(f2(A.sr), r, f2(A.tc));
  }
  float *orow = io.out + off + (long long)yo * io.pitch + x0;
  const bool full = FULL || (A.vec_out && x0 + C <= io.W);
  if (full) {
#pragma unroll
    for (int j = 0; j < C / 4; ++j)
      reinterpret_cast<float4 *>(orow)[j] =
          make_float4(o[2 * j].x, o[2 * j].y, o[2 * j + 1].x, o[2 * j + 1].y);
  } else {
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (x0 + k < io.W) orow[k] = k & 1 ? o[k / 2].y : o[k / 2].x;
  }
  if (io.qaux) {
    float2 q[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) q[p] = __fmul2_rn(__fmul2_rn(ws_u0(K, fc[p]), Qa[p]), f2(A.qscale));
    float *qrow = io.qaux + off + (long long)yo * io.pitch + x0;
    if (full) {
#pragma unroll
      for (int j = 0; j < C / 4; ++j)
        reinterpret_cast<float4 *>(qrow)[j] =
            make_float4(q[2 * j].x, q[2 * j].y, q[2 * j + 1].x, q[2 * j + 1].y);
    } else {
#pragma unroll
      for (int k = 0; k < C; ++k)
        if (x0 + k < io.W) qrow[k] = k & 1 ? q[k / 2].y : q[k / 2].x;
    }
  }
}

// The band loop.  FAST: every row the loop touches is inside the image and
// every lane's C columns are inside the image with 16-byte aligned rows.
template <int R, int NN, int DP, int C, bool FAST>
__device__ __forceinline__ void ws_band(const WarpStripArgs &A, const WsConst &K, float *my,
                                        int x0, int yo0, int yo1, int cnt0, int cnt1,
                                        long long off) {
  using G = WarpStripGeom<R, DP, C>;
  constexpr int SW = G::SW, L = G::L, RS = G::RS, NP = C / 2, HL = G::HL;
  const TileIO &io = A.io;
  const bool vec0 = FAST || (A.vec_in && cnt0 == 4), vec1 = FAST || (A.vec_in && cnt1 == 4);
  auto issue = [&](int y, int slot) {
    if (FAST || (y >= 0 && y < io.H)) {
      const float *src = io.in + off + (long long)y * io.pitch + x0;
      float *dst = my + slot * SW;
      if (vec0) {
        cp_async16(dst, src);
      } else {
        for (int e = 0; e < cnt0; ++e) cp_async4(dst + e, src + e);
      }
      if constexpr (C == 8) {
        if (vec1) {
          cp_async16(dst + 128, src + 4);
        } else {
          for (int e = 0; e < cnt1; ++e) cp_async4(dst + 128 + e, src + 4 + e);
        }
      }
    }
  };
  auto wrap = [](int s) { return s >= RS ? s - RS : s; };  // s < 2 RS

  float2 V[NN][NP];
#pragma unroll
  for (int n = 0; n < NN; ++n)
#pragma unroll
    for (int p = 0; p < NP; ++p) V[n][p] = make_float2(0.f, 0.f);

  const int lane = threadIdx.x & 31;
  const bool writer = lane >= HL && lane < 32 - HL;
  // region row rho = 0.. is image row yo0 - R + rho and lives in ring slot
  // rho mod RS; rows rho >= 2W complete the window of output row rho - 2W
  const int nrows = (yo1 - yo0) + 2 * R;
#pragma unroll
  for (int k = 0; k < DP; ++k) {  // the first DP pairs
    issue(yo0 - R + 2 * k, 2 * k);
    issue(yo0 - R + 2 * k + 1, 2 * k + 1);
    cp_async_commit();
  }
  int s0 = 0;  // slot of row rho
  for (int rho = 0; rho < nrows; rho += 2) {
    const int y = yo0 - R + rho;
    // pair rho + 2 DP goes to the slots of rows rho - L - 2 and rho - L - 1,
    // which left the window in the previous iteration
    issue(y + 2 * DP, wrap(s0 + 2 * DP));
    issue(y + 2 * DP + 1, wrap(s0 + 2 * DP + 1));
    cp_async_commit();
    cp_async_wait<DP>();  // rows rho and rho + 1 have landed
    const int s1 = wrap(s0 + 1);
    float2 fe0[NP], fe1[NP];
    ws_load<C>(my + s0 * SW, fe0);
    ws_load<C>(my + s1 * SW, fe1);
    if (rho < 2 * R) {  // warm-up: the window above the band's first output row
      if (FAST || (y >= 0 && y < io.H)) ws_update<NN, NP, true>(K, V, fe0);
      if (FAST || (y + 1 >= 0 && y + 1 < io.H)) ws_update<NN, NP, true>(K, V, fe1);
    } else {
      const int sl0 = wrap(s0 + RS - L), sl1 = wrap(s1 + RS - L);
      const int sc0 = wrap(s0 + RS - R), sc1 = wrap(s1 + RS - R);
      float2 fl0[NP], fl1[NP], fc0[NP], fc1[NP];
      ws_load<C>(my + sl0 * SW, fl0);
      ws_load<C>(my + sl1 * SW, fl1);
      ws_load<C>(my + sc0 * SW, fc0);
      ws_load<C>(my + sc1 * SW, fc1);
      const int yo = y - R;  // output rows yo, yo + 1 (the second may be past the band)
      // entering rows y, y + 1; leaving rows y - L, y + 1 - L (entered in this band
      // when rho >= L)
      if (FAST || y < io.H) ws_update<NN, NP, true>(K, V, fe0);
      if (rho >= L && (FAST || y - L >= 0)) ws_update<NN, NP, false>(K, V, fl0);
      ws_row_out<R, NN, C, FAST>(A, K, V, fc0, yo, x0, writer, off);
      if (FAST || y + 1 < io.H) ws_update<NN, NP, true>(K, V, fe1);
      if (FAST || y + 1 - L >= 0) ws_update<NN, NP, false>(K, V, fl1);
      ws_row_out<R, NN, C, FAST>(A, K, V, fc1, yo + 1, x0, writer && yo + 1 < yo1, off);
    }
    s0 = wrap(s0 + 2);
  }
  cp_async_wait<0>();
}

// One warp: strip `strip` (TW output columns), band `band` (A.band output rows)
// of the image whose in, out and Q' start `off` elements after io's.  The
// warp's ring holds RS rows of SW floats, lane l's chunk j of a row at offset
// 128 j + 4 l.
template <int R, int NN, int DP = 1, int C = 8>
__device__ __forceinline__ void box_warp_strip(const WarpStripArgs &A, int strip, int band,
                                               long long off, float *ring) {
  using G = WarpStripGeom<R, DP, C>;
  constexpr int SW = G::SW, RS = G::RS;
  static_assert(R >= 1 && R <= 8 && G::HL <= 2, "the halo comes from at most two lanes");
  static_assert(NN >= 2 && NN <= 9, "order range of the warp-strip kernel");
  const TileIO &io = A.io;
  const int lane = threadIdx.x & 31;
  const int x0 = strip * G::TW - G::HL * C + C * lane;  // first region column of this lane
  const int yo0 = band * A.band, yo1 = min(io.H, yo0 + A.band);
  float *my = ring + 4 * lane;
  WsConst K;
  K.kg = f2(A.kg);
  K.kg0 = f2(A.kg0);
  K.hs = f2(A.hs);
  K.hs0 = f2(A.hs0);

  // per chunk of 4 columns: valid column count (chunks start on multiples of 4);
  // out-of-image columns of every ring row hold the sentinel
  const int cnt0 = x0 < 0 ? 0 : max(0, min(4, io.W - x0));
  const int cnt1 = C == 4 ? 4 : (x0 + 4 < 0 ? 0 : max(0, min(4, io.W - x0 - 4)));
  for (int e = cnt0; e < 4; ++e)
    for (int r = 0; r < RS; ++r) my[r * SW + e] = A.sentinel;
  if constexpr (C == 8)
    for (int e = cnt1; e < 4; ++e)
      for (int r = 0; r < RS; ++r) my[r * SW + 128 + e] = A.sentinel;
  // rows touched: yo0 - W .. yo1 + W + 2 DP - 1 (the last prefetches)
  const bool rows_in = yo0 - R >= 0 && yo1 + R + 2 * DP <= io.H;
  const bool fast = __all_sync(0xffffffffu, rows_in && A.vec_in && A.vec_out && cnt0 == 4 &&
                                                cnt1 == 4);
  if (fast)
    ws_band<R, NN, DP, C, true>(A, K, my, x0, yo0, yo1, cnt0, cnt1, off);
  else
    ws_band<R, NN, DP, C, false>(A, K, my, x0, yo0, yo1, cnt0, cnt1, off);
}

}  // namespace bfk
