// Device side of the two-pass banded forward (Algorithm 2 for large radii):
// the tile bodies of the column pass (pass V) and the row pass (pass H),
// shared by the single-image launches and the batched plan.
//   pass V  per tile of 64 columns x 64 output rows: loads f for the tile's
//           rows plus the W-row halos, generates a_0 and then a_n in shared
//           memory (Algorithm 2's recursion, rescaled by 1/sqrt(n!)), and
//           writes the vertical filtering (w_1 * a_n) of every channel
//           n = 0..N to a workspace of N + 1 planes covering the band;
//   pass H  per tile of 32 rows x 128 output columns: for each channel reads
//           the plane with the W-column halos (cp.async, one channel ahead),
//           filters along the rows, regenerates a_n at the tile's pixels and
//           accumulates Q' and P' (eqs. P, Q), then f_GPA = t_c + sigma_r P'/Q'.
// Out-of-image pixels carry a_n = 0 (zero extension), as in the fused kernels.
#pragma once

#include <type_traits>

#include "bf_internal.h"
#include "gpa_fixed.cuh"

namespace bfk {

constexpr int kBandNT = 256;        // pass H threads per CTA
constexpr int kVNT = 256;           // pass V threads per CTA (two columns, 8 output rows each)
constexpr int kVC = 64, kVB = 64;   // pass V tile: columns, output rows
constexpr int kHT = 32, kHW = 128;  // pass H tile: rows, output columns

struct BandArgs {
  const float *in;
  float *out, *qaux;
  float *ws;        // N + 1 planes of rows x Wp floats
  long long plane;  // floats per plane
  int Wp;           // workspace row pitch: W rounded up to a multiple of 4
  int H, W, pitch;
  int y0, rows;     // the band: image rows y0 .. y0 + rows - 1
  bfi::FilterConsts fc;
};

// Region rows of a pass-V tile: the rotating 16-tap windows read up to row
// 63 + ntaps_pad (taps padded with zeros); a box reads 64 + 2W rows.
__host__ __device__ inline int vpass_rows(int kind, int R, int ntp) {
  return kind == BF_SPATIAL_GAUSS ? kVB + ntp : kVB + 2 * R;
}
// Region columns of a pass-H tile, and the row pitch (1 mod 32: the 32 lanes
// of a warp, one row each, read distinct banks).
__host__ __device__ inline int hpass_cols(int kind, int R, int ntp) {
  return kind == BF_SPATIAL_GAUSS ? kHW + ntp : kHW + 2 * R;
}
__host__ __device__ inline int hpass_pitch(int cols) { return (cols + 31) / 32 * 32 + 1; }

// Whether the forward takes the banded path: Gaussian radii from 12 (except
// 15, which has a compile-time-radius fused kernel) and box radii above 15;
// below these the fused single-pass tiles are faster (measured at 2048^2).
inline bool banded_forward_preferred(int kind, int R) {
  return kind == BF_SPATIAL_GAUSS ? (R >= 12 && R != 15) : R > 15;
}

inline size_t vpass_smem(int kind, int R, int ntp) { return 2 * (size_t)vpass_rows(kind, R, ntp) * kVC * sizeof(float); }
inline size_t hpass_smem(int kind, int R, int ntp) {
  return 2 * (size_t)kHT * hpass_pitch(hpass_cols(kind, R, ntp)) * sizeof(float);
}

// Pass V of tile (bx, by): columns 64 bx.., band rows 64 by.. .
// `taps` holds fc.taps (2W + 1 normalised taps, zero-padded to fc.ntaps_pad):
// the single-image kernels pass their parameter block's copy, the batch its
// launch's table, both constant-bank reads.
template <int KIND>
__device__ __forceinline__ void band_vpass_tile(const BandArgs &A, int bx, int by, float *sm,
                                                const float *taps) {
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RR = vpass_rows(KIND, R, fc.ntaps_pad);
  float *sH = sm, *sA = sm + RR * kVC;
  const int tx = bx * kVC;
  const int tyb = by * kVB;  // band-relative first output row
  const int ty = A.y0 + tyb;
  const int halo = kVB + 2 * R;      // rows of real data; the rest are zero padding
  for (int i = threadIdx.x; i < RR * kVC; i += kVNT) {
    const int r = i / kVC, c = i % kVC;
    const int gy = ty - R + r, gx = tx + c;
    float h = 0.f, a0 = 0.f;
    if (r < halo && gy >= 0 && gy < A.H && gx < A.W) {
      const float d = __ldg(A.in + (long long)gy * A.pitch + gx) - fc.tc;
      h = d * fc.inv_sr;
      a0 = exp2f(d * d * fc.e2c);  // exp(-H^2/2)
    }
    sH[i] = h;
    sA[i] = a0;
  }
  // each thread: two adjacent columns (a packed pair) x RPT output rows; a
  // warp holds one block of RPT rows (the 32 column pairs of the tile)
  constexpr int CS = kVC / 2;                // row stride in column pairs
  constexpr int RPT = kVB * CS / kVNT;       // output rows per thread
  static_assert(CS == 32 && RPT == 8, "a warp per block of 8 output rows");
  const int cp = threadIdx.x % CS, yb = threadIdx.x / CS;  // kVB / RPT blocks of RPT rows
  const int gx = tx + 2 * cp;
  const float2 *col = reinterpret_cast<const float2 *>(sA + RPT * yb * kVC) + cp;
  for (int n = 0; n <= N; ++n) {
    __syncthreads();  // region loaded / previous channel's filtering done
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
      float4 *a4 = reinterpret_cast<float4 *>(sA);
      const float4 *h4 = reinterpret_cast<const float4 *>(sH);
      for (int i = threadIdx.x; i < RR * kVC / 4; i += kVNT) {
        const float4 h = h4[i];
        float4 v = a4[i];
        v.x *= h.x * rs;
        v.y *= h.y * rs;
        v.z *= h.z * rs;
        v.w *= h.w * rs;
        a4[i] = v;
      }
      __syncthreads();
    }
    // a warp whose output rows all lie past the band has nothing to filter
    // (warp-uniform; it still takes part in the advance and the barriers)
    if (tyb + RPT * yb >= A.rows) continue;
    float2 acc[RPT];
    if (KIND == BF_SPATIAL_GAUSS) {
      // window of the RPT rows tap t reads, rotated one row per tap; taps
      // in blocks of RPT (those past 2W are zeros: the table is padded to a
      // multiple of 16, and the region's rows to the padded count)
      float2 win[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        acc[i] = make_float2(0.f, 0.f);
        win[i] = col[i * CS];
      }
      const int L = 2 * R + 1;
      for (int k = 0; k < L; k += RPT) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          const float w = taps[k + j];
          const float2 w2 = make_float2(w, w);
#pragma unroll
          for (int i = 0; i < RPT; ++i) acc[i] = __ffma2_rn(w2, win[(j + i) % RPT], acc[i]);
          win[j] = col[(k + j + RPT) * CS];
        }
      }
    } else {
      float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
      int r = 0;
      for (; r + 3 <= 2 * R; r += 4) {
        s0 = __fadd2_rn(s0, col[r * CS]);
        s1 = __fadd2_rn(s1, col[(r + 1) * CS]);
        s2 = __fadd2_rn(s2, col[(r + 2) * CS]);
        s3 = __fadd2_rn(s3, col[(r + 3) * CS]);
      }
      for (; r <= 2 * R; ++r) s0 = __fadd2_rn(s0, col[r * CS]);
      float2 s = __fadd2_rn(__fadd2_rn(s0, s1), __fadd2_rn(s2, s3));
      acc[0] = s;
#pragma unroll
      for (int i = 1; i < RPT; ++i) {
        const float2 in = col[(i + 2 * R) * CS], out = col[(i - 1) * CS];
        s = __fadd2_rn(s, __fadd2_rn(in, make_float2(-out.x, -out.y)));
        acc[i] = s;
      }
    }
    // columns W..Wp-1 of the workspace receive zeros (their a_n are 0)
    if (gx < A.Wp) {
      float *dst = A.ws + (long long)n * A.plane + gx;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int orow = tyb + RPT * yb + i;
        if (orow < A.rows) *reinterpret_cast<float2 *>(dst + (long long)orow * A.Wp) = acc[i];
      }
    }
  }
}

// Pass H of tile (bx, by): output columns 128 bx.., band rows 32 by.. .
template <int KIND>
__device__ __forceinline__ void band_hpass_tile(const BandArgs &A, int bx, int by, float *sm,
                                                const float *taps) {
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RC = hpass_cols(KIND, R, fc.ntaps_pad), P = hpass_pitch(RC);
  float *const buf0 = sm, *const buf1 = sm + kHT * P;
  const int tx = bx * kHW;
  const int tyb = by * kHT;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;  // row lane, 16 columns seg

  // plane n of rows tyb.., columns tx - W.., into b; each warp copies four
  // rows, its lanes consecutive columns.  The region's in-image columns are
  // j in [j0, j1) of every row, the same for every channel; the cells outside
  // the image or the band are zeroed once in both buffers here (no copy ever
  // writes them), so each channel copies the in-image cells and nothing else.
  const int j0 = max(0, R - tx), j1 = min(RC, A.W - tx + R);
  for (int r = seg; r < kHT; r += kBandNT / 32) {
    const bool rin = tyb + r < A.rows;
    for (int j = lane; j < RC; j += 32)
      if (!rin || j < j0 || j >= j1) buf0[r * P + j] = buf1[r * P + j] = 0.f;
  }
  auto load = [&](int n, float *b) {
    // column j of the region is image column tx - W + j (>= 0 for j >= j0)
    const float *src = A.ws + (long long)n * A.plane + (long long)tyb * A.Wp + (tx - R);
    for (int r = seg; r < kHT && tyb + r < A.rows; r += kBandNT / 32) {
      const float *srow = src + (long long)r * A.Wp;
      float *drow = b + r * P;
      for (int j = j0 + lane; j < j1; j += 32) bfk::cp_async4(drow + j, srow + j);
    }
  };

  // the thread's 16 pixels: row ty + lane, columns tx + 16 seg + i
  const int gy = A.y0 + tyb + lane;
  const bool rowin = tyb + lane < A.rows;
  float a[16], H[16], Q[16], Pp[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int gx = tx + 16 * seg + i;
    float h = 0.f, a0 = 0.f;
    if (rowin && gx < A.W) {
      const float d = __ldg(A.in + (long long)gy * A.pitch + gx) - fc.tc;
      h = d * fc.inv_sr;
      a0 = exp2f(d * d * fc.e2c);
    }
    a[i] = a0;
    H[i] = h;
    Q[i] = Pp[i] = 0.f;
  }

  load(0, buf0);
  bfk::cp_async_commit();
  const float *vrow0 = nullptr;
  for (int n = 0; n <= N; ++n) {
    if (n < N) {
      load(n + 1, (n & 1) ? buf0 : buf1);
      bfk::cp_async_commit();
      bfk::cp_async_wait<1>();
    } else {
      bfk::cp_async_wait<0>();
    }
    __syncthreads();  // plane n is in buffer n & 1 for every thread
    vrow0 = ((n & 1) ? buf1 : buf0) + lane * P + 16 * seg;
    if (tx + 16 * seg >= A.W) {  // the warp's 16 columns lie past the image (warp-uniform)
      __syncthreads();           // the barrier that frees buffer n & 1
      continue;
    }
    float Ab[16];
    if (KIND == BF_SPATIAL_GAUSS) {
      float win[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        Ab[i] = 0.f;
        win[i] = vrow0[i];
      }
      const int L = 2 * R + 1, kl = (L - 1) & ~15;  // as in pass V: a last block of 8 or 16
      auto block = [&](int k, auto taps_tag) {
        constexpr int NTB = decltype(taps_tag)::value;
#pragma unroll
        for (int j = 0; j < NTB; ++j) {
          const float w = taps[k + j];
#pragma unroll
          for (int i = 0; i < 16; ++i) Ab[i] = fmaf(w, win[(j + i) & 15], Ab[i]);
          win[j] = vrow0[k + j + 16];
        }
      };
      for (int k = 0; k < kl; k += 16) block(k, std::integral_constant<int, 16>{});
      if (L - kl > 8) block(kl, std::integral_constant<int, 16>{});
      else block(kl, std::integral_constant<int, 8>{});
    } else {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int j = 0;
      for (; j + 3 <= 2 * R; j += 4) {
        s0 += vrow0[j];
        s1 += vrow0[j + 1];
        s2 += vrow0[j + 2];
        s3 += vrow0[j + 3];
      }
      for (; j <= 2 * R; ++j) s0 += vrow0[j];
      float s = (s0 + s1) + (s2 + s3);
      Ab[0] = s;
#pragma unroll
      for (int i = 1; i < 16; ++i) {
        s += vrow0[i + 2 * R] - vrow0[i - 1];
        Ab[i] = s;
      }
    }
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float aold = a[i];  // a_{n-1}
      const float an = n > 0 ? aold * (H[i] * rs) : aold;
      if (n < N) Q[i] = fmaf(an, Ab[i], Q[i]);
      if (n > 0) Pp[i] = fmaf(sq * aold, Ab[i], Pp[i]);
      a[i] = an;
    }
    __syncthreads();  // buffer n & 1 is free for plane n + 2
  }

  if (!rowin) return;
  const long long ro = (long long)gy * A.pitch;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int gx = tx + 16 * seg + i;
    if (gx < A.W) {
      A.out[ro + gx] = fmaf(fc.sr, __fdividef(Pp[i], Q[i]), fc.tc);  // 2-ulp division
      if (A.qaux) A.qaux[ro + gx] = Q[i] * fc.qscale;
    }
  }
}

}  // namespace bfk
