// Fused forward tile specialised for a compile-time radius R.
//
// Same algorithm and tile geometry as gpa_tile.cuh (phase V down region
// columns, phase H along output rows, N + 1 channels per tile), but with R
// known at compile time every loop over rows and taps is unrolled, so:
//  - each column thread keeps its RH = TH + 2R power-image values a_n in
//    registers (only H = (f - t_c)/sigma_r stays in shared memory, read once
//    per row per channel);
//  - Gaussian taps are read as constant-bank operands of the FMAs (the
//    kernel's parameter block), with no shared-memory loads;
//  - the shared rows are padded so that no index needs clamping.
// Phase V also copies the TH centre rows of a_n to shared memory (sC) for the
// recombination in phase H.
#pragma once

#include "gpa_tile.cuh"

namespace bfk {

template <int R, int NT, int TH>
struct FixedGeom {
  static constexpr int RH = TH + 2 * R;
  static constexpr int TW = NT - 2 * R;
  static constexpr int KH = TH;
  static constexpr int L = 2 * R + 1;
  static constexpr int VP = NT + KH + 1;  // odd; phase-H windows never need clamping
  static constexpr size_t smem_bytes() {
    return ((size_t)2 * TH * VP + (size_t)RH * NT) * sizeof(float);
  }
};

template <int KIND, int R, int NT, int TH>
__device__ __forceinline__ void gpa_fwd_tile_fixed(const TileIO &io, const bfi::FilterConsts &fc,
                                                   int ty0, int tx0, float *smem) {
  using G = FixedGeom<R, NT, TH>;
  constexpr int RH = G::RH, TW = G::TW, KH = G::KH, L = G::L, VP = G::VP;
  static_assert(TW >= KH, "tile too narrow for this radius");
  static_assert(NT % TH == 0, "NT must be a multiple of TH");
  float *sV = smem;            // TH x VP   vertical-pass results
  float *sC = sV + TH * VP;    // TH x VP   centre rows of a_n
  float *sH = sC + TH * VP;    // RH x NT   H of the region
  const int c = threadIdx.x;
  const int N = fc.N;

  float a[RH];
  {
    // all loads of the column first (RH independent loads in flight), then
    // the arithmetic; out-of-image pixels read as t_c with a_0 = 0
    const int gx = tx0 - R + c;
    const bool colin = gx >= 0 && gx < io.W;
    const float *src = io.in + gx;
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      const int gy = ty0 - R + r;
      a[r] = (colin && gy >= 0 && gy < io.H) ? __ldg(src + (long long)gy * io.pitch) : fc.tc;
    }
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      const int gy = ty0 - R + r;
      const bool in = colin && gy >= 0 && gy < io.H;
      const float h = (a[r] - fc.tc) * fc.inv_sr;
      a[r] = in ? expf(-0.5f * h * h) : 0.f;  // the one transcendental of Algorithm 2
      sH[r * NT + c] = h;
    }
  }

  const int hy = c % TH;
  const int hx0 = (c / TH) * KH;
  const bool hact = hx0 < TW;
  float Q[KH], P[KH], ap[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) Q[k] = P[k] = ap[k] = 0.f;
  const float *vrow = sV + hy * VP + hx0;
  const float *crow = sC + hy * VP + R + hx0;

  for (int n = 0; n <= N; ++n) {
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
    __syncthreads();  // phase H of the previous channel is done with sV / sC

    // ---------------- phase V (registers): advance, centre copy, vertical pass
    if (n > 0) {
#pragma unroll
      for (int r = 0; r < RH; ++r) a[r] *= sH[r * NT + c] * rs;
    }
#pragma unroll
    for (int y = 0; y < TH; ++y) sC[y * VP + c] = a[y + R];
    if (KIND == BF_SPATIAL_GAUSS) {
#pragma unroll
      for (int y = 0; y < TH; ++y) {
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < L; ++t) acc = fmaf(fc.taps[t], a[y + t], acc);
        sV[y * VP + c] = acc;
      }
    } else {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < L; ++r) s += a[r];
      sV[c] = s;
#pragma unroll
      for (int y = 1; y < TH; ++y) {
        s += a[y + 2 * R] - a[y - 1];
        sV[y * VP + c] = s;
      }
    }
    __syncthreads();

    // ---------------- phase H: horizontal pass + recombination
    if (hact) {
      float Ab[KH];
      if (KIND == BF_SPATIAL_GAUSS) {
        float win[KH];
#pragma unroll
        for (int i = 0; i < KH; ++i) {
          Ab[i] = 0.f;
          win[i] = vrow[i];
        }
#pragma unroll
        for (int t = 0; t < L; ++t) {
          const float w = fc.taps[t];
#pragma unroll
          for (int i = 0; i < KH; ++i) Ab[i] = fmaf(w, win[(t + i) % KH], Ab[i]);
          win[t % KH] = vrow[t + KH];
        }
      } else {
        float v[KH + 2 * R];
#pragma unroll
        for (int i = 0; i < KH + 2 * R; ++i) v[i] = vrow[i];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) s += v[i];
        Ab[0] = s;
#pragma unroll
        for (int j = 1; j < KH; ++j) {
          s += v[j + 2 * R] - v[j - 1];
          Ab[j] = s;
        }
      }
      const bool qn = n < N, pn = n > 0;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const float av = crow[k];
        if (qn) Q[k] = fmaf(av, Ab[k], Q[k]);
        if (pn) P[k] = fmaf(sq * ap[k], Ab[k], P[k]);
        ap[k] = av;
      }
    }
  }

  if (hact) {
    const int gy = ty0 + hy;
    if (gy < io.H) {
      float *orow = io.out + (long long)gy * io.pitch;
      float *qrow = io.qaux ? io.qaux + (long long)gy * io.pitch : nullptr;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const int gx = tx0 + hx0 + k;
        if (hx0 + k < TW && gx < io.W) {
          orow[gx] = fmaf(fc.sr, P[k] / Q[k], fc.tc);
          if (qrow) qrow[gx] = Q[k] * fc.qscale;
        }
      }
    }
  }
}

}  // namespace bfk
