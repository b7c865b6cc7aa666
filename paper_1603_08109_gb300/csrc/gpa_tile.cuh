// Fused Gaussian-polynomial bilateral filter: the per-tile device code.
//
// One CTA computes an output tile of TH rows x TW = NT - 2R columns.  Its
// region (the tile plus an R-pixel halo, RH = TH + 2R rows x NT columns) is
// read once from global memory; shared memory then holds, per region pixel,
// the current power image value a_n and H = (f - t_c) / sigma_r
// (Algorithm 2's images F and H, rescaled by 1/sqrt(n!)).  For every channel
// n = 0..N (the N + 1 filterings of Algorithm 2):
//
//   phase V  thread c owns region column c.  It streams down the column,
//            advancing a_n = a_{n-1} * H / sqrt(n) in place (eq. intImg) and
//            feeding the values straight into the vertical pass of the
//            separable spatial filter (eq. spatialFiltering): a running sum
//            for the box, a register-window FIR for the Gaussian.  The TH
//            vertical results per column go to shared memory (sV).
//   phase H  thread (y, segment) owns KH consecutive outputs of row y.  It
//            applies the horizontal pass on sV and accumulates
//            Q' += a_n (w*a_n) [n < N] and P' += sqrt(n) a_{n-1} (w*a_n) [n >= 1]
//            in registers (eqs. P and Q after rescaling).
//
// Out-of-image region pixels carry a_0 = 0, so every sum runs over the
// in-image neighbours only.  Only f is read and out (plus optional Q') is
// written: the N + 1 power images never leave the SM.
//
// Shared-memory layout: the region rows are NT + 1 float2 apart so that the
// phase-H reads of centre values (lanes walk down rows) fall in distinct
// banks; sV rows are NT + 1 floats apart for the same reason.  Gaussian taps
// beyond 2R are skipped with a warp-uniform branch (no padded FMAs).
#pragma once

#include <cuda_runtime.h>

#include "bf_internal.h"

namespace bfk {

struct TileIO {
  const float *in;
  float *out;
  float *qaux;      // optional normalised Q'
  float *abar;      // optional stored filtered power images (planes)
  long long plane_stride;
  int H, W, pitch;
};

__host__ __device__ constexpr int vpitch(int nt) { return nt + 1; }
__host__ __device__ constexpr int rpitch(int nt) { return nt + 1; }

// Shared-memory bytes of the forward tile body.
__host__ __device__ inline size_t fwd_smem_bytes(int NT, int TH, int R, int ntaps_pad) {
  return (size_t)(TH + 2 * R) * rpitch(NT) * sizeof(float2) +
         (size_t)TH * vpitch(NT) * sizeof(float) +
         (size_t)(ntaps_pad > 0 ? ntaps_pad : 1) * sizeof(float);
}

// Advance the power image of one region pixel to channel n (n > 0) in place.
__device__ __forceinline__ float advance(float2 *p, int n, float rs) {
  if (n == 0) return p->x;
  const float2 v = *p;
  const float a = v.x * (v.y * rs);
  p->x = a;
  return a;
}

template <int KIND, int NT, int TH, int KH, bool STORE>
__device__ __forceinline__ void gpa_fwd_tile(const TileIO &io, const bfi::FilterConsts &fc,
                                             const float *taps_src, int ty0, int tx0,
                                             float *smem) {
  static_assert(KH == TH, "phase H covers TH x ceil(TW/KH) <= NT items only when KH == TH");
  static_assert(NT % TH == 0, "NT must be a multiple of TH");
  const int R = fc.R;
  const int RH = TH + 2 * R;
  const int TW = NT - 2 * R;
  const int N = fc.N;
  const int ntaps = 2 * R + 1;
  constexpr int VP = vpitch(NT);
  constexpr int RP = rpitch(NT);
  float2 *sAH = reinterpret_cast<float2 *>(smem);
  float *sV = smem + 2 * RH * RP;
  float *sT = sV + TH * VP;
  const int tid = threadIdx.x;

  if (KIND == BF_SPATIAL_GAUSS)
    for (int i = tid; i < fc.ntaps_pad; i += NT) sT[i] = taps_src[i];

  // ---- region load: f -> (a_0, H); one pass over the tile + halo
  {
    const int gx = tx0 - R + tid;
    const bool colin = gx >= 0 && gx < io.W;
    const float *src = io.in + gx;
    for (int r = 0; r < RH; ++r) {
      const int gy = ty0 - R + r;
      float a0 = 0.f, h = 0.f;
      if (colin && gy >= 0 && gy < io.H) {
        const float f = __ldg(src + (long long)gy * io.pitch);
        h = (f - fc.tc) * fc.inv_sr;
        a0 = expf(-0.5f * h * h);  // the one transcendental of Algorithm 2
      }
      sAH[r * RP + tid] = make_float2(a0, h);
    }
  }

  // ---- phase-H ownership (fixed for the whole channel loop)
  const int hy = tid % TH;
  const int hx0 = (tid / TH) * KH;
  const bool hact = hx0 < TW;
  float Q[KH], P[KH], ap[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) Q[k] = P[k] = ap[k] = 0.f;

  float2 *col = sAH + tid;
  const float *vrow = sV + hy * VP;
  const float2 *crow = sAH + (hy + R) * RP + R + hx0;

  for (int n = 0; n <= N; ++n) {
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
    __syncthreads();  // previous phase H done with sV / sAH; region load done

    // ---------------- phase V: generate a_n in place, vertical pass
    if (KIND == BF_SPATIAL_BOX) {
      float s = 0.f;
      const int L = 2 * R + 1;
      for (int r = 0; r < RH; ++r) {
        s += advance(col + r * RP, n, rs);
        if (r >= L) s -= col[(r - L) * RP].x;  // already a_n
        if (r >= L - 1) sV[(r - L + 1) * VP + tid] = s;
      }
    } else {
      float acc[TH], win[TH];
#pragma unroll
      for (int i = 0; i < TH; ++i) {
        acc[i] = 0.f;
        win[i] = advance(col + i * RP, n, rs);
      }
      for (int kb = 0; kb < ntaps; kb += TH) {
#pragma unroll
        for (int u = 0; u < TH; ++u) {
          if (kb + u < ntaps) {  // warp-uniform
            const float w = sT[kb + u];
#pragma unroll
            for (int y = 0; y < TH; ++y) acc[y] = fmaf(w, win[(u + y) % TH], acc[y]);
            const int r = kb + u + TH;
            win[u] = (r < RH) ? advance(col + r * RP, n, rs) : 0.f;
          }
        }
      }
#pragma unroll
      for (int y = 0; y < TH; ++y) sV[y * VP + tid] = acc[y];
    }
    __syncthreads();

    // ---------------- phase H: horizontal pass + recombination
    if (hact) {
      float Ab[KH];
      if (KIND == BF_SPATIAL_BOX) {
        float head[KH];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < KH; ++i) {
          head[i] = vrow[min(hx0 + i, NT - 1)];
          if (i <= 2 * R) s += head[i];
        }
        for (int i = KH; i <= 2 * R; ++i) s += vrow[hx0 + i];
        Ab[0] = s;
#pragma unroll
        for (int j = 1; j < KH; ++j) {
          s += vrow[min(hx0 + j + 2 * R, NT - 1)] - head[j - 1];
          Ab[j] = s;
        }
      } else {
        float win[KH];
#pragma unroll
        for (int i = 0; i < KH; ++i) {
          Ab[i] = 0.f;
          win[i] = vrow[min(hx0 + i, NT - 1)];
        }
        for (int kb = 0; kb < ntaps; kb += KH) {
#pragma unroll
          for (int u = 0; u < KH; ++u) {
            if (kb + u < ntaps) {  // warp-uniform
              const float w = sT[kb + u];
#pragma unroll
              for (int i = 0; i < KH; ++i) Ab[i] = fmaf(w, win[(u + i) % KH], Ab[i]);
              win[u] = vrow[min(hx0 + kb + u + KH, NT - 1)];
            }
          }
        }
      }
      const bool qn = n < N, pn = n > 0;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const float a = crow[min(k, NT - 1 - R - hx0)].x;
        if (qn) Q[k] = fmaf(a, Ab[k], Q[k]);
        if (pn) P[k] = fmaf(sq * ap[k], Ab[k], P[k]);
        ap[k] = a;
      }
      if (STORE) {
        const int gy = ty0 + hy;
        if (gy < io.H) {
          float *dst = io.abar + (long long)n * io.plane_stride + (long long)gy * io.pitch;
#pragma unroll
          for (int k = 0; k < KH; ++k) {
            const int gx = tx0 + hx0 + k;
            if (hx0 + k < TW && gx < io.W) dst[gx] = Ab[k] * fc.qscale;
          }
        }
      }
    }
  }

  // ---- epilogue: f_GPA = t_c + sigma_r P'/Q' (eq. PbyQ with the centre added back)
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
