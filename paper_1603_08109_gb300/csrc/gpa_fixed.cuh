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
// recombination in phase H.  With STORE, each channel's w * a_n (normalised)
// also goes to plane n of io.abar for the stored-plane backward: staged in sV
// once phase H is done reading it, then written row by row so that a warp
// stores 32 consecutive floats (a thread's own KH columns would scatter one
// store instruction over 32 rows and segments).
//
// The kernel is persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ...
// and copies the next tile's region (f) into a second shared buffer with
// cp.async while it computes the current tile, so the HBM latency of the
// load overlaps the arithmetic.  Outputs are staged in shared memory and
// written row by row (coalesced).
#pragma once

#include "gpa_tile.cuh"

namespace bfk {

// Gaussian tap pairs for the vertical pass over pairs of output rows:
// tap2[k] = (w[k], w[k - 1]), w[-1] = w[L] = 0, k = 0 .. L (L <= 31).
constexpr int kTap2 = 32;

template <int R, int NT, int TH>
struct FixedGeom {
  static constexpr int RH = TH + 2 * R;
  static constexpr int TW = NT - 2 * R;
  static constexpr int KH = TH;
  static constexpr int L = 2 * R + 1;
  static constexpr int VP = NT + KH + 1;  // 17 mod 32; phase-H windows never need clamping
  // sV, sC, two region buffers, and the (1/sqrt(n), sqrt(n)) table for n <= N
  static constexpr size_t smem_bytes(int N) {
    return ((size_t)2 * TH * VP + (size_t)2 * RH * NT) * sizeof(float) +
           (size_t)(N + 1) * sizeof(float2);
  }
};

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Copy the f column of region column c of the tile at (ty0, tx0) into buf
// (RH x NT floats).  Out-of-image pixels are not copied (the consumer masks
// them by their coordinates).
template <int R, int NT, int TH>
__device__ __forceinline__ void prefetch_region(const TileIO &io, int ty0, int tx0, float *buf) {
  using G = FixedGeom<R, NT, TH>;
  const int c = threadIdx.x;
  const int gx = tx0 - R + c;
  if (gx < 0 || gx >= io.W) return;
  const float *src = io.in + gx;
  if (ty0 - R >= 0 && ty0 - R + G::RH <= io.H) {  // interior rows: no per-row test
#pragma unroll
    for (int r = 0; r < G::RH; ++r)
      cp_async4(buf + r * NT + c, src + (long long)(ty0 - R + r) * io.pitch);
  } else {
#pragma unroll
    for (int r = 0; r < G::RH; ++r) {
      const int gy = ty0 - R + r;
      if (gy >= 0 && gy < io.H) cp_async4(buf + r * NT + c, src + (long long)gy * io.pitch);
    }
  }
}

// DB: sV / sC are pairs of buffers (sV1 / sC1 the second) that alternate
// between channels, so one block barrier per channel suffices (phase V of
// channel n + 1 writes the pair that phase H of channel n - 1 read, and every
// thread has passed channel n's barrier after finishing that phase H).
template <int KIND, int R, int NT, int TH, bool STORE, bool DB = false>
__device__ __forceinline__ void gpa_fwd_tile_fixed(const TileIO &io, const bfi::FilterConsts &fc,
                                                   const float2 *tap2, int ty0, int tx0, float *sH,
                                                   float *sV0, float *sC0, const float2 *sRS,
                                                   float *sV1 = nullptr, float *sC1 = nullptr) {
  static_assert(!(DB && STORE), "the stored planes are staged in the single pair");
  using G = FixedGeom<R, NT, TH>;
  constexpr int RH = G::RH, TW = G::TW, KH = G::KH, L = G::L, VP = G::VP;
  static_assert(TW >= KH, "tile too narrow for this radius");
  static_assert(NT % TH == 0, "NT must be a multiple of TH");
  const int c = threadIdx.x;
  const int N = fc.N;

  // sH holds this column's f (copied asynchronously); turn it into H in place
  float a[RH];
  {
    const int gx = tx0 - R + c;
    const bool colin = gx >= 0 && gx < io.W;
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      const int gy = ty0 - R + r;
      const bool in = colin && gy >= 0 && gy < io.H;
      const float d = sH[r * NT + c] - fc.tc;
      const float h = in ? d * fc.inv_sr : 0.f;
      // the one transcendental of Algorithm 2: exp(-H^2/2) = 2^(e2c d^2)
      a[r] = in ? exp2f(d * d * fc.e2c) : 0.f;
      sH[r * NT + c] = h;
    }
  }

  const int hy = c % TH;
  const int hx0 = (c / TH) * KH;
  const bool hact = hx0 < TW;
  float Q[KH], P[KH], ap[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) Q[k] = P[k] = ap[k] = 0.f;

  for (int n = 0; n <= N; ++n) {
    const float2 rsq = sRS[n];  // (1/sqrt(n), sqrt(n)), correctly rounded
    const float rs = rsq.x, sq = rsq.y;
    float *sV = DB && (n & 1) ? sV1 : sV0;
    float *sC = DB && (n & 1) ? sC1 : sC0;
    const float *vrow = sV + hy * VP + hx0;
    const float *crow = sC + hy * VP + R + hx0;
    if (!DB) __syncthreads();  // phase H of the previous channel (or tile) is done with sV / sC

    // ---------------- phase V (registers): advance, centre copy, vertical pass
    if (n > 0) {
#pragma unroll
      for (int r = 0; r < RH; ++r) a[r] *= sH[r * NT + c] * rs;
    }
#pragma unroll
    for (int y = 0; y < TH; ++y) sC[y * VP + c] = a[y + R];
    if (KIND == BF_SPATIAL_GAUSS) {
      // rows (y, y + 1) as one packed pair: (acc_y, acc_y+1) += (w[r-y], w[r-y-1]) a_r,
      // taps in ascending order per row as in the scalar sum (the extra terms
      // have weight 0 and leave each sum unchanged)
      static_assert(TH % 2 == 0 && L + 1 <= kTap2, "row pairs");
      float2 acc[TH / 2];
#pragma unroll
      for (int p = 0; p < TH / 2; ++p) acc[p] = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < RH; ++r) {
        const float2 ar = make_float2(a[r], a[r]);
#pragma unroll
        for (int p = 0; p < TH / 2; ++p) {
          const int t = r - 2 * p;
          if (t >= 0 && t <= L) acc[p] = __ffma2_rn(tap2[t >= 0 && t <= L ? t : 0], ar, acc[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < TH / 2; ++p) {
        sV[2 * p * VP + c] = acc[p].x;
        sV[(2 * p + 1) * VP + c] = acc[p].y;
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
    float Ab[KH];
    if (hact) {
      if (KIND == BF_SPATIAL_GAUSS) {
        // columns (i, i + 1) as one packed pair, element by element of the
        // window: (Ab_i, Ab_i+1) += (w[e-i], w[e-i-1]) v_e, each sum in
        // ascending tap order as in the scalar form
        static_assert(KH % 2 == 0, "column pairs");
        float2 ab[KH / 2];
#pragma unroll
        for (int p = 0; p < KH / 2; ++p) ab[p] = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < KH + 2 * R; ++e) {
          const float v = vrow[e];
          const float2 vv = make_float2(v, v);
#pragma unroll
          for (int p = 0; p < KH / 2; ++p) {
            const int t = e - 2 * p;
            if (t >= 0 && t <= L) ab[p] = __ffma2_rn(tap2[t >= 0 && t <= L ? t : 0], vv, ab[p]);
          }
        }
#pragma unroll
        for (int p = 0; p < KH / 2; ++p) {
          Ab[2 * p] = ab[p].x;
          Ab[2 * p + 1] = ab[p].y;
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
    if (STORE) {
      __syncthreads();  // every thread is done reading sV for this channel
      if (hact) {
#pragma unroll
        for (int k = 0; k < KH; ++k) sV[hy * VP + hx0 + k] = Ab[k] * fc.qscale;
      }
      __syncthreads();
      if (c < min(TW, io.W - tx0)) {
        float *dst = io.abar + (long long)n * io.plane_stride + tx0 + c;
#pragma unroll
        for (int y = 0; y < TH; ++y)
          if (ty0 + y < io.H) dst[(long long)(ty0 + y) * io.pitch] = sV[y * VP + c];
      }
    }
  }

  // ---- epilogue: f_GPA = t_c + sigma_r P'/Q', staged in sV / sC (DB: the
  // pair channel N's phase H does not read), stored row-wise
  float *sV = DB && ((N + 1) & 1) ? sV1 : sV0;
  float *sC = DB && ((N + 1) & 1) ? sC1 : sC0;
  if (!DB) __syncthreads();  // every thread is done reading sV / sC
  if (hact) {
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      // approximate division (2 ulp): <= 3e-5 on the 0..255 scale
      sV[hy * VP + hx0 + k] = fmaf(fc.sr, __fdividef(P[k], Q[k]), fc.tc);
      sC[hy * VP + hx0 + k] = Q[k] * fc.qscale;
    }
  }
  __syncthreads();
  const int wmax = min(TW, io.W - tx0);
  for (int y = 0; y < TH; ++y) {
    const int gy = ty0 + y;
    if (gy >= io.H) break;
    if (c < wmax) {
      io.out[(long long)gy * io.pitch + tx0 + c] = sV[y * VP + c];
      if (io.qaux) io.qaux[(long long)gy * io.pitch + tx0 + c] = sC[y * VP + c];
    }
  }
}

// Persistent driver: tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (row-major over the tile grid), double-buffered region copies.
template <int KIND, int R, int NT, int TH, bool STORE>
__device__ __forceinline__ void gpa_fwd_fixed_persistent(const TileIO &io,
                                                         const bfi::FilterConsts &fc,
                                                         const float2 *tap2, float *smem) {
  using G = FixedGeom<R, NT, TH>;
  float *sV = smem;
  float *sC = sV + TH * G::VP;
  float *sF0 = sC + TH * G::VP;
  float *sF1 = sF0 + G::RH * NT;
  float2 *sRS = reinterpret_cast<float2 *>(sF1 + G::RH * NT);
  const int ntx = (io.W + G::TW - 1) / G::TW;
  const int nty = (io.H + TH - 1) / TH;
  const int ntiles = ntx * nty;
  int t = blockIdx.x;
  if (t >= ntiles) return;
  prefetch_region<R, NT, TH>(io, (t / ntx) * TH, (t % ntx) * G::TW, sF0);
  cp_async_commit();
  // channel constants 1/sqrt(n), sqrt(n), correctly rounded, once per CTA
  for (int n = threadIdx.x; n <= fc.N; n += NT)
    sRS[n] = make_float2(n > 0 ? __frsqrt_rn((float)n) : 0.f, __fsqrt_rn((float)n));
  __syncthreads();
  int buf = 0;
  for (; t < ntiles; t += gridDim.x) {
    const int next = t + gridDim.x;
    float *cur = buf ? sF1 : sF0;
    if (next < ntiles) {
      prefetch_region<R, NT, TH>(io, (next / ntx) * TH, (next % ntx) * G::TW, buf ? sF0 : sF1);
      cp_async_commit();
      cp_async_wait<1>();  // the current tile's copies are complete
    } else {
      cp_async_wait<0>();
    }
    gpa_fwd_tile_fixed<KIND, R, NT, TH, STORE>(io, fc, tap2, (t / ntx) * TH, (t % ntx) * G::TW, cur,
                                               sV, sC, sRS);
    buf ^= 1;
  }
}

// Without stored planes: a single region buffer, filled at the start of
// each tile, and two alternating pairs of phase rows (one block barrier per
// channel, see gpa_fwd_tile_fixed), the second pair taking the shared memory
// of the region copy that would otherwise be in flight.  Where two such
// pairs keep the CTA from sharing an SM with a second one (W = 15: 46 region
// rows), a single pair and two barriers per channel: 2 CTAs per SM instead
// of 1.
template <int R, int NT, int TH>
struct FixedDbGeom {
  using G = FixedGeom<R, NT, TH>;
  static constexpr size_t bytes(int pairs, int N) {
    return ((size_t)2 * pairs * TH * G::VP + (size_t)G::RH * NT) * sizeof(float) +
           (size_t)(N + 1) * sizeof(float2);
  }
  // two CTAs (and their 1 KB reserves) in an SM's 228 KB at every order
  static constexpr bool DB = 2 * (bytes(2, BF_MAX_ORDER) + 1024) <= 228 * 1024;
  static constexpr size_t smem_bytes(int N, bool store = false) {
    return bytes(DB && !store ? 2 : 1, N);
  }
  // with stored planes: the layout with the next tile's region in flight
  // (G::smem_bytes) where it fits two CTAs per SM, else this one
  static constexpr bool STORE_PREFETCH = 2 * (G::smem_bytes(BF_MAX_ORDER) + 1024) <= 228 * 1024;
};

// STORE: the stored planes are staged in the single pair (DB off); this
// layout serves them where the one with the next tile's region in flight
// does not fit two CTAs per SM.
template <int KIND, int R, int NT, int TH, bool STORE = false>
__device__ __forceinline__ void gpa_fwd_fixed_persistent_db(const TileIO &io,
                                                            const bfi::FilterConsts &fc,
                                                            const float2 *tap2, float *smem) {
  using G = FixedGeom<R, NT, TH>;
  constexpr bool DB = FixedDbGeom<R, NT, TH>::DB && !STORE;
  float *sV0 = smem;
  float *sC0 = sV0 + TH * G::VP;
  float *sV1 = DB ? sC0 + TH * G::VP : nullptr;
  float *sC1 = DB ? sV1 + TH * G::VP : nullptr;
  float *sF = sC0 + (DB ? 3 : 1) * TH * G::VP;
  float2 *sRS = reinterpret_cast<float2 *>(sF + G::RH * NT);
  const int ntx = (io.W + G::TW - 1) / G::TW;
  const int nty = (io.H + TH - 1) / TH;
  const int ntiles = ntx * nty;
  int t = blockIdx.x;
  if (t >= ntiles) return;
  // channel constants 1/sqrt(n), sqrt(n), correctly rounded, once per CTA
  for (int n = threadIdx.x; n <= fc.N; n += NT)
    sRS[n] = make_float2(n > 0 ? __frsqrt_rn((float)n) : 0.f, __fsqrt_rn((float)n));
  for (; t < ntiles; t += gridDim.x) {
    const int ty0 = (t / ntx) * TH, tx0 = (t % ntx) * G::TW;
    prefetch_region<R, NT, TH>(io, ty0, tx0, sF);  // each thread its own column
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();  // sRS written; the previous tile's epilogue is done with the pairs
    gpa_fwd_tile_fixed<KIND, R, NT, TH, STORE, DB>(io, fc, tap2, ty0, tx0, sF, sV0, sC0, sRS,
                                                   sV1, sC1);
  }
}

}  // namespace bfk
