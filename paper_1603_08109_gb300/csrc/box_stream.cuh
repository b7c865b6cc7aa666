// Streaming forward for the box spatial kernel at small order (N + 1 <= 6
// channels) and small radius (W <= 7): the memory-bound regime.
//
// A CTA owns a strip of TW = 240 output columns (region: TW + 2W columns,
// one thread per region column) and a band of BAND output rows.  It streams
// down the band once:
//   phase C  thread c keeps, per channel n, the running vertical window sum
//            V_n = sum of a_n over the last 2W + 1 region rows of its column.
//            A row entering adds a_n (power images generated from f by the
//            recursion of Algorithm 2); the row leaving (2W + 1 rows back)
//            subtracts a_n regenerated with the identical recursion from a
//            ring of (a_0, H) in shared memory, so every value added is
//            exactly the value later subtracted.  V_n of each output row of
//            an 8-row block goes to shared memory.  The input rows of the next
//            block are loaded into registers one block ahead.
//   phase S  thread (row, segment) produces 8 consecutive outputs of one row:
//            horizontal window sums of V_n, the centre power images
//            regenerated from the ring's (a_0, H), Q' and P' over the
//            channels, then f_GPA = t_c + sigma_r P'/Q', stored with two
//            16-byte stores when aligned.
// The ring holds 2W + 2 + 8 rows, so the centre rows of the block are still
// in it during phase S; ring columns are shifted so that the 8 centre values
// of a segment start on a 16-byte boundary, and the V_n rows have a pitch of
// 4 (mod 32) floats: every phase-S read is a conflict-free 16-byte load.
// Bands are 64 rows, so the running sums' rounding stays a few ulp of the
// window sum.  f is read once per band (plus the 2W-row halo); out (and Q')
// are written once.
#pragma once

#include "gpa_tile.cuh"

namespace bfk {

struct StreamArgs {
  TileIO io;
  bfi::FilterConsts fc;
  float rsq[8];  // 1/sqrt(n), n = 1..7 (entry 0 unused), correctly rounded
  float sq[8];   // sqrt(n)
  int vec_ok;    // 16-byte aligned rows: vector stores allowed
};

template <int R, int NN>
struct StreamGeom {
  static constexpr int NT = 256, TW = 240, RW = TW + 2 * R, RB = 8, K = 8;
  static constexpr int L = 2 * R + 1, RING = 2 * R + 2 + RB, BAND = 64;
  static constexpr int SH = R & 1;   // ring column shift: centre of output x at x + R + SH (even)
  static constexpr int RP = NT + 2;  // ring pitch in float2 (2 mod 16)
  static constexpr int VP = 292;     // V row pitch in floats (4 mod 32, multiple of 4)
  static constexpr size_t smem_bytes() {
    return (size_t)RING * RP * sizeof(float2) + (size_t)RB * NN * VP * sizeof(float);
  }
};

template <int R, int NN>
__device__ __forceinline__ void box_stream_band(const StreamArgs &A, int tx0, int yo0, int yo1,
                                                float *smem) {
  using G = StreamGeom<R, NN>;
  constexpr int NT = G::NT, TW = G::TW, RW = G::RW, RB = G::RB, K = G::K, L = G::L;
  constexpr int RING = G::RING, RP = G::RP, VP = G::VP, SH = G::SH;
  constexpr int NV = (K + 2 * R + 3) / 4;  // float4 loads per phase-S window
  static_assert(RW + SH <= RP, "radius too large for the streaming strip");
  static_assert(NN >= 2 && NN <= 6, "order range of the streaming kernel");
  static_assert(VP % 32 == 4 && VP >= TW + 4 * NV - K + 8, "V row pitch");
  const TileIO &io = A.io;
  const bfi::FilterConsts &fc = A.fc;
  float2 *ring = reinterpret_cast<float2 *>(smem);        // RING x RP: (a_0, H)
  float *sV = reinterpret_cast<float *>(ring + RING * RP);  // NN x RB x VP
  const int c = threadIdx.x;
  const int gx = tx0 - R + c;
  const bool colin = c < RW && gx >= 0 && gx < io.W;
  const float *src = io.in + gx;
  float2 *ringc = ring + c + SH;

  auto load = [&](int y) -> float {
    return (colin && y >= 0 && y < io.H) ? __ldg(src + (long long)y * io.pitch) : fc.tc;
  };
  auto next = [](int s) { return s + 1 == RING ? 0 : s + 1; };
  // (a_0, H) of region row y from its f; out-of-image pixels carry a_0 = 0.
  // a_0 = 2^(e2c d^2) with the hardware base-2 exponential (ex2.approx,
  // <= 2 ulp relative); the exponent is >= -122 for |H| <= 13, so the result
  // is a normal float and flushing subnormals changes nothing.
  auto enter = [&](int y, float f, int s) -> float2 {
    const bool in = colin && y >= 0 && y < io.H;
    const float d = f - fc.tc;
    float a0;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a0) : "f"(d * d * fc.e2c));
    const float2 v = make_float2(in ? a0 : 0.f, in ? d * fc.inv_sr : 0.f);
    ringc[s * RP] = v;
    return v;
  };

  float V[NN];
#pragma unroll
  for (int n = 0; n < NN; ++n) V[n] = 0.f;
  {  // warm-up: the 2W region rows above the first block's entering rows
    float fw[2 * R];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) fw[i] = load(yo0 - R + i);
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
      const float2 v = enter(yo0 - R + i, fw[i], i);
      float a = v.x;
#pragma unroll
      for (int n = 0; n < NN; ++n) {
        if (n > 0) a *= v.y * A.rsq[n];
        V[n] += a;
      }
    }
  }
  float fnext[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) fnext[j] = load(yo0 + R + j);

  const int hj = c % RB, hx0 = (c / RB) * K;
  const bool hact = hx0 < TW;
  // ring slot of region row rho = y - (yo0 - R) is rho mod RING; the slots of
  // the entering (yo + R), leaving (yo - R - 1) and centre (yo) rows advance
  // by one per output row
  int s_in = 2 * R, s_out = RING - 1, s_cen = R;
  for (int yb = yo0; yb < yo1; yb += RB) {
    const int s_block = s_cen;  // slot of the block's first centre row
    float fcur[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      fcur[j] = fnext[j];
      fnext[j] = load(yb + RB + R + j);  // next block's entering rows, in flight meanwhile
    }
    // ---------------- phase C: 8 output rows of running vertical sums
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      const int yo = yb + j;
      const float2 ve = enter(yo + R, fcur[j], s_in);
      float ae = ve.x;
#pragma unroll
      for (int n = 0; n < NN; ++n) {
        if (n > 0) ae *= ve.y * A.rsq[n];
        V[n] += ae;
      }
      if (yo > yo0) {  // the leaving row yo - R - 1 entered in this band
        const float2 vl = ringc[s_out * RP];
        float al = vl.x;
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          if (n > 0) al *= vl.y * A.rsq[n];
          V[n] -= al;
        }
      }
#pragma unroll
      for (int n = 0; n < NN; ++n) sV[(n * RB + j) * VP + c] = V[n];
      s_in = next(s_in);
      s_out = next(s_out);
      s_cen = next(s_cen);
    }
    __syncthreads();

    // ---------------- phase S: horizontal sums, recombination, stores
    if (hact && yb + hj < yo1) {
      const int sc = s_block + hj < RING ? s_block + hj : s_block + hj - RING;
      const float4 *cen = reinterpret_cast<const float4 *>(ring + sc * RP + hx0 + R + SH);
      float Q[K], P[K], ac[K], ap[K], hc[K];
#pragma unroll
      for (int k = 0; k < K / 2; ++k) {
        const float4 cv = cen[k];  // (a_0, H) of two consecutive centre pixels
        ac[2 * k] = cv.x;
        hc[2 * k] = cv.y;
        ac[2 * k + 1] = cv.z;
        hc[2 * k + 1] = cv.w;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) Q[k] = P[k] = ap[k] = 0.f;
#pragma unroll
      for (int n = 0; n < NN; ++n) {
        const float4 *row = reinterpret_cast<const float4 *>(sV + (n * RB + hj) * VP + hx0);
        float v[4 * NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const float4 t = row[i];
          v[4 * i] = t.x;
          v[4 * i + 1] = t.y;
          v[4 * i + 2] = t.z;
          v[4 * i + 3] = t.w;
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) s += v[i];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k > 0) s += v[k + 2 * R] - v[k - 1];
          if (n > 0) ac[k] *= hc[k] * A.rsq[n];
          if (n < NN - 1) Q[k] = fmaf(ac[k], s, Q[k]);
          if (n > 0) P[k] = fmaf(A.sq[n] * ap[k], s, P[k]);
          ap[k] = ac[k];
        }
      }
      const int gy = yb + hj;
      float o[K], q[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        o[k] = fmaf(fc.sr, __fdividef(P[k], Q[k]), fc.tc);  // 2-ulp division
        q[k] = Q[k] * fc.qscale;
      }
      float *orow = io.out + (long long)gy * io.pitch + tx0 + hx0;
      float *qrow = io.qaux ? io.qaux + (long long)gy * io.pitch + tx0 + hx0 : nullptr;
      const int nvalid = min(K, io.W - (tx0 + hx0));
      if (A.vec_ok && nvalid == K) {
        reinterpret_cast<float4 *>(orow)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4 *>(orow)[1] = make_float4(o[4], o[5], o[6], o[7]);
        if (qrow) {
          reinterpret_cast<float4 *>(qrow)[0] = make_float4(q[0], q[1], q[2], q[3]);
          reinterpret_cast<float4 *>(qrow)[1] = make_float4(q[4], q[5], q[6], q[7]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k < nvalid) {
            orow[k] = o[k];
            if (qrow) qrow[k] = q[k];
          }
        }
      }
    }
    __syncthreads();  // phase C of the next block overwrites sV and ring rows
  }
}

}  // namespace bfk
