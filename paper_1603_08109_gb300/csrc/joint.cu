// Cross (joint) bilateral filter: the range kernel compares a guide image e,
// the data f is averaged (the extension named in Sec. I and Sec. V).
//
// Gaussian-polynomial form: with E = (e - t_c)/sigma_r, b_n = e^{-E^2/2} E^n / sqrt(n!)
// and f~ = f - t_c,
//   out = t_c + U'/Q',  Q' = sum_{n<N} b_n (w*b_n),  U' = sum_{n<N} b_n (w*(b_n f~)),
// i.e. 2N spatial filterings (eq. GPA with phi_N on guide values; for e = f it
// reduces to Algorithm 2 because b_n f~ = sigma_r sqrt(n+1) b_{n+1}).
// The fused tile mirrors gpa_tile.cuh with two channels per order: phase V
// streams region columns (advancing b_n in place, forming b_n f~) through the
// vertical pass of both channels; phase H applies the horizontal passes and
// accumulates Q', U' in registers.  Shared memory holds b_n, E and f~ per
// region pixel (row pitch NT + 1: conflict-free phase-H reads).
//
// The direct joint filter (exact range kernel, O((2W+1)^2) per pixel) is the
// same-GPU comparison.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "bf_internal.h"
#include "tmem.cuh"

namespace {

struct JointArgs {
  const float *in, *guide;
  float *out, *qaux;
  int H, W, pitch;
  bfi::FilterConsts fc;
};

__host__ __device__ constexpr int jrp(int nt) { return nt + 1; }

size_t joint_smem(int NT, int TH, int R, int ntaps_pad) {
  return (size_t)(TH + 2 * R) * jrp(NT) * 3 * sizeof(float) +
         (size_t)2 * TH * jrp(NT) * sizeof(float) +
         (size_t)(ntaps_pad > 0 ? ntaps_pad : 1) * sizeof(float);
}

template <int KIND, int NT, int TH>
__global__ void __launch_bounds__(NT) joint_kernel(const __grid_constant__ JointArgs A) {
  extern __shared__ __align__(16) float smem[];
  constexpr int KH = TH;
  constexpr int RP = jrp(NT), VP = jrp(NT);
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, RH = TH + 2 * R, TW = NT - 2 * R, N = fc.N, ntaps = 2 * R + 1;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
  float *sB = smem;              // b_n (advanced in place)
  float *sE = sB + RH * RP;      // E of the guide
  float *sF = sE + RH * RP;      // f - t_c
  float *sVb = sF + RH * RP;     // vertical pass of b_n
  float *sVc = sVb + TH * VP;    // vertical pass of b_n f~
  float *sT = sVc + TH * VP;     // taps
  const int tid = threadIdx.x;
  if (KIND == BF_SPATIAL_GAUSS)
    for (int i = tid; i < fc.ntaps_pad; i += NT) sT[i] = fc.taps[i];
  {
    const int gx = tx0 - R + tid;
    const bool colin = gx >= 0 && gx < A.W;
    for (int r = 0; r < RH; ++r) {
      const int gy = ty0 - R + r;
      float b = 0.f, E = 0.f, ft = 0.f;
      if (colin && gy >= 0 && gy < A.H) {
        const long long o = (long long)gy * A.pitch + gx;
        E = (__ldg(A.guide + o) - fc.tc) * fc.inv_sr;
        ft = __ldg(A.in + o) - fc.tc;
        b = expf(-0.5f * E * E);
      }
      sB[r * RP + tid] = b;
      sE[r * RP + tid] = E;
      sF[r * RP + tid] = ft;
    }
  }
  const int hy = tid % TH, hx0 = (tid / TH) * KH;
  const bool hact = hx0 < TW;
  float Q[KH], U[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) Q[k] = U[k] = 0.f;

  for (int n = 0; n < N; ++n) {
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    __syncthreads();
    auto gen = [&](int r, float &c) -> float {
      float b = sB[r * RP + tid];
      if (n > 0) {
        b *= sE[r * RP + tid] * rs;
        sB[r * RP + tid] = b;
      }
      c = b * sF[r * RP + tid];
      return b;
    };
    if (KIND == BF_SPATIAL_BOX) {
      float sb = 0.f, sc = 0.f;
      const int L = 2 * R + 1;
      for (int r = 0; r < RH; ++r) {
        float c;
        sb += gen(r, c);
        sc += c;
        if (r >= L) {
          const float bo = sB[(r - L) * RP + tid];  // already b_n
          sb -= bo;
          sc -= bo * sF[(r - L) * RP + tid];
        }
        if (r >= L - 1) {
          sVb[(r - L + 1) * VP + tid] = sb;
          sVc[(r - L + 1) * VP + tid] = sc;
        }
      }
    } else {
      float ab[TH], ac[TH], wb[TH], wc[TH];
#pragma unroll
      for (int i = 0; i < TH; ++i) {
        ab[i] = ac[i] = 0.f;
        wb[i] = gen(i, wc[i]);
      }
      for (int kb = 0; kb < ntaps; kb += TH) {
#pragma unroll
        for (int u = 0; u < TH; ++u) {
          if (kb + u < ntaps) {  // warp-uniform
            const float w = sT[kb + u];
#pragma unroll
            for (int y = 0; y < TH; ++y) {
              ab[y] = fmaf(w, wb[(u + y) % TH], ab[y]);
              ac[y] = fmaf(w, wc[(u + y) % TH], ac[y]);
            }
            const int r = kb + u + TH;
            if (r < RH) {
              wb[u] = gen(r, wc[u]);
            } else {
              wb[u] = 0.f;
              wc[u] = 0.f;
            }
          }
        }
      }
#pragma unroll
      for (int y = 0; y < TH; ++y) {
        sVb[y * VP + tid] = ab[y];
        sVc[y * VP + tid] = ac[y];
      }
    }
    __syncthreads();
    if (hact) {
      const float *rb = sVb + hy * VP, *rc = sVc + hy * VP;
      float Bb[KH], Cb[KH];
      if (KIND == BF_SPATIAL_BOX) {
        float hb[KH], hc[KH], s_b = 0.f, s_c = 0.f;
#pragma unroll
        for (int i = 0; i < KH; ++i) {
          const int x = min(hx0 + i, NT - 1);
          hb[i] = rb[x];
          hc[i] = rc[x];
          if (i <= 2 * R) {
            s_b += hb[i];
            s_c += hc[i];
          }
        }
        for (int i = KH; i <= 2 * R; ++i) {
          s_b += rb[hx0 + i];
          s_c += rc[hx0 + i];
        }
        Bb[0] = s_b;
        Cb[0] = s_c;
#pragma unroll
        for (int j = 1; j < KH; ++j) {
          const int x = min(hx0 + j + 2 * R, NT - 1);
          s_b += rb[x] - hb[j - 1];
          s_c += rc[x] - hc[j - 1];
          Bb[j] = s_b;
          Cb[j] = s_c;
        }
      } else {
        float wb[KH], wc[KH];
#pragma unroll
        for (int i = 0; i < KH; ++i) {
          Bb[i] = Cb[i] = 0.f;
          const int x = min(hx0 + i, NT - 1);
          wb[i] = rb[x];
          wc[i] = rc[x];
        }
        for (int kb = 0; kb < ntaps; kb += KH) {
#pragma unroll
          for (int u = 0; u < KH; ++u) {
            if (kb + u < ntaps) {
              const float w = sT[kb + u];
#pragma unroll
              for (int i = 0; i < KH; ++i) {
                Bb[i] = fmaf(w, wb[(u + i) % KH], Bb[i]);
                Cb[i] = fmaf(w, wc[(u + i) % KH], Cb[i]);
              }
              const int x = min(hx0 + kb + u + KH, NT - 1);
              wb[u] = rb[x];
              wc[u] = rc[x];
            }
          }
        }
      }
      const float *crow = sB + (hy + R) * RP + R + hx0;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const float b = crow[min(k, NT - 1 - R - hx0)];
        Q[k] = fmaf(b, Bb[k], Q[k]);
        U[k] = fmaf(b, Cb[k], U[k]);
      }
    }
  }
  if (hact) {
    const int gy = ty0 + hy;
    if (gy < A.H) {
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const int gx = tx0 + hx0 + k;
        if (hx0 + k < TW && gx < A.W) {
          A.out[(long long)gy * A.pitch + gx] = fc.tc + U[k] / Q[k];
          if (A.qaux) A.qaux[(long long)gy * A.pitch + gx] = Q[k] * fc.qscale;
        }
      }
    }
  }
}

// Compile-time-radius joint tile (W in {3, 5, 9, 15}): 128 threads, 8-row
// tiles; each column thread keeps its RH = 8 + 2W guide power images b_n in
// registers, (E, f~) of the thread's region column in its own tensor-memory
// lane (three TMEM columns per region row, read with tcgen05.ld in every
// channel instead of from shared memory), Gaussian taps are constant-bank FMA
// operands; phase V writes the centre rows of b_n for the recombination.  The
// rows of the two phases alternate between two shared buffers, so one block
// barrier per channel suffices (phase V of channel n + 1 writes the buffer
// that phase H of channel n - 1 read, and every thread has passed channel n's
// barrier after finishing that phase H).  The two filterings of a channel (b_n and b_n f~ share
// every tap) run as one filtering of the pair with the packed two-lane FP32
// instructions (each lane rounded exactly as the scalar operation), and the
// recombination updates (Q', U') as a pair.
template <int R>
struct JointFixedGeom {
  static constexpr int NT = 128, TH = 8, KH = 8;
  static constexpr int RH = TH + 2 * R, TW = NT - 2 * R, L = 2 * R + 1;
  // 1 (mod 32): the 4 x 8 phase-H lanes read distinct bank pairs of the
  // (b, c) rows (per half-warp) and distinct banks of the b_n centre rows
  static constexpr int VP = NT + 33;
  static constexpr int NG = (RH + 3) / 4;  // groups of four region rows in TMEM
  static_assert(RH % 4 == 2 && 3 * RH <= bft::kCols, "region rows in the TMEM lane");
  static constexpr size_t buf_floats = (size_t)3 * TH * VP;  // (b, c) pairs + b_n centre rows
  static constexpr size_t smem_used = 2 * buf_floats * sizeof(float);
  // more than a fifth of an SM's shared memory: at most four CTAs (4 x 128
  // TMEM columns) per SM, so an allocation never waits
  static constexpr size_t smem_bytes() { return smem_used > 47 * 1024 ? smem_used : 47 * 1024; }
  // a fifth CTA (with its 1 KB reserve) does not fit an SM's 228 KB
  static_assert(5 * (smem_bytes() + 1024) > 228 * 1024, "at most four CTAs per SM");
};

template <int KIND, int R>
__global__ void __launch_bounds__(128) joint_fixed_kernel(const __grid_constant__ JointArgs A) {
  using G = JointFixedGeom<R>;
  constexpr int NT = G::NT, TH = G::TH, KH = G::KH, RH = G::RH, TW = G::TW, L = G::L, VP = G::VP;
  static_assert(G::VP % 32 == 1 && TW >= KH, "geometry");
  extern __shared__ __align__(16) float smem[];
  __shared__ uint32_t s_tmem;
  const bfi::FilterConsts &fc = A.fc;
  const int N = fc.N;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
  const int c = threadIdx.x;
  if (c < 32) bft::alloc(&s_tmem);
  bft::fence_before_sync();
  __syncthreads();
  bft::fence_after_sync();
  const uint32_t tl = s_tmem + ((uint32_t)(c & ~31) << 16);  // this warp's lane quadrant
  float b[RH];
  {  // (E, f - t_c) of the region column to TMEM, b_0 to registers
    const int gx = tx0 - R + c;
    const bool colin = gx >= 0 && gx < A.W;
#pragma unroll
    for (int g = 0; g < G::NG; ++g) {
      float t[12];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * g + j, gy = ty0 - R + r;
        float E = 0.f, ft = 0.f, b0 = 0.f;
        if (r < RH && colin && gy >= 0 && gy < A.H) {
          const long long o = (long long)gy * A.pitch + gx;
          E = (__ldg(A.guide + o) - fc.tc) * fc.inv_sr;
          ft = __ldg(A.in + o) - fc.tc;
          b0 = expf(-0.5f * E * E);
        }
        if (r < RH) b[r] = b0;
        t[3 * j] = E;
        t[3 * j + 1] = ft;
        t[3 * j + 2] = 0.f;
      }
      if (4 * g + 4 <= RH) {
        bft::st12(tl + 12 * g, t);
      } else {
        const float t6[6] = {t[0], t[1], t[2], t[3], t[4], t[5]};
        bft::st6(tl + 12 * g, t6);
      }
    }
  }
  bft::wait_st();
  const int hy = c % TH, hx0 = (c / TH) * KH;
  const bool hact = hx0 < TW;
  float2 QU[KH];  // (Q', U')
#pragma unroll
  for (int k = 0; k < KH; ++k) QU[k] = make_float2(0.f, 0.f);

  for (int n = 0; n < N; ++n) {
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    float2 *sV = reinterpret_cast<float2 *>(smem + (n & 1) * G::buf_floats);  // (b_n, b_n f~)
    float *sCb = smem + (n & 1) * G::buf_floats + 2 * TH * VP;               // b_n centre rows
    const float2 *rv = sV + hy * VP + hx0;
    const float *cb = sCb + hy * VP + R + hx0;
    float2 acc[TH];  // (b_n, b_n f~) of the TH output rows
#pragma unroll
    for (int y = 0; y < TH; ++y) acc[y] = make_float2(0.f, 0.f);
    float cbox[KIND == BF_SPATIAL_BOX ? RH : 1];
    float t[12];  // (E, f~, -) of the current group of four rows
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      if (r % 4 == 0) {  // (E, f~) of rows r .. r + 3 from TMEM
        if (r + 4 <= RH) {
          bft::ld12(tl + 3 * r, t);
        } else {
          float t6[6];
          bft::ld6(tl + 3 * r, t6);
#pragma unroll
          for (int i = 0; i < 6; ++i) t[i] = t6[i];
        }
      }
      const float2 ef = make_float2(t[3 * (r % 4)], t[3 * (r % 4) + 1]);
      if (n > 0) b[r] *= ef.x * rs;
      const float cn = b[r] * ef.y;
      if (r >= R && r < R + TH) sCb[(r - R) * VP + c] = b[r];
      if (KIND == BF_SPATIAL_GAUSS) {
        const float2 bc = make_float2(b[r], cn);
#pragma unroll
        for (int y = 0; y < TH; ++y) {
          if (r - y >= 0 && r - y < L) {
            const float w = fc.taps[r - y];
            acc[y] = __ffma2_rn(make_float2(w, w), bc, acc[y]);
          }
        }
      } else {
        cbox[KIND == BF_SPATIAL_BOX ? r : 0] = cn;
      }
    }
    if (KIND == BF_SPATIAL_BOX) {
      float sb = 0.f, sc = 0.f;
#pragma unroll
      for (int r = 0; r < L; ++r) {
        sb += b[r];
        sc += cbox[KIND == BF_SPATIAL_BOX ? r : 0];
      }
      acc[0] = make_float2(sb, sc);
#pragma unroll
      for (int y = 1; y < TH; ++y) {
        sb += b[y + 2 * R] - b[y - 1];
        sc += cbox[KIND == BF_SPATIAL_BOX ? y + 2 * R : 0] - cbox[KIND == BF_SPATIAL_BOX ? y - 1 : 0];
        acc[y] = make_float2(sb, sc);
      }
    }
#pragma unroll
    for (int y = 0; y < TH; ++y) sV[y * VP + c] = acc[y];
    __syncthreads();
    if (hact) {
      float2 BC[KH];  // (w * b_n, w * (b_n f~)) of the item's KH columns
      if (KIND == BF_SPATIAL_GAUSS) {
        float2 win[KH];
#pragma unroll
        for (int i = 0; i < KH; ++i) {
          BC[i] = make_float2(0.f, 0.f);
          win[i] = rv[i];
        }
#pragma unroll
        for (int t = 0; t < L; ++t) {
          const float w = fc.taps[t];
#pragma unroll
          for (int i = 0; i < KH; ++i) BC[i] = __ffma2_rn(make_float2(w, w), win[(t + i) % KH], BC[i]);
          win[t % KH] = rv[t + KH];
        }
      } else {
        float vb[KH + 2 * R], vc[KH + 2 * R];
#pragma unroll
        for (int i = 0; i < KH + 2 * R; ++i) {
          vb[i] = rv[i].x;
          vc[i] = rv[i].y;
        }
        float sb = 0.f, sc = 0.f;
#pragma unroll
        for (int i = 0; i < L; ++i) {
          sb += vb[i];
          sc += vc[i];
        }
        BC[0] = make_float2(sb, sc);
#pragma unroll
        for (int j = 1; j < KH; ++j) {
          sb += vb[j + 2 * R] - vb[j - 1];
          sc += vc[j + 2 * R] - vc[j - 1];
          BC[j] = make_float2(sb, sc);
        }
      }
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const float bk = cb[k];
        QU[k] = __ffma2_rn(make_float2(bk, bk), BC[k], QU[k]);
      }
    }
  }
  // every warp's TMEM reads are complete: free the columns
  bft::fence_before_sync();
  __syncthreads();
  if (c < 32) {
    bft::fence_after_sync();
    bft::dealloc(s_tmem);
  }
  if (hact) {
    const int gy = ty0 + hy;
    if (gy < A.H) {
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const int gx = tx0 + hx0 + k;
        if (hx0 + k < TW && gx < A.W) {
          A.out[(long long)gy * A.pitch + gx] = fc.tc + QU[k].y / QU[k].x;
          if (A.qaux) A.qaux[(long long)gy * A.pitch + gx] = QU[k].x * fc.qscale;
        }
      }
    }
  }
}

template <int KIND, int R>
bf_status launch_joint_fixed_r(const JointArgs &A, cudaStream_t s) {
  using G = JointFixedGeom<R>;
  auto kern = joint_fixed_kernel<KIND, R>;
  const bf_status st = bfi::ensure_smem(reinterpret_cast<const void *>(kern), G::smem_bytes());
  if (st != BF_OK) return st;
  dim3 grid((A.W + G::TW - 1) / G::TW, (A.H + G::TH - 1) / G::TH);
  kern<<<grid, G::NT, G::smem_bytes(), s>>>(A);
  return bfi::check_launch();
}

template <int KIND>
bf_status launch_joint_fixed(const JointArgs &A, cudaStream_t s) {
  switch (A.fc.R) {
    case 3: return launch_joint_fixed_r<KIND, 3>(A, s);
    case 5: return launch_joint_fixed_r<KIND, 5>(A, s);
    case 9: return launch_joint_fixed_r<KIND, 9>(A, s);
    case 15: return launch_joint_fixed_r<KIND, 15>(A, s);
    default: return BF_ERR_UNSUPPORTED;
  }
}

bool joint_fixed_radius(int R) { return R == 3 || R == 5 || R == 9 || R == 15; }

// Direct joint filter: out(i) = f(i) + sum_j w(j) g(e(i-j) - e(i)) (f(i-j) - f(i)) / sum_j (...)
constexpr int DTH = 16, DKX = 4, DNT = 256, DTW = (DNT / DTH) * DKX;

struct JointDirectArgs {
  const float *in, *guide;
  float *out;
  int H, W, pitch, R;
  float negc;
  float lx[2 * BF_MAX_RADIUS + 1];
};

__host__ __device__ inline size_t jd_plane(int R) { return (size_t)(DTH + 2 * R) * (DTW + 2 * R + 1); }

__global__ void __launch_bounds__(DNT) joint_direct_kernel(const __grid_constant__ JointDirectArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int R = A.R, sp = DTW + 2 * R + 1;
  const size_t plane = jd_plane(R);
  float *sf = sm, *se = sm + plane;
  const int ty0 = blockIdx.y * DTH, tx0 = blockIdx.x * DTW;
  const int RH = DTH + 2 * R, RW = DTW + 2 * R;
  for (int i = threadIdx.x; i < RH * RW; i += blockDim.x) {
    const int r = i / RW, c = i % RW;
    const int gy = ty0 - R + r, gx = tx0 - R + c;
    float f = 0.f, e = __int_as_float(0x7fc00000);  // NaN guide marks out-of-image
    if (gy >= 0 && gy < A.H && gx >= 0 && gx < A.W) {
      f = __ldg(A.in + (long long)gy * A.pitch + gx);
      e = __ldg(A.guide + (long long)gy * A.pitch + gx);
    }
    sf[r * sp + c] = f;
    se[r * sp + c] = e;
  }
  __syncthreads();
  const int y = threadIdx.x % DTH, x0 = (threadIdx.x / DTH) * DKX;
  float fc[DKX], ec[DKX], num[DKX], den[DKX];
#pragma unroll
  for (int k = 0; k < DKX; ++k) {
    fc[k] = sf[(y + R) * sp + x0 + k + R];
    ec[k] = se[(y + R) * sp + x0 + k + R];
    num[k] = den[k] = 0.f;
  }
  for (int dy = -R; dy <= R; ++dy) {
    const int rb = (y + R + dy) * sp + x0;
    const float ly = A.lx[dy + R];
    for (int dx = 0; dx <= 2 * R; ++dx) {
      const float lw = ly + A.lx[dx];
#pragma unroll
      for (int k = 0; k < DKX; ++k) {
        const float e = se[rb + dx + k];
        const float d = e - ec[k];
        const float wt = exp2f(fmaf(d * d, A.negc, lw));
        if (e == e) {
          num[k] = fmaf(wt, sf[rb + dx + k] - fc[k], num[k]);
          den[k] += wt;
        }
      }
    }
  }
  const int gy = ty0 + y;
  if (gy < A.H) {
#pragma unroll
    for (int k = 0; k < DKX; ++k) {
      const int gx = tx0 + x0 + k;
      if (gx < A.W) A.out[(long long)gy * A.pitch + gx] = fc[k] + num[k] / den[k];
    }
  }
}

int smem_optin_j() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      v = 232448;
    cudaGetLastError();
  }
  return v;
}

template <int KIND, int NT, int TH>
bf_status launch_joint(const JointArgs &A, cudaStream_t s) {
  const size_t smem = joint_smem(NT, TH, A.fc.R, A.fc.ntaps_pad);
  auto kern = joint_kernel<KIND, NT, TH>;
  const bf_status st = bfi::ensure_smem(reinterpret_cast<const void *>(kern), smem);
  if (st != BF_OK) return st;
  const int TW = NT - 2 * A.fc.R;
  dim3 grid((A.W + TW - 1) / TW, (A.H + TH - 1) / TH);
  kern<<<grid, NT, smem, s>>>(A);
  return bfi::check_launch();
}

}  // namespace

extern "C" {

bf_status bf_joint_forward(const float *d_in, const float *d_guide, float *d_out, float *d_qaux,
                           int height, int width, int pitch, const bf_params *p, void *stream) {
  bf_status st = bfi::check_image(d_in, d_out, height, width, pitch);
  if (st != BF_OK) return st;
  if (!d_guide || (reinterpret_cast<uintptr_t>(d_guide) & 3u)) return BF_ERR_INVALID_ARG;
  JointArgs A;
  st = bfi::resolve(p, true, &A.fc);
  if (st != BF_OK) return st;
  A.in = d_in;
  A.guide = d_guide;
  A.out = d_out;
  A.qaux = d_qaux;
  A.H = height;
  A.W = width;
  A.pitch = pitch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int R = A.fc.R;
  const size_t optin = (size_t)smem_optin_j();
  const bool g = A.fc.kind == BF_SPATIAL_GAUSS;
  if (joint_fixed_radius(R)) return g ? launch_joint_fixed<1>(A, s) : launch_joint_fixed<0>(A, s);
  if (256 - 2 * R >= 16 && joint_smem(256, 16, R, A.fc.ntaps_pad) <= optin)
    return g ? launch_joint<1, 256, 16>(A, s) : launch_joint<0, 256, 16>(A, s);
  if (128 - 2 * R >= 16 && joint_smem(128, 16, R, A.fc.ntaps_pad) <= optin)
    return g ? launch_joint<1, 128, 16>(A, s) : launch_joint<0, 128, 16>(A, s);
  return BF_ERR_UNSUPPORTED;
}

bf_status bf_joint_direct(const float *d_in, const float *d_guide, float *d_out, int height,
                          int width, int pitch, const bf_params *p, void *stream) {
  bf_status st = bfi::check_image(d_in, d_out, height, width, pitch);
  if (st != BF_OK) return st;
  if (!d_guide || (reinterpret_cast<uintptr_t>(d_guide) & 3u)) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  st = bfi::resolve(p, false, &fc);
  if (st != BF_OK) return st;
  JointDirectArgs A;
  memset(&A, 0, sizeof(A));
  A.in = d_in;
  A.guide = d_guide;
  A.out = d_out;
  A.H = height;
  A.W = width;
  A.pitch = pitch;
  A.R = fc.R;
  const double log2e = 1.4426950408889634, sr = p->sigma_r;
  A.negc = (float)(-log2e / (2.0 * sr * sr));
  for (int k = -fc.R; k <= fc.R; ++k)
    A.lx[k + fc.R] = fc.kind == BF_SPATIAL_GAUSS
                         ? (float)(-(double)k * k * log2e / (2.0 * (double)p->sigma_s * p->sigma_s))
                         : 0.f;
  const size_t smem = 2 * jd_plane(fc.R) * sizeof(float);
  if (smem > (size_t)smem_optin_j()) return BF_ERR_UNSUPPORTED;
  st = bfi::ensure_smem(reinterpret_cast<const void *>(joint_direct_kernel), smem);
  if (st != BF_OK) return st;
  dim3 grid((width + DTW - 1) / DTW, (height + DTH - 1) / DTH);
  joint_direct_kernel<<<grid, DNT, smem, static_cast<cudaStream_t>(stream)>>>(A);
  return bfi::check_launch();
}

}  // extern "C"
