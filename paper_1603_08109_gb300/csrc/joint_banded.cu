// Two-pass banded cross (joint) bilateral filter for large radii (Gaussian
// W > 15, box W > 24).
//
// The Gaussian-polynomial joint filter (joint.cu) is
//   out = t_c + U'/Q',  Q' = sum_{n<N} b_n (w*b_n),  U' = sum_{n<N} b_n (w*(b_n f~)),
// with b_n = e^{-E^2/2} E^n / sqrt(n!) the guide's rescaled power images and
// f~ = f - t_c.  Both b_n and b_n f~ follow Algorithm 2's recursion (f~ does
// not depend on n), so, as in the banded forward:
//   pass V  per tile of 32 columns x 64 output rows: E and the recursions b_n,
//           b_n f~ of the region (with the W-row halos) in shared memory; the
//           column filterings of both, for every channel n < N, go to 2N
//           workspace planes of the band;
//   pass H  per tile of 32 rows x 64 output columns: for each channel filters
//           the two planes along the rows (W-column halos), regenerates b_n
//           at the tile's pixels and accumulates Q' and U'.
// Out-of-image pixels carry b_n = 0 (zero extension).
#include <algorithm>
#include <mutex>

#include "gpa_banded.cuh"

namespace {

using namespace bfk;

constexpr int kJVC = 32;             // pass V: columns per tile (16 column pairs)
constexpr int kJVNT = 128;           // pass V: 16 column pairs x 8 blocks of 8 output rows
constexpr int kJHT = 32, kJHW = 64;  // pass H: rows, output columns per tile
constexpr int kJHNT = 256;           // pass H: 32 rows x 8 segments of 8 columns
constexpr size_t kJointBandCap = 2ull << 30;
constexpr long long kJointBandCTAs = 8 * 152;

struct JointBandArgs {
  const float *in, *guide;
  float *out, *qaux;
  float *ws;         // 2 N planes of rows x Wp for the band
  long long plane;   // floats per band plane
  int Wp, H, W, pitch;
  int y0, rows;
  bfi::FilterConsts fc;
};

__host__ __device__ inline int jv_rows(int kind, int R, int ntp) {
  return kind == BF_SPATIAL_GAUSS ? kVB + ntp : kVB + 2 * R;
}
__host__ __device__ inline int jh_cols(int kind, int R, int ntp) {
  return kind == BF_SPATIAL_GAUSS ? kJHW + ntp : kJHW + 2 * R;
}
size_t jv_smem(int kind, int R, int ntp) { return 3 * (size_t)jv_rows(kind, R, ntp) * kJVC * sizeof(float); }
size_t jh_smem(int kind, int R, int ntp) {
  return 2 * (size_t)kJHT * hpass_pitch(jh_cols(kind, R, ntp)) * sizeof(float);
}

template <int KIND>
__global__ void __launch_bounds__(kJVNT) joint_band_vpass(const __grid_constant__ JointBandArgs A) {
  extern __shared__ __align__(16) float sm[];
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RR = jv_rows(KIND, R, fc.ntaps_pad);
  float *sE = sm, *sB = sE + RR * kJVC, *sF = sB + RR * kJVC;
  const int tx = blockIdx.x * kJVC;
  const int tyb = blockIdx.y * kVB;  // band-relative first output row
  const int ty = A.y0 + tyb;
  const int halo = kVB + 2 * R;      // rows of real data; the rest are zero padding
  for (int i = threadIdx.x; i < RR * kJVC; i += kJVNT) {
    const int r = i / kJVC, c = i % kJVC;
    const int gy = ty - R + r, gx = tx + c;
    float E = 0.f, b0 = 0.f, bf = 0.f;
    if (r < halo && gy >= 0 && gy < A.H && gx < A.W) {
      const long long o = (long long)gy * A.pitch + gx;
      const float d = __ldg(A.guide + o) - fc.tc;
      E = d * fc.inv_sr;
      b0 = exp2f(d * d * fc.e2c);  // exp(-E^2/2)
      bf = b0 * (__ldg(A.in + o) - fc.tc);
    }
    sE[i] = E;
    sB[i] = b0;
    sF[i] = bf;
  }
  constexpr int CS = kJVC / 2;
  const int cp = threadIdx.x % CS, yb = threadIdx.x / CS;  // 8 blocks of 8 output rows
  const int gx = tx + 2 * cp;
  const float2 *cB = reinterpret_cast<const float2 *>(sB + 8 * yb * kJVC) + cp;
  const float2 *cF = reinterpret_cast<const float2 *>(sF + 8 * yb * kJVC) + cp;
  for (int n = 0; n < N; ++n) {
    __syncthreads();  // region loaded / previous channel's filtering done
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
      for (int i = threadIdx.x; i < RR * kJVC / 4; i += kJVNT) {
        const float4 e = reinterpret_cast<const float4 *>(sE)[i];
        const float4 m = make_float4(e.x * rs, e.y * rs, e.z * rs, e.w * rs);
        float4 *pb = reinterpret_cast<float4 *>(sB) + i;
        float4 *pf = reinterpret_cast<float4 *>(sF) + i;
        float4 v = *pb;
        *pb = make_float4(v.x * m.x, v.y * m.y, v.z * m.z, v.w * m.w);
        v = *pf;
        *pf = make_float4(v.x * m.x, v.y * m.y, v.z * m.z, v.w * m.w);
      }
      __syncthreads();
    }
    float2 aB[8], aF[8];
    if (KIND == BF_SPATIAL_GAUSS) {
      float2 wB[8], wF[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        aB[i] = aF[i] = make_float2(0.f, 0.f);
        wB[i] = cB[i * CS];
        wF[i] = cF[i * CS];
      }
      for (int k = 0; k < fc.ntaps_pad; k += 8) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float w = fc.taps[k + j];
          const float2 w2 = make_float2(w, w);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            aB[i] = __ffma2_rn(w2, wB[(j + i) & 7], aB[i]);
            aF[i] = __ffma2_rn(w2, wF[(j + i) & 7], aF[i]);
          }
          wB[j] = cB[(k + j + 8) * CS];
          wF[j] = cF[(k + j + 8) * CS];
        }
      }
    } else {
      float2 sb = make_float2(0.f, 0.f), sf = sb;
      for (int r = 0; r <= 2 * R; ++r) {
        sb = __fadd2_rn(sb, cB[r * CS]);
        sf = __fadd2_rn(sf, cF[r * CS]);
      }
      aB[0] = sb;
      aF[0] = sf;
#pragma unroll
      for (int i = 1; i < 8; ++i) {
        const float2 ib = cB[(i + 2 * R) * CS], ob = cB[(i - 1) * CS];
        const float2 iff = cF[(i + 2 * R) * CS], of = cF[(i - 1) * CS];
        sb = __fadd2_rn(sb, __fadd2_rn(ib, make_float2(-ob.x, -ob.y)));
        sf = __fadd2_rn(sf, __fadd2_rn(iff, make_float2(-of.x, -of.y)));
        aB[i] = sb;
        aF[i] = sf;
      }
    }
    if (gx < A.Wp) {
      float *dB = A.ws + (2LL * n) * A.plane + gx;
      float *dF = dB + A.plane;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int orow = tyb + 8 * yb + i;
        if (orow < A.rows) {
          const long long o = (long long)orow * A.Wp;
          *reinterpret_cast<float2 *>(dB + o) = aB[i];
          *reinterpret_cast<float2 *>(dF + o) = aF[i];
        }
      }
    }
  }
}

// Row filtering of one plane at the thread's 8 pixels (rotating window).
template <int KIND>
__device__ __forceinline__ void jh_filter(const bfi::FilterConsts &fc, const float *v, float (&o)[8]) {
  if (KIND == BF_SPATIAL_GAUSS) {
    float win[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      o[i] = 0.f;
      win[i] = v[i];
    }
    for (int k = 0; k < fc.ntaps_pad; k += 8) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float w = fc.taps[k + j];
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = fmaf(w, win[(j + i) & 7], o[i]);
        win[j] = v[k + j + 8];
      }
    }
  } else {
    const int R = fc.R;
    float s = 0.f;
    for (int j = 0; j <= 2 * R; ++j) s += v[j];
    o[0] = s;
#pragma unroll
    for (int i = 1; i < 8; ++i) {
      s += v[i + 2 * R] - v[i - 1];
      o[i] = s;
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(kJHNT) joint_band_hpass(const __grid_constant__ JointBandArgs A) {
  extern __shared__ __align__(16) float sm[];
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RC = jh_cols(KIND, R, fc.ntaps_pad), P = hpass_pitch(RC);
  const int tx = blockIdx.x * kJHW;
  const int tyb = blockIdx.y * kJHT;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;  // row lane, 8-column segment
  const int gy = A.y0 + tyb + lane;
  const bool rowin = tyb + lane < A.rows;

  float b[8], E[8], Q[8], U[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gx = tx + 8 * seg + i;
    float e = 0.f, b0 = 0.f;
    if (rowin && gx < A.W) {
      const float d = __ldg(A.guide + (long long)gy * A.pitch + gx) - fc.tc;
      e = d * fc.inv_sr;
      b0 = exp2f(d * d * fc.e2c);
    }
    b[i] = b0;
    E[i] = e;
    Q[i] = U[i] = 0.f;
  }

  // the region's in-image columns are j in [j0, j1) of every row; the cells
  // outside the image or the band are zeroed once here (no copy writes them)
  const int j0 = max(0, R - tx), j1 = min(RC, A.W - tx + R);
  for (int pl = 0; pl < 2; ++pl)
    for (int r = seg; r < kJHT; r += kJHNT / 32) {
      const bool rin = tyb + r < A.rows;
      for (int j = lane; j < RC; j += 32)
        if (!rin || j < j0 || j >= j1) sm[pl * kJHT * P + r * P + j] = 0.f;
    }
  for (int n = 0; n < N; ++n) {
    for (int pl = 0; pl < 2; ++pl) {
      // column j of the region is image column tx - W + j
      const float *src = A.ws + (2LL * n + pl) * A.plane + (long long)tyb * A.Wp + (tx - R);
      float *buf = sm + pl * kJHT * P;
      for (int r = seg; r < kJHT && tyb + r < A.rows; r += kJHNT / 32) {
        const float *srow = src + (long long)r * A.Wp;
        float *drow = buf + r * P;
        for (int j = j0 + lane; j < j1; j += 32) cp_async4(drow + j, srow + j);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    float RB[8], RF[8];
    const int off = lane * P + 8 * seg;
    jh_filter<KIND>(fc, sm + off, RB);
    jh_filter<KIND>(fc, sm + kJHT * P + off, RF);
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float bn = n > 0 ? b[i] * (E[i] * rs) : b[i];
      Q[i] = fmaf(bn, RB[i], Q[i]);
      U[i] = fmaf(bn, RF[i], U[i]);
      b[i] = bn;
    }
    __syncthreads();  // the planes' buffers are refilled for the next channel
  }

  if (!rowin) return;
  const long long ro = (long long)gy * A.pitch;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gx = tx + 8 * seg + i;
    if (gx < A.W) {
      A.out[ro + gx] = fc.tc + __fdividef(U[i], Q[i]);  // 2-ulp division
      if (A.qaux) A.qaux[ro + gx] = Q[i] * fc.qscale;
    }
  }
}

int round_up4(int w) { return (w + 3) / 4 * 4; }

// The banded form pays off above radius 15 for the Gaussian; the box's fused
// running sums stay faster up to radius 24 (measured at 2048^2).
bool joint_banded_fits(const bfi::FilterConsts &fc) {
  return fc.kind == BF_SPATIAL_GAUSS ? fc.R > 15 : fc.R > 24;
}

int joint_band_rows(int height, int width, int N, size_t ws_bytes) {
  const size_t row_bytes = 2 * (size_t)N * round_up4(width) * sizeof(float);
  const int cap = (height + kVB - 1) / kVB * kVB;
  if (ws_bytes == 0) {  // preferred: several waves of pass-V CTAs, within the cap
    const long long col_tiles = (round_up4(width) + kJVC - 1) / kJVC;
    long long rows = (kJointBandCTAs + col_tiles - 1) / col_tiles * kVB;
    rows = std::min<long long>(rows, cap);
    const long long fit = (long long)(kJointBandCap / row_bytes) / kVB * kVB;
    if (fit >= kVB) rows = std::min(rows, fit);
    return (int)std::max<long long>(rows, kVB);
  }
  const size_t fit = ws_bytes / row_bytes / kVB * kVB;
  return (int)std::min<size_t>(fit, (size_t)cap);
}

template <int KIND>
bf_status run_joint_band(JointBandArgs &A, cudaStream_t s) {
  const int ntp_max = (2 * BF_MAX_RADIUS + 1 + 15) / 16 * 16;
  bf_status est = bfi::ensure_smem(reinterpret_cast<const void *>(joint_band_vpass<KIND>),
                                   jv_smem(KIND, BF_MAX_RADIUS, ntp_max));
  if (est == BF_OK)
    est = bfi::ensure_smem(reinterpret_cast<const void *>(joint_band_hpass<KIND>),
                           jh_smem(KIND, BF_MAX_RADIUS, ntp_max));
  if (est != BF_OK) return est;
  const int R = A.fc.R, ntp = A.fc.ntaps_pad;
  const size_t vs = jv_smem(KIND, R, ntp), hs = jh_smem(KIND, R, ntp);
  const int band = A.rows;
  for (int y0 = 0; y0 < A.H; y0 += band) {
    A.y0 = y0;
    A.rows = std::min(band, A.H - y0);
    dim3 gv((A.Wp + kJVC - 1) / kJVC, (A.rows + kVB - 1) / kVB);
    joint_band_vpass<KIND><<<gv, kJVNT, vs, s>>>(A);
    bf_status st = bfi::check_launch();
    if (st != BF_OK) return st;
    dim3 gh((A.W + kJHW - 1) / kJHW, (A.rows + kJHT - 1) / kJHT);
    joint_band_hpass<KIND><<<gh, kJHNT, hs, s>>>(A);
    st = bfi::check_launch();
    if (st != BF_OK) return st;
  }
  return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_joint_forward_workspace(int height, int width, const bf_params *p, size_t *bytes) {
  if (!bytes || height < 1 || width < 1) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  bf_status st = bfi::resolve(p, true, &fc);
  if (st != BF_OK) return st;
  *bytes = 0;
  if (!joint_banded_fits(fc)) return BF_OK;
  const size_t row_bytes = 2 * (size_t)fc.N * round_up4(width) * sizeof(float);
  *bytes = row_bytes * (size_t)joint_band_rows(height, width, fc.N, 0);
  return BF_OK;
}

bf_status bf_joint_forward_ws(const float *d_in, const float *d_guide, float *d_out,
                              float *d_qaux, int height, int width, int pitch, const bf_params *p,
                              void *d_workspace, size_t ws_bytes, void *stream) {
  bf_status st = bfi::check_image(d_in, d_out, height, width, pitch);
  if (st != BF_OK) return st;
  if (!d_guide || (reinterpret_cast<uintptr_t>(d_guide) & 3u)) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  st = bfi::resolve(p, true, &fc);
  if (st != BF_OK) return st;
  if (!joint_banded_fits(fc))
    return bf_joint_forward(d_in, d_guide, d_out, d_qaux, height, width, pitch, p, stream);
  if (!d_workspace) return BF_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(d_workspace) & 15u) return BF_ERR_INVALID_ARG;
  const int rows = joint_band_rows(height, width, fc.N, ws_bytes);
  if (rows < kVB) return BF_ERR_WORKSPACE;
  JointBandArgs A;
  A.in = d_in;
  A.guide = d_guide;
  A.out = d_out;
  A.qaux = d_qaux;
  A.ws = static_cast<float *>(d_workspace);
  A.Wp = round_up4(width);
  A.plane = (long long)rows * A.Wp;
  A.H = height;
  A.W = width;
  A.pitch = pitch;
  A.y0 = 0;
  A.rows = rows;
  A.fc = fc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return fc.kind == BF_SPATIAL_GAUSS ? run_joint_band<BF_SPATIAL_GAUSS>(A, s)
                                     : run_joint_band<BF_SPATIAL_BOX>(A, s);
}

}  // extern "C"
