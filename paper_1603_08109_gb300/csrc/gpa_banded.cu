// Two-pass banded forward of Algorithm 2 for large radii (W > 15).
//
// A fused 2-D tile needs a 2W halo in both directions: at W = 60 its region
// is tens of times the tile, does not fit shared memory at a useful size, and
// the tile runs at a few per cent of the FP32 pipe.  The spatial filter is
// separable (eq. spatial_kernel1 on the square Omega), so here the image is cut
// into bands of rows and each band goes through two kernels:
//   pass V  per tile of 64 columns x 64 output rows: loads f for the tile's
//           rows plus the W-row halos, generates a_0 and then a_n in shared
//           memory (Algorithm 2's recursion, rescaled by 1/sqrt(n!)), and
//           writes the vertical filtering (w_1 * a_n) of every channel
//           n = 0..N to a workspace of N + 1 planes covering the band;
//   pass H  per tile of 32 rows x 128 output columns: for each channel reads
//           the plane with the W-column halos (cp.async, one channel ahead),
//           filters along the rows, regenerates a_n at the tile's pixels and
//           accumulates Q' and P' (eqs. P, Q), then f_GPA = t_c + sigma_r P'/Q'.
// Each pass carries a halo in one direction only.  Bands are as tall as
// needed to give each launch several waves of CTAs (the workspace is capped
// at 2 GiB by default).  Out-of-image pixels carry a_n = 0 (zero extension),
// as in the fused kernels.
#include <algorithm>
#include <mutex>

#include "bf_internal.h"
#include "gpa_fixed.cuh"

namespace {

constexpr int kBandNT = 256;
constexpr int kVC = 64, kVB = 64;   // pass V tile: columns, output rows
constexpr int kHT = 32, kHW = 128;  // pass H tile: rows, output columns
constexpr size_t kBandCap = 2ull << 30;   // default workspace cap (bytes)
constexpr long long kBandCTAs = 8 * 152;   // pass-V CTAs per band wanted

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

size_t vpass_smem(int kind, int R, int ntp) { return 2 * (size_t)vpass_rows(kind, R, ntp) * kVC * sizeof(float); }
size_t hpass_smem(int kind, int R, int ntp) {
  return 2 * (size_t)kHT * hpass_pitch(hpass_cols(kind, R, ntp)) * sizeof(float);
}

template <int KIND>
__global__ void __launch_bounds__(kBandNT) band_vpass(const __grid_constant__ BandArgs A) {
  extern __shared__ __align__(16) float sm[];
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RR = vpass_rows(KIND, R, fc.ntaps_pad);
  float *sH = sm, *sA = sm + RR * kVC;
  const int tx = blockIdx.x * kVC;
  const int tyb = blockIdx.y * kVB;  // band-relative first output row
  const int ty = A.y0 + tyb;
  const int halo = kVB + 2 * R;      // rows of real data; the rest are zero padding
  for (int i = threadIdx.x; i < RR * kVC; i += kBandNT) {
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
  const int c = threadIdx.x % kVC, yb = threadIdx.x / kVC;  // 4 blocks of 16 output rows
  const int gx = tx + c;
  const float *col = sA + 16 * yb * kVC + c;
  for (int n = 0; n <= N; ++n) {
    __syncthreads();  // region loaded / previous channel's filtering done
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
      float4 *a4 = reinterpret_cast<float4 *>(sA);
      const float4 *h4 = reinterpret_cast<const float4 *>(sH);
      for (int i = threadIdx.x; i < RR * kVC / 4; i += kBandNT) {
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
    float acc[16];
    if (KIND == BF_SPATIAL_GAUSS) {
      float win[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        acc[i] = 0.f;
        win[i] = col[i * kVC];
      }
      for (int k = 0; k < fc.ntaps_pad; k += 16) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float w = fc.taps[k + j];
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[i] = fmaf(w, win[(j + i) & 15], acc[i]);
          win[j] = col[(k + j + 16) * kVC];
        }
      }
    } else {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int r = 0;
      for (; r + 3 <= 2 * R; r += 4) {
        s0 += col[r * kVC];
        s1 += col[(r + 1) * kVC];
        s2 += col[(r + 2) * kVC];
        s3 += col[(r + 3) * kVC];
      }
      for (; r <= 2 * R; ++r) s0 += col[r * kVC];
      float s = (s0 + s1) + (s2 + s3);
      acc[0] = s;
#pragma unroll
      for (int i = 1; i < 16; ++i) {
        s += col[(i + 2 * R) * kVC] - col[(i - 1) * kVC];
        acc[i] = s;
      }
    }
    if (c < A.Wp - tx) {  // columns W..Wp-1 of the workspace are written as zeros
      float *dst = A.ws + (long long)n * A.plane + gx;
      const bool colin = gx < A.W;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int orow = tyb + 16 * yb + i;
        if (orow < A.rows) dst[(long long)orow * A.Wp] = colin ? acc[i] : 0.f;
      }
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(kBandNT) band_hpass(const __grid_constant__ BandArgs A) {
  extern __shared__ __align__(16) float sm[];
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RC = hpass_cols(KIND, R, fc.ntaps_pad), P = hpass_pitch(RC);
  float *const buf0 = sm, *const buf1 = sm + kHT * P;
  const int tx = blockIdx.x * kHW;
  const int tyb = blockIdx.y * kHT;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;  // row lane, 16 columns seg

  // plane n of rows tyb.., columns tx - W.., into b; each warp copies four
  // rows, its lanes consecutive columns (zeros outside the image / band)
  auto load = [&](int n, float *b) {
    const float *src = A.ws + (long long)n * A.plane;
    for (int r = seg; r < kHT; r += kBandNT / 32) {
      const int orow = tyb + r;
      const float *srow = src + (long long)orow * A.Wp;
      float *drow = b + r * P;
      for (int j = lane; j < RC; j += 32) {
        const int gx = tx - R + j;
        if (orow < A.rows && gx >= 0 && gx < A.W)
          bfk::cp_async4(drow + j, srow + gx);
        else
          drow[j] = 0.f;
      }
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
    float Ab[16];
    if (KIND == BF_SPATIAL_GAUSS) {
      float win[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        Ab[i] = 0.f;
        win[i] = vrow0[i];
      }
      for (int k = 0; k < fc.ntaps_pad; k += 16) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float w = fc.taps[k + j];
#pragma unroll
          for (int i = 0; i < 16; ++i) Ab[i] = fmaf(w, win[(j + i) & 15], Ab[i]);
          win[j] = vrow0[k + j + 16];
        }
      }
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

bool banded_fits(const bfi::FilterConsts &fc) { return fc.R > 15; }

int round_up4(int w) { return (w + 3) / 4 * 4; }

// Band rows for a workspace of ws_bytes (multiple of 64, at most the image
// height rounded up), or 0 when the workspace holds fewer than 64 rows.
int band_rows(int height, int width, int N, size_t ws_bytes) {
  const size_t row_bytes = (size_t)(N + 1) * (size_t)round_up4(width) * sizeof(float);
  const size_t fit = ws_bytes / row_bytes;
  const int cap = (height + kVB - 1) / kVB * kVB;
  if (fit < (size_t)kVB) return 0;
  return (int)std::min<size_t>(fit / kVB * kVB, (size_t)cap);
}

// Preferred band rows: enough pass-V tiles for several waves, within the cap.
int preferred_band_rows(int height, int width, int N) {
  const long long col_tiles = (width + kVC - 1) / kVC;
  long long rows = (kBandCTAs + col_tiles - 1) / col_tiles * kVB;
  rows = std::min<long long>(rows, (height + kVB - 1) / kVB * kVB);
  const int fit = band_rows(height, width, N, kBandCap);
  if (fit > 0) rows = std::min<long long>(rows, fit);
  return (int)std::max<long long>(rows, kVB);
}

template <int KIND>
bf_status launch_band(BandArgs &A, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t init_err = cudaSuccess;
  std::call_once(once, [] {
    const int ntp_max = (2 * BF_MAX_RADIUS + 1 + 15) / 16 * 16;
    cudaError_t e = cudaFuncSetAttribute(band_vpass<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)vpass_smem(KIND, BF_MAX_RADIUS, ntp_max));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(band_hpass<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)hpass_smem(KIND, BF_MAX_RADIUS, ntp_max));
    init_err = e;
  });
  if (init_err != cudaSuccess) return bfi::cuda_status(init_err);
  const int R = A.fc.R, ntp = A.fc.ntaps_pad;
  const size_t vs = vpass_smem(KIND, R, ntp), hs = hpass_smem(KIND, R, ntp);
  const int band = A.rows;
  for (int y0 = 0; y0 < A.H; y0 += band) {
    A.y0 = y0;
    A.rows = std::min(band, A.H - y0);
    dim3 gv((A.Wp + kVC - 1) / kVC, (A.rows + kVB - 1) / kVB);
    band_vpass<KIND><<<gv, kBandNT, vs, s>>>(A);
    bf_status st = bfi::check_launch();
    if (st != BF_OK) return st;
    dim3 gh((A.W + kHW - 1) / kHW, (A.rows + kHT - 1) / kHT);
    band_hpass<KIND><<<gh, kBandNT, hs, s>>>(A);
    st = bfi::check_launch();
    if (st != BF_OK) return st;
  }
  return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_fast_forward_workspace(int height, int width, const bf_params *p, size_t *bytes) {
  if (!bytes || height < 1 || width < 1) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  bf_status st = bfi::resolve(p, true, &fc);
  if (st != BF_OK) return st;
  *bytes = 0;
  if (!banded_fits(fc)) return BF_OK;
  const size_t row_bytes = (size_t)(fc.N + 1) * (size_t)round_up4(width) * sizeof(float);
  *bytes = row_bytes * (size_t)preferred_band_rows(height, width, fc.N);
  return BF_OK;
}

bf_status bf_fast_forward_ws(const float *d_in, float *d_out, float *d_qaux, int height, int width,
                             int pitch, const bf_params *p, void *d_workspace, size_t ws_bytes,
                             void *stream) {
  bf_status st = bfi::check_image(d_in, d_out, height, width, pitch);
  if (st != BF_OK) return st;
  bfi::FilterConsts fc;
  st = bfi::resolve(p, true, &fc);
  if (st != BF_OK) return st;
  if (!banded_fits(fc)) return bf_fast_forward(d_in, d_out, d_qaux, height, width, pitch, p, stream);
  if (!d_workspace) return BF_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(d_workspace) & 15u) return BF_ERR_INVALID_ARG;
  const int rows = band_rows(height, width, fc.N, ws_bytes);
  if (rows == 0) return BF_ERR_WORKSPACE;
  BandArgs A;
  A.in = d_in;
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
  return fc.kind == BF_SPATIAL_GAUSS ? launch_band<BF_SPATIAL_GAUSS>(A, s)
                                     : launch_band<BF_SPATIAL_BOX>(A, s);
}

}  // extern "C"
