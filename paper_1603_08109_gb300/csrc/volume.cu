// Algorithm 2 on volume (video) data: the straightforward extension of the
// filter to a box of Z^3 that Sec. I and Sec. V mention.  f is a grayscale
// volume (depth x height x width, packed: x fastest), the range kernel is the
// Gaussian of the planar filter, and the spatial kernel is the separable
// w(j) = w1(j_z) w1(j_y) w1(j_x) with the normalised 1-D box or Gaussian w1 of
// the planar filter along every axis; neighbours outside the volume do not
// contribute (zero extension).  With the rescaled power images
// a_n = e^{-H^2/2} H^n / sqrt(n!), H = (f - t_c) / sigma_r,
//   Q' = sum_{n<N} a_n (w * a_n),  P' = sum_{n=1..N} sqrt(n) a_{n-1} (w * a_n),
//   f_GPA = t_c + sigma_r P'/Q',
// exactly as for images; only the N + 1 filterings are 3-D.
//
// Two kernels:
//   vol_zpass   one thread per (y, x) column and 16 output planes z0..z0+15:
//               the column's f over the tile plus the W-plane halos is turned
//               into a_0 and H in shared memory (each thread its own column,
//               so no barriers), then channel by channel a_n is advanced in
//               place and filtered along z into the workspace plane Z_n
//               (N + 1 volumes of floats);
//   vol_yxpass  one CTA per 32 x 32 output tile of one z-plane: per channel
//               the Z_n region with the W-pixel halos is staged in shared
//               memory (cp.async, the next channel's region copied while the
//               current one is filtered), filtered along y, then along x, and the result
//               (w * a_n at the tile's voxels) is recombined with a_n at the
//               voxel itself (regenerated from f in registers) into Q', P'.
#include <algorithm>
#include <cmath>

#include "bf_internal.h"
#include "gpa_fixed.cuh"  // cp.async helpers

namespace {

constexpr int kVolMaxR = 31;   // radius limit of the volume path (taps <= 63)
constexpr int kZT = 16;        // z-pass output planes per thread
constexpr int kZNT = 128;      // z-pass threads per CTA (consecutive x)
constexpr int kYT = 32;        // y/x-pass output tile side
constexpr int kYNT = 256;      // y/x-pass threads per CTA (32 x 8)

struct VolArgs {
  const float *in;
  float *out, *qaux, *ws;
  long long plane;  // D * H * W: floats per workspace volume
  int D, H, W, R, L, N;
  float tc, sr, inv_sr, e2c;
  float taps[2 * kVolMaxR + 1];  // normalised w1(k - R), k = 0 .. 2R
};

__global__ void __launch_bounds__(kZNT) vol_zpass(const __grid_constant__ VolArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int RZ = kZT + 2 * A.R;
  float *sA = sm, *sH = sm + RZ * kZNT;  // [r][thread]
  const int t = threadIdx.x;
  const int x = blockIdx.x * kZNT + t, y = blockIdx.y, z0 = blockIdx.z * kZT;
  if (x >= A.W) return;  // no barriers: every thread owns its column
  const long long col = (long long)y * A.W + x, zs = (long long)A.H * A.W;
  for (int r = 0; r < RZ; ++r) {
    const int z = z0 - A.R + r;
    float a = 0.f, h = 0.f;
    if (z >= 0 && z < A.D) {
      const float d = __ldg(A.in + z * zs + col) - A.tc;
      h = d * A.inv_sr;
      a = exp2f(d * d * A.e2c);  // exp(-H^2/2)
    }
    sA[r * kZNT + t] = a;
    sH[r * kZNT + t] = h;
  }
  const int zn = min(kZT, A.D - z0);
  for (int n = 0; n <= A.N; ++n) {
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
      for (int r = 0; r < RZ; ++r) sA[r * kZNT + t] *= sH[r * kZNT + t] * rs;
    }
    float *dst = A.ws + (long long)n * A.plane + z0 * zs + col;
    for (int zo = 0; zo < zn; ++zo) {
      float acc = 0.f;
      for (int k = 0; k < A.L; ++k) acc = fmaf(A.taps[k], sA[(zo + k) * kZNT + t], acc);
      dst[zo * zs] = acc;
    }
  }
}

__global__ void __launch_bounds__(kYNT) vol_yxpass(const __grid_constant__ VolArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int RC = kYT + 2 * A.R, RP = RC + 1;  // region side, row pitch
  float *sR0 = sm, *sR1 = sm + RC * RP;       // two regions (RC x RP): channels n, n + 1
  float *sV = sm + 2 * RC * RP;               // vertical pass (32 x RP)
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  const int x0 = blockIdx.x * kYT, y0 = blockIdx.y * kYT, z = blockIdx.z;
  const long long zs = (long long)A.H * A.W, zoff = z * zs;
  constexpr int KR = kYT / (kYNT / 32);  // output rows per thread: ty, ty + 8, ...
  float a[KR], H[KR], Q[KR], P[KR];
  const int x = x0 + tx;
  for (int k = 0; k < KR; ++k) {
    const int y = y0 + ty + 8 * k;
    float av = 0.f, h = 0.f;
    if (x < A.W && y < A.H) {
      const float d = __ldg(A.in + zoff + (long long)y * A.W + x) - A.tc;
      h = d * A.inv_sr;
      av = exp2f(d * d * A.e2c);
    }
    a[k] = av;
    H[k] = h;
    Q[k] = P[k] = 0.f;
  }
  // channel n's region into buffer b (zeros outside the plane)
  auto issue = [&](int n, float *b) {
    const float *src = A.ws + (long long)n * A.plane + zoff;
    for (int e = t; e < RC * RC; e += kYNT) {
      const int rr = e / RC, cc = e - rr * RC;
      const int gy = y0 - A.R + rr, gx = x0 - A.R + cc;
      if (gy >= 0 && gy < A.H && gx >= 0 && gx < A.W)
        bfk::cp_async4(b + rr * RP + cc, src + (long long)gy * A.W + gx);
      else
        b[rr * RP + cc] = 0.f;
    }
  };
  issue(0, sR0);
  bfk::cp_async_commit();
  for (int n = 0; n <= A.N; ++n) {
    // the other buffer was last read by the previous channel's y pass, which
    // every thread finished before the barrier that ended it
    if (n + 1 <= A.N) issue(n + 1, (n & 1) ? sR0 : sR1);
    bfk::cp_async_commit();
    bfk::cp_async_wait<1>();  // this thread's copies of channel n have landed
    __syncthreads();          // ... and every thread's; the x pass of n - 1 is done with sV
    const float *sR = (n & 1) ? sR1 : sR0;
    for (int e = t; e < kYT * RC; e += kYNT) {  // along y: 32 output rows, every region column
      const int row = e / RC, cc = e - row * RC;
      float acc = 0.f;
      for (int k = 0; k < A.L; ++k) acc = fmaf(A.taps[k], sR[(row + k) * RP + cc], acc);
      sV[row * RP + cc] = acc;
    }
    __syncthreads();
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
    for (int k = 0; k < KR; ++k) {  // along x, then the recursion and the sums
      const float *vr = sV + (ty + 8 * k) * RP + tx;
      float ab = 0.f;
      for (int j = 0; j < A.L; ++j) ab = fmaf(A.taps[j], vr[j], ab);
      const float aold = a[k];  // a_{n-1}
      const float an = n > 0 ? aold * (H[k] * rs) : aold;
      if (n < A.N) Q[k] = fmaf(an, ab, Q[k]);
      if (n > 0) P[k] = fmaf(sq * aold, ab, P[k]);
      a[k] = an;
    }
  }
  if (x >= A.W) return;
  for (int k = 0; k < KR; ++k) {
    const int y = y0 + ty + 8 * k;
    if (y >= A.H) break;
    const long long o = zoff + (long long)y * A.W + x;
    A.out[o] = fmaf(A.sr, __fdividef(P[k], Q[k]), A.tc);  // approximate division (2 ulp)
    if (A.qaux) A.qaux[o] = Q[k];
  }
}

// Compile-time radius (W <= 8): the same two passes with every filter loop
// unrolled, the taps as constant operands and register windows, so that a
// shared-memory load serves several FMAs.  z-pass: the column's a_n and H in
// registers.  y/x pass: the y filter per (region column, 8 output rows), the
// x filter per (output row, 4 consecutive voxels), which are also the
// thread's voxels for the recursion and the sums.
constexpr int kVolFixedMaxR = 8;

template <int R>
__global__ void __launch_bounds__(kZNT) vol_zpass_r(const __grid_constant__ VolArgs A) {
  constexpr int L = 2 * R + 1, RZ = kZT + 2 * R;
  const int t = threadIdx.x;
  const int x = blockIdx.x * kZNT + t, y = blockIdx.y, z0 = blockIdx.z * kZT;
  if (x >= A.W) return;
  const long long col = (long long)y * A.W + x, zs = (long long)A.H * A.W;
  float a[RZ], h[RZ];
#pragma unroll
  for (int r = 0; r < RZ; ++r) {
    const int z = z0 - R + r;
    float av = 0.f, hv = 0.f;
    if (z >= 0 && z < A.D) {
      const float d = __ldg(A.in + z * zs + col) - A.tc;
      hv = d * A.inv_sr;
      av = exp2f(d * d * A.e2c);  // exp(-H^2/2)
    }
    a[r] = av;
    h[r] = hv;
  }
  const int zn = min(kZT, A.D - z0);
  for (int n = 0; n <= A.N; ++n) {
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
#pragma unroll
      for (int r = 0; r < RZ; ++r) a[r] *= h[r] * rs;
    }
    float *dst = A.ws + (long long)n * A.plane + z0 * zs + col;
#pragma unroll
    for (int zo = 0; zo < kZT; ++zo) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < L; ++k) acc = fmaf(A.taps[k], a[zo + k], acc);
      if (zo < zn) dst[zo * zs] = acc;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kYNT) vol_yxpass_r(const __grid_constant__ VolArgs A) {
  constexpr int L = 2 * R + 1, RC = kYT + 2 * R, RP = RC + 1;  // RP odd
  static_assert(4 * RC <= kYNT && kYT * kYT == 4 * kYNT, "thread mapping");
  extern __shared__ __align__(16) float sm[];
  float *sR0 = sm, *sR1 = sm + RC * RP, *sV = sm + 2 * RC * RP;
  const int t = threadIdx.x;
  const int x0 = blockIdx.x * kYT, y0 = blockIdx.y * kYT, z = blockIdx.z;
  const long long zs = (long long)A.H * A.W, zoff = z * zs;
  const int orow = t >> 3, oc = 4 * (t & 7);  // the thread's voxels: row orow, columns oc..oc+3
  const int y = y0 + orow;
  const int vcc = t % RC, vch = t / RC;        // y filter item: region column, 8-row chunk
  const bool vact = vch < 4;
  float a[4], H[4], Q[4], P[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int x = x0 + oc + k;
    float av = 0.f, h = 0.f;
    if (x < A.W && y < A.H) {
      const float d = __ldg(A.in + zoff + (long long)y * A.W + x) - A.tc;
      h = d * A.inv_sr;
      av = exp2f(d * d * A.e2c);
    }
    a[k] = av;
    H[k] = h;
    Q[k] = P[k] = 0.f;
  }
  auto issue = [&](int n, float *b) {  // channel n's region (zeros outside the plane)
    const float *src = A.ws + (long long)n * A.plane + zoff;
    for (int e = t; e < RC * RC; e += kYNT) {
      const int rr = e / RC, cc = e - rr * RC;
      const int gy = y0 - R + rr, gx = x0 - R + cc;
      if (gy >= 0 && gy < A.H && gx >= 0 && gx < A.W)
        bfk::cp_async4(b + rr * RP + cc, src + (long long)gy * A.W + gx);
      else
        b[rr * RP + cc] = 0.f;
    }
  };
  issue(0, sR0);
  bfk::cp_async_commit();
  for (int n = 0; n <= A.N; ++n) {
    if (n + 1 <= A.N) issue(n + 1, (n & 1) ? sR0 : sR1);  // last read by the y filter of n - 1
    bfk::cp_async_commit();
    bfk::cp_async_wait<1>();
    __syncthreads();
    const float *sR = (n & 1) ? sR1 : sR0;
    if (vact) {
      float w[8 + 2 * R];
#pragma unroll
      for (int i = 0; i < 8 + 2 * R; ++i) w[i] = sR[(8 * vch + i) * RP + vcc];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < L; ++k) acc = fmaf(A.taps[k], w[r + k], acc);
        sV[(8 * vch + r) * RP + vcc] = acc;
      }
    }
    __syncthreads();
    float w[4 + 2 * R];
#pragma unroll
    for (int i = 0; i < 4 + 2 * R; ++i) w[i] = sV[orow * RP + oc + i];
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float ab = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) ab = fmaf(A.taps[j], w[k + j], ab);
      const float aold = a[k];  // a_{n-1}
      const float an = n > 0 ? aold * (H[k] * rs) : aold;
      if (n < A.N) Q[k] = fmaf(an, ab, Q[k]);
      if (n > 0) P[k] = fmaf(sq * aold, ab, P[k]);
      a[k] = an;
    }
  }
  if (y >= A.H) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int x = x0 + oc + k;
    if (x < A.W) {
      const long long o = zoff + (long long)y * A.W + x;
      A.out[o] = fmaf(A.sr, __fdividef(P[k], Q[k]), A.tc);  // approximate division (2 ulp)
      if (A.qaux) A.qaux[o] = Q[k];
    }
  }
}

template <int R>
bf_status launch_volume_r(const VolArgs &A, cudaStream_t s) {
  constexpr int RC = kYT + 2 * R;
  constexpr size_t ys = (size_t)(2 * RC + kYT) * (RC + 1) * sizeof(float);
  bf_status st = bfi::ensure_smem(reinterpret_cast<const void *>(vol_yxpass_r<R>), ys);
  if (st != BF_OK) return st;
  dim3 gz((A.W + kZNT - 1) / kZNT, A.H, (A.D + kZT - 1) / kZT);
  vol_zpass_r<R><<<gz, kZNT, 0, s>>>(A);
  st = bfi::check_launch();
  if (st != BF_OK) return st;
  dim3 gy((A.W + kYT - 1) / kYT, (A.H + kYT - 1) / kYT, A.D);
  vol_yxpass_r<R><<<gy, kYNT, ys, s>>>(A);
  return bfi::check_launch();
}

bf_status launch_volume_fixed(const VolArgs &A, cudaStream_t s) {
  switch (A.R) {
    case 0: return launch_volume_r<0>(A, s);
    case 1: return launch_volume_r<1>(A, s);
    case 2: return launch_volume_r<2>(A, s);
    case 3: return launch_volume_r<3>(A, s);
    case 4: return launch_volume_r<4>(A, s);
    case 5: return launch_volume_r<5>(A, s);
    case 6: return launch_volume_r<6>(A, s);
    case 7: return launch_volume_r<7>(A, s);
    case 8: return launch_volume_r<8>(A, s);
    default: return BF_ERR_UNSUPPORTED;
  }
}

size_t zpass_smem(int R) { return (size_t)2 * (kZT + 2 * R) * kZNT * sizeof(float); }
size_t yxpass_smem(int R) {
  const size_t RC = kYT + 2 * (size_t)R;
  return (2 * RC + kYT) * (RC + 1) * sizeof(float);
}

bf_status resolve_volume(const bf_params *p, bfi::FilterConsts *fc) {
  bf_status st = bfi::resolve(p, true, fc);
  if (st != BF_OK) return st;
  if (fc->kind != BF_SPATIAL_BOX && fc->kind != BF_SPATIAL_GAUSS) return BF_ERR_INVALID_ARG;
  if (fc->R > kVolMaxR) return BF_ERR_UNSUPPORTED;
  return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_volume_workspace(int depth, int height, int width, const bf_params *p,
                              size_t *bytes) {
  if (!bytes || depth < 1 || height < 1 || width < 1) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  const bf_status st = resolve_volume(p, &fc);
  if (st != BF_OK) return st;
  *bytes = (size_t)(fc.N + 1) * (size_t)depth * (size_t)height * (size_t)width * sizeof(float);
  return BF_OK;
}

bf_status bf_volume_forward(const float *d_in, float *d_out, float *d_qaux, int depth,
                            int height, int width, const bf_params *p, void *d_ws,
                            size_t ws_bytes, void *stream) {
  if (!d_in || !d_out || d_in == d_out || depth < 1 || height < 1 || width < 1)
    return BF_ERR_INVALID_ARG;
  if (d_qaux && (d_qaux == d_in || d_qaux == d_out)) return BF_ERR_INVALID_ARG;
  if (height > 65535 || depth > 65535) return BF_ERR_UNSUPPORTED;  // grid limits
  bfi::FilterConsts fc;
  bf_status st = resolve_volume(p, &fc);
  if (st != BF_OK) return st;
  const size_t need = (size_t)(fc.N + 1) * (size_t)depth * (size_t)height * (size_t)width *
                      sizeof(float);
  if (!d_ws || ws_bytes < need) return BF_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(d_ws) & 15u) != 0) return BF_ERR_INVALID_ARG;
  VolArgs A = {};
  A.in = d_in;
  A.out = d_out;
  A.qaux = d_qaux;
  A.ws = static_cast<float *>(d_ws);
  A.plane = (long long)depth * height * width;
  A.D = depth;
  A.H = height;
  A.W = width;
  A.R = fc.R;
  A.L = 2 * fc.R + 1;
  A.N = fc.N;
  A.tc = fc.tc;
  A.sr = fc.sr;
  A.inv_sr = fc.inv_sr;
  A.e2c = fc.e2c;
  for (int k = 0; k < A.L; ++k)
    A.taps[k] = fc.kind == BF_SPATIAL_GAUSS ? fc.taps[k] : (float)(1.0 / (double)A.L);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fc.R <= kVolFixedMaxR) return launch_volume_fixed(A, s);
  const size_t zs = zpass_smem(fc.R), ys = yxpass_smem(fc.R);
  st = bfi::ensure_smem(reinterpret_cast<const void *>(vol_zpass), zpass_smem(kVolMaxR));
  if (st == BF_OK)
    st = bfi::ensure_smem(reinterpret_cast<const void *>(vol_yxpass), yxpass_smem(kVolMaxR));
  if (st != BF_OK) return st;
  dim3 gz((width + kZNT - 1) / kZNT, height, (depth + kZT - 1) / kZT);
  vol_zpass<<<gz, kZNT, zs, s>>>(A);
  st = bfi::check_launch();
  if (st != BF_OK) return st;
  dim3 gy((width + kYT - 1) / kYT, (height + kYT - 1) / kYT, depth);
  vol_yxpass<<<gy, kYNT, ys, s>>>(A);
  return bfi::check_launch();
}

}  // extern "C"
