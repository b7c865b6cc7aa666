// Direct bilateral filter (eq. BF): O((2W+1)^2) range-kernel evaluations per
// pixel, float32.  The same-GPU comparison for the fast filter, plus its
// exact gradient with respect to the image and sigma_r (gather form).
//
// Each CTA stages its output tile plus an R-pixel halo of f in shared memory;
// each thread produces KX consecutive outputs of one row and walks the
// (2R+1)^2 neighbours with a KX-wide register window along x.  The spatial
// and range weights are combined into one base-2 exponent:
//   w(j) g(t - tau) = 2^( -(t - tau)^2 log2(e) / (2 sigma_r^2) + lw(j) ),
// lw(j) = log2 of the unnormalised spatial weight (0 for the box,
// -(dx^2 + dy^2) log2(e) / (2 sigma_s^2) for the Gaussian); the kernel's
// normalisation cancels in the ratio.
#include <math.h>

#include "bf_internal.h"

namespace {

constexpr int DTH = 16;   // output rows per tile
constexpr int DKX = 4;    // outputs per thread along x
constexpr int DNT = 256;  // threads
constexpr int DTW = (DNT / DTH) * DKX;  // 64 output columns

struct DirectArgs {
  const float *in;
  float *out;
  // backward extras
  const float *gout;
  float *gin;
  float *ws_out, *ws_u, *ws_self;  // per-pixel out, g/D, centre term
  double *partials;
  int H, W, pitch, R;
  float tc, negc;       // negc = -log2(e) / (2 sigma_r^2)
  float inv_sr2;        // 1 / sigma_r^2
  float inv_sr;
  float lx[2 * BF_MAX_RADIUS + 1];  // log2 spatial weight per axis offset
};

__host__ __device__ inline size_t region_floats(int R) { return (size_t)(DTH + 2 * R) * (DTW + 2 * R + 1); }

__device__ __forceinline__ void load_region(const float *src, int H, int W, int pitch, int ty0,
                                            int tx0, int R, float *s, int sp, float fill) {
  const int RH = DTH + 2 * R, RW = DTW + 2 * R;
  for (int i = threadIdx.x; i < RH * RW; i += blockDim.x) {
    const int r = i / RW, c = i % RW;
    const int gy = ty0 - R + r, gx = tx0 - R + c;
    float v = fill;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = __ldg(src + (long long)gy * pitch + gx);
    s[r * sp + c] = v;
  }
}

__device__ __forceinline__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// MODE 0: forward (out).  MODE 1: backward pass 1 (out, g/D, centre term,
// sigma_r partials) -- everything of the gradient that is local to pixel i.
template <int MODE>
__global__ void __launch_bounds__(DNT) direct_kernel(const __grid_constant__ DirectArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int R = A.R;
  const int sp = DTW + 2 * R + 1;
  const int ty0 = blockIdx.y * DTH, tx0 = blockIdx.x * DTW;
  // in-image mask: out-of-image neighbours carry NaN and are skipped
  load_region(A.in, A.H, A.W, A.pitch, ty0, tx0, R, sm, sp, __int_as_float(0x7fc00000));
  __syncthreads();
  const int y = threadIdx.x % DTH;
  const int x0 = (threadIdx.x / DTH) * DKX;
  float tau[DKX], num[DKX], den[DKX], cen[DKX], sig[DKX];
#pragma unroll
  for (int k = 0; k < DKX; ++k) {
    tau[k] = sm[(y + R) * sp + x0 + k + R];
    num[k] = den[k] = cen[k] = sig[k] = 0.f;
  }
  // pass A: numerator and denominator
  for (int dy = -R; dy <= R; ++dy) {
    const float *row = sm + (y + R + dy) * sp + x0;
    const float ly = A.lx[dy + R];
    float win[DKX];
#pragma unroll
    for (int i = 0; i < DKX; ++i) win[i] = row[i];
    for (int db = 0; db < 2 * R + 1; db += DKX) {
#pragma unroll
      for (int u = 0; u < DKX; ++u) {
        const int dx = db + u;  // window holds columns dx .. dx + DKX - 1
        if (dx <= 2 * R) {
          const float lw = ly + A.lx[dx];
#pragma unroll
          for (int k = 0; k < DKX; ++k) {
            const float t = win[(u + k) % DKX];
            const float d = t - tau[k];
            const float wt = exp2f(fmaf(d * d, A.negc, lw));
            if (t == t) {  // skip out-of-image neighbours
              num[k] = fmaf(wt, d, num[k]);  // centred on f(i): small summands
              den[k] += wt;
            }
          }
          win[u] = row[min(dx + DKX, sp - 1)];
        }
      }
    }
  }
  if (MODE == 1) {
    // pass B: centre-derivative and sigma_r sums need out_i first
    float o[DKX];
#pragma unroll
    for (int k = 0; k < DKX; ++k) o[k] = tau[k] + num[k] / den[k];
    for (int dy = -R; dy <= R; ++dy) {
      const float *row = sm + (y + R + dy) * sp + x0;
      const float ly = A.lx[dy + R];
      for (int dx = 0; dx <= 2 * R; ++dx) {
        const float lw = ly + A.lx[dx];
#pragma unroll
        for (int k = 0; k < DKX; ++k) {
          const float t = row[min(dx + k, sp - 1)];
          const float d = t - tau[k];
          const float wt = exp2f(fmaf(d * d, A.negc, lw));
          if (t == t) {
            const float e = (t - o[k]) * wt * d;
            cen[k] = fmaf(e, 1.0f, cen[k]);
            sig[k] = fmaf(e, d, sig[k]);
          }
        }
      }
    }
    double part = 0.0;
    const int gy = ty0 + y;
#pragma unroll
    for (int k = 0; k < DKX; ++k) {
      const int gx = tx0 + x0 + k;
      if (gy < A.H && gx < A.W) {
        const long long off = (long long)gy * A.W + gx;  // workspace is dense
        const float g = __ldg(A.gout + (long long)gy * A.pitch + gx);
        const float u = g / den[k];
        A.ws_out[off] = o[k];
        A.ws_u[off] = u;
        A.ws_self[off] = u * cen[k] * A.inv_sr2;
        part += (double)u * (double)sig[k];
      }
    }
    if (A.partials) {
      __shared__ double red[32];
      const double t = block_sum_d(part * (double)A.inv_sr2 * (double)A.inv_sr, red);
      if (threadIdx.x == 0) A.partials[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  } else {
    const int gy = ty0 + y;
    if (gy < A.H) {
#pragma unroll
      for (int k = 0; k < DKX; ++k) {
        const int gx = tx0 + x0 + k;
        if (gx < A.W) A.out[(long long)gy * A.pitch + gx] = tau[k] + num[k] / den[k];
      }
    }
  }
}

// Backward pass 2 (gather): pixel k is the neighbour t of every i = k + j:
//   gin_k = self_k + sum_j (g_i / D_i) w(j) g(f_k - f_i) [1 - (f_k - out_i)(f_k - f_i)/sigma_r^2]
__global__ void __launch_bounds__(DNT) direct_bwd_gather(const __grid_constant__ DirectArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int R = A.R;
  const int sp = DTW + 2 * R + 1;
  const size_t plane = region_floats(R);
  float *sf = sm, *so = sm + plane, *su = sm + 2 * plane;
  const int ty0 = blockIdx.y * DTH, tx0 = blockIdx.x * DTW;
  load_region(A.in, A.H, A.W, A.pitch, ty0, tx0, R, sf, sp, 0.f);
  load_region(A.ws_out, A.H, A.W, A.W, ty0, tx0, R, so, sp, 0.f);
  load_region(A.ws_u, A.H, A.W, A.W, ty0, tx0, R, su, sp, 0.f);  // u = 0 outside the image
  __syncthreads();
  const int y = threadIdx.x % DTH;
  const int x0 = (threadIdx.x / DTH) * DKX;
  float fk[DKX], acc[DKX];
#pragma unroll
  for (int k = 0; k < DKX; ++k) {
    fk[k] = sf[(y + R) * sp + x0 + k + R];
    acc[k] = 0.f;
  }
  for (int dy = -R; dy <= R; ++dy) {
    const int rbase = (y + R + dy) * sp + x0;
    const float ly = A.lx[dy + R];
    for (int dx = 0; dx <= 2 * R; ++dx) {
      const float lw = ly + A.lx[dx];
#pragma unroll
      for (int k = 0; k < DKX; ++k) {
        const int idx = rbase + min(dx + k, sp - 1);
        const float fi = sf[idx], oi = so[idx], ui = su[idx];
        const float d = fk[k] - fi;
        const float wt = exp2f(fmaf(d * d, A.negc, lw));
        const float term = fmaf(-(fk[k] - oi) * d, A.inv_sr2, 1.0f);
        acc[k] = fmaf(ui * wt, term, acc[k]);
      }
    }
  }
  const int gy = ty0 + y;
  if (gy < A.H) {
#pragma unroll
    for (int k = 0; k < DKX; ++k) {
      const int gx = tx0 + x0 + k;
      if (gx < A.W) {
        const long long off = (long long)gy * A.W + gx;
        A.gin[(long long)gy * A.pitch + gx] = A.ws_self[off] + acc[k];
      }
    }
  }
}

__global__ void __launch_bounds__(256) reduce_partials_d(const double *p, int n, double *out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
  const double t = block_sum_d(v, red);
  if (threadIdx.x == 0) *out = t;
}

bf_status fill_args(const bf_params *p, int H, int W, int pitch, DirectArgs *A) {
  bfi::FilterConsts fc;
  bf_status st = bfi::resolve(p, false, &fc);
  if (st != BF_OK) return st;
  memset(A, 0, sizeof(*A));
  A->H = H;
  A->W = W;
  A->pitch = pitch;
  A->R = fc.R;
  A->tc = fc.tc;
  const double log2e = 1.4426950408889634;
  const double sr = p->sigma_r;
  A->negc = (float)(-log2e / (2.0 * sr * sr));
  A->inv_sr2 = (float)(1.0 / (sr * sr));
  A->inv_sr = (float)(1.0 / sr);
  for (int k = -fc.R; k <= fc.R; ++k) {
    double v = 0.0;
    if (fc.kind == BF_SPATIAL_GAUSS) v = -(double)k * k * log2e / (2.0 * (double)p->sigma_s * p->sigma_s);
    A->lx[k + fc.R] = (float)v;
  }
  return BF_OK;
}

template <typename K>
bf_status set_smem(K kern, size_t bytes) {
  return bfi::ensure_smem(reinterpret_cast<const void *>(kern), bytes);
}

dim3 direct_grid(int H, int W) { return dim3((W + DTW - 1) / DTW, (H + DTH - 1) / DTH); }

}  // namespace

extern "C" {

bf_status bf_direct(const float *d_in, float *d_out, int height, int width, int pitch,
                    const bf_params *p, void *stream) {
  bf_status st = bfi::check_image(d_in, d_out, height, width, pitch);
  if (st != BF_OK) return st;
  DirectArgs A;
  st = fill_args(p, height, width, pitch, &A);
  if (st != BF_OK) return st;
  A.in = d_in;
  A.out = d_out;
  const size_t smem = region_floats(A.R) * sizeof(float);
  st = set_smem(direct_kernel<0>, smem);
  if (st != BF_OK) return st;
  direct_kernel<0><<<direct_grid(height, width), DNT, smem, static_cast<cudaStream_t>(stream)>>>(A);
  return bfi::check_launch();
}

bf_status bf_direct_backward_workspace(int height, int width, const bf_params *p, size_t *bytes) {
  if (!bytes || height < 1 || width < 1) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  bf_status st = bfi::resolve(p, false, &fc);
  if (st != BF_OK) return st;
  const dim3 g = direct_grid(height, width);
  const size_t px = (size_t)height * width;
  size_t b = 3 * px * sizeof(float);
  b = (b + 255) / 256 * 256;
  *bytes = b + (size_t)g.x * g.y * sizeof(double);
  return BF_OK;
}

bf_status bf_direct_backward(const float *d_in, const float *d_gout, float *d_gin,
                             double *d_gsigma, int height, int width, int pitch,
                             const bf_params *p, void *d_workspace, size_t workspace_bytes,
                             void *stream) {
  bf_status st = bfi::check_image(d_in, d_gin, height, width, pitch);
  if (st != BF_OK) return st;
  if (!d_gout) return BF_ERR_INVALID_ARG;
  size_t need = 0;
  st = bf_direct_backward_workspace(height, width, p, &need);
  if (st != BF_OK) return st;
  if (!d_workspace || workspace_bytes < need) return BF_ERR_WORKSPACE;
  DirectArgs A;
  st = fill_args(p, height, width, pitch, &A);
  if (st != BF_OK) return st;
  const size_t px = (size_t)height * width;
  char *ws = static_cast<char *>(d_workspace);
  A.in = d_in;
  A.gout = d_gout;
  A.gin = d_gin;
  A.ws_out = reinterpret_cast<float *>(ws);
  A.ws_u = A.ws_out + px;
  A.ws_self = A.ws_u + px;
  A.partials = reinterpret_cast<double *>(ws + (3 * px * sizeof(float) + 255) / 256 * 256);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 g = direct_grid(height, width);
  const size_t smem1 = region_floats(A.R) * sizeof(float);
  st = set_smem(direct_kernel<1>, smem1);
  if (st != BF_OK) return st;
  direct_kernel<1><<<g, DNT, smem1, s>>>(A);
  st = bfi::check_launch();
  if (st != BF_OK) return st;
  const size_t smem2 = 3 * region_floats(A.R) * sizeof(float);
  if (smem2 > 232448) return BF_ERR_UNSUPPORTED;
  st = set_smem(direct_bwd_gather, smem2);
  if (st != BF_OK) return st;
  direct_bwd_gather<<<g, DNT, smem2, s>>>(A);
  st = bfi::check_launch();
  if (st != BF_OK || !d_gsigma) return st;
  reduce_partials_d<<<1, 256, 0, s>>>(A.partials, (int)(g.x * g.y), d_gsigma);
  return bfi::check_launch();
}

}  // extern "C"
