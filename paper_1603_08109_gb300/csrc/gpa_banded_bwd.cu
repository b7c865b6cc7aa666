// Two-pass banded backward for large radii (W > 15): the adjoint of the
// rescaled P'/Q' ratio (same formulas as the fused backward kernels), with the
// separable spatial filter split into a column pass and a row pass over bands
// of rows, as in the banded forward.
//
// With pbar = gout sigma_r / Q', qbar = -gout (out - t_c) / Q' (kernel-sum
// units), D_n = sqrt(n) a_{n-1} - H a_n and Abar_n = w * a_n:
//   c_n   = qbar a_n [n < N] + pbar sqrt(n) a_{n-1}
//   Hbar  = qbar sum_{n<N} Abar_n D_n + sum_n (w * c_n) D_n
//           + pbar sum_{m>=1} sqrt(m) Abar_m D_{m-1}
//   d in  = Hbar / sigma_r,   d sigma_r = sum (gout (out - t_c) - Hbar H) / sigma_r.
// Because qbar and pbar vary per pixel, w * c_n needs the filterings of the
// products qbar a_n and pbar a_n: w * c_n = w*(qbar a_n) [n < N]
// + sqrt(n) w*(pbar a_{n-1}).  Both products follow Algorithm 2's recursion
// (qbar and pbar do not depend on n), so
//   prep    writes the qbar and pbar planes of the image to the workspace;
//   pass V  per tile of 32 columns x 64 output rows: H and the three
//           recursions a_n, qbar a_n, pbar a_n of the region (with the W-row
//           halos) in shared memory; writes the column filterings of all
//           three for every channel (3 (N+1) planes of the band);
//   pass H  per tile of 32 rows x 64 output columns: for each channel filters
//           the three planes along the rows (W-column halos), regenerates a_n
//           and D_n at the tile's pixels and accumulates the three sums; then
//           d in and the tile's sigma_r partial (double);
//   reduce  sums the partials in a fixed order.
#include <algorithm>
#include <mutex>

#include "gpa_banded.cuh"

namespace {

using namespace bfk;

constexpr int kBVC = 32;             // pass V: columns per tile (16 column pairs)
constexpr int kBVNT = 128;           // pass V: 16 column pairs x 8 blocks of 8 output rows
constexpr int kBHT = 32, kBHW = 64;  // pass H: rows, output columns per tile
constexpr int kBHNT = 256;           // pass H: 32 rows x 8 segments of 8 columns
constexpr size_t kBwdBandCap = 2ull << 30;  // band planes, default bytes
constexpr long long kBwdBandCTAs = 8 * 152;  // pass-V CTAs per band wanted

struct BandBwdArgs {
  const float *in, *out, *qaux, *gout;
  float *gin;
  float *qb, *pb;    // qbar and pbar planes, H x Wp (workspace)
  float *ws;         // 3 (N + 1) planes of rows x Wp for the band (workspace)
  double *partials;  // one per pass-H CTA over all bands, or NULL
  long long plane;   // floats per band plane
  int Wp, H, W, pitch;
  int y0, rows, part0;
  bfi::FilterConsts fc;
};

__host__ __device__ inline int bv_rows(int kind, int R, int ntp) {
  return kind == BF_SPATIAL_GAUSS ? kVB + ntp : kVB + 2 * R;
}
__host__ __device__ inline int bh_cols(int kind, int R, int ntp) {
  return kind == BF_SPATIAL_GAUSS ? kBHW + ntp : kBHW + 2 * R;
}
size_t bv_smem(int kind, int R, int ntp) { return 4 * (size_t)bv_rows(kind, R, ntp) * kBVC * sizeof(float); }
size_t bh_smem(int kind, int R, int ntp) {
  return 3 * (size_t)kBHT * hpass_pitch(bh_cols(kind, R, ntp)) * sizeof(float);
}

__global__ void __launch_bounds__(256) band_bwd_prep(const __grid_constant__ BandBwdArgs A) {
  const bfi::FilterConsts &fc = A.fc;
  const long long n = (long long)A.H * A.Wp;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const int y = (int)(i / A.Wp), x = (int)(i - (long long)y * A.Wp);
    float qv = 0.f, pv = 0.f;
    if (x < A.W) {
      const long long o = (long long)y * A.pitch + x;
      const float g = __ldg(A.gout + o);
      // kernel-sum units: Q_u = Q' / qscale; approximate division (2 ulp)
      const float iq = __fdividef(fc.qscale, __ldg(A.qaux + o));
      qv = -(g * (__ldg(A.out + o) - fc.tc)) * iq;
      pv = g * fc.sr * iq;
    }
    A.qb[i] = qv;
    A.pb[i] = pv;
  }
}

template <int KIND>
__global__ void __launch_bounds__(kBVNT) band_bwd_vpass(const __grid_constant__ BandBwdArgs A) {
  extern __shared__ __align__(16) float sm[];
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RR = bv_rows(KIND, R, fc.ntaps_pad);
  float *sH = sm, *sA = sH + RR * kBVC, *sQ = sA + RR * kBVC, *sP = sQ + RR * kBVC;
  const int tx = blockIdx.x * kBVC;
  const int tyb = blockIdx.y * kVB;  // band-relative first output row
  const int ty = A.y0 + tyb;
  const int halo = kVB + 2 * R;      // rows of real data; the rest are zero padding
  for (int i = threadIdx.x; i < RR * kBVC; i += kBVNT) {
    const int r = i / kBVC, c = i % kBVC;
    const int gy = ty - R + r, gx = tx + c;
    float h = 0.f, a0 = 0.f, q = 0.f, p = 0.f;
    if (r < halo && gy >= 0 && gy < A.H && gx < A.W) {
      const float d = __ldg(A.in + (long long)gy * A.pitch + gx) - fc.tc;
      h = d * fc.inv_sr;
      a0 = exp2f(d * d * fc.e2c);  // exp(-H^2/2), as in the forward
      const long long k = (long long)gy * A.Wp + gx;
      q = A.qb[k] * a0;
      p = A.pb[k] * a0;
    }
    sH[i] = h;
    sA[i] = a0;
    sQ[i] = q;
    sP[i] = p;
  }
  constexpr int CS = kBVC / 2;  // row stride in column pairs
  const int cp = threadIdx.x % CS, yb = threadIdx.x / CS;  // 8 blocks of 8 output rows
  const int gx = tx + 2 * cp;
  const float2 *cA = reinterpret_cast<const float2 *>(sA + 8 * yb * kBVC) + cp;
  const float2 *cQ = reinterpret_cast<const float2 *>(sQ + 8 * yb * kBVC) + cp;
  const float2 *cP = reinterpret_cast<const float2 *>(sP + 8 * yb * kBVC) + cp;
  for (int n = 0; n <= N; ++n) {
    __syncthreads();  // region loaded / previous channel's filtering done
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
      for (int i = threadIdx.x; i < RR * kBVC / 4; i += kBVNT) {
        const float4 h = reinterpret_cast<const float4 *>(sH)[i];
        const float4 m = make_float4(h.x * rs, h.y * rs, h.z * rs, h.w * rs);
        float4 *pa = reinterpret_cast<float4 *>(sA) + i;
        float4 *pq = reinterpret_cast<float4 *>(sQ) + i;
        float4 *pp = reinterpret_cast<float4 *>(sP) + i;
        float4 v = *pa;
        *pa = make_float4(v.x * m.x, v.y * m.y, v.z * m.z, v.w * m.w);
        v = *pq;
        *pq = make_float4(v.x * m.x, v.y * m.y, v.z * m.z, v.w * m.w);
        v = *pp;
        *pp = make_float4(v.x * m.x, v.y * m.y, v.z * m.z, v.w * m.w);
      }
      __syncthreads();
    }
    float2 aA[8], aQ[8], aP[8];
    if (KIND == BF_SPATIAL_GAUSS) {
      float2 wA[8], wQ[8], wP[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        aA[i] = aQ[i] = aP[i] = make_float2(0.f, 0.f);
        wA[i] = cA[i * CS];
        wQ[i] = cQ[i * CS];
        wP[i] = cP[i * CS];
      }
      for (int k = 0; k < fc.ntaps_pad; k += 8) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float w = fc.taps[k + j];
          const float2 w2 = make_float2(w, w);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            aA[i] = __ffma2_rn(w2, wA[(j + i) & 7], aA[i]);
            aQ[i] = __ffma2_rn(w2, wQ[(j + i) & 7], aQ[i]);
            aP[i] = __ffma2_rn(w2, wP[(j + i) & 7], aP[i]);
          }
          wA[j] = cA[(k + j + 8) * CS];
          wQ[j] = cQ[(k + j + 8) * CS];
          wP[j] = cP[(k + j + 8) * CS];
        }
      }
    } else {
      float2 sa = make_float2(0.f, 0.f), sq = sa, sp = sa;
      for (int r = 0; r <= 2 * R; ++r) {
        sa = __fadd2_rn(sa, cA[r * CS]);
        sq = __fadd2_rn(sq, cQ[r * CS]);
        sp = __fadd2_rn(sp, cP[r * CS]);
      }
      aA[0] = sa;
      aQ[0] = sq;
      aP[0] = sp;
#pragma unroll
      for (int i = 1; i < 8; ++i) {
        const float2 ia = cA[(i + 2 * R) * CS], oa = cA[(i - 1) * CS];
        const float2 iqv = cQ[(i + 2 * R) * CS], oq = cQ[(i - 1) * CS];
        const float2 ipv = cP[(i + 2 * R) * CS], op = cP[(i - 1) * CS];
        sa = __fadd2_rn(sa, __fadd2_rn(ia, make_float2(-oa.x, -oa.y)));
        sq = __fadd2_rn(sq, __fadd2_rn(iqv, make_float2(-oq.x, -oq.y)));
        sp = __fadd2_rn(sp, __fadd2_rn(ipv, make_float2(-op.x, -op.y)));
        aA[i] = sa;
        aQ[i] = sq;
        aP[i] = sp;
      }
    }
    if (gx < A.Wp) {
      float *dA = A.ws + (3LL * n) * A.plane + gx;
      float *dQ = dA + A.plane;
      float *dP = dQ + A.plane;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int orow = tyb + 8 * yb + i;
        if (orow < A.rows) {
          const long long o = (long long)orow * A.Wp;
          *reinterpret_cast<float2 *>(dA + o) = aA[i];
          *reinterpret_cast<float2 *>(dQ + o) = aQ[i];
          *reinterpret_cast<float2 *>(dP + o) = aP[i];
        }
      }
    }
  }
}

// Row filtering of one plane at the thread's 8 pixels (rotating window).
template <int KIND>
__device__ __forceinline__ void bh_filter(const bfi::FilterConsts &fc, const float *v, float (&o)[8]) {
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
__global__ void __launch_bounds__(kBHNT) band_bwd_hpass(const __grid_constant__ BandBwdArgs A) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[kBHNT / 32];
  const bfi::FilterConsts &fc = A.fc;
  const int R = fc.R, N = fc.N;
  const int RC = bh_cols(KIND, R, fc.ntaps_pad), P = hpass_pitch(RC);
  const int tx = blockIdx.x * kBHW;
  const int tyb = blockIdx.y * kBHT;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;  // row lane, 8-column segment
  const int gy = A.y0 + tyb + lane;
  const bool rowin = tyb + lane < A.rows;

  float a[8], H[8], X[8], Y[8], Z[8], Dp[8], RPp[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gx = tx + 8 * seg + i;
    float h = 0.f, a0 = 0.f;
    if (rowin && gx < A.W) {
      const float d = __ldg(A.in + (long long)gy * A.pitch + gx) - fc.tc;
      h = d * fc.inv_sr;
      a0 = exp2f(d * d * fc.e2c);
    }
    a[i] = a0;
    H[i] = h;
    X[i] = Y[i] = Z[i] = Dp[i] = RPp[i] = 0.f;
  }

  // the region's in-image columns are j in [j0, j1) of every row; the cells
  // outside the image or the band are zeroed once here (no copy writes them)
  const int j0 = max(0, R - tx), j1 = min(RC, A.W - tx + R);
  for (int pl = 0; pl < 3; ++pl)
    for (int r = seg; r < kBHT; r += kBHNT / 32) {
      const bool rin = tyb + r < A.rows;
      for (int j = lane; j < RC; j += 32)
        if (!rin || j < j0 || j >= j1) sm[pl * kBHT * P + r * P + j] = 0.f;
    }
  for (int n = 0; n <= N; ++n) {
    // the channel's three column-filtered planes, rows tyb.., columns tx - W..
    // (column j of the region is image column tx - W + j)
    for (int pl = 0; pl < 3; ++pl) {
      const float *src = A.ws + (3LL * n + pl) * A.plane + (long long)tyb * A.Wp + (tx - R);
      float *b = sm + pl * kBHT * P;
      for (int r = seg; r < kBHT && tyb + r < A.rows; r += kBHNT / 32) {
        const float *srow = src + (long long)r * A.Wp;
        float *drow = b + r * P;
        for (int j = j0 + lane; j < j1; j += 32) cp_async4(drow + j, srow + j);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    float RA[8], RQ[8], RP[8];
    const int off = lane * P + 8 * seg;
    bh_filter<KIND>(fc, sm + off, RA);
    bh_filter<KIND>(fc, sm + kBHT * P + off, RQ);
    bh_filter<KIND>(fc, sm + 2 * kBHT * P + off, RP);
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float aold = a[i];
      const float an = n > 0 ? aold * (H[i] * rs) : aold;
      const float D = fmaf(sq, aold, -H[i] * an);  // d a_n / dH
      const float Cb = (n < N ? RQ[i] : 0.f) + sq * RPp[i];
      if (n < N) X[i] = fmaf(RA[i], D, X[i]);
      Y[i] = fmaf(Cb, D, Y[i]);
      if (n > 0) Z[i] = fmaf(RA[i] * sq, Dp[i], Z[i]);
      Dp[i] = D;
      RPp[i] = RP[i];
      a[i] = an;
    }
    __syncthreads();  // the planes' buffers are refilled for the next channel
  }

  double part = 0.0;
  if (rowin) {
    float pf = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gx = tx + 8 * seg + i;
      if (gx < A.W) {
        const long long k = (long long)gy * A.Wp + gx, o = (long long)gy * A.pitch + gx;
        const float hbar = fmaf(A.qb[k], X[i], fmaf(A.pb[k], Z[i], Y[i]));
        A.gin[o] = hbar * fc.inv_sr;
        if (A.partials)
          pf += fmaf(__ldg(A.gout + o), __ldg(A.out + o) - fc.tc, -hbar * H[i]);
      }
    }
    part = (double)pf * (double)fc.inv_sr;
  }
  if (A.partials) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if (lane == 0) red[seg] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kBHNT / 32; ++w) t += red[w];
      A.partials[A.part0 + blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Fixed-order sum of the partials (one CTA, deterministic).
__global__ void __launch_bounds__(256) band_bwd_reduce(const double *p, int n, double *out) {
  __shared__ double red[8];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) v += p[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *out = t;
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
int round_up4(int w) { return (w + 3) / 4 * 4; }

struct BwdLayout {
  size_t off_qb, off_pb, off_part, off_planes, total;
  int rows;
};

BwdLayout layout(int height, int width, int N, size_t ws_bytes) {
  BwdLayout L{};
  const int Wp = round_up4(width);
  const size_t plane_img = align256((size_t)height * Wp * sizeof(float));
  const size_t nparts = (size_t)((width + kBHW - 1) / kBHW) * ((height + kBHT - 1) / kBHT);
  L.off_qb = 0;
  L.off_pb = plane_img;
  L.off_part = 2 * plane_img;
  L.off_planes = align256(L.off_part + nparts * sizeof(double));
  const size_t row_bytes = 3 * (size_t)(N + 1) * Wp * sizeof(float);
  const int cap = (height + kVB - 1) / kVB * kVB;
  if (ws_bytes == 0) {  // preferred: several waves of pass-V CTAs, within the cap
    const long long col_tiles = (Wp + kBVC - 1) / kBVC;
    long long rows = (kBwdBandCTAs + col_tiles - 1) / col_tiles * kVB;
    rows = std::min<long long>(rows, cap);
    const long long fit = (long long)(kBwdBandCap / row_bytes) / kVB * kVB;
    if (fit >= kVB) rows = std::min(rows, fit);
    L.rows = (int)std::max<long long>(rows, kVB);
  } else {
    const size_t avail = ws_bytes > L.off_planes ? ws_bytes - L.off_planes : 0;
    const size_t fit = avail / row_bytes / kVB * kVB;
    L.rows = (int)std::min<size_t>(fit, (size_t)cap);
  }
  L.total = L.off_planes + row_bytes * (size_t)L.rows;
  return L;
}

template <int KIND>
bf_status run_banded_bwd(BandBwdArgs &A, const BwdLayout &L, double *gsigma, cudaStream_t s) {
  const int ntp_max = (2 * BF_MAX_RADIUS + 1 + 15) / 16 * 16;
  bf_status est = bfi::ensure_smem(reinterpret_cast<const void *>(band_bwd_vpass<KIND>),
                                   bv_smem(KIND, BF_MAX_RADIUS, ntp_max));
  if (est == BF_OK)
    est = bfi::ensure_smem(reinterpret_cast<const void *>(band_bwd_hpass<KIND>),
                           bh_smem(KIND, BF_MAX_RADIUS, ntp_max));
  if (est != BF_OK) return est;
  const int R = A.fc.R, ntp = A.fc.ntaps_pad;
  const size_t vs = bv_smem(KIND, R, ntp), hs = bh_smem(KIND, R, ntp);
  const long long n = (long long)A.H * A.Wp;
  const int pgrid = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
  band_bwd_prep<<<pgrid, 256, 0, s>>>(A);
  bf_status st = bfi::check_launch();
  if (st != BF_OK) return st;
  const int band = L.rows;
  int part0 = 0;
  for (int y0 = 0; y0 < A.H; y0 += band) {
    A.y0 = y0;
    A.rows = std::min(band, A.H - y0);
    A.part0 = part0;
    dim3 gv((A.Wp + kBVC - 1) / kBVC, (A.rows + kVB - 1) / kVB);
    band_bwd_vpass<KIND><<<gv, kBVNT, vs, s>>>(A);
    st = bfi::check_launch();
    if (st != BF_OK) return st;
    dim3 gh((A.W + kBHW - 1) / kBHW, (A.rows + kBHT - 1) / kBHT);
    band_bwd_hpass<KIND><<<gh, kBHNT, hs, s>>>(A);
    st = bfi::check_launch();
    if (st != BF_OK) return st;
    part0 += (int)(gh.x * gh.y);
  }
  if (!gsigma) return BF_OK;
  band_bwd_reduce<<<1, 256, 0, s>>>(A.partials, part0, gsigma);
  return bfi::check_launch();
}

}  // namespace

namespace bfi {

bool banded_backward_fits(const FilterConsts &fc) { return fc.R > 15; }

size_t banded_backward_bytes(int height, int width, const FilterConsts &fc) {
  return layout(height, width, fc.N, 0).total;
}

bf_status banded_backward(const float *in, const float *out, const float *qaux, const float *gout,
                          float *gin, double *gsigma, int height, int width, int pitch,
                          const FilterConsts &fc, void *ws, size_t ws_bytes, void *stream) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return BF_ERR_WORKSPACE;
  const BwdLayout L = layout(height, width, fc.N, ws_bytes);
  if (L.rows < kVB) return BF_ERR_WORKSPACE;
  char *base = static_cast<char *>(ws);
  BandBwdArgs A;
  A.in = in;
  A.out = out;
  A.qaux = qaux;
  A.gout = gout;
  A.gin = gin;
  A.qb = reinterpret_cast<float *>(base + L.off_qb);
  A.pb = reinterpret_cast<float *>(base + L.off_pb);
  A.partials = gsigma ? reinterpret_cast<double *>(base + L.off_part) : nullptr;
  A.ws = reinterpret_cast<float *>(base + L.off_planes);
  A.Wp = round_up4(width);
  A.plane = (long long)L.rows * A.Wp;
  A.H = height;
  A.W = width;
  A.pitch = pitch;
  A.y0 = 0;
  A.rows = L.rows;
  A.part0 = 0;
  A.fc = fc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return fc.kind == BF_SPATIAL_GAUSS ? run_banded_bwd<BF_SPATIAL_GAUSS>(A, L, gsigma, s)
                                     : run_banded_bwd<BF_SPATIAL_BOX>(A, L, gsigma, s);
}

}  // namespace bfi
