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
//   vol_zpass   one thread per (y, x) column (two adjacent columns as packed
//               pairs for W <= 8) and 16 output planes z0..z0+15:
//               the column's f over the tile plus the W-plane halos is turned
//               into a_0 and H in shared memory (each thread its own column,
//               so no barriers), then channel by channel a_n is advanced in
//               place and filtered along z into the workspace plane Z_n
//               (N + 1 volumes of floats);
//   vol_yxpass  one CTA per output tile of one z-plane: per channel the Z_n
//               region with the W-pixel halos is staged in shared memory (the
//               next channel's region copied while the current one is
//               filtered), filtered along y, then along x, and the result
//               (w * a_n at the tile's voxels) is recombined with a_n at the
//               voxel itself (regenerated from f in registers) into Q', P'.
//               For W <= 8 (vol_yxpass_tma) the region arrives by one tiled
//               tensor copy per channel and the filters run as packed
//               two-lane FP32 pairs; larger radii copy per thread.
#include <cuda.h>  // CUtensorMap and its enums (types only; no driver library link)

#include <algorithm>
#include <cmath>
#include <mutex>

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
  int *status;      // the workspace's status word (BF_OK, or BF_ERR_TIMEOUT)
  long long plane;  // D * H * Wp: floats per workspace volume
  int D, H, W, Wp, R, L, N;  // Wp: workspace row pitch, W rounded up to a multiple of 4
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
  const long long wcol = (long long)y * A.Wp + x, wzs = (long long)A.H * A.Wp;
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
    float *dst = A.ws + (long long)n * A.plane + z0 * wzs + wcol;
    for (int zo = 0; zo < zn; ++zo) {
      float acc = 0.f;
      for (int k = 0; k < A.L; ++k) acc = fmaf(A.taps[k], sA[(zo + k) * kZNT + t], acc);
      dst[zo * wzs] = acc;
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
  const long long wzoff = z * (long long)A.H * A.Wp;
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
    const float *src = A.ws + (long long)n * A.plane + wzoff;
    for (int e = t; e < RC * RC; e += kYNT) {
      const int rr = e / RC, cc = e - rr * RC;
      const int gy = y0 - A.R + rr, gx = x0 - A.R + cc;
      if (gy >= 0 && gy < A.H && gx >= 0 && gx < A.W)
        bfk::cp_async4(b + rr * RP + cc, src + (long long)gy * A.Wp + gx);
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

// ---------------------------------------------------------------------------
// y/x pass for W <= 8 with TMA staging.  One CTA of 256 threads per 64 x 48
// output tile of one z-plane.  Per channel n the tile's Z_n region (rows
// y0 - W .. y0 + 63 + W, columns x0 - 8 .. x0 + 55) arrives by one tiled
// tensor copy (cp.async.bulk.tensor, zero fill outside the plane) into one of
// two shared buffers, the next channel's copy in flight while the current one
// is filtered; an mbarrier per buffer signals its completion.
//   y filter: thread (column pair 2p, 2p + 1; rows 8c .. 8c + 7) over the
//             region's 64 columns, the column pair as one packed two-lane
//             FP32 filtering (both columns take the same taps);
//   x filter: thread (row, 12 consecutive output columns), output pairs
//             (j, j + 1) as one packed filtering with the tap pairs
//             (w[k], w[k - 1]); then the recursion a_n and the sums Q', P' of
//             the thread's 12 voxels in registers, as packed pairs.
// Every wait on an mbarrier is bounded: past about a second the CTA records
// BF_ERR_TIMEOUT in the status word, drains its copies (bounded too) and
// returns.
constexpr int kTY = 64, kTX = 48, kTC = 64, kTNT = 256;  // tile rows, columns, region columns

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase `parity` of an mbarrier (about 1 s at 2 GHz).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (2ll << 30)) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map,
                                            unsigned long long *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

struct VolTapPairs {
  float2 dup[2 * kVolFixedMaxR + 1];   // (w[k], w[k]): the y filter's column pairs
  float2 pair[2 * kVolFixedMaxR + 2];  // (w[k], w[k - 1]), w[-1] = w[L] = 0: the x filter's output pairs
};

template <int R>
__global__ void __launch_bounds__(kTNT, 3) vol_yxpass_tma(const __grid_constant__ VolArgs A,
                                                       const __grid_constant__ VolTapPairs T,
                                                       const __grid_constant__ CUtensorMap map) {
  constexpr int L = 2 * R + 1, RR = kTY + 2 * R;  // region rows
  constexpr int VP = kTC + 2;                     // sV row pitch (floats): rows 33 float2 apart
  constexpr unsigned kBytes = RR * kTC * sizeof(float);
  extern __shared__ __align__(1024) float sm[];  // the only shared memory: buffers first
  float *buf0 = sm, *buf1 = sm + RR * kTC, *sV = sm + 2 * RR * kTC;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(sV + kTY * VP);
  const int t = threadIdx.x;
  if (smem_u32(sm) & 127u) {  // a tensor copy needs a 128-byte aligned destination
    if (t == 0) atomicExch(A.status, (int)BF_ERR_INVALID_ARG);
    return;
  }
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z = blockIdx.z;
  const long long zin = (long long)A.H * A.W;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int n) {  // thread 0: channel n's region into buffer n & 1
    unsigned long long *b = &bar[n & 1];
    mbar_expect_tx(b, kBytes);
    tma_load_3d((n & 1) ? buf1 : buf0, &map, b, x0 - 8, y0 - R, n * A.D + z);
  };
  if (t == 0) issue(0);

  // the thread's voxels: row xr, output columns 12 xs .. 12 xs + 11 (six pairs)
  const int xr = t & 63, xs = t >> 6;
  const int gy = y0 + xr;
  float2 a2[6], h2[6], q2[6], p2[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float av[2] = {0.f, 0.f}, hv[2] = {0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int gx = x0 + 12 * xs + 2 * k + e;
      if (gx < A.W && gy < A.H) {
        const float d = __ldg(A.in + z * zin + (long long)gy * A.W + gx) - A.tc;
        hv[e] = d * A.inv_sr;
        av[e] = exp2f(d * d * A.e2c);  // exp(-H^2/2)
      }
    }
    a2[k] = make_float2(av[0], av[1]);
    h2[k] = make_float2(hv[0], hv[1]);
    q2[k] = p2[k] = make_float2(0.f, 0.f);
  }
  const int yp = t & 31, yc = t >> 5;  // y filter: columns 2 yp, 2 yp + 1; rows 8 yc .. 8 yc + 7
  bool bad = false;
  int issued = 0;  // thread 0: the last channel whose copy was issued
  for (int n = 0; n <= A.N; ++n) {
    // the other buffer was last read by the y filter of channel n - 1, finished
    // before the barrier that ended it; sV was last read by the x filter of n - 1
    __syncthreads();
    if (t == 0 && n + 1 <= A.N) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(n + 1);
      issued = n + 1;
    }
    const bool ok = mbar_wait(&bar[n & 1], (n >> 1) & 1);
    const float *sR = (n & 1) ? buf1 : buf0;
    {
      float2 w[8 + 2 * R];
#pragma unroll
      for (int i = 0; i < 8 + 2 * R; ++i)
        w[i] = *reinterpret_cast<const float2 *>(sR + (8 * yc + i) * kTC + 2 * yp);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < L; ++k) acc = __ffma2_rn(T.dup[k], w[r + k], acc);
        *reinterpret_cast<float2 *>(sV + (8 * yc + r) * VP + 2 * yp) = acc;
      }
    }
    if (__syncthreads_or(!ok)) {  // every thread leaves the loop together
      bad = true;
      break;
    }
    // x filter: output column j of the tile is region column j + 8
    constexpr int X0 = 8 - R - (R & 1);  // first (even) region column the window needs, less 12 xs
    constexpr int OFF = R & 1;           // window index of output column 12 xs's first tap
    constexpr int NW = (12 + 2 * R + OFF + 1) / 2 * 2;
    float v[NW];
#pragma unroll
    for (int i = 0; i < NW; i += 2) {
      const float2 e = *reinterpret_cast<const float2 *>(sV + xr * VP + 12 * xs + X0 + i);
      v[i] = e.x;
      v[i + 1] = e.y;
    }
    const float rs = n > 0 ? __frsqrt_rn((float)n) : 0.f;
    const float sq = __fsqrt_rn((float)n);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      // outputs (2k, 2k + 1): sum over window values e of (w[e - 2k], w[e - 2k - 1]) v_e
      float2 ab = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j <= L; ++j) {
        const float ve = v[OFF + 2 * k + j];
        ab = __ffma2_rn(T.pair[j], make_float2(ve, ve), ab);
      }
      const float2 aold = a2[k];  // a_{n-1}
      const float2 an = n > 0 ? __fmul2_rn(aold, __fmul2_rn(h2[k], make_float2(rs, rs))) : aold;
      if (n < A.N) q2[k] = __ffma2_rn(an, ab, q2[k]);
      if (n > 0) p2[k] = __ffma2_rn(__fmul2_rn(aold, make_float2(sq, sq)), ab, p2[k]);
      a2[k] = an;
    }
  }
  if (bad) {  // a copy did not arrive: record it, let the copies in flight land, leave
    if (t == 0) {
      atomicExch(A.status, (int)BF_ERR_TIMEOUT);
      for (int b = 0; b < 2; ++b) {  // each buffer's last issued phase
        const int last = issued - ((issued - b) & 1);
        if (last >= 0) mbar_wait(&bar[b], (last >> 1) & 1);
      }
    }
    return;
  }
  if (gy >= A.H) return;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float pk[2] = {p2[k].x, p2[k].y}, qk[2] = {q2[k].x, q2[k].y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int gx = x0 + 12 * xs + 2 * k + e;
      if (gx < A.W) {
        const long long o = z * zin + (long long)gy * A.W + gx;
        A.out[o] = fmaf(A.sr, __fdividef(pk[e], qk[e]), A.tc);  // approximate division (2 ulp)
        if (A.qaux) A.qaux[o] = qk[e];
      }
    }
  }
}

// z-pass for W <= 8: each thread owns two adjacent (y, x) columns and 16
// output planes; the two columns' a_n over the planes and their W-plane halos
// are packed pairs in registers (both columns take the same taps, so each tap
// is one two-lane FMA), H of the pairs in shared memory (each thread reads only
// its own), and Z_n = w1 *_z a_n is stored as pairs (the workspace rows hold a
// multiple of 4 floats, so a pair starting at an even column never leaves them).
template <int R>
__global__ void __launch_bounds__(kZNT) vol_zpass_pairs(const __grid_constant__ VolArgs A,
                                                        const __grid_constant__ VolTapPairs T) {
  constexpr int L = 2 * R + 1, RZ = kZT + 2 * R;
  extern __shared__ __align__(16) float2 sH2[];  // [r][thread]
  const int t = threadIdx.x;
  const int x = 2 * (blockIdx.x * kZNT + t), y = blockIdx.y, z0 = blockIdx.z * kZT;
  if (x >= A.W) return;  // no barriers: every thread owns its columns
  const bool x1in = x + 1 < A.W;
  const long long col = (long long)y * A.W + x, zs = (long long)A.H * A.W;
  const long long wcol = (long long)y * A.Wp + x, wzs = (long long)A.H * A.Wp;
  float2 a[RZ];
#pragma unroll
  for (int r = 0; r < RZ; ++r) {
    const int z = z0 - R + r;
    float av[2] = {0.f, 0.f}, hv[2] = {0.f, 0.f};
    if (z >= 0 && z < A.D) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (e == 1 && !x1in) break;
        const float d = __ldg(A.in + z * zs + col + e) - A.tc;
        hv[e] = d * A.inv_sr;
        av[e] = exp2f(d * d * A.e2c);  // exp(-H^2/2)
      }
    }
    a[r] = make_float2(av[0], av[1]);
    sH2[r * kZNT + t] = make_float2(hv[0], hv[1]);
  }
  const int zn = min(kZT, A.D - z0);
  for (int n = 0; n <= A.N; ++n) {
    if (n > 0) {
      const float rs = __frsqrt_rn((float)n);
#pragma unroll
      for (int r = 0; r < RZ; ++r) a[r] = __fmul2_rn(a[r], __fmul2_rn(sH2[r * kZNT + t], make_float2(rs, rs)));
    }
    float *dst = A.ws + (long long)n * A.plane + z0 * wzs + wcol;
#pragma unroll
    for (int zo = 0; zo < kZT; ++zo) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < L; ++k) acc = __ffma2_rn(T.dup[k], a[zo + k], acc);
      if (zo < zn) *reinterpret_cast<float2 *>(dst + zo * wzs) = acc;
    }
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); looked up once.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// The workspace planes as a 3-D tensor (x, y, n D + z) with row pitch Wp; the
// box is one y/x-pass region of one plane.  Coordinates outside (W, H) read 0.
bf_status volume_tensor_map(const VolArgs &A, int R, CUtensorMap *map) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    bfi::set_error_text("cuTensorMapEncodeTiled is not available from the CUDA driver");
    return BF_ERR_CUDA;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)A.W, (cuuint64_t)A.H,
                              (cuuint64_t)A.D * (cuuint64_t)(A.N + 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)A.Wp * sizeof(float),
                                 (cuuint64_t)A.H * (cuuint64_t)A.Wp * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kTC, (cuuint32_t)(kTY + 2 * R), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, A.ws, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    bfi::set_error_text("cuTensorMapEncodeTiled rejected the volume workspace layout");
    return BF_ERR_CUDA;
  }
  return BF_OK;
}

template <int R>
bf_status launch_volume_r(const VolArgs &A, cudaStream_t s) {
  constexpr size_t ys = ((size_t)2 * (kTY + 2 * R) * kTC + (size_t)kTY * (kTC + 2)) * sizeof(float) +
                        2 * sizeof(unsigned long long);  // two buffers, sV, two mbarriers
  bf_status st = bfi::ensure_smem(reinterpret_cast<const void *>(vol_yxpass_tma<R>), ys);
  if (st != BF_OK) return st;
  CUtensorMap map;
  st = volume_tensor_map(A, R, &map);
  if (st != BF_OK) return st;
  VolTapPairs T;
  constexpr int L = 2 * R + 1;
  for (int k = 0; k < 2 * kVolFixedMaxR + 1; ++k) T.dup[k] = k < L ? make_float2(A.taps[k], A.taps[k]) : make_float2(0.f, 0.f);
  for (int k = 0; k < 2 * kVolFixedMaxR + 2; ++k)
    T.pair[k] = make_float2(k < L ? A.taps[k] : 0.f, k >= 1 && k <= L ? A.taps[k - 1] : 0.f);
  constexpr size_t zsm = (size_t)(kZT + 2 * R) * kZNT * sizeof(float2);
  dim3 gz((A.W + 2 * kZNT - 1) / (2 * kZNT), A.H, (A.D + kZT - 1) / kZT);
  vol_zpass_pairs<R><<<gz, kZNT, zsm, s>>>(A, T);
  st = bfi::check_launch();
  if (st != BF_OK) return st;
  dim3 gy((A.W + kTX - 1) / kTX, (A.H + kTY - 1) / kTY, A.D);
  vol_yxpass_tma<R><<<gy, kTNT, ys, s>>>(A, T, map);
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

// Workspace: a 256-byte header (the status word) and the N + 1 planes of
// depth x height x Wp floats (Wp = width rounded up to a multiple of 4, the
// 16-byte row pitch a tensor copy needs).
constexpr size_t kVolHeader = 256;
int round_up4(int w) { return (w + 3) / 4 * 4; }
size_t volume_ws_bytes(int depth, int height, int width, int N) {
  return kVolHeader + (size_t)(N + 1) * (size_t)depth * (size_t)height *
                          (size_t)round_up4(width) * sizeof(float);
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
  *bytes = volume_ws_bytes(depth, height, width, fc.N);
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
  const size_t need = volume_ws_bytes(depth, height, width, fc.N);
  if (!d_ws || ws_bytes < need) return BF_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(d_ws) & 15u) != 0) return BF_ERR_INVALID_ARG;
  if ((long long)depth * (fc.N + 1) > 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
  VolArgs A = {};
  A.in = d_in;
  A.out = d_out;
  A.qaux = d_qaux;
  A.status = static_cast<int *>(d_ws);
  A.ws = reinterpret_cast<float *>(static_cast<char *>(d_ws) + kVolHeader);
  A.Wp = round_up4(width);
  A.plane = (long long)depth * height * A.Wp;
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
  const cudaError_t me = cudaMemsetAsync(A.status, 0, sizeof(int), s);
  if (me != cudaSuccess) return bfi::cuda_status(me);
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
