// Fused forward of the Gaussian-polynomial bilateral filter (Algorithm 2):
// kernels, tile-variant dispatch and the tile autotuner.
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "bf_internal.h"
#include "box_warp.cuh"
#include "gpa_banded.cuh"
#include "gpa_fixed.cuh"
#include "gpa_tile.cuh"

namespace {

struct FwdArgs {
  bfk::TileIO io;
  bfi::FilterConsts fc;
  float2 tap2[bfk::kTap2];  // compile-time-radius Gaussian: (w[k], w[k - 1]) pairs
  int count = 1;            // images (same size and parameters), image_stride apart
  long long image_stride = 0;
};

template <int KIND, int NT, int TH, bool STORE>
__global__ void __launch_bounds__(NT) gpa_fwd_kernel(const __grid_constant__ FwdArgs args) {
  extern __shared__ __align__(16) float smem[];
  const int TW = NT - 2 * args.fc.R;
  bfk::gpa_fwd_tile<KIND, NT, TH, TH, STORE>(args.io, args.fc, args.fc.taps, blockIdx.y * TH,
                                             blockIdx.x * TW, smem);
}

// Compile-time-radius kernel (gpa_fixed.cuh): persistent, 256 threads,
// 16-row tiles, double-buffered region copies.
template <int KIND, int R, bool STORE>
__global__ void __launch_bounds__(256, 2) gpa_fwd_fixed_kernel(const __grid_constant__ FwdArgs args) {
  extern __shared__ __align__(16) float smem[];
  bfk::gpa_fwd_fixed_persistent<KIND, R, 256, 16, STORE>(args.io, args.fc, args.tap2, smem);
}

// The same without stored planes: alternating pairs of phase rows, one
// barrier per channel.
template <int KIND, int R, bool STORE = false>
__global__ void __launch_bounds__(256, 2) gpa_fwd_fixed_db_kernel(const __grid_constant__ FwdArgs args) {
  extern __shared__ __align__(16) float smem[];
  bfk::gpa_fwd_fixed_persistent_db<KIND, R, 256, 16, STORE>(args.io, args.fc, args.tap2, smem);
}

// Warp-strip box kernel for small N (box_warp.cuh): one warp per strip of
// output columns (C columns per lane) and band of rows, one warp per CTA.
constexpr int kWarpWPB = 1;
template <int R, int NN, int C>
__global__ void __launch_bounds__(32 * kWarpWPB, 8) box_warp_kernel(const __grid_constant__ bfk::WarpStripArgs A) {
  extern __shared__ __align__(16) float smem[];
  using G = bfk::WarpStripGeom<R, 1, C>;
  const int w = threadIdx.x >> 5;
  const int wid = blockIdx.x * kWarpWPB + w;
  const int strip = wid % A.nstrips, rest = wid / A.nstrips;
  const int band = rest % A.nbands, img = rest / A.nbands;
  if (img >= A.nimg) return;
  bfk::box_warp_strip<R, NN, 1, C>(A, strip, band, (long long)img * A.img_stride,
                                   smem + w * G::warp_floats);
}

// Tile variants 0..4: runtime-radius kernel, (threads per CTA = region
// columns, output rows per tile).  Variant 5: the compile-time-radius kernel
// for the radii in kFixedRadii (with or without stored planes).
// Variants 6 and 7: the warp-strip streaming box kernel (box, W in {3, 5})
// with 8 columns per lane (N <= 5) and 4 columns per lane (N <= 8; fewer
// registers per channel).  Variant 8: the two-pass banded forward
// (gpa_banded.cu), which needs a caller workspace: only the entry points
// that take one run it.
struct Variant {
  int NT, TH;
};
constexpr Variant kVariants[] = {{256, 16}, {512, 8}, {256, 8}, {128, 16}, {192, 8}};
constexpr int kNumGeneric = sizeof(kVariants) / sizeof(kVariants[0]);
constexpr int kFixedVariant = kNumGeneric;
constexpr int kStreamVariant = kNumGeneric + 1;
constexpr int kStream4Variant = kNumGeneric + 2;
constexpr int kBandedVariant = kNumGeneric + 3;
constexpr int kNumVariants = kNumGeneric + 4;
static_assert(kBandedVariant == bfi::kFwdBandedVariant && kNumVariants == bfi::kFwdNumVariants,
              "variant numbering shared with the banded forward and the batch plan");

bool fixed_radius(int R) { return R == 3 || R == 5 || R == 9 || R == 15; }
bool stream_fits(const bfi::FilterConsts &fc, int max_n) {
  return fc.kind == BF_SPATIAL_BOX && (fc.R == 3 || fc.R == 5) && fc.N >= 1 && fc.N <= max_n;
}

int max_smem_optin() {
  static int v = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      v = 232448;
    cudaGetLastError();
  });
  return v;
}

bool variant_fits(int v, const bfi::FilterConsts &fc, bool store = false) {
  if (v == kBandedVariant) return !store;
  if (v == kFixedVariant) return fixed_radius(fc.R);
  if (v == kStreamVariant) return !store && stream_fits(fc, 5);
  if (v == kStream4Variant) return !store && stream_fits(fc, 8);
  const Variant &var = kVariants[v];
  const int TW = var.NT - 2 * fc.R;
  if (TW < var.TH) return false;
  return bfk::fwd_smem_bytes(var.NT, var.TH, fc.R, fc.ntaps_pad) <= (size_t)max_smem_optin();
}

// Measured at 2048^2, 4096^2 and 8192^2: 4 columns per lane is faster for
// W = 3 at every N <= 5 and for W = 5 at N <= 3; at W = 5, N in {4, 5} the
// extra halo shuffles and halo lanes of 4 columns per lane cost more than
// the added resident warps gain.  N in 6..8 runs with 4 columns per lane only.
int default_variant(const bfi::FilterConsts &fc, bool store) {
  if (!store && stream_fits(fc, 5)) return fc.R == 3 || fc.N <= 3 ? kStream4Variant : kStreamVariant;
  if (!store && stream_fits(fc, 8)) return kStream4Variant;
  static const int order[] = {kFixedVariant, 0, 2, 4, 3, 1};
  for (int v : order)
    if (variant_fits(v, fc, store)) return v;
  return -1;
}

template <int KIND, int R, bool STORE>
bf_status launch_fixed_r(const FwdArgs &args, cudaStream_t s) {
  using G = bfk::FixedGeom<R, 256, 16>;
  using D = bfk::FixedDbGeom<R, 256, 16>;
  // stored planes: the next tile's region in flight where two CTAs fit, else
  // (W = 15) the single-buffer layout
  constexpr bool PF = STORE && D::STORE_PREFETCH;
  const size_t smem = PF ? G::smem_bytes(args.fc.N) : D::smem_bytes(args.fc.N, STORE);
  void (*kern)(const FwdArgs);
  if constexpr (PF) kern = gpa_fwd_fixed_kernel<KIND, R, true>;
  else kern = gpa_fwd_fixed_db_kernel<KIND, R, STORE>;
  const void *fn = reinterpret_cast<const void *>(kern);
  bf_status st = bfi::ensure_smem(fn, PF ? G::smem_bytes(BF_MAX_ORDER)
                                        : D::smem_bytes(BF_MAX_ORDER, STORE));
  int resident = 0;  // resident CTAs (SMs x CTAs per SM) at this shared-memory size
  if (st == BF_OK) st = bfi::resident_ctas(fn, 256, smem, &resident);
  if (st != BF_OK) return st;
  if (resident < 1) return BF_ERR_UNSUPPORTED;
  const long long tiles = (long long)((args.io.W + G::TW - 1) / G::TW) * ((args.io.H + 15) / 16);
  if (tiles > 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
  const int grid = (int)std::min<long long>(tiles, resident);
  FwdArgs a = args;
  constexpr int L = 2 * R + 1;
  for (int k = 0; k < bfk::kTap2; ++k)
    a.tap2[k] = make_float2(k < L ? args.fc.taps[k] : 0.f, k >= 1 && k <= L ? args.fc.taps[k - 1] : 0.f);
  kern<<<grid, 256, smem, s>>>(a);
  return bfi::check_launch();
}

// Rows per warp band (even, 16..64).  The 2W warm-up rows of a band are read
// and entered but produce no output.  Measured at 4096^2 (W in {3, 5},
// N in {1, 3}): with 8 columns per lane (14-16 resident warps per SM) about
// one wave of warps, or half a wave for N <= 2, is fastest; with 4 columns
// per lane (20-28 resident warps per SM) short bands filling two or more
// waves are fastest, the warm-up rows being mostly L2 hits.  A batch of
// images counts the rows of all of them (longer bands, fewer warm-up rows).
template <int R, int NN, int C>
bf_status launch_warp_rn(const FwdArgs &a, cudaStream_t s) {
  using G = bfk::WarpStripGeom<R, 1, C>;
  constexpr size_t smem = kWarpWPB * G::warp_floats * sizeof(float);
  auto kern = box_warp_kernel<R, NN, C>;
  const void *fn = reinterpret_cast<const void *>(kern);
  bf_status st = bfi::ensure_smem(fn, smem);
  int resident_ctas = 0;
  if (st == BF_OK) st = bfi::resident_ctas(fn, 32 * kWarpWPB, smem, &resident_ctas);
  if (st != BF_OK) return st;
  const int resident_warps = resident_ctas * kWarpWPB;
  if (resident_warps < 1) return BF_ERR_UNSUPPORTED;
  bfk::WarpStripArgs A;
  A.io = a.io;
  const double sr = a.fc.sr, tc = a.fc.tc;
  const double kg = sqrt(1.4426950408889634 / 2.0) / sr;
  A.tc = a.fc.tc;
  A.sr = a.fc.sr;
  A.kg = (float)kg;
  A.kg0 = (float)(-tc * kg);
  A.hs = (float)(1.0 / sr);
  A.hs0 = (float)(-tc / sr);
  A.qscale = a.fc.qscale;
  A.sentinel = (float)(tc + 1e4 * sr);
  for (int n = 0; n < 12; ++n) A.inv_n[n] = n > 0 ? (float)(1.0 / n) : 0.f;
  const bool in_al = (reinterpret_cast<uintptr_t>(a.io.in) & 15u) == 0;
  const bool out_al = (reinterpret_cast<uintptr_t>(a.io.out) & 15u) == 0;
  const bool q_al = !a.io.qaux || (reinterpret_cast<uintptr_t>(a.io.qaux) & 15u) == 0;
  const bool st_al = a.count == 1 || a.image_stride % 4 == 0;  // every image's rows 16-byte aligned
  A.vec_in = (in_al && st_al && a.io.pitch % 4 == 0) ? 1 : 0;
  A.vec_out = (out_al && q_al && st_al && a.io.pitch % 4 == 0) ? 1 : 0;
  A.nimg = a.count;
  A.img_stride = a.image_stride;
  A.nstrips = (a.io.W + G::TW - 1) / G::TW;
  const long long per_strip = std::max(1, resident_warps / A.nstrips);
  const long long all_rows = (long long)a.io.H * a.count;
  const long long one_wave = (all_rows + per_strip - 1) / per_strip;  // band rows for one wave
  const long long rows = C == 4 ? (one_wave + 1) / 2 : (NN <= 3 ? 2 : 1) * one_wave;
  const int band = (int)std::min<long long>(64, std::max<long long>(16, rows));
  A.band = (band + 1) & ~1;
  A.nbands = (a.io.H + A.band - 1) / A.band;
  const long long warps = (long long)A.nstrips * A.nbands * A.nimg;
  const long long ctas = (warps + kWarpWPB - 1) / kWarpWPB;
  if (ctas > 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
  kern<<<(int)ctas, 32 * kWarpWPB, smem, s>>>(A);
  return bfi::check_launch();
}

template <int R, int C>
bf_status launch_warp_r(const FwdArgs &a, cudaStream_t s) {
  switch (a.fc.N + 1) {
    case 2: return launch_warp_rn<R, 2, C>(a, s);
    case 3: return launch_warp_rn<R, 3, C>(a, s);
    case 4: return launch_warp_rn<R, 4, C>(a, s);
    case 5: return launch_warp_rn<R, 5, C>(a, s);
    case 6: return launch_warp_rn<R, 6, C>(a, s);
    default: break;
  }
  if constexpr (C == 4) {
    switch (a.fc.N + 1) {
      case 7: return launch_warp_rn<R, 7, C>(a, s);
      case 8: return launch_warp_rn<R, 8, C>(a, s);
      case 9: return launch_warp_rn<R, 9, C>(a, s);
      default: break;
    }
  }
  return BF_ERR_UNSUPPORTED;
}

template <int C>
bf_status launch_warp(const FwdArgs &a, cudaStream_t s) {
  if (a.fc.R == 3) return launch_warp_r<3, C>(a, s);
  if (a.fc.R == 5) return launch_warp_r<5, C>(a, s);
  return BF_ERR_UNSUPPORTED;
}

template <int KIND, bool STORE>
bf_status launch_fixed(const FwdArgs &a, cudaStream_t s) {
  switch (a.fc.R) {
    case 3: return launch_fixed_r<KIND, 3, STORE>(a, s);
    case 5: return launch_fixed_r<KIND, 5, STORE>(a, s);
    case 9: return launch_fixed_r<KIND, 9, STORE>(a, s);
    case 15: return launch_fixed_r<KIND, 15, STORE>(a, s);
    default: return BF_ERR_UNSUPPORTED;
  }
}

template <int KIND, int NT, int TH, bool STORE>
bf_status launch_fwd(const FwdArgs &args, cudaStream_t s) {
  const int TW = NT - 2 * args.fc.R;
  const size_t smem = bfk::fwd_smem_bytes(NT, TH, args.fc.R, args.fc.ntaps_pad);
  auto kern = gpa_fwd_kernel<KIND, NT, TH, STORE>;
  const bf_status st = bfi::ensure_smem(reinterpret_cast<const void *>(kern), smem);
  if (st != BF_OK) return st;
  dim3 grid((args.io.W + TW - 1) / TW, (args.io.H + TH - 1) / TH);
  kern<<<grid, NT, smem, s>>>(args);
  return bfi::check_launch();
}

template <bool STORE>
bf_status dispatch(int v, const FwdArgs &a, cudaStream_t s) {
  const bool g = a.fc.kind == BF_SPATIAL_GAUSS;
  if (v == kFixedVariant) return g ? launch_fixed<1, STORE>(a, s) : launch_fixed<0, STORE>(a, s);
  if (v == kStreamVariant || v == kStream4Variant) {
    if (STORE) return BF_ERR_UNSUPPORTED;
    return v == kStreamVariant ? launch_warp<8>(a, s) : launch_warp<4>(a, s);
  }
  switch (v) {
    case 0: return g ? launch_fwd<1, 256, 16, STORE>(a, s) : launch_fwd<0, 256, 16, STORE>(a, s);
    case 1: return g ? launch_fwd<1, 512, 8, STORE>(a, s) : launch_fwd<0, 512, 8, STORE>(a, s);
    case 2: return g ? launch_fwd<1, 256, 8, STORE>(a, s) : launch_fwd<0, 256, 8, STORE>(a, s);
    case 3: return g ? launch_fwd<1, 128, 16, STORE>(a, s) : launch_fwd<0, 128, 16, STORE>(a, s);
    case 4: return g ? launch_fwd<1, 192, 8, STORE>(a, s) : launch_fwd<0, 192, 8, STORE>(a, s);
    default: return BF_ERR_INVALID_ARG;
  }
}

// count > 1: images k = 0 .. count - 1 at in / out / qaux + k image_stride
// (same size and parameters); the warp-strip kernels take them in one launch,
// the tile kernels in one launch per image.
bf_status forward_impl(const float *in, float *out, float *qaux, float *abar, size_t plane_stride,
                       int height, int width, int pitch, const bf_params *p, int variant,
                       void *stream, int count = 1, size_t image_stride = 0) {
  bf_status st = bfi::check_image(in, out, height, width, pitch);
  if (st != BF_OK) return st;
  if (count < 1 || (count > 1 && (abar || image_stride < (size_t)height * (size_t)pitch)))
    return BF_ERR_INVALID_ARG;
  FwdArgs a;
  st = bfi::resolve(p, true, &a.fc);
  if (st != BF_OK) return st;
  a.io = {in, out, qaux, abar, (long long)plane_stride, height, width, pitch};
  if (abar && plane_stride < (size_t)height * (size_t)pitch) return BF_ERR_INVALID_ARG;
  const bool store = abar != nullptr;
  int v = variant;
  if (v < 0) {
    v = bfi::tuned_variant(a.fc.kind, a.fc.R, a.fc.N);
    // the banded forward needs a workspace, which this path does not have
    if (v == kBandedVariant || (v >= 0 && !variant_fits(v, a.fc, store))) v = -1;
    if (v < 0) v = default_variant(a.fc, store);
    if (v < 0) return BF_ERR_UNSUPPORTED;
  } else {
    if (v >= kNumVariants) return BF_ERR_INVALID_ARG;
    if (v == kBandedVariant) return BF_ERR_WORKSPACE;
    if (!variant_fits(v, a.fc, store)) return BF_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (abar) return dispatch<true>(v, a, s);
  if (count == 1 || v == kStreamVariant || v == kStream4Variant) {
    a.count = count;
    a.image_stride = (long long)image_stride;
    return dispatch<false>(v, a, s);
  }
  for (int k = 0; k < count; ++k) {
    const size_t o = (size_t)k * image_stride;
    a.io.in = in + o;
    a.io.out = out + o;
    a.io.qaux = qaux ? qaux + o : nullptr;
    st = dispatch<false>(v, a, s);
    if (st != BF_OK) return st;
  }
  return BF_OK;
}

}  // namespace

namespace bfi {

bool forward_variant_fits(int v, const FilterConsts &fc) {
  return v >= 0 && v < kNumVariants && variant_fits(v, fc, false);
}

int forward_variant(const FilterConsts &fc, bool allow_banded) {
  int v = tuned_variant(fc.kind, fc.R, fc.N);
  if (v == kBandedVariant && !allow_banded) v = -1;
  if (v >= 0 && !variant_fits(v, fc, false)) v = -1;
  if (v >= 0) return v;
  if (allow_banded && bfk::banded_forward_preferred(fc.kind, fc.R)) return kBandedVariant;
  return default_variant(fc, false);
}

bool tile_variant_shape(int v, int *NT, int *TH) {
  if (v < 0 || v >= kNumGeneric) return false;
  *NT = kVariants[v].NT;
  *TH = kVariants[v].TH;
  return true;
}

}  // namespace bfi

extern "C" {

int bf_variant_count(int kind) {
  (void)kind;
  return kNumVariants;
}

bf_status bf_fast_forward(const float *d_in, float *d_out, float *d_qaux, int height, int width,
                          int pitch, const bf_params *p, void *stream) {
  return forward_impl(d_in, d_out, d_qaux, nullptr, 0, height, width, pitch, p, -1, stream);
}

bf_status bf_fast_forward_variant(const float *d_in, float *d_out, float *d_qaux, int height,
                                  int width, int pitch, const bf_params *p, int variant,
                                  void *stream) {
  return forward_impl(d_in, d_out, d_qaux, nullptr, 0, height, width, pitch, p, variant, stream);
}

bf_status bf_fast_forward_many(const float *d_in, float *d_out, float *d_qaux, int count,
                               size_t image_stride, int height, int width, int pitch,
                               const bf_params *p, void *stream) {
  return forward_impl(d_in, d_out, d_qaux, nullptr, 0, height, width, pitch, p, -1, stream, count,
                      image_stride);
}

bf_status bf_fast_forward_stored(const float *d_in, float *d_out, float *d_qaux, float *d_abar,
                                 size_t plane_stride, int height, int width, int pitch,
                                 const bf_params *p, void *stream) {
  if (!d_abar) return BF_ERR_INVALID_ARG;
  return forward_impl(d_in, d_out, d_qaux, d_abar, plane_stride, height, width, pitch, p, -1,
                      stream);
}

// Times every fitting variant (CUDA events on `stream` around each of `reps`
// launches after one warm-up launch; the fastest launch counts) and records
// the fastest variant in the tuning table, keeping the built-in choice unless
// another variant beats it by more than 3%.  Synchronises.  With a workspace
// that holds at least 64 band rows the two-pass banded forward (variant 8) is
// timed too.
bf_status bf_autotune_ws(const float *d_in, float *d_out, int height, int width, int pitch,
                         const bf_params *p, void *d_workspace, size_t workspace_bytes, int reps,
                         void *stream, int *best, float *best_ms) {
  if (!best || reps < 1) return BF_ERR_INVALID_ARG;
  bfi::FilterConsts fc;
  bf_status st = bfi::resolve(p, true, &fc);
  if (st != BF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return bfi::check_launch();
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfi::check_launch();
  }
  int bv = -1;
  float bms = 0.f;
  // the built-in choice for these constants (the table is not consulted)
  const bool have_ws = d_workspace && workspace_bytes > 0;
  const int incumbent = have_ws && bfk::banded_forward_preferred(fc.kind, fc.R)
                            ? kBandedVariant : default_variant(fc, false);
  float inc_ms = -1.f;
  auto run = [&](int v) {
    if (v == kBandedVariant)
      return bf_fast_forward_ws_variant(d_in, d_out, nullptr, height, width, pitch, p, v,
                                        d_workspace, workspace_bytes, stream);
    return bf_fast_forward_variant(d_in, d_out, nullptr, height, width, pitch, p, v, stream);
  };
  for (int v = 0; v < kNumVariants; ++v) {
    if (!variant_fits(v, fc)) continue;
    st = run(v);
    if (v == kBandedVariant && st == BF_ERR_WORKSPACE) {  // no room for it: not a candidate
      st = BF_OK;
      continue;
    }
    if (st != BF_OK) break;
    float ms = -1.f;  // the fastest of the timed launches
    for (int r = 0; r < reps && st == BF_OK; ++r) {
      cudaEventRecord(e0, s);
      st = run(v);
      cudaEventRecord(e1, s);
      const cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) st = bfi::cuda_status(ce);
      float t = 0.f;
      if (st == BF_OK) cudaEventElapsedTime(&t, e0, e1);
      if (ms < 0.f || t < ms) ms = t;
    }
    if (st != BF_OK) break;
    if (v == incumbent) inc_ms = ms;
    if (bv < 0 || ms < bms) {
      bv = v;
      bms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BF_OK) return st;
  if (bv < 0) return BF_ERR_UNSUPPORTED;
  // timing noise should not displace the built-in choice: a challenger must
  // be faster by more than kTuneMargin
  constexpr float kTuneMargin = 0.03f;
  if (inc_ms >= 0.f && bv != incumbent && bms > (1.f - kTuneMargin) * inc_ms) {
    bv = incumbent;
    bms = inc_ms;
  }
  *best = bv;
  if (best_ms) *best_ms = bms;
  return bf_tuning_set(fc.kind, bf_tuning_radius_bucket(fc.R), bf_tuning_order_bucket(fc.N), bv);
}

bf_status bf_autotune(const float *d_in, float *d_out, int height, int width, int pitch,
                      const bf_params *p, int reps, void *stream, int *best, float *best_ms) {
  return bf_autotune_ws(d_in, d_out, height, width, pitch, p, nullptr, 0, reps, stream, best,
                        best_ms);
}

}  // extern "C"
