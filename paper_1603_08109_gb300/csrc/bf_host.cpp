// Host-side parts of the library: status codes, argument validation,
// spatial-kernel tables and order selection (Sec. II-B, Sec. III-C).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "bf_internal.h"

namespace {
thread_local char g_err[256] = "no CUDA error";

// Tuning table: variant index per (kind, radius bucket, order bucket).
// -1 means "use the built-in rule".  Written by bf_tuning_set / bf_autotune.
constexpr int kRadiusBuckets = 8;
constexpr int kOrderBuckets = 6;
std::atomic<int> g_table[2][kRadiusBuckets][kOrderBuckets];
std::atomic<bool> g_table_init{false};

void init_table() {
  bool expected = false;
  if (g_table_init.compare_exchange_strong(expected, true)) {
    for (auto &k : g_table)
      for (auto &r : k)
        for (auto &o : r) o.store(-1);
  }
}
}  // namespace

namespace bfi {

void set_error_text(const char *msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg ? msg : "");
}

bf_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BF_OK;
  set_error_text(cudaGetErrorString(e));
  return BF_ERR_CUDA;
}

bf_status check_launch() { return cuda_status(cudaGetLastError()); }

bf_status ensure_smem(const void *func, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> set;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(dev, func);
  const auto it = set.find(key);
  if (it != set.end() && it->second >= bytes) return BF_OK;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return cuda_status(e);
  set[key] = bytes;
  return BF_OK;
}

bf_status resident_ctas(const void *func, int threads, size_t smem, int *ctas) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, func, threads, smem);
  const auto it = cache.find(key);
  if (it != cache.end()) {
    *ctas = it->second;
    return BF_OK;
  }
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e);
  cache[key] = per_sm * sms;
  *ctas = per_sm * sms;
  return BF_OK;
}

bf_status check_image(const void *in, const void *out, int height, int width, int pitch) {
  if (!in || !out) return BF_ERR_INVALID_ARG;
  // the tiles read neighbours' pixels that other CTAs write: no in-place filtering
  if (in == out) return BF_ERR_INVALID_ARG;
  if (height < 1 || width < 1 || pitch < width) return BF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) & 3u) || (reinterpret_cast<uintptr_t>(out) & 3u))
    return BF_ERR_INVALID_ARG;
  // Pixel offsets are formed in 64-bit; the row index fits an int by the checks above.
  return BF_OK;
}

// Normalised 1-D Gaussian taps exp(-k^2 / 2 s^2) / Z on k = -R..R (eq.
// spatial_kernel1 is separable on the square Omega, so the 2-D kernel is the
// outer product and sums to 1, eq. normal).  Computed in double, rounded once.
static void gaussian_taps(int R, double sigma_s, float *taps, int ntaps_pad) {
  double tmp[2 * BF_MAX_RADIUS + 1];
  double z = 0.0;
  for (int k = -R; k <= R; ++k) {
    tmp[k + R] = exp(-(double)k * k / (2.0 * sigma_s * sigma_s));
    z += tmp[k + R];
  }
  for (int i = 0; i < ntaps_pad; ++i) taps[i] = (i <= 2 * R) ? (float)(tmp[i] / z) : 0.0f;
}

bf_status resolve(const bf_params *p, bool need_order, FilterConsts *fc) {
  if (!p || !fc) return BF_ERR_INVALID_ARG;
  memset(fc, 0, sizeof(*fc));
  if (p->kind != BF_SPATIAL_BOX && p->kind != BF_SPATIAL_GAUSS) return BF_ERR_INVALID_ARG;
  if (!(p->sigma_r > 0.0f) || !isfinite(p->sigma_r)) return BF_ERR_INVALID_ARG;
  if (!isfinite(p->t_c)) return BF_ERR_INVALID_ARG;
  int R = p->radius;
  if (p->kind == BF_SPATIAL_GAUSS) {
    if (!(p->sigma_s > 0.0f) || !isfinite(p->sigma_s)) return BF_ERR_INVALID_ARG;
    if (R <= 0) R = (int)ceil(3.0 * (double)p->sigma_s - 1e-9);
  }
  if (R < 0) return BF_ERR_INVALID_ARG;
  if (R > BF_MAX_RADIUS) return BF_ERR_UNSUPPORTED;
  if (need_order) {
    if (p->order_N < 1) return BF_ERR_INVALID_ARG;
    if (p->order_N > BF_MAX_ORDER) return BF_ERR_UNSUPPORTED;
    // exp(-H^2/2) must stay a normal float32 for |f - t_c| <= t_c.
    if ((double)p->t_c / (double)p->sigma_r > 13.0) return BF_ERR_UNSUPPORTED;
  }
  fc->kind = p->kind;
  fc->R = R;
  fc->N = p->order_N;
  fc->sr = p->sigma_r;
  fc->inv_sr = (float)(1.0 / (double)p->sigma_r);
  fc->e2c = (float)(-1.4426950408889634 / (2.0 * (double)p->sigma_r * (double)p->sigma_r));
  fc->tc = p->t_c;
  if (p->kind == BF_SPATIAL_GAUSS) {
    fc->ntaps_pad = ((2 * R + 1) + 15) / 16 * 16;
    gaussian_taps(R, p->sigma_s, fc->taps, fc->ntaps_pad);
    fc->qscale = 1.0f;
  } else {
    fc->ntaps_pad = 0;
    fc->qscale = (float)(1.0 / ((double)(2 * R + 1) * (double)(2 * R + 1)));
  }
  return BF_OK;
}

int tuned_variant(int kind, int R, int N) {
  init_table();
  if (kind < 0 || kind > 1) return -1;
  return g_table[kind][bf_tuning_radius_bucket(R)][bf_tuning_order_bucket(N)].load();
}

}  // namespace bfi

using namespace bfi;

extern "C" {

const char *bf_status_string(int status) {
  switch (status) {
    case BF_OK: return "ok";
    case BF_ERR_INVALID_ARG: return "invalid argument";
    case BF_ERR_CUDA: return "CUDA error";
    case BF_ERR_UNSUPPORTED: return "unsupported parameters";
    case BF_ERR_TIMEOUT: return "device wait timed out";
    case BF_ERR_WORKSPACE: return "workspace missing or too small";
    case BF_ERR_NONFINITE: return "non-finite result";
    default: return "unknown status";
  }
}

const char *bf_last_cuda_error(void) { return g_err; }

int bf_version(void) { return BF_VERSION; }

bf_status bf_centre_weight(int kind, int radius, float sigma_s, double *w0_out) {
  if (!w0_out || radius < 0) return BF_ERR_INVALID_ARG;
  if (kind == BF_SPATIAL_BOX) {
    double s = 2.0 * radius + 1.0;
    *w0_out = 1.0 / (s * s);
    return BF_OK;
  }
  if (kind == BF_SPATIAL_GAUSS_RECURSIVE) {
    if (!(sigma_s >= 0.5f) || !isfinite(sigma_s)) return BF_ERR_INVALID_ARG;
    *w0_out = recursive_centre_weight(sigma_s);
    return BF_OK;
  }
  if (kind != BF_SPATIAL_GAUSS || !(sigma_s > 0.0f)) return BF_ERR_INVALID_ARG;
  if (radius > 100000) return BF_ERR_UNSUPPORTED;
  double z = 0.0;
  for (int k = -radius; k <= radius; ++k) z += exp(-(double)k * k / (2.0 * (double)sigma_s * sigma_s));
  *w0_out = 1.0 / (z * z);
  return BF_OK;
}

}  // extern "C"

namespace {

// w(0) of the planar kernel of (kind, radius, sigma_s), the Gaussian radius
// defaulting to ceil(3 sigma_s) (the recursive Gaussian has no radius).
bf_status planar_centre_weight(int kind, int radius, float sigma_s, double *w0) {
  int R = kind == BF_SPATIAL_GAUSS_RECURSIVE ? 0 : radius;
  if (kind == BF_SPATIAL_GAUSS && R <= 0) {
    if (!(sigma_s > 0.0f)) return BF_ERR_INVALID_ARG;
    R = (int)ceil(3.0 * (double)sigma_s - 1e-9);
  }
  return bf_centre_weight(kind, R, sigma_s, w0);
}

// Order from the accuracy target (Sec. III-C and App. A): eps from eq. eps,
// then the root theta of nu.  nu(x) = x log x - p x - q is strictly convex
// with its minimum at lambda, and nu(lambda) = log(eps) < 0, so exactly one
// root theta > lambda exists; nu is increasing there.  Bracket it by
// doubling, then take Newton steps (eq. Newton_method), falling back to
// bisection whenever a step leaves the bracket.
bf_status order_from_centre_weight(double w0, float sigma_r, float delta, float T, int *N_out) {
  const double t = T, d = delta;
  const double eps = w0 * d / (2.0 * t + d);  // eq. eps
  if (!(eps > 0.0) || eps >= 1.0) return BF_ERR_INVALID_ARG;
  const double lam = (t / sigma_r) * (t / sigma_r);
  const double p = 1.0 + log(lam), q = -lam - log(eps);
  auto nu = [&](double x) { return x * log(x) - p * x - q; };
  double lo = lam, hi = 2.0 * lam + 1.0;
  int guard = 0;
  while (nu(hi) <= 0.0) {
    lo = hi;
    hi *= 2.0;
    if (++guard > 200 || hi > 1e12) return BF_ERR_UNSUPPORTED;
  }
  double x = hi;
  for (int it = 0; it < 200; ++it) {
    double fx = nu(x);
    if (fx > 0.0) hi = x; else lo = x;
    double step = fx / (log(x) + 1.0 - p);
    double xn = x - step;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) <= 1e-13 * x || hi - lo <= 1e-13 * hi) {
      x = xn;
      break;
    }
    x = xn;
  }
  double N = ceil(x - 1e-9 * x);
  if (N < 1.0) N = 1.0;
  if (N > BF_MAX_ORDER) return BF_ERR_UNSUPPORTED;
  *N_out = (int)N;
  return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_order_from_delta(int kind, int radius, float sigma_s, float sigma_r, float delta,
                              float T, int *N_out) {
  if (!N_out || !(delta > 0.0f) || !(T > 0.0f) || !(sigma_r > 0.0f)) return BF_ERR_INVALID_ARG;
  double w0 = 0.0;
  const bf_status st = planar_centre_weight(kind, radius, sigma_s, &w0);
  if (st != BF_OK) return st;
  return order_from_centre_weight(w0, sigma_r, delta, T, N_out);
}

// Volume / video data (the Sec. I and Sec. V extension): the spatial kernel
// is w1(j_z) w1(j_y) w1(j_x) with the planar filter's normalised 1-D kernel
// w1, so its centre weight is w1(0)^3 = (planar w(0))^(3/2); eq. eps and the
// root of nu then follow unchanged (Prop. accuracy holds for any normalised
// non-negative kernel).
bf_status bf_volume_order_from_delta(int kind, int radius, float sigma_s, float sigma_r,
                                     float delta, float T, int *N_out) {
  if (!N_out || !(delta > 0.0f) || !(T > 0.0f) || !(sigma_r > 0.0f)) return BF_ERR_INVALID_ARG;
  if (kind != BF_SPATIAL_BOX && kind != BF_SPATIAL_GAUSS) return BF_ERR_INVALID_ARG;
  double w0 = 0.0;
  const bf_status st = planar_centre_weight(kind, radius, sigma_s, &w0);
  if (st != BF_OK) return st;
  return order_from_centre_weight(w0 * sqrt(w0), sigma_r, delta, T, N_out);
}

int bf_tuning_radius_bucket(int radius) {
  // 0-4, 5-8, 9-12, 13-20, 21-30, 31-44, 45-50, 51+
  if (radius <= 4) return 0;
  if (radius <= 8) return 1;
  if (radius <= 12) return 2;
  if (radius <= 20) return 3;
  if (radius <= 30) return 4;
  if (radius <= 44) return 5;
  if (radius <= 50) return 6;
  return 7;
}

int bf_tuning_order_bucket(int order_N) {
  // 1-4, 5-12, 13-32, 33-64, 65-128, 129+
  if (order_N <= 4) return 0;
  if (order_N <= 12) return 1;
  if (order_N <= 32) return 2;
  if (order_N <= 64) return 3;
  if (order_N <= 128) return 4;
  return 5;
}

bf_status bf_tuning_get(int kind, int rb, int ob, int *variant) {
  init_table();
  if (!variant || kind < 0 || kind > 1 || rb < 0 || rb >= kRadiusBuckets || ob < 0 ||
      ob >= kOrderBuckets)
    return BF_ERR_INVALID_ARG;
  *variant = g_table[kind][rb][ob].load();
  return BF_OK;
}

bf_status bf_tuning_set(int kind, int rb, int ob, int variant) {
  init_table();
  if (kind < 0 || kind > 1 || rb < 0 || rb >= kRadiusBuckets || ob < 0 || ob >= kOrderBuckets)
    return BF_ERR_INVALID_ARG;
  if (variant < -1 || variant >= bf_variant_count(kind)) return BF_ERR_INVALID_ARG;
  g_table[kind][rb][ob].store(variant);
  return BF_OK;
}

}  // extern "C"
