// Kernel-error analysis of the Gaussian-polynomial (Sec. II).
//
// bf_kernel_error_max evaluates the sup-norm of eq. Linf,
//   max |E_N(t, tau)|,  E_N = g(t - tau) - phi_N(t, tau)   (eq. error),
// over a G x G grid of [-T, T]^2 in double precision (kernel errors of 1e-9
// and below are not resolvable in float32).  One thread per grid point; the
// block maxima are combined with an integer atomicMax on the bit patterns of
// the non-negative doubles, so the result does not depend on the order.
// Host-side order estimates for a kernel-error budget eps: Chebyshev
// (eq. cheby2), Chernoff (eq. LambW: the root of nu above lambda, App. A,
// found by bisection), and the exact Poisson tail of Prop. upperBound.
#include <math.h>

#include "bf_internal.h"

namespace {

__device__ __forceinline__ double kernel_error_at(double t, double tau, double inv2s2, double inv_s2,
                                                  int N) {
  const double x = t * tau * inv_s2;
  double s = 0.0, term = 1.0;
  for (int n = 0; n < N; ++n) {
    s += term;
    term *= x / (double)(n + 1);
  }
  const double phi = exp(-(t * t + tau * tau) * inv2s2) * s;
  const double g = exp(-(t - tau) * (t - tau) * inv2s2);
  return fabs(g - phi);
}

__global__ void __launch_bounds__(256) kernel_error_kernel(int N, double sr, double T, int G,
                                                           unsigned long long *out) {
  const double inv_s2 = 1.0 / (sr * sr), inv2s2 = 0.5 * inv_s2;
  const double step = G > 1 ? 2.0 * T / (double)(G - 1) : 0.0;
  double m = 0.0;
  const long long total = (long long)G * G;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const double t = -T + step * (double)(k % G);
    const double tau = -T + step * (double)(k / G);
    m = fmax(m, kernel_error_at(t, tau, inv2s2, inv_s2, N));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) b = fmax(b, red[i]);
    atomicMax(out, (unsigned long long)__double_as_longlong(b));  // b >= 0: bits order as values
  }
}

double poisson_tail(int N, double lam) {
  // P(X >= N) = 1 - sum_{n<N} e^{-lam} lam^n / n!, summed in log space; for
  // large N sum the tail directly (terms decrease once n > lam).
  if (N <= 0) return 1.0;
  if ((double)N > lam) {
    double s = 0.0;
    for (int n = N; n < N + 100000; ++n) {
      const double tn = exp(-lam + n * log(lam) - lgamma((double)n + 1.0));
      s += tn;
      if (tn < 1e-300 || tn < s * 1e-17) break;
    }
    return s;
  }
  double s = 0.0;
  for (int n = 0; n < N; ++n) s += exp(-lam + n * log(lam) - lgamma((double)n + 1.0));
  return s >= 1.0 ? 0.0 : 1.0 - s;
}

}  // namespace

extern "C" {

bf_status bf_kernel_error_max(int N, double sigma_r, double T, int grid, double *d_out,
                              void *stream) {
  if (!d_out || N < 1 || !(sigma_r > 0.0) || !(T > 0.0) || grid < 1 || grid > 65536)
    return BF_ERR_INVALID_ARG;
  if (N > BF_MAX_ORDER) return BF_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double), s);
  if (e != cudaSuccess) return bfi::cuda_status(e);
  const long long total = (long long)grid * grid;
  const int blocks = (int)((total + 255) / 256 < 152LL * 16 ? (total + 255) / 256 : 152LL * 16);
  kernel_error_kernel<<<blocks, 256, 0, s>>>(N, sigma_r, T, grid,
                                             reinterpret_cast<unsigned long long *>(d_out));
  return bfi::check_launch();
}

bf_status bf_order_estimates(double sigma_r, double eps, double T, int *N_chebyshev,
                             int *N_chernoff, int *N_poisson) {
  if (!(sigma_r > 0.0) || !(eps > 0.0) || eps >= 1.0 || !(T > 0.0)) return BF_ERR_INVALID_ARG;
  const double lam = (T / sigma_r) * (T / sigma_r);
  // estimates are plain numbers (not limited to BF_MAX_ORDER); cap at 1e8
  if (N_chebyshev) {  // eq. cheby2
    const double n = ceil(lam + sqrt(lam / eps));
    if (n > 1e8) return BF_ERR_UNSUPPORTED;
    *N_chebyshev = (int)n;
  }
  if (N_chernoff) {  // eq. LambW: the root above lambda of x log x - p x - q (App. A)
    const double p = 1.0 + log(lam), q = -lam - log(eps);
    auto nu = [&](double x) { return x * log(x) - p * x - q; };
    double lo = lam, hi = 2.0 * lam + 1.0;
    int guard = 0;
    while (nu(hi) <= 0.0) {
      lo = hi;
      hi *= 2.0;
      if (++guard > 200) return BF_ERR_UNSUPPORTED;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
      const double mid = 0.5 * (lo + hi);
      (nu(mid) > 0.0 ? hi : lo) = mid;
    }
    const double n = ceil(hi - 1e-9 * hi);
    if (n > 1e8) return BF_ERR_UNSUPPORTED;
    *N_chernoff = n < 1.0 ? 1 : (int)n;
  }
  if (N_poisson) {  // smallest N with P(X >= N) <= eps (Prop. upperBound)
    int n = 1;
    while (poisson_tail(n, lam) > eps) {
      if (++n > 1000000) return BF_ERR_UNSUPPORTED;
    }
    *N_poisson = n;
  }
  return BF_OK;
}

}  // extern "C"
