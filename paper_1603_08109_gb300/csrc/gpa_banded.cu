// Two-pass banded forward of Algorithm 2 for large radii (by default
// Gaussian W >= 12 except 15, box W > 15; the tuning table may choose it for
// any radius): single-image launches and the workspace entry points (tile
// bodies in gpa_banded.cuh).
//
// A fused 2-D tile needs a 2W halo in both directions: at W = 60 its region
// is tens of times the tile, does not fit shared memory at a useful size, and
// the tile runs at a few per cent of the FP32 pipe.  The spatial filter is
// separable (eq. spatial_kernel1 on the square Omega), so here the image is cut
// into bands of rows and each band goes through a column pass and a row pass.
// Each pass carries a halo in one direction only.  Bands are as tall as the
// workspace allows (by default the whole image, up to 8 GiB of planes).
// Out-of-image pixels carry a_n = 0 (zero extension), as in the fused kernels.
#include <algorithm>
#include <mutex>

#include "gpa_banded.cuh"

namespace {

using namespace bfk;

constexpr size_t kBandCap = 8ull << 30;   // default workspace cap (bytes)

template <int KIND>
__global__ void __launch_bounds__(kVNT) band_vpass(const __grid_constant__ BandArgs A) {
  extern __shared__ __align__(16) float sm[];
  band_vpass_tile<KIND>(A, blockIdx.x, blockIdx.y, sm, A.fc.taps);
}

template <int KIND>
__global__ void __launch_bounds__(kBandNT) band_hpass(const __grid_constant__ BandArgs A) {
  extern __shared__ __align__(16) float sm[];
  band_hpass_tile<KIND>(A, blockIdx.x, blockIdx.y, sm, A.fc.taps);
}

// Whether a forward with a workspace takes the banded path: the tuning
// table's choice, else the built-in radius rule.
bool banded_route(const bfi::FilterConsts &fc) {
  return bfi::forward_variant(fc, true) == bfi::kFwdBandedVariant;
}

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

// Preferred band rows: the whole image when its planes fit the cap, else as
// many rows as fit.  Every band is a column-pass launch followed by a row-pass
// launch that waits for it, so fewer bands lose fewer launch tails (8192^2,
// W = 60, N = 32: 640-row bands 24.4 ms, 4096-row bands 22.3 ms, one band
// 22.2 ms).
int preferred_band_rows(int height, int width, int N) {
  const long long rows = (height + kVB - 1) / kVB * kVB;
  const int fit = band_rows(height, width, N, kBandCap);
  if (fit <= 0 || fit >= rows) return (int)std::max<long long>(fit > 0 ? rows : kVB, kVB);
  // the fewest bands that fit, of equal height (no short last band)
  const long long nb = (rows + fit - 1) / fit;
  const long long even = ((rows + nb - 1) / nb + kVB - 1) / kVB * kVB;
  return (int)std::min<long long>(even, fit);
}

template <int KIND>
bf_status launch_band(BandArgs &A, cudaStream_t s) {
  const int ntp_max = (2 * BF_MAX_RADIUS + 1 + 15) / 16 * 16;
  bf_status est = bfi::ensure_smem(reinterpret_cast<const void *>(band_vpass<KIND>),
                                   vpass_smem(KIND, BF_MAX_RADIUS, ntp_max));
  if (est == BF_OK)
    est = bfi::ensure_smem(reinterpret_cast<const void *>(band_hpass<KIND>),
                           hpass_smem(KIND, BF_MAX_RADIUS, ntp_max));
  if (est != BF_OK) return est;
  const int R = A.fc.R, ntp = A.fc.ntaps_pad;
  const size_t vs = vpass_smem(KIND, R, ntp), hs = hpass_smem(KIND, R, ntp);
  const int band = A.rows;
  for (int y0 = 0; y0 < A.H; y0 += band) {
    A.y0 = y0;
    A.rows = std::min(band, A.H - y0);
    dim3 gv((A.Wp + kVC - 1) / kVC, (A.rows + kVB - 1) / kVB);
    band_vpass<KIND><<<gv, kVNT, vs, s>>>(A);
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
  if (!banded_route(fc)) return BF_OK;
  const size_t row_bytes = (size_t)(fc.N + 1) * (size_t)round_up4(width) * sizeof(float);
  *bytes = row_bytes * (size_t)preferred_band_rows(height, width, fc.N);
  return BF_OK;
}

bf_status bf_fast_forward_ws_variant(const float *d_in, float *d_out, float *d_qaux, int height,
                                     int width, int pitch, const bf_params *p, int variant,
                                     void *d_workspace, size_t ws_bytes, void *stream) {
  bf_status st = bfi::check_image(d_in, d_out, height, width, pitch);
  if (st != BF_OK) return st;
  bfi::FilterConsts fc;
  st = bfi::resolve(p, true, &fc);
  if (st != BF_OK) return st;
  if (variant >= bfi::kFwdNumVariants) return BF_ERR_INVALID_ARG;
  const int v = variant >= 0 ? variant : bfi::forward_variant(fc, true);
  if (v < 0) return BF_ERR_UNSUPPORTED;
  if (v != bfi::kFwdBandedVariant)
    return bf_fast_forward_variant(d_in, d_out, d_qaux, height, width, pitch, p, v, stream);
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

bf_status bf_fast_forward_ws(const float *d_in, float *d_out, float *d_qaux, int height, int width,
                             int pitch, const bf_params *p, void *d_workspace, size_t ws_bytes,
                             void *stream) {
  return bf_fast_forward_ws_variant(d_in, d_out, d_qaux, height, width, pitch, p, -1, d_workspace,
                                    ws_bytes, stream);
}

}  // extern "C"
