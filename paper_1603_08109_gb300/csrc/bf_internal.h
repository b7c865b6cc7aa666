// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/bf.h"

#define BF_VERSION 10400  // 1.4.0: video / volume data (bf_volume_forward)

// Gaussian taps are padded with zeros to a multiple of 16 (the register-window
// unroll of the separable passes); 2 * BF_MAX_RADIUS + 1 = 193 -> 208 <= 224.
#define BF_TAPS_MAX 224

namespace bfi {

// One image's filter constants as the device sees them (resolved params).
struct FilterConsts {
  int kind;        // BF_SPATIAL_BOX / BF_SPATIAL_GAUSS
  int R;           // radius W
  int N;           // number of Taylor terms
  int ntaps_pad;   // Gaussian: 2R+1 rounded up to a multiple of 16; box: 0
  float sr;        // sigma_r
  float inv_sr;    // 1 / sigma_r
  float tc;        // centre t_c
  float qscale;    // kernel-sum normalisation: box 1/(2R+1)^2, Gaussian 1
  float e2c;       // -log2(e) / (2 sigma_r^2): a_0 = 2^(e2c (f - t_c)^2)
  float taps[BF_TAPS_MAX];  // normalised 1-D Gaussian taps, taps[k] = w1(k - R)
};

// Status helpers (bf_host.cpp).
bf_status cuda_status(cudaError_t e);
bf_status check_launch();
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device (cached per device and kernel; thread-safe).
bf_status ensure_smem(const void *func, size_t bytes);
// Resident CTAs of a kernel on the current device (SMs x CTAs per SM) for a
// block size and dynamic shared memory (cached; thread-safe).
bf_status resident_ctas(const void *func, int threads, size_t smem, int *ctas);
void set_error_text(const char *msg);

// Validates image sizes / pointers / params and fills the device constants.
// `need_order` is false for the direct filter (order_N ignored).
bf_status resolve(const bf_params *p, bool need_order, FilterConsts *fc);
bf_status check_image(const void *in, const void *out, int height, int width, int pitch);

// Two-pass banded backward for W > 15 (gpa_banded_bwd.cu): whether it applies,
// the workspace it prefers, and the launch sequence (prep, per band a column
// and a row pass, the sigma_r reduce).  BF_ERR_WORKSPACE when ws holds fewer
// than 64 band rows.
bool banded_backward_fits(const FilterConsts &fc);
size_t banded_backward_bytes(int height, int width, const FilterConsts &fc);
bf_status banded_backward(const float *in, const float *out, const float *qaux, const float *gout,
                          float *gin, double *gsigma, int height, int width, int pitch,
                          const FilterConsts &fc, void *ws, size_t ws_bytes, void *stream);

// w(0) = h(0)^2 of the normalised recursive (Deriche) Gaussian (recursive.cu).
double recursive_centre_weight(double sigma_s);

// Fastest compiled-in tile variant for (kind, R, N) from the tuning table.
int tuned_variant(int kind, int R, int N);

// Forward variants (gpa_fwd.cu): 0..4 runtime-radius tiles, 5 compile-time
// radius, 6 / 7 warp-strip box, 8 the two-pass banded forward (workspace).
constexpr int kFwdBandedVariant = 8;
constexpr int kFwdNumVariants = 9;
// Whether variant v can run these constants (without stored planes).
bool forward_variant_fits(int v, const FilterConsts &fc);
// The variant a forward runs: the tuning table's entry for (kind, radius
// bucket, order bucket) when it fits, else the built-in rule (banded for
// Gaussian W >= 12 except 15 and box W > 15 when allow_banded, then the
// compile-time-radius, warp-strip and runtime-radius kernels).  -1: none fits.
int forward_variant(const FilterConsts &fc, bool allow_banded);
// (threads per CTA, output rows per tile) of a runtime-radius tile variant.
bool tile_variant_shape(int v, int *NT, int *TH);

}  // namespace bfi
