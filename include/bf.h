/*
 * bf.h -- C ABI of the GB300 (sm_103a) Gaussian-polynomial bilateral filter.
 *
 * Method: K. N. Chaudhury and S. D. Dabhade, "Fast and Provably Accurate
 * Bilateral Filtering", arXiv 1603.08109.  The bilateral filter (eq. BF) with
 * a Gaussian range kernel (eq. range_kernel) and a box (eq. spatial_kernel2)
 * or Gaussian (eq. spatial_kernel1) spatial kernel on Omega = [-W, W]^2 is
 * approximated by replacing each translated range kernel with the
 * Gaussian-polynomial phi_N of eq. GaussPolynomial (eq. GPA).  With centred
 * intensities h = f - t_c (eq. shift) and H = h / sigma_r the result is
 *      f_GPA = t_c + sigma_r * P' / Q',
 *      Q' = sum_{n<N} a_n (w * a_n),   P' = sum_{n<N} sqrt(n+1) a_n (w * a_{n+1}),
 *      a_n = exp(-H^2/2) H^n / sqrt(n!),
 * which is eqs. PbyQ, P, Q of Sec. III-A (Algorithm 2) with every auxiliary
 * image divided by sqrt(n!) and the common factor exp(-H^2/2) of P and Q
 * cancelled (an exact rescaling; it keeps every intermediate in [-1, 1]).
 *
 * Conventions shared by every entry point:
 *  - Images are single-channel float32, row-major, `height` rows of `width`
 *    pixels, consecutive rows `pitch` elements apart (pitch >= width).
 *    Intensities are expected in [0, 2 t_c] (8-bit data: t_c = 128).
 *  - The image domain is finite (Sec. I): every spatial sum runs over the
 *    neighbours that lie inside the image only, without renormalisation
 *    (w cancels in the ratio).  This is the same as zero-extending the
 *    power images before filtering.
 *  - `d_*` pointers are device pointers; the caller owns all device memory.
 *    The library never allocates device memory and never synchronises the
 *    stream: every GPU entry point only enqueues work on `stream` (a
 *    cudaStream_t passed as void*, NULL = legacy default stream).
 *  - float arrays must be 4-byte aligned; inputs and outputs may not alias
 *    (an output equal to the input is rejected with BF_ERR_INVALID_ARG;
 *    partial overlaps are not detected).
 *  - Errors are returned, never raised: nothing traps or aborts.  A CUDA
 *    launch error is reported as BF_ERR_CUDA (the CUDA error string is
 *    available from bf_last_cuda_error()).
 */
#ifndef BF_GB300_H
#define BF_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,  /* a size, pointer or parameter is out of range  */
    BF_ERR_CUDA = 2,         /* a CUDA runtime call or launch failed          */
    BF_ERR_UNSUPPORTED = 3,  /* valid, but beyond this build's limits         */
    BF_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up            */
    BF_ERR_WORKSPACE = 5,    /* workspace missing or smaller than required    */
    BF_ERR_NONFINITE = 6     /* reserved: non-finite result reported by a check */
} bf_status;

typedef enum {
    BF_SPATIAL_BOX = 0,      /* eq. spatial_kernel2: w = 1/|Omega|            */
    BF_SPATIAL_GAUSS = 1,    /* eq. spatial_kernel1: w = exp(-|j|^2 / 2 s^2)  */
    BF_SPATIAL_GAUSS_RECURSIVE = 2  /* Deriche's recursive Gaussian (Sec. I,
                                       Sec. III-A); only bf_recursive_* and the
                                       order-selection helpers accept it      */
} bf_spatial_kind;

/* Filter parameters (Sec. I, Sec. III).
 *  kind     bf_spatial_kind.
 *  radius   W, the half-width of Omega = [-W, W]^2 (support 2W+1 per axis).
 *           For the Gaussian, radius <= 0 selects W = ceil(3 sigma_s) (Sec. I).
 *  sigma_s  Gaussian spatial standard deviation (ignored for the box).
 *  sigma_r  range standard deviation, > 0.  Because the rescaled power images
 *           start from exp(-H^2/2) in float32, |f - t_c| / sigma_r must stay
 *           below 13 (sigma_r >= 9.85 for 8-bit data); smaller sigma_r is
 *           rejected with BF_ERR_UNSUPPORTED.
 *  order_N  N, the number of Taylor terms of eq. approx (1 <= N <= BF_MAX_ORDER);
 *           the method performs N + 1 spatial filterings (Algorithm 2).
 *  t_c      centre of the intensity range (eq. shift); 128 for 8-bit data.   */
typedef struct {
    int kind;
    int radius;
    float sigma_s;
    float sigma_r;
    int order_N;
    float t_c;
} bf_params;

#define BF_MAX_ORDER 1024
#define BF_MAX_RADIUS 96

/* ------------------------------------------------------------------ misc */
const char *bf_status_string(int status);
/* Message of the last CUDA error seen by this library in this thread, or the
 * reason given with the last BF_ERR_UNSUPPORTED that carries one. */
const char *bf_last_cuda_error(void);
/* Library version, as major * 10000 + minor * 100 + patch. */
int bf_version(void);

/* --------------------------------------------------- order selection (host)
 * Centre weight w(0) of the normalised spatial kernel (eq. normal):
 * 1/(2W+1)^2 for the box, 1/(sum_k exp(-k^2/2 sigma_s^2))^2 for the
 * Gaussian on [-W, W]^2, h(0)^2 for the recursive Gaussian (radius ignored;
 * h is its normalised 1-D impulse response, see bf_recursive_forward).
 * Host only; no GPU work. */
bf_status bf_centre_weight(int kind, int radius, float sigma_s, double *w0_out);

/* Order N for a filter accuracy delta (Sec. III-C): eps from eq. eps,
 * eps = w(0) delta / (2T + delta), then N = ceil(theta) where theta is the
 * root above lambda = T^2/sigma_r^2 of nu(x) = x log x - p x - q
 * (App. A; p = 1 + log lambda, q = -lambda - log eps), i.e. eq. LambW.
 * The root is bracketed and refined by safeguarded Newton steps
 * (eq. Newton_method).  T is the half dynamic range (128 for 8-bit data).
 * BF_ERR_INVALID_ARG if delta <= 0, T <= 0, sigma_r <= 0 or radius < 0;
 * BF_ERR_UNSUPPORTED if the order exceeds BF_MAX_ORDER.  Host only. */
bf_status bf_order_from_delta(int kind, int radius, float sigma_s, float sigma_r,
                              float delta, float T, int *N_out);

/* Order N for a volume (video) filter accuracy delta: as bf_order_from_delta
 * with the centre weight of the separable 3-D kernel w1(j_z) w1(j_y) w1(j_x)
 * of bf_volume_forward, w1(0)^3 = (planar w(0))^(3/2) in eq. eps (the Sec. I
 * and Sec. V extension to video and volume data).  kind: BF_SPATIAL_BOX or
 * BF_SPATIAL_GAUSS (radius <= 0: ceil(3 sigma_s)).  Same errors.  Host only. */
bf_status bf_volume_order_from_delta(int kind, int radius, float sigma_s, float sigma_r,
                                     float delta, float T, int *N_out);

/* -------------------------------------------- kernel-error analysis (Sec. II)
 * bf_kernel_error_max: sup-norm of the kernel error (eq. Linf),
 *   max |g(t - tau) - phi_N(t, tau)|  (eq. error)
 * over a grid x grid lattice of [-T, T]^2 (end points included), evaluated
 * in double precision on the GPU; writes one double to d_out (device).
 * BF_ERR_INVALID_ARG for N < 1, sigma_r <= 0, T <= 0, grid outside [1, 65536].
 * bf_order_estimates (host only): for a kernel-error budget eps in (0, 1),
 * the Chebyshev order (eq. cheby2), the Chernoff order (eq. LambW, the
 * root of nu above lambda = T^2/sigma_r^2, App. A) and the exact Poisson
 * order (smallest N with P(X >= N) <= eps, Prop. upperBound); any output
 * pointer may be NULL. */
bf_status bf_kernel_error_max(int N, double sigma_r, double T, int grid, double *d_out,
                              void *stream);
bf_status bf_order_estimates(double sigma_r, double eps, double T, int *N_chebyshev,
                             int *N_chernoff, int *N_poisson);

/* ---------------------------------------------------------- fast forward
 * f_GPA of eq. GPA via Algorithm 2 (eqs. intImg, spatialFiltering, PbyQ,
 * P, Q), fused: each output tile reads its input tile plus a W-pixel halo
 * once, generates the N+1 power images a_0..a_N in on-chip memory, filters
 * them and accumulates P', Q' in registers.
 *  d_in    input image (height x width, pitch elements per row).
 *  d_out   output image, same layout as d_in.
 *  d_qaux  optional (NULL allowed): receives Q' at every pixel, normalised
 *          as sum_j w(j) phi_N(h(i-j), h(i)) with sum_Omega w = 1 (this is
 *          Q_2 of App. C).  Needed by bf_fast_backward.
 * BF_ERR_INVALID_ARG for null in/out, height or width < 1, pitch < width,
 * or invalid params. */
bf_status bf_fast_forward(const float *d_in, float *d_out, float *d_qaux,
                          int height, int width, int pitch,
                          const bf_params *p, void *stream);

/* Forward with a caller-provided workspace, for large radii (by default
 * Gaussian W >= 12 except 15, box W > 15, where it is faster than the fused
 * kernels; the tuning table below can choose it, variant 8, for other radii
 * and keep the fused kernels at some of these).  The
 * spatial filter is separable (eq. spatial_kernel1 on the square Omega), so
 * the image is processed in bands of rows, two kernels per band: the first
 * filters the columns of every power image a_0..a_N of the band (with the
 * W-row halos) into the workspace, the second filters those planes along the
 * rows (with the W-column halos) and forms P', Q' and f_GPA (Algorithm 2).
 * Results equal bf_fast_forward's up to float rounding.
 * bf_fast_forward_workspace: the workspace in bytes for bands as tall as
 *   the image, or as fit 8 GiB (64 rows at least; fewer, taller bands lose
 *   fewer launch tails); 0 when the banded path is not chosen (bf_fast_forward_ws
 *   then runs the fused kernels, as bf_fast_forward).
 * bf_fast_forward_ws: d_workspace device memory, 16-byte aligned, owned by
 *   the caller, of ws_bytes >= 64 rows of N + 1 planes, i.e. 64 (N+1) Wp
 *   floats with Wp = width rounded up to a multiple of 4; a larger workspace
 *   gives taller bands.  Same arguments and outputs as bf_fast_forward.
 *   BF_ERR_WORKSPACE for a missing or too small workspace when the banded
 *   path is chosen.
 * bf_fast_forward_ws_variant: the same with an explicit variant (see the
 *   tuning section; -1 = the table / built-in choice, as bf_fast_forward_ws). */
bf_status bf_fast_forward_workspace(int height, int width, const bf_params *p,
                                    size_t *bytes);
bf_status bf_fast_forward_ws(const float *d_in, float *d_out, float *d_qaux,
                             int height, int width, int pitch, const bf_params *p,
                             void *d_workspace, size_t ws_bytes, void *stream);
bf_status bf_fast_forward_ws_variant(const float *d_in, float *d_out, float *d_qaux,
                                     int height, int width, int pitch, const bf_params *p,
                                     int variant, void *d_workspace, size_t ws_bytes,
                                     void *stream);

/* bf_fast_forward for `count` images of the same height, width, pitch and
 * parameters (e.g. the frames of a video): image k is read from
 * d_in + k * image_stride and written to d_out (and d_qaux, if not NULL)
 * + k * image_stride; image_stride >= height * pitch (elements), and the
 * input and output blocks must not overlap.  Each image is filtered on its
 * own (zero extension at its edges), with the same results as bf_fast_forward
 * image by image.  The warp-strip box kernel (box, W in {3, 5}, N <= 8) takes
 * the whole batch in one launch, which amortises its ramp-up and tail over
 * the batch; the other kernels run one launch per image.
 * BF_ERR_INVALID_ARG for count < 1 or a smaller image_stride. */
bf_status bf_fast_forward_many(const float *d_in, float *d_out, float *d_qaux, int count,
                               size_t image_stride, int height, int width, int pitch,
                               const bf_params *p, void *stream);

/* Same as bf_fast_forward, and also stores the N+1 filtered power images
 * w * a_n (normalised kernel) to d_abar: plane n at d_abar + n * plane_stride,
 * each plane height x width with row pitch `pitch`; plane_stride >=
 * height * pitch.  For the stored-power-image backward. */
bf_status bf_fast_forward_stored(const float *d_in, float *d_out, float *d_qaux,
                                 float *d_abar, size_t plane_stride,
                                 int height, int width, int pitch,
                                 const bf_params *p, void *stream);

/* --------------------------------------------------------- fast backward
 * Gradient of a loss L through f_GPA with respect to the input image and
 * sigma_r (N and W held fixed), given gout = dL/d f_GPA.  The paper has no
 * backward pass; this is the exact adjoint of the rescaled P'/Q' ratio:
 *   pbar = gout sigma_r / Q',  qbar = -gout (out - t_c) / Q',
 *   abar_n = qbar (w*a_n) [n<N] + pbar sqrt(n+1) (w*a_{n+1}) [n<N]
 *            + w * (qbar a_n [n<N] + pbar sqrt(n) a_{n-1} [n>=1]),
 *   Hbar = sum_n abar_n (sqrt(n) a_{n-1} - H a_n),  gin = Hbar / sigma_r,
 *   gsigma = sum_i gout (out - t_c) / sigma_r - sum_i Hbar H / sigma_r.
 * The power images are recomputed (not stored).
 *  d_in, d_out, d_qaux  the forward's input, output and Q' (from the same params).
 *  d_gout               dL/d out.           d_gin: dL/d in (written).
 *  d_gsigma             optional: one double on the device, written (not added).
 *  d_workspace          >= bf_fast_backward_workspace() bytes (may be NULL
 *                       only if d_gsigma is NULL), 256-byte aligned.  The
 *                       sigma_r sum is reduced deterministically in a fixed
 *                       order.
 * For W > 15 the gradient is computed by a two-pass banded backward (a column
 * pass of a_n, qbar a_n and pbar a_n into workspace planes, then a row pass
 * that forms the sums above), the adjoint of bf_fast_forward_ws; its
 * workspace (the query's value) also holds the qbar and pbar planes.  With a
 * workspace too small for 64 band rows, or none, the fused runtime-W kernel
 * runs instead where its tile fits (W up to about 52).
 * For W in {3, 5, 9, 15} (without stored planes) the fused kernel keeps each
 * thread's region inputs in tensor memory: every CTA of 128 threads
 * allocates 128 TMEM columns for its lifetime and frees them before it
 * exits, and at most four of its CTAs share an SM (4 x 128 = the SM's 512
 * columns).  A kernel of another library that holds TMEM columns on the same
 * SMs at the same time (another stream) makes an allocation wait until
 * columns are free; it never fails.
 * BF_ERR_WORKSPACE if the workspace is missing or too small. */
bf_status bf_fast_backward_workspace(int height, int width, const bf_params *p,
                                     size_t *bytes);
bf_status bf_fast_backward(const float *d_in, const float *d_out, const float *d_qaux,
                           const float *d_gout, float *d_gin, double *d_gsigma,
                           int height, int width, int pitch, const bf_params *p,
                           void *d_workspace, size_t workspace_bytes, void *stream);

/* Same gradient, reading the N+1 filtered power images written by
 * bf_fast_forward_stored instead of recomputing them (only the adjoint
 * channels are filtered).  Same workspace rule. */
bf_status bf_fast_backward_stored(const float *d_in, const float *d_out, const float *d_qaux,
                                  const float *d_abar, size_t plane_stride,
                                  const float *d_gout, float *d_gin, double *d_gsigma,
                                  int height, int width, int pitch, const bf_params *p,
                                  void *d_workspace, size_t workspace_bytes, void *stream);

/* Allocation-free variant of bf_fast_backward (the paper has no counterpart;
 * it exists for callers of this library, not for the method).  Some callers
 * cannot call cudaMalloc: plug-ins hosted by an application that owns the
 * device allocator, and real-time pipelines that must not allocate after
 * start-up because cudaMalloc can synchronise the device and take an
 * unbounded time.  This entry point needs no workspace: the per-CTA sigma_r
 * partial sums go to a fixed 65536-entry (512 KiB) static device array that
 * every GPU loading the library holds until the process exits.  The caller
 * still passes every input and output, as for bf_fast_backward, and gets the
 * same results.
 *  - The first call on a device (with d_gsigma non-NULL) looks up the
 *    array's device address for that device, so make that first call before
 *    any stream capture.
 *  - All calls share the array and it keeps the last call's partial sums;
 *    each call writes every entry it reads, so nothing needs clearing, but
 *    calls that overlap on the GPU (e.g. on two streams) race on it.
 *  - With d_gsigma non-NULL, an image that needs more than 65536 partial
 *    sums (one per CTA of the backward grid: roughly beyond 5.7e7 pixels at
 *    W = 9, e.g. above 7500 x 7500) is rejected with BF_ERR_UNSUPPORTED
 *    before any GPU work.  With d_gsigma NULL no scratch is used and any
 *    image size is accepted.
 *  - Radii are limited to those whose fused backward tile fits in shared
 *    memory (227 KB per block): Gaussian W <= 50, box W <= 39.  Larger radii
 *    return BF_ERR_UNSUPPORTED with that reason in bf_last_cuda_error();
 *    bf_fast_backward takes them through its banded backward, which needs a
 *    caller workspace.
 *  - The cached address outlives a cudaDeviceReset, so a device that was
 *    reset after the first call is not supported.
 *  Nothing here calls cudaMalloc, cudaFree or any allocating library
 *  routine. */
bf_status bf_fast_backward_noalloc(const float *d_in, const float *d_out, const float *d_qaux,
                                   const float *d_gout, float *d_gin, double *d_gsigma,
                                   int height, int width, int pitch, const bf_params *p,
                                   void *stream);

/* ------------------------------------------------------ direct filter
 * eq. BF computed directly, O((2W+1)^2) exponentials per pixel (Sec. I-A),
 * float32 accumulation; order_N is ignored.  The same-GPU comparison. */
bf_status bf_direct(const float *d_in, float *d_out, int height, int width, int pitch,
                    const bf_params *p, void *stream);

/* Gradient of eq. BF with respect to the image and sigma_r (the paper has
 * none; exact chain rule on the ratio, gather form).  Workspace: >=
 * bf_direct_backward_workspace() bytes, always required (per-pixel
 * denominators and partial sums). */
bf_status bf_direct_backward_workspace(int height, int width, const bf_params *p,
                                       size_t *bytes);
bf_status bf_direct_backward(const float *d_in, const float *d_gout, float *d_gin,
                             double *d_gsigma, int height, int width, int pitch,
                             const bf_params *p, void *d_workspace,
                             size_t workspace_bytes, void *stream);

/* ------------------------------------------------ cross (joint) filter
 * The cross (joint) bilateral filter, named as an extension in Sec. I and
 * Sec. V: the range kernel compares a guide image e while the data f is
 * averaged,
 *   out(i) = t_c + sum_j w(j) k(e(i-j), e(i)) (f(i-j) - t_c) / sum_j w(j) k(e(i-j), e(i)).
 * bf_joint_forward uses k = phi_N on centred guide values (eq. GaussPolynomial):
 * with b_n the guide's rescaled power images, out = t_c + U'/Q',
 * Q' = sum_{n<N} b_n (w*b_n), U' = sum_{n<N} b_n (w*(b_n (f - t_c))): 2N
 * spatial filterings in one fused pass.  For e = f it equals bf_fast_forward.
 * d_qaux (optional) receives Q' as in bf_fast_forward.  The guide follows the
 * image's layout (same height, width, pitch).  Radius limit: W <= 56.
 * For W in {3, 5, 9, 15} the kernel keeps each thread's region inputs in
 * tensor memory (128 TMEM columns per CTA of 128 threads, at most four CTAs
 * per SM; see bf_fast_backward).
 * bf_joint_forward_workspace / bf_joint_forward_ws: the same filter for
 * Gaussian W > 15 and box W > 24 (where the fused box tile stops being the
 * faster form) by the two-pass banded split (see bf_fast_forward_ws): a column pass
 * of b_n and b_n (f - t_c) into 2N workspace planes per band, then a row pass
 * forming Q' and U'.  Workspace rule as for bf_fast_forward_ws with 2N planes
 * per band row (64 rows at least); radii up to BF_MAX_RADIUS; below those
 * radii the workspace query returns 0 and the call runs bf_joint_forward.
 * bf_joint_direct computes the same filter with the exact Gaussian range
 * kernel, O((2W+1)^2) per pixel (the same-GPU comparison). */
bf_status bf_joint_forward(const float *d_in, const float *d_guide, float *d_out, float *d_qaux,
                           int height, int width, int pitch, const bf_params *p, void *stream);
bf_status bf_joint_forward_workspace(int height, int width, const bf_params *p, size_t *bytes);
bf_status bf_joint_forward_ws(const float *d_in, const float *d_guide, float *d_out,
                              float *d_qaux, int height, int width, int pitch, const bf_params *p,
                              void *d_workspace, size_t ws_bytes, void *stream);
bf_status bf_joint_direct(const float *d_in, const float *d_guide, float *d_out, int height,
                          int width, int pitch, const bf_params *p, void *stream);

/* --------------------------------------------------- batched forward
 * Many images of uneven sizes, each with its own spatial kind, W, sigma_s,
 * sigma_r and N.  Each image runs the variant that the tuning table (below)
 * holds for its (kind, radius bucket, order bucket), or the built-in choice
 * of bf_fast_forward_ws where the table has no entry or its entry does not
 * fit the image's radius:
 *  - runtime-radius tiles (variants 0..4): ONE persistent launch per tile
 *    shape present, whose CTAs take output tiles from a device work queue
 *    (longest work first) until it is empty;
 *  - compile-time-radius and warp-strip kernels (variants 5..7): one launch
 *    per image (their filter taps are constant-bank operands of a launch);
 *  - the two-pass banded forward (variant 8): one column-pass launch and one
 *    row-pass launch over the tiles of a group of images, their planes in the
 *    plan's workspace (groups keep the plane region at most 4 GiB, reused
 *    group after group).
 * The three groups run on the caller's stream and two side streams of the
 * plan, forked from and joined back into the caller's stream with events.
 * Each image's result equals the single-image call with its variant bit for
 * bit.  The table is read when the plan is created.
 * Usage: bf_batch_plan_create (host: validates, picks the variants, orders
 * the work) -> bf_batch_workspace -> bf_batch_upload (enqueue the plan's
 * tables into the workspace; the plan must stay alive until that copy has
 * completed) -> bf_batch_forward, any number of times (graph-capturable: a
 * memset node, the persistent kernels, the per-image kernels and two kernels
 * per banded group as parallel branches; no allocation, no host
 * synchronisation) -> bf_batch_plan_destroy.
 * bf_batch_variants: the variant each image runs (count = the plan's image
 * count). */
typedef struct {
    const float *d_in;   /* device input image                    */
    float *d_out;        /* device output image                   */
    float *d_qaux;       /* optional Q' output (NULL = none)       */
    int height, width, pitch;
    bf_params params;
} bf_image_desc;

typedef struct bf_batch_plan bf_batch_plan;

bf_status bf_batch_plan_create(const bf_image_desc *descs, int count, bf_batch_plan **plan);
bf_status bf_batch_workspace(const bf_batch_plan *plan, size_t *bytes);
/* Number of work items (tiles of the persistent and banded launches, plus
 * one per whole-image launch) and CTAs of the persistent launches. */
bf_status bf_batch_info(const bf_batch_plan *plan, int *items, int *ctas);
bf_status bf_batch_variants(const bf_batch_plan *plan, int *variants, int count);
bf_status bf_batch_upload(const bf_batch_plan *plan, void *d_workspace,
                          size_t workspace_bytes, void *stream);
/* d_status (optional, device int): set to BF_ERR_INVALID_ARG by the kernel
 * if a work item names a descriptor outside the plan; left unchanged
 * otherwise.  CTAs never wait on one another (work is taken with one atomic
 * add per item), so the launch has no device-side wait to time out. */
bf_status bf_batch_forward(const bf_batch_plan *plan, void *d_workspace,
                           size_t workspace_bytes, int *d_status, void *stream);
void bf_batch_plan_destroy(bf_batch_plan *plan);

/* Capture bf_batch_forward into a CUDA graph on `stream` and instantiate
 * it; bf_graph_launch replays it; bf_graph_destroy frees it. */
bf_status bf_batch_graph_create(const bf_batch_plan *plan, void *d_workspace,
                                size_t workspace_bytes, int *d_status, void *stream,
                                void **graph_exec_out);
bf_status bf_graph_launch(void *graph_exec, void *stream);
void bf_graph_destroy(void *graph_exec);

/* ---------------------------------------------------- tile autotuning
 * The forward comes in several kernels and tile shapes (variants):
 *   0..4  the runtime-radius fused tile with (threads, output rows) =
 *         (256, 16), (512, 8), (256, 8), (128, 16), (192, 8);
 *   5     the compile-time-radius fused tile (W in {3, 5, 9, 15});
 *   6, 7  the warp-strip streaming box kernel, 8 / 4 columns per lane
 *         (box, W in {3, 5}, N <= 5 / N <= 8);
 *   8     the two-pass banded forward (needs the workspace of
 *         bf_fast_forward_ws; the calls without one skip it).
 * The library keeps a table variant[kind][radius bucket][order bucket]
 * (-1 = the built-in choice); bf_autotune times every variant that fits on
 * caller-provided device buffers (it synchronises `stream`; each variant's
 * fastest of `reps` launches counts) and records the fastest, keeping the
 * built-in choice unless another variant beats it by more than 3%.  The
 * single-image forwards and the batch plan read the table.
 *  bf_variant_count        number of variants for a kind (>= 1).
 *  bf_fast_forward_variant forward with an explicit variant (-1 = table);
 *                          variant 8 returns BF_ERR_WORKSPACE here.
 *  bf_autotune(_ws)        time all variants for (kind, W, N) at this size
 *                          (with a workspace of at least 64 band rows, see
 *                          bf_fast_forward_ws, the banded forward too);
 *                          writes the winner to *best and into the table.
 *  bf_tuning_get/set       read / write one table entry (for a JSON cache). */
int bf_variant_count(int kind);
bf_status bf_fast_forward_variant(const float *d_in, float *d_out, float *d_qaux,
                                  int height, int width, int pitch, const bf_params *p,
                                  int variant, void *stream);
bf_status bf_autotune(const float *d_in, float *d_out, int height, int width, int pitch,
                      const bf_params *p, int reps, void *stream, int *best,
                      float *best_ms);
bf_status bf_autotune_ws(const float *d_in, float *d_out, int height, int width, int pitch,
                         const bf_params *p, void *d_workspace, size_t workspace_bytes,
                         int reps, void *stream, int *best, float *best_ms);
int bf_tuning_radius_bucket(int radius);
int bf_tuning_order_bucket(int order_N);
bf_status bf_tuning_get(int kind, int radius_bucket, int order_bucket, int *variant);
bf_status bf_tuning_set(int kind, int radius_bucket, int order_bucket, int variant);

/* ------------------------------------------- recursive Gaussian (Sec. III-A)
 * The paper notes (Sec. I, Sec. III-A) that the N + 1 spatial filterings of
 * Algorithm 2 cost O(1) per pixel, independent of the filter size, when the
 * Gaussian is implemented by recursion (Deriche).  These entry points use
 * Deriche's fourth-order fit: the 1-D impulse response
 *     h(k) = (1.680 cos(0.6318 k/s) + 3.735 sin(0.6318 k/s)) exp(-1.783 k/s)
 *          - (0.6803 cos(1.997 k/s) + 0.2598 sin(1.997 k/s)) exp(-1.723 k/s)
 * for k >= 0, mirrored for k < 0, s = sigma_s, normalised to unit sum over
 * all integers (within 5e-4 of the sampled Gaussian's peak).  Its causal and
 * anticausal recursions start from zero state at both ends of every row and
 * column, which is exactly the convolution of the zero-extended image with
 * w(j) = h(j_y) h(j_x) over the whole image (the in-image-neighbours rule of
 * the other kinds, with unbounded support); the cost per pixel and channel
 * does not depend on sigma_s.  Floating point: FP32, each mode a complex
 * one-pole recursion; rows and columns cut into 32-pixel tiles made exact by
 * a carry pass (no halos).
 *
 * bf_recursive_workspace: bytes of the caller-owned device workspace for an
 *   image of height x width and order N (N = 0: the plain filter):
 *   1.5 (N + 1) 4 Hp P bytes (Hp, P = height, width rounded up to 32;
 *   N + 1 planes and two carry arrays of a quarter plane each), rounded to
 *   256-byte blocks.
 * bf_recursive_gauss: d_out = w * d_in (the plain filter, one image), for
 *   tests and as a building block.  sigma_s >= 0.5.
 * bf_recursive_forward: Algorithm 2 (f_GPA, optional Q') with w the
 *   recursive Gaussian; p->kind must be BF_SPATIAL_GAUSS_RECURSIVE,
 *   p->sigma_s >= 0.5, p->radius is ignored; otherwise as bf_fast_forward
 *   (the same sigma_r limit).  Choose N with bf_order_from_delta (kind 2:
 *   w(0) = h(0)^2).
 * bf_recursive_backward_workspace / bf_recursive_backward: the exact adjoint
 *   of bf_recursive_forward (the paper has none; the same derivation as
 *   bf_fast_backward): with qbar = -g (out - t_c) / Q', pbar = g sigma_r / Q',
 *   the seeds c_n = qbar a_n [n<N] + pbar sqrt(n) a_{n-1} [n>=1] and the power
 *   images a_n are both filtered (the zero-extended recursive filter is
 *   self-adjoint), Hbar = sum_n abar_n (sqrt(n) a_{n-1} - H a_n), d in =
 *   Hbar / sigma_r, d sigma_r = sum_i (g (out - t_c) - Hbar H) / sigma_r (N
 *   held fixed).  d_out and d_qaux are the forward's out and Q' (order N,
 *   same image and parameters); d_gout the cotangent of out; d_gin receives
 *   d loss / d in; d_gsigma_r (device double, may be NULL) receives the sigma_r
 *   gradient, summed in a fixed order (deterministic).  Workspace:
 *   2.75 (N + 1) 4 Hp P bytes plus 8 bytes per 16 x 32 column tile.
 * Workspace: 256-byte aligned, at least the queried size, else
 * BF_ERR_WORKSPACE / BF_ERR_INVALID_ARG.  Asynchronous on `stream`. */
bf_status bf_recursive_workspace(int height, int width, int order_N, size_t *bytes);
/* bf_recursive_joint_workspace / bf_recursive_joint_forward: the cross (joint)
 *   filter of bf_joint_forward (guide d_guide, averaged image d_in, same
 *   layout) with the recursive Gaussian as w: the guide's power images b_n
 *   and the products b_n (f - t_c), n < N, through the same row and column
 *   passes (2N filterings), out = t_c + U'/Q' and optionally Q' (d_qaux).
 *   Workspace: (2.75 N) 4 Hp P bytes plus 8 bytes per 16 x 32 column tile. */
bf_status bf_recursive_joint_workspace(int height, int width, int order_N, size_t *bytes);
bf_status bf_recursive_joint_forward(const float *d_in, const float *d_guide, float *d_out,
                                     float *d_qaux, int height, int width, int pitch,
                                     const bf_params *p, void *d_ws, size_t ws_bytes,
                                     void *stream);
bf_status bf_recursive_backward_workspace(int height, int width, int order_N, size_t *bytes);
bf_status bf_recursive_backward(const float *d_in, const float *d_out, const float *d_qaux,
                                const float *d_gout, float *d_gin, double *d_gsigma_r, int height,
                                int width, int pitch, const bf_params *p, void *d_ws,
                                size_t ws_bytes, void *stream);
bf_status bf_recursive_gauss(const float *d_in, float *d_out, int height, int width, int pitch,
                             float sigma_s, void *d_ws, size_t ws_bytes, void *stream);
bf_status bf_recursive_forward(const float *d_in, float *d_out, float *d_qaux, int height,
                               int width, int pitch, const bf_params *p, void *d_ws,
                               size_t ws_bytes, void *stream);
/* bf_recursive_forward_stored / bf_recursive_backward_stored: the same
 *   forward and gradient, with the power images' row-pass planes kept between
 *   them instead of recomputed (the paper has no backward; this trades memory
 *   for the backward's repeat of those row passes).  The forward takes a
 *   workspace of the backward's size (bf_recursive_backward_workspace, same
 *   height, width and N) and writes the same out and Q' as
 *   bf_recursive_forward; afterwards the workspace holds the N + 1 row-filtered
 *   power planes and their scanned column-tile states.  The backward then
 *   runs only the adjoint seeds' passes and the gather, and returns the same
 *   bits as bf_recursive_backward.  Contract (not checkable on the host): the
 *   backward gets the workspace the stored forward wrote, unmodified, with the
 *   same d_in contents, height, width, pitch and parameters; anything else
 *   gives wrong gradients (never an out-of-bounds access: every index comes
 *   from the sizes).  The backward overwrites only the seeds' part, so one
 *   stored forward serves several backwards (e.g. several cotangents). */
bf_status bf_recursive_forward_stored(const float *d_in, float *d_out, float *d_qaux,
                                      int height, int width, int pitch, const bf_params *p,
                                      void *d_ws, size_t ws_bytes, void *stream);
bf_status bf_recursive_backward_stored(const float *d_in, const float *d_out,
                                       const float *d_qaux, const float *d_gout, float *d_gin,
                                       double *d_gsigma_r, int height, int width, int pitch,
                                       const bf_params *p, void *d_ws, size_t ws_bytes,
                                       void *stream);

/* ------------------------------------------------ volume / video (Sec. I, V)
 * The paper notes that the filter extends directly to video and volume data.
 * bf_volume_forward runs Algorithm 2 on a grayscale volume f of depth x
 * height x width voxels (packed: x fastest, then y, then z; for video, z is
 * time) with the same Gaussian range kernel and the separable spatial kernel
 * w(j) = w1(j_z) w1(j_y) w1(j_x), w1 the normalised 1-D box (p->kind =
 * BF_SPATIAL_BOX) or truncated Gaussian (BF_SPATIAL_GAUSS, radius = ceil(3
 * sigma_s) if p->radius <= 0) of the planar filter, the same along every
 * axis; neighbours outside the volume do not contribute.  Outputs f_GPA and
 * optionally Q' (normalised), as bf_fast_forward per voxel.  Choose N with
 * bf_volume_order_from_delta (eq. eps with w(0) = w1(0)^3).  Two passes: the
 * z-filtering of the N + 1 power images into the workspace, then per z-plane
 * the y- and x-filterings and the ratio (for W <= 8 each channel's plane
 * region reaches shared memory by one tiled tensor copy).  Workspace:
 * bf_volume_workspace bytes = 256 + 4 (N + 1) depth height Wp, Wp = width
 * rounded up to a multiple of 4; device memory owned by the caller, 16-byte
 * aligned.  Its first 4 bytes are a status word that each call sets to
 * BF_OK; a copy wait that gives up after about a second (which a healthy GPU
 * never reaches) leaves BF_ERR_TIMEOUT there and the outputs undefined.
 * BF_ERR_UNSUPPORTED for radius > 31 or depth or height > 65535;
 * BF_ERR_WORKSPACE for a missing or small workspace; BF_ERR_INVALID_ARG for
 * other kinds, aliasing outputs or sizes < 1.  Asynchronous on `stream`. */
bf_status bf_volume_workspace(int depth, int height, int width, const bf_params *p,
                              size_t *bytes);
bf_status bf_volume_forward(const float *d_in, float *d_out, float *d_qaux, int depth,
                            int height, int width, const bf_params *p, void *d_ws,
                            size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BF_GB300_H */
