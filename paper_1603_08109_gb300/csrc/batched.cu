// Batched forward: many images of uneven sizes, each with its own spatial
// kind, W, sigma_s, sigma_r and N.
//
// Each image runs the forward variant that the tuning table names for its
// (kind, radius bucket, order bucket), or the built-in choice where the table
// has no entry (bfi::forward_variant, the same rule a single-image call with
// a workspace follows), so every image's result equals the single-image call
// with that variant bit for bit.  The variants fall into three groups:
//
//  * runtime-radius tiles (variants 0..4, one (threads, rows) shape each):
//    ONE persistent launch per shape present.  The host plan splits the
//    images into output tiles (work items), estimates each item's cost from
//    its (N + 1) filterings and tile geometry and sorts the items longest
//    first.  The grid is sized to the device (SMs x resident CTAs); each CTA
//    repeatedly takes the next item index from the shape's device counter
//    (atomicAdd; no CTA ever waits on another) and runs the single-image
//    tile body with that item's parameters;
//  * whole-image kernels (variant 5, compile-time radius, and variants 6 / 7,
//    warp-strip box): these keep the image's filter taps as constant-bank
//    operands of a launch, so each such image is its own launch;
//  * the two-pass banded forward (variant 8, gpa_banded.cuh): one launch per
//    pass over the tiles of a group of images (longest first); each image's
//    N + 1 column-filtered planes live in the plan's workspace, groups are
//    formed so that one group's planes fit a 4 GiB region that the next group
//    reuses.
//
// The persistent launches run on the caller's stream, the whole-image
// launches and the banded groups on two side streams of the plan that fork
// from and join back into it with events, so the three groups overlap and a
// captured CUDA graph holds them as parallel branches.  A launch is a memset
// of the counters plus these kernels, so it can be captured and replayed.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "bf_internal.h"
#include "gpa_banded.cuh"
#include "gpa_tile.cuh"

namespace {

constexpr int kMaxTileGroups = 5;  // runtime-radius tile variants 0..4

struct BatchDesc {
  bfk::TileIO io;
  bfi::FilterConsts fc;
};

struct WorkItem {
  int desc, ty0, tx0, pad;
};

struct BatchArgs {
  const BatchDesc *descs;
  const WorkItem *items;  // this launch's items
  int *counter;
  int *status;
  int count, nitems;
};

template <int NT, int TH>
__global__ void __launch_bounds__(NT) gpa_batched_kernel(const __grid_constant__ BatchArgs A) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();  // everyone has read s_item before thread 0 may overwrite it
    if (it >= A.nitems) break;
    const WorkItem w = A.items[it];
    if (w.desc < 0 || w.desc >= A.count) {
      if (threadIdx.x == 0 && A.status) atomicExch(A.status, (int)BF_ERR_INVALID_ARG);
      continue;
    }
    const BatchDesc &d = A.descs[w.desc];
    const bfi::FilterConsts &fc = d.fc;
    if (fc.kind == BF_SPATIAL_GAUSS)
      bfk::gpa_fwd_tile<1, NT, TH, TH, false>(d.io, fc, fc.taps, w.ty0, w.tx0, smem);
    else
      bfk::gpa_fwd_tile<0, NT, TH, TH, false>(d.io, fc, fc.taps, w.ty0, w.tx0, smem);
    __syncthreads();  // the next item's region load reuses shared memory
  }
}

// The persistent kernel of tile variant v (shapes as in gpa_fwd.cu).
const void *tile_kernel(int v) {
  switch (v) {
    case 0: return reinterpret_cast<const void *>(gpa_batched_kernel<256, 16>);
    case 1: return reinterpret_cast<const void *>(gpa_batched_kernel<512, 8>);
    case 2: return reinterpret_cast<const void *>(gpa_batched_kernel<256, 8>);
    case 3: return reinterpret_cast<const void *>(gpa_batched_kernel<128, 16>);
    case 4: return reinterpret_cast<const void *>(gpa_batched_kernel<192, 8>);
    default: return nullptr;
  }
}

void launch_tile_kernel(int v, int ctas, size_t smem, cudaStream_t s, const BatchArgs &A) {
  switch (v) {
    case 0: gpa_batched_kernel<256, 16><<<ctas, 256, smem, s>>>(A); break;
    case 1: gpa_batched_kernel<512, 8><<<ctas, 512, smem, s>>>(A); break;
    case 2: gpa_batched_kernel<256, 8><<<ctas, 256, smem, s>>>(A); break;
    case 3: gpa_batched_kernel<128, 16><<<ctas, 128, smem, s>>>(A); break;
    case 4: gpa_batched_kernel<192, 8><<<ctas, 192, smem, s>>>(A); break;
    default: break;
  }
}

// ---- banded items
// slot: the item's image in its launch's tap table, or -1 when its taps do not
// fit the table (radius above 63): then they are read from the descriptor copy
struct BandItem {
  int desc, bx, by, slot;
};

// A launch carries the taps of (at most) kBandLaunchImages images in its
// parameter block, so that the filters read them as constant-bank operands,
// as the single-image kernels do (from a per-CTA shared copy they cost a
// shared-memory load per tap and left the batch's passes waiting on them).
constexpr int kBandLaunchImages = 48, kBandTapsMax = 128;

struct BandBatchArgs {
  const bfk::BandArgs *descs;  // .ws holds the byte offset of the image's planes
  const BandItem *items;       // this launch's items, one per CTA
  char *planes;                // the workspace's plane region
  float taps[kBandLaunchImages][kBandTapsMax];
};
static_assert(sizeof(BandBatchArgs) <= 32764, "kernel parameter block");

template <bool VPASS>
__global__ void __launch_bounds__(VPASS ? bfk::kVNT : bfk::kBandNT) gpa_batched_band_kernel(
    const __grid_constant__ BandBatchArgs A) {
  extern __shared__ __align__(16) float smem[];
  __shared__ bfk::BandArgs sA;
  const BandItem it = A.items[blockIdx.x];
  const int *src = reinterpret_cast<const int *>(A.descs + it.desc);
  int *dst = reinterpret_cast<int *>(&sA);
  for (int i = threadIdx.x; i < (int)(sizeof(bfk::BandArgs) / sizeof(int)); i += blockDim.x)
    dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x == 0)
    sA.ws = reinterpret_cast<float *>(A.planes + reinterpret_cast<uintptr_t>(sA.ws));
  __syncthreads();
  if (sA.fc.kind != BF_SPATIAL_GAUSS) {  // the box filter has no taps
    if (VPASS) bfk::band_vpass_tile<BF_SPATIAL_BOX>(sA, it.bx, it.by, smem, sA.fc.taps);
    else bfk::band_hpass_tile<BF_SPATIAL_BOX>(sA, it.bx, it.by, smem, sA.fc.taps);
  } else if (it.slot >= 0) {
    if (VPASS) bfk::band_vpass_tile<BF_SPATIAL_GAUSS>(sA, it.bx, it.by, smem, A.taps[it.slot]);
    else bfk::band_hpass_tile<BF_SPATIAL_GAUSS>(sA, it.bx, it.by, smem, A.taps[it.slot]);
  } else {
    if (VPASS) bfk::band_vpass_tile<BF_SPATIAL_GAUSS>(sA, it.bx, it.by, smem, sA.fc.taps);
    else bfk::band_hpass_tile<BF_SPATIAL_GAUSS>(sA, it.bx, it.by, smem, sA.fc.taps);
  }
}

struct BandGroup {
  int v0, nv, h0, nh;
  size_t vsmem, hsmem;
  std::vector<float> taps;  // kBandLaunchImages x kBandTapsMax: the launches' tap table
};

struct TileGroup {
  int variant, NT, TH;
  int item0, nitems;  // range in the plan's item table
  size_t smem;
  int ctas;
};

struct WholeImage {
  bf_image_desc d;
  int variant;
};

constexpr size_t kBatchPlaneCap = 4ull << 30;  // plane bytes per group

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct bf_batch_plan {
  std::vector<BatchDesc> descs;
  std::vector<int> variants;  // per image
  std::vector<WorkItem> items;
  std::vector<TileGroup> tgroups;
  std::vector<WholeImage> whole;
  std::vector<bfk::BandArgs> bdescs;
  std::vector<BandItem> bitems;
  std::vector<BandGroup> groups;
  cudaStream_t side[2] = {nullptr, nullptr};  // whole-image launches, banded groups
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  size_t off_descs = 0, off_items = 0, off_bdescs = 0, off_bitems = 0, off_planes = 0;
  size_t ws_bytes = 0;
  std::vector<unsigned char> staging;  // tables, laid out as in the workspace
  ~bf_batch_plan() {
    for (cudaStream_t s : side)
      if (s) cudaStreamDestroy(s);
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : join)
      if (e) cudaEventDestroy(e);
  }
};

extern "C" {

bf_status bf_batch_plan_create(const bf_image_desc *descs, int count, bf_batch_plan **plan_out) {
  if (!descs || count < 1 || !plan_out) return BF_ERR_INVALID_ARG;
  *plan_out = nullptr;
  bf_batch_plan *plan = new (std::nothrow) bf_batch_plan();
  if (!plan) return BF_ERR_INVALID_ARG;
  auto fail = [&](bf_status st) {
    delete plan;
    return st;
  };
  struct Cost {
    double c;
    WorkItem w;
  };
  std::vector<Cost> costs[kMaxTileGroups];
  size_t gsmem[kMaxTileGroups] = {};
  std::vector<int> large;  // images for the banded path
  plan->descs.resize(count);
  plan->variants.resize(count);
  for (int i = 0; i < count; ++i) {
    const bf_image_desc &d = descs[i];
    bf_status st = bfi::check_image(d.d_in, d.d_out, d.height, d.width, d.pitch);
    BatchDesc &bd = plan->descs[i];
    if (st == BF_OK) st = bfi::resolve(&d.params, true, &bd.fc);
    if (st != BF_OK) return fail(st);
    bd.io = {d.d_in, d.d_out, d.d_qaux, nullptr, 0, d.height, d.width, d.pitch};
    const int v = bfi::forward_variant(bd.fc, true);
    if (v < 0) return fail(BF_ERR_UNSUPPORTED);
    plan->variants[i] = v;
    int NT = 0, TH = 0;
    if (v == bfi::kFwdBandedVariant) {
      large.push_back(i);
      continue;
    }
    if (!bfi::tile_variant_shape(v, &NT, &TH)) {  // a whole-image kernel
      plan->whole.push_back({d, v});
      continue;
    }
    const int R = bd.fc.R, TW = NT - 2 * R;
    gsmem[v] = std::max(gsmem[v], bfk::fwd_smem_bytes(NT, TH, R, bd.fc.ntaps_pad));
    // cost model per tile: (N+1) x (region generation + both filter passes)
    const double taps = bd.fc.kind == BF_SPATIAL_GAUSS ? (double)bd.fc.ntaps_pad : 4.0;
    const double per_ch = (double)(TH + 2 * R) * NT * 3.0 + (double)TH * NT * taps +
                          (double)TH * TW * (taps + 4.0);
    const double c = (bd.fc.N + 1.0) * per_ch + (double)(TH + 2 * R) * NT * 8.0;
    for (int y = 0; y < d.height; y += TH)
      for (int x = 0; x < d.width; x += TW) costs[v].push_back({c, {i, y, x, 0}});
  }
  for (int v = 0; v < kMaxTileGroups; ++v) {
    if (costs[v].empty()) continue;
    std::stable_sort(costs[v].begin(), costs[v].end(),
                     [](const Cost &a, const Cost &b) { return a.c > b.c; });
    TileGroup g{};
    g.variant = v;
    bfi::tile_variant_shape(v, &g.NT, &g.TH);
    g.item0 = (int)plan->items.size();
    g.nitems = (int)costs[v].size();
    g.smem = gsmem[v];
    for (const Cost &c : costs[v]) plan->items.push_back(c.w);
    const void *fn = tile_kernel(v);
    int resident = 0;
    bf_status st = bfi::ensure_smem(fn, g.smem);
    if (st == BF_OK) st = bfi::resident_ctas(fn, g.NT, g.smem, &resident);
    if (st != BF_OK || resident < 1) return fail(st != BF_OK ? st : BF_ERR_UNSUPPORTED);
    g.ctas = (int)std::min<long long>((long long)resident, (long long)g.nitems);
    plan->tgroups.push_back(g);
  }

  // banded images: descriptors, groups of planes, tile items (longest first)
  size_t planes_max = 0;
  {
    struct BCost {
      double c;
      BandItem it;
    };
    size_t cur = 0;
    int slots = 0;  // images in the open group
    std::vector<BCost> vq, hq;
    std::vector<float> gtaps((size_t)kBandLaunchImages * kBandTapsMax, 0.f);
    auto close_group = [&]() {
      if (vq.empty()) return;
      auto by_cost = [](const BCost &a, const BCost &b) { return a.c > b.c; };
      std::stable_sort(vq.begin(), vq.end(), by_cost);
      std::stable_sort(hq.begin(), hq.end(), by_cost);
      BandGroup g{};
      g.v0 = (int)plan->bitems.size();
      g.nv = (int)vq.size();
      for (const BCost &b : vq) plan->bitems.push_back(b.it);
      g.h0 = (int)plan->bitems.size();
      g.nh = (int)hq.size();
      for (const BCost &b : hq) plan->bitems.push_back(b.it);
      for (const BCost &b : vq) {
        const bfi::FilterConsts &fc = plan->bdescs[b.it.desc].fc;
        g.vsmem = std::max(g.vsmem, bfk::vpass_smem(fc.kind, fc.R, fc.ntaps_pad));
        g.hsmem = std::max(g.hsmem, bfk::hpass_smem(fc.kind, fc.R, fc.ntaps_pad));
      }
      g.taps = gtaps;
      plan->groups.push_back(std::move(g));
      planes_max = std::max(planes_max, cur);
      vq.clear();
      hq.clear();
      cur = 0;
      slots = 0;
      std::fill(gtaps.begin(), gtaps.end(), 0.f);
    };
    // images of similar radii share a group: a launch's shared memory is sized
    // for its largest radius, so small-radius groups keep more CTAs resident
    std::stable_sort(large.begin(), large.end(), [&](int a, int b) {
      return plan->descs[a].fc.ntaps_pad < plan->descs[b].fc.ntaps_pad;
    });
    for (int i : large) {
      const BatchDesc &bd = plan->descs[i];
      const int H = bd.io.H, W = bd.io.W, Wp = (W + 3) / 4 * 4, N = bd.fc.N;
      const size_t pbytes = align256((size_t)(N + 1) * (size_t)H * (size_t)Wp * sizeof(float));
      if (cur > 0 && (cur + pbytes > kBatchPlaneCap || slots == kBandLaunchImages)) close_group();
      bfk::BandArgs a{};
      a.in = bd.io.in;
      a.out = bd.io.out;
      a.qaux = bd.io.qaux;
      a.ws = reinterpret_cast<float *>(static_cast<uintptr_t>(cur));  // offset, patched on device
      a.plane = (long long)H * Wp;
      a.Wp = Wp;
      a.H = H;
      a.W = W;
      a.pitch = bd.io.pitch;
      a.y0 = 0;
      a.rows = H;
      a.fc = bd.fc;
      const int di = (int)plan->bdescs.size();
      plan->bdescs.push_back(a);
      cur += pbytes;
      int slot = -1;
      if (bd.fc.ntaps_pad <= kBandTapsMax) {
        slot = slots;
        for (int k = 0; k < bd.fc.ntaps_pad; ++k) gtaps[(size_t)slot * kBandTapsMax + k] = bd.fc.taps[k];
      }
      ++slots;
      const double c = (N + 1.0) * (bd.fc.kind == BF_SPATIAL_GAUSS ? bd.fc.ntaps_pad : 8.0);
      for (int by = 0; by < (H + bfk::kVB - 1) / bfk::kVB; ++by)
        for (int bx = 0; bx < (Wp + bfk::kVC - 1) / bfk::kVC; ++bx) vq.push_back({c, {di, bx, by, slot}});
      for (int by = 0; by < (H + bfk::kHT - 1) / bfk::kHT; ++by)
        for (int bx = 0; bx < (W + bfk::kHW - 1) / bfk::kHW; ++bx) hq.push_back({c, {di, bx, by, slot}});
    }
    close_group();
  }
  if (plan->items.size() > 0x7fffffff || plan->bitems.size() > 0x7fffffff)
    return fail(BF_ERR_UNSUPPORTED);
  if (!large.empty()) {
    const int ntp_max = (2 * BF_MAX_RADIUS + 1 + 15) / 16 * 16;
    const size_t vs = std::max(bfk::vpass_smem(BF_SPATIAL_GAUSS, BF_MAX_RADIUS, ntp_max),
                               bfk::vpass_smem(BF_SPATIAL_BOX, BF_MAX_RADIUS, 0));
    const size_t hs = std::max(bfk::hpass_smem(BF_SPATIAL_GAUSS, BF_MAX_RADIUS, ntp_max),
                               bfk::hpass_smem(BF_SPATIAL_BOX, BF_MAX_RADIUS, 0));
    bf_status st = bfi::ensure_smem(reinterpret_cast<const void *>(gpa_batched_band_kernel<true>), vs);
    if (st == BF_OK)
      st = bfi::ensure_smem(reinterpret_cast<const void *>(gpa_batched_band_kernel<false>), hs);
    if (st != BF_OK) return fail(st);
  }
  // side streams for the whole-image launches and the banded groups
  const bool sides[2] = {!plan->whole.empty(), !plan->groups.empty()};
  if (sides[0] || sides[1]) {
    cudaError_t e = cudaEventCreateWithFlags(&plan->fork, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      if (!sides[k]) continue;
      e = cudaStreamCreateWithFlags(&plan->side[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(bfi::cuda_status(e));
  }
  plan->off_descs = 256;  // the first 256 bytes hold the tile groups' counters
  plan->off_items = align256(plan->off_descs + sizeof(BatchDesc) * plan->descs.size());
  plan->off_bdescs = align256(plan->off_items + sizeof(WorkItem) * plan->items.size());
  plan->off_bitems = align256(plan->off_bdescs + sizeof(bfk::BandArgs) * plan->bdescs.size());
  plan->off_planes = align256(plan->off_bitems + sizeof(BandItem) * plan->bitems.size());
  plan->ws_bytes = plan->off_planes + planes_max;
  plan->staging.assign(plan->off_planes - plan->off_descs, 0);
  unsigned char *st0 = plan->staging.data() - plan->off_descs;  // workspace offset -> staging
  memcpy(st0 + plan->off_descs, plan->descs.data(), sizeof(BatchDesc) * plan->descs.size());
  memcpy(st0 + plan->off_items, plan->items.data(), sizeof(WorkItem) * plan->items.size());
  memcpy(st0 + plan->off_bdescs, plan->bdescs.data(), sizeof(bfk::BandArgs) * plan->bdescs.size());
  memcpy(st0 + plan->off_bitems, plan->bitems.data(), sizeof(BandItem) * plan->bitems.size());
  *plan_out = plan;
  return BF_OK;
}

bf_status bf_batch_workspace(const bf_batch_plan *plan, size_t *bytes) {
  if (!plan || !bytes) return BF_ERR_INVALID_ARG;
  *bytes = plan->ws_bytes;
  return BF_OK;
}

bf_status bf_batch_info(const bf_batch_plan *plan, int *items, int *ctas) {
  if (!plan) return BF_ERR_INVALID_ARG;
  if (items) *items = (int)(plan->items.size() + plan->bitems.size() + plan->whole.size());
  if (ctas) {
    int c = 0;
    for (const TileGroup &g : plan->tgroups) c += g.ctas;
    *ctas = c;
  }
  return BF_OK;
}

bf_status bf_batch_variants(const bf_batch_plan *plan, int *variants, int count) {
  if (!plan || !variants || count != (int)plan->variants.size()) return BF_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) variants[i] = plan->variants[i];
  return BF_OK;
}

bf_status bf_batch_upload(const bf_batch_plan *plan, void *d_ws, size_t ws_bytes, void *stream) {
  if (!plan || !d_ws) return BF_ERR_INVALID_ARG;
  if (ws_bytes < plan->ws_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
    return BF_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(d_ws);
  cudaError_t e = cudaMemcpyAsync(base + plan->off_descs, plan->staging.data(),
                                  plan->staging.size(), cudaMemcpyHostToDevice, s);
  return bfi::cuda_status(e);
}

bf_status bf_batch_forward(const bf_batch_plan *plan, void *d_ws, size_t ws_bytes, int *d_status,
                           void *stream) {
  if (!plan || !d_ws) return BF_ERR_INVALID_ARG;
  if (ws_bytes < plan->ws_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
    return BF_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(d_ws);
  cudaError_t e = cudaSuccess;
  // fork: the side streams start after everything already on s
  if (plan->fork) {
    e = cudaEventRecord(plan->fork, s);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      if (plan->side[k]) e = cudaStreamWaitEvent(plan->side[k], plan->fork, 0);
    if (e != cudaSuccess) return bfi::cuda_status(e);
  }
  // whole-image kernels, one launch per image (side stream 0)
  for (const WholeImage &w : plan->whole) {
    const bf_status st = bf_fast_forward_variant(w.d.d_in, w.d.d_out, w.d.d_qaux, w.d.height,
                                                 w.d.width, w.d.pitch, &w.d.params, w.variant,
                                                 plan->side[0]);
    if (st != BF_OK) return st;
  }
  // banded groups (side stream 1)
  for (const BandGroup &g : plan->groups) {
    BandBatchArgs B;
    memcpy(B.taps, g.taps.data(), sizeof(B.taps));
    B.descs = reinterpret_cast<const bfk::BandArgs *>(base + plan->off_bdescs);
    B.planes = base + plan->off_planes;
    B.items = reinterpret_cast<const BandItem *>(base + plan->off_bitems) + g.v0;
    gpa_batched_band_kernel<true><<<g.nv, bfk::kVNT, g.vsmem, plan->side[1]>>>(B);
    bf_status st = bfi::check_launch();
    if (st != BF_OK) return st;
    B.items = reinterpret_cast<const BandItem *>(base + plan->off_bitems) + g.h0;
    gpa_batched_band_kernel<false><<<g.nh, bfk::kBandNT, g.hsmem, plan->side[1]>>>(B);
    st = bfi::check_launch();
    if (st != BF_OK) return st;
  }
  // one persistent launch per runtime-radius tile shape (caller's stream)
  if (!plan->tgroups.empty()) {
    int *counters = reinterpret_cast<int *>(base);
    e = cudaMemsetAsync(counters, 0, kMaxTileGroups * sizeof(int), s);
    if (e != cudaSuccess) return bfi::cuda_status(e);
    for (const TileGroup &g : plan->tgroups) {
      const bf_status sm = bfi::ensure_smem(tile_kernel(g.variant), g.smem);
      if (sm != BF_OK) return sm;
      BatchArgs A;
      A.descs = reinterpret_cast<const BatchDesc *>(base + plan->off_descs);
      A.items = reinterpret_cast<const WorkItem *>(base + plan->off_items) + g.item0;
      A.counter = counters + g.variant;
      A.status = d_status;
      A.count = (int)plan->descs.size();
      A.nitems = g.nitems;
      launch_tile_kernel(g.variant, g.ctas, g.smem, s, A);
      const bf_status st = bfi::check_launch();
      if (st != BF_OK) return st;
    }
  }
  // join
  for (int k = 0; k < 2; ++k) {
    if (!plan->side[k]) continue;
    e = cudaEventRecord(plan->join[k], plan->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->join[k], 0);
    if (e != cudaSuccess) return bfi::cuda_status(e);
  }
  return BF_OK;
}

void bf_batch_plan_destroy(bf_batch_plan *plan) { delete plan; }

bf_status bf_batch_graph_create(const bf_batch_plan *plan, void *d_ws, size_t ws_bytes,
                                int *d_status, void *stream, void **graph_exec_out) {
  if (!plan || !graph_exec_out || !stream) return BF_ERR_INVALID_ARG;
  *graph_exec_out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfi::cuda_status(e);
  bf_status st = bf_batch_forward(plan, d_ws, ws_bytes, d_status, stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(s, &graph);
  if (st != BF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return bfi::cuda_status(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfi::cuda_status(e);
  *graph_exec_out = exec;
  return BF_OK;
}

bf_status bf_graph_launch(void *graph_exec, void *stream) {
  if (!graph_exec) return BF_ERR_INVALID_ARG;
  return bfi::cuda_status(
      cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream)));
}

void bf_graph_destroy(void *graph_exec) {
  if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
}

}  // extern "C"
