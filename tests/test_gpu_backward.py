"""GPU gradients: the fast filter's adjoint (recompute and stored variants)
and the direct filter's gradient, against the checker's exact derivatives
of eq. GPA / eq. BF, central finite differences of the GPU forward, and the
direct filter's FP64 gradient."""
import numpy as np
import pytest
import torch

import oracle
import paper_1603_08109_gb300 as bf
from helpers import image, needs_gpu, spatial
from paper_1603_08109_gb300 import synth

pytestmark = [pytest.mark.gpu, needs_gpu]

GIN_RTOL = 2e-3   # relative to max |gradient|
GSIG_RTOL = 1e-3


def _fast_grads(img, g, kind, r, ss, sr, N, store=False):
    x = torch.from_numpy(img).cuda()
    if store:
        out, q, abar = bf.gpa_forward_stored(x, kind, sr, N, radius=r, sigma_s=ss)
    else:
        out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
        abar = None
    gin, gs = bf.gpa_backward(x, out, q, torch.from_numpy(g).cuda(), kind, sr, N, radius=r,
                              sigma_s=ss, abar=abar)
    torch.cuda.synchronize()
    return gin.cpu().numpy().astype(np.float64), float(gs.item())


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("case", [
    (bf.GAUSS, 9, 3.0, 30.0, 40, (40, 300)),
    (bf.GAUSS, 15, 5.0, 25.0, 54, (40, 130)),
    (bf.GAUSS, 6, 2.0, 60.0, 8, (25, 90)),
    (bf.BOX, 5, 0.0, 30.0, 41, (30, 270)),
    (bf.BOX, 9, 0.0, 40.0, 25, (21, 60)),
], ids=lambda c: "k%d_r%d_sr%g_N%d" % (c[0], c[1], c[3], c[4]))
def test_fast_backward_matches_exact_derivatives(case):
    kind, r, ss, sr, N, (H, W) = case
    img = image(H, W, seed=H * 31 + W)
    g = synth.random_like((H, W), seed=H + W)
    gin, gs = _fast_grads(img, g, kind, r, ss, sr, N)
    rgin, rgs = oracle.gpa_grad(img, spatial(kind, r, ss), sr, N, g.astype(np.float64))
    assert _rel(gin, rgin) <= GIN_RTOL
    assert abs(gs - rgs) <= GSIG_RTOL * abs(rgs)
    # stored planes vs recompute: same math, float32 (for radii 3, 5, 9, 15 both
    # run the compile-time-radius kernels; otherwise the stored planes go
    # through the runtime-radius kernel and the sums are associated differently)
    gin2, gs2 = _fast_grads(img, g, kind, r, ss, sr, N, store=True)
    assert _rel(gin2, gin) <= 1e-4
    assert abs(gs2 - gs) <= 1e-4 * abs(gs)
    assert abs(gs2 - rgs) <= GSIG_RTOL * abs(rgs)


@pytest.mark.parametrize("case", [
    (bf.GAUSS, 3, 1.0, 30.0, 37, (70, 301)),
    (bf.GAUSS, 5, 5 / 3.0, 40.0, 25, (33, 250)),
    (bf.GAUSS, 9, 3.0, 30.0, 40, (17, 229)),
    (bf.GAUSS, 15, 5.0, 25.0, 54, (41, 200)),
    (bf.BOX, 3, 0.0, 30.0, 41, (26, 127)),
    (bf.BOX, 15, 0.0, 50.0, 22, (9, 333)),
], ids=lambda c: "k%d_r%d" % (c[0], c[1]))
def test_stored_fixed_radius_backward(case):
    """The stored-plane pair at the compile-time radii: the forward stages each
    plane through shared memory and writes whole rows, the backward copies
    each channel's plane block into shared memory and filters only the
    adjoint seeds.  Images several tiles wide (238 and 110 output columns per
    tile) and tall with ragged edges; gradients against recompute and against
    the checker's exact derivatives.  The recompute kernel carries the powers
    unnormalised (a_n = s_n ã_n) where the stored planes hold the normalised
    a_n, so the two are different float32 roundings of the same sums: each
    sigma_r gradient lies within about 2e-5 (relative) of the exact one, and
    the two agree to 1e-4."""
    kind, r, ss, sr, N, (H, W) = case
    img = image(H, W, seed=H * 13 + W)
    g = synth.random_like((H, W), seed=H * W)
    gin, gs = _fast_grads(img, g, kind, r, ss, sr, N)
    gin2, gs2 = _fast_grads(img, g, kind, r, ss, sr, N, store=True)
    assert _rel(gin2, gin) <= 1e-5
    assert abs(gs2 - gs) <= 1e-4 * abs(gs)
    rgin, rgs = oracle.gpa_grad(img, spatial(kind, r, ss), sr, N, g.astype(np.float64))
    assert _rel(gin2, rgin) <= GIN_RTOL
    assert abs(gs2 - rgs) <= GSIG_RTOL * abs(rgs)


@pytest.mark.parametrize("case", [
    (bf.GAUSS, 20, 20 / 3.0, 60.0, 18, (150, 173)),
    (bf.GAUSS, 60, 20.0, 60.0, 12, (140, 150)),
    (bf.BOX, 25, 0.0, 60.0, 18, (150, 131)),
], ids=lambda c: "k%d_r%d" % (c[0], c[1]))
def test_banded_backward(case):
    """The banded two-pass backward (radius > 15) against the checker's exact
    derivatives, with the workspace from the query (one band) and with smaller
    workspaces (several bands of 64 or 128 rows); W = 60 is beyond what the
    fused runtime-radius backward supports."""
    import ctypes
    from paper_1603_08109_gb300 import _lib
    kind, r, ss, sr, N, (H, W) = case
    img = image(H, W, seed=H * 7 + W)
    g = synth.random_like((H, W), seed=H + 2 * W)
    rgin, rgs = oracle.gpa_grad(img, spatial(kind, r, ss), sr, N, g.astype(np.float64))
    x = torch.from_numpy(img).cuda()
    out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
    gt = torch.from_numpy(g).cuda()
    p = _lib.make_params(kind, r, ss, sr, N)
    lib = _lib.lib()
    need = ctypes.c_size_t()
    assert lib.bf_fast_backward_workspace(H, W, ctypes.byref(p), ctypes.byref(need)) == 0
    band_bytes = 3 * (N + 1) * 64 * ((W + 3) // 4 * 4) * 4   # 64 rows of band planes
    ran = 0
    for nbytes in (need.value, need.value - band_bytes, need.value - 2 * band_bytes):
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        gin = torch.empty_like(x)
        gs = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = lib.bf_fast_backward(x.data_ptr(), out.data_ptr(), q.data_ptr(), gt.data_ptr(),
                                  gin.data_ptr(), gs.data_ptr(), H, W, W, ctypes.byref(p),
                                  ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
        if st == 5 and r > 52:
            continue  # below 64 band rows, and no fused fallback at this radius
        assert st == 0, st
        torch.cuda.synchronize()
        assert _rel(gin.cpu().numpy().astype(np.float64), rgin) <= GIN_RTOL, nbytes
        assert abs(float(gs.item()) - rgs) <= GSIG_RTOL * abs(rgs), nbytes
        ran += 1
    assert ran >= 2
    # through autograd: the default path for this radius
    xg = x.clone().requires_grad_(True)
    srt = torch.tensor(sr, dtype=torch.float64, device="cuda", requires_grad=True)
    y = bf.gpa_bilateral(xg, srt, kind, N, radius=r, sigma_s=ss)
    (y * gt).sum().backward()
    assert _rel(xg.grad.cpu().numpy().astype(np.float64), rgin) <= GIN_RTOL
    assert abs(float(srt.grad.item()) - rgs) <= GSIG_RTOL * abs(rgs)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (5, 7), (3, 300), (260, 3)])
def test_fast_backward_tiny_and_thin_images(shape):
    """Radius beyond the image, single rows/columns, ragged tiles: both the
    compile-time-radius (W=9) and the runtime-radius (W=12) backward."""
    img = image(*shape, seed=7, block=2)
    g = synth.random_like(shape, seed=8)
    for kind, r, ss, sr, N in ((bf.GAUSS, 9, 3.0, 30.0, 40), (bf.BOX, 12, 0.0, 30.0, 44)):
        gin, gs = _fast_grads(img, g, kind, r, ss, sr, N)
        rgin, rgs = oracle.gpa_grad(img, spatial(kind, r, ss), sr, N, g.astype(np.float64))
        assert _rel(gin, rgin) <= GIN_RTOL, (shape, kind)
        # absolute floor: a 1x1 image has an exactly zero sigma_r gradient
        assert abs(gs - rgs) <= GSIG_RTOL * abs(rgs) + 1e-4, (shape, kind)


def test_fast_backward_deterministic_and_autograd():
    img = image(40, 200, seed=3)
    g = synth.random_like(img.shape, seed=4)
    a = _fast_grads(img, g, bf.GAUSS, 9, 3.0, 30.0, 40)
    b = _fast_grads(img, g, bf.GAUSS, 9, 3.0, 30.0, 40)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    x = torch.from_numpy(img).cuda().requires_grad_(True)
    s = torch.tensor(30.0, device="cuda", requires_grad=True)
    out = bf.gpa_bilateral(x, s, kind=bf.GAUSS, N=40, radius=9, sigma_s=3.0)
    (out * torch.from_numpy(g).cuda()).sum().backward()
    assert np.array_equal(x.grad.cpu().numpy().astype(np.float64), a[0])
    assert float(s.grad) == pytest.approx(a[1], rel=1e-6)


def test_fast_backward_finite_differences_of_gpu_forward():
    """Central differences of the GPU forward, loss <r, out> accumulated in
    FP64.  Image: step h = 1e-2 along a direction d built from the analytic
    gradient's signs times random magnitudes, so that the directional
    derivative (order of the pixel count) dominates the float32 rounding
    noise of the forward (about sqrt(pixels) * 1e-5 / h).  sigma_r: step 0.25
    (1% of sigma_r; truncation error O(1e-4) relative)."""
    H, W = 64, 96
    img = image(H, W, seed=8)
    kind, r, ss, sr, N = bf.GAUSS, 15, 5.0, 25.0, 54
    rr = synth.random_like((H, W), seed=9).astype(np.float64)

    def loss(x, s):
        o = bf.gpa_forward(torch.from_numpy(x).cuda(), kind, s, N, radius=r, sigma_s=ss)
        return float(np.sum(rr * o.cpu().numpy().astype(np.float64)))

    gin, gs = _fast_grads(img, rr.astype(np.float32), kind, r, ss, sr, N)
    mag = np.abs(synth.random_like((H, W), seed=10)).astype(np.float64)
    d = (np.sign(gin) * mag).astype(np.float32)
    h = 1e-2
    fd = (loss(img + h * d, sr) - loss(img - h * d, sr)) / (2 * h)
    an = float(np.sum(gin * d))
    assert an == pytest.approx(fd, rel=2e-3)
    hs = 0.25
    fds = (loss(img, sr + hs) - loss(img, sr - hs)) / (2 * hs)
    assert gs == pytest.approx(fds, rel=2e-3)


def test_fast_gradient_approaches_direct_gradient():
    """At the order from delta the fast gradient is close to the exact
    FP64 gradient of eq. BF (and the gap shrinks with N)."""
    img = image(30, 60, seed=12)
    g = synth.random_like(img.shape, seed=13)
    kind, r, ss, sr = bf.GAUSS, 6, 2.0, 30.0
    w = spatial(kind, r, ss)
    dgin, dgs = oracle.bf_direct_grad(img, w, sr, g.astype(np.float64))
    errs = []
    for N in (25, 40, 55):
        gin, gs = _fast_grads(img, g, kind, r, ss, sr, N)
        errs.append(_rel(gin, dgin))
    assert errs[2] < errs[0]
    assert errs[2] <= 5e-3


@pytest.mark.parametrize("case", [
    (bf.GAUSS, 9, 3.0, 30.0, (40, 150)),
    (bf.BOX, 5, 0.0, 20.0, (30, 100)),
    (bf.GAUSS, 15, 5.0, 25.0, (33, 70)),
])
def test_direct_backward_matches_exact_derivatives(case):
    kind, r, ss, sr, (H, W) = case
    img = image(H, W, seed=H + W)
    g = synth.random_like((H, W), seed=2 * H)
    x = torch.from_numpy(img).cuda()
    gin, gs = bf.direct_backward(x, torch.from_numpy(g).cuda(), kind, sr, radius=r, sigma_s=ss)
    rgin, rgs = oracle.bf_direct_grad(img, spatial(kind, r, ss), sr, g.astype(np.float64))
    assert _rel(gin.cpu().numpy().astype(np.float64), rgin) <= GIN_RTOL
    assert abs(float(gs.item()) - rgs) <= GSIG_RTOL * abs(rgs)
    xs = x.clone().requires_grad_(True)
    s = torch.tensor(sr, device="cuda", requires_grad=True)
    (bf.direct_bilateral(xs, s, kind=kind, radius=r, sigma_s=ss) * torch.from_numpy(g).cuda()).sum().backward()
    assert torch.equal(xs.grad, gin)


def test_backward_full_size_512_sampled():
    """One 512^2 image of the differentiated workload (Gaussian sigma_s = 5,
    sigma_r = 25, N = 54): image gradient at sampled pixels and sigma_r."""
    H = W = 512
    img = image(H, W, seed=4000)
    g = synth.random_like((H, W), seed=4001)
    kind, r, ss, sr, N = bf.GAUSS, 15, 5.0, 25.0, 54
    gin, gs = _fast_grads(img, g, kind, r, ss, sr, N)
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.integers(0, H, 12), [0, H - 1]])
    xs = np.concatenate([rng.integers(0, W, 12), [W - 1, 0]])
    rgin, _ = oracle.gpa_grad(img, spatial(kind, r, ss), sr, N, g.astype(np.float64),
                              samples=(ys, xs))
    scale = np.abs(gin).max()
    assert np.abs(gin[ys, xs] - rgin).max() <= GIN_RTOL * scale


@pytest.mark.parametrize("kind,r,ss,sr", [(bf.GAUSS, 3, 1.0, 35.0), (bf.GAUSS, 9, 3.0, 30.0),
                                          (bf.GAUSS, 15, 5.0, 45.0), (bf.BOX, 9, 0.0, 40.0)],
                         ids=lambda v: str(v))
def test_compile_time_radius_backward_orders(kind, r, ss, sr):
    """The compile-time-radius backward carries the powers unnormalised and
    resets their scale every 8 channels: orders that end before, on and just
    after a reset (and N = 1, 2, a long run at N = 200, the largest order at
    W = 3, where the scale s_n is smallest) against the checker's exact
    derivatives, on a ragged image several tiles wide.

    The sigma_r gradient is a sum over pixels of g (out - t_c) / sigma_r -
    Hbar H / sigma_r whose terms can nearly cancel (at W = 9, N = 33 it is
    1.6e-6 of the sum of their magnitudes S); float32 terms then fix it only
    to a few units of 2^-24 S, so its bar is 1e-3 of the exact value plus
    2^-24 S (the conditioning allowance of the forward's bar, from the terms'
    magnitudes)."""
    H, W = 23, 251
    img = image(H, W, seed=400 + r)
    g = synth.random_like((H, W), seed=401 + r)
    w = spatial(kind, r, ss)
    orders = (1, 2, 7, 8, 9, 16, 17, 33, 200) + ((1024,) if r == 3 else ())  # BF_MAX_ORDER
    for N in orders:
        gin, gs = _fast_grads(img, g, kind, r, ss, sr, N)
        rgin, rgs = oracle.gpa_grad(img, w, sr, N, g.astype(np.float64))
        assert _rel(gin, rgin) <= GIN_RTOL, (N, _rel(gin, rgin))
        ro = oracle.gpa_definition(img, w, sr, N)  # eq. GPA: Algorithm 2's output, any N
        S = (np.abs(g * (ro - 128.0)).sum() + np.abs(rgin * (img - 128.0)).sum()) / sr
        assert abs(gs - rgs) <= GSIG_RTOL * abs(rgs) + 2.0 ** -24 * S, (N, gs, rgs, S)


def test_backward_concurrent_streams_match_sequential():
    """Backward launches on four streams at once (their CTAs share the SMs'
    tensor memory) give bitwise the results of the same calls one after
    another."""
    S, N = 700, 40
    imgs = [torch.from_numpy(image(S, S + 37 * k, seed=500 + k)).cuda() for k in range(4)]
    gs = [torch.from_numpy(synth.random_like(tuple(x.shape), seed=510 + k)).cuda()
          for k, x in enumerate(imgs)]
    fw = [bf.gpa_forward(x, bf.GAUSS, 30.0, N, radius=9, sigma_s=3.0, return_q=True) for x in imgs]
    seq = [bf.gpa_backward(x, o, q, g, bf.GAUSS, 30.0, N, radius=9, sigma_s=3.0)
           for x, (o, q), g in zip(imgs, fw, gs)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in imgs]
    for _ in range(3):
        par = [None] * len(imgs)
        for k, (s, x, (o, q), g) in enumerate(zip(streams, imgs, fw, gs)):
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                par[k] = bf.gpa_backward(x, o, q, g, bf.GAUSS, 30.0, N, radius=9, sigma_s=3.0)
        torch.cuda.synchronize()
        for (a_gin, a_gs), (b_gin, b_gs) in zip(seq, par):
            assert torch.equal(a_gin, b_gin)
            assert float(a_gs.item()) == float(b_gs.item())
