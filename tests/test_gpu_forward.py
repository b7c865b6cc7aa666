"""GPU parity of the fused forward (bf_fast_forward) against the checker's
Algorithm 2 at the same N, element by element, at sizes spanning several
tiles with ragged tails; plus every tile variant, edge cases, the stored
planes, and sampled pixels at the full 2048^2 / 4096^2 workload sizes."""
import numpy as np
import pytest
import torch

import oracle
import paper_1603_08109_gb300 as bf
from helpers import compare_forward, image, needs_gpu, scaled_q, spatial

pytestmark = [pytest.mark.gpu, needs_gpu]

CASES = [
    # kind, radius, sigma_s, sigma_r, N, (H, W)
    (bf.GAUSS, 9, 3.0, 30.0, 40, (70, 500)),     # 256^2 workload's filter, several tiles
    (bf.GAUSS, 9, 3.0, 30.0, 2, (40, 300)),
    (bf.GAUSS, 30, 10.0, 60.0, 19, (90, 260)),
    (bf.GAUSS, 15, 5.0, 25.0, 54, (45, 470)),
    (bf.GAUSS, 9, 3.0, 10.0, 223, (34, 260)),
    (bf.BOX, 5, 0.0, 30.0, 41, (70, 520)),
    (bf.BOX, 20, 0.0, 60.0, 20, (60, 300)),
    (bf.BOX, 5, 0.0, 10.0, 226, (30, 270)),
    (bf.BOX, 50, 0.0, 60.0, 21, (40, 200)),
    (bf.BOX, 3, 0.0, 40.0, 1, (33, 100)),
]


def _run(img, kind, r, ss, sr, N, variant=-1):
    x = torch.from_numpy(img).cuda()
    out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True, variant=variant)
    torch.cuda.synchronize()
    return out.cpu().numpy(), q.cpu().numpy()


def _ref(img, kind, r, ss, sr, N):
    w = spatial(kind, r, ss)
    o, P, Q = oracle.gpa_alg2(img, w, sr, N, return_parts=True)
    return o, scaled_q(img, Q, sr), w[r, r]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "k%d_r%d_sr%g_N%d" % (c[0], c[1], c[3], c[4]))
def test_forward_matches_algorithm2(case):
    kind, r, ss, sr, N, (H, W) = case
    img = image(H, W, seed=H * 1000 + W)
    out, q = _run(img, kind, r, ss, sr, N)
    ro, rq, w0 = _ref(img, kind, r, ss, sr, N)
    compare_forward(out, q, ro, rq, w0, str(case), sigma_r=sr, N=N, img=img, w=spatial(kind, r, ss))


@pytest.mark.parametrize("variant", range(6))
def test_every_tile_variant(variant):
    img = image(50, 330, seed=77)
    ran = 0
    for kind, r, ss in ((bf.GAUSS, 9, 3.0), (bf.BOX, 7, 0.0), (bf.BOX, 5, 0.0)):
        ro, rq, w0 = _ref(img, kind, r, ss, 30.0, 40)
        try:
            out, q = _run(img, kind, r, ss, 30.0, 40, variant=variant)
        except bf._lib.BFError as e:  # the fixed-radius variant covers W in {3, 5, 9, 15} only
            assert e.status == 3 and variant == 5 and r == 7
            continue
        compare_forward(out, q, ro, rq, w0, "variant %d kind %d" % (variant, kind), sigma_r=30.0,
                        N=40, img=img, w=spatial(kind, r, ss))
        ran += 1
    assert ran >= 2


@pytest.mark.parametrize("variant", [6, 7])
@pytest.mark.parametrize("r", [3, 5])
def test_streaming_box_kernel(r, variant):
    """Variants 6 and 7 (warp-strip streaming box, 8 columns per lane for
    N <= 5, 4 columns per lane for N <= 8, halos from one or two lanes away):
    several strips and bands with
    ragged tails, every supported N, aligned (vector copies and stores) and
    odd-pitch (scalar) rows, widths that end inside a 4-column chunk, and
    images smaller than one strip or band."""
    H, W = 150, 500
    img = image(H, W, seed=40 + r)
    orders = ((40.0, 1), (40.0, 2), (60.0, 3), (80.0, 5), (30.0, 4))
    if variant == 7:
        orders += ((50.0, 6), (35.0, 7), (70.0, 8))
    for sr, N in orders:
        ro, rq, w0 = _ref(img, bf.BOX, r, 0.0, sr, N)
        out, q = _run(img, bf.BOX, r, 0.0, sr, N, variant=variant)
        compare_forward(out, q, ro, rq, w0, "stream v%d r=%d N=%d" % (variant, r, N), sigma_r=sr, N=N,
                        img=img, w=spatial(bf.BOX, r, 0.0))
    base = torch.zeros((H, W + 1), dtype=torch.float32, device="cuda")
    base[:, :W] = torch.from_numpy(img).cuda()
    o = bf.gpa_forward(base[:, :W], bf.BOX, 60.0, 3, radius=r, variant=variant)
    ro, rq, w0 = _ref(img, bf.BOX, r, 0.0, 60.0, 3)
    compare_forward(o.cpu().numpy(), None, ro, rq, w0, "stream odd pitch", sigma_r=60.0, N=3,
                    img=img, w=spatial(bf.BOX, r, 0.0))
    for shape in ((70, 517), (37, 243), (9, 5), (1, 1), (300, 3)):
        im = image(*shape, seed=shape[0] + shape[1], block=4)
        ro, rq, w0 = _ref(im, bf.BOX, r, 0.0, 70.0, 4)
        out, q = _run(im, bf.BOX, r, 0.0, 70.0, 4, variant=variant)
        compare_forward(out, q, ro, rq, w0, "stream v%d shape %s" % (variant, shape), sigma_r=70.0, N=4,
                        img=im, w=spatial(bf.BOX, r, 0.0))
    with pytest.raises(bf._lib.BFError):
        bf.gpa_forward(torch.from_numpy(img).cuda(), bf.BOX, 30.0, 6 if variant == 6 else 9,
                       radius=r, variant=variant)


@pytest.mark.parametrize("kind,r,ss,sr,N", [(bf.BOX, 3, 0.0, 40.0, 1), (bf.BOX, 5, 0.0, 60.0, 3),
                                             (bf.BOX, 3, 0.0, 35.0, 7), (bf.GAUSS, 9, 3.0, 30.0, 12)])
def test_forward_many(kind, r, ss, sr, N):
    """bf_fast_forward_many: a batch of images of one size in one call (one
    launch on the warp-strip box kernel, one per image on the tile kernels);
    each image is filtered on its own (zero extension at its edges), against
    the checker image by image and against single-image calls, with ragged
    strips and bands, odd image strides and padded rows (scalar copies)."""
    B, H, W = 3, 61, 301
    imgs = np.stack([image(H, W, seed=500 + 7 * k + r) for k in range(B)])
    x = torch.from_numpy(imgs).cuda()
    out, q = bf.gpa_forward_many(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
    padded = torch.zeros((B, H, W + 3), device="cuda")
    padded[:, :, :W] = x
    out_p = bf.gpa_forward_many(padded[:, :, :W], kind, sr, N, radius=r, sigma_s=ss)
    torch.cuda.synchronize()
    for k in range(B):
        ro, rq, w0 = _ref(imgs[k], kind, r, ss, sr, N)
        where = "many k=%d kind %d r=%d N=%d" % (k, kind, r, N)
        wk = spatial(kind, r, ss)
        compare_forward(out[k].cpu().numpy(), q[k].cpu().numpy(), ro, rq, w0, where, sigma_r=sr, N=N,
                        img=imgs[k], w=wk)
        compare_forward(out_p[k].cpu().numpy(), None, ro, rq, w0, where + " padded", sigma_r=sr, N=N,
                        img=imgs[k], w=wk)
        one, _ = _run(imgs[k], kind, r, ss, sr, N)
        assert np.abs(out[k].cpu().numpy() - one).max() <= 1e-3, where
    # the last image alone past a batch of one: count 1 behaves as bf_fast_forward
    o1 = bf.gpa_forward_many(x[2:], kind, sr, N, radius=r, sigma_s=ss)
    one, _ = _run(imgs[2], kind, r, ss, sr, N)
    assert np.abs(o1[0].cpu().numpy() - one).max() == 0.0
    import ctypes
    p = bf._lib.make_params(kind, r, ss, sr, N)
    ptr = ctypes.c_void_p(x.data_ptr())
    optr = ctypes.c_void_p(out.data_ptr())
    lib = bf._lib.lib()
    assert lib.bf_fast_forward_many(ptr, optr, None, 0, H * W, H, W, W, ctypes.byref(p), None) == 1
    assert lib.bf_fast_forward_many(ptr, optr, None, 2, H * W - 1, H, W, W, ctypes.byref(p), None) == 1


@pytest.mark.parametrize("kind,r,ss", [(bf.GAUSS, 12, 4.0), (bf.GAUSS, 20, 20 / 3.0),
                                       (bf.GAUSS, 60, 20.0), (bf.BOX, 20, 0.0), (bf.BOX, 50, 0.0)])
def test_banded_two_pass(kind, r, ss):
    """The banded two-pass forward (Gaussian radius >= 12, box > 15): several bands of 64 rows with
    a ragged last band, several column tiles with ragged edges, the band
    height from the default workspace, and Q'."""
    H, W = 150, 301
    img = image(H, W, seed=r + 7)
    sr, N = 60.0, 18
    ro, rq, w0 = _ref(img, kind, r, ss, sr, N)
    x = torch.from_numpy(img).cuda()
    assert bf.forward_workspace_bytes(H, W, kind, sr, N, radius=r, sigma_s=ss) > 0
    for band in (64, 128, None):
        out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True, band_rows=band)
        compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, rq, w0,
                        "banded kind %d r %d band %s" % (kind, r, band), sigma_r=sr, N=N,
                        img=img, w=spatial(kind, r, ss))


@pytest.mark.parametrize("r", [3, 5, 9, 15])
def test_fixed_radius_kernel(r):
    """The compile-time-radius kernel at every radius it is built for, both
    kinds, ragged sizes, small and large N (including N = 1 and 2)."""
    img = image(45, 600, seed=r)
    for kind, ss in ((bf.GAUSS, r / 3.0), (bf.BOX, 0.0)):
        for sr, N in ((30.0, 40), (60.0, 2), (40.0, 1), (12.0, 180)):
            ro, rq, w0 = _ref(img, kind, r, ss, sr, N)
            out, q = _run(img, kind, r, ss, sr, N, variant=5)
            compare_forward(out, q, ro, rq, w0, "fixed r=%d kind %d N=%d" % (r, kind, N),
                            sigma_r=sr, N=N, img=img, w=spatial(kind, r, ss))


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (5, 7), (3, 400), (300, 3)])
def test_tiny_and_thin_images_radius_beyond_image(shape):
    img = image(*shape, seed=5, block=2)
    for kind, r, ss in ((bf.GAUSS, 9, 3.0), (bf.BOX, 12, 0.0)):
        ro, rq, w0 = _ref(img, kind, r, ss, 30.0, 40)
        out, q = _run(img, kind, r, ss, 30.0, 40)
        compare_forward(out, q, ro, rq, w0, "shape %s kind %d" % (shape, kind), sigma_r=30.0, N=40,
                        img=img, w=spatial(kind, r, ss))


def test_constant_image_is_fixed_point():
    img = np.full((40, 300), 201.0, np.float32)
    for kind, r, ss in ((bf.GAUSS, 9, 3.0), (bf.BOX, 5, 0.0)):
        out, _ = _run(img, kind, r, ss, 30.0, 40)
        assert np.abs(out - 201.0).max() <= 1e-3


def test_pitched_input_and_cpu_tensor_roundtrip():
    img = image(40, 150, seed=9)
    base = torch.zeros((40, 160), dtype=torch.float32, device="cuda")
    base[:, :150] = torch.from_numpy(img).cuda()
    view = base[:, :150]
    assert view.stride(0) == 160
    out = bf.gpa_forward(view, bf.GAUSS, 30.0, 40, radius=9, sigma_s=3.0)
    ro, rq, w0 = _ref(img, bf.GAUSS, 9, 3.0, 30.0, 40)
    compare_forward(out.cpu().numpy(), None, ro, rq, w0, "pitched", sigma_r=30.0, N=40, img=img,
                    w=spatial(bf.GAUSS, 9, 3.0))
    out_cpu = bf.gpa_forward(torch.from_numpy(img), bf.GAUSS, 30.0, 40, radius=9, sigma_s=3.0)
    assert out_cpu.device.type == "cpu"
    assert torch.equal(out_cpu, out.cpu())


@pytest.mark.parametrize("kind,r,ss,shape", [(bf.GAUSS, 6, 2.0, (40, 280)),
                                              (bf.GAUSS, 9, 3.0, (37, 500)),
                                              (bf.BOX, 5, 0.0, (19, 250))])
def test_stored_planes_match_filtered_images(kind, r, ss, shape):
    """bf_fast_forward_stored plane n = Fbar_n / sqrt(n!) (the rescaled
    filtered image of Algorithm 2), and out is bitwise the plain forward's:
    the runtime-radius kernel (radius 6) and the compile-time-radius kernel
    with its row-wise staged plane stores (radii 9 and 5, several tiles)."""
    img = image(*shape, seed=31 + r)
    sr, N = 30.0, 30
    w = spatial(kind, r, ss)
    _, _, _, planes = oracle.gpa_alg2(img, w, sr, N, return_parts=True, return_planes=True)
    x = torch.from_numpy(img).cuda()
    out_s, q_s, abar = bf.gpa_forward_stored(x, kind, sr, N, radius=r, sigma_s=ss)
    out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
    assert torch.equal(out_s, out) and torch.equal(q_s, q)
    ab = abar.cpu().numpy()
    from math import lgamma, exp
    for n in range(N + 1):
        ref = planes[n] / np.sqrt(exp(lgamma(n + 1)))
        assert np.abs(ab[n] - ref).max() <= 2e-6 + 1e-5 * np.abs(ref).max(), n


def _sampled_case(H, W, gen, kind, r, ss, sr, N, nsamp, seed):
    img = gen(H, W, seed)
    x = torch.from_numpy(img).cuda()
    out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    ys = np.concatenate([rng.integers(0, H, nsamp), [0, 0, H - 1, H - 1, H // 2]])
    xs = np.concatenate([rng.integers(0, W, nsamp), [0, W - 1, 0, W - 1, W // 2]])
    w = spatial(kind, r, ss)
    ro, P, Q = oracle.gpa_alg2_at(img, w, sr, N, (ys, xs), return_parts=True)
    rq = scaled_q(img[ys, xs], Q, sr)
    o = out[ys, xs].cpu().numpy()
    qq = q[ys, xs].cpu().numpy()
    return compare_forward(o, qq, ro, rq, w[r, r], "sampled %dx%d" % (H, W), sigma_r=sr, N=N,
                           img=img, w=w, pixels=(ys, xs))


def test_full_size_2048_sampled():
    """2048^2 blocks (64) + noise 10 at the benchmark's launch configuration."""
    gen = lambda h, w, s: image(h, w, s, block=64, noise=10.0)  # noqa: E731
    _sampled_case(2048, 2048, gen, bf.GAUSS, 9, 3.0, 30.0, 40, 400, 1000)
    _sampled_case(2048, 2048, gen, bf.BOX, 20, 0.0, 30.0, 44, 300, 1001)


def test_full_size_4096_sampled_gradient_polygons():
    from paper_1603_08109_gb300 import synth
    gen = lambda h, w, s: synth.gradient_polygons_image(h, w, 64, 15.0, seed=s)  # noqa: E731
    _sampled_case(4096, 4096, gen, bf.BOX, 5, 0.0, 40.0, 3, 300, 2000)
    _sampled_case(4096, 4096, gen, bf.GAUSS, 60, 20.0, 40.0, 32, 60, 2001)
