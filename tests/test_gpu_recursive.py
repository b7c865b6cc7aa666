"""GPU parity of the recursive-Gaussian path (bf_recursive_gauss,
bf_recursive_forward, bf_recursive_backward) against the checker's full-line
Toeplitz-product evaluation (oracle.recursive), which is the zero-extended
convolution with Deriche's fit written out, and its FP64 reverse-mode
gradient.

Sizes span several 32-pixel carry tiles in both directions with ragged last
tiles, single-row / single-column / single-pixel images, pitched rows, the
smallest accepted sigma_s and sigma_s far above the tile length (the carries
then cross many tiles)."""
import numpy as np
import pytest
import torch

import paper_1603_08109_gb300 as bf
from helpers import compare_forward, image, needs_gpu, scaled_q
from oracle import recursive as rec
from paper_1603_08109_gb300 import synth

pytestmark = [pytest.mark.gpu, needs_gpu]

# plain filter: FP32 recursions over values in [0, 255]; the complex one-pole
# form keeps the error near 1e-6 of the largest value
FILTER_RTOL = 1e-5


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (45, 1), (5, 7), (33, 65), (97, 301),
                                   (256, 200)])
@pytest.mark.parametrize("s", [0.5, 2.5, 9.0, 40.0])
def test_recursive_filter(shape, s):
    img = image(*shape, seed=shape[0] * 7 + shape[1], block=8)
    out = bf.recursive_gauss(torch.from_numpy(img).cuda(), s).cpu().numpy().astype(np.float64)
    ref = rec.recursive_filter(img, s)
    scale = max(np.abs(ref).max(), 1e-30)
    assert np.abs(out - ref).max() <= FILTER_RTOL * scale, (shape, s)


def test_recursive_filter_impulse_and_pitch():
    """A unit impulse gives the separable kernel h(j_y) h(j_x) itself; a
    pitched (non-contiguous) view gives the same result as a packed copy."""
    s = 6.0
    H, W = 81, 95
    img = np.zeros((H, W), np.float32)
    img[40, 47] = 1.0
    out = bf.recursive_gauss(torch.from_numpy(img).cuda(), s).cpu().numpy().astype(np.float64)
    h = rec.deriche_impulse(s, 100)
    ref = np.outer(h[np.abs(np.arange(H) - 40)], h[np.abs(np.arange(W) - 47)])
    assert np.abs(out - ref).max() <= 1e-5 * ref.max()
    base = torch.zeros((70, 131), device="cuda")
    im2 = image(70, 120, seed=3)
    base[:, :120] = torch.from_numpy(im2).cuda()
    o1 = bf.recursive_gauss(base[:, :120], 3.0)
    o2 = bf.recursive_gauss(base[:, :120].contiguous(), 3.0)
    torch.testing.assert_close(o1, o2, rtol=0, atol=0)


CASES = [  # (sigma_s, sigma_r, shape)
    (1.5, 30.0, (70, 130)),
    (5.0, 60.0, (64, 64)),
    (20.0, 40.0, (97, 211)),
    (3.0, 25.0, (33, 1)),
    (0.5, 50.0, (1, 90)),
]


@pytest.mark.parametrize("s,sr,shape", CASES)
def test_recursive_forward(s, sr, shape):
    img = image(*shape, seed=int(s * 10) + shape[1], block=6)
    w0 = rec.centre_weight_recursive(s)
    assert bf.centre_weight(bf.GAUSS_RECURSIVE, 0, s) == pytest.approx(w0, rel=1e-6)
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    out, q = bf.recursive_forward(torch.from_numpy(img).cuda(), sr, N, s, return_q=True)
    ro, P, Q = rec.gpa_alg2_recursive(img, s, sr, N, return_parts=True)
    compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, scaled_q(img, Q, sr), w0,
                    "recursive s=%g sr=%g N=%d %s" % (s, sr, N, shape), sigma_r=sr, N=N)


def test_recursive_forward_small_orders_and_ws_reuse():
    """Orders below the bound (N = 1, 2, 3) and a reused workspace tensor."""
    img = image(50, 77, seed=9)
    s = 4.0
    w0 = rec.centre_weight_recursive(s)
    x = torch.from_numpy(img).cuda()
    ws = torch.empty(bf.recursive_workspace_bytes(50, 77, 3) // 4, device="cuda")
    for sr, N in ((40.0, 1), (40.0, 2), (60.0, 3)):
        out, q = bf.recursive_forward(x, sr, N, s, return_q=True, ws=ws)
        ro, P, Q = rec.gpa_alg2_recursive(img, s, sr, N, return_parts=True)
        compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, scaled_q(img, Q, sr), w0,
                        "recursive small N=%d" % N, sigma_r=sr, N=N)


def test_recursive_full_size_sampled_rows():
    """8192^2-style content at 2048^2 (the launch configuration of the
    benchmark's recursive sweep): rows sampled across the image, including
    the first and last, against the checker's rows."""
    H = W = 2048
    s, sr = 20.0, 40.0
    img = synth.gradient_polygons_image(H, W, 64, 15.0, seed=2001)
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 0.5)
    out, q = bf.recursive_forward(torch.from_numpy(img).cuda(), sr, N, s, return_q=True)
    rows = [0, 1, 31, 32, 777, 1024, 2016, 2047]
    ro, P, Q = rec.gpa_alg2_recursive(img, s, sr, N, rows=rows, return_parts=True)
    w0 = rec.centre_weight_recursive(s)
    compare_forward(out.cpu().numpy()[rows], q.cpu().numpy()[rows], ro,
                    scaled_q(img[rows], Q, sr), w0, "recursive 2048^2 rows", sigma_r=sr, N=N)


def test_recursive_errors():
    x = torch.from_numpy(image(20, 30, seed=1)).cuda()
    with pytest.raises(bf._lib.BFError) as e:
        bf.recursive_gauss(x, 0.4)
    assert e.value.status == 1
    with pytest.raises(bf._lib.BFError) as e:
        bf.recursive_forward(x, 5.0, 10, 3.0)  # t_c / sigma_r > 13
    assert e.value.status == 3
    # the fused entry points reject the recursive kind
    with pytest.raises(bf._lib.BFError) as e:
        bf.gpa_forward(x, bf.GAUSS_RECURSIVE, 40.0, 10, sigma_s=3.0)
    assert e.value.status == 1
    # too small a workspace
    p = bf._lib.make_params(bf.GAUSS_RECURSIVE, 0, 3.0, 40.0, 10)
    o = torch.empty_like(x)
    need = bf.recursive_workspace_bytes(20, 30, 10)
    ws = torch.empty(need // 4, device="cuda")
    import ctypes
    st = bf._lib.lib().bf_recursive_forward(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(o.data_ptr()), None, 20, 30, 30,
        ctypes.byref(p), ctypes.c_void_p(ws.data_ptr()), need - 256, None)
    assert st == 5


GRAD_CASES = [  # (sigma_s, sigma_r, shape)
    (1.5, 30.0, (40, 70)),
    (5.0, 60.0, (64, 64)),
    (20.0, 40.0, (50, 97)),
    (3.0, 25.0, (33, 1)),
    (0.5, 50.0, (1, 90)),
]


@pytest.mark.parametrize("s,sr,shape", GRAD_CASES)
def test_recursive_backward(s, sr, shape):
    """bf_recursive_backward against the checker's FP64 reverse-mode gradient
    of the same Algorithm 2 (image: 2e-3 of the largest entry; sigma_r: 1e-3
    relative), through the autograd wrapper as well."""
    img = image(*shape, seed=int(s * 7) + shape[0], block=5)
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    g = synth.random_like(shape, seed=shape[1] + 3)
    rgin, rgs = rec.gpa_grad_recursive(img, s, sr, N, g.astype(np.float64))
    x = torch.from_numpy(img).cuda()
    out, q = bf.recursive_forward(x, sr, N, s, return_q=True)
    gin, gs = bf.recursive_backward(x, out, q, torch.from_numpy(g).cuda(), sr, N, s)
    torch.cuda.synchronize()
    scale = max(np.abs(rgin).max(), 1e-30)
    where = "s=%g sr=%g N=%d %s" % (s, sr, N, shape)
    assert np.abs(gin.cpu().numpy() - rgin).max() <= 2e-3 * scale, where
    assert abs(float(gs.item()) - rgs) <= max(1e-3 * abs(rgs), 1e-4), where
    # the autograd wrapper
    xin = x.clone().requires_grad_(True)
    sig = torch.tensor(sr, dtype=torch.float32, device="cuda", requires_grad=True)
    (bf.recursive_bilateral(xin, sig, s, N=N) * torch.from_numpy(g).cuda()).sum().backward()
    assert np.abs(xin.grad.cpu().numpy() - rgin).max() <= 2e-3 * scale, where
    assert abs(float(sig.grad) - rgs) <= max(1e-3 * abs(rgs), 1e-4), where


def test_recursive_backward_pitched_and_errors():
    """A pitched image gives the same gradient as its packed copy (the wrapper
    packs mismatched layouts); too small a workspace is rejected."""
    import ctypes
    H, W, s, sr = 45, 80, 4.0, 40.0
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    base = torch.zeros((H, W + 3), device="cuda")
    base[:, :W] = torch.from_numpy(image(H, W, seed=4)).cuda()
    x = base[:, :W]
    out, q = bf.recursive_forward(x, sr, N, s, return_q=True)
    g = torch.from_numpy(synth.random_like((H, W), seed=6)).cuda()
    gin, gs = bf.recursive_backward(x, out, q, g, sr, N, s)
    gin2, gs2 = bf.recursive_backward(x.contiguous(), out, q, g, sr, N, s)
    torch.testing.assert_close(gin, gin2, rtol=0, atol=0)
    assert float(gs.item()) == float(gs2.item())
    n = ctypes.c_size_t(0)
    assert bf._lib.lib().bf_recursive_backward_workspace(H, W, N, ctypes.byref(n)) == 0
    p = bf._lib.make_params(bf.GAUSS_RECURSIVE, 0, s, sr, N)
    xc = x.contiguous()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    ws = torch.empty(n.value // 4, device="cuda")
    st = bf._lib.lib().bf_recursive_backward(ptr(xc), ptr(out), ptr(q), ptr(g), ptr(gin), None, H, W,
                                             W, ctypes.byref(p), ptr(ws), n.value - 256, None)
    assert st == 5


@pytest.mark.parametrize("s,sr,shape", [(3.0, 30.0, (97, 130)), (15.0, 45.0, (64, 33)),
                                        (0.5, 60.0, (1, 70))])
def test_recursive_stored_pair(s, sr, shape):
    """The stored pair keeps the power images' row-pass planes from the
    forward for the backward: out, Q' and both gradients equal the recompute
    pair's bitwise (the same kernels on the same data), for two cotangents
    from one stored forward, through the autograd wrapper as well; and the
    gradient matches the checker's FP64 reverse-mode gradient."""
    img = image(*shape, seed=int(s * 11) + shape[1], block=5)
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    x = torch.from_numpy(img).cuda()
    out, q = bf.recursive_forward(x, sr, N, s, return_q=True)
    so, sq, ws = bf.recursive_forward_stored(x, sr, N, s)
    torch.cuda.synchronize()
    where = "s=%g sr=%g N=%d %s" % (s, sr, N, shape)
    torch.testing.assert_close(so, out, rtol=0, atol=0, msg=where)
    torch.testing.assert_close(sq, q, rtol=0, atol=0, msg=where)
    for seed in (41, 42):
        g = torch.from_numpy(synth.random_like(shape, seed=seed)).cuda()
        gin, gs = bf.recursive_backward(x, out, q, g, sr, N, s)
        sgin, sgs = bf.recursive_backward_stored(x, so, sq, g, sr, N, s, ws)
        torch.cuda.synchronize()
        torch.testing.assert_close(sgin, gin, rtol=0, atol=0, msg=where)
        assert float(sgs.item()) == float(gs.item()), where
    rgin, rgs = rec.gpa_grad_recursive(img, s, sr, N, g.cpu().numpy().astype(np.float64))
    scale = max(np.abs(rgin).max(), 1e-30)
    assert np.abs(sgin.cpu().numpy() - rgin).max() <= 2e-3 * scale, where
    assert abs(float(sgs.item()) - rgs) <= max(1e-3 * abs(rgs), 1e-4), where
    grads = []
    for store in (False, True):
        xin = x.clone().requires_grad_(True)
        sig = torch.tensor(sr, dtype=torch.float32, device="cuda", requires_grad=True)
        (bf.recursive_bilateral(xin, sig, s, N=N, store=store) * g).sum().backward()
        grads.append((xin.grad, sig.grad))
    torch.testing.assert_close(grads[1][0], grads[0][0], rtol=0, atol=0, msg=where)
    assert float(grads[1][1]) == float(grads[0][1]), where
    with pytest.raises(ValueError):  # the stored backward needs the stored forward's workspace
        bf.recursive_backward_stored(x, so, sq, g, sr, N, s, ws[:16])


def test_recursive_graph_capture():
    """The forward and the backward enqueue only kernels (no allocation, no
    synchronisation inside the library), so both capture into a CUDA graph;
    replays on new image contents match eager calls bitwise."""
    H, W, s, sr = 70, 90, 6.0, 40.0
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    x = torch.from_numpy(image(H, W, seed=31)).cuda()
    g = torch.from_numpy(synth.random_like((H, W), seed=32)).cuda()
    out = torch.empty_like(x)
    q = torch.empty_like(x)
    ws = torch.empty(bf.recursive_backward_workspace_bytes(H, W, N) // 4, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up (module loading) outside the capture
        bf.recursive_forward(x, sr, N, s, return_q=False, out=out, ws=ws)
        o0, q0 = bf.recursive_forward(x, sr, N, s, return_q=True, ws=ws)
        bf.recursive_backward(x, o0, q0, g, sr, N, s, ws=ws)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        o, qq = bf.recursive_forward(x, sr, N, s, return_q=True, ws=ws)
        gin, gs = bf.recursive_backward(x, o, qq, g, sr, N, s, ws=ws)
    for seed in (33, 34):
        x.copy_(torch.from_numpy(image(H, W, seed=seed)).cuda())
        graph.replay()
        torch.cuda.synchronize()
        eo, eq = bf.recursive_forward(x, sr, N, s, return_q=True)
        egin, egs = bf.recursive_backward(x, eo, eq, g, sr, N, s)
        torch.testing.assert_close(o, eo, rtol=0, atol=0)
        torch.testing.assert_close(gin, egin, rtol=0, atol=0)
        assert float(gs.item()) == float(egs.item())


@pytest.mark.parametrize("s,sr,shape", [(2.0, 30.0, (60, 110)), (15.0, 45.0, (97, 64)),
                                        (0.5, 60.0, (1, 77))])
def test_recursive_joint(s, sr, shape):
    """The cross filter with the recursive Gaussian against the checker's 2N
    filterings (Q' is the checker's Q as is: the guide's factors are already
    rescaled); with guide = image it equals the Algorithm 2 route."""
    img = image(*shape, seed=shape[0] + 5, block=6)
    guide = synth.gradient_polygons_image(*shape, 8, 10.0, seed=shape[1] + 9)
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    x = torch.from_numpy(img).cuda()
    out, q = bf.recursive_joint_forward(x, torch.from_numpy(guide).cuda(), sr, N, s, return_q=True)
    ro, U, Q = rec.joint_gpa_recursive(img, guide, s, sr, N, return_parts=True)
    compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, Q, rec.centre_weight_recursive(s),
                    "joint s=%g sr=%g N=%d %s" % (s, sr, N, shape), sigma_r=sr, N=N)
    same = bf.recursive_joint_forward(x, x, sr, N, s)
    gpa = bf.recursive_forward(x, sr, N, s)
    assert float((same - gpa).abs().max()) <= 1e-3


def test_recursive_large_order():
    """sigma_r = 10.5 (the bound asks N ~ 230): hundreds of channels through
    the carries and the ring, forward and backward."""
    H, W, s, sr = 37, 70, 3.0, 10.5
    N = bf.order_from_delta(bf.GAUSS_RECURSIVE, 0, s, sr, 1.0)
    assert N > 150
    img = image(H, W, seed=77, block=5)
    x = torch.from_numpy(img).cuda()
    out, q = bf.recursive_forward(x, sr, N, s, return_q=True)
    ro, P, Q = rec.gpa_alg2_recursive(img, s, sr, N, return_parts=True)
    compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, scaled_q(img, Q, sr),
                    rec.centre_weight_recursive(s), "recursive N=%d" % N, sigma_r=sr, N=N)
    g = synth.random_like((H, W), seed=78)
    gin, gs = bf.recursive_backward(x, out, q, torch.from_numpy(g).cuda(), sr, N, s)
    rgin, rgs = rec.gpa_grad_recursive(img, s, sr, N, g.astype(np.float64))
    scale = max(np.abs(rgin).max(), 1e-30)
    assert np.abs(gin.cpu().numpy() - rgin).max() <= 2e-3 * scale
    assert abs(float(gs.item()) - rgs) <= max(1e-3 * abs(rgs), 1e-4)
