"""The allocation-free backward (bf_fast_backward_noalloc) against the
workspace backward (bf_fast_backward) and the checker's exact gradient,
through the C ABI.

Some callers of this library cannot call cudaMalloc (plug-ins whose host
application owns the device allocator; real-time loops that must not
allocate after start-up), so bf_fast_backward_noalloc keeps its scratch in a
static device array.  This file is collected last so that a failure here
cannot hide any other test's result; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import image, needs_gpu
from paper_1603_08109_gb300 import _lib, synth

pytestmark = [pytest.mark.gpu, needs_gpu]

GIN_RTOL = 2e-3    # same bars as the other gradient tests
GSIG_RTOL = 1e-3


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _forward(lib, x, p, stream):
    H, W = x.shape
    out = torch.empty_like(x)
    q = torch.empty_like(x)
    _lib.check(lib.bf_fast_forward(_ptr(x), _ptr(out), _ptr(q), H, W, W, ctypes.byref(p), stream),
               "bf_fast_forward")
    return out, q


def _with_workspace(lib, x, out, q, g, p, stream):
    H, W = x.shape
    n = ctypes.c_size_t()
    _lib.check(lib.bf_fast_backward_workspace(H, W, ctypes.byref(p), ctypes.byref(n)), "ws")
    ws = torch.empty(n.value, dtype=torch.uint8, device=x.device)
    gin = torch.empty_like(x)
    gs = torch.zeros(1, dtype=torch.float64, device=x.device)
    _lib.check(lib.bf_fast_backward(_ptr(x), _ptr(out), _ptr(q), _ptr(g), _ptr(gin), _ptr(gs),
                                    H, W, W, ctypes.byref(p), _ptr(ws), n, stream),
               "bf_fast_backward")
    return gin, gs


def _no_alloc(lib, x, out, q, g, p, stream, sigma=True):
    H, W = x.shape
    gin = torch.empty_like(x)
    gs = torch.full((1,), float("nan"), dtype=torch.float64, device=x.device) if sigma else None
    _lib.check(lib.bf_fast_backward_noalloc(_ptr(x), _ptr(out), _ptr(q), _ptr(g), _ptr(gin),
                                            _ptr(gs), H, W, W, ctypes.byref(p), stream),
               "bf_fast_backward_noalloc")
    return gin, gs


def _rel(a, ref):
    ref = np.asarray(ref, np.float64)
    return np.abs(np.asarray(a, np.float64) - ref).max() / np.abs(ref).max()


def test_no_alloc_backward_matches_workspace_backward_on_two_calls():
    lib = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [((120, 530), _lib.GAUSS, 9, 3.0, 30.0, 40, 1),
             ((77, 301), _lib.BOX, 5, 0.0, 20.0, 60, 2)]  # a smaller second call
    for (H, W), kind, r, ss, sr, N, seed in cases:
        p = _lib.make_params(kind, r, ss, sr, N)
        x = torch.from_numpy(image(H, W, seed=seed)).cuda()
        g = torch.from_numpy(synth.random_like((H, W), seed=seed + 10)).cuda()
        out, q = _forward(lib, x, p, stream)
        ref_gin, ref_gs = _with_workspace(lib, x, out, q, g, p, stream)
        gin, gs = _no_alloc(lib, x, out, q, g, p, stream)
        torch.cuda.synchronize()
        rg = ref_gin.double().cpu().numpy()
        err = np.abs(gin.double().cpu().numpy() - rg).max() / np.abs(rg).max()
        assert err <= GIN_RTOL
        assert abs(float(gs.item()) - float(ref_gs.item())) <= GSIG_RTOL * abs(float(ref_gs.item()))


def test_no_alloc_backward_rejects_images_beyond_its_scratch():
    lib = _lib.lib()
    p = _lib.make_params(_lib.GAUSS, 9, 3.0, 30.0, 40)
    fake = ctypes.c_void_p(256)
    # 16384 x 16384 needs about 2.4e5 partial sums: rejected before any GPU work
    st = lib.bf_fast_backward_noalloc(fake, fake, fake, fake, fake, fake, 16384, 16384, 16384,
                                      ctypes.byref(p), None)
    assert st == 3


def test_no_alloc_backward_against_checker_runtime_radius_and_no_sigma():
    """A radius above the compile-time set (Gaussian W = 22: the runtime-radius
    fused tile, since the static scratch is too small for the banded backward)
    against the checker's exact gradient; then the same call without a sigma_r
    gradient (no scratch at all), whose image gradient is bitwise the same."""
    lib = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (H, W), kind, r, ss, sr, N, seed in (((70, 260), _lib.GAUSS, 22, 22 / 3.0, 30.0, 41, 3),
                                             ((50, 140), _lib.GAUSS, 9, 3.0, 30.0, 40, 4)):
        p = _lib.make_params(kind, r, ss, sr, N)
        img = image(H, W, seed=seed)
        x = torch.from_numpy(img).cuda()
        gh = synth.random_like((H, W), seed=seed + 10)
        g = torch.from_numpy(gh).cuda()
        out, q = _forward(lib, x, p, stream)
        gin, gs = _no_alloc(lib, x, out, q, g, p, stream)
        gin0, _ = _no_alloc(lib, x, out, q, g, p, stream, sigma=False)
        torch.cuda.synchronize()
        w = oracle.spatial_kernel(kind, r, ss)
        ref_gin, ref_gs = oracle.gpa_grad(img, w, sr, N, gh.astype(np.float64))
        assert _rel(gin.cpu().numpy(), ref_gin) <= GIN_RTOL
        assert abs(float(gs.item()) - ref_gs) <= GSIG_RTOL * abs(ref_gs)
        assert torch.equal(gin0, gin)


def test_no_alloc_backward_rejects_radii_beyond_its_tiles():
    """Gaussian W = 60 (the 8192^2 workload's radius): no fused tile holds its
    region, so the allocation-free backward returns BF_ERR_UNSUPPORTED with a
    reason, before any GPU work; the workspace backward takes it."""
    lib = _lib.lib()
    p = _lib.make_params(_lib.GAUSS, 60, 20.0, 40.0, 32)
    fake = ctypes.c_void_p(256)
    st = lib.bf_fast_backward_noalloc(fake, fake, fake, fake, fake, fake, 300, 300, 300,
                                      ctypes.byref(p), None)
    assert st == 3
    assert b"radius" in lib.bf_last_cuda_error()
    n = ctypes.c_size_t()
    assert lib.bf_fast_backward_workspace(300, 300, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value > 0
