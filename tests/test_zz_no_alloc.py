"""The allocation-free backward (bf_fast_backward_noalloc) against the
workspace backward (bf_fast_backward), through the C ABI.

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


def _no_alloc(lib, x, out, q, g, p, stream):
    H, W = x.shape
    gin = torch.empty_like(x)
    gs = torch.full((1,), float("nan"), dtype=torch.float64, device=x.device)
    _lib.check(lib.bf_fast_backward_noalloc(_ptr(x), _ptr(out), _ptr(q), _ptr(g), _ptr(gin),
                                            _ptr(gs), H, W, W, ctypes.byref(p), stream),
               "bf_fast_backward_noalloc")
    return gin, gs


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
