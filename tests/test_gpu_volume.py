"""GPU parity of the volume (video) filter, bf_volume_forward, against the
checker's Algorithm 2 on volumes (oracle.volume, pinned by the planar checker
and brute force): several z-tiles (16 planes) and y/x tiles (32 x 32) with
ragged edges, a single voxel, box and Gaussian kernels, orders from the
volume kernel's w(0) = w1(0)^3, a z-constant volume against the planar GPU
filter of its slice, and the argument errors."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1603_08109_gb300 as bf
from helpers import compare_forward, needs_gpu, scaled_q
from oracle import volume as vol
from paper_1603_08109_gb300 import synth

pytestmark = [pytest.mark.gpu, needs_gpu]

CASES = [  # (kind, radius, sigma_s, sigma_r, (D, H, W))
    (bf.GAUSS, 2, 0.7, 30.0, (5, 40, 70)),
    (bf.BOX, 3, 0.0, 40.0, (20, 33, 45)),
    (bf.GAUSS, 6, 2.0, 30.0, (17, 37, 100)),
    (bf.GAUSS, 9, 3.0, 50.0, (3, 70, 33)),
    (bf.BOX, 1, 0.0, 25.0, (1, 1, 1)),
    (bf.GAUSS, 4, 4.0 / 3.0, 60.0, (35, 9, 8)),
    (bf.GAUSS, 7, 7 / 3.0, 40.0, (3, 150, 131)),   # odd radius, several 64 x 48 y/x tiles
    (bf.BOX, 8, 0.0, 45.0, (4, 129, 97)),          # the largest tensor-copy radius
    (bf.BOX, 0, 0.0, 30.0, (2, 65, 49)),           # W = 0: the range kernel alone
]


def _volume(D, H, W, seed):
    return np.stack([synth.blocks_image(H, W, 6, 15.0, seed=seed + k) for k in range(D)])


@pytest.mark.parametrize("case", CASES, ids=lambda c: "k%d_r%d_%dx%dx%d" % ((c[0], c[1]) + c[4]))
def test_volume_forward(case):
    kind, r, ss, sr, (D, H, W) = case
    v = _volume(D, H, W, seed=D * 100 + H)
    N = bf.volume_order_from_delta(kind, r, ss, sr, 1.0)
    x = torch.from_numpy(v).cuda()
    out, q = bf.gpa_volume(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
    torch.cuda.synchronize()
    ro, P, Q = vol.gpa_alg2_volume(v, kind, r, ss, sr, N, return_parts=True)
    compare_forward(out.cpu().numpy(), q.cpu().numpy(), ro, scaled_q(v, Q, sr),
                    vol.centre_weight_volume(kind, r, ss), "volume %s N=%d" % (case, N),
                    sigma_r=sr, N=N)


def test_volume_z_constant_matches_planar_filter():
    """A volume constant along z: each output plane equals the planar filter of
    the slice (the z-weights cancel in P'/Q'), here against the GPU planar
    forward; and a reused workspace gives the same bits."""
    img = synth.blocks_image(45, 77, 5, 20.0, seed=3)
    D, r, ss, sr, N = 19, 5, 5.0 / 3.0, 35.0, 30
    x = torch.from_numpy(np.repeat(img[None], D, axis=0)).cuda()
    ws = torch.empty(bf.volume_workspace_bytes(D, 45, 77, bf.GAUSS, sr, N, r, ss) // 4, device="cuda")
    out = bf.gpa_volume(x, bf.GAUSS, sr, N, radius=r, sigma_s=ss, ws=ws)
    out2 = bf.gpa_volume(x, bf.GAUSS, sr, N, radius=r, sigma_s=ss, ws=ws)
    ref = bf.gpa_forward(torch.from_numpy(img).cuda(), bf.GAUSS, sr, N, radius=r, sigma_s=ss)
    torch.cuda.synchronize()
    assert int(ws[:1].view(torch.int32).item()) == 0  # the workspace's status word: no timeout
    assert torch.equal(out, out2)
    for z in range(D):
        assert float((out[z] - ref).abs().max()) <= 1e-3, z


def test_volume_errors():
    lib = bf._lib.lib()
    x = torch.zeros((4, 8, 8), device="cuda")
    o = torch.empty_like(x)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    p = bf._lib.make_params(bf.GAUSS, 32, 10.0, 30.0, 10)  # radius above the volume limit
    n = ctypes.c_size_t()
    assert lib.bf_volume_workspace(4, 8, 8, ctypes.byref(p), ctypes.byref(n)) == 3
    p = bf._lib.make_params(bf.BOX, 2, 0.0, 30.0, 10)
    assert lib.bf_volume_workspace(4, 8, 8, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value == 256 + 11 * 4 * 8 * 8 * 4  # status header + N + 1 planes
    assert lib.bf_volume_workspace(4, 8, 6, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value == 256 + 11 * 4 * 8 * 8 * 4  # rows padded to a multiple of 4 floats
    assert lib.bf_volume_workspace(4, 8, 8, ctypes.byref(p), ctypes.byref(n)) == 0
    ws = torch.empty(n.value // 4, device="cuda")
    assert lib.bf_volume_forward(ptr(x), ptr(o), None, 4, 8, 8, ctypes.byref(p), ptr(ws),
                                 n.value - 4, None) == 5
    assert lib.bf_volume_forward(ptr(x), ptr(x), None, 4, 8, 8, ctypes.byref(p), ptr(ws),
                                 n.value, None) == 1
    rp = bf._lib.make_params(bf.GAUSS_RECURSIVE, 0, 3.0, 30.0, 10)
    assert lib.bf_volume_forward(ptr(x), ptr(o), None, 4, 8, 8, ctypes.byref(rp), ptr(ws),
                                 n.value, None) == 1
    assert lib.bf_volume_forward(ptr(x), ptr(o), None, 4, 8, 8, ctypes.byref(p), ptr(ws),
                                 n.value, None) == 0
    torch.cuda.synchronize()
