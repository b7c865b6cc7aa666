"""The row-band split of one image (the multi-GPU decomposition of
paper_1603_08109_gb300.shard) checked on the CUDA path, on one GPU.

A rank that outputs rows [y0, y1) filters the input window [y0 - W, y1 + W)
(clipped to the image): each band is launched on the device pointer of its
window's first row (d_in + in0 * pitch), its output rows are stitched, and
the result is compared with the unsplit launch.  For the image gradient the
window is [y0 - 2W, y1 + 2W) and the output cotangent is kept on
[y0 - W, y1 + W) only; the per-band sigma_r gradients (each band's own
pixels' cotangent) are summed as the one all-reduce of the split would.
Neighbours outside the image do not contribute (zero extension), and a
window edge inside the image is at least W rows from every output row that
is kept, so the Gaussian FIR kernels, whose per-pixel sums do not depend on
where a tile starts, give bitwise the unsplit values; the box kernels' running
sums start at their tile's first row, so they agree to float rounding."""
import numpy as np
import pytest
import torch

import paper_1603_08109_gb300 as bf
from helpers import needs_gpu
from paper_1603_08109_gb300 import shard, synth

pytestmark = [pytest.mark.gpu, needs_gpu]


def _forward_bands(x, world, kind, r, ss, sr, N):
    H = x.shape[0]
    out = torch.empty_like(x)
    for b in shard.row_bands(H, world, r):
        o = bf.gpa_forward(x[b.in0:b.in1], kind, sr, N, radius=r, sigma_s=ss)
        out[b.y0:b.y1] = o[b.y0 - b.in0:b.y1 - b.in0]
    return out


@pytest.mark.parametrize("kind,r,ss,sr,N,exact", [(bf.GAUSS, 9, 3.0, 30.0, 40, True),
                                                  (bf.GAUSS, 20, 20 / 3.0, 40.0, 30, True),
                                                  (bf.BOX, 5, 0.0, 30.0, 41, False)])
def test_row_band_forward_equals_unsplit(kind, r, ss, sr, N, exact):
    """2048^2, four bands (fused compile-time-radius kernels; the banded
    two-pass forward at W = 20)."""
    S = 2048
    x = torch.from_numpy(synth.blocks_image(S, S, 64, 10.0, seed=1000)).cuda()
    full = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss)
    split = _forward_bands(x, 4, kind, r, ss, sr, N)
    torch.cuda.synchronize()
    if exact:
        assert torch.equal(split, full)
    else:
        assert float((split - full).abs().max()) <= 1e-3


@pytest.mark.parametrize("kind,r,ss,sr,N", [(bf.GAUSS, 9, 3.0, 30.0, 40),
                                            (bf.GAUSS, 5, 5 / 3.0, 25.0, 50)])
def test_row_band_gradient_equals_unsplit(kind, r, ss, sr, N):
    """1024 x 1536, three bands: the image gradient bitwise, the summed
    sigma_r gradient to FP32 rounding of the per-tile partial sums."""
    H, W = 1024, 1536
    x = torch.from_numpy(synth.blocks_image(H, W, 64, 10.0, seed=1001)).cuda()
    g = torch.from_numpy(synth.random_like((H, W), seed=1002)).cuda()
    out, q = bf.gpa_forward(x, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
    gin, gs = bf.gpa_backward(x, out, q, g, kind, sr, N, radius=r, sigma_s=ss)
    gin_split = torch.empty_like(x)
    gs_split = 0.0
    for b in shard.row_bands(H, 3, r, grad=True):
        xw = x[b.in0:b.in1]
        ow, qw = bf.gpa_forward(xw, kind, sr, N, radius=r, sigma_s=ss, return_q=True)
        gw = torch.zeros_like(xw)
        gw[b.g0 - b.in0:b.g1 - b.in0] = g[b.g0:b.g1]
        gi, _ = bf.gpa_backward(xw, ow, qw, gw, kind, sr, N, radius=r, sigma_s=ss,
                                need_sigma=False)
        gin_split[b.y0:b.y1] = gi[b.y0 - b.in0:b.y1 - b.in0]
        own = torch.zeros_like(xw)  # sigma_r: only the band's own pixels' cotangent
        own[b.y0 - b.in0:b.y1 - b.in0] = g[b.y0:b.y1]
        _, gsb = bf.gpa_backward(xw, ow, qw, own, kind, sr, N, radius=r, sigma_s=ss)
        gs_split += float(gsb.item())
    torch.cuda.synchronize()
    assert torch.equal(gin_split, gin)
    ref = float(gs.item())
    assert abs(gs_split - ref) <= 1e-5 * abs(ref) + 1e-9 * float(np.abs(g.cpu().numpy()).sum())
