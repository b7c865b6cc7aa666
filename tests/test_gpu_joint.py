"""GPU parity of the cross (joint) bilateral filter: the fused Gaussian-
polynomial kernel against the checker's definition at the same N, the
direct joint kernel against the exact joint filter, and the reduction to
the plain filter when the guide is the image."""
import numpy as np
import pytest
import torch

import oracle
import paper_1603_08109_gb300 as bf
from helpers import OUT_TOL, Q_ATOL, Q_RTOL, image, in_bound_regime, needs_gpu, spatial
from paper_1603_08109_gb300 import synth

pytestmark = [pytest.mark.gpu, needs_gpu]


def _pair(H, W, seed):
    f = image(H, W, seed=seed)
    e = synth.gradient_polygons_image(H, W, 6, 10.0, seed=seed + 1)
    return f, e


@pytest.mark.parametrize("case", [
    (bf.GAUSS, 9, 3.0, 30.0, 40, (40, 300)),
    (bf.GAUSS, 20, 6.7, 45.0, 25, (50, 200)),
    (bf.BOX, 5, 0.0, 30.0, 41, (37, 260)),
    (bf.BOX, 30, 0.0, 60.0, 19, (70, 140)),
    (bf.GAUSS, 3, 1.0, 20.0, 70, (1, 9)),
    (bf.GAUSS, 15, 5.0, 25.0, 54, (33, 250)),
    (bf.BOX, 15, 0.0, 40.0, 30, (9, 131)),
    (bf.GAUSS, 3, 1.0, 35.0, 30, (45, 290)),
    (bf.GAUSS, 5, 5 / 3.0, 40.0, 26, (26, 240)),
    (bf.BOX, 9, 0.0, 40.0, 30, (30, 280)),
], ids=lambda c: "k%d_r%d_sr%g_N%d" % (c[0], c[1], c[3], c[4]))
def test_joint_forward_matches_definition(case):
    kind, r, ss, sr, N, (H, W) = case
    f, e = _pair(H, W, seed=H + W)
    out, q = bf.joint_forward(torch.from_numpy(f).cuda(), torch.from_numpy(e).cuda(), kind, sr, N,
                              radius=r, sigma_s=ss, return_q=True)
    w = spatial(kind, r, ss)
    ro, num, den = oracle.joint_gpa(f, e, w, sr, N, return_parts=True)
    qg = q.cpu().numpy().astype(np.float64)
    assert (np.abs(qg - den) <= Q_ATOL + Q_RTOL * np.abs(den)).all()
    assert in_bound_regime(sr, N, w[r, r])
    mask = np.abs(den) >= 0.5 * w[r, r]
    assert np.abs(out.cpu().numpy() - ro)[mask].max() <= OUT_TOL


@pytest.mark.parametrize("case", [(bf.GAUSS, 20, 20 / 3.0, 45.0, 25), (bf.GAUSS, 60, 20.0, 60.0, 12),
                                  (bf.BOX, 30, 0.0, 60.0, 19)], ids=lambda c: "k%d_r%d" % c[:2])
def test_joint_banded_two_pass(case):
    """The banded joint filter (radius > 15): several bands (64 rows, ragged last
    band), several column tiles, against the checker's definition."""
    kind, r, ss, sr, N = case
    H, W = 150, 181
    f, e = _pair(H, W, seed=r + 3)
    w = spatial(kind, r, ss)
    ro, num, den = oracle.joint_gpa(f, e, w, sr, N, return_parts=True)
    mask = den >= 0.5 * w[r, r]
    for band in (64, None):
        out, q = bf.joint_forward(torch.from_numpy(f).cuda(), torch.from_numpy(e).cuda(), kind, sr,
                                  N, radius=r, sigma_s=ss, return_q=True, band_rows=band)
        qg = q.cpu().numpy().astype(np.float64)
        assert (np.abs(qg - den) <= Q_ATOL + Q_RTOL * np.abs(den)).all()
        og = out.cpu().numpy().astype(np.float64)
        assert np.abs(og - ro)[mask].max() <= OUT_TOL


def test_joint_with_guide_equal_to_image_is_plain_filter():
    f = image(45, 280, seed=3)
    x = torch.from_numpy(f).cuda()
    for kind, r, ss in ((bf.GAUSS, 9, 3.0), (bf.BOX, 7, 0.0)):
        a = bf.joint_forward(x, x, kind, 30.0, 40, radius=r, sigma_s=ss)
        b = bf.gpa_forward(x, kind, 30.0, 40, radius=r, sigma_s=ss)
        assert float((a - b).abs().max()) <= OUT_TOL


@pytest.mark.parametrize("case", [(bf.GAUSS, 9, 3.0, 30.0), (bf.BOX, 12, 0.0, 25.0)])
def test_joint_direct_matches_exact_joint_filter(case):
    kind, r, ss, sr = case
    f, e = _pair(60, 150, seed=11)
    out = bf.joint_direct(torch.from_numpy(f).cuda(), torch.from_numpy(e).cuda(), kind, sr,
                          radius=r, sigma_s=ss)
    ref = oracle.joint_direct(f, e, spatial(kind, r, ss), sr)
    assert np.abs(out.cpu().numpy() - ref).max() <= OUT_TOL


def test_joint_full_size_sampled():
    H = W = 2048
    f = image(H, W, seed=5, block=64, noise=10.0)
    e = synth.gradient_polygons_image(H, W, 64, 15.0, seed=6)
    N = bf.order_from_delta(bf.GAUSS, 9, 3.0, 30.0, 1.0)
    out = bf.joint_forward(torch.from_numpy(f).cuda(), torch.from_numpy(e).cuda(), bf.GAUSS, 30.0,
                           N, radius=9, sigma_s=3.0)
    rng = np.random.default_rng(2)
    ys = np.concatenate([rng.integers(0, H, 200), [0, H - 1]])
    xs = np.concatenate([rng.integers(0, W, 200), [W - 1, 0]])
    ref = oracle.joint_gpa(f, e, spatial(bf.GAUSS, 9, 3.0), 30.0, N, samples=(ys, xs))
    assert np.abs(out.cpu().numpy()[ys, xs] - ref).max() <= OUT_TOL
