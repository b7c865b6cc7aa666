"""GPU parity of the direct filter (eq. BF) against the checker's brute force."""
import numpy as np
import pytest
import torch

import oracle
import paper_1603_08109_gb300 as bf
from helpers import OUT_TOL, image, needs_gpu, spatial

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("case", [
    (bf.GAUSS, 9, 3.0, 30.0, (70, 150)),
    (bf.GAUSS, 15, 5.0, 25.0, (40, 90)),
    (bf.BOX, 5, 0.0, 10.0, (33, 140)),
    (bf.BOX, 20, 0.0, 60.0, (50, 70)),
    (bf.GAUSS, 2, 0.7, 40.0, (1, 1)),
    (bf.BOX, 12, 0.0, 30.0, (5, 300)),
], ids=lambda c: "k%d_r%d_sr%g_%dx%d" % (c[0], c[1], c[3], c[4][0], c[4][1]))
def test_direct_matches_eq_bf(case):
    kind, r, ss, sr, (H, W) = case
    img = image(H, W, seed=H + 7 * W)
    out = bf.direct(torch.from_numpy(img).cuda(), kind, sr, radius=r, sigma_s=ss)
    ref = oracle.bf_direct(img, spatial(kind, r, ss), sr)
    err = np.abs(out.cpu().numpy() - ref).max()
    assert err <= OUT_TOL, err


def test_direct_full_size_sampled():
    H = W = 2048
    img = image(H, W, seed=1000, block=64, noise=10.0)
    out = bf.direct(torch.from_numpy(img).cuda(), bf.GAUSS, 30.0, radius=9, sigma_s=3.0)
    rng = np.random.default_rng(3)
    ys = np.concatenate([rng.integers(0, H, 500), [0, H - 1, 0, H - 1]])
    xs = np.concatenate([rng.integers(0, W, 500), [0, W - 1, W - 1, 0]])
    ref = oracle.bf_direct(img, spatial(bf.GAUSS, 9, 3.0), 30.0, samples=(ys, xs))
    assert np.abs(out.cpu().numpy()[ys, xs] - ref).max() <= OUT_TOL
