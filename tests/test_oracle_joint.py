"""Pins for the checker's cross (joint) bilateral filter (Sec. I, Sec. V)."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import order
from paper_1603_08109_gb300 import synth

T = 128.0


def _asym(r, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.1, 1.0, size=(2 * r + 1, 2 * r + 1))
    return w / w.sum()


def test_guide_equal_to_image_is_the_plain_filter():
    """e = f: the joint GPA equals Algorithm 2 (independent route) and the
    exact joint filter equals eq. BF."""
    img = synth.blocks_image(19, 27, 6, 20.0, seed=1)
    w = _asym(3, 2)
    for sr, N in ((30.0, 40), (50.0, 12)):
        a = oracle.joint_gpa(img, img, w, sr, N)
        b = oracle.gpa_alg2(img, w, sr, N)
        assert np.abs(a - b).max() < 1e-9
    assert np.abs(oracle.joint_direct(img, img, w, 25.0) - oracle.bf_direct(img, w, 25.0)).max() < 1e-11


def test_constant_guide_gives_the_spatial_filter():
    img = synth.blocks_image(17, 23, 5, 20.0, seed=3).astype(np.float64)
    guide = np.full_like(img, 91.0)
    w = _asym(2, 4)
    ref = ndimage.convolve(img, w, mode="constant") / ndimage.convolve(np.ones_like(img), w, mode="constant")
    assert np.abs(oracle.joint_direct(img, guide, w, 30.0) - ref).max() < 1e-10
    assert np.abs(oracle.joint_gpa(img, guide, w, 30.0, 20) - ref).max() < 1e-10


def test_linear_in_the_averaged_image():
    """For a fixed guide, out - T is linear in f - T."""
    f1 = synth.blocks_image(16, 21, 4, 20.0, seed=5).astype(np.float64)
    f2 = synth.blocks_image(16, 21, 7, 20.0, seed=6).astype(np.float64)
    e = synth.blocks_image(16, 21, 5, 20.0, seed=7)
    w = oracle.spatial_kernel(1, 3, 1.2)
    al, be = 0.3, -0.45
    mix = T + al * (f1 - T) + be * (f2 - T)
    for fn in (lambda x: oracle.joint_gpa(x, e, w, 30.0, 30), lambda x: oracle.joint_direct(x, e, w, 30.0)):
        lhs = fn(mix) - T
        rhs = al * (fn(f1) - T) + be * (fn(f2) - T)
        assert np.abs(lhs - rhs).max() < 1e-9


def test_joint_gpa_within_accuracy_bound():
    """The proof of Prop. accuracy only uses |f - T| <= T and the kernel
    error on the guide, so the same bound holds for the joint filter."""
    img = synth.blocks_image(30, 34, 8, 20.0, seed=8)
    guide = synth.blocks_image(30, 34, 10, 15.0, seed=9)
    for kind, r, ss, sr in ((1, 6, 2.0, 30.0), (0, 4, 0.0, 40.0)):
        w = oracle.spatial_kernel(kind, r, ss)
        w0 = w[r, r]
        ex = oracle.joint_direct(img, guide, w, sr)
        lam = (T / sr) ** 2
        for N in (int(lam) + 6, int(2 * lam) + 10, int(3 * lam) + 15):
            E = order.poisson_tail(N, lam)
            if E >= w0:
                continue
            err = np.abs(oracle.joint_gpa(img, guide, w, sr, N) - ex).max()
            assert err <= 2 * T * E / (w0 - E) + 1e-9


def test_large_sigma_r_and_constant_image():
    img = synth.blocks_image(14, 18, 5, 20.0, seed=10).astype(np.float64)
    guide = synth.blocks_image(14, 18, 3, 30.0, seed=11)
    w = oracle.spatial_kernel(0, 2)
    ref = ndimage.convolve(img, w, mode="constant") / ndimage.convolve(np.ones_like(img), w, mode="constant")
    assert np.abs(oracle.joint_gpa(img, guide, w, 1e6, 3) - ref).max() < 1e-6
    c = np.full_like(img, 33.0)
    assert np.abs(oracle.joint_gpa(c, guide, w, 30.0, 25) - 33.0).max() < 1e-9
