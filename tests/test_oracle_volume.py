"""Pins for the checker's volume mode (oracle.volume): the straightforward
extension of eq. BF and Algorithm 2 to a box of Z^3 with the separable
kernel w1 (x) w1 (x) w1 (Sec. I, Sec. V).

Each check is fixed by something other than the module's own formulas: a
volume of depth 1 is an image, so every function must reproduce the C
checker's planar brute force and Algorithm 2 (pinned by their own tests); a
volume constant along z reduces exactly to the planar filter of each slice
(the z-weights are a common factor of every filtered power image and cancel
in P/Q, also at the z-edges), which catches a wrong or transposed axis; the
brute-force filter pins the separable one on a tiny anisotropic box; the
brute-force definition with phi_N pins Algorithm 2 in 3-D; and the error
against eq. BF stays within delta when N comes from eq. eps with
w(0) = w1(0)^3."""
import numpy as np
import pytest

import oracle
from oracle import order
from oracle import volume as vol
from paper_1603_08109_gb300 import synth

T = 128.0


def _volume(D, H, W, seed, block=3, noise=20.0):
    return np.stack([synth.blocks_image(H, W, block, noise, seed=seed + k) for k in range(D)]).astype(
        np.float64)


@pytest.mark.parametrize("kind,r,ss", [(oracle.GAUSS, 2, 0.8), (oracle.BOX, 1, 0.0),
                                       (oracle.GAUSS, 3, 1.0)])
def test_depth_one_is_the_planar_filter(kind, r, ss):
    img = synth.blocks_image(9, 13, 3, 25.0, seed=r + 5).astype(np.float64)
    w = oracle.spatial_kernel(kind, r, ss)
    w1 = vol.taps_1d(kind, r, ss)
    assert np.abs(np.outer(w1, w1) - w).max() < 1e-15 and abs(w1.sum() - 1.0) < 1e-14
    v = img[None]
    sr, N = 35.0, 9
    o3, P3, Q3 = vol.gpa_alg2_volume(v, kind, r, ss, sr, N, return_parts=True)
    o2, P2, Q2 = oracle.gpa_alg2(img, w, sr, N, return_parts=True)
    # the planar checker's Q carries w as given; depth 1 multiplies by w1(0) (the
    # only z-tap inside the volume): a common factor of P and Q
    c = w1[r]
    assert np.abs(o3[0] - o2).max() < 1e-10
    assert np.abs(Q3[0] - c * Q2).max() <= 1e-12 * np.abs(Q2).max()
    assert np.abs(P3[0] - c * P2).max() <= 1e-12 * np.abs(P2).max()
    assert np.abs(vol.bf_direct_volume(v, kind, r, ss, sr)[0] - oracle.bf_direct(img, w, sr)).max() < 1e-10
    assert np.abs(vol.gpa_definition_volume(v, kind, r, ss, sr, N)[0]
                  - oracle.gpa_definition(img, w, sr, N)).max() < 1e-10


@pytest.mark.parametrize("kind,r,ss,D", [(oracle.GAUSS, 2, 0.8, 5), (oracle.BOX, 2, 0.0, 3)])
def test_z_constant_volume_reduces_to_slices(kind, r, ss, D):
    img = synth.blocks_image(11, 8, 3, 20.0, seed=40 + D).astype(np.float64)
    v = np.repeat(img[None], D, axis=0)
    w = oracle.spatial_kernel(kind, r, ss)
    sr, N = 40.0, 12
    o3 = vol.gpa_alg2_volume(v, kind, r, ss, sr, N)
    o2 = oracle.gpa_alg2(img, w, sr, N)
    for z in range(D):
        assert np.abs(o3[z] - o2).max() < 1e-10, z
    d3 = vol.bf_direct_volume(v, kind, r, ss, sr)
    d2 = oracle.bf_direct(img, w, sr)
    for z in range(D):
        assert np.abs(d3[z] - d2).max() < 1e-10, z


def test_separable_filter_against_brute_force():
    """filter3 equals the triple sum over in-volume neighbours with the
    explicit kernel w1(j_z) w1(j_y) w1(j_x) on an anisotropic box."""
    rng = np.random.default_rng(3)
    F = rng.uniform(-1, 1, size=(4, 5, 7))
    r = 2
    w1 = vol.taps_1d(oracle.GAUSS, r, 0.9)
    got = vol.filter3(F, w1)
    D, H, W = F.shape
    ref = np.zeros_like(F)
    for z in range(D):
        for y in range(H):
            for x in range(W):
                s = 0.0
                for dz in range(-r, r + 1):
                    for dy in range(-r, r + 1):
                        for dx in range(-r, r + 1):
                            zz, yy, xx = z - dz, y - dy, x - dx
                            if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W:
                                s += w1[dz + r] * w1[dy + r] * w1[dx + r] * F[zz, yy, xx]
                ref[z, y, x] = s
    assert np.abs(got - ref).max() < 1e-14


@pytest.mark.parametrize("kind,r,ss,N", [(oracle.GAUSS, 1, 0.6, 6), (oracle.BOX, 1, 0.0, 11)])
def test_algorithm2_matches_definition(kind, r, ss, N):
    v = _volume(4, 5, 6, seed=11 * N)
    for sr in (25.0, 60.0):
        a2 = vol.gpa_alg2_volume(v, kind, r, ss, sr, N)
        df = vol.gpa_definition_volume(v, kind, r, ss, sr, N)
        assert np.abs(a2 - df).max() < 1e-9


@pytest.mark.parametrize("kind,r,ss,sr", [(oracle.GAUSS, 2, 0.8, 30.0), (oracle.BOX, 1, 0.0, 45.0)])
def test_accuracy_against_direct_filter(kind, r, ss, sr):
    """With N from delta (eq. eps with w(0) = w1(0)^3, eq. LambW) the GPA is
    within delta of eq. BF on the volume, and the error falls as N grows."""
    v = _volume(6, 9, 10, seed=5, block=4)
    direct = vol.bf_direct_volume(v, kind, r, ss, sr)
    w0 = vol.centre_weight_volume(kind, r, ss)
    lam = T * T / (sr * sr)
    errs = []
    for delta in (1.0, 0.1, 0.01):
        N, _ = order.chernoff_order_lambertw(lam, order.eps_from_delta(w0, delta))
        err = np.abs(vol.gpa_alg2_volume(v, kind, r, ss, sr, N) - direct).max()
        assert err <= delta
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]


def test_support_larger_than_the_volume():
    """Depth 2 with a radius of 3 (whole z-offsets outside the volume): the
    z-constant reduction and the agreement of Algorithm 2 with the brute-force
    definition still hold."""
    img = synth.blocks_image(6, 7, 2, 25.0, seed=77).astype(np.float64)
    v = np.repeat(img[None], 2, axis=0)
    w = oracle.spatial_kernel(oracle.BOX, 3, 0.0)
    o3 = vol.gpa_alg2_volume(v, oracle.BOX, 3, 0.0, 40.0, 10)
    o2 = oracle.gpa_alg2(img, w, 40.0, 10)
    assert np.abs(o3 - o2[None]).max() < 1e-10
    v2 = _volume(2, 4, 5, seed=91)
    a2 = vol.gpa_alg2_volume(v2, oracle.GAUSS, 3, 1.0, 30.0, 8)
    df = vol.gpa_definition_volume(v2, oracle.GAUSS, 3, 1.0, 30.0, 8)
    assert np.abs(a2 - df).max() < 1e-9
