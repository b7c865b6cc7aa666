"""Pins for the checker's filters: eq. BF, eq. GPA (definition and
Algorithm 2) and their gradients.

Each check is fixed by the mathematics rather than by the checker itself:
library routines for the special cases (scipy.ndimage.convolve), exact
invariants, agreement of two independent routes (definition vs the
recursion of Algorithm 2), the accuracy bound of Prop. accuracy, and
central finite differences for the gradients.  An asymmetric spatial kernel
on non-square images exposes swapped indices or transposed operands.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import order
from paper_1603_08109_gb300 import synth

T = 128.0


def _asym_kernel(r, seed=5):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.1, 1.0, size=(2 * r + 1, 2 * r + 1))
    return w / w.sum()


def _ratio_conv(num_img, den_img, w):
    """sum_j w(j) a(i-j) over in-image neighbours == convolution, zero fill."""
    num = ndimage.convolve(num_img, w, mode="constant", cval=0.0)
    den = ndimage.convolve(den_img, w, mode="constant", cval=0.0)
    return num / den


# --------------------------------------------------------------- spatial kernel
def test_spatial_kernels_normalised_and_separable():
    wb = oracle.spatial_kernel(0, 4)
    assert wb.shape == (9, 9)
    assert np.allclose(wb, 1.0 / 81.0)
    wg = oracle.spatial_kernel(1, 9, 3.0)
    assert wg.sum() == pytest.approx(1.0, abs=1e-14)
    k = np.arange(-9, 10)
    g1 = np.exp(-k * k / 18.0)
    assert np.allclose(wg, np.outer(g1, g1) / g1.sum() ** 2, rtol=1e-13, atol=0)
    assert wg[9, 9] == pytest.approx(order.centre_weight(1, 9, 3.0), rel=1e-13)


# -------------------------------------------------------------------- eq. BF
def test_bf_large_sigma_r_is_spatial_filter_asymmetric_kernel():
    img = synth.blocks_image(23, 31, 8, 20.0, seed=11).astype(np.float64)
    w = _asym_kernel(3)
    out = oracle.bf_direct(img, w, 1e7)
    ref = _ratio_conv(img, np.ones_like(img), w)
    assert np.abs(out - ref).max() < 1e-7


def test_bf_constant_image_and_shift_equivariance():
    w = oracle.spatial_kernel(1, 4, 1.5)
    c = np.full((12, 17), 77.0)
    assert np.abs(oracle.bf_direct(c, w, 20.0) - 77.0).max() < 1e-12
    img = synth.blocks_image(19, 26, 8, 20.0, seed=3).astype(np.float64)
    a = oracle.bf_direct(img, w, 25.0)
    b = oracle.bf_direct(img + 13.5, w, 25.0)  # Prop. centering: shifts commute
    assert np.abs(b - a - 13.5).max() < 1e-10


def test_bf_small_sigma_r_is_identity():
    img = synth.blocks_image(15, 21, 5, 20.0, seed=4).astype(np.float64)
    out = oracle.bf_direct(img, oracle.spatial_kernel(0, 3), 1e-3)
    assert np.abs(out - img).max() < 1e-9


def test_bf_transpose_equivariance():
    img = synth.blocks_image(13, 29, 6, 20.0, seed=7).astype(np.float64)
    w = _asym_kernel(2)
    a = oracle.bf_direct(img, w, 30.0)
    b = oracle.bf_direct(img.T.copy(), w.T.copy(), 30.0)
    assert np.abs(a - b.T).max() < 1e-11


# ------------------------------------------------------------------- eq. GPA
def test_gpa_definition_equals_algorithm2_asymmetric_kernel():
    """Two independent routes to eq. GPA: brute force with phi_N
    (eq. GaussPolynomial) and the recursions of Algorithm 2 with
    eqs. intImg / spatialFiltering / P / Q."""
    img = synth.blocks_image(21, 34, 8, 20.0, seed=12)
    w = _asym_kernel(4, seed=9)
    for sr, N in ((30.0, 40), (30.0, 7), (12.0, 150), (60.0, 3)):
        out_d, p2, q2 = oracle.gpa_definition(img, w, sr, N, return_parts=True)
        out_a, P, Q = oracle.gpa_alg2(img, w, sr, N, return_parts=True)
        H = (img.astype(np.float64) - T) / sr
        scale = np.exp(-H * H / 2)  # App. B: P_2 = e^{-H^2/2} P, Q_2 = e^{-H^2/2} Q
        assert np.abs(q2 - scale * Q).max() < 1e-12 * max(1.0, np.abs(q2).max())
        assert np.abs(p2 - scale * P).max() < 1e-10 * max(1.0, np.abs(p2).max())
        good = np.abs(q2) > 1e-6
        assert np.abs(out_d - out_a)[good].max() < 1e-8


def test_alg2_sampled_is_bitwise_full():
    img = synth.blocks_image(30, 41, 8, 20.0, seed=13)
    w = oracle.spatial_kernel(1, 6, 2.0)
    full, P, Q = oracle.gpa_alg2(img, w, 25.0, 33, return_parts=True)
    rng = np.random.default_rng(0)
    ys = rng.integers(0, 30, 50)
    xs = rng.integers(0, 41, 50)
    ys[:4] = [0, 29, 0, 29]
    xs[:4] = [0, 40, 40, 0]
    s, Ps, Qs = oracle.gpa_alg2_at(img, w, 25.0, 33, (ys, xs), return_parts=True)
    assert np.array_equal(s, full[ys, xs])
    assert np.array_equal(Qs, Q[ys, xs]) and np.array_equal(Ps, P[ys, xs])


def test_gpa_order1_is_range_weighted_spatial_filter():
    """N = 1: phi_1(t, tau) = exp(-(t^2+tau^2)/2 sigma_r^2), so the ratio is
    the spatial filter of h e^{-h^2/2s^2} over the filter of e^{-h^2/2s^2}."""
    img = synth.blocks_image(17, 27, 6, 20.0, seed=14).astype(np.float64)
    w = _asym_kernel(3, seed=2)
    sr = 40.0
    h = img - T
    e = np.exp(-h * h / (2 * sr * sr))
    ref = T + _ratio_conv(h * e, e, w)
    assert np.abs(oracle.gpa_alg2(img, w, sr, 1) - ref).max() < 1e-10
    assert np.abs(oracle.gpa_definition(img, w, sr, 1) - ref).max() < 1e-10


def test_gpa_large_sigma_r_is_spatial_filter():
    img = synth.blocks_image(18, 22, 6, 20.0, seed=15).astype(np.float64)
    w = oracle.spatial_kernel(1, 5, 2.0)
    ref = _ratio_conv(img, np.ones_like(img), w)
    for N in (1, 2, 5):
        assert np.abs(oracle.gpa_alg2(img, w, 1e6, N) - ref).max() < 1e-6


def test_gpa_constant_image_fixed_point():
    w = oracle.spatial_kernel(0, 5)
    for level in (3.0, 128.0, 250.0):
        c = np.full((14, 19), level)
        assert np.abs(oracle.gpa_alg2(c, w, 30.0, 40) - level).max() < 1e-9


def test_gpa_negation_and_scaling_symmetry():
    """a_n(-H) = (-1)^n a_n(H) gives GPA(2T - f) = 2T - GPA(f); phi_N depends
    on t/sigma_r and tau/sigma_r only, so scaling (f - T, sigma_r) by alpha
    scales GPA - T by alpha."""
    img = synth.blocks_image(20, 25, 7, 20.0, seed=16).astype(np.float64)
    w = oracle.spatial_kernel(1, 4, 1.7)
    a = oracle.gpa_alg2(img, w, 30.0, 25)
    b = oracle.gpa_alg2(2 * T - img, w, 30.0, 25)
    assert np.abs(b - (2 * T - a)).max() < 1e-9
    alpha = 0.37
    c = oracle.gpa_alg2(T + alpha * (img - T), w, 30.0 * alpha, 25)
    assert np.abs((c - T) - alpha * (a - T)).max() < 1e-9


def test_gpa_within_accuracy_bound_of_bf():
    """Prop. accuracy with the Poisson tail of Prop. upperBound, and the
    corollary: N from eq. eps + eq. LambW keeps |BF - GPA| <= delta."""
    img = synth.blocks_image(48, 40, 16, 20.0, seed=17)
    for kind, r, ss, sr in ((1, 9, 3.0, 30.0), (0, 5, 0.0, 20.0), (1, 6, 2.0, 60.0)):
        w = oracle.spatial_kernel(kind, r, ss)
        w0 = w[r, r]
        bf = oracle.bf_direct(img, w, sr)
        lam = (T / sr) ** 2
        for N in (int(lam) + 5, int(1.5 * lam) + 8, int(2.5 * lam) + 12):
            E = order.poisson_tail(N, lam)
            if E >= w0:
                continue
            err = np.abs(oracle.gpa_alg2(img, w, sr, N) - bf).max()
            assert err <= 2 * T * E / (w0 - E) + 1e-9
        for delta in (1.0, 0.1):
            N = order.order_from_delta(kind, r, ss, sr, delta)
            assert np.abs(oracle.gpa_alg2(img, w, sr, N) - bf).max() <= delta


def test_gpa_error_decreases_to_fp64_floor():
    """Table (GPA vs N, sigma_s = 5 / box W = 4, sigma_r = 30): the error to
    the exact filter falls with N and saturates at the FP64 floor by N = 60."""
    img = synth.blocks_image(40, 40, 10, 20.0, seed=18)
    for w in (oracle.spatial_kernel(1, 15, 5.0), oracle.spatial_kernel(0, 4)):
        bf = oracle.bf_direct(img, w, 30.0)
        errs = [np.abs(oracle.gpa_alg2(img, w, 30.0, N) - bf).max() for N in (10, 20, 30, 40, 50)]
        assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1))
        floor = [np.abs(oracle.gpa_alg2(img, w, 30.0, N) - bf).max() for N in (60, 70)]
        assert max(floor) < 1e-9


# ---------------------------------------------------------------- gradients
def _fd_check(kind, img, w, sr, N, seed):
    H, W = img.shape
    g = synth.random_like((H, W), seed).astype(np.float64)
    d = synth.random_like((H, W), seed + 1).astype(np.float64)

    def loss(x, s):
        if kind == 0:
            return float(np.sum(g * oracle.bf_direct(x, w, s)))
        return float(np.sum(g * oracle.gpa_definition(x, w, s, N)))

    if kind == 0:
        gin, gs = oracle.bf_direct_grad(img, w, sr, g)
    else:
        gin, gs = oracle.gpa_grad(img, w, sr, N, g)
    x = img.astype(np.float64)
    hstep = 1e-4
    fd = (loss(x + hstep * d, sr) - loss(x - hstep * d, sr)) / (2 * hstep)
    an = float(np.sum(gin * d))
    assert an == pytest.approx(fd, rel=2e-6, abs=1e-9)
    hs = 1e-4 * sr
    fds = (loss(x, sr + hs) - loss(x, sr - hs)) / (2 * hs)
    assert gs == pytest.approx(fds, rel=2e-6, abs=1e-9)
    return gin


@pytest.mark.parametrize("kind", [0, 1])
def test_gradients_match_central_differences(kind):
    img = synth.blocks_image(14, 19, 5, 20.0, seed=21)
    w = _asym_kernel(2, seed=4)
    _fd_check(kind, img, w, 30.0, 30, seed=100)
    _fd_check(kind, img, oracle.spatial_kernel(1, 3, 1.2), 45.0, 12, seed=200)


def test_gradient_sampled_equals_full():
    img = synth.blocks_image(16, 21, 5, 20.0, seed=22)
    w = oracle.spatial_kernel(1, 3, 1.0)
    g = synth.random_like(img.shape, 5).astype(np.float64)
    full, _ = oracle.gpa_grad(img, w, 25.0, 30, g)
    ys = np.array([0, 15, 7, 3])
    xs = np.array([20, 0, 10, 4])
    part, _ = oracle.gpa_grad(img, w, 25.0, 30, g, samples=(ys, xs))
    assert np.array_equal(part, full[ys, xs])


# ------------------------------------------------ term magnitudes (conditioning)
def test_term_magnitudes_order1_is_spatial_filter_of_positive_terms():
    """N = 1: the single term e^{-(t^2+tau^2)/2 s^2} is positive, so S_Q = Q'
    = e(i) (w * e)(i) and S_P = e(i) (w * |h| e)(i) (scipy convolution with an
    asymmetric kernel on a non-square image)."""
    img = synth.blocks_image(17, 27, 6, 20.0, seed=24).astype(np.float64)
    w = _asym_kernel(3, seed=8)
    sr = 35.0
    h = img - T
    e = np.exp(-h * h / (2 * sr * sr))
    sp, sq = oracle.gpa_term_magnitudes(img, w, sr, 1)
    ref_q = e * ndimage.convolve(e, w, mode="constant", cval=0.0)
    ref_p = e * ndimage.convolve(np.abs(h) * e, w, mode="constant", cval=0.0)
    assert np.abs(sq - ref_q).max() < 1e-13
    assert np.abs(sp - ref_p).max() < 1e-11


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_term_magnitudes_equal_algorithm2_sums_on_one_sided_images(sign):
    """Every intensity on one side of t_c: all terms t^n tau^n are >= 0, so the
    magnitudes are Algorithm 2's own sums (Q' = e^{-H^2/2} Q and
    P' = (out - t_c) Q'), evaluated by its recursion (an independent route);
    for intensities below t_c the numerator is the negated P'."""
    rng = np.random.default_rng(4)
    img = T + sign * rng.uniform(0.0, 127.0, size=(19, 23))
    w = _asym_kernel(2, seed=3)
    sr, N = 30.0, 7
    out, P, Q = oracle.gpa_alg2(img, w, sr, N, return_parts=True)
    H = (img - T) / sr
    qs = Q * np.exp(-H * H / 2)
    sp, sq = oracle.gpa_term_magnitudes(img, w, sr, N)
    assert np.abs(sq - qs).max() < 1e-12
    assert np.abs(sp - sign * (out - T) * qs).max() < 1e-9


def test_term_magnitudes_large_order_limit_brute_force():
    """As N grows, sum_n |t tau|^n / (s^2n n!) -> e^{|t tau|/s^2}, so each term
    sum tends to e^{-(|t| - |tau|)^2 / 2 s^2}: brute force over a tiny image."""
    img = synth.blocks_image(9, 11, 3, 25.0, seed=6).astype(np.float64)
    w = _asym_kernel(2, seed=12)
    sr = 45.0
    sp, sq = oracle.gpa_term_magnitudes(img, w, sr, 200)
    h = np.abs(img - T)
    r = 2
    Hh, Ww = img.shape
    for y in range(Hh):
        for x in range(Ww):
            rq = rp = 0.0
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    yy, xx = y - dy, x - dx
                    if 0 <= yy < Hh and 0 <= xx < Ww:
                        g = np.exp(-(h[yy, xx] - h[y, x]) ** 2 / (2 * sr * sr))
                        rq += w[dy + r, dx + r] * g
                        rp += w[dy + r, dx + r] * g * h[yy, xx]
            assert abs(sq[y, x] - rq) < 1e-12 and abs(sp[y, x] - rp) < 1e-10


def test_term_magnitudes_bound_the_signed_sums():
    """|num| <= S_P and |den| <= S_Q everywhere; at N = 2 with intensities on
    both sides of t_c some terms cancel (strict inequality somewhere)."""
    img = synth.blocks_image(20, 30, 5, 20.0, seed=9).astype(np.float64)
    w = oracle.spatial_kernel(0, 3)
    for N in (2, 3, 10):
        sp, sq = oracle.gpa_term_magnitudes(img, w, 40.0, N)
        _, num, den = oracle.gpa_definition(img, w, 40.0, N, return_parts=True)
        assert (np.abs(den) <= sq * (1 + 1e-12)).all() and (np.abs(num) <= sp * (1 + 1e-12)).all()
        assert (sq > np.abs(den) * 1.01).any()
