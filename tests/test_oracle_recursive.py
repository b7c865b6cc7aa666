"""Pins for the checker's recursive-Gaussian mode (oracle.recursive).

Each check is fixed by something other than the checker's own formula:
the sampled Gaussian the fit approximates (to the fit's published accuracy),
the unit sum over all integers, an independent route through the C checker's
brute-force 2-D filter with the explicit kernel h(j_y) h(j_x) on non-square
images (catches a transposed operand), the causal + anticausal recursions
started from zero state (catches a wrong sign, a dropped mode or a missing
centre correction), the interior of a constant image, and the accuracy of
the resulting GPA against the direct bilateral filter with the same kernel.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import order
from oracle import recursive as rec
from paper_1603_08109_gb300 import synth

T = 128.0


@pytest.mark.parametrize("s", [1.5, 3.0, 10.0, 20.0])
def test_impulse_approximates_sampled_gaussian(s):
    """The fit's maximum deviation from the normalised sampled Gaussian stays
    within 1e-3 of the Gaussian's peak (Deriche's fourth-order fit is accurate
    to a few 1e-4 of the peak); a wrong constant or a swapped sine and cosine
    is off by tens of percent."""
    K = int(math.ceil(12 * s)) + 8
    h = rec.deriche_impulse(s, K + 1)
    k = np.arange(-400 * int(math.ceil(s)), 400 * int(math.ceil(s)) + 1)
    g = np.exp(-k * k / (2.0 * s * s))
    g = g / g.sum()
    g = g[np.abs(k) <= K][K:]  # k = 0 .. K
    assert np.abs(h - g).max() <= 1e-3 * g[0]
    assert h[0] == pytest.approx(g[0], rel=1e-3)


@pytest.mark.parametrize("s", [0.8, 2.0, 7.5, 33.0])
def test_unit_sum_and_centre_weight(s):
    K = int(math.ceil(100 * s)) + 64
    h = rec.deriche_impulse(s, K + 1)
    assert 2.0 * h.sum() - h[0] == pytest.approx(1.0, abs=1e-12)
    assert rec.centre_weight_recursive(s) == pytest.approx(h[0] ** 2, rel=1e-15)


def _explicit_kernel(s, Hh, Ww):
    """h(j_y) h(j_x) on [-r, r]^2 with r covering every in-image offset."""
    r = max(Hh, Ww) - 1
    h = rec.deriche_impulse(s, r + 1)
    j = np.abs(np.arange(-r, r + 1))
    return np.outer(h[j], h[j])


@pytest.mark.parametrize("s,Hh,Ww", [(1.3, 9, 14), (4.0, 13, 7)])
def test_gpa_matches_bruteforce_route(s, Hh, Ww):
    """Algorithm 2 with the Toeplitz-product filter equals the C checker's
    Algorithm 2 with the explicit 2-D kernel (brute-force sum over in-image
    neighbours); also the filtered planes and the parts P, Q."""
    img = synth.blocks_image(Hh, Ww, 3, 25.0, seed=int(10 * s) + Hh).astype(np.float64)
    w = _explicit_kernel(s, Hh, Ww)
    for sr, N in ((30.0, 5), (60.0, 9)):
        ro, rP, rQ = oracle.gpa_alg2(img, w, sr, N, return_parts=True)
        o, P, Q = rec.gpa_alg2_recursive(img, s, sr, N, return_parts=True)
        assert np.abs(o - ro).max() < 1e-10
        assert np.abs(P - rP).max() <= 1e-11 * np.abs(rP).max()
        assert np.abs(Q - rQ).max() <= 1e-11 * np.abs(rQ).max()
    # the filter alone: the C checker's filtered planes F_n * w of the same image
    sr = 40.0
    _, _, _, planes = oracle.gpa_alg2(img, w, sr, 3, return_parts=True, return_planes=True)
    Hs = (img - T) / sr
    F = np.exp(-Hs * Hs / 2.0)
    for n in range(4):
        assert np.abs(rec.recursive_filter(F, s) - planes[n]).max() < 1e-13
        F = Hs * F
    rows = [Hh - 1, 0, Hh // 2]
    assert np.abs(rec.recursive_filter(F, s, rows=rows) - rec.recursive_filter(F, s)[rows]).max() < 1e-13


@pytest.mark.parametrize("s,L", [(0.9, 37), (5.0, 120), (25.0, 300)])
def test_zero_state_recursions_reproduce_the_operator(s, L):
    """The two damped-cosine modes of the fit as complex one-pole recursions,
    causal from the line's start and anticausal from its end, both from zero
    state: y = sum_j 2 Re(alpha_j (s_j + q_j)) - h(0) x.  The result equals the
    checker's full-line convolution, which fixes the normalisation and every
    sign of the formula."""
    d = rec.DERICHE4
    norm = rec.deriche_raw(0, s) / rec.deriche_impulse(s, 1)[0]
    alpha = [complex(d["a0"], -d["a1"]) / 2 / norm, complex(d["c0"], -d["c1"]) / 2 / norm]
    pole = [np.exp(complex(-d["b0"], d["w0"]) / s), np.exp(complex(-d["b1"], d["w1"]) / s)]
    x = np.random.default_rng(int(L)).uniform(-1, 1, size=L)
    y = np.zeros(L)
    h0 = 0.0
    for a, r in zip(alpha, pole):
        h0 += 2 * a.real
        sc = np.zeros(L, dtype=complex)
        acc = 0j
        for i in range(L):
            acc = x[i] + r * acc
            sc[i] = acc
        qa = np.zeros(L, dtype=complex)
        acc = 0j
        for i in range(L - 1, -1, -1):
            acc = x[i] + r * acc
            qa[i] = acc
        y += 2 * (a * (sc + qa)).real
    y -= h0 * x
    ref = rec.toeplitz_line(s, L) @ x
    assert h0 == pytest.approx(rec.deriche_impulse(s, 1)[0], rel=1e-13)
    assert np.abs(y - ref).max() < 1e-12


def test_constant_image_interior():
    s = 2.5
    c = np.full((90, 110), 55.0)
    out = rec.recursive_filter(c, s)
    m = int(math.ceil(16 * s))
    assert np.abs(out[m:-m, m:-m] - 55.0).max() < 1e-9
    # and GPA of a constant image is the constant everywhere (Q cancels the edge loss)
    o = rec.gpa_alg2_recursive(c[:20, :30], s, 30.0, 8)
    assert np.abs(o - 55.0).max() < 1e-9


@pytest.mark.parametrize("s,sr", [(2.0, 30.0), (3.0, 50.0)])
def test_gpa_accuracy_against_direct_filter(s, sr):
    """With N from delta (eq. eps with w(0) = h(0)^2, eq. LambW) the GPA with
    the recursive kernel is within delta of eq. BF with the same kernel, and
    the error falls as N grows (Sec. III-C)."""
    Hh, Ww = 21, 26
    img = synth.blocks_image(Hh, Ww, 5, 20.0, seed=77).astype(np.float64)
    w = _explicit_kernel(s, Hh, Ww)
    direct = oracle.bf_direct(img, w, sr)
    w0 = rec.centre_weight_recursive(s)
    assert w0 == pytest.approx(w[w.shape[0] // 2, w.shape[1] // 2], rel=1e-14)
    lam = T * T / (sr * sr)
    errs = []
    for delta in (1.0, 0.1, 0.01):
        N, _ = order.chernoff_order_lambertw(lam, order.eps_from_delta(w0, delta))
        err = np.abs(rec.gpa_alg2_recursive(img, s, sr, N) - direct).max()
        assert err <= delta
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("s,sr,N,Hh,Ww", [(1.5, 30.0, 6, 9, 13), (3.0, 45.0, 10, 12, 8)])
def test_gradient_matches_bruteforce_chain_rule(s, sr, N, Hh, Ww):
    """The autograd gradient of the recursive Algorithm 2 equals the C
    checker's brute-force chain rule on eq. GPA (a different route: the
    ratio's derivative per neighbour) with the explicit kernel h(j_y) h(j_x)."""
    img = synth.blocks_image(Hh, Ww, 3, 25.0, seed=Hh * Ww).astype(np.float64)
    g = np.random.default_rng(5).standard_normal((Hh, Ww))
    gin, gs = rec.gpa_grad_recursive(img, s, sr, N, g)
    rgin, rgs = oracle.gpa_grad(img, _explicit_kernel(s, Hh, Ww), sr, N, g)
    assert np.abs(gin - rgin).max() <= 1e-9 * max(np.abs(rgin).max(), 1.0)
    assert gs == pytest.approx(rgs, rel=1e-9, abs=1e-12)


def test_gradient_matches_finite_differences():
    """Central differences of gpa_alg2_recursive along a random direction and
    in sigma_r (step 1e-3 / 1e-4, FP64)."""
    s, sr, N = 2.0, 35.0, 12
    img = synth.blocks_image(14, 19, 4, 20.0, seed=21).astype(np.float64)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(img.shape)
    d = rng.standard_normal(img.shape)
    gin, gs = rec.gpa_grad_recursive(img, s, sr, N, g)
    e = 1e-3
    fd = (np.sum(g * rec.gpa_alg2_recursive(img + e * d, s, sr, N))
          - np.sum(g * rec.gpa_alg2_recursive(img - e * d, s, sr, N))) / (2 * e)
    assert np.sum(gin * d) == pytest.approx(fd, rel=1e-6)
    e = 1e-4
    fds = (np.sum(g * rec.gpa_alg2_recursive(img, s, sr + e, N))
           - np.sum(g * rec.gpa_alg2_recursive(img, s, sr - e, N))) / (2 * e)
    assert gs == pytest.approx(fds, rel=1e-6)


@pytest.mark.parametrize("s,sr,N,Hh,Ww", [(1.5, 30.0, 6, 9, 13), (4.0, 50.0, 9, 12, 8)])
def test_joint_matches_bruteforce(s, sr, N, Hh, Ww):
    """The joint filter with the recursive kernel equals the C checker's
    brute-force cross filter with phi_N and the explicit kernel h(j_y) h(j_x)
    (outputs and both sums), and with guide = image it is Algorithm 2."""
    img = synth.blocks_image(Hh, Ww, 3, 25.0, seed=Hh + 2 * Ww).astype(np.float64)
    guide = synth.blocks_image(Hh, Ww, 4, 15.0, seed=Hh * Ww).astype(np.float64)
    w = _explicit_kernel(s, Hh, Ww)
    o, U, Q = rec.joint_gpa_recursive(img, guide, s, sr, N, return_parts=True)
    ro, rU, rQ = oracle.joint_gpa(img, guide, w, sr, N, return_parts=True)
    assert np.abs(o - ro).max() < 1e-9
    assert np.abs(Q - rQ).max() <= 1e-11 * np.abs(rQ).max()
    assert np.abs(U - rU).max() <= 1e-11 * max(np.abs(rU).max(), 1e-300)
    same = rec.joint_gpa_recursive(img, img, s, sr, N)
    assert np.abs(same - rec.gpa_alg2_recursive(img, s, sr, N)).max() < 1e-9
