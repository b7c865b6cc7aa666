"""Pins for the checker's order selection and kernel-error analysis (Sec. II).

Each test ties the checker to something the paper prints or the mathematics
fixes: the order tables (golden files), the Poisson-tail bound of
Prop. upperBound on a dense grid, the Chernoff inequality at the returned
order, and the closed forms of eq. cheby2 / eq. Nvsdelta.
"""
import math
import os

import numpy as np
import pytest

from oracle import order

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_table1_lambertw_row():
    """N0' of Table 1: ceil(q / W0(q e^{-p})) with eps = 1e-3, T = 128."""
    for sr, n1, _, _ in _rows("order_vs_sigma_r.txt"):
        assert order.chernoff_order_lambertw((128.0 / sr) ** 2, 1e-3)[0] == int(n1)


def test_table1_series_row_needs_corrected_fourth_term():
    """N0'' of Table 1 comes from eq. series with -8t^4/3; Algorithm 1's
    printed -8t^3/4 does not reproduce it (the printed term is a typo)."""
    rows = _rows("order_vs_sigma_r.txt")
    mism = 0
    for sr, _, n2, _ in rows:
        lam = (128.0 / sr) ** 2
        q = -lam - math.log(1e-3)
        t = q / (math.e * lam)
        assert math.ceil(q / order.w0_series(t)) == int(n2)
        printed = q / (t - t * t + 1.5 * t ** 3 - 8.0 * t ** 3 / 4.0)
        mism += math.ceil(printed) != int(n2)
    assert mism >= 3


def test_table1_newton_row_is_algorithm1():
    """N0''' of Table 1 equals Algorithm 1 (series, Newton below sigma_r=30)."""
    for sr, _, _, n3 in _rows("order_vs_sigma_r.txt"):
        assert order.algorithm1(sr, 1e-3) == int(n3)
        assert order.algorithm1(sr, 1e-3, force_newton=True) == int(n3)


def test_chernoff_order_is_smallest_integer_satisfying_inequality():
    """ceil(theta) satisfies eq. inequality and ceil(theta) - 1 does not."""
    for sr in (10.0, 17.0, 25.0, 40.0, 60.0):
        lam = (128.0 / sr) ** 2
        for eps in (1e-1, 1e-3, 1e-6, 1e-9):
            n0, theta = order.chernoff_order_lambertw(lam, eps)
            assert theta > lam
            assert order.chernoff_lhs(n0, lam) <= eps * (1 + 1e-12)
            if n0 - 1 > lam:
                assert order.chernoff_lhs(n0 - 1, lam) > eps


def test_order_vs_delta_table():
    """Table orderComp: LambW row exact with T=127, +-1 with T=128;
    Nvsdelta row exact with T=128 (nearest integer)."""
    w0 = order.centre_weight(1, 15, 5.0)
    assert w0 == pytest.approx(6.3905e-3, rel=1e-3)
    for delta, n_lw, n_nd in _rows("order_vs_delta.txt"):
        eps127 = order.eps_from_delta(w0, delta, 127.0)
        assert order.chernoff_order_lambertw((127.0 / 30.0) ** 2, eps127)[0] == int(n_lw)
        eps128 = order.eps_from_delta(w0, delta, 128.0)
        n128 = order.chernoff_order_lambertw((128.0 / 30.0) ** 2, eps128)[0]
        assert abs(n128 - int(n_lw)) <= 1
        assert round(order.order_vs_delta_approx(30.0, w0, delta, 128.0)) == int(n_nd)


def test_text_example_nvsdelta_box3x3():
    """Sec. IV text: box 3x3, sigma_r = 50 gives N0 of about 24 at delta=0.01
    and about 19 at delta = 3 (eq. Nvsdelta)."""
    w0 = order.centre_weight(0, 1)
    assert w0 == pytest.approx(1.0 / 9.0)
    assert abs(order.order_vs_delta_approx(50.0, w0, 0.01) - 24) < 1.0
    assert abs(order.order_vs_delta_approx(50.0, w0, 3.0) - 19) < 1.5


def test_poisson_tail_matches_direct_sum_and_bounds():
    """P(X >= N) from the incomplete gamma equals the summed Poisson pmf
    (computed with lgamma), and lies below the Chernoff and Chebyshev
    bounds whenever N > lambda."""
    for lam in (0.5, 4.0, 18.2, 163.84):
        for N in (1, 2, int(lam) + 3, int(2 * lam) + 10):
            tail = order.poisson_tail(N, lam)
            terms = [math.exp(-lam + n * math.log(lam) - math.lgamma(n + 1))
                     for n in range(N, N + 2000)]
            assert tail == pytest.approx(math.fsum(terms), rel=1e-10, abs=1e-300)
            if N > lam:
                assert tail <= order.chernoff_lhs(N, lam) * (1 + 1e-12)
                assert tail <= lam / (N - lam) ** 2 * (1 + 1e-12)


def test_chebyshev_order_closed_form():
    lam, eps = (128.0 / 30.0) ** 2, 1e-3
    n0 = order.chebyshev_order(lam, eps)
    assert n0 == math.ceil(lam + math.sqrt(lam / eps))
    assert lam / (n0 - lam) ** 2 <= eps


@pytest.mark.parametrize("sr,N", [(30.0, 40), (30.0, 20), (50.0, 19), (15.0, 107), (80.0, 6)])
def test_kernel_error_below_poisson_tail_on_dense_grid(sr, N):
    """Prop. upperBound: max |E_N| over [-T, T]^2 <= P(X >= N)."""
    T = 128.0
    t = np.linspace(-T, T, 513)
    tt, uu = np.meshgrid(t, t)
    err = np.abs(order.kernel_error(N, sr, tt, uu)).max()
    bound = order.poisson_tail(N, (T / sr) ** 2)
    assert err <= bound * (1 + 1e-9) + 1e-15


def test_kernel_error_bound_same_order_of_magnitude():
    """Fig. errorBound (T = 128, sigma_r = 30, N = 40): the grid supremum of
    the error and the bound are of the same order of magnitude; the
    supremum sits on the boundary t tau = +-T^2 as the proof predicts."""
    T, sr, N = 128.0, 30.0, 40
    t = np.linspace(-T, T, 1025)
    tt, uu = np.meshgrid(t, t)
    e = np.abs(order.kernel_error(N, sr, tt, uu))
    bound = order.poisson_tail(N, (T / sr) ** 2)
    assert 0.1 * bound <= e.max() <= bound
    iy, ix = np.unravel_index(np.argmax(e), e.shape)
    assert abs(tt[iy, ix] * uu[iy, ix]) == pytest.approx(T * T, rel=0.02)


def test_kernel_error_converges():
    """eq. asymp2: phi_N -> g pointwise as N grows."""
    t = np.linspace(-128, 128, 65)
    tt, uu = np.meshgrid(t, t)
    prev = np.inf
    for N in (10, 30, 60, 120):
        e = np.abs(order.kernel_error(N, 30.0, tt, uu)).max()
        assert e < prev
        prev = e
    assert prev < 1e-12


def test_poisson_order_not_above_chernoff_order():
    for sr in (10.0, 30.0, 60.0):
        lam = (128.0 / sr) ** 2
        for eps in (1e-3, 1e-6):
            assert order.poisson_order(lam, eps) <= order.chernoff_order_lambertw(lam, eps)[0]
