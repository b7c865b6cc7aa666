"""CPU checker: order selection and kernel-error analysis, FP64 (Sec. II).

Test infrastructure only. Written from the paper's equations; it shares no
code with the GPU library's own order selection.

Readings (listed in the design notes):
* ``T`` is the half dynamic range (8-bit images: T = 128, Sec. III-A).
* The order N is the number of Taylor terms (eq. approx), so the kernel error
  is the Poisson tail P(X >= N), X ~ Poisson(lambda = T^2 / sigma_r^2)
  (Prop. upperBound).
* The spatial kernel is normalised to unit sum (eq. normal), so its centre
  weight is w(0) = 1 / (2r + 1)^2 for the box and 1 / (sum_k e^{-k^2/2 s^2})^2
  for the Gaussian on [-r, r]^2 (it is separable on a square).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

__all__ = [
    "centre_weight", "eps_from_delta", "poisson_tail", "chebyshev_order",
    "chernoff_order_lambertw", "chernoff_lhs", "w0_series", "algorithm1",
    "order_vs_delta_approx", "yang_order", "kernel_error", "order_from_delta",
    "poisson_order",
]


def centre_weight(kind: int, radius: int, sigma_s: float = 0.0) -> float:
    """w(0) of the normalised spatial kernel (eqs. spatial_kernel1/2, normal)."""
    if kind == 0:
        return 1.0 / float(2 * radius + 1) ** 2
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    s = float(np.sum(np.exp(-k * k / (2.0 * sigma_s * sigma_s))))
    return 1.0 / (s * s)


def eps_from_delta(w0: float, delta: float, T: float = 128.0) -> float:
    """Kernel-error budget that guarantees filter error <= delta (eq. eps)."""
    return w0 * delta / (2.0 * T + delta)


def poisson_tail(N: int, lam: float) -> float:
    """P(X >= N) for X ~ Poisson(lam): right side of Prop. upperBound.
    P(X >= N) is the regularised lower incomplete gamma P(N, lam)."""
    if N <= 0:
        return 1.0
    return float(special.gammainc(N, lam))


def chebyshev_order(lam: float, eps: float) -> int:
    """eq. cheby2: N0 = ceil(lambda + sqrt(lambda / eps))."""
    return int(math.ceil(lam + math.sqrt(lam / eps)))


def chernoff_lhs(N: float, lam: float) -> float:
    """Left side of eq. inequality: e^{-lam} (e lam)^N / N^N (in log space)."""
    return math.exp(-lam + N * (1.0 + math.log(lam)) - N * math.log(N))


def chernoff_order_lambertw(lam: float, eps: float) -> tuple[int, float]:
    """eq. LambW with p = 1 + log(lam), q = -lam - log(eps):
    theta = q / W0(q e^{-p}); returns (ceil(theta), theta).  The principal
    branch W0 gives the root of nu(x) = x log x - p x - q above lambda
    (App. A) also when q < 0."""
    p = 1.0 + math.log(lam)
    q = -lam - math.log(eps)
    z = q * math.exp(-p)
    w = special.lambertw(z, 0)
    theta = q / float(w.real)
    return int(math.ceil(theta)), theta


def w0_series(t: float) -> float:
    """Four-term series of the Lambert W0 function (eq. series)."""
    return t - t * t + 1.5 * t ** 3 - (8.0 / 3.0) * t ** 4


def algorithm1(sigma_r: float, eps: float, T: float = 128.0, as_printed: bool = False,
               newton_iters: int = 3, newton_below: float = 30.0, large_sigma: float = 70.0,
               force_newton: bool = False) -> int:
    """Algorithm 1 (estimation of the order).  ``as_printed`` uses the
    printed fourth series term 8t^3/4 instead of 8t^4/3 (eq. series); the
    printed form is kept only to show the typo."""
    if sigma_r >= large_sigma:
        return 10
    lam = (T / sigma_r) ** 2
    p = 1.0 + math.log(lam)
    q = -lam - math.log(eps)
    t = q / (math.e * lam)
    if as_printed:
        w0 = t - t * t + 1.5 * t ** 3 - 8.0 * t ** 3 / 4.0
    else:
        w0 = w0_series(t)
    n0 = q / w0
    if sigma_r < newton_below or force_newton:
        for _ in range(newton_iters):
            n0 = n0 - (n0 * math.log(n0) - p * n0 - q) / (math.log(n0) + 1.0 - p)
    return int(math.ceil(n0))


def order_vs_delta_approx(sigma_r: float, w0: float, delta: float, T: float = 128.0) -> float:
    """eq. Nvsdelta: N0 ~ 1.72 (T/sigma_r)^2 + log(2T / (w(0) delta))."""
    return 1.72 * (T / sigma_r) ** 2 + math.log(2.0 * T / (w0 * delta))


def yang_order(sigma_r: float, delta: float) -> float:
    """eq. Nest (the comparison method's estimate, quoted by the paper)."""
    return 1.14e5 / (math.sqrt(delta) * sigma_r ** 2)


def kernel_error(N: int, sigma_r: float, t: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """E_{N,sigma_r}(t, tau) of eq. error, as g(t - tau) - phi_N(t, tau)."""
    t = np.asarray(t, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    s2 = sigma_r * sigma_r
    x = t * tau / s2
    poly = np.zeros_like(x)
    term = np.ones_like(x)
    for n in range(N):
        poly += term
        term = term * x / (n + 1)
    phi = np.exp(-(t * t + tau * tau) / (2 * s2)) * poly
    return np.exp(-((t - tau) ** 2) / (2 * s2)) - phi


def order_from_delta(kind: int, radius: int, sigma_s: float, sigma_r: float, delta: float,
                     T: float = 128.0) -> int:
    """N from the filter accuracy delta: eq. eps then eq. LambW."""
    eps = eps_from_delta(centre_weight(kind, radius, sigma_s), delta, T)
    return chernoff_order_lambertw((T / sigma_r) ** 2, eps)[0]


def poisson_order(lam: float, eps: float) -> int:
    """Smallest N with P(X >= N) <= eps (the exact tail, Prop. upperBound)."""
    N = 1
    while poisson_tail(N, lam) > eps:
        N += 1
    return N
