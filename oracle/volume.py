"""CPU checker: the bilateral filter and Algorithm 2 on volume (or video) data --
test infrastructure only (tests, the smoke check and the benchmark's CPU
leg); it shares no code, constant or table with the GPU library.

Sec. I and Sec. V note that the filter extends directly to video and volume
data.  The reading checked here keeps everything of eq. BF and Algorithm 2
except the dimension of the domain: f is a grayscale volume on a finite box
of Z^3 (depth, height, width), the range kernel is the same Gaussian of the
intensity difference, and the spatial kernel is the separable product
w(j) = w1(j_z) w1(j_y) w1(j_x) of the normalised 1-D box or Gaussian of the
planar filter, the same along every axis.  Neighbours outside the volume do
not contribute (zero extension, as for images).  Then w(0) = w1(0)^3 enters
the order selection (eq. eps) in place of the planar w(0).  Colour data would
need a range kernel on vectors, which the paper does not give; it is not
covered.

Functions (FP64):
* ``taps_1d``            -- w1 from the planar kernel of the C checker.
* ``filter3``            -- F * w: zero-extended correlation with w1 along
                            each axis (scipy.ndimage.correlate1d, mode constant).
* ``gpa_alg2_volume``    -- Algorithm 2 step by step with filter3 as F * w.
* ``bf_direct_volume``   -- eq. BF over the in-volume neighbours, brute force.
* ``gpa_definition_volume`` -- eq. GPA with phi_N of eq. GaussPolynomial,
                            brute force (tiny volumes).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

from . import spatial_kernel

__all__ = ["taps_1d", "centre_weight_volume", "filter3", "gpa_alg2_volume",
           "bf_direct_volume", "gpa_definition_volume"]


def taps_1d(kind: int, radius: int, sigma_s: float = 0.0) -> np.ndarray:
    """Normalised 1-D kernel w1 on [-r, r]: the column sums of the checker's
    normalised planar kernel w1 (x) w1 (w1 sums to 1)."""
    return spatial_kernel(kind, radius, sigma_s).sum(axis=0)


def centre_weight_volume(kind: int, radius: int, sigma_s: float = 0.0) -> float:
    """w(0) = w1(0)^3 of the separable volume kernel."""
    w1 = taps_1d(kind, radius, sigma_s)
    return float(w1[radius] ** 3)


def filter3(vol, w1) -> np.ndarray:
    """F * w with w = w1 (x) w1 (x) w1 over the in-volume neighbours."""
    F = np.asarray(vol, dtype=np.float64)
    w1 = np.asarray(w1, dtype=np.float64)
    for axis in range(3):
        F = ndimage.correlate1d(F, w1, axis=axis, mode="constant", cval=0.0)
    return F


def gpa_alg2_volume(vol, kind: int, radius: int, sigma_s: float, sigma_r: float, N: int,
                    T: float = 128.0, return_parts: bool = False):
    """Algorithm 2 (GPA) on a volume, in the paper's order of steps, FP64.
    P includes the factor sigma_r of the last step (out = P / Q + T)."""
    f = np.asarray(vol, dtype=np.float64)
    w1 = taps_1d(kind, radius, sigma_s)
    h = f - T
    F = np.exp(-h * h / (2.0 * sigma_r * sigma_r))
    Hs = h / sigma_r
    G = np.ones_like(f)
    P = np.zeros_like(f)
    Q = np.zeros_like(f)
    Fbar = filter3(F, w1)
    for n in range(1, N + 1):
        Q = Q + G * Fbar
        F = Hs * F
        Fbar = filter3(F, w1)
        P = P + G * Fbar
        G = Hs * G / n
    out = sigma_r * (P / Q) + T
    if return_parts:
        return out, sigma_r * P, Q
    return out


def _span(n, d):
    """Along an axis of length n: the indices i with i - d inside [0, n), and
    the matching source indices i - d (both empty when |d| >= n)."""
    lo = max(d, 0)
    hi = max(n + min(d, 0), lo)
    return slice(lo, hi), slice(lo - d, hi - d)


def _shifted(f, dz, dy, dx):
    """(f(i - j), inside) for the offset j = (dz, dy, dx): the neighbour's
    value and whether it lies in the volume."""
    D, H, W = f.shape
    val = np.zeros_like(f)
    ins = np.zeros(f.shape, dtype=bool)
    (zs, zt), (ys, yt), (xs, xt) = _span(D, dz), _span(H, dy), _span(W, dx)
    val[zs, ys, xs] = f[zt, yt, xt]
    ins[zs, ys, xs] = True
    return val, ins


def bf_direct_volume(vol, kind: int, radius: int, sigma_s: float, sigma_r: float) -> np.ndarray:
    """Eq. BF with i, j in Z^3: sum over the in-volume neighbours i - j of
    w(j) g(f(i - j) - f(i)) f(i - j), divided by the sum of the weights."""
    f = np.asarray(vol, dtype=np.float64)
    w1 = taps_1d(kind, radius, sigma_s)
    num = np.zeros_like(f)
    den = np.zeros_like(f)
    r = radius
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                w = w1[dz + r] * w1[dy + r] * w1[dx + r]
                val, ins = _shifted(f, dz, dy, dx)
                g = np.exp(-(val - f) ** 2 / (2.0 * sigma_r * sigma_r)) * ins
                num += w * g * val
                den += w * g
    return num / den


def gpa_definition_volume(vol, kind: int, radius: int, sigma_s: float, sigma_r: float, N: int,
                          T: float = 128.0) -> np.ndarray:
    """Eq. GPA with i, j in Z^3: the Gaussian range kernel replaced by
    phi_N(t, tau) = exp(-(s^2 + u^2) / 2) sum_{n<N} (s u)^n / n!, with s, u the
    centred intensities (t - T) / sigma_r, (tau - T) / sigma_r (eq.
    GaussPolynomial), summed over the in-volume neighbours."""
    f = np.asarray(vol, dtype=np.float64)
    w1 = taps_1d(kind, radius, sigma_s)
    u = (f - T) / sigma_r
    num = np.zeros_like(f)
    den = np.zeros_like(f)
    r = radius
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                w = w1[dz + r] * w1[dy + r] * w1[dx + r]
                val, ins = _shifted(f, dz, dy, dx)
                s = (val - T) / sigma_r
                series = np.zeros_like(f)
                for n in range(N):
                    series += (s * u) ** n / math.factorial(n)
                phi = np.exp(-(s * s + u * u) / 2.0) * series * ins
                num += w * phi * (val - T)
                den += w * phi
    return T + num / den
