"""CPU checker: Algorithm 2 with the recursive O(1) Gaussian spatial filter --
test infrastructure only (tests, the smoke check and the benchmark's CPU
leg); it shares no code, constant or table with the GPU library.

Sec. I and Sec. III-A state that the N + 1 spatial filterings of Algorithm 2
cost O(1) per pixel for a Gaussian w when the Gaussian is implemented by
recursion, citing Deriche's recursive Gaussian.  The operator checked here is
Deriche's fourth-order approximation: for k >= 0 the (unnormalised) impulse
response is

    h(k) = (a0 cos(w0 k/s) + a1 sin(w0 k/s)) exp(-b0 k/s)
         + (c0 cos(w1 k/s) + c1 sin(w1 k/s)) exp(-b1 k/s),

s = sigma_s, mirrored for k < 0, with Deriche's published fit constants
(DERICHE4 below; h(0) = a0 + c0 ~ 1 approximates exp(-k^2 / 2 s^2)).  The
checker normalises h to unit sum over all integers (eq. normal).  A recursive
implementation that starts its causal and anticausal recursions from zero
state at the two ends of each image line computes exactly the convolution of
the zero-extended line with h; this checker evaluates that convolution as
written -- every in-line neighbour, no truncation -- once along columns and
once along rows, as products with the Toeplitz matrices T[i, k] = h(|i - k|).
The zero extension is the same reading of the finite image domain (Sec. I) as
for the truncated kernels: only neighbours inside the image contribute.

Algorithm 2 then runs step by step in FP64 with this operator as F * w;
its gradient (image and sigma_r, N fixed) is taken by FP64 reverse-mode
differentiation of those same steps.  The cross (joint) filter with the same
operator is written out as its 2N filterings.

Readings (also listed in the design notes):
* The spatial support is the whole image (the recursion has an infinite
  impulse response); w(j) = h(j_y) h(j_x), so w(0) = h(0)^2 enters the order
  selection (eq. eps) in place of the truncated Gaussian's w(0).
* h has tiny negative lobes (about -1.4e-4 of its peak near k = 3.6 s): the
  fit is not a positive kernel, so Prop. upperBound's guarantee is checked
  numerically rather than assumed.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["DERICHE4", "deriche_raw", "deriche_impulse", "toeplitz_line",
           "recursive_filter", "gpa_alg2_recursive", "gpa_grad_recursive",
           "joint_gpa_recursive", "centre_weight_recursive"]

# Deriche's fourth-order fit of the Gaussian (two damped cosine/sine pairs).
DERICHE4 = {"a0": 1.680, "a1": 3.735, "b0": 1.783, "w0": 0.6318,
            "c0": -0.6803, "c1": -0.2598, "b1": 1.723, "w1": 1.997}


def deriche_raw(k, sigma_s: float) -> np.ndarray:
    """Unnormalised impulse response h(|k|) of the fit (the formula above)."""
    d = DERICHE4
    x = np.abs(np.asarray(k, dtype=np.float64)) / float(sigma_s)
    return ((d["a0"] * np.cos(d["w0"] * x) + d["a1"] * np.sin(d["w0"] * x)) * np.exp(-d["b0"] * x)
            + (d["c0"] * np.cos(d["w1"] * x) + d["c1"] * np.sin(d["w1"] * x)) * np.exp(-d["b1"] * x))


def _unit_sum(sigma_s: float) -> float:
    """Sum of the unnormalised h over all integers, by a direct sum over
    |k| <= 80 s + 64 (the envelope exp(-1.72 |k| / s) is below 1e-59 there)."""
    K = int(math.ceil(80.0 * sigma_s)) + 64
    k = np.arange(-K, K + 1)
    return float(np.sum(deriche_raw(k, sigma_s)))


def deriche_impulse(sigma_s: float, L: int) -> np.ndarray:
    """Normalised h(k), k = 0 .. L-1 (sum over all integers of h(|k|) is 1)."""
    if not sigma_s > 0:
        raise ValueError("sigma_s must be > 0")
    return deriche_raw(np.arange(L), sigma_s) / _unit_sum(sigma_s)


def centre_weight_recursive(sigma_s: float) -> float:
    """w(0) = h(0)^2 of the separable recursive kernel."""
    h0 = float(deriche_impulse(sigma_s, 1)[0])
    return h0 * h0


def toeplitz_line(sigma_s: float, L: int) -> np.ndarray:
    """L x L matrix T[i, k] = h(|i - k|): one image line of length L filtered
    with every in-line neighbour (zero extension outside the line)."""
    h = deriche_impulse(sigma_s, L)
    i = np.arange(L)
    return h[np.abs(i[:, None] - i[None, :])]


def recursive_filter(img, sigma_s: float, rows=None) -> np.ndarray:
    """F * w for w = h (x) h over the whole (zero-extended) image: columns
    filtered by T_H, rows by T_W.  `rows` (optional) selects output rows."""
    F = np.asarray(img, dtype=np.float64)
    Hh, Ww = F.shape
    TH = toeplitz_line(sigma_s, Hh)
    TW = toeplitz_line(sigma_s, Ww)
    if rows is not None:
        TH = TH[np.asarray(rows)]
    return TH @ F @ TW.T


def gpa_alg2_recursive(img, sigma_s: float, sigma_r: float, N: int, T: float = 128.0,
                       rows=None, return_parts: bool = False):
    """Algorithm 2 (GPA) with the recursive Gaussian as the spatial filter, in
    the paper's order of steps, FP64.  P includes the factor sigma_r of the
    last step (out = P / Q + T).  `rows` (optional) evaluates the output rows
    listed only (the filter still reads the whole image)."""
    f = np.asarray(img, dtype=np.float64)
    Hh, Ww = f.shape
    TH = toeplitz_line(sigma_s, Hh)
    TW = toeplitz_line(sigma_s, Ww)
    THr = TH if rows is None else TH[np.asarray(rows)]
    sel = (lambda a: a) if rows is None else (lambda a: a[np.asarray(rows)])

    def filt(F):
        return THr @ F @ TW.T

    h = f - T
    F = np.exp(-h * h / (2.0 * sigma_r * sigma_r))  # the one transcendental
    Hs = h / sigma_r
    G = np.ones_like(sel(f))
    P = np.zeros_like(G)
    Q = np.zeros_like(G)
    Hsel = sel(Hs)
    Fbar = filt(F)
    for n in range(1, N + 1):
        Q = Q + G * Fbar
        F = Hs * F
        Fbar = filt(F)
        P = P + G * Fbar
        G = Hsel * G / n
    out = sigma_r * (P / Q) + T
    if return_parts:
        return out, sigma_r * P, Q
    return out


def gpa_grad_recursive(img, sigma_s: float, sigma_r: float, N: int, gout, T: float = 128.0):
    """(d loss / d image, d loss / d sigma_r) of gpa_alg2_recursive for
    loss = sum(gout * out), N held fixed: reverse-mode differentiation in
    FP64 (plain PyTorch CPU autograd) through the same Algorithm 2 steps with
    the same Toeplitz-product filter."""
    import torch
    f = torch.tensor(np.asarray(img, dtype=np.float64), requires_grad=True)
    sr = torch.tensor(float(sigma_r), dtype=torch.float64, requires_grad=True)
    Hh, Ww = f.shape
    TH = torch.from_numpy(toeplitz_line(sigma_s, Hh))
    TW = torch.from_numpy(toeplitz_line(sigma_s, Ww))

    def filt(F):
        return TH @ F @ TW.T

    h = f - T
    F = torch.exp(-h * h / (2.0 * sr * sr))
    Hs = h / sr
    G = torch.ones_like(f)
    P = torch.zeros_like(f)
    Q = torch.zeros_like(f)
    Fbar = filt(F)
    for n in range(1, N + 1):
        Q = Q + G * Fbar
        F = Hs * F
        Fbar = filt(F)
        P = P + G * Fbar
        G = Hs * G / n
    out = sr * (P / Q) + T
    (out * torch.from_numpy(np.asarray(gout, dtype=np.float64))).sum().backward()
    return f.grad.numpy(), float(sr.grad)


def joint_gpa_recursive(img, guide, sigma_s: float, sigma_r: float, N: int, T: float = 128.0,
                        return_parts: bool = False):
    """Cross (joint) bilateral filter (Sec. I, Sec. V) with phi_N on centred
    guide values and the recursive Gaussian as w, written as its N + N
    filterings: with B_n = e^{-G^2/2} G^n / n!-weighted guide power images
    (G = (guide - T) / sigma_r), out = T + U / Q where
    Q = sum_{n<N} (G^n / n!) e^{-G^2/2} (w * (e^{-G^2/2} G^n)) and
    U = sum_{n<N} (G^n / n!) e^{-G^2/2} (w * (e^{-G^2/2} G^n (img - T))),
    in FP64 with the Toeplitz-product filter.  Parts are U and Q."""
    f = np.asarray(img, dtype=np.float64)
    e = np.asarray(guide, dtype=np.float64)
    Hh, Ww = f.shape
    TH = toeplitz_line(sigma_s, Hh)
    TW = toeplitz_line(sigma_s, Ww)

    def filt(F):
        return TH @ F @ TW.T

    g = e - T
    E = np.exp(-g * g / (2.0 * sigma_r * sigma_r))
    Gs = g / sigma_r
    F = E.copy()         # e^{-G^2/2} G^n
    C = E.copy()         # e^{-G^2/2} G^n / n!  (the centre's factor)
    U = np.zeros_like(f)
    Q = np.zeros_like(f)
    for n in range(N):
        if n > 0:
            F = Gs * F
            C = Gs * C / n
        Q = Q + C * filt(F)
        U = U + C * filt(F * (f - T))
    out = U / Q + T
    return (out, U, Q) if return_parts else out
