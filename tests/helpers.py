"""Shared helpers of the GPU parity tests (comparison logic and tolerances).

Tolerances (derived in the design notes):
* filter outputs: max |GPU - checker| <= 1e-3 on the 0..255 scale, the
  accuracy target for the float32 path, on every pixel whose checker
  Q' = sum_j w(j) phi_N is at least w(0)/2, whatever N.  A pixel may exceed
  1e-3 only where eq. GPA's ratio is ill-conditioned: its numerator and
  denominator are sums of terms of both signs that nearly cancel (small N,
  outputs far outside the data range).  There the allowance is the error
  that a float32 evaluation may carry, first order:
      (7N + 2L + 4) u (S_P + |out - t_c| S_Q) / |Q'|  +  4 u |out - t_c|,
  u = 2^-24, L = taps per filter pass (2W + 1), S_P and S_Q the sums of the
  terms' magnitudes (oracle.gpa_term_magnitudes): (6N + 4) u for a term
  a_n(t) a_n(tau) built by n recursion steps from one exponential on each
  side, 2L u for the two filter passes, N u for the sum over n, and the
  final ratio.  At N = 1 every term is positive (S = |Q'|), so this never
  exceeds 1e-3 there.  Pixels with Q' < w(0)/2 compare P' and Q' directly.
* Q' (a sum of at most N+1 products of numbers in [-1, 1]): absolute error
  <= 2e-5 + 1e-5 * |Q'|.
* gradients: relative (to the largest gradient entry) 2e-3 for the image
  gradient, 1e-3 for the scalar sigma_r gradient.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1603_08109_gb300 import synth

OUT_TOL = 1e-3
Q_ATOL, Q_RTOL = 2e-5, 1e-5
U32 = 2.0 ** -24

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def image(h, w, seed, block=16, noise=20.0):
    return synth.blocks_image(h, w, block, noise, seed=seed)


def spatial(kind, radius, sigma_s):
    return oracle.spatial_kernel(kind, radius, sigma_s)


def scaled_q(img, Q_alg2, sigma_r, T=128.0):
    """Q' = Q_2 = e^{-H^2/2} Q of Algorithm 2 (App. B)."""
    H = (np.asarray(img, np.float64) - T) / sigma_r
    return Q_alg2 * np.exp(-H * H / 2)


def in_bound_regime(sigma_r, N, w0, T=128.0):
    """True when the kernel error E_N <= P(X >= N) (Prop. upperBound) is
    below w(0)/2, so Prop. accuracy guarantees Q' >= w(0)/2 at every pixel."""
    from oracle import order
    return order.poisson_tail(N, (T / sigma_r) ** 2) < 0.5 * w0


def ratio_allowance(img, w, sigma_r, N, ref_out, ref_q, pixels, tc=128.0):
    """The float32 rounding allowance of eq. GPA's ratio at `pixels` (ys, xs)
    of img (see the module docstring), or OUT_TOL where that is larger."""
    L = w.shape[0]
    sp, sq = oracle.gpa_term_magnitudes(img, w, sigma_r, N, T=tc, samples=pixels)
    dev = np.abs(ref_out - tc)
    cond = (7 * N + 2 * L + 4) * U32 * (sp + dev * sq) / np.abs(ref_q) + 4 * U32 * dev
    return np.maximum(OUT_TOL, cond)


def compare_forward(out, q, ref_out, ref_q, w0, where="", sigma_r=None, N=None, tc=128.0,
                    img=None, w=None, pixels=None):
    """Assert the parity bar; return (max out err on the mask, max Q err, unmasked count).

    Every pixel with |Q'| >= w(0)/2 must match to OUT_TOL, or, where eq. GPA's
    ratio is ill-conditioned, to its float32 rounding allowance, which needs the
    input image `img` and kernel `w` (and sigma_r, N).  `pixels` = (ys, xs)
    locates the compared values in img when they are samples."""
    out = np.asarray(out, np.float64)
    ref_out = np.asarray(ref_out, np.float64)
    ref_q = np.asarray(ref_q, np.float64)
    mask = np.abs(ref_q) >= 0.5 * w0
    err = np.abs(out - ref_out)
    emax = float(err[mask].max()) if mask.any() else 0.0
    over = mask & ~(err <= OUT_TOL)
    if over.any():
        assert img is not None and w is not None and sigma_r is not None and N is not None, \
            "%s: max |out err| %.3e > %.1e" % (where, emax, OUT_TOL)
        idx = np.nonzero(over)
        if pixels is None:
            assert out.ndim == 2, where
            pix = idx
        else:
            pix = (np.asarray(pixels[0])[idx], np.asarray(pixels[1])[idx])
        allowed = ratio_allowance(img, w, sigma_r, N, ref_out[idx], ref_q[idx], pix, tc)
        bad = ~(err[idx] <= allowed)
        assert not bad.any(), "%s: out error %.3e beyond the float32 allowance %.3e of the ratio" % (
            where, float(err[idx][bad].max()), float(allowed[bad].min()))
    if q is not None:
        q = np.asarray(q, np.float64)
        qtol = Q_ATOL + Q_RTOL * np.abs(ref_q)
        qerr = float(np.abs(q - ref_q).max())
        assert (np.abs(q - ref_q) <= qtol).all(), "%s: Q' error %.3e" % (where, qerr)
        if sigma_r is not None and (~mask).any():  # P' where the ratio is not compared
            p_gpu = (out - tc) * q / sigma_r
            p_ref = (ref_out - tc) * ref_q / sigma_r
            fin = ~mask & np.isfinite(p_gpu)
            assert (np.abs(p_gpu - p_ref)[fin] <= 2 * (Q_ATOL + Q_RTOL * np.abs(p_ref))[fin]).all(), \
                "%s: P' error" % where
    else:
        qerr = 0.0
    return emax, qerr, int((~mask).sum())
