"""Shared helpers of the GPU parity tests (comparison logic and tolerances).

Tolerances (derived in the design notes):
* filter outputs: max |GPU - checker| <= 1e-3 on the 0..255 scale, the
  accuracy target for the float32 path; compared on pixels whose checker
  Q' = sum_j w(j) phi_N is at least w(0)/2 (elsewhere the ratio P'/Q' is
  ill-conditioned or undefined for small N, and Q' itself is compared).
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


def compare_forward(out, q, ref_out, ref_q, w0, where="", sigma_r=None, N=None, tc=128.0):
    """Assert the parity bar; return (max out err on the mask, max Q err, masked count).

    In the accuracy-bound regime (or when sigma_r/N are not given) every pixel
    with |Q'| >= w(0)/2 must match to OUT_TOL.  Below it (N far under the
    order the bound asks for, e.g. N = 2), Q' nearly cancels at some pixels and
    the ratio is ill-conditioned in any finite precision; there Q' and
    P' = (out - t_c) Q' / sigma_r are compared directly to the Q' tolerance,
    and out to max(OUT_TOL, the error those tolerances propagate to the ratio)."""
    out = np.asarray(out, np.float64)
    mask = np.abs(ref_q) >= 0.5 * w0
    err = np.abs(out - ref_out)
    strict = sigma_r is None or N is None or in_bound_regime(sigma_r, N, w0)
    if strict or q is None:
        emax = float(err[mask].max()) if mask.any() else 0.0
        assert emax <= OUT_TOL, "%s: max |out err| %.3e > %.1e" % (where, emax, OUT_TOL)
    else:
        eps = Q_ATOL + Q_RTOL * np.abs(ref_q)
        bound = (sigma_r * eps + np.abs(ref_out - tc) * eps) / np.maximum(np.abs(ref_q) - eps, 1e-30)
        allowed = np.maximum(OUT_TOL, 2.0 * bound)
        assert (err[mask] <= allowed[mask]).all(), "%s: out error beyond the propagated bound" % where
        emax = float(err[mask].max()) if mask.any() else 0.0
        qq = np.asarray(q, np.float64)
        p_gpu = (out - tc) * qq / sigma_r
        p_ref = (ref_out - tc) * ref_q / sigma_r
        fin = np.isfinite(p_gpu)
        assert (np.abs(p_gpu - p_ref)[fin] <= (Q_ATOL + Q_RTOL * np.abs(p_ref))[fin] * 2).all(), \
            "%s: P' error" % where
    qerr = 0.0
    if q is not None:
        q = np.asarray(q, np.float64)
        qd = np.abs(q - ref_q) - (Q_ATOL + Q_RTOL * np.abs(ref_q))
        qerr = float(np.abs(q - ref_q).max())
        assert qd.max() <= 0, "%s: Q' error %.3e" % (where, qerr)
    return emax, qerr, int((~mask).sum())
