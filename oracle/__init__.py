"""CPU checker for the GPU bilateral-filter library -- test infrastructure.

Plain FP64 implementations written from Chaudhury & Dabhade, "Fast and
Provably Accurate Bilateral Filtering" (arXiv 1603.08109):

* ``bf_direct``          -- eq. BF (direct bilateral filter), brute force.
* ``gpa_definition``     -- eq. GPA with phi_N of eq. GaussPolynomial, brute force.
* ``gpa_alg2``           -- Algorithm 2 (GPA) step by step over whole images.
* ``gpa_alg2_at``        -- Algorithm 2 evaluated at sampled pixels.
* ``gpa_term_magnitudes`` -- the sums of eq. GPA's terms in absolute value
                            (the conditioning of its ratio).
* ``*_grad``             -- exact derivatives of eq. BF / eq. GPA with respect
                            to the image and sigma_r (chain rule on the ratio).
* ``order``              -- order selection and kernel error (Sec. II).
* ``recursive``          -- Algorithm 2 with the recursive (Deriche) Gaussian
                            as the spatial filter, the O(1) route of Sec. III-A.
* ``volume``             -- eq. BF, eq. GPA and Algorithm 2 on volume / video
                            data (a box of Z^3, separable kernel), Sec. I, Sec. V.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package. It shares no code with the GPU library. Parity status of each
function is pinned by ``tests/test_oracle_*.py``; nothing here is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_bf.c")
_LIB = os.path.join(_HERE, "liboracle_bf.so")
_lib = None

BOX, GAUSS = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle_bf.c with gcc (FP64, OpenMP, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared",
           "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_spatial_kernel.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        lib.orc_range_filter.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ip, ip, ctypes.c_long, dp, dp, dp]
        lib.orc_range_filter_grad.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_double, dp, ip, ip, ctypes.c_long, dp, dp]
        lib.orc_gpa_alg2.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp, dp,
                                     dp]
        lib.orc_gpa_alg2_at.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_double, ip, ip,
                                        ctypes.c_long, dp, dp, dp]
        lib.orc_joint_filter.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ip, ip, ctypes.c_long, dp, dp, dp]
        for fn in ("orc_spatial_kernel", "orc_range_filter", "orc_range_filter_grad",
                   "orc_gpa_alg2", "orc_gpa_alg2_at", "orc_joint_filter"):
            getattr(lib, fn).restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(img):
    return np.ascontiguousarray(np.asarray(img, dtype=np.float64))


def _check(rc, name):
    if rc < 0:
        raise ValueError("%s: bad arguments (rc=%d)" % (name, rc))
    if rc > 0:
        raise FloatingPointError("%s: non-finite value (rc=%d)" % (name, rc))


def spatial_kernel(kind: int, radius: int, sigma_s: float = 0.0) -> np.ndarray:
    """Normalised 2-D spatial kernel on [-r, r]^2 (eqs. spatial_kernel1/2, normal)."""
    S = 2 * radius + 1
    w = np.zeros((S, S), dtype=np.float64)
    _check(_load().orc_spatial_kernel(int(kind), int(radius), float(sigma_s), _dp(w)),
           "spatial_kernel")
    return w


def _samples(samples):
    if samples is None:
        return None, None, 0
    ys = np.ascontiguousarray(np.asarray(samples[0], dtype=np.int32))
    xs = np.ascontiguousarray(np.asarray(samples[1], dtype=np.int32))
    return ys, xs, int(ys.size)


def _range_filter(kind, img, w, sigma_r, N, T, samples):
    f = _f64(img)
    H, W = f.shape
    r = (w.shape[0] - 1) // 2
    ys, xs, ns = _samples(samples)
    n = ns if ys is not None else H * W
    out = np.empty(n, dtype=np.float64)
    num = np.empty(n, dtype=np.float64)
    den = np.empty(n, dtype=np.float64)
    rc = _load().orc_range_filter(kind, _dp(f), H, W, _dp(np.ascontiguousarray(w)), r,
                                  float(sigma_r), int(N), float(T), _ip(ys), _ip(xs), ns,
                                  _dp(out), _dp(num), _dp(den))
    _check(rc, "range_filter")
    if ys is None:
        return out.reshape(H, W), num.reshape(H, W), den.reshape(H, W)
    return out, num, den


def bf_direct(img, w, sigma_r, T=128.0, samples=None, return_parts=False):
    """eq. BF, brute force. ``samples``: optional (ys, xs) pixel lists."""
    out, num, den = _range_filter(0, img, w, sigma_r, 1, T, samples)
    return (out, num, den) if return_parts else out


def gpa_definition(img, w, sigma_r, N, T=128.0, samples=None, return_parts=False):
    """eq. GPA with the Gaussian-polynomial phi_N (eq. GaussPolynomial),
    brute force. Parts: num = P_2, den = Q_2 of App. C."""
    out, num, den = _range_filter(1, img, w, sigma_r, N, T, samples)
    return (out, num, den) if return_parts else out


def gpa_term_magnitudes(img, w, sigma_r, N, T=128.0, samples=None):
    """Magnitudes of the sums behind eq. GPA's ratio, term by term:
    S_P = sum_j w(j) |t| sum_{n<N} |a_n(t) a_n(tau)| and
    S_Q = sum_j w(j) sum_{n<N} |a_n(t) a_n(tau)| (t = f(i-j) - T, tau = f(i) - T,
    the n-th term of phi_N in eq. GaussPolynomial taken in absolute value).
    Same units as ``gpa_definition``'s (num, den).  A finite-precision
    evaluation of eq. GPA in any summation order carries absolute errors of
    order u * S_P and u * S_Q in its numerator and denominator; where the terms
    cancel (S_Q >> |den|) the ratio is ill-conditioned."""
    _, num, den = _range_filter(2, img, w, sigma_r, N, T, samples)
    return num, den


def _joint(kind, img, guide, w, sigma_r, N, T, samples):
    f = _f64(img)
    e = _f64(guide)
    assert f.shape == e.shape
    H, W = f.shape
    r = (w.shape[0] - 1) // 2
    ys, xs, ns = _samples(samples)
    n = ns if ys is not None else H * W
    out = np.empty(n)
    num = np.empty(n)
    den = np.empty(n)
    rc = _load().orc_joint_filter(kind, _dp(f), _dp(e), H, W, _dp(np.ascontiguousarray(w)), r,
                                  float(sigma_r), int(N), float(T), _ip(ys), _ip(xs), ns,
                                  _dp(out), _dp(num), _dp(den))
    _check(rc, "joint_filter")
    if ys is None:
        return out.reshape(H, W), num.reshape(H, W), den.reshape(H, W)
    return out, num, den


def joint_direct(img, guide, w, sigma_r, T=128.0, samples=None, return_parts=False):
    """Cross (joint) bilateral filter (Sec. I, Sec. V): exact Gaussian range
    kernel on the guide, average of img."""
    res = _joint(0, img, guide, w, sigma_r, 1, T, samples)
    return res if return_parts else res[0]


def joint_gpa(img, guide, w, sigma_r, N, T=128.0, samples=None, return_parts=False):
    """Cross bilateral filter with the range kernel replaced by phi_N
    (eq. GaussPolynomial) on guide values, brute force."""
    res = _joint(1, img, guide, w, sigma_r, N, T, samples)
    return res if return_parts else res[0]


def gpa_alg2(img, w, sigma_r, N, T=128.0, return_parts=False, return_planes=False):
    """Algorithm 2 over the whole image; parts are eq. P and eq. Q; planes
    are the N + 1 filtered images Fbar_n = F_n * w of eq. spatialFiltering."""
    f = _f64(img)
    H, W = f.shape
    r = (w.shape[0] - 1) // 2
    out = np.empty((H, W))
    P = np.empty((H, W))
    Q = np.empty((H, W))
    planes = np.empty((N + 1, H, W)) if return_planes else None
    rc = _load().orc_gpa_alg2(_dp(f), H, W, _dp(np.ascontiguousarray(w)), r, float(sigma_r),
                              int(N), float(T), _dp(out), _dp(P), _dp(Q), _dp(planes))
    _check(rc, "gpa_alg2")
    res = (out, P, Q) if return_parts else (out,)
    if return_planes:
        res = res + (planes,)
    return res if len(res) > 1 else res[0]


def gpa_alg2_at(img, w, sigma_r, N, samples, T=128.0, return_parts=False):
    """Algorithm 2 evaluated at sampled pixels (ys, xs)."""
    f = _f64(img)
    H, W = f.shape
    r = (w.shape[0] - 1) // 2
    ys, xs, ns = _samples(samples)
    out = np.empty(ns)
    P = np.empty(ns)
    Q = np.empty(ns)
    rc = _load().orc_gpa_alg2_at(_dp(f), H, W, _dp(np.ascontiguousarray(w)), r, float(sigma_r),
                                 int(N), float(T), _ip(ys), _ip(xs), ns, _dp(out), _dp(P), _dp(Q))
    _check(rc, "gpa_alg2_at")
    return (out, P, Q) if return_parts else out


def _grad(kind, img, w, sigma_r, N, gout, T, samples):
    f = _f64(img)
    H, W = f.shape
    r = (w.shape[0] - 1) // 2
    g = _f64(gout)
    assert g.shape == f.shape
    ys, xs, ns = _samples(samples)
    n = ns if ys is not None else H * W
    gin = np.empty(n)
    gs = np.zeros(1)
    rc = _load().orc_range_filter_grad(kind, _dp(f), H, W, _dp(np.ascontiguousarray(w)), r,
                                       float(sigma_r), int(N), float(T), _dp(g), _ip(ys),
                                       _ip(xs), ns, _dp(gin), _dp(gs))
    _check(rc, "range_filter_grad")
    if ys is None:
        gin = gin.reshape(H, W)
    return gin, float(gs[0])


def bf_direct_grad(img, w, sigma_r, gout, T=128.0, samples=None):
    """(d loss / d image, d loss / d sigma_r) for eq. BF."""
    return _grad(0, img, w, sigma_r, 1, gout, T, samples)


def gpa_grad(img, w, sigma_r, N, gout, T=128.0, samples=None):
    """(d loss / d image, d loss / d sigma_r) for eq. GPA (N held fixed)."""
    return _grad(1, img, w, sigma_r, N, gout, T, samples)


def set_threads(n: int) -> None:
    """Limit the checker's OpenMP threads (takes effect for new parallel regions)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        libgomp = ctypes.CDLL("libgomp.so.1")
        libgomp.omp_set_num_threads(int(n))
    except OSError:  # pragma: no cover
        pass


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
