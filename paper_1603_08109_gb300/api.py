"""PyTorch-facing wrappers of the C ABI (include/bf.h).

PyTorch supplies device memory and the current CUDA stream; every filter
step runs inside libbf_gb300.so.  Inputs may be CUDA tensors (no copies) or
CPU tensors (copied to the GPU and back around the library call).
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional

import torch

from . import _lib
from ._lib import BOX, GAUSS, GAUSS_RECURSIVE, check, lib, make_params

__all__ = [
    "BOX", "GAUSS", "resolve_radius", "centre_weight", "order_from_delta", "gpa_forward",
    "gpa_forward_stored", "gpa_backward", "direct", "direct_backward", "GPABilateral",
    "DirectBilateral", "gpa_bilateral", "direct_bilateral", "BatchPlan", "autotune",
    "variant_count", "forward_workspace_bytes", "tuning_get", "tuning_set", "radius_bucket", "order_bucket",
    "joint_forward", "joint_direct", "order_estimates", "kernel_error_max", "exhaustive_order",
    "GAUSS_RECURSIVE", "recursive_workspace_bytes", "recursive_gauss", "recursive_forward",
    "recursive_backward", "recursive_backward_workspace_bytes", "RecursiveBilateral",
    "recursive_bilateral", "recursive_joint_forward", "recursive_forward_stored",
    "recursive_backward_stored", "gpa_forward_many", "gpa_volume", "volume_order_from_delta",
    "volume_workspace_bytes", "BANDED_VARIANT",
]

BANDED_VARIANT = 8  # the two-pass banded forward in the variant numbering of bf.h


def resolve_radius(kind: int, radius: int, sigma_s: float) -> int:
    """W = ceil(3 sigma_s) for the Gaussian when radius <= 0 (Sec. I)."""
    if kind == GAUSS and radius <= 0:
        return int(math.ceil(3.0 * float(sigma_s) - 1e-9))
    return int(radius)


def centre_weight(kind: int, radius: int, sigma_s: float = 0.0) -> float:
    out = ctypes.c_double()
    check(lib().bf_centre_weight(int(kind), int(radius), float(sigma_s), ctypes.byref(out)),
          "bf_centre_weight")
    return out.value


def order_from_delta(kind: int, radius: int, sigma_s: float, sigma_r: float, delta: float = 1.0,
                     T: float = 128.0) -> int:
    """Order N for filter accuracy delta (eq. eps + eq. LambW), host only."""
    n = ctypes.c_int()
    check(lib().bf_order_from_delta(int(kind), int(radius), float(sigma_s), float(sigma_r),
                                    float(delta), float(T), ctypes.byref(n)), "bf_order_from_delta")
    return n.value


def order_estimates(sigma_r: float, eps: float, T: float = 128.0):
    """(Chebyshev, Chernoff, exact Poisson) orders for kernel-error budget eps."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().bf_order_estimates(float(sigma_r), float(eps), float(T), ctypes.byref(a),
                                   ctypes.byref(b), ctypes.byref(c)), "bf_order_estimates")
    return a.value, b.value, c.value


def kernel_error_max(N: int, sigma_r: float, T: float = 128.0, grid: int = 1025,
                     device="cuda") -> float:
    """sup |g - phi_N| over a grid x grid lattice of [-T, T]^2 (eq. Linf), on the GPU."""
    out = torch.empty(1, dtype=torch.float64, device=device)
    check(lib().bf_kernel_error_max(int(N), float(sigma_r), float(T), int(grid), _ptr(out),
                                    _stream(out.device)), "bf_kernel_error_max")
    return float(out.item())


def exhaustive_order(sigma_r: float, eps: float, T: float = 128.0, grid: int = 1025) -> int:
    """Smallest N whose grid sup-norm kernel error is <= eps (the 'exhaustive
    search' order of Sec. II-B), found by bisection between 1 and the exact
    Poisson order (the error decreases with N)."""
    _, _, hi = order_estimates(sigma_r, eps, T)
    lo = 1
    if kernel_error_max(lo, sigma_r, T, grid) <= eps:
        return lo
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if kernel_error_max(mid, sigma_r, T, grid) <= eps:
            hi = mid
        else:
            lo = mid
    return hi


def _stream(dev: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[ctypes.c_void_p]:
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _as_device_image(img: torch.Tensor):
    """Return (device tensor with unit column stride, was_on_cpu)."""
    if not isinstance(img, torch.Tensor) or img.dim() != 2:
        raise ValueError("expected a 2-D tensor (height x width)")
    if img.dtype != torch.float32:
        raise ValueError("expected float32 input")
    on_cpu = img.device.type == "cpu"
    if on_cpu:
        src = img if img.is_pinned() or not torch.cuda.is_available() else img
        img = src.to("cuda", non_blocking=src.is_pinned())
    if img.device.type != "cuda":
        raise ValueError("expected a CUDA or CPU tensor")
    if img.stride(1) != 1 or img.stride(0) < img.shape[1] or img.storage_offset() % 1:
        img = img.contiguous()
    return img, on_cpu


def _image_like(img: torch.Tensor, out: Optional[torch.Tensor]) -> torch.Tensor:
    """Output with the input's row pitch (the ABI takes one pitch for both)."""
    if out is None:
        return torch.empty_strided(img.shape, img.stride(), dtype=img.dtype, device=img.device)
    if out.shape != img.shape or out.dtype != torch.float32 or out.device != img.device \
            or out.stride() != img.stride():
        raise ValueError("out must match the input's shape, dtype, device and strides")
    return out


def _like(x: torch.Tensor) -> torch.Tensor:
    return torch.empty_strided(x.shape, x.stride(), dtype=x.dtype, device=x.device)


def _params(kind, radius, sigma_s, sigma_r, N, t_c):
    return make_params(kind, radius, sigma_s, float(sigma_r), N, t_c)


def forward_workspace_bytes(H: int, W: int, kind: int, sigma_r: float, N: int, radius: int = 0,
                            sigma_s: float = 0.0, t_c: float = 128.0) -> int:
    """Workspace of the banded two-pass forward (0 when the radius is <= 15)."""
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    n = ctypes.c_size_t(0)
    check(lib().bf_fast_forward_workspace(H, W, ctypes.byref(p), ctypes.byref(n)),
          "bf_fast_forward_workspace")
    return int(n.value)


def gpa_forward(img: torch.Tensor, kind: int, sigma_r: float, N: int, radius: int = 0,
                sigma_s: float = 0.0, t_c: float = 128.0, return_q: bool = False,
                out: Optional[torch.Tensor] = None, variant: int = -1,
                band_rows: Optional[int] = None):
    """f_GPA of eq. GPA (Algorithm 2).  Returns out, or (out, Q').

    variant -1 picks the kernel from the tuning table or the built-in rule:
    the banded two-pass forward (by default for radii above 15) with a
    workspace from torch's allocator (band_rows, a multiple of 64, overrides
    its band height), else the fused single-pass kernels.  An explicit
    variant runs that kernel (BANDED_VARIANT: the banded forward)."""
    x, on_cpu = _as_device_image(img)
    o = _image_like(x, out if not on_cpu else None)
    q = _like(x) if return_q else None
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    H, W = x.shape
    nbytes = 0
    row_bytes = (int(N) + 1) * ((W + 3) // 4 * 4) * 4
    if variant < 0:
        n = ctypes.c_size_t(0)
        check(lib().bf_fast_forward_workspace(H, W, ctypes.byref(p), ctypes.byref(n)),
              "bf_fast_forward_workspace")
        nbytes = int(n.value)
    elif variant == BANDED_VARIANT:  # the whole image as one band, up to 1 GiB of planes
        rows = min((H + 63) // 64 * 64, max(64, (1 << 30) // row_bytes // 64 * 64))
        nbytes = rows * row_bytes
    if nbytes > 0:
        if band_rows is not None:
            nbytes = int(band_rows) * row_bytes
        ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=x.device)
        st = lib().bf_fast_forward_ws_variant(_ptr(x), _ptr(o), _ptr(q), H, W, x.stride(0),
                                              ctypes.byref(p), int(variant), _ptr(ws), nbytes,
                                              _stream(x.device))
    else:
        st = lib().bf_fast_forward_variant(_ptr(x), _ptr(o), _ptr(q), H, W, x.stride(0),
                                           ctypes.byref(p), int(variant), _stream(x.device))
    check(st, "bf_fast_forward")
    if on_cpu:
        o = o.cpu()
        q = q.cpu() if q is not None else None
    return (o, q) if return_q else o


def recursive_workspace_bytes(H: int, W: int, N: int = 0) -> int:
    """Workspace of the recursive-Gaussian path (N = 0: the plain filter)."""
    n = ctypes.c_size_t(0)
    check(lib().bf_recursive_workspace(int(H), int(W), int(N), ctypes.byref(n)),
          "bf_recursive_workspace")
    return int(n.value)


def _recursive_ws(H, W, N, dev, ws):
    nbytes = recursive_workspace_bytes(H, W, N)
    if ws is None or ws.numel() * ws.element_size() < nbytes or ws.device != dev:
        ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=dev)
    return ws, ws.numel() * ws.element_size()


def recursive_gauss(img: torch.Tensor, sigma_s: float, out: Optional[torch.Tensor] = None,
                    ws: Optional[torch.Tensor] = None) -> torch.Tensor:
    """w * img with w the recursive (Deriche) Gaussian over the whole image."""
    x, on_cpu = _as_device_image(img)
    o = _image_like(x, out if not on_cpu else None)
    H, W = x.shape
    ws, nbytes = _recursive_ws(H, W, 0, x.device, ws)
    check(lib().bf_recursive_gauss(_ptr(x), _ptr(o), H, W, x.stride(0), float(sigma_s), _ptr(ws),
                                   nbytes, _stream(x.device)), "bf_recursive_gauss")
    return o.cpu() if on_cpu else o


def recursive_forward(img: torch.Tensor, sigma_r: float, N: int, sigma_s: float,
                      t_c: float = 128.0, return_q: bool = False,
                      out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None):
    """f_GPA (Algorithm 2) with the recursive Gaussian as the spatial filter.
    Returns out, or (out, Q').  `ws` may hold a reusable workspace tensor."""
    x, on_cpu = _as_device_image(img)
    o = _image_like(x, out if not on_cpu else None)
    q = _like(x) if return_q else None
    H, W = x.shape
    ws, nbytes = _recursive_ws(H, W, N, x.device, ws)
    p = _params(GAUSS_RECURSIVE, 0, sigma_s, sigma_r, N, t_c)
    check(lib().bf_recursive_forward(_ptr(x), _ptr(o), _ptr(q), H, W, x.stride(0), ctypes.byref(p),
                                     _ptr(ws), nbytes, _stream(x.device)), "bf_recursive_forward")
    if on_cpu:
        o = o.cpu()
        q = q.cpu() if q is not None else None
    return (o, q) if return_q else o


def recursive_joint_forward(img: torch.Tensor, guide: torch.Tensor, sigma_r: float, N: int,
                            sigma_s: float, t_c: float = 128.0, return_q: bool = False,
                            out: Optional[torch.Tensor] = None,
                            ws: Optional[torch.Tensor] = None):
    """Cross (joint) filter with the recursive Gaussian: range kernel on the
    guide, average of img.  Returns out, or (out, Q')."""
    x, on_cpu = _as_device_image(img)
    gd, _ = _as_device_image(guide)
    if gd.shape != x.shape or gd.stride() != x.stride():
        x = x.contiguous()
        gd = gd.contiguous()
    o = _image_like(x, out if not on_cpu else None)
    q = _like(x) if return_q else None
    H, W = x.shape
    n = ctypes.c_size_t(0)
    check(lib().bf_recursive_joint_workspace(H, W, int(N), ctypes.byref(n)),
          "bf_recursive_joint_workspace")
    nbytes = int(n.value)
    if ws is None or ws.numel() * ws.element_size() < nbytes or ws.device != x.device:
        ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=x.device)
    p = _params(GAUSS_RECURSIVE, 0, sigma_s, sigma_r, N, t_c)
    check(lib().bf_recursive_joint_forward(_ptr(x), _ptr(gd), _ptr(o), _ptr(q), H, W, x.stride(0),
                                           ctypes.byref(p), _ptr(ws), ws.numel() * ws.element_size(),
                                           _stream(x.device)), "bf_recursive_joint_forward")
    if on_cpu:
        o = o.cpu()
        q = q.cpu() if q is not None else None
    return (o, q) if return_q else o


def recursive_backward_workspace_bytes(H: int, W: int, N: int) -> int:
    """Workspace of bf_recursive_backward (it also covers the forward's)."""
    n = ctypes.c_size_t(0)
    check(lib().bf_recursive_backward_workspace(int(H), int(W), int(N), ctypes.byref(n)),
          "bf_recursive_backward_workspace")
    return int(n.value)


def _backward_ws(H, W, N, dev, ws):
    nbytes = recursive_backward_workspace_bytes(H, W, N)
    if ws is None or ws.numel() * ws.element_size() < nbytes or ws.device != dev:
        ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=dev)
    return ws


def recursive_forward_stored(img: torch.Tensor, sigma_r: float, N: int, sigma_s: float,
                             t_c: float = 128.0, out: Optional[torch.Tensor] = None,
                             ws: Optional[torch.Tensor] = None):
    """recursive_forward that keeps the power images' row-pass planes for
    recursive_backward_stored: returns (out, Q', ws).  Pass the returned
    workspace, unmodified, with the same image and parameters to the
    backward."""
    x, on_cpu = _as_device_image(img)
    if on_cpu:
        raise ValueError("the stored forward keeps device state: pass a CUDA image")
    x = x.contiguous()
    o = _image_like(x, out)
    q = _like(x)
    H, W = x.shape
    ws = _backward_ws(H, W, N, x.device, ws)
    p = _params(GAUSS_RECURSIVE, 0, sigma_s, sigma_r, N, t_c)
    check(lib().bf_recursive_forward_stored(_ptr(x), _ptr(o), _ptr(q), H, W, x.stride(0),
                                            ctypes.byref(p), _ptr(ws),
                                            ws.numel() * ws.element_size(), _stream(x.device)),
          "bf_recursive_forward_stored")
    return o, q, ws


def recursive_backward_stored(img, out, q, gout, sigma_r: float, N: int, sigma_s: float,
                              ws: torch.Tensor, t_c: float = 128.0, need_sigma: bool = True):
    """(dL/d img, dL/d sigma_r or None) from the workspace that
    recursive_forward_stored returned (same image and parameters)."""
    return recursive_backward(img, out, q, gout, sigma_r, N, sigma_s, t_c, need_sigma, ws,
                              stored=True)


def recursive_backward(img, out, q, gout, sigma_r: float, N: int, sigma_s: float,
                       t_c: float = 128.0, need_sigma: bool = True,
                       ws: Optional[torch.Tensor] = None, stored: bool = False):
    """(dL/d img, dL/d sigma_r or None) of recursive_forward, given gout."""
    x, _ = _as_device_image(img)
    if stored and (x.stride(-1) != 1 or x.stride(0) != x.shape[1]):
        raise ValueError("the stored backward takes the contiguous image of the stored forward")
    tensors = []
    for t in (out, q, gout):
        if t.shape != x.shape or t.device != x.device or t.dtype != torch.float32:
            raise ValueError("out, q, gout must match the image")
        tensors.append(t)
    if any(t.stride() != x.stride() for t in tensors):
        x = x.contiguous()
        tensors = [t.contiguous() for t in tensors]
    o, qq, g = tensors
    H, W = x.shape
    gin = _like(x)
    gs = torch.zeros(1, dtype=torch.float64, device=x.device) if need_sigma else None
    nbytes = recursive_backward_workspace_bytes(H, W, N)
    if stored:
        if ws is None or ws.device != x.device or ws.numel() * ws.element_size() < nbytes:
            raise ValueError("the stored backward needs the stored forward's workspace")
    else:
        ws = _backward_ws(H, W, N, x.device, ws)
    p = _params(GAUSS_RECURSIVE, 0, sigma_s, sigma_r, N, t_c)
    fn = lib().bf_recursive_backward_stored if stored else lib().bf_recursive_backward
    check(fn(_ptr(x), _ptr(o), _ptr(qq), _ptr(g), _ptr(gin), _ptr(gs), H, W, x.stride(0),
             ctypes.byref(p), _ptr(ws), ws.numel() * ws.element_size(), _stream(x.device)),
          "bf_recursive_backward_stored" if stored else "bf_recursive_backward")
    return gin, gs


def gpa_forward_many(imgs: torch.Tensor, kind: int, sigma_r: float, N: int, radius: int = 0,
                     sigma_s: float = 0.0, t_c: float = 128.0, return_q: bool = False,
                     out: Optional[torch.Tensor] = None):
    """f_GPA of each image of a (B, H, W) CUDA tensor (same parameters, e.g.
    video frames) through bf_fast_forward_many: one launch for the whole batch
    on the warp-strip box kernel, one per image otherwise.  Returns out, or
    (out, Q')."""
    if imgs.dim() != 3 or imgs.device.type != "cuda":
        raise ValueError("imgs must be a (B, H, W) CUDA tensor")
    x = imgs.to(torch.float32)
    if x.stride(2) != 1 or x.stride(0) < x.shape[1] * x.stride(1):
        x = x.contiguous()
    B, H, W = x.shape
    out = _image_like(x, out)
    q = _like(x) if return_q else None
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    check(lib().bf_fast_forward_many(_ptr(x), _ptr(out), _ptr(q), B, ctypes.c_size_t(x.stride(0)), H, W,
                                     x.stride(1), ctypes.byref(p), _stream(x.device)),
          "bf_fast_forward_many")
    return (out, q) if return_q else out


def volume_order_from_delta(kind: int, radius: int, sigma_s: float, sigma_r: float, delta: float,
                            t_c: float = 128.0) -> int:
    """N for a volume filter accuracy delta (bf_volume_order_from_delta: eq.
    eps with the volume kernel's w(0) = w1(0)^3, then eq. LambW)."""
    n = ctypes.c_int()
    check(lib().bf_volume_order_from_delta(int(kind), int(radius), float(sigma_s), float(sigma_r),
                                           float(delta), float(t_c), ctypes.byref(n)),
          "bf_volume_order_from_delta")
    return n.value


def volume_workspace_bytes(D: int, H: int, W: int, kind: int, sigma_r: float, N: int,
                           radius: int = 0, sigma_s: float = 0.0, t_c: float = 128.0) -> int:
    n = ctypes.c_size_t(0)
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    check(lib().bf_volume_workspace(int(D), int(H), int(W), ctypes.byref(p), ctypes.byref(n)),
          "bf_volume_workspace")
    return int(n.value)


def gpa_volume(vol: torch.Tensor, kind: int, sigma_r: float, N: int, radius: int = 0,
               sigma_s: float = 0.0, t_c: float = 128.0, return_q: bool = False,
               out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None):
    """f_GPA of a (D, H, W) grayscale volume or video (Algorithm 2 with the
    separable 3-D kernel; bf_volume_forward).  Returns out, or (out, Q')."""
    if vol.dim() != 3 or vol.device.type != "cuda":
        raise ValueError("vol must be a (D, H, W) CUDA tensor")
    x = vol.to(torch.float32).contiguous()
    D, H, W = x.shape
    o = _image_like(x, out)
    q = _like(x) if return_q else None
    nbytes = volume_workspace_bytes(D, H, W, kind, sigma_r, N, radius, sigma_s, t_c)
    if ws is None or ws.numel() * ws.element_size() < nbytes or ws.device != x.device:
        ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=x.device)
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    check(lib().bf_volume_forward(_ptr(x), _ptr(o), _ptr(q), D, H, W, ctypes.byref(p), _ptr(ws),
                                  ws.numel() * ws.element_size(), _stream(x.device)),
          "bf_volume_forward")
    return (o, q) if return_q else o


def gpa_forward_stored(img: torch.Tensor, kind: int, sigma_r: float, N: int, radius: int = 0,
                       sigma_s: float = 0.0, t_c: float = 128.0):
    """Forward that also keeps the N+1 filtered power images: (out, Q', Abar)."""
    x, _ = _as_device_image(img)
    o = _like(x)
    q = _like(x)
    H, W = x.shape
    abar = torch.empty((N + 1, H, x.stride(0)), dtype=torch.float32, device=x.device)
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    st = lib().bf_fast_forward_stored(_ptr(x), _ptr(o), _ptr(q), _ptr(abar),
                                      ctypes.c_size_t(H * x.stride(0)), H, W, x.stride(0),
                                      ctypes.byref(p), _stream(x.device))
    check(st, "bf_fast_forward_stored")
    return o, q, abar[:, :, :W]


def _workspace(fn_name, H, W, p, dev):
    n = ctypes.c_size_t()
    check(getattr(lib(), fn_name)(H, W, ctypes.byref(p), ctypes.byref(n)), fn_name)
    return torch.empty(max(int(n.value), 1), dtype=torch.uint8, device=dev), int(n.value)


def gpa_backward(img, out, q, gout, kind: int, sigma_r: float, N: int, radius: int = 0,
                 sigma_s: float = 0.0, t_c: float = 128.0, need_sigma: bool = True,
                 abar: Optional[torch.Tensor] = None):
    """(dL/d img, dL/d sigma_r or None) of the fast filter, given gout."""
    x, _ = _as_device_image(img)
    H, W = x.shape
    tensors = []
    for t in (out, q, gout):
        if t.shape != x.shape or t.device != x.device or t.dtype != torch.float32:
            raise ValueError("out, q, gout must match the image")
        tensors.append(t)
    if abar is None and any(t.stride() != x.stride() for t in tensors):
        x = x.contiguous()
        tensors = [t.contiguous() for t in tensors]
    elif abar is not None and any(t.stride() != x.stride() for t in tensors):
        raise ValueError("with stored planes, out, q and gout must share the image's layout")
    pitch = x.stride(0)
    o, qq, g = tensors
    gin = _like(x)
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    gs = torch.zeros(1, dtype=torch.float64, device=x.device) if need_sigma else None
    ws, nbytes = _workspace("bf_fast_backward_workspace", H, W, p, x.device)
    if abar is None:
        st = lib().bf_fast_backward(_ptr(x), _ptr(o), _ptr(qq), _ptr(g), _ptr(gin), _ptr(gs),
                                    H, W, pitch, ctypes.byref(p), _ptr(ws), ctypes.c_size_t(nbytes),
                                    _stream(x.device))
        check(st, "bf_fast_backward")
    else:
        if abar.dim() != 3 or abar.shape[0] != N + 1 or abar.stride(2) != 1 \
                or abar.stride(1) != pitch:
            raise ValueError("abar must come from gpa_forward_stored on this image")
        st = lib().bf_fast_backward_stored(_ptr(x), _ptr(o), _ptr(qq), _ptr(abar),
                                           ctypes.c_size_t(abar.stride(0)), _ptr(g), _ptr(gin),
                                           _ptr(gs), H, W, pitch, ctypes.byref(p), _ptr(ws),
                                           ctypes.c_size_t(nbytes), _stream(x.device))
        check(st, "bf_fast_backward_stored")
    return gin, gs


def direct(img: torch.Tensor, kind: int, sigma_r: float, radius: int = 0, sigma_s: float = 0.0,
           t_c: float = 128.0, out: Optional[torch.Tensor] = None):
    """eq. BF computed directly (the O(W^2) comparison filter)."""
    x, on_cpu = _as_device_image(img)
    o = _image_like(x, out if not on_cpu else None)
    p = _params(kind, radius, sigma_s, sigma_r, 1, t_c)
    H, W = x.shape
    check(lib().bf_direct(_ptr(x), _ptr(o), H, W, x.stride(0), ctypes.byref(p), _stream(x.device)),
          "bf_direct")
    return o.cpu() if on_cpu else o


def _guide_like(x: torch.Tensor, guide: torch.Tensor) -> torch.Tensor:
    g, _ = _as_device_image(guide)
    if g.shape != x.shape or g.device != x.device:
        raise ValueError("guide must have the image's shape and device")
    if g.stride() != x.stride():
        g = torch.empty_strided(x.shape, x.stride(), dtype=x.dtype, device=x.device).copy_(g)
    return g


def joint_forward(img: torch.Tensor, guide: torch.Tensor, kind: int, sigma_r: float, N: int,
                  radius: int = 0, sigma_s: float = 0.0, t_c: float = 128.0,
                  return_q: bool = False, out: Optional[torch.Tensor] = None,
                  band_rows: Optional[int] = None):
    """Cross (joint) bilateral filter, Gaussian-polynomial form (range kernel on guide).

    For radii above 15 the banded two-pass form with a workspace from torch's
    allocator (band_rows, a multiple of 64, overrides its band height)."""
    x, on_cpu = _as_device_image(img)
    g = _guide_like(x, guide)
    o = _image_like(x, out if not on_cpu else None)
    q = _like(x) if return_q else None
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    H, W = x.shape
    n = ctypes.c_size_t(0)
    check(lib().bf_joint_forward_workspace(H, W, ctypes.byref(p), ctypes.byref(n)),
          "bf_joint_forward_workspace")
    nbytes = int(n.value)
    if nbytes > 0:
        if band_rows is not None:
            nbytes = int(band_rows) * 2 * int(N) * ((W + 3) // 4 * 4) * 4
        ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=x.device)
        check(lib().bf_joint_forward_ws(_ptr(x), _ptr(g), _ptr(o), _ptr(q), H, W, x.stride(0),
                                        ctypes.byref(p), _ptr(ws), nbytes, _stream(x.device)),
              "bf_joint_forward")
    else:
        check(lib().bf_joint_forward(_ptr(x), _ptr(g), _ptr(o), _ptr(q), H, W, x.stride(0),
                                     ctypes.byref(p), _stream(x.device)), "bf_joint_forward")
    if on_cpu:
        o = o.cpu()
        q = q.cpu() if q is not None else None
    return (o, q) if return_q else o


def joint_direct(img: torch.Tensor, guide: torch.Tensor, kind: int, sigma_r: float,
                 radius: int = 0, sigma_s: float = 0.0, t_c: float = 128.0,
                 out: Optional[torch.Tensor] = None):
    """Cross (joint) bilateral filter with the exact range kernel (comparison)."""
    x, on_cpu = _as_device_image(img)
    g = _guide_like(x, guide)
    o = _image_like(x, out if not on_cpu else None)
    p = _params(kind, radius, sigma_s, sigma_r, 1, t_c)
    H, W = x.shape
    check(lib().bf_joint_direct(_ptr(x), _ptr(g), _ptr(o), H, W, x.stride(0), ctypes.byref(p),
                                _stream(x.device)), "bf_joint_direct")
    return o.cpu() if on_cpu else o


def direct_backward(img, gout, kind: int, sigma_r: float, radius: int = 0, sigma_s: float = 0.0,
                    t_c: float = 128.0, need_sigma: bool = True):
    x, _ = _as_device_image(img)
    H, W = x.shape
    g = gout
    if g.stride() != x.stride():
        x, g = x.contiguous(), g.contiguous()
    gin = _like(x)
    p = _params(kind, radius, sigma_s, sigma_r, 1, t_c)
    gs = torch.zeros(1, dtype=torch.float64, device=x.device) if need_sigma else None
    ws, nbytes = _workspace("bf_direct_backward_workspace", H, W, p, x.device)
    st = lib().bf_direct_backward(_ptr(x), _ptr(g), _ptr(gin), _ptr(gs), H, W, x.stride(0),
                                  ctypes.byref(p), _ptr(ws), ctypes.c_size_t(nbytes),
                                  _stream(x.device))
    check(st, "bf_direct_backward")
    return gin, gs


# ------------------------------------------------------------------ autograd
def _sigma_value(sigma_r) -> float:
    """sigma_r as the host float the library takes.  A tensor's value is read
    (a device-to-host copy that waits for the stream) once per version: its
    version counter changes with every in-place update through torch (an
    optimizer step), so calls with an unchanged sigma_r tensor do not stall
    the host on the device.  A tensor written behind torch's back (e.g. by a
    raw kernel) needs a new tensor or a torch in-place op to be re-read."""
    if not isinstance(sigma_r, torch.Tensor):
        return float(sigma_r)
    key = (sigma_r._version, sigma_r.data_ptr(), sigma_r.device)
    cached = getattr(sigma_r, "_bf_sigma_host", None)
    if cached is not None and cached[0] == key:
        return cached[1]
    v = float(sigma_r.detach().item())
    try:
        sigma_r._bf_sigma_host = (key, v)
    except (AttributeError, RuntimeError):  # pragma: no cover - tensor subclasses without a dict
        pass
    return v


class GPABilateral(torch.autograd.Function):
    """Autograd wrapper: forward = bf_fast_forward, backward = bf_fast_backward
    (power images recomputed) or bf_fast_backward_stored (store=True)."""

    @staticmethod
    def forward(ctx, img, sigma_r, kind, N, radius, sigma_s, t_c, store):
        sr = _sigma_value(sigma_r)
        if store:
            out, q, abar = gpa_forward_stored(img, kind, sr, N, radius, sigma_s, t_c)
        else:
            out, q = gpa_forward(img, kind, sr, N, radius, sigma_s, t_c, return_q=True)
            abar = None
        ctx.cfg = (kind, sr, N, radius, sigma_s, t_c)
        ctx.abar = abar
        ctx.sigma_is_tensor = isinstance(sigma_r, torch.Tensor)
        ctx.save_for_backward(img, out, q)
        return out

    @staticmethod
    def backward(ctx, gout):
        img, out, q = ctx.saved_tensors
        kind, sr, N, radius, sigma_s, t_c = ctx.cfg
        need_s = ctx.sigma_is_tensor and ctx.needs_input_grad[1]
        gin, gs = gpa_backward(img, out, q, gout.contiguous(), kind, sr, N, radius, sigma_s, t_c,
                               need_sigma=need_s, abar=ctx.abar)
        gsig = gs.reshape(()).to(torch.float32) if need_s else None
        return gin, gsig, None, None, None, None, None, None


class DirectBilateral(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, sigma_r, kind, radius, sigma_s, t_c):
        sr = _sigma_value(sigma_r)
        out = direct(img, kind, sr, radius, sigma_s, t_c)
        ctx.cfg = (kind, sr, radius, sigma_s, t_c)
        ctx.sigma_is_tensor = isinstance(sigma_r, torch.Tensor)
        ctx.save_for_backward(img)
        return out

    @staticmethod
    def backward(ctx, gout):
        (img,) = ctx.saved_tensors
        kind, sr, radius, sigma_s, t_c = ctx.cfg
        need_s = ctx.sigma_is_tensor and ctx.needs_input_grad[1]
        gin, gs = direct_backward(img, gout.contiguous(), kind, sr, radius, sigma_s, t_c, need_s)
        gsig = gs.reshape(()).to(torch.float32) if need_s else None
        return gin, gsig, None, None, None, None


class RecursiveBilateral(torch.autograd.Function):
    """Autograd wrapper of the recursive-Gaussian route: forward =
    bf_recursive_forward, backward = bf_recursive_backward; with store, the
    stored pair (the workspace with the power images' row-pass planes is held
    from forward to backward)."""

    @staticmethod
    def forward(ctx, img, sigma_r, N, sigma_s, t_c, store):
        sr = _sigma_value(sigma_r)
        if store:
            x = img.contiguous()
            out, q, ctx.ws = recursive_forward_stored(x, sr, N, sigma_s, t_c)
        else:
            x = img
            out, q = recursive_forward(x, sr, N, sigma_s, t_c, return_q=True)
            ctx.ws = None
        ctx.cfg = (sr, N, sigma_s, t_c)
        ctx.sigma_is_tensor = isinstance(sigma_r, torch.Tensor)
        ctx.save_for_backward(x, out, q)
        return out

    @staticmethod
    def backward(ctx, gout):
        img, out, q = ctx.saved_tensors
        sr, N, sigma_s, t_c = ctx.cfg
        need_s = ctx.sigma_is_tensor and ctx.needs_input_grad[1]
        gin, gs = recursive_backward(img, out, q, gout.contiguous(), sr, N, sigma_s, t_c,
                                     need_sigma=need_s, ws=ctx.ws, stored=ctx.ws is not None)
        gsig = gs.reshape(()).to(torch.float32) if need_s else None
        return gin, gsig, None, None, None, None


def recursive_bilateral(img, sigma_r, sigma_s, N=None, t_c=128.0, delta=1.0, store=True):
    """Differentiable fast bilateral filter with the recursive Gaussian;
    N from delta (w(0) = h(0)^2) when not given.  store (default): keep the
    power images' row-pass planes from forward to backward, which holds the
    backward workspace, 2.75 (N + 1) planes, between them; the backward then
    skips those row passes (same gradients, about 25% less fwd+bwd time).
    store=False recomputes them and holds only out and Q'."""
    if N is None:
        N = order_from_delta(GAUSS_RECURSIVE, 0, sigma_s, _sigma_value(sigma_r), delta, t_c)
    return RecursiveBilateral.apply(img, sigma_r, int(N), float(sigma_s), float(t_c), bool(store))


def gpa_bilateral(img, sigma_r, kind=GAUSS, N=None, radius=0, sigma_s=0.0, t_c=128.0,
                  delta=1.0, store=False):
    """Differentiable fast bilateral filter; N from delta when not given."""
    r = resolve_radius(kind, radius, sigma_s)
    if N is None:
        N = order_from_delta(kind, r, sigma_s, _sigma_value(sigma_r), delta, t_c)
    return GPABilateral.apply(img, sigma_r, kind, int(N), r, float(sigma_s), float(t_c),
                              bool(store))


def direct_bilateral(img, sigma_r, kind=GAUSS, radius=0, sigma_s=0.0, t_c=128.0):
    r = resolve_radius(kind, radius, sigma_s)
    return DirectBilateral.apply(img, sigma_r, kind, r, float(sigma_s), float(t_c))


# ------------------------------------------------------------------ batched
class BatchPlan:
    """Persistent batched forward over images of uneven sizes and parameters.

    specs: list of dicts with kind, radius, sigma_s, sigma_r, N (t_c optional).
    Each image runs the variant the tuning table names for it when the plan is
    created (variants()).  The plan owns its workspace; run() enqueues the
    counters' memset, the persistent launches, the per-image launches and the
    banded groups (the last two on side streams forked from the current one);
    graph() captures that into a CUDA graph, replay() launches it."""

    def __init__(self, images, outs, specs, qaux=None):
        if not (len(images) == len(outs) == len(specs)) or not images:
            raise ValueError("images, outs and specs must be non-empty lists of equal length")
        self.device = images[0].device
        self.images, self.outs, self.qaux = images, outs, qaux
        descs = (_lib.BfImageDesc * len(images))()
        for k, (x, o, sp) in enumerate(zip(images, outs, specs)):
            if x.device != self.device or x.dtype != torch.float32 or x.stride(1) != 1:
                raise ValueError("image %d must be a float32 CUDA tensor with unit column stride" % k)
            if o.shape != x.shape or o.stride() != x.stride():
                raise ValueError("output %d must match its image" % k)
            q = qaux[k] if qaux is not None else None
            p = _params(sp["kind"], sp.get("radius", 0), sp.get("sigma_s", 0.0), sp["sigma_r"],
                        sp["N"], sp.get("t_c", 128.0))
            descs[k] = _lib.BfImageDesc(x.data_ptr(), o.data_ptr(), q.data_ptr() if q is not None
                                        else None, x.shape[0], x.shape[1], x.stride(0), p)
        self._descs = descs
        plan = ctypes.c_void_p()
        check(lib().bf_batch_plan_create(descs, len(images), ctypes.byref(plan)),
              "bf_batch_plan_create")
        self._plan = plan
        n = ctypes.c_size_t()
        check(lib().bf_batch_workspace(plan, ctypes.byref(n)), "bf_batch_workspace")
        self.ws_bytes = int(n.value)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        check(lib().bf_batch_upload(plan, _ptr(self.ws), ctypes.c_size_t(self.ws_bytes),
                                    _stream(self.device)), "bf_batch_upload")
        torch.cuda.current_stream(self.device).synchronize()  # plan tables are now on the device
        self._graph = None

    def info(self):
        items, ctas = ctypes.c_int(), ctypes.c_int()
        check(lib().bf_batch_info(self._plan, ctypes.byref(items), ctypes.byref(ctas)),
              "bf_batch_info")
        return items.value, ctas.value

    def variants(self):
        """The forward variant each image runs (read from the tuning table when
        the plan was created)."""
        n = len(self.images)
        v = (ctypes.c_int * n)()
        check(lib().bf_batch_variants(self._plan, v, n), "bf_batch_variants")
        return list(v)

    def run(self):
        check(lib().bf_batch_forward(self._plan, _ptr(self.ws), ctypes.c_size_t(self.ws_bytes),
                                     _ptr(self.status), _stream(self.device)), "bf_batch_forward")

    def graph(self):
        if self._graph is None:
            g = ctypes.c_void_p()
            s = torch.cuda.Stream(self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            check(lib().bf_batch_graph_create(self._plan, _ptr(self.ws),
                                              ctypes.c_size_t(self.ws_bytes), _ptr(self.status),
                                              ctypes.c_void_p(s.cuda_stream), ctypes.byref(g)),
                  "bf_batch_graph_create")
            s.synchronize()
            self._graph = g
        return self._graph

    def replay(self):
        check(lib().bf_graph_launch(self.graph(), _stream(self.device)), "bf_graph_launch")

    def close(self):
        if getattr(self, "_graph", None):
            lib().bf_graph_destroy(self._graph)
            self._graph = None
        if getattr(self, "_plan", None):
            lib().bf_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ tuning
def variant_count(kind: int = GAUSS) -> int:
    return int(lib().bf_variant_count(int(kind)))


def radius_bucket(radius: int) -> int:
    return int(lib().bf_tuning_radius_bucket(int(radius)))


def order_bucket(N: int) -> int:
    return int(lib().bf_tuning_order_bucket(int(N)))


def tuning_get(kind: int, rb: int, ob: int) -> int:
    v = ctypes.c_int()
    check(lib().bf_tuning_get(int(kind), int(rb), int(ob), ctypes.byref(v)), "bf_tuning_get")
    return v.value


def tuning_set(kind: int, rb: int, ob: int, variant: int) -> None:
    check(lib().bf_tuning_set(int(kind), int(rb), int(ob), int(variant)), "bf_tuning_set")


def autotune(img: torch.Tensor, kind: int, sigma_r: float, N: int, radius: int = 0,
             sigma_s: float = 0.0, t_c: float = 128.0, reps: int = 5, banded: bool = True):
    """Time every variant on this image (with banded=True also the two-pass
    banded forward, in a workspace of 64 band rows from torch's allocator);
    record the fastest in the tuning table and return (variant, ms)."""
    x, _ = _as_device_image(img)
    o = _like(x)
    p = _params(kind, radius, sigma_s, sigma_r, N, t_c)
    best, ms = ctypes.c_int(), ctypes.c_float()
    H, W = x.shape
    row_bytes = (int(N) + 1) * ((W + 3) // 4 * 4) * 4
    rows = min((H + 63) // 64 * 64, max(64, (1 << 30) // row_bytes // 64 * 64))
    nbytes = rows * row_bytes if banded else 0
    ws = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=x.device) if banded else None
    check(lib().bf_autotune_ws(_ptr(x), _ptr(o), H, W, x.stride(0), ctypes.byref(p), _ptr(ws),
                               nbytes, int(reps), _stream(x.device), ctypes.byref(best),
                               ctypes.byref(ms)), "bf_autotune_ws")
    return best.value, ms.value
