"""CPU checks of the C ABI: the library loads, exports every function that
include/bf.h declares, validates arguments without touching a GPU, and its
own host-side order selection reproduces the paper's tables."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bf.h")
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _lib():
    from paper_1603_08109_gb300 import _lib as L
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_08109_gb300 import build
        build.build()
    return L


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z0-9_]+)\s*\(", text)))


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([float(v) for v in line.split()])
    return out


def test_every_declared_symbol_is_exported_and_bound():
    L = _lib()
    handle = ctypes.CDLL(L.LIB_PATH)
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(handle, n), "missing export " + n
    assert set(names) <= set(L.SIGNATURES), "binding lacks " + str(set(names) - set(L.SIGNATURES))
    L.lib()


def test_version_and_status_strings():
    L = _lib()
    assert L.lib().bf_version() == 10400
    for code, text in L.STATUS.items():
        assert L.lib().bf_status_string(code).decode() == text


def test_library_order_selection_reproduces_table1():
    """The library's own bracketing + Newton root of nu (App. A) returns the
    N0' row of Table 1 for eps = 1e-3, T = 128 (independent of the checker)."""
    L = _lib()
    from paper_1603_08109_gb300 import api
    # eps = w(0) delta / (2T + delta): choose delta so that eps = 1e-3 for a box of radius 0
    for sr, n1, _, _ in _rows("order_vs_sigma_r.txt"):
        delta = 1e-3 * 256.0 / (1.0 - 1e-3)  # w(0) = 1 for radius 0
        assert api.order_from_delta(L.BOX, 0, 0.0, sr, delta, 128.0) == int(n1)


def test_library_order_vs_delta_table():
    L = _lib()
    from paper_1603_08109_gb300 import api
    for delta, n_lw, _ in _rows("order_vs_delta.txt"):
        assert api.order_from_delta(L.GAUSS, 15, 5.0, 30.0, delta, 127.0) == int(n_lw)
        assert abs(api.order_from_delta(L.GAUSS, 0, 5.0, 30.0, delta, 128.0) - int(n_lw)) <= 1


def test_library_volume_order_matches_checker():
    """bf_volume_order_from_delta (C++) against the checker: eq. eps with the
    volume kernel's w(0) = w1(0)^3 (w1 from the checker's planar kernel), then
    its Lambert-W order (eq. LambW)."""
    L = _lib()
    from oracle import order, volume
    from paper_1603_08109_gb300 import api
    for kind, r, ss in ((L.BOX, 3, 0.0), (L.GAUSS, 6, 2.0), (L.GAUSS, 15, 5.0), (L.BOX, 1, 0.0)):
        w0 = volume.centre_weight_volume(kind, r, ss)
        for sr in (12.0, 30.0, 70.0):
            for delta in (0.1, 1.0):
                eps = order.eps_from_delta(w0, delta, 128.0)
                ref = order.chernoff_order_lambertw((128.0 / sr) ** 2, eps)[0]
                assert api.volume_order_from_delta(kind, r, ss, sr, delta) == ref, (kind, r, sr)
    # the Gaussian radius defaults to ceil(3 sigma_s); invalid arguments
    assert api.volume_order_from_delta(L.GAUSS, 0, 2.0, 30.0, 1.0) == \
        api.volume_order_from_delta(L.GAUSS, 6, 2.0, 30.0, 1.0)
    n = ctypes.c_int()
    assert L.lib().bf_volume_order_from_delta(2, 0, 3.0, 30.0, 1.0, 128.0, ctypes.byref(n)) == 1
    assert L.lib().bf_volume_order_from_delta(0, 3, 0.0, 30.0, -1.0, 128.0, ctypes.byref(n)) == 1


def test_library_centre_weight():
    from paper_1603_08109_gb300 import api
    assert api.centre_weight(0, 4) == pytest.approx(1.0 / 81.0, rel=1e-15)
    assert api.centre_weight(1, 15, 5.0) == pytest.approx(6.3905e-3, rel=1e-4)


def test_argument_validation_without_gpu():
    """Invalid arguments are rejected before any CUDA call is made."""
    L = _lib()
    lib = L.lib()
    good = L.make_params(L.GAUSS, 9, 3.0, 30.0, 40)
    p = ctypes.byref(good)
    fake = ctypes.c_void_p(0x1000)
    out = ctypes.c_void_p(0x9000)  # a distinct output (an output equal to the input is rejected)
    assert lib.bf_fast_forward(None, fake, None, 8, 8, 8, p, None) == 1
    assert lib.bf_fast_forward(fake, fake, None, 8, 8, 8, p, None) == 1
    assert lib.bf_fast_forward(fake, out, None, 0, 8, 8, p, None) == 1
    assert lib.bf_fast_forward(fake, out, None, 8, 8, 4, p, None) == 1
    for bad in (L.make_params(L.GAUSS, 9, 3.0, 0.0, 40), L.make_params(L.GAUSS, 9, 3.0, 30.0, 0),
                L.make_params(7, 9, 3.0, 30.0, 40), L.make_params(L.GAUSS, 0, 0.0, 30.0, 4),
                L.make_params(L.BOX, -1, 0.0, 30.0, 4)):
        assert lib.bf_fast_forward(fake, out, None, 8, 8, 8, ctypes.byref(bad), None) == 1
    assert lib.bf_fast_forward(fake, out, None, 8, 8, 8,
                               ctypes.byref(L.make_params(L.BOX, 2, 0.0, 30.0, 5000)), None) == 3
    assert lib.bf_fast_forward(fake, out, None, 8, 8, 8,
                               ctypes.byref(L.make_params(L.BOX, 2, 0.0, 5.0, 5)), None) == 3
    n = ctypes.c_int()
    assert lib.bf_order_from_delta(0, 2, 0.0, 30.0, 0.0, 128.0, ctypes.byref(n)) == 1
    assert lib.bf_order_from_delta(0, 2, 0.0, 30.0, 1.0, 128.0, None) == 1
    sz = ctypes.c_size_t()
    assert lib.bf_fast_backward_workspace(64, 64, p, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.bf_direct_backward_workspace(64, 64, p, ctypes.byref(sz)) == 0 and sz.value > 0
    # backward asking for the sigma_r gradient without a workspace
    assert lib.bf_fast_backward(fake, fake, fake, fake, out, fake, 8, 8, 8, p, None, 0,
                                None) in (5, 3)
    assert lib.bf_batch_plan_create(None, 0, None) == 1
    # banded forward: no workspace for radius <= 15; for W = 60 a workspace of
    # at least 64 rows of N + 1 planes, checked before any launch
    assert lib.bf_fast_forward_workspace(64, 64, p, ctypes.byref(sz)) == 0 and sz.value == 0
    big = ctypes.byref(L.make_params(L.GAUSS, 60, 20.0, 40.0, 32))
    assert lib.bf_fast_forward_workspace(8192, 8192, big, ctypes.byref(sz)) == 0
    assert sz.value >= 64 * 33 * 8192 * 4 and sz.value % (33 * 8192 * 4) == 0
    assert lib.bf_fast_forward_ws(fake, out, None, 300, 200, 200, big, None, 0, None) == 5
    too_small = 63 * 33 * 200 * 4
    assert lib.bf_fast_forward_ws(fake, out, None, 300, 200, 200, big, fake, too_small, None) == 5
    assert lib.bf_fast_forward_ws(fake, out, None, 300, 200, 200, big,
                                  ctypes.c_void_p(0x1004), 64 * 33 * 200 * 4, None) == 1


def test_recursive_host_side():
    """The recursive Gaussian's centre weight and order agree with the checker
    (an independent derivation: closed-form geometric series on the library
    side, a direct sum over the integers in the checker); workspace size and
    argument checks need no GPU."""
    from oracle import order
    from oracle import recursive as rec
    from paper_1603_08109_gb300 import api
    L = _lib()
    lib = L.lib()
    for s in (0.5, 1.25, 3.0, 20.0, 64.0):
        assert api.centre_weight(L.GAUSS_RECURSIVE, 0, s) == pytest.approx(
            rec.centre_weight_recursive(float(np.float32(s))), rel=1e-12)
    for s, sr, delta in ((20.0, 40.0, 0.5), (3.0, 30.0, 1.0), (10.0, 15.0, 0.1)):
        w0 = rec.centre_weight_recursive(s)
        N, _ = order.chernoff_order_lambertw((128.0 / sr) ** 2, order.eps_from_delta(w0, delta))
        assert api.order_from_delta(L.GAUSS_RECURSIVE, 0, s, sr, delta) == N
    sz = ctypes.c_size_t()
    assert lib.bf_recursive_workspace(100, 70, 9, ctypes.byref(sz)) == 0
    planes = 10 * 128 * 96 * 4
    assert sz.value == planes + 2 * (planes // 4)
    assert lib.bf_recursive_workspace(100, 70, -1, ctypes.byref(sz)) == 1
    assert lib.bf_recursive_workspace(100, 70, 5000, ctypes.byref(sz)) == 3
    fake = ctypes.c_void_p(0x1000)
    good = L.make_params(L.GAUSS_RECURSIVE, 0, 3.0, 40.0, 9)
    args = (fake, ctypes.c_void_p(0x9000), None, 100, 70, 70)
    assert lib.bf_recursive_forward(*args, ctypes.byref(good), None, 0, None) == 5
    assert lib.bf_recursive_forward(*args, ctypes.byref(good), ctypes.c_void_p(0x1010),
                                    sz.value, None) == 1  # workspace not 256-byte aligned
    for bad in (L.make_params(L.GAUSS, 0, 3.0, 40.0, 9), L.make_params(L.GAUSS_RECURSIVE, 0, 0.4, 40.0, 9),
                L.make_params(L.GAUSS_RECURSIVE, 0, 3.0, 40.0, 0)):
        assert lib.bf_recursive_forward(*args, ctypes.byref(bad), fake, 1 << 30, None) == 1
    assert lib.bf_recursive_gauss(fake, ctypes.c_void_p(0x9000), 100, 70, 70, ctypes.c_float(0.3), fake, 1 << 30,
                                  None) == 1
    assert lib.bf_recursive_gauss(None, fake, 100, 70, 70, ctypes.c_float(3.0), fake, 1 << 30,
                                  None) == 1
    # backward and cross filter: workspace queries and checks made before any launch
    bsz, jsz = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.bf_recursive_backward_workspace(100, 70, 9, ctypes.byref(bsz)) == 0
    assert lib.bf_recursive_joint_workspace(100, 70, 9, ctypes.byref(jsz)) == 0
    assert bsz.value > sz.value and jsz.value > sz.value
    assert lib.bf_recursive_backward_workspace(100, 70, 0, ctypes.byref(bsz)) == 1
    assert lib.bf_recursive_joint_workspace(100, 70, 0, ctypes.byref(jsz)) == 1
    g = ctypes.c_void_p(0x2000)
    bargs = (fake, g, g, g, ctypes.c_void_p(0x3000), None, 100, 70, 70)
    assert lib.bf_recursive_backward(*bargs, ctypes.byref(good), fake, 0, None) == 5
    assert lib.bf_recursive_backward(fake, None, g, g, ctypes.c_void_p(0x3000), None, 100, 70, 70,
                                     ctypes.byref(good), fake, 1 << 30, None) == 1
    assert lib.bf_recursive_backward(fake, g, g, g, g, None, 100, 70, 70,  # d_gin aliases d_out
                                     ctypes.byref(good), fake, 1 << 30, None) == 1
    # the stored pair: the forward wants the backward's workspace size
    ws = ctypes.c_void_p(0x100000)
    assert lib.bf_recursive_forward_stored(*args, ctypes.byref(good), ws, sz.value, None) == 5
    assert lib.bf_recursive_forward_stored(*args, ctypes.byref(good), None, bsz.value, None) == 5
    assert lib.bf_recursive_forward_stored(fake, ctypes.c_void_p(0x9000), fake, 100, 70, 70,  # Q' = in
                                           ctypes.byref(good), ws, bsz.value, None) == 1
    assert lib.bf_recursive_forward_stored(*args, ctypes.byref(L.make_params(L.GAUSS, 9, 3.0, 40.0, 9)),
                                           ws, bsz.value, None) == 1
    assert lib.bf_recursive_backward_stored(*bargs, ctypes.byref(good), ws, sz.value, None) == 5
    assert lib.bf_recursive_backward_stored(fake, g, g, g, g, None, 100, 70, 70,
                                            ctypes.byref(good), ws, bsz.value, None) == 1
    jargs = (fake, g, ctypes.c_void_p(0x3000), None, 100, 70, 70)
    assert lib.bf_recursive_joint_forward(*jargs, ctypes.byref(good), fake, 0, None) == 5
    assert lib.bf_recursive_joint_forward(fake, None, ctypes.c_void_p(0x3000), None, 100, 70, 70,
                                          ctypes.byref(good), fake, 1 << 30, None) == 1
    assert lib.bf_recursive_joint_forward(*jargs, ctypes.byref(L.make_params(L.GAUSS, 9, 3.0, 40.0,
                                                                             9)),
                                          fake, 1 << 30, None) == 1


def test_forward_many_host_side():
    """bf_fast_forward_many rejects a batch count below 1 and an image stride
    smaller than one image before any launch."""
    L = _lib()
    lib = L.lib()
    p = L.make_params(L.BOX, 3, 0.0, 40.0, 1)
    a, b = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x900000)
    assert lib.bf_fast_forward_many(a, b, None, 0, 64 * 64, 64, 64, 64, ctypes.byref(p), None) == 1
    assert lib.bf_fast_forward_many(a, b, None, 3, 64 * 64 - 1, 64, 64, 64, ctypes.byref(p),
                                    None) == 1
    assert lib.bf_fast_forward_many(a, a, None, 3, 64 * 64, 64, 64, 64, ctypes.byref(p), None) == 1


def test_volume_host_side():
    """Workspace query and the argument checks made before any launch."""
    L = _lib()
    lib = L.lib()
    n = ctypes.c_size_t()
    p = L.make_params(L.BOX, 3, 0.0, 40.0, 7)
    assert lib.bf_volume_workspace(5, 6, 7, ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value == 256 + 8 * 5 * 6 * 8 * 4  # status word header; rows padded to 8 floats
    assert lib.bf_volume_workspace(0, 6, 7, ctypes.byref(p), ctypes.byref(n)) == 1
    big = L.make_params(L.BOX, 32, 0.0, 40.0, 7)
    assert lib.bf_volume_workspace(5, 6, 7, ctypes.byref(big), ctypes.byref(n)) == 3
    fake = ctypes.c_void_p(0x1000)
    out = ctypes.c_void_p(0x2000)
    assert lib.bf_volume_forward(fake, out, None, 5, 6, 7, ctypes.byref(p), None, 0, None) == 5
    assert lib.bf_volume_forward(fake, fake, None, 5, 6, 7, ctypes.byref(p), fake, 1 << 20,
                                 None) == 1
    assert lib.bf_volume_forward(fake, out, None, 5, 70000, 7, ctypes.byref(p), fake, 1 << 40,
                                 None) == 3


def test_tuning_table_roundtrip():
    from paper_1603_08109_gb300 import api
    nv = api.variant_count(1)
    assert nv >= 3
    rb, ob = api.radius_bucket(9), api.order_bucket(40)
    old = api.tuning_get(1, rb, ob)
    api.tuning_set(1, rb, ob, nv - 1)
    assert api.tuning_get(1, rb, ob) == nv - 1
    api.tuning_set(1, rb, ob, old)
    with pytest.raises(Exception):
        api.tuning_set(1, rb, ob, nv)


def test_library_order_estimates_match_checker():
    """bf_order_estimates (C++, own root finder and tail sum) vs the
    checker's Chebyshev formula, Lambert-W order and Poisson order."""
    from oracle import order
    from paper_1603_08109_gb300 import api
    for sr in (10.0, 17.0, 30.0, 55.0):
        lam = (128.0 / sr) ** 2
        for eps in (1e-1, 1e-3, 1e-7):
            ch, cn, po = api.order_estimates(sr, eps, 128.0)
            assert ch == order.chebyshev_order(lam, eps)
            assert cn == order.chernoff_order_lambertw(lam, eps)[0]
            assert po == order.poisson_order(lam, eps)
            assert po <= cn <= ch or eps > 0.05


def test_variant_routing_host_side():
    """The banded forward is variant 8: the calls without a workspace refuse it
    when asked for it explicitly, the workspace query follows the tuning table
    (a table entry of 8 makes a radius-9 forward take the banded path, so it
    asks for a workspace), and the new entry points check their arguments
    before any GPU work."""
    L = _lib()
    lib = L.lib()
    from paper_1603_08109_gb300 import api
    fake = ctypes.c_void_p(256)
    out = ctypes.c_void_p(512)
    p = ctypes.byref(L.make_params(L.GAUSS, 9, 3.0, 30.0, 40))
    assert api.variant_count() == 9 and api.BANDED_VARIANT == 8
    assert lib.bf_fast_forward_variant(fake, out, None, 64, 64, 64, p, 8, None) == 5
    assert lib.bf_fast_forward_ws_variant(fake, out, None, 64, 64, 64, p, 9, None, 0, None) == 1
    assert lib.bf_fast_forward_ws_variant(fake, out, None, 64, 64, 64, p, 8, None, 0, None) == 5
    best, ms = ctypes.c_int(), ctypes.c_float()
    assert lib.bf_autotune_ws(fake, out, 64, 64, 64, p, None, 0, 0, None, ctypes.byref(best),
                              ctypes.byref(ms)) == 1
    assert lib.bf_batch_variants(None, ctypes.byref(best), 1) == 1
    sz = ctypes.c_size_t()
    rb, ob = api.radius_bucket(9), api.order_bucket(40)
    old = api.tuning_get(L.GAUSS, rb, ob)
    try:
        api.tuning_set(L.GAUSS, rb, ob, -1)
        assert lib.bf_fast_forward_workspace(512, 512, p, ctypes.byref(sz)) == 0 and sz.value == 0
        api.tuning_set(L.GAUSS, rb, ob, 8)
        assert lib.bf_fast_forward_workspace(512, 512, p, ctypes.byref(sz)) == 0
        assert sz.value >= 64 * 41 * 512 * 4
        # without a workspace the table's banded entry is passed over (variant 5 runs)
        assert lib.bf_fast_forward_ws_variant(fake, out, None, 64, 64, 64, p, 8, fake,
                                              63 * 41 * 64 * 4, None) == 5
    finally:
        api.tuning_set(L.GAUSS, rb, ob, old)
