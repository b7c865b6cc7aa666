"""GPU kernel-error toolkit (Sec. II): the dense-grid sup-norm of eq. Linf
against the checker's FP64 grid evaluation, the Poisson bound of
Prop. upperBound, and the ordering of the order estimates (Fig. tightness)."""
import numpy as np
import pytest

import paper_1603_08109_gb300 as bf
from helpers import needs_gpu
from oracle import order

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("sr,N", [(30.0, 40), (30.0, 10), (15.0, 107), (50.0, 19), (80.0, 3)])
def test_grid_sup_norm_matches_checker_and_bound(sr, N):
    G = 257
    t = np.linspace(-128.0, 128.0, G)
    tt, uu = np.meshgrid(t, t)
    ref = np.abs(order.kernel_error(N, sr, tt, uu)).max()
    got = bf.kernel_error_max(N, sr, 128.0, G)
    assert got == pytest.approx(ref, rel=1e-9, abs=1e-15)
    assert got <= order.poisson_tail(N, (128.0 / sr) ** 2) * (1 + 1e-9) + 1e-15


def test_tightness_ordering_of_order_estimates():
    """For eps = 1e-3 (Fig. tightness, right): exhaustive <= Poisson <=
    Chernoff <= Chebyshev, and the Chernoff order reproduces Table 1."""
    table = {10.0: 214, 20.0: 67, 30.0: 37, 50.0: 19}
    for sr, n_table in table.items():
        ex = bf.exhaustive_order(sr, 1e-3, 128.0, grid=513)
        ch, cn, po = bf.order_estimates(sr, 1e-3, 128.0)
        assert ex <= po <= cn <= ch
        assert cn == n_table
        assert bf.kernel_error_max(ex, sr, 128.0, 513) <= 1e-3
