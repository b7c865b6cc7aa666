"""GB300 (sm_103a) Gaussian-polynomial bilateral filter.

Chaudhury & Dabhade, "Fast and Provably Accurate Bilateral Filtering"
(arXiv 1603.08109): the bilateral filter with a Gaussian range kernel and a
box or Gaussian spatial kernel, approximated to order N by N + 1 spatial
filterings of power images (Algorithm 2), as hand-written CUDA kernels
behind the C ABI in include/bf.h.  This package is the thin Python layer:
``api`` (PyTorch tensors in, library calls out), ``_lib`` (ctypes
signatures), ``build`` (nvcc), ``synth`` (seeded synthetic inputs).
"""
from .api import (BANDED_VARIANT, BOX, GAUSS, GAUSS_RECURSIVE, BatchPlan, DirectBilateral, GPABilateral, autotune,  # noqa: F401
                  centre_weight, direct, direct_backward, direct_bilateral, gpa_backward,
                  exhaustive_order, forward_workspace_bytes, gpa_bilateral, gpa_forward,
                  gpa_forward_many, gpa_forward_stored, gpa_volume, joint_direct,
                  joint_forward, kernel_error_max, order_bucket, order_estimates, order_from_delta,
                  radius_bucket, RecursiveBilateral, recursive_backward,
                  recursive_backward_workspace_bytes, recursive_bilateral, recursive_joint_forward,
                  recursive_forward, recursive_gauss, recursive_workspace_bytes,
                  recursive_forward_stored, recursive_backward_stored, volume_order_from_delta,
                  volume_workspace_bytes,
                  resolve_radius, tuning_get, tuning_set, variant_count)

__version__ = "1.4.0"
