"""Host-side behaviour of the Python binding that needs no GPU."""
import torch

from paper_1603_08109_gb300 import api


def test_sigma_value_follows_in_place_updates():
    """sigma_r's host copy is read once per tensor version: every in-place
    update through torch (an optimizer step, a copy) is seen, views and clones
    carry their own values."""
    s = torch.tensor(30.0, requires_grad=True)
    assert api._sigma_value(s) == 30.0
    assert api._sigma_value(s) == 30.0
    with torch.no_grad():
        s.add_(1.5)
    assert api._sigma_value(s) == 31.5
    opt = torch.optim.SGD([s], lr=1.0)
    s.grad = torch.tensor(2.0)
    opt.step()
    assert api._sigma_value(s) == 29.5
    c = s.detach().clone()
    with torch.no_grad():
        s.copy_(torch.tensor(7.0))
    assert api._sigma_value(s) == 7.0 and api._sigma_value(c) == 29.5
    assert api._sigma_value(12.0) == 12.0
