"""The Python binding's argument checks and layout helpers, on the CPU: every
malformed tensor is refused with a Python error before the library is
called, so no GPU is needed (a stand-in model carries only the sizes)."""
import pytest
import torch

from paper_2605_31481_gb300 import api


class StandIn:
    nq, nv, n_bodies = 7, 6, 5
    device = torch.device("cpu")
    handle = None


def _ok(rows, B=8):
    return torch.zeros(rows, B, dtype=torch.float32)


@pytest.mark.parametrize("bad, err", [
    (lambda m: [0.0] * 7, TypeError),                                        # not a tensor
    (lambda m: _ok(m.nq).double(), ValueError),                               # wrong dtype
    (lambda m: _ok(m.nq + 1), ValueError),                                     # wrong row count
    (lambda m: torch.zeros(8, m.nq).t(), ValueError),                          # not contiguous
    (lambda m: torch.zeros(m.nq, 2, 4), ValueError),                           # not 2-D
])
def test_inputs_are_checked_before_any_call(bad, err):
    m = StandIn()
    with pytest.raises(err):
        api.fk(m, bad(m))
    with pytest.raises(err):
        api.rnea(m, bad(m), _ok(m.nv), _ok(m.nv))


def test_outputs_and_theta_are_checked():
    m = StandIn()
    q, v = _ok(m.nq), _ok(m.nv)
    with pytest.raises(ValueError):
        api.fk(m, q, out=torch.zeros(m.n_bodies, 12, 9))                      # B mismatch
    with pytest.raises(ValueError):
        api.crba(m, q, out=torch.zeros(m.nv, m.nv, 8, dtype=torch.float64))
    with pytest.raises(ValueError):
        api.rnea(m, q, v, v, theta=torch.zeros(m.n_bodies, 9))
    with pytest.raises(ValueError):
        api.aba(m, q, v, _ok(m.nv + 1))


def test_layout_helpers_round_trip():
    x = torch.arange(2 * 3 * 5, dtype=torch.float32).reshape(5, 2, 3)       # (B, ...)
    s = api.soa(x)
    assert s.shape == (2, 3, 5) and s.is_contiguous()
    assert torch.equal(api.aos(s), x)
    assert torch.equal(s[1, 2], x[:, 1, 2])                                   # environment index last
