"""Host logic of the autograd wrapper, without a GPU: the native calls are replaced by fakes, so
only the bookkeeping of FdtdGrad and Problem runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _FakeNative:
    """Stands in for the C-ABI: F = sum(rho^2) of the last density, gradient 2 rho."""

    def __init__(self):
        self.rho = None
        self.calls = []

    def fdtd_set_density(self, h, rho):
        self.calls.append("set_density")
        self.rho = np.array(rho.cpu() if hasattr(rho, "cpu") else rho, dtype=np.float64)

    def fdtd_forward(self, h, ng):
        self.calls.append("forward")
        return float(np.sum(self.rho ** 2)), np.zeros(ng)

    def fdtd_adjoint(self, h):
        self.calls.append("adjoint")

    def fdtd_gradient(self, h, out):
        self.calls.append("gradient")
        out[...] = 2.0 * self.rho.reshape(out.shape)
        return out


def _fake_problem(monkeypatch, shape=(2, 3, 4)):
    import importlib
    P = importlib.import_module("paper_2305_00234_gb300.problem")
    fake = _FakeNative()
    for name in ("fdtd_set_density", "fdtd_forward", "fdtd_adjoint", "fdtd_gradient"):
        monkeypatch.setattr(P.N, name, getattr(fake, name))
    p = P.Problem.__new__(P.Problem)
    p.h = None
    p.version = 0
    p.nf, p.ngap, p.gshape, p.dshape = 1, 0, (0, 0, 0), shape
    return p, fake


def test_backward_runs_adjoint_and_gradient_of_its_own_forward(monkeypatch):
    from paper_2305_00234_gb300.grad import FdtdGrad
    p, fake = _fake_problem(monkeypatch)
    rho = torch.rand(2, 3, 4, dtype=torch.float64, requires_grad=True)
    F = FdtdGrad.apply(rho, p)
    (3.0 * F).backward()
    assert fake.calls == ["set_density", "forward", "adjoint", "gradient"]
    assert torch.allclose(rho.grad, 6.0 * rho.detach())


def test_second_forward_before_backward_raises(monkeypatch):
    from paper_2305_00234_gb300.grad import FdtdGrad
    p, fake = _fake_problem(monkeypatch)
    r1 = torch.rand(2, 3, 4, dtype=torch.float64, requires_grad=True)
    r2 = torch.rand(2, 3, 4, dtype=torch.float64, requires_grad=True)
    F1 = FdtdGrad.apply(r1, p)
    F2 = FdtdGrad.apply(r2, p)
    with pytest.raises(RuntimeError, match="another forward"):
        F1.backward()
    F2.backward()                                   # the latest forward is still valid
    assert torch.allclose(r2.grad, 2.0 * r2.detach())
    assert "adjoint" in fake.calls
