"""The autograd wrapper's wiring, on CPU with a stand-in solver. The
parameters reach the solver; S comes back as a float64 scalar. Backward
gives upstream x dS/dtheta for each parameter that asks for a gradient,
on that parameter's device and in its dtype, and none for a plain
number."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1907_00908_gb300.autograd import signal  # noqa: E402


class FakeSolver:
    def __init__(self):
        self.seen = {}

    def set_phases(self, D, T2):
        self.seen["D"], self.seen["T2"] = np.asarray(D), np.asarray(T2)

    def set_permeability(self, kappa):
        self.seen["kappa"] = kappa

    def grad(self, checkpoint_every):
        self.seen["ck"] = checkpoint_every
        self.seen["called"] = "grad"
        return {"S": 0.75, "dD": np.array([0.5, -2.0]), "dT2": np.array([0.125, 4.0]), "dkappa": -3.0}

    def run(self):
        self.seen["called"] = "run"
        return {"S": 0.75}


def test_parameters_in_signal_out_and_gradients_back():
    s = FakeSolver()
    D = torch.tensor([2.0, 1.0], dtype=torch.float64, requires_grad=True)
    T2 = torch.tensor([80.0, 50.0], dtype=torch.float32, requires_grad=True)
    kap = torch.tensor(0.02, dtype=torch.float64, requires_grad=True)
    S = signal(s, D, T2, kap, checkpoint_every=16)
    assert S.dtype == torch.float64 and float(S.detach()) == 0.75
    assert np.allclose(s.seen["D"], [2.0, 1.0]) and np.allclose(s.seen["T2"], [80.0, 50.0])
    assert s.seen["kappa"] == pytest.approx(0.02) and s.seen["ck"] == 16
    (3.0 * S).backward()
    assert D.grad.dtype == torch.float64 and torch.equal(D.grad, torch.tensor([1.5, -6.0], dtype=torch.float64))
    assert T2.grad.dtype == torch.float32 and torch.equal(T2.grad, torch.tensor([0.375, 12.0]))
    assert float(kap.grad) == -9.0


def test_plain_number_and_frozen_parameters_get_no_gradient():
    s = FakeSolver()
    D = torch.tensor([2.0, 1.0], dtype=torch.float64, requires_grad=True)
    T2 = torch.tensor([80.0, 50.0], dtype=torch.float64)            # frozen
    S = signal(s, D, T2, 0.02)                                      # kappa a plain number
    S.backward()
    assert torch.equal(D.grad, torch.tensor([0.5, -2.0], dtype=torch.float64))
    assert T2.grad is None


def test_no_gradient_wanted_runs_the_forward_only():
    """Under no_grad, or with no input requiring a gradient, the signal comes
    from a plain forward run: the adjoint (about 4x the cost) is not run."""
    s = FakeSolver()
    D = torch.tensor([2.0, 1.0], dtype=torch.float64, requires_grad=True)
    with torch.no_grad():
        S = signal(s, D, [80.0, 50.0], 0.02)
    assert s.seen["called"] == "run" and float(S) == 0.75 and not S.requires_grad
    s = FakeSolver()
    S = signal(s, torch.tensor([2.0, 1.0]), torch.tensor([80.0, 50.0]), 0.02)
    assert s.seen["called"] == "run"
    s = FakeSolver()
    S = signal(s, D, [80.0, 50.0], 0.02)
    assert s.seen["called"] == "grad" and S.requires_grad
