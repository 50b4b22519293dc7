"""Host logic of the torch.autograd front end on CPU, with the CUDA device
replaced by a stand-in: forward returns the traces as float64 tensors,
backward hands the incoming gradients to the gradient pass as the weights of
J and of the zone counts, returns its result for theta, zeroes the fill
entry when the placement does not depend on fill, and releases the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_09413_gb300 import autograd as AG  # noqa: E402
from paper_2511_09413_gb300 import workloads as W  # noqa: E402


class _FakeSim:
    made = []

    def __init__(self, dev, V, init_mode, fill=0.0, occ0=None):
        self.dev, self.init_mode, self.fill = dev, init_mode, fill
        self.steps, self.closed, self.weights = 0, False, None
        _FakeSim.made.append(self)

    def step_n(self, n):
        self.steps += n

    def traces(self):
        n, Z = self.steps, self.dev.Z
        J = np.arange(n, dtype=np.int64) - 2
        Zc = np.arange(n * Z, dtype=np.int64).reshape(n, Z)
        return J, Zc

    def grad(self, wJ, wZ):
        self.weights = (wJ, wZ)
        return np.array([1.0, 2.0, 3.0, 4.0]), np.array([0.1, 0.2, 0.3, 0.4])

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    _FakeSim.made.clear()
    monkeypatch.setattr(AG.K, "Sim", _FakeSim)
    return _FakeSim


def test_forward_traces_and_backward_weights(fake):
    dev = W.Device(R=3, L=20, Z=4)
    theta = torch.tensor([0.41, 1e12, 0.8, 0.25], dtype=torch.float64, requires_grad=True)
    J, Zc = AG.simulate(theta, dev, np.zeros(7), 7)
    sim = fake.made[-1]
    assert sim.steps == 7 and sim.init_mode == 1 and sim.fill == 0.25
    assert (sim.dev.Ea, sim.dev.nu, sim.dev.kappa) == (0.41, 1e12, 0.8)
    assert J.dtype == torch.float64 and Zc.shape == (7, 4)
    assert torch.equal(J, torch.arange(7, dtype=torch.float64) - 2)
    loss = 3.0 * J[-2:].sum() + Zc[:, 1].sum()
    loss.backward()
    wJ, wZ = sim.weights
    assert np.array_equal(wJ, [0, 0, 0, 0, 0, 3.0, 3.0])
    expect = np.zeros((7, 4))
    expect[:, 1] = 1.0
    assert np.array_equal(wZ, expect)
    assert torch.equal(theta.grad, torch.tensor([1.0, 2.0, 3.0, 4.0], dtype=torch.float64))
    assert sim.closed


def test_unused_trace_passes_no_weights(fake):
    dev = W.Device(R=3, L=20, Z=4)
    theta = torch.tensor([0.4, 1e12, 1.0, 0.2], dtype=torch.float64, requires_grad=True)
    J, _ = AG.simulate(theta, dev, np.zeros(5), 5)
    J.sum().backward()
    wJ, wZ = fake.made[-1].weights
    assert np.array_equal(wJ, np.ones(5)) and wZ is None


def test_fill_entry_is_zero_without_bernoulli_placement(fake):
    dev = W.Device(R=3, L=20, Z=4)
    theta = torch.tensor([0.4, 1e12, 1.0, 0.2], dtype=torch.float64, requires_grad=True)
    occ0 = np.zeros((3, 20), dtype=np.uint8)
    J, _ = AG.simulate(theta, dev, np.zeros(5), 5, init_mode=2, occ0=occ0)
    J.sum().backward()
    assert theta.grad.tolist() == [1.0, 2.0, 3.0, 0.0]


def test_theta_must_have_four_entries():
    with pytest.raises(ValueError):
        AG.simulate(torch.zeros(3, dtype=torch.float64), W.Device(R=1, L=4), np.zeros(2), 2)
