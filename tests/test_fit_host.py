"""Host logic of the material fit on CPU: the Adam iteration of
MaterialFit.run on a loss with a known minimum (the GPU loss and gradient
are replaced by a closed form), and the shape checks of the constructor."""
import numpy as np
import pytest

from paper_2511_09413_gb300 import fit as F
from paper_2511_09413_gb300 import workloads as W


class _Quadratic(F.MaterialFit):
    """loss = a (Ea - Ea*)^2 + b (kappa - kappa*)^2 with its exact gradient."""

    def __init__(self, target=(0.42, 0.9), scale=(400.0, 4.0), noise=0.0, seed=0):
        devs = [W.Device(R=4, L=16)]
        super().__init__(devs, np.zeros(10), [0.2], np.array([4, 9]), np.zeros((1, 2)))
        self.t, self.s, self.noise = np.array(target), np.array(scale), noise
        self.rng = np.random.default_rng(seed)
        self.calls = []

    def loss_and_grad(self, Ea, kappa):
        th = np.array([Ea, kappa])
        self.calls.append(th)
        g = 2.0 * self.s * (th - self.t)
        g = g + self.noise * self.rng.standard_normal(2) * np.abs(g).max()
        return F.FitStep(Ea, kappa, float((self.s * (th - self.t) ** 2).sum()), g,
                         np.zeros(2), 0.0, 0.0)


def test_adam_first_step_is_the_learning_rate_against_the_gradient():
    f = _Quadratic()
    hist = f.run(0.40, 1.0, iters=1, lr=(6e-3, 5e-2))
    assert len(hist) == 2                                  # one step + the final evaluation
    # with bias correction Adam's first step is lr * sign(-grad)
    assert np.allclose(f.calls[1], [0.40 + 6e-3, 1.0 - 5e-2])


def test_adam_converges_to_the_minimum():
    f = _Quadratic()
    hist = f.run(0.40, 1.0, iters=120, lr=(6e-3, 5e-2))
    assert len(hist) == 121
    assert abs(hist[-1].Ea - 0.42) < 2e-3 and abs(hist[-1].kappa - 0.9) < 2e-2
    assert hist[-1].loss < 1e-2 * hist[0].loss


def test_adam_tolerates_gradient_noise():
    f = _Quadratic(noise=0.3, seed=4)
    hist = f.run(0.40, 1.0, iters=150, lr=(3e-3, 2.5e-2))
    assert abs(hist[-1].Ea - 0.42) < 5e-3 and abs(hist[-1].kappa - 0.9) < 5e-2


def test_target_shape_is_checked():
    devs = [W.Device(R=4, L=16), W.Device(R=4, L=16)]
    with pytest.raises(ValueError):
        F.MaterialFit(devs, np.zeros(10), [0.2, 0.2], np.array([4, 9]), np.zeros((1, 2)))
    f = F.MaterialFit(devs, np.zeros(10), [0.2, 0.2], np.array([4, 9]), np.zeros((2, 2)))
    assert f.n_steps == 10
