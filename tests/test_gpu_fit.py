"""GPU tests of the batched gradient (kmc_batch_grad) and of the material
fit driven by it: a device's gradient in a batch equals its gradient alone,
and gradient descent from (0.40 eV, 1.0) moves toward the hidden parameters
of target curves that the oracle produced."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2511_09413_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09413_gb300 import build, kmc as K
    build.build()
    K.load()
    torch.cuda.init()
    return K


def test_batch_gradient_equals_single_device_gradient(kmc):
    devs, V, fills, samples = W.fit_batch(5, seed=3, n_pulses=2, forget_steps=1000)
    devs = [dataclasses.replace(d, R=d.R // 16, L=d.L // 4) for d in devs]
    n = len(V)
    b = kmc.Batch(devs, [V] * len(devs), [1] * len(devs), fills=fills)
    b.set_launch(4, 256)
    b.step_n(n)
    rng = np.random.default_rng(0)
    for i, d in enumerate(devs):
        wJ = rng.normal(size=n)
        wZ = rng.normal(size=(n, d.Z))
        gb, sb = b.grad(i, wJ, wZ)
        sim = kmc.Sim(d, V, init_mode=1, fill=fills[i])
        sim.step_n(n)
        gs, ss = sim.grad(wJ, wZ)
        sim.close()
        assert np.array_equal(gb, gs) and np.array_equal(sb, ss), i
    b.close()


def test_batched_gradient_passes_equal_per_device_passes(kmc):
    """kmc_batch_grad_all (one launch for all devices) returns, bit for bit,
    each device's own kmc_batch_grad, with weights missing for some devices."""
    devs, V, fills, samples = W.fit_batch(6, seed=4, n_pulses=2, forget_steps=1000)
    devs = [dataclasses.replace(d, R=d.R // 16, L=d.L // 2) for d in devs]
    devs[1] = dataclasses.replace(devs[1], electrodes=1, k_e=2e5, rho_e=0.2)
    n = len(V)
    b = kmc.Batch(devs, [V] * len(devs), [1] * len(devs), fills=fills)
    b.step_n(n)
    rng = np.random.default_rng(1)
    wJs = [rng.normal(size=n) if i != 2 else None for i in range(len(devs))]
    wZs = [rng.normal(size=(n, d.Z)) if i != 4 else None for i, d in enumerate(devs)]
    g, se = b.grad_all(wJs, wZs)
    for i in range(len(devs)):
        gi, si = b.grad(i, wJs[i], wZs[i])
        assert np.array_equal(g[i], gi, equal_nan=True) and np.array_equal(se[i], si, equal_nan=True), i
    b.close()


def test_batched_gradient_passes_of_every_kernel_shape(kmc):
    """One device of every tile shape (lanes per rail 1 ... 32, and 32 lanes of
    two words): the batched gradient pass runs one launch per shape and
    returns, bit for bit, each device's own pass, with dense weights on some
    devices and the fit's sparse first-zone weights on others."""
    devs, V, fills, samples = W.fit_batch(7, seed=6, n_pulses=2, forget_steps=1000)
    Ls = [20, 40, 100, 200, 400, 900, 1500]
    devs = [dataclasses.replace(d, R=max(8, d.R // 64), L=L, Z=min(10, L)) for d, L in zip(devs, Ls)]
    n = len(V)
    b = kmc.Batch(devs, [V] * len(devs), [1] * len(devs), fills=fills)
    b.step_n(n)
    rng = np.random.default_rng(2)
    wJs, wZs = [], []
    for i, d in enumerate(devs):
        if i % 2:
            wZ = np.zeros((n, d.Z))
            wZ[samples, 0] = rng.normal(size=len(samples))
            wJs.append(None)
            wZs.append(wZ)
        else:
            wJs.append(rng.normal(size=n))
            wZs.append(rng.normal(size=(n, d.Z)))
    g, se = b.grad_all(wJs, wZs)
    for i in range(len(devs)):
        gi, si = b.grad(i, wJs[i], wZs[i])
        assert np.array_equal(g[i], gi, equal_nan=True) and np.array_equal(se[i], si, equal_nan=True), i
    b.close()


def _fit_case():
    """4 devices of 8,192 rails x 160 sites, 4 pulses + 4,000 steps; targets are
    the oracle's curves at the hidden (0.42 eV, 0.9) from 32 rails per device."""
    devs, V, fills, samples = W.fit_batch(4, seed=5, n_pulses=4, forget_steps=4000,
                                          sample_every=250)
    devs = [dataclasses.replace(d, R=8192, L=160) for d in devs]
    n = int(samples.max()) + 1
    target = np.zeros((len(devs), len(samples)))
    for i, (d, fill) in enumerate(zip(devs, fills)):
        dev = dict(d.as_dict(), Ea=0.42, kappa=0.9)
        ids = np.arange(0, d.R, d.R // 32, dtype=np.int32)
        occ0 = oracle.init_occupancy(dev, 1, fill=fill, rail_ids=ids)
        _, Zc = oracle.OracleSim(dev, V[:n], occ0, rail_ids=ids).step_n(n)
        target[i] = Zc[samples, 0] / occ0.sum()
    return devs, V, fills, samples, target


def test_fit_gradient_agrees_with_finite_differences(kmc):
    from paper_2511_09413_gb300.fit import MaterialFit
    devs, V, fills, samples, target = _fit_case()
    fit = MaterialFit(devs, V, fills, samples, target, warps=8, steps_per_launch=1024)
    st = fit.loss_and_grad(0.40, 1.0)
    h = 0.004      # the same draws at Ea +- h (common random numbers)
    fd = (fit.loss_and_grad(0.40 + h, 1.0).loss - fit.loss_and_grad(0.40 - h, 1.0).loss) / (2 * h)
    assert fd < 0 and st.grad[0] < 0, (fd, st.grad, st.stderr)
    assert abs(st.grad[0] - fd) < 4.0 * st.stderr[0] + 0.2 * abs(fd), (fd, st.grad, st.stderr)


def test_fit_moves_toward_hidden_parameters(kmc):
    from paper_2511_09413_gb300.fit import MaterialFit
    devs, V, fills, samples, target = _fit_case()
    fit = MaterialFit(devs, V, fills, samples, target, warps=8, steps_per_launch=1024)
    hist = fit.run(0.40, 1.0, iters=5, lr=(3e-3, 3e-2))
    assert hist[-1].Ea > 0.405, [h.Ea for h in hist]
    assert hist[-1].loss < 0.7 * hist[0].loss, [h.loss for h in hist]
