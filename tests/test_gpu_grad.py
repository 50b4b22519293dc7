"""GPU parity of the likelihood-ratio gradient pass (kmc_grad) against the
oracle's estimator (orc_run_lr) on the same seeded inputs, its agreement with
central finite differences under common random numbers, and the
torch.autograd front end."""
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


def _dev(**kw):
    d = dict(R=48, L=100, Z=10, electrodes=0, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=21, instance=3)
    d.update(kw)
    return d


def _pulse(n_write, n_relax, v=1.0):
    return np.concatenate([np.full(n_write, v), np.zeros(n_relax)])


def _weights(n, Z, seed, with_J=True, with_Z=True):
    rng = np.random.default_rng(seed)
    wJ = rng.normal(size=n) if with_J else None
    wZ = rng.normal(size=(n, Z)) if with_Z else None
    return wJ, wZ


@pytest.mark.parametrize("L,Z,electrodes", [(100, 10, 0), (100, 10, 1), (7, 3, 1), (40, 5, 0),
                                            (700, 10, 1), (1500, 12, 0), (2048, 32, 1)])
def test_grad_matches_oracle_estimator(kmc, L, Z, electrodes):
    """Same trajectory, same per-trial scores: the GPU's FP64 estimator equals
    the oracle's up to summation order."""
    R = 40
    dev = _dev(R=R, L=L, Z=Z, electrodes=electrodes, k_e=1e6 if electrodes else 0.0,
               rho_e=0.3 if electrodes else 0.0, alpha=0.4)
    fill = 0.3
    V = _pulse(90, 150, 1.5)
    n = len(V)
    wJ, wZ = _weights(n, Z, seed=L + Z)
    sim = kmc.Sim(dev, V, init_mode=1, fill=fill)
    sim.step_n(n)
    g, se = sim.grad(wJ, wZ)
    occ0 = oracle.init_occupancy(dev, 1, fill=fill)
    ref = oracle.lr_gradient(dev, V, occ0, n, wJ=wJ, wZ=wZ, fill=fill)
    scale = np.abs(ref["G"]).sum(axis=0)
    assert np.all(scale > 0)
    np.testing.assert_allclose(g, ref["grad"], rtol=1e-10, atol=1e-11 * scale.max())
    for i in range(4):
        assert abs(g[i] - ref["grad"][i]) <= 1e-11 * scale[i] + 1e-10 * abs(ref["grad"][i])
    np.testing.assert_allclose(se, ref["stderr"], rtol=1e-8)
    sim.close()


def test_grad_observables_separately_and_deterministic(kmc):
    dev = _dev(R=64, L=128, Z=8, electrodes=1, k_e=5e5, rho_e=0.25)
    V = _pulse(60, 140, 1.0)
    n = len(V)
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.25)
    sim.step_n(n)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.25)
    for with_J, with_Z in [(True, False), (False, True)]:
        wJ, wZ = _weights(n, 8, seed=5, with_J=with_J, with_Z=with_Z)
        g1, _ = sim.grad(wJ, wZ)
        g2, _ = sim.grad(wJ, wZ)
        assert np.array_equal(g1, g2), "gradient pass not deterministic"
        ref = oracle.lr_gradient(dev, V, occ0, n, wJ=wJ, wZ=wZ, fill=0.25)
        scale = np.abs(ref["G"]).sum(axis=0)
        assert np.all(np.abs(g1 - ref["grad"]) <= 1e-11 * scale + 1e-10 * np.abs(ref["grad"]))
    sim.close()


@pytest.mark.parametrize("with_J", [False, True])
def test_grad_sparse_zone_weights_match_oracle(kmc, with_J):
    """Zone weights set at a few steps and zones only, as the fit's samples of
    the first-zone count: the replay skips the zones outside each step's range
    of nonzero weights and the steps without any, and still equals the
    oracle's estimator (which sums every zone of every step)."""
    Z = 10
    dev = _dev(R=40, L=200, Z=Z, electrodes=1, k_e=1e6, rho_e=0.3, alpha=0.4)
    V = _pulse(80, 170, 1.2)
    n = len(V)
    rng = np.random.default_rng(77)
    wZ = np.zeros((n, Z))
    wZ[::25, 0] = rng.normal(size=len(range(0, n, 25)))     # first zone, every 25th step
    wZ[101, 3] = 0.7                                         # a range with a zero inside
    wZ[101, 6] = -0.4
    wZ[157, Z - 1] = 1.3                                     # the last zone alone
    wZ[203, 4] = -0.0                                        # a signed zero counts as no weight
    wJ = rng.normal(size=n) if with_J else None
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.3)
    sim.step_n(n)
    g, se = sim.grad(wJ, wZ)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    ref = oracle.lr_gradient(dev, V, occ0, n, wJ=wJ, wZ=wZ, fill=0.3)
    scale = np.abs(ref["G"]).sum(axis=0)
    assert np.all(scale > 0)
    assert np.all(np.abs(g - ref["grad"]) <= 1e-11 * scale + 1e-10 * np.abs(ref["grad"]))
    np.testing.assert_allclose(se, ref["stderr"], rtol=1e-8)
    sim.close()


def test_grad_leaves_forward_state_unchanged(kmc):
    """The backward pass replays on its own buffers: stepping on after a
    gradient call gives the oracle's trajectory."""
    dev = _dev(R=32, L=90, Z=6)
    V = _pulse(100, 200, 1.0)
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.3)
    sim.step_n(120)
    wJ = np.ones(120) / 120
    sim.grad(wJ, None)
    sim.step_n(180)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    orc = oracle.OracleSim(dev, V, occ0)
    Jo, Zo = orc.step_n(300)
    Jg, Zg = sim.traces()
    assert np.array_equal(Jg, Jo) and np.array_equal(Zg, Zo)
    assert np.array_equal(sim.occupancy(), orc.occ)
    sim.close()


def test_grad_special_cases(kmc):
    # no weights, no steps: zero; exact-count placement: no fill entry
    dev = _dev(R=8, L=50, Z=5)
    V = _pulse(10, 10)
    sim = kmc.Sim(dev, V, init_mode=0, n_ions=100)
    g, se = sim.grad(None, None)
    assert np.all(g[:3] == 0.0) and np.isnan(g[3])
    sim.step_n(20)
    g, se = sim.grad(np.ones(20), None)
    assert np.all(np.isfinite(g[:3])) and np.isnan(g[3])
    sim.close()
    # alpha = 0: the field coupling drops out of every probability
    dev = _dev(R=16, L=60, Z=4, alpha=0.0)
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.3)
    sim.step_n(20)
    g, _ = sim.grad(np.ones(20), np.ones((20, 4)))
    assert g[2] == 0.0
    sim.close()
    # per-site barriers are rejected
    dev = _dev(R=4, L=30, Z=3)
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.3, Ea_site=W.normal_barriers(4, 30, 0.4, 0.02, 1))
    sim.step_n(5)
    with pytest.raises(kmc.KmcError):
        sim.grad(np.ones(5), None)
    sim.close()


def _mean_relax_current(kmc, dev, V, n_write, fill):
    sim = kmc.Sim(dev, V, init_mode=1, fill=fill)
    sim.step_n(len(V))
    J, _ = sim.traces()
    sim.close()
    return J[n_write:].mean() / dev["R"]


def test_grad_agrees_with_crn_finite_differences(kmc):
    """Mean relaxation current per rail after a write pulse; LR gradient
    against central differences (h = 1e-3 relative) with common random numbers,
    over independent instances, within 4 combined standard errors."""
    n_write, n_relax = 150, 250
    V = _pulse(n_write, n_relax, 1.0)
    n = len(V)
    fill = 0.2
    R = 1 << 16
    base = _dev(R=R, L=64, Z=8, alpha=0.3)
    wJ = np.zeros(n)
    wJ[n_write:] = 1.0 / (n_relax * R)
    n_inst = 8
    lr, lr_se = [], []
    fd = {k: [] for k in range(4)}
    for inst in range(n_inst):
        dev = dict(base, instance=100 + inst)
        sim = kmc.Sim(dev, V, init_mode=1, fill=fill)
        sim.step_n(n)
        g, se = sim.grad(wJ, None)
        sim.close()
        lr.append(g)
        lr_se.append(se)
        for k, nm in enumerate(["Ea", "nu", "kappa"]):
            h = 1e-3 * abs(dev[nm])
            fp = _mean_relax_current(kmc, dict(dev, **{nm: dev[nm] + h}), V, n_write, fill)
            fm = _mean_relax_current(kmc, dict(dev, **{nm: dev[nm] - h}), V, n_write, fill)
            fd[k].append((fp - fm) / (2 * h))
        h = 1e-3 * fill
        fp = _mean_relax_current(kmc, dev, V, n_write, fill + h)
        fm = _mean_relax_current(kmc, dev, V, n_write, fill - h)
        fd[3].append((fp - fm) / (2 * h))
    lr = np.mean(lr, axis=0)
    lr_se = np.sqrt(np.sum(np.square(lr_se), axis=0)) / n_inst
    for k in range(4):
        f = np.array(fd[k])
        f_se = f.std(ddof=1) / np.sqrt(len(f))
        tol = 4.0 * np.hypot(lr_se[k], f_se)
        assert abs(lr[k] - f.mean()) <= tol, (k, lr[k], f.mean(), lr_se[k], f_se)
        # the check has power: the LR gradient is resolved to 10 % and the
        # combined tolerance is below the gradient itself
        assert lr_se[k] < 0.1 * abs(lr[k]), (k, lr[k], lr_se[k])
        assert tol < abs(f.mean()), (k, lr[k], f.mean(), lr_se[k], f_se)


def test_autograd_function(kmc):
    import torch
    from paper_2511_09413_gb300 import autograd as KA
    from paper_2511_09413_gb300.workloads import Device
    dev = Device(R=256, L=80, Z=8, dt=5e-7, alpha=0.3, seed=3)
    V = _pulse(50, 70, 1.0)
    theta = torch.tensor([0.40, 1e12, 1.0, 0.25], dtype=torch.float64, requires_grad=True)
    J, Zc = KA.simulate(theta, dev, V, len(V))
    loss = J[50:].mean() + 0.1 * Zc[-1, 0]
    loss.backward()
    wJ = np.zeros(len(V))
    wJ[50:] = 1.0 / 70
    wZ = np.zeros((len(V), 8))
    wZ[-1, 0] = 0.1
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.25)
    sim.step_n(len(V))
    g, _ = sim.grad(wJ, wZ)
    sim.close()
    np.testing.assert_allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0)
