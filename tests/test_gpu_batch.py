"""GPU parity of the batched launch: many devices of different sizes,
parameters and voltage tables advanced together, each bit-identical to the
oracle; graph replays, odd chunk sizes and the autotuner (which must leave
the simulation unchanged)."""
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
    return K


def _batch_case(n, n_steps, seed=0):
    rng = np.random.default_rng(seed)
    devs, Vs, occs = [], [], []
    for i in range(n):
        L = int(rng.choice([2, 31, 64, 100, 200, 257, 700, 1024, 1500, 2048]))
        R = int(rng.integers(1, 90))
        Z = int(min(L, rng.choice([1, 4, 10])))
        el = int(rng.integers(0, 2))
        devs.append(dict(R=R, L=L, Z=Z, electrodes=el, d=1.0, dt=float(rng.choice([2e-7, 5e-7])),
                         T=300.0, Ea=float(rng.uniform(0.38, 0.42)), nu=1e12,
                         alpha=float(rng.uniform(0.0, 0.5)), kappa=1.0, k_e=2e6 if el else 0.0,
                         rho_e=float(rng.uniform(0.1, 0.6)) if el else 0.0, seed=77,
                         instance=1000 + i, rail_base=int(rng.choice([0, 0, 5000]))))
        # each device its own protocol: a triangle of random amplitude and period
        period = int(rng.integers(50, 400))
        Vs.append(W.triangle_protocol(float(rng.uniform(0.5, 4.0)), period,
                                      n_steps // period + 1)[:n_steps])
        occs.append(W.random_occupancy(R, L, float(rng.uniform(0.05, 0.6)), seed=int(rng.integers(1 << 30))))
    return devs, Vs, occs


def _check_against_oracle(b, devs, Vs, occs, n_steps, Eas=None):
    for i, (dev, V, occ0) in enumerate(zip(devs, Vs, occs)):
        orc = oracle.OracleSim(dev, V, occ0, None if Eas is None else Eas[i])
        Jo, Zo = orc.step_n(n_steps)
        Jg, Zg = b.traces(i)
        assert np.array_equal(Zg, Zo), i
        assert np.array_equal(Jg, Jo), i
        assert np.array_equal(b.occupancy(i), orc.occ), i
        assert np.array_equal(b.rail_current(i), orc.J_rail), i


def test_batch_bit_exact_with_graph_replays(kmc):
    n_steps = 530
    devs, Vs, occs = _batch_case(14, n_steps, seed=1)
    b = kmc.Batch(devs, Vs, [2] * len(devs), occ0s=occs)
    b.set_launch(8, 128)                 # graph of 128 steps, replayed; odd remainders
    b.step_n(300)
    b.step_n(230)
    assert b.t == n_steps
    _check_against_oracle(b, devs, Vs, occs, n_steps)
    b.close()


def test_batch_small_ctas_and_direct_launches(kmc):
    n_steps = 211
    devs, Vs, occs = _batch_case(9, n_steps, seed=2)
    b = kmc.Batch(devs, Vs, [2] * len(devs), occ0s=occs)
    b.set_launch(2, 1000)                # every call is a direct launch
    for n in (1, 7, 64, 139):
        b.step_n(n)
    _check_against_oracle(b, devs, Vs, occs, n_steps)
    b.close()


def test_batch_autotuner_leaves_the_simulation_unchanged(kmc):
    n_steps = 400
    devs, Vs, occs = _batch_case(10, 2 * n_steps, seed=3)
    b = kmc.Batch(devs, Vs, [2] * len(devs), occ0s=occs)
    b.step_n(37)
    warps, steps = b.tune(256)
    assert warps in (4, 8) and steps in (64, 128, 256)
    assert b.t == 37
    b.step_n(n_steps - 37)
    _check_against_oracle(b, devs, [v[:n_steps] for v in Vs], occs, n_steps)
    b.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_accept_path_modes_bit_exact(kmc, mode):
    """Both batch kernels (with and without the inline accept path) on the same
    mixed batch, against the oracle."""
    n_steps = 260
    devs, Vs, occs = _batch_case(8, n_steps, seed=5)
    b = kmc.Batch(devs, Vs, [2] * len(devs), occ0s=occs)
    b.set_accept_path(mode)
    assert b.accept_path == mode
    b.set_launch(4, 100)
    b.step_n(n_steps)
    _check_against_oracle(b, devs, Vs, occs, n_steps)
    b.close()


def test_batch_rejects_mixed_seeds(kmc):
    devs, Vs, occs = _batch_case(2, 10, seed=4)
    devs[1]["seed"] = 78
    with pytest.raises(kmc.KmcError):
        kmc.Batch(devs, Vs, [2, 2], occ0s=occs)


def test_batch_with_brick_wall_devices(kmc):
    """Devices of either update rule in one batch, each equal to the oracle."""
    n_steps = 240
    devs, Vs, occs = _batch_case(10, n_steps, seed=6)
    for i in range(0, len(devs), 2):
        devs[i]["rule"] = 1
    b = kmc.Batch(devs, Vs, [2] * len(devs), occ0s=occs)
    b.set_launch(8, 64)
    b.step_n(n_steps)
    _check_against_oracle(b, devs, Vs, occs, n_steps)
    b.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_with_per_site_barriers_bit_exact(kmc, mode):
    """Devices with per-site barrier tables (every other device of a batch of
    mixed tile shapes) next to scalar-barrier devices, with graph replays and
    either accept path: each device equals the oracle, and a gradient pass on
    a per-site device is refused."""
    n_steps = 300
    devs, Vs, occs = _batch_case(12, n_steps, seed=8)
    Eas = [W.normal_barriers(d["R"], d["L"], 0.40, 0.03, seed=100 + i) if i % 2 == 0 else None
           for i, d in enumerate(devs)]
    b = kmc.Batch(devs, Vs, [2] * len(devs), occ0s=occs, Ea_sites=Eas)
    b.set_accept_path(mode)
    b.set_launch(8, 128)
    b.step_n(200)
    b.step_n(100)
    _check_against_oracle(b, devs, Vs, occs, n_steps, Eas)
    with pytest.raises(kmc.KmcError):
        b.grad(0, np.ones(n_steps), None)
    b.close()
