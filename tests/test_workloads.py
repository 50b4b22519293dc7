"""The synthetic inputs against the readings they implement (CPU): voltage
protocols (relaxation, S2.2.2; the hysteresis triangle, R19; the STDP spike
pair, R20; the potentiation train of the fit, R23) and the named devices'
sizes, parameters and value distributions."""
import numpy as np
import pytest

from paper_2511_09413_gb300 import workloads as W


def test_relaxation_protocol_polarises_then_holds():
    V = W.relaxation_protocol(5, 1.5, 12, -0.25)
    assert V.dtype == np.float64 and V.shape == (12,)
    assert np.all(V[:5] == 1.5) and np.all(V[5:] == -0.25)


@pytest.mark.parametrize("spc", [4, 100, 100000])
def test_triangle_is_zero_up_zero_down_zero_per_cycle(spc):
    A = 2.0
    V = W.triangle_protocol(A, spc, 2)
    assert V.shape == (2 * spc,)
    q = spc // 4
    assert V[0] == 0.0 and V[q] == A and V[2 * q] == 0.0 and V[3 * q] == -A
    assert np.array_equal(V[:spc], V[spc:])                  # periodic
    assert V.max() == A and V.min() == -A
    if spc >= 8:
        d = np.diff(V[:spc])                                  # slopes +-4A/spc, sampled at step start
        assert np.allclose(np.abs(d), 4 * A / spc)
        assert np.all(d[:q] > 0) and np.all(d[q:3 * q] < 0) and np.all(d[3 * q:] > 0)


@pytest.mark.parametrize("delay", [-50.0, -3.5, 0.0, 0.5, 2.0, 50.0])
def test_spike_pair_has_one_pulse_of_each_sign(delay):
    spm, t_pre, pulse = 2000, 55.0, 1.0
    V = W.spike_pair_protocol(delay, spm)
    assert V.shape == (120 * spm,)
    t = np.arange(V.size) / spm
    pre = (t >= t_pre) & (t < t_pre + pulse)
    post = (t >= t_pre + delay) & (t < t_pre + delay + pulse)
    assert np.array_equal(V, pre.astype(float) - post.astype(float))   # summed where overlapping
    assert pre.sum() == pulse * spm
    assert V.sum() == 0.0
    if delay == 0.0:
        assert not V.any()


def test_potentiation_train_then_forgetting():
    V = W.potentiation_protocol(3, 700)
    on = off = 1000                     # 0.5 ms at 2,000 steps per ms
    assert V.size == 3 * (on + off) + 700
    for k in range(3):
        p = V[k * (on + off):(k + 1) * (on + off)]
        assert np.all(p[:on] == 0.8) and not p[on:].any()
    assert not V[3 * (on + off):].any()


def test_relaxation_device_is_the_64x100_parity_case():
    wl = W.relaxation_64x100()
    d = wl.device
    assert (d.R, d.L, d.Z, d.electrodes, d.seed) == (64, 100, 10, 0, 0)
    assert (d.Ea, d.nu, d.T, d.d, d.dt) == (0.40, 1e12, 300.0, 1.0, 1e-9)
    assert wl.init_mode == 0 and wl.n_ions == 800 and wl.n_steps == 10000
    assert np.all(wl.V[:5000] == 1.0) and not wl.V[5000:].any()


def test_hysteresis_device_recipe():
    wl = W.hysteresis_65536x1024(R=512, L=1024)     # same recipe, fewer rails
    d = wl.device
    assert (d.L, d.Z, d.electrodes, d.k_e, d.rho_e, d.dt) == (1024, 10, 1, 1e9, 0.25, 1e-9)
    assert wl.init_mode == 1 and wl.fill == 0.25 and wl.n_steps == 200000
    assert np.array_equal(wl.V, W.triangle_protocol(2.0, 100000, 2))
    Ea = wl.Ea_site
    assert Ea.shape == (512, 1024)
    assert abs(Ea.mean() - 0.40) < 3 * 0.02 / np.sqrt(Ea.size)
    assert abs(Ea.std() - 0.02) < 0.02 * 0.01
    full = W.hysteresis_65536x1024(with_barriers=False)
    assert (full.device.R, full.device.L) == (65536, 1024) and full.Ea_site is None


def test_stdp_batch_distributions():
    devs, Vs, fills, delays = W.stdp_batch(512, n_steps=10)
    R = np.array([d.R for d in devs])
    L = np.array([d.L for d in devs])
    assert len(devs) == 512 and len(set(d.instance for d in devs)) == 512
    assert R.min() >= 256 and R.max() <= 16384 and L.min() >= 128 and L.max() <= 2048
    # log-uniform: the mean of log R sits at the middle of [log 256, log 16384]
    assert abs(np.log(R).mean() - np.log(2048)) < 0.15
    assert abs(np.log(L).mean() - np.log(512)) < 0.15
    assert min(fills) >= 0.05 and max(fills) <= 0.4
    assert min(delays) >= -50 and max(delays) <= 50
    assert all(d.dt == 5e-7 and d.electrodes == 0 for d in devs)
    assert all(v.shape == (10,) for v in Vs)


def test_adjoint_device_recipe():
    wl = W.adjoint_relaxation(replicas=2, n_write=10, n_relax=30)
    d = wl.device
    assert (d.R, d.L, d.Z, d.electrodes, d.dt) == (2 * 4096, 512, 10, 0, 5e-7)
    assert wl.init_mode == 1 and wl.fill == 0.2
    assert np.all(wl.V[:10] == 1.0) and not wl.V[10:].any() and wl.n_steps == 40


def test_fit_batch_recipe():
    devs, V, fills, samples = W.fit_batch(n_dev=256, n_pulses=2, forget_steps=1000)
    R = np.array([d.R for d in devs])
    L = np.array([d.L for d in devs])
    assert len(devs) == 256
    assert R.min() >= 2048 and R.max() <= 8192 and L.min() >= 256 and L.max() <= 1024
    assert min(fills) >= 0.1 and max(fills) <= 0.3
    assert np.array_equal(V, W.potentiation_protocol(2, 1000))
    assert np.array_equal(samples, np.arange(499, V.size, 500))


def test_seeded_inputs_are_reproducible():
    a = W.random_occupancy(7, 33, 0.3, seed=5)
    assert a.dtype == np.uint8 and set(np.unique(a)) <= {0, 1}
    assert np.array_equal(a, W.random_occupancy(7, 33, 0.3, seed=5))
    assert not np.array_equal(a, W.random_occupancy(7, 33, 0.3, seed=6))
    b = W.normal_barriers(5, 9, 0.4, 0.02, seed=1)
    assert np.array_equal(b, W.normal_barriers(5, 9, 0.4, 0.02, seed=1))


def test_barrier_table_rows_of_a_shard_equal_the_whole_table():
    """A rank generating only its rows of the per-site barrier table gets
    exactly those rows of the whole device's table (blockwise streams)."""
    whole = W.normal_barriers(50, 200_000, 0.4, 0.02, seed=3)      # blocks of 20 rows
    for r0, r1 in [(0, 7), (7, 20), (19, 41), (40, 50), (0, 50)]:
        part = W.normal_barriers(r1 - r0, 200_000, 0.4, 0.02, seed=3, row0=r0)
        assert np.array_equal(part, whole[r0:r1])
    wl = W.hysteresis_65536x1024(R=8, L=64, rail_base=24)
    assert wl.device.rail_base == 24
    assert np.array_equal(wl.Ea_site, W.normal_barriers(40, 64, 0.40, 0.02, 1001)[24:32])
