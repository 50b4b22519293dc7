"""Shapes the paper validates, checked on the oracle (Sec. 4, Figs. 1-2;
Supplementary S4, Figs. S1 and S3).  The paper prints no figure data, so the
magnitudes are unpinned; only the qualitative trends it states are tested:

- relaxation decay (Fig. 1): the decile-1 ion ratio grows with polarisation
  voltage and time, linearly at low voltage and time, saturates at high
  voltage, and decays monotonically toward a common value once the bias is off;
- I-V hysteresis (Fig. 2, Fig. S3): faster sweeps give lower peak current and
  narrower loops;
- rails vs noise (S4.1): rails fluctuate independently, so the fluctuation of
  the device signal falls as 1/sqrt(rails);
- potentiation and forgetting under a pulse train (Fig. 3, Fig. S4): the
  conductance rises pulse by pulse and relaxes once the pulses stop; a longer
  relaxation time tau is slower and more persistent, and its relaxation is
  less noisy (Fig. S2).  tau is the hop time scale (Gamma_0 of Eq. 1 is
  proportional to 1/tau), so a tau k times longer is nu / k here;
- the spike-timing (STDP) analogue of the abstract (reading R20, on a
  shortened window): a post pulse (-1 V) before the pre pulse (+1 V)
  potentiates, most when the pulses are close; the reverse order depresses,
  the more the later the post pulse comes before the fixed readout.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09413_gb300 import workloads as W


def _dev(R, **kw):
    d = dict(R=R, L=100, Z=10, electrodes=0, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=1, instance=0)
    d.update(kw)
    return d


def _decile1_trace(dev, V, fill=0.3):
    occ0 = oracle.init_occupancy(dev, 1, fill=fill)
    sim = oracle.OracleSim(dev, V, occ0)
    J, Zc = sim.step_n(len(V))
    N = occ0.sum()
    return Zc[:, 0] / N, Zc[:, -1] / N, J / N


@pytest.fixture(scope="module")
def relaxation_by_voltage():
    out = {}
    for Vp in (0.25, 0.5, 1.0, 2.0):
        r, _, _ = _decile1_trace(_dev(256), W.relaxation_protocol(1000, Vp, 3500))
        out[Vp] = r
    return out


def test_relaxation_grows_with_polarisation_voltage(relaxation_by_voltage):
    r = relaxation_by_voltage
    start = np.mean([r[v][:50].mean() for v in r])
    at_removal = {v: r[v][950:1000].mean() for v in r}
    vals = [at_removal[v] for v in sorted(r)]
    assert all(a < b for a, b in zip(vals, vals[1:]))
    gain = {v: at_removal[v] - start for v in r}
    # linear response at moderate voltage ...
    assert 1.6 < gain[0.5] / gain[0.25] < 2.4
    # ... and saturation / Coulombic crowding at high voltage
    assert gain[2.0] / gain[1.0] < 1.6


def test_relaxation_decays_monotonically_toward_common_value(relaxation_by_voltage):
    r = relaxation_by_voltage
    for v in (0.5, 1.0, 2.0):
        blocks = r[v][1000:3500].reshape(5, 500).mean(axis=1)
        assert np.all(np.diff(blocks) < 0), (v, blocks)
    # curves approach each other once the bias is off
    gap_removal = r[2.0][950:1000].mean() - r[0.5][950:1000].mean()
    gap_end = r[2.0][-200:].mean() - r[0.5][-200:].mean()
    assert 0 < gap_end < 0.75 * gap_removal
    # higher polarisation relaxes more slowly (still higher at the end)
    ends = [r[v][-200:].mean() for v in sorted(r)]
    assert all(a < b for a, b in zip(ends, ends[1:]))


def test_relaxation_accumulation_linear_in_polarisation_time():
    gains = {}
    for npol in (250, 500):
        r, _, _ = _decile1_trace(_dev(256, seed=4), W.relaxation_protocol(npol, 0.5, npol + 10))
        gains[npol] = r[npol - 20:npol].mean() - r[:20].mean()
    assert 1.6 < gains[500] / gains[250] < 2.4


def _loop(steps_per_cycle, R=256, amp=1.0):
    V = W.triangle_protocol(amp, steps_per_cycle, 2)
    d1, d10, _ = _decile1_trace(_dev(R, seed=3), V)
    # current (a.u.): decile 1 at V >= 0, decile 10 at V < 0 (Fig. 2 caption, S3)
    I = np.where(V >= 0, d1, d10)
    v, i = V[-steps_per_cycle:], I[-steps_per_cycle:]
    area = abs(np.sum(0.5 * (i[1:] + i[:-1]) * np.diff(v)))
    return i.max(), area


def test_hysteresis_faster_sweeps_give_smaller_loops():
    peak_slow, area_slow = _loop(2000)
    peak_fast, area_fast = _loop(500)
    peak_slowest, _ = _loop(8000)
    assert peak_slowest > peak_slow > peak_fast
    assert area_fast < area_slow
    assert area_fast > 0.0


def test_noise_falls_as_inverse_sqrt_rails():
    def fluct(R):
        _, _, j = _decile1_trace(_dev(R, seed=5), np.zeros(800))
        r, _, _ = _decile1_trace(_dev(R, seed=5), np.zeros(800))
        return np.diff(r).std(), j.std()
    small, big = fluct(64), fluct(1024)
    for a, b in zip(small, big):
        assert 3.4 < a / b < 4.6     # sqrt(1024 / 64) = 4


def _pulse_train(nu, R=128, n_pulses=8, forget=8000):
    """Decile-1 conductance G(t) under n_pulses pulses of 0.8 V (0.25 ms on,
    0.25 ms off at 2,000 steps per ms), then `forget` steps at 0 V."""
    V = W.potentiation_protocol(n_pulses, forget, V_pulse=0.8, pulse_ms=0.25, gap_ms=0.25,
                                steps_per_ms=2000)
    G, _, _ = _decile1_trace(_dev(R, nu=nu, seed=7), V)
    return G


@pytest.fixture(scope="module")
def pulse_trains():
    # tau and 5 tau (Figs. 3 and S4 compare relaxation times 1 ms and 5 ms)
    return {1: _pulse_train(1e12), 5: _pulse_train(2e11)}


def _pulse_ends(G, n_pulses=8, period=1000, on=500):
    return np.array([G[k * period + on - 20:k * period + on].mean() for k in range(n_pulses)])


def test_pulse_train_potentiates_then_forgets(pulse_trains):
    for tau, G in pulse_trains.items():
        G0 = G[:20].mean()
        ends = _pulse_ends(G)
        assert G0 < ends[0] < ends[-1], (tau, G0, ends)
        # forgetting: the conductance falls in every 2,000-step block after the train
        blocks = G[8000:].reshape(4, 2000).mean(axis=1)
        assert np.all(np.diff(blocks) < 0), (tau, blocks)
        assert blocks[-1] > G0              # not yet back to the start
    # the short tau saturates under the train: most of its gain comes from the
    # first pulses, while the long tau keeps rising
    e1, e5 = _pulse_ends(pulse_trains[1]), _pulse_ends(pulse_trains[5])
    assert (e1[3] - e1[0]) > 3.0 * (e1[7] - e1[4])
    assert np.all(np.diff(e5) > 0)


def test_longer_tau_is_slower_and_more_persistent(pulse_trains):
    gain, kept = {}, {}
    for tau, G in pulse_trains.items():
        G0 = G[:20].mean()
        gain[tau] = _pulse_ends(G)[0] - G0
        trained = G[7980:8000].mean() - G0
        kept[tau] = (G[-200:].mean() - G0) / trained
    assert gain[5] < 0.5 * gain[1]          # slower: less gained in the first pulse
    assert kept[5] > 2.0 * kept[1]          # more persistent after the train


def test_longer_tau_relaxes_with_less_noise(pulse_trains):
    noise = {tau: np.diff(G[10000:]).std() for tau, G in pulse_trains.items()}
    assert noise[5] < 0.75 * noise[1]


def test_spike_pair_timing_sign_and_closeness():
    """Delta G = G(t_pre + 10 ms) - G(t_pre^-) for pre/post delays of -8, -2,
    +2 and +8 ms (1 ms pulses of +-1 V, 500 steps per ms)."""
    spm, t_pre = 500, 10.0
    dG = {}
    for delay in (-8.0, -2.0, 2.0, 8.0):
        V = W.spike_pair_protocol(delay, spm, t_pre_ms=t_pre, window_ms=t_pre + 10.0)
        G, _, _ = _decile1_trace(_dev(128, dt=1e-3 / spm, seed=9), V)
        i_pre = int(round(t_pre * spm))
        dG[delay] = G[-1] - G[i_pre - 1]
    assert dG[-2.0] > dG[-8.0] > 0.0, dG      # post before pre: potentiation, closer is stronger
    assert dG[8.0] < dG[2.0] < 0.0, dG        # pre before post: depression, read at a fixed time
