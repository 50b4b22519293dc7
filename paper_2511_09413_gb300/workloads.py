"""Seeded synthetic workloads for the rail-based KMC sweep.

This module is the one piece shared by the CUDA path, the oracle, the tests
and the benchmark.  It holds device descriptions (sizes and physical
parameters), the applied-voltage protocols as per-step tables, and seeded
random inputs (initial occupancies, per-site barriers).  It holds none of the
method's arithmetic: no field, rate, probability or update rule.

Protocols follow the paper's simulation types (Supplementary S2.2.2-S2.2.4,
Table S1): relaxation decay (polarise, then hold a constant voltage) and the
hysteresis sweep.  The hysteresis waveform is the triangle
0 -> +A -> 0 -> -A -> 0 per cycle, sampled at the start of each step.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Device:
    """Physical description of one simulated device (one instance).

    Units: lengths in nm, energies in eV, times in s, rates in Hz, volts.
    ``alpha`` is the rail-local space-charge voltage per excess ion and
    ``kappa`` its dimensionless coupling; ``electrodes`` is 0 for blocking and
    1 for injecting/extracting contacts with exchange rate ``k_e`` and
    reservoir density ``rho_e``.
    """

    R: int
    L: int
    Z: int = 10
    electrodes: int = 0
    d: float = 1.0
    dt: float = 1e-9
    T: float = 300.0
    Ea: float = 0.40
    nu: float = 1e12
    alpha: float = 0.2
    kappa: float = 1.0
    k_e: float = 0.0
    rho_e: float = 0.0
    seed: int = 0
    instance: int = 0
    rule: int = 0          # 0 synchronous update, 1 brick-wall (even/odd bonds)
    rail_base: int = 0     # global index of rail 0: this device is rows
                           # [rail_base, rail_base + R) of a larger one (a shard)

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Workload:
    """A device, its voltage table, its initial condition and its barriers."""

    name: str
    device: Device
    V: np.ndarray                      # float64 [n_steps]
    init_mode: int                     # 0 exact count, 1 Bernoulli(fill), 2 given occupancy
    n_ions: int = 0
    fill: float = 0.0
    occ0: Optional[np.ndarray] = None  # uint8 [R, L] when init_mode == 2
    Ea_site: Optional[np.ndarray] = None  # float64 [R, L] or None (scalar Ea)

    @property
    def n_steps(self) -> int:
        return int(self.V.shape[0])


# ---------------------------------------------------------------- protocols

def relaxation_protocol(n_polarise: int, V_polarise: float, n_total: int,
                        V_hold: float = 0.0) -> np.ndarray:
    """Relaxation decay (S2.2.2): V_polarise for n_polarise steps, then V_hold."""
    V = np.full(n_total, float(V_hold), dtype=np.float64)
    V[:n_polarise] = float(V_polarise)
    return V


def triangle_protocol(amplitude: float, steps_per_cycle: int, cycles: int) -> np.ndarray:
    """Hysteresis sweep (S2.2.3): 0 -> +A -> 0 -> -A -> 0 per cycle."""
    t = np.arange(steps_per_cycle * cycles, dtype=np.float64)
    phase = np.mod(t, steps_per_cycle) / float(steps_per_cycle)
    tri = np.where(phase < 0.25, 4.0 * phase,
                   np.where(phase < 0.75, 2.0 - 4.0 * phase, 4.0 * phase - 4.0))
    return amplitude * tri


def constant_protocol(V: float, n_steps: int) -> np.ndarray:
    return np.full(n_steps, float(V), dtype=np.float64)


def spike_pair_protocol(dt_pre_post_ms: float, steps_per_ms: int = 2000, t_pre_ms: float = 55.0,
                        window_ms: float = 120.0, amplitude: float = 1.0,
                        pulse_ms: float = 1.0) -> np.ndarray:
    """Spike-timing protocol for the STDP analogue named in the abstract: a
    +amplitude pulse of pulse_ms at t_pre and a -amplitude pulse at
    t_post = t_pre + dt_pre_post, summed where they overlap, over a window."""
    n = int(round(window_ms * steps_per_ms))
    t = np.arange(n, dtype=np.float64) / steps_per_ms
    t_post = t_pre_ms + dt_pre_post_ms
    V = np.zeros(n, dtype=np.float64)
    V += np.where((t >= t_pre_ms) & (t < t_pre_ms + pulse_ms), amplitude, 0.0)
    V -= np.where((t >= t_post) & (t < t_post + pulse_ms), amplitude, 0.0)
    return V


# ------------------------------------------------------------ seeded inputs

def random_occupancy(R: int, L: int, fill: float, seed: int) -> np.ndarray:
    """Independent Bernoulli(fill) sites from numpy's PCG64 stream."""
    rng = np.random.default_rng(seed)
    return (rng.random((R, L)) < fill).astype(np.uint8)


def normal_barriers(R: int, L: int, mean: float, sigma: float, seed: int,
                    row0: int = 0) -> np.ndarray:
    """Per-site migration barriers Ea ~ N(mean, sigma) in eV: rows
    [row0, row0 + R) of a device's table.  The table is drawn in blocks of
    B = max(1, 2^22 // L) rows, block b from its own PCG64 stream seeded with
    (seed, b), so that any range of rows (the shard of one rank) is generated
    alone and equals those rows of the whole table."""
    out = np.empty((R, L), dtype=np.float64)
    B = max(1, (1 << 22) // max(L, 1))
    g0, g1 = row0, row0 + R
    for b in range(g0 // B, (g1 - 1) // B + 1 if R > 0 else 0):
        blk = np.random.default_rng([seed, b]).normal(mean, sigma, size=(B, L))
        lo, hi = max(g0, b * B), min(g1, (b + 1) * B)
        out[lo - g0:hi - g0] = blk[lo - b * B:hi - b * B]
    return out


# ----------------------------------------------------------- named devices

def relaxation_64x100(n_polarise: int = 5000, n_total: int = 10000) -> Workload:
    """Plain single device: 64 rails x 100 sites, 800 ions placed uniformly
    at random (seed 0), Ea = 0.40 eV, nu = 1e12 Hz, T = 300 K, d = 1 nm,
    dt = 1e-9 s, 1 V for 5,000 steps then 0 V for 5,000 steps, blocking."""
    dev = Device(R=64, L=100, Z=10, electrodes=0, seed=0)
    return Workload("relaxation_64x100", dev,
                    relaxation_protocol(n_polarise, 1.0, n_total, 0.0),
                    init_mode=0, n_ions=800)


def hysteresis_65536x1024(R: int = 65536, L: int = 1024, steps_per_cycle: int = 100000,
                          cycles: int = 2, seed: int = 1, with_barriers: bool = True,
                          rail_base: int = 0) -> Workload:
    """Plain large device: 65,536 rails x 1,024 sites, 25 % filling,
    Ea per site ~ N(0.40, 0.02) eV, T = 300 K, triangular sweep +-2 V at
    1e5 steps per cycle for 2 cycles, injecting/extracting electrodes with
    rate 1e9 Hz (reservoir density = the initial filling).  With rail_base,
    rails [rail_base, rail_base + R) of a larger device of the same recipe."""
    dev = Device(R=R, L=L, Z=10, electrodes=1, k_e=1e9, rho_e=0.25, seed=seed,
                 rail_base=rail_base)
    Ea = (normal_barriers(R, L, 0.40, 0.02, seed + 1000, row0=rail_base)
          if with_barriers else None)
    return Workload("hysteresis_%dx%d" % (R, L), dev,
                    triangle_protocol(2.0, steps_per_cycle, cycles),
                    init_mode=1, fill=0.25, Ea_site=Ea)


def stdp_batch(n_inst: int = 512, seed: int = 7, n_steps: Optional[int] = None,
               steps_per_ms: int = 2000):
    """Batched devices: rails log-uniform in [256, 16,384], sites log-uniform
    in [128, 2,048], filling U(0.05, 0.4), each with a spike-pair protocol of
    1 V, 1 ms pulses and pre-post delay U(-50, 50) ms at 2,000 steps per ms.
    Returns (devices, voltage tables, fills, delays_ms); n_steps truncates the
    tables (for timing a bounded window)."""
    rng = np.random.default_rng(seed)
    devs, Vs, fills, delays = [], [], [], []
    for i in range(n_inst):
        R = int(round(np.exp(rng.uniform(np.log(256), np.log(16384)))))
        L = int(round(np.exp(rng.uniform(np.log(128), np.log(2048)))))
        fill = float(rng.uniform(0.05, 0.4))
        d = float(rng.uniform(-50.0, 50.0))
        V = spike_pair_protocol(d, steps_per_ms)
        if n_steps is not None:
            V = V[:n_steps]
        devs.append(Device(R=R, L=L, Z=10, electrodes=0, dt=1e-3 / steps_per_ms, seed=seed,
                           instance=i))
        Vs.append(V)
        fills.append(fill)
        delays.append(d)
    return devs, Vs, fills, delays


def adjoint_relaxation(replicas: int = 256, rails: int = 4096, L: int = 512, fill: float = 0.2,
                       n_write: int = 10000, n_relax: int = 50000, V_write: float = 1.0,
                       seed: int = 13, instance: int = 0) -> Workload:
    """Write pulse and relaxation on independent replicas of a 4,096-rail x
    512-site device, 20 % Bernoulli filling, Ea = 0.40 eV, dt = 5e-7 s
    (2,000 steps per ms), blocking electrodes: V_write for n_write steps, then
    0 V for n_relax steps.  Rails are independent, so the replicas are laid end
    to end as one device of replicas x rails rails (rail index r of replica q
    is q * rails + r; every rail has its own Philox counters)."""
    dev = Device(R=replicas * rails, L=L, Z=10, electrodes=0, dt=5e-7, seed=seed,
                 instance=instance)
    return Workload("adjoint_relaxation_%dx%dx%d" % (replicas, rails, L), dev,
                    relaxation_protocol(n_write, V_write, n_write + n_relax, 0.0),
                    init_mode=1, fill=fill)


def potentiation_protocol(n_pulses: int, forget_steps: int, V_pulse: float = 0.8,
                          pulse_ms: float = 0.5, gap_ms: float = 0.5,
                          steps_per_ms: int = 2000) -> np.ndarray:
    """Learning then forgetting: n_pulses pulses of V_pulse lasting pulse_ms,
    each followed by gap_ms at 0 V, then forget_steps steps at 0 V."""
    on = int(round(pulse_ms * steps_per_ms))
    off = int(round(gap_ms * steps_per_ms))
    period = np.concatenate([np.full(on, float(V_pulse)), np.zeros(off)])
    return np.concatenate([np.tile(period, n_pulses), np.zeros(forget_steps)])


def fit_batch(n_dev: int = 256, seed: int = 11, n_pulses: int = 100, forget_steps: int = 100000,
              steps_per_ms: int = 2000, sample_every: int = 500):
    """Devices of the material fit: rails log-uniform in [2,048, 8,192], sites
    log-uniform in [256, 1,024], filling U(0.1, 0.3), Ea = 0.40 eV, coupling 1,
    blocking electrodes, dt = 1 ms / steps_per_ms, all driven by the same
    potentiation protocol (n_pulses pulses of 0.8 V, 0.5 ms, 0.5 ms apart,
    then forget_steps steps at 0 V).  Returns (devices, V, fills, sample_steps):
    the learning/forgetting curve is sampled every sample_every steps."""
    rng = np.random.default_rng(seed)
    V = potentiation_protocol(n_pulses, forget_steps, steps_per_ms=steps_per_ms)
    devs, fills = [], []
    for i in range(n_dev):
        R = int(round(np.exp(rng.uniform(np.log(2048), np.log(8192)))))
        L = int(round(np.exp(rng.uniform(np.log(256), np.log(1024)))))
        fills.append(float(rng.uniform(0.1, 0.3)))
        devs.append(Device(R=R, L=L, Z=10, electrodes=0, dt=1e-3 / steps_per_ms, seed=seed,
                           instance=i))
    sample_steps = np.arange(sample_every - 1, len(V), sample_every, dtype=np.int64)
    return devs, V, fills, sample_steps
