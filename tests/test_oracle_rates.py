"""Pins of the oracle's rate, probability, zone and field functions against
values the paper prints, closed forms evaluated in 50-digit arithmetic
(mpmath), exact rational arithmetic, and physical invariants (Gauss law,
Dirichlet constraint, mirror symmetry, sign of the space-charge push)."""
import math
import os
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

import oracle

mp.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                name, val, _cite = line.split()
                out[name] = float(val)
    return out


def _dev(**kw):
    d = dict(R=1, L=100, Z=10, electrodes=0, d=1.0, dt=1e-9, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=0, instance=0)
    d.update(kw)
    return d


# ------------------------------------------------------------------ Eq. 1

def test_gamma0_barrier_zero_is_attempt_frequency():
    assert oracle.gamma0(3.7e12, 0.0, 300.0) == 3.7e12


def test_gamma0_uses_printed_boltzmann_constant():
    # Ea = k_B T with the k_B printed under Eq. 4 gives exactly nu / e;
    # the CODATA value 8.617333e-5 would miss by 3.9e-6 relative.
    kB = _golden()["k_B_eV_per_K"]
    for T in (250.0, 300.0, 400.0):
        g = oracle.gamma0(1e12, kB * T, T)
        assert g == pytest.approx(1e12 / math.e, rel=1e-14)


@pytest.mark.parametrize("Ea,T,nu", [(0.40, 300.0, 1e12), (0.42, 300.0, 1e12),
                                      (0.30, 350.0, 5e11), (0.55, 280.0, 2e13)])
def test_gamma0_closed_form_50_digits(Ea, T, nu):
    x = mp.mpf(Ea) / (mp.mpf("8.6173e-5") * mp.mpf(T))
    exact = mp.mpf(nu) * mp.exp(-x)
    # FP64 rounding of the exponent x costs |x| ulps of relative error in exp(-x)
    tol = (float(x) + 4.0) * 2.0 ** -52
    assert oracle.gamma0(nu, Ea, T) == pytest.approx(float(exact), rel=tol)


def test_gamma0_reference_value():
    # Eq. 1 at Ea = 0.40 eV, T = 300 K, nu = 1e12 Hz
    assert oracle.gamma0(1e12, 0.40, 300.0) == pytest.approx(1.906645e5, rel=1e-6)


def test_arrhenius_slope():
    # d ln Gamma / d(1/T) = -Ea / k_B  (Eq. 1), by a centred difference
    Ea, T, h = 0.40, 300.0, 1e-3
    lo = math.log(oracle.gamma0(1e12, Ea, T + h))
    hi = math.log(oracle.gamma0(1e12, Ea, T - h))
    slope = (hi - lo) / (1.0 / (T - h) - 1.0 / (T + h))
    assert slope == pytest.approx(-Ea / 8.6173e-5, rel=1e-6)


# ------------------------------------------------------------- P0 reading

def test_p0_closed_form_and_limits():
    # P0 = 1 - exp(-2 Gamma0 dt)
    for dt in (1e-12, 1e-9, 5e-7, 1e-5, 1e-3):
        g = mp.mpf(oracle.gamma0(1e12, 0.40, 300.0))
        exact = 1 - mp.exp(-2 * g * mp.mpf(dt))
        assert oracle.p0(1e12, 0.40, 300.0, dt) == pytest.approx(float(exact), rel=1e-15)
    # small-step limit: P0 ~ 2 Gamma0 dt
    g = oracle.gamma0(1e12, 0.40, 300.0)
    assert oracle.p0(1e12, 0.40, 300.0, 1e-15) == pytest.approx(2 * g * 1e-15, rel=1e-9)
    # 2 Gamma0 dt = ln 2  =>  P0 = 1/2
    dt = math.log(2.0) / (2.0 * g)
    assert oracle.p0(1e12, 0.40, 300.0, dt) == pytest.approx(0.5, rel=1e-15)


def test_p0_table_per_site():
    dev = _dev(R=2, L=3)
    Ea = np.array([[0.38, 0.40, 0.42], [0.41, 0.39, 0.40]])
    tab = oracle.p0_table(dev, Ea)
    for r in range(2):
        for k in range(3):
            assert tab[r, k] == oracle.p0(1e12, Ea[r, k], 300.0, 1e-9)
    assert tab[0, 0] > tab[0, 1] > tab[0, 2]   # higher barrier, slower hopping


# ------------------------------------------------------------ Eqs. 3 - 6

def test_energy_gap_eq3_and_boltzmann_eq4():
    # 1 V across a 100-site rail of 1 nm spacing: dE = 1 e * 1 V * 1 nm / 100 nm = 0.01 eV
    dev = _dev(L=100, Z=10)
    N0 = 30
    Nz = np.full(10, 3)         # background density exactly: no space charge
    dV, B, inv = oracle.zone_field(dev, Nz, N0, 1.0)
    assert np.all(dV == 1.0)
    kT = 8.6173e-5 * 300.0
    dE = -kT * np.log(B)
    assert np.allclose(dE, 0.01, rtol=1e-13, atol=0)
    assert B[0] == pytest.approx(float(mp.exp(mp.mpf("-0.01") / (mp.mpf("8.6173e-5") * 300))),
                                 rel=1e-15)
    assert B[0] == pytest.approx(0.679214, rel=1e-6)
    assert np.allclose(inv * (1.0 + B), 1.0, rtol=2e-16, atol=0)


def test_hop_probabilities_eqs_5_6():
    for base in (1e-6, 3.8e-4, 0.3, 1.0):
        for B in (1e-3, 0.679214, 1.0, 1.47, 50.0):
            inv = 1.0 / (1.0 + B)
            pl, pr = oracle.hop_probs(base, B, inv)
            assert pr / pl == pytest.approx(B, rel=4e-16)          # Eq. 6
            assert pl + pr == pytest.approx(base, rel=4e-16)       # normalisation
            assert pl == pytest.approx(base / (1.0 + B), rel=4e-16)  # Eq. 5
    # zero bias: forward and backward equal (detailed balance, Sec. 3)
    pl, pr = oracle.hop_probs(0.37, 1.0, 0.5)
    assert pl == pr == 0.185


def test_positive_bias_drives_cations_toward_site_0():
    # decile 1 (site 0 side) is the active decile at V > 0 (Fig. 2 caption)
    dev = _dev()
    dV, B, inv = oracle.zone_field(dev, np.full(10, 3), 30, 2.0)
    pl, pr = oracle.hop_probs(0.1, B[4], inv[4])
    assert pl > pr
    dV, B, inv = oracle.zone_field(dev, np.full(10, 3), 30, -2.0)
    pl, pr = oracle.hop_probs(0.1, B[4], inv[4])
    assert pl < pr


# ------------------------------------------------------------------ zones

def test_zone_index_matches_paper_formula_exactly():
    # z = ceil(X / (L_x / Z)) with X = k + 1 (1-based), in exact rationals
    for L in list(range(2, 80)) + [100, 127, 128, 1000, 1024, 2047, 2048]:
        for Z in range(1, min(L, 32) + 1):
            for k in range(L):
                paper = math.ceil(Fraction(k + 1) / Fraction(L, Z)) - 1
                assert oracle.zone_of(k, L, Z) == paper


def test_zone_widths_equal_up_to_one():
    for L in (100, 101, 1024, 37, 2048):
        for Z in (1, 3, 10, 16, 32):
            if Z > L:
                continue
            w = oracle.zone_widths(L, Z)
            assert w.sum() == L
            assert w.max() - w.min() <= 1
    assert list(oracle.zone_widths(100, 10)) == [10] * 10


# ---------------------------------------------------- space-charge field

def _random_counts(rng, L, Z, fill):
    occ = rng.random(L) < fill
    z = np.array([oracle.zone_of(k, L, Z) for k in range(L)])
    return np.bincount(z[occ], minlength=Z), int(occ.sum())


def test_field_uniform_background_is_applied_bias():
    dev = _dev(L=100, Z=10)
    for V in (-3.0, 0.0, 1.0, 7.5):
        dV, _, _ = oracle.zone_field(dev, np.full(10, 4), 40, V)
        assert np.all(dV == V)


def test_field_no_coupling_is_applied_bias():
    rng = np.random.default_rng(1)
    dev = _dev(L=100, Z=10, kappa=0.0)
    Nz, _ = _random_counts(rng, 100, 10, 0.3)
    dV, _, _ = oracle.zone_field(dev, Nz, 30, 1.25)
    assert np.all(dV == 1.25)


@pytest.mark.parametrize("L,Z", [(100, 10), (103, 10), (1024, 10), (37, 5), (64, 16)])
def test_field_dirichlet_and_discrete_gauss_law(L, Z):
    rng = np.random.default_rng(L * 100 + Z)
    dev = _dev(L=L, Z=Z, alpha=0.2, kappa=0.9)
    w = oracle.zone_widths(L, Z)
    for trial in range(20):
        Nz, N = _random_counts(rng, L, Z, rng.uniform(0.05, 0.6))
        N0 = int(rng.integers(0, L // 2 + 1))
        V = float(rng.uniform(-5, 5))
        dV, _, _ = oracle.zone_field(dev, Nz, N0, V)
        C = Nz - N0 * w / L
        scale = 0.18 * (np.abs(C).sum() + 1.0)
        # the potential drop over the whole rail is the applied bias (Dirichlet, S1.4)
        assert np.dot(w, dV) / L == pytest.approx(V, abs=1e-12 * (abs(V) + scale))
        # the field changes between zone centres by the enclosed charge (Gauss)
        jump = dV[1:] - dV[:-1]
        assert np.allclose(jump, -0.18 * (C[1:] + C[:-1]) / 2.0, rtol=0, atol=1e-12 * scale)


def test_field_pile_pushes_neighbours_away():
    # ions piled in zone 0 at zero bias: the field in zone 1 pushes ions to the
    # right, away from the pile (repulsion lowers drift into dense regions, Sec. 3)
    dev = _dev(L=100, Z=10)
    Nz = np.array([10, 2, 2, 2, 2, 2, 2, 2, 2, 2])
    dV, B, inv = oracle.zone_field(dev, Nz, 28, 0.0)
    assert dV[1] < 0.0 and B[1] > 1.0
    pl, pr = oracle.hop_probs(0.1, B[1], inv[1])
    assert pr > pl
    # the mirror image pushes to the left
    dV2, _, _ = oracle.zone_field(dev, Nz[::-1].copy(), 28, 0.0)
    assert dV2[8] > 0.0


def test_field_mirror_symmetry():
    rng = np.random.default_rng(7)
    dev = _dev(L=100, Z=10)
    for _ in range(10):
        Nz, N = _random_counts(rng, 100, 10, 0.3)
        V = float(rng.uniform(-3, 3))
        dV, _, _ = oracle.zone_field(dev, Nz, N, V)
        dVm, _, _ = oracle.zone_field(dev, Nz[::-1].copy(), N, -V)
        assert np.allclose(dVm[::-1], -dV, rtol=0, atol=1e-12)
