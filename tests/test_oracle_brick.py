"""Pins of the oracle's brick-wall (even/odd bond) variant against its
brute-force master equation (tests/master_eq.py, written separately):

* the exact chain is flat at zero bias without space charge: the stationary
  law of two steps (one even, one odd) is uniform over the configurations of
  a given ion count, so every site has the same occupancy (the synchronous
  rule is not: its walls are depleted by O(p));
* the oracle's k-step distribution from a fixed start agrees with the exact
  chain (chi-square over all 2^6 configurations), with blocking and open
  electrodes and with space charge;
* the same test rejects the synchronous rule's chain (the pin has power);
* blocking electrodes conserve the ion count, and J is the position sum's loss.
"""
import numpy as np
import pytest

import oracle
from tests import master_eq as me
from tests.test_oracle_dynamics import _chi2_pvalue


def _dev(**kw):
    d = dict(R=1, L=6, Z=3, electrodes=0, d=1.0, dt=1e-6, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=2024, instance=0, rule=1)
    d.update(kw)
    return d


def _stationary(M):
    w, v = np.linalg.eig(M.T)
    pi = np.real(v[:, int(np.argmin(np.abs(w - 1.0)))])
    return pi / pi.sum()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_exact_chain_is_flat_at_zero_bias(N):
    dev = _dev(alpha=0.0)
    L = dev["L"]
    pops = np.array([bin(s).count("1") for s in range(1 << L)])
    idx = np.where(pops == N)[0]
    M = me.transition_matrix_brick(dev, 0.0, N, 0) @ me.transition_matrix_brick(dev, 0.0, N, 1)
    pi = _stationary(M[np.ix_(idx, idx)])
    assert np.abs(pi - 1.0 / len(idx)).max() < 1e-12
    bits = np.array([[(s >> k) & 1 for k in range(L)] for s in idx], dtype=float)
    np.testing.assert_allclose(bits.T @ pi, N / L, atol=1e-12)
    # the synchronous rule on the same rail is not flat
    sync = _stationary(me.transition_matrix(dev, 0.0, N)[np.ix_(idx, idx)])
    assert np.abs(bits.T @ sync - N / L).max() > 1e-3


CASES = {
    "blocking": dict(electrodes=0),
    "open": dict(electrodes=1, k_e=2e5, rho_e=0.4),
    "open_strong_field": dict(electrodes=1, k_e=5e5, rho_e=0.7, alpha=0.5),
}


def _distribution_after(dev, start, k, V):
    p = np.zeros(1 << dev["L"])
    p[me.state_index(start)] = 1.0
    for t in range(k):
        p = p @ me.transition_matrix_brick(dev, V, sum(start), t % 2)
    return p


def _oracle_states(dev, start, k, V):
    occ0 = np.tile(np.asarray(start, dtype=np.uint8), (dev["R"], 1))
    sim = oracle.OracleSim(dev, np.full(k, float(V)), occ0)
    sim.step_n(k)
    return np.array([me.state_index(row) for row in sim.occ])


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("k", [1, 2, 5])
def test_k_step_distribution_matches_master_equation(case, k):
    dev = _dev(R=120000, **CASES[case])
    start = [1, 0, 1, 1, 0, 1]
    p = _distribution_after(dev, start, k, 0.3)
    counts = np.bincount(_oracle_states(dev, start, k, 0.3), minlength=64).astype(float)
    pval, chi2, dof = _chi2_pvalue(counts, p)
    assert pval > 1e-5, (case, k, chi2, dof)


def test_master_equation_rejects_the_synchronous_chain():
    dev = _dev(R=60000)
    start = [1, 0, 1, 1, 0, 1]
    counts = np.bincount(_oracle_states(dev, start, 3, 0.3), minlength=64).astype(float)
    p = np.zeros(64)
    p[me.state_index(start)] = 1.0
    T = me.transition_matrix(dev, 0.3, N0=sum(start))
    p = p @ T @ T @ T
    # states the synchronous chain cannot reach get a tiny expectation, not zero
    pval, _, _ = _chi2_pvalue(counts, np.maximum(p, 1e-300))
    assert pval < 1e-10


def test_conservation_and_current_with_blocking_electrodes():
    dev = _dev(R=300, L=40, Z=5, alpha=0.4)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.35)
    V = np.concatenate([np.full(150, 2.0), np.full(150, -1.0)])
    sim = oracle.OracleSim(dev, V, occ0)
    pos = np.arange(40)
    X0 = (occ0 * pos).sum()
    J, Zc = sim.step_n(300)
    assert np.array_equal(sim.occ.sum(axis=1), occ0.sum(axis=1))
    assert np.all(Zc.sum(axis=1) == occ0.sum())
    # each leftward crossing lowers the position sum by one, each rightward raises it
    assert J.sum() == X0 - (sim.occ * pos).sum()
