"""Pins of the oracle's likelihood-ratio gradient (orc_run_lr), independent of
the oracle's own arithmetic:

* the analytic per-trial score equals the derivative of the trajectory's
  log-probability, taken by central differences of the log-probability of the
  same trial outcomes re-evaluated at shifted parameters (a dropped term, a
  wrong sign or a wrong chain-rule factor in d ln p / d theta fails here);
* the estimator is unbiased: on a 1-rail x 6-site chain its mean over many
  independent rails agrees, within its own standard error, with the exact
  gradient of the observable's expectation, obtained by differencing the
  brute-force master equation (every configuration and every joint trial
  outcome enumerated; no sampling);
* the replay that accumulates the score reproduces the plain run's trajectory.
"""
import numpy as np
import pytest

from tests import master_eq as M
import oracle
from paper_2511_09413_gb300 import workloads as W

NAMES = ["Ea", "nu", "kappa"]


def _dev(**kw):
    d = dict(R=6, L=12, Z=3, electrodes=0, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.5, kappa=1.0, k_e=0.0, rho_e=0.0, seed=5, instance=0)
    d.update(kw)
    return d


@pytest.mark.parametrize("electrodes", [0, 1])
def test_score_is_derivative_of_log_probability(electrodes):
    dev = _dev(electrodes=electrodes, k_e=3e5 if electrodes else 0.0,
               rho_e=0.3 if electrodes else 0.0)
    occ0 = W.random_occupancy(6, 12, 0.4, seed=2)
    V = W.triangle_protocol(0.5, 60, 4)
    n = 200
    base = oracle.lr_gradient(dev, V, occ0, n)
    S = base["S"]
    assert np.array_equal(base["J"], base["J_tot"]), "replay differs from the plain run"
    assert np.all(np.abs(S[:, 0]) > 0) and np.all(np.abs(S[:, 2]) > 0)
    for i, nm in enumerate(NAMES):
        h = 1e-5 * abs(dev[nm])
        dp, dm = dict(dev), dict(dev)
        dp[nm] += h
        dm[nm] -= h
        lp = oracle.lr_gradient(dev, V, occ0, n, dev_eval=dp)["loglik"]
        lm = oracle.lr_gradient(dev, V, occ0, n, dev_eval=dm)["loglik"]
        fd = (lp - lm) / (2.0 * h)
        np.testing.assert_allclose(S[:, i], fd, rtol=2e-5, atol=1e-8 * np.abs(S[:, i]).max(),
                                   err_msg=nm)


def test_rho_score_is_derivative_of_initial_log_probability():
    occ0 = W.random_occupancy(50, 40, 0.3, seed=9)
    rho, h = 0.3, 1e-6
    n = occ0.sum(axis=1)

    def ll(r):
        return n * np.log(r) + (40 - n) * np.log1p(-r)

    fd = (ll(rho + h) - ll(rho - h)) / (2 * h)
    np.testing.assert_allclose(oracle.init_score_rho(occ0, rho), fd, rtol=1e-7)


def _exact_F(dev, V, wJ, wZ, fill):
    """E[F] from the master equation, Bernoulli(fill) initial placement."""
    L, Z = dev["L"], dev["Z"]
    n_states = 1 << L
    pops = np.array([bin(s).count("1") for s in range(n_states)])
    zones = [M.zone_index(k, L, Z) for k in range(L)]
    Nz = np.array([[sum((s >> k) & 1 for k in range(L) if zones[k] == z) for z in range(Z)]
                   for s in range(n_states)], dtype=np.float64)
    pi0 = fill ** pops * (1.0 - fill) ** (L - pops)
    F = 0.0
    for N0 in range(L + 1):
        mats = {v: M.transition_matrix(dev, v, N0, with_current=True) for v in sorted(set(V))}
        pi = np.where(pops == N0, pi0, 0.0)
        for t in range(len(V)):
            T, Jm = mats[V[t]]
            F += pi @ (Nz @ wZ[t])          # zone counts at the start of step t
            F += wJ[t] * (pi @ Jm)          # current of step t
            pi = pi @ T
    return F


@pytest.mark.parametrize("electrodes,observable,nR,k_e,Vw", [
    (0, "current", 30, 0.0, 0.3), (0, "zone", 10, 0.0, 0.3), (1, "current", 5, 1e6, 0.5)])
def test_lr_gradient_matches_master_equation(electrodes, observable, nR, k_e, Vw):
    """Write pulse then relaxation on a 1 x 6 chain; F = mean relaxation
    current, or mean zone-0 count, per rail."""
    dev = _dev(R=1, L=6, Z=3, dt=1e-6, alpha=0.3, seed=11, electrodes=electrodes,
               k_e=k_e, rho_e=0.35 if electrodes else 0.0)
    fill = 0.4
    nW = 15
    V = np.concatenate([np.full(nW, Vw), np.zeros(nR)])
    n = len(V)
    wJ = np.zeros(n)
    wZ = np.zeros((n, dev["Z"]))
    if observable == "current":
        wJ[nW:] = 1.0 / nR
    else:
        wZ[nW:, 0] = 1.0 / nR
    exact = []
    for nm in NAMES:
        h = 1e-5 * dev[nm]
        dp, dm = dict(dev), dict(dev)
        dp[nm] += h
        dm[nm] -= h
        exact.append((_exact_F(dp, V, wJ, wZ, fill) - _exact_F(dm, V, wJ, wZ, fill)) / (2 * h))
    h = 1e-5
    exact.append((_exact_F(dev, V, wJ, wZ, fill + h) - _exact_F(dev, V, wJ, wZ, fill - h)) / (2 * h))
    exact = np.array(exact)

    R = 100000
    d2 = dict(dev, R=R)
    occ0 = oracle.init_occupancy(d2, 1, fill=fill)
    r = oracle.lr_gradient(d2, V, occ0, n, wJ=wJ / R if observable == "current" else None,
                           wZ=wZ / R if observable == "zone" else None, fill=fill, cv_windows=5)
    z = (r["grad"] - exact) / r["stderr"]
    assert np.all(np.abs(z) < 4.0), (r["grad"], r["stderr"], exact)
    # the comparison has power: every component is resolved to better than 35 %
    assert np.all(r["stderr"] < 0.35 * np.abs(exact)), (r["stderr"], exact)
    # the cross-fitted state-dependent control variate keeps the estimator unbiased
    z_cv = (r["grad_cv"] - exact) / r["stderr_cv"]
    assert np.all(np.abs(z_cv) < 4.0), (r["grad_cv"], r["stderr_cv"], exact)


def test_control_variate_features_have_zero_mean():
    """Every feature sum of the control variate (a score increment times a
    step-start feature) averages to zero over independent rails."""
    dev = _dev(R=20000, L=16, Z=4, electrodes=1, k_e=2e5, rho_e=0.3, dt=1e-6)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    V = W.triangle_protocol(0.4, 40, 2)
    r = oracle.lr_gradient(dev, V, occ0, len(V), fill=0.3, cv_windows=4)
    A = r["cv"].reshape(dev["R"], -1)
    m = A.mean(axis=0)
    se = A.std(axis=0, ddof=1) / np.sqrt(A.shape[0])
    ok = se > 0
    assert ok.sum() > 0.9 * A.shape[1]
    assert np.all(np.abs(m[ok]) < 4.5 * se[ok]), np.abs(m[ok] / se[ok]).max()


def test_control_variate_reduces_the_standard_error():
    """Write pulse and relaxation on 4,096 rails x 64 sites, F = mean
    relaxation current: the cross-fitted control variate over 10 time windows
    cuts the standard error of the Ea, nu and kappa entries by more than a
    third, and moves each estimate by less than the combined errors."""
    R, nw, nr = 4096, 200, 800
    dev = _dev(R=R, L=64, Z=8, dt=5e-7, alpha=0.2, seed=17)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.2)
    V = np.concatenate([np.full(nw, 1.0), np.zeros(nr)])
    w = np.zeros(nw + nr)
    w[nw:] = 1.0 / (nr * R)
    r = oracle.lr_gradient(dev, V, occ0, nw + nr, wJ=w, fill=0.2, cv_windows=10)
    gain = r["stderr"][:3] / r["stderr_cv"][:3]
    assert np.all(gain > 1.35), gain
    assert np.all(np.abs(r["grad_cv"][:3] - r["grad"][:3]) < 3.0 * r["stderr"][:3])
    assert r["grad_cv"][3] == r["grad"][3]          # no features for the filling


def test_score_has_zero_mean():
    """E[d log p] = 0: the cumulative score over many independent rails
    averages to zero within its standard error."""
    dev = _dev(R=20000, L=16, Z=4, electrodes=1, k_e=2e5, rho_e=0.3, dt=1e-6)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    V = W.triangle_protocol(0.4, 40, 2)
    r = oracle.lr_gradient(dev, V, occ0, len(V), fill=0.3)
    S = r["S"]
    m = S.mean(axis=0)
    se = S.std(axis=0, ddof=1) / np.sqrt(S.shape[0])
    assert np.all(np.abs(m) < 4.0 * se), (m, se)
