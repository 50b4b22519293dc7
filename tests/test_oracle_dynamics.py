"""Pins of the oracle's synchronous update rule (S2.1.6 - S2.1.7) against the
brute-force master equation of a short rail, single-ion closed forms,
conservation laws and exact identities.

Every rail of an oracle run draws from its own Philox stream (the rail index is
a counter word), so R rails started from the same configuration are R
independent samples of the chain."""
import numpy as np
import pytest
from scipy import stats

import oracle
from tests import master_eq as me


def _dev(**kw):
    d = dict(R=1, L=6, Z=3, electrodes=0, d=1.0, dt=1e-6, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=12345, instance=0)
    d.update(kw)
    return d


def _run_from(dev, start_row, n_steps, V, Ea_site=None):
    R, L = dev["R"], dev["L"]
    occ0 = np.tile(np.asarray(start_row, dtype=np.uint8), (R, 1))
    Vtab = np.full(n_steps, float(V))
    Ea = None if Ea_site is None else np.tile(np.asarray(Ea_site, dtype=np.float64), (R, 1))
    sim = oracle.OracleSim(dev, Vtab, occ0, Ea)
    J, Zc = sim.step_n(n_steps)
    return sim, J, Zc


def _chi2_pvalue(counts, probs):
    n = counts.sum()
    expct = probs * n
    # pool bins with small expectation into one
    small = expct < 5
    obs = list(counts[~small])
    exp_ = list(expct[~small])
    if small.any():
        obs.append(counts[small].sum())
        exp_.append(expct[small].sum())
    obs, exp_ = np.array(obs, dtype=float), np.array(exp_, dtype=float)
    keep = exp_ > 0
    assert obs[~keep].sum() == 0, "oracle reached a state the exact chain forbids"
    chi2 = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    dof = max(1, keep.sum() - 1)
    return stats.chi2.sf(chi2, dof), chi2, dof


CASES = {
    "blocking": dict(electrodes=0),
    "open": dict(electrodes=1, k_e=2e5, rho_e=0.4),
    "open_strong_field": dict(electrodes=1, k_e=5e5, rho_e=0.7, alpha=0.5),
    "blocking_no_coupling": dict(electrodes=0, kappa=0.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("k", [1, 4])
def test_k_step_distribution_matches_master_equation(case, k):
    dev = _dev(R=120000, **CASES[case])
    start = [1, 0, 1, 1, 0, 0]
    V = 0.3
    sim, _, _ = _run_from(dev, start, k, V)
    T = me.transition_matrix(dev, V, N0=sum(start))
    p = np.zeros(1 << dev["L"])
    p[me.state_index(start)] = 1.0
    for _ in range(k):
        p = p @ T
    idx = np.array([me.state_index(row) for row in sim.occ])
    counts = np.bincount(idx, minlength=1 << dev["L"]).astype(float)
    pval, chi2, dof = _chi2_pvalue(counts, p)
    assert pval > 1e-5, (case, k, chi2, dof)


def test_per_site_barriers_match_master_equation():
    # a barrier per site acts on hops leaving that site
    dev = _dev(R=120000, electrodes=1, k_e=2e5, rho_e=0.3)
    Ea = [0.38, 0.41, 0.40, 0.37, 0.43, 0.39]
    start = [0, 1, 1, 0, 1, 0]
    V = -0.2
    sim, _, _ = _run_from(dev, start, 2, V, Ea_site=Ea)
    T = me.transition_matrix(dev, V, N0=sum(start), Ea_site=Ea)
    p = np.zeros(64)
    p[me.state_index(start)] = 1.0
    p = p @ T @ T
    counts = np.bincount([me.state_index(r) for r in sim.occ], minlength=64).astype(float)
    pval, chi2, dof = _chi2_pvalue(counts, p)
    assert pval > 1e-5, (chi2, dof)


def test_master_equation_rejects_a_wrong_rule():
    # sanity of the pin itself: a chain with conflicting hops *not* cancelled
    # (first come first served is impossible synchronously, so emulate a plain
    # sign flip of the bias) must be rejected by the same test
    dev = _dev(R=60000)
    start = [1, 0, 1, 1, 0, 0]
    sim, _, _ = _run_from(dev, start, 3, 0.3)
    T_wrong = me.transition_matrix(dev, -0.3, N0=3)
    p = np.zeros(64)
    p[me.state_index(start)] = 1.0
    for _ in range(3):
        p = p @ T_wrong
    counts = np.bincount([me.state_index(r) for r in sim.occ], minlength=64).astype(float)
    pval, _, _ = _chi2_pvalue(counts, p)
    assert pval < 1e-10


def test_single_ion_step_closed_form():
    # one ion far from the walls, no space-charge coupling: the two trials are
    # independent, so P(+1) = pR (1 - pL), P(-1) = pL (1 - pR)  (S2.1.7)
    dev = _dev(R=400000, L=5, Z=5, kappa=0.0)
    V = 0.5
    sim, _, _ = _run_from(dev, [0, 0, 1, 0, 0], 1, V)
    pos = np.argmax(sim.occ, axis=1)
    _, B, inv = oracle.zone_field(dev, np.array([0, 0, 1, 0, 0]), 1, V)
    pl, pr = oracle.hop_probs(oracle.p0(1e12, 0.40, 300.0, 1e-6), B[2], inv[2])
    n = dev["R"]
    for site, prob in ((3, pr * (1 - pl)), (1, pl * (1 - pr)), (2, 1 - pr * (1 - pl) - pl * (1 - pr))):
        obs = np.count_nonzero(pos == site)
        sd = np.sqrt(n * prob * (1 - prob))
        assert abs(obs - n * prob) < 4.5 * sd, (site, obs, n * prob)
    # net current: J_rail = -(displacement)
    assert np.array_equal(sim.J_rail, -(pos - 2))


def test_single_ion_next_to_blocking_wall_stationary():
    # single ion, three sites, zero bias: pi_0 / pi_1 = 1 - p  (from the exact chain)
    dev = _dev(R=200000, L=3, Z=3, kappa=0.0)
    sim, _, _ = _run_from(dev, [0, 1, 0], 60, 0.0)
    p = oracle.p0(1e12, 0.40, 300.0, 1e-6) / 2.0
    pi = np.array([1 - p, 1.0, 1 - p]) / (3 - 2 * p)
    pos = np.argmax(sim.occ, axis=1)
    counts = np.bincount(pos, minlength=3)
    pval, chi2, dof = _chi2_pvalue(counts.astype(float), pi)
    assert pval > 1e-5, (counts, pi * dev["R"])


def test_zero_bias_profile_matches_exact_stationary_state():
    # zero bias, blocking, space charge on: long-run site occupation equals the
    # exact chain's stationary law (nearly flat; the walls perturb it at O(p))
    dev = _dev(R=40000, L=6, Z=3)
    start = [1, 1, 0, 0, 0, 0]
    sim, _, _ = _run_from(dev, start, 150, 0.0)
    T = me.transition_matrix(dev, 0.0, N0=2)
    p = np.zeros(64)
    p[me.state_index(start)] = 1.0
    for _ in range(150):
        p = p @ T
    counts = np.bincount([me.state_index(r) for r in sim.occ], minlength=64).astype(float)
    pval, chi2, dof = _chi2_pvalue(counts, p)
    assert pval > 1e-5, (chi2, dof)
    # the stationary law itself: mirror symmetric, flat up to O(p) at the walls
    pi = np.linalg.matrix_power(T, 4096)[me.state_index(start)]
    dens = np.array([sum(pi[s] for s in range(64) if (s >> k) & 1) for k in range(6)])
    assert np.allclose(dens, dens[::-1], atol=1e-9)
    p_hop = oracle.p0(1e12, 0.40, 300.0, 1e-6) / 2.0
    assert dens.max() - dens.min() < 2.0 * p_hop * dens.mean()
    assert np.allclose(dens[1:5], dens[1:5].mean(), rtol=0.05)


def test_blocking_conserves_ions_and_position_identity():
    rng = np.random.default_rng(3)
    dev = dict(R=32, L=100, Z=10, electrodes=0, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=9, instance=2)
    occ0 = (rng.random((32, 100)) < 0.3).astype(np.uint8)
    V = np.concatenate([np.full(300, 2.0), np.full(300, -1.0)])
    sim = oracle.OracleSim(dev, V, occ0)
    J, Zc = sim.step_n(600)
    assert np.all(Zc.sum(axis=1) == occ0.sum())
    assert np.all(sim.occ.sum(axis=1) == occ0.sum(axis=1))
    k = np.arange(100)
    assert J.sum() == (occ0 * k).sum() - (sim.occ.astype(np.int64) * k).sum()
    assert np.array_equal(sim.J_rail, (occ0 * k).sum(axis=1) - (sim.occ.astype(np.int64) * k).sum(axis=1))


def test_ions_never_pass_each_other():
    """Exclusion against the step-start occupancy and the cancellation of
    conflicting entries (R3, R4) keep the ions' order: step by step, each
    rail's k-th ion (by position) moves by at most one site, and every site
    holds 0 or 1 ion."""
    dev = dict(R=32, L=40, Z=4, electrodes=0, d=1.0, dt=5e-6, T=300.0, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=31, instance=2)
    occ0 = (np.random.default_rng(3).random((32, 40)) < 0.45).astype(np.uint8)
    V = np.concatenate([np.full(100, 2.0), np.full(100, -2.0), np.zeros(100)])
    sim = oracle.OracleSim(dev, V, occ0)
    prev = sim.occ.copy()
    moved = 0
    for _ in range(len(V)):
        sim.step_n(1)
        cur = sim.occ
        assert cur.max() <= 1 and cur.min() >= 0
        for r in range(32):
            a, b = np.flatnonzero(prev[r]), np.flatnonzero(cur[r])
            assert len(a) == len(b)
            assert np.all(np.abs(b - a) <= 1), (r, a, b)
            moved += int(np.count_nonzero(b != a))
        prev = cur.copy()
    assert moved > 1000          # the test sees many moves, not a frozen lattice


def test_resume_is_bit_identical():
    dev = dict(R=16, L=64, Z=8, electrodes=1, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=1.0, k_e=1e6, rho_e=0.25, seed=77, instance=5)
    occ0 = (np.random.default_rng(5).random((16, 64)) < 0.25).astype(np.uint8)
    V = np.linspace(-2, 2, 400)
    a = oracle.OracleSim(dev, V, occ0)
    Ja, Za = a.step_n(400)
    b = oracle.OracleSim(dev, V, occ0)
    Jb1, Zb1 = b.step_n(150)
    Jb2, Zb2 = b.step_n(250)
    assert np.array_equal(a.occ, b.occ)
    assert np.array_equal(Ja, np.concatenate([Jb1, Jb2]))
    assert np.array_equal(Za, np.concatenate([Zb1, Zb2]))


def test_init_modes():
    dev = dict(R=64, L=100, Z=10, electrodes=0, d=1.0, dt=1e-9, T=300.0, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=0, instance=0)
    occ = oracle.init_occupancy(dev, 0, n_ions=800)
    assert occ.sum() == 800 and occ.max() == 1
    # uniform placement: every site equally likely -> per-zone counts ~ 80
    z = np.array([oracle.zone_of(k, 100, 10) for k in range(100)])
    per_zone = np.bincount(np.repeat(z[None, :], 64, 0)[occ == 1], minlength=10)
    assert stats.chisquare(per_zone).pvalue > 1e-4
    occ1 = oracle.init_occupancy(dict(dev, R=256), 1, fill=0.25)
    frac = occ1.mean()
    assert abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / occ1.size)
    assert oracle.init_occupancy(dev, 1, fill=0.0).sum() == 0
    assert oracle.init_occupancy(dev, 1, fill=1.0).sum() == 6400


def test_near_threshold_decisions_are_logged():
    # choose P0 so that p_left = P0 / 2 equals the left draw of site 2 of
    # some rail at step 0 to within rounding: that decision must be logged
    dev = dict(R=1, L=5, Z=1, electrodes=0, d=1.0, dt=1e-6, T=300.0, Ea=0.0, nu=1e12,
               alpha=0.0, kappa=0.0, k_e=0.0, rho_e=0.0, seed=42, instance=0)
    for rail in range(64):
        x = oracle.philox4x32_10([2, rail, 0, 0], [42, 0])
        uL = float(((int(x[3]) << 32) | int(x[2])) >> 11) * 2.0 ** -53
        if 0.05 < uL < 0.45:
            break
    # P0 = 1 - exp(-2 nu dt) with Ea = 0; solve for nu
    dev["nu"] = -np.log1p(-2.0 * uL) / (2.0 * dev["dt"])
    dev["R"] = rail + 1
    occ0 = np.tile(np.array([0, 0, 1, 0, 0], dtype=np.uint8), (rail + 1, 1))
    sim = oracle.OracleSim(dev, np.zeros(1), occ0)
    sim.step_n(1)
    log = sim.near_threshold_log()
    hits = [e for e in log if e["rail"] == rail]
    assert len(hits) == 1
    e = hits[0]
    assert (e["step"], e["site"], e["dir"], e["kind"]) == (0, 2, 1, 0)
    assert abs(e["diff"]) < 1e-12


def test_rail_sample_matches_full_device():
    # a sample of rails advanced on its own (rail index map) equals those rows
    # of the whole device: rails are independent and keyed by their index
    dev = dict(R=20, L=48, Z=6, electrodes=1, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=1.0, k_e=1e6, rho_e=0.25, seed=11, instance=3)
    V = np.linspace(1.5, -1.5, 300)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    ids = np.array([5, 17, 0, 19])
    assert np.array_equal(oracle.init_occupancy(dev, 1, fill=0.3, rail_ids=ids), occ0[ids])
    Ea = 0.40 + 0.02 * np.random.default_rng(2).standard_normal((20, 48))
    full = oracle.OracleSim(dev, V, occ0, Ea)
    full.step_n(300)
    part = oracle.OracleSim(dev, V, occ0[ids], Ea[ids], rail_ids=ids)
    part.step_n(300)
    assert np.array_equal(part.occ, full.occ[ids])
    assert np.array_equal(part.J_rail, full.J_rail[ids])


def _init_keys(dev, rails):
    """64-bit placement keys (R5, R17): Philox4x32-10 block at counter
    (site, rail, 0xFFFFFFFF, instance) under key (seed lo, seed hi), words
    (x1:x0); the generator itself is pinned against cuRAND elsewhere."""
    key = [dev["seed"] & 0xFFFFFFFF, dev["seed"] >> 32]
    out = np.zeros((len(rails), dev["L"]), dtype=np.uint64)
    for i, r in enumerate(rails):
        for k in range(dev["L"]):
            x = oracle.philox4x32_10([k, int(r), 0xFFFFFFFF, dev["instance"]], key)
            out[i, k] = (np.uint64(x[1]) << np.uint64(32)) | np.uint64(x[0])
    return out


def test_placement_is_the_smallest_keys_and_the_bernoulli_rule():
    dev = dict(R=5, L=13, Z=3, electrodes=0, d=1.0, dt=1e-9, T=300.0, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=0x1234_5678_9ABC_DEF1,
               instance=7)
    keys = _init_keys(dev, range(dev["R"]))
    flat = keys.ravel()
    for n in (0, 1, 17, 64, 65):
        want = np.zeros(flat.size, dtype=np.uint8)
        want[np.lexsort((np.arange(flat.size), flat))[:n]] = 1      # by key, ties by index
        assert np.array_equal(oracle.init_occupancy(dev, 0, n_ions=n).ravel(), want)
    for fill in (0.0, 0.3, 0.75, 1.0):
        u = (keys >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        assert np.array_equal(oracle.init_occupancy(dev, 1, fill=fill), (u < fill).astype(np.uint8))
    # a sample of rails (index map) draws the rails' own keys
    ids = np.array([4, 0, 2], dtype=np.int32)
    u = (_init_keys(dev, ids) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    assert np.array_equal(oracle.init_occupancy(dev, 1, fill=0.5, rail_ids=ids),
                          (u < 0.5).astype(np.uint8))


@pytest.mark.parametrize("electrodes", [0, 1])
def test_per_step_trace_definitions(electrodes):
    """Zone counts are those of each step's start occupancy (R16's trace);
    with blocking electrodes the step's current is the drop of the summed
    ion position over that step (each leftward crossing lowers it by one)."""
    rng = np.random.default_rng(11 + electrodes)
    dev = dict(R=12, L=47, Z=5, electrodes=electrodes, d=1.0, dt=5e-7, T=300.0, Ea=0.40,
               nu=1e12, alpha=0.2, kappa=1.0, k_e=2e6 if electrodes else 0.0,
               rho_e=0.3 if electrodes else 0.0, seed=21, instance=3)
    occ = (rng.random((12, 47)) < 0.35).astype(np.uint8)
    V = np.concatenate([np.linspace(0.0, 2.5, 20), np.linspace(2.5, -2.5, 40), np.zeros(20)])
    sim = oracle.OracleSim(dev, V, occ)
    z = np.array([oracle.zone_of(k, 47, 5) for k in range(47)])
    k = np.arange(47)
    moved = 0
    for t in range(len(V)):
        before = sim.occ.copy()
        J, Zc = sim.step_n(1)
        assert np.array_equal(Zc[0], np.bincount(z, weights=before.sum(axis=0), minlength=5))
        if electrodes == 0:
            assert J[0] == (before * k).sum() - (sim.occ.astype(np.int64) * k).sum()
        moved += int(np.any(before != sim.occ))
    assert moved > len(V) // 2


def test_single_ion_follows_its_own_draws_exactly():
    """One ion, no space charge, blocking walls: each step its right trial
    uses u = ((x1:x0) >> 11) 2^-53 and its left trial ((x3:x2) >> 11) 2^-53
    of the Philox block at counter (site, rail, step, instance) (R5, R6); it
    moves right iff only the right trial is accepted, left iff only the left
    one is, and stays if both or neither are (R2); trials into a wall are not
    made (R14).  Checked move by move against the oracle."""
    L, V, T, dt = 6, 0.3, 300.0, 2e-6
    dev = dict(R=1, L=L, Z=2, electrodes=0, d=1.0, dt=dt, T=T, Ea=0.40, nu=1e12,
               alpha=0.2, kappa=0.0, k_e=0.0, rho_e=0.0, seed=0xC0FFEE, instance=9)
    P0 = -np.expm1(-2.0 * 1e12 * np.exp(-0.40 / (8.6173e-5 * T)) * dt)
    B = np.exp(-(V / L) / (8.6173e-5 * T))          # Eqs. 3-4, t_dev = L d
    pL = P0 / (1.0 + B)                              # Eq. 5
    pR = pL * B                                      # Eq. 6
    occ = np.zeros((1, L), dtype=np.uint8)
    occ[0, 2] = 1
    n = 400
    sim = oracle.OracleSim(dev, np.full(n, V), occ)
    key = [0xC0FFEE, 0]
    pos, kinds = 2, set()
    for t in range(n):
        x = [int(w) for w in oracle.philox4x32_10([pos, 0, t, 9], key)]
        uR = ((x[1] << 32 | x[0]) >> 11) * 2.0 ** -53
        uL = ((x[3] << 32 | x[2]) >> 11) * 2.0 ** -53
        aR = pos < L - 1 and uR <= pR
        aL = pos > 0 and uL <= pL
        step = (1 if aR else 0) - (1 if aL else 0)
        kinds.add((aR, aL))
        J, _ = sim.step_n(1)
        pos += step
        assert sim.occ[0, pos] == 1 and sim.occ.sum() == 1, "step %d" % t
        assert J[0] == -step
    assert kinds == {(False, False), (True, False), (False, True), (True, True)}
