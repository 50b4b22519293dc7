"""Brute-force master equation of one short rail (test tool, independent of
the C oracle and of the CUDA path).

For a rail of L <= 8 sites every configuration is enumerated; for each one,
every joint outcome of the Bernoulli trials the synchronous rule draws
(S2.1.6 - S2.1.7) is enumerated too, and the rule's deterministic part
(exclusion against the step-start state, both-trials-succeed => stay,
two hops into one empty site => both cancelled, electrode exchange) maps the
outcome to the next configuration.  The result is the exact one-step
transition matrix T of the Markov chain.  Written separately from the oracle
so that a shared mistake is unlikely.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

KB = 8.6173e-5  # eV/K, as printed next to Eq. 4


def zone_index(k, L, Z):
    return math.ceil((k + 1) * Z / L) - 1


def field_B(occ_bits, L, Z, N0, V, dev):
    """Boltzmann factor per zone for one configuration (1-D Gauss law)."""
    zones = [zone_index(k, L, Z) for k in range(L)]
    w = [zones.count(z) for z in range(Z)]
    N = [0] * Z
    for k in range(L):
        if occ_bits[k]:
            N[zones[k]] += 1
    excess = [N[z] - N0 * w[z] / L for z in range(Z)]
    enclosed_mid = []
    left_sum = 0.0
    for z in range(Z):
        enclosed_mid.append(left_sum + excess[z] / 2)
        left_sum += excess[z]
    mean_enclosed = sum(w[z] * enclosed_mid[z] for z in range(Z)) / L
    B = []
    for z in range(Z):
        v_loc = V - dev["kappa"] * dev["alpha"] * (enclosed_mid[z] - mean_enclosed)
        gap = v_loc * dev["d"] / (L * dev["d"])
        B.append(math.exp(-gap / (KB * dev["T"])))
    return B, zones


def transition_matrix(dev, V, N0, Ea_site=None, with_current=False):
    """Exact one-step transition matrix over all 2^L configurations
    (bit k of the state index = site k occupied).  ``Ea_site`` gives a
    barrier per site for hops leaving that site (else the scalar Ea).  With
    ``with_current`` also the expected net leftward crossings of one step from
    each configuration (electrode bonds included)."""
    L, Z = dev["L"], dev["Z"]
    open_ = dev["electrodes"] == 1
    kT = KB * dev["T"]
    def base_prob(Ea):
        gamma = dev["nu"] * math.exp(-Ea / kT)          # Eq. 1
        return 1.0 - math.exp(-2.0 * gamma * dev["dt"])
    P0_scalar = base_prob(dev["Ea"])
    P0_site = [base_prob(e) for e in Ea_site] if Ea_site is not None else None
    E = 1.0 - math.exp(-2.0 * dev["k_e"] * dev["dt"])
    E_in, E_out = E * dev["rho_e"], E * (1.0 - dev["rho_e"])
    n = 1 << L
    T = np.zeros((n, n))
    Jmean = np.zeros(n)
    for s in range(n):
        occ = [(s >> k) & 1 for k in range(L)]
        B, zones = field_B(occ, L, Z, N0, V, dev)
        trials = []  # (site, direction, probability); direction +1 right, -1 left
        for k in range(L):
            z = zones[k]
            pk = P0_site[k] if P0_site is not None else P0_scalar
            split_left = 1.0 / (1.0 + B[z])
            split_right = B[z] / (1.0 + B[z])
            if occ[k]:
                # right neighbour free, or the right electrode when open
                if k + 1 < L:
                    if not occ[k + 1]:
                        trials.append((k, +1, pk * split_right))
                elif open_:
                    trials.append((k, +1, E_out * split_right))
                if k - 1 >= 0:
                    if not occ[k - 1]:
                        trials.append((k, -1, pk * split_left))
                elif open_:
                    trials.append((k, -1, E_out * split_left))
            elif open_ and k == 0:
                trials.append((-1, +1, E_in * split_right))   # from the left reservoir
            elif open_ and k == L - 1:
                trials.append((L, -1, E_in * split_left))     # from the right reservoir
        for outcome in itertools.product((0, 1), repeat=len(trials)):
            prob = 1.0
            for (site, dirn, p), hit in zip(trials, outcome):
                prob *= p if hit else (1.0 - p)
            if prob == 0.0:
                continue
            # per source: net displacement (both directions succeeding => stay)
            net = {}
            for (site, dirn, p), hit in zip(trials, outcome):
                if hit:
                    net[site] = net.get(site, 0) + dirn
            moves = {src: d for src, d in net.items() if d != 0}
            # targets; two hops into one site cancel both
            target_count = {}
            for src, d in moves.items():
                target_count[src + d] = target_count.get(src + d, 0) + 1
            moves = {src: d for src, d in moves.items()
                     if not (0 <= src + d < L and target_count[src + d] > 1)}
            nxt = list(occ)
            for src, d in moves.items():
                if 0 <= src < L:
                    nxt[src] = 0
            for src, d in moves.items():
                if 0 <= src + d < L:
                    nxt[src + d] = 1
            s2 = sum(b << k for k, b in enumerate(nxt))
            T[s, s2] += prob
            Jmean[s] += prob * sum(-d for d in moves.values())
    if with_current:
        return T, Jmean
    return T


def state_index(occ_row):
    return int(sum(int(b) << k for k, b in enumerate(occ_row)))


def stationary(T):
    """Left eigenvector of T for eigenvalue 1, normalised (restricted to the
    states reachable from anywhere it is supported on)."""
    w, v = np.linalg.eig(T.T)
    i = int(np.argmin(np.abs(w - 1.0)))
    pi = np.real(v[:, i])
    pi = pi / pi.sum()
    return pi


def transition_matrix_brick(dev, V, N0, parity, Ea_site=None):
    """Exact one-step transition matrix of the brick-wall variant at a step of
    the given parity: only bonds (b, b+1) with b = parity (mod 2) are active,
    b = -1 being the left reservoir's bond and b = L-1 the right one's.  An
    active bond holding exactly one ion tries that ion's hop across it; the
    trials of different bonds touch disjoint sites, so every joint outcome
    maps to a configuration directly (no exclusion conflicts exist)."""
    L, Z = dev["L"], dev["Z"]
    open_ = dev["electrodes"] == 1
    kT = KB * dev["T"]

    def base_prob(Ea):
        return 1.0 - math.exp(-2.0 * dev["nu"] * math.exp(-Ea / kT) * dev["dt"])

    P0 = [base_prob(e) for e in Ea_site] if Ea_site is not None else [base_prob(dev["Ea"])] * L
    E = 1.0 - math.exp(-2.0 * dev["k_e"] * dev["dt"])
    E_in, E_out = E * dev["rho_e"], E * (1.0 - dev["rho_e"])
    n = 1 << L
    T = np.zeros((n, n))
    for s in range(n):
        occ = [(s >> k) & 1 for k in range(L)]
        B, zones = field_B(occ, L, Z, N0, V, dev)

        def right(k):   # Boltzmann share of a rightward hop in the zone of site k
            return B[zones[k]] / (1.0 + B[zones[k]])

        def left(k):
            return 1.0 / (1.0 + B[zones[k]])

        # (probability, site that empties or -1, site that fills or -1)
        trials = []
        for b in range(-1, L):
            if b % 2 != parity % 2:
                continue
            if b == -1:
                if open_:
                    trials.append((E_out * left(0), 0, -1) if occ[0] else (E_in * right(0), -1, 0))
            elif b == L - 1:
                if open_:
                    trials.append((E_out * right(L - 1), L - 1, -1) if occ[L - 1]
                                  else (E_in * left(L - 1), -1, L - 1))
            elif occ[b] and not occ[b + 1]:
                trials.append((P0[b] * right(b), b, b + 1))
            elif occ[b + 1] and not occ[b]:
                trials.append((P0[b + 1] * left(b + 1), b + 1, b))
        for outcome in itertools.product((0, 1), repeat=len(trials)):
            prob = 1.0
            nxt = list(occ)
            for (p, src, dst), hit in zip(trials, outcome):
                prob *= p if hit else 1.0 - p
                if hit:
                    if src >= 0:
                        nxt[src] = 0
                    if dst >= 0:
                        nxt[dst] = 1
            if prob > 0.0:
                T[s, sum(v << k for k, v in enumerate(nxt))] += prob
    return T
