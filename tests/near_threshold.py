"""Devices whose step-0 decisions are forced next to their thresholds.

A decision accepts a trial when its uniform u is at most p (S2.1.7).  The
near-threshold log records the decisions with |u - p| < 1e-12.  Random inputs
almost never produce one (about 2e-12 per trial), so these devices are built
to: for chosen occupied sites the per-site barrier Ea_k is solved so that, at
step 0, the site's left-trial probability p = P0_k / (1 + B_z) (Eqs. 1, 4, 5)
sits a chosen delta below or above the site's own left uniform u; on open
rails the electrode rate and reservoir density are solved so that one
injection (site 0, right draw, Eq. 6) and one extraction (site L-1, right
draw) sit that close too.  |delta| is 2e-14 .. 9e-14: inside the logging
window and far outside the last-ulp differences of exp/expm1 between two
implementations (about 1e-17 here), so both sides take the same decisions
and log the same entries.

The uniforms come from the oracle's Philox (counter (site, rail, step,
instance), u from the 53 high bits of (x1:x0) for the right trial and
(x3:x2) for the left), the zone factors from the oracle's field; the solved
parameters then go through each side's own arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_2511_09413_gb300 import workloads as W

KB = 8.6173e-5


def _uniforms(site, rail, step, instance, seed):
    x = oracle.philox4x32_10([site, rail, step, instance],
                             [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    uR = float(((int(x[1]) << 32) | int(x[0])) >> 11) * 2.0 ** -53
    uL = float(((int(x[3]) << 32) | int(x[2])) >> 11) * 2.0 ** -53
    return uR, uL


def forced_device(R, L, electrodes, seed, per_rail=3, n_steps=40, V0=0.7):
    """(dev, V, occ0, Ea_site, targets): targets lists the forced step-0
    decisions as (rail, step, site, dir, kind) with dir 0 right, 1 left and
    kind 0 inner hop, 1 injection, 2 extraction."""
    rng = np.random.default_rng(seed)
    Z = min(10, L)
    dev = dict(R=R, L=L, Z=Z, electrodes=electrodes, d=1.0, dt=5e-7, T=300.0, Ea=0.40,
               nu=1e12, alpha=0.2, kappa=1.0, k_e=1e6 if electrodes else 0.0,
               rho_e=0.3 if electrodes else 0.0, seed=int(rng.integers(1, 2 ** 62)),
               instance=int(rng.integers(0, 100)))
    inst, key = dev["instance"], dev["seed"]
    occ0 = W.random_occupancy(R, L, 0.3, seed=seed + 1)
    V = np.full(n_steps, V0)
    kT = KB * dev["T"]
    zone = np.array([oracle.zone_of(k, L, Z) for k in range(L)])
    targets = []

    def delta():
        return float(rng.choice([-1.0, 1.0]) * rng.uniform(2e-14, 9e-14))

    def field(r):
        Nz = np.bincount(zone, weights=occ0[r], minlength=Z).astype(np.int32)
        _, B, inv = oracle.zone_field(dev, Nz, int(occ0[r].sum()), V[0])
        return B, inv

    if electrodes:
        # an injection into the empty site 0 of rail r0 and an extraction from
        # the occupied site L-1 of rail r1, both decided by the right draw:
        # p_in = E rho inv_0 B_0,  p_out = E (1 - rho) inv_{Z-1} B_{Z-1}
        found = False
        for r0 in range(R):
            for r1 in range(R):
                if r1 == r0:
                    continue
                o0, o1 = occ0[r0, 0], occ0[r1, L - 1]
                occ0[r0, 0], occ0[r1, L - 1] = 0, 1
                B0, inv0 = field(r0)
                B1, inv1 = field(r1)
                u0, _ = _uniforms(0, r0, 0, inst, key)
                u1, _ = _uniforms(L - 1, r1, 0, inst, key)
                a = (u0 - delta()) / (inv0[0] * B0[0])
                b = (u1 - delta()) / (inv1[Z - 1] * B1[Z - 1])
                if 0.0 < a and 0.0 < b and a + b < 0.95:
                    E = a + b
                    dev["rho_e"] = a / E
                    dev["k_e"] = -math.log1p(-E) / (2.0 * dev["dt"])
                    targets += [(r0, 0, 0, 0, 1), (r1, 0, L - 1, 0, 2)]
                    found = True
                    break
                occ0[r0, 0], occ0[r1, L - 1] = o0, o1
            if found:
                break
        assert found, "no rail pair admits the electrode targets"

    Ea = np.full((R, L), dev["Ea"])
    Ea += rng.normal(0.0, 0.02, size=(R, L))
    for r in range(R):
        B, inv = field(r)
        sites = [k for k in range(1, L) if occ0[r, k] == 1 and occ0[r, k - 1] == 0]
        rng.shuffle(sites)
        taken = 0
        for k in sites:
            if taken == per_rail:
                break
            _, uL = _uniforms(k, r, 0, inst, key)
            p = uL - delta()
            P0 = p / inv[zone[k]]
            if not 1e-6 < P0 < 0.9:
                continue
            x = -math.log1p(-P0)                       # P0 = 1 - exp(-x), x = 2 nu exp(-Ea/kT) dt
            Ea[r, k] = -kT * math.log(x / (2.0 * dev["nu"] * dev["dt"]))
            targets.append((r, 0, k, 1, 0))
            taken += 1
    return dev, V, occ0, Ea, targets
