"""Writes the target learning/forgetting curves of the material fit:
the oracle's conductance curves G*(t) = (ions in zone 0) / (ions) of the
fit devices (paper_2511_09413_gb300.workloads.fit_batch) at the hidden
parameters Ea = 0.42 eV, coupling kappa = 0.9, each from a fixed sample of
its rails (every rail has its own Philox stream, so a sample of rails is the
oracle's exact trajectory of those rails).  Calls only the oracle.

    python tests/golden/make_fit_target.py [n_dev n_pulses forget_steps rails_per_device]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2511_09413_gb300 import workloads as W  # noqa: E402

EA_HIDDEN, KAPPA_HIDDEN = 0.42, 0.9


def target_name(n_dev, n_pulses, forget_steps):
    return os.path.join(HERE, "fit_target_%ddev_%dp_%df.npz" % (n_dev, n_pulses, forget_steps))


def device_curve(job):
    """The oracle's G*(t) of one device from `rails` evenly spaced rails."""
    i, n_dev, n_pulses, forget_steps, rails = job
    devs, V, fills, samples = W.fit_batch(n_dev, n_pulses=n_pulses, forget_steps=forget_steps)
    d, fill = devs[i], fills[i]
    dev = dict(d.as_dict(), Ea=EA_HIDDEN, kappa=KAPPA_HIDDEN)
    ids = np.unique(np.linspace(0, d.R - 1, rails).astype(np.int32))
    occ0 = oracle.init_occupancy(dev, 1, fill=fill, rail_ids=ids)
    sim = oracle.OracleSim(dev, V, occ0, rail_ids=ids, nthreads=1)
    _, Zc = sim.step_n(int(samples.max()) + 1)
    return i, Zc[samples, 0] / max(float(occ0.sum()), 1.0)


def main(n_dev=256, n_pulses=8, forget_steps=8000, rails=24):
    import multiprocessing as mp
    _, _, _, samples = W.fit_batch(n_dev, n_pulses=n_pulses, forget_steps=forget_steps)
    target = np.zeros((n_dev, len(samples)))
    jobs = [(i, n_dev, n_pulses, forget_steps, rails) for i in range(n_dev)]
    # one single-threaded oracle per process: the rail samples are too small
    # for threads within a step to pay
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for i, curve in pool.imap_unordered(device_curve, jobs):
            target[i] = curve
            print("device %d: G* %.4f -> %.4f" % (i, curve[0], curve[-1]), flush=True)
    np.savez(target_name(n_dev, n_pulses, forget_steps), target=target, sample_steps=samples,
             Ea=EA_HIDDEN, kappa=KAPPA_HIDDEN, rails_per_device=rails)


if __name__ == "__main__":
    main(*[int(x) for x in sys.argv[1:]])
