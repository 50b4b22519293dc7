"""The forced near-threshold devices (tests/near_threshold.py) against the
oracle: every forced step-0 decision (inner left hops with solved per-site
barriers; an injection and an extraction with a solved electrode rate and
reservoir density on open rails) appears in the oracle's near-threshold log
with u - p at the constructed 2e-14 .. 9e-14 distance, and of both signs, so
that the GPU comparison of the logs has entries of every kind to compare."""
import numpy as np
import pytest

import oracle
from tests.near_threshold import forced_device


@pytest.mark.parametrize("R,L,electrodes", [(12, 100, 0), (9, 37, 1), (5, 1024, 1),
                                            (3, 2048, 0), (20, 300, 1)])
def test_forced_decisions_are_logged_by_the_oracle(R, L, electrodes):
    dev, V, occ0, Ea, targets = forced_device(R, L, electrodes, seed=R * 1000 + L)
    assert len(targets) >= 3
    orc = oracle.OracleSim(dev, V, occ0, Ea)
    orc.step_n(1)
    log = orc.near_threshold_log()
    got = {(int(e["rail"]), int(e["step"]), int(e["site"]), int(e["dir"]), int(e["kind"])): e["diff"]
           for e in log}
    for t in targets:
        assert t in got, t
        assert 1.5e-14 < abs(got[t]) < 1e-13, (t, got[t])
    diffs = np.array([got[t] for t in targets])
    if len(targets) >= 8:
        assert (diffs > 0).any() and (diffs < 0).any()
    if electrodes:
        kinds = {t[4] for t in targets}
        assert kinds == {0, 1, 2}
