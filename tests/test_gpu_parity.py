"""GPU parity: the CUDA sweep (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Occupancy trajectories, per-step current, per-rail
current and zone counts must be bit-identical; integer traces leave no room
for tolerance.  Near-threshold decisions (|u - p| < 1e-12, S2.1.7's "u <= p")
must be logged identically: the same (rail, step, site, direction, kind) set,
and u - p equal to 1e-15 (both sides compute it in FP64 from the same u and a
p that can differ by an ulp of exp)."""
import numpy as np
import pytest

import oracle
from paper_2511_09413_gb300 import workloads as W
from tests.near_threshold import forced_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09413_gb300 import build, kmc as K
    build.build()
    K.load()
    torch.cuda.init()
    return K


def _dev(**kw):
    d = dict(R=8, L=100, Z=10, electrodes=0, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
             alpha=0.2, kappa=1.0, k_e=0.0, rho_e=0.0, seed=7, instance=0)
    d.update(kw)
    return d


LOG_KEYS = ("rail", "step", "site", "dir", "kind")


def _sorted_log(log):
    order = np.lexsort(tuple(log[k] for k in reversed(LOG_KEYS)))
    return log[order]


def assert_logs_equal(lg, lo):
    """Near-threshold logs: equal as sets of (rail, step, site, dir, kind), with
    u - p equal to 1e-15 (the logs are filled in a nondeterministic order)."""
    assert len(lg) == len(lo), (len(lg), len(lo))
    a, b = _sorted_log(lg), _sorted_log(lo)
    for k in LOG_KEYS:
        assert np.array_equal(a[k], b[k]), k
    assert np.all(np.abs(a["diff"] - b["diff"]) <= 1e-15)
    assert np.all(np.abs(a["diff"]) < 1e-12)


def _compare(kmc, dev, V, occ0, Ea=None, chunks=None, warps=0, flush=0, accept=-1):
    """Run GPU and oracle from the same occupancy; compare everything."""
    n = len(V)
    sim = kmc.Sim(dev, V, init_mode=2, occ0=occ0, Ea_site=Ea)
    if warps or flush:
        sim.set_launch(warps, flush)
    if accept >= 0:
        sim.set_accept_path(accept)
        assert sim.accept_path == accept
    orc = oracle.OracleSim(dev, V, occ0, Ea)
    for c in (chunks or [n]):
        sim.step_n(c)
    Jo, Zo = orc.step_n(n)
    Jg, Zg = sim.traces()
    occ_g = sim.occupancy()
    assert np.array_equal(Zg, Zo), "zone-count traces differ"
    assert np.array_equal(Jg, Jo), "current traces differ"
    assert np.array_equal(occ_g, orc.occ), "final occupancy differs"
    Jr = sim.rail_current()
    assert np.array_equal(Jr, orc.J_rail), "per-rail current differs"
    assert Jr.sum() == Jg.sum()
    lg, n_lg = sim.near_threshold_log(with_total=True)
    assert n_lg == len(lg) and int(orc.log_count[0]) == n_lg, "log overflowed or counts differ"
    assert_logs_equal(lg, orc.near_threshold_log())
    cnt = sim.counters()
    sim.close()
    return Jg, Zg, occ_g, cnt, lg


def test_relaxation_64x100_full_run_bit_exact(kmc):
    """64 rails x 100 sites, 800 ions at seed 0, 1 V x 5000 then 0 V x 5000."""
    wl = W.relaxation_64x100()
    sim = kmc.Sim.from_workload(wl)
    orc = oracle.OracleSim.from_workload(wl)
    assert np.array_equal(sim.occupancy(), orc.occ), "initial placement differs"
    assert sim.occupancy().sum() == 800
    sim.step_n(5000)
    sim.step_n(5000)
    Jo, Zo = orc.step_n(10000)
    Jg, Zg = sim.traces()
    assert np.array_equal(Zg, Zo)
    assert np.array_equal(Jg, Jo)
    assert np.array_equal(sim.occupancy(), orc.occ)
    assert np.array_equal(sim.rail_current(), orc.J_rail)
    assert_logs_equal(sim.near_threshold_log(), orc.near_threshold_log())
    sim.close()


@pytest.mark.parametrize("L", [2, 3, 5, 31, 32, 33, 37, 64, 100, 127, 128, 129, 255, 500, 1000,
                               1023, 1024, 1025, 1500, 2047, 2048])
@pytest.mark.parametrize("electrodes", [0, 1])
def test_shapes_bit_exact(kmc, L, electrodes):
    rng = np.random.default_rng(L * 3 + electrodes)
    Z = int(min(L, [1, 3, 10, 32][L % 4]))
    R = int(rng.integers(1, 41))
    dev = _dev(R=R, L=L, Z=Z, electrodes=electrodes, k_e=2e6 if electrodes else 0.0,
               rho_e=0.3 if electrodes else 0.0, seed=int(rng.integers(0, 2 ** 63)),
               instance=int(rng.integers(0, 1000)))
    occ0 = W.random_occupancy(R, L, float(rng.uniform(0.05, 0.7)), seed=L)
    V = W.triangle_protocol(3.0, 150, 2)
    _compare(kmc, dev, V, occ0)


@pytest.mark.parametrize("L,electrodes", [(100, 0), (1024, 1), (2048, 1), (37, 1)])
def test_per_site_barriers_bit_exact(kmc, L, electrodes):
    R = 24
    dev = _dev(R=R, L=L, electrodes=electrodes, k_e=1e6, rho_e=0.25, seed=99)
    occ0 = W.random_occupancy(R, L, 0.3, seed=5)
    Ea = W.normal_barriers(R, L, 0.40, 0.02, seed=6)
    V = W.triangle_protocol(2.0, 200, 2)
    _compare(kmc, dev, V, occ0, Ea=Ea)


@pytest.mark.parametrize("Z,sigma", [(3, 0.05), (10, 0.02), (12, 0.05), (16, 0.03), (20, 0.05),
                                     (10, 0.0)])
@pytest.mark.parametrize("accept", [0, 1])
def test_per_site_barriers_zones_and_accept_paths_bit_exact(kmc, Z, sigma, accept):
    """Per-site barriers on 513-1,024-site rails (the shape whose list entries
    carry their bound row), from 3 to 20 zones, with a spread of barriers or
    all equal, on both accept paths: the oracle's trajectory."""
    R, L = 20, 700
    dev = _dev(R=R, L=L, Z=Z, dt=5e-7 if accept else 1e-9, electrodes=1, k_e=1e6, rho_e=0.3,
               seed=123 + Z)
    occ0 = W.random_occupancy(R, L, 0.3, seed=Z)
    Ea = W.normal_barriers(R, L, 0.40, sigma, seed=Z + 1) if sigma > 0 else np.full((R, L), 0.40)
    V = W.triangle_protocol(2.5, 150, 2)
    _compare(kmc, dev, V, occ0, Ea=Ea, accept=accept)


def test_chunked_steps_and_launch_shapes_identical(kmc):
    dev = _dev(R=50, L=300, Z=7, electrodes=1, k_e=3e6, rho_e=0.4)
    occ0 = W.random_occupancy(50, 300, 0.35, seed=1)
    V = W.triangle_protocol(4.0, 97, 3)
    a = _compare(kmc, dev, V, occ0)
    b = _compare(kmc, dev, V, occ0, chunks=[1, 2, 30, 100, len(V) - 133], warps=2, flush=7)
    c = _compare(kmc, dev, V, occ0, warps=1, flush=1)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    for x, y in zip(a[:3], c[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("dt", [1e-9, 5e-7, 5e-6])
@pytest.mark.parametrize("L,electrodes,per_site", [(100, 0, False), (33, 1, False), (1024, 1, True),
                                                   (2048, 1, False), (7, 0, True)])
def test_accept_path_modes_bit_exact(kmc, dt, L, electrodes, per_site):
    """The kernels with and without the inline accept path, at small and large
    hop probabilities (P0 from 4e-4 to 0.9), give the oracle's trajectory."""
    R = 24
    dev = _dev(R=R, L=L, Z=min(10, L), dt=dt, electrodes=electrodes, k_e=1e6 if electrodes else 0.0,
               rho_e=0.3 if electrodes else 0.0)
    occ0 = W.random_occupancy(R, L, 0.3, seed=L + 11)
    Ea = W.normal_barriers(R, L, 0.40, 0.02, seed=L) if per_site else None
    V = W.triangle_protocol(3.0, 120, 2)
    res = [_compare(kmc, dev, V, occ0, Ea=Ea, accept=m) for m in (0, 1)]
    for x, y in zip(res[0][:3], res[1][:3]):
        assert np.array_equal(x, y)


def test_strong_space_charge_and_large_bias(kmc):
    # large |exponent| drives decisions through the exact FP64 path
    dev = _dev(R=16, L=200, Z=10, alpha=3.0, kappa=1.0, electrodes=1, k_e=1e7, rho_e=0.9)
    occ0 = W.random_occupancy(16, 200, 0.6, seed=3)
    V = np.concatenate([np.full(200, 60.0), np.full(200, -60.0), np.zeros(100)])
    _, _, _, cnt, _ = _compare(kmc, dev, V, occ0)
    assert cnt[1] > 0   # some decisions needed the exact path


def test_empty_and_full_rails(kmc):
    for fill in (0.0, 1.0):
        for electrodes in (0, 1):
            dev = _dev(R=9, L=70, electrodes=electrodes, k_e=5e6, rho_e=0.5)
            occ0 = np.full((9, 70), int(fill), dtype=np.uint8)
            _compare(kmc, dev, W.constant_protocol(1.0, 120), occ0)


def test_zero_steps_and_range_errors(kmc):
    dev = _dev(R=3, L=40)
    sim = kmc.Sim(dev, np.zeros(10), init_mode=1, fill=0.5)
    sim.step_n(0)
    assert sim.t == 0
    sim.step_n(10)
    with pytest.raises(kmc.KmcError) as e:
        sim.step_n(1)
    assert e.value.code == kmc.KMC_E_RANGE
    with pytest.raises(kmc.KmcError):
        sim.traces(5, 10)
    sim.close()


@pytest.mark.parametrize("R,L,fill", [(64, 100, 0.25), (1000, 1024, 0.25), (3, 2048, 0.9)])
def test_bernoulli_placement_bit_exact(kmc, R, L, fill):
    dev = _dev(R=R, L=L)
    sim = kmc.Sim(dev, np.zeros(1), init_mode=1, fill=fill)
    assert np.array_equal(sim.occupancy(), oracle.init_occupancy(dev, 1, fill=fill))
    sim.close()


@pytest.mark.parametrize("R,L,n", [(64, 100, 800), (5, 37, 0), (5, 37, 185), (7, 300, 1),
                                   (300, 64, 5000)])
def test_exact_count_placement_bit_exact(kmc, R, L, n):
    dev = _dev(R=R, L=L)
    sim = kmc.Sim(dev, np.zeros(1), init_mode=0, n_ions=n)
    got = sim.occupancy()
    assert got.sum() == n
    assert np.array_equal(got, oracle.init_occupancy(dev, 0, n_ions=n))
    sim.close()


def test_near_threshold_decision_logged(kmc):
    dev = dict(R=1, L=5, Z=1, electrodes=0, d=1.0, dt=1e-6, T=300.0, Ea=0.0, nu=1e12,
               alpha=0.0, kappa=0.0, k_e=0.0, rho_e=0.0, seed=42, instance=0)
    for rail in range(64):
        x = oracle.philox4x32_10([2, rail, 0, 0], [42, 0])
        uL = float(((int(x[3]) << 32) | int(x[2])) >> 11) * 2.0 ** -53
        if 0.05 < uL < 0.45:
            break
    dev["nu"] = -np.log1p(-2.0 * uL) / (2.0 * dev["dt"])
    dev["R"] = rail + 1
    occ0 = np.tile(np.array([0, 0, 1, 0, 0], dtype=np.uint8), (rail + 1, 1))
    sim = kmc.Sim(dev, np.zeros(1), init_mode=2, occ0=occ0)
    sim.step_n(1)
    log = [e for e in sim.near_threshold_log() if e["rail"] == rail]
    assert len(log) == 1
    assert (log[0]["step"], log[0]["site"], log[0]["dir"], log[0]["kind"]) == (0, 2, 1, 0)
    assert abs(log[0]["diff"]) < 1e-12
    sim.close()


@pytest.mark.parametrize("accept", [0, 1])
@pytest.mark.parametrize("R,L,electrodes", [(12, 100, 0), (9, 37, 1), (5, 1024, 1),
                                            (3, 2048, 0), (20, 300, 1)])
def test_forced_near_threshold_decisions_logged_identically(kmc, R, L, electrodes, accept):
    """Step-0 decisions forced 2e-14 .. 9e-14 from their thresholds (inner hops
    through solved per-site barriers; an injection and an extraction through a
    solved electrode rate on open rails): the GPU logs exactly the oracle's
    entries, field by field, and every forced one among them, on both accept
    paths and on one-rail-per-warp, several-rails-per-warp and two-words-per-
    lane shapes; trajectories stay bit-exact."""
    dev, V, occ0, Ea, targets = forced_device(R, L, electrodes, seed=R * 1000 + L)
    *_, lg = _compare(kmc, dev, V, occ0, Ea=Ea, accept=accept)
    got = {(int(e["rail"]), int(e["step"]), int(e["site"]), int(e["dir"]), int(e["kind"]))
           for e in lg}
    for t in targets:
        assert t in got, t


def test_rail_shards_reproduce_the_whole_device(kmc):
    """A device split by rails into parts with rail_base (the multi-GPU
    partition) advances exactly the rows of the whole device: occupancy,
    per-rail current, and traces that sum to the whole device's."""
    R, L = 40, 300
    dev = _dev(R=R, L=L, Z=10, electrodes=1, k_e=2e6, rho_e=0.3, seed=31, instance=4)
    Ea = W.normal_barriers(R, L, 0.40, 0.02, seed=8)
    V = W.triangle_protocol(3.0, 100, 2)
    whole = kmc.Sim(dev, V, init_mode=1, fill=0.3, Ea_site=Ea)
    whole.step_n(len(V))
    Jw, Zw = whole.traces()
    occ_w, jr_w = whole.occupancy(), whole.rail_current()
    whole.close()
    J = np.zeros_like(Jw)
    Zc = np.zeros_like(Zw)
    for r0, r1 in [(0, 13), (13, 14), (14, 40)]:
        part = dict(dev, R=r1 - r0, rail_base=r0)
        sim = kmc.Sim(part, V, init_mode=1, fill=0.3, Ea_site=Ea[r0:r1])
        sim.step_n(len(V))
        j, z = sim.traces()
        J += j
        Zc += z
        assert np.array_equal(sim.occupancy(), occ_w[r0:r1])
        assert np.array_equal(sim.rail_current(), jr_w[r0:r1])
        sim.close()
    assert np.array_equal(J, Jw) and np.array_equal(Zc, Zw)
    # the oracle advances a part by the same global rail indices
    part = dict(dev, R=27, rail_base=13)
    occ_p = oracle.init_occupancy(part, 1, fill=0.3)
    orc = oracle.OracleSim(part, V, occ_p, Ea[13:40])
    orc.step_n(len(V))
    assert np.array_equal(orc.occ, occ_w[13:40])
    assert np.array_equal(orc.J_rail, jr_w[13:40])


def test_hysteresis_device_sampled_rails_full_size(kmc):
    """65,536 x 1,024 device, per-site barriers, open electrodes, +-2 V sweep:
    the GPU advances the whole device; every 256th rail is re-run on the
    oracle (rails are independent and keyed by their index) and must match."""
    wl = W.hysteresis_65536x1024(steps_per_cycle=100000, cycles=2)
    n = 300
    sim = kmc.Sim.from_workload(wl)
    occ_init = sim.occupancy()
    ids = np.arange(0, wl.device.R, 256)
    assert np.array_equal(occ_init[ids], oracle.init_occupancy(wl.device, 1, fill=wl.fill,
                                                               rail_ids=ids))
    sim.step_n(n)
    Jg, Zg = sim.traces()
    occ_g = sim.occupancy()
    orc = oracle.OracleSim(wl.device, wl.V, occ_init[ids], wl.Ea_site[ids], rail_ids=ids)
    orc.step_n(n)
    assert np.array_equal(occ_g[ids], orc.occ)
    Jr = sim.rail_current()
    assert np.array_equal(Jr[ids], orc.J_rail), "per-rail current of the sampled rails differs"
    assert Jr.sum() == Jg.sum()
    # the first zone-count row is the initial occupancy summed per zone
    z = np.array([oracle.zone_of(k, wl.device.L, wl.device.Z) for k in range(wl.device.L)])
    assert np.array_equal(Zg[0], np.bincount(z, weights=occ_init.sum(axis=0), minlength=10))
    sim.close()


def test_hysteresis_device_sampled_rails_whole_protocol(kmc):
    """The same device through its whole protocol (two +-2 V cycles, 2e5
    steps, in the bench's 10,000-step kmc_step_n calls): every 256th rail
    re-run on the oracle matches, occupancy and per-rail current, at every
    50,000-step checkpoint, and the near-threshold decisions of those rails
    are logged identically."""
    wl = W.hysteresis_65536x1024(steps_per_cycle=100000, cycles=2)
    n_total, chunk, launch = len(wl.V), 50000, 10000
    assert n_total == 200000
    sim = kmc.Sim.from_workload(wl)
    ids = np.arange(0, wl.device.R, 256)
    orc = oracle.OracleSim(wl.device, wl.V, sim.occupancy()[ids], wl.Ea_site[ids], rail_ids=ids)
    for t in range(chunk, n_total + 1, chunk):
        for _ in range(chunk // launch):
            sim.step_n(launch)
        orc.step_n(chunk)
        assert np.array_equal(sim.occupancy()[ids], orc.occ), "rails differ by step %d" % t
        assert np.array_equal(sim.rail_current()[ids], orc.J_rail), \
            "per-rail current differs by step %d" % t
    assert orc.occ.sum() > 0
    lg, n_lg = sim.near_threshold_log(with_total=True)
    assert n_lg == len(lg), "the near-threshold log overflowed"
    assert_logs_equal(lg[np.isin(lg["rail"], ids)], orc.near_threshold_log())
    sim.close()


@pytest.mark.parametrize("L,electrodes", [(128, 0), (40, 1), (1024, 1)])
def test_rapidly_varying_bias_bit_exact(kmc, L, electrodes):
    # the bias jumps every step, so the FP32 bands must cover a wide voltage window
    rng = np.random.default_rng(L)
    dev = _dev(R=20, L=L, Z=8, electrodes=electrodes, k_e=2e6, rho_e=0.35)
    occ0 = W.random_occupancy(20, L, 0.4, seed=L + 1)
    V = rng.uniform(-4.0, 4.0, size=300)
    V[::7] = 0.0
    _compare(kmc, dev, V, occ0)


@pytest.mark.parametrize("L,electrodes,per_site,dt", [
    (2, 1, False, 5e-7), (3, 0, False, 5e-7), (31, 1, False, 5e-7), (33, 1, True, 5e-7),
    (100, 0, False, 1e-9), (100, 1, False, 5e-6), (512, 1, True, 5e-7), (1024, 1, False, 5e-7),
    (1500, 0, True, 5e-7), (2048, 1, False, 5e-6)])
def test_brick_wall_rule_bit_exact(kmc, L, electrodes, per_site, dt):
    """The brick-wall variant (even/odd bonds) against the oracle's, with both
    accept paths and chunked launches."""
    R = 20
    dev = _dev(R=R, L=L, Z=min(10, L), dt=dt, electrodes=electrodes,
               k_e=1e6 if electrodes else 0.0, rho_e=0.3 if electrodes else 0.0, rule=1)
    occ0 = W.random_occupancy(R, L, 0.3, seed=L + 5)
    Ea = W.normal_barriers(R, L, 0.40, 0.02, seed=L + 1) if per_site else None
    V = W.triangle_protocol(3.0, 90, 2)
    res = [_compare(kmc, dev, V, occ0, Ea=Ea, accept=m, chunks=[7, 53, len(V) - 60])
           for m in (0, 1)]
    for x, y in zip(res[0][:3], res[1][:3]):
        assert np.array_equal(x, y)
    # the two rules differ on the same draws
    sync = _compare(kmc, dict(dev, rule=0), V, occ0, Ea=Ea)
    assert not np.array_equal(sync[2], res[0][2])


def test_brick_wall_rule_rejected_by_gradient_pass(kmc):
    dev = _dev(R=4, L=30, Z=3, rule=1)
    V = np.zeros(10)
    sim = kmc.Sim(dev, V, init_mode=1, fill=0.3)
    sim.step_n(10)
    with pytest.raises(kmc.KmcError):
        sim.grad(np.ones(10), None)
    sim.close()


def test_philox_probe_reports_a_rate(kmc):
    """The Philox-only probe runs and reports a rate between the sweep's own
    draw rate and the IMAD-issue bound (152 SMs x 64 lanes x 2.07 GHz / 40)."""
    r = kmc.kmc_philox_probe()
    assert 1e11 < r < 8e11, r
