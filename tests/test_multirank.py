"""The multi-GPU path's host logic on CPU, as two gloo ranks (spawned
processes).  The per-rank engine is the oracle: the data path needs no GPU
and has no exchange.

- Rail partition: each rank advances its contiguous rails of one device (a
  device of r1 - r0 rails starting at global rail r0); the ranks' summed
  traces equal one process advancing the whole device, and each rank's rows
  equal those rows of the whole device.
- Instance partition: each rank advances its share of four instances; the
  summed traces equal one process running all four.
- The timing collective takes the slower rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import oracle  # noqa: E402
from paper_2511_09413_gb300 import multigpu as MG  # noqa: E402
from paper_2511_09413_gb300 import workloads as W  # noqa: E402

N_INST, N_STEPS = 4, 60
R_WHOLE, L_WHOLE = 23, 40


def _device(instance, R=12, rail_base=0):
    return dict(R=R, L=L_WHOLE, Z=5, electrodes=1, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
                alpha=0.3, kappa=1.0, k_e=2e5, rho_e=0.3, seed=99, instance=instance,
                rail_base=rail_base)


def _V():
    return W.triangle_protocol(1.5, 40, 2)[:N_STEPS]


def _run_instance(instance):
    dev = _device(instance)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    return oracle.OracleSim(dev, _V(), occ0, nthreads=1).step_n(N_STEPS)


def _run_rails(r0, r1):
    """Rails [r0, r1) of the whole device, advanced as a device of their own."""
    dev = _device(7, R=r1 - r0, rail_base=r0)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    sim = oracle.OracleSim(dev, _V(), occ0, nthreads=1)
    J, Zc = sim.step_n(N_STEPS)
    return J, Zc, sim.occ, sim.J_rail


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # instance partition
    J = np.zeros(N_STEPS, dtype=np.int64)
    Zc = np.zeros((N_STEPS, 5), dtype=np.int64)
    mine = MG.shard_instances(N_INST, rank, world)
    for i in mine:
        j, z = _run_instance(i)
        J += j
        Zc += z
    J, Zc = MG.sum_traces(J, Zc)
    # rail partition of one device
    r0, r1 = MG.shard_rails(R_WHOLE, rank, world)
    Jr, Zr, occ, jrail = _run_rails(r0, r1)
    Jr, Zr = MG.sum_traces(Jr, Zr)
    t = MG.max_over_ranks(1.5 + rank)
    MG.barrier()
    np.savez(out % rank, J=J, Zc=Zc, t=t, mine=np.array(mine), Jr=Jr, Zr=Zr, occ=occ,
             jrail=jrail, rows=np.array([r0, r1]))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharding_is_a_partition():
    for world in (1, 2, 3, 8):
        got = sorted(i for r in range(world) for i in MG.shard_instances(10, r, world))
        assert got == list(range(10))
        rows = [MG.shard_rails(23, r, world) for r in range(world)]
        assert rows[0][0] == 0 and rows[-1][1] == 23
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
        sizes = [b - a for a, b in rows]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        MG.shard_instances(4, 2, 2)
    with pytest.raises(ValueError):
        MG.shard_rails(4, 2, 2)
    assert MG.whole_job_rate([3.0, 5.0], 2.0) == 4.0


def test_two_gloo_ranks_match_one_process(tmp_path):
    oracle.lib()                      # build the oracle before spawning
    out = str(tmp_path / "rank%d.npz")
    tmp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                        start_method="spawn")
    r = [np.load(out % k) for k in range(2)]
    # instance partition
    J = np.zeros(N_STEPS, dtype=np.int64)
    Zc = np.zeros((N_STEPS, 5), dtype=np.int64)
    per = []
    for i in range(N_INST):
        j, z = _run_instance(i)
        J += j
        Zc += z
        per.append(z)
    assert np.array_equal(r[0]["J"], J) and np.array_equal(r[0]["Zc"], Zc)
    assert float(r[0]["t"]) == 2.5 and float(r[1]["t"]) == 2.5   # the slower rank's time
    assert list(r[0]["mine"]) == [0, 2]
    assert not np.array_equal(per[0], per[1])      # distinct instances are distinct streams
    # rail partition: the whole device in one process
    Jw, Zw, occ_w, jrail_w = _run_rails(0, R_WHOLE)
    assert [list(x["rows"]) for x in r] == [[0, 12], [12, 23]]
    for x in r:
        assert np.array_equal(x["Jr"], Jw) and np.array_equal(x["Zr"], Zw)
        a, b = x["rows"]
        assert np.array_equal(x["occ"], occ_w[a:b])
        assert np.array_equal(x["jrail"], jrail_w[a:b])
    assert Jw.sum() == jrail_w.sum()
