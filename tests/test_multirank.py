"""The multi-GPU path's host logic on CPU: two gloo ranks (spawned
processes), each advancing its shard of four device instances, sum their
traces in the readout collective and take the maximum of their timings.
The per-rank engine here is the oracle (the data path needs no GPU and has
no exchange); the summed traces must equal one process running all four
instances, and the instances must be distinct streams."""
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


def _device(instance):
    return dict(R=12, L=40, Z=5, electrodes=1, d=1.0, dt=5e-7, T=300.0, Ea=0.40, nu=1e12,
                alpha=0.3, kappa=1.0, k_e=2e5, rho_e=0.3, seed=99, instance=instance)


def _run_instance(instance):
    dev = _device(instance)
    occ0 = oracle.init_occupancy(dev, 1, fill=0.3)
    V = W.triangle_protocol(1.5, 40, 2)[:N_STEPS]
    return oracle.OracleSim(dev, V, occ0, nthreads=1).step_n(N_STEPS)


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    J = np.zeros(N_STEPS, dtype=np.int64)
    Zc = np.zeros((N_STEPS, 5), dtype=np.int64)
    mine = MG.shard_instances(N_INST, rank, world)
    for i in mine:
        j, z = _run_instance(i)
        J += j
        Zc += z
    J, Zc = MG.sum_traces(J, Zc)
    t = MG.max_over_ranks(1.5 + rank)
    MG.barrier()
    if rank == 0:
        np.savez(out, J=J, Zc=Zc, t=t, mine=np.array(mine))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharding_is_a_partition():
    for world in (1, 2, 3, 8):
        got = sorted(i for r in range(world) for i in MG.shard_instances(10, r, world))
        assert got == list(range(10))
    with pytest.raises(ValueError):
        MG.shard_instances(4, 2, 2)
    assert MG.whole_job_rate([3.0, 5.0], 2.0) == 4.0


def test_two_gloo_ranks_match_one_process(tmp_path):
    oracle.lib()                      # build the oracle before spawning
    out = str(tmp_path / "rank0.npz")
    tmp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                        start_method="spawn")
    r = np.load(out)
    J = np.zeros(N_STEPS, dtype=np.int64)
    Zc = np.zeros((N_STEPS, 5), dtype=np.int64)
    per = []
    for i in range(N_INST):
        j, z = _run_instance(i)
        J += j
        Zc += z
        per.append(z)
    assert np.array_equal(r["J"], J) and np.array_equal(r["Zc"], Zc)
    assert float(r["t"]) == 2.5                    # the slower rank's time
    assert list(r["mine"]) == [0, 2]
    # distinct instances are distinct streams
    assert not np.array_equal(per[0], per[1])
