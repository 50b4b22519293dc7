"""kmc_sweep_noalloc, the entry point for callers that cannot allocate device
memory (a framework allocator that owns the whole GPU, latency-bound loops
that cannot afford cudaMalloc's synchronisation, services with a fixed device
footprint).  It must give exactly the results of the handle-based path: two
calls in a row, against kmc_create / kmc_step_n on the same device.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2511_09413_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09413_gb300 import build, kmc
    build.build()
    kmc.load()
    return torch, kmc


def _device(electrodes):
    return dict(R=300, L=100, Z=10, electrodes=electrodes, d=1.0, dt=5e-7, T=300.0, Ea=0.40,
                nu=1e12, alpha=0.2, kappa=1.0, k_e=2e6 if electrodes else 0.0,
                rho_e=0.3 if electrodes else 0.0, seed=2024, instance=3)


@pytest.mark.parametrize("electrodes", [0, 1])
def test_no_alloc_sweep_matches_handle_path_on_two_calls(env, electrodes):
    torch, kmc = env
    dev = _device(electrodes)
    R, L, Z = dev["R"], dev["L"], dev["Z"]
    n1, n2 = 170, 230
    V = W.triangle_protocol(3.0, 120, 4)[: n1 + n2]
    occ0 = W.random_occupancy(R, L, 0.35, seed=11)

    # the existing path: a handle owning its device memory
    sim = kmc.Sim(dev, V, init_mode=2, occ0=occ0)
    sim.step_n(n1)
    occ_mid = sim.occupancy()
    sim.step_n(n2)
    J_ref, Zc_ref = sim.traces()
    occ_ref = sim.occupancy()
    sim.close()

    # the no-allocation path: all device memory belongs to the caller
    stream = torch.cuda.current_stream()
    stride = (L + 15) // 16 * 16
    occ_dev = torch.zeros((R, stride), dtype=torch.uint8, device="cuda")
    occ_dev[:, :L] = torch.from_numpy(occ0).cuda()
    V_dev = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    N0_dev = torch.from_numpy(occ0.sum(axis=1).astype(np.int32)).cuda()
    J_dev = torch.full((n1 + n2,), -7, dtype=torch.int64, device="cuda")   # must be overwritten
    Zc_dev = torch.full((n1 + n2, Z), -7, dtype=torch.int64, device="cuda")
    p = kmc.params_from_device(dev, init_mode=2)

    # first call: background counts taken from the occupancy (the device's first step)
    kmc.kmc_sweep_noalloc(p, occ_dev.data_ptr(), stride, None, V_dev.data_ptr(), 0, n1,
                          J_dev.data_ptr(), Zc_dev.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(occ_dev[:, :L].cpu().numpy(), occ_mid)
    # second call continues from the first, with the background counts given
    kmc.kmc_sweep_noalloc(p, occ_dev.data_ptr(), stride, N0_dev.data_ptr(),
                          V_dev[n1:].data_ptr(), n1, n2, J_dev[n1:].data_ptr(),
                          Zc_dev[n1:].data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()

    assert np.array_equal(J_dev.cpu().numpy(), J_ref)
    assert np.array_equal(Zc_dev.cpu().numpy(), Zc_ref)
    assert np.array_equal(occ_dev[:, :L].cpu().numpy(), occ_ref)
    assert not occ_dev[:, L:].any()


def test_no_alloc_rejects_sizes_beyond_its_scratch(env):
    torch, kmc = env
    dev = _device(0)
    dev["R"] = (1 << 20) + 1
    p = kmc.params_from_device(dev, init_mode=2)
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_sweep_noalloc(p, buf.data_ptr(), 112, None, buf.data_ptr(), 0, 1, buf.data_ptr(),
                              buf.data_ptr(), 0)
    assert e.value.code == kmc.KMC_E_ARG
    assert "KMC_NOALLOC_MAX_RAILS" in str(e.value)
