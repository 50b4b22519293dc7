"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
include/kmc.h declares, the ctypes structures match the C layout, and host-side
argument validation rejects bad input before touching a GPU."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kmc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(kmc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2511_09413_gb300 import build, kmc
    build.build()
    return kmc.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("kmc_create", "kmc_step_n", "kmc_observables", "kmc_destroy", "kmc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2511_09413_gb300 import kmc
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(kmc.EXPORTS) == _declared()


def test_struct_layouts_match_header(lib):
    from paper_2511_09413_gb300 import kmc
    # kmc_params: 4 int32, 9 double, uint64, uint32, int32, int64, double, int32, int32
    assert ctypes.sizeof(kmc.kmc_params) == 4 * 4 + 9 * 8 + 8 + 4 + 4 + 8 + 8 + 4 + 4
    assert kmc.kmc_params.seed.offset == 16 + 72
    assert kmc.kmc_params.update_rule.offset == 16 + 72 + 8 + 4 + 4 + 8 + 8
    assert kmc.kmc_params.rail_base.offset == kmc.kmc_params.update_rule.offset + 4
    assert ctypes.sizeof(kmc.kmc_log_entry) == 32
    assert kmc.LOG_DTYPE.itemsize == 32


def _params(**kw):
    from paper_2511_09413_gb300 import kmc
    d = dict(n_rails=4, n_sites=100, n_zones=10, electrodes=0, site_spacing_nm=1.0, dt_s=1e-9,
             T_K=300.0, Ea_eV=0.4, nu_Hz=1e12, alpha_V=0.2, kappa=1.0, k_electrode_Hz=0.0,
             rho_electrode=0.0, seed=0, instance=0, init_mode=1, n_ions=0, fill=0.25)
    d.update(kw)
    return kmc.kmc_params(**d)


@pytest.mark.parametrize("bad", [
    dict(n_rails=0), dict(n_sites=1), dict(n_sites=4096), dict(n_zones=0), dict(n_zones=33),
    dict(n_sites=8, n_zones=9), dict(electrodes=2), dict(dt_s=0.0), dict(T_K=-1.0),
    dict(site_spacing_nm=float("nan")), dict(nu_Hz=-1.0), dict(init_mode=3),
    dict(init_mode=1, fill=1.5), dict(init_mode=0, n_ions=401), dict(init_mode=2),
    dict(electrodes=1, rho_electrode=1.5), dict(kappa=float("inf")), dict(update_rule=2),
    dict(update_rule=-1), dict(rail_base=-1), dict(rail_base=2 ** 31 - 3),
    dict(init_mode=0, n_ions=10, rail_base=8),
])
def test_validation_rejects_bad_parameters_on_host(lib, bad):
    from paper_2511_09413_gb300 import kmc
    p = _params(**bad)
    V = np.zeros(10)
    h = ctypes.c_void_p()
    rc = lib.kmc_create(ctypes.byref(p), V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 10,
                        None, None, None, ctypes.byref(h))
    assert rc == kmc.KMC_E_ARG
    assert h.value is None
    assert len(lib.kmc_last_error()) > 0


def test_validation_rejects_non_finite_voltage(lib):
    from paper_2511_09413_gb300 import kmc
    p = _params()
    V = np.array([0.0, np.nan, 1.0])
    h = ctypes.c_void_p()
    rc = lib.kmc_create(ctypes.byref(p), V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 3,
                        None, None, None, ctypes.byref(h))
    assert rc == kmc.KMC_E_ARG
    assert b"not finite" in lib.kmc_last_error()


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2511_09413_gb300 import kmc
    assert lib.kmc_step_n(None, 1) == kmc.KMC_E_ARG
    assert lib.kmc_observables(None, 0, 0, None, None, None) == kmc.KMC_E_ARG
    assert lib.kmc_rail_current(None, None) == kmc.KMC_E_ARG
    assert lib.kmc_batch_rail_current(None, 0, None) == kmc.KMC_E_ARG
    assert lib.kmc_current_step(None) == -1
    lib.kmc_destroy(None)
    g = (ctypes.c_double * 4)()
    assert lib.kmc_grad(None, None, None, g, None) == kmc.KMC_E_ARG
    assert lib.kmc_batch_grad(None, 0, None, None, g, None) == kmc.KMC_E_ARG
    assert lib.kmc_batch_grad_all(None, None, None, g, None) == kmc.KMC_E_ARG
    assert lib.kmc_batch_step_n(None, 1) == kmc.KMC_E_ARG
    assert lib.kmc_set_accept_path(None, 1) == kmc.KMC_E_ARG
    assert lib.kmc_philox_probe(None, None) == kmc.KMC_E_ARG
    assert lib.kmc_batch_current_step(None) == -1
    lib.kmc_batch_destroy(None)
    assert len(lib.kmc_last_error()) > 0


def test_missing_library_raises(tmp_path):
    from paper_2511_09413_gb300 import kmc
    saved = kmc._lib
    kmc._lib = None
    try:
        with pytest.raises(ImportError):
            kmc.load(str(tmp_path / "libkmc.so"))
    finally:
        kmc._lib = saved


def test_device_maps_to_the_same_quantities_on_both_sides():
    """A workloads.Device reaches the C ABI (kmc_params) and the oracle
    (OrcParams) as the same physical quantities, field by field."""
    import oracle
    from paper_2511_09413_gb300 import kmc, workloads as W
    dev = W.Device(R=7, L=33, Z=5, electrodes=1, d=0.7, dt=3e-7, T=310.0, Ea=0.37, nu=2e12,
                   alpha=0.15, kappa=0.8, k_e=4e6, rho_e=0.35, seed=-5, instance=11, rule=1)
    p = kmc.params_from_device(dev, init_mode=1, fill=0.3)
    q = oracle.params(dev)
    pairs = [("n_rails", "R"), ("n_sites", "L"), ("n_zones", "Z"), ("electrodes", "electrodes"),
             ("site_spacing_nm", "d"), ("dt_s", "dt"), ("T_K", "T"), ("Ea_eV", "Ea"),
             ("nu_Hz", "nu"), ("alpha_V", "alpha"), ("kappa", "kappa"),
             ("k_electrode_Hz", "k_e"), ("rho_electrode", "rho_e"), ("seed", "seed"),
             ("instance", "instance"), ("update_rule", "rule")]
    for a, b in pairs:
        assert getattr(p, a) == getattr(q, b), (a, b)
        assert getattr(q, b) == {"seed": (-5) & 0xFFFFFFFFFFFFFFFF}.get(b, dev.as_dict()[b])
    assert p.init_mode == 1 and p.fill == 0.3 and p.rail_base == 0
    assert kmc.params_from_device(dev.as_dict(), init_mode=0, n_ions=9).n_ions == 9


@pytest.mark.parametrize("bad,code", [
    (dict(n_rails=(1 << 20) + 1), "KMC_NOALLOC_MAX_RAILS"),
    (dict(rail_base=-1), "rail_base"),
    (dict(n_sites=1), "n_sites"),
    (dict(update_rule=3), "update_rule"),
])
def test_noalloc_rejects_bad_parameters_before_touching_a_gpu(lib, bad, code):
    """kmc_sweep_noalloc checks every argument on the host and returns
    KMC_E_ARG before any CUDA call: these run without a GPU."""
    from paper_2511_09413_gb300 import kmc
    p = _params(**bad)
    fake = ctypes.c_void_p(1 << 20)              # 16-byte aligned, never dereferenced
    rc = lib.kmc_sweep_noalloc(ctypes.byref(p), fake, 112, None, fake, 0, 5, fake, fake, None)
    assert rc == kmc.KMC_E_ARG
    assert code.encode() in lib.kmc_last_error()


def test_noalloc_checks_layout_arguments_on_the_host(lib):
    from paper_2511_09413_gb300 import kmc
    p = _params()
    fake = ctypes.c_void_p(1 << 20)
    # row stride not a multiple of 16, or shorter than a row
    assert lib.kmc_sweep_noalloc(ctypes.byref(p), fake, 100, None, fake, 0, 5, fake, fake, None) == kmc.KMC_E_ARG
    assert lib.kmc_sweep_noalloc(ctypes.byref(p), fake, 96, None, fake, 0, 5, fake, fake, None) == kmc.KMC_E_ARG
    # occupancy not 16-byte aligned
    assert lib.kmc_sweep_noalloc(ctypes.byref(p), ctypes.c_void_p((1 << 20) + 8), 112, None, fake, 0, 5,
                                 fake, fake, None) == kmc.KMC_E_ARG
    # missing voltage or trace buffers for a non-empty call
    assert lib.kmc_sweep_noalloc(ctypes.byref(p), fake, 112, None, None, 0, 5, fake, fake, None) == kmc.KMC_E_ARG
    # zero steps: nothing to do, nothing touched
    assert lib.kmc_sweep_noalloc(ctypes.byref(p), fake, 112, None, None, 0, 0, None, None, None) == kmc.KMC_OK


def test_header_states_the_contracts_it_promises():
    """The boundary's declarations carry their passages and the no-alloc entry
    point's undocumented-input rule."""
    src = open(HEADER).read()
    step = src[:src.index("int kmc_step_n(")]
    step = step[step.rindex("/*"):]
    assert "S2.1.2 - S2.1.7" in step and "Eq. 3" in step and "Eqs. 5-6" in step
    obs = src[:src.index("int kmc_observables(")]
    obs = obs[obs.rindex("/* Read observables"):]
    assert "S3" in obs and "S2.1.7" in obs
    noalloc = src[src.index("---- Sweep without any device allocation"):src.index("int kmc_sweep_noalloc(")]
    assert "other than 0 or 1 gives" in noalloc and "undefined results" in noalloc
    assert "rail_base" in src[src.index("typedef struct kmc_params"):src.index("} kmc_params;")]
