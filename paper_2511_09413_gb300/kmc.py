"""Python binding of the C ABI in include/kmc.h (argument marshalling only).

The functions keep the C names (``kmc_create``, ``kmc_step_n``,
``kmc_observables`` ...).  Every step of the simulation runs in the CUDA
kernels of ``libkmc.so``; this module never computes any part of it.  PyTorch
supplies the CUDA stream and, through ``kmc_set_allocator``, device memory
from its caching allocator.

If ``libkmc.so`` is missing or cannot be loaded, importing the binding raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkmc.so")

KMC_OK = 0
KMC_E_ARG = -1
KMC_E_PROB = -2
KMC_E_NOMEM = -3
KMC_E_CUDA = -4
KMC_E_TIMEOUT = -5
KMC_E_RANGE = -6
KMC_MAX_SITES = 2048
KMC_MAX_ZONES = 32


class KmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("kmc error %d: %s" % (code, msg))
        self.code = code


class kmc_params(ctypes.Structure):
    _fields_ = [
        ("n_rails", ctypes.c_int32), ("n_sites", ctypes.c_int32), ("n_zones", ctypes.c_int32),
        ("electrodes", ctypes.c_int32),
        ("site_spacing_nm", ctypes.c_double), ("dt_s", ctypes.c_double), ("T_K", ctypes.c_double),
        ("Ea_eV", ctypes.c_double), ("nu_Hz", ctypes.c_double), ("alpha_V", ctypes.c_double),
        ("kappa", ctypes.c_double), ("k_electrode_Hz", ctypes.c_double),
        ("rho_electrode", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint32), ("init_mode", ctypes.c_int32),
        ("n_ions", ctypes.c_int64), ("fill", ctypes.c_double),
        ("update_rule", ctypes.c_int32), ("rail_base", ctypes.c_int32),
    ]


class kmc_log_entry(ctypes.Structure):
    _fields_ = [
        ("rail", ctypes.c_int32), ("step", ctypes.c_uint32), ("site", ctypes.c_int32),
        ("dir", ctypes.c_int32), ("kind", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("diff", ctypes.c_double),
    ]


LOG_DTYPE = np.dtype([("rail", "<i4"), ("step", "<u4"), ("site", "<i4"), ("dir", "<i4"),
                      ("kind", "<i4"), ("pad", "<i4"), ("diff", "<f8")])

kmc_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
kmc_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                               ctypes.c_void_p)

# every symbol include/kmc.h declares
EXPORTS = ["kmc_set_allocator", "kmc_create", "kmc_step_n", "kmc_observables", "kmc_set_voltage",
           "kmc_near_threshold_log", "kmc_counters", "kmc_set_launch", "kmc_current_step",
           "kmc_destroy", "kmc_last_error", "kmc_sweep_noalloc", "kmc_batch_create",
           "kmc_batch_step_n", "kmc_batch_observables", "kmc_batch_set_launch", "kmc_batch_tune",
           "kmc_batch_current_step", "kmc_batch_destroy", "kmc_set_accept_path",
           "kmc_accept_path", "kmc_batch_set_accept_path", "kmc_batch_accept_path", "kmc_grad",
           "kmc_batch_grad", "kmc_philox_probe", "kmc_batch_grad_all", "kmc_rail_current",
           "kmc_batch_rail_current"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libkmc.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libkmc.so not built at %s: run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    P = ctypes.POINTER
    L.kmc_set_allocator.argtypes = [kmc_alloc_fn, kmc_free_fn, vp]
    L.kmc_create.argtypes = [P(kmc_params), P(ctypes.c_double), i64, P(ctypes.c_uint8),
                             P(ctypes.c_double), vp, P(vp)]
    L.kmc_step_n.argtypes = [vp, i64]
    L.kmc_observables.argtypes = [vp, i64, i64, P(ctypes.c_int64), P(ctypes.c_int64),
                                  P(ctypes.c_uint8)]
    L.kmc_set_voltage.argtypes = [vp, i64, i64, P(ctypes.c_double)]
    L.kmc_rail_current.argtypes = [vp, P(ctypes.c_int64)]
    L.kmc_rail_current.restype = ctypes.c_int
    L.kmc_batch_rail_current.argtypes = [vp, ctypes.c_int32, P(ctypes.c_int64)]
    L.kmc_batch_rail_current.restype = ctypes.c_int
    L.kmc_near_threshold_log.argtypes = [vp, P(kmc_log_entry), i64, P(ctypes.c_int64)]
    L.kmc_counters.argtypes = [vp, P(ctypes.c_uint64)]
    L.kmc_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.kmc_current_step.argtypes = [vp]
    L.kmc_current_step.restype = i64
    L.kmc_destroy.argtypes = [vp]
    L.kmc_destroy.restype = None
    L.kmc_last_error.restype = ctypes.c_char_p
    L.kmc_sweep_noalloc.argtypes = [P(kmc_params), vp, i64, vp, vp, i64, i64, vp, vp, vp]
    L.kmc_sweep_noalloc.restype = ctypes.c_int
    L.kmc_batch_create.argtypes = [P(kmc_params), ctypes.c_int32, P(P(ctypes.c_double)), i64,
                                   P(P(ctypes.c_uint8)), P(P(ctypes.c_double)), vp, P(vp)]
    L.kmc_batch_step_n.argtypes = [vp, i64]
    L.kmc_batch_observables.argtypes = [vp, ctypes.c_int32, i64, i64, P(ctypes.c_int64),
                                        P(ctypes.c_int64), P(ctypes.c_uint8)]
    L.kmc_batch_set_launch.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    L.kmc_batch_tune.argtypes = [vp, i64, P(ctypes.c_int32), P(ctypes.c_int32)]
    L.kmc_batch_current_step.argtypes = [vp]
    L.kmc_batch_current_step.restype = i64
    L.kmc_batch_destroy.argtypes = [vp]
    L.kmc_batch_destroy.restype = None
    L.kmc_grad.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                           P(ctypes.c_double)]
    L.kmc_batch_grad_all.argtypes = [vp, P(P(ctypes.c_double)), P(P(ctypes.c_double)),
                                     P(ctypes.c_double), P(ctypes.c_double)]
    L.kmc_batch_grad_all.restype = ctypes.c_int
    L.kmc_philox_probe.argtypes = [vp, P(ctypes.c_double)]
    L.kmc_philox_probe.restype = ctypes.c_int
    L.kmc_batch_grad.argtypes = [vp, ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double),
                                 P(ctypes.c_double), P(ctypes.c_double)]
    L.kmc_batch_grad.restype = ctypes.c_int
    L.kmc_set_accept_path.argtypes = [vp, ctypes.c_int]
    L.kmc_accept_path.argtypes = [vp]
    L.kmc_batch_set_accept_path.argtypes = [vp, ctypes.c_int32]
    L.kmc_batch_accept_path.argtypes = [vp]
    for name in ("kmc_batch_create", "kmc_batch_step_n", "kmc_batch_observables",
                 "kmc_batch_set_launch", "kmc_batch_tune", "kmc_set_accept_path",
                 "kmc_accept_path", "kmc_batch_set_accept_path", "kmc_batch_accept_path",
                 "kmc_grad"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("kmc_set_allocator", "kmc_create", "kmc_step_n", "kmc_observables",
                 "kmc_set_voltage", "kmc_near_threshold_log", "kmc_counters", "kmc_set_launch"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != KMC_OK:
        raise KmcError(rc, load().kmc_last_error().decode(errors="replace"))


def _ptr(a: Optional[np.ndarray], ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


# ------------------------------------------------------------------ C names

def kmc_set_allocator(alloc, free_fn, ctx=None):
    _check(load().kmc_set_allocator(alloc, free_fn, ctx))


def kmc_create(params: kmc_params, V_per_step: np.ndarray, init_occ: Optional[np.ndarray] = None,
               Ea_site: Optional[np.ndarray] = None, stream: int = 0) -> int:
    V = np.ascontiguousarray(V_per_step, dtype=np.float64)
    occ = None if init_occ is None else np.ascontiguousarray(init_occ, dtype=np.uint8)
    Ea = None if Ea_site is None else np.ascontiguousarray(Ea_site, dtype=np.float64)
    n = params.n_rails * params.n_sites
    if occ is not None and occ.size != n:
        raise ValueError("init_occ must have n_rails * n_sites entries")
    if Ea is not None and Ea.size != n:
        raise ValueError("Ea_site must have n_rails * n_sites entries")
    h = ctypes.c_void_p()
    _check(load().kmc_create(ctypes.byref(params), _ptr(V, ctypes.c_double), V.shape[0],
                             _ptr(occ, ctypes.c_uint8), _ptr(Ea, ctypes.c_double),
                             ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def kmc_step_n(h: int, n_steps: int):
    _check(load().kmc_step_n(ctypes.c_void_p(h), int(n_steps)))


def kmc_observables(h: int, first_step: int, count: int, J_out: Optional[np.ndarray],
                    zone_counts_out: Optional[np.ndarray], occ_out: Optional[np.ndarray]):
    _check(load().kmc_observables(ctypes.c_void_p(h), int(first_step), int(count),
                                  _ptr(J_out, ctypes.c_int64), _ptr(zone_counts_out, ctypes.c_int64),
                                  _ptr(occ_out, ctypes.c_uint8)))


def kmc_rail_current(h: int, n_rails: int) -> np.ndarray:
    out = np.zeros(n_rails, dtype=np.int64)
    _check(load().kmc_rail_current(ctypes.c_void_p(h), _ptr(out, ctypes.c_int64)))
    return out


def kmc_set_voltage(h: int, first_step: int, V_host: np.ndarray):
    V = np.ascontiguousarray(V_host, dtype=np.float64)
    _check(load().kmc_set_voltage(ctypes.c_void_p(h), int(first_step), V.shape[0],
                                  _ptr(V, ctypes.c_double)))


def kmc_near_threshold_log(h: int, cap: int = 4096, with_total: bool = False):
    """Logged near-threshold decisions (at most cap); with_total also returns
    how many were logged in all (more than returned if the log overflowed)."""
    buf = np.zeros(cap, dtype=LOG_DTYPE)
    n = ctypes.c_int64()
    _check(load().kmc_near_threshold_log(ctypes.c_void_p(h),
                                         buf.ctypes.data_as(ctypes.POINTER(kmc_log_entry)), cap,
                                         ctypes.byref(n)))
    out = buf[:min(n.value, cap)].copy()
    return (out, int(n.value)) if with_total else out


def kmc_counters(h: int) -> np.ndarray:
    out = np.zeros(3, dtype=np.uint64)
    _check(load().kmc_counters(ctypes.c_void_p(h), _ptr(out, ctypes.c_uint64)))
    return out


def kmc_set_launch(h: int, warps_per_cta: int = 0, flush_steps: int = 0):
    _check(load().kmc_set_launch(ctypes.c_void_p(h), int(warps_per_cta), int(flush_steps)))


def kmc_grad(h: int, n: int, Z: int, dLoss_dJ: Optional[np.ndarray] = None,
             dLoss_dZc: Optional[np.ndarray] = None):
    """(grad[4], stderr[4]) of E[F] with respect to (Ea, nu, kappa, fill) for
    F = sum_s dLoss_dJ[s] J_s + sum_{s,z} dLoss_dZc[s, z] Zc_s[z] over the n
    steps simulated so far."""
    wJ = None if dLoss_dJ is None else np.ascontiguousarray(dLoss_dJ, dtype=np.float64)
    wZ = None if dLoss_dZc is None else np.ascontiguousarray(dLoss_dZc, dtype=np.float64)
    if wJ is not None and wJ.shape != (n,):
        raise ValueError("dLoss_dJ must have shape (%d,)" % n)
    if wZ is not None and wZ.shape != (n, Z):
        raise ValueError("dLoss_dZc must have shape (%d, %d)" % (n, Z))
    g = np.zeros(4)
    se = np.zeros(4)
    _check(load().kmc_grad(ctypes.c_void_p(h), _ptr(wJ, ctypes.c_double), _ptr(wZ, ctypes.c_double),
                           _ptr(g, ctypes.c_double), _ptr(se, ctypes.c_double)))
    return g, se


def kmc_set_accept_path(h: int, mode: int = -1):
    _check(load().kmc_set_accept_path(ctypes.c_void_p(h), int(mode)))


def kmc_accept_path(h: int) -> int:
    return int(load().kmc_accept_path(ctypes.c_void_p(h)))


def kmc_current_step(h: int) -> int:
    return int(load().kmc_current_step(ctypes.c_void_p(h)))


def kmc_destroy(h: int):
    load().kmc_destroy(ctypes.c_void_p(h))


def kmc_last_error() -> str:
    return load().kmc_last_error().decode(errors="replace")


def kmc_sweep_noalloc(params: kmc_params, occ_dev: int, row_stride: int, N0_dev: Optional[int],
                      V_dev: int, t0: int, n_steps: int, J_dev: int, zone_counts_dev: int,
                      stream: int = 0):
    """Advance caller-owned device state without allocating (device pointers
    as integers, e.g. torch ``tensor.data_ptr()``); see include/kmc.h."""
    _check(load().kmc_sweep_noalloc(ctypes.byref(params), ctypes.c_void_p(occ_dev), int(row_stride),
                                    ctypes.c_void_p(N0_dev) if N0_dev else None,
                                    ctypes.c_void_p(V_dev), int(t0), int(n_steps),
                                    ctypes.c_void_p(J_dev), ctypes.c_void_p(zone_counts_dev),
                                    ctypes.c_void_p(stream)))


# ------------------------------------------------------------ conveniences

def params_from_device(dev, init_mode: int, n_ions: int = 0, fill: float = 0.0) -> kmc_params:
    """kmc_params from a workloads.Device (or an equivalent dict)."""
    d = dev if isinstance(dev, dict) else dev.as_dict()
    return kmc_params(n_rails=d["R"], n_sites=d["L"], n_zones=d["Z"], electrodes=d["electrodes"],
                      site_spacing_nm=d["d"], dt_s=d["dt"], T_K=d["T"], Ea_eV=d["Ea"],
                      nu_Hz=d["nu"], alpha_V=d["alpha"], kappa=d["kappa"],
                      k_electrode_Hz=d["k_e"], rho_electrode=d["rho_e"],
                      seed=d["seed"] & 0xFFFFFFFFFFFFFFFF, instance=d["instance"],
                      init_mode=init_mode, n_ions=n_ions, fill=fill,
                      update_rule=d.get("rule", 0), rail_base=d.get("rail_base", 0))


_torch_alloc_cb = None


def use_torch_allocator(device: int = 0):
    """Route libkmc device allocations through PyTorch's caching allocator."""
    global _torch_alloc_cb
    import torch

    def _alloc(nbytes, stream, ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _torch_alloc_cb = (kmc_alloc_fn(_alloc), kmc_free_fn(_free))
    kmc_set_allocator(_torch_alloc_cb[0], _torch_alloc_cb[1], None)


class Sim:
    """One device on the GPU behind a kmc handle."""

    def __init__(self, dev, V: np.ndarray, init_mode: int, n_ions: int = 0, fill: float = 0.0,
                 occ0: Optional[np.ndarray] = None, Ea_site: Optional[np.ndarray] = None,
                 stream: Optional[int] = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.params = params_from_device(dev, init_mode, n_ions, fill)
        self.R, self.L, self.Z = self.params.n_rails, self.params.n_sites, self.params.n_zones
        self.h = kmc_create(self.params, V, occ0, Ea_site, stream)
        self.n_total = int(np.asarray(V).shape[0])

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.device, wl.V, wl.init_mode, wl.n_ions, wl.fill, wl.occ0, wl.Ea_site, **kw)

    @property
    def t(self) -> int:
        return kmc_current_step(self.h)

    def step_n(self, n: int):
        kmc_step_n(self.h, n)

    def traces(self, first: int = 0, count: Optional[int] = None):
        count = self.t - first if count is None else count
        J = np.zeros(count, dtype=np.int64)
        Zc = np.zeros((count, self.Z), dtype=np.int64)
        kmc_observables(self.h, first, count, J, Zc, None)
        return J, Zc

    def occupancy(self) -> np.ndarray:
        occ = np.zeros((self.R, self.L), dtype=np.uint8)
        kmc_observables(self.h, 0, 0, None, None, occ)
        return occ

    def rail_current(self) -> np.ndarray:
        """Net leftward crossings of each rail over every step so far (kmc_rail_current)."""
        return kmc_rail_current(self.h, self.R)

    def grad(self, dLoss_dJ: Optional[np.ndarray] = None, dLoss_dZc: Optional[np.ndarray] = None):
        """Likelihood-ratio gradient of E[F] (kmc_grad): (grad[4], stderr[4])
        with respect to (Ea, nu, kappa, fill)."""
        return kmc_grad(self.h, self.t, self.Z, dLoss_dJ, dLoss_dZc)

    def near_threshold_log(self, cap: int = 4096, with_total: bool = False):
        return kmc_near_threshold_log(self.h, cap, with_total)

    def counters(self) -> np.ndarray:
        return kmc_counters(self.h)

    def set_launch(self, warps_per_cta: int = 0, flush_steps: int = 0):
        kmc_set_launch(self.h, warps_per_cta, flush_steps)

    def set_accept_path(self, mode: int = -1):
        kmc_set_accept_path(self.h, mode)

    @property
    def accept_path(self) -> int:
        return kmc_accept_path(self.h)

    def close(self):
        if getattr(self, "h", None):
            kmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- batches

def kmc_batch_create(params_list, V_list, init_occ_list=None, stream: int = 0,
                     Ea_site_list=None) -> int:
    n = len(params_list)
    P = (kmc_params * n)(*params_list)
    Vs = [np.ascontiguousarray(v, dtype=np.float64) for v in V_list]
    n_total = Vs[0].shape[0]
    if any(v.shape[0] != n_total for v in Vs):
        raise ValueError("all voltage tables of a batch have the same length")
    Vp = (ctypes.POINTER(ctypes.c_double) * n)(*[_ptr(v, ctypes.c_double) for v in Vs])
    occs = None
    Op = None
    if init_occ_list is not None:
        occs = [None if o is None else np.ascontiguousarray(o, dtype=np.uint8) for o in init_occ_list]
        Op = (ctypes.POINTER(ctypes.c_uint8) * n)(*[_ptr(o, ctypes.c_uint8) for o in occs])
    eas = None
    Ep = None
    if Ea_site_list is not None:
        eas = [None if e is None else np.ascontiguousarray(e, dtype=np.float64) for e in Ea_site_list]
        for p, e in zip(params_list, eas):
            if e is not None and e.size != p.n_rails * p.n_sites:
                raise ValueError("Ea_site must have n_rails * n_sites entries")
        Ep = (ctypes.POINTER(ctypes.c_double) * n)(*[_ptr(e, ctypes.c_double) for e in eas])
    h = ctypes.c_void_p()
    _check(load().kmc_batch_create(P, n, Vp, n_total, Op, Ep, ctypes.c_void_p(stream),
                                   ctypes.byref(h)))
    return h.value


def kmc_batch_step_n(b: int, n_steps: int):
    _check(load().kmc_batch_step_n(ctypes.c_void_p(b), int(n_steps)))


def kmc_batch_observables(b: int, inst: int, first_step: int, count: int,
                          J_out: Optional[np.ndarray], zone_counts_out: Optional[np.ndarray],
                          occ_out: Optional[np.ndarray]):
    _check(load().kmc_batch_observables(ctypes.c_void_p(b), int(inst), int(first_step), int(count),
                                        _ptr(J_out, ctypes.c_int64),
                                        _ptr(zone_counts_out, ctypes.c_int64),
                                        _ptr(occ_out, ctypes.c_uint8)))


def kmc_batch_rail_current(b: int, inst: int, n_rails: int) -> np.ndarray:
    out = np.zeros(n_rails, dtype=np.int64)
    _check(load().kmc_batch_rail_current(ctypes.c_void_p(b), int(inst), _ptr(out, ctypes.c_int64)))
    return out


def kmc_batch_set_launch(b: int, warps_per_cta: int, steps_per_launch: int):
    _check(load().kmc_batch_set_launch(ctypes.c_void_p(b), int(warps_per_cta), int(steps_per_launch)))


def kmc_batch_tune(b: int, probe_steps: int):
    w = ctypes.c_int32()
    st = ctypes.c_int32()
    _check(load().kmc_batch_tune(ctypes.c_void_p(b), int(probe_steps), ctypes.byref(w),
                                 ctypes.byref(st)))
    return w.value, st.value


def kmc_batch_set_accept_path(b: int, mode: int = -1):
    _check(load().kmc_batch_set_accept_path(ctypes.c_void_p(b), int(mode)))


def kmc_batch_accept_path(b: int) -> int:
    return int(load().kmc_batch_accept_path(ctypes.c_void_p(b)))


def kmc_batch_grad(b: int, inst: int, n: int, Z: int, dLoss_dJ: Optional[np.ndarray] = None,
                   dLoss_dZc: Optional[np.ndarray] = None):
    """(grad[4], stderr[4]) for device inst of a batch, as kmc_grad."""
    wJ = None if dLoss_dJ is None else np.ascontiguousarray(dLoss_dJ, dtype=np.float64)
    wZ = None if dLoss_dZc is None else np.ascontiguousarray(dLoss_dZc, dtype=np.float64)
    if wJ is not None and wJ.shape != (n,):
        raise ValueError("dLoss_dJ must have shape (%d,)" % n)
    if wZ is not None and wZ.shape != (n, Z):
        raise ValueError("dLoss_dZc must have shape (%d, %d)" % (n, Z))
    g = np.zeros(4)
    se = np.zeros(4)
    _check(load().kmc_batch_grad(ctypes.c_void_p(b), int(inst), _ptr(wJ, ctypes.c_double),
                                 _ptr(wZ, ctypes.c_double), _ptr(g, ctypes.c_double),
                                 _ptr(se, ctypes.c_double)))
    return g, se


def kmc_batch_grad_all(b: int, shapes, n: int, dLoss_dJ=None, dLoss_dZc=None):
    """(grad [n_inst, 4], stderr [n_inst, 4]) of every device in one launch;
    dLoss_dJ / dLoss_dZc are sequences (entries may be None) or None."""
    k = len(shapes)
    keep = []

    def table(ws, shape_of):
        if ws is None:
            return None
        arr = (ctypes.POINTER(ctypes.c_double) * k)()
        for i, w in enumerate(ws):
            if w is None:
                continue
            a = np.ascontiguousarray(w, dtype=np.float64)
            if a.shape != shape_of(i):
                raise ValueError("weights of device %d must have shape %s" % (i, shape_of(i)))
            keep.append(a)
            arr[i] = _ptr(a, ctypes.c_double)
        return arr

    tJ = table(dLoss_dJ, lambda i: (n,))
    tZ = table(dLoss_dZc, lambda i: (n, shapes[i][2]))
    g = np.zeros((k, 4))
    se = np.zeros((k, 4))
    _check(load().kmc_batch_grad_all(ctypes.c_void_p(b), tJ, tZ, _ptr(g, ctypes.c_double),
                                     _ptr(se, ctypes.c_double)))
    return g, se


def kmc_philox_probe(stream: Optional[int] = None) -> float:
    """Philox4x32-10 blocks per second with no other work (kmc_philox_probe)."""
    out = ctypes.c_double()
    _check(load().kmc_philox_probe(ctypes.c_void_p(stream or 0), ctypes.byref(out)))
    return out.value


def kmc_batch_current_step(b: int) -> int:
    return int(load().kmc_batch_current_step(ctypes.c_void_p(b)))


def kmc_batch_destroy(b: int):
    load().kmc_batch_destroy(ctypes.c_void_p(b))


class Batch:
    """Many devices advanced together: per chunk of steps, one persistent launch
    per tile shape."""

    def __init__(self, devs, Vs, init_modes, n_ions=None, fills=None, occ0s=None,
                 stream: Optional[int] = None, Ea_sites=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        n = len(devs)
        n_ions = n_ions or [0] * n
        fills = fills or [0.0] * n
        self.params = [params_from_device(d, m, ni, f)
                       for d, m, ni, f in zip(devs, init_modes, n_ions, fills)]
        self.shapes = [(p.n_rails, p.n_sites, p.n_zones) for p in self.params]
        self.h = kmc_batch_create(self.params, Vs, occ0s, stream, Ea_sites)

    @property
    def t(self) -> int:
        return kmc_batch_current_step(self.h)

    def step_n(self, n: int):
        kmc_batch_step_n(self.h, n)

    def tune(self, probe_steps: int):
        return kmc_batch_tune(self.h, probe_steps)

    def set_launch(self, warps_per_cta: int, steps_per_launch: int):
        kmc_batch_set_launch(self.h, warps_per_cta, steps_per_launch)

    def set_accept_path(self, mode: int = -1):
        kmc_batch_set_accept_path(self.h, mode)

    def grad_all(self, dLoss_dJ=None, dLoss_dZc=None):
        """Gradients of every device, one persistent launch per tile shape
        (kmc_batch_grad_all)."""
        return kmc_batch_grad_all(self.h, self.shapes, self.t, dLoss_dJ, dLoss_dZc)

    def grad(self, inst: int, dLoss_dJ: Optional[np.ndarray] = None,
             dLoss_dZc: Optional[np.ndarray] = None):
        """Likelihood-ratio gradient of device inst (kmc_batch_grad)."""
        R, L, Z = self.shapes[inst]
        return kmc_batch_grad(self.h, inst, self.t, Z, dLoss_dJ, dLoss_dZc)

    @property
    def accept_path(self) -> int:
        return kmc_batch_accept_path(self.h)

    def traces(self, inst: int, first: int = 0, count: Optional[int] = None):
        R, L, Z = self.shapes[inst]
        count = self.t - first if count is None else count
        J = np.zeros(count, dtype=np.int64)
        Zc = np.zeros((count, Z), dtype=np.int64)
        kmc_batch_observables(self.h, inst, first, count, J, Zc, None)
        return J, Zc

    def occupancy(self, inst: int) -> np.ndarray:
        R, L, Z = self.shapes[inst]
        occ = np.zeros((R, L), dtype=np.uint8)
        kmc_batch_observables(self.h, inst, 0, 0, None, None, occ)
        return occ

    def rail_current(self, inst: int) -> np.ndarray:
        return kmc_batch_rail_current(self.h, inst, self.shapes[inst][0])

    def close(self):
        if getattr(self, "h", None):
            kmc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
