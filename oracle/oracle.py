"""ctypes front end of the FP64 C oracle (kmc_oracle.c).

Test infrastructure only (tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg and reference arm): it builds and loads ``liboracle.so``
from the C source next to it.  Every function here is a thin marshalling wrapper; the
arithmetic of the method is in kmc_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmc_oracle.c")
_HDR = os.path.join(_HERE, "kmc_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INIT_STEP = 0xFFFFFFFF
MAX_ZONES = 32


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_int32), ("L", ctypes.c_int32), ("Z", ctypes.c_int32),
        ("electrodes", ctypes.c_int32),
        ("d", ctypes.c_double), ("dt", ctypes.c_double), ("T", ctypes.c_double),
        ("Ea", ctypes.c_double), ("nu", ctypes.c_double), ("alpha", ctypes.c_double),
        ("kappa", ctypes.c_double), ("k_e", ctypes.c_double), ("rho_e", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint32), ("rule", ctypes.c_int32),
    ]


class OrcLogEntry(ctypes.Structure):
    _fields_ = [
        ("rail", ctypes.c_int32), ("step", ctypes.c_uint32), ("site", ctypes.c_int32),
        ("dir", ctypes.c_int32), ("kind", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("diff", ctypes.c_double),
    ]


LOG_DTYPE = np.dtype([("rail", "<i4"), ("step", "<u4"), ("site", "<i4"), ("dir", "<i4"),
                      ("kind", "<i4"), ("pad", "<i4"), ("diff", "<f8")])


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, FP64, no contraction, OpenMP over rails)."""
    with _lock:
        fresh = (os.path.exists(_LIB)
                 and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or not fresh:
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                   "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        P = ctypes.POINTER(OrcParams)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_zone_of.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_zone_of.restype = ctypes.c_int
        L.orc_zone_widths.argtypes = [ctypes.c_int, ctypes.c_int, i32p]
        L.orc_gamma0.argtypes = [ctypes.c_double] * 3
        L.orc_gamma0.restype = ctypes.c_double
        L.orc_p0.argtypes = [ctypes.c_double] * 4
        L.orc_p0.restype = ctypes.c_double
        L.orc_p0_table.argtypes = [P, f64p, f64p]
        L.orc_hop_probs.argtypes = [ctypes.c_double] * 3 + [f64p, f64p]
        L.orc_zone_field.argtypes = [P, i32p, ctypes.c_int32, ctypes.c_double, f64p, f64p, f64p]
        L.orc_init_occupancy.argtypes = [P, ctypes.c_int, ctypes.c_int64, ctypes.c_double, i32p,
                                         u8p]
        L.orc_init_occupancy.restype = ctypes.c_int
        L.orc_run.argtypes = [P, f64p, ctypes.c_int64, ctypes.c_int64, u8p, i32p, f64p, i32p,
                              i64p, i64p, i64p, ctypes.POINTER(OrcLogEntry), ctypes.c_int64, i64p,
                              ctypes.c_int]
        L.orc_run.restype = ctypes.c_int
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_run_lr.argtypes = [P, P, f64p, ctypes.c_int64, ctypes.c_int64, u8p, i32p, f64p, f64p,
                                 i64p, i64p, f64p, f64p, f64p, i64p, ctypes.c_int, ctypes.c_int64,
                                 f64p]
        L.orc_run_lr.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def params(dev) -> OrcParams:
    """Oracle parameter block from a workloads.Device (or a dict)."""
    d = dev if isinstance(dev, dict) else dev.as_dict()
    return OrcParams(R=d["R"], L=d["L"], Z=d["Z"], electrodes=d["electrodes"], d=d["d"],
                     dt=d["dt"], T=d["T"], Ea=d["Ea"], nu=d["nu"], alpha=d["alpha"],
                     kappa=d["kappa"], k_e=d["k_e"], rho_e=d["rho_e"],
                     seed=d["seed"] & 0xFFFFFFFFFFFFFFFF, instance=d["instance"],
                     rule=d.get("rule", 0))


# ------------------------------------------------------------- primitives

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def zone_of(k: int, L: int, Z: int) -> int:
    return lib().orc_zone_of(k, L, Z)


def zone_widths(L: int, Z: int) -> np.ndarray:
    w = np.zeros(Z, dtype=np.int32)
    lib().orc_zone_widths(L, Z, _ptr(w, ctypes.c_int32))
    return w


def gamma0(nu: float, Ea: float, T: float) -> float:
    return lib().orc_gamma0(nu, Ea, T)


def p0(nu: float, Ea: float, T: float, dt: float) -> float:
    return lib().orc_p0(nu, Ea, T, dt)


def p0_table(dev, Ea_site: np.ndarray) -> np.ndarray:
    P = params(dev)
    Ea = np.ascontiguousarray(Ea_site, dtype=np.float64)
    out = np.empty(Ea.shape, dtype=np.float64)
    lib().orc_p0_table(ctypes.byref(P), _ptr(Ea, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def hop_probs(base: float, B: float, inv: float):
    """(p_left, p_right) of Eqs. 5-6 for a base probability and a zone's B."""
    pl = ctypes.c_double()
    pr = ctypes.c_double()
    lib().orc_hop_probs(float(base), float(B), float(inv), ctypes.byref(pl), ctypes.byref(pr))
    return pl.value, pr.value


def zone_field(dev, Nz, N0: int, V: float):
    """(dV, B, inv) per zone for zone counts Nz of one rail."""
    P = params(dev)
    n = np.ascontiguousarray(Nz, dtype=np.int32)
    Z = P.Z
    dV = np.empty(Z)
    B = np.empty(Z)
    inv = np.empty(Z)
    lib().orc_zone_field(ctypes.byref(P), _ptr(n, ctypes.c_int32), int(N0), float(V),
                         _ptr(dV, ctypes.c_double), _ptr(B, ctypes.c_double),
                         _ptr(inv, ctypes.c_double))
    return dV, B, inv


def _shard_rails(dev, rail_ids):
    """Global rail indices of a device that is a shard (rail_base != 0)."""
    d = dev if isinstance(dev, dict) else dev.as_dict()
    base = int(d.get("rail_base", 0))
    if rail_ids is None and base != 0:
        return np.arange(base, base + d["R"], dtype=np.int32)
    return rail_ids


def init_occupancy(dev, mode: int, n_ions: int = 0, fill: float = 0.0,
                   rail_ids: Optional[np.ndarray] = None) -> np.ndarray:
    """Initial placement; with rail_ids (Bernoulli only) the rows are those
    global rails of the device, so P.R must equal len(rail_ids).  A device
    with rail_base != 0 stands for rails [rail_base, rail_base + R)."""
    P = params(dev)
    rail_ids = _shard_rails(dev, rail_ids)
    ids = None if rail_ids is None else np.ascontiguousarray(rail_ids, dtype=np.int32)
    if ids is not None:
        P.R = len(ids)
    occ = np.zeros((P.R, P.L), dtype=np.uint8)
    rc = lib().orc_init_occupancy(ctypes.byref(P), int(mode), int(n_ions), float(fill),
                                  _ptr(ids, ctypes.c_int32), _ptr(occ, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("orc_init_occupancy failed (%d)" % rc)
    return occ


def max_threads() -> int:
    return lib().orc_max_threads()


# ------------------------------------------------------------- simulation

class OracleSim:
    """Oracle state of one device: occupancy, N0 per rail, step counter."""

    def __init__(self, dev, V: np.ndarray, occ0: np.ndarray, Ea_site: Optional[np.ndarray] = None,
                 log_cap: int = 4096, nthreads: int = 0, rail_ids: Optional[np.ndarray] = None):
        """rail_ids: global rail index of each row of occ0 (a sample of a larger
        device); by default row r is rail rail_base + r."""
        self.dev = dev
        self.P = params(dev)
        rail_ids = _shard_rails(dev, rail_ids)
        self.rail_ids = None if rail_ids is None else np.ascontiguousarray(rail_ids, dtype=np.int32)
        if self.rail_ids is not None:
            self.P.R = len(self.rail_ids)
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.occ = np.ascontiguousarray(occ0, dtype=np.uint8).reshape(self.P.R, self.P.L).copy()
        self.N0 = self.occ.sum(axis=1).astype(np.int32)
        self.P0site = None
        if Ea_site is not None:
            Ea = np.ascontiguousarray(Ea_site, dtype=np.float64).reshape(self.P.R, self.P.L)
            self.P0site = np.empty_like(Ea)
            lib().orc_p0_table(ctypes.byref(self.P), _ptr(Ea, ctypes.c_double),
                               _ptr(self.P0site, ctypes.c_double))
        self.t = 0
        self.J_rail = np.zeros(self.P.R, dtype=np.int64)
        self.log = np.zeros(log_cap, dtype=LOG_DTYPE)
        self.log_count = np.zeros(1, dtype=np.int64)
        self.nthreads = nthreads

    @classmethod
    def from_workload(cls, wl, **kw):
        dev = wl.device
        if wl.init_mode == 2:
            occ0 = wl.occ0
        else:
            occ0 = init_occupancy(dev, wl.init_mode, wl.n_ions, wl.fill)
        return cls(dev, wl.V, occ0, wl.Ea_site, **kw)

    def step_n(self, n: int):
        """Advance n steps; returns (J[n], Zc[n, Z]) for those steps."""
        P = self.P
        J = np.zeros(n, dtype=np.int64)
        Zc = np.zeros((n, P.Z), dtype=np.int64)
        rc = lib().orc_run(ctypes.byref(P), _ptr(self.V, ctypes.c_double), self.t, n,
                           _ptr(self.occ, ctypes.c_uint8), _ptr(self.N0, ctypes.c_int32),
                           _ptr(self.P0site, ctypes.c_double), _ptr(self.rail_ids, ctypes.c_int32),
                           _ptr(J, ctypes.c_int64),
                           _ptr(Zc, ctypes.c_int64), _ptr(self.J_rail, ctypes.c_int64),
                           self.log.ctypes.data_as(ctypes.POINTER(OrcLogEntry)),
                           len(self.log), _ptr(self.log_count, ctypes.c_int64), self.nthreads)
        if rc != 0:
            raise ValueError("orc_run failed (%d)" % rc)
        self.t += n
        return J, Zc

    def near_threshold_log(self) -> np.ndarray:
        n = int(min(self.log_count[0], len(self.log)))
        return self.log[:n].copy()


__all__ = ["build", "lib", "philox4x32_10", "zone_of", "zone_widths", "gamma0", "p0",
           "p0_table", "zone_field", "hop_probs", "init_occupancy", "max_threads", "OracleSim", "params",
           "INIT_STEP", "MAX_ZONES", "LOG_DTYPE", "init_score_rho", "lr_gradient"]


# ------------------------------------------------- likelihood-ratio gradient

def init_score_rho(occ0: np.ndarray, fill: float) -> np.ndarray:
    """d/drho of the log-probability of each rail's initial Bernoulli(rho)
    placement: (N0 - L rho) / (rho (1 - rho))."""
    occ = np.asarray(occ0).reshape(occ0.shape[0], -1)
    n0 = occ.sum(axis=1).astype(np.float64)
    L = occ.shape[1]
    return (n0 - L * fill) / (fill * (1.0 - fill))


def lr_gradient(dev, V: np.ndarray, occ0: np.ndarray, n_steps: int,
                wJ: Optional[np.ndarray] = None, wZ: Optional[np.ndarray] = None,
                fill: Optional[float] = None, dev_eval=None, nthreads: int = 0,
                cv_windows: int = 0) -> dict:
    """Likelihood-ratio gradient of F = sum_s wJ[s] J_s + sum_{s,z} wZ[s,z] Zc_s[z]
    over steps 0 .. n_steps-1 of a device started from occ0 (scalar barrier).

    A plain oracle run gives the totals J_s, Zc_s; orc_run_lr then replays the
    same trajectory and accumulates the per-rail estimator.  The gradient is
    with respect to (Ea, nu, kappa, rho); the rho entry is NaN unless fill
    (the Bernoulli filling that produced occ0) is given.  Returns a dict with
    grad, stderr (from the spread of the independent per-rail terms), G (per
    rail), S (cumulative score per rail), loglik (per rail, at dev_eval or dev)
    and J (the replayed totals).

    With cv_windows = K > 0 it also returns the state-dependent control
    variate's features (orc_run_lr's cv_out, [R][2][K][Z + 2]: the Ea and
    kappa score increments of each of K equal time windows times the
    step-start features 1, first moment / L and zone counts) and grad_cv,
    stderr_cv, G_cv: the per-rail terms less their cross-fitted linear
    prediction from those features (`cross_fit`), for Ea and nu from the Ea
    features and for kappa from the kappa features; rho is left as is."""
    P = params(dev)
    Pe = params(dev_eval if dev_eval is not None else dev)
    occ = np.ascontiguousarray(occ0, dtype=np.uint8).reshape(P.R, P.L).copy()
    Vc = np.ascontiguousarray(V, dtype=np.float64)
    fwd = OracleSim(dev, Vc, occ, nthreads=nthreads)
    J_tot, Zc_tot = fwd.step_n(n_steps)
    N0 = occ.sum(axis=1).astype(np.int32)
    S = np.zeros((P.R, 4))
    if fill is not None:
        S[:, 3] = init_score_rho(occ, fill)
    G = np.zeros((P.R, 4))
    ll = np.zeros(P.R)
    J = np.zeros(n_steps, dtype=np.int64)
    wJc = None if wJ is None else np.ascontiguousarray(wJ, dtype=np.float64)
    wZc = None if wZ is None else np.ascontiguousarray(wZ, dtype=np.float64).reshape(n_steps, P.Z)
    cv = None
    window = 0
    if cv_windows > 0:
        window = -(-n_steps // cv_windows)
        K = -(-n_steps // window)
        cv = np.zeros((P.R, 2, K, P.Z + 2))
    rc = lib().orc_run_lr(ctypes.byref(P), ctypes.byref(Pe), _ptr(Vc, ctypes.c_double), 0,
                          n_steps, _ptr(occ, ctypes.c_uint8), _ptr(N0, ctypes.c_int32),
                          _ptr(wJc, ctypes.c_double), _ptr(wZc, ctypes.c_double),
                          _ptr(J_tot, ctypes.c_int64), _ptr(Zc_tot, ctypes.c_int64),
                          _ptr(S, ctypes.c_double), _ptr(G, ctypes.c_double),
                          _ptr(ll, ctypes.c_double), _ptr(J, ctypes.c_int64), nthreads,
                          window, _ptr(cv, ctypes.c_double))
    if rc != 0:
        raise ValueError("orc_run_lr failed (%d)" % rc)
    R = P.R

    def summary(T):
        g = T.sum(axis=0)
        se = np.sqrt(R / max(R - 1, 1) * ((T - T.mean(axis=0)) ** 2).sum(axis=0))
        if fill is None:
            g[3] = np.nan
            se[3] = np.nan
        return g, se

    grad, stderr = summary(G)
    out = {"grad": grad, "stderr": stderr, "G": G, "S": S, "loglik": ll, "J": J,
           "J_tot": J_tot, "Zc_tot": Zc_tot}
    if cv is not None:
        Xe = cv[:, 0].reshape(R, -1)
        Xk = cv[:, 1].reshape(R, -1)
        G_cv = G.copy()
        G_cv[:, 0] = cross_fit(G[:, 0], Xe)
        G_cv[:, 1] = cross_fit(G[:, 1], Xe)
        G_cv[:, 2] = cross_fit(G[:, 2], Xk)
        out["cv"] = cv
        out["G_cv"] = G_cv
        out["grad_cv"], out["stderr_cv"] = summary(G_cv)
    return out


def cross_fit(y: np.ndarray, X: np.ndarray) -> np.ndarray:
    """y less its cross-fitted linear prediction from zero-mean features X
    (one row per rail): the coefficients for the even rails are fitted (least
    squares with an intercept) on the odd rails and vice versa, so each rail's
    correction is independent of its own terms, and since E[X] = 0 the sum of
    the corrected terms keeps the expectation of the sum of y."""
    y = np.asarray(y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    out = y.copy()
    idx = np.arange(len(y))
    for half in (0, 1):
        fit, app = idx % 2 != half, idx % 2 == half
        if fit.sum() <= X.shape[1] + 1 or not app.any():
            continue
        Xf = X[fit] - X[fit].mean(axis=0)
        beta = np.linalg.lstsq(Xf, y[fit] - y[fit].mean(), rcond=None)[0]
        out[app] = y[app] - X[app] @ beta
    return out
