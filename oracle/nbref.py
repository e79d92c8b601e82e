"""ctypes wrapper of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. It loads ``oracle/libnbref.so`` (built on
demand by ``oracle/build.py``) and never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class RefParams(C.Structure):
    _fields_ = [
        ("G", C.c_double),
        ("m0", C.c_double),
        ("dt_rcrit", C.c_double),
        ("hill_factor", C.c_double),
        ("vel_factor", C.c_double),
        ("vel_mode", C.c_int),
        ("merge", C.c_int),
        ("bs_tol", C.c_double),
        ("bs_kmax", C.c_int),
        ("bs_max_halvings", C.c_int),
        ("kepler_max_iter", C.c_int),
        ("rcrit_refresh", C.c_int),
        ("gas", C.c_int),
        ("gas_rho0", C.c_double),
        ("gas_p", C.c_double),
        ("gas_eta", C.c_double),
        ("gas_cd", C.c_double),
        ("gas_iter", C.c_int),
        ("eject_r", C.c_double),
        ("ml_levels", C.c_int),
        ("ml_factor", C.c_int),
    ]


class RefStats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in (
        "steps", "force_evals", "encounter_pairs", "groups", "bs_substeps", "bs_halvings",
        "bs_derivs", "merges", "kepler_iters", "ejections")] + [("m_ejected", C.c_double)] + [
        (k, C.c_longlong) for k in ("ml_substeps", "ml_groups")]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.nbref_default_params.argtypes = [C.POINTER(RefParams)]
        L.nbref_changeover.argtypes = [C.c_double, C.c_double, _D, _D]
        L.nbref_stumpff.argtypes = [C.c_double, _D]
        L.nbref_kepler_drift.argtypes = [C.c_double, _D, _D, C.c_double, C.c_int, _I]
        L.nbref_kepler_drift.restype = C.c_int
        L.nbref_kepler_fg.argtypes = [C.c_double, _D, _D, C.c_double, C.c_int, _D]
        L.nbref_kepler_fg.restype = C.c_int
        L.nbref_rcrit.argtypes = [C.POINTER(RefParams), _D, _D, C.c_double]
        L.nbref_rcrit.restype = C.c_double
        L.nbref_forces.argtypes = [C.c_int, _D, _D, _D, C.c_double, _D, _I, C.c_int, _I]
        L.nbref_forces_targets.argtypes = [C.c_int, _D, _D, _D, C.c_double, _I, C.c_int, _D,
                                           _I, C.c_int, _I]
        L.nbref_bs_group.argtypes = [C.POINTER(RefParams), C.c_int, _D, _D, _D, _D, _D, _I,
                                     C.c_double, _D, C.POINTER(RefStats)]
        L.nbref_bs_group.restype = C.c_int
        L.nbref_ml_group.argtypes = L.nbref_bs_group.argtypes
        L.nbref_ml_group.restype = C.c_int
        L.nbref_create.argtypes = [C.POINTER(RefParams), C.c_int, _D, _D, _D, _D, _D, _I, _I]
        L.nbref_create.restype = C.c_void_p
        L.nbref_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.nbref_step.restype = C.c_int
        L.nbref_energy_momentum.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.nbref_n_active.argtypes = [C.c_void_p]
        L.nbref_get_state.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _I, _I]
        L.nbref_get_accel.argtypes = [C.c_void_p, _D]
        L.nbref_encounter_list.argtypes = [C.c_void_p, _I, C.c_int, _I]
        L.nbref_stats_get.argtypes = [C.c_void_p, C.POINTER(RefStats)]
        L.nbref_step_index.argtypes = [C.c_void_p]
        L.nbref_step_index.restype = C.c_longlong
        L.nbref_destroy.argtypes = [C.c_void_p]
        L.nbref_set_threads.argtypes = [C.c_int]
        L.nbref_implicit_drag.argtypes = [C.POINTER(RefParams)] + [C.c_void_p] * 3 + [
            C.c_double, C.c_double, C.c_double, C.c_void_p]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def set_threads(n: int):
    """Host threads of the oracle's OpenMP loops (results do not depend on it)."""
    lib().nbref_set_threads(int(n))


def implicit_drag(p: RefParams, x, v, Pm0, m, R, tau):
    """One body's implicit-midpoint drag update; returns (v', status)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    P = np.ascontiguousarray(Pm0, dtype=np.float64)
    out = np.zeros(3)
    st = lib().nbref_implicit_drag(C.byref(p), _dp(x), _dp(v), _dp(P), float(m), float(R),
                                   float(tau), _dp(out))
    return out, st


def params(**kw) -> RefParams:
    p = RefParams()
    lib().nbref_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def changeover(r: float, rc: float):
    K, dK = C.c_double(), C.c_double()
    lib().nbref_changeover(r, rc, C.byref(K), C.byref(dK))
    return K.value, dK.value


def stumpff(z: float) -> np.ndarray:
    c = np.zeros(4)
    lib().nbref_stumpff(z, _dp(c))
    return c


def kepler_drift(mu, x, v, h, max_iter=30):
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    it = C.c_int()
    st = lib().nbref_kepler_drift(mu, _dp(x), _dp(v), h, max_iter, C.byref(it))
    return st, x, v, it.value


def kepler_fg(mu, x, v, h, max_iter=30):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    fg = np.zeros(4)
    st = lib().nbref_kepler_fg(mu, _dp(x), _dp(v), h, max_iter, _dp(fg))
    return st, fg


def rcrit(p: RefParams, x, v, m):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().nbref_rcrit(C.byref(p), _dp(x), _dp(v), m)


def forces(x, m, rc, G=2.959122082855911e-4, cap=None):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    m = np.ascontiguousarray(m, dtype=np.float64)
    rc = np.ascontiguousarray(rc, dtype=np.float64)
    a = np.zeros((n, 3))
    cap = 16 * n + 64 if cap is None else cap
    pairs = np.zeros((cap, 2), dtype=np.int32)
    npairs = C.c_int()
    lib().nbref_forces(n, _dp(x), _dp(m), _dp(rc), G, _dp(a), _ip(pairs), cap, C.byref(npairs))
    k = npairs.value
    if k > cap:
        return forces(x, m, rc, G, cap=k)
    return a, pairs[:k].copy()


def forces_targets(x, m, rc, targets, G=2.959122082855911e-4, cap=None):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    m = np.ascontiguousarray(m, dtype=np.float64)
    rc = np.ascontiguousarray(rc, dtype=np.float64)
    t = np.ascontiguousarray(targets, dtype=np.int32)
    a = np.zeros((t.shape[0], 3))
    cap = 64 * t.shape[0] + 64 if cap is None else cap
    pairs = np.zeros((cap, 2), dtype=np.int32)
    npairs = C.c_int()
    lib().nbref_forces_targets(n, _dp(x), _dp(m), _dp(rc), G, _ip(t), t.shape[0], _dp(a),
                               _ip(pairs), cap, C.byref(npairs))
    k = npairs.value
    if k > cap:
        return forces_targets(x, m, rc, targets, G, cap=k)
    return a, pairs[:k].copy()


def bs_group(p: RefParams, x, v, m, R, rc, h, multilevel=False):
    """One group over h by the direct solver, or by the multi-level
    changeover (p.ml_levels levels) when multilevel is set."""
    x = np.array(x, dtype=np.float64).reshape(-1, 3)
    v = np.array(v, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    m = np.array(m, dtype=np.float64)
    R = np.array(R, dtype=np.float64)
    rc = np.array(rc, dtype=np.float64)
    alive = np.ones(n, dtype=np.int32)
    El = C.c_double(0.0)
    st = RefStats()
    fn = lib().nbref_ml_group if multilevel else lib().nbref_bs_group
    status = fn(C.byref(p), n, _dp(x), _dp(v), _dp(m), _dp(R), _dp(rc), _ip(alive), h,
                C.byref(El), C.byref(st))
    return dict(status=status, x=x, v=v, m=m, R=R, rc=rc, alive=alive, E_lost=El.value,
                stats={k: getattr(st, k) for k, _ in RefStats._fields_})


class RefSystem:
    """One planetary system integrated by the oracle."""

    def __init__(self, p: RefParams, x, v, m, R, rc=None, ids=None):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        n = x.shape[0]
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(n, 3)
        m = np.ascontiguousarray(m, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        rcp = None if rc is None else np.ascontiguousarray(rc, dtype=np.float64)
        idp = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        status = C.c_int()
        self.p = p
        self._h = lib().nbref_create(C.byref(p), n, _dp(x), _dp(v), _dp(m), _dp(R),
                                     None if rcp is None else _dp(rcp),
                                     None if idp is None else _ip(idp), C.byref(status))
        if not self._h:
            raise ValueError("nbref_create failed with status %d" % status.value)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().nbref_destroy(self._h)
            self._h = None

    def step(self, nsteps: int, dt: float) -> int:
        return lib().nbref_step(self._h, nsteps, dt)

    @property
    def n_active(self) -> int:
        return lib().nbref_n_active(self._h)

    @property
    def step_index(self) -> int:
        return lib().nbref_step_index(self._h)

    def state(self):
        n = self.n_active
        x = np.zeros((n, 3)); v = np.zeros((n, 3)); m = np.zeros(n); R = np.zeros(n)
        rc = np.zeros(n); ids = np.zeros(n, dtype=np.int32); na = C.c_int()
        lib().nbref_get_state(self._h, _dp(x), _dp(v), _dp(m), _dp(R), _dp(rc), _ip(ids),
                              C.byref(na))
        return dict(x=x, v=v, m=m, R=R, rc=rc, ids=ids)

    def accel(self):
        a = np.zeros((self.n_active, 3))
        lib().nbref_get_accel(self._h, _dp(a))
        return a

    def energy_momentum(self):
        E = C.c_double(); L = np.zeros(3); P = np.zeros(3); El = C.c_double()
        lib().nbref_energy_momentum(self._h, C.byref(E), _dp(L), _dp(P), C.byref(El))
        return dict(E=E.value, L=L, P=P, E_lost=El.value)

    def encounter_list(self) -> np.ndarray:
        cnt = C.c_int()
        lib().nbref_encounter_list(self._h, None, 0, C.byref(cnt))
        out = np.zeros((cnt.value, 3), dtype=np.int32)
        if cnt.value:
            lib().nbref_encounter_list(self._h, _ip(out), cnt.value, C.byref(cnt))
        return out

    def stats(self) -> dict:
        st = RefStats()
        lib().nbref_stats_get(self._h, C.byref(st))
        return {k: getattr(st, k) for k, _ in RefStats._fields_}
