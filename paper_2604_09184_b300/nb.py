"""Thin ctypes binding of libnb.so (include/nb.h).

Argument marshalling only: every step of the integrator runs in the library's
CUDA kernels. PyTorch provides the device memory (the workspace is a uint8
CUDA tensor) and the stream. A missing library or a missing GPU raises; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# NB_DEBUG=1 selects the debug build (index checks that report NB_E_INVALID)
LIB_PATH = os.path.join(_HERE, "libnb_debug.so" if os.environ.get("NB_DEBUG") == "1"
                        else "libnb.so")

NB_OK = 0
NB_E_INVALID = -1
NB_E_CUDA = -2
NB_E_OVERFLOW = -3
NB_E_NOCONV = -4
NB_E_TIMEOUT = -5
NB_E_WORKSPACE = -6
NB_PREC_FP64 = 0
NB_PREC_MIXED = 1
NB_PREC_DS = 2
NB_MATH_EXP, NB_MATH_RCP, NB_MATH_RSQRT, NB_MATH_RPOW32 = 0, 1, 2, 3
NB_MATH_RPOW32_MIXED, NB_MATH_RPOW32_M, NB_MATH_CLOSE_WEIGHT = 4, 5, 6
NB_MATH_MASS15, NB_MATH_MASS1875, NB_MATH_NEVILLE, NB_MATH_RATIO_LE = 7, 8, 9, 10
NB_MATH_RINV3 = 11


class NbParams(C.Structure):
    _fields_ = [
        ("G", C.c_double), ("m0", C.c_double), ("dt_rcrit", C.c_double),
        ("hill_factor", C.c_double), ("vel_factor", C.c_double),
        ("vel_mode", C.c_int), ("merge", C.c_int), ("precision", C.c_int),
        ("kepler_max_iter", C.c_int), ("bs_tol", C.c_double), ("bs_kmax", C.c_int),
        ("bs_max_halvings", C.c_int), ("pair_capacity", C.c_int), ("log_capacity", C.c_int),
        ("kick_split", C.c_int), ("rcrit_refresh", C.c_int),
        ("gas", C.c_int), ("gas_rho0", C.c_double), ("gas_p", C.c_double),
        ("gas_eta", C.c_double), ("gas_cd", C.c_double), ("gas_iter", C.c_int),
        ("eject_r", C.c_double), ("bs_cluster_min", C.c_int), ("ml_levels", C.c_int),
        ("ml_factor", C.c_int), ("bs_speculate", C.c_int), ("kick_symmetric", C.c_int),
    ]


class NbStats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in (
        "steps", "force_evals", "encounter_pairs", "groups", "bs_substeps", "bs_halvings",
        "bs_derivs", "merges", "kepler_iters", "moved_bodies", "log_dropped")] + [
        ("n_active", C.c_int), ("last_pairs", C.c_int), ("ejections", C.c_longlong),
        ("m_ejected", C.c_double), ("ml_substeps", C.c_longlong), ("ml_groups", C.c_longlong),
        ("kick_symmetric", C.c_int)]


# nb_allgather_fn: int (*)(void* user, const void* send, void* recv, size_t bytes, void* stream)
ALLGATHER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class NbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (status_string(code), code, msg))
        self.code = code


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_lib = None


def lib():
    """Load libnb.so (built in-tree by paper_2604_09184_b300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is missing: run `python -m paper_2604_09184_b300.build%s`"
                              % (os.path.basename(LIB_PATH),
                                 " --debug" if LIB_PATH.endswith("_debug.so") else ""))
        L = C.CDLL(LIB_PATH)
        L.nb_default_params.argtypes = [C.POINTER(NbParams)]
        L.nb_workspace_bytes.argtypes = [C.POINTER(NbParams), C.c_int]
        L.nb_workspace_bytes.restype = C.c_size_t
        L.nb_init_system.argtypes = [C.POINTER(C.c_void_p), C.POINTER(NbParams), C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_int]
        L.nb_set_fsal.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.nb_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.nb_set_state.argtypes = [C.c_void_p] + [C.c_void_p] * 8 + [C.c_int, C.c_int]
        L.nb_set_timing.argtypes = [C.c_void_p, C.c_int]
        L.nb_timing.argtypes = [C.c_void_p, _D, C.POINTER(C.c_longlong),
                                C.POINTER(C.c_longlong)]
        L.nb_energy_momentum.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.nb_get_state.argtypes = [C.c_void_p] + [C.c_void_p] * 6 + [_I, C.c_int]
        L.nb_get_fsal.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, _I, C.c_int]
        L.nb_encounter_list.argtypes = [C.c_void_p, C.c_void_p, C.c_int, _I]
        L.nb_stats.argtypes = [C.c_void_p, C.POINTER(NbStats)]
        L.nb_destroy.argtypes = [C.c_void_p]
        L.nb_last_error.argtypes = [C.c_void_p]
        L.nb_last_error.restype = C.c_char_p
        L.nb_status_string.argtypes = [C.c_int]
        L.nb_status_string.restype = C.c_char_p
        L.nb_kick_scratch_bytes.argtypes = [C.c_int, C.c_int]
        L.nb_kick_scratch_bytes.restype = C.c_size_t
        L.nb_kick.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                              C.c_int, C.c_void_p, C.c_void_p, C.c_int, _I, C.c_void_p,
                              C.c_size_t, C.c_void_p]
        L.nb_kick_rows.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                   _I, C.c_void_p, C.c_size_t, C.c_void_p]
        L.nb_kick_noalloc.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                      C.c_int, C.c_void_p, C.c_void_p, C.c_int, _I, C.c_void_p]
        L.nb_kepler_drift.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_double,
                                      C.c_int, C.c_void_p, C.c_void_p]
        L.nb_shard_rows.argtypes = [C.c_int, C.c_int, C.c_int, _I, _I]
        L.nb_shard_buffer_bytes.argtypes = [C.c_void_p, C.c_int]
        L.nb_shard_buffer_bytes.restype = C.c_size_t
        L.nb_set_shard.argtypes = [C.c_void_p, C.c_int, C.c_int, ALLGATHER_FN, C.c_void_p,
                                   C.c_void_p, C.c_size_t]
        L.nb_batch_get_shape.argtypes = [C.c_void_p, _I, _I, _I, _I]
        L.nb_batch_set_schedule.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.nb_batch_encounter_list.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, _I]
        L.nb_energy_grad_scratch_bytes.argtypes = [C.c_int]
        L.nb_energy_grad_scratch_bytes.restype = C.c_size_t
        L.nb_energy_grad.argtypes = [C.c_int] + [C.c_void_p] * 4 + [C.c_double, C.c_double] + [
            C.c_void_p] * 4 + [C.c_size_t, C.c_void_p]
        L.nb_batch_workspace_bytes.argtypes = [C.POINTER(NbParams), C.c_int, C.c_void_p]
        L.nb_batch_workspace_bytes.restype = C.c_size_t
        L.nb_batch_init.argtypes = [C.POINTER(C.c_void_p), C.POINTER(NbParams), C.c_int,
                                    C.c_void_p] + [C.c_void_p] * 5 + [C.c_void_p, C.c_size_t,
                                                                      C.c_void_p, C.c_int]
        L.nb_batch_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.nb_batch_set_shape.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.nb_batch_autotune.argtypes = [C.c_void_p, C.c_double, _I, _D]
        L.nb_batch_get_state.argtypes = [C.c_void_p] + [C.c_void_p] * 5 + [C.c_int]
        L.nb_batch_energy.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.nb_batch_stats.argtypes = [C.c_void_p, C.POINTER(NbStats)]
        L.nb_batch_destroy.argtypes = [C.c_void_p]
        L.nb_batch_set_budget.argtypes = [C.c_void_p, C.c_double]
        L.nb_batch_balance.argtypes = [C.c_void_p, _D, _D, _I]
        L.nb_peak_scratch_bytes.argtypes = []
        L.nb_peak_scratch_bytes.restype = C.c_size_t
        L.nb_measure_peaks.argtypes = [_D, _D, C.c_void_p, C.c_void_p]
        L.nb_math_eval.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.nb_adjoint_workspace_bytes.argtypes = [C.POINTER(NbParams), C.c_int, C.c_int, C.c_int]
        L.nb_adjoint_workspace_bytes.restype = C.c_size_t
        L.nb_adjoint_init.argtypes = [C.POINTER(C.c_void_p), C.POINTER(NbParams), C.c_int] + [
            C.c_void_p] * 5 + [C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, C.c_int]
        L.nb_adjoint_forward.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.nb_adjoint_state.argtypes = [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]
        L.nb_adjoint_backward.argtypes = [C.c_void_p] + [C.c_void_p] * 6 + [C.c_int]
        L.nb_adjoint_last_error.argtypes = [C.c_void_p]
        L.nb_adjoint_last_error.restype = C.c_char_p
        L.nb_adjoint_destroy.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().nb_status_string(code).decode()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libnb needs a CUDA device; there is no CPU fallback")
    return torch


def _stream(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def params(**kw) -> NbParams:
    p = NbParams()
    lib().nb_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _shape_ok(got, want, min_rows):
    if len(got) != len(want):
        return False
    if any(w >= 0 and g != w for g, w in zip(got[1:], want[1:])):
        return False
    if want[0] < 0:
        return True
    return got[0] >= want[0] if min_rows else got[0] == want[0]


def _dev_buf(torch, name, t, dtype, shape, convert=False, min_rows=False):
    """t as a buffer the library may read or write through a raw device
    pointer. It must be a CUDA tensor on the current device: a host pointer,
    or another device's memory, handed to a kernel faults it. With convert a
    tensor of another dtype or layout is copied to a contiguous one of dtype;
    without, it must already be one (outputs are written in place). Its shape
    must equal shape (-1 matches any extent; min_rows: at least shape[0]
    rows), else the kernel would run past it. ValueError otherwise."""
    dev = torch.device("cuda", torch.cuda.current_device())
    if not isinstance(t, torch.Tensor) or t.device != dev:
        raise ValueError("%s must be a CUDA tensor on %s" % (name, dev))
    if convert:
        t = t.contiguous().to(dtype)
    elif t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor" % (name, dtype))
    if not _shape_ok(tuple(t.shape), tuple(shape), min_rows):
        raise ValueError("%s must have shape %s%s, got %s" % (
            name, tuple(shape), " (or more rows)" if min_rows else "", tuple(t.shape)))
    return t


def _host_buf(name, a, dtype, shape):
    """a as a contiguous host array of dtype and exactly shape (the library
    reads that many elements through its pointer); ValueError otherwise."""
    a = np.ascontiguousarray(a, dtype=dtype)
    if not _shape_ok(a.shape, tuple(shape), False):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), a.shape))
    return a


def _len0(t):
    """Leading extent of an array or tensor (-1 for a scalar)."""
    s = tuple(t.shape) if hasattr(t, "shape") else np.shape(t)
    return int(s[0]) if len(s) else -1


class NBodySystem:
    """A planetary system integrated on the GPU by libnb.

    x, v: (n, 3) heliocentric positions / barycentric velocities (AU, AU/day);
    m, R: (n,) masses (Msun) and radii (AU). numpy arrays are copied from the
    host by the library; CUDA float64 tensors are read on the device.
    """

    def __init__(self, p: NbParams, x, v, m, R, rc=None, ids=None):
        torch = _torch()
        L = lib()
        self.p = p
        on_dev = isinstance(x, torch.Tensor) and x.is_cuda
        n = _len0(m)
        shapes = {"x": (n, 3), "v": (n, 3), "m": (n,), "R": (n,)}
        names = ("x", "v", "m", "R")
        if on_dev:
            args = [_dev_buf(torch, k, t, torch.float64, shapes[k], convert=True)
                    for k, t in zip(names, (x, v, m, R))]
            rcv = None if rc is None else _dev_buf(torch, "rc", rc, torch.float64, (n,), True)
            idv = None if ids is None else _dev_buf(torch, "ids", ids, torch.int32, (n,), True)
            self._keep = (args, rcv, idv)
            ptrs = [_ptr(t) for t in args]
            rcp = None if rcv is None else _ptr(rcv)
            idp = None if idv is None else _ptr(idv)
        else:
            args = [_host_buf(k, a, np.float64, shapes[k]) for k, a in zip(names, (x, v, m, R))]
            rcv = None if rc is None else _host_buf("rc", rc, np.float64, (n,))
            idv = None if ids is None else _host_buf("ids", ids, np.int32, (n,))
            self._keep = (args, rcv, idv)
            ptrs = [C.c_void_p(a.ctypes.data) for a in args]
            rcp = None if rcv is None else C.c_void_p(rcv.ctypes.data)
            idp = None if idv is None else C.c_void_p(idv.ctypes.data)
        self.n = int(n)
        nbytes = L.nb_workspace_bytes(C.byref(p), self.n)
        if nbytes == 0:
            raise NbError(NB_E_INVALID, "bad parameters or n")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self._ws_ptr = C.c_void_p(base + off)
        self._ws_bytes = nbytes
        h = C.c_void_p()
        self._stream = _stream(torch)
        rcode = L.nb_init_system(C.byref(h), C.byref(p), self.n, ptrs[0], ptrs[1], ptrs[2],
                                 ptrs[3], rcp, idp, self._ws_ptr, self._ws_bytes, self._stream,
                                 1 if on_dev else 0)
        if rcode != NB_OK:
            raise NbError(rcode, "nb_init_system failed")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().nb_destroy(h)
            self._h = None

    def _check(self, code):
        if code != NB_OK:
            raise NbError(code, lib().nb_last_error(self._h).decode())

    def step(self, nsteps: int, dt: float):
        self._check(lib().nb_step(self._h, int(nsteps), float(dt)))

    def step_status(self, nsteps: int, dt: float) -> int:
        return lib().nb_step(self._h, int(nsteps), float(dt))

    def energy_momentum(self) -> dict:
        E, El = C.c_double(), C.c_double()
        Lv, P = np.zeros(3), np.zeros(3)
        self._check(lib().nb_energy_momentum(self._h, C.byref(E), Lv.ctypes.data_as(_D),
                                             P.ctypes.data_as(_D), C.byref(El)))
        return dict(E=E.value, L=Lv, P=P, E_lost=El.value)

    def state(self) -> dict:
        n = self.n
        x = np.zeros((n, 3)); v = np.zeros((n, 3)); m = np.zeros(n); R = np.zeros(n)
        rc = np.zeros(n); ids = np.zeros(n, dtype=np.int32); k = C.c_int()
        self._check(lib().nb_get_state(self._h, C.c_void_p(x.ctypes.data),
                                       C.c_void_p(v.ctypes.data), C.c_void_p(m.ctypes.data),
                                       C.c_void_p(R.ctypes.data), C.c_void_p(rc.ctypes.data),
                                       C.c_void_p(ids.ctypes.data), C.byref(k), 0))
        k = k.value
        return dict(x=x[:k], v=v[:k], m=m[:k], R=R[:k], rc=rc[:k], ids=ids[:k])

    def state_device(self, out: dict) -> int:
        """Gather the active bodies into caller CUDA tensors; returns their count.
        Each tensor needs room for all n slots: x, v (n, 3), m, R, rc (n,)
        float64 and ids (n,) int32, contiguous (more rows are fine)."""
        torch = _torch()
        n = self.n
        for k, dt, sh in (("x", torch.float64, (n, 3)), ("v", torch.float64, (n, 3)),
                          ("m", torch.float64, (n,)), ("R", torch.float64, (n,)),
                          ("rc", torch.float64, (n,)), ("ids", torch.int32, (n,))):
            _dev_buf(torch, k, out[k], dt, sh, min_rows=True)
        k = C.c_int()
        self._check(lib().nb_get_state(self._h, _ptr(out["x"]), _ptr(out["v"]), _ptr(out["m"]),
                                       _ptr(out["R"]), _ptr(out["rc"]), _ptr(out["ids"]),
                                       C.byref(k), 1))
        return k.value

    def fsal(self):
        a = np.zeros((self.n, 3))
        cnt = C.c_int()
        self._check(lib().nb_get_fsal(self._h, C.c_void_p(a.ctypes.data), None, 0,
                                      C.byref(cnt), 0))
        pairs = np.zeros((max(cnt.value, 1), 2), dtype=np.int32)
        code = lib().nb_get_fsal(self._h, None, C.c_void_p(pairs.ctypes.data), cnt.value,
                                 C.byref(cnt), 0)
        self._check(code)
        return a, pairs[:cnt.value]

    def set_fsal(self, a, pairs):
        a = _host_buf("a", a, np.float64, (self.n, 3))
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        self._check(lib().nb_set_fsal(self._h, C.c_void_p(a.ctypes.data),
                                      C.c_void_p(pairs.ctypes.data), pairs.shape[0], 0))

    def set_state(self, x, v, m, R, rc, ids, a, pairs):
        """Load a full state (host numpy arrays or CUDA tensors) without a force
        evaluation; a is the cached force [n][3], pairs the cached flags."""
        import torch
        on_dev = isinstance(x, torch.Tensor) and x.is_cuda
        n = self.n
        f64 = ((n, 3), (n, 3), (n,), (n,), (n,), (n, 3))
        names = ("x", "v", "m", "R", "rc", "a")
        if on_dev:
            x, v, m, R, rc, a = (_dev_buf(torch, k, t, torch.float64, sh, convert=True)
                                 for k, t, sh in zip(names, (x, v, m, R, rc, a), f64))
            ids = None if ids is None else _dev_buf(torch, "ids", ids, torch.int32, (n,), True)
            pairs = _dev_buf(torch, "pairs", pairs, torch.int32, (-1, 2), True)
            npairs = int(pairs.shape[0])
            ptr = _ptr
        else:
            x, v, m, R, rc, a = (_host_buf(k, t, np.float64, sh)
                                 for k, t, sh in zip(names, (x, v, m, R, rc, a), f64))
            ids = None if ids is None else _host_buf("ids", ids, np.int32, (n,))
            pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
            npairs = int(pairs.shape[0])

            def ptr(t):
                return C.c_void_p(t.ctypes.data)
        idp = None if ids is None else ptr(ids)
        self._check(lib().nb_set_state(self._h, ptr(x), ptr(v), ptr(m), ptr(R), ptr(rc), idp,
                                       ptr(a), ptr(pairs) if npairs else None, npairs,
                                       1 if on_dev else 0))

    def set_timing(self, enable: bool = True):
        self._check(lib().nb_set_timing(self._h, 1 if enable else 0))

    def timing(self) -> dict:
        ms, kl, la = C.c_double(), C.c_longlong(), C.c_longlong()
        self._check(lib().nb_timing(self._h, C.byref(ms), C.byref(kl), C.byref(la)))
        return dict(kick_ms=ms.value, kick_launches=kl.value, launches=la.value)

    def encounter_list(self) -> np.ndarray:
        cnt = C.c_int()
        lib().nb_encounter_list(self._h, None, 0, C.byref(cnt))
        out = np.zeros((max(cnt.value, 1), 3), dtype=np.int32)
        code = lib().nb_encounter_list(self._h, C.c_void_p(out.ctypes.data), cnt.value,
                                       C.byref(cnt))
        self._check(code)
        return out[:cnt.value]

    def stats(self) -> dict:
        st = NbStats()
        self._check(lib().nb_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in NbStats._fields_}


def kick(x, m, rc, G=2.959122082855911e-4, precision=NB_PREC_FP64, split=0, cap=None,
         rows=None):
    """One launch of the kick+flag kernel on CUDA tensors. Returns (a, pairs,
    status); with rows = (row0, row1) only those target rows (nb_kick_rows)."""
    torch = _torch()
    L = lib()
    n = _len0(x)
    x = _dev_buf(torch, "x", x, torch.float64, (n, 3), convert=True)
    m = _dev_buf(torch, "m", m, torch.float64, (n,), convert=True)
    rc = _dev_buf(torch, "rc", rc, torch.float64, (n,), convert=True)
    r0, r1 = (0, n) if rows is None else rows
    a = torch.empty((max(r1 - r0, 1), 3), dtype=torch.float64, device="cuda")
    cap = 16 * n + 64 if cap is None else cap
    pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    nb = L.nb_kick_scratch_bytes(n, split)
    scratch = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    sp = scratch.data_ptr() + ((-scratch.data_ptr()) % 256)
    cnt = C.c_int()
    code = L.nb_kick_rows(n, r0, r1, _ptr(x), _ptr(m), _ptr(rc), G,
                          precision, split, _ptr(a), _ptr(pairs), cap, C.byref(cnt),
                          C.c_void_p(sp), nb, _stream(torch))
    return a[:max(r1 - r0, 0)], pairs[:min(cnt.value, cap)], code


NB_NOALLOC_MAX_N = 65600
NB_BATCH_MAX_N = 512


class NBodyBatch:
    """Independent systems integrated together by libnb's batched kernel.

    systems: list of objects with x (n,3), v (n,3), m (n,), R (n,) (numpy).
    """

    def __init__(self, p: NbParams, systems, rc=None):
        torch = _torch()
        L = lib()
        self.p = p
        ns = [int(np.asarray(d.m).shape[0]) for d in systems]
        self.offsets = np.concatenate([[0], np.cumsum(ns)]).astype(np.int32)
        self.nsys = len(systems)
        cat = lambda k: np.ascontiguousarray(np.concatenate([np.asarray(getattr(d, k), dtype=np.float64)  # noqa: E731
                                                             for d in systems]))
        self._x, self._v, self._m, self._R = cat("x"), cat("v"), cat("m"), cat("R")
        tot = int(self.offsets[-1])
        for k, sh in (("x", (tot, 3)), ("v", (tot, 3)), ("m", (tot,)), ("R", (tot,))):
            _host_buf(k, getattr(self, "_" + k), np.float64, sh)
        self._rc = None if rc is None else _host_buf("rc", rc, np.float64, (tot,))
        nbytes = L.nb_batch_workspace_bytes(C.byref(p), self.nsys,
                                            C.c_void_p(self.offsets.ctypes.data))
        if nbytes == 0:
            raise NbError(NB_E_INVALID, "bad parameters, sizes or offsets")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        ws = C.c_void_p(base + ((-base) % 256))
        h = C.c_void_p()
        code = L.nb_batch_init(C.byref(h), C.byref(p), self.nsys,
                               C.c_void_p(self.offsets.ctypes.data),
                               C.c_void_p(self._x.ctypes.data), C.c_void_p(self._v.ctypes.data),
                               C.c_void_p(self._m.ctypes.data), C.c_void_p(self._R.ctypes.data),
                               None if self._rc is None else C.c_void_p(self._rc.ctypes.data),
                               ws, nbytes, _stream(torch), 0)
        if code != NB_OK:
            raise NbError(code, "nb_batch_init failed")
        self._h = h
        self.total = int(self.offsets[-1])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().nb_batch_destroy(h)
            self._h = None

    def _check(self, code):
        if code != NB_OK:
            raise NbError(code, "batched call failed")

    def step(self, nsteps: int, dt: float):
        self._check(lib().nb_batch_step(self._h, int(nsteps), float(dt)))

    def step_status(self, nsteps: int, dt: float) -> int:
        return lib().nb_batch_step(self._h, int(nsteps), float(dt))

    def set_shape(self, threads: int, chunk: int):
        self._check(lib().nb_batch_set_shape(self._h, threads, chunk))

    def autotune(self, dt: float):
        t, ms = C.c_int(), C.c_double()
        self._check(lib().nb_batch_autotune(self._h, dt, C.byref(t), C.byref(ms)))
        return t.value, ms.value

    def encounter_list(self, s: int) -> np.ndarray:
        """(step, i, j) encounter pairs of system s during the last step() call
        (i < j, indices within the system)."""
        cnt = C.c_int()
        code = lib().nb_batch_encounter_list(self._h, int(s), None, 0, C.byref(cnt))
        if code not in (NB_OK, NB_E_OVERFLOW):
            self._check(code)
        out = np.zeros((cnt.value, 3), dtype=np.int32)
        if cnt.value:
            self._check(lib().nb_batch_encounter_list(self._h, int(s),
                                                      C.c_void_p(out.ctypes.data), cnt.value,
                                                      C.byref(cnt)))
        return out

    def shape(self) -> dict:
        """The launch shape and schedule in use: threads per CTA, steps per
        graph chunk, kick tile rows and buckets of independent launch chains."""
        t, c, r, k = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._check(lib().nb_batch_get_shape(self._h, C.byref(t), C.byref(c), C.byref(r),
                                             C.byref(k)))
        return {"threads": t.value, "chunk": c.value, "tile_rows": r.value, "buckets": k.value}

    def set_schedule(self, tile_rows: int, buckets: int):
        self._check(lib().nb_batch_set_schedule(self._h, int(tile_rows), int(buckets)))

    def state(self) -> dict:
        n = self.total
        x = np.zeros((n, 3)); v = np.zeros((n, 3)); m = np.zeros(n); R = np.zeros(n)
        alive = np.zeros(n, dtype=np.int32)
        self._check(lib().nb_batch_get_state(self._h, C.c_void_p(x.ctypes.data),
                                             C.c_void_p(v.ctypes.data), C.c_void_p(m.ctypes.data),
                                             C.c_void_p(R.ctypes.data),
                                             C.c_void_p(alive.ctypes.data), 0))
        return dict(x=x, v=v, m=m, R=R, alive=alive)

    def system_state(self, s: int, st=None) -> dict:
        st = st or self.state()
        a, b = self.offsets[s], self.offsets[s + 1]
        keep = st["alive"][a:b] != 0
        return {k: st[k][a:b][keep] for k in ("x", "v", "m", "R")} | {
            "ids": np.nonzero(keep)[0].astype(np.int32)}

    def energy(self):
        E = np.zeros(self.nsys); El = np.zeros(self.nsys)
        self._check(lib().nb_batch_energy(self._h, C.c_void_p(E.ctypes.data),
                                          C.c_void_p(El.ctypes.data)))
        return E, El

    def stats(self) -> dict:
        st = NbStats()
        self._check(lib().nb_batch_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in NbStats._fields_}

    def set_budget(self, max_ms_per_launch: float):
        self._check(lib().nb_batch_set_budget(self._h, float(max_ms_per_launch)))

    def balance(self) -> dict:
        """Load balance of the last launch (efficiency, longest CTA in ms, CTAs)."""
        e, mx, g = C.c_double(), C.c_double(), C.c_int()
        self._check(lib().nb_batch_balance(self._h, C.byref(e), C.byref(mx), C.byref(g)))
        return {"efficiency": e.value, "max_cta_ms": mx.value, "ctas": g.value}


def kick_noalloc(x, m, rc, a, pairs, G=2.959122082855911e-4, precision=NB_PREC_FP64):
    """nb_kick_noalloc on caller-provided CUDA tensors a (n, 3) and pairs
    (cap, 2): nothing is allocated by this call. Returns (npairs, status).

    The kernel writes n x 3 doubles through a and up to cap int32 pairs
    through pairs, so every tensor must be a contiguous CUDA tensor on the
    current device with the stated dtype and shape (ValueError otherwise;
    the checks allocate nothing)."""
    torch = _torch()
    n = int(x.shape[0]) if x.dim() >= 1 else -1
    dev = torch.device("cuda", torch.cuda.current_device())
    want = [("x", x, torch.float64, (n, 3)), ("m", m, torch.float64, (n,)),
            ("rc", rc, torch.float64, (n,)), ("a", a, torch.float64, (n, 3)),
            ("pairs", pairs, torch.int32, None)]
    for name, t, dt, shape in want:
        if not isinstance(t, torch.Tensor) or t.device != dev:
            raise ValueError("%s must be a CUDA tensor on %s" % (name, dev))
        if t.dtype != dt or not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor" % (name, dt))
        if shape is not None and tuple(t.shape) != shape:
            raise ValueError("%s must have shape %s, got %s" % (name, shape, tuple(t.shape)))
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    cnt = C.c_int()
    code = lib().nb_kick_noalloc(x.shape[0], _ptr(x), _ptr(m), _ptr(rc), G, precision, _ptr(a),
                                 _ptr(pairs), pairs.shape[0], C.byref(cnt), _stream(torch))
    return cnt.value, code


def energy_grad(x, v, m, alive=None, G=2.959122082855911e-4, m0=1.0):
    """Gradient of the total energy (Eqs. Ha-Hc) with respect to the state on
    CUDA tensors x, v (n, 3), m (n,), alive (n,) int32 or None (nb_energy_grad).
    Returns (dE/dx, dE/dv, dE/dm) as new tensors; zero for absorbed bodies."""
    torch = _torch()
    n = _len0(m)
    x = _dev_buf(torch, "x", x, torch.float64, (n, 3), convert=True)
    v = _dev_buf(torch, "v", v, torch.float64, (n, 3), convert=True)
    m = _dev_buf(torch, "m", m, torch.float64, (n,), convert=True)
    al = None if alive is None else _dev_buf(torch, "alive", alive, torch.int32, (n,), True)
    gx = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gv = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gm = torch.empty(n, dtype=torch.float64, device="cuda")
    L = lib()
    nbytes = L.nb_energy_grad_scratch_bytes(n)
    scratch = torch.empty(max(nbytes, 8), dtype=torch.uint8, device="cuda")
    code = L.nb_energy_grad(n, _ptr(x), _ptr(v), _ptr(m), None if al is None else _ptr(al), G,
                            m0, _ptr(gx), _ptr(gv), _ptr(gm), _ptr(scratch), nbytes,
                            _stream(torch))
    if code != NB_OK:
        raise NbError(code, "nb_energy_grad")
    return gx, gv, gm


def kepler_drift(x, v, mu, dt, max_iter=30):
    """Kepler-drift CUDA tensors x, v (n, 3) in place (contiguous float64);
    returns the status code."""
    torch = _torch()
    n = _len0(x)
    _dev_buf(torch, "x", x, torch.float64, (n, 3))
    _dev_buf(torch, "v", v, torch.float64, (n, 3))
    scratch = torch.zeros(64, dtype=torch.uint8, device="cuda")
    return lib().nb_kepler_drift(x.shape[0], mu, _ptr(x), _ptr(v), dt, max_iter,
                                 _ptr(scratch), _stream(torch))


def math_eval(fn: int, x):
    """Evaluate device arithmetic helper fn (NB_MATH_*) element-wise on a
    float64 CUDA tensor (nb_math_eval); returns a new tensor."""
    torch = _torch()
    x = _dev_buf(torch, "x", x, torch.float64, tuple(-1 for _ in x.shape))
    out = torch.empty_like(x)
    code = lib().nb_math_eval(fn, x.numel(), _ptr(x), _ptr(out), _stream(torch))
    if code != NB_OK:
        raise NbError(code, "nb_math_eval")
    return out


def ratio_le(a, b, tol):
    """The direct solver's acceptance test fl(a / b) <= tol, element-wise on
    float64 CUDA tensors a, b, tol of one length (NB_MATH_RATIO_LE); returns
    a float64 tensor of 1.0 / 0.0."""
    torch = _torch()
    k = _len0(a)
    a, b, tol = (_dev_buf(torch, nm, t, torch.float64, (k,), convert=True)
                 for nm, t in (("a", a), ("b", b), ("tol", tol)))
    tri = torch.stack([a, b, tol], dim=1).contiguous()
    out = torch.empty(tri.shape[0], dtype=torch.float64, device=tri.device)
    code = lib().nb_math_eval(NB_MATH_RATIO_LE, tri.shape[0], _ptr(tri), _ptr(out),
                              _stream(torch))
    if code != NB_OK:
        raise NbError(code, "nb_math_eval")
    return out


def measure_peaks():
    """(FP64 FLOP/s, FP32 FLOP/s) from the library's own FMA loops."""
    torch = _torch()
    L = lib()
    scratch = torch.empty(L.nb_peak_scratch_bytes(), dtype=torch.uint8, device="cuda")
    f64, f32 = C.c_double(), C.c_double()
    code = L.nb_measure_peaks(C.byref(f64), C.byref(f32), _ptr(scratch), _stream(torch))
    if code != NB_OK:
        raise NbError(code, "nb_measure_peaks")
    return f64.value, f32.value


class NBodyAdjoint:
    """Forward integration with checkpoints and its discrete adjoint
    (nb_adjoint_*): gradients of a loss on the final state with respect to
    the initial positions, velocities and masses. rc is required and held
    fixed, as are the encounter events of the forward.

    Inputs are host numpy arrays or CUDA float64 tensors; results come back
    in the same kind.
    """

    def __init__(self, p: NbParams, x, v, m, R, rc, nsteps: int, every: int = 100):
        torch = _torch()
        L = lib()
        self.p = p
        self.on_dev = isinstance(x, torch.Tensor) and x.is_cuda
        n = _len0(m)
        names = ("x", "v", "m", "R", "rc")
        shapes = ((n, 3), (n, 3), (n,), (n,), (n,))
        if self.on_dev:
            args = [_dev_buf(torch, k, t, torch.float64, sh, convert=True)
                    for k, t, sh in zip(names, (x, v, m, R, rc), shapes)]
            ptrs = [_ptr(t) for t in args]
        else:
            args = [_host_buf(k, a, np.float64, sh)
                    for k, a, sh in zip(names, (x, v, m, R, rc), shapes)]
            ptrs = [C.c_void_p(a.ctypes.data) for a in args]
        self._keep = args
        self.n = int(n)
        self.nsteps = int(nsteps)
        nbytes = L.nb_adjoint_workspace_bytes(C.byref(p), self.n, self.nsteps, int(every))
        if nbytes == 0:
            raise NbError(NB_E_INVALID, "bad parameters, n, nsteps or checkpoint interval")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        self._ws_ptr = C.c_void_p(base + (-base) % 256)
        h = C.c_void_p()
        self._stream = _stream(torch)
        code = L.nb_adjoint_init(C.byref(h), C.byref(p), self.n, *ptrs, self.nsteps, int(every),
                                 self._ws_ptr, nbytes, self._stream, 1 if self.on_dev else 0)
        if code != NB_OK:
            raise NbError(code, "nb_adjoint_init failed")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().nb_adjoint_destroy(h)
            self._h = None

    def _check(self, code):
        if code != NB_OK:
            raise NbError(code, lib().nb_adjoint_last_error(self._h).decode())

    def forward(self, dt: float, nsteps: int | None = None):
        self._check(lib().nb_adjoint_forward(self._h, int(nsteps or self.nsteps), float(dt)))

    def state(self) -> dict:
        """Final state of all n slots: x, v (n, 3), m (n,), alive (n,)."""
        n = self.n
        if self.on_dev:
            import torch
            out = dict(x=torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                       v=torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                       m=torch.empty(n, dtype=torch.float64, device="cuda"),
                       alive=torch.empty(n, dtype=torch.int32, device="cuda"))
            ptrs = [_ptr(out[k]) for k in ("x", "v", "m", "alive")]
        else:
            out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), m=np.zeros(n),
                       alive=np.zeros(n, dtype=np.int32))
            ptrs = [C.c_void_p(out[k].ctypes.data) for k in ("x", "v", "m", "alive")]
        self._check(lib().nb_adjoint_state(self._h, *ptrs, 1 if self.on_dev else 0))
        return out

    def backward(self, gx, gv, gm):
        """Pull back (dL/dx_T, dL/dv_T, dL/dm_T) to (dL/dx_0, dL/dv_0, dL/dm_0)."""
        n = self.n
        if self.on_dev:
            import torch
            g = [_dev_buf(torch, k, t, torch.float64, sh, convert=True)
                 for k, t, sh in (("gx", gx, (n, 3)), ("gv", gv, (n, 3)), ("gm", gm, (n,)))]
            out = (torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                   torch.empty((n, 3), dtype=torch.float64, device="cuda"),
                   torch.empty(n, dtype=torch.float64, device="cuda"))
            gp = [_ptr(t) for t in g]
            op = [_ptr(t) for t in out]
        else:
            g = [_host_buf(k, a, np.float64, sh)
                 for k, a, sh in (("gx", gx, (n, 3)), ("gv", gv, (n, 3)), ("gm", gm, (n,)))]
            out = (np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n))
            gp = [C.c_void_p(a.ctypes.data) for a in g]
            op = [C.c_void_p(a.ctypes.data) for a in out]
        self._check(lib().nb_adjoint_backward(self._h, *gp, *op, 1 if self.on_dev else 0))
        return out


def _autograd_fn():
    import torch

    class NBodyFn(torch.autograd.Function):
        """(x0, v0, m0) -> (x_T, v_T, m_T) through libnb, differentiable by the
        library's discrete adjoint. R and rc are constants."""

        @staticmethod
        def forward(ctx, x0, v0, m0, R, rc, p, nsteps, dt, every):
            adj = NBodyAdjoint(p, x0.detach(), v0.detach(), m0.detach(), R.detach(),
                               rc.detach(), nsteps, every)
            adj.forward(dt)
            st = adj.state()
            ctx.adj = adj
            ctx.mark_non_differentiable(st["alive"])
            return st["x"], st["v"], st["m"], st["alive"]

        @staticmethod
        def backward(ctx, gx, gv, gm, _galive):
            n = ctx.adj.n
            z3 = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
            z1 = torch.zeros(n, dtype=torch.float64, device="cuda")
            dx, dv, dm = ctx.adj.backward(z3 if gx is None else gx, z3 if gv is None else gv,
                                          z1 if gm is None else gm)
            return dx, dv, dm, None, None, None, None, None, None

    return NBodyFn


_NBodyFn = None


def integrate(x0, v0, m0, R, rc, p: NbParams, nsteps: int, dt: float, every: int = 100):
    """Differentiable integration of CUDA float64 tensors: returns
    (x_T, v_T, m_T, alive_T); gradients reach x0, v0 and m0 through the
    library's adjoint kernels."""
    global _NBodyFn
    if _NBodyFn is None:
        _NBodyFn = _autograd_fn()
    return _NBodyFn.apply(x0, v0, m0, R, rc, p, int(nsteps), float(dt), int(every))
