"""GB300-native coupled central-moment lattice Boltzmann stepper (arXiv 2210.07501).

Thin ctypes binding of the C ABI in ``include/lbm_gb300.h``: argument marshalling only.
Every step of the method runs in the CUDA library ``_lib/liblbm_gb300.so`` (built for
sm_103a by :func:`build`); there is no CPU path.  If the library cannot be loaded the
import of :func:`load` raises.

PyTorch is optional: a torch CUDA stream can be handed to :class:`Lbm`, and torch device
tensors can receive fields through :meth:`Lbm.fields_device`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EIO, LBM_EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7
LBM_FP64, LBM_FP32, LBM_FP16 = 0, 1, 2
LBM_DTYPE_F64, LBM_DTYPE_F32 = 0, 1
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16}

LIB_PATH = _build.LIB
_lock = threading.Lock()
_lib = None


class LbmError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = load().lbm_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class LbmDomain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("heat_periods", ctypes.c_int32),
                ("q_phi", ctypes.c_int32), ("q_T", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("b", ctypes.c_double), ("W", ctypes.c_double)]


class LbmParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "sigma0", "sigma1", "sigma2", "T_ref", "T_hot", "T_cold", "dT", "tau_flow", "visc_ratio", "tau_T",
        "cond_ratio", "tau_phi", "rho_bottom", "rho_top", "Fx_ext", "Fy_ext")]


_D = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); the names are those of include/lbm_gb300.h
SIGNATURES = {
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(LbmDomain), ctypes.POINTER(LbmParams), ctypes.c_void_p,
                                  ctypes.POINTER(_H)]),
    "lbm_init_fields": (ctypes.c_int, [_H, _D, _D, _D, _D, _D]),
    "lbm_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "lbm_fields": (ctypes.c_int, [_H, _D, _D, _D, _D, _D]),
    "lbm_fields_device": (ctypes.c_int, [_H] + [ctypes.c_void_p] * 5 + [ctypes.c_int]),
    "lbm_diag": (ctypes.c_int, [_H, _D, _D, _I64P]),
    "lbm_set_check_interval": (ctypes.c_int, [_H, ctypes.c_int32]),
    "lbm_run_to_steady": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_int64, _I64P]),
    "lbm_get_state": (ctypes.c_int, [_H, _D, _D, _D, _D]),
    "lbm_set_state": (ctypes.c_int, [_H, _D, _D, _D, _D]),
    "lbm_save": (ctypes.c_int, [_H, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_H, ctypes.c_char_p]),
    "lbm_set_segment": (ctypes.c_int, [_H, ctypes.c_int32]),
    "lbm_test_stall_copies": (ctypes.c_int, [_H, ctypes.c_int32]),
    "lbm_autotune": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_bytes_per_node": (ctypes.c_int, [_H, _I64P]),
    "lbm_launch_count": (ctypes.c_int, [_H, _I64P]),
    "lbm_reduce_fields_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_void_p,
                                                                      ctypes.c_void_p]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(LbmDomain), ctypes.POINTER(LbmParams),
                                        ctypes.c_void_p, ctypes.POINTER(_H)]),
    "lbm_batch_set_check_interval": (ctypes.c_int, [_H, ctypes.c_int32]),
    "lbm_batch_autotune": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "lbm_batch_run_to_steady": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_int64, _I64P,
                                               ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_fields": (ctypes.c_int, [_H, ctypes.c_int32, _D, _D, _D, _D, _D]),
    "lbm_batch_diag": (ctypes.c_int, [_H, ctypes.c_int32, _D, _I64P]),
    "lbm_batch_init_fields": (ctypes.c_int, [_H, ctypes.c_int32, _D, _D, _D, _D, _D]),
    "lbm_batch_size": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_destroy": (None, [_H]),
    "lbm_cnn_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_void_p, ctypes.POINTER(_H)]),
    "lbm_cnn_num_params": (ctypes.c_int, [_H, _I64P]),
    "lbm_cnn_get_params": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float)]),
    "lbm_cnn_set_params": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float)]),
    "lbm_cnn_forward": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "lbm_cnn_gradients": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_float), _D]),
    "lbm_cnn_train_step": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, _D]),
    "lbm_cnn_strerror": (ctypes.c_char_p, []),
    "lbm_cnn_destroy": (None, [_H]),
    "lbm_destroy": (None, [_H]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a in-tree (nvcc)."""
    return _build.build(force=force)


def load(path: str | None = None):
    """Load the CUDA library (no fallback: raises OSError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise OSError(f"CUDA library {p} is not built; run paper_2210_07501_gb300.build()")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc, where):
    if rc != LBM_OK:
        raise LbmError(rc, where)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _field(a, shape):
    if a is None:
        return None
    return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))


_CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream as an explicit handle


def stream_handle(stream):
    """ctypes value for a stream argument: None (the library makes its own stream), an int,
    or a torch.cuda.Stream.  Torch's default stream has handle 0, which the C ABI would read
    as "none given", so it is passed as cudaStreamLegacy to keep the caller's ordering."""
    if stream is None:
        return None
    h = stream if isinstance(stream, int) else stream.cuda_stream
    return ctypes.c_void_p(h if h else _CUDA_STREAM_LEGACY)


def make_domain(domain: dict, precision="fp64") -> LbmDomain:
    d = LbmDomain()
    for k in ("nx", "ny", "heat_periods", "q_phi", "q_T"):
        setattr(d, k, int(domain[k]))
    d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d.b = float(domain["b"])
    d.W = float(domain["W"])
    return d


def make_params(params: dict) -> LbmParams:
    p = LbmParams()
    for k, _ in LbmParams._fields_:
        setattr(p, k, float(params.get(k, 0.0)))
    return p


class Lbm:
    """One solver instance (one lbm_handle).  Fields are [ny][nx] float64 arrays."""

    def __init__(self, domain: dict, params: dict, precision="fp64", stream=None):
        self._lib = load()
        self.domain = dict(domain)
        self.params = dict(params)
        self.nx, self.ny = int(domain["nx"]), int(domain["ny"])
        self.q_phi, self.q_T = int(domain["q_phi"]), int(domain["q_T"])
        self.precision = precision
        self._h = _H()
        s = stream_handle(stream)
        self._dom = make_domain(domain, precision)
        self._prm = make_params(params)
        _check(self._lib.lbm_create(ctypes.byref(self._dom), ctypes.byref(self._prm), s, ctypes.byref(self._h)),
               "lbm_create")

    # -- lifetime
    def lbm_destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbm_destroy(self._h)
            self._h = _H()

    close = lbm_destroy

    def __del__(self):
        try:
            self.lbm_destroy()
        except Exception:
            pass

    # -- C-ABI entry points, same names
    def lbm_init_fields(self, phi=None, u=None, v=None, T=None, dp=None):
        shape = (self.ny, self.nx)
        a = [_field(x, shape) for x in (phi, u, v, T, dp)]
        _check(self._lib.lbm_init_fields(self._h, *[_dptr(x) for x in a]), "lbm_init_fields")

    def lbm_step(self, n: int = 1):
        _check(self._lib.lbm_step(self._h, int(n)), "lbm_step")

    def lbm_fields(self) -> dict:
        shape = (self.ny, self.nx)
        out = {k: np.empty(shape) for k in ("phi", "u", "v", "T", "dp")}
        _check(self._lib.lbm_fields(self._h, *[_dptr(out[k]) for k in ("phi", "u", "v", "T", "dp")]), "lbm_fields")
        return out

    def lbm_fields_device(self, phi=None, u=None, v=None, T=None, dp=None, dtype=LBM_DTYPE_F64):
        ptrs = [None if t is None else ctypes.c_void_p(t.data_ptr()) for t in (phi, u, v, T, dp)]
        _check(self._lib.lbm_fields_device(self._h, *ptrs, int(dtype)), "lbm_fields_device")

    def lbm_diag(self, raise_unstable=True):
        m, r, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        rc = self._lib.lbm_diag(self._h, ctypes.byref(m), ctypes.byref(r), ctypes.byref(s))
        if rc == LBM_EUNSTABLE and not raise_unstable:
            return {"mass": m.value, "residual": r.value, "step": s.value, "unstable": True}
        _check(rc, "lbm_diag")
        return {"mass": m.value, "residual": r.value, "step": s.value, "unstable": False}

    def lbm_set_check_interval(self, K: int):
        _check(self._lib.lbm_set_check_interval(self._h, int(K)), "lbm_set_check_interval")

    def lbm_run_to_steady(self, tol: float, max_steps: int):
        n = ctypes.c_int64()
        rc = self._lib.lbm_run_to_steady(self._h, float(tol), int(max_steps), ctypes.byref(n))
        if rc not in (LBM_OK, LBM_ETIMEOUT):
            _check(rc, "lbm_run_to_steady")
        return rc == LBM_OK, n.value

    def lbm_get_state(self) -> dict:
        N = (self.ny, self.nx)
        st = {"f": np.empty((self.q_phi,) + N), "g": np.empty((9,) + N), "h": np.empty((self.q_T,) + N),
              "dp": np.empty(N)}
        _check(self._lib.lbm_get_state(self._h, _dptr(st["f"]), _dptr(st["g"]), _dptr(st["h"]), _dptr(st["dp"])),
               "lbm_get_state")
        return st

    def lbm_set_state(self, st: dict):
        N = (self.ny, self.nx)
        a = [np.ascontiguousarray(st["f"], dtype=np.float64).reshape((self.q_phi,) + N),
             np.ascontiguousarray(st["g"], dtype=np.float64).reshape((9,) + N),
             np.ascontiguousarray(st["h"], dtype=np.float64).reshape((self.q_T,) + N),
             np.ascontiguousarray(st["dp"], dtype=np.float64).reshape(N)]
        _check(self._lib.lbm_set_state(self._h, *[_dptr(x) for x in a]), "lbm_set_state")

    def lbm_save(self, path: str):
        _check(self._lib.lbm_save(self._h, os.fsencode(path)), "lbm_save")

    def lbm_load(self, path: str):
        _check(self._lib.lbm_load(self._h, os.fsencode(path)), "lbm_load")

    def lbm_set_segment(self, rows: int):
        _check(self._lib.lbm_set_segment(self._h, int(rows)), "lbm_set_segment")

    def lbm_test_stall_copies(self, on: bool):
        _check(self._lib.lbm_test_stall_copies(self._h, int(bool(on))), "lbm_test_stall_copies")

    def lbm_autotune(self, reps: int = 20) -> int:
        r = ctypes.c_int32()
        _check(self._lib.lbm_autotune(self._h, int(reps), ctypes.byref(r)), "lbm_autotune")
        return r.value

    def lbm_bytes_per_node(self) -> int:
        b = ctypes.c_int64()
        _check(self._lib.lbm_bytes_per_node(self._h, ctypes.byref(b)), "lbm_bytes_per_node")
        return b.value

    def lbm_launch_count(self) -> int:
        b = ctypes.c_int64()
        _check(self._lib.lbm_launch_count(self._h, ctypes.byref(b)), "lbm_launch_count")
        return b.value

    # -- short aliases
    step = lbm_step
    fields = lbm_fields
    diag = lbm_diag
    init_fields = lbm_init_fields
    get_state = lbm_get_state
    set_state = lbm_set_state


class LbmBatch:
    """Many channels of uneven size stepped together (one lbm_batch)."""

    def __init__(self, workloads: list, precision="fp32", stream=None):
        self._lib = load()
        self.workloads = [dict(w) for w in workloads]
        n = len(workloads)
        doms = (LbmDomain * n)(*[make_domain(w["domain"], precision) for w in workloads])
        prms = (LbmParams * n)(*[make_params(w["params"]) for w in workloads])
        self.n = n
        self.shapes = [(int(w["domain"]["ny"]), int(w["domain"]["nx"])) for w in workloads]
        self._h = _H()
        s = stream_handle(stream)
        _check(self._lib.lbm_batch_create(n, doms, prms, s, ctypes.byref(self._h)), "lbm_batch_create")

    def lbm_batch_destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbm_batch_destroy(self._h)
            self._h = _H()

    close = lbm_batch_destroy

    def __del__(self):
        try:
            self.lbm_batch_destroy()
        except Exception:
            pass

    def lbm_batch_set_check_interval(self, K: int):
        _check(self._lib.lbm_batch_set_check_interval(self._h, int(K)), "lbm_batch_set_check_interval")

    def lbm_batch_autotune(self, reps: int = 10) -> int:
        r = ctypes.c_int32()
        _check(self._lib.lbm_batch_autotune(self._h, int(reps), ctypes.byref(r)), "lbm_batch_autotune")
        return r.value

    def lbm_batch_step(self, n: int):
        _check(self._lib.lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def lbm_batch_run_to_steady(self, tol: float, max_steps: int):
        steps = (ctypes.c_int64 * self.n)()
        conv = (ctypes.c_int32 * self.n)()
        rc = self._lib.lbm_batch_run_to_steady(self._h, float(tol), int(max_steps), steps, conv)
        if rc not in (LBM_OK, LBM_ETIMEOUT):
            _check(rc, "lbm_batch_run_to_steady")
        return list(steps), [bool(c) for c in conv]

    def lbm_batch_fields(self, c: int) -> dict:
        shape = self.shapes[c]
        out = {k: np.empty(shape) for k in ("phi", "u", "v", "T", "dp")}
        _check(self._lib.lbm_batch_fields(self._h, int(c), *[_dptr(out[k]) for k in ("phi", "u", "v", "T", "dp")]),
               "lbm_batch_fields")
        return out

    def lbm_batch_diag(self, c: int):
        r, st = ctypes.c_double(), ctypes.c_int64()
        _check(self._lib.lbm_batch_diag(self._h, int(c), ctypes.byref(r), ctypes.byref(st)), "lbm_batch_diag")
        return {"residual": r.value, "steps": st.value}

    def lbm_batch_init_fields(self, c: int, phi=None, u=None, v=None, T=None, dp=None):
        shape = self.shapes[c]
        a = [_field(x, shape) for x in (phi, u, v, T, dp)]
        _check(self._lib.lbm_batch_init_fields(self._h, int(c), *[_dptr(x) for x in a]), "lbm_batch_init_fields")

    def lbm_batch_size(self):
        n, c, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lbm_batch_size(self._h, ctypes.byref(n), ctypes.byref(c), ctypes.byref(r)), "lbm_batch_size")
        return {"cases": n.value, "ctas": c.value, "rows": r.value}


class Cnn:
    """The warm-start surrogate (one lbm_cnn).  x, y, target: float32 CUDA tensors.

    The kernels run on `stream` (default: torch's current stream), so that tensors made by
    torch on that stream are ready when the kernels read them and the outputs are ready
    for torch's next operation on it."""

    def __init__(self, H: int, W: int, batch_max: int, bf16: bool = True, seed: int = 0, stream=None):
        self._lib = load()
        self.H, self.W = int(H), int(W)
        self._h = _H()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        s = stream_handle(stream)
        _check(self._lib.lbm_cnn_create(self.H, self.W, int(batch_max), int(bool(bf16)), int(seed), s,
                                        ctypes.byref(self._h)), "lbm_cnn_create")
        n = ctypes.c_int64()
        _check(self._lib.lbm_cnn_num_params(self._h, ctypes.byref(n)), "lbm_cnn_num_params")
        self.n_params = n.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbm_cnn_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self._lib.lbm_cnn_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "lbm_cnn_get_params")
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.lbm_cnn_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "lbm_cnn_set_params")

    def forward(self, x, y):
        _check(self._lib.lbm_cnn_forward(self._h, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                         ctypes.c_void_p(y.data_ptr())), "lbm_cnn_forward")

    def gradients(self, x, target):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self._lib.lbm_cnn_gradients(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                           int(x.shape[0]), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           ctypes.byref(loss)), "lbm_cnn_gradients")
        return g, loss.value

    def train_step(self, x, target, lr: float) -> float:
        loss = ctypes.c_double()
        _check(self._lib.lbm_cnn_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                            int(x.shape[0]), float(lr), ctypes.byref(loss)), "lbm_cnn_train_step")
        return loss.value
