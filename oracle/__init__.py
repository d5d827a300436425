"""CPU oracle of the coupled central-moment LB step (arXiv 2210.07501, Sec. 4, App. B).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only code allowed to import, link or run anything in this
package.  It shares no code with the CUDA library in ``paper_2210_07501_gb300``; the
two meet only through the seeded inputs of ``lbm_workloads``.

``lbm_oracle.c`` is the plain FP64 step (see its header for every reading of the paper
it fixes); ``analytic.py`` is the paper's closed-form creeping-flow solution (Sec. 3,
App. A, App. C) used to pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_ORACLE_SRC points the wrapper at another copy of the source; the mutation test
# uses it to plant mistakes in a copy of the oracle and check that the pins catch them.
_SRC = os.environ.get("LBM_ORACLE_SRC") or os.path.join(_HERE, "lbm_oracle.c")
_BUILD_DIR = (os.path.join(os.path.dirname(os.path.abspath(_SRC)), "_build")
              if os.environ.get("LBM_ORACLE_SRC") else os.path.join(_HERE, "_build"))
_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_libs = {}


_FMA_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle_fma.so")


def build(force: bool = False, fma: bool = False) -> str:
    """Compile the oracle with gcc: FP64, OpenMP over rows, no FMA contraction.

    ``fma=True`` builds the same source with floating-point contraction allowed (fused
    multiply-adds wherever the compiler finds them).  The two builds differ only in
    round-off; their difference measures how strongly each field amplifies FP64
    rounding, which is what the GPU parity tests derive their bars from.
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    path = _FMA_LIB_PATH if fma else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    contract = ["-ffp-contract=fast"] + (["-mfma"] if os.uname().machine in ("x86_64", "AMD64") else []) \
        if fma else ["-ffp-contract=off"]
    cmd = ["gcc", "-O2", "-std=c11"] + contract + ["-fno-fast-math", "-fopenmp",
                                                    "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class OrParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("heat_periods", ctypes.c_int32),
        ("q_phi", ctypes.c_int32), ("q_T", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("b", ctypes.c_double), ("W", ctypes.c_double),
        ("sigma0", ctypes.c_double), ("sigma1", ctypes.c_double), ("sigma2", ctypes.c_double),
        ("T_ref", ctypes.c_double), ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double),
        ("dT", ctypes.c_double),
        ("tau_flow", ctypes.c_double), ("visc_ratio", ctypes.c_double),
        ("tau_T", ctypes.c_double), ("cond_ratio", ctypes.c_double), ("tau_phi", ctypes.c_double),
        ("rho_bottom", ctypes.c_double), ("rho_top", ctypes.c_double),
        ("Fx_ext", ctypes.c_double), ("Fy_ext", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def _lib_handle(fma: bool = False):
    with _lock:
        if fma not in _libs:
            lib = ctypes.CDLL(build(fma=fma))
            lib.or_create.restype = ctypes.c_void_p
            lib.or_create.argtypes = [ctypes.POINTER(OrParams)]
            lib.or_destroy.argtypes = [ctypes.c_void_p]
            lib.or_init.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _D]
            lib.or_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            lib.or_fields.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _D]
            lib.or_get_state.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
            lib.or_set_state.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
            lib.or_mass.restype = ctypes.c_double
            lib.or_mass.argtypes = [ctypes.c_void_p]
            lib.or_step_count.restype = ctypes.c_long
            lib.or_step_count.argtypes = [ctypes.c_void_p]
            lib.or_set_threads.argtypes = [ctypes.c_int]
            lib.or_matrices.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D]
            lib.or_collide_phase_site.argtypes = [ctypes.c_int, _D] + [ctypes.c_double] * 6
            lib.or_collide_energy_site.argtypes = [ctypes.c_int, _D] + [ctypes.c_double] * 4
            lib.or_collide_flow_site.argtypes = [_D] + [ctypes.c_double] * 9
            lib.or_debug_fields.argtypes = [ctypes.c_void_p] + [_D] * 6
            lib.or_streamed.argtypes = [ctypes.c_void_p, _D, _D, _D]
            if lib.or_sizeof_params() != ctypes.sizeof(OrParams):
                raise RuntimeError("oracle parameter struct layout mismatch")
            _libs[fma] = lib
    return _libs[fma]


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _as_field(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
    return a


def make_params(domain: dict, params: dict) -> OrParams:
    p = OrParams()
    for k in ("nx", "ny", "heat_periods", "q_phi", "q_T"):
        setattr(p, k, int(domain[k]))
    p.b = float(domain["b"])
    p.W = float(domain["W"])
    for k in ("sigma0", "sigma1", "sigma2", "T_ref", "T_hot", "T_cold", "dT", "tau_flow", "visc_ratio",
              "tau_T", "cond_ratio", "tau_phi", "rho_bottom", "rho_top", "Fx_ext", "Fy_ext"):
        setattr(p, k, float(params.get(k, 0.0)))
    return p


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the oracle (0 = leave); returns the count in use."""
    r = _lib_handle().or_set_threads(int(n))
    _lib_handle(True).or_set_threads(int(n))
    return r


class Oracle:
    """Plain FP64 three-lattice LB solver on the host.

    Fields are row-major [ny][nx]; row j = 0 is next to the heated bottom wall (y = 1/2).
    """

    def __init__(self, domain: dict, params: dict, fma: bool = False):
        self._lib = _lib_handle(fma)
        self._prm = make_params(domain, params)
        self.nx, self.ny = int(domain["nx"]), int(domain["ny"])
        self.q_phi, self.q_T = int(domain["q_phi"]), int(domain["q_T"])
        self._h = self._lib.or_create(ctypes.byref(self._prm))
        if not self._h:
            raise ValueError("oracle rejected the domain/parameters")
        self.init()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.or_destroy(self._h)
            self._h = None

    __del__ = close

    def init(self, phi=None, u=None, v=None, T=None, dp=None):
        """Equilibrium state from macroscopic fields; None = default (tanh interface, rest, T_ref)."""
        shape = (self.ny, self.nx)
        arrs = [_as_field(a, shape) for a in (phi, u, v, T, dp)]
        self._keep = arrs
        rc = self._lib.or_init(self._h, *[_ptr(a) for a in arrs])
        if rc != 0:
            raise RuntimeError("or_init failed")

    def step(self, n: int = 1):
        if self._lib.or_step(self._h, int(n)) != 0:
            raise RuntimeError("or_step failed")

    @property
    def step_count(self) -> int:
        return int(self._lib.or_step_count(self._h))

    def fields(self) -> dict:
        shape = (self.ny, self.nx)
        out = {k: np.empty(shape) for k in ("phi", "u", "v", "T", "dp")}
        self._lib.or_fields(self._h, *[_ptr(out[k]) for k in ("phi", "u", "v", "T", "dp")])
        return out

    def get_state(self) -> dict:
        N = (self.ny, self.nx)
        st = {"f": np.empty((self.q_phi,) + N), "g": np.empty((9,) + N),
              "h": np.empty((self.q_T,) + N), "dp": np.empty(N)}
        self._lib.or_get_state(self._h, _ptr(st["f"]), _ptr(st["g"]), _ptr(st["h"]), _ptr(st["dp"]))
        return st

    def set_state(self, st: dict):
        N = (self.ny, self.nx)
        a = [np.ascontiguousarray(st["f"], dtype=np.float64).reshape((self.q_phi,) + N),
             np.ascontiguousarray(st["g"], dtype=np.float64).reshape((9,) + N),
             np.ascontiguousarray(st["h"], dtype=np.float64).reshape((self.q_T,) + N),
             np.ascontiguousarray(st["dp"], dtype=np.float64).reshape(N)]
        self._lib.or_set_state(self._h, *[_ptr(x) for x in a])

    def mass(self) -> float:
        return float(self._lib.or_mass(self._h))

    def debug_fields(self) -> dict:
        """grad sigma, F_t and F_p of the last step."""
        keys = ("dsx", "dsy", "ftx", "fty", "fpx", "fpy")
        out = {k: np.empty((self.ny, self.nx)) for k in keys}
        self._lib.or_debug_fields(self._h, *[_ptr(out[k]) for k in keys])
        return out

    def streamed(self) -> dict:
        """Streaming (with the wall rules) of the current state, without collision."""
        N = (self.ny, self.nx)
        st = {"f": np.empty((self.q_phi,) + N), "g": np.empty((9,) + N), "h": np.empty((self.q_T,) + N)}
        self._lib.or_streamed(self._h, _ptr(st["f"]), _ptr(st["g"]), _ptr(st["h"]))
        return st


# ---- site-level access for the pins -------------------------------------------------

def matrices(Q: int, ux: float, uy: float):
    lib = _lib_handle()
    P, Pi, F, Fi = (np.empty((Q, Q)) for _ in range(4))
    if lib.or_matrices(Q, ux, uy, _ptr(P), _ptr(Pi), _ptr(F), _ptr(Fi)) != 0:
        raise ValueError("Q must be 5 or 9")
    return P, Pi, F, Fi


def collide_phase_site(pop, phi, ux, uy, Mtnx, Mtny, omega_phi):
    p = np.array(pop, dtype=np.float64)
    _lib_handle().or_collide_phase_site(len(p), _ptr(p), phi, ux, uy, Mtnx, Mtny, omega_phi)
    return p


def collide_energy_site(pop, T, ux, uy, omega_T):
    p = np.array(pop, dtype=np.float64)
    _lib_handle().or_collide_energy_site(len(p), _ptr(p), T, ux, uy, omega_T)
    return p


def collide_flow_site(pop, rho, dp, ux, uy, Fpx, Fpy, Ftx, Fty, omega_nu):
    """Flow collision on deviation populations g - w p0 (p0 = rho_A c^2)."""
    p = np.array(pop, dtype=np.float64)
    _lib_handle().or_collide_flow_site(_ptr(p), rho, dp, ux, uy, Fpx, Fpy, Ftx, Fty, omega_nu)
    return p
