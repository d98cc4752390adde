"""FP64 CPU oracle of the coupled power-law / Cahn-Hilliard LB step (arXiv 2207.09431).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library under ``paper_2207_09431_gb300/`` and never
imports it; both sides only share the seeded input generators.

The numerics live in ``lbm_oracle.c`` (plain C, double precision, one
whole-field pass per quantity).  This module compiles it with gcc on first use
and wraps it with ctypes.

Parity status per function (what pins it lives in ``tests/test_oracle_pins.py``):
  step / set_fields / init_bubbles   pinned (closed forms, invariants, hand step)
  raw observable sums                pinned (prescribed symmetric disc: centroid,
                                     mean velocity, masses, brute-force extents)
  observables post-processing        pinned (Tables 5-7 of the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

from .observables import postprocess  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATHS = {"f64": os.path.join(_BUILD_DIR, "liblbm_oracle.so"),
              "f32": os.path.join(_BUILD_DIR, "liblbm_oracle_f32.so"),
              "f64-omp": os.path.join(_BUILD_DIR, "liblbm_oracle_omp.so"),
              "f32-omp": os.path.join(_BUILD_DIR, "liblbm_oracle_f32_omp.so")}
_libs = {}


def build(force: bool = False, precision: str = "f64") -> str:
    """Compile the oracle into a shared library (gcc -O3, no machine-specific
    flags, ISO C so that no multiply-add is contracted).

    precision "f64" is the oracle.  "f32" compiles the same source with FP32
    internals; the GPU parity tests use it only to measure the FP32 rounding
    floor of the scheme on a case.  "f64-omp" and "f32-omp" are those builds
    with OpenMP, whose whole-field passes share their nodes among the host's
    threads (the same results, bit for bit): the timed CPU baseline and the
    tests on paper-size lattices use them."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    path = _LIB_PATHS[precision]
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD_DIR)
    os.close(fd)
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    if precision.startswith("f32"):
        cmd.insert(1, "-DORACLE_REAL=float")
    if precision.endswith("-omp"):
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("ncomp", ctypes.c_int),
        ("periodic_y", ctypes.c_int),
        ("rho", ctypes.c_double * 3), ("tau", ctypes.c_double * 3),
        ("powerlaw", ctypes.c_int),
        ("pl_n", ctypes.c_double), ("pl_k", ctypes.c_double),
        ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
        ("sigma12", ctypes.c_double), ("sigma13", ctypes.c_double),
        ("sigma23", ctypes.c_double), ("Lambda", ctypes.c_double),
        ("xi", ctypes.c_double), ("D0", ctypes.c_double),
        ("mobility", ctypes.c_int),
        ("gravity", ctypes.c_double), ("force_x", ctypes.c_double),
        ("fd_scheme", ctypes.c_int),
        ("open_x", ctypes.c_int), ("u_in", ctypes.c_double), ("c_in", ctypes.c_double * 2),
    ]


def _load(precision: str = "f64"):
    if precision in _libs:
        return _libs[precision]
    lib = ctypes.CDLL(build(precision=precision))
    P = ctypes.POINTER
    d = P(ctypes.c_double)
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [P(_Params)]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_set_fields.argtypes = [ctypes.c_void_p, d, d, d, d]
    lib.orc_init_bubbles.argtypes = [ctypes.c_void_p, d, ctypes.c_int, ctypes.c_ulonglong,
                                     ctypes.c_double]
    lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    lib.orc_get_step.restype = ctypes.c_longlong
    lib.orc_get_step.argtypes = [ctypes.c_void_p]
    lib.orc_get_field.restype = ctypes.c_longlong
    lib.orc_get_field.argtypes = [ctypes.c_void_p, ctypes.c_int, d]
    lib.orc_observables.argtypes = [ctypes.c_void_p, ctypes.c_int, d]
    _libs[precision] = lib
    return lib


FIELD_IDS = {"C1": 0, "C2": 1, "C3": 2, "rho": 3, "p": 4, "ux": 5, "uy": 6, "tau": 7,
             "mu1": 8, "mu2": 9, "mu3": 10, "g": 11, "h": 12, "shear": 13, "S": 14, "V": 15}

DEFAULTS = dict(periodic_y=0, rho=(1.0, 1.0, 1.0), tau=(0.5, 0.5, 0.5), powerlaw=0,
                pl_n=1.0, pl_k=1.0 / 6.0, tau_min=0.01, tau_max=3.0, sigma12=1e-3,
                sigma13=1e-3, sigma23=1e-3, Lambda=0.0, xi=4.0, D0=4.0 / 300.0,
                mobility=0, gravity=0.0, force_x=0.0, fd_scheme=0, gas_comp=3,
                open_x=0, u_in=0.0, c_in=(1.0, 0.0))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One FP64 lattice; ``params`` is a dict with the keys of ``DEFAULTS`` plus
    nx, ny, ncomp."""

    def __init__(self, params: dict, precision: str = "f64"):
        lib = _load(precision)
        full = dict(DEFAULTS)
        full.update(params)
        self.params = full
        pr = _Params()
        for name, ctype in _Params._fields_:
            v = full[name]
            if name in ("rho", "tau"):
                arr = (ctypes.c_double * 3)(*[float(x) for x in v])
                setattr(pr, name, arr)
            elif name == "c_in":
                setattr(pr, name, (ctypes.c_double * 2)(*[float(x) for x in v]))
            elif ctype is ctypes.c_int:
                setattr(pr, name, int(v))
            else:
                setattr(pr, name, float(v))
        self._h = lib.orc_create(ctypes.byref(pr))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self._lib = lib
        self.nx, self.ny, self.ncomp = int(full["nx"]), int(full["ny"]), int(full["ncomp"])
        self.nh = self.ncomp - 1
        self.n = self.nx * self.ny

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def set_fields(self, C, p=None, ux=None, uy=None):
        C = np.ascontiguousarray(C, dtype=np.float64).reshape(self.nh, self.n)
        arrs = [C]
        ptrs = [_dptr(C)]
        for f in (p, ux, uy):
            if f is None:
                ptrs.append(None)
            else:
                a = np.ascontiguousarray(f, dtype=np.float64).reshape(self.n)
                arrs.append(a)
                ptrs.append(_dptr(a))
        rc = self._lib.orc_set_fields(self._h, *ptrs)
        if rc != 0:
            raise RuntimeError("orc_set_fields failed")

    def init_bubbles(self, bubbles, seed=0, noise=0.0):
        b = np.ascontiguousarray(np.asarray(bubbles, dtype=np.float64).reshape(-1, 4))
        rc = self._lib.orc_init_bubbles(self._h, _dptr(b), b.shape[0], int(seed), float(noise))
        if rc != 0:
            raise ValueError("orc_init_bubbles rejected the bubbles")

    def step(self, nsteps: int = 1):
        self._lib.orc_step(self._h, int(nsteps))

    @property
    def step_count(self) -> int:
        return int(self._lib.orc_get_step(self._h))

    def field(self, name: str) -> np.ndarray:
        fid = FIELD_IDS[name]
        if name == "g":
            shape = (9, self.ny, self.nx)
        elif name == "h":
            shape = (self.nh, 9, self.ny, self.nx)
        elif name in ("S", "V"):
            shape = (self.nh, self.ny, self.nx)
        else:
            shape = (self.ny, self.nx)
        out = np.empty(int(np.prod(shape)), dtype=np.float64)
        got = self._lib.orc_get_field(self._h, fid, _dptr(out))
        if got != out.size:
            raise RuntimeError(f"orc_get_field({name}) returned {got}")
        return out.reshape(shape)

    def raw_observables(self, gas_comp=None) -> np.ndarray:
        gc = int(self.params["gas_comp"] if gas_comp is None else gas_comp)
        out = np.empty(15, dtype=np.float64)
        self._lib.orc_observables(self._h, gc, _dptr(out))
        return out

    def observables(self, gas_comp=None) -> dict:
        return postprocess(self.params, self.raw_observables(gas_comp), gas_comp)
