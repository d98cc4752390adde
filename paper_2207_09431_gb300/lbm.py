"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (same names).

Argument marshalling only: every step of the method runs in the CUDA library
``liblbm_gb300.so`` built from ``csrc/`` for sm_103a.  PyTorch supplies the
device arena and the stream.  There is no fallback: if the library or a GPU
is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB
_lib = None

STATUS = {0: "LBM_OK", -1: "LBM_E_INVAL", -2: "LBM_E_NOMEM", -3: "LBM_E_CUDA", -4: "LBM_E_DIVERGED",
          -5: "LBM_E_TIMEOUT", -6: "LBM_E_STATE", -7: "LBM_E_IO", -8: "LBM_E_RANGE"}
STATIC_MAX_NODES = 1 << 20
FIELD_IDS = {"C1": 0, "C2": 1, "C3": 2, "rho": 3, "p": 4, "ux": 5, "uy": 6, "tau": 7, "mu1": 8,
             "mu2": 9, "mu3": 10, "g": 11, "h": 12, "shear": 13, "SV": 16}


class LbmError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("ncomp", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("rho", ctypes.c_double * 3), ("tau", ctypes.c_double * 3),
        ("powerlaw", ctypes.c_int), ("pl_n", ctypes.c_double), ("pl_k", ctypes.c_double),
        ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
        ("sigma12", ctypes.c_double), ("sigma13", ctypes.c_double), ("sigma23", ctypes.c_double),
        ("Lambda", ctypes.c_double), ("xi", ctypes.c_double), ("D0", ctypes.c_double),
        ("mobility", ctypes.c_int), ("gravity", ctypes.c_double), ("force_x", ctypes.c_double),
        ("fd_scheme", ctypes.c_int), ("storage", ctypes.c_int), ("gas_comp", ctypes.c_int),
        ("collapse_h", ctypes.c_int), ("open_x", ctypes.c_int), ("u_in", ctypes.c_double),
        ("c_in", ctypes.c_double * 2),
    ]


class lbm_bubble(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("r", ctypes.c_double), ("comp", ctypes.c_int)]


class lbm_run_opts(ctypes.Structure):
    _fields_ = [("window", ctypes.c_longlong), ("rtol", ctypes.c_double), ("max_steps", ctypes.c_longlong),
                ("top_margin", ctypes.c_double)]


RUN_OUTCOMES = {0: "max_steps", 1: "terminal", 2: "top", -1: "diverged", -2: "skipped"}


class lbm_obs(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_longlong), ("mass", ctypes.c_double * 3), ("mass_thr", ctypes.c_double * 3),
        ("area", ctypes.c_double), ("centroid", ctypes.c_double * 2), ("velocity", ctypes.c_double * 2),
        ("rise_velocity", ctypes.c_double), ("y_integrated", ctypes.c_double), ("d_eq", ctypes.c_double),
        ("aspect_E", ctypes.c_double), ("drag_coefficient", ctypes.c_double), ("Re", ctypes.c_double),
        ("Eo", ctypes.c_double), ("Mo", ctypes.c_double), ("raw", ctypes.c_double * 15),
    ]


DEFAULTS = dict(periodic_y=0, rho=(1.0, 1.0, 1.0), tau=(0.5, 0.5, 0.5), powerlaw=0, pl_n=1.0,
                pl_k=1.0 / 6.0, tau_min=0.01, tau_max=3.0, sigma12=1e-3, sigma13=1e-3, sigma23=1e-3,
                Lambda=0.0, xi=4.0, D0=4.0 / 300.0, mobility=0, gravity=0.0, force_x=0.0, fd_scheme=0,
                storage=0, gas_comp=3, collapse_h=0, open_x=0, u_in=0.0, c_in=(1.0, 0.0))

EXPORTED = ["lbm_version", "lbm_required_bytes", "lbm_create", "lbm_init_bubbles", "lbm_set_fields",
            "lbm_step", "lbm_observables", "lbm_get_field", "lbm_save", "lbm_load", "lbm_destroy",
            "lbm_last_error", "lbm_postprocess", "lbm_kernels_per_step", "lbm_kernel_name",
            "lbm_profile_step", "lbm_observables_static", "lbm_autotune", "lbm_kernel_config_count",
            "lbm_set_kernel_config", "lbm_batch_required_bytes", "lbm_batch_create", "lbm_batch_case",
            "lbm_batch_set_active", "lbm_batch_step", "lbm_batch_autotune", "lbm_batch_destroy",
            "lbm_batch_last_error", "lbm_batch_set_persistent", "lbm_batch_run", "surr_param_count", "surr_required_bytes", "surr_create", "surr_destroy",
            "surr_last_error", "surr_get_weights", "surr_forward_backward", "surr_train", "surr_predict", "surr_answer",
            "surr_train_cv", "surr_local_residual", "surr_set_local_trust"]


def load_library(path: str | None = None):
    """Loads the CUDA library (building it first if it is missing)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        _build.build()
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    vp, d = ctypes.c_void_p, P(ctypes.c_double)
    lib.lbm_version.restype = ctypes.c_int
    lib.lbm_required_bytes.restype = ctypes.c_size_t
    lib.lbm_required_bytes.argtypes = [P(lbm_params)]
    lib.lbm_create.argtypes = [P(lbm_params), vp, ctypes.c_size_t, vp, P(vp)]
    lib.lbm_init_bubbles.argtypes = [vp, P(lbm_bubble), ctypes.c_int, ctypes.c_ulonglong, ctypes.c_double]
    lib.lbm_set_fields.argtypes = [vp, d, d, d, d]
    lib.lbm_step.argtypes = [vp, ctypes.c_longlong]
    lib.lbm_observables.argtypes = [vp, P(lbm_obs)]
    lib.lbm_get_field.argtypes = [vp, ctypes.c_int, d, ctypes.c_size_t]
    lib.lbm_save.argtypes = [vp, ctypes.c_char_p]
    lib.lbm_load.argtypes = [vp, ctypes.c_char_p]
    lib.lbm_destroy.argtypes = [vp]
    lib.lbm_destroy.restype = None
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_postprocess.argtypes = [P(lbm_params), d, P(lbm_obs)]
    lib.lbm_kernels_per_step.argtypes = [vp]
    lib.lbm_kernel_name.argtypes = [vp, ctypes.c_int]
    lib.lbm_kernel_name.restype = ctypes.c_char_p
    lib.lbm_profile_step.argtypes = [vp, ctypes.c_longlong, d, ctypes.c_int]
    lib.lbm_autotune.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
    lib.lbm_kernel_config_count.argtypes = [vp]
    lib.lbm_set_kernel_config.argtypes = [vp, ctypes.c_int]
    lib.lbm_batch_required_bytes.restype = ctypes.c_size_t
    lib.lbm_batch_required_bytes.argtypes = [P(lbm_params), ctypes.c_int]
    lib.lbm_batch_create.argtypes = [P(lbm_params), ctypes.c_int, vp, ctypes.c_size_t, vp, P(vp)]
    lib.lbm_batch_case.restype = vp
    lib.lbm_batch_case.argtypes = [vp, ctypes.c_int]
    lib.lbm_batch_set_active.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.lbm_batch_step.argtypes = [vp, ctypes.c_longlong]
    lib.lbm_batch_autotune.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
    lib.lbm_batch_set_persistent.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    lib.lbm_batch_run.argtypes = [vp, P(lbm_run_opts), P(lbm_obs), P(ctypes.c_int), P(ctypes.c_longlong)]
    lib.lbm_batch_destroy.argtypes = [vp]
    lib.lbm_batch_destroy.restype = None
    lib.lbm_batch_last_error.argtypes = [vp]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    lib.surr_param_count.restype = ctypes.c_int
    lib.surr_required_bytes.restype = ctypes.c_size_t
    lib.surr_required_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.surr_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, vp, ctypes.c_size_t, vp, P(vp)]
    lib.surr_destroy.argtypes = [vp]
    lib.surr_destroy.restype = None
    lib.surr_last_error.argtypes = [vp]
    lib.surr_last_error.restype = ctypes.c_char_p
    lib.surr_get_weights.argtypes = [vp, ctypes.c_int, d]
    lib.surr_forward_backward.argtypes = [vp, ctypes.c_int, d, d, ctypes.c_int, d, d, d]
    lib.surr_train.argtypes = [vp, d, d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_ulonglong, d]
    lib.surr_predict.argtypes = [vp, d, ctypes.c_int, d, d, P(ctypes.c_int)]
    lib.surr_train_cv.argtypes = [vp, d, d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_ulonglong, d, d]
    lib.surr_local_residual.argtypes = [vp, d, ctypes.c_int, ctypes.c_int, d]
    lib.surr_set_local_trust.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    lib.surr_answer.argtypes = [vp, d, P(lbm_params), P(lbm_bubble), ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, P(lbm_run_opts), vp, ctypes.c_size_t, d, P(ctypes.c_int),
                                P(ctypes.c_int)]
    lib.lbm_observables_static.argtypes = [P(lbm_params), vp, vp, ctypes.c_int, ctypes.c_longlong, d, vp]
    for name in EXPORTED:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def make_params(params: dict) -> lbm_params:
    full = dict(DEFAULTS)
    full.update(params)
    pr = lbm_params()
    for name, ctype in lbm_params._fields_:
        v = full[name]
        if name in ("rho", "tau"):
            setattr(pr, name, (ctypes.c_double * 3)(*[float(x) for x in v]))
        elif name == "c_in":
            setattr(pr, name, (ctypes.c_double * 2)(*[float(x) for x in v]))
        elif ctype is ctypes.c_int:
            setattr(pr, name, int(v))
        else:
            setattr(pr, name, float(v))
    return pr


def obs_to_dict(o: lbm_obs) -> dict:
    out = {}
    for name, _ in lbm_obs._fields_:
        v = getattr(o, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


def _check(h, rc, what):
    if rc != 0:
        msg = load_library().lbm_last_error(h).decode() if h else ""
        raise LbmError(rc, f"{what}: {msg}")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --- the C ABI, same names ------------------------------------------------

def lbm_version() -> int:
    return load_library().lbm_version()


def lbm_required_bytes(params) -> int:
    pr = params if isinstance(params, lbm_params) else make_params(params)
    return int(load_library().lbm_required_bytes(ctypes.byref(pr)))


def lbm_create(params, arena_ptr: int, arena_bytes: int, stream_ptr: int):
    pr = params if isinstance(params, lbm_params) else make_params(params)
    h = ctypes.c_void_p()
    rc = load_library().lbm_create(ctypes.byref(pr), ctypes.c_void_p(arena_ptr), arena_bytes,
                                   ctypes.c_void_p(stream_ptr), ctypes.byref(h))
    _check(None, rc, "lbm_create")
    return h


def lbm_init_bubbles(h, bubbles, seed=0, noise=0.0):
    arr = (lbm_bubble * max(1, len(bubbles)))()
    for i, (cx, cy, r, c) in enumerate(bubbles):
        arr[i] = lbm_bubble(float(cx), float(cy), float(r), int(c))
    _check(h, load_library().lbm_init_bubbles(h, arr, len(bubbles), int(seed), float(noise)), "lbm_init_bubbles")


def lbm_set_fields(h, C, p=None, ux=None, uy=None):
    C = np.ascontiguousarray(C, dtype=np.float64)
    keep = [C]
    ptrs = [_dptr(C)]
    for f in (p, ux, uy):
        if f is None:
            ptrs.append(None)
        else:
            a = np.ascontiguousarray(f, dtype=np.float64)
            keep.append(a)
            ptrs.append(_dptr(a))
    _check(h, load_library().lbm_set_fields(h, *ptrs), "lbm_set_fields")


def lbm_step(h, nsteps: int = 1):
    _check(h, load_library().lbm_step(h, int(nsteps)), "lbm_step")


def lbm_observables(h) -> dict:
    o = lbm_obs()
    _check(h, load_library().lbm_observables(h, ctypes.byref(o)), "lbm_observables")
    return obs_to_dict(o)


def lbm_get_field(h, name: str, nx: int, ny: int, nh: int) -> np.ndarray:
    fid = FIELD_IDS[name]
    if name == "g":
        shape = (9, ny, nx)
    elif name == "h":
        shape = (nh, 9, ny, nx)
    elif name == "SV":
        shape = (nh, ny, nx)
    else:
        shape = (ny, nx)
    out = np.empty(shape, dtype=np.float64)
    _check(h, load_library().lbm_get_field(h, fid, _dptr(out), out.size), "lbm_get_field")
    return out


def lbm_save(h, path: str):
    _check(h, load_library().lbm_save(h, path.encode()), "lbm_save")


def lbm_load(h, path: str):
    _check(h, load_library().lbm_load(h, path.encode()), "lbm_load")


def lbm_destroy(h):
    if h:
        load_library().lbm_destroy(h)


def lbm_last_error(h) -> str:
    return load_library().lbm_last_error(h).decode()


def lbm_postprocess(params, raw) -> dict:
    pr = params if isinstance(params, lbm_params) else make_params(params)
    r = np.ascontiguousarray(raw, dtype=np.float64)
    o = lbm_obs()
    _check(None, load_library().lbm_postprocess(ctypes.byref(pr), _dptr(r), ctypes.byref(o)), "lbm_postprocess")
    return obs_to_dict(o)


def lbm_kernels_per_step(h) -> int:
    return int(load_library().lbm_kernels_per_step(h))


def lbm_kernel_name(h, i: int) -> str:
    return load_library().lbm_kernel_name(h, int(i)).decode()


def lbm_profile_step(h, nsteps: int) -> dict:
    k = lbm_kernels_per_step(h)
    out = np.zeros(max(k, 1), dtype=np.float64)
    _check(h, load_library().lbm_profile_step(h, int(nsteps), _dptr(out), out.size), "lbm_profile_step")
    return {lbm_kernel_name(h, i): float(out[i]) for i in range(k)}


def lbm_autotune(h, reps: int = 5) -> int:
    chosen = ctypes.c_int(0)
    _check(h, load_library().lbm_autotune(h, int(reps), ctypes.byref(chosen)), "lbm_autotune")
    return int(chosen.value)


def lbm_kernel_config_count(h) -> int:
    return int(load_library().lbm_kernel_config_count(h))


def lbm_set_kernel_config(h, config: int):
    _check(h, load_library().lbm_set_kernel_config(h, int(config)), "lbm_set_kernel_config")


def lbm_observables_static(params, g_ptr: int, hc_ptr: int, pitch: int, plane_stride: int,
                           stream_ptr: int = 0) -> np.ndarray:
    """Raw observable sums (15 doubles) of a state in caller-held device buffers;
    allocates no device memory (see include/lbm.h)."""
    pr = params if isinstance(params, lbm_params) else make_params(params)
    out = np.zeros(15, dtype=np.float64)
    rc = load_library().lbm_observables_static(ctypes.byref(pr), ctypes.c_void_p(g_ptr), ctypes.c_void_p(hc_ptr),
                                               int(pitch), int(plane_stride), _dptr(out),
                                               ctypes.c_void_p(stream_ptr))
    _check(None, rc, "lbm_observables_static")
    return out


def _check_batch(b, rc, what):
    if rc != 0:
        raise LbmError(rc, f"{what}: {load_library().lbm_batch_last_error(b).decode()}")


def lbm_batch_required_bytes(cases) -> int:
    arr = (lbm_params * len(cases))(*[c if isinstance(c, lbm_params) else make_params(c) for c in cases])
    return int(load_library().lbm_batch_required_bytes(arr, len(cases)))


def lbm_batch_create(cases, arena_ptr: int, arena_bytes: int, stream_ptr: int):
    arr = (lbm_params * len(cases))(*[c if isinstance(c, lbm_params) else make_params(c) for c in cases])
    b = ctypes.c_void_p()
    rc = load_library().lbm_batch_create(arr, len(cases), ctypes.c_void_p(arena_ptr), arena_bytes,
                                         ctypes.c_void_p(stream_ptr), ctypes.byref(b))
    _check(None, rc, "lbm_batch_create")
    return b


def lbm_batch_case(b, i: int):
    return ctypes.c_void_p(load_library().lbm_batch_case(b, int(i)))


def lbm_batch_set_active(b, i: int, active: bool):
    _check_batch(b, load_library().lbm_batch_set_active(b, int(i), int(bool(active))), "lbm_batch_set_active")


def lbm_batch_step(b, nsteps: int):
    _check_batch(b, load_library().lbm_batch_step(b, int(nsteps)), "lbm_batch_step")


def lbm_batch_autotune(b, reps: int = 3) -> int:
    chosen = ctypes.c_int(0)
    _check_batch(b, load_library().lbm_batch_autotune(b, int(reps), ctypes.byref(chosen)), "lbm_batch_autotune")
    return int(chosen.value)


def lbm_batch_set_persistent(b, on: bool = True, spin_limit: int = 0):
    _check_batch(b, load_library().lbm_batch_set_persistent(b, 1 if on else 0, int(spin_limit)),
                 "lbm_batch_set_persistent")


def lbm_batch_run(b, ncases: int, window=2000, rtol=0.01, max_steps=40000, top_margin=1.5) -> list:
    """Runs the batch's active cases to their terminal state; per case a dict
    of the observables at the stop (rise_velocity = window-averaged U_t) with
    'outcome' and 'steps_run'."""
    opts = lbm_run_opts(int(window), float(rtol), int(max_steps), float(top_margin))
    obs = (lbm_obs * ncases)()
    outcome = (ctypes.c_int * ncases)()
    steps = (ctypes.c_longlong * ncases)()
    _check_batch(b, load_library().lbm_batch_run(b, ctypes.byref(opts), obs, outcome, steps), "lbm_batch_run")
    res = []
    for i in range(ncases):
        d = obs_to_dict(obs[i])
        d["outcome"] = RUN_OUTCOMES[outcome[i]]
        d["steps_run"] = int(steps[i])
        res.append(d)
    return res


def lbm_batch_destroy(b):
    if b:
        load_library().lbm_batch_destroy(b)


def lbm_batch_last_error(b) -> str:
    return load_library().lbm_batch_last_error(b).decode()


class Batch:
    """Cases advancing together in one launch per step; `case(i)` gives a view
    with the single-lattice methods (init, fields, observables)."""

    def __init__(self, cases, device="cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU path exists)")
        self.params = []
        for c in cases:
            full = dict(DEFAULTS)
            full.update(c)
            self.params.append(full)
        prs = [make_params(c) for c in self.params]
        self.nbytes = lbm_batch_required_bytes(prs)
        if self.nbytes == 0:
            raise LbmError(-1, "invalid batch parameters")
        self.arena = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        # a created stream, so that runs of steps can be captured as CUDA graphs
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.arena.device)
        torch.cuda.current_stream(self.arena.device).synchronize()
        self.b = lbm_batch_create(prs, self.arena.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            lbm_batch_destroy(b)
            self.b = None

    def __len__(self):
        return len(self.params)

    def case(self, i) -> "CaseView":
        return CaseView(self, i)

    def step(self, nsteps):
        lbm_batch_step(self.b, nsteps)

    def set_active(self, i, active):
        lbm_batch_set_active(self.b, i, active)

    def autotune(self, reps=3) -> int:
        return lbm_batch_autotune(self.b, reps)

    def run(self, window=2000, rtol=0.01, max_steps=40000, top_margin=1.5) -> list:
        """Every active case to its terminal state (see lbm_batch_run)."""
        return lbm_batch_run(self.b, len(self.params), window, rtol, max_steps, top_margin)

    def set_persistent(self, on=True, spin_limit=0):
        """One cooperative launch for many steps (see lbm_batch_set_persistent)."""
        lbm_batch_set_persistent(self.b, on, spin_limit)


class CaseView:
    """Single-lattice calls on case i of a Batch (the batch owns the handle)."""

    def __init__(self, batch, i):
        self._batch = batch
        self.h = lbm_batch_case(batch.b, i)
        p = batch.params[i]
        self.nx, self.ny, self.nh = int(p["nx"]), int(p["ny"]), int(p["ncomp"]) - 1

    def init_bubbles(self, bubbles, seed=0, noise=0.0):
        lbm_init_bubbles(self.h, bubbles, seed, noise)

    def set_fields(self, C, p=None, ux=None, uy=None):
        lbm_set_fields(self.h, C, p, ux, uy)

    def observables(self) -> dict:
        return lbm_observables(self.h)

    def field(self, name) -> np.ndarray:
        return lbm_get_field(self.h, name, self.nx, self.ny, self.nh)


def _check_surr(n, rc, what):
    if rc != 0:
        msg = load_library().surr_last_error(n).decode() if n else ""
        raise LbmError(rc, f"{what}: {msg}")


def surr_param_count() -> int:
    return int(load_library().surr_param_count())


def surr_required_bytes(members: int, max_batch: int, max_rows: int) -> int:
    return int(load_library().surr_required_bytes(members, max_batch, max_rows))


def surr_create(members, max_batch, max_rows, init_weights, arena_ptr, arena_bytes, stream_ptr):
    w = np.ascontiguousarray(init_weights, dtype=np.float64)
    n = ctypes.c_void_p()
    rc = load_library().surr_create(int(members), int(max_batch), int(max_rows), _dptr(w), ctypes.c_void_p(arena_ptr),
                                    arena_bytes, ctypes.c_void_p(stream_ptr), ctypes.byref(n))
    _check_surr(None, rc, "surr_create")
    return n


def surr_destroy(n):
    if n:
        load_library().surr_destroy(n)


def surr_get_weights(n, member: int) -> np.ndarray:
    out = np.zeros(surr_param_count())
    _check_surr(n, load_library().surr_get_weights(n, int(member), _dptr(out)), "surr_get_weights")
    return out


def surr_forward_backward(n, member, X, T=None):
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows = X.shape[0]
    Y = np.zeros((rows, 2))
    loss = np.zeros(1)
    grads = np.zeros(surr_param_count())
    Tp = None
    if T is not None:
        T = np.ascontiguousarray(T, dtype=np.float64)
        Tp = _dptr(T)
    rc = load_library().surr_forward_backward(n, int(member), _dptr(X), Tp, rows, _dptr(Y), _dptr(loss), _dptr(grads))
    _check_surr(n, rc, "surr_forward_backward")
    return Y, float(loss[0]), grads


def surr_train(n, X, Y, epochs, batch, lr, seed=0) -> float:
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    fl = np.zeros(1)
    rc = load_library().surr_train(n, _dptr(X), _dptr(Y), X.shape[0], int(epochs), int(batch), float(lr), int(seed),
                                   _dptr(fl))
    _check_surr(n, rc, "surr_train")
    return float(fl[0])


def surr_train_cv(n, X, Y, folds, epochs, batch, lr, seed, init_weights) -> float:
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    w = np.ascontiguousarray(init_weights, dtype=np.float64)
    fl = np.zeros(1)
    rc = load_library().surr_train_cv(n, _dptr(X), _dptr(Y), X.shape[0], int(folds), int(epochs), int(batch),
                                      float(lr), int(seed), _dptr(w), _dptr(fl))
    _check_surr(n, rc, "surr_train_cv")
    return float(fl[0])


def surr_local_residual(n, X, k) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0])
    _check_surr(n, load_library().surr_local_residual(n, _dptr(X), X.shape[0], int(k), _dptr(out)),
                "surr_local_residual")
    return out


def surr_set_local_trust(n, k, max_residual):
    _check_surr(n, load_library().surr_set_local_trust(n, int(k), float(max_residual)), "surr_set_local_trust")


def surr_predict(n, X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows = X.shape[0]
    mean, spread = np.zeros((rows, 2)), np.zeros((rows, 2))
    outside = (ctypes.c_int * rows)()
    rc = load_library().surr_predict(n, _dptr(X), rows, _dptr(mean), _dptr(spread), outside)
    _check_surr(n, rc, "surr_predict")
    return mean, spread, np.array(list(outside), dtype=bool)


def surr_answer(n, X, cases, bubbles, max_spread, noise_amp, window, rtol, max_steps, top_margin, arena_ptr,
                arena_bytes):
    """(y (rows x 2: U_t, C_D), used_fallback, fallback outcome per row) from
    the network where trusted and the solver elsewhere (see include/lbm.h)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows = X.shape[0]
    prs = (lbm_params * rows)(*[make_params(c) for c in cases])
    bs = (lbm_bubble * rows)(*[lbm_bubble(float(b[0]), float(b[1]), float(b[2]), int(b[3])) for b in bubbles])
    opts = lbm_run_opts(int(window), float(rtol), int(max_steps), float(top_margin))
    y = np.zeros((rows, 2))
    used = (ctypes.c_int * rows)()
    outc = (ctypes.c_int * rows)()
    _check_surr(n, load_library().surr_answer(n, _dptr(X), prs, bs, rows, float(max_spread), float(noise_amp),
                                              ctypes.byref(opts), ctypes.c_void_p(arena_ptr), int(arena_bytes),
                                              _dptr(y), used, outc), "surr_answer")
    return y, np.array(used[:], dtype=bool), [RUN_OUTCOMES[o] for o in outc]


class Surrogate:
    """Ensemble network with its torch-allocated arena and stream."""

    def __init__(self, init_weights, max_batch=1024, max_rows=4096, device="cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU path exists)")
        w = np.atleast_2d(np.asarray(init_weights, dtype=np.float64))
        self.members = w.shape[0]
        self.nbytes = surr_required_bytes(self.members, max_batch, max_rows)
        self.arena = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.arena.device)
        self.n = surr_create(self.members, max_batch, max_rows, w, self.arena.data_ptr(), self.nbytes,
                             self.stream.cuda_stream)

    def __del__(self):
        n = getattr(self, "n", None)
        if n:
            surr_destroy(n)
            self.n = None

    def forward_backward(self, member, X, T=None):
        return surr_forward_backward(self.n, member, X, T)

    def weights(self, member=0):
        return surr_get_weights(self.n, member)

    def train(self, X, Y, epochs, batch, lr, seed=0):
        return surr_train(self.n, X, Y, epochs, batch, lr, seed)

    def train_cv(self, X, Y, folds, epochs, batch, lr, seed, init_weights):
        return surr_train_cv(self.n, X, Y, folds, epochs, batch, lr, seed, init_weights)

    def predict(self, X):
        return surr_predict(self.n, X)

    def local_residual(self, X, k):
        return surr_local_residual(self.n, X, k)

    def set_local_trust(self, k, max_residual):
        surr_set_local_trust(self.n, k, max_residual)

    def answer(self, X, cases, bubbles, max_spread=0.05, noise_amp=1e-8, window=2000, rtol=0.05, max_steps=40000,
               top_margin=1.5):
        """Network where trusted, solver elsewhere (surr_answer); the solver's
        batch arena is allocated here for every case, the most it can need."""
        import torch

        full = []
        for c in cases:
            q = dict(DEFAULTS)
            q.update(c)
            full.append(q)
        nbytes = lbm_batch_required_bytes([make_params(c) for c in full])
        arena = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.arena.device)
        return surr_answer(self.n, X, full, bubbles, max_spread, noise_amp, window, rtol, max_steps, top_margin,
                           arena.data_ptr(), nbytes)


class Lattice:
    """A handle plus its torch-allocated device arena and stream."""

    def __init__(self, params: dict, device="cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU path exists)")
        self.params = dict(DEFAULTS)
        self.params.update(params)
        self.nx, self.ny = int(self.params["nx"]), int(self.params["ny"])
        self.nh = int(self.params["ncomp"]) - 1
        self._pr = make_params(self.params)
        self.nbytes = lbm_required_bytes(self._pr)
        if self.nbytes == 0:
            raise LbmError(-1, "invalid parameters")
        self.arena = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.arena.device)
        self.h = lbm_create(self._pr, self.arena.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lbm_destroy(h)
            self.h = None

    def init_bubbles(self, bubbles, seed=0, noise=0.0):
        lbm_init_bubbles(self.h, bubbles, seed, noise)

    def set_fields(self, C, p=None, ux=None, uy=None):
        lbm_set_fields(self.h, C, p, ux, uy)

    def step(self, nsteps=1):
        lbm_step(self.h, nsteps)

    def observables(self) -> dict:
        return lbm_observables(self.h)

    def field(self, name) -> np.ndarray:
        return lbm_get_field(self.h, name, self.nx, self.ny, self.nh)

    def kernel_times(self, reps=5) -> dict:
        """Mean device ms of each kernel of the step (advances `reps` steps)."""
        return lbm_profile_step(self.h, reps)

    def autotune(self, reps=5) -> str:
        """Picks the fastest launch configuration; returns the kernel's name."""
        lbm_autotune(self.h, reps)
        return lbm_kernel_name(self.h, 0)

    def launches_per_step(self) -> int:
        return lbm_kernels_per_step(self.h)

    def save(self, path):
        lbm_save(self.h, path)

    def load(self, path):
        lbm_load(self.h, path)
