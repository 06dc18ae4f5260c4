"""ctypes binding of libflic (include/flic.h): argument marshalling only.

Every step of the computation runs in the CUDA library; there is no Python or CPU
fallback.  If libflic.so is missing or cannot be loaded, ``load()`` raises.
Host arrays may be numpy float64 arrays or CPU torch tensors (pinned or not);
CUDA torch tensors (float64) are passed to the device-pointer entry points.
"""
from __future__ import annotations

import ctypes
import os
from typing import Mapping, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflic.so")

FIELDS = ("rho", "mx", "my", "mz", "E", "e",
          "n", "qx", "qy", "qz",
          "nExx", "nEyy", "nEzz", "nExy", "nExz", "nEyz",
          "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz")
NFIELDS = 22

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_OOM = 0, -1, -2, -3, -4, -5
FP64, MIXED = 0, 1
PERIODIC, ISOLATED = 0, 1
HYDRO_PERIODIC, HYDRO_OUTFLOW = 0, 1

# every entry point declared in include/flic.h
EXPORTS = ("flic_init_grid", "flic_set_state", "flic_set_state_device", "flic_get_state",
           "flic_get_state_device", "flic_step", "flic_run", "flic_solve_poisson",
           "flic_step_diagnostics", "flic_diagnostics", "flic_sync", "flic_destroy",
           "flic_last_error", "flic_version", "flic_profile", "flic_launches_per_step",
           "flic_state_diagnostics_noalloc", "flic_autotune", "flic_num_tile_configs", "flic_set_tile_config",
           "flic_tile_config", "flic_ensemble_autotune", "flic_ensemble_num_tile_configs", "flic_ensemble_set_tile_config",
           "flic_ensemble_tile_config",
           "flic_ensemble_create", "flic_ensemble_set_state", "flic_ensemble_get_state", "flic_ensemble_step",
           "flic_ensemble_diagnostics", "flic_ensemble_profile", "flic_ensemble_launches_per_step",
           "flic_ensemble_destroy", "flic_ensemble_last_error")
NSTAGES = 4
STAGES = ("poisson", "gas", "bme", "finalize")


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("box_min", ctypes.c_double), ("box_max", ctypes.c_double),
                ("gamma", ctypes.c_double), ("G", ctypes.c_double), ("courant", ctypes.c_double),
                ("eta", ctypes.c_double), ("precision", ctypes.c_int), ("poisson_bc", ctypes.c_int),
                ("hydro_bc", ctypes.c_int), ("cooling", ctypes.c_double), ("flux_reading", ctypes.c_int)]


class Diag(ctypes.Structure):
    _fields_ = [("mass_gas", ctypes.c_double), ("mass_bme", ctypes.c_double),
                ("mom", ctypes.c_double * 3), ("ekin_gas", ctypes.c_double),
                ("eint_gas", ctypes.c_double), ("ekin_bme", ctypes.c_double),
                ("etherm_bme", ctypes.c_double), ("epot", ctypes.c_double),
                ("kappa_gas", ctypes.c_double), ("kappa_bme", ctypes.c_double),
                ("vmax", ctypes.c_double), ("dt", ctypes.c_double), ("time", ctypes.c_double),
                ("step", ctypes.c_longlong), ("status", ctypes.c_int)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "mom"}
        d["mom_x"], d["mom_y"], d["mom_z"] = self.mom[0], self.mom[1], self.mom[2]
        d["nonphysical"] = self.status != OK
        return d


class FlicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libflic error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libflic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FlicError(ERR_INVALID_ARG, f"{path} not found: build it with paper_1311_0861_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.flic_init_grid.argtypes = [ctypes.POINTER(GridDesc), P, ctypes.POINTER(P)]
    for name in ("flic_set_state", "flic_set_state_device", "flic_get_state", "flic_get_state_device"):
        getattr(lib, name).argtypes = [P, ctypes.POINTER(P)]
    lib.flic_step.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.flic_run.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.flic_solve_poisson.argtypes = [P, P]
    lib.flic_profile.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.flic_launches_per_step.argtypes = [P]
    lib.flic_ensemble_create.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int, P, ctypes.POINTER(P)]
    lib.flic_ensemble_set_state.argtypes = [P, ctypes.c_int, ctypes.POINTER(P)]
    lib.flic_ensemble_get_state.argtypes = [P, ctypes.c_int, ctypes.POINTER(P)]
    lib.flic_ensemble_step.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.flic_ensemble_diagnostics.argtypes = [P, ctypes.c_int, ctypes.POINTER(Diag)]
    lib.flic_ensemble_profile.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.flic_ensemble_launches_per_step.argtypes = [P]
    lib.flic_ensemble_destroy.argtypes = [P]
    lib.flic_ensemble_last_error.argtypes = [P]
    lib.flic_ensemble_last_error.restype = ctypes.c_char_p
    lib.flic_state_diagnostics_noalloc.argtypes = [ctypes.POINTER(P), P, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double, P, ctypes.POINTER(Diag)]
    IP = ctypes.POINTER(ctypes.c_int)
    DP = ctypes.POINTER(ctypes.c_double)
    lib.flic_autotune.argtypes = [P, ctypes.c_int, ctypes.c_int, DP]
    lib.flic_num_tile_configs.argtypes = [P, IP, IP]
    lib.flic_set_tile_config.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.flic_tile_config.argtypes = [P, IP, IP, ctypes.c_char_p, ctypes.c_int]
    lib.flic_ensemble_autotune.argtypes = [P, ctypes.c_int, DP]
    lib.flic_ensemble_num_tile_configs.argtypes = [P, IP, IP]
    lib.flic_ensemble_set_tile_config.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.flic_ensemble_tile_config.argtypes = [P, IP, IP, IP, IP, ctypes.c_char_p, ctypes.c_int]
    lib.flic_step_diagnostics.argtypes = [P, ctypes.POINTER(Diag)]
    lib.flic_diagnostics.argtypes = [P, ctypes.POINTER(Diag)]
    lib.flic_sync.argtypes = [P]
    lib.flic_destroy.argtypes = [P]
    lib.flic_last_error.argtypes = [P]
    lib.flic_last_error.restype = ctypes.c_char_p
    lib.flic_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("flic_last_error", "flic_version", "flic_ensemble_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr_of(a, want_device):
    """(pointer, on_device) of a float64 array-like (numpy or torch)."""
    mod = type(a).__module__
    if mod.startswith("torch"):
        if a.dtype.__repr__() != "torch.float64" or not a.is_contiguous():
            raise FlicError(ERR_INVALID_ARG, "torch tensors must be contiguous float64")
        return a.data_ptr(), a.is_cuda
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags.c_contiguous:
        raise FlicError(ERR_INVALID_ARG, "numpy arrays must be C-contiguous float64")
    return arr.ctypes.data, False


def _field_list(state, n):
    if isinstance(state, Mapping):
        arrs = [state[f] for f in FIELDS]
    else:
        arrs = [state[i] for i in range(NFIELDS)]
    for a in arrs:
        if tuple(a.shape) != (n, n, n) and int(np.prod(a.shape)) != n ** 3:
            raise FlicError(ERR_INVALID_ARG, f"field shape {tuple(a.shape)} != ({n},{n},{n})")
    return arrs


def state_diagnostics_noalloc(fields, phi, n: int, h: float, gamma: float = 5.0 / 3.0, stream: int = 0,
                              allow_nonphysical: bool = False) -> dict:
    """Diagnostics of 22 caller-owned device float64 arrays (and an optional
    device potential) through flic_state_diagnostics_noalloc, which allocates no
    device memory (for callers that cannot allocate; see include/flic.h)."""
    lib = load()
    arrs = _field_list(fields, n)
    ptrs = []
    for a in arrs:
        p, dev = _ptr_of(a, True)
        if not dev:
            raise FlicError(ERR_INVALID_ARG, "fields must be device arrays")
        ptrs.append(p)
    pp = None
    if phi is not None:
        pp, dev = _ptr_of(phi, True)
        if not dev:
            raise FlicError(ERR_INVALID_ARG, "phi must be a device array")
    d = Diag()
    rc = lib.flic_state_diagnostics_noalloc((ctypes.c_void_p * NFIELDS)(*ptrs), ctypes.c_void_p(pp), int(n),
                                            float(h), float(gamma), ctypes.c_void_p(stream or None),
                                            ctypes.byref(d))
    if rc != OK and not (rc == ERR_NONPHYSICAL and allow_nonphysical):
        raise FlicError(rc, lib.flic_last_error(None).decode())
    return d.as_dict()


class Grid:
    """One N^3 grid of the two-fluid step (a libflic handle).  ``poisson``:
    "periodic" or "isolated" gravity; ``boundary``: "periodic" or "outflow" hydro;
    ``cooling``: Lambda of the cooling placeholder; ``flux``: reading "A" or "B"
    of the Lagrangian transport velocity."""

    def __init__(self, n: int, *, box=(-1.0, 1.0), gamma=5.0 / 3.0, G=1.0, courant=0.2, eta=1e-3,
                 precision: str = "fp64", poisson: str = "periodic", boundary: str = "periodic",
                 cooling: float = 0.0, flux: str = "A", stream: int = 0):
        self.lib = load()
        self.n = int(n)
        self.h = (box[1] - box[0]) / n
        d = GridDesc(int(n), box[0], box[1], gamma, G, courant, eta,
                     {"fp64": FP64, "mixed": MIXED}[precision],
                     {"periodic": PERIODIC, "isolated": ISOLATED}[poisson],
                     {"periodic": HYDRO_PERIODIC, "outflow": HYDRO_OUTFLOW}[boundary], float(cooling),
                     {"A": 0, "B": 1}[flux])
        self._h = ctypes.c_void_p()
        rc = self.lib.flic_init_grid(ctypes.byref(d), ctypes.c_void_p(stream or None), ctypes.byref(self._h))
        if rc != OK:
            raise FlicError(rc, self.lib.flic_last_error(None).decode())
        self.precision = precision

    # -- helpers ---------------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            raise FlicError(rc, self.lib.flic_last_error(self._h).decode())
        return rc

    def _ptrs(self, arrs):
        ptrs, dev = [], None
        for a in arrs:
            p, is_dev = _ptr_of(a, None)
            if dev is None:
                dev = is_dev
            elif dev != is_dev:
                raise FlicError(ERR_INVALID_ARG, "mix of host and device arrays")
            ptrs.append(p)
        return (ctypes.c_void_p * NFIELDS)(*ptrs), dev

    # -- ABI calls ---------------------------------------------------------------
    def set_state(self, state, *, allow_nonphysical=False):
        arrs = _field_list(state, self.n)
        p, dev = self._ptrs(arrs)
        fn = self.lib.flic_set_state_device if dev else self.lib.flic_set_state
        rc = fn(self._h, p)
        if rc == ERR_NONPHYSICAL and allow_nonphysical:
            return rc
        return self._check(rc)

    def get_state(self, out=None):
        """Returns a dict of float64 (N, N, N) numpy arrays, or fills ``out``
        (dict or sequence of 22 host or device float64 arrays)."""
        if out is None:
            res = {f: np.empty((self.n, self.n, self.n)) for f in FIELDS}
            p, _ = self._ptrs([res[f] for f in FIELDS])
            self._check(self.lib.flic_get_state(self._h, p))
            return res
        arrs = _field_list(out, self.n)
        p, dev = self._ptrs(arrs)
        fn = self.lib.flic_get_state_device if dev else self.lib.flic_get_state
        self._check(fn(self._h, p))
        return out

    def step(self, dt: float = 0.0, wait: bool = True):
        if wait:
            used = ctypes.c_double()
            self._check(self.lib.flic_step(self._h, dt, ctypes.byref(used)))
            return used.value
        self._check(self.lib.flic_step(self._h, dt, None))
        return None

    def run(self, nsteps: int, dt: float = 0.0, sync: bool = True):
        self._check(self.lib.flic_run(self._h, int(nsteps), dt, int(bool(sync))))

    def profile(self, nsteps: int, dt: float = 0.0):
        """Per-stage device milliseconds summed over ``nsteps`` plain-launch steps,
        and the total elapsed milliseconds."""
        ms = (ctypes.c_double * NSTAGES)()
        tot = ctypes.c_double()
        self._check(self.lib.flic_profile(self._h, int(nsteps), dt, ms, ctypes.byref(tot)))
        return dict(zip(STAGES, list(ms))), tot.value

    def launches_per_step(self) -> int:
        return self._check_count(self.lib.flic_launches_per_step(self._h))

    def _check_count(self, rc):
        if rc < 0:
            raise FlicError(rc, self.lib.flic_last_error(self._h).decode())
        return rc

    # -- launch-shape tuner ---------------------------------------------------------
    def num_tile_configs(self):
        """(number of compiled gas-kernel shapes, number of moment-kernel shapes)."""
        ng, nb = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.flic_num_tile_configs(self._h, ctypes.byref(ng), ctypes.byref(nb)))
        return ng.value, nb.value

    def set_tile_config(self, gas: int = -1, bme: int = -1):
        self._check(self.lib.flic_set_tile_config(self._h, int(gas), int(bme)))

    def tile_config(self) -> dict:
        """{"gas": index, "bme": index, "text": description} of the shapes in use."""
        g, b = ctypes.c_int(), ctypes.c_int()
        buf = ctypes.create_string_buffer(512)
        self._check(self.lib.flic_tile_config(self._h, ctypes.byref(g), ctypes.byref(b), buf, len(buf)))
        return {"gas": g.value, "bme": b.value, "text": buf.value.decode()}

    def autotune(self, reps: int = 5, use_cache: bool = True) -> dict:
        """Times every compiled shape of both fluid kernels on the current state and
        keeps the fastest; returns {"cached": bool, "ms_gas": [...], "ms_bme": [...]}
        (the lists are empty when a cached choice was applied)."""
        ng, nb = self.num_tile_configs()
        ms = (ctypes.c_double * (ng + nb))()
        rc = self.lib.flic_autotune(self._h, int(reps), int(bool(use_cache)), ms)
        if rc < 0:
            self._check(rc)
        if rc == 1:
            return {"cached": True, "ms_gas": [], "ms_bme": []}
        return {"cached": False, "ms_gas": list(ms)[:ng], "ms_bme": list(ms)[ng:]}

    def solve_poisson(self, want=True):
        if not want:
            self._check(self.lib.flic_solve_poisson(self._h, None))
            return None
        phi = np.empty((self.n, self.n, self.n))
        self._check(self.lib.flic_solve_poisson(self._h, ctypes.c_void_p(phi.ctypes.data)))
        return phi

    def step_diagnostics(self) -> dict:
        d = Diag()
        self._check(self.lib.flic_step_diagnostics(self._h, ctypes.byref(d)))
        return d.as_dict()

    def diagnostics(self) -> dict:
        d = Diag()
        self._check(self.lib.flic_diagnostics(self._h, ctypes.byref(d)))
        return d.as_dict()

    def sync(self):
        self._check(self.lib.flic_sync(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.flic_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent runs of uneven sizes advanced together (a libflic ensemble)."""

    def __init__(self, sizes, *, box=(-1.0, 1.0), gamma=5.0 / 3.0, G=1.0, courant=0.2, eta=1e-3,
                 precision: str = "mixed", poisson: str = "periodic", boundary: str = "periodic",
                 cooling: float = 0.0, stream: int = 0):
        self.lib = load()
        self.sizes = [int(n) for n in sizes]
        hb = {"periodic": HYDRO_PERIODIC, "outflow": HYDRO_OUTFLOW}[boundary]
        descs = (GridDesc * len(self.sizes))(*[
            GridDesc(n, box[0], box[1], gamma, G, courant, eta, {"fp64": FP64, "mixed": MIXED}[precision],
                     {"periodic": PERIODIC, "isolated": ISOLATED}[poisson], hb, float(cooling))
            for n in self.sizes])
        self._e = ctypes.c_void_p()
        rc = self.lib.flic_ensemble_create(descs, len(self.sizes), ctypes.c_void_p(stream or None),
                                           ctypes.byref(self._e))
        if rc != OK:
            raise FlicError(rc, self.lib.flic_last_error(None).decode())

    def _check(self, rc):
        if rc < 0:
            raise FlicError(rc, self.lib.flic_ensemble_last_error(self._e).decode())
        return rc

    def set_state(self, run: int, state):
        n = self.sizes[run]
        arrs = _field_list(state, n)
        ptrs = []
        for a in arrs:
            p, dev = _ptr_of(a, False)
            if dev:
                raise FlicError(ERR_INVALID_ARG, "ensemble states are host arrays")
            ptrs.append(p)
        self._check(self.lib.flic_ensemble_set_state(self._e, run, (ctypes.c_void_p * NFIELDS)(*ptrs)))

    def get_state(self, run: int, out=None):
        """The run's state as a dict of float64 (n, n, n) numpy arrays, or into
        ``out`` (dict or sequence of 22 host float64 arrays, numpy or torch)."""
        n = self.sizes[run]
        if out is None:
            res = {f: np.empty((n, n, n)) for f in FIELDS}
            arrs = [res[f] for f in FIELDS]
        else:
            res = out
            arrs = _field_list(out, n)
        ptrs = []
        for a in arrs:
            p, dev = _ptr_of(a, False)
            if dev:
                raise FlicError(ERR_INVALID_ARG, "ensemble states are host arrays")
            ptrs.append(p)
        self._check(self.lib.flic_ensemble_get_state(self._e, run, (ctypes.c_void_p * NFIELDS)(*ptrs)))
        return res

    def step(self, nsteps: int = 1, dt: float = 0.0, sync: bool = True):
        self._check(self.lib.flic_ensemble_step(self._e, int(nsteps), dt, int(bool(sync))))

    def diagnostics(self, run: int) -> dict:
        d = Diag()
        self._check(self.lib.flic_ensemble_diagnostics(self._e, run, ctypes.byref(d)))
        return d.as_dict()

    def profile(self, nsteps: int, dt: float = 0.0):
        """Per-stage device milliseconds summed over ``nsteps`` plain-launch steps,
        and the total elapsed milliseconds."""
        ms = (ctypes.c_double * NSTAGES)()
        tot = ctypes.c_double()
        self._check(self.lib.flic_ensemble_profile(self._e, int(nsteps), dt, ms, ctypes.byref(tot)))
        return dict(zip(STAGES, list(ms))), tot.value

    def launches_per_step(self) -> int:
        return self._check(self.lib.flic_ensemble_launches_per_step(self._e))

    def num_tile_configs(self):
        ng, nb = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.flic_ensemble_num_tile_configs(self._e, ctypes.byref(ng), ctypes.byref(nb)))
        return ng.value, nb.value

    def autotune(self, reps: int = 3) -> dict:
        """Times every (compiled shape, z-chunk cap 16/32/64) of both fluid kernels
        over the work list and keeps the fastest of each; returns the mean ms per
        launch as {"ms_gas": [[cap16, cap32, cap64] per shape], "ms_bme": [...]}
        (-1: skipped)."""
        ng, nb = self.num_tile_configs()
        ms = (ctypes.c_double * (3 * (ng + nb)))()
        self._check(self.lib.flic_ensemble_autotune(self._e, int(reps), ms))
        v = list(ms)
        rows = [v[3 * i:3 * i + 3] for i in range(ng + nb)]
        return {"ms_gas": rows[:ng], "ms_bme": rows[ng:]}

    def set_tile_config(self, gas: int = -1, bme: int = -1, tz_gas: int = -1, tz_bme: int = -1):
        self._check(self.lib.flic_ensemble_set_tile_config(self._e, int(gas), int(bme), int(tz_gas), int(tz_bme)))

    def tile_config(self) -> dict:
        g, b, tg, tb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        buf = ctypes.create_string_buffer(512)
        self._check(self.lib.flic_ensemble_tile_config(self._e, ctypes.byref(g), ctypes.byref(b), ctypes.byref(tg),
                                                       ctypes.byref(tb), buf, len(buf)))
        return {"gas": g.value, "bme": b.value, "tz_gas": tg.value, "tz_bme": tb.value, "text": buf.value.decode()}


    def close(self):
        if getattr(self, "_e", None) and self._e.value:
            self.lib.flic_ensemble_destroy(self._e)
            self._e = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
