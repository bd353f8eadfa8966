"""Thin ctypes binding of libeulbfs (include/eulbfs.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  If the library has not been built, or there is no CUDA device, the
calls fail loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

from .build import LIB as LIB_PATH

FP64, FP32C = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EBUSY = range(7)
_STATUS = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ENONFINITE: "ENONFINITE",
           ETIMEOUT: "ETIMEOUT", EBUSY: "EBUSY"}


class EulbfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int)]


class Phase(ct.Structure):
    _fields_ = [("rho", ct.c_double), ("mu", ct.c_double), ("lam", ct.c_double), ("cp", ct.c_double)]


class Props(ct.Structure):
    _fields_ = [("s", Phase), ("l", Phase), ("g", Phase), ("L", ct.c_double), ("Ts", ct.c_double),
                ("Tl", ct.c_double), ("sigma", ct.c_double), ("xi", ct.c_double), ("Mc", ct.c_double),
                ("tau_g", ct.c_double), ("gx", ct.c_double), ("gy", ct.c_double),
                ("zero_solid_velocity", ct.c_int), ("literal_eq7", ct.c_int)]


class Side(ct.Structure):
    _fields_ = [("thermal", ct.c_int), ("flow", ct.c_int), ("phase", ct.c_int), ("Tw", ct.c_double),
                ("theta_deg", ct.c_double), ("theta_adv_deg", ct.c_double), ("theta_rec_deg", ct.c_double)]


class BC(ct.Structure):
    _fields_ = [("xlo", Side), ("xhi", Side), ("ylo", Side), ("yhi", Side)]


class Numerics(ct.Structure):
    _fields_ = [("dt", ct.c_double), ("axisymmetric", ct.c_int), ("dt_stream_h", ct.c_double),
                ("dt_stream_f", ct.c_double), ("dt_stream_g", ct.c_double)]


_DP = ct.POINTER(ct.c_double)


class Init(ct.Structure):
    _fields_ = [("T", _DP), ("Fl", _DP), ("C", _DP), ("u", _DP), ("v", _DP), ("p", _DP)]


class Domain(ct.Structure):
    _fields_ = [("grid", Grid), ("props", Props), ("bc", BC), ("num", Numerics), ("init", Init)]


class FieldsOut(ct.Structure):
    _fields_ = [("H", _DP), ("T", _DP), ("Fl", _DP), ("C", _DP), ("p", _DP), ("u", _DP), ("v", _DP)]


class Diag(ct.Structure):
    _fields_ = [("step", ct.c_longlong), ("t", ct.c_double), ("mass", ct.c_double),
                ("enthalpy", ct.c_double), ("phase_vol", ct.c_double), ("solid_vol", ct.c_double),
                ("front_pos", ct.c_double), ("interface_pos", ct.c_double),
                ("max_speed", ct.c_double), ("nonfinite", ct.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every entry point the header declares
SIGNATURES = [
    ("eulbfs_create", ct.c_int, [ct.POINTER(Grid), ct.POINTER(Props), ct.POINTER(BC), ct.POINTER(Numerics),
                                 ct.POINTER(Init), ct.c_int, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    ("eulbfs_batch_create", ct.c_int, [ct.c_int, ct.POINTER(Domain), ct.c_int, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    ("eulbfs_set_memory_budget", ct.c_int, [ct.c_void_p, ct.c_ulonglong]),
    ("eulbfs_domain_bytes", ct.c_ulonglong, [ct.c_int, ct.c_int, ct.c_int]),
    ("eulbfs_add_domain", ct.c_int, [ct.c_void_p, ct.POINTER(Domain), ct.c_longlong, ct.POINTER(ct.c_int)]),
    ("eulbfs_add_split_domain", ct.c_int, [ct.c_void_p, ct.POINTER(Domain), ct.c_int, ct.c_longlong,
                                           ct.POINTER(ct.c_int)]),
    ("eulbfs_remove_domain", ct.c_int, [ct.c_void_p, ct.c_int]),
    ("eulbfs_num_slots", ct.c_int, [ct.c_void_p]),
    ("eulbfs_domain_progress", ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]),
    ("eulbfs_step", ct.c_int, [ct.c_void_p, ct.c_longlong]),
    ("eulbfs_sync", ct.c_int, [ct.c_void_p]),
    ("eulbfs_nonfinite_domains", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int), ct.c_int, ct.POINTER(ct.c_int)]),
    ("eulbfs_fields", ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(FieldsOut)]),
    ("eulbfs_get_state", ct.c_int, [ct.c_void_p, ct.c_int] + [_DP] * 7 + [ct.POINTER(ct.c_longlong)]),
    ("eulbfs_set_state", ct.c_int, [ct.c_void_p, ct.c_int] + [_DP] * 6 + [ct.c_double, ct.c_longlong]),
    ("eulbfs_checkpoint_bytes", ct.c_ulonglong, [ct.c_void_p, ct.c_int]),
    ("eulbfs_save", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_ulonglong, ct.POINTER(ct.c_longlong)]),
    ("eulbfs_load", ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_ulonglong, ct.c_longlong]),
    ("eulbfs_diagnostics", ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(Diag)]),
    ("eulbfs_launches_per_step", ct.c_int, [ct.c_void_p]),
    ("eulbfs_set_whole_step", ct.c_int, [ct.c_void_p, ct.c_int]),
    ("eulbfs_launch_count", ct.c_ulonglong, [ct.c_void_p]),
    ("eulbfs_use_graphs", ct.c_int, [ct.c_void_p, ct.c_int]),
    ("eulbfs_autotune", ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_float)]),
    ("eulbfs_set_tile", ct.c_int, [ct.c_void_p, ct.c_int]),
    ("eulbfs_set_tile_wait_probe", ct.c_int, [ct.c_void_p, ct.c_int]),
    ("eulbfs_autotune_report", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int), ct.POINTER(ct.c_float), ct.c_int,
                                          ct.POINTER(ct.c_int)]),
    ("eulbfs_diagnostics_noalloc", ct.c_int, [ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.POINTER(Props),
                                              ct.c_void_p, ct.c_void_p]),
    ("eulbfs_destroy", None, [ct.c_void_p]),
    ("eulbfs_last_error", ct.c_char_p, []),
    ("eulbfs_version", ct.c_char_p, []),
]


# entry points of include/eulbfs_peaks.h (measured FMA throughput)
PEAK_SIGNATURES = [
    ("eulbfs_peak_fma", ct.c_int, [ct.c_int, ct.c_longlong, ct.c_void_p, ct.POINTER(ct.c_double),
                                   ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
]
PEAK_FP32, PEAK_FP32X2, PEAK_FP64 = range(3)


def lib():
    """Load libeulbfs.so; raises if it has not been built.  EULBFS_LIB names
    another build of the same library (e.g. one compiled with other flags)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("EULBFS_LIB") or LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with `python -c \"import __graft_entry__ as g; "
                                   f"g.build()\"` (there is no CPU fallback)")
            L = ct.CDLL(path)
            for name, res, args in SIGNATURES + PEAK_SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def peak_fma(kind: int, iters: int, stream: Optional[int] = None) -> dict:
    """One timed launch of the FMA-chain kernel of `kind` (PEAK_*)."""
    fl, ms, wi = ct.c_double(), ct.c_double(), ct.c_double()
    _check(lib().eulbfs_peak_fma(kind, iters, ct.c_void_p(stream) if stream else None, ct.byref(fl), ct.byref(ms),
                                 ct.byref(wi)))
    return {"flops_per_s": fl.value, "ms": ms.value, "fma_warp_inst_per_s": wi.value}


def _check(rc: int):
    if rc != OK:
        raise EulbfsError(rc, lib().eulbfs_last_error().decode())


def _ptr(a: Optional[np.ndarray]):
    return a.ctypes.data_as(_DP) if a is not None else None


def _props(p) -> Props:
    ph = lambda q: Phase(q.rho, q.mu, q.lam, q.cp)  # noqa: E731
    return Props(ph(p.s), ph(p.l), ph(p.g), p.L, p.Ts, p.Tl, p.sigma, p.xi, p.Mc, p.tau_g, p.gx, p.gy,
                 int(p.zero_solid_velocity), int(getattr(p, "literal_eq7", 0)))


def _bc(b) -> BC:
    sd = lambda q: Side(q.thermal, q.flow, q.phase, q.Tw, q.theta_deg,  # noqa: E731
                        getattr(q, "theta_adv_deg", q.theta_deg), getattr(q, "theta_rec_deg", q.theta_deg))
    return BC(sd(b.xlo), sd(b.xhi), sd(b.ylo), sd(b.yhi))


def _numerics(case) -> Numerics:
    """Time step, geometry and the three streaming steps (a case's
    dt_stream stands for any step it leaves at 0)."""
    base = float(getattr(case, "dt_stream", 0.5))
    steps = [float(getattr(case, k, 0.0) or 0.0) or base for k in ("dt_h", "dt_f", "dt_g")]
    return Numerics(case.dt, int(getattr(case, "axisymmetric", 0)), *steps)


def domain_struct(case, keep: list) -> Domain:
    """Marshal a workloads.Case into an eulbfs_domain (arrays kept alive in `keep`)."""
    arrs = {k: np.ascontiguousarray(case.init[k], dtype=np.float64).ravel() for k in ("T", "Fl", "C", "u", "v", "p")}
    keep.append(arrs)
    init = Init(*[_ptr(arrs[k]) for k in ("T", "Fl", "C", "u", "v", "p")])
    return Domain(Grid(case.nx, case.ny), _props(case.props), _bc(case.bc), _numerics(case), init)


class Solver:
    """A set of domains advanced together on the GPU (eulbfs_solver)."""

    def __init__(self, cases: Sequence, precision: int = FP32C, stream: Optional[int] = None):
        cases = list(cases)
        keep: list = []
        arr = (Domain * len(cases))(*[domain_struct(c, keep) for c in cases])
        h = ct.c_void_p()
        _check(lib().eulbfs_batch_create(len(cases), arr, precision, ct.c_void_p(stream) if stream else None,
                                         ct.byref(h)))
        self._h = h
        self.precision = precision
        self.shapes: List = [(c.ny, c.nx) for c in cases]
        self.cases = cases

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.eulbfs_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # -- continuous batching
    def add(self, case, max_steps: int = 0) -> int:
        keep: list = []
        d = domain_struct(case, keep)
        slot = ct.c_int()
        _check(lib().eulbfs_add_domain(self._h, ct.byref(d), max_steps, ct.byref(slot)))
        while len(self.shapes) <= slot.value:
            self.shapes.append(None)
            self.cases.append(None)
        self.shapes[slot.value] = (case.ny, case.nx)
        self.cases[slot.value] = case
        return slot.value

    def add_split(self, case, k: int, max_steps: int = 0) -> List[int]:
        """Add `case` split along y into k slabs; returns their slots (bottom first)."""
        keep: list = []
        d = domain_struct(case, keep)
        slots = (ct.c_int * k)()
        _check(lib().eulbfs_add_split_domain(self._h, ct.byref(d), k, max_steps, slots))
        out = [slots[i] for i in range(k)]
        for i, sl in enumerate(out):
            y0, y1 = i * case.ny // k, (i + 1) * case.ny // k
            while len(self.shapes) <= sl:
                self.shapes.append(None)
                self.cases.append(None)
            self.shapes[sl] = (y1 - y0, case.nx)
            self.cases[sl] = case
        return out

    def split_fields(self, slots: Sequence[int]) -> dict:
        """Fields of a split domain, its slabs stacked back along y."""
        parts = [self.fields(sl) for sl in slots]
        return {k: np.concatenate([p[k] for p in parts], axis=0) for k in parts[0]}

    def remove(self, slot: int):
        _check(lib().eulbfs_remove_domain(self._h, slot))

    def progress(self, slot: int):
        done, left = ct.c_longlong(), ct.c_longlong()
        _check(lib().eulbfs_domain_progress(self._h, slot, ct.byref(done), ct.byref(left)))
        return done.value, left.value

    def set_memory_budget(self, nbytes: int):
        _check(lib().eulbfs_set_memory_budget(self._h, nbytes))

    # -- stepping
    def step(self, n: int = 1):
        _check(lib().eulbfs_step(self._h, n))

    def sync(self):
        _check(lib().eulbfs_sync(self._h))

    def nonfinite_slots(self) -> List[int]:
        """Slots whose own state became NaN or Inf (synchronises the stream)."""
        cap = max(1, len(self.shapes))
        buf = (ct.c_int * cap)()
        n = ct.c_int()
        _check(lib().eulbfs_nonfinite_domains(self._h, buf, cap, ct.byref(n)))
        return [buf[k] for k in range(min(n.value, cap))]

    def use_graphs(self, steps: int):
        _check(lib().eulbfs_use_graphs(self._h, steps))

    def set_tile(self, tile_y: int):
        _check(lib().eulbfs_set_tile(self._h, tile_y))

    def autotune(self, steps_per_candidate: int = 10):
        """Time the work-item heights on the live batch; returns (rows, ms per step)."""
        rows, ms = ct.c_int(), ct.c_float()
        _check(lib().eulbfs_autotune(self._h, steps_per_candidate, ct.byref(rows), ct.byref(ms)))
        return rows.value, ms.value

    def autotune_report(self) -> dict:
        """{rows: best ms per step} of the candidates the last autotune timed."""
        rows, ms, n = (ct.c_int * 8)(), (ct.c_float * 8)(), ct.c_int()
        _check(lib().eulbfs_autotune_report(self._h, rows, ms, 8, ct.byref(n)))
        return {rows[k]: ms[k] for k in range(min(n.value, 8))}

    def launches_per_step(self) -> int:
        return lib().eulbfs_launches_per_step(self._h)

    def launch_count(self) -> int:
        """Kernel launches of the time-stepping path since creation."""
        return int(lib().eulbfs_launch_count(self._h))

    def set_whole_step(self, on: bool = True):
        """One kernel launch per time step (default) or one per Runge-Kutta stage."""
        _check(lib().eulbfs_set_whole_step(self._h, 1 if on else 0))

    # -- outputs
    def fields(self, slot: int = 0, which=("H", "T", "Fl", "C", "p", "u", "v")) -> dict:
        ny, nx = self.shapes[slot]
        out = {k: np.empty(nx * ny) for k in which}
        fo = FieldsOut(*[_ptr(out.get(k)) for k in ("H", "T", "Fl", "C", "p", "u", "v")])
        _check(lib().eulbfs_fields(self._h, slot, ct.byref(fo)))
        return {k: v.reshape(ny, nx) for k, v in out.items()}

    def state(self, slot: int = 0) -> dict:
        ny, nx = self.shapes[slot]
        out = {k: np.empty(nx * ny) for k in ("H", "p", "mx", "my", "C", "Fsp")}
        t, step = ct.c_double(), ct.c_longlong()
        _check(lib().eulbfs_get_state(self._h, slot, *[_ptr(out[k]) for k in ("H", "p", "mx", "my", "C", "Fsp")],
                                      ct.byref(t), ct.byref(step)))
        res = {k: v.reshape(ny, nx) for k, v in out.items()}
        res["t"], res["step"] = t.value, step.value
        return res

    def set_state(self, st: dict, slot: int = 0):
        arrs = [np.ascontiguousarray(st[k], dtype=np.float64).ravel() for k in ("H", "p", "mx", "my", "C", "Fsp")]
        _check(lib().eulbfs_set_state(self._h, slot, *[_ptr(a) for a in arrs], float(st.get("t", 0.0)),
                                      int(st.get("step", 0))))

    def save(self, slot: int = 0):
        """Bitwise-exact checkpoint: (bytes, step)."""
        n = lib().eulbfs_checkpoint_bytes(self._h, slot)
        buf = ct.create_string_buffer(n)
        step = ct.c_longlong()
        _check(lib().eulbfs_save(self._h, slot, buf, n, ct.byref(step)))
        return buf.raw, step.value

    def load(self, blob: bytes, step: int, slot: int = 0):
        _check(lib().eulbfs_load(self._h, slot, blob, len(blob), step))

    def diag(self, slot: int = 0) -> dict:
        d = Diag()
        _check(lib().eulbfs_diagnostics(self._h, slot, ct.byref(d)))
        return d.as_dict()
