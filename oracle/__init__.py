"""Python binding of the FP64 CPU oracle (oracle.h / eulbfs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke entry point
and the CPU-baseline leg of the benchmark.  The product path never imports it.
It shares no code with the CUDA library; its inputs come from the seeded
problem descriptions in ``paper_2507_03366_gb300.workloads``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eulbfs_oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, reading R23).

    EULBFS_ORACLE_LIB names a prebuilt library instead (used by the mutation
    test, which plants mistakes in a copy of the oracle source)."""
    override = os.environ.get("EULBFS_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared", "-D_DEFAULT_SOURCE"]
        # OpenMP over independent loops where the compiler has it (same
        # results for any thread count); a plain build otherwise
        r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


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
    _fields_ = [("dt", ct.c_double), ("dt_stream", ct.c_double), ("axisymmetric", ct.c_int),
                ("dt_h", ct.c_double), ("dt_f", ct.c_double), ("dt_g", ct.c_double)]


_DP = ct.POINTER(ct.c_double)


class Init(ct.Structure):
    _fields_ = [("T", _DP), ("Fl", _DP), ("C", _DP), ("u", _DP), ("v", _DP), ("p", _DP)]


class Diag(ct.Structure):
    _fields_ = [("step", ct.c_longlong), ("t", ct.c_double), ("mass", ct.c_double),
                ("enthalpy", ct.c_double), ("phase_vol", ct.c_double), ("solid_vol", ct.c_double),
                ("front_pos", ct.c_double), ("interface_pos", ct.c_double),
                ("max_speed", ct.c_double), ("nonfinite", ct.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            L.or_create.restype = ct.c_void_p
            L.or_create.argtypes = [ct.c_int, ct.c_int, ct.POINTER(Props), ct.POINTER(BC),
                                    ct.POINTER(Numerics), ct.POINTER(Init), ct.c_char_p]
            L.or_destroy.argtypes = [ct.c_void_p]
            L.or_step.argtypes = [ct.c_void_p, ct.c_longlong]
            L.or_step.restype = ct.c_int
            L.or_diagnostics.argtypes = [ct.c_void_p, ct.POINTER(Diag)]
            L.or_get_state.argtypes = [ct.c_void_p] + [_DP] * 6
            L.or_set_state.argtypes = [ct.c_void_p] + [_DP] * 6 + [ct.c_double, ct.c_longlong]
            L.or_get_primitives.argtypes = [ct.c_void_p] + [_DP] * 4
            for name in ("or_heq",):
                getattr(L, name).argtypes = [ct.c_int] + [ct.c_double] * 6
            L.or_feq.argtypes = [ct.c_int] + [ct.c_double] * 4
            L.or_feqm.argtypes = [ct.c_int] + [ct.c_double] * 4
            L.or_geq.argtypes = [ct.c_int] + [ct.c_double] * 5
            for name in ("or_heq", "or_feq", "or_feqm", "or_geq", "or_enthalpy_of", "or_mix"):
                getattr(L, name).restype = ct.c_double
            L.or_invert_enthalpy.argtypes = [ct.POINTER(Props), ct.c_double, ct.c_double, _DP, _DP]
            L.or_enthalpy_of.argtypes = [ct.POINTER(Props), ct.c_double, ct.c_double, ct.c_double]
            L.or_mix.argtypes = [ct.POINTER(Props), ct.c_double, ct.c_double, ct.c_int]
            L.or_face_flux.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, _DP]
            L.or_residual.argtypes = [ct.c_void_p, _DP]
            L.or_get_muc.argtypes = [ct.c_void_p, _DP]
            L.or_set_threads.argtypes = [ct.c_int]
            L.or_set_threads.restype = ct.c_int
            L.or_set_threads(1)     # single-threaded unless a caller asks for more
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def props_struct(p) -> Props:
    ph = lambda q: Phase(q.rho, q.mu, q.lam, q.cp)  # noqa: E731
    return Props(ph(p.s), ph(p.l), ph(p.g), p.L, p.Ts, p.Tl, p.sigma, p.xi, p.Mc, p.tau_g, p.gx, p.gy,
                 int(p.zero_solid_velocity), int(getattr(p, "literal_eq7", 0)))


def bc_struct(b) -> BC:
    sd = lambda q: Side(q.thermal, q.flow, q.phase, q.Tw, q.theta_deg,  # noqa: E731
                        getattr(q, "theta_adv_deg", q.theta_deg), getattr(q, "theta_rec_deg", q.theta_deg))
    return BC(sd(b.xlo), sd(b.xhi), sd(b.ylo), sd(b.yhi))


def set_threads(n: int) -> int:
    """Host threads the oracle's independent loops use (OpenMP builds);
    returns the count in use.  Results are bitwise the same for any count."""
    return lib().or_set_threads(int(n))


# ---- equilibria and closure, exposed for the pin tests ----
def heq(a, H, T, Cp, Cref, u, v):
    return lib().or_heq(a, H, T, Cp, Cref, u, v)


def feq(a, p, rho, u, v):
    return lib().or_feq(a, p, rho, u, v)


def feqm(a, p, rho_face, u, v):
    return lib().or_feqm(a, p, rho_face, u, v)


def geq(a, C, muc, Qg, u, v):
    return lib().or_geq(a, C, muc, Qg, u, v)


def invert_enthalpy(props, H, C):
    T, Fl = ct.c_double(), ct.c_double()
    P = props_struct(props)
    lib().or_invert_enthalpy(ct.byref(P), H, C, ct.byref(T), ct.byref(Fl))
    return T.value, Fl.value


def enthalpy_of(props, T, Fl, C):
    P = props_struct(props)
    return lib().or_enthalpy_of(ct.byref(P), T, Fl, C)


def mix(props, C, Fl, which):
    P = props_struct(props)
    return lib().or_mix(ct.byref(P), C, Fl, which)


class OracleSolver:
    """One domain advanced by the oracle.  ``case`` is a workloads.Case."""

    def __init__(self, case):
        self.case = case
        self.nx, self.ny = case.nx, case.ny
        self._keep = {k: np.ascontiguousarray(case.init[k], dtype=np.float64).ravel()
                      for k in ("T", "Fl", "C", "u", "v", "p")}
        init = Init(*[_ptr(self._keep[k]) for k in ("T", "Fl", "C", "u", "v", "p")])
        P, B = props_struct(case.props), bc_struct(case.bc)
        N = Numerics(case.dt, case.dt_stream, int(getattr(case, "axisymmetric", 0)),
                     *[float(getattr(case, k, 0.0) or 0.0) for k in ("dt_h", "dt_f", "dt_g")])
        err = ct.create_string_buffer(256)
        h = lib().or_create(case.nx, case.ny, ct.byref(P), ct.byref(B), ct.byref(N), ct.byref(init), err)
        if not h:
            raise ValueError(err.value.decode())
        self._h = ct.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    def step(self, n: int = 1) -> int:
        rc = lib().or_step(self._h, n)
        if rc != 0:
            raise FloatingPointError(f"oracle state became non-finite (status {rc})")
        return rc

    def diag(self) -> dict:
        d = Diag()
        lib().or_diagnostics(self._h, ct.byref(d))
        return d.as_dict()

    def state(self) -> dict:
        n = self.nx * self.ny
        out = {k: np.empty(n) for k in ("H", "p", "mx", "my", "C", "Fsp")}
        lib().or_get_state(self._h, *[_ptr(out[k]) for k in ("H", "p", "mx", "my", "C", "Fsp")])
        return {k: v.reshape(self.ny, self.nx) for k, v in out.items()}

    def set_state(self, st: dict, t: float, step: int):
        arrs = [np.ascontiguousarray(st[k], dtype=np.float64).ravel() for k in ("H", "p", "mx", "my", "C", "Fsp")]
        lib().or_set_state(self._h, *[_ptr(a) for a in arrs], t, step)

    def fields(self) -> dict:
        """H, T, Fl, C, p, u, v as (ny, nx) arrays."""
        n = self.nx * self.ny
        st = self.state()
        T, Fl, u, v = (np.empty(n) for _ in range(4))
        lib().or_get_primitives(self._h, _ptr(T), _ptr(Fl), _ptr(u), _ptr(v))
        shp = (self.ny, self.nx)
        return {"H": st["H"], "T": T.reshape(shp), "Fl": Fl.reshape(shp), "C": st["C"],
                "p": st["p"], "u": u.reshape(shp), "v": v.reshape(shp)}

    def face_flux(self, direction: int, i: int, j: int) -> np.ndarray:
        out = np.empty(6)
        lib().or_face_flux(self._h, direction, i, j, _ptr(out))
        return out

    def residual(self) -> np.ndarray:
        out = np.empty(5 * self.nx * self.ny)
        lib().or_residual(self._h, _ptr(out))
        return out.reshape(5, self.ny, self.nx)

    def muc(self) -> np.ndarray:
        out = np.empty(self.nx * self.ny)
        lib().or_get_muc(self._h, _ptr(out))
        return out.reshape(self.ny, self.nx)
