"""A domain at the largest size that is practical to test, through the C ABI.

The library accepts up to 2^31 cells per domain, and all its cell indices
and plane offsets are 64-bit.  This test drives a domain whose FP32C state
planes reach past 2^31 elements: 20480 x 16384 = 335.5 M cells, with the
seven planes of a state buffer spanning 2.35 G elements (31 GB of device
memory in all).  No oracle can step such a domain, so the check is a property
that holds at any size.  The domain is periodic in both directions and
starts as a tiling of one 32 x 32 periodic tile, so every tile stays a copy
of that tile run alone: the per-cell arithmetic does not depend on where the
cell sits.  The FP64 integrals of the big domain must therefore be the
number of tiles times those of the single tile, and its largest speed the
same, to the rounding of the sums.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TILE = 32
TX, TY = 640, 512          # tiles along x and y: 20480 x 16384 cells


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()


def _tile():
    """A freezing drop in a doubly periodic 32 x 32 tile."""
    x = np.arange(TILE) + 0.5
    X, Y = np.meshgrid(x, x)
    d = np.sqrt((X - 16.0) ** 2 + (Y - 16.0) ** 2)
    C = 0.5 * (1 + np.tanh(2 * (8.0 - d) / 4.0))
    T = 0.3 - 0.7 * np.exp(-((X - 12.0) ** 2 + (Y - 12.0) ** 2) / 20.0)
    return T, C


def _run(T, C, steps):
    """Create one FP32C domain from T and C (the other fields default), step
    it and return its diagnostics."""
    ny, nx = T.shape
    case = wl.droplet(32, theta_deg=90.0, St=0.3)
    case.bc = wl.BC(wl.PER, wl.PER, wl.PER, wl.PER)
    T = np.ascontiguousarray(T, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    init = eulbfs.Init(eulbfs._ptr(T), None, eulbfs._ptr(C), None, None, None)
    dom = eulbfs.Domain(eulbfs.Grid(nx, ny), eulbfs._props(case.props), eulbfs._bc(case.bc),
                        eulbfs.Numerics(case.dt, 0, 0.5, 0.5, 0.5), init)
    lib = eulbfs.lib()
    h = ct.c_void_p()
    rc = lib.eulbfs_batch_create(1, ct.byref(dom), eulbfs.FP32C, None, ct.byref(h))
    assert rc == eulbfs.OK, lib.eulbfs_last_error()
    try:
        assert lib.eulbfs_step(h, steps) == eulbfs.OK, lib.eulbfs_last_error()
        d = eulbfs.Diag()
        assert lib.eulbfs_diagnostics(h, 0, ct.byref(d)) == eulbfs.OK, lib.eulbfs_last_error()
        return d.as_dict()
    finally:
        lib.eulbfs_destroy(h)


def test_tiled_domain_past_2_31_plane_elements():
    Tt, Ct = _tile()
    small = _run(Tt, Ct, 2)
    assert small["solid_vol"] > 0 and small["max_speed"] > 0    # freezing and flow are under way
    big = _run(np.tile(Tt, (TY, TX)), np.tile(Ct, (TY, TX)), 2)
    assert TILE * TILE * TX * TY * 7 > 2 ** 31                    # FP32C plane offsets pass 2^31
    n = TX * TY
    for k in ("mass", "enthalpy", "phase_vol", "solid_vol"):
        assert abs(big[k] - n * small[k]) <= 1e-9 * abs(n * small[k]), (k, big[k], n * small[k])
    assert big["max_speed"] == small["max_speed"]
    assert big["step"] == 2 and not big["nonfinite"]
