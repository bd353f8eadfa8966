"""The C-ABI library builds, loads and exports every entry point of
include/eulbfs.h; on a machine without a GPU it refuses to run instead of
falling back to the CPU."""
import ctypes as ct
import os
import re

import pytest

from paper_2507_03366_gb300 import build as B
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="eulbfs.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eulbfs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return eulbfs.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared entry points
    assert sorted(n for n, _, _ in eulbfs.SIGNATURES) == names


def test_every_header_in_include_is_exported(lib):
    """Every header under include/ declares entry points of libeulbfs.so."""
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert "eulbfs_peaks.h" in headers
    for h in headers:
        for n in _declared(h):
            assert hasattr(lib, n), (h, n)
    assert sorted(n for n, _, _ in eulbfs.PEAK_SIGNATURES) == _declared("eulbfs_peaks.h")


def test_version_and_sizes(lib):
    assert b"sm_103a" in lib.eulbfs_version()
    # 3 state buffers x 7 FP32 planes + 2 FP32 planes per cell, plus a descriptor
    n = 128 * 64
    assert lib.eulbfs_domain_bytes(128, 64, eulbfs.FP32C) >= n * (3 * 7 * 4 + 2 * 4)
    assert lib.eulbfs_domain_bytes(128, 64, eulbfs.FP64) >= n * (3 * 5 * 8 + 2 * 8)
    assert lib.eulbfs_domain_bytes(0, 64, eulbfs.FP64) == 0


def test_no_cpu_fallback_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(eulbfs.EulbfsError) as e:
        eulbfs.Solver([wl.conductive(32, 2)], precision=eulbfs.FP64)
    assert e.value.code in (eulbfs.ECUDA,)


def test_invalid_arguments_rejected_before_device_work(lib):
    h = ct.c_void_p()
    # negative domain count, and a non-empty batch without a domain list
    assert lib.eulbfs_batch_create(-1, None, eulbfs.FP32C, None, ct.byref(h)) == eulbfs.EINVAL
    assert lib.eulbfs_batch_create(2, None, eulbfs.FP32C, None, ct.byref(h)) == eulbfs.EINVAL
    # tau_g <= 0.5 is invalid (Sec. 2.3.2: M_c = (tau_g - 0.5) Q_g dt_s)
    case = wl.conductive(32, 2)
    case.props.tau_g = 0.5
    keep = []
    d = eulbfs.domain_struct(case, keep)
    assert lib.eulbfs_batch_create(1, ct.byref(d), eulbfs.FP32C, None, ct.byref(h)) == eulbfs.EINVAL
    assert b"tau_g" in lib.eulbfs_last_error()
    # periodic on one side only
    case = wl.conductive(32, 2)
    case.bc.yhi = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)
    d = eulbfs.domain_struct(case, keep)
    assert lib.eulbfs_batch_create(1, ct.byref(d), eulbfs.FP64, None, ct.byref(h)) == eulbfs.EINVAL
    # an axisymmetric domain needs its axis (xlo) adiabatic, symmetric and no-flux
    case = wl.conductive(32, 2)
    case.axisymmetric = 1
    d = eulbfs.domain_struct(case, keep)
    assert lib.eulbfs_batch_create(1, ct.byref(d), eulbfs.FP64, None, ct.byref(h)) == eulbfs.EINVAL
    assert b"axis" in lib.eulbfs_last_error()
    # a domain of more than 2^31 cells is refused before any array is read
    big = eulbfs.Domain(eulbfs.Grid(65536, 32769), d.props, d.bc, d.num, eulbfs.Init())
    assert lib.eulbfs_batch_create(1, ct.byref(big), eulbfs.FP32C, None, ct.byref(h)) == eulbfs.EINVAL
    assert b"too large" in lib.eulbfs_last_error()
    # streaming steps lie in (0, 0.5]
    case = wl.droplet(32)
    case.dt_f = 0.6
    d = eulbfs.domain_struct(case, keep)
    assert lib.eulbfs_batch_create(1, ct.byref(d), eulbfs.FP64, None, ct.byref(h)) == eulbfs.EINVAL
    assert b"streaming" in lib.eulbfs_last_error()
    # a hysteresis window needs theta_rec <= theta_adv
    case = wl.droplet(32)
    case.bc.ylo = wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING_HYST, Tw=-0.5, theta_deg=90.0,
                          theta_adv_deg=60.0, theta_rec_deg=100.0)
    d = eulbfs.domain_struct(case, keep)
    assert lib.eulbfs_batch_create(1, ct.byref(d), eulbfs.FP64, None, ct.byref(h)) == eulbfs.EINVAL
    assert lib.eulbfs_step(None, 1) == eulbfs.EINVAL


def test_streaming_steps_marshalled():
    """A case's single streaming step stands for each distribution's step it
    leaves unset (the oracle's convention); explicit steps win."""
    case = wl.droplet(32)
    case.dt_stream = 0.4
    case.dt_f = 0.3
    d = eulbfs.domain_struct(case, [])
    assert (d.num.dt_stream_h, d.num.dt_stream_f, d.num.dt_stream_g) == (0.4, 0.3, 0.4)
    d = eulbfs.domain_struct(wl.droplet(32), [])
    assert (d.num.dt_stream_h, d.num.dt_stream_f, d.num.dt_stream_g) == (0.5, 0.5, 0.5)
