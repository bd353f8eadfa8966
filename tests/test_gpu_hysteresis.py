"""Contact-angle hysteresis walls (reading R25): CUDA path vs the FP64 oracle.

FP64 every field element within 1e-10 of the field's magnitude; FP32C within
the stated FP32 tolerances.  Cases: the oracle pins' tilted contact line
(pinned inside the window) and both limits, the impact problem's angles of
Sec. 3.5 case (a) (theta_adv 100, theta_r 39, theta_eq 82) on planar and
axisymmetric droplets, a wetting wall along a periodic axis, ragged tiles,
and hysteresis and static walls in one batch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

from test_gpu_parity import FIELDS, assert_fields_close, check_fp32c, run_pair
from test_oracle_hysteresis import NX, NY, _interface, _props_wet
from test_oracle_pins import _case, _walls

pytestmark = pytest.mark.gpu

CASE_A = dict(theta_deg=82.0, hysteresis=(100.0, 39.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()
    oracle.build()


def tilted(theta0, theta, adv, rec, name):
    side = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.WETTING_HYST, theta_deg=theta, theta_adv_deg=adv, theta_rec_deg=rec)
    c = _case(NX, NY, _props_wet(), _walls(ylo=side), T=0.0, C=_interface(theta0), dt=1.0)
    c.name = name
    return c


def periodic_film():
    """A wavy liquid film on a hysteresis wall, periodic along the wall."""
    nx, ny = 48, 24
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    h = 8.0 + 3.0 * np.sin(2 * math.pi * x / nx)
    C = 0.5 * (1 + np.tanh(2 * (h[None, :] - y[:, None]) / 4.0))
    side = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.WETTING_HYST, theta_deg=70.0, theta_adv_deg=110.0, theta_rec_deg=50.0)
    bc = wl.BC(wl.PER, wl.PER, side, wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX))
    c = _case(nx, ny, _props_wet(), bc, T=0.0, C=C, dt=1.0)
    c.name = "periodic_film_48x24"
    return c


FP64_CASES = [
    ("tilted_pinned", lambda: tilted(75.0, 90.0, 120.0, 60.0, "tilted_pinned"), 300),
    ("advancing_limit", lambda: tilted(90.0, 45.0, 60.0, 30.0, "advancing_limit"), 300),
    ("receding_limit", lambda: tilted(90.0, 130.0, 150.0, 110.0, "receding_limit"), 300),
    ("periodic_film_48x24", periodic_film, 300),
    ("droplet_case_a_64", lambda: wl.droplet(64, St=0.2, Tw=-0.8, **CASE_A), 300),
    ("droplet_rz_case_a_64", lambda: wl.droplet(64, St=0.2, Tw=-0.8, axisymmetric=True, **CASE_A), 300),
    ("impact_rz_case_a_64", lambda: wl.droplet(64, St=0.3, Tw=-1.0, impact_speed=0.05, We=50.0, Re=500.0,
                                               axisymmetric=True, **CASE_A), 120),
]


@pytest.mark.parametrize("name,make,steps", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_hysteresis_matches_oracle(name, make, steps):
    case = make()
    gpu, ref = run_pair(case, steps)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=name, floor=1e-8)
    dg, dr = gpu.diag(), ref.diag()
    for k in ("mass", "enthalpy", "phase_vol", "solid_vol"):
        assert abs(dg[k] - dr[k]) <= 1e-10 * max(abs(dr[k]), 1.0), k


@pytest.mark.parametrize("nx,ny", [(33, 5), (37, 18)])
def test_fp64_hysteresis_ragged_tiles(nx, ny):
    rng = np.random.default_rng(nx * 7 + ny)
    case = wl.droplet(max(nx, ny), St=0.25, Tw=-0.6, **CASE_A).crop(nx, ny)
    case.init["T"] = case.init["T"] + 0.05 * rng.standard_normal((ny, nx))
    gpu, ref = run_pair(case, 40)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=f"hyst {nx}x{ny}", floor=1e-8)


def test_fp32c_hysteresis_droplet_within_tolerances():
    case = wl.droplet(64, St=0.2, Tw=-0.8, axisymmetric=True, **CASE_A)
    gpu = eulbfs.Solver([case], precision=eulbfs.FP32C)
    d0g = gpu.diag()
    gpu.step(1000)
    ref = oracle.OracleSolver(case)
    d0r = ref.diag()
    ref.step(1000)
    check_fp32c(gpu.fields(), ref.fields(), gpu.diag(), ref.diag(), d0g, d0r)


def test_hysteresis_and_static_walls_in_one_batch():
    cases = [wl.droplet(48, St=0.3, name="hyst", **CASE_A), wl.droplet(48, theta_deg=82.0, St=0.3, name="static"),
             periodic_film()]
    batch = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    batch.step(80)
    for k, c in enumerate(cases):
        alone = eulbfs.Solver([c], precision=eulbfs.FP32C)
        alone.step(80)
        fa, fb = alone.fields(), batch.fields(k)
        for key in FIELDS:
            assert np.array_equal(fa[key], fb[key]), (c.name, key)
