"""Axisymmetric (r, z) domains: CUDA path vs the FP64 oracle, through the C ABI.

The same bars as the planar parity tests: FP64 every field element within
1e-10 of the field's magnitude, the r-weighted diagnostics within 1e-10;
FP32C within the stated FP32 tolerances.  Cases: the closed-form problems of
the oracle's axisymmetric pins (cylinder conduction, pipe flow, a relaxing
liquid column), droplets of revolution on a cold wetting plate (static and
impacting), ragged tiles, and a batch that mixes planar and axisymmetric
domains in one launch.
"""
import math

import numpy as np
import pytest
from scipy.special import j0

import oracle
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

from test_gpu_parity import FIELDS, assert_fields_close, check_fp32c, run_pair

pytestmark = pytest.mark.gpu

AXIS = wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX)
WALL = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()
    oracle.build()


def _props(**kw):
    base = dict(rho=(1.0, 1.0, 1.0), mu=(0.1, 0.1, 0.1), lam=(0.1, 0.1, 0.1), cp=(1.0, 1.0, 1.0), L=1.0,
                Ts=-5.0, Tl=-5.0, sigma=0.0, xi=4.0, Mc=0.0, tau_g=1.0, gx=0.0, gy=0.0, zsv=0)
    base.update(kw)
    ph = [wl.Phase(base["rho"][k], base["mu"][k], base["lam"][k], base["cp"][k]) for k in range(3)]
    return wl.Props(ph[0], ph[1], ph[2], base["L"], base["Ts"], base["Tl"], base["sigma"], base["xi"],
                    base["Mc"], base["tau_g"], base["gx"], base["gy"], base["zsv"])


def _case(name, nx, ny, props, bc, dt=1.0, **fields):
    f = dict(T=0.0, Fl=1.0, C=1.0)
    f.update(fields)
    return wl.Case(name, nx, ny, props, bc, dt, wl._fields(nx, ny, **f), axisymmetric=1)


def cylinder_conduction():
    R = 24
    r = np.arange(R) + 0.5
    T0 = np.broadcast_to(j0(2.404825557695773 / R * r), (2, R))
    cold = wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.NOFLUX, Tw=0.0)
    return _case("cylinder_conduction_24x2", R, 2, _props(), wl.BC(AXIS, cold, wl.PER, wl.PER), T=T0)


def pipe_flow():
    return _case("pipe_flow_8x2", 8, 2, _props(gy=1e-5), wl.BC(AXIS, WALL, wl.PER, wl.PER))


def liquid_column():
    nx, ny = 32, 32
    r = np.arange(nx) + 0.5
    z = np.arange(ny) + 0.5
    Rz = 8.0 + 1.5 * np.cos(2 * math.pi * z / ny)
    C = 0.5 * (1 + np.tanh(2 * (Rz[:, None] - r[None, :]) / 4.0))
    P = _props(rho=(1.0, 1.0, 0.1), mu=(0.1, 0.1, 0.01), sigma=0.01, Mc=0.1)
    return _case("liquid_column_32x32", nx, ny, P, wl.BC(AXIS, WALL, wl.PER, wl.PER), C=C)


def stagnation_flow():
    nx, ny, a = 40, 24, 2e-4
    r = np.arange(nx) + 0.5
    z = np.arange(ny) + 0.5 - ny / 2
    out = wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX)
    return _case("stagnation_flow_40x24", nx, ny, _props(), wl.BC(AXIS, out, out, out), T=1.0,
                 u=a * r[None, :] * np.ones((ny, 1)), v=-2 * a * z[:, None] * np.ones((1, nx)))


FP64_CASES = [
    ("cylinder_conduction_24x2", cylinder_conduction, 500),
    ("pipe_flow_8x2", pipe_flow, 500),
    ("liquid_column_32x32", liquid_column, 200),
    ("stagnation_flow_40x24", stagnation_flow, 100),
    ("droplet_rz_64_wet60", lambda: wl.droplet(64, theta_deg=60.0, St=0.2, Tw=-0.8, axisymmetric=True), 300),
    ("droplet_rz_crop_70x45",
     lambda: wl.droplet(80, theta_deg=120.0, St=0.3, axisymmetric=True).crop(70, 45), 300),
    ("impact_rz_64",
     lambda: wl.droplet(64, theta_deg=90.0, St=0.3, Tw=-1.0, impact_speed=0.05, We=50.0, Re=500.0,
                        axisymmetric=True), 120),
]


@pytest.mark.parametrize("name,make,steps", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_axisymmetric_matches_oracle(name, make, steps):
    case = make()
    gpu, ref = run_pair(case, steps)
    # fields that stay at round-off level (p of the pipe flow) are held to 1e-18
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=name, floor=1e-8)
    dg, dr = gpu.diag(), ref.diag()
    for k in ("mass", "enthalpy", "phase_vol", "solid_vol", "front_pos", "interface_pos"):
        assert abs(dg[k] - dr[k]) <= 1e-10 * max(abs(dr[k]), 1.0), k
    assert dg["step"] == steps and not dg["nonfinite"]


@pytest.mark.parametrize("nx,ny", [(33, 5), (2, 17), (65, 3)])
def test_fp64_axisymmetric_ragged_tiles(nx, ny):
    """Ragged x and y tails, and the narrowest walled radius (2 cells)."""
    rng = np.random.default_rng(nx * 31 + ny)
    case = wl.droplet(max(nx, ny), theta_deg=75.0, St=0.25, Tw=-0.6, axisymmetric=True).crop(nx, ny)
    case.init["T"] = case.init["T"] + 0.05 * rng.standard_normal((ny, nx))
    case.init["u"] = 1e-3 * rng.standard_normal((ny, nx)) * case.init["C"]
    gpu, ref = run_pair(case, 40)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=f"rz {nx}x{ny}")


def test_fp32c_axisymmetric_droplet_within_tolerances():
    case = wl.droplet(64, theta_deg=60.0, St=0.2, Tw=-0.8, axisymmetric=True)
    gpu = eulbfs.Solver([case], precision=eulbfs.FP32C)
    d0g = gpu.diag()
    gpu.step(1000)
    ref = oracle.OracleSolver(case)
    d0r = ref.diag()
    ref.step(1000)
    check_fp32c(gpu.fields(), ref.fields(), gpu.diag(), ref.diag(), d0g, d0r)


@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_mixed_planar_and_axisymmetric_batch(precision):
    """Planar and axisymmetric domains share the stage launches; each result
    is bit for bit the one it has alone, and the FP64 ones match the oracle."""
    cases = [wl.droplet(48, theta_deg=100.0, St=0.3, axisymmetric=True, name="rz48"),
             wl.droplet(48, theta_deg=100.0, St=0.3, name="xy48"),
             wl.droplet(72, theta_deg=70.0, St=0.2, axisymmetric=True).crop(72, 40, name="rz72"),
             wl.film(256).crop(40, 33, name="film40")]
    steps = 60
    batch = eulbfs.Solver(cases, precision=precision)
    batch.step(steps)
    for k, c in enumerate(cases):
        alone = eulbfs.Solver([c], precision=precision)
        alone.step(steps)
        fa, fb = alone.fields(), batch.fields(k)
        for key in FIELDS:
            assert np.array_equal(fa[key], fb[key]), (c.name, key)
        if precision == eulbfs.FP64:
            ref = oracle.OracleSolver(c)
            ref.step(steps)
            assert_fields_close(fb, ref.fields(), 1e-10, what=c.name)
    # the planar and axisymmetric twins differ (the geometry is not ignored)
    assert not np.allclose(batch.fields(0)["C"], batch.fields(1)["C"], atol=1e-6)
