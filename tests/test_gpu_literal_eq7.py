"""Eq. 5-7 exactly as printed (``literal_eq7``) on the GPU against the oracle.

Reading R1 gates Eq. 7 by the phase field; the switch turns the gate off in
both implementations.  Where no gas gets colder than T_s (the three-phase
Stefan layers, the film under warm gas) the printed form runs, and the FP64
path matches the oracle element by element within 1e-10, FP32C within the
FP32 tolerances.  Where cold gas touches a cold wall (a droplet on a cold
plate), Eq. 7 as printed turns that gas into solid of about 900 times its
density and both implementations lose the state within 20 steps, while
reading R1 runs on.
"""
import numpy as np
import pytest

import oracle
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

from test_gpu_parity import assert_fields_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()
    oracle.build()


def _literal(case):
    case.props.literal_eq7 = 1
    return case


CASES = [
    ("three_phase_256x4_St1", lambda: wl.three_phase(256, 4, St=1.0, H0=128), 1000),
    ("film_crop_72x40", lambda: wl.film(256).crop(72, 40), 300),
]


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_fp64_literal_eq7_matches_oracle(name, make, steps):
    case = _literal(make())
    gpu = eulbfs.Solver([case], precision=eulbfs.FP64)
    gpu.step(steps)
    ref = oracle.OracleSolver(case)
    ref.step(steps)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=name)
    dg, dr = gpu.diag(), ref.diag()
    for k in ("mass", "enthalpy", "phase_vol", "solid_vol"):
        assert abs(dg[k] - dr[k]) <= 1e-10 * max(abs(dr[k]), 1.0), k


def test_fp32c_literal_eq7_within_fp32_tolerances():
    case = _literal(wl.three_phase(256, 4, St=1.0, H0=128))
    gpu = eulbfs.Solver([case], precision=eulbfs.FP32C)
    gpu.step(1000)
    ref = oracle.OracleSolver(case)
    ref.step(1000)
    g, r = gpu.fields(), ref.fields()
    for k in ("T", "C"):
        rel = np.linalg.norm(g[k] - r[k]) / np.linalg.norm(r[k])
        assert rel <= 1e-3, (k, rel)
    dg, dr = gpu.diag(), ref.diag()
    assert abs(dg["front_pos"] - dr["front_pos"]) <= 5e-3 * abs(dr["front_pos"])
    assert abs(dg["interface_pos"] - dr["interface_pos"]) <= 5e-3 * abs(dr["interface_pos"])


def test_literal_eq7_loses_the_cold_gas_droplet_on_both_sides():
    """The printed Eq. 7 freezes the cold gas at the plate; the GPU path and
    the oracle both report a non-finite state within 20 steps, and with
    reading R1 the same droplet runs 200 steps on both."""
    case = _literal(wl.droplet(48, theta_deg=60.0, St=0.2, Tw=-0.8))
    ref = oracle.OracleSolver(case)
    with pytest.raises(FloatingPointError):
        ref.step(20)
    gpu = eulbfs.Solver([case], precision=eulbfs.FP64)
    gpu.step(20)
    with pytest.raises(eulbfs.EulbfsError) as e:
        gpu.sync()
    assert e.value.code == eulbfs.ENONFINITE
    gated = wl.droplet(48, theta_deg=60.0, St=0.2, Tw=-0.8)
    g2 = eulbfs.Solver([gated], precision=eulbfs.FP64)
    g2.step(200)
    g2.sync()
    assert not g2.diag()["nonfinite"]
