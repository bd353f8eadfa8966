"""Per-distribution streaming steps (reading R26): CUDA path vs the FP64 oracle.

Domains whose h, f, g streaming steps differ from 1/2 take the general face
path of the stage kernel.  FP64 every field element within 1e-10 of the
field's magnitude; FP32C within the stated FP32 tolerances; mixed with
default domains in one batch, each result bit for bit its result alone.
"""
import numpy as np
import pytest

import oracle
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

from test_gpu_parity import FIELDS, assert_fields_close, check_fp32c, ragged_case, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()
    oracle.build()


def steps(case, h, f, g):
    case.dt_h, case.dt_f, case.dt_g = h, f, g
    return case


FP64_CASES = [
    ("conductive_256x4_h0.3", lambda: steps(wl.conductive(256, 4), 0.3, 0.5, 0.5), 1000),
    ("three_phase_256x4_mixed", lambda: steps(wl.three_phase(256, 4, St=1.0, H0=128), 0.35, 0.45, 0.4), 600),
    ("droplet_64_mixed", lambda: steps(wl.droplet(64, theta_deg=60.0, St=0.2, Tw=-0.8), 0.4, 0.45, 0.35), 300),
    ("droplet_rz_64_mixed",
     lambda: steps(wl.droplet(64, theta_deg=100.0, St=0.3, axisymmetric=True), 0.45, 0.4, 0.42), 300),
    ("film_crop_72x40_uniform0.4", lambda: steps(wl.film(256).crop(72, 40), 0.4, 0.4, 0.4), 200),
]


@pytest.mark.parametrize("name,make,nsteps", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_streaming_steps_match_oracle(name, make, nsteps):
    case = make()
    gpu, ref = run_pair(case, nsteps)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=name, floor=1e-8)
    dg, dr = gpu.diag(), ref.diag()
    for k in ("mass", "enthalpy", "phase_vol", "solid_vol"):
        assert abs(dg[k] - dr[k]) <= 1e-10 * max(abs(dr[k]), 1.0), k


def test_fp64_benchmark_steps_on_a_batch_domain():
    """The steps the benchmark's general-streaming leg times, (0.3, 0.4, 0.3),
    on the smallest droplet of its (r, z) batch."""
    cases = wl.static_droplet_batch(64, seed=4, axisymmetric=True)
    case = steps(min(cases, key=lambda c: c.cells), 0.3, 0.4, 0.3)
    gpu, ref = run_pair(case, 60)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=case.name, floor=1e-8)


@pytest.mark.parametrize("nx,ny,per", [(33, 5, False), (37, 9, True)])
def test_fp64_streaming_steps_ragged(nx, ny, per):
    case = steps(ragged_case(nx, ny, per), 0.3, 0.45, 0.4)
    gpu, ref = run_pair(case, 40)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=f"{nx}x{ny}", floor=1e-8)


def test_fp32c_streaming_steps_within_tolerances():
    case = steps(wl.droplet(64, theta_deg=60.0, St=0.2, Tw=-0.8, axisymmetric=True), 0.4, 0.45, 0.4)
    gpu = eulbfs.Solver([case], precision=eulbfs.FP32C)
    d0g = gpu.diag()
    gpu.step(1000)
    ref = oracle.OracleSolver(case)
    d0r = ref.diag()
    ref.step(1000)
    check_fp32c(gpu.fields(), ref.fields(), gpu.diag(), ref.diag(), d0g, d0r)


def test_general_and_default_steps_in_one_batch():
    cases = [steps(wl.droplet(48, theta_deg=80.0, St=0.3, name="general"), 0.4, 0.45, 0.35),
             wl.droplet(48, theta_deg=80.0, St=0.3, name="default"),
             steps(wl.droplet(48, theta_deg=80.0, St=0.3, axisymmetric=True, name="general_rz"), 0.45, 0.4, 0.4)]
    batch = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    batch.step(80)
    for k, c in enumerate(cases):
        alone = eulbfs.Solver([c], precision=eulbfs.FP32C)
        alone.step(80)
        fa, fb = alone.fields(), batch.fields(k)
        for key in FIELDS:
            assert np.array_equal(fa[key], fb[key]), (c.name, key)
    # the general path does change the result
    assert not np.array_equal(batch.fields(0)["T"], batch.fields(1)["T"])
