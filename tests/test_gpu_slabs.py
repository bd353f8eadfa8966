"""One domain split along y into slabs that exchange 3-row halos after every
Runge-Kutta stage (eulbfs_add_split_domain).

The stencil of the step reaches two rows for the gradients of Eq. 54 and a
third for the Laplacian of C in mu_c, so with the halo rows copied from the
neighbouring slab every slab sees exactly what the undivided domain does:
the fields, stacked back, must equal the undivided domain's bit for bit.
Cases: the 512^2 film (walls on every side) in 2 and 4 slabs in both
precisions, a periodic-y three-phase problem in 2 slabs (the wrap is a halo
link too), and an axisymmetric droplet on a hysteresis plate in 3 uneven
slabs (the wall's apparent angle reads tangential neighbours in the halo).
"""
import numpy as np
import pytest

from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("H", "T", "Fl", "C", "p", "u", "v")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()


def _whole_and_split(case, k, steps, precision):
    whole = eulbfs.Solver([case], precision=precision)
    whole.step(steps)
    split = eulbfs.Solver([], precision=precision)
    slots = split.add_split(case, k)
    assert split.launches_per_step() == 6
    split.step(steps)
    return whole, split, slots


@pytest.mark.parametrize("precision", [eulbfs.FP32C, eulbfs.FP64])
@pytest.mark.parametrize("k", [2, 4])
def test_film_slabs_equal_undivided_domain(k, precision):
    case = wl.film(512)
    whole, split, slots = _whole_and_split(case, k, 100, precision)
    got, ref = split.split_fields(slots), whole.fields()
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f
    # the slabs' integrals add up to the domain's (different summation order)
    dw = whole.diag()
    for key in ("mass", "enthalpy", "phase_vol", "solid_vol"):
        tot = sum(split.diag(sl)[key] for sl in slots)
        assert abs(tot - dw[key]) <= 1e-12 * abs(dw[key]), key


def test_periodic_axis_split_links_the_wrap():
    case = wl.three_phase(128, 32, St=1.0, H0=64)        # periodic in y
    whole, split, slots = _whole_and_split(case, 2, 80, eulbfs.FP32C)
    got, ref = split.split_fields(slots), whole.fields()
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f


def test_axisymmetric_hysteresis_droplet_in_uneven_slabs():
    case = wl.droplet(128, theta_deg=82.0, St=0.3, axisymmetric=True, hysteresis=(100.0, 39.0),
                      impact_speed=0.03)
    whole, split, slots = _whole_and_split(case, 3, 60, eulbfs.FP32C)   # 42, 43, 43 rows
    assert [split.shapes[s][0] for s in slots] == [42, 43, 43]
    got, ref = split.split_fields(slots), whole.fields()
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f


def test_split_checkpoint_and_graphs_bitwise():
    """Halo rows are refreshed after set_state/load, and a captured graph
    replays the halo copies with the stages."""
    case = wl.film(256)
    ref = eulbfs.Solver([case], precision=eulbfs.FP32C)
    ref.step(40)
    s = eulbfs.Solver([], precision=eulbfs.FP32C)
    slots = s.add_split(case, 2)
    s.use_graphs(5)
    s.step(20)
    blobs = [s.save(sl) for sl in slots]
    t = eulbfs.Solver([], precision=eulbfs.FP32C)
    slots2 = t.add_split(case, 2)
    for sl, (blob, step) in zip(slots2, blobs):
        t.load(blob, step, sl)
    t.step(20)
    got, want = t.split_fields(slots2), ref.fields()
    for f in FIELDS:
        assert np.array_equal(got[f], want[f]), f


def test_split_rejects_too_thin_slabs():
    s = eulbfs.Solver([], precision=eulbfs.FP32C)
    with pytest.raises(eulbfs.EulbfsError) as e:
        s.add_split(wl.film(64), 9)          # 64 rows < 8 x 9
    assert e.value.code == eulbfs.EINVAL
