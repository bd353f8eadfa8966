"""One launch per time step (eulbfs_set_whole_step, the default) against one
launch per Runge-Kutta stage.

In a whole-step launch the work items of stage 1, 2 and 3 run in one grid;
an item starts once the items of the previous stage whose output it reads
are done (its strip and the strips beside it, its rows and 4 rows beyond,
wrapped on periodic axes).  A missing neighbour in that list, or a wait that
let an item read a neighbour's output too early, changes the result, so the
two launch forms must agree bit for bit: on a mix of planar, axisymmetric,
periodic-x, periodic-y, hysteresis-wall and general-streaming domains of
ragged sizes, over several work-item heights, and on the 64-domain batch
(more items than resident CTAs, so stages overlap).
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


def _periodic_x(nx, ny):
    rng = np.random.default_rng(nx + 7 * ny)
    case = wl.droplet(max(nx, ny), theta_deg=70.0, St=0.25, Tw=-0.6).crop(nx, ny)
    case.bc = wl.BC(wl.PER, wl.PER, wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, Tw=-0.6, theta_deg=70.0),
                    wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX))
    y = np.arange(ny) + 0.5
    case.init["C"] = np.ascontiguousarray(np.broadcast_to((0.5 * (1 + np.tanh(2 * (ny / 2 - y) / 4.0)))[:, None],
                                                          (ny, nx)))
    case.init["T"] = case.init["T"] + 0.05 * rng.standard_normal((ny, nx))
    case.init["u"] = 1e-3 * rng.standard_normal((ny, nx)) * case.init["C"]
    return case


def _periodic_y(nx, ny):
    rng = np.random.default_rng(nx * 100 + ny)
    case = wl.droplet(max(nx, ny), theta_deg=75.0, St=0.25, Tw=-0.6).crop(nx, ny)
    case.bc = wl.BC(wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, Tw=-0.6, theta_deg=75.0),
                    wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX), wl.PER, wl.PER)
    x = np.arange(nx) + 0.5
    case.init["C"] = np.ascontiguousarray(np.broadcast_to(0.5 * (1 + np.tanh(2 * (nx / 2 - x) / 4.0)), (ny, nx)))
    case.init["T"] = case.init["T"] + 0.05 * rng.standard_normal((ny, nx))
    return case


def _mix():
    gen = wl.droplet(70, theta_deg=95.0, St=0.3)
    gen.dt_h, gen.dt_f, gen.dt_g = 0.3, 0.4, 0.3
    return [
        wl.droplet(96, theta_deg=82.0, St=0.3, axisymmetric=True, hysteresis=(100.0, 39.0), impact_speed=0.03),
        _periodic_x(100, 48),
        _periodic_y(37, 90),
        wl.droplet(65, theta_deg=60.0, St=0.2),
        gen,
        wl.droplet(40, theta_deg=110.0, St=0.25, axisymmetric=True),
        wl.film(128),
    ]


def _run(cases, precision, whole, steps, tile=0, graphs=0):
    s = eulbfs.Solver(cases, precision=precision)
    s.set_whole_step(whole)
    if tile:
        s.set_tile(tile)
    if graphs:
        s.use_graphs(graphs)
    s.step(steps)
    return s


@pytest.mark.parametrize("precision", [eulbfs.FP32C, eulbfs.FP64])
def test_whole_step_equals_stage_launches_on_a_mixed_batch(precision):
    cases = _mix()
    ref = _run(cases, precision, False, 30)
    assert ref.launches_per_step() == 3
    for tile in (8, 24, 64):
        got = _run(cases, precision, True, 30, tile=tile, graphs=5 if tile == 24 else 0)
        assert got.launches_per_step() == 1
        for k in range(len(cases)):
            a, b = got.fields(k), ref.fields(k)
            for f in FIELDS:
                assert np.array_equal(a[f], b[f]), (tile, k, f)
        for k in range(len(cases)):
            assert got.diag(k)["step"] == 30


def test_whole_step_on_the_64_domain_batch():
    """More items than resident CTAs: a stage's last items run while the next
    stage's first ones do."""
    cases = wl.static_droplet_batch(64, axisymmetric=True)
    ref = _run(cases, eulbfs.FP32C, False, 6, tile=64)
    got = _run(cases, eulbfs.FP32C, True, 6, tile=64)
    for k in range(0, 64, 7):
        a, b = got.fields(k), ref.fields(k)
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), (k, f)
    # every domain, through its integrals
    for k in range(64):
        assert got.diag(k)["mass"] == ref.diag(k)["mass"], k


def test_split_domains_launch_per_stage():
    s = eulbfs.Solver([], precision=eulbfs.FP32C)
    s.add_split(wl.film(256), 2)
    assert s.launches_per_step() == 6
    s.set_whole_step(False)
    assert s.launches_per_step() == 6


def test_whole_step_argument_checks():
    s = eulbfs.Solver([wl.droplet(32)], precision=eulbfs.FP32C)
    with pytest.raises(eulbfs.EulbfsError) as e:
        eulbfs._check(eulbfs.lib().eulbfs_set_whole_step(s._h, 2))
    assert e.value.code == eulbfs.EINVAL
    s.set_whole_step(False)
    assert s.launches_per_step() == 3
    s.set_whole_step(True)
    assert s.launches_per_step() == 1


@pytest.mark.parametrize("precision", [eulbfs.FP32C, eulbfs.FP64])
def test_bounded_neighbour_wait_reports_timeout_and_context_survives(precision):
    """Failure detection without a fault: with probe 2 no work item marks
    itself done, so every stage-2 item waits out its bound (about a second of
    SM clocks) for the items it reads, the kernel stops and the host reads
    ETIMEOUT.  The context stays usable: two fresh solvers then agree bit for
    bit."""
    import time
    case = wl.droplet(96, theta_deg=90.0, St=0.3)
    s = eulbfs.Solver([case], precision=precision)
    with pytest.raises(eulbfs.EulbfsError) as e:
        eulbfs._check(eulbfs.lib().eulbfs_set_tile_wait_probe(s._h, 3))
    assert e.value.code == eulbfs.EINVAL
    eulbfs._check(eulbfs.lib().eulbfs_set_tile_wait_probe(s._h, 2))
    t0 = time.perf_counter()
    s.step(1)
    with pytest.raises(eulbfs.EulbfsError) as e:
        s.sync()
    assert e.value.code == eulbfs.ETIMEOUT
    assert time.perf_counter() - t0 < 60.0
    s.close()
    a = _run([case], precision, True, 5)
    b = _run([case], precision, False, 5)
    for f in FIELDS:
        assert np.array_equal(a.fields()[f], b.fields()[f]), f


def test_several_steps_per_launch_equal_single_steps():
    """An eulbfs_step of many steps runs up to 16 whole steps in one launch
    (stage 1 of a step waits for stage 3 of the step before, item by item);
    a domain's step limit inside that span cuts the launch there."""
    cases = _mix()[:4]
    a = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    n0 = a.launch_count()
    a.step(37)                                   # launches of 16, 16 and 5 steps
    assert a.launch_count() - n0 == 3
    b = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    for _ in range(37):
        b.step(1)
    assert b.launch_count() == 37
    for k in range(len(cases)):
        for f in FIELDS:
            assert np.array_equal(a.fields(k)[f], b.fields(k)[f]), (k, f)
    # a step limit at 7: the first launch stops there, the rest carry on
    c = eulbfs.Solver([cases[0]], precision=eulbfs.FP32C)
    slot = c.add(cases[1], max_steps=7)
    c.step(20)
    assert c.progress(slot)[0] == 7 and c.progress(0)[0] == 20
    alone = eulbfs.Solver([cases[1]], precision=eulbfs.FP32C)
    alone.step(7)
    ref0 = eulbfs.Solver([cases[0]], precision=eulbfs.FP32C)
    ref0.step(20)
    for f in FIELDS:
        assert np.array_equal(c.fields(slot)[f], alone.fields()[f]), f
        assert np.array_equal(c.fields(0)[f], ref0.fields()[f]), f
