"""CUDA path vs the FP64 CPU oracle, through the C ABI.

FP64: every field element within 1e-10 of the field's magnitude after up to
1000 steps.  FP32C (FP32 arithmetic, compensated H and C): relative L2 of T,
u, C within 1e-3, front and interface positions within 0.5 %, relative total
mass drift within 1e-6 of the oracle's drift.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("H", "T", "Fl", "C", "p", "u", "v")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()
    oracle.build()


def assert_fields_close(g, r, rtol, keys=FIELDS, what="", floor=1e-12):
    """Max-norm error of each field relative to the field's magnitude (at
    least `floor`); the two velocity components share the speed scale (one is
    pure round-off noise in the quasi-1D problems).  T is recovered from the
    enthalpy (Eq. 5-6: T = (H - L F_l) / C_p, C_p = O(1) here), so its
    round-off is relative to |H| as well as to |T|: a droplet near T_m = 0
    has |T| << |H|."""
    speed = max(float(np.max(np.abs(r["u"]))), float(np.max(np.abs(r["v"]))), floor)
    hscale = float(np.max(np.abs(r["H"]))) if "H" in r else 0.0
    for k in keys:
        scale = speed if k in ("u", "v") else max(float(np.max(np.abs(r[k]))), floor)
        if k == "T":
            scale = max(scale, hscale)
        err = float(np.max(np.abs(g[k] - r[k])))
        assert err <= rtol * scale, f"{what} field {k}: max|gpu - oracle| = {err:.3e} > {rtol:g} * {scale:.3e}"


def run_pair(case, steps, precision=eulbfs.FP64):
    gpu = eulbfs.Solver([case], precision=precision)
    gpu.step(steps)
    ref = oracle.OracleSolver(case)
    ref.step(steps)
    return gpu, ref


# ---------------------------------------------------------------------------
# FP64 element-wise parity
# ---------------------------------------------------------------------------
FP64_CASES = [
    ("conductive_256x4", lambda: wl.conductive(256, 4), 1000),
    ("three_phase_256x4_St0.1", lambda: wl.three_phase(256, 4, St=0.1, H0=128), 1000),
    ("three_phase_256x4_St1", lambda: wl.three_phase(256, 4, St=1.0, H0=128), 1000),
    ("film_crop_72x40", lambda: wl.film(256).crop(72, 40), 300),
    ("droplet_crop_70x45", lambda: wl.droplet(80, theta_deg=120.0, St=0.3).crop(70, 45), 300),
    ("droplet_64_wet60", lambda: wl.droplet(64, theta_deg=60.0, St=0.2, Tw=-0.8), 300),
]


@pytest.mark.parametrize("name,make,steps", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_matches_oracle(name, make, steps):
    case = make()
    gpu, ref = run_pair(case, steps)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=name)
    dg, dr = gpu.diag(), ref.diag()
    for k in ("mass", "enthalpy", "phase_vol", "solid_vol"):
        assert abs(dg[k] - dr[k]) <= 1e-10 * max(abs(dr[k]), 1.0), k
    assert dg["step"] == steps and not dg["nonfinite"]


def test_fp64_full_size_three_phase():
    """Three-phase Stefan problem at its full 1024 x 4 size, 1000 steps."""
    case = wl.three_phase(1024, 4, St=1.0)
    gpu, ref = run_pair(case, 1000)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what="three_phase_1024x4")


def ragged_case(nx, ny, per):
    """Droplet crop on walled grids; on a periodic y axis a liquid layer along
    x (continuous across the seam) frozen from a wetting cold wall at x = 0."""
    rng = np.random.default_rng(nx * 100 + ny)
    case = wl.droplet(max(nx, ny), theta_deg=75.0, St=0.25, Tw=-0.6).crop(nx, ny)
    if per:
        case.bc = wl.BC(wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, Tw=-0.6, theta_deg=75.0),
                        wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX), wl.PER, wl.PER)
        x = np.arange(nx) + 0.5
        case.init["C"] = np.ascontiguousarray(np.broadcast_to(0.5 * (1 + np.tanh(2 * (nx / 2 - x) / 4.0)), (ny, nx)))
    case.init["T"] = case.init["T"] + 0.05 * rng.standard_normal((ny, nx))
    case.init["u"] = 1e-3 * rng.standard_normal((ny, nx)) * case.init["C"]
    return case


@pytest.mark.parametrize("nx,ny,per", [(33, 5, False), (37, 9, True), (2, 17, False), (40, 1, True), (65, 3, True)])
def test_fp64_ragged_and_degenerate_grids(nx, ny, per):
    """Tiles with ragged tails in x and y, a 1-row periodic domain and the
    narrowest walled domain (2 cells)."""
    case = ragged_case(nx, ny, per)
    gpu, ref = run_pair(case, 40)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-10, what=f"{nx}x{ny}")


# ---------------------------------------------------------------------------
# Full-size cases in the batched launch configuration: one step from a
# common state, compared on whole fields (film) or sampled domains (batch).
# ---------------------------------------------------------------------------
def _one_step_from_gpu_state(gpu, slot, case, precision):
    st = gpu.state(slot)
    ref = oracle.OracleSolver(case)
    ref.set_state(st, st["t"], st["step"])
    ref.step(1)
    return ref


def test_fp64_full_size_film_one_step():
    case = wl.film(512)
    gpu = eulbfs.Solver([case], precision=eulbfs.FP64)
    gpu.step(20)
    ref = _one_step_from_gpu_state(gpu, 0, case, eulbfs.FP64)
    gpu.step(1)
    assert_fields_close(gpu.fields(), ref.fields(), 1e-12, what="film_512 one step")


def test_fp64_batch_sampled_domains_one_step():
    cases = wl.static_droplet_batch(64)
    gpu = eulbfs.Solver(cases, precision=eulbfs.FP64)
    gpu.step(10)
    sizes = [c.nx for c in cases]
    sample = [sizes.index(min(sizes)), sizes.index(max(sizes)), 7]
    refs = {k: _one_step_from_gpu_state(gpu, k, cases[k], eulbfs.FP64) for k in sample}
    gpu.step(1)
    for k in sample:
        assert_fields_close(gpu.fields(k), refs[k].fields(), 1e-12, what=f"batch domain {k}")


# ---------------------------------------------------------------------------
# FP32C against the oracle, tolerances as stated for the FP32 form.
# ---------------------------------------------------------------------------
def rel_l2(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / max(nb, 1e-30)


def check_fp32c(g, r, dg, dr, d0g, d0r):
    """The tolerances stated for the FP32 form against the FP64 oracle."""
    assert rel_l2(g["T"], r["T"]) <= 1e-3
    assert rel_l2(g["C"], r["C"]) <= 1e-3
    if np.linalg.norm(r["u"]) > 0:
        assert rel_l2(g["u"], r["u"]) <= 1e-3, rel_l2(g["u"], r["u"])
    assert abs(dg["front_pos"] - dr["front_pos"]) <= 5e-3 * dr["front_pos"]
    disp_g = dg["interface_pos"] - d0g["interface_pos"]
    disp_r = dr["interface_pos"] - d0r["interface_pos"]
    assert abs(disp_g - disp_r) <= 5e-3 * max(abs(disp_r), 1e-3 * dr["interface_pos"])
    drift_g = dg["mass"] / d0g["mass"] - 1.0
    drift_r = dr["mass"] / d0r["mass"] - 1.0
    assert abs(drift_g - drift_r) <= 1e-6


FP32C_CASES = [
    ("conductive_256x4", lambda: wl.conductive(256, 4), 1000),
    ("three_phase_1024x4_St0.1", lambda: wl.three_phase(1024, 4, St=0.1), 1000),
    ("three_phase_1024x4_St1", lambda: wl.three_phase(1024, 4, St=1.0), 1000),
    ("droplet_64_wet60", lambda: wl.droplet(64, theta_deg=60.0, St=0.2, Tw=-0.8), 1000),
    ("film_crop_72x40", lambda: wl.film(256).crop(72, 40), 1000),
]


@pytest.mark.parametrize("name,make,steps", FP32C_CASES, ids=[c[0] for c in FP32C_CASES])
def test_fp32c_within_tolerances(name, make, steps):
    case = make()
    gpu = eulbfs.Solver([case], precision=eulbfs.FP32C)
    d0g = gpu.diag()
    gpu.step(steps)
    ref = oracle.OracleSolver(case)
    d0r = ref.diag()
    ref.step(steps)
    check_fp32c(gpu.fields(), ref.fields(), gpu.diag(), ref.diag(), d0g, d0r)


def test_fp32c_batch_domain_in_launch_configuration():
    """A 128 x 128 domain advanced inside the full 64-domain FP32C batch (the
    benchmark's launch configuration) against the oracle run on it alone."""
    cases = wl.static_droplet_batch(64)
    k = [c.nx for c in cases].index(128)
    gpu = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    d0g = gpu.diag(k)
    gpu.step(300)
    ref = oracle.OracleSolver(cases[k])
    d0r = ref.diag()
    ref.step(300)
    check_fp32c(gpu.fields(k), ref.fields(), gpu.diag(k), ref.diag(), d0g, d0r)


# ---------------------------------------------------------------------------
# Batching, checkpoints, graphs, tiles: results independent of placement.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_domain_alone_equals_domain_in_mix(precision):
    cases = wl.static_droplet_batch(6, sides=(32, 48, 64, 96))
    mix = eulbfs.Solver(cases, precision=precision)
    mix.step(30)
    for k in (0, 3, 5):
        alone = eulbfs.Solver([cases[k]], precision=precision)
        alone.step(30)
        a, m = alone.fields(0), mix.fields(k)
        for f in FIELDS:
            assert np.array_equal(a[f], m[f]), (k, f)


@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_checkpoint_resume_bitwise(precision):
    """2n steps == n steps, save, new solver, load, n steps (bit for bit)."""
    case = wl.droplet(48, theta_deg=110.0, St=0.2)
    full = eulbfs.Solver([case], precision=precision)
    full.step(40)
    half = eulbfs.Solver([case], precision=precision)
    half.step(20)
    blob, step = half.save()
    assert step == 20
    resumed = eulbfs.Solver([case], precision=precision)
    resumed.load(blob, step)
    resumed.step(20)
    assert full.save()[0] == resumed.save()[0]
    assert resumed.progress(0)[0] == 40


@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_state_round_trip_through_doubles(precision):
    """get_state/set_state: exact in FP64; FP32C pairs to 2^-53 relative."""
    case = wl.droplet(48, theta_deg=80.0, St=0.3)
    a = eulbfs.Solver([case], precision=precision)
    a.step(15)
    st = a.state()
    b = eulbfs.Solver([case], precision=precision)
    b.set_state(st)
    st2 = b.state()
    for k in ("H", "p", "mx", "my", "C", "Fsp"):
        if precision == eulbfs.FP64 or k not in ("H", "C"):
            assert np.array_equal(st[k], st2[k]), k
        else:
            assert np.max(np.abs(st[k] - st2[k])) <= 2.0 ** -52 * np.max(np.abs(st[k])), k
    assert st2["step"] == 15


@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_graph_replay_and_work_item_shapes_bitwise(precision):
    cases = wl.static_droplet_batch(3, sides=(40, 72))
    ref = eulbfs.Solver(cases, precision=precision)
    ref.step(12)
    for tile in (8, 24, 64):
        s = eulbfs.Solver(cases, precision=precision)
        s.set_tile(tile)
        s.use_graphs(4)
        s.step(12)
        for k in range(3):
            for f in FIELDS:
                assert np.array_equal(s.fields(k)[f], ref.fields(k)[f]), (tile, k, f)


def test_autotune_picks_a_candidate_and_steps_as_documented():
    cases = wl.static_droplet_batch(3, sides=(40, 72), axisymmetric=True)
    s = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    rows, ms = s.autotune(2)
    assert rows in (32, 48, 64, 96, 128, 160, 192, 256) and ms > 0
    assert sorted(s.autotune_report()) == [32, 48, 64, 96, 128, 160, 192, 256]
    steps = 2 * 8 * (2 + 1)               # two rounds over eight heights, each 1 + 2 steps
    assert s.diag(0)["step"] == steps
    ref = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    ref.step(steps)
    for k in range(3):                    # the heights it ran do not change the result
        for f in FIELDS:
            assert np.array_equal(s.fields(k)[f], ref.fields(k)[f]), (k, f)
    with pytest.raises(eulbfs.EulbfsError):
        s.autotune(0)


# ---------------------------------------------------------------------------
# Continuous batching and failure detection (host-side faults only).
# ---------------------------------------------------------------------------
def test_add_remove_step_limits_and_budget():
    a, b = wl.droplet(32), wl.droplet(48, theta_deg=100.0)
    s = eulbfs.Solver([a], precision=eulbfs.FP32C)
    slot = s.add(b, max_steps=5)
    s.step(8)
    assert s.progress(0) == (8, -1)
    assert s.progress(slot) == (5, 0)
    ref = eulbfs.Solver([b], precision=eulbfs.FP32C)
    ref.step(5)
    assert np.array_equal(ref.fields(0)["H"], s.fields(slot)["H"])
    s.remove(slot)
    with pytest.raises(eulbfs.EulbfsError):
        s.fields(slot)
    s.set_memory_budget(eulbfs.lib().eulbfs_domain_bytes(32, 32, eulbfs.FP32C) + 1024)
    with pytest.raises(eulbfs.EulbfsError) as e:
        s.add(wl.droplet(64))
    assert e.value.code == eulbfs.EBUSY


def test_nonfinite_input_rejected():
    case = wl.droplet(32)
    case.init["T"][5, 7] = float("nan")
    with pytest.raises(eulbfs.EulbfsError) as e:
        eulbfs.Solver([case], precision=eulbfs.FP32C)
    assert e.value.code == eulbfs.EINVAL


@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_nonfinite_state_is_reported(precision):
    """A poisoned state, planted from the host through the checkpoint API,
    is reported by sync and by the diagnostics."""
    s = eulbfs.Solver([wl.droplet(32)], precision=precision)
    s.step(2)
    st = s.state()
    st["p"][5, 7] = float("nan")
    s.set_state(st)
    s.step(2)
    with pytest.raises(eulbfs.EulbfsError) as e:
        s.sync()
    assert e.value.code == eulbfs.ENONFINITE
    with pytest.raises(eulbfs.EulbfsError) as e:
        s.diag()
    assert e.value.code == eulbfs.ENONFINITE


# ---------------------------------------------------------------------------
# Long runs of the two Stefan problems at their full sizes, both precisions,
# against the closed forms (Neumann front, Eq. 59-60 one-phase limit; the
# mass-conservation displacement (1 - rho_s/rho_l) x_s of Sec. 3.2).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_conductive_20k_steps_front_follows_neumann(precision):
    """Conductive freezing, 256 x 4, 20 000 steps: the front stays within 1 %
    of 2 k sqrt(alpha t) once it is 16 cells from the wall."""
    c = wl.conductive(256, 4)
    k = wl.neumann_k(0.1)
    s = eulbfs.Solver([c], precision=precision)
    fronts = []
    for _ in range(4):
        s.step(5000)
        d = s.diag()
        xs = 2 * k * math.sqrt(0.1 * d["t"])
        if xs >= 16.0:
            assert abs(d["front_pos"] / xs - 1.0) < 0.01, (d["t"], d["front_pos"], xs)
        fronts.append(d["front_pos"])
    assert d["step"] == 20000 and fronts[-1] > 16.0


def test_three_phase_long_run_fp32c_against_fp64():
    """Three-phase Stefan, 1024 x 4, St = 1, 20 000 steps: the FP64 step follows
    the Neumann front and the expansion law; the FP32C step stays within
    0.5 % of it in front and interface displacement, and its relative mass
    drift within 1e-6 of the FP64 one."""
    c = wl.three_phase(1024, 4, St=1.0)
    kv = 1.0 - c.props.s.rho / c.props.l.rho
    k = wl.neumann_k(1.0)
    out = {}
    for prec in (eulbfs.FP64, eulbfs.FP32C):
        s = eulbfs.Solver([c], precision=prec)
        d0 = s.diag()
        s.step(20000)
        out[prec] = (d0, s.diag())
    d0, d = out[eulbfs.FP64]
    xs = d["front_pos"]
    assert abs(xs / (2 * k * math.sqrt(0.1 * d["t"])) - 1.0) < 0.01
    disp = d["interface_pos"] - d0["interface_pos"]
    assert abs(disp / (kv * xs) - 1.0) < 0.02
    e0, e = out[eulbfs.FP32C]
    assert abs(e["front_pos"] - xs) <= 5e-3 * xs
    assert abs((e["interface_pos"] - e0["interface_pos"]) - disp) <= 5e-3 * abs(disp)
    assert abs((e["mass"] / e0["mass"] - 1.0) - (d["mass"] / d0["mass"] - 1.0)) <= 1e-6


def test_film_512_long_run_fp32c_against_fp64():
    """Liquid film freezing, 512 x 512, 50 000 steps (the film configuration's
    length): the FP32C step within the stated FP32 tolerances of the FP64
    step on the full-size film.  (Measured: T and C within 5e-8 relative L2,
    front within 1e-7, mass drift within 4e-9.)"""
    c = wl.film(512)
    runs = {}
    for prec in (eulbfs.FP64, eulbfs.FP32C):
        s = eulbfs.Solver([c], precision=prec)
        d0 = s.diag()
        s.step(50000)
        runs[prec] = (s.fields(), s.diag(), d0)
    r, dr, d0r = runs[eulbfs.FP64]
    g, dg, d0g = runs[eulbfs.FP32C]
    assert dr["solid_vol"] > 0 and not dr["nonfinite"]
    check_fp32c(g, r, dg, dr, d0g, d0r)


def test_solvers_on_two_host_threads():
    """FP64 and FP32C solvers created and stepped from two host threads at
    once (the stage kernel's launch set-up is per device and locked) give
    the results of the same solvers run one after the other."""
    import threading
    cases = [lambda: wl.droplet(48, theta_deg=80.0, St=0.3), lambda: wl.three_phase(128, 4, St=1.0, H0=64)]

    def run(make, precision, out, key):
        s = eulbfs.Solver([make()], precision=precision)
        s.step(60)
        out[key] = s.fields()
        s.close()

    serial, threaded = {}, {}
    for k, make in enumerate(cases):
        for prec in (eulbfs.FP64, eulbfs.FP32C):
            run(make, prec, serial, (k, prec))
    threads = [threading.Thread(target=run, args=(make, prec, threaded, (k, prec)))
               for k, make in enumerate(cases) for prec in (eulbfs.FP64, eulbfs.FP32C)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert set(threaded) == set(serial)
    for key in serial:
        for f in FIELDS:
            assert np.array_equal(threaded[key][f], serial[key][f]), (key, f)


def test_bounded_tile_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: with the wait probe on, every TMA
    tile barrier expects 16 bytes that never arrive, each wait gives up after
    its bound (about a second of SM clocks), the kernel stops and the host
    reads ETIMEOUT.  The context stays usable: a new solver on the same case
    then matches a third, fresh one bit for bit."""
    import time
    case = wl.droplet(96, theta_deg=90.0, St=0.3)     # nx = 96: tensor maps and two interior strips
    s = eulbfs.Solver([case], precision=eulbfs.FP32C)
    eulbfs._check(eulbfs.lib().eulbfs_set_tile_wait_probe(s._h, 1))
    t0 = time.perf_counter()
    s.step(1)
    with pytest.raises(eulbfs.EulbfsError) as e:
        s.sync()
    assert e.value.code == eulbfs.ETIMEOUT
    assert time.perf_counter() - t0 < 60.0
    s.close()
    a = eulbfs.Solver([case], precision=eulbfs.FP32C)
    a.step(5)
    a.sync()
    b = eulbfs.Solver([case], precision=eulbfs.FP32C)
    b.step(5)
    for f in FIELDS:
        assert np.array_equal(a.fields()[f], b.fields()[f]), f
