"""Brute-force pin of the oracle's face flux and time step on random fields.

Every other face-flux pin uses fields that are uniform, linear or vary in one
quantity at a time.  Here rho, mu, lambda, C_p (through random H and C in
the solid, mushy and liquid ranges), T, p, u, v, C and mu_c all vary at
random on 4x4, 5x3 and 5x4 grids, with walls of every kind (contact-angle
hysteresis included), periodic sides, the axisymmetric (r, z) form and
per-distribution streaming steps.  The
reference is ``brute_eulbfs``, a second transcription of Sec. 2.5 steps
(2)-(4) (Eq. 54, 9/29/33/42, 56, 13/16, 35/37, 44/46, 53) and of Eq. 51-52,
58 written from the paper in 40-digit arithmetic.  The oracle must agree with
it to FP64 rounding on every face flux (all five components and u_n) and on
one full Runge-Kutta step (with a non-zero lagged solid-fraction rate).
"""
import numpy as np
import pytest

pytest.importorskip("mpmath")

import oracle  # noqa: E402
from paper_2507_03366_gb300 import workloads as wl  # noqa: E402

import brute_eulbfs as bf  # noqa: E402

TOL = 1e-13


def _props(literal=False, gy=0.0):
    ph = [wl.Phase(0.9, 0.02, 0.12, 0.8), wl.Phase(1.0, 0.05, 0.08, 1.2), wl.Phase(0.2, 0.01, 0.03, 0.5)]
    p = wl.Props(ph[0], ph[1], ph[2], L=0.5, Ts=-0.05, Tl=0.05, sigma=0.02, xi=2.5, Mc=0.05, tau_g=0.9,
                 gx=0.0, gy=gy, zero_solid_velocity=1)
    if literal:
        p.literal_eq7 = 1
    return p


def _random_state(nx, ny, seed):
    """H over the solid, mushy and liquid ranges, C slightly beyond [0, 1]."""
    rng = np.random.default_rng(seed)
    return {"H": rng.uniform(-0.4, 1.1, (ny, nx)), "p": rng.uniform(-0.05, 0.05, (ny, nx)),
            "mx": rng.uniform(-0.02, 0.02, (ny, nx)), "my": rng.uniform(-0.02, 0.02, (ny, nx)),
            "C": rng.uniform(-0.05, 1.05, (ny, nx)), "Fsp": rng.uniform(0.0, 1.0, (ny, nx))}


def _walls():
    return wl.BC(wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, -0.3, 60.0),
                 wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX),
                 wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, 0.2, 120.0),
                 wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX))


def _axis_walls():
    return wl.BC(wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX),
                 wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, -0.2, 75.0),
                 wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING, -0.1, 110.0),
                 wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX))


def _hysteresis_walls():
    """Hysteresis windows on three walls (R25): the apparent angles of random
    fields fall inside and outside them."""
    return wl.BC(wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING_HYST, -0.3, 70.0, 110.0, 40.0),
                 wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.WETTING_HYST, 0.0, 95.0, 120.0, 80.0),
                 wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.WETTING_HYST, 0.1, 60.0, 150.0, 30.0),
                 wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX))


PER = wl.BC(wl.PER, wl.PER, wl.PER, wl.PER)
AXI_PER_Y = wl.BC(wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX), wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.WETTING, 0, 70.0),
                  wl.PER, wl.PER)

# (id, nx, ny, bc, axisymmetric, streaming steps (h, f, g), gravity, seed)
CASES = [
    ("periodic_4x4", 4, 4, PER, 0, (0.5, 0.5, 0.5), 0.0, 1),
    ("walls_5x3", 5, 3, _walls(), 0, (0.5, 0.5, 0.5), -1e-3, 2),
    ("axisymmetric_4x4", 4, 4, AXI_PER_Y, 1, (0.5, 0.5, 0.5), 0.0, 3),
    ("walls_steps_4x4", 4, 4, _walls(), 0, (0.3, 0.4, 0.25), -1e-3, 4),
    ("axisymmetric_steps_5x3", 5, 3, _axis_walls(), 1, (0.35, 0.3, 0.45), -1e-3, 5),
    ("hysteresis_walls_5x4", 5, 4, _hysteresis_walls(), 0, (0.5, 0.5, 0.5), -1e-3, 8),
]
# Eq. 5-7 as printed (literal_eq7) instead of reading R1
LITERAL = [("literal_walls_5x3", 5, 3, _walls(), 0, (0.5, 0.5, 0.5), -1e-3, 6),
           ("literal_axisymmetric_4x4", 4, 4, _axis_walls(), 1, (0.5, 0.5, 0.5), 0.0, 7)]


def _setup(nx, ny, bc, axi, steps, gy, seed, literal=False):
    props = _props(literal, gy)
    dt = 0.7
    init = wl._fields(nx, ny, T=0.0, Fl=1.0, C=0.5)
    case = wl.Case("brute", nx, ny, props, bc, dt, init, axisymmetric=axi, dt_h=steps[0], dt_f=steps[1],
                   dt_g=steps[2])
    orc = oracle.OracleSolver(case)
    st = _random_state(nx, ny, seed)
    orc.set_state(st, 0.0, 0)
    model = bf.Model(nx, ny, props, bc, dt, steps=steps, axisymmetric=bool(axi))
    W = [[[bf.N(st[k][j, i]) for i in range(nx)] for j in range(ny)] for k in ("H", "p", "mx", "my", "C")]
    Fsp = [[bf.N(st["Fsp"][j, i]) for i in range(nx)] for j in range(ny)]
    return orc, model, W, Fsp


def _check_faces(orc, model, W):
    g = bf.Grid(model, W)
    faces = [(0, i, j) for j in range(model.ny) for i in range(model.nx + 1)] + \
            [(1, i, j) for j in range(model.ny + 1) for i in range(model.nx)]
    got = np.array([orc.face_flux(*f) for f in faces])
    ref = np.array([[float(x) for x in g.face_flux(*f)] for f in faces])
    scale = np.abs(ref).max(axis=0) + 1e-300
    err = (np.abs(got - ref) / scale).max(axis=0)
    assert np.all(err <= TOL), f"face flux components (F_H, F_p, F_mx, F_my, F_C, u_n) relative errors {err}"
    # the fields really vary together: the surrounding densities differ from the face density
    rho = np.array([[float(g.prim["rho"][(i, j)]) for i in range(model.nx)] for j in range(model.ny)])
    assert rho.max() - rho.min() > 0.2


def _check_step(orc, model, W, Fsp):
    ref, _ = bf.step(model, W, Fsp)
    orc.step(1)
    got = orc.state()
    for k, name in enumerate(("H", "p", "mx", "my", "C")):
        r = np.array([[float(x) for x in row] for row in ref[k]])
        scale = np.abs(r).max() + 1e-300
        err = np.abs(got[name] - r).max() / scale
        assert err <= TOL, f"{name} after one RK3 step: relative error {err:.2e}"


@pytest.mark.parametrize("cid,nx,ny,bc,axi,steps,gy,seed", CASES, ids=[c[0] for c in CASES])
def test_face_flux_matches_brute_force(cid, nx, ny, bc, axi, steps, gy, seed):
    orc, model, W, _ = _setup(nx, ny, bc, axi, steps, gy, seed)
    _check_faces(orc, model, W)


@pytest.mark.parametrize("cid,nx,ny,bc,axi,steps,gy,seed", CASES, ids=[c[0] for c in CASES])
def test_rk3_step_matches_brute_force(cid, nx, ny, bc, axi, steps, gy, seed):
    orc, model, W, Fsp = _setup(nx, ny, bc, axi, steps, gy, seed)
    _check_step(orc, model, W, Fsp)


@pytest.mark.parametrize("cid,nx,ny,bc,axi,steps,gy,seed", LITERAL, ids=[c[0] for c in LITERAL])
def test_literal_eq7_matches_brute_force(cid, nx, ny, bc, axi, steps, gy, seed):
    orc, model, W, Fsp = _setup(nx, ny, bc, axi, steps, gy, seed, literal=True)
    _check_faces(orc, model, W)
    _check_step(orc, model, W, Fsp)
