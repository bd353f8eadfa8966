"""Pins of the oracle's per-distribution streaming steps (reading R26).

Each of the three distributions (h: enthalpy, f: flow, g: phase field)
takes its surrounding points at x_f - e_alpha dt with its own streaming step,
and its relaxation time follows from the same step (tau - 1/2 = transport
coefficient / (cs^2 dt) with the field's factors).  The Chapman-Enskog
fluxes of Eq. 15, 32 and 45 do not depend on dt, so the closed forms of the
linear-field pins hold for every choice; the phase field's advective O(u^2)
term is the one that scales with dt_g.  For a field that is not linear the
u = 0 fluxes are the hand-expanded sums: with the surrounding points inside
the two cells, each side contributes its reconstruction at distance
1/2 - dt from its centre, f' = f + (1/2 - dt)(f_next - f_prev)/2, and the
D2Q9 sums reduce to (transport coefficient) (f'_L - f'_R) / (2 dt), which is
the textbook central flux at dt = 1/2.  Every pin runs with the three steps
all different, so a step taken from the wrong distribution fails it.
"""
import numpy as np
import pytest

import oracle
from paper_2507_03366_gb300 import workloads as wl

from test_oracle_pins import CS2, PERIODIC_BC, _case, _props, _walls

STEPS = [(0.2, 0.35, 0.45), (0.45, 0.2, 0.35), (0.35, 0.45, 0.2)]


def _with_steps(case, steps):
    case.dt_h, case.dt_f, case.dt_g = steps
    return case


def test_equal_steps_are_the_single_streaming_step():
    a = wl.droplet(32, theta_deg=70.0, St=0.3)
    a.dt_stream = 0.4
    b = _with_steps(wl.droplet(32, theta_deg=70.0, St=0.3), (0.4, 0.4, 0.4))
    sa, sb = oracle.OracleSolver(a), oracle.OracleSolver(b)
    sa.step(30)
    sb.step(30)
    for k in ("H", "p", "mx", "my", "C"):
        assert np.array_equal(sa.state()[k], sb.state()[k]), k


def _side_values(f, i, a):
    """Reconstructions of row f at distance a from the centres of cells i-1
    (towards +x) and i (towards -x), central slopes (R6)."""
    return f[i - 1] + a * 0.5 * (f[i] - f[i - 2]), f[i] - a * 0.5 * (f[i + 1] - f[i - 1])


@pytest.mark.parametrize("steps", STEPS)
def test_conduction_flux_hand_expanded(steps):
    """u = 0, random T: F_h = (lambda/rho) (T'_L - T'_R) / (2 dt_h)."""
    rng = np.random.default_rng(5)
    nx, ny = 9, 6
    P = _props(rho=(1.3,) * 3, lam=(0.26,) * 3, cp=(0.7, 1.4, 1.0), L=2.0, Ts=0.0, Tl=0.0)
    T = rng.uniform(-1.0, 1.0, (ny, nx))
    s = oracle.OracleSolver(_with_steps(_case(nx, ny, P, _walls(), T=T, Fl=rng.uniform(0, 1, (ny, nx))), steps))
    Tc = s.fields()["T"]
    dth = steps[0]
    for j in range(ny):
        for i in range(2, nx - 1):
            tl, tr = _side_values(Tc[j], i, 0.5 - dth)
            assert abs(s.face_flux(0, i, j)[0] - 0.2 * (tl - tr) / (2 * dth)) < 1e-13


@pytest.mark.parametrize("steps", STEPS)
def test_linear_temperature_flux_independent_of_steps(steps):
    """Linear T, uniform u: C_p T_f u_n - (lambda/rho) dT/dn - (lambda/(rho C_ref cs^2)) C_p u_n (u.grad T),
    where (tau_h - 1/2) dt_h = lambda/(rho C_ref cs^2) whatever dt_h is."""
    nx, ny = 10, 8
    lam, rho, cp = 0.3, 1.2, 1.1
    P = _props(rho=(rho,) * 3, lam=(lam,) * 3, cp=(cp,) * 3, L=1.0, Ts=5.0, Tl=5.0)
    gxT, gyT = 0.013, -0.021
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    T = -1.0 + gxT * x[None, :] + gyT * y[:, None]
    u, v = 0.04, 0.025
    s = oracle.OracleSolver(_with_steps(_case(nx, ny, P, _walls(), T=T, u=u, v=v, Fl=0.0), steps))
    for d, (nx_, ny_) in enumerate([(1, 0), (0, 1)]):
        i, j = 4, 3
        xf, yf = (i, j + 0.5) if d == 0 else (i + 0.5, j)
        Tf = -1.0 + gxT * xf + gyT * yf
        un = u * nx_ + v * ny_
        expect = cp * Tf * un - (lam / rho) * (gxT * nx_ + gyT * ny_) - (lam / (rho * cp * CS2)) * cp * un * (
            u * gxT + v * gyT)
        assert abs(s.face_flux(d, i, j)[0] - expect) < 1e-14


@pytest.mark.parametrize("steps", STEPS)
def test_shear_flux_independent_of_steps(steps):
    """u = (0, gamma x): the tangential momentum flux is -cs^2 mu gamma for any dt_f."""
    nx, ny, mu, gam = 9, 9, 0.04, 0.011
    P = _props(rho=(1.1,) * 3, mu=(mu,) * 3, L=1.0, Ts=-5.0, Tl=-5.0)
    X, _ = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    s = oracle.OracleSolver(_with_steps(_case(nx, ny, P, _walls(), T=0.0, u=0.0 * X, v=gam * X, p=0.3), steps))
    for (i, j) in [(4, 4), (5, 3)]:
        assert abs(s.face_flux(0, i, j)[3] + CS2 * mu * gam) < 1e-15


@pytest.mark.parametrize("steps", STEPS)
def test_phase_field_fluxes_with_steps(steps):
    """(a) u = 0: M_c (mu'_L - mu'_R) / (2 dt_g) (Q_g = M_c / ((tau_g - 1/2) dt_g));
    (b) linear C, uniform u: C_f u_n - (3/2 - tau_g) dt_g u_n (u.grad C)."""
    Mc, tau_g = 0.07, 1.3
    nx, ny = 16, 3
    P = _props(L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.02, xi=4.0, Mc=Mc, tau_g=tau_g)
    x = np.arange(nx) + 0.5
    C = 0.5 * (1 + np.tanh(2 * (8.3 - x) / 4.0))
    w = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)
    s = oracle.OracleSolver(_with_steps(_case(nx, ny, P, wl.BC(w, w, wl.PER, wl.PER), T=0.0,
                                              C=np.broadcast_to(C, (ny, nx))), steps))
    muc = s.muc()
    dtg = steps[2]
    for i in range(2, nx - 1):
        ml, mr = _side_values(muc[1], i, 0.5 - dtg)
        assert abs(s.face_flux(0, i, 1)[4] - Mc * (ml - mr) / (2 * dtg)) < 1e-15

    P = _props(L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.0, Mc=0.05, tau_g=1.4)
    nx = ny = 10
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    gC = (0.031, -0.017)
    C = 0.5 + gC[0] * (x[None, :] - 5) + gC[1] * (y[:, None] - 5)
    u, v = 0.05, -0.03
    s = oracle.OracleSolver(_with_steps(_case(nx, ny, P, _walls(), T=0.0, C=C, u=u, v=v), steps))
    for d, (nx_, ny_) in enumerate([(1, 0), (0, 1)]):
        xf, yf = (4, 4.5) if d == 0 else (4.5, 4)
        Cf = 0.5 + gC[0] * (xf - 5) + gC[1] * (yf - 5)
        un = u * nx_ + v * ny_
        expect = Cf * un - (1.5 - 1.4) * steps[2] * un * (u * gC[0] + v * gC[1])
        assert abs(s.face_flux(d, 4, 4)[4] - expect) < 1e-15


@pytest.mark.parametrize("steps", STEPS)
def test_uniform_state_euler_fluxes_with_steps(steps):
    P = _props(rho=(0.9, 1.0, 0.1), mu=(0.1, 0.07, 0.01), lam=(0.2, 0.1, 0.01), cp=(1.0, 1.5, 0.8),
               L=1.0, Ts=0.0, Tl=0.0, sigma=0.01, xi=4.0, Mc=0.1)
    T, C, u, v, p = 0.7, 0.6, 0.031, -0.017, 0.02
    s = oracle.OracleSolver(_with_steps(_case(6, 5, P, PERIODIC_BC, T=T, C=C, u=u, v=v, p=p), steps))
    rho, Cp = oracle.mix(P, C, 1.0, 0), oracle.mix(P, C, 1.0, 3)
    for d, (nx_, ny_) in enumerate([(1, 0), (0, 1)]):
        un = u * nx_ + v * ny_
        expect = [Cp * T * un, rho * CS2 * un, CS2 * (rho * un * u + p * nx_), CS2 * (rho * un * v + p * ny_),
                  C * un, un]
        np.testing.assert_allclose(s.face_flux(d, 2, 3), expect, atol=2e-15, rtol=1e-12)


@pytest.mark.parametrize("steps", STEPS)
def test_axisymmetric_stagnation_flow_with_steps(steps):
    """The R24 source and the advanced hoop pressure stream over dt_f: the
    stagnation flow (a r, -2 a z) still leaves no linear residual."""
    nx, ny, a = 16, 16, 1e-6
    P = _props(mu=(0.1,) * 3, Ts=-5.0, Tl=-5.0)
    r = np.arange(nx) + 0.5
    z = np.arange(ny) + 0.5 - ny / 2
    Rr, Zz = np.meshgrid(r, z)
    axis = wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX)
    out = wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX)
    res = []
    for sgn in (1.0, -1.0):
        c = _with_steps(_case(nx, ny, P, wl.BC(axis, out, out, out), T=1.0, C=1.0, u=sgn * a * Rr,
                              v=-2 * sgn * a * Zz), steps)
        c.axisymmetric = 1
        res.append(oracle.OracleSolver(c).residual())
    lin = (res[0] - res[1]) / (2 * a)
    for k in range(5):
        assert np.max(np.abs(lin[k][3:ny - 3, :nx - 3])) < 1e-8, k


@pytest.mark.parametrize("steps", STEPS)
def test_axisymmetric_radial_expansion_with_steps(steps):
    """Uniform radial expansion (a r, 0): the isotropic stress of the faces
    and of the hoop term are both advanced over dt_f, so the radial momentum
    still has no linear residual."""
    nx, ny, a = 16, 4, 1e-6
    P = _props(mu=(0.1,) * 3, Ts=-5.0, Tl=-5.0)
    r = np.arange(nx) + 0.5
    axis = wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX)
    out = wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX)
    res = []
    for sgn in (1.0, -1.0):
        c = _with_steps(_case(nx, ny, P, wl.BC(axis, out, wl.PER, wl.PER), T=1.0, C=1.0,
                              u=np.broadcast_to(sgn * a * r, (ny, nx))), steps)
        c.axisymmetric = 1
        res.append(oracle.OracleSolver(c).residual())
    lin = (res[0] - res[1]) / (2 * a)
    assert np.max(np.abs(lin[2][:, :nx - 3])) < 1e-8
