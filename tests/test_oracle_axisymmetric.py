"""Pins of the oracle's axisymmetric (r, z) form against closed forms.

In an axisymmetric run x is the radius r (the axis at x = 0, a symmetric,
adiabatic, no-flux side) and y the axial coordinate z.  The finite-volume
balance of Eq. 52 then takes per-radian volumes r_i and face areas r_f, the
radial momentum gains the hoop term cs^2 (p - 2 mu u_r / r) / r, the
chemical potential takes the axisymmetric Laplacian, and the face pressure
sees the full divergence (reading R24).  Each pin below is a textbook result
for a cylinder or a body of revolution that the planar scheme gets wrong:

  * the Laplacian of r^2 is 4 (planar: 2), exactly on the lattice;
  * a fluid at rest under a uniform pressure feels no force;
  * the stagnation flow u = (a r, -2 a z) is divergence-free and free of
    viscous force, so the part of the residual linear in a vanishes;
  * the uniform radial expansion u = (a r, 0) feels no force (its stresses
    are uniform and isotropic in (r, theta)) and compresses at div u = 2a;
  * a drop of revolution at rest in a gas 1000 times lighter stays at rest
    (no mode of the linearised scheme grows);
  * heat conduction in a cylinder decays as J0(k r) exp(-alpha k^2 t) with
    k R = 2.4048 (the first zero of J0);
  * steady pipe flow is Hagen-Poiseuille, u_z = g (R^2 - r^2) / (4 nu);
  * a diffuse sphere's volume of revolution and its Gibbs-Thomson
    chemical potential 2 sigma / R;
  * the phase volume integral of r C is conserved while a liquid column
    relaxes.
"""
import math

import numpy as np
from scipy.special import j0

import oracle
from paper_2507_03366_gb300 import workloads as wl

from test_oracle_pins import _case, _props

CS2 = 1.0 / 3.0
J0_ZERO = 2.404825557695773
AXIS = wl.Side(wl.ADIABATIC, wl.SYMMETRY, wl.NOFLUX)
WALL = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)
OUTLET = wl.Side(wl.ADIABATIC, wl.OUTLET, wl.NOFLUX)


def _axi_case(nx, ny, props, bc, axisymmetric=1, **kw):
    c = _case(nx, ny, props, bc, **kw)
    c.axisymmetric = axisymmetric
    return c


def _sphere(nx, ny, R, xi):
    r = np.arange(nx) + 0.5
    z = np.arange(ny) + 0.5 - ny / 2
    d = np.sqrt(r[None, :] ** 2 + z[:, None] ** 2)
    return d, 0.5 * (1 + np.tanh(2 * (R - d) / xi))


# ---------------------------------------------------------------------------
# 1. The axisymmetric Laplacian (1/r) d/dr (r dC/dr) of C = eps r^2 is 4 eps,
#    exactly for the conservative three-point form on faces r = i, i + 1.
#    mu_c = 2 beta C (C - 1)(2C - 1) - 4 kappa eps (Sec. 2.3.1, reading R5).
# ---------------------------------------------------------------------------
def test_laplacian_of_r_squared():
    nx, ny, sigma, xi, eps = 16, 4, 0.01, 4.0, 1.0 / 256
    P = _props(sigma=sigma, xi=xi, Mc=0.1, Ts=-5.0, Tl=-5.0)
    r = np.arange(nx) + 0.5
    C = np.broadcast_to(eps * r ** 2, (ny, nx))
    s = oracle.OracleSolver(_axi_case(nx, ny, P, wl.BC(AXIS, WALL, wl.PER, wl.PER), T=0.0, C=C))
    beta, kappa = 12 * sigma / xi, 1.5 * xi * sigma
    c = C[0]
    expect = 2 * beta * c * (c - 1) * (2 * c - 1) - 4.0 * kappa * eps
    # the last column sees the zero-gradient ghost of the outer wall
    np.testing.assert_allclose(s.muc()[:, :-1], np.broadcast_to(expect[:-1], (ny, nx - 1)), rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# 2. Uniform pressure at rest: the pressure on the radial faces (areas r_f)
#    is balanced by the hoop term cs^2 p / r_i, so every residual is zero.
# ---------------------------------------------------------------------------
def test_uniform_pressure_is_force_free():
    nx, ny, p0 = 12, 4, 0.3
    P = _props(Ts=-5.0, Tl=-5.0)
    s = oracle.OracleSolver(_axi_case(nx, ny, P, wl.BC(AXIS, WALL, wl.PER, wl.PER), T=0.0, C=1.0, p=p0))
    R = s.residual()
    assert np.max(np.abs(R)) < 1e-14 * p0


# ---------------------------------------------------------------------------
# 3. Stagnation flow u_r = a r, u_z = -2 a z: (1/r) d(r u_r)/dr + du_z/dz = 0
#    and the viscous force of the axisymmetric Navier-Stokes equations,
#    mu (lap u_r - u_r / r^2, lap u_z), vanishes.  All fields are linear, so
#    the reconstruction (Eq. 54) is exact and the part of the residual linear
#    in a must vanish to rounding in every equation: the pressure equation
#    (r-weighted mass flux), the enthalpy equation (C_p T div u source), the
#    radial momentum (hoop viscous stress and the streamed pressure source of
#    reading R24) and the axial momentum.
# ---------------------------------------------------------------------------
def test_stagnation_flow_residual_linear_part_vanishes():
    nx, ny, a = 16, 16, 1e-6
    P = _props(mu=(0.1,) * 3, Ts=-5.0, Tl=-5.0)
    r = np.arange(nx) + 0.5
    z = np.arange(ny) + 0.5 - ny / 2
    Rr, Zz = np.meshgrid(r, z)
    res = []
    for sgn in (1.0, -1.0):
        s = oracle.OracleSolver(_axi_case(nx, ny, P, wl.BC(AXIS, OUTLET, OUTLET, OUTLET), T=1.0, C=1.0,
                                          u=sgn * a * Rr, v=-2 * sgn * a * Zz))
        res.append(s.residual())
    lin = (res[0] - res[1]) / (2 * a)
    inner = (slice(3, ny - 3), slice(0, nx - 3))     # away from the outlet ghosts
    for k in range(5):
        assert np.max(np.abs(lin[k][inner])) < 1e-8, k


# ---------------------------------------------------------------------------
# 3b. Uniform radial expansion u_r = a r, u_z = 0: div u = 2a, the viscous
#     stress 2 mu a is the same in r and theta and the isotropic part of the
#     face fluxes (the pressure advanced over dt_s) is uniform, so the
#     radial momentum feels no force: its residual has no part linear in a.
#     The pressure and phase equations compress at -rho cs^2 2a and -C 2a.
# ---------------------------------------------------------------------------
def test_uniform_radial_expansion():
    nx, ny, a = 16, 4, 1e-6
    P = _props(mu=(0.1,) * 3, Ts=-5.0, Tl=-5.0)
    r = np.arange(nx) + 0.5
    res = []
    for sgn in (1.0, -1.0):
        s = oracle.OracleSolver(_axi_case(nx, ny, P, wl.BC(AXIS, OUTLET, wl.PER, wl.PER), T=1.0, C=1.0,
                                          u=np.broadcast_to(sgn * a * r, (ny, nx))))
        res.append(s.residual())
    lin = (res[0] - res[1]) / (2 * a)
    inner = (slice(None), slice(0, nx - 3))
    for k in (0, 2, 3):
        assert np.max(np.abs(lin[k][inner])) < 1e-8, k
    np.testing.assert_allclose(lin[1][inner], -2.0 * CS2, atol=1e-8)
    np.testing.assert_allclose(lin[4][inner], -2.0, atol=1e-8)


# ---------------------------------------------------------------------------
# 3c. A drop of revolution at rest in a gas 1000 times lighter (the impact
#     problem's fluids) stays at rest up to the diffuse interface's small
#     parasitic currents: no mode of the scheme grows near the axis.
# ---------------------------------------------------------------------------
def test_resting_drop_in_light_gas_stays_bounded():
    side, R = 24, 6.0
    P = wl.Props(wl.Phase(1.0, 0.0032, 0.05, 1.0), wl.Phase(1.0, 0.0032, 0.05, 1.0), wl.Phase(1e-3, 3.2e-5, 5e-5, 1.0),
                 L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.0016, xi=4.0, Mc=0.1, tau_g=1.0, gx=0.0, gy=0.0,
                 zero_solid_velocity=0)
    r = np.arange(side) + 0.5
    z = np.arange(side) + 0.5 - side / 2
    C = 0.5 * (1 + np.tanh(2 * (R - np.sqrt(r[None, :] ** 2 + z[:, None] ** 2)) / 4.0))
    s = oracle.OracleSolver(_axi_case(side, side, P, wl.BC(AXIS, WALL, WALL, WALL), T=0.0, C=C))
    for _ in range(8):
        s.step(50)
        assert s.diag()["max_speed"] < 0.01


# ---------------------------------------------------------------------------
# 4. Conduction in a cylinder of radius R with T = 0 on r = R: the first mode
#    J0(k r), k = 2.4048 / R, decays at the rate alpha k^2 (Carslaw & Jaeger).
#    The planar scheme would pick cos(pi r / 2R) and the rate alpha pi^2/4R^2.
# ---------------------------------------------------------------------------
def test_cylinder_conduction_mode_decay():
    R, lam, n = 24, 0.1, 500
    P = _props(lam=(lam,) * 3, Ts=-5.0, Tl=-5.0)
    k = J0_ZERO / R
    r = np.arange(R) + 0.5
    T0 = j0(k * r)
    cold = wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.NOFLUX, Tw=0.0)
    s = oracle.OracleSolver(_axi_case(R, 2, P, wl.BC(AXIS, cold, wl.PER, wl.PER), T=np.broadcast_to(T0, (2, R)),
                                      dt=1.0))
    s.step(n)
    T = s.fields()["T"][0]
    amp = T @ T0 / (T0 @ T0)
    rate = -math.log(amp) / n
    assert abs(rate / (lam * k * k) - 1.0) < 0.005
    assert np.max(np.abs(T - amp * T0)) < 1e-3      # the shape stays J0


# ---------------------------------------------------------------------------
# 5. Hagen-Poiseuille: axial flow in a pipe of radius R driven by a body force
#    g along z settles to u_z = g (R^2 - r^2) / (4 nu) (planar channel: /2).
# ---------------------------------------------------------------------------
def test_hagen_poiseuille_profile():
    R, nu, g = 8, 0.1, 1e-5
    P = _props(mu=(nu,) * 3, Ts=-5.0, Tl=-5.0, gy=g)
    s = oracle.OracleSolver(_axi_case(R, 2, P, wl.BC(AXIS, WALL, wl.PER, wl.PER), T=0.0, dt=1.0))
    s.step(6000)
    r = np.arange(R) + 0.5
    exact = g * (R * R - r * r) / (4 * nu)
    assert np.max(np.abs(s.fields()["v"][0] - exact)) < 0.01 * exact.max()


# ---------------------------------------------------------------------------
# 6. A diffuse sphere C = (1 + tanh(2 (R - d) / xi)) / 2 on the axis:
#    2 pi sum r_i C_i = 4/3 pi R^3 + pi^3 R xi^2 / 12 (the tanh correction of
#    the volume of revolution, from the integral of x / (1 + e^(4x/xi))),
#    and the C'-weighted mean of mu_c over the interface is the
#    Gibbs-Thomson value 2 sigma / R (the Laplace jump of a sphere).  A flat
#    solid layer of height h across the cylinder gives front_pos = h.
# ---------------------------------------------------------------------------
def test_sphere_volume_and_gibbs_thomson():
    nx, ny, R, sigma, xi = 40, 80, 20.0, 0.01, 4.0
    P = _props(sigma=sigma, xi=xi, Mc=0.1, Ts=-5.0, Tl=-5.0)
    d, C = _sphere(nx, ny, R, xi)
    s = oracle.OracleSolver(_axi_case(nx, ny, P, wl.BC(AXIS, WALL, WALL, WALL), T=0.0, C=C))
    vol = 2 * math.pi * s.diag()["phase_vol"]
    exact = 4.0 / 3.0 * math.pi * R ** 3 + math.pi ** 3 * R * xi ** 2 / 12.0
    assert abs(vol / exact - 1.0) < 1e-3
    w = 1.0 / np.cosh(2 * (R - d) / xi) ** 2
    mu_gt = float((s.muc() * w).sum() / w.sum())
    assert abs(mu_gt / (2 * sigma / R) - 1.0) < 0.03

    h, nx2, ny2 = 5, 12, 10
    P2 = _props(Ts=0.0, Tl=0.0)
    T = np.where((np.arange(ny2) < h)[:, None], -1.0, 1.0) * np.ones((ny2, nx2))
    s2 = oracle.OracleSolver(_axi_case(nx2, ny2, P2, wl.BC(AXIS, WALL, WALL, WALL), T=T, C=1.0))
    assert abs(s2.diag()["front_pos"] - h) < 1e-12


# ---------------------------------------------------------------------------
# 7. Conservation: with no phase change the phase equation is a pure flux
#    divergence with r-weighted faces, so sum r_i C_i is constant to rounding
#    while a perturbed liquid column (periodic in z, clear of the outer wall)
#    relaxes; the plain sum of C is not.
# ---------------------------------------------------------------------------
def test_liquid_column_phase_volume_conserved():
    nx, ny, xi = 32, 32, 4.0
    P = _props(rho=(1.0, 1.0, 0.1), mu=(0.1, 0.1, 0.01), sigma=0.01, xi=xi, Mc=0.1, Ts=-5.0, Tl=-5.0)
    r = np.arange(nx) + 0.5
    z = np.arange(ny) + 0.5
    Rz = 8.0 + 1.5 * np.cos(2 * math.pi * z / ny)
    C = 0.5 * (1 + np.tanh(2 * (Rz[:, None] - r[None, :]) / xi))
    s = oracle.OracleSolver(_axi_case(nx, ny, P, wl.BC(AXIS, WALL, wl.PER, wl.PER), T=0.0, C=C, dt=1.0))
    v0 = s.diag()["phase_vol"]
    c0 = s.state()["C"].sum()
    s.step(200)
    assert s.diag()["max_speed"] > 1e-5          # the column moved
    assert abs(s.diag()["phase_vol"] / v0 - 1.0) < 1e-12
    assert abs(s.state()["C"].sum() / c0 - 1.0) > 1e-6
