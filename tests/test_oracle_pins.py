"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins a part of the oracle to something other than the oracle
itself: a moment identity the paper states (Eq. 11, 29, 42), a closed form
that the Chapman-Enskog relations (Eq. 15, 32, 45) give for linear fields, an
exact reduction to a textbook scheme, the Neumann solution (Eq. 59-60), the
mass-conservation law behind H_f = (rho_l/rho_s) H_0 (Sec. 3.2), discrete
conservation and symmetry.  A dropped term, a wrong sign, weight or index in
the oracle breaks at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import erf, erfc

import oracle
from paper_2507_03366_gb300 import workloads as wl

CS2 = 1.0 / 3.0
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _case(nx, ny, props, bc, T, C=1.0, u=0.0, v=0.0, p=0.0, Fl=1.0, dt=0.5, name="pin"):
    init = wl._fields(nx, ny, T=T, Fl=Fl, C=C, u=u, v=v, p=p)
    return wl.Case(name, nx, ny, props, bc, dt, init)


def _props(rho=(1.0, 1.0, 1.0), mu=(0.05, 0.05, 0.05), lam=(0.1, 0.1, 0.1), cp=(1.0, 1.0, 1.0),
           L=1.0, Ts=0.0, Tl=0.0, sigma=0.0, xi=4.0, Mc=0.0, tau_g=1.0, gx=0.0, gy=0.0, zsv=0):
    ph = [wl.Phase(rho[k], mu[k], lam[k], cp[k]) for k in range(3)]
    return wl.Props(ph[0], ph[1], ph[2], L, Ts, Tl, sigma, xi, Mc, tau_g, gx, gy, zsv)


PERIODIC_BC = wl.BC(wl.PER, wl.PER, wl.PER, wl.PER)


def _walls(**kw):
    w = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)
    return wl.BC(kw.get("xlo", w), kw.get("xhi", w), kw.get("ylo", w), kw.get("yhi", w))


# ---------------------------------------------------------------------------
# 1. Moment identities of the equilibria (Eq. 11, and the textbook D2Q9
#    moments of Eq. 29 and Eq. 42 that Eq. 56 relies on).
# ---------------------------------------------------------------------------
def test_equilibria_moments():
    rng = np.random.default_rng(11)
    for _ in range(20):
        H, T, Cp, Cref = rng.uniform(-3, 3), rng.uniform(-2, 2), rng.uniform(0.3, 3), rng.uniform(0.3, 3)
        u, v, p, rho = rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-1, 1), rng.uniform(0.01, 2)
        C, muc, Qg = rng.uniform(-0.1, 1.1), rng.uniform(-1, 1), rng.uniform(0, 2)
        U = np.array([u, v])
        h = np.array([oracle.heq(a, H, T, Cp, Cref, u, v) for a in range(9)])
        f = np.array([oracle.feq(a, p, rho, u, v) for a in range(9)])
        fm = np.array([oracle.feqm(a, p, rho, u, v) for a in range(9)])
        g = np.array([oracle.geq(a, C, muc, Qg, u, v) for a in range(9)])
        E = np.stack([EX, EY])                     # 2 x 9
        EE = np.einsum("ia,ja->ija", E, E)
        I2 = np.eye(2)
        # Eq. 11 (third line with reading R17: C_ref T cs^2 I)
        np.testing.assert_allclose(h.sum(), H, atol=1e-13)
        np.testing.assert_allclose(E @ h, Cp * T * U, atol=1e-13)
        np.testing.assert_allclose(EE @ h, Cp * T * np.outer(U, U) + Cref * T * CS2 * I2, atol=1e-13)
        # Eq. 29: sum f = p, sum e f = rho cs^2 u (Eq. 32 first line), sum ee f = cs^2 (p I + rho uu)
        np.testing.assert_allclose(f.sum(), p, atol=1e-13)
        np.testing.assert_allclose(E @ f, rho * CS2 * U, atol=1e-13)
        np.testing.assert_allclose(EE @ f, CS2 * (p * I2 + rho * np.outer(U, U)), atol=1e-13)
        # Eq. 33 with R8: same moments with the face density
        np.testing.assert_allclose(EE @ fm, CS2 * (p * I2 + rho * np.outer(U, U)), atol=1e-13)
        # Eq. 42: sum g = C, sum e g = C u (Eq. 45 convective part), sum ee g = mu_c Q_g I
        np.testing.assert_allclose(g.sum(), C, atol=1e-13)
        np.testing.assert_allclose(E @ g, C * U, atol=1e-13)
        np.testing.assert_allclose(EE @ g, muc * Qg * I2, atol=1e-13)


# ---------------------------------------------------------------------------
# 2. Enthalpy closure (Eq. 5-7) at hand-computed points.
# ---------------------------------------------------------------------------
def test_enthalpy_inversion_values():
    P = _props(cp=(2.0, 1.0, 0.5), L=3.0, Ts=0.5, Tl=0.5)
    # C = 1: H_s = 2*0.5 = 1.0, H_l = 1*0.5 + 3 = 3.5
    for H, T, Fl in [(0.4, 0.2, 0.0), (2.25, 0.5, 0.5), (4.5, 1.5, 1.0), (1.0, 0.5, 0.0), (3.5, 0.5, 1.0)]:
        t, f = oracle.invert_enthalpy(P, H, 1.0)
        assert abs(t - T) < 1e-14 and abs(f - Fl) < 1e-14, (H, t, f)
    # gas (C = 0): both branches use cp_g = 0.5, latent heat uniform (R1)
    t, f = oracle.invert_enthalpy(P, 0.1, 0.0)
    assert abs(t - 0.2) < 1e-14 and f == 0.0
    t, f = oracle.invert_enthalpy(P, 4.0, 0.0)          # H_l = 0.25 + 3 = 3.25
    assert abs(t - (0.5 + 0.75 / 0.5)) < 1e-14 and f == 1.0
    # non-isothermal mushy range: T linear in F_l (Eq. 6 second branch)
    P2 = _props(cp=(1.0, 1.0, 1.0), L=2.0, Ts=-0.5, Tl=0.5)   # H_s = -0.5, H_l = 2.5
    t, f = oracle.invert_enthalpy(P2, 1.0, 1.0)
    assert abs(f - 0.5) < 1e-14 and abs(t - 0.0) < 1e-14
    # round trip of the initial-state map
    rng = np.random.default_rng(2)
    for _ in range(50):
        T, C = rng.uniform(-2, 3), rng.uniform(-0.2, 1.2)
        H = oracle.enthalpy_of(P, T, 1.0, C)
        t, _ = oracle.invert_enthalpy(P, H, C)
        assert abs(t - T) < 1e-12


def test_literal_eq7_closure_values():
    """Eq. 5-7 exactly as printed (literal_eq7) at hand-computed points, next
    to reading R1 where the two differ: cold gas counts as solid."""
    P = _props(rho=(0.9, 1.0, 0.01), cp=(2.0, 4.0, 1.0), L=3.0, Ts=0.5, Tl=0.5)
    P.literal_eq7 = 1
    # printed: H_s = C_p,s T_s = 1, H_l = C_p,l T_l + L = 5, whatever C is
    t, f = oracle.invert_enthalpy(P, 0.6, 0.0)          # gas below H_s: solid branch, T = H / C_p,s
    assert abs(t - 0.3) < 1e-15 and f == 0.0
    assert abs(oracle.mix(P, 0.0, f, 0) - 0.9) < 1e-15   # and it takes the solid density
    t, f = oracle.invert_enthalpy(P, 7.0, 0.0)          # gas above H_l: T = T_l + (H - H_l) / C_p,g
    assert abs(t - 2.5) < 1e-15 and f == 1.0
    t, f = oracle.invert_enthalpy(P, 7.0, 0.5)          # liquid branch C_p = 0.5 * 4 + 0.5 * 1 = 2.5
    assert abs(t - 1.3) < 1e-15 and f == 1.0
    t, f = oracle.invert_enthalpy(P, 3.0, 0.5)          # mushy: F_l = (3 - 1) / (5 - 1)
    assert abs(f - 0.5) < 1e-15 and abs(t - 0.5) < 1e-15
    # Eq. 7 with F_s = 0.5, C = 0.5: 0.5 * 0.9 + 0.5 * 0.5 * 1.0 + 0.5 * 0.5 * 0.01
    assert abs(oracle.mix(P, 0.5, 0.5, 0) - 0.7025) < 1e-15
    assert abs(oracle.enthalpy_of(P, 0.3, 1.0, 0.0) - 0.6) < 1e-15
    # reading R1 on the same gas cell: C_p,g in both branches, so H_s = 0.5,
    # H_l = 3.5 and H = 0.6 is mushy with F_l = 0.1 / 3; the density stays the gas's
    P.literal_eq7 = 0
    t, f = oracle.invert_enthalpy(P, 0.6, 0.0)
    assert abs(f - 0.1 / 3.0) < 1e-15 and abs(t - 0.5) < 1e-15
    assert abs(oracle.mix(P, 0.0, f, 0) - 0.01) < 1e-15


def test_property_mixing():
    P = _props(rho=(0.9, 1.0, 0.001), mu=(0.3, 0.2, 0.002), lam=(2.2, 0.56, 0.02), cp=(2.0, 4.0, 1.0))
    for which, vals in enumerate([(0.9, 1.0, 0.001), (0.3, 0.2, 0.002), (2.2, 0.56, 0.02), (2.0, 4.0, 1.0)]):
        s, l, g = vals
        assert oracle.mix(P, 1.0, 0.0, which) == pytest.approx(s, abs=1e-15)
        assert oracle.mix(P, 1.0, 1.0, which) == pytest.approx(l, abs=1e-15)
        assert oracle.mix(P, 0.0, 0.3, which) == pytest.approx(g, abs=1e-15)
        assert oracle.mix(P, 0.5, 1.0, which) == pytest.approx(0.5 * (l + g), abs=1e-15)
        assert oracle.mix(P, 1.0, 0.25, which) == pytest.approx(0.75 * s + 0.25 * l, abs=1e-15)
        assert oracle.mix(P, 1.4, 0.0, which) == pytest.approx(s, abs=1e-15)      # clamp
        assert oracle.mix(P, -0.2, 1.0, which) == pytest.approx(g, abs=1e-15)


# ---------------------------------------------------------------------------
# 3. Pure conduction: with u = 0 and uniform lambda/rho the enthalpy flux of
#    Eq. 16/53 reduces exactly to -(lambda/rho)(T_R - T_L)/dx, because
#    omega_1 + 2 omega_5 = 1/6 and tau_h - 0.5 = lambda/(rho C_ref cs^2 dt_s).
# ---------------------------------------------------------------------------
def test_pure_conduction_face_flux():
    rng = np.random.default_rng(3)
    nx, ny = 9, 7
    P = _props(rho=(1.3, 1.3, 1.3), lam=(0.26, 0.26, 0.26), cp=(0.7, 1.4, 1.0), L=2.0, Ts=0.0, Tl=0.0)
    T = rng.uniform(-1.0, 1.0, (ny, nx))
    s = oracle.OracleSolver(_case(nx, ny, P, _walls(), T=T, Fl=rng.uniform(0, 1, (ny, nx))))
    Tcell = s.fields()["T"]
    lr = 0.26 / 1.3
    for j in range(ny):
        for i in range(1, nx):
            F = s.face_flux(0, i, j)
            assert abs(F[0] + lr * (Tcell[j, i] - Tcell[j, i - 1])) < 1e-13
            assert np.all(np.abs(F[1:]) < 1e-13)
    for j in range(1, ny):
        for i in range(nx):
            F = s.face_flux(1, i, j)
            assert abs(F[0] + lr * (Tcell[j, i] - Tcell[j - 1, i])) < 1e-13


# ---------------------------------------------------------------------------
# 4. Uniform state: all non-equilibrium parts vanish and the fluxes are the
#    Euler fluxes (C_p T u, rho cs^2 u, cs^2 (rho u u + p I), C u).  The "1"
#    in Gamma_alpha of Eq. 34 would add mu cs^2/dt_s to the normal momentum
#    flux, so this also pins reading R8.
# ---------------------------------------------------------------------------
def test_uniform_state_euler_fluxes():
    P = _props(rho=(0.9, 1.0, 0.1), mu=(0.1, 0.07, 0.01), lam=(0.2, 0.1, 0.01), cp=(1.0, 1.5, 0.8),
               L=1.0, Ts=0.0, Tl=0.0, sigma=0.01, xi=4.0, Mc=0.1)
    T, C, u, v, p = 0.7, 0.6, 0.031, -0.017, 0.02
    s = oracle.OracleSolver(_case(6, 5, P, PERIODIC_BC, T=T, C=C, u=u, v=v, p=p))
    rho = oracle.mix(P, C, 1.0, 0)
    Cp = oracle.mix(P, C, 1.0, 3)
    for d, (nx_, ny_) in enumerate([(1, 0), (0, 1)]):
        un = u * nx_ + v * ny_
        expect = [Cp * T * un, rho * CS2 * un, CS2 * (rho * un * u + p * nx_),
                  CS2 * (rho * un * v + p * ny_), C * un, un]
        for (i, j) in [(0, 0), (2, 3), (4, 1)]:
            np.testing.assert_allclose(s.face_flux(d, i, j), expect, atol=2e-15, rtol=1e-12)


# ---------------------------------------------------------------------------
# 5. Linear temperature, uniform velocity: the enthalpy flux takes the closed
#    form C_p T_f u_n - (lambda/rho) dT/dn - (lambda/(rho C_ref cs^2)) C_p u_n (u.grad T),
#    the Chapman-Enskog flux of Eq. 15 plus the O(u^2) term that the
#    expansion (A-8/A-9) neglects.
# ---------------------------------------------------------------------------
def test_linear_temperature_convective_diffusive_flux():
    nx, ny = 10, 8
    lam, rho, cp, cref = 0.3, 1.2, 1.1, 1.1
    P = _props(rho=(rho,) * 3, lam=(lam,) * 3, cp=(cp,) * 3, L=1.0, Ts=5.0, Tl=5.0)  # all solid
    gxT, gyT = 0.013, -0.021
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    T = -1.0 + gxT * x[None, :] + gyT * y[:, None]
    u, v = 0.04, 0.025
    s = oracle.OracleSolver(_case(nx, ny, P, _walls(), T=T, u=u, v=v, Fl=0.0))
    for d, (nx_, ny_) in enumerate([(1, 0), (0, 1)]):
        for (i, j) in [(4, 3), (5, 4), (3, 5)]:
            xf, yf = (i, j + 0.5) if d == 0 else (i + 0.5, j)
            Tf = -1.0 + gxT * xf + gyT * yf
            un = u * nx_ + v * ny_
            dTn = gxT * nx_ + gyT * ny_
            udT = u * gxT + v * gyT
            expect = cp * Tf * un - (lam / rho) * dTn - (lam / (rho * cref * CS2)) * cp * un * udT
            F = s.face_flux(d, i, j)
            assert abs(F[0] - expect) < 1e-14, (d, i, j, F[0], expect)
            assert abs(F[5] - un) < 1e-14


# ---------------------------------------------------------------------------
# 6. Simple shear u = (0, gamma x) (and its transpose): the tangential
#    momentum flux is exactly -cs^2 mu gamma at every face (Eq. 32/36 with the
#    viscous sign of reading R3; the opposite sign of Eq. 37 gives +).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("transpose", [False, True])
def test_simple_shear_viscous_flux(transpose):
    nx, ny = 9, 9
    mu, rho = 0.04, 1.1
    P = _props(rho=(rho,) * 3, mu=(mu,) * 3, L=1.0, Ts=-5.0, Tl=-5.0)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    gam = 0.011
    X, Y = np.meshgrid(x, y)
    if transpose:
        u, v = gam * Y, 0.0 * X
    else:
        u, v = 0.0 * X, gam * X
    s = oracle.OracleSolver(_case(nx, ny, P, _walls(), T=0.0, u=u, v=v, p=0.3))
    for d in (0, 1):
        for (i, j) in [(4, 4), (5, 3), (3, 5)]:
            F = s.face_flux(d, i, j)
            tang = F[3] if d == 0 else F[2]
            assert abs(tang - (-CS2 * mu * gam)) < 1e-15, (d, i, j, tang)


# ---------------------------------------------------------------------------
# 7. Cahn-Hilliard fluxes: (a) u = 0, C varying in x only: the phase flux is
#    exactly -M_c (mu_c,R - mu_c,L) (M_c = (tau_g - 0.5) Q_g dt_s, Sec. 2.3.2);
#    (b) linear C, uniform u, mu_c = 0: F = C(x_f) u_n - (1.5 - tau_g) dt_s u_n (u.grad C).
# ---------------------------------------------------------------------------
def test_phase_field_diffusive_flux():
    nx, ny = 16, 3
    Mc, tau_g = 0.07, 1.3
    P = _props(L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.02, xi=4.0, Mc=Mc, tau_g=tau_g)
    x = np.arange(nx) + 0.5
    C = 0.5 * (1 + np.tanh(2 * (8.3 - x) / 4.0))
    s = oracle.OracleSolver(_case(nx, ny, P, wl.BC(wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX),
                                                   wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX), wl.PER, wl.PER),
                                  T=0.0, C=np.broadcast_to(C, (ny, nx))))
    muc = s.muc()
    for i in range(1, nx):
        F = s.face_flux(0, i, 1)
        assert abs(F[4] + Mc * (muc[1, i] - muc[1, i - 1])) < 1e-15


def test_phase_field_advective_flux():
    nx, ny = 10, 10
    tau_g, dts = 1.4, 0.5
    P = _props(L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.0, Mc=0.05, tau_g=tau_g)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    gC = (0.031, -0.017)
    C = 0.5 + gC[0] * (x[None, :] - 5) + gC[1] * (y[:, None] - 5)
    u, v = 0.05, -0.03
    s = oracle.OracleSolver(_case(nx, ny, P, _walls(), T=0.0, C=C, u=u, v=v))
    for d, (nx_, ny_) in enumerate([(1, 0), (0, 1)]):
        for (i, j) in [(4, 4), (5, 6)]:
            xf, yf = (i, j + 0.5) if d == 0 else (i + 0.5, j)
            Cf = 0.5 + gC[0] * (xf - 5) + gC[1] * (yf - 5)
            un = u * nx_ + v * ny_
            udC = u * gC[0] + v * gC[1]
            expect = Cf * un - (1.5 - tau_g) * dts * un * udC
            assert abs(s.face_flux(d, i, j)[4] - expect) < 1e-15


# ---------------------------------------------------------------------------
# 8. SSP-RK3 (Eq. 58) on pure conduction of a periodic sine: the discrete
#    operator is lambda/(rho cp) times the 3-point Laplacian (pin 3), so each
#    step multiplies the mode by 1 + z + z^2/2 + z^3/6, z = -4 dt alpha sin^2(pi k/N).
# ---------------------------------------------------------------------------
def test_rk3_mode_decay():
    nx, ny, k = 32, 1, 3
    lam, rho, cp, dt = 0.12, 1.0, 0.8, 1.7
    P = _props(rho=(rho,) * 3, lam=(lam,) * 3, cp=(cp, 2.0, 1.0), L=1.0, Ts=0.0, Tl=0.0)
    x = np.arange(nx)
    A, T0 = 0.3, -2.0
    T = T0 + A * np.sin(2 * np.pi * k * x / nx)
    s = oracle.OracleSolver(_case(nx, ny, P, PERIODIC_BC, T=T[None, :], Fl=0.0, dt=dt))
    nsteps = 40
    s.step(nsteps)
    z = -4.0 * dt * (lam / (rho * cp)) * np.sin(np.pi * k / nx) ** 2
    g = 1 + z + z * z / 2 + z ** 3 / 6
    expect = T0 + A * g ** nsteps * np.sin(2 * np.pi * k * x / nx)
    np.testing.assert_allclose(s.fields()["T"][0], expect, atol=1e-13)


# ---------------------------------------------------------------------------
# 9. Neumann solution (Eq. 59-60): freezing front X_i = 2 k sqrt(alpha t).
# ---------------------------------------------------------------------------


def test_neumann_one_phase_front_and_profile():
    """Liquid at T_m (Sec. 3.1 with T_0 = T_m): k e^{k^2} erf k = St/sqrt(pi).
    Front within 1% once it is 16 cells from the wall, T within 1e-2."""
    c = wl.conductive(256, 1)
    St, alpha = 0.1, 0.1
    k = wl.neumann_k(St)
    s = oracle.OracleSolver(c)
    checked = 0
    for _ in range(4):
        s.step(1600)
        d = s.diag()
        xs = 2 * k * math.sqrt(alpha * d["t"])
        if xs >= 16.0:
            assert abs(d["front_pos"] / xs - 1.0) < 0.01, (d["t"], d["front_pos"], xs)
            checked += 1
    assert checked >= 1
    x = np.arange(256) + 0.5
    t = s.diag()["t"]
    xs = 2 * k * math.sqrt(alpha * t)
    Tex = np.where(x < xs, 0.0 + (1.0 - 0.0) * erf(x / (2 * math.sqrt(alpha * t))) / erf(k), 1.0)
    assert np.max(np.abs(s.fields()["T"][0] - Tex)) < 1e-2


def _neumann_two_phase_k(St_s, St_l, ratio=1.0):
    """Root of St_s/(e^{k^2} erf k) - St_l sqrt(a_l/a_s)/(e^{k^2 a_s/a_l} erfc(k sqrt(a_s/a_l))) = k sqrt(pi)
    (Eq. 60 read with erfc in the liquid term; equal diffusivities by default)."""
    def F(k):
        return (St_s / (math.exp(k * k) * erf(k))
                - St_l * math.sqrt(ratio) / (math.exp(k * k / ratio) * erfc(k / math.sqrt(ratio))) - k * math.sqrt(math.pi))
    lo, hi = 1e-6, 3.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if F(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_neumann_two_phase_front():
    """Superheated liquid (Sec. 3.1 setup): wall T_b = 0, T_m = 1, T_0 = 1.2."""
    nx = 256
    alpha, L, Tb, Tm, T0 = 0.1, 10.0, 0.0, 1.0, 1.2
    ph = wl.Phase(1.0, 0.1, alpha, 1.0)
    P = wl.Props(ph, ph, ph, L, Tm, Tm, 0.0, 4.0, 0.0, 1.0, zero_solid_velocity=0)
    bc = wl.BC(wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.NOFLUX, Tw=Tb), wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.NOFLUX, Tw=T0),
               wl.PER, wl.PER)
    s = oracle.OracleSolver(_case(nx, 1, P, bc, T=T0, dt=2.5))
    k = _neumann_two_phase_k((Tm - Tb) / L, (T0 - Tm) / L)
    s.step(6000)
    d = s.diag()
    xs = 2 * k * math.sqrt(alpha * d["t"])
    assert xs >= 16.0
    assert abs(d["front_pos"] / xs - 1.0) < 0.01, (d["front_pos"], xs)


# ---------------------------------------------------------------------------
# 10. Three-phase Stefan (Sec. 3.2): mass conservation behind H_f = (rho_l/rho_s) H_0
#     gives an interface displacement (1 - rho_s/rho_l) x_s while the solid
#     front follows the one-phase Neumann law.
# ---------------------------------------------------------------------------
def test_three_phase_expansion_law():
    c = wl.three_phase(256, 1, St=1.0, H0=128)
    kv = 1.0 - c.props.s.rho / c.props.l.rho
    k = wl.neumann_k(1.0)
    s = oracle.OracleSolver(c)
    d0 = s.diag()
    s.step(3000)
    d = s.diag()
    xs = d["front_pos"]
    assert abs(xs / (2 * k * math.sqrt(0.1 * d["t"])) - 1.0) < 0.01
    disp = d["interface_pos"] - d0["interface_pos"]
    assert abs(disp / (kv * xs) - 1.0) < 0.02, (disp, kv * xs)


# ---------------------------------------------------------------------------
# 11. Discrete conservation of the flux form (Eq. 52).
# ---------------------------------------------------------------------------
def test_enthalpy_conserved_without_flow():
    rng = np.random.default_rng(7)
    nx, ny = 12, 10
    P = _props(lam=(0.2, 0.1, 0.1), cp=(0.8, 1.2, 1.0), L=0.5, Ts=0.0, Tl=0.0)
    T = rng.uniform(-0.5, 0.5, (ny, nx))
    s = oracle.OracleSolver(_case(nx, ny, P, wl.BC(wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX),
                                                   wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX), wl.PER, wl.PER),
                                  T=T, Fl=rng.uniform(0, 1, (ny, nx)), dt=0.8))
    E0 = s.diag()["enthalpy"]
    s.step(60)
    assert abs(s.diag()["enthalpy"] - E0) < 1e-12 * nx * ny


def test_phase_and_momentum_conserved_periodic():
    rng = np.random.default_rng(8)
    nx, ny = 16, 12
    P = _props(mu=(0.05, 0.05, 0.02), L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.0, Mc=0.1)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    C = 0.5 + 0.4 * np.sin(2 * np.pi * x[None, :] / nx) * np.cos(2 * np.pi * y[:, None] / ny)
    u = 0.02 * np.sin(2 * np.pi * y[:, None] / ny) + 0 * x[None, :]
    v = 0.015 * np.cos(2 * np.pi * x[None, :] / nx) + 0 * y[:, None]
    s = oracle.OracleSolver(_case(nx, ny, P, PERIODIC_BC, T=0.5, C=C, u=u, v=v, p=rng.uniform(-1e-3, 1e-3, (ny, nx))))
    st0 = s.state()
    s.step(40)
    st = s.state()
    for k in ("C", "mx", "my", "p"):
        assert abs(st[k].sum() - st0[k].sum()) < 1e-13 * nx * ny, k


# ---------------------------------------------------------------------------
# 12. Mirror symmetry of symmetric data.
# ---------------------------------------------------------------------------
def test_mirror_symmetry():
    nx, ny = 24, 16
    P = _props(rho=(0.9, 1.0, 0.05), mu=(0.05, 0.05, 0.01), lam=(0.1, 0.1, 0.02), L=2.0, Ts=0.0, Tl=0.0,
               sigma=0.01, xi=4.0, Mc=0.1, gy=-1e-4, zsv=1)
    cold = wl.Side(wl.DIRICHLET_T, wl.NOSLIP, wl.NOFLUX, Tw=-0.5)
    bc = _walls(ylo=cold)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    r = np.sqrt((x[None, :] - nx / 2) ** 2 + (y[:, None] - 3.0) ** 2)
    C = 0.5 * (1 + np.tanh(2 * (6.0 - r) / 4.0))
    s = oracle.OracleSolver(_case(nx, ny, P, bc, T=0.2, C=C))
    s.step(150)
    f = s.fields()
    for k in ("T", "C", "p", "v", "H"):
        a = f[k]
        scale = max(np.max(np.abs(a)), 1e-300)
        assert np.max(np.abs(a - a[:, ::-1])) <= 1e-12 * scale, k
    a = f["u"]
    assert np.max(np.abs(a + a[:, ::-1])) <= 1e-12 * max(np.max(np.abs(a)), 1e-300)
    assert np.max(np.abs(f["u"])) > 0  # the flow is not trivially zero


# ---------------------------------------------------------------------------
# 13. Flat interface (Eq. 61): the tanh profile is the exact continuum
#     equilibrium of mu_c = 2 beta C (C-1)(2C-1) - kappa lap C with
#     beta = 12 sigma/xi, kappa = 3 xi sigma/2 (reading R5); discretely mu_c
#     is a small fraction of the double-well term and the interface stays put.
# ---------------------------------------------------------------------------
def test_flat_interface_equilibrium():
    nx, ny, xi, sigma = 64, 1, 4.0, 0.01
    P = _props(rho=(1.0, 1.0, 0.01), mu=(0.01, 0.01, 0.001), L=1.0, Ts=-5.0, Tl=-5.0, sigma=sigma, xi=xi, Mc=0.1)
    x = np.arange(nx) + 0.5
    C = 0.5 * (1 + np.tanh(2 * (32.0 - x) / xi))
    bc = wl.BC(wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX), wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX), wl.PER, wl.PER)
    s = oracle.OracleSolver(_case(nx, ny, P, bc, T=0.0, C=C[None, :]))
    beta = 12 * sigma / xi
    well = np.max(np.abs(2 * beta * C * (C - 1) * (2 * C - 1)))
    assert np.max(np.abs(s.muc())) < 0.1 * well
    d0 = s.diag()
    s.step(2000)
    d = s.diag()
    assert abs(d["interface_pos"] - d0["interface_pos"]) < 0.01
    assert d["max_speed"] < 1e-4


# ---------------------------------------------------------------------------
# 14. Hydrostatics: a closed box of uniform fluid under gravity settles to
#     dp/dy = rho g_y (momentum equation, Eq. 27/38 with G = rho g).
# ---------------------------------------------------------------------------
def test_hydrostatic_pressure():
    ny, gy, rho = 16, -1e-3, 1.2
    P = _props(rho=(rho,) * 3, mu=(0.15 * rho,) * 3, L=1.0, Ts=-5.0, Tl=-5.0, gy=gy)
    wall = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)
    s = oracle.OracleSolver(_case(2, ny, P, wl.BC(wl.PER, wl.PER, wall, wall), T=0.0, dt=1.0))
    s.step(3000)
    dp = np.diff(s.fields()["p"][:, 0])
    np.testing.assert_allclose(dp, rho * gy, rtol=0.02)


# ---------------------------------------------------------------------------
# 15. Plane Poiseuille flow between no-slip walls driven by a body force:
#     u(y) = g/(2 nu) y (h - y) (textbook closed form; pins the no-slip rule
#     on the tangential velocity and the viscous flux).
# ---------------------------------------------------------------------------
def test_poiseuille_profile():
    ny, nu, g = 16, 0.1, 1e-5
    P = _props(mu=(nu,) * 3, L=1.0, Ts=-5.0, Tl=-5.0, gx=g)
    wall = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.NOFLUX)
    s = oracle.OracleSolver(_case(4, ny, P, wl.BC(wl.PER, wl.PER, wall, wall), T=0.0, dt=1.0))
    s.step(8000)
    u = s.fields()["u"][:, 1]
    y = np.arange(ny) + 0.5
    exact = g / (2 * nu) * y * (ny - y)
    assert np.max(np.abs(u - exact)) < 0.01 * exact.max()


# ---------------------------------------------------------------------------
# 16. Volume-change sources on a spatially uniform freezing state (all
#     fluxes uniform, so dW/dt = F_E): with d_t F_s = D prescribed through the
#     previous-step solid fraction (R14),
#       Eq. 27:  d(rho cs^2 u)/dt = -D (rho cs^2 u)     (F_IBM = -rho u d_t F_s)
#       Eq. 26:  dp/dt = rho cs^2 (1 - rho_s/rho_l) D
#       Eq. 40:  dC/dt = C (1 - rho_s/rho_l) d_t F_s
#     and SSP-RK3 multiplies a linear mode by 1 + z + z^2/2 + z^3/6.  In a
#     cell that is only partly condensed (C = 0.6) the rates follow the cell's
#     solid volume D = C~ d_t F_s (reading R1) for p, while the phase field
#     keeps Eq. 40's single factor C: the condensed volume grows by
#     (1 - rho_s/rho_l) times the volume that froze, no more.
# ---------------------------------------------------------------------------
def _uniform_mushy(kv, u0, dt, C=1.0):
    P = _props(rho=(1.0 - kv, 1.0, 1.0), L=2.0, Ts=0.0, Tl=0.0, zsv=0)
    s = oracle.OracleSolver(_case(4, 4, P, PERIODIC_BC, T=0.0, Fl=0.5, u=u0, dt=dt, C=C))
    st = s.state()
    st["Fsp"] = np.full_like(st["Fsp"], 0.4)           # F_s^n = 0.5, F_s^{n-1} = 0.4
    s.set_state(st, 0.0, 0)
    return s, st


def test_freezing_momentum_decay():
    dt = 0.8
    s, st0 = _uniform_mushy(0.0, 0.03, dt)
    s.step(1)
    z = -(0.1 / dt) * dt
    g = 1 + z + z * z / 2 + z ** 3 / 6
    np.testing.assert_allclose(s.state()["mx"], st0["mx"] * g, rtol=1e-13)


def test_volume_change_sources():
    dt, kv = 0.8, 0.1
    s, st0 = _uniform_mushy(kv, 0.0, dt)
    rho = oracle.mix(s.case.props, 1.0, 0.5, 0)
    D = 0.1 / dt
    s.step(1)
    st = s.state()
    np.testing.assert_allclose(st["p"], st0["p"] + dt * rho * CS2 * kv * D, rtol=1e-12, atol=1e-15)
    z = kv * D * dt
    np.testing.assert_allclose(st["C"], 1.0 * (1 + z + z * z / 2 + z ** 3 / 6), rtol=1e-13)


def test_volume_change_sources_in_a_mixed_cell():
    dt, kv, C0 = 0.8, 0.1, 0.6
    s, st0 = _uniform_mushy(kv, 0.0, dt, C=C0)
    dFs = 0.1 / dt
    s.step(1)
    st = s.state()
    # SSP-RK3 by hand on dC/dt = kv C dFs and dp/dt = rho(C) cs^2 kv C dFs
    # (F_l stays 0.5: H has no source and C_p is the same in every phase)
    src_p = lambda C: oracle.mix(s.case.props, C, 0.5, 0) * CS2 * kv * C * dFs   # noqa: E731
    src_c = lambda C: kv * C * dFs                                             # noqa: E731
    c1, p1 = C0 + dt * src_c(C0), dt * src_p(C0)
    c2 = 0.75 * C0 + 0.25 * (c1 + dt * src_c(c1))
    p2 = 0.25 * (p1 + dt * src_p(c1))
    p3 = 2.0 / 3.0 * (p2 + dt * src_p(c2))
    np.testing.assert_allclose(st["p"], st0["p"] + p3, rtol=1e-12)
    z = kv * dFs * dt
    np.testing.assert_allclose(st["C"], C0 * (1 + z + z * z / 2 + z ** 3 / 6), rtol=1e-13)


# ---------------------------------------------------------------------------
# 17. Reading R15: with zero_solid_velocity the solid does not move.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("zsv", [0, 1])
def test_rigid_solid(zsv):
    P = _props(L=1.0, Ts=0.0, Tl=0.0, zsv=zsv)
    s = oracle.OracleSolver(_case(5, 4, P, PERIODIC_BC, T=-0.5, Fl=0.0, u=0.02, v=-0.01))
    s.step(2)
    sp = s.diag()["max_speed"]
    if zsv:
        assert sp == 0.0
    else:
        assert abs(sp - math.hypot(0.02, 0.01)) < 1e-15


# ---------------------------------------------------------------------------
# 18. Wetting wall (reading R11, dC/dn = (4 cos theta/xi) C(1-C)): an interface
#     meeting the wall relaxes to the contact angle theta.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [60.0])
def test_contact_angle(theta):
    nx, ny = 32, 16
    P = _props(rho=(1.0, 1.0, 0.1), mu=(0.1, 0.1, 0.01), L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.01, xi=4.0, Mc=0.2)
    wet = wl.Side(wl.ADIABATIC, wl.NOSLIP, wl.WETTING, theta_deg=theta)
    x = np.arange(nx) + 0.5
    C = 0.5 * (1 + np.tanh(2 * (nx / 2 - x) / 4.0))
    s = oracle.OracleSolver(_case(nx, ny, P, _walls(ylo=wet), T=0.0, C=np.broadcast_to(C, (ny, nx)), dt=1.0))
    s.step(2000)
    Cf = s.fields()["C"]
    xs = []
    for j in range(1, 4):        # C = 0.5 contour in the rows next to the wall
        row = Cf[j]
        i = int(np.where(row < 0.5)[0][0])
        xs.append(i - 0.5 + (row[i - 1] - 0.5) / (row[i - 1] - row[i]))
    slope = np.polyfit(np.arange(1, 4) + 0.5, xs, 1)[0]   # dx/dy of the interface, liquid at x < x_c
    measured = math.degrees(math.acos(-slope / math.sqrt(1 + slope * slope)))
    assert abs(measured - theta) < 10.0, measured
