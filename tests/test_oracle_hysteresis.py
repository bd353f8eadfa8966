"""Pins of the oracle's contact-angle hysteresis (reading R25).

Sec. 3.5 gives advancing, receding and equilibrium contact angles for the
impact cases but no model for them.  The model taken (R25): the wetting rule
of R11 uses the apparent angle read from the wall layers, clamped to
[theta_rec, theta_adv].  What fixes its behaviour:

  * with theta_adv = theta_rec = theta it is the static wetting rule of R11,
    bit for bit;
  * inside the window the contact line is pinned: an interface that meets
    the wall at 75 deg keeps that angle, where the no-flux wall (90 deg)
    turns it to 90;
  * outside the window the nearer limit acts like a static contact angle:
    a 90 deg interface with the window [30, 60] ends where the static
    60 deg wall puts it, with [110, 150] where the static 110 deg wall does.
"""
import math

import numpy as np

import oracle
from paper_2507_03366_gb300 import workloads as wl

from test_oracle_pins import _case, _props, _walls

NX, NY = 32, 16


def _props_wet():
    return _props(rho=(1.0, 1.0, 0.1), mu=(0.1, 0.1, 0.01), L=1.0, Ts=-5.0, Tl=-5.0, sigma=0.01, xi=4.0, Mc=0.2)


def _interface(theta0):
    """Liquid (C = 1) at small x; a tanh interface crossing the wall y = 0 at
    x = NX/2 under the angle theta0 measured inside the liquid."""
    x = np.arange(NX) + 0.5
    y = np.arange(NY) + 0.5
    s = -1.0 / math.tan(math.radians(theta0))          # dx/dy of the interface line
    d = (x[None, :] - NX / 2 - s * y[:, None]) / math.sqrt(1 + s * s)
    return 0.5 * (1 + np.tanh(-2 * d / 4.0))


def _angle_and_contact(C):
    """Angle inside the liquid from the C = 0.5 contour of rows 1-3 and the
    contour position in the wall row."""
    xs = []
    for j in range(4):
        row = C[j]
        i = int(np.where(row < 0.5)[0][0])
        xs.append(i - 0.5 + (row[i - 1] - 0.5) / (row[i - 1] - row[i]))
    slope = np.polyfit(np.arange(1, 4) + 0.5, xs[1:], 1)[0]
    return math.degrees(math.acos(-slope / math.sqrt(1 + slope * slope))), xs[0]


def _run(side, theta0=90.0, steps=1500):
    s = oracle.OracleSolver(_case(NX, NY, _props_wet(), _walls(ylo=side), T=0.0, C=_interface(theta0), dt=1.0))
    s.step(steps)
    return s.fields()["C"]


def _side(phase, theta, adv=None, rec=None):
    return wl.Side(wl.ADIABATIC, wl.NOSLIP, phase, theta_deg=theta, theta_adv_deg=adv, theta_rec_deg=rec)


def test_hysteresis_without_window_is_static_wetting():
    a = _run(_side(wl.WETTING, 60.0), steps=400)
    b = _run(_side(wl.WETTING_HYST, 60.0, 60.0, 60.0), steps=400)
    assert np.array_equal(a, b)


def test_contact_line_pinned_inside_window():
    start = _angle_and_contact(_interface(75.0))
    pinned = _angle_and_contact(_run(_side(wl.WETTING_HYST, 90.0, 120.0, 60.0), theta0=75.0, steps=2000))
    free = _angle_and_contact(_run(_side(wl.NOFLUX, 90.0), theta0=75.0, steps=2000))
    assert abs(free[0] - 90.0) < 2.0                  # without hysteresis the angle turns to 90
    assert abs(pinned[0] - start[0]) < 6.0            # with it, it stays near 75
    assert abs(pinned[1] - start[1]) < 1.2 < abs(free[1] - start[1])


def test_limits_act_as_static_angles_outside_window():
    for window, theta in (((60.0, 30.0), 60.0), ((150.0, 110.0), 110.0)):
        adv, rec = window
        hyst = _angle_and_contact(_run(_side(wl.WETTING_HYST, 0.5 * (adv + rec), adv, rec)))
        static = _angle_and_contact(_run(_side(wl.WETTING, theta)))
        assert abs(hyst[0] - static[0]) < 0.05 and abs(hyst[1] - static[1]) < 0.01, (window, hyst, static)
        assert abs(static[0] - theta) < 10.0
