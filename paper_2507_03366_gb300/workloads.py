"""Seeded synthetic workloads for the EULBFS solidification step.

This module only describes problems: grid sizes, material properties,
boundary conditions, time steps and initial primitive fields (T, F_l, C, u,
v, p).  It holds none of the method's arithmetic -- no enthalpy inversion,
no equilibria, no fluxes -- so that both the CUDA library binding and the CPU
oracle can take their inputs from it without sharing any of the computation.

Everything is in lattice units (dx = 1, lattice speed c = 1, cs^2 = 1/3,
streaming step 0.5).  The problems stand in for the paper's benchmark cases
(arXiv 2507.03366, Sec. 3.1-3.5); no data set is involved.  Initial phase
fields follow Eq. 61 (flat interface) and Eq. 62 read as a circle (R20).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Dict, List

import numpy as np

# Boundary-condition kinds.  The numeric values are the ones of the C ABI.
PERIODIC, DIRICHLET_T, ADIABATIC, NOSLIP, SYMMETRY, OUTLET, NOFLUX, WETTING, WETTING_HYST = range(9)


@dataclass
class Phase:
    rho: float
    mu: float
    lam: float
    cp: float


@dataclass
class Props:
    s: Phase
    l: Phase
    g: Phase
    L: float
    Ts: float
    Tl: float
    sigma: float
    xi: float
    Mc: float
    tau_g: float = 1.0
    gx: float = 0.0
    gy: float = 0.0
    zero_solid_velocity: int = 1
    literal_eq7: int = 0       # 1: Eq. 5-7 exactly as printed instead of reading R1


@dataclass
class Side:
    thermal: int
    flow: int
    phase: int
    Tw: float = 0.0
    theta_deg: float = 90.0
    theta_adv_deg: float | None = None     # WETTING_HYST: advancing and receding limits
    theta_rec_deg: float | None = None     # (None: the equilibrium angle)

    def __post_init__(self):
        if self.theta_adv_deg is None:
            self.theta_adv_deg = self.theta_deg
        if self.theta_rec_deg is None:
            self.theta_rec_deg = self.theta_deg


@dataclass
class BC:
    xlo: Side
    xhi: Side
    ylo: Side
    yhi: Side


@dataclass
class Case:
    """One domain: grid, properties, boundaries, time step and initial fields.

    ``init`` maps "T", "Fl", "C", "u", "v", "p" to float64 arrays of shape
    (ny, nx) (row-major, x fastest when flattened)."""

    name: str
    nx: int
    ny: int
    props: Props
    bc: BC
    dt: float
    init: Dict[str, np.ndarray] = field(repr=False)
    dt_stream: float = 0.5
    axisymmetric: int = 0      # 1: x is the radius r (axis at x = 0), y the axial z
    dt_h: float = 0.0          # streaming steps of the h, f, g distributions (0: dt_stream)
    dt_f: float = 0.0
    dt_g: float = 0.0

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def crop(self, nx: int, ny: int, name: str | None = None) -> "Case":
        """Lower-left nx x ny window of this case (same physics, smaller grid)."""
        init = {k: np.ascontiguousarray(v[:ny, :nx]) for k, v in self.init.items()}
        return replace(self, name=name or f"{self.name}_crop{nx}x{ny}", nx=nx, ny=ny, init=init)


PER = Side(PERIODIC, PERIODIC, PERIODIC)


def _wall(thermal=ADIABATIC, flow=NOSLIP, phase=NOFLUX, Tw=0.0, theta=90.0) -> Side:
    return Side(thermal, flow, phase, Tw, theta)


def _fields(nx: int, ny: int, T, Fl, C, u=None, v=None, p=None) -> Dict[str, np.ndarray]:
    z = np.zeros((ny, nx))

    def full(a):
        return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (ny, nx)).copy())

    return {"T": full(T), "Fl": full(Fl), "C": full(C),
            "u": full(z if u is None else u), "v": full(z if v is None else v),
            "p": full(z if p is None else p)}


def neumann_k(St: float) -> float:
    """Root of k exp(k^2) erf(k) = St / sqrt(pi): one-phase limit of Eq. 60
    (liquid initially at the melting temperature)."""
    lo, hi = 1e-9, 5.0
    target = St / math.sqrt(math.pi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid * math.exp(mid * mid) * math.erf(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------------------
# Problem 1: conductive freezing, one-phase Stefan (Sec. 3.1 with T_0 = T_m).
# ---------------------------------------------------------------------------
def conductive(nx: int = 256, ny: int = 4, St: float = 0.1, alpha: float = 0.1,
               dt: float = 2.5) -> Case:
    """Liquid at the melting point T_m = 1 against a wall at T = 0 (x = 0),
    adiabatic at x = nx, periodic in y; no flow, C = 1 everywhere."""
    Tm, Tw = 1.0, 0.0
    L = 1.0 * (Tm - Tw) / St
    ph = Phase(rho=1.0, mu=0.1, lam=alpha, cp=1.0)
    props = Props(s=ph, l=ph, g=ph, L=L, Ts=Tm, Tl=Tm, sigma=0.0, xi=4.0, Mc=0.0,
                  tau_g=1.0, zero_solid_velocity=0)
    bc = BC(xlo=_wall(DIRICHLET_T, NOSLIP, NOFLUX, Tw=Tw), xhi=_wall(ADIABATIC, NOSLIP, NOFLUX),
            ylo=PER, yhi=PER)
    init = _fields(nx, ny, T=Tm, Fl=1.0, C=1.0)
    return Case(f"conductive_{nx}x{ny}", nx, ny, props, bc, dt, init)


# ---------------------------------------------------------------------------
# Problem 2: three-phase Stefan with volume change (Sec. 3.2), layers along x.
# ---------------------------------------------------------------------------
def three_phase(nx: int = 1024, ny: int = 4, St: float = 0.1, H0: float | None = None,
                rho_ratio_sl: float = 0.9, rho_ratio_lg: float = 100.0, dt: float = 1.0,
                xi: float = 4.0) -> Case:
    """Solid grows from the cold wall at x = 0 into liquid (0 < x < H0) under
    gas (x > H0); the far end is an outlet so displaced gas can leave."""
    Tm, Tw, alpha = 1.0, 0.0, 0.1
    H0 = nx / 2 if H0 is None else H0
    L = 1.0 * (Tm - Tw) / St
    rl, rs, rg = 1.0, rho_ratio_sl, 1.0 / rho_ratio_lg
    props = Props(
        s=Phase(rho=rs, mu=0.01, lam=alpha * rs * 1.0, cp=1.0),
        l=Phase(rho=rl, mu=0.01, lam=alpha * rl * 1.0, cp=1.0),
        g=Phase(rho=rg, mu=0.001, lam=alpha * rg * 1.0, cp=1.0),
        L=L, Ts=Tm, Tl=Tm, sigma=0.01, xi=xi, Mc=0.1, tau_g=1.0, zero_solid_velocity=1)
    bc = BC(xlo=_wall(DIRICHLET_T, NOSLIP, NOFLUX, Tw=Tw), xhi=_wall(ADIABATIC, OUTLET, NOFLUX),
            ylo=PER, yhi=PER)
    x = np.arange(nx) + 0.5
    C = 0.5 * (1.0 + np.tanh(2.0 * (H0 - x) / xi))          # Eq. 61 along x
    init = _fields(nx, ny, T=Tm, Fl=1.0, C=np.broadcast_to(C, (ny, nx)))
    return Case(f"three_phase_{nx}x{ny}_St{St:g}", nx, ny, props, bc, dt, init)


# ---------------------------------------------------------------------------
# Problem 3: liquid film freezing in a closed 2D container (Sec. 3.3).
# ---------------------------------------------------------------------------
def film(n: int = 512, seed: int = 3, dt: float = 0.5, height: float = 0.3,
         St: float = 0.2, modes: int = 8, amp: float = 0.01) -> Case:
    """Film of height 0.3 n under gas; bottom wall at T = 0, other walls
    adiabatic; no-slip bottom and sides, outlet on top.  Water-like ratios:
    rho_l/rho_g = 1000, mu_l/mu_g = 100, rho_s/rho_l = 0.917, Oh = 0.01,
    Bo = 1, St = 0.2, lambda_s/lambda_l = 3.93, cp_s/cp_l = 0.482."""
    Tm, Tw = 1.0, 0.0
    h = height * n
    sigma = 0.01
    rl, rg, rs = 1.0, 1e-3, 0.917
    mu_l = 0.01 * math.sqrt(rl * sigma * h)                 # Oh = mu / sqrt(rho sigma h)
    g = 1.0 * sigma / (rl * h * h)                           # Bo = rho g h^2 / sigma
    cpl = 1.0
    L = cpl * (Tm - Tw) / St
    lam_l = 0.05
    props = Props(
        s=Phase(rho=rs, mu=mu_l, lam=3.93 * lam_l, cp=0.482 * cpl),
        l=Phase(rho=rl, mu=mu_l, lam=lam_l, cp=cpl),
        g=Phase(rho=rg, mu=mu_l / 100.0, lam=1e-4, cp=cpl),
        L=L, Ts=Tm, Tl=Tm, sigma=sigma, xi=4.0, Mc=0.1, tau_g=1.0, gy=-g,
        zero_solid_velocity=1)
    bc = BC(xlo=_wall(ADIABATIC, NOSLIP, NOFLUX), xhi=_wall(ADIABATIC, NOSLIP, NOFLUX),
            ylo=_wall(DIRICHLET_T, NOSLIP, NOFLUX, Tw=Tw), yhi=_wall(ADIABATIC, OUTLET, NOFLUX))
    rng = np.random.default_rng(seed)
    k = np.arange(1, modes + 1)
    a = rng.uniform(0.2, 1.0, modes)
    a *= amp * h / a.sum()                                   # total amplitude 1% of h
    phi = rng.uniform(0.0, 2.0 * math.pi, modes)
    x = np.arange(n) + 0.5
    surf = h + (a[:, None] * np.sin(2.0 * math.pi * k[:, None] * x[None, :] / n + phi[:, None])).sum(0)
    y = np.arange(n) + 0.5
    C = 0.5 * (1.0 + np.tanh(2.0 * (surf[None, :] - y[:, None]) / props.xi))
    init = _fields(n, n, T=Tm, Fl=1.0, C=C)
    return Case(f"film_{n}", n, n, props, bc, dt, init)


# ---------------------------------------------------------------------------
# Problem 4: static droplets freezing on a cold plate (Sec. 3.4), batched.
# ---------------------------------------------------------------------------
def droplet(side: int, theta_deg: float = 90.0, St: float = 0.2, rho_sl: float = 0.917,
            Tw: float = -0.5, dt: float = 0.5, name: str | None = None,
            impact_speed: float = 0.0, We: float | None = None, Re: float | None = None,
            axisymmetric: bool = False, hysteresis: tuple | None = None) -> Case:
    """Half droplet of radius 0.25*side on the plate y = 0 with its axis at
    x = 0: a planar 2-D drop with a symmetry plane there, or with
    axisymmetric=True the drop of revolution in (r, z) (reading R18).
    Plate at Tw < T_m = 0, liquid and gas initially at T_m; rho_l/rho_g = 1000.
    With impact_speed U > 0 the drop is released at rest 0.1*side above the
    plate under gravity g = U^2 / (2 gap), reaching U at contact (an impulsive
    start would send pressure waves through the light gas), and We, Re are
    defined with U and the diameter D = 2R.  hysteresis = (theta_adv,
    theta_rec) makes the plate a hysteresis wetting wall (reading R25) with
    theta_deg as its equilibrium angle."""
    Tm = 0.0
    R = 0.25 * side
    rl, rg, rs = 1.0, 1e-3, rho_sl
    cpl = 1.0
    L = cpl * (Tm - Tw) / St
    lam_l = 0.05
    if impact_speed > 0.0:
        D = 2.0 * R
        sigma = rl * impact_speed ** 2 * D / (We if We else 50.0)
        mu_l = rl * impact_speed * D / (Re if Re else 500.0)
    else:
        sigma, mu_l = 0.005, 0.02
    props = Props(
        s=Phase(rho=rs, mu=mu_l, lam=lam_l, cp=cpl),
        l=Phase(rho=rl, mu=mu_l, lam=lam_l, cp=cpl),
        g=Phase(rho=rg, mu=mu_l / 100.0, lam=5e-5, cp=cpl),
        L=L, Ts=Tm, Tl=Tm, sigma=sigma, xi=4.0, Mc=0.1, tau_g=1.0, zero_solid_velocity=1)
    if impact_speed > 0.0:
        props.gy = -impact_speed ** 2 / (2.0 * 0.1 * side)
    # explicit-step bounds: kinematic viscosity of either fluid x dt <= 0.1
    # (compressive modes of the scheme diffuse with 2 nu, so 16 nu dt <= 1.6 in
    # 2-D) and the Cahn-Hilliard biharmonic term 64 M_c kappa dt <= 1.5
    nu_max = max(mu_l / rl, (mu_l / 100.0) / rg)
    dt = min(dt, 0.1 / nu_max, 1.5 / (64.0 * props.Mc * 1.5 * props.xi * props.sigma))
    bc = BC(xlo=_wall(ADIABATIC, SYMMETRY, NOFLUX), xhi=_wall(ADIABATIC, NOSLIP, NOFLUX),
            ylo=_wall(DIRICHLET_T, NOSLIP, WETTING, Tw=Tw, theta=theta_deg) if hysteresis is None else
            Side(DIRICHLET_T, NOSLIP, WETTING_HYST, Tw, theta_deg, hysteresis[0], hysteresis[1]),
            yhi=_wall(ADIABATIC, NOSLIP, NOFLUX))
    x = np.arange(side) + 0.5
    y = np.arange(side) + 0.5
    if impact_speed > 0.0:
        y0 = R + 0.1 * side
    else:
        y0 = -R * math.cos(math.radians(theta_deg))       # circle meets the plate at theta
    dist = np.sqrt(x[None, :] ** 2 + (y[:, None] - y0) ** 2)
    C = 0.5 * (1.0 + np.tanh(2.0 * (R - dist) / props.xi))   # Eq. 62 read as a circle (R20)
    init = _fields(side, side, T=Tm, Fl=1.0, C=C)
    tag = "_rz" if axisymmetric else ""
    return Case(name or f"droplet_{side}{tag}", side, side, props, bc, dt, init, axisymmetric=int(axisymmetric))


BATCH_SIDES = (128, 192, 256, 384, 512)


def static_droplet_batch(n: int = 64, seed: int = 4, sides=BATCH_SIDES, axisymmetric: bool = False) -> List[Case]:
    """n droplet domains, side uniform over `sides`, seeded contact angle in
    [60, 150] deg, St in [0.05, 0.5], rho_s/rho_l in [0.85, 0.95] and plate
    temperature in [-1, -0.2] (melting point 0); planar or axisymmetric."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.choice(sides))
        out.append(droplet(side, theta_deg=float(rng.uniform(60, 150)),
                           St=float(rng.uniform(0.05, 0.5)), rho_sl=float(rng.uniform(0.85, 0.95)),
                           Tw=float(rng.uniform(-1.0, -0.2)), name=f"drop{k}_{side}",
                           axisymmetric=axisymmetric))
    return out


# ---------------------------------------------------------------------------
# Problem 5: droplet impact on a cold surface (Sec. 3.5) as serving requests.
# ---------------------------------------------------------------------------
@dataclass
class Request:
    rid: int
    arrival_s: float
    case: Case
    steps: int


def impact_requests(n: int = 500, rate_hz: float = 20.0, seed: int = 5, lo: int = 256,
                    hi: int = 1024, U: float = 0.05, end_time_UD: float = 0.015,
                    axisymmetric: bool = False, hysteresis: bool = False) -> List[Request]:
    """Poisson arrivals; side uniform in [lo, hi] rounded to 32; seeded We in
    [10, 200], Re in [100, 2000], St in [0.05, 0.5]; impact speed U (lattice)
    with D = side/2, rho_l/rho_g = 1000, rho_s/rho_l = 0.917.  Each request
    runs to the fixed dimensionless end time t U / D = end_time_UD (0.015 puts
    the offered load near 0.7 of one GB300's FP32C throughput at 20/s).
    hysteresis=True gives the plate the angles of Sec. 3.5 case (a):
    theta_eq 82, theta_adv 100, theta_r 39 deg (reading R25)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        side = int(round(rng.uniform(lo, hi) / 32.0)) * 32
        We = float(rng.uniform(10, 200))
        Re = float(rng.uniform(100, 2000))
        St = float(rng.uniform(0.05, 0.5))
        case = droplet(side, theta_deg=82.0 if hysteresis else 90.0, St=St, rho_sl=0.917, Tw=-1.0, impact_speed=U,
                       We=We, Re=Re, name=f"impact{k}_{side}", axisymmetric=axisymmetric,
                       hysteresis=(100.0, 39.0) if hysteresis else None)
        D = 0.5 * side
        steps = max(1, int(round(end_time_UD * D / U / case.dt)))
        reqs.append(Request(k, t, case, steps))
    return reqs
