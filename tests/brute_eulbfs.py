"""A second, independent transcription of the EULBFS face flux and time step.

It is written from the paper (arXiv 2507.03366, Sec. 2.1-2.5) and the
readings listed with the oracle, in 40-digit arithmetic (mpmath), so that it
serves as a brute-force pin of the FP64 oracle on small grids where every
field varies at once.  It is deliberately organised differently from the
oracle: every surrounding point is an explicit position, every equilibrium a
9-vector, every flux a moment of a 9-vector, and the grid a dictionary of
padded cells.  It shares no code with the oracle or the CUDA library and is
used only by the tests.

Conventions: lattice units, cs^2 = 1/3, cell (i, j) centred at (i + 1/2,
j + 1/2); the x-face with index (i, j) lies at x = i between cells i - 1 and
i, the y-face (i, j) at y = j between rows j - 1 and j.
"""
from __future__ import annotations

import math

from mpmath import mp, mpf

mp.dps = 40

CS2 = mpf(1) / 3
# D2Q9 (Eq. 10, Fig. 1) with the standard weights (the paper does not print them)
E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WT = [mpf(4) / 9] + [mpf(1) / 9] * 4 + [mpf(1) / 36] * 4
GHOST = 2

# boundary kinds (the values of the C ABI)
PERIODIC, DIRICHLET_T, ADIABATIC, NOSLIP, SYMMETRY, OUTLET, NOFLUX, WETTING, WETTING_HYST = range(9)

FIELDS = ("H", "T", "Fl", "Cp", "rho", "lam", "mu", "p", "u", "v", "C")


def N(x) -> mpf:
    return mpf(float(x))


class Model:
    """Problem constants in 40-digit numbers.  ``props``/``bc`` follow the
    dataclasses of ``paper_2507_03366_gb300.workloads``."""

    def __init__(self, nx, ny, props, bc, dt, steps=(0.5, 0.5, 0.5), axisymmetric=False):
        self.nx, self.ny = nx, ny
        self.ph = {k: {q: N(getattr(getattr(props, k), q)) for q in ("rho", "mu", "lam", "cp")}
                   for k in ("s", "l", "g")}
        self.L, self.Ts, self.Tl = N(props.L), N(props.Ts), N(props.Tl)
        sigma, xi = N(props.sigma), N(props.xi)
        self.xi = xi
        self.beta = 12 * sigma / xi if sigma > 0 else mpf(0)      # Sec. 2.3.1
        self.kappa = 3 * xi * sigma / 2
        self.tau_g = N(props.tau_g)
        self.gx, self.gy = N(props.gx), N(props.gy)
        self.zsv = bool(props.zero_solid_velocity)
        self.literal_eq7 = bool(getattr(props, "literal_eq7", 0))
        self.Cref = (self.ph["s"]["cp"] + self.ph["l"]["cp"]) / 2           # Sec. 2.1.2, arithmetic mean
        self.dh, self.df, self.dg = (N(s) for s in steps)                   # streaming steps of h, f, g
        self.Qg = N(props.Mc) / ((self.tau_g - mpf(0.5)) * self.dg)          # M_c = (tau_g - 1/2) Q_g dt_g
        self.kv = 1 - self.ph["s"]["rho"] / self.ph["l"]["rho"]
        self.dt = N(dt)
        self.axi = bool(axisymmetric)
        self.sides = {"xlo": bc.xlo, "xhi": bc.xhi, "ylo": bc.ylo, "yhi": bc.yhi}
        self.per_x = bc.xlo.thermal == PERIODIC
        self.per_y = bc.ylo.thermal == PERIODIC

    # ---- Eq. 5-7 ---------------------------------------------------------
    def cell_state(self, H, C):
        """T, F_l and the mixed properties of a cell from its H and C."""
        Cg = min(max(C, mpf(0)), mpf(1))
        cps, cpl, cpg = self.ph["s"]["cp"], self.ph["l"]["cp"], self.ph["g"]["cp"]
        if self.literal_eq7:
            # Eq. 5-7 as printed: H_s, H_l with the pure solid / liquid heat
            # capacities; the branches' C_p is Eq. 7 at F_s = 1 and F_s = 0
            c_solid, c_liquid = cps, Cg * cpl + (1 - Cg) * cpg
            Hs, Hl = cps * self.Ts, cpl * self.Tl + self.L
        else:
            # reading R1/R2: the heat capacities gated by C~, uniform latent heat
            c_solid, c_liquid = Cg * cps + (1 - Cg) * cpg, Cg * cpl + (1 - Cg) * cpg
            Hs, Hl = c_solid * self.Ts, c_liquid * self.Tl + self.L
        if H < Hs:
            Fl, T = mpf(0), H / c_solid
        elif H > Hl:
            Fl, T = mpf(1), self.Tl + (H - Hl) / c_liquid
        elif Hl > Hs:
            Fl = (H - Hs) / (Hl - Hs)
            T = self.Ts + Fl * (self.Tl - self.Ts)
        else:
            Fl, T = mpf(1), self.Tl
        props = {}
        for q in ("rho", "mu", "lam", "cp"):
            gs, gl, gg = self.ph["s"][q], self.ph["l"][q], self.ph["g"][q]
            Fs = 1 - Fl
            if self.literal_eq7:
                props[q] = Fs * gs + (1 - Fs) * Cg * gl + (1 - Fs) * (1 - Cg) * gg
            else:
                props[q] = Cg * (Fs * gs + Fl * gl) + (1 - Cg) * gg
        return T, Fl, props

    def solid_gate(self, C):
        """The factor on F_s in the volume-change sources and the solid
        projection: C~ (reading R1), or 1 with Eq. 7 as printed."""
        return mpf(1) if self.literal_eq7 else min(max(C, mpf(0)), mpf(1))

    # ---- Eq. 9, 29, 33 (R8), 42 --------------------------------------------
    def h_eq(self, H, T, Cp, u, v):
        out = []
        uu = u * u + v * v
        for a, (ex, ey) in enumerate(E):
            eu = ex * u + ey * v
            if a == 0:
                out.append(H - self.Cref * T + WT[0] * Cp * T * (self.Cref / Cp - uu / (2 * CS2)))
            else:
                out.append(WT[a] * Cp * T * (self.Cref / Cp + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2)))
        return out

    def f_eq(self, p, rho, u, v, rho_face=None):
        """Eq. 29; with rho_face given, Eq. 33 read as R8 (no leading 1 in
        Gamma, density of the face point)."""
        r = rho if rho_face is None else rho_face
        uu = u * u + v * v
        out = []
        for a, (ex, ey) in enumerate(E):
            eu = ex * u + ey * v
            out.append(WT[a] * (p + r * CS2 * (eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2))))
        return out

    def g_eq(self, C, muc, u, v):
        out = []
        for a, (ex, ey) in enumerate(E):
            if a == 0:
                out.append(C - muc * self.Qg * (1 - WT[0]) / CS2)
            else:
                out.append(WT[a] * (muc * self.Qg + C * (ex * u + ey * v)) / CS2)
        return out


class Grid:
    """Padded cell fields of one Runge-Kutta stage input: prim[name][(i, j)]."""

    def __init__(self, m: Model, W):
        self.m = m
        nx, ny = m.nx, m.ny
        self.prim = {f: {} for f in FIELDS + ("muc",)}
        for j in range(ny):
            for i in range(nx):
                H, p, mx, my, C = (W[k][j][i] for k in range(5))
                T, Fl, pr = m.cell_state(H, C)
                vals = {"H": H, "T": T, "Fl": Fl, "Cp": pr["cp"], "rho": pr["rho"], "lam": pr["lam"],
                        "mu": pr["mu"], "p": p, "u": mx / (pr["rho"] * CS2), "v": my / (pr["rho"] * CS2), "C": C}
                for f, x in vals.items():
                    self.prim[f][(i, j)] = x
        self._ghosts(FIELDS)
        for j in range(ny):
            for i in range(nx):
                self.prim["muc"][(i, j)] = self._chemical_potential(i, j)
        self._ghosts(("muc",))
        # central differences (R6) on the interior and the first ghost layer
        self.gx = {f: {} for f in self.prim}
        self.gy = {f: {} for f in self.prim}
        for f, d in self.prim.items():
            for j in range(-1, ny + 1):
                for i in range(-1, nx + 1):
                    self.gx[f][(i, j)] = (d[(i + 1, j)] - d[(i - 1, j)]) / 2
                    self.gy[f][(i, j)] = (d[(i, j + 1)] - d[(i, j - 1)]) / 2

    def _ghost_rule(self, side, name, k, normal, v):
        """Boundary conditions on macroscopic variables (Sec. 3): the value of
        ghost layer k from its mirror cell's value v."""
        sd = self.m.sides[side]
        if name == "T" and sd.thermal == DIRICHLET_T:
            return 2 * N(sd.Tw) - v
        if name == "p" and sd.flow == OUTLET:
            return -v
        if name in ("u", "v"):
            if sd.flow == NOSLIP:
                return -v
            if sd.flow == SYMMETRY and name == normal:
                return -v
        if name == "C" and sd.phase in (WETTING, WETTING_HYST):
            # reading R11: dC/dn_out = (4 cos(theta) / xi) C (1 - C) at distance 2k - 1
            c = self._cos_theta(side) if sd.phase == WETTING_HYST else N(math.cos(sd.theta_deg * (math.pi / 180.0)))
            return v + (2 * k - 1) * (4 * c / self.m.xi) * v * (1 - v)
        return v

    def _cos_theta(self, side):
        """Reading R25 (contact-angle hysteresis, Sec. 3.5): the apparent angle
        of the wall position now being filled, read from the phase field of
        the two wall layers: cos = (C_0 - C_1) / |grad C|, the tangential
        derivative a central difference along layer 0 (one-sided where the
        tangential axis ends at a wall, wrapped where it is periodic), clamped
        to [cos theta_adv, cos theta_rec]; the equilibrium angle where the
        wall cell carries no interface (C_0 (1 - C_0) < 1e-3)."""
        sd = self.m.sides[side]
        C = self.prim["C"]
        nx, ny = self.m.nx, self.m.ny
        xs = side in ("xlo", "xhi")
        n = ny if xs else nx
        per = self.m.per_y if xs else self.m.per_x
        t = self._t
        if per:
            tc, tp, tm = t % n, (t + 1) % n, (t - 1) % n
        else:
            tc = min(max(t, 0), n - 1)
            tp, tm = min(tc + 1, n - 1), max(tc - 1, 0)
        m = nx if xs else ny
        l0, l1 = (0, 1) if side in ("xlo", "ylo") else (m - 1, m - 2)

        def at(layer, tt):
            return C[(layer, tt)] if xs else C[(tt, layer)]

        ceq = N(math.cos(sd.theta_deg * (math.pi / 180.0)))
        c0 = at(l0, tc)
        if not (c0 * (1 - c0) >= mpf("1e-3")):
            return ceq
        dn = c0 - at(l1, tc)
        dt = (at(l0, tp) - at(l0, tm)) / (2 if per else (tp - tm))
        g = mp.sqrt(dn * dn + dt * dt)
        if not g > 0:
            return ceq
        c = dn / g
        lo = N(math.cos(sd.theta_adv_deg * (math.pi / 180.0)))
        hi = N(math.cos(sd.theta_rec_deg * (math.pi / 180.0)))
        return lo if c < lo else (hi if c > hi else c)

    def _ghosts(self, names):
        nx, ny = self.m.nx, self.m.ny
        for name in names:
            d = self.prim[name]
            for j in range(ny):               # x sides first, on interior rows
                self._t = j                   # the wall position (R25)
                for k in range(1, GHOST + 1):
                    if self.m.per_x:
                        d[(-k, j)] = d[(nx - k, j)]
                        d[(nx - 1 + k, j)] = d[(k - 1, j)]
                    else:
                        d[(-k, j)] = self._ghost_rule("xlo", name, k, "u", d[(k - 1, j)])
                        d[(nx - 1 + k, j)] = self._ghost_rule("xhi", name, k, "u", d[(nx - k, j)])
            for i in range(-GHOST, nx + GHOST):   # then y sides on every column
                self._t = i
                for k in range(1, GHOST + 1):
                    if self.m.per_y:
                        d[(i, -k)] = d[(i, ny - k)]
                        d[(i, ny - 1 + k)] = d[(i, k - 1)]
                    else:
                        d[(i, -k)] = self._ghost_rule("ylo", name, k, "v", d[(i, k - 1)])
                        d[(i, ny - 1 + k)] = self._ghost_rule("yhi", name, k, "v", d[(i, ny - k)])

    def _chemical_potential(self, i, j):
        """mu_c = 2 beta C (C-1)(2C-1) - kappa lap C (reading R5)."""
        C = self.prim["C"]
        c = C[(i, j)]
        if self.m.axi:
            r, rw, re = mpf(i) + mpf(0.5), mpf(i), mpf(i + 1)
            lap = (re * (C[(i + 1, j)] - c) - rw * (c - C[(i - 1, j)])) / r + C[(i, j + 1)] + C[(i, j - 1)] - 2 * c
        else:
            lap = C[(i + 1, j)] + C[(i - 1, j)] + C[(i, j + 1)] + C[(i, j - 1)] - 4 * c
        return 2 * self.m.beta * c * (c - 1) * (2 * c - 1) - self.m.kappa * lap

    def at(self, name, cell, x, y):
        """Eq. 54: the linear reconstruction of a field from a cell at (x, y)."""
        i, j = cell
        return (self.prim[name][cell] + (x - (mpf(i) + mpf(0.5))) * self.gx[name][cell]
                + (y - (mpf(j) + mpf(0.5))) * self.gy[name][cell])

    def point_values(self, names, face, left, right, normal, point):
        """Values at a surrounding point: from the cell on whose side of the
        face it lies, or the mean of both reconstructions on the face (R7)."""
        off = (point[0] - face[0]) * normal[0] + (point[1] - face[1]) * normal[1]
        out = {}
        for n in names:
            if off < 0:
                out[n] = self.at(n, left, *point)
            elif off > 0:
                out[n] = self.at(n, right, *point)
            else:
                out[n] = (self.at(n, left, *point) + self.at(n, right, *point)) / 2
        return out

    def face_flux(self, direction, i, j):
        """Sec. 2.5 steps (2)-(4) and Eq. 53 at one face: (F_H, F_p, F_mx,
        F_my, F_C, u_n)."""
        m = self.m
        if direction == 0:
            face, normal, left, right = (mpf(i), mpf(j) + mpf(0.5)), (1, 0), (i - 1, j), (i, j)
        else:
            face, normal, left, right = (mpf(i) + mpf(0.5), mpf(j)), (0, 1), (i, j - 1), (i, j)

        def points(step):
            return [(face[0] - ex * step, face[1] - ey * step) for ex, ey in E]

        # the face itself (alpha = 0 point) at the current time: R9
        fv = self.point_values(("rho", "T", "Cp", "lam", "mu", "muc", "u"), face, left, right, normal, face)
        rho_f = fv["rho"]
        # step (2): surrounding equilibria, each distribution on its own points (R26)
        heq_s, feq_s, feqm_s, geq_s = [], [], [], []
        for a, pt in enumerate(points(m.dh)):
            q = self.point_values(("H", "T", "Cp", "u", "v"), face, left, right, normal, pt)
            heq_s.append(m.h_eq(q["H"], q["T"], q["Cp"], q["u"], q["v"])[a])
        for a, pt in enumerate(points(m.df)):
            q = self.point_values(("p", "rho", "u", "v"), face, left, right, normal, pt)
            feq_s.append(m.f_eq(q["p"], q["rho"], q["u"], q["v"])[a])
            feqm_s.append(m.f_eq(q["p"], q["rho"], q["u"], q["v"], rho_face=rho_f)[a])
        for a, pt in enumerate(points(m.dg)):
            q = self.point_values(("C", "muc", "u", "v"), face, left, right, normal, pt)
            geq_s.append(m.g_eq(q["C"], q["muc"], q["u"], q["v"])[a])
        if m.axi and face[0] > 0:
            # reading R24: the axisymmetric mass source -rho cs^2 u_r / r
            # streamed with weight w_a over dt_f into f^eq and f^eq-m
            S = -m.df * rho_f * CS2 * fv["u"] / face[0]
            feq_s = [f + WT[a] * S for a, f in enumerate(feq_s)]
            feqm_s = [f + WT[a] * S for a, f in enumerate(feqm_s)]
        # step (3): Eq. 56, then the equilibria at the face
        H_f = sum(heq_s)
        p_f = sum(feq_s)
        mx_f = sum(E[a][0] * feq_s[a] for a in range(9))
        my_f = sum(E[a][1] * feq_s[a] for a in range(9))
        C_f = sum(geq_s)
        u_f, v_f = mx_f / (rho_f * CS2), my_f / (rho_f * CS2)
        heq_f = m.h_eq(H_f, fv["T"], fv["Cp"], u_f, v_f)
        feq_f = m.f_eq(p_f, rho_f, u_f, v_f)
        geq_f = m.g_eq(C_f, fv["muc"], u_f, v_f)
        tau_h = mpf(0.5) + fv["lam"] / (rho_f * m.Cref * CS2 * m.dh)
        tau_f = mpf(0.5) + fv["mu"] / (rho_f * CS2 * m.df)
        tau_g = m.tau_g
        # step (4): Eq. 13/16, 35/37 (R3 sign), 44/46
        h_star = [heq_f[a] + (1 - 1 / (2 * tau_h)) * (-tau_h * (heq_f[a] - heq_s[a])) for a in range(9)]
        f_star = [feq_f[a] + (1 - 1 / (2 * tau_f)) * (-tau_f * (feq_f[a] - feqm_s[a])) for a in range(9)]
        g_star = [geq_f[a] + (1 - 1 / (2 * tau_g)) * (-tau_g * (geq_f[a] - geq_s[a])) for a in range(9)]
        # Eq. 53 along the face normal
        en = [E[a][0] * normal[0] + E[a][1] * normal[1] for a in range(9)]
        return (sum(en[a] * h_star[a] for a in range(9)),
                sum(en[a] * feq_f[a] for a in range(9)),
                sum(en[a] * E[a][0] * f_star[a] for a in range(9)),
                sum(en[a] * E[a][1] * f_star[a] for a in range(9)),
                sum(en[a] * g_star[a] for a in range(9)),
                u_f * normal[0] + v_f * normal[1])


def residual(m: Model, W, dFs):
    """R(W) of Eq. 52 with the sources of Eq. 51 (readings R12-R14, R24);
    dFs[j][i] is the lagged solid-fraction rate of the step."""
    g = Grid(m, W)
    nx, ny = m.nx, m.ny
    fx = {(i, j): g.face_flux(0, i, j) for j in range(ny) for i in range(nx + 1)}
    fy = {(i, j): g.face_flux(1, i, j) for j in range(ny + 1) for i in range(nx)}
    R = [[[None] * nx for _ in range(ny)] for _ in range(5)]
    for j in range(ny):
        for i in range(nx):
            w, e, s, n = fx[(i, j)], fx[(i + 1, j)], fy[(i, j)], fy[(i, j + 1)]
            if m.axi:
                rc, rw, re = mpf(i) + mpf(0.5), mpf(i), mpf(i + 1)
                div = [(re * e[k] - rw * w[k]) / rc + (n[k] - s[k]) for k in range(6)]
            else:
                div = [(e[k] - w[k]) + (n[k] - s[k]) for k in range(6)]
            c = (i, j)
            P = g.prim
            T, Fl, Cp, rho, C = P["T"][c], P["Fl"][c], P["Cp"][c], P["rho"][c], P["C"][c]
            u, v = P["u"][c], P["v"][c]
            D = m.solid_gate(C) * dFs[j][i]          # solid-volume rate (R1, R14)
            src = [Cp * T * div[5],
                   CS2 * (u * g.gx["rho"][c] + v * g.gy["rho"][c]) + rho * CS2 * m.kv * D,
                   CS2 * (-Fl * C * g.gx["muc"][c] + rho * m.gx - rho * u * D),
                   CS2 * (-Fl * C * g.gy["muc"][c] + rho * m.gy - rho * v * D),
                   C * m.kv * dFs[j][i]]
            if m.axi:
                rc = mpf(i) + mpf(0.5)
                src[2] += CS2 * (P["p"][c] - m.df * div[1] - 2 * P["mu"][c] * u / rc) / rc
            for k in range(5):
                R[k][j][i] = -div[k] + src[k]
    return R


def _project(m: Model, W):
    """Reading R15: the momentum of the solid part of each cell set to zero."""
    if not m.zsv:
        return
    for j in range(m.ny):
        for i in range(m.nx):
            _, Fl, _ = m.cell_state(W[0][j][i], W[4][j][i])
            keep = 1 - m.solid_gate(W[4][j][i]) * (1 - Fl)
            W[2][j][i] *= keep
            W[3][j][i] *= keep


def step(m: Model, W, Fs_prev):
    """One SSP-RK3 time step (Eq. 58) from the state W (5 lists of rows) and
    the previous step's solid fraction; returns (W^{n+1}, F_s^n)."""
    nx, ny = m.nx, m.ny
    Fs = [[1 - m.cell_state(W[0][j][i], W[4][j][i])[1] for i in range(nx)] for j in range(ny)]
    dFs = [[(Fs[j][i] - Fs_prev[j][i]) / m.dt for i in range(nx)] for j in range(ny)]   # R14
    Wn = [[row[:] for row in W[k]] for k in range(5)]
    coef = [(mpf(1), mpf(0), mpf(1)), (mpf(3) / 4, mpf(1) / 4, mpf(1) / 4), (mpf(1) / 3, mpf(2) / 3, mpf(2) / 3)]
    cur = Wn
    for a, b, c in coef:
        R = residual(m, cur, dFs)
        nxt = [[[a * Wn[k][j][i] + b * cur[k][j][i] + c * m.dt * R[k][j][i] for i in range(nx)]
                for j in range(ny)] for k in range(5)]
        _project(m, nxt)
        cur = nxt
    return cur, Fs
