/*
 * eulbfs_oracle.c -- plain FP64 CPU oracle of the EULBFS explicit step.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Deliberately slow and literal:
 * every face, every D2Q9 direction, every field is evaluated as the paper
 * writes it, with no algebraic contraction, fusion or reordering.
 * Build: gcc -O2 -ffp-contract=off -std=c99 -shared -fPIC (reading R23).
 *
 * Function map (paper: arXiv 2507.03366):
 *   or_invert_enthalpy  Eq. 5-6 with uniform latent heat, gated Cp (R1, R2)
 *   or_mix              Eq. 7 (R1)
 *   or_heq              Eq. 9        or_feq   Eq. 29
 *   or_feqm             Eq. 33-34 (R8)   or_geq Eq. 42
 *   face_flux           Sec. 2.5 steps (2)-(4): Eq. 54, 56, 13/16, 35/37, 44/46, 53
 *   residual            Eq. 51-52, 57 (planar, or axisymmetric (r, z) with
 *                       r-weighted volumes/areas and the hoop source)
 *   or_step             Eq. 58 and Sec. 2.5 steps (5)-(7)
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* Loops whose iterations write disjoint elements may run on several host
 * threads (OpenMP, when the oracle is built with it).  Nothing is reduced
 * across threads, so the results are bitwise the same for any thread count. */
#ifdef _OPENMP
#include <omp.h>
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OMP_FOR
#endif

#define NG 2              /* ghost ring width */
#define CS2 (1.0 / 3.0)   /* cs^2 = c^2/3 with lattice speed c = 1 */

/* D2Q9 velocities (Eq. 10, Fig. 1).  The weights are not printed in the
 * paper; these are the standard D2Q9 weights 4/9, 1/9, 1/36. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WA[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* primitive (macroscopic) fields held on the padded grid */
enum { P_H, P_T, P_FL, P_CP, P_RHO, P_LAM, P_MU, P_P, P_U, P_V, P_C, P_MUC, NPRIM };

/* variables interpolated to the surrounding points (Sec. 2.5 step (2)),
 * plus rho (needed by Eq. 29) and lambda, mu (needed at the face, R9) */
static const int RECON[] = {P_H, P_T, P_CP, P_RHO, P_LAM, P_MU, P_P, P_U, P_V, P_C, P_MUC};
#define NRECON ((int)(sizeof(RECON) / sizeof(RECON[0])))

struct or_solver {
    int nx, ny, px, py;
    or_props P;
    or_bc B;
    or_numerics N;
    double Cref, beta, kappa, Qg;
    double dth, dtf, dtg;  /* streaming steps of h, f, g (R26) */
    double* W[5];          /* conserved state (Eq. 49) */
    double* Fsp;           /* F_s at the previous step (R14) */
    double* dFs;           /* (F_s^n - F_s^{n-1}) / dt, fixed during one step */
    double* prim[NPRIM];   /* padded primitive fields */
    double* grx[NPRIM];    /* central x-gradients, valid on interior + ghost layer 1 */
    double* gry[NPRIM];
    double* Wn[5];
    double* R[5];
    double* fx;            /* x-face fluxes, 6 per face, (nx+1)*ny faces */
    double* fy;            /* y-face fluxes, 6 per face, nx*(ny+1) faces */
    double t;
    long long step;
};

static double clamp01(double c) { return c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c); }
static int wrapi(int g, int n) { return ((g % n) + n) % n; }
static int PI(const or_solver* s, int i, int j) { return (j + NG) * s->px + (i + NG); }

/* ------------------------------------------------------------------ */
/* Closure: enthalpy inversion (Eq. 5-6) and property mixing (Eq. 7).  */
/* ------------------------------------------------------------------ */

/* Reading R1: the latent heat is uniform, H = Cp*T + L*F_l in every cell
 * (the assumption under Eq. 2 that drops the advection of Delta H), while
 * the heat capacity is the Eq. 7 mixture gated by C~ = clamp(C, 0, 1).
 * H_s and H_l of Eq. 5-6 are the enthalpies of the cell fully solid at T_s
 * and fully liquid at T_l.  Reading R2: the solid branch uses the
 * solid-state mixture Cp, the liquid branch the liquid-state mixture Cp. */
/* The heat capacities of the solid and liquid branches of Eq. 6 and the
 * enthalpies H_s, H_l of Eq. 5-6.  Reading R1: gated mixtures.  Eq. 7 as
 * printed (literal_eq7): H_s = C_p,s T_s and H_l = C_p,l T_l + L with the pure
 * phases' heat capacities; the solid branch's C_p is Eq. 7 at F_s = 1, i.e.
 * C_p,s, the liquid branch's is Eq. 7 at F_s = 0, C~ C_p,l + (1 - C~) C_p,g. */
static void branch_constants(const or_props* P, double C, double* cps, double* cpl, double* Hs, double* Hl) {
    const double Ct = clamp01(C);
    *cpl = Ct * P->l.cp + (1.0 - Ct) * P->g.cp;
    if (P->literal_eq7) {
        *cps = P->s.cp;
        *Hs = P->s.cp * P->Ts;
        *Hl = P->l.cp * P->Tl + P->L;
    } else {
        *cps = Ct * P->s.cp + (1.0 - Ct) * P->g.cp;
        *Hs = *cps * P->Ts;
        *Hl = *cpl * P->Tl + P->L;
    }
}

void or_invert_enthalpy(const or_props* P, double H, double C, double* T, double* Fl) {
    double cps, cpl, Hs, Hl;
    branch_constants(P, C, &cps, &cpl, &Hs, &Hl);
    if (H < Hs) {                 /* Eq. 5-6, first branch */
        *Fl = 0.0;
        *T = H / cps;
    } else if (H > Hl) {          /* third branch */
        *Fl = 1.0;
        *T = P->Tl + (H - Hl) / cpl;
    } else if (Hl > Hs) {         /* mushy branch */
        *Fl = (H - Hs) / (Hl - Hs);
        *T = P->Ts + (*Fl) * (P->Tl - P->Ts);
    } else {                      /* zero-width mushy range (L = 0 and Ts == Tl) */
        *Fl = 1.0;
        *T = P->Tl;
    }
}

/* Inverse of Eq. 5-6 used only to build the initial H from (T, F_l, C). */
double or_enthalpy_of(const or_props* P, double T, double Fl, double C) {
    double cps, cpl, Hs, Hl;
    branch_constants(P, C, &cps, &cpl, &Hs, &Hl);
    if (T < P->Ts) return cps * T;
    if (T > P->Tl) return Hl + cpl * (T - P->Tl);
    double f = (P->Tl > P->Ts) ? (T - P->Ts) / (P->Tl - P->Ts) : Fl;
    if (f >= 1.0) return Hl;
    if (f <= 0.0) return Hs;
    return Hs + f * (Hl - Hs);
}

/* Eq. 7 with reading R1: gamma = C~[F_s gamma_s + F_l gamma_l] + (1 - C~) gamma_g;
 * as printed (literal_eq7): F_s gamma_s + (1 - F_s) C~ gamma_l + (1 - F_s)(1 - C~) gamma_g. */
double or_mix(const or_props* P, double C, double Fl, int which) {
    const double Ct = clamp01(C);
    const double Fs = 1.0 - Fl;
    double gs, gl, gg;
    switch (which) {
        case 0: gs = P->s.rho; gl = P->l.rho; gg = P->g.rho; break;
        case 1: gs = P->s.mu; gl = P->l.mu; gg = P->g.mu; break;
        case 2: gs = P->s.lambda; gl = P->l.lambda; gg = P->g.lambda; break;
        default: gs = P->s.cp; gl = P->l.cp; gg = P->g.cp; break;
    }
    if (P->literal_eq7) return Fs * gs + (1.0 - Fs) * Ct * gl + (1.0 - Fs) * (1.0 - Ct) * gg;
    return Ct * (Fs * gs + Fl * gl) + (1.0 - Ct) * gg;
}

/* The factor on F_s in the volume-change sources and the solid projection:
 * C~ under reading R1, 1 with Eq. 7 as printed. */
static double solid_gate(const or_props* P, double C) { return P->literal_eq7 ? 1.0 : clamp01(C); }

/* ------------------------------------------------------------------ */
/* Equilibria.                                                          */
/* ------------------------------------------------------------------ */

/* Eq. 9 */
double or_heq(int a, double H, double T, double Cp, double Cref, double u, double v) {
    const double eu = EX[a] * u + EY[a] * v;
    const double uu = u * u + v * v;
    if (a == 0) return H - Cref * T + WA[0] * Cp * T * (Cref / Cp - uu / (2.0 * CS2));
    return WA[a] * Cp * T *
           (Cref / Cp + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 29 */
double or_feq(int a, double p, double rho, double u, double v) {
    const double eu = EX[a] * u + EY[a] * v;
    const double uu = u * u + v * v;
    return WA[a] * (p + rho * CS2 * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
}

/* Eq. 33-34 with reading R8: Gamma_alpha without the leading "1", so that
 * f^eq-m is f^eq with the density taken at the face point x. */
double or_feqm(int a, double p, double rho_face, double u, double v) {
    const double eu = EX[a] * u + EY[a] * v;
    const double uu = u * u + v * v;
    const double Gamma = CS2 * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    return WA[a] * (p + rho_face * Gamma);
}

/* Eq. 42 */
double or_geq(int a, double C, double muc, double Qg, double u, double v) {
    const double eu = EX[a] * u + EY[a] * v;
    if (a == 0) return C - muc * Qg * (1.0 - WA[0]) / CS2;
    return WA[a] * (muc * Qg + C * eu) / CS2;
}

/* ------------------------------------------------------------------ */
/* Primitive fields and ghost cells.                                    */
/* ------------------------------------------------------------------ */

static void derive_interior(or_solver* s, double* const W[5]) {
    OMP_FOR
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            const int c = j * s->nx + i, q = PI(s, i, j);
            const double H = W[0][c], C = W[4][c];
            double T, Fl;
            or_invert_enthalpy(&s->P, H, C, &T, &Fl);
            const double rho = or_mix(&s->P, C, Fl, 0);
            s->prim[P_H][q] = H;
            s->prim[P_T][q] = T;
            s->prim[P_FL][q] = Fl;
            s->prim[P_CP][q] = or_mix(&s->P, C, Fl, 3);
            s->prim[P_RHO][q] = rho;
            s->prim[P_LAM][q] = or_mix(&s->P, C, Fl, 2);
            s->prim[P_MU][q] = or_mix(&s->P, C, Fl, 1);
            s->prim[P_P][q] = W[1][c];
            s->prim[P_U][q] = W[2][c] / (rho * CS2);   /* W3 = rho cs^2 u (Eq. 49) */
            s->prim[P_V][q] = W[3][c] / (rho * CS2);
            s->prim[P_C][q] = C;
        }
}

/* Ghost value k layers outside a wall side from the value vm in its mirror
 * cell.  The boundary conditions act directly on macroscopic variables.
 * normal_f is the wall-normal velocity component. */
/* Reading R25, contact-angle hysteresis (Sec. 3.5 gives theta_adv and theta_r
 * but no model; this is a literature-style choice).  The apparent angle at
 * the wall position t (the row of an x side, the column of a y side, clamped
 * to the domain or wrapped on a periodic axis) is read from the phase field
 * of the two wall layers: cos(theta_app) = dC/dn_out / |grad C| with
 * dC/dn_out = C_0 - C_1 and the tangential central difference along layer 0
 * (one-sided at a walled end).  The wetting rule of R11 then takes
 * cos(theta) = cos(theta_app) clamped to [cos(theta_adv), cos(theta_rec)]:
 * inside that window the contact line keeps its current angle (pinned),
 * outside it the nearer limit applies.  Where the wall cell carries no
 * interface, C_0 (1 - C_0) < 1e-3, the equilibrium angle is used: there the
 * direction of grad C is set by round-off and the R11 correction, which
 * scales with C (1 - C), is negligible anyway. */
static double wall_cos_theta(const or_solver* s, const or_side* sd, int side, int t) {
    const double ceq = cos(sd->theta_deg * (M_PI / 180.0));
    if (sd->phase != OR_BC_WETTING_HYST) return ceq;
    const int xs = side < 2;                       /* an x side: t runs along y */
    const int n = xs ? s->ny : s->nx, m = xs ? s->nx : s->ny;
    const int per = xs ? (s->B.ylo.thermal == OR_BC_PERIODIC) : (s->B.xlo.thermal == OR_BC_PERIODIC);
    int tc = t, tp = t + 1, tm = t - 1;
    if (per) {
        tc = wrapi(t, n); tp = wrapi(t + 1, n); tm = wrapi(t - 1, n);
    } else {
        tc = t < 0 ? 0 : (t > n - 1 ? n - 1 : t);
        tp = tc + 1 > n - 1 ? n - 1 : tc + 1;
        tm = tc - 1 < 0 ? 0 : tc - 1;
    }
    const int l0 = (side == 0 || side == 2) ? 0 : m - 1;     /* wall layer and the one inside */
    const int l1 = (side == 0 || side == 2) ? 1 : m - 2;
    const double* C = s->prim[P_C];
#define CAT(layer, tt) (xs ? C[PI(s, (layer), (tt))] : C[PI(s, (tt), (layer))])
    const double dn = CAT(l0, tc) - CAT(l1, tc);
    const double dt = per ? 0.5 * (CAT(l0, tp) - CAT(l0, tm)) : (CAT(l0, tp) - CAT(l0, tm)) / (double)(tp - tm);
    const double c0 = CAT(l0, tc);
    if (!(c0 * (1.0 - c0) >= 1e-3)) return ceq;
#undef CAT
    const double g = sqrt(dn * dn + dt * dt);
    if (!(g > 0.0)) return ceq;
    const double c = dn / g, lo = cos(sd->theta_adv_deg * (M_PI / 180.0)), hi = cos(sd->theta_rec_deg * (M_PI / 180.0));
    return c < lo ? lo : (c > hi ? hi : c);
}

static double ghost_value(const or_solver* s, const or_side* sd, int f, int k, int normal_f,
                          double vm, double cth) {
    switch (f) {
        case P_T: return sd->thermal == OR_BC_DIRICHLET_T ? 2.0 * sd->Tw - vm : vm;
        case P_P: return sd->flow == OR_BC_OUTLET ? -vm : vm;
        case P_U:
        case P_V:
            if (sd->flow == OR_BC_NOSLIP) return -vm;
            if (sd->flow == OR_BC_SYMMETRY) return f == normal_f ? -vm : vm;
            return vm;
        case P_C:
            if (sd->phase == OR_BC_WETTING || sd->phase == OR_BC_WETTING_HYST) {
                /* R11: dC/dn_out = (4 cos(theta)/xi) C (1 - C), ghost k at distance (2k-1);
                 * cth = cos(theta) of this wall position (R25 for hysteresis) */
                return vm + (2.0 * k - 1.0) * (4.0 * cth / s->P.xi) * vm * (1.0 - vm);
            }
            return vm;
        default: return vm;   /* H, F_l, properties, mu_c: mirror copy */
    }
}

/* Fill the ghost ring for the listed fields: x sides on interior rows first,
 * then y sides on every column (so corners take the y rule of the x ghost). */
static void fill_ghosts(or_solver* s, const int* fields, int nf) {
    const int nx = s->nx, ny = s->ny;
    const int perx = s->B.xlo.thermal == OR_BC_PERIODIC;
    const int pery = s->B.ylo.thermal == OR_BC_PERIODIC;
    OMP_FOR
    for (int j = 0; j < ny; ++j)
        for (int k = 1; k <= NG; ++k) {
            const int gl = -k, gh = nx - 1 + k;
            const int ml = perx ? wrapi(gl, nx) : k - 1;
            const int mh = perx ? wrapi(gh, nx) : nx - k;
            const double cl = perx ? 0.0 : wall_cos_theta(s, &s->B.xlo, 0, j);
            const double ch = perx ? 0.0 : wall_cos_theta(s, &s->B.xhi, 1, j);
            for (int n = 0; n < nf; ++n) {
                const int f = fields[n];
                const double vl = s->prim[f][PI(s, ml, j)], vh = s->prim[f][PI(s, mh, j)];
                s->prim[f][PI(s, gl, j)] = perx ? vl : ghost_value(s, &s->B.xlo, f, k, P_U, vl, cl);
                s->prim[f][PI(s, gh, j)] = perx ? vh : ghost_value(s, &s->B.xhi, f, k, P_U, vh, ch);
            }
        }
    OMP_FOR
    for (int i = -NG; i < nx + NG; ++i)
        for (int k = 1; k <= NG; ++k) {
            const int gl = -k, gh = ny - 1 + k;
            const int ml = pery ? wrapi(gl, ny) : k - 1;
            const int mh = pery ? wrapi(gh, ny) : ny - k;
            const double cl = pery ? 0.0 : wall_cos_theta(s, &s->B.ylo, 2, i);
            const double ch = pery ? 0.0 : wall_cos_theta(s, &s->B.yhi, 3, i);
            for (int n = 0; n < nf; ++n) {
                const int f = fields[n];
                const double vl = s->prim[f][PI(s, i, ml)], vh = s->prim[f][PI(s, i, mh)];
                s->prim[f][PI(s, i, gl)] = pery ? vl : ghost_value(s, &s->B.ylo, f, k, P_V, vl, cl);
                s->prim[f][PI(s, i, gh)] = pery ? vh : ghost_value(s, &s->B.yhi, f, k, P_V, vh, ch);
            }
        }
}

/* Chemical potential, Sec. 2.3.1 with reading R5 (minus sign on kappa lap C),
 * 5-point Laplacian (R6), on interior cells; ghosts are then mirrored. */
static void compute_muc(or_solver* s) {
    const double* C = s->prim[P_C];
    OMP_FOR
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            const int q = PI(s, i, j);
            const double c = C[q];
            double lap;
            if (s->N.axisymmetric) {
                /* (1/r) d/dr (r dC/dr) + d2C/dz2, faces at r = i and i + 1 */
                const double rc = i + 0.5;
                lap = (((i + 1.0) * (C[PI(s, i + 1, j)] - c) - i * (c - C[PI(s, i - 1, j)])) / rc) +
                      (C[PI(s, i, j + 1)] + C[PI(s, i, j - 1)] - 2.0 * c);
            } else {
                lap = C[PI(s, i + 1, j)] + C[PI(s, i - 1, j)] + C[PI(s, i, j + 1)] + C[PI(s, i, j - 1)] - 4.0 * c;
            }
            s->prim[P_MUC][q] = 2.0 * s->beta * c * (c - 1.0) * (2.0 * c - 1.0) - s->kappa * lap;
        }
    const int f = P_MUC;
    fill_ghosts(s, &f, 1);
}

/* Central differences (R6) on interior cells and ghost layer 1. */
static void compute_gradients(or_solver* s) {
    OMP_FOR
    for (int f = 0; f < NPRIM; ++f)
        for (int j = -1; j <= s->ny; ++j)
            for (int i = -1; i <= s->nx; ++i) {
                const int q = PI(s, i, j);
                s->grx[f][q] = 0.5 * (s->prim[f][PI(s, i + 1, j)] - s->prim[f][PI(s, i - 1, j)]);
                s->gry[f][q] = 0.5 * (s->prim[f][PI(s, i, j + 1)] - s->prim[f][PI(s, i, j - 1)]);
            }
}

static void prepare(or_solver* s, double* const W[5]) {
    static const int base[] = {P_H, P_T, P_FL, P_CP, P_RHO, P_LAM, P_MU, P_P, P_U, P_V, P_C};
    derive_interior(s, W);
    fill_ghosts(s, base, (int)(sizeof(base) / sizeof(base[0])));
    compute_muc(s);
    compute_gradients(s);
}

/* Eq. 54: linear reconstruction from cell (ci, cj) at the point (x, y). */
static double recon(const or_solver* s, int f, int ci, int cj, double x, double y) {
    const int q = PI(s, ci, cj);
    return s->prim[f][q] + (x - (ci + 0.5)) * s->grx[f][q] + (y - (cj + 0.5)) * s->gry[f][q];
}

/* ------------------------------------------------------------------ */
/* Face flux: Sec. 2.5 steps (2)-(4) and Eq. 53.                        */
/* ------------------------------------------------------------------ */

/* step (2): macroscopic variables at the points x_f - e_alpha dts of the
 * face (xf, yf) with normal (nxv, nyv) by Eq. 54.  The point belongs to the
 * cell on whose side of the face it lies; on the face itself the values are
 * the mean of the two reconstructions (R7). */
static void surrounding(const or_solver* s, double xf, double yf, double nxv, double nyv, int Li, int Lj,
                        int Ri, int Rj, double dts, double q[9][NPRIM]) {
    for (int a = 0; a < 9; ++a) {
        const double sx = xf - EX[a] * dts, sy = yf - EY[a] * dts;
        const double off = (sx - xf) * nxv + (sy - yf) * nyv;
        for (int n = 0; n < NRECON; ++n) {
            const int f = RECON[n];
            if (off < 0.0)
                q[a][f] = recon(s, f, Li, Lj, sx, sy);
            else if (off > 0.0)
                q[a][f] = recon(s, f, Ri, Rj, sx, sy);
            else
                q[a][f] = 0.5 * (recon(s, f, Li, Lj, sx, sy) + recon(s, f, Ri, Rj, sx, sy));
        }
    }
}

static void face_flux(const or_solver* s, int dir, int i, int j, double out[6]) {
    const double dts = s->dtf;   /* flow streaming step: R24 terms */
    double xf, yf, nxv, nyv;
    int Li, Lj, Ri, Rj;
    if (dir == 0) {
        xf = i; yf = j + 0.5; nxv = 1.0; nyv = 0.0;
        Li = i - 1; Lj = j; Ri = i; Rj = j;
    } else {
        xf = i + 0.5; yf = j; nxv = 0.0; nyv = 1.0;
        Li = i; Lj = j - 1; Ri = i; Rj = j;
    }

    /* Reading R26: each distribution streams over its own step, so h, f and
     * g take their surrounding points at x_f - e_alpha dt_h, dt_f, dt_g.  The
     * alpha = 0 point is the face itself for all three. */
    double qh[9][NPRIM], qf[9][NPRIM], qg[9][NPRIM];
    surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dtf, qf);
    if (s->dth == s->dtf) memcpy(qh, qf, sizeof(qh));
    else surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dth, qh);
    if (s->dtg == s->dtf) memcpy(qg, qf, sizeof(qg));
    else surrounding(s, xf, yf, nxv, nyv, Li, Lj, Ri, Rj, s->dtg, qg);
    double (*q)[NPRIM] = qf;

    /* face values at the current time: mean of the L/R reconstructions at
     * the face (text under Eq. 54), i.e. the alpha = 0 point (R9). */
    const double rho_f = q[0][P_RHO], Tf = q[0][P_T], Cpf = q[0][P_CP];
    const double lamf = q[0][P_LAM], muf = q[0][P_MU], mucf = q[0][P_MUC];

    /* step (2): surrounding equilibria, Eq. 9, 29, 33, 42 */
    double heqs[9], feqs[9], feqms[9], geqs[9];
    for (int a = 0; a < 9; ++a) {
        heqs[a] = or_heq(a, qh[a][P_H], qh[a][P_T], qh[a][P_CP], s->Cref, qh[a][P_U], qh[a][P_V]);
        feqs[a] = or_feq(a, qf[a][P_P], qf[a][P_RHO], qf[a][P_U], qf[a][P_V]);
        feqms[a] = or_feqm(a, qf[a][P_P], rho_f, qf[a][P_U], qf[a][P_V]);
        geqs[a] = or_geq(a, qg[a][P_C], qg[a][P_MUC], s->Qg, qg[a][P_U], qg[a][P_V]);
    }
    if (s->N.axisymmetric && xf > 0.0) {
        /* Axisymmetric runs (reading R24): the pressure equation has the
         * extra source -rho cs^2 u_r / r, which the planar stencil does not
         * see.  It is streamed with the surrounding distributions (weight
         * w_alpha, over dt_s) so that p at the face is advanced with the full
         * 3-D divergence; evaluated with the face values.  On the axis the
         * face area is zero and nothing is added. */
        const double Sp = -dts * rho_f * CS2 * q[0][P_U] / xf;
        for (int a = 0; a < 9; ++a) {
            feqs[a] += WA[a] * Sp;
            feqms[a] += WA[a] * Sp;
        }
    }

    /* step (3): face macroscopic variables, Eq. 56 */
    double Hf = 0.0, pf = 0.0, mxf = 0.0, myf = 0.0, Cf = 0.0;
    for (int a = 0; a < 9; ++a) {
        Hf += heqs[a];
        pf += feqs[a];
        mxf += EX[a] * feqs[a];
        myf += EY[a] * feqs[a];
        Cf += geqs[a];
    }
    const double uf = mxf / (rho_f * CS2), vf = myf / (rho_f * CS2);

    /* relaxation parameters with the face properties (Sec. 2.1.2, 2.2.3, 2.3.2) */
    const double tau_h = 0.5 + lamf / (rho_f * s->Cref * CS2 * s->dth);
    const double tau_f = 0.5 + muf / (rho_f * CS2 * s->dtf);
    const double tau_g = s->P.tau_g;

    /* steps (3)-(4) and Eq. 53 */
    double Fh = 0.0, Fp = 0.0, Fmx = 0.0, Fmy = 0.0, Fc = 0.0;
    for (int a = 0; a < 9; ++a) {
        const double en = EX[a] * nxv + EY[a] * nyv;
        const double heqf = or_heq(a, Hf, Tf, Cpf, s->Cref, uf, vf);
        const double feqf = or_feq(a, pf, rho_f, uf, vf);
        const double geqf = or_geq(a, Cf, mucf, s->Qg, uf, vf);
        const double hneq = -tau_h * (heqf - heqs[a]);             /* Eq. 13 */
        const double hstar = heqf + (1.0 - 1.0 / (2.0 * tau_h)) * hneq;   /* Eq. 16 */
        const double fneqm = -tau_f * (feqf - feqms[a]);           /* Eq. 35 */
        const double fstar = feqf + (1.0 - 1.0 / (2.0 * tau_f)) * fneqm;  /* Eq. 37, R3 */
        const double gneq = -tau_g * (geqf - geqs[a]);             /* Eq. 44 */
        const double gstar = geqf + (1.0 - 1.0 / (2.0 * tau_g)) * gneq;   /* Eq. 46 */
        Fh += en * hstar;
        Fp += en * feqf;
        Fmx += en * EX[a] * fstar;
        Fmy += en * EY[a] * fstar;
        Fc += en * gstar;
    }
    out[0] = Fh;
    out[1] = Fp;
    out[2] = Fmx;
    out[3] = Fmy;
    out[4] = Fc;
    out[5] = uf * nxv + vf * nyv;
}

/* ------------------------------------------------------------------ */
/* Residual R(W): Eq. 51, 52, 57.                                       */
/* ------------------------------------------------------------------ */

static void residual(or_solver* s, double* const W[5], double* const R[5]) {
    const int nx = s->nx, ny = s->ny;
    prepare(s, W);
    OMP_FOR
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) face_flux(s, 0, i, j, &s->fx[(j * (nx + 1) + i) * 6]);
    OMP_FOR
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) face_flux(s, 1, i, j, &s->fy[(j * nx + i) * 6]);

    const double kv = 1.0 - s->P.s.rho / s->P.l.rho;   /* (1 - rho_s/rho_l) */
    OMP_FOR
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int c = j * nx + i, q = PI(s, i, j);
            const double* fw = &s->fx[(j * (nx + 1) + i) * 6];
            const double* fe = &s->fx[(j * (nx + 1) + i + 1) * 6];
            const double* fs = &s->fy[(j * nx + i) * 6];
            const double* fn = &s->fy[((j + 1) * nx + i) * 6];
            /* Eq. 52: planar V = S = 1; axisymmetric (per radian) V = r_i,
             * S = r_f on the radial faces and r_i on the axial faces. */
            double divF[5], divu;
            if (s->N.axisymmetric) {
                const double rc = i + 0.5, rw = i, re = i + 1.0;
                for (int k = 0; k < 5; ++k) divF[k] = (re * fe[k] - rw * fw[k]) / rc + (fn[k] - fs[k]);
                divu = (re * fe[5] - rw * fw[5]) / rc + (fn[5] - fs[5]);
            } else {
                for (int k = 0; k < 5; ++k) divF[k] = (fe[k] - fw[k]) + (fn[k] - fs[k]);
                divu = (fe[5] - fw[5]) + (fn[5] - fs[5]);   /* R6 */
            }

            const double T = s->prim[P_T][q], Fl = s->prim[P_FL][q], Cp = s->prim[P_CP][q];
            const double rho = s->prim[P_RHO][q], u = s->prim[P_U][q], v = s->prim[P_V][q];
            const double C = s->prim[P_C][q];
            const double D = solid_gate(&s->P, C) * s->dFs[c];   /* solid-volume rate, R1 + R14 */
            const double Fsx = -Fl * C * s->grx[P_MUC][q];   /* F_surf, R13 */
            const double Fsy = -Fl * C * s->gry[P_MUC][q];
            const double Fix = -rho * u * D, Fiy = -rho * v * D;   /* F_IBM (Eq. 27) */
            double FE[5];
            FE[0] = Cp * T * divu;
            FE[1] = u * (s->grx[P_RHO][q] * CS2) + v * (s->gry[P_RHO][q] * CS2) +
                    rho * CS2 * kv * D;
            FE[2] = CS2 * (Fsx + rho * s->P.gx + Fix);
            FE[3] = CS2 * (Fsy + rho * s->P.gy + Fiy);
            FE[4] = C * kv * s->dFs[c];   /* R12: Eq. 40 / 47 as printed, C (1 - rho_s/rho_l) d_t F_s */
            if (s->N.axisymmetric) {
                /* hoop stress of the radial momentum equation, + Pi_thetatheta / r
                 * (reading R24): the pressure advanced over dt_s like the face
                 * pressures, p - dt_s div(rho cs^2 u), and the viscous -2 mu u_r / r */
                const double rc = i + 0.5;
                FE[2] += CS2 * (s->prim[P_P][q] - s->dtf * divF[1] -
                                2.0 * s->prim[P_MU][q] * u / rc) / rc;
            }
            for (int k = 0; k < 5; ++k) R[k][c] = -divF[k] + FE[k];
        }
}

/* Reading R15: momentum projected to zero in the solid part of the cell. */
static void project_solid(or_solver* s) {
    if (!s->P.zero_solid_velocity) return;
    const int n = s->nx * s->ny;
    OMP_FOR
    for (int c = 0; c < n; ++c) {
        double T, Fl;
        or_invert_enthalpy(&s->P, s->W[0][c], s->W[4][c], &T, &Fl);
        const double keep = 1.0 - solid_gate(&s->P, s->W[4][c]) * (1.0 - Fl);
        s->W[2][c] *= keep;
        s->W[3][c] *= keep;
    }
}

/* ------------------------------------------------------------------ */
/* Public API.                                                          */
/* ------------------------------------------------------------------ */

static int bad(char* err, const char* msg) {
    if (err) snprintf(err, 256, "%s", msg);
    return 1;
}

static int check_side(const or_side* sd, int periodic) {
    if (periodic) return sd->thermal == OR_BC_PERIODIC && sd->flow == OR_BC_PERIODIC &&
                         sd->phase == OR_BC_PERIODIC;
    if (sd->thermal != OR_BC_DIRICHLET_T && sd->thermal != OR_BC_ADIABATIC) return 0;
    if (sd->flow != OR_BC_NOSLIP && sd->flow != OR_BC_SYMMETRY && sd->flow != OR_BC_OUTLET)
        return 0;
    if (sd->phase != OR_BC_NOFLUX && sd->phase != OR_BC_WETTING && sd->phase != OR_BC_WETTING_HYST) return 0;
    if (sd->phase == OR_BC_WETTING_HYST &&
        !(sd->theta_rec_deg >= 0.0 && sd->theta_rec_deg <= sd->theta_adv_deg && sd->theta_adv_deg <= 180.0))
        return 0;
    return 1;
}

static double* alloc0(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

or_solver* or_create(int nx, int ny, const or_props* P, const or_bc* B, const or_numerics* N,
                     const or_init* I, char* err) {
    if (nx < 1 || ny < 1) { bad(err, "nx and ny must be >= 1"); return NULL; }
    const int perx = B->xlo.thermal == OR_BC_PERIODIC, pery = B->ylo.thermal == OR_BC_PERIODIC;
    if (!check_side(&B->xlo, perx) || !check_side(&B->xhi, perx) || !check_side(&B->ylo, pery) ||
        !check_side(&B->yhi, pery)) {
        bad(err, "inconsistent boundary conditions");
        return NULL;
    }
    if ((!perx && nx < NG) || (!pery && ny < NG)) { bad(err, "grid too small for walls"); return NULL; }
    const or_phase* ph[3] = {&P->s, &P->l, &P->g};
    for (int k = 0; k < 3; ++k)
        if (!(ph[k]->rho > 0 && ph[k]->cp > 0 && ph[k]->lambda > 0 && ph[k]->mu >= 0)) {
            bad(err, "phase properties must be positive");
            return NULL;
        }
    if (!(P->L >= 0 && P->Ts <= P->Tl && P->sigma >= 0 && P->Mc >= 0 && P->tau_g > 0.5)) {
        bad(err, "invalid latent heat, temperatures, sigma, Mc or tau_g");
        return NULL;
    }
    if (P->sigma > 0 && !(P->xi > 0)) { bad(err, "xi must be > 0"); return NULL; }
    const double dsx[3] = {N->dt_h, N->dt_f, N->dt_g};
    int dts_ok = N->dt > 0 && N->dt_stream > 0 && N->dt_stream <= 0.5;
    for (int k = 0; k < 3; ++k) dts_ok &= dsx[k] == 0.0 || (dsx[k] > 0.0 && dsx[k] <= 0.5);
    if (!dts_ok) {
        bad(err, "need dt > 0 and streaming steps in (0, 0.5]");
        return NULL;
    }
    if (!I || !I->T || !I->C) { bad(err, "initial T and C are required"); return NULL; }
    if (N->axisymmetric && !(B->xlo.thermal == OR_BC_ADIABATIC && B->xlo.flow == OR_BC_SYMMETRY &&
                             B->xlo.phase == OR_BC_NOFLUX)) {
        bad(err, "axisymmetric runs need the axis x = 0 as an adiabatic, symmetric, no-flux side");
        return NULL;
    }

    or_solver* s = (or_solver*)calloc(1, sizeof(or_solver));
    s->nx = nx; s->ny = ny; s->px = nx + 2 * NG; s->py = ny + 2 * NG;
    s->P = *P; s->B = *B; s->N = *N;
    s->Cref = 0.5 * (P->s.cp + P->l.cp);                 /* R16 */
    s->beta = P->sigma > 0 ? 12.0 * P->sigma / P->xi : 0.0;   /* Sec. 2.3.1 */
    s->kappa = 1.5 * P->xi * P->sigma;
    s->dth = N->dt_h > 0 ? N->dt_h : N->dt_stream;
    s->dtf = N->dt_f > 0 ? N->dt_f : N->dt_stream;
    s->dtg = N->dt_g > 0 ? N->dt_g : N->dt_stream;
    s->Qg = P->Mc / ((P->tau_g - 0.5) * s->dtg);   /* M_c = (tau_g - 0.5) Q_g dt_g */
    const size_t n = (size_t)nx * ny, np = (size_t)s->px * s->py;
    for (int k = 0; k < 5; ++k) { s->W[k] = alloc0(n); s->Wn[k] = alloc0(n); s->R[k] = alloc0(n); }
    s->Fsp = alloc0(n); s->dFs = alloc0(n);
    for (int f = 0; f < NPRIM; ++f) { s->prim[f] = alloc0(np); s->grx[f] = alloc0(np); s->gry[f] = alloc0(np); }
    s->fx = alloc0((size_t)(nx + 1) * ny * 6);
    s->fy = alloc0((size_t)nx * (ny + 1) * 6);

    for (size_t c = 0; c < n; ++c) {
        const double C = I->C[c];
        const double H = or_enthalpy_of(P, I->T[c], I->Fl ? I->Fl[c] : 1.0, C);
        double T, Fl;
        or_invert_enthalpy(P, H, C, &T, &Fl);
        const double rho = or_mix(P, C, Fl, 0);
        s->W[0][c] = H;
        s->W[1][c] = I->p ? I->p[c] : 0.0;
        s->W[2][c] = I->u ? rho * CS2 * I->u[c] : 0.0;
        s->W[3][c] = I->v ? rho * CS2 * I->v[c] : 0.0;
        s->W[4][c] = C;
        s->Fsp[c] = 1.0 - Fl;       /* dF_s/dt = 0 on the first step (R14) */
    }
    return s;
}

void or_destroy(or_solver* s) {
    if (!s) return;
    for (int k = 0; k < 5; ++k) { free(s->W[k]); free(s->Wn[k]); free(s->R[k]); }
    free(s->Fsp); free(s->dFs);
    for (int f = 0; f < NPRIM; ++f) { free(s->prim[f]); free(s->grx[f]); free(s->gry[f]); }
    free(s->fx); free(s->fy);
    free(s);
}

int or_step(or_solver* s, long long nsteps) {
    const int n = s->nx * s->ny;
    const double dt = s->N.dt;
    for (long long it = 0; it < nsteps; ++it) {
        /* R14: lagged dF_s/dt from the last two time levels, fixed over the stages */
        OMP_FOR
        for (int c = 0; c < n; ++c) {
            double T, Fl;
            or_invert_enthalpy(&s->P, s->W[0][c], s->W[4][c], &T, &Fl);
            const double Fs = 1.0 - Fl;
            s->dFs[c] = (Fs - s->Fsp[c]) / dt;
            s->Fsp[c] = Fs;
        }
        for (int k = 0; k < 5; ++k) memcpy(s->Wn[k], s->W[k], sizeof(double) * n);
        /* Eq. 58, stage 1 */
        residual(s, s->W, s->R);
        for (int k = 0; k < 5; ++k)
            OMP_FOR
            for (int c = 0; c < n; ++c) s->W[k][c] = s->Wn[k][c] + dt * s->R[k][c];
        project_solid(s);
        /* stage 2 */
        residual(s, s->W, s->R);
        for (int k = 0; k < 5; ++k)
            OMP_FOR
            for (int c = 0; c < n; ++c)
                s->W[k][c] = 0.75 * s->Wn[k][c] + 0.25 * s->W[k][c] + 0.25 * dt * s->R[k][c];
        project_solid(s);
        /* stage 3 */
        residual(s, s->W, s->R);
        for (int k = 0; k < 5; ++k)
            OMP_FOR
            for (int c = 0; c < n; ++c)
                s->W[k][c] = (1.0 / 3.0) * s->Wn[k][c] + (2.0 / 3.0) * s->W[k][c] +
                             (2.0 / 3.0) * dt * s->R[k][c];
        project_solid(s);
        s->t += dt;
        s->step += 1;
        for (int k = 0; k < 5; ++k)
            for (int c = 0; c < n; ++c)
                if (!isfinite(s->W[k][c])) return 4;
    }
    return 0;
}

void or_diagnostics(const or_solver* s, or_diag* d) {
    const int n = s->nx * s->ny;
    memset(d, 0, sizeof(*d));
    d->step = s->step;
    d->t = s->t;
    for (int c = 0; c < n; ++c) {
        const double H = s->W[0][c], C = s->W[4][c];
        const double w = s->N.axisymmetric ? (c % s->nx) + 0.5 : 1.0;   /* cell volume */
        for (int k = 0; k < 5; ++k)
            if (!isfinite(s->W[k][c])) d->nonfinite = 1;
        double T, Fl;
        or_invert_enthalpy(&s->P, H, C, &T, &Fl);
        const double rho = or_mix(&s->P, C, Fl, 0);
        d->mass += w * rho;
        d->enthalpy += w * H;
        d->phase_vol += w * C;
        d->solid_vol += w * clamp01(C) * (1.0 - Fl);
        const double sp = sqrt(s->W[2][c] * s->W[2][c] + s->W[3][c] * s->W[3][c]) / (rho * CS2);
        if (sp > d->max_speed) d->max_speed = sp;
    }
    const double base = s->N.axisymmetric ? 0.5 * (double)s->nx * s->nx : (double)s->ny;
    d->front_pos = d->solid_vol / base;
    d->interface_pos = d->phase_vol / base;
}

void or_get_state(const or_solver* s, double* H, double* p, double* mx, double* my, double* C,
                  double* Fsp) {
    const size_t b = sizeof(double) * (size_t)s->nx * s->ny;
    double* dst[5] = {H, p, mx, my, C};
    for (int k = 0; k < 5; ++k)
        if (dst[k]) memcpy(dst[k], s->W[k], b);
    if (Fsp) memcpy(Fsp, s->Fsp, b);
}

void or_set_state(or_solver* s, const double* H, const double* p, const double* mx,
                  const double* my, const double* C, const double* Fsp, double t,
                  long long step) {
    const size_t b = sizeof(double) * (size_t)s->nx * s->ny;
    const double* src[5] = {H, p, mx, my, C};
    for (int k = 0; k < 5; ++k)
        if (src[k]) memcpy(s->W[k], src[k], b);
    if (Fsp) memcpy(s->Fsp, Fsp, b);
    s->t = t;
    s->step = step;
}

void or_get_primitives(or_solver* s, double* T, double* Fl, double* u, double* v) {
    derive_interior(s, s->W);
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            const int c = j * s->nx + i, q = PI(s, i, j);
            if (T) T[c] = s->prim[P_T][q];
            if (Fl) Fl[c] = s->prim[P_FL][q];
            if (u) u[c] = s->prim[P_U][q];
            if (v) v[c] = s->prim[P_V][q];
        }
}

void or_face_flux(or_solver* s, int dir, int i, int j, double* out) {
    prepare(s, s->W);
    face_flux(s, dir, i, j, out);
}

void or_residual(or_solver* s, double* out) {
    const size_t n = (size_t)s->nx * s->ny;
    double* R[5];
    for (int k = 0; k < 5; ++k) R[k] = out + k * n;
    residual(s, s->W, R);
}

void or_get_muc(or_solver* s, double* muc) {
    prepare(s, s->W);
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) muc[j * s->nx + i] = s->prim[P_MUC][PI(s, i, j)];
}

int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
