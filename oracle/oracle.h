/*
 * oracle.h -- plain, slow FP64 CPU oracle of the EULBFS explicit time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This program exists so that the CUDA path can be
 * checked against something obviously correct.  Only the test suite, the smoke
 * entry point and the CPU-baseline leg of the benchmark may load it; the
 * product path never does, and nothing here is shared with the CUDA sources
 * (no common headers, helpers or tables).
 *
 * Method: Zhou, Yang, Wang, Wu, Niu, "An Enthalpy-Based Unified Lattice
 * Boltzmann Flux Solver for Liquid Solidification" (arXiv 2507.03366).
 * The oracle follows the procedure of Sec. 2.5, steps (1)-(7), literally:
 * for every cell face and every D2Q9 direction alpha it reconstructs the
 * macroscopic variables at x_f - e_alpha*dt_s (Eq. 54), evaluates the
 * equilibria (Eq. 9, 29, 33, 42), forms the face variables (Eq. 56), the
 * non-equilibrium parts and the star distributions (Eq. 13/16, 35/37, 44/46),
 * takes the flux moments (Eq. 53), adds the cell sources (Eq. 51) and
 * advances with SSP-RK3 (Eq. 58), inverting enthalpy with Eq. 5-6.
 * Where the paper is silent or inconsistent, the reading taken is stated at
 * the code that implements it, labelled R1, R2, ... so that the CUDA path
 * can name the same reading.
 *
 * Units: lattice units, dx = dy = 1, lattice speed c = 1, cs^2 = 1/3.
 * Cell (i, j) has its centre at (i + 1/2, j + 1/2); arrays are row-major
 * with x fastest: index = j*nx + i.
 */
#ifndef EULBFS_ORACLE_H
#define EULBFS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double rho, mu, lambda, cp; } or_phase;

/* Physical properties of the three phases and of the phase-field model. */
typedef struct {
    or_phase s, l, g;   /* solid, liquid, gas (Eq. 7) */
    double L;           /* latent heat (Eq. 5-6) */
    double Ts, Tl;      /* solidus and liquidus temperatures, Ts <= Tl */
    double sigma, xi;   /* interfacial tension, interface thickness (Sec. 2.3.1) */
    double Mc;          /* mobility M_c (Eq. 39) */
    double tau_g;       /* phase-field relaxation parameter (Sec. 2.3.2) */
    double gx, gy;      /* gravitational acceleration; G = rho*g (Eq. 51) */
    int zero_solid_velocity; /* reading R15: project momentum to zero in solid */
    /* 0: reading R1 (properties and the volume-change sources gated by
     * C~ = clamp(C, 0, 1), uniform latent heat).  1: Eq. 5-7 as printed:
     * F_s = 1 - F_l of every cell (gas included) enters Eq. 7 and the sources,
     * H_s = C_p,s T_s and H_l = C_p,l T_l + L (C~ still bounds the mixture). */
    int literal_eq7;
} or_props;

enum {
    OR_BC_PERIODIC = 0,
    OR_BC_DIRICHLET_T = 1, /* thermal: T = Tw on the wall face */
    OR_BC_ADIABATIC = 2,   /* thermal: zero normal gradient of T */
    OR_BC_NOSLIP = 3,      /* flow: u = 0 on the wall face */
    OR_BC_SYMMETRY = 4,    /* flow: normal u = 0, zero gradient of tangential u */
    OR_BC_OUTLET = 5,      /* flow: p = 0 on the face, zero gradient of u */
    OR_BC_NOFLUX = 6,      /* phase: zero normal gradient of C and mu_c */
    OR_BC_WETTING = 7,     /* phase: contact angle theta (reading R11) */
    OR_BC_WETTING_HYST = 8 /* phase: contact angle within [theta_rec, theta_adv] (reading R25) */
};

/* theta_deg: (equilibrium) contact angle; theta_adv_deg >= theta_rec_deg bound
 * the apparent angle for OR_BC_WETTING_HYST. */
typedef struct { int thermal, flow, phase; double Tw, theta_deg, theta_adv_deg, theta_rec_deg; } or_side;
typedef struct { or_side xlo, xhi, ylo, yhi; } or_bc;

typedef struct {
    double dt;        /* Runge-Kutta time step Delta t (Eq. 58) */
    double dt_stream; /* streaming step delta t (Sec. 2.5 step 1), 0 < dt_stream <= 0.5 */
    int axisymmetric; /* 1: x is the radius r (axis at x = 0), y the axial coordinate z */
    /* per-distribution streaming steps of h (enthalpy), f (flow) and g (phase
     * field), each in (0, 0.5]; 0 means dt_stream (reading R26) */
    double dt_h, dt_f, dt_g;
} or_numerics;

/* Initial primitive fields, host arrays of nx*ny doubles, copied at create.
 * Fl is the initial liquid fraction, used only where Ts <= T <= Tl. */
typedef struct { const double *T, *Fl, *C, *u, *v, *p; } or_init;

/* Integrals over the domain; in axisymmetric runs every cell is weighted by
 * its radius r_i (volumes per radian). */
typedef struct {
    long long step;
    double t;
    double mass;          /* sum of rho over cells (dx = 1) */
    double enthalpy;      /* sum of H */
    double phase_vol;     /* sum of C */
    double solid_vol;     /* sum of clamp(C)*F_s */
    double front_pos;     /* solid_vol / (ny, or sum of r_i over a row) */
    double interface_pos; /* phase_vol / (ny, or sum of r_i over a row) */
    double max_speed;     /* max |u| */
    int nonfinite;        /* 1 if any conserved value is NaN or Inf */
} or_diag;

typedef struct or_solver or_solver;

/* Returns NULL and writes a message to err (if non-NULL, 256 bytes) on bad input. */
or_solver* or_create(int nx, int ny, const or_props* P, const or_bc* B,
                     const or_numerics* N, const or_init* I, char* err);
void or_destroy(or_solver* s);
int or_step(or_solver* s, long long n);   /* returns 0, or 4 on a non-finite state */
void or_diagnostics(const or_solver* s, or_diag* d);

/* Conserved state W = (H, p, rho cs^2 u, rho cs^2 v, C) (Eq. 49), each nx*ny;
 * Fsp = F_s of the previous step.  Any pointer may be NULL. */
void or_get_state(const or_solver* s, double* H, double* p, double* mx, double* my,
                  double* C, double* Fsp);
void or_set_state(or_solver* s, const double* H, const double* p, const double* mx,
                  const double* my, const double* C, const double* Fsp,
                  double t, long long step);
/* Primitive fields of the current state: T, F_l, u, v (each nx*ny, may be NULL). */
void or_get_primitives(or_solver* s, double* T, double* Fl, double* u, double* v);

/* ---- pieces exposed for the pin tests ---- */
double or_heq(int a, double H, double T, double Cp, double Cref, double u, double v);
double or_feq(int a, double p, double rho, double u, double v);
double or_feqm(int a, double p, double rho_face, double u, double v);
double or_geq(int a, double C, double muc, double Qg, double u, double v);
void or_invert_enthalpy(const or_props* P, double H, double C, double* T, double* Fl);
double or_enthalpy_of(const or_props* P, double T, double Fl, double C);
/* Mixture property (Eq. 7, reading R1): which = 0 rho, 1 mu, 2 lambda, 3 cp. */
double or_mix(const or_props* P, double C, double Fl, int which);
/* Flux through face (dir 0: x-face at x = i between cells (i-1,j),(i,j);
 * dir 1: y-face at y = j between (i,j-1),(i,j)) for the current state:
 * out[0..4] = F.n (Eq. 53), out[5] = u_f.n (Eq. 56). */
void or_face_flux(or_solver* s, int dir, int i, int j, double* out);
/* R(W) of Eq. 57 for the current state, out = 5 arrays of nx*ny back to back. */
void or_residual(or_solver* s, double* out);
/* Chemical potential mu_c (Sec. 2.3.1, reading R5) of the current state, nx*ny. */
void or_get_muc(or_solver* s, double* muc);

/* Host threads for the loops whose iterations are independent (OpenMP
 * builds; n <= 0 keeps the current count).  Returns the count in use (1
 * without OpenMP).  Results do not depend on it. */
int or_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
