/*
 * eulbfs.h -- C ABI of the GB300 (sm_103a) EULBFS explicit time step.
 *
 * Method: Zhou, Yang, Wang, Wu, Niu, "An Enthalpy-Based Unified Lattice
 * Boltzmann Flux Solver for Liquid Solidification", arXiv 2507.03366.
 * One call of eulbfs_step advances every resident domain by whole time
 * steps of Sec. 2.5: face fluxes of H, p, rho cs^2 u and C reconstructed from
 * local D2Q9 equilibria (Eq. 54-56, 13/16, 35/37, 44/46, 53), cell sources
 * (Eq. 51), SSP-RK3 (Eq. 58) and enthalpy inversion (Eq. 5-7).
 *
 * Units are lattice units: cell size 1, lattice speed 1, cs^2 = 1/3 and by
 * default the streaming step dt_s = 0.5, so the surrounding points
 * x_f - e_a dt_s of a face lie on the neighbouring cell centres and face
 * midpoints (Sec. 2.5 step (1): they must stay inside the two cells of the
 * face).  Each distribution's step can be set in eulbfs_numerics.
 * Arrays are row-major with x fastest: element (i, j) is at j*nx + i.
 *
 * Conventions for every call:
 *  - The return value is an eulbfs_status; EULBFS_OK is 0.  On failure a
 *    message is available from eulbfs_last_error() (thread-local).
 *  - Host arrays passed in are read during the call only (copied); host
 *    arrays passed out are owned by the caller and must hold nx*ny doubles.
 *  - All device memory is owned by the solver and released by
 *    eulbfs_destroy.  There is no CPU fallback: without a usable CUDA device
 *    creation fails with EULBFS_ECUDA.
 *  - A solver is not thread-safe; use one host thread per solver.
 */
#ifndef EULBFS_H
#define EULBFS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EULBFS_OK = 0,
    EULBFS_EINVAL = 1,     /* invalid argument or physically invalid parameters */
    EULBFS_ENOMEM = 2,     /* device or host allocation failed */
    EULBFS_ECUDA = 3,      /* CUDA runtime error (no device, launch failure, ...) */
    EULBFS_ENONFINITE = 4, /* the state of some domain became NaN or Inf */
    EULBFS_ETIMEOUT = 5,   /* a bounded device wait gave up (the stage kernel waits about a second
                            * for each input tile it copies by TMA, then stops and reports this) */
    EULBFS_EBUSY = 6       /* a domain does not fit in the solver's memory budget */
} eulbfs_status;

typedef enum {
    EULBFS_FP64 = 0,  /* all state and arithmetic in FP64 */
    EULBFS_FP32C = 1  /* FP32 arithmetic; H and C carried as compensated hi/lo FP32 pairs */
} eulbfs_precision;

/* Boundary-condition kinds, per field family and side (Sec. 3.1-3.5).
 * A side is periodic only if all three kinds are EULBFS_BC_PERIODIC, and then
 * so is the opposite side. */
typedef enum {
    EULBFS_BC_PERIODIC = 0,
    EULBFS_BC_DIRICHLET_T = 1, /* thermal: T = Tw on the wall face */
    EULBFS_BC_ADIABATIC = 2,   /* thermal: zero normal gradient */
    EULBFS_BC_NOSLIP = 3,      /* flow: u = 0 on the wall face */
    EULBFS_BC_SYMMETRY = 4,    /* flow: zero normal velocity, free slip */
    EULBFS_BC_OUTLET = 5,      /* flow: p = 0 on the face, zero gradient of u */
    EULBFS_BC_NOFLUX = 6,      /* phase field: zero normal gradient of C and mu_c */
    EULBFS_BC_WETTING = 7,     /* phase field: contact angle theta_deg */
    /* phase field: contact-angle hysteresis.  The apparent angle at each wall
     * position, read from the two wall layers (cos = dC/dn_out / |grad C|),
     * is clamped to [theta_rec_deg, theta_adv_deg] and used as the contact
     * angle: inside that window the contact line is pinned, outside it the
     * nearer limit applies (Sec. 3.5 quotes theta_adv and theta_r; the paper
     * gives no model, this is one).  theta_deg is used where the wall layers
     * carry no interface. */
    EULBFS_BC_WETTING_HYST = 8
} eulbfs_bc_kind;

typedef struct { int nx, ny; } eulbfs_grid;   /* cells; nx, ny >= 2 on walled axes */

/* Properties of one phase: density, dynamic viscosity, thermal conductivity,
 * specific heat (all > 0 except mu >= 0). */
typedef struct { double rho, mu, lambda, cp; } eulbfs_phase;

typedef struct {
    eulbfs_phase s, l, g;  /* solid, liquid, gas; mixed by Eq. 7 */
    double L;              /* latent heat (Eq. 5-6), >= 0 */
    double Ts, Tl;         /* solidus <= liquidus temperature */
    double sigma, xi;      /* interfacial tension, interface thickness (Sec. 2.3.1) */
    double Mc;             /* mobility M_c = (tau_g - 0.5) Q_g dt_s (Sec. 2.3.2) */
    double tau_g;          /* phase-field relaxation parameter, > 0.5 */
    double gx, gy;         /* gravitational acceleration, G = rho g (Eq. 51) */
    int zero_solid_velocity; /* 1: momentum of the solid part projected to zero */
    /* 0 (default): Eq. 5-7 gated by the phase field, C~ = clamp(C, 0, 1):
     * gamma = C~ [F_s gamma_s + F_l gamma_l] + (1 - C~) gamma_g, heat
     * capacities of both branches of Eq. 6 mixed the same way, and C~ F_s as
     * the solid fraction of the volume-change sources (Eq. 26, 27) and of the
     * solid projection.  Without the gate, Eq. 7 with F_s from Eq. 5 turns gas
     * colder than T_s into solid.  1: Eq. 5-7 exactly as printed:
     * gamma = F_s gamma_s + (1 - F_s) C~ gamma_l + (1 - F_s)(1 - C~) gamma_g,
     * H_s = C_p,s T_s, H_l = C_p,l T_l + L, and F_s itself in those sources
     * (C~ still bounds the mixture, so an overshoot of C cannot make rho <= 0). */
    int literal_eq7;
} eulbfs_props;

/* Tw: wall temperature (DIRICHLET_T).  theta_deg: contact angle (WETTING),
 * or the angle where no interface touches the wall (WETTING_HYST).
 * theta_adv_deg, theta_rec_deg: the hysteresis window of WETTING_HYST,
 * 0 <= theta_rec_deg <= theta_adv_deg <= 180 (EINVAL otherwise); ignored by
 * the other kinds. */
typedef struct { int thermal, flow, phase; double Tw, theta_deg, theta_adv_deg, theta_rec_deg; } eulbfs_side;
typedef struct { eulbfs_side xlo, xhi, ylo, yhi; } eulbfs_bc;

typedef struct {
    double dt;  /* Runge-Kutta time step Delta t (Eq. 58), chosen by the caller's CFL bound */
    /* 0: planar 2-D.  1: axisymmetric (r, z): x is the radius r with the axis
     * at x = 0 and y the axial coordinate.  The finite-volume balance (Eq. 52)
     * then uses per-radian cell volumes r_i and face areas r_f (radial faces)
     * or r_i (axial faces), adds the hoop term cs^2 (p - 2 mu u_r / r) / r to
     * the radial momentum, takes the axisymmetric Laplacian in mu_c and the
     * axisymmetric mass source -rho cs^2 u_r / r in the face pressure.  The
     * xlo side must be ADIABATIC / SYMMETRY / NOFLUX (EINVAL otherwise). */
    int axisymmetric;
    /* Streaming steps of the enthalpy (h), flow (f) and phase-field (g)
     * distributions in lattice units (Sec. 2.5 step (1)): each takes its
     * surrounding points at x_f - e_a dt and its relaxation time from its own
     * step.  0 selects 0.5, where the points fall on cell centres and face
     * midpoints (the fast path); any value must lie in (0, 0.5] (EINVAL
     * otherwise).  Smaller steps carry less numerical dissipation. */
    double dt_stream_h, dt_stream_f, dt_stream_g;
} eulbfs_numerics;

/* Initial primitive fields: host arrays of nx*ny doubles, copied at creation.
 * T and C are required; Fl (initial liquid fraction, used only where
 * Ts <= T <= Tl), u, v, p may be NULL (1, 0, 0, 0). */
typedef struct { const double *T, *Fl, *C, *u, *v, *p; } eulbfs_init;

/* One domain of a batch. */
typedef struct {
    eulbfs_grid grid;
    eulbfs_props props;
    eulbfs_bc bc;
    eulbfs_numerics num;
    eulbfs_init init;
} eulbfs_domain;

/* Host output of eulbfs_fields; any pointer may be NULL (skipped). */
typedef struct { double *H, *T, *Fl, *C, *p, *u, *v; } eulbfs_fields_out;

/* Global diagnostics of one domain, accumulated in FP64 on the device
 * (fixed-order reduction, bitwise reproducible).  Sums are over cell volumes:
 * 1 per cell in planar domains, r_i = i + 1/2 (per radian) in axisymmetric
 * ones. */
typedef struct {
    long long step;       /* completed time steps */
    double t;             /* simulated time = step * dt */
    double mass;          /* sum of rho */
    double enthalpy;      /* sum of H */
    double phase_vol;     /* sum of C */
    double solid_vol;     /* sum of clamp(C,0,1) * F_s */
    double front_pos;     /* solid_vol / ny (axisymmetric: / (nx^2 / 2)): flat-front solid thickness */
    double interface_pos; /* phase_vol / ny (axisymmetric: / (nx^2 / 2)): flat condensed thickness */
    double max_speed;     /* max |u| */
    int nonfinite;        /* 1 if any state value is NaN or Inf */
} eulbfs_diag;

typedef struct eulbfs_solver eulbfs_solver;

/* Create a solver holding one domain: the problem as Sec. 3 states each
 * case -- a uniform grid (Sec. 3.1-3.5), the three phases' properties
 * (Tables 1 and 3: rho, mu, lambda, C_p; L, T_s, T_l, sigma, xi, M_c), the
 * boundary conditions per field and side (Sec. 3.1-3.5), the time steps
 * (Sec. 2.4 after Eq. 58, Sec. 2.5 step (1)) and the initial fields (e.g.
 * Eq. 61-62), from which H = C_p T + L F_l (Eq. 5-7) is formed on the device.
 * stream is a cudaStream_t the solver enqueues all its work on, or NULL for a
 * stream the solver owns.
 * Errors: EINVAL (bad sizes or parameters: tau <= 0.5, rho/lambda/cp <= 0,
 * inconsistent periodic sides, dt <= 0), ECUDA, ENOMEM. */
int eulbfs_create(const eulbfs_grid* grid, const eulbfs_props* props, const eulbfs_bc* bc,
                  const eulbfs_numerics* num, const eulbfs_init* init, int precision,
                  void* stream, eulbfs_solver** out);

/* Create a solver holding n >= 0 domains of any sizes and parameters that
 * advance together (no counterpart in the paper, which runs one domain at a
 * time; each domain is the problem eulbfs_create describes): every stage of
 * every domain runs in one launch over a
 * work list of strip segments (many uneven domains).  n = 0 creates an empty
 * solver that eulbfs_add_domain fills (a serving loop). */
int eulbfs_batch_create(int n, const eulbfs_domain* domains, int precision, void* stream,
                        eulbfs_solver** out);

/* Limit the device memory the solver may hold (bytes, 0 = unlimited).
 * eulbfs_add_domain fails with EBUSY instead of exceeding it. */
int eulbfs_set_memory_budget(eulbfs_solver* s, unsigned long long bytes);

/* Bytes of device memory a domain of this size needs in this precision. */
unsigned long long eulbfs_domain_bytes(int nx, int ny, int precision);

/* Add a domain to a live solver (continuous batching).  max_steps > 0 stops
 * the domain after that many steps; 0 = no limit.  *slot receives its index.
 * Errors: EINVAL, EBUSY (memory budget), ENOMEM, ECUDA. */
int eulbfs_add_domain(eulbfs_solver* s, const eulbfs_domain* d, long long max_steps, int* slot);

/* Add one domain split along y into k slabs that advance as k domains of
 * this solver (the paper has no counterpart: it is the decomposition a
 * domain spread over several devices needs, here within one device).  Slab i
 * holds rows [i ny / k, (i + 1) ny / k) (integer division), at least 8 rows
 * each, and 3 halo rows on each side it shares with a neighbour (both sides
 * if y is periodic): the ghost width of the stencil (two rows for the
 * gradients, a third for the Laplacian of C in mu_c).  After every
 * Runge-Kutta stage the solver copies each slab's 3 outermost interior rows
 * into its neighbours' halo rows, so every slab sees the rows the undivided
 * domain would; results are bit for bit those of the undivided domain.
 * slots: caller array of k slot indices (bottom slab first); each slab is
 * read back (fields, state, diagnostics) as a domain of ny_i rows.  Remove
 * the slabs of a split domain together.  k = 1 adds the domain whole.
 * Errors: EINVAL (k < 1, ny < 8 k, or the domain's own errors), EBUSY,
 * ENOMEM, ECUDA. */
int eulbfs_add_split_domain(eulbfs_solver* s, const eulbfs_domain* d, int k, long long max_steps, int* slots);

/* Remove a domain and release its memory; its slot index is not reused. */
int eulbfs_remove_domain(eulbfs_solver* s, int slot);

/* Number of slots ever created (removed slots included). */
int eulbfs_num_slots(const eulbfs_solver* s);

/* Steps completed and steps left (-1 = unlimited) of a domain. */
int eulbfs_domain_progress(const eulbfs_solver* s, int slot, long long* done, long long* left);

/* Advance every active domain by n >= 0 time steps of Sec. 2.5, steps
 * (1)-(7): per Runge-Kutta stage of Eq. 58, the face fluxes of Eq. 53 from
 * the reconstruction (Eq. 54), the surrounding and face equilibria (Eq. 9,
 * 29, 33, 42, 56) and the star distributions (Eq. 13/16, 35/37, 44/46), the
 * sources of Eq. 51 and the residual of Eq. 52; then Eq. 5-7 on the new state
 * (a domain with a step limit stops at it).  Work is enqueued on the solver's stream and the call
 * returns without waiting; launch errors are reported, a non-finite state is
 * reported by eulbfs_sync / eulbfs_diagnostics / eulbfs_fields. */
int eulbfs_step(eulbfs_solver* s, long long n);

/* Wait for the solver's stream.  Returns ENONFINITE if a stage of any
 * domain produced a NaN or Inf since the solver was created, ETIMEOUT if a
 * stage kernel gave up waiting for an input tile (its results are then not
 * valid). */
int eulbfs_sync(eulbfs_solver* s);

/* Slots of the live domains whose own state became NaN or Inf (their
 * per-domain flag; other domains are unaffected and keep stepping).
 * Synchronises the solver's stream.  Up to `cap` slot indices are written to
 * the caller-owned `slots`; *count receives the number of such domains (it
 * may exceed cap).  A serving loop calls it after each batch of steps to
 * retire a diverged case at once instead of at its step limit.
 * Errors: EINVAL (null solver or count, cap < 0, slots NULL with cap > 0),
 * ENOMEM, ECUDA. */
int eulbfs_nonfinite_domains(eulbfs_solver* s, int* slots, int cap, int* count);

/* Copy primitive fields of domain `slot` to caller-owned host arrays
 * (synchronises the solver's stream): H and C from the state W (Eq. 49), T
 * and F_l by Eq. 5-6, u = W_3 / (rho cs^2), v = W_4 / (rho cs^2) with rho from
 * Eq. 7, and p.  Returns ENONFINITE (after copying) if
 * this domain produced a NaN or Inf; other domains do not affect it. */
int eulbfs_fields(eulbfs_solver* s, int slot, const eulbfs_fields_out* out);

/* Conserved state W = (H, p, rho cs^2 u, rho cs^2 v, C) (Eq. 49), the
 * previous-step solid fraction F_s^{n-1}, time and step, as doubles.  Exact in
 * FP64; in FP32C H and C are the hi + lo pairs rounded to double (a pair can
 * carry more than 53 significant bits), so a round trip perturbs them by at
 * most 2^-53 relative.  Any pointer may be NULL.  set_state sets the step
 * counter to `step` (t is recomputed as step * dt). */
int eulbfs_get_state(eulbfs_solver* s, int slot, double* H, double* p, double* mx, double* my,
                     double* C, double* Fs_prev, double* t, long long* step);
int eulbfs_set_state(eulbfs_solver* s, int slot, const double* H, const double* p,
                     const double* mx, const double* my, const double* C,
                     const double* Fs_prev, double t, long long step);

/* Bytes of a domain's raw checkpoint: its state planes and F_s^{n-1} in the
 * solver's working precision. */
unsigned long long eulbfs_checkpoint_bytes(const eulbfs_solver* s, int slot);
/* Bitwise-exact checkpoint of domain `slot` into / from a caller-owned host
 * buffer of eulbfs_checkpoint_bytes bytes (same precision and grid size on
 * load; EINVAL otherwise).  *step receives / step sets the step counter. */
int eulbfs_save(eulbfs_solver* s, int slot, void* buf, unsigned long long bytes, long long* step);
int eulbfs_load(eulbfs_solver* s, int slot, const void* buf, unsigned long long bytes, long long step);

/* FP64 diagnostics of domain `slot` (synchronises the solver's stream);
 * ENONFINITE (with d filled) if this domain's state is not finite.  They are
 * the quantities Sec. 3 measures: the front position of the Neumann problem
 * (Sec. 3.1, Eq. 59-60) and the interface position of the expansion law
 * H_f = (rho_l / rho_s) H_0 (Sec. 3.2) as flat-layer heights of the solid
 * and condensed volumes, those volumes themselves (Table 2, Table 5), the
 * total mass, enthalpy and largest speed. */
int eulbfs_diagnostics(eulbfs_solver* s, int slot, eulbfs_diag* d);

/* Number of kernels the solver launches per time step of the current batch:
 * one whole-step launch (eulbfs_set_whole_step; an eulbfs_step of several
 * steps runs up to 16 of them in one launch); three stage launches with it
 * off; and while a split domain's slabs are active, three stage launches
 * with a halo copy after each. */
int eulbfs_launches_per_step(const eulbfs_solver* s);

/* Kernel launches of the time-stepping path (stage kernels and halo copies,
 * including those replayed from captured graphs) since the solver was
 * created; 0 for a null solver. */
unsigned long long eulbfs_launch_count(const eulbfs_solver* s);

/* Whole-step launches (on = 1, the default) or one launch per Runge-Kutta
 * stage (on = 0).  A whole-step launch runs the work items of stage 1, then
 * stage 2, then stage 3 (Eq. 58) of one time step, or of up to 16 steps in
 * sequence (an eulbfs_step of several steps, up to the next domain's step
 * limit), each item as soon as the items of the previous stage whose output
 * it reads (its strip and the strips beside it, its rows and 4 rows beyond)
 * are done, so one stage's last items overlap the next stage's first.  Batches with split domains always launch per
 * stage (their halo copies run between stages).  Results are the same bit
 * for bit.  A wait for a neighbour's item is bounded (about a second) and
 * reports EULBFS_ETIMEOUT like a tile wait.  Errors: EINVAL. */
int eulbfs_set_whole_step(eulbfs_solver* s, int on);

/* Capture eulbfs_step's per-step launches in a CUDA graph of `steps_per_graph`
 * steps (0 disables); replays are used when n is a multiple of it. */
int eulbfs_use_graphs(eulbfs_solver* s, int steps_per_graph);

/* Work-item shape of the stage kernel: each item is a 31-column strip of a
 * domain and a run of its rows.  `rows` (a multiple of 8 in [8, 1024];
 * 0 = 64) is the target height: a domain of ny rows is cut into
 * round(ny / rows) runs (at least one) of nearly equal height, in whole
 * 8-row chunks.  The persistent CTAs claim items from a counter, tallest
 * first.  Results do not depend on it. */
int eulbfs_set_tile(eulbfs_solver* s, int rows);

/* Diagnostics of a caller-held domain state that allocates no device memory.
 * The paper has no counterpart to this call; it exists for callers that
 * cannot let a library call cudaMalloc or cudaFree: programs whose device
 * memory is fully committed to another framework's allocator, and loops that
 * cannot afford cudaFree's device-wide synchronisation or a driver allocation
 * in the middle of a step.  It computes what eulbfs_diagnostics computes
 * for a planar domain (every cell volume 1; it is not told the geometry, so
 * for an axisymmetric domain the sums are unweighted).
 *   state: device pointer to the conserved-state planes of one domain in the
 *          working precision, nx*ny values per plane, planes back to back:
 *          FP64 5 planes of doubles (H, p, rho cs^2 u, rho cs^2 v, C); FP32C
 *          7 planes of floats (H_hi, H_lo, p, m_x, m_y, C_hi, C_lo), e.g. the
 *          first part of an eulbfs_save buffer copied to the device.
 *   props: host struct of the domain's properties (used for rho and F_s).
 *   out:   device pointer to 6 doubles: mass, enthalpy, phase_vol, solid_vol,
 *          max_speed, nonfinite (1.0 or 0.0).
 *   stream: cudaStream_t to enqueue on (NULL: the legacy default stream);
 *          the call returns after enqueueing.
 * Limit: nx*ny <= EULBFS_NOALLOC_MAX_CELLS; larger domains return EINVAL.
 * The block partials live in one fixed 48 KiB device array inside the
 * library (1024 x 6 doubles), held on every GPU that loads the library until
 * the process exits and shared by all calls: each call overwrites the
 * partials it uses, so nothing needs clearing, but calls that overlap on the
 * GPU (different streams or host threads) race on it and must be serialised.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again
 * when the device's context has changed (after cudaDeviceReset); make that
 * first call before any stream capture. */
#define EULBFS_NOALLOC_MAX_CELLS 2097152
int eulbfs_diagnostics_noalloc(int precision, const void* state, int nx, int ny,
                               const eulbfs_props* props, double* out, void* stream);

/* Pick the work-item height of the current batch by timing each candidate
 * (32, 48, 64, 96, 128, 160, 192, 256 rows) over steps_per_candidate steps on
 * the solver's stream, in two rounds, and keeping the candidate with the
 * fastest of its two timings (*best_ms_per_step).  The timed steps are real
 * steps of every active domain (results do not depend on the height), so the
 * simulation advances by 2 * 8 * (steps_per_candidate + 1) steps.  Synchronises the
 * stream.  EULBFS_EINVAL for a null solver or steps_per_candidate < 1; a
 * failing step returns its error and leaves the height unchanged. */
int eulbfs_autotune(eulbfs_solver* s, int steps_per_candidate, int* best_rows, float* best_ms_per_step);

/* Test hook for the bounded device waits (no counterpart in the paper).
 * With on = 1 every input-tile barrier of the stage kernel expects 16 bytes
 * more than its copy delivers, so every tile wait runs out after its bound
 * (about a second of SM clocks, twice: the wait and the wait for the copy in
 * flight) and the kernel stops; eulbfs_sync then returns ETIMEOUT and the
 * CUDA context stays usable.  on = 0 (the default) restores normal waits.
 * Only domains whose state buffers get tensor maps (nx a multiple of 4 in
 * FP32C) and interior work items wait on tiles.  With on = 2 the tiles are
 * normal but no work item of a whole-step launch (eulbfs_set_whole_step)
 * marks itself done, so every item of stages 2 and 3 waits out its bound
 * for the items it reads and the kernel stops with the same ETIMEOUT (both
 * precisions).  Errors: EINVAL. */
int eulbfs_set_tile_wait_probe(eulbfs_solver* s, int on);

/* The candidates the last eulbfs_autotune of this solver timed: up to `cap`
 * heights (rows) and their best milliseconds per step; *n receives how many
 * it timed (0 before any autotune).  Errors: EINVAL (null solver or n,
 * cap < 0, null arrays with cap > 0). */
int eulbfs_autotune_report(const eulbfs_solver* s, int* rows, float* ms_per_step, int cap, int* n);

void eulbfs_destroy(eulbfs_solver* s);

/* Message of the last failed call on this thread ("" if none). */
const char* eulbfs_last_error(void);

/* Library version string. */
const char* eulbfs_version(void);

#ifdef __cplusplus
}
#endif
#endif
