// eulbfs_internal.h -- declarations shared by the kernel and host translation
// units of libeulbfs (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eulbfs {

constexpr int kHalo = 3;     // C halo; every other field needs 2 (gradient ring + its neighbours)
constexpr int kMaxDomains = 1 << 20;

// Sides in descriptor arrays.
enum { XLO = 0, XHI = 1, YLO = 2, YHI = 3 };

// Per-domain descriptor, stored in device memory.  Physical constants are in
// double; the kernels convert them to their working precision.
struct DomainDesc {
    int nx, ny;
    int strips, segs;        // work items of this domain along x and y
    int per_x, per_y;        // periodic axes
    int bc_t[4], bc_f[4], bc_c[4];  // thermal, flow, phase kind per side
    int zero_solid_velocity;
    int axi;                 // 1: axisymmetric (r, z), x = r with the axis at x = 0
    int literal_eq7;         // 1: Eq. 5-7 as printed instead of reading R1
    // A slab of a domain split along y: its planes hold hlo halo rows below
    // and hhi above its ny interior rows (0 or kHalo each); halo rows are
    // copies of the neighbouring slab's rows, not boundary ghosts.
    int hlo, hhi;
    double Tw[4];            // wall temperature per side (Dirichlet)
    double wet[4];           // 4 cos(theta) / xi per side (wetting)
    double cos_adv[4], cos_rec[4];   // hysteresis window per side (WETTING_HYST)
    double four_over_xi;
    double rho[3], mu[3], lam[3], cp[3];   // solid, liquid, gas
    double L, Ts, Tl;
    double beta, kappa;      // double-well and gradient coefficients (Sec. 2.3.1)
    double Qg, tau_g;        // phase-field diffusion parameter and relaxation (Sec. 2.3.2)
    double dts[3];           // streaming steps of h, f, g (0.5 unless chosen otherwise)
    double Cref;             // 0.5 (cp_s + cp_l) (Sec. 2.1.2)
    double kv;               // 1 - rho_s / rho_l
    double gx, gy;
    double dt;
    // device state: three buffers (W^n, stage 1, stage 2) of NP planes each,
    // NP = 5 doubles (FP64) or 7 floats (FP32C: Hhi Hlo p mx my Chi Clo).
    void* st[3];
    void* Fsp;               // F_s of the previous step
    void* dFs;               // (F_s^n - F_s^{n-1}) / dt of the current step
    int* flag;               // bit 0: this domain produced a non-finite state
    long long plane;         // nx * (ny + hlo + hhi): elements per plane
    long long off;           // hlo * nx: plane index of interior cell (0, 0)
};

// Four constants that the kernels read together: one 16-byte shared-memory
// load in FP32 (two in FP64) instead of four.
template <class R>
struct alignas(16) Q4 { R x, y, z, w; };

// Working-precision copy of a domain's constants.  Built on the host for the
// stage kernel (one per domain, copied into shared memory per work item) and
// on the device by the auxiliary kernels.
template <class R>
struct Consts {
    // groups read with one load (Q4):
    //  - Eq. 7 mixtures of C_p, rho, lambda, mu: gamma = m.x + X (m.y + Y m.z)
    //    with reading R1's {g_g, g_s - g_g, g_l - g_s} and (X, Y) = (C~, F_l),
    //    or, with Eq. 7 as printed, {g_s, g_g - g_s, g_l - g_g} and
    //    (X, Y) = (F_l, C~);
    //  - {T_s, T_l, L, T_l - T_s};
    //  - the heat capacities of Eq. 6's branches, C_p^sol = x + C~ y and
    //    C_p^liq = z + C~ w: R1 {cp_g, cp_s - cp_g, cp_g, cp_l - cp_g}, as
    //    printed {cp_s, 0, cp_g, cp_l - cp_g};
    //  - face {Q, C_ref / 6, 6 / C_ref, tau_g - 1/2}; cell {kv, g_x, g_y, 1 / dt}
    //    and {2 beta, kappa, dt, dt_f}
    Q4<R> mcp, mrho, mlam, mmu, enth, enthc, facec, cellc, cellc2;
    // H_l = C_p^liq hl[0] + hl[1]: R1 {T_l, L}, as printed {0, cp_l T_l + L}
    alignas(2 * sizeof(R)) R hl[2];
    R printed;                 // 1 with Eq. 5-7 as printed, 0 with reading R1
    R cp[3];                   // solid, liquid, gas (the forward closure of the initial state)
    R L, Ts, Tl;
    R dth, dtf, dtg;           // streaming steps of h, f, g
    R th_coef, tf_coef;        // 3 / (C_ref dt_h), 3 / dt_f: tau - 1/2 = coef x lambda (or mu) / rho
    R Tw[4], wet[4], cos_adv[4], cos_rec[4];
    R four_over_xi;
    int nx, ny, per_x, per_y, zsv, axi;
    int gen;                   // 1: some streaming step differs from 0.5 (general face path)
    int lit;                   // 1: Eq. 5-7 as printed instead of reading R1
    int tma;                   // 1: the state buffers have tensor maps (stage kernel tiles by TMA)
    int pad_;
    int hlo, hhi;              // halo rows below / above (a slab of a split domain)
    long long off;             // plane index of interior cell (0, 0)
    int bc_t[4], bc_f[4], bc_c[4];
    long long plane;
    void* st[3];
    void* Fsp;
    void* dFs;
    int* flag;
};

template <class R>
__host__ __device__ inline Q4<R> make_q4(double x, double y, double z, double w) {
    Q4<R> q;
    q.x = (R)x; q.y = (R)y; q.z = (R)z; q.w = (R)w;
    return q;
}

// The Eq. 7 group of one property (solid, liquid, gas): reading R1
// {g_g, g_s - g_g, g_l - g_s}, Eq. 7 as printed {g_s, g_g - g_s, g_l - g_g}.
template <class R>
__host__ __device__ inline Q4<R> mixture_q4(const double g[3], bool printed) {
    if (printed) return make_q4<R>(g[0], g[2] - g[0], g[1] - g[2], 0.0);
    return make_q4<R>(g[2], g[0] - g[2], g[1] - g[0], 0.0);
}

template <class R>
__host__ __device__ inline void fill_consts(const DomainDesc& d, Consts<R>& K) {
    const bool printed = d.literal_eq7 != 0;
    K.mcp = mixture_q4<R>(d.cp, printed);
    K.mrho = mixture_q4<R>(d.rho, printed);
    K.mlam = mixture_q4<R>(d.lam, printed);
    K.mmu = mixture_q4<R>(d.mu, printed);
    K.enth = make_q4<R>(d.Ts, d.Tl, d.L, d.Tl - d.Ts);
    K.enthc = printed ? make_q4<R>(d.cp[0], 0.0, d.cp[2], d.cp[1] - d.cp[2])
                      : make_q4<R>(d.cp[2], d.cp[0] - d.cp[2], d.cp[2], d.cp[1] - d.cp[2]);
    K.hl[0] = printed ? R(0) : (R)d.Tl;
    K.hl[1] = printed ? (R)(d.cp[1] * d.Tl + d.L) : (R)d.L;
    K.printed = printed ? R(1) : R(0);
    K.facec = make_q4<R>(d.Qg, d.Cref / 6.0, 6.0 / d.Cref, d.tau_g - 0.5);
    K.cellc = make_q4<R>(d.kv, d.gx, d.gy, 1.0 / d.dt);
    K.cellc2 = make_q4<R>(2.0 * d.beta, d.kappa, d.dt, d.dts[1]);
    for (int k = 0; k < 3; ++k) K.cp[k] = (R)d.cp[k];
    K.L = (R)d.L; K.Ts = (R)d.Ts; K.Tl = (R)d.Tl;
    K.four_over_xi = (R)d.four_over_xi;
    K.dth = (R)d.dts[0]; K.dtf = (R)d.dts[1]; K.dtg = (R)d.dts[2];
    K.th_coef = (R)(3.0 / (d.Cref * d.dts[0]));
    K.tf_coef = (R)(3.0 / d.dts[1]);
    K.gen = (d.dts[0] != 0.5 || d.dts[1] != 0.5 || d.dts[2] != 0.5) ? 1 : 0;
    K.lit = d.literal_eq7;
    K.tma = 0;                 // set by the host where the tensor maps exist
    K.pad_ = 0;
    for (int k = 0; k < 4; ++k) {
        K.Tw[k] = (R)d.Tw[k]; K.wet[k] = (R)d.wet[k];
        K.cos_adv[k] = (R)d.cos_adv[k]; K.cos_rec[k] = (R)d.cos_rec[k];
        K.bc_t[k] = d.bc_t[k]; K.bc_f[k] = d.bc_f[k]; K.bc_c[k] = d.bc_c[k];
    }
    K.nx = d.nx; K.ny = d.ny; K.per_x = d.per_x; K.per_y = d.per_y;
    K.zsv = d.zero_solid_velocity; K.axi = d.axi;
    K.plane = d.plane;
    K.hlo = d.hlo;
    K.hhi = d.hhi;
    K.off = d.off;
    for (int k = 0; k < 3; ++k) K.st[k] = d.st[k];
    K.Fsp = d.Fsp;
    K.dFs = d.dFs;
    K.flag = d.flag;
}

// Stage kernel geometry: a work item is a strip segment of one domain,
// kStripX interior columns wide and rows [y0, y1) high, swept in chunks of
// kChunk rows (one warp per row, so kChunk warps per CTA).
constexpr int kStripX = 31;   // 31 cells -> 32 x-faces per row: one per lane
constexpr int kChunk = 8;
constexpr int kStageThreads = 32 * kChunk;

// The stage kernel's input tiles: kChunk rows x kTileX columns x all state
// planes of one buffer, copied into shared memory by a TMA tensor copy.  The
// first column is rounded down to a 16-byte boundary, so kTileX covers the
// strip, its halo and up to three columns of offset.
constexpr int kTileX = 40;
constexpr int kTmapBytes = 128;   // sizeof(CUtensorMap)

struct StageLaunch {
    const void* consts;      // Consts<R>[ndomains] in device memory
    const void* tmaps;       // CUtensorMap[ndomains][3]: one per state buffer (used where Consts::tma)
    const int4* items;       // (domain, strip, y0, y1), tallest first
    int nitems;
    int stage;               // the stage of a one-stage launch: 0, 1, 2
    int stages;              // 1: stage `stage` alone; 3 k: k whole time steps (items of stage 0, 1, 2 of the first step, then of the next)
    int* work;               // item counters (per stage; [0] for a whole-step launch), zeroed before each step
    // whole-step launches: item i of stage s reads the output of the stage
    // s - 1 items dep_idx[dep_off[i] .. dep_off[i + 1]) (its neighbourhood),
    // and waits until done[(s - 1) * nitems + j] is set for each of them
    const int* dep_off;
    const int* dep_idx;
    int* done;               // [stages][nitems], zeroed before each launch
    int* flag;               // bit 0: non-finite state seen; bit 1: a bounded wait (tile or neighbour) gave up
    unsigned tile_probe;     // bytes each tile barrier expects beyond its copy (0; > 0 only to test the bounded waits)
    int dep_probe;           // 1: items never mark themselves done (only to test the bounded neighbour waits)
};

// Launch one Runge-Kutta stage (stages == 1) or k whole steps (stages == 3 k)
// over every work item of the batch.
cudaError_t launch_stage(int precision, const StageLaunch& a, int grid, cudaStream_t s);
// Resident CTAs per SM of the stage kernel (for sizing the persistent grid).
int stage_blocks_per_sm(int precision);
size_t stage_smem_bytes(int precision);

// Initial state from primitive fields (device double arrays); *bad is set
// to 1 if any input value is NaN or Inf.
cudaError_t launch_init(int precision, const DomainDesc* d_desc, const double* T, const double* Fl,
                        const double* C, const double* u, const double* v, const double* p,
                        long long n, int* bad, cudaStream_t s);
// Primitive fields of the current state W^n (device double outputs, NULL skipped).
cudaError_t launch_fields(int precision, const DomainDesc* d_desc, long long n, double* H, double* T,
                          double* Fl, double* C, double* p, double* u, double* v, cudaStream_t s);
// Checkpoint conversion between the state planes and double arrays.
cudaError_t launch_get_state(int precision, const DomainDesc* d_desc, long long n, double* H, double* p,
                             double* mx, double* my, double* C, double* Fsp, cudaStream_t s);
cudaError_t launch_set_state(int precision, const DomainDesc* d_desc, long long n, const double* H,
                             const double* p, const double* mx, const double* my, const double* C,
                             const double* Fsp, cudaStream_t s);

// Halo rows of the slabs of split domains: for every link (lower slab, upper
// slab) of `links`, the lower slab's top kHalo interior rows go to the upper
// slab's lower halo and the upper slab's bottom kHalo rows to the lower
// slab's upper halo, in state buffer `buffer` (all planes).
cudaError_t launch_halo(int precision, const void* consts, const int2* links, int nlinks, int max_nx, int buffer,
                        cudaStream_t s);

// FP64 diagnostics: per-block partial sums (deterministic order) and the final pass.
constexpr int kDiagThreads = 256;
constexpr int kDiagFields = 6;   // mass, enthalpy, phase, solid, max speed, nonfinite
int diag_blocks(long long n);
cudaError_t launch_diag(int precision, const DomainDesc* d_desc, long long n, double* partial,
                        int nblocks, double* out, cudaStream_t s);

// Record the message returned by eulbfs_last_error() on this thread.
int set_error(int code, const char* msg);

}  // namespace eulbfs
