// eulbfs_internal.h -- declarations shared by the kernel and host translation
// units of libeulbfs (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eulbfs {

constexpr int kTileX = 32;   // tile width in cells: one warp spans a tile row
constexpr int kHalo = 3;     // C halo; every other field needs 2 (gradient ring + its neighbours)
constexpr int kMaxDomains = 1 << 20;

// Sides in descriptor arrays.
enum { XLO = 0, XHI = 1, YLO = 2, YHI = 3 };

// Per-domain descriptor, stored in device memory.  Physical constants are in
// double; the kernels convert them to their working precision.
struct DomainDesc {
    int nx, ny;
    int tiles_x, tiles_y;
    int tile0;               // first global tile index of this domain
    int per_x, per_y;        // periodic axes
    int bc_t[4], bc_f[4], bc_c[4];  // thermal, flow, phase kind per side
    int zero_solid_velocity;
    int pad_;
    double Tw[4];            // wall temperature per side (Dirichlet)
    double wet[4];           // 4 cos(theta) / xi per side (wetting)
    double rho[3], mu[3], lam[3], cp[3];   // solid, liquid, gas
    double L, Ts, Tl;
    double beta, kappa;      // double-well and gradient coefficients (Sec. 2.3.1)
    double Qg, tau_g;        // phase-field diffusion parameter and relaxation (Sec. 2.3.2)
    double Cref;             // 0.5 (cp_s + cp_l) (Sec. 2.1.2)
    double kv;               // 1 - rho_s / rho_l
    double gx, gy;
    double dt;
    // device state: three buffers (W^n, stage 1, stage 2) of NP planes each,
    // NP = 5 doubles (FP64) or 7 floats (FP32C: Hhi Hlo p mx my Chi Clo).
    void* st[3];
    void* Fsp;               // F_s of the previous step
    void* dFs;               // (F_s^n - F_s^{n-1}) / dt of the current step
    long long plane;         // nx * ny
};

struct StageLaunch {
    const DomainDesc* descs;
    const int* tile_domain;  // domain of each global tile
    int ntiles;
    int stage;               // 0, 1, 2
    int* flag;               // bit 0: non-finite state seen
};

// Tile heights compiled into the stage kernel.
constexpr int kTileYChoices[3] = {4, 8, 16};

// Launch one Runge-Kutta stage over every tile of the batch.
cudaError_t launch_stage(int precision, int tile_y, const StageLaunch& a, int grid, cudaStream_t s);
// Resident CTAs per SM of the stage kernel (for sizing the persistent grid).
int stage_blocks_per_sm(int precision, int tile_y);
size_t stage_smem_bytes(int precision, int tile_y);

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

// FP64 diagnostics: per-block partial sums (deterministic order) and the final pass.
constexpr int kDiagThreads = 256;
constexpr int kDiagFields = 6;   // mass, enthalpy, phase, solid, max speed, nonfinite
int diag_blocks(long long n);
cudaError_t launch_diag(int precision, const DomainDesc* d_desc, long long n, double* partial,
                        int nblocks, double* out, cudaStream_t s);

// Record the message returned by eulbfs_last_error() on this thread.
int set_error(int code, const char* msg);

}  // namespace eulbfs
