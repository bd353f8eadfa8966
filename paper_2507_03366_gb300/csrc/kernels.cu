// kernels.cu -- auxiliary kernels of libeulbfs (sm_103a): initial state from
// primitive fields, field output, checkpoint conversion, the deterministic
// FP64 diagnostics reduction and its no-allocation variant.  The hot path is
// the stage kernel in stage.cu.
#include <math.h>
#include <stdint.h>

#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "device_common.cuh"
#include "eulbfs.h"

namespace eulbfs {

// ---------------------------------------------------------------------------
// Initial state, field output, checkpoints (double precision arithmetic).
// ---------------------------------------------------------------------------
// Inverse of Eq. 5-6 for the initial state (same rule as the oracle).
__device__ double enthalpy_of(const Consts<double>& K, double T, double Fl, double C) {
    const double Ct = clamp01(C);
    const double cpl = Ct * K.cp[1] + (1.0 - Ct) * K.cp[2];
    const double cps = K.lit ? K.cp[0] : Ct * K.cp[0] + (1.0 - Ct) * K.cp[2];
    const double Hs = cps * K.Ts;
    const double HL = (K.lit ? K.cp[1] : cpl) * K.Tl + K.L;
    if (T < K.Ts) return cps * T;
    if (T > K.Tl) return HL + cpl * (T - K.Tl);
    const double f = (K.Tl > K.Ts) ? (T - K.Ts) / (K.Tl - K.Ts) : Fl;
    if (f >= 1.0) return HL;
    if (f <= 0.0) return Hs;
    return Hs + f * (HL - Hs);
}

template <class R>
__global__ void init_kernel(const DomainDesc* dd, const double* T, const double* Fl, const double* C,
                            const double* u, const double* v, const double* p, long long n, int* bad) {
    __shared__ Consts<double> Kd;
    __shared__ Consts<R> K;
    if (threadIdx.x == 0) { fill_consts(*dd, Kd); fill_consts(*dd, K); }
    __syncthreads();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double Cc = C[c];
        if (!(isfinite(T[c]) && isfinite(Cc) && (!Fl || isfinite(Fl[c])) && (!u || isfinite(u[c])) &&
              (!v || isfinite(v[c])) && (!p || isfinite(p[c]))))
            atomicOr(bad, 1);
        const double H = enthalpy_of(Kd, T[c], Fl ? Fl[c] : 1.0, Cc);
        double Td, Fld;
        invert_enthalpy(Kd, H, 0.0, clamp01(Cc), Td, Fld);
        const double rho = mix(mix_weights(Kd, clamp01(Cc), Fld), Kd.mrho);
        SV<R> s;
        if (sizeof(R) == 8) { s.Hh = (R)H; s.Hl = 0; s.Ch = (R)Cc; s.Cl = 0; }
        else { put_pair(s.Hh, s.Hl, H); put_pair(s.Ch, s.Cl, Cc); }
        s.p = (R)(p ? p[c] : 0.0);
        s.mx = (R)(u ? rho * (1.0 / 3.0) * u[c] : 0.0);
        s.my = (R)(v ? rho * (1.0 / 3.0) * v[c] : 0.0);
        store_state(reinterpret_cast<R*>(K.st[0]), K.plane, c + K.off, s);
        // previous-step solid fraction from the stored state, in working precision (R14)
        R Tw, Flw;
        invert_enthalpy(K, s.Hh, s.Hl, clamp01(s.Ch + s.Cl), Tw, Flw);
        reinterpret_cast<R*>(K.Fsp)[c + K.off] = R(1) - Flw;
    }
}

template <class R>
__global__ void fields_kernel(const DomainDesc* dd, long long n, double* H, double* T, double* Fl, double* C,
                              double* p, double* u, double* v) {
    __shared__ Consts<double> Kd;
    __shared__ const void* base;
    if (threadIdx.x == 0) { fill_consts(*dd, Kd); base = dd->st[0]; }
    __syncthreads();
    const R* b = reinterpret_cast<const R*>(base);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, Kd.plane, c + Kd.off);
        const double Hd = pair_value(w.Hh, w.Hl), Cd = pair_value(w.Ch, w.Cl);
        double Td, Fld;
        invert_enthalpy(Kd, Hd, 0.0, clamp01(Cd), Td, Fld);
        const double rho = mix(mix_weights(Kd, clamp01(Cd), Fld), Kd.mrho);
        if (H) H[c] = Hd;
        if (T) T[c] = Td;
        if (Fl) Fl[c] = Fld;
        if (C) C[c] = Cd;
        if (p) p[c] = (double)w.p;
        if (u) u[c] = (double)w.mx / (rho * (1.0 / 3.0));
        if (v) v[c] = (double)w.my / (rho * (1.0 / 3.0));
    }
}

template <class R>
__global__ void get_state_kernel(const DomainDesc* dd, long long n, double* H, double* p, double* mx, double* my,
                                 double* C, double* Fsp) {
    const R* b = reinterpret_cast<const R*>(dd->st[0]);
    const R* fs = reinterpret_cast<const R*>(dd->Fsp);
    const long long P = dd->plane, off = dd->off;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, P, c + off);
        if (H) H[c] = pair_value(w.Hh, w.Hl);
        if (p) p[c] = (double)w.p;
        if (mx) mx[c] = (double)w.mx;
        if (my) my[c] = (double)w.my;
        if (C) C[c] = pair_value(w.Ch, w.Cl);
        if (Fsp) Fsp[c] = (double)fs[c + off];
    }
}

template <class R>
__global__ void set_state_kernel(const DomainDesc* dd, long long n, const double* H, const double* p,
                                 const double* mx, const double* my, const double* C, const double* Fsp) {
    R* b = reinterpret_cast<R*>(dd->st[0]);
    R* fs = reinterpret_cast<R*>(dd->Fsp);
    const long long P = dd->plane, off = dd->off;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        SV<R> w = load_state(b, P, c + off);
        if (sizeof(R) == 8) {
            if (H) w.Hh = (R)H[c];
            if (C) w.Ch = (R)C[c];
        } else {
            if (H) put_pair(w.Hh, w.Hl, H[c]);
            if (C) put_pair(w.Ch, w.Cl, C[c]);
        }
        if (p) w.p = (R)p[c];
        if (mx) w.mx = (R)mx[c];
        if (my) w.my = (R)my[c];
        store_state(b, P, c + off, w);
        if (Fsp) fs[c + off] = (R)Fsp[c];
    }
}

// ---------------------------------------------------------------------------
// Halo rows of the slabs of split domains.  Link l joins a lower slab A (its
// top interior rows) and an upper slab B (its bottom interior rows); both
// have the domain's nx.  Every plane of state buffer `buffer` gets A's rows
// ny_A - kHalo .. ny_A - 1 in B's halo rows -kHalo .. -1 and B's rows
// 0 .. kHalo - 1 in A's halo rows ny_A .. ny_A + kHalo - 1.  Plain copies:
// the halo rows hold the neighbour's values bit for bit.
// ---------------------------------------------------------------------------
template <class R>
__global__ void halo_kernel(const Consts<R>* consts, const int2* links, int buffer) {
    const int2 lk = links[blockIdx.y];
    const Consts<R>& A = consts[lk.x];
    const Consts<R>& B = consts[lk.y];
    const int nx = A.nx;
    const long long rows = (long long)kHalo * nx, per_dir = (long long)Prec<R>::NP * rows;
    const R* a_in = reinterpret_cast<const R*>(A.st[buffer]);
    const R* b_in = reinterpret_cast<const R*>(B.st[buffer]);
    R* a_out = reinterpret_cast<R*>(A.st[buffer]);
    R* b_out = reinterpret_cast<R*>(B.st[buffer]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2 * per_dir;
         i += (long long)gridDim.x * blockDim.x) {
        const bool up = i < per_dir;              // A -> B's lower halo
        const long long j = up ? i : i - per_dir;
        const long long k = j / rows, e = j - k * rows;   // plane, element within the kHalo rows
        if (up)
            b_out[k * B.plane + B.off - rows + e] = a_in[k * A.plane + A.off + (long long)(A.ny - kHalo) * nx + e];
        else
            a_out[k * A.plane + A.off + (long long)A.ny * nx + e] = b_in[k * B.plane + B.off + e];
    }
}

cudaError_t launch_halo(int precision, const void* consts, const int2* links, int nlinks, int max_nx, int buffer,
                        cudaStream_t s) {
    if (nlinks <= 0) return cudaSuccess;
    const long long work = 2LL * (precision == 0 ? 5 : 7) * kHalo * max_nx;
    const dim3 grid((unsigned)std::min<long long>((work + 255) / 256, 1024), (unsigned)nlinks);
    if (precision == 0)
        halo_kernel<double><<<grid, 256, 0, s>>>(static_cast<const Consts<double>*>(consts), links, buffer);
    else
        halo_kernel<float><<<grid, 256, 0, s>>>(static_cast<const Consts<float>*>(consts), links, buffer);
    return cudaGetLastError();
}

static int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_init(int precision, const DomainDesc* d, const double* T, const double* Fl, const double* C,
                        const double* u, const double* v, const double* p, long long n, int* bad, cudaStream_t s) {
    if (precision == 0) init_kernel<double><<<grid_for(n), 256, 0, s>>>(d, T, Fl, C, u, v, p, n, bad);
    else init_kernel<float><<<grid_for(n), 256, 0, s>>>(d, T, Fl, C, u, v, p, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_fields(int precision, const DomainDesc* d, long long n, double* H, double* T, double* Fl,
                          double* C, double* p, double* u, double* v, cudaStream_t s) {
    if (precision == 0) fields_kernel<double><<<grid_for(n), 256, 0, s>>>(d, n, H, T, Fl, C, p, u, v);
    else fields_kernel<float><<<grid_for(n), 256, 0, s>>>(d, n, H, T, Fl, C, p, u, v);
    return cudaGetLastError();
}

cudaError_t launch_get_state(int precision, const DomainDesc* d, long long n, double* H, double* p, double* mx,
                             double* my, double* C, double* Fsp, cudaStream_t s) {
    if (precision == 0) get_state_kernel<double><<<grid_for(n), 256, 0, s>>>(d, n, H, p, mx, my, C, Fsp);
    else get_state_kernel<float><<<grid_for(n), 256, 0, s>>>(d, n, H, p, mx, my, C, Fsp);
    return cudaGetLastError();
}

cudaError_t launch_set_state(int precision, const DomainDesc* d, long long n, const double* H, const double* p,
                             const double* mx, const double* my, const double* C, const double* Fsp,
                             cudaStream_t s) {
    if (precision == 0) set_state_kernel<double><<<grid_for(n), 256, 0, s>>>(d, n, H, p, mx, my, C, Fsp);
    else set_state_kernel<float><<<grid_for(n), 256, 0, s>>>(d, n, H, p, mx, my, C, Fsp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: fixed-order warp-shuffle tree per block, then one block
// sums the block partials in index order, so the result is bitwise
// reproducible for a given grid size.
// ---------------------------------------------------------------------------
int diag_blocks(long long n) {
    long long b = (n + kDiagThreads * 8 - 1) / (kDiagThreads * 8);
    if (b > 2048) b = 2048;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_max(double x) {
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    return x;
}

template <class R>
__global__ void __launch_bounds__(kDiagThreads) diag_partial_kernel(const DomainDesc* dd, long long n, double* partial) {
    __shared__ Consts<double> Kd;
    __shared__ const void* base;
    __shared__ double red[kDiagThreads / 32][kDiagFields];
    if (threadIdx.x == 0) { fill_consts(*dd, Kd); base = dd->st[0]; }
    __syncthreads();
    const R* b = reinterpret_cast<const R*>(base);
    double acc[kDiagFields] = {0, 0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, Kd.plane, c + Kd.off);
        const double H = pair_value(w.Hh, w.Hl), C = pair_value(w.Ch, w.Cl);
        double T, Fl;
        invert_enthalpy(Kd, H, 0.0, clamp01(C), T, Fl);
        const double rho = mix(mix_weights(Kd, clamp01(C), Fl), Kd.mrho);
        // cell volume: 1, or the radius r_i = i + 1/2 per radian (axisymmetric)
        const double vol = Kd.axi ? (double)(c % Kd.nx) + 0.5 : 1.0;
        acc[0] += vol * rho;
        acc[1] += vol * H;
        acc[2] += vol * C;
        acc[3] += vol * (clamp01(C) * (1.0 - Fl));
        const double mx = (double)w.mx, my = (double)w.my;
        acc[4] = fmax(acc[4], sqrt(mx * mx + my * my) / (rho * (1.0 / 3.0)));
        if (!(isfinite(H) && isfinite(C) && isfinite((double)w.p) && isfinite(mx) && isfinite(my))) acc[5] = 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagFields; ++k) {
        const double r = (k == 4 || k == 5) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) red[wid][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < kDiagFields) {
        const int k = threadIdx.x;
        double r = red[0][k];
        for (int w2 = 1; w2 < kDiagThreads / 32; ++w2) r = (k == 4 || k == 5) ? fmax(r, red[w2][k]) : r + red[w2][k];
        partial[(long long)blockIdx.x * kDiagFields + k] = r;
    }
}

__global__ void diag_final_kernel(const double* partial, int nblocks, double* out) {
    if (threadIdx.x < kDiagFields) {
        const int k = threadIdx.x;
        double r = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            const double x = partial[(long long)b * kDiagFields + k];
            r = (k == 4 || k == 5) ? fmax(r, x) : r + x;
        }
        out[k] = r;
    }
}

cudaError_t launch_diag(int precision, const DomainDesc* d, long long n, double* partial, int nblocks, double* out,
                        cudaStream_t s) {
    if (precision == 0) diag_partial_kernel<double><<<nblocks, kDiagThreads, 0, s>>>(d, n, partial);
    else diag_partial_kernel<float><<<nblocks, kDiagThreads, 0, s>>>(d, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, 32, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

}  // namespace eulbfs

// ---------------------------------------------------------------------------
// Diagnostics of a caller-held state without any device allocation.
//
// Some callers cannot let a library call cudaMalloc / cudaFree: programs whose
// device memory is fully committed to another framework's pool, and loops
// that cannot afford the implicit device synchronisation of cudaFree or a
// driver allocation in the middle of a latency-bound step.  For them the
// block partials of the diagnostics reduction live in this fixed, file-scope
// device array instead of a buffer from cudaMalloc.  Every GPU that loads the
// library holds the array (kNoAllocMaxBlocks x 6 doubles = 48 KiB) until the
// process exits.  All calls share it: each call overwrites exactly the
// partials it reads back, so nothing has to start at zero, but two calls that
// overlap on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace eulbfs {

constexpr int kNoAllocMaxBlocks = 1024;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * kDiagFields];

template <class R>
__global__ void __launch_bounds__(kDiagThreads)
diag_partial_noalloc_kernel(Consts<double> Kd, const R* b, long long n, double* partial) {
    __shared__ double red[kDiagThreads / 32][kDiagFields];
    double acc[kDiagFields] = {0, 0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, n, c);
        const double H = pair_value(w.Hh, w.Hl), C = pair_value(w.Ch, w.Cl);
        double T, Fl;
        invert_enthalpy(Kd, H, 0.0, clamp01(C), T, Fl);
        const double rho = mix(mix_weights(Kd, clamp01(C), Fl), Kd.mrho);
        acc[0] += rho;
        acc[1] += H;
        acc[2] += C;
        acc[3] += clamp01(C) * (1.0 - Fl);
        const double mx = (double)w.mx, my = (double)w.my;
        acc[4] = fmax(acc[4], sqrt(mx * mx + my * my) / (rho * (1.0 / 3.0)));
        if (!(isfinite(H) && isfinite(C) && isfinite((double)w.p) && isfinite(mx) && isfinite(my))) acc[5] = 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagFields; ++k) {
        const double r = (k == 4 || k == 5) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) red[wid][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < kDiagFields) {
        const int k = threadIdx.x;
        double r = red[0][k];
        for (int w2 = 1; w2 < kDiagThreads / 32; ++w2) r = (k == 4 || k == 5) ? fmax(r, red[w2][k]) : r + red[w2][k];
        partial[(long long)blockIdx.x * kDiagFields + k] = r;
    }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};

typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

// Identifier of the current CUDA context (unique for the life of the
// process; 0 if there is none or the driver does not provide it).  The
// driver calls are fetched through the runtime, so the library needs no link
// against the driver library.  Called with g_noalloc_mutex held.
unsigned long long current_context_id() {
    static bool tried = false;
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<ctx_get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<ctx_get_id_fn>(f);
        cudaGetLastError();
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of g_noalloc_partials on the current device.  In host code
// the array's name is only a host-side stand-in, never a device address, so
// the address is resolved with the device current: once per device and
// context, and again whenever the device's context has changed (after a
// cudaDeviceReset the old address is not valid).
int noalloc_scratch(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(EULBFS_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(EULBFS_ECUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);   // makes the context current if it was not
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(EULBFS_ECUDA, "cudaGetSymbolAddress of the diagnostics scratch array failed");
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
        g_noalloc_ctx[dev] = current_context_id();
    }
    *out = g_noalloc_ptr[dev];
    return EULBFS_OK;
}
}  // namespace

}  // namespace eulbfs

extern "C" int eulbfs_diagnostics_noalloc(int precision, const void* state, int nx, int ny, const eulbfs_props* props,
                                          double* out, void* stream) {
    using namespace eulbfs;
    if (precision != EULBFS_FP64 && precision != EULBFS_FP32C) return set_error(EULBFS_EINVAL, "unknown precision");
    if (!state || !out || !props) return set_error(EULBFS_EINVAL, "state, props and out must be non-null");
    if (nx < 1 || ny < 1) return set_error(EULBFS_EINVAL, "nx and ny must be >= 1");
    const long long n = (long long)nx * ny;
    const int nb = diag_blocks(n);
    if (n > EULBFS_NOALLOC_MAX_CELLS || nb > kNoAllocMaxBlocks)
        return set_error(EULBFS_EINVAL, "domain exceeds the no-allocation diagnostics limit of "
                                        "EULBFS_NOALLOC_MAX_CELLS (2097152) cells");
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != EULBFS_OK) return rc;
    // the constants the closure and the integrals use (Eq. 5-7), as the
    // other entry points fill them
    DomainDesc d = {};
    const eulbfs_phase* ph[3] = {&props->s, &props->l, &props->g};
    for (int k = 0; k < 3; ++k) { d.rho[k] = ph[k]->rho; d.cp[k] = ph[k]->cp; }
    d.literal_eq7 = props->literal_eq7 ? 1 : 0;
    d.Ts = props->Ts;
    d.Tl = props->Tl;
    d.L = props->L;
    d.Cref = 1.0;
    d.dt = 1.0;
    d.dts[0] = d.dts[1] = d.dts[2] = 0.5;
    d.plane = n;
    Consts<double> Kd = {};
    fill_consts(d, Kd);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == EULBFS_FP64)
        diag_partial_noalloc_kernel<double><<<nb, kDiagThreads, 0, s>>>(Kd, static_cast<const double*>(state), n, scratch);
    else
        diag_partial_noalloc_kernel<float><<<nb, kDiagThreads, 0, s>>>(Kd, static_cast<const float*>(state), n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        diag_final_kernel<<<1, 32, 0, s>>>(scratch, nb, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(EULBFS_ECUDA, cudaGetErrorString(e));
    return EULBFS_OK;
}
