// api.cu -- host side of libeulbfs: the C ABI of include/eulbfs.h.
//
// A solver holds a set of domains ("slots").  Each domain owns one device
// allocation: its descriptor, three state buffers (W^n and the two
// intermediate Runge-Kutta stages), F_s of the previous step and the lagged
// dF_s/dt.  The active domains form one tile work list; a time step is three
// launches of the stage kernel over that list (Eq. 58), optionally replayed
// from a captured CUDA graph; each stage launch and each graph replay is an
// NVTX range for profilers.  Domains can be added and removed between steps
// (continuous batching) under a device-memory budget.
#include <cuda.h>           // CUtensorMap and its enums only: the encoder is fetched through the runtime
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>   // header-only: ranges cost a pointer test unless a profiler is attached

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "eulbfs.h"
#include "eulbfs_internal.h"

using namespace eulbfs;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(EULBFS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr double kDtStream = 0.5;   // c dt_s = dx / 2 (Sec. 2.5 step (1))
constexpr int kMinSlabRows = 8;     // interior rows of each slab of a split domain

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int planes_of(int precision) { return precision == EULBFS_FP64 ? 5 : 7; }
size_t elem_of(int precision) { return precision == EULBFS_FP64 ? 8 : 4; }

struct Dom {
    eulbfs_grid grid{};
    eulbfs_props props{};
    eulbfs_bc bc{};
    eulbfs_numerics num{};
    DomainDesc desc{};     // host copy (device pointers filled in)
    DomainDesc* d_desc = nullptr;  // device copy at the start of `mem`
    void* mem = nullptr;
    size_t bytes = 0;
    long long done = 0;
    long long max_steps = 0;
    bool alive = false;    // allocated and not removed
    bool finished() const { return max_steps > 0 && done >= max_steps; }
    bool active() const { return alive && !finished(); }
};

bool valid_kind_side(const eulbfs_side& s, bool periodic) {
    if (periodic)
        return s.thermal == EULBFS_BC_PERIODIC && s.flow == EULBFS_BC_PERIODIC && s.phase == EULBFS_BC_PERIODIC;
    return (s.thermal == EULBFS_BC_DIRICHLET_T || s.thermal == EULBFS_BC_ADIABATIC) &&
           (s.flow == EULBFS_BC_NOSLIP || s.flow == EULBFS_BC_SYMMETRY || s.flow == EULBFS_BC_OUTLET) &&
           (s.phase == EULBFS_BC_NOFLUX || s.phase == EULBFS_BC_WETTING ||
            (s.phase == EULBFS_BC_WETTING_HYST && s.theta_rec_deg >= 0.0 && s.theta_rec_deg <= s.theta_adv_deg &&
             s.theta_adv_deg <= 180.0));
}

int validate(const eulbfs_grid& g, const eulbfs_props& P, const eulbfs_bc& B, const eulbfs_numerics& N) {
    if (g.nx < 1 || g.ny < 1) return fail(EULBFS_EINVAL, "nx and ny must be >= 1");
    if ((long long)g.nx * g.ny > (1LL << 31)) return fail(EULBFS_EINVAL, "domain too large");
    const bool px = B.xlo.thermal == EULBFS_BC_PERIODIC, py = B.ylo.thermal == EULBFS_BC_PERIODIC;
    if (!valid_kind_side(B.xlo, px) || !valid_kind_side(B.xhi, px) || !valid_kind_side(B.ylo, py) ||
        !valid_kind_side(B.yhi, py))
        return fail(EULBFS_EINVAL, "inconsistent boundary conditions (a periodic side needs a periodic partner)");
    if ((!px && g.nx < 2) || (!py && g.ny < 2)) return fail(EULBFS_EINVAL, "a walled axis needs at least 2 cells");
    const eulbfs_phase* ph[3] = {&P.s, &P.l, &P.g};
    for (auto* q : ph)
        if (!(q->rho > 0 && q->cp > 0 && q->lambda > 0 && q->mu >= 0 && std::isfinite(q->rho) &&
              std::isfinite(q->cp) && std::isfinite(q->lambda) && std::isfinite(q->mu)))
            return fail(EULBFS_EINVAL, "phase properties must be finite, rho, lambda, cp > 0 and mu >= 0");
    if (!(P.L >= 0 && P.Ts <= P.Tl && P.sigma >= 0 && P.Mc >= 0 && P.tau_g > 0.5))
        return fail(EULBFS_EINVAL, "need L >= 0, Ts <= Tl, sigma >= 0, Mc >= 0, tau_g > 0.5");
    if (P.sigma > 0 && !(P.xi > 0)) return fail(EULBFS_EINVAL, "xi must be > 0 when sigma > 0");
    if (!(N.dt > 0 && std::isfinite(N.dt))) return fail(EULBFS_EINVAL, "dt must be > 0");
    if (N.axisymmetric != 0 && N.axisymmetric != 1) return fail(EULBFS_EINVAL, "axisymmetric must be 0 or 1");
    for (double ds : {N.dt_stream_h, N.dt_stream_f, N.dt_stream_g})
        if (!(ds == 0.0 || (ds > 0.0 && ds <= 0.5)))
            return fail(EULBFS_EINVAL, "streaming steps must be 0 (default 0.5) or in (0, 0.5]");
    if (N.axisymmetric && !(B.xlo.thermal == EULBFS_BC_ADIABATIC && B.xlo.flow == EULBFS_BC_SYMMETRY &&
                            B.xlo.phase == EULBFS_BC_NOFLUX))
        return fail(EULBFS_EINVAL, "an axisymmetric domain needs the axis (xlo) adiabatic, symmetric and no-flux");
    return EULBFS_OK;
}

// hlo, hhi: halo rows below / above a slab of a split domain (0 otherwise).
DomainDesc make_desc(const eulbfs_grid& g, const eulbfs_props& P, const eulbfs_bc& B, const eulbfs_numerics& N,
                     int hlo = 0, int hhi = 0) {
    DomainDesc d{};
    d.nx = g.nx;
    d.ny = g.ny;
    d.hlo = hlo;
    d.hhi = hhi;
    d.per_x = B.xlo.thermal == EULBFS_BC_PERIODIC;
    // a slab with halos reaches its neighbours through them, not by wrapping
    d.per_y = B.ylo.thermal == EULBFS_BC_PERIODIC && !hlo && !hhi;
    const eulbfs_side* sides[4] = {&B.xlo, &B.xhi, &B.ylo, &B.yhi};
    for (int k = 0; k < 4; ++k) {
        d.bc_t[k] = sides[k]->thermal;
        d.bc_f[k] = sides[k]->flow;
        d.bc_c[k] = sides[k]->phase;
        d.Tw[k] = sides[k]->Tw;
        d.wet[k] = (P.xi > 0) ? 4.0 * std::cos(sides[k]->theta_deg * M_PI / 180.0) / P.xi : 0.0;
        d.cos_adv[k] = std::cos(sides[k]->theta_adv_deg * M_PI / 180.0);
        d.cos_rec[k] = std::cos(sides[k]->theta_rec_deg * M_PI / 180.0);
    }
    d.zero_solid_velocity = P.zero_solid_velocity ? 1 : 0;
    d.literal_eq7 = P.literal_eq7 ? 1 : 0;
    d.axi = N.axisymmetric ? 1 : 0;
    const eulbfs_phase* ph[3] = {&P.s, &P.l, &P.g};
    for (int k = 0; k < 3; ++k) {
        d.rho[k] = ph[k]->rho;
        d.mu[k] = ph[k]->mu;
        d.lam[k] = ph[k]->lambda;
        d.cp[k] = ph[k]->cp;
    }
    d.L = P.L;
    d.Ts = P.Ts;
    d.Tl = P.Tl;
    d.beta = P.sigma > 0 ? 12.0 * P.sigma / P.xi : 0.0;   // Sec. 2.3.1
    d.kappa = 1.5 * P.xi * P.sigma;
    d.four_over_xi = P.xi > 0 ? 4.0 / P.xi : 0.0;
    d.tau_g = P.tau_g;
    d.dts[0] = N.dt_stream_h > 0 ? N.dt_stream_h : kDtStream;
    d.dts[1] = N.dt_stream_f > 0 ? N.dt_stream_f : kDtStream;
    d.dts[2] = N.dt_stream_g > 0 ? N.dt_stream_g : kDtStream;
    d.Qg = P.Mc / ((P.tau_g - 0.5) * d.dts[2]);          // M_c = (tau_g - 0.5) Q_g dt_g
    d.Cref = 0.5 * (P.s.cp + P.l.cp);                    // Sec. 2.1.2
    d.kv = 1.0 - P.s.rho / P.l.rho;
    d.gx = P.gx;
    d.gy = P.gy;
    d.dt = N.dt;
    d.plane = (long long)g.nx * (g.ny + hlo + hhi);
    d.off = (long long)hlo * g.nx;
    return d;
}

// Bytes of one domain's allocation; n = elements per plane (halo rows included).
size_t domain_bytes(long long n, int precision) {
    const size_t e = elem_of(precision);
    return align256(sizeof(DomainDesc)) + 256 /* flag */ + 3 * align256((size_t)planes_of(precision) * n * e) +
           2 * align256(n * e);
}

}  // namespace

int eulbfs::set_error(int code, const char* msg) { return fail(code, msg); }

constexpr int kMaxTune = 8;   // autotune candidates kept for eulbfs_autotune_report
constexpr int kTailLevels = 2;   // halvings of the work list's last wave (launches per stage)
constexpr int kMaxLaunchSteps = 16;   // time steps in one whole-step launch at most

struct eulbfs_solver {
    int precision = EULBFS_FP32C;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<Dom> doms;
    void* d_consts = nullptr;      // Consts<R>[ndomains] in the working precision
    size_t consts_cap = 0;
    void* d_tmaps = nullptr;       // CUtensorMap[ndomains][3] of the state buffers
    size_t tmaps_cap = 0;
    int4* d_items = nullptr;       // work items (domain, strip, segment, 0)
    int items_cap = 0;
    int nitems = 0;
    bool dirty = true;
    int seg = 64;                  // segment height of a work item (rows)
    int sms = 1;
    int grid = 1;
    int* d_flag = nullptr;
    // item counters ([0..3]) and the whole-step launch's done flags ([3][nitems])
    int* d_sched = nullptr;
    size_t sched_cap = 0;
    // whole-step launches: each item's neighbourhood (CSR: offsets, then indices)
    int* d_deps = nullptr;
    int deps_cap = 0;
    int ndeps = 0;
    bool whole_step = true;        // eulbfs_set_whole_step: one launch per step where possible
    bool fused = false;            // this batch runs whole-step launches
    unsigned long long launches = 0;        // kernel launches run so far (eulbfs_launch_count)
    unsigned long long graph_launches = 0;  // kernel launches in one replay of the captured graph
    int* h_flag = nullptr;
    int* h_flags = nullptr;        // pinned, one per slot: per-domain non-finite flags
    int h_flags_cap = 0;
    double* d_partial = nullptr;
    int partial_cap = 0;
    double* d_diag = nullptr;
    double* h_diag = nullptr;
    unsigned long long budget = 0;
    unsigned long long used = 0;
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    // the last eulbfs_autotune: candidate heights and their best ms per step
    int tune_n = 0;
    int tune_rows[kMaxTune] = {};
    float tune_ms[kMaxTune] = {};
    unsigned tile_probe = 0;       // eulbfs_set_tile_wait_probe(1)
    int dep_probe = 0;             // eulbfs_set_tile_wait_probe(2)
    // split domains: (lower slab, upper slab) pairs whose halo rows are
    // exchanged after every stage; the active ones on the device
    std::vector<int2> links;
    int2* d_links = nullptr;
    int links_cap = 0;
    int nlinks = 0;                // active links uploaded
    int link_nx = 0;               // widest linked slab
    bool halo_stale = false;       // W^n was written outside a stage: refresh its halos before stepping
};

namespace {

void drop_graph(eulbfs_solver* s) {
    if (s->graph) cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
    s->graph_valid = false;
}

static_assert(sizeof(CUtensorMap) == kTmapBytes, "tensor map size");

typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry points (no link
// against the driver library); null if the driver does not provide it.
encode_tiled_fn tensor_map_encoder() {
    static encode_tiled_fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<encode_tiled_fn>(f);
        cudaGetLastError();
    }
    return fn;
}

// Tensor map of one state buffer: columns x rows x planes, box kTileX x
// kChunk x all planes.  A TMA copy needs 16-byte aligned rows and planes, so
// domains whose row (nx elements) is not a multiple of 16 bytes get none and
// the stage kernel loads their cells directly.
bool encode_state_map(CUtensorMap* m, void* base, int precision, int nx, long long rows, long long plane) {
    encode_tiled_fn enc = tensor_map_encoder();
    const size_t e = elem_of(precision);
    if (!enc || (nx * e) % 16 != 0 || (plane * e) % 16 != 0 || reinterpret_cast<uintptr_t>(base) % 16 != 0)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)rows, (cuuint64_t)planes_of(precision)};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * e, (cuuint64_t)plane * e};
    const cuuint32_t box[3] = {(cuuint32_t)kTileX, (cuuint32_t)kChunk, (cuuint32_t)planes_of(precision)};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, precision == EULBFS_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <class R>
std::vector<unsigned char> consts_image(const std::vector<Dom>& doms, const std::vector<char>& tma) {
    std::vector<unsigned char> img(sizeof(Consts<R>) * doms.size());
    for (size_t k = 0; k < doms.size(); ++k) {
        Consts<R> K{};
        fill_consts(doms[k].desc, K);
        K.tma = tma[k];
        std::memcpy(img.data() + k * sizeof(Consts<R>), &K, sizeof(K));
    }
    return img;
}

// Rebuild the work list (strip segments of every active domain) and the
// per-domain constants after the set of domains or the segment height changed.
// A whole-step launch runs the items of stage s once the stage s - 1 items
// they read are done.  Item i reads its strip and the strips on either side
// (the 3-column halo, and the wall-wetting column beyond), rows
// [y0 - 4, y1 + 4) (the 3-row halo and the wall-wetting row beyond), both
// wrapped on periodic axes: those are the items listed here (CSR).
void build_deps(const eulbfs_solver* s, const std::vector<int4>& items, std::vector<int>& dep) {
    const int n = (int)items.size();
    std::vector<std::vector<std::vector<int>>> by(s->doms.size());   // [domain][strip] -> items
    for (int i = 0; i < n; ++i) {
        const int4& t = items[i];
        auto& v = by[t.x];
        if (v.empty()) v.resize(s->doms[t.x].desc.strips);
        v[t.y].push_back(i);
    }
    dep.assign(n + 1, 0);
    std::vector<char> mark;
    for (int i = 0; i < n; ++i) {
        const int4& t = items[i];
        const DomainDesc& d = s->doms[t.x].desc;
        mark.assign(d.strips, 0);
        const int x0 = t.y * kStripX;
        for (int c = x0 - kHalo - 1; c < x0 + kStripX + kHalo + 1; ++c) {
            int cc = c;
            if (d.per_x) cc = ((c % d.nx) + d.nx) % d.nx;
            else if (c < 0 || c >= d.nx) continue;
            mark[cc / kStripX] = 1;
        }
        // row intervals of [y0 - 4, y1 + 4) within [0, ny)
        int iv[2][2];
        int niv = 0;
        const int lo = t.z - kHalo - 1, hi = t.w + kHalo + 1;
        if (!d.per_y || hi - lo >= d.ny) {
            iv[0][0] = std::max(0, lo); iv[0][1] = std::min(d.ny, hi); niv = 1;
        } else {
            const int a = ((lo % d.ny) + d.ny) % d.ny, b = a + (hi - lo);
            if (b <= d.ny) { iv[0][0] = a; iv[0][1] = b; niv = 1; }
            else { iv[0][0] = a; iv[0][1] = d.ny; iv[1][0] = 0; iv[1][1] = b - d.ny; niv = 2; }
        }
        for (int sx = 0; sx < d.strips; ++sx) {
            if (!mark[sx]) continue;
            for (int j : by[t.x][sx]) {
                const int4& u = items[j];
                bool hit = false;
                for (int k = 0; k < niv; ++k) hit |= u.z < iv[k][1] && iv[k][0] < u.w;
                if (hit) dep.push_back(j);
            }
        }
        dep[i + 1] = (int)dep.size() - (n + 1);
    }
}

int rebuild(eulbfs_solver* s) {
    const int nd = (int)s->doms.size();
    // tensor maps of every live domain's three state buffers
    std::vector<CUtensorMap> maps((size_t)nd * 3);
    std::vector<char> tma(nd, 0);
    for (int k = 0; k < nd; ++k) {
        const Dom& d = s->doms[k];
        if (!d.alive) continue;
        bool ok = true;
        for (int b = 0; b < 3 && ok; ++b)
            ok = encode_state_map(&maps[(size_t)k * 3 + b], d.desc.st[b], s->precision, d.grid.nx,
                                  (long long)d.grid.ny + d.desc.hlo + d.desc.hhi, d.desc.plane);
        tma[k] = ok ? 1 : 0;
    }
    std::vector<unsigned char> img =
        s->precision == EULBFS_FP64 ? consts_image<double>(s->doms, tma) : consts_image<float>(s->doms, tma);
    const size_t map_bytes = sizeof(CUtensorMap) * maps.size();
    if (map_bytes > s->tmaps_cap) {
        if (s->d_tmaps) cudaFree(s->d_tmaps);
        s->d_tmaps = nullptr;
        s->tmaps_cap = std::max(map_bytes, 2 * s->tmaps_cap);
        CK(cudaMalloc(&s->d_tmaps, s->tmaps_cap), "tensor maps");
    }
    if (map_bytes) CK(cudaMemcpyAsync(s->d_tmaps, maps.data(), map_bytes, cudaMemcpyHostToDevice, s->stream), "upload tensor maps");
    if (img.size() > s->consts_cap) {
        if (s->d_consts) cudaFree(s->d_consts);
        s->consts_cap = std::max(img.size(), 2 * s->consts_cap);
        CK(cudaMalloc(&s->d_consts, s->consts_cap), "constants array");
    }
    // work items: each domain's kChunk-row chunks split into round(ny / seg)
    // runs of nearly equal length; the list runs the tallest items first, so
    // that the persistent CTAs, which claim items in list order, end on the
    // shortest
    std::vector<int4> items;
    for (int k = 0; k < nd; ++k) {
        Dom& d = s->doms[k];
        const int chunks = (d.grid.ny + kChunk - 1) / kChunk, per = std::max(1, s->seg / kChunk);
        d.desc.strips = (d.grid.nx + kStripX - 1) / kStripX;
        d.desc.segs = std::min(chunks, std::max(1, (chunks + per / 2) / per));
        if (!d.active()) continue;
        for (int sy = 0; sy < d.desc.segs; ++sy) {
            const int y0 = (int)((long long)sy * chunks / d.desc.segs) * kChunk;
            const int y1 = std::min(d.grid.ny, (int)((long long)(sy + 1) * chunks / d.desc.segs) * kChunk);
            for (int sx = 0; sx < d.desc.strips; ++sx) items.push_back(make_int4(k, sx, y0, y1));
        }
    }
    const auto taller = [](const int4& a, const int4& b) { return a.w - a.z > b.w - b.z; };
    std::stable_sort(items.begin(), items.end(), taller);
    // launches per stage (split domains exchange halos between stages, or
    // eulbfs_set_whole_step(0)): the end of the list in shorter items --
    // kTailLevels times, the last wave (one item per resident CTA) is cut in
    // half, so each launch ends on items 2^-kTailLevels as tall and the first
    // CTAs to run out of work wait less for the last.  A whole-step launch
    // has no stage ends to shorten (the next stage's items fill them), and
    // its one end gains less than the extra prologues cost.
    bool linked = false;
    for (const int2& l : s->links)
        linked |= l.x < nd && l.y < nd && s->doms[l.x].active() && s->doms[l.y].active();
    const int tail_levels = s->whole_step && !linked ? 0 : kTailLevels;
    const int resident = stage_blocks_per_sm(s->precision) * s->sms;
    for (int level = 0; level < tail_levels && (long long)items.size() > 2LL * resident; ++level) {
        std::vector<int4> tail;
        for (size_t i = items.size() - resident; i < items.size(); ++i) {
            const int4 t = items[i];
            const int chunks = (t.w - t.z + kChunk - 1) / kChunk;
            if (chunks < 2) { tail.push_back(t); continue; }
            const int ym = t.z + (chunks / 2) * kChunk;
            tail.push_back(make_int4(t.x, t.y, t.z, ym));
            tail.push_back(make_int4(t.x, t.y, ym, t.w));
        }
        items.resize(items.size() - resident);
        std::stable_sort(tail.begin(), tail.end(), taller);
        items.insert(items.end(), tail.begin(), tail.end());
    }
    if (!img.empty()) CK(cudaMemcpyAsync(s->d_consts, img.data(), img.size(), cudaMemcpyHostToDevice, s->stream), "upload constants");
    s->nitems = (int)items.size();
    if (s->nitems > s->items_cap) {
        if (s->d_items) cudaFree(s->d_items);
        s->items_cap = std::max(s->nitems, 2 * s->items_cap);
        CK(cudaMalloc(&s->d_items, sizeof(int4) * s->items_cap), "work list");
    }
    if (s->nitems) CK(cudaMemcpyAsync(s->d_items, items.data(), sizeof(int4) * s->nitems, cudaMemcpyHostToDevice, s->stream), "upload work list");
    // halo links between active slabs
    std::vector<int2> act;
    s->link_nx = 0;
    for (const int2& l : s->links)
        if (l.x < nd && l.y < nd && s->doms[l.x].active() && s->doms[l.y].active()) {
            act.push_back(l);
            s->link_nx = std::max(s->link_nx, s->doms[l.x].grid.nx);
        }
    s->nlinks = (int)act.size();
    if (s->nlinks > s->links_cap) {
        if (s->d_links) cudaFree(s->d_links);
        s->d_links = nullptr;
        s->links_cap = std::max(s->nlinks, 2 * s->links_cap);
        CK(cudaMalloc(&s->d_links, sizeof(int2) * s->links_cap), "halo links");
    }
    if (s->nlinks) CK(cudaMemcpyAsync(s->d_links, act.data(), sizeof(int2) * s->nlinks, cudaMemcpyHostToDevice, s->stream), "upload links");
    // counters and done flags; the neighbourhoods of a whole-step launch
    // (split domains exchange halos between stages: one launch per stage)
    const size_t sched = 4 + (size_t)3 * kMaxLaunchSteps * s->nitems;
    if (sched > s->sched_cap) {
        if (s->d_sched) cudaFree(s->d_sched);
        s->d_sched = nullptr;
        s->sched_cap = std::max(sched, 2 * s->sched_cap);
        CK(cudaMalloc(&s->d_sched, sizeof(int) * s->sched_cap), "work counters");
    }
    s->fused = s->whole_step && s->nlinks == 0 && s->nitems > 0;
    std::vector<int> dep;
    if (s->fused) {
        build_deps(s, items, dep);
        s->ndeps = (int)dep.size();
        if (s->ndeps > s->deps_cap) {
            if (s->d_deps) cudaFree(s->d_deps);
            s->d_deps = nullptr;
            s->deps_cap = std::max(s->ndeps, 2 * s->deps_cap);
            CK(cudaMalloc(&s->d_deps, sizeof(int) * s->deps_cap), "item neighbourhoods");
        }
        CK(cudaMemcpyAsync(s->d_deps, dep.data(), sizeof(int) * s->ndeps, cudaMemcpyHostToDevice, s->stream), "upload neighbourhoods");
    }
    // the host vectors die here: make the copies complete before returning
    CK(cudaStreamSynchronize(s->stream), "rebuild sync");
    const int per_sm = stage_blocks_per_sm(s->precision);
    s->grid = std::max(1, std::min(s->nitems, per_sm * s->sms));
    drop_graph(s);
    s->dirty = false;
    return EULBFS_OK;
}

// k time steps on the solver's stream: whole-step launches of up to
// kMaxLaunchSteps steps each, or three stage launches per step (with the
// split domains' halo copies after each).
int launch_steps_direct(eulbfs_solver* s, long long k) {
    StageLaunch a;
    a.consts = s->d_consts;
    a.tmaps = s->d_tmaps;
    a.tile_probe = s->tile_probe;
    a.dep_probe = s->dep_probe;
    a.items = s->d_items;
    a.nitems = s->nitems;
    a.flag = s->d_flag;
    a.work = s->d_sched;
    a.done = s->d_sched + 4;
    a.dep_off = s->d_deps;
    a.dep_idx = s->d_deps + (s->nitems + 1);
    a.stage = 0;
    static const char* const kStageRange[3] = {"eulbfs RK stage 1", "eulbfs RK stage 2", "eulbfs RK stage 3"};
    while (k > 0) {
        // counters and done flags start at zero every launch: an aborted launch cannot leave one behind
        const int steps = s->fused ? (int)std::min<long long>(k, kMaxLaunchSteps) : 1;
        const size_t zero = sizeof(int) * (s->fused ? 4 + 3 * (size_t)steps * s->nitems : 4);
        if (cudaMemsetAsync(s->d_sched, 0, zero, s->stream) != cudaSuccess) return cuda_fail(cudaGetLastError(), "work counters");
        if (s->fused) {
            a.stages = 3 * steps;
            nvtxRangePushA("eulbfs steps");
            const cudaError_t e = launch_stage(s->precision, a, s->grid, s->stream);
            nvtxRangePop();
            if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
            ++s->launches;
        } else {
            a.stages = 1;
            for (int st = 0; st < 3; ++st) {
                a.stage = st;
                nvtxRangePushA(kStageRange[st]);
                cudaError_t e = launch_stage(s->precision, a, s->grid, s->stream);
                ++s->launches;
                // split domains: the stage's output halos from the neighbouring slabs
                if (e == cudaSuccess && s->nlinks) {
                    e = launch_halo(s->precision, s->d_consts, s->d_links, s->nlinks, s->link_nx, st == 2 ? 0 : st + 1,
                                    s->stream);
                    ++s->launches;
                }
                nvtxRangePop();
                if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
            }
        }
        k -= steps;
    }
    return EULBFS_OK;
}

int capture_graph(eulbfs_solver* s) {
    drop_graph(s);
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return EULBFS_ECUDA;
    }
    // the capture records launches without running them: count them once per replay
    const unsigned long long before = s->launches;
    int rc = launch_steps_direct(s, s->graph_steps);
    s->graph_launches = s->launches - before;
    s->launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (rc != EULBFS_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return EULBFS_ECUDA;
    }
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph = nullptr;
        cudaGetLastError();
        return EULBFS_ECUDA;
    }
    s->graph_valid = true;
    return EULBFS_OK;
}

// 1 if the domain's own non-finite flag is set (synchronises the stream).
int domain_nonfinite(eulbfs_solver* s, const Dom& d, int* out) {
    CK(cudaMemcpyAsync(s->h_flag, d.desc.flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "flag copy");
    CK(cudaStreamSynchronize(s->stream), "stream sync");
    *out = *s->h_flag & 1;
    return EULBFS_OK;
}

int check_slot(const eulbfs_solver* s, int slot) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    if (slot < 0 || slot >= (int)s->doms.size() || !s->doms[slot].alive)
        return fail(EULBFS_EINVAL, "no such domain slot");
    return EULBFS_OK;
}

int add_domain(eulbfs_solver* s, const eulbfs_domain& dm, long long max_steps, int* slot, int hlo = 0, int hhi = 0) {
    int rc = validate(dm.grid, dm.props, dm.bc, dm.num);
    if (rc) return rc;
    if (!dm.init.T || !dm.init.C) return fail(EULBFS_EINVAL, "initial T and C are required");
    if (max_steps < 0) return fail(EULBFS_EINVAL, "max_steps must be >= 0");
    const long long n = (long long)dm.grid.nx * dm.grid.ny;                  // interior cells
    const long long np = (long long)dm.grid.nx * (dm.grid.ny + hlo + hhi);   // elements per plane
    const size_t bytes = domain_bytes(np, s->precision);
    if (s->budget && s->used + bytes > s->budget)
        return fail(EULBFS_EBUSY, "domain does not fit in the memory budget");
    Dom d;
    d.grid = dm.grid;
    d.props = dm.props;
    d.bc = dm.bc;
    d.num = dm.num;
    d.max_steps = max_steps;
    d.desc = make_desc(dm.grid, dm.props, dm.bc, dm.num, hlo, hhi);
    if (cudaMalloc(&d.mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(EULBFS_ENOMEM, "device allocation of a domain failed");
    }
    d.bytes = bytes;
    char* p = static_cast<char*>(d.mem);
    d.d_desc = reinterpret_cast<DomainDesc*>(p);
    p += align256(sizeof(DomainDesc));
    d.desc.flag = reinterpret_cast<int*>(p);
    p += 256;
    const size_t e = elem_of(s->precision);
    for (int k = 0; k < 3; ++k) {
        d.desc.st[k] = p;
        p += align256((size_t)planes_of(s->precision) * np * e);
    }
    d.desc.Fsp = p;
    p += align256(np * e);
    d.desc.dFs = p;
    CK(cudaMemsetAsync(d.mem, 0, bytes, s->stream), "clear domain");
    CK(cudaMemcpyAsync(d.d_desc, &d.desc, sizeof(DomainDesc), cudaMemcpyHostToDevice, s->stream), "upload descriptor");
    // initial fields: H from (T, F_l, C), m = rho cs^2 u, F_s^{-1} = F_s^0
    double* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * n * 6 + 256) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d.mem);
        return fail(EULBFS_ENOMEM, "init scratch allocation failed");
    }
    int* d_bad = reinterpret_cast<int*>(buf + 6 * n);
    const double* src[6] = {dm.init.T, dm.init.Fl, dm.init.C, dm.init.u, dm.init.v, dm.init.p};
    double* dst[6];
    cudaError_t ce = cudaMemsetAsync(d_bad, 0, sizeof(int), s->stream);
    for (int k = 0; k < 6; ++k) {
        dst[k] = src[k] ? buf + k * n : nullptr;
        if (src[k] && ce == cudaSuccess)
            ce = cudaMemcpyAsync(dst[k], src[k], sizeof(double) * n, cudaMemcpyHostToDevice, s->stream);
    }
    if (ce == cudaSuccess) ce = launch_init(s->precision, d.d_desc, dst[0], dst[1], dst[2], dst[3], dst[4], dst[5], n, d_bad, s->stream);
    int bad = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->h_flag, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    if (ce == cudaSuccess) bad = *s->h_flag;
    cudaFree(buf);
    if (ce != cudaSuccess) {
        cudaFree(d.mem);
        return cuda_fail(ce, "domain initialisation");
    }
    if (bad) {
        cudaFree(d.mem);
        return fail(EULBFS_EINVAL, "initial fields contain NaN or Inf");
    }
    d.alive = true;
    s->used += bytes;
    s->doms.push_back(d);
    if (slot) *slot = (int)s->doms.size() - 1;
    s->dirty = true;
    if (hlo || hhi) s->halo_stale = true;
    return EULBFS_OK;
}

int new_solver(int precision, void* stream, eulbfs_solver** out) {
    if (!out) return fail(EULBFS_EINVAL, "out is null");
    *out = nullptr;
    if (precision != EULBFS_FP64 && precision != EULBFS_FP32C) return fail(EULBFS_EINVAL, "unknown precision");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(EULBFS_ECUDA, "no CUDA device available (there is no CPU fallback)");
    }
    eulbfs_solver* s = new eulbfs_solver();
    s->precision = precision;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return fail(EULBFS_ECUDA, "stream creation failed");
        }
        s->own_stream = true;
    }
    if (cudaMalloc(&s->d_flag, sizeof(int)) != cudaSuccess || cudaMallocHost(&s->h_flag, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s->d_diag, sizeof(double) * kDiagFields) != cudaSuccess ||
        cudaMallocHost(&s->h_diag, sizeof(double) * kDiagFields) != cudaSuccess) {
        eulbfs_destroy(s);
        return fail(EULBFS_ENOMEM, "solver allocation failed");
    }
    cudaMemsetAsync(s->d_flag, 0, sizeof(int), s->stream);
    *out = s;
    return EULBFS_OK;
}

}  // namespace

extern "C" {

const char* eulbfs_last_error(void) { return g_err.c_str(); }

const char* eulbfs_version(void) { return "eulbfs-gb300 0.1 (sm_103a)"; }

unsigned long long eulbfs_domain_bytes(int nx, int ny, int precision) {
    if (nx < 1 || ny < 1) return 0;
    return (unsigned long long)domain_bytes((long long)nx * ny, precision);
}

int eulbfs_create(const eulbfs_grid* grid, const eulbfs_props* props, const eulbfs_bc* bc,
                  const eulbfs_numerics* num, const eulbfs_init* init, int precision, void* stream,
                  eulbfs_solver** out) {
    if (!grid || !props || !bc || !num || !init) return fail(EULBFS_EINVAL, "null argument");
    eulbfs_domain d;
    d.grid = *grid;
    d.props = *props;
    d.bc = *bc;
    d.num = *num;
    d.init = *init;
    return eulbfs_batch_create(1, &d, precision, stream, out);
}

int eulbfs_batch_create(int n, const eulbfs_domain* domains, int precision, void* stream, eulbfs_solver** out) {
    if (n < 0 || (n > 0 && !domains)) return fail(EULBFS_EINVAL, "need n >= 0 domains");
    if (!out) return fail(EULBFS_EINVAL, "out is null");
    for (int k = 0; k < n; ++k) {
        int rc = validate(domains[k].grid, domains[k].props, domains[k].bc, domains[k].num);
        if (rc) return fail(rc, "domain " + std::to_string(k) + ": " + g_err);
    }
    eulbfs_solver* s = nullptr;
    int rc = new_solver(precision, stream, &s);
    if (rc) return rc;
    for (int k = 0; k < n; ++k) {
        rc = add_domain(s, domains[k], 0, nullptr);
        if (rc) {
            std::string m = g_err;
            eulbfs_destroy(s);
            return fail(rc, "domain " + std::to_string(k) + ": " + m);
        }
    }
    *out = s;
    return EULBFS_OK;
}

int eulbfs_set_memory_budget(eulbfs_solver* s, unsigned long long bytes) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    s->budget = bytes;
    return EULBFS_OK;
}

int eulbfs_add_domain(eulbfs_solver* s, const eulbfs_domain* d, long long max_steps, int* slot) {
    if (!s || !d) return fail(EULBFS_EINVAL, "null argument");
    return add_domain(s, *d, max_steps, slot);
}

int eulbfs_remove_domain(eulbfs_solver* s, int slot) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    Dom& d = s->doms[slot];
    CK(cudaStreamSynchronize(s->stream), "sync before remove");
    cudaFree(d.mem);
    d.mem = nullptr;
    d.alive = false;
    s->used -= d.bytes;
    s->dirty = true;
    return EULBFS_OK;
}

int eulbfs_num_slots(const eulbfs_solver* s) { return s ? (int)s->doms.size() : 0; }

int eulbfs_domain_progress(const eulbfs_solver* s, int slot, long long* done, long long* left) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    const Dom& d = s->doms[slot];
    if (done) *done = d.done;
    if (left) *left = d.max_steps > 0 ? std::max(0LL, d.max_steps - d.done) : -1;
    return EULBFS_OK;
}

int eulbfs_set_tile(eulbfs_solver* s, int rows) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    if (rows == 0) rows = 64;
    if (rows < kChunk || rows > 1024 || rows % kChunk) return fail(EULBFS_EINVAL, "segment height must be a multiple of 8 in [8, 1024]");
    if (rows != s->seg) {
        s->seg = rows;
        s->dirty = true;
    }
    return EULBFS_OK;
}

int eulbfs_autotune(eulbfs_solver* s, int steps_per_candidate, int* best_rows, float* best_ms_per_step) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    if (steps_per_candidate < 1) return fail(EULBFS_EINVAL, "steps_per_candidate must be >= 1");
    static const int kCandidates[] = {32, 48, 64, 96, 128, 160, 192, 256};
    static_assert(sizeof(kCandidates) / sizeof(kCandidates[0]) <= kMaxTune, "report arrays");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const int saved_graph = s->graph_steps, saved_seg = s->seg;
    s->graph_steps = 0;                      // time the launches themselves
    constexpr int kNC = (int)(sizeof(kCandidates) / sizeof(kCandidates[0]));
    constexpr int kRounds = 2;               // each candidate's best of two rounds
    float cand_ms[kNC] = {};
    int best = s->seg;
    float best_ms = 0.f;
    int rc = EULBFS_OK;
    for (int round = 0; round < kRounds && rc == EULBFS_OK; ++round) {
        for (int k = 0; k < kNC; ++k) {
            rc = eulbfs_set_tile(s, kCandidates[k]);
            if (rc == EULBFS_OK) rc = eulbfs_step(s, 1);   // rebuild + warm the work list
            if (rc != EULBFS_OK) break;
            if (s->nitems == 0) break;                     // nothing to time
            cudaEventRecord(e0, s->stream);
            rc = eulbfs_step(s, steps_per_candidate);
            cudaEventRecord(e1, s->stream);
            if (rc != EULBFS_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "autotune timing"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= steps_per_candidate;
            if (cand_ms[k] == 0.f || ms < cand_ms[k]) cand_ms[k] = ms;
        }
    }
    s->tune_n = 0;
    for (int k = 0; k < kNC; ++k) {
        if (cand_ms[k] > 0.f && (best_ms == 0.f || cand_ms[k] < best_ms)) { best_ms = cand_ms[k]; best = kCandidates[k]; }
        if (cand_ms[k] > 0.f && s->tune_n < kMaxTune) {
            s->tune_rows[s->tune_n] = kCandidates[k];
            s->tune_ms[s->tune_n] = cand_ms[k];
            ++s->tune_n;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->graph_steps = saved_graph;
    if (rc != EULBFS_OK) {
        const std::string msg = eulbfs_last_error();   // the step's error, kept over the restore
        eulbfs_set_tile(s, saved_seg);
        return fail(rc, msg.c_str());
    }
    eulbfs_set_tile(s, best);
    if (best_rows) *best_rows = best;
    if (best_ms_per_step) *best_ms_per_step = best_ms;
    return EULBFS_OK;
}

int eulbfs_autotune_report(const eulbfs_solver* s, int* rows, float* ms_per_step, int cap, int* n) {
    if (!s || !n || cap < 0 || (cap > 0 && (!rows || !ms_per_step))) return fail(EULBFS_EINVAL, "bad arguments");
    for (int k = 0; k < s->tune_n && k < cap; ++k) {
        rows[k] = s->tune_rows[k];
        ms_per_step[k] = s->tune_ms[k];
    }
    *n = s->tune_n;
    return EULBFS_OK;
}

int eulbfs_set_tile_wait_probe(eulbfs_solver* s, int on) {
    if (!s || on < 0 || on > 2) return fail(EULBFS_EINVAL, "null solver or on not 0, 1 or 2");
    s->tile_probe = on == 1 ? 16u : 0u;
    s->dep_probe = on == 2 ? 1 : 0;
    drop_graph(s);
    return EULBFS_OK;
}

int eulbfs_use_graphs(eulbfs_solver* s, int steps_per_graph) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    if (steps_per_graph < 0) return fail(EULBFS_EINVAL, "steps_per_graph must be >= 0");
    s->graph_steps = steps_per_graph;
    drop_graph(s);
    return EULBFS_OK;
}

int eulbfs_launches_per_step(const eulbfs_solver* s) {
    if (!s) return 0;
    const int nd = (int)s->doms.size();
    for (const int2& l : s->links)   // a halo copy after each stage while two linked slabs are active
        if (l.x < nd && l.y < nd && s->doms[l.x].active() && s->doms[l.y].active()) return 6;
    bool any = false;
    for (const Dom& d : s->doms) any |= d.active();
    return s->whole_step && any ? 1 : 3;
}

unsigned long long eulbfs_launch_count(const eulbfs_solver* s) { return s ? s->launches : 0; }

int eulbfs_set_whole_step(eulbfs_solver* s, int on) {
    if (!s || (on != 0 && on != 1)) return fail(EULBFS_EINVAL, "null solver or on not 0/1");
    if (s->whole_step != (on == 1)) {
        s->whole_step = on == 1;
        s->dirty = true;
    }
    return EULBFS_OK;
}

int eulbfs_add_split_domain(eulbfs_solver* s, const eulbfs_domain* d, int k, long long max_steps, int* slots) {
    if (!s || !d || !slots) return fail(EULBFS_EINVAL, "null argument");
    if (k < 1) return fail(EULBFS_EINVAL, "k must be >= 1");
    if (k == 1) return add_domain(s, *d, max_steps, slots);
    const int ny = d->grid.ny, nx = d->grid.nx;
    if (ny < k * kMinSlabRows) return fail(EULBFS_EINVAL, "each slab needs at least 8 rows (ny >= 8 k)");
    const bool per_y = d->bc.ylo.thermal == EULBFS_BC_PERIODIC;
    const int first = (int)s->doms.size();
    for (int i = 0; i < k; ++i) {
        const int y0 = (int)((long long)i * ny / k), y1 = (int)((long long)(i + 1) * ny / k);
        eulbfs_domain sl = *d;
        sl.grid.ny = y1 - y0;
        const long long o = (long long)y0 * nx;
        const double* const* src[6] = {&d->init.T, &d->init.Fl, &d->init.C, &d->init.u, &d->init.v, &d->init.p};
        const double** dst[6] = {&sl.init.T, &sl.init.Fl, &sl.init.C, &sl.init.u, &sl.init.v, &sl.init.p};
        for (int f = 0; f < 6; ++f) *dst[f] = *src[f] ? *src[f] + o : nullptr;
        const int hlo = (i > 0 || per_y) ? kHalo : 0, hhi = (i < k - 1 || per_y) ? kHalo : 0;
        int slot = -1;
        const int rc = add_domain(s, sl, max_steps, &slot, hlo, hhi);
        if (rc) {
            const std::string msg = eulbfs_last_error();
            for (int j = first; j < (int)s->doms.size(); ++j) eulbfs_remove_domain(s, j);
            return fail(rc, msg);
        }
        slots[i] = slot;
    }
    for (int i = 0; i + 1 < k; ++i) s->links.push_back(make_int2(slots[i], slots[i + 1]));
    if (per_y) s->links.push_back(make_int2(slots[k - 1], slots[0]));
    s->dirty = true;
    s->halo_stale = true;
    return EULBFS_OK;
}

int eulbfs_step(eulbfs_solver* s, long long n) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    if (n < 0) return fail(EULBFS_EINVAL, "n must be >= 0");
    while (n > 0) {
        if (s->dirty) {
            int rc = rebuild(s);
            if (rc) return rc;
        }
        if (s->nitems == 0) break;
        if (s->halo_stale) {   // W^n written by creation, set_state or load: its halos first
            if (s->nlinks) {
                CK(launch_halo(s->precision, s->d_consts, s->d_links, s->nlinks, s->link_nx, 0, s->stream), "halo rows");
                ++s->launches;
            }
            s->halo_stale = false;
        }
        long long k = n;
        for (const Dom& d : s->doms)
            if (d.active() && d.max_steps > 0) k = std::min(k, d.max_steps - d.done);
        long long left = k;
        if (s->graph_steps > 0) {
            if (!s->graph_valid && left >= s->graph_steps) capture_graph(s);
            while (s->graph_valid && left >= s->graph_steps) {
                nvtxRangePushA("eulbfs graph replay");
                const cudaError_t ge = cudaGraphLaunch(s->graph, s->stream);
                nvtxRangePop();
                CK(ge, "graph launch");
                s->launches += s->graph_launches;
                left -= s->graph_steps;
            }
        }
        if (left > 0) {
            int rc = launch_steps_direct(s, left);
            if (rc) return rc;
        }
        for (Dom& d : s->doms)
            if (d.active()) {
                d.done += k;
                if (d.finished()) s->dirty = true;
            }
        n -= k;
    }
    return EULBFS_OK;
}

int eulbfs_sync(eulbfs_solver* s) {
    if (!s) return fail(EULBFS_EINVAL, "null solver");
    CK(cudaMemcpyAsync(s->h_flag, s->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "flag copy");
    CK(cudaStreamSynchronize(s->stream), "stream sync");
    if (*s->h_flag & 2) return fail(EULBFS_ETIMEOUT, "a bounded device wait for an input tile gave up");
    if (*s->h_flag & 1) return fail(EULBFS_ENONFINITE, "a non-finite state value was produced");
    return EULBFS_OK;
}

int eulbfs_nonfinite_domains(eulbfs_solver* s, int* slots, int cap, int* count) {
    if (!s || !count || cap < 0 || (cap > 0 && !slots)) return fail(EULBFS_EINVAL, "bad arguments");
    const int nd = (int)s->doms.size();
    if (nd > s->h_flags_cap) {
        if (s->h_flags) cudaFreeHost(s->h_flags);
        s->h_flags = nullptr;
        s->h_flags_cap = 0;
        const int want = std::max(nd, 2 * s->h_flags_cap + 16);
        CK(cudaMallocHost(&s->h_flags, sizeof(int) * want), "flag staging");
        s->h_flags_cap = want;
    }
    for (int k = 0; k < nd; ++k)
        if (s->doms[k].alive)
            CK(cudaMemcpyAsync(s->h_flags + k, s->doms[k].desc.flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
               "flag copy");
    CK(cudaStreamSynchronize(s->stream), "stream sync");
    int n = 0;
    for (int k = 0; k < nd; ++k)
        if (s->doms[k].alive && (s->h_flags[k] & 1)) {
            if (n < cap) slots[n] = k;
            ++n;
        }
    *count = n;
    return EULBFS_OK;
}

int eulbfs_fields(eulbfs_solver* s, int slot, const eulbfs_fields_out* out) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    if (!out) return fail(EULBFS_EINVAL, "null output");
    const Dom& d = s->doms[slot];
    const long long n = (long long)d.grid.nx * d.grid.ny;   // interior cells
    double* host[7] = {out->H, out->T, out->Fl, out->C, out->p, out->u, out->v};
    double* buf = nullptr;
    CK(cudaMalloc(&buf, sizeof(double) * n * 7), "fields scratch");
    double* dev[7];
    for (int k = 0; k < 7; ++k) dev[k] = host[k] ? buf + k * n : nullptr;
    cudaError_t e = launch_fields(s->precision, d.d_desc, n, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], dev[6], s->stream);
    for (int k = 0; k < 7 && e == cudaSuccess; ++k)
        if (host[k]) e = cudaMemcpyAsync(host[k], dev[k], sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "fields");
    int bad = 0;
    rc = domain_nonfinite(s, d, &bad);
    if (rc) return rc;
    return bad ? fail(EULBFS_ENONFINITE, "this domain produced a non-finite state") : EULBFS_OK;
}

int eulbfs_get_state(eulbfs_solver* s, int slot, double* H, double* p, double* mx, double* my, double* C,
                     double* Fs_prev, double* t, long long* step) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    const Dom& d = s->doms[slot];
    const long long n = (long long)d.grid.nx * d.grid.ny;   // interior cells
    double* host[6] = {H, p, mx, my, C, Fs_prev};
    double* buf = nullptr;
    CK(cudaMalloc(&buf, sizeof(double) * n * 6), "state scratch");
    double* dev[6];
    for (int k = 0; k < 6; ++k) dev[k] = host[k] ? buf + k * n : nullptr;
    cudaError_t e = launch_get_state(s->precision, d.d_desc, n, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], s->stream);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        if (host[k]) e = cudaMemcpyAsync(host[k], dev[k], sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "get_state");
    if (t) *t = d.done * d.num.dt;
    if (step) *step = d.done;
    return EULBFS_OK;
}

int eulbfs_set_state(eulbfs_solver* s, int slot, const double* H, const double* p, const double* mx,
                     const double* my, const double* C, const double* Fs_prev, double t, long long step) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    (void)t;
    if (step < 0) return fail(EULBFS_EINVAL, "step must be >= 0");
    Dom& d = s->doms[slot];
    const long long n = (long long)d.grid.nx * d.grid.ny;   // interior cells
    const double* host[6] = {H, p, mx, my, C, Fs_prev};
    double* buf = nullptr;
    CK(cudaMalloc(&buf, sizeof(double) * n * 6), "state scratch");
    const double* dev[6];
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6; ++k) {
        dev[k] = host[k] ? buf + k * n : nullptr;
        if (host[k] && e == cudaSuccess)
            e = cudaMemcpyAsync(buf + k * n, host[k], sizeof(double) * n, cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess) e = launch_set_state(s->precision, d.d_desc, n, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "set_state");
    s->halo_stale = true;
    d.done = step;
    if (d.finished()) s->dirty = true;
    return EULBFS_OK;
}

unsigned long long eulbfs_checkpoint_bytes(const eulbfs_solver* s, int slot) {
    if (check_slot(s, slot)) return 0;
    const long long n = s->doms[slot].desc.plane;
    return (unsigned long long)((planes_of(s->precision) + 1) * n * elem_of(s->precision));
}

int eulbfs_save(eulbfs_solver* s, int slot, void* buf, unsigned long long bytes, long long* step) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    if (!buf || bytes != eulbfs_checkpoint_bytes(s, slot)) return fail(EULBFS_EINVAL, "checkpoint buffer size mismatch");
    const Dom& d = s->doms[slot];
    const size_t st = (size_t)planes_of(s->precision) * d.desc.plane * elem_of(s->precision);
    const size_t fs = (size_t)d.desc.plane * elem_of(s->precision);
    char* h = static_cast<char*>(buf);
    CK(cudaMemcpyAsync(h, d.desc.st[0], st, cudaMemcpyDeviceToHost, s->stream), "save state");
    CK(cudaMemcpyAsync(h + st, d.desc.Fsp, fs, cudaMemcpyDeviceToHost, s->stream), "save F_s");
    CK(cudaStreamSynchronize(s->stream), "save sync");
    if (step) *step = d.done;
    return EULBFS_OK;
}

int eulbfs_load(eulbfs_solver* s, int slot, const void* buf, unsigned long long bytes, long long step) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    if (!buf || bytes != eulbfs_checkpoint_bytes(s, slot)) return fail(EULBFS_EINVAL, "checkpoint buffer size mismatch");
    if (step < 0) return fail(EULBFS_EINVAL, "step must be >= 0");
    Dom& d = s->doms[slot];
    const size_t st = (size_t)planes_of(s->precision) * d.desc.plane * elem_of(s->precision);
    const size_t fs = (size_t)d.desc.plane * elem_of(s->precision);
    const char* h = static_cast<const char*>(buf);
    CK(cudaMemcpyAsync(d.desc.st[0], h, st, cudaMemcpyHostToDevice, s->stream), "load state");
    CK(cudaMemcpyAsync(d.desc.Fsp, h + st, fs, cudaMemcpyHostToDevice, s->stream), "load F_s");
    CK(cudaStreamSynchronize(s->stream), "load sync");
    s->halo_stale = true;
    d.done = step;
    if (d.finished()) s->dirty = true;
    return EULBFS_OK;
}

int eulbfs_diagnostics(eulbfs_solver* s, int slot, eulbfs_diag* out) {
    int rc = check_slot(s, slot);
    if (rc) return rc;
    if (!out) return fail(EULBFS_EINVAL, "null output");
    const Dom& d = s->doms[slot];
    const long long n = (long long)d.grid.nx * d.grid.ny;   // interior cells
    const int nb = diag_blocks(n);
    if (nb > s->partial_cap) {
        CK(cudaStreamSynchronize(s->stream), "sync");
        if (s->d_partial) cudaFree(s->d_partial);
        s->partial_cap = std::max(nb, 64);
        CK(cudaMalloc(&s->d_partial, sizeof(double) * kDiagFields * s->partial_cap), "diag scratch");
    }
    CK(launch_diag(s->precision, d.d_desc, n, s->d_partial, nb, s->d_diag, s->stream), "diag kernels");
    CK(cudaMemcpyAsync(s->h_diag, s->d_diag, sizeof(double) * kDiagFields, cudaMemcpyDeviceToHost, s->stream), "diag copy");
    int bad = 0;
    rc = domain_nonfinite(s, d, &bad);   // synchronises the stream
    if (rc) return rc;
    out->step = d.done;
    out->t = d.done * d.num.dt;
    out->mass = s->h_diag[0];
    out->enthalpy = s->h_diag[1];
    out->phase_vol = s->h_diag[2];
    out->solid_vol = s->h_diag[3];
    out->max_speed = s->h_diag[4];
    out->nonfinite = s->h_diag[5] != 0.0 ? 1 : 0;
    // flat-front thickness: planar per unit width, axisymmetric over the
    // cylinder's per-radian cross-section sum_i r_i = nx^2 / 2
    const double base = d.desc.axi ? 0.5 * (double)d.grid.nx * d.grid.nx : (double)d.grid.ny;
    out->front_pos = out->solid_vol / base;
    out->interface_pos = out->phase_vol / base;
    if (out->nonfinite || bad) {
        out->nonfinite = 1;
        return fail(EULBFS_ENONFINITE, "domain state is not finite");
    }
    return EULBFS_OK;
}

void eulbfs_destroy(eulbfs_solver* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    for (Dom& d : s->doms)
        if (d.mem) cudaFree(d.mem);
    if (s->d_consts) cudaFree(s->d_consts);
    if (s->d_tmaps) cudaFree(s->d_tmaps);
    if (s->d_links) cudaFree(s->d_links);
    if (s->d_sched) cudaFree(s->d_sched);
    if (s->d_deps) cudaFree(s->d_deps);
    if (s->d_items) cudaFree(s->d_items);
    if (s->d_flag) cudaFree(s->d_flag);
    if (s->h_flag) cudaFreeHost(s->h_flag);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    if (s->d_partial) cudaFree(s->d_partial);
    if (s->d_diag) cudaFree(s->d_diag);
    if (s->h_diag) cudaFreeHost(s->h_diag);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
