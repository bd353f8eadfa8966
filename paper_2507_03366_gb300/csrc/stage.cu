// stage.cu -- the hot path of libeulbfs (sm_103a): one SSP-RK3 stage (Eq. 58)
// of the EULBFS explicit step over every domain of a batch.
//
// Work decomposition.  A work item is a strip segment of one domain: 31
// interior columns wide, `seg` rows high.  A CTA of 8 warps sweeps its segment
// upwards in chunks of 8 rows, keeping the derived fields of the rows it needs
// in a 16-row ring buffer in shared memory, so every cell of the segment is
// loaded and derived once per stage (plus a 3-column halo on each side and a
// 6-row prologue per segment).  Per chunk:
//   1. load and derive 8 new rows: stage state -> T, F_l, C_p, rho, lambda,
//      mu (Eq. 5-7), u = m / (rho cs^2), p, C; halo cells outside the domain
//      are mapped through the boundary rules (mirror + value rule, or wrap);
//   2. mu_c = 2 beta C (C-1)(2C-1) - kappa lap C (Sec. 2.3.1) for 8 rows;
//      a wall ghost takes the value at its mirror cell;
//   3. every face once: warp w computes the 32 x-faces of chunk row w (one
//      per lane: 31 cells have 32 x-faces) and the 31 y-faces below row w+1
//      (the face row below the chunk comes from the previous chunk);
//   4. per cell: R(W) = -div F + F_E (Eq. 51-52), the Runge-Kutta stage, the
//      optional solid projection, a non-finite check, and the store.
// Work items span all domains of the batch, so one launch advances every
// domain by one stage; the grid is persistent and strides over the items.
//
// The face computation is written in the face frame (n, t): an x-face has
// n = x, t = y and a y-face n = y, t = x (D2Q9 is symmetric under the swap).
// With dt_s = 0.5 the surrounding points x_f - e_a dt_s of a face are the two
// cell centres (e_n = +-1, e_t = 0), the two cells' extrapolations half a cell
// along t (e_n = +-1, e_t = +-1) and three points on the face itself (e_n = 0),
// which take the mean of the two one-sided reconstructions (Eq. 54, R7).
#include <mutex>

#include "device_common.cuh"

namespace eulbfs {

namespace {

constexpr int RW = kStripX + 2 * kHalo;   // ring columns: strip plus halo (37)
constexpr int RING = 16;                  // ring rows (power of two)
constexpr int NT = kStageThreads;         // 8 warps

// Two fields of a cell side by side, read and written with one 8-byte
// (FP64: 16-byte) shared-memory access.
template <class R> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };
template <class R> using P2 = typename Pair<R>::T;


// Derived fields of the ring rows (row r in slot r & 15), paired by the
// places that read them together: every face point needs (u, v), (rho, C)
// and (T, C_p); p is needed at every point and mu_c at the cell and outer
// n-neighbours; lambda and mu only at the face.
template <class R>
struct Ring {
    P2<R> uv[RING][RW];       // u, v
    P2<R> rc[RING][RW];       // rho, C
    P2<R> tc[RING][RW];       // T, C_p
    P2<R> pm[RING][RW];       // p, mu_c
    P2<R> lm[RING][RW];       // lambda, mu
    R fl[RING][RW];           // F_l
};

template <class R>
struct Smem {
    Ring<R> P;
    // face fluxes in pairs (F_h, F_p), (F_mx, F_my), (F_C, u_n): y-faces in a
    // ring of face rows, x-faces of the current chunk
    P2<R> YF[3][RING][32];
    P2<R> XF[3][kChunk][32];
    // the next rows' stage input, all planes, copied by TMA while the
    // current chunk computes (planes x rows x columns, as the tensor map's box)
    // (FP32C only: the FP64 step is bound by the FP64 pipe, not by its loads)
    alignas(128) R tile[sizeof(R) == 4 ? Prec<R>::NP : 1][kChunk][kTileX];
    unsigned long long tile_bar;      // mbarrier: the tile's copy has landed
    int cur_domain;
    int next;                         // the CTA's next work item
    int ready;                        // whole-step launches: the current item's inputs are done
    int stage, item;                  // the current item's stage and work-list index
    int pre;                          // 1: the tile holds (or is receiving) this item's prologue rows
    Consts<R> K;
};

__device__ __forceinline__ int slot(int r) { return r & (RING - 1); }

// ---------------------------------------------------------------------------
// Input tiles by TMA.  One thread issues a 3-D tensor copy (columns x rows x
// planes) into the shared tile with an mbarrier that counts its bytes; every
// thread waits on the barrier's phase.  A wait gives up after about 2^31 SM
// clocks (a second at 2 GHz): the kernel then sets bit 1 of the launch's
// flag, waits the same bound once more for the copy in flight, and returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Per-CTA count of the tile copies waited for (the barrier's phase).
struct TileIO {
    unsigned phase;
};

// The first column of a tile: x0 - kHalo rounded down to 16 bytes.
template <class R>
__device__ __forceinline__ int tile_x(int x0) { return (x0 - kHalo) & ~(int)(16 / sizeof(R) - 1); }

// Rows [r0, r0 + nrows) of the strip at x0 come from a tile when the domain
// has tensor maps and every cell of those rows, with the column halo, is
// inside it (the chunks that need boundary rules load their cells directly).
template <class R>
__device__ __forceinline__ bool tile_rows(const Consts<R>& K, int x0, int r0, int nrows) {
    if constexpr (sizeof(R) != 4) return false;
    return K.tma && x0 >= kHalo && x0 + kStripX + kHalo <= K.nx && r0 >= -K.hlo && r0 + nrows <= K.ny + K.hhi;
}

// Thread 0 issues the copy of rows [r0, r0 + kChunk) of domain dom's stage
// buffer (its tensor map in the launch's map array; hlo: its halo rows below).
template <class R>
__device__ __forceinline__ void tile_fetch_from(Smem<R>& S, const StageLaunch& a, int stage, int dom, int hlo, int x0,
                                                int r0) {
    const unsigned bar = smem_addr(&S.tile_bar);
    const unsigned bytes = (unsigned)sizeof(S.tile) + a.tile_probe;
    const char* map = static_cast<const char*>(a.tmaps) + ((size_t)dom * 3 + stage) * kTmapBytes;
    // the tile's previous contents were read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(&S.tile[0][0][0])), "l"(map), "r"(tile_x<R>(x0)), "r"(r0 + hlo), "r"(0), "r"(bar)
        : "memory");
}

// The same for the current domain.
template <class R>
__device__ __forceinline__ void tile_fetch(Smem<R>& S, const StageLaunch& a, int stage, int x0, int r0) {
    if (threadIdx.x == 0) tile_fetch_from(S, a, stage, S.cur_domain, S.K.hlo, x0, r0);
}

// Position g of a launch's item sequence: its stage (counted over the
// launch: 3 k + s for Runge-Kutta stage s of the launch's step k) and work item.
__device__ __forceinline__ int2 stage_item(const StageLaunch& a, int g) {
    if (a.stages == 1) return make_int2(a.stage, g);
    const int st = g / a.nitems;
    return make_int2(st, g - st * a.nitems);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Whole-step launches: true once every stage st - 1 item whose output item i
// of stage st reads is done (acquire loads; the caller's barrier then
// publishes the data to its CTA).  Lanes of one warp take one neighbour each.
// A bounded wait: after 2^31 clocks it gives up and returns false.
__device__ __forceinline__ bool deps_ready(const StageLaunch& a, int st, int i, int lane, bool wait) {
    // one-stage launches have no neighbourhood lists (kernel boundaries order the stages)
    if (a.stages == 1 || st == 0) return true;
    const int* done = a.done + (size_t)(st - 1) * a.nitems;
    bool ok = true;
    for (int j = a.dep_off[i] + lane; j < a.dep_off[i + 1]; j += 32) {
        const int* f = done + a.dep_idx[j];
        if (ld_acquire(f)) continue;
        if (!wait) { ok = false; continue; }
        const long long t0 = clock64();
        while (!ld_acquire(f)) {
            if (clock64() - t0 > (1LL << 31)) { ok = false; break; }
            __nanosleep(256);
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// During the last chunk of a work item (the tile is free): thread 0 copies
// the prologue rows of the CTA's next work item, if they come from a tile
// (and, in a whole-step launch, if the items it reads are already done),
// and records in S.pre whether it did (read after the next barrier).
template <class R>
__device__ __forceinline__ void tile_prefetch_next(Smem<R>& S, const StageLaunch& a) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int pre = 0;
    const int next = S.next;
    if (next < a.nitems * a.stages) {
        const int2 si = stage_item(a, next);
        const int4 item = a.items[si.y];
        const Consts<R>& Kn = static_cast<const Consts<R>*>(a.consts)[item.x];
        const int x0 = item.y * kStripX, y0 = item.z;
        if (tile_rows(Kn, x0, y0 - kHalo, 2 * kHalo) && deps_ready(a, si.x, si.y, lane, false)) {
            __syncwarp();   // the lanes' acquire loads before lane 0's proxy fence
            if (lane == 0) {
                // the rows were written by other CTAs through the generic proxy
                asm volatile("fence.proxy.async.global;" ::: "memory");
                tile_fetch_from(S, a, si.x % 3, item.x, Kn.hlo, x0, y0 - kHalo);
            }
            pre = 1;
        }
    }
    if (lane == 0) S.pre = pre;
}

// The cell update reads W^n and dF_s/dt (stages 2 and 3) or F_s^{n-1}
// (stage 1) straight from global memory, where nothing has touched them
// during the step.  One warp asks L2 for rows r0 .. r0+7 of those arrays
// a chunk before their update: lane l takes row r0 + l % 8 and arrays
// l / 8 and l / 8 + 4 (the 7 state planes, then dF_s/dt), both ends of the
// strip's segment of each row.  Prefetches are hints: they change no value.
__device__ __forceinline__ void l2_prefetch(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

template <class R>
__device__ __forceinline__ void prefetch_update_rows(const Consts<R>& K, int stage, int x0, int r0, int y1, int lane) {
    const int r = r0 + (lane & 7);
    if (r >= y1) return;
    const long long c0 = (long long)r * K.nx + K.off + x0;
    const long long c1 = (long long)r * K.nx + K.off + min(x0 + kStripX, K.nx) - 1;
    const int k = lane >> 3;
    if (stage == 0) {
        if (k == 0) {
            const R* f = reinterpret_cast<const R*>(K.Fsp);
            l2_prefetch(f + c0);
            l2_prefetch(f + c1);
        }
        return;
    }
    const R* w = reinterpret_cast<const R*>(K.st[0]);
    l2_prefetch(w + k * K.plane + c0);
    l2_prefetch(w + k * K.plane + c1);
    const R* b = k + 4 < Prec<R>::NP ? w + (k + 4) * K.plane : reinterpret_cast<const R*>(K.dFs);
    if (k + 4 <= Prec<R>::NP) {
        l2_prefetch(b + c0);
        l2_prefetch(b + c1);
    }
}

__device__ __forceinline__ bool bar_try_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

// The bounded retry loop (out of line: the tile has normally landed long
// before its chunk starts, and the first try succeeds).
__device__ __noinline__ bool bar_wait_bounded(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    while (!bar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}

// Wait for the copy issued last; false if the bound ran out.
template <class R>
__device__ __forceinline__ bool tile_wait(Smem<R>& S, TileIO& io) {
    const unsigned bar = smem_addr(&S.tile_bar), parity = io.phase & 1u;
    ++io.phase;
    return bar_try_wait(bar, parity) || bar_wait_bounded(bar, parity);
}

// The state of tile column cc (0 .. RW-1 of the strip) in row rr.
__device__ __forceinline__ SV<float> tile_state(const float* t) {
    constexpr int PS = kChunk * kTileX;
    SV<float> s;
    s.Hh = t[0]; s.Hl = t[PS]; s.p = t[2 * PS]; s.mx = t[3 * PS]; s.my = t[4 * PS]; s.Ch = t[5 * PS]; s.Cl = t[6 * PS];
    return s;
}
__device__ __forceinline__ SV<double> tile_state(const double* t) {
    constexpr int PS = kChunk * kTileX;
    SV<double> s;
    s.Hh = t[0]; s.Hl = 0.0; s.p = t[PS]; s.mx = t[2 * PS]; s.my = t[3 * PS]; s.Ch = t[4 * PS]; s.Cl = 0.0;
    return s;
}

// Step 1: rows [r0, r0 + nrows) of the strip (all RW columns).
template <class R>
__device__ __forceinline__ void store_prim(Smem<R>& S, int s, int cc, const Prim<R>& q) {
    S.P.uv[s][cc] = P2<R>{q.u, q.v};
    S.P.rc[s][cc] = P2<R>{q.rho, q.C};
    S.P.tc[s][cc] = P2<R>{q.T, q.cp};
    S.P.pm[s][cc].x = q.p;     // mu_c follows in step 2
    S.P.lm[s][cc] = P2<R>{q.lam, q.mu};
    S.P.fl[s][cc] = q.Fl;
}

template <class R>
__device__ __forceinline__ void load_rows(Smem<R>& S, const R* in, int x0, int r0, int nrows) {
    const Consts<R>& K = S.K;
    const int total = nrows * RW;
    if (x0 >= kHalo && x0 + kStripX + kHalo <= K.nx && r0 >= -K.hlo && r0 + nrows <= K.ny + K.hhi) {
        // every cell of these rows is inside the domain (or a slab's halo):
        // no boundary mapping
        const long long base = (long long)r0 * K.nx + (x0 - kHalo) + K.off;
        for (int idx = threadIdx.x; idx < total; idx += NT) {
            const int rr = idx / RW, cc = idx - rr * RW;
            const SV<R> w = load_state(in, K.plane, base + (long long)rr * K.nx + cc);
            store_prim(S, slot(r0 + rr), cc, derive(K, w));
        }
        return;
    }
    for (int idx = threadIdx.x; idx < total; idx += NT) {
        const int rr = idx / RW, cc = idx - rr * RW;
        const int gy = r0 + rr, gx = x0 + cc - kHalo;
        int sx, kx, sdx, sy, ky, sdy;
        map_axis(gx, K.nx, K.per_x, XLO, sx, kx, sdx);
        map_row(K, gy, sy, ky, sdy);
        const SV<R> w = load_state(in, K.plane, (long long)sy * K.nx + sx + K.off);
        Prim<R> q = derive(K, w);
        // x sides first, then y (corners); an x ghost takes the wetting of its
        // (interior) row, a y ghost that of its column
        if (kx) apply_ghost(K, sdx, kx, true, wall_wetting(K, in, sdx, sy), q);
        if (ky) apply_ghost(K, sdy, ky, false, wall_wetting(K, in, sdy, gx), q);
        store_prim(S, slot(gy), cc, q);
    }
}

// Step 1 from a tile: rows [r0, r0 + nrows) (all inside the domain, see
// tile_rows) read from shared memory instead of global memory.
template <class R>
__device__ __forceinline__ void load_rows_tile(Smem<R>& S, int x0, int r0, int nrows) {
    const Consts<R>& K = S.K;
    const int xoff = (x0 - kHalo) - tile_x<R>(x0);
    const int total = nrows * RW;
    for (int idx = threadIdx.x; idx < total; idx += NT) {
        const int rr = idx / RW, cc = idx - rr * RW;
        store_prim(S, slot(r0 + rr), cc, derive(K, tile_state(&S.tile[0][rr][cc + xoff])));
    }
}

// The barrier after a load phase; true (on every thread) if some thread's
// tile wait gave up.  Without tiles (FP64) a plain barrier.
template <class R>
__device__ __forceinline__ bool load_barrier_failed(Smem<R>& S, bool ok) {
    if constexpr (sizeof(R) == 4) {
        return __syncthreads_or(!ok) != 0;
    } else {
        __syncthreads();
        return false;
    }
}
// A tile wait gave up: report it, wait (with the same bound) for the copy
// still in flight so that it cannot land in shared memory after the CTA has
// left, and stop.
// A wait for the items an item reads gave up (whole-step launches): report
// it as a bounded wait that gave up, wait for a prologue tile that may be in
// flight, and stop.
template <class R>
__device__ __noinline__ void dep_abort(Smem<R>& S, TileIO io, int* flag) {
    if (threadIdx.x == 0) atomicOr(flag, 2);
    if constexpr (sizeof(R) == 4)
        if (S.pre) tile_wait(S, io);
}

template <class R>
__device__ __noinline__ bool tile_abort(Smem<R>& S, TileIO io, int* flag) {
    if (threadIdx.x == 0) atomicOr(flag, 2);
    --io.phase;
    tile_wait(S, io);
    return false;
}

// mu_c = 2 beta C (C-1)(2C-1) - kappa lap C (reading R5) at ring offset s0
// (column gx of the domain) with the y-neighbours at sN, sS.  The Laplacian
// is the 5-point one, or in an axisymmetric domain the conservative
// (1/r) d/dr (r dC/dr) + d2C/dz2 with faces at r = gx and gx + 1.
template <class R, bool AXI>
__device__ __forceinline__ R chem_potential_of(const Consts<R>& K, R c, R ce, R cw, R cn, R cs, int gx) {
    R lap;
    if (AXI) {
        const R rw = (R)gx, re = rw + R(1);
        lap = wdiv(re * (ce - c) - rw * (c - cw), rw + R(0.5)) + (cn + cs - R(2) * c);
    } else {
        lap = ce + cw + cn + cs - R(4) * c;
    }
    const Q4<R> cc = ld4(K.cellc2);   // 2 beta, kappa
    return cc.x * c * (c - R(1)) * (R(2) * c - R(1)) - cc.y * lap;
}

template <class R, bool AXI>
__device__ __forceinline__ R chem_potential(const Consts<R>& K, const P2<R>* RC, int s0, int sN, int sS, int gx) {
    return chem_potential_of<R, AXI>(K, RC[s0].y, RC[s0 + 1].y, RC[s0 - 1].y, RC[sN].y, RC[sS].y, gx);
}

// True if mu_c of rows [r0, r0 + nrows) of the strip involves no wall ghost
// (the in-place Laplacian of muc_rows' first branch applies to all of them).
template <class R>
__device__ __forceinline__ bool muc_in_place(const Consts<R>& K, int x0, int r0, int nrows) {
    const int rlo = K.hlo ? 1 - K.hlo : 0, rhi = K.hhi ? K.ny + K.hhi - 1 : K.ny;
    return x0 >= kHalo - 1 && x0 + (RW - 2) - (kHalo - 1) <= K.nx && r0 >= rlo && r0 + nrows <= rhi;
}

// Steps 1 and 2 of an interior chunk from its tile (FP32C): rows
// [r0, r0 + kChunk) derived as in load_rows_tile and, by the same threads,
// mu_c of rows [r0 - 1, r0 + kChunk - 1) (muc_in_place must hold).  Their
// C comes from the tile (rows >= r0, C_hi + C_lo as derive forms it) or
// from the ring (rows r0 - 2, r0 - 1, derived by the previous chunk), so
// mu_c needs no barrier after the derive; the values are those muc_rows
// computes.
template <class R, bool AXI>
__device__ __forceinline__ void load_rows_tile_muc(Smem<R>& S, int x0, int r0, bool with_muc) {
    const Consts<R>& K = S.K;
    constexpr int PS = kChunk * kTileX;
    const int xoff = (x0 - kHalo) - tile_x<R>(x0);
    const R* t = &S.tile[0][0][0];
    for (int idx = threadIdx.x; idx < kChunk * RW; idx += NT) {
        const int rr = idx / RW, cc = idx - rr * RW;
        store_prim(S, slot(r0 + rr), cc, derive(K, tile_state(t + rr * kTileX + cc + xoff)));
    }
    if (!with_muc) return;
    // mu_c of ring row r0 + m, m = -1 .. kChunk-2, columns 1 .. RW-2
    const P2<R>* RC = &S.P.rc[0][0];
    constexpr int NC = RW - 2;
    for (int idx = threadIdx.x; idx < kChunk * NC; idx += NT) {
        const int m = idx / NC - 1, cc = 1 + idx - (m + 1) * NC;
        // C of row r0 + k at column cc + d: the tile for k >= 0, the ring below
        auto Cat = [&](int k, int d) -> R {
            const int ti = k * kTileX + cc + d + xoff;
            return k >= 0 ? t[5 * PS + ti] + t[6 * PS + ti] : RC[slot(r0 + k) * RW + cc + d].y;
        };
        S.P.pm[slot(r0 + m)][cc].y =
            chem_potential_of<R, AXI>(K, Cat(m, 0), Cat(m, 1), Cat(m, -1), Cat(m + 1, 0), Cat(m - 1, 0), x0 + cc - kHalo);
    }
}

// Step 2: mu_c for rows [r0, r0 + nrows), columns 1 .. RW-2.  A wall ghost
// (layer 1 or 2) evaluates mu_c at its mirror cell, which equals mirroring
// the interior value; deeper layers are never read by a face of the strip
// and get 0.
template <class R, bool AXI>
__device__ __forceinline__ void muc_rows(Smem<R>& S, int x0, int r0, int nrows) {
    const Consts<R>& K = S.K;
    constexpr int NC = RW - 2;
    const int total = nrows * NC;
    const P2<R>* C = &S.P.rc[0][0];
    // a slab's halo rows take mu_c in place, except the outermost (never read)
    const int rlo = K.hlo ? 1 - K.hlo : 0, rhi = K.hhi ? K.ny + K.hhi - 1 : K.ny;
    if (x0 >= kHalo - 1 && x0 + NC - (kHalo - 1) <= K.nx && r0 >= rlo && r0 + nrows <= rhi) {
        // no wall ghost among these cells: the Laplacian in place
        for (int idx = threadIdx.x; idx < total; idx += NT) {
            const int rr = idx / NC, cc = 1 + idx - rr * NC;
            const int gy = r0 + rr;
            const int s0 = slot(gy) * RW + cc;
            S.P.pm[slot(gy)][cc].y =
                chem_potential<R, AXI>(K, C, s0, slot(gy + 1) * RW + cc, slot(gy - 1) * RW + cc, x0 + cc - kHalo);
        }
        return;
    }
    for (int idx = threadIdx.x; idx < total; idx += NT) {
        const int rr = idx / NC, cc = 1 + idx - rr * NC;
        const int gy = r0 + rr, gx = x0 + cc - kHalo;
        int mc = cc, my = gy, deep = 0;
        if (!K.per_x) {
            if (gx < 0) { const int k = -gx; mc = cc + 2 * k - 1; deep |= k > 2; }
            else if (gx >= K.nx) { const int k = gx - K.nx + 1; mc = cc - (2 * k - 1); deep |= k > 2; }
        }
        if (gy < 0 && K.hlo) {
            deep |= gy < rlo;
        } else if (gy >= K.ny && K.hhi) {
            deep |= gy >= rhi;
        } else if (!K.per_y) {
            if (gy < 0) { const int k = -gy; my = gy + 2 * k - 1; deep |= k > 2; }
            else if (gy >= K.ny) { const int k = gy - K.ny + 1; my = gy - (2 * k - 1); deep |= k > 2; }
        }
        R mu = R(0);
        if (!deep)
            mu = chem_potential<R, AXI>(K, C, slot(my) * RW + mc, slot(my + 1) * RW + mc, slot(my - 1) * RW + mc,
                                x0 + mc - kHalo);
        S.P.pm[slot(gy)][cc].y = mu;
    }
}

// The 9 surrounding-point values of one field of a face (Eq. 54, R7), given
// the ring offsets of the L and R cells, their outer n-neighbours and their
// t-neighbours.
struct FaceIdx { int L, R, LL, RR, Lp, Lm, Rp, Rm; };

template <class R>
struct FaceFlux { R Fh, Fp, Fmn, Fmt, Fc, un; };

// Reconstruction pieces of one field: the cell values l, r, the face value
// o0 (mean of the two one-sided reconstructions l + (r - ll)/4 and
// r - (rr - l)/4, i.e. 5/8 (l + r) - 1/8 (ll + rr)) and the central
// t-differences dtl, dtr of the two cells (half-cell t-step = dt / 4).
template <class R>
struct Rec { R l, r, o0, dtl, dtr; };

template <class R>
__device__ __forceinline__ R face_value(R l, R r, R ll, R rr) {
    return R(0.625) * (l + r) - R(0.125) * (ll + rr);
}

template <class R>
__device__ __forceinline__ Rec<R> rec_of(R l, R r, R ll, R rr, R lp, R lm, R rp, R rm) {
    Rec<R> z;
    z.l = l;
    z.r = r;
    z.o0 = face_value(l, r, ll, rr);
    z.dtl = lp - lm;
    z.dtr = rp - rm;
    return z;
}

// The reconstruction pieces of both fields of a pair.
template <class R>
__device__ __forceinline__ void rec2(const P2<R>* f, const FaceIdx& x, Rec<R>& a, Rec<R>& b) {
    const P2<R> l = f[x.L], r = f[x.R], ll = f[x.LL], rr = f[x.RR];
    const P2<R> lp = f[x.Lp], lm = f[x.Lm], rp = f[x.Rp], rm = f[x.Rm];
    a = rec_of(l.x, r.x, ll.x, rr.x, lp.x, lm.x, rp.x, rm.x);
    b = rec_of(l.y, r.y, ll.y, rr.y, lp.y, lm.y, rp.y, rm.y);
}

// Face values of both fields of a pair (cells L, R and their outer n-neighbours).
template <class R>
__device__ __forceinline__ void face_value2(const P2<R>* f, const FaceIdx& x, R& a, R& b) {
    const P2<R> l = f[x.L], r = f[x.R], ll = f[x.LL], rr = f[x.RR];
    a = face_value(l.x, r.x, ll.x, rr.x);
    b = face_value(l.y, r.y, ll.y, rr.y);
}

// The nonlinear parts of the equilibrium moments over the surrounding points
// of one side column of a face: the points x_f - e_a dt_s with e_n = sn
// (+1: the L cell, points 1, 5, 8; -1: the R cell, points 3, 6, 7).  The
// column's centre point (e_t = 0) takes the cell values; its t-points
// (e_t = +1 / -1) the cell value minus / plus a quarter of the central
// t-difference.  With q = e.u + 3/2 (e.u)^2 - 1/2 u^2 (cs^2 = 1/3):
//   centre:   q = sn u_n + u_n^2 - u_t^2 / 2
//   t-points: q = e.u (1 + e.u) + e_n e_t u_n u_t
// Returned: at the centre rho q, C u_n, q, C_p T q; over the t-points the sum
// (e_t = +1 plus e_t = -1) of rho q, C e.u, q and C_p T q, and the difference
// (+1 minus -1) of rho q and q.
template <class R>
struct SideSums { R f0, c0, q0, h0, fs, fd, cs, qs, qd, hs; };

template <class R, int SN>
__device__ __forceinline__ SideSums<R> side_sums(R un, R ut, R rho, R C, R T, R cp, R dun, R dut, R drho, R dC,
                                                 R dT, R dcp) {
    SideSums<R> s;
    const R sun = SN > 0 ? un : -un;
    s.q0 = fma(un, un, fma(R(-0.5) * ut, ut, sun));
    s.f0 = rho * s.q0;
    s.c0 = C * un;
    s.h0 = (cp * T) * s.q0;
    // e_t = +1: value - d/4; e_t = -1: value + d/4
    const R unp = fma(R(-0.25), dun, un), unm = fma(R(0.25), dun, un);
    const R utp = fma(R(-0.25), dut, ut), utm = fma(R(0.25), dut, ut);
    const R eup = (SN > 0 ? unp : -unp) + utp;
    const R eum = (SN > 0 ? unm : -unm) - utm;
    const R qp = fma(SN > 0 ? unp : -unp, utp, fma(eup, eup, eup));      // e_n e_t = sn
    const R qm = fma(SN > 0 ? -unm : unm, utm, fma(eum, eum, eum));      // e_n e_t = -sn
    const R rp = fma(R(-0.25), drho, rho), rm = fma(R(0.25), drho, rho);
    const R am = rm * qm;
    s.fs = fma(rp, qp, am);
    s.fd = fma(rp, qp, -am);
    const R Cp_ = fma(R(-0.25), dC, C), Cm_ = fma(R(0.25), dC, C);
    s.cs = fma(Cp_, eup, Cm_ * eum);
    s.qs = qp + qm;
    s.qd = qp - qm;
    const R hp = fma(R(-0.25), dcp, cp) * fma(R(-0.25), dT, T);
    const R hm = fma(R(0.25), dcp, cp) * fma(R(0.25), dT, T);
    s.hs = fma(hp, qp, hm * qm);
    return s;
}

// Sec. 2.5 steps (2)-(4) and Eq. 53 for one face.
//
// The face equilibria enter only through their closed moments (C_p T u_n,
// cs^2 (p + rho u_n^2), cs^2 rho u_n u_t, C u_n; Eq. 11 and the moments of
// Eq. 29, 42).  The sums over the surrounding points x_f - e_a dt_s are
// split into their parts linear in one reconstructed field, which have
// closed forms because the reconstruction is linear (the t-offsets cancel in
// pairs):
//   sum w p = 2/3 p_0 + (p_L + p_R)/6          sum e_n w p = (p_L - p_R)/6
//   sum e_t w p = -(dp_L + dp_R)/24             sum e_n e_t w p = (dp_R - dp_L)/72
//   sum_{e_n != 0} w p = (p_L + p_R)/6
//   mu_c part of sum g = Q ((mu_L + mu_R)/2 - mu_0), of sum e_n g = Q (mu_L - mu_R)/2
//   C_ref T part of sum e_n h = C_ref (T_L - T_R)/6
// (dp = central t-difference), and the nonlinear parts (rho q, C e.u,
// C_p T q, q), which are summed over the points by columns of equal e_n
// (side_sums above, and the face column e_n = 0 below) so that each sign
// pattern of the moments is one sum or difference of column sums.
//
// Axisymmetric domains (reading R24): the face pressure is advanced with the
// axisymmetric mass source -rho cs^2 u_r / r as well, streamed with weight
// w_a over dt_s.  Of the fluxes only the normal momentum flux changes, by
// cs^2 dt_s (-rho_f cs^2 u_r / r) = -rho_f u_r / (18 r) with the face values;
// inv_r = 1 / r of the face (0 on the axis, where the face area is zero).
//
// The arithmetic is written for a value type T (the working precision) and a
// source Src of the reconstruction pieces (RingFace: one face of the ring).
template <class T, class R, bool AXI, class Src>
__device__ __forceinline__ FaceFlux<T> face_math(const Q4<R>& fc, const Src& src, T inv_r) {
    Rec<T> n, t, rho, C, T_, cp;
    src.vel(n, t);               // normal and tangential velocity
    src.rc(rho, C);
    src.tc(T_, cp);

    // side columns: L (points 1, 5, 8) and R (points 3, 6, 7)
    const SideSums<T> L = side_sums<T, 1>(n.l, t.l, rho.l, C.l, T_.l, cp.l, n.dtl, t.dtl, rho.dtl, C.dtl, T_.dtl,
                                          cp.dtl);
    const SideSums<T> Rs = side_sums<T, -1>(n.r, t.r, rho.r, C.r, T_.r, cp.r, n.dtr, t.dtr, rho.dtr, C.dtr, T_.dtr,
                                            cp.dtr);

    // face column (e_n = 0): point 0 at the face value, points 2 (e_t = +1)
    // and 4 (e_t = -1) shifted by the mean t-step; there
    // q = e_t u_t + u_t^2 - u_n^2 / 2, and at point 0 q = -u^2 / 2
    const T stn = T(0.125) * (n.dtl + n.dtr), stt = T(0.125) * (t.dtl + t.dtr);
    const T str = T(0.125) * (rho.dtl + rho.dtr), stc = T(0.125) * (C.dtl + C.dtr);
    const T un2 = n.o0 - stn, un4 = n.o0 + stn, ut2 = t.o0 - stt, ut4 = t.o0 + stt;
    const T q2 = fma(ut2, ut2, fma(T(-0.5) * un2, un2, ut2));
    const T q4 = fma(ut4, ut4, fma(T(-0.5) * un4, un4, -ut4));
    const T a4 = (rho.o0 + str) * q4;
    const T f24s = fma(rho.o0 - str, q2, a4);     // rho q at 2 plus at 4
    const T f24d = fma(rho.o0 - str, q2, -a4);    // rho q at 2 minus at 4
    const T c24 = fma(C.o0 - stc, ut2, -((C.o0 + stc) * ut4));   // C e.u at 2 plus at 4
    const T rho_f = rho.o0;
    const T ruu0 = rho_f * fma(n.o0, n.o0, t.o0 * t.o0);       // -2 rho q at point 0

    Rec<T> p, muc;
    src.pm(p, muc);
    T lamf, muf;
    src.lm(lamf, muf);
    const T fQ = T(fc.x), fC = T(fc.y), fI = T(fc.z);   // Q, C_ref / 6, 6 / C_ref; fc.w = tau_g - 1/2

    // Eq. 56 and the moments of the surrounding equilibria; weights 4/9, 1/9
    // (e_n or e_t zero) and 1/36 (diagonal)
    const T w1 = T(1.0 / 9.0), w5 = T(1.0 / 36.0);
    const T pf = T(2.0 / 3.0) * p.o0 + T(1.0 / 6.0) * (p.l + p.r) - T(2.0 / 9.0) * ruu0 +
                 w1 * ((L.f0 + Rs.f0) + f24s) + w5 * (L.fs + Rs.fs);
    const T mn = T(1.0 / 6.0) * (p.l - p.r) + w1 * (L.f0 - Rs.f0) + w5 * (L.fs - Rs.fs);
    const T mt = T(-1.0 / 24.0) * (p.dtl + p.dtr) + w1 * f24d + w5 * (L.fd + Rs.fd);
    const T Cf = C.o0 + fQ * (T(0.5) * (muc.l + muc.r) - muc.o0) + T(1.0 / 3.0) * ((L.c0 - Rs.c0) + c24) +
                 T(1.0 / 12.0) * (L.cs + Rs.cs);
    const T Sg = T(0.5) * fQ * (muc.l - muc.r) + T(1.0 / 3.0) * (L.c0 + Rs.c0) + T(1.0 / 12.0) * (L.cs - Rs.cs);
    const T Sh = fC * (T_.l - T_.r) + T(1.0 / 3.0) * (L.h0 - Rs.h0) + T(1.0 / 12.0) * (L.hs - Rs.hs);
    const T Snn_p = T(1.0 / 6.0) * (p.l + p.r);
    const T Snt_p = T(1.0 / 72.0) * (p.dtr - p.dtl);
    const T Snn_q = w1 * (L.q0 + Rs.q0) + w5 * (L.qs + Rs.qs);
    const T Snt_q = w5 * (L.qd - Rs.qd);
    // rho_f cs^2 u_f = sum e f^eq (Eq. 56); tau from the face properties (R9)
    const T irf = wdiv(T(1), rho_f);
    const T unf = T(3) * mn * irf, utf = T(3) * mt * irf;
    const T th = fI * lamf * irf;                // tau_h - 0.5 = lambda / (rho C_ref cs^2 dt_s)
    const T tf = T(6) * muf * irf;               // tau_f - 0.5 = mu / (rho cs^2 dt_s)
    const T tg = T(fc.w);
    const T cs2 = T(1.0 / 3.0);
    FaceFlux<T> F;
    // h* = (1.5 - tau) h^eq(x_f) + (tau - 0.5) h^eq(x_f - e dt_s) (Eq. 13, 16)
    F.Fh = (T(1) - th) * (cp.o0 * T_.o0) * unf + th * Sh;
    F.Fp = mn;                                    // sum e_n f^eq(x_f) = rho_f cs^2 u_n,f
    // f* = (1.5 - tau_f) f^eq(x_f) + (tau_f - 0.5) f^eq-m (Eq. 35, 37 with R3)
    F.Fmn = (T(1) - tf) * cs2 * (pf + rho_f * unf * unf) + tf * (Snn_p + rho_f * Snn_q);
    F.Fmt = (T(1) - tf) * cs2 * rho_f * unf * utf + tf * (Snt_p + rho_f * Snt_q);
    F.Fc = (T(1) - tg) * Cf * unf + tg * Sg;     // Eq. 44, 46
    F.un = unf;
    if (AXI) F.Fmn += T(-1.0 / 18.0) * rho_f * src.radial(n.o0, t.o0) * inv_r;
    return F;
}

// The pieces of one face from the ring, in the working precision.
template <class R>
struct RingFace {
    const Ring<R>& P;
    const FaceIdx& x;
    bool normal_x, normal_is_r;
    __device__ __forceinline__ void vel(Rec<R>& n, Rec<R>& t) const {
        Rec<R> ru, rv;
        rec2(&P.uv[0][0], x, ru, rv);
        n = normal_x ? ru : rv;
        t = normal_x ? rv : ru;
    }
    __device__ __forceinline__ void rc(Rec<R>& a, Rec<R>& b) const { rec2(&P.rc[0][0], x, a, b); }
    __device__ __forceinline__ void tc(Rec<R>& a, Rec<R>& b) const { rec2(&P.tc[0][0], x, a, b); }
    __device__ __forceinline__ void pm(Rec<R>& a, Rec<R>& b) const { rec2(&P.pm[0][0], x, a, b); }
    __device__ __forceinline__ void lm(R& a, R& b) const { face_value2(&P.lm[0][0], x, a, b); }
    __device__ __forceinline__ R radial(R n0, R t0) const { return normal_is_r ? n0 : t0; }
};

template <class R, bool AXI>
__device__ __forceinline__ FaceFlux<R> face_flux(const Consts<R>& K, const Ring<R>& P, const FaceIdx& x, bool normal_x,
                                                 bool normal_is_r, R inv_r) {
    const RingFace<R> src{P, x, normal_x, normal_is_r};
    return face_math<R, R, AXI>(ld4(K.facec), src, inv_r);
}


// ---------------------------------------------------------------------------
// General streaming steps (reading R26): h, f and g take their surrounding
// points at x_f - e_a dt_h, dt_f, dt_g.  A side point then lies inside its
// cell at distance a = 1/2 - dt from the centre along n and dt along t, so
// its value is f' -/+ (dt/2) d_t f with f' = f + a g_n (g_n the central
// n-slope of that cell); the face points move by -/+ (dt/4)(d_t f_L + d_t f_R).
// The closed forms of the linear parts keep their shape with f' for f and
// dt/12, dt/36 for the t-moments; the nonlinear sums run once per
// distribution on its own points, by face columns as in face_flux (the
// centre of a side column at f', its t-points at f' -/+ (dt/2) d_t f).  Used
// only when some step differs from 1/2; face_flux above is this with a = 0,
// dt = 1/2.
// ---------------------------------------------------------------------------
template <class R>
struct RecN { R l, r, gl, gr, o0, dtl, dtr; };

template <class R>
__device__ __forceinline__ RecN<R> recn_of(R l, R r, R ll, R rr, R lp, R lm, R rp, R rm) {
    RecN<R> z;
    z.l = l;
    z.r = r;
    z.gl = R(0.5) * (r - ll);
    z.gr = R(0.5) * (rr - l);
    z.o0 = R(0.5) * ((z.l + R(0.5) * z.gl) + (z.r - R(0.5) * z.gr));
    z.dtl = lp - lm;
    z.dtr = rp - rm;
    return z;
}

template <class R>
__device__ __forceinline__ void recn2(const P2<R>* f, const FaceIdx& x, RecN<R>& a, RecN<R>& b) {
    const P2<R> l = f[x.L], r = f[x.R], ll = f[x.LL], rr = f[x.RR];
    const P2<R> lp = f[x.Lp], lm = f[x.Lm], rp = f[x.Rp], rm = f[x.Rm];
    a = recn_of(l.x, r.x, ll.x, rr.x, lp.x, lm.x, rp.x, rm.x);
    b = recn_of(l.y, r.y, ll.y, rr.y, lp.y, lm.y, rp.y, rm.y);
}

// q at the centre of a side column (e_n = SN, e_t = 0) and at its t-points
// (e_t = +1: value - d, e_t = -1: value + d), with e.u at the t-points; the
// forms of side_sums above.
template <class R, int SN>
__device__ __forceinline__ R q_centre(R un, R ut) {
    return fma(un, un, fma(R(-0.5) * ut, ut, SN > 0 ? un : -un));
}

template <class R, int SN>
__device__ __forceinline__ void eu_tpoints(R un, R ut, R dun, R dut, R& unp, R& utp, R& unm, R& utm, R& eup, R& eum) {
    unp = un - dun; unm = un + dun; utp = ut - dut; utm = ut + dut;
    eup = (SN > 0 ? unp : -unp) + utp;
    eum = (SN > 0 ? unm : -unm) - utm;
}

template <class R, int SN>
__device__ __forceinline__ void q_tpoints(R un, R ut, R dun, R dut, R& qp, R& qm) {
    R unp, utp, unm, utm, eup, eum;
    eu_tpoints<R, SN>(un, ut, dun, dut, unp, utp, unm, utm, eup, eum);
    qp = fma(SN > 0 ? unp : -unp, utp, fma(eup, eup, eup));      // e_n e_t = SN
    qm = fma(SN > 0 ? -unm : unm, utm, fma(eum, eum, eum));      // e_n e_t = -SN
}

// The value of one field at the centre of a side column for a streaming step
// with a = 1/2 - dt: the L cell's f + a g_n, the R cell's f - a g_n.
template <class R, int SN>
__device__ __forceinline__ R col_centre(const RecN<R>& z, R a) {
    return SN > 0 ? fma(a, z.gl, z.l) : fma(-a, z.gr, z.r);
}
template <class R, int SN>
__device__ __forceinline__ R col_dt(const RecN<R>& z) { return SN > 0 ? z.dtl : z.dtr; }

// f (points at dt_f): rho q and q of one side column; sums and differences
// over the t-points as in side_sums.
template <class R>
struct ColF { R f0, q0, fs, fd, qs, qd; };

template <class R, int SN>
__device__ __forceinline__ ColF<R> col_f(const RecN<R>& Un, const RecN<R>& Ut, const RecN<R>& Rho, R a, R b) {
    ColF<R> s;
    const R un = col_centre<R, SN>(Un, a), ut = col_centre<R, SN>(Ut, a), rho = col_centre<R, SN>(Rho, a);
    s.q0 = q_centre<R, SN>(un, ut);
    s.f0 = rho * s.q0;
    R qp, qm;
    q_tpoints<R, SN>(un, ut, b * col_dt<R, SN>(Un), b * col_dt<R, SN>(Ut), qp, qm);
    const R dr = b * col_dt<R, SN>(Rho);
    const R am = (rho + dr) * qm;
    s.fs = fma(rho - dr, qp, am);
    s.fd = fma(rho - dr, qp, -am);
    s.qs = qp + qm;
    s.qd = qp - qm;
    return s;
}

// g (points at dt_g): C u_n at the centre and the t-points' sum of C e.u.
template <class R, int SN>
__device__ __forceinline__ void col_g(const RecN<R>& Un, const RecN<R>& Ut, const RecN<R>& Cc, R a, R b, R& c0, R& cs) {
    const R un = col_centre<R, SN>(Un, a), ut = col_centre<R, SN>(Ut, a), C = col_centre<R, SN>(Cc, a);
    c0 = C * un;
    R unp, utp, unm, utm, eup, eum;
    eu_tpoints<R, SN>(un, ut, b * col_dt<R, SN>(Un), b * col_dt<R, SN>(Ut), unp, utp, unm, utm, eup, eum);
    const R dC = b * col_dt<R, SN>(Cc);
    cs = fma(C - dC, eup, (C + dC) * eum);
}

// h (points at dt_h): C_p T q at the centre and the t-points' sum.
template <class R, int SN>
__device__ __forceinline__ void col_h(const RecN<R>& Un, const RecN<R>& Ut, const RecN<R>& T, const RecN<R>& cp, R a,
                                      R b, R& h0, R& hs) {
    const R un = col_centre<R, SN>(Un, a), ut = col_centre<R, SN>(Ut, a);
    const R Tc = col_centre<R, SN>(T, a), cc = col_centre<R, SN>(cp, a);
    h0 = (cc * Tc) * q_centre<R, SN>(un, ut);
    R qp, qm;
    q_tpoints<R, SN>(un, ut, b * col_dt<R, SN>(Un), b * col_dt<R, SN>(Ut), qp, qm);
    const R dT = b * col_dt<R, SN>(T), dc = b * col_dt<R, SN>(cp);
    hs = fma((cc - dc) * (Tc - dT), qp, ((cc + dc) * (Tc + dT)) * qm);
}

template <class R, bool AXI>
__device__ __forceinline__ FaceFlux<R> face_flux_gen(const Consts<R>& K, const Ring<R>& P, const FaceIdx& x,
                                                     bool normal_x, bool normal_is_r, R inv_r) {
    const R w1 = R(1.0 / 9.0), w5 = R(1.0 / 36.0);
    RecN<R> Un, Ut;
    recn2(&P.uv[0][0], x, Un, Ut);
    if (!normal_x) { const RecN<R> t = Un; Un = Ut; Ut = t; }
    RecN<R> Rho, Cc;
    recn2(&P.rc[0][0], x, Rho, Cc);
    // f: points at dt_f; the face column (e_n = 0) shifts by (dt/4)(d_t f_L + d_t f_R)
    R pf_n, mn_n, mt_n, Snn_q, Snt_q;
    const R rho_f = Rho.o0;
    {
        const R a = R(0.5) - K.dtf, b = R(0.5) * K.dtf, h = R(0.5) * b;
        const ColF<R> L = col_f<R, 1>(Un, Ut, Rho, a, b);
        const ColF<R> Rs = col_f<R, -1>(Un, Ut, Rho, a, b);
        const R stn = h * (Un.dtl + Un.dtr), stt = h * (Ut.dtl + Ut.dtr), str = h * (Rho.dtl + Rho.dtr);
        const R un2 = Un.o0 - stn, un4 = Un.o0 + stn, ut2 = Ut.o0 - stt, ut4 = Ut.o0 + stt;
        const R q2 = fma(ut2, ut2, fma(R(-0.5) * un2, un2, ut2));
        const R q4 = fma(ut4, ut4, fma(R(-0.5) * un4, un4, -ut4));
        const R a4 = (Rho.o0 + str) * q4;
        const R f24s = fma(Rho.o0 - str, q2, a4), f24d = fma(Rho.o0 - str, q2, -a4);
        const R ruu0 = rho_f * fma(Un.o0, Un.o0, Ut.o0 * Ut.o0);
        pf_n = R(-2.0 / 9.0) * ruu0 + w1 * ((L.f0 + Rs.f0) + f24s) + w5 * (L.fs + Rs.fs);
        mn_n = w1 * (L.f0 - Rs.f0) + w5 * (L.fs - Rs.fs);
        mt_n = w1 * f24d + w5 * (L.fd + Rs.fd);
        Snn_q = w1 * (L.q0 + Rs.q0) + w5 * (L.qs + Rs.qs);
        Snt_q = w5 * (L.qd - Rs.qd);
    }
    // g: points at dt_g
    R ce_a, cen_a, ce_d, cen_d;
    {
        const R a = R(0.5) - K.dtg, b = R(0.5) * K.dtg, h = R(0.5) * b;
        R c0L, csL, c0R, csR;
        col_g<R, 1>(Un, Ut, Cc, a, b, c0L, csL);
        col_g<R, -1>(Un, Ut, Cc, a, b, c0R, csR);
        const R stt = h * (Ut.dtl + Ut.dtr), stc = h * (Cc.dtl + Cc.dtr);
        const R c24 = fma(Cc.o0 - stc, Ut.o0 - stt, -((Cc.o0 + stc) * (Ut.o0 + stt)));
        ce_a = (c0L - c0R) + c24;
        cen_a = c0L + c0R;
        ce_d = csL + csR;
        cen_d = csL - csR;
    }
    // h: points at dt_h (only e_n != 0 points carry C_p T q into the flux)
    RecN<R> T, cp;
    recn2(&P.tc[0][0], x, T, cp);
    R th_a, th_d;
    {
        const R a = R(0.5) - K.dth, b = R(0.5) * K.dth;
        R h0L, hsL, h0R, hsR;
        col_h<R, 1>(Un, Ut, T, cp, a, b, h0L, hsL);
        col_h<R, -1>(Un, Ut, T, cp, a, b, h0R, hsR);
        th_a = h0L - h0R;
        th_d = hsL - hsR;
    }
    RecN<R> p, mu;
    recn2(&P.pm[0][0], x, p, mu);
    R lamf, muf;
    face_value2(&P.lm[0][0], x, lamf, muf);
    const Q4<R> fc = ld4(K.facec);   // Q, C_ref / 6, 6 / C_ref, tau_g - 1/2
    const R af = R(0.5) - K.dtf, ag = R(0.5) - K.dtg, ah = R(0.5) - K.dth;
    const R pl = p.l + af * p.gl, pr = p.r - af * p.gr;
    const R ml = mu.l + ag * mu.gl, mr = mu.r - ag * mu.gr;
    const R Tl = T.l + ah * T.gl, Tr = T.r - ah * T.gr;
    const R pf = R(2.0 / 3.0) * p.o0 + R(1.0 / 6.0) * (pl + pr) + pf_n;
    const R mn = R(1.0 / 6.0) * (pl - pr) + mn_n;
    const R mt = -(K.dtf * R(1.0 / 12.0)) * (p.dtl + p.dtr) + mt_n;
    const R Cf = Cc.o0 + fc.x * (R(0.5) * (ml + mr) - mu.o0) + R(1.0 / 3.0) * ce_a + R(1.0 / 12.0) * ce_d;
    const R Sg = R(0.5) * fc.x * (ml - mr) + R(1.0 / 3.0) * cen_a + R(1.0 / 12.0) * cen_d;
    const R Sh = fc.y * (Tl - Tr) + R(1.0 / 3.0) * th_a + R(1.0 / 12.0) * th_d;
    const R Snn_p = R(1.0 / 6.0) * (pl + pr);
    const R Snt_p = (K.dtf * R(1.0 / 36.0)) * (p.dtr - p.dtl);
    const R irf = wdiv(R(1), rho_f);
    const R unf = R(3) * mn * irf, utf = R(3) * mt * irf;
    const R th = K.th_coef * lamf * irf;
    const R tf = K.tf_coef * muf * irf;
    const R tg = fc.w;
    const R cs2 = R(1.0 / 3.0);
    FaceFlux<R> F;
    F.Fh = (R(1) - th) * (cp.o0 * T.o0) * unf + th * Sh;
    F.Fp = mn;
    F.Fmn = (R(1) - tf) * cs2 * (pf + rho_f * unf * unf) + tf * (Snn_p + rho_f * Snn_q);
    F.Fmt = (R(1) - tf) * cs2 * rho_f * unf * utf + tf * (Snt_p + rho_f * Snt_q);
    F.Fc = (R(1) - tg) * Cf * unf + tg * Sg;
    F.un = unf;
    if (AXI) F.Fmn += -(K.dtf * R(1.0 / 9.0)) * rho_f * (normal_is_r ? Un.o0 : Ut.o0) * inv_r;
    return F;
}

// Step 3, x-faces of ring row r: lane l computes the face between columns
// l+2 and l+3 (cells x0+l-1 and x0+l), at x = x0 + l.  In an axisymmetric
// domain the stored fluxes are multiplied by the face area r_f = x0 + l.
template <class R, bool AXI, bool GEN>
__device__ __forceinline__ void x_face(Smem<R>& S, int x0, int r, int row_in_chunk, int lane, R inv_rf) {
    FaceIdx x;
    const int cL = lane + 2;
    x.L = slot(r) * RW + cL;
    x.R = x.L + 1;
    x.LL = x.L - 1;
    x.RR = x.L + 2;
    x.Lp = slot(r + 1) * RW + cL;
    x.Lm = slot(r - 1) * RW + cL;
    x.Rp = x.Lp + 1;
    x.Rm = x.Lm + 1;
    const R rf = AXI ? (R)(x0 + lane) : R(1);
    FaceFlux<R> F = GEN ? face_flux_gen<R, AXI>(S.K, S.P, x, true, true, inv_rf)
                        : face_flux<R, AXI>(S.K, S.P, x, true, true, inv_rf);
    if (AXI) {
        F.Fh *= rf; F.Fp *= rf; F.Fmn *= rf; F.Fmt *= rf; F.Fc *= rf; F.un *= rf;
    }
    S.XF[0][row_in_chunk][lane] = P2<R>{F.Fh, F.Fp};
    S.XF[1][row_in_chunk][lane] = P2<R>{F.Fmn, F.Fmt};   // x-, y-momentum
    S.XF[2][row_in_chunk][lane] = P2<R>{F.Fc, F.un};
}

// Step 3, y-faces of face row r (between rows r-1 and r), lane l < 31 at
// column l+3 (cell x0 + l, radius x0 + l + 1/2 in an axisymmetric domain).
template <class R, bool AXI, bool GEN>
__device__ __forceinline__ void y_face(Smem<R>& S, int r, int lane, R inv_r) {
    FaceIdx x;
    const int c = lane + kHalo;
    x.L = slot(r - 1) * RW + c;
    x.R = slot(r) * RW + c;
    x.LL = slot(r - 2) * RW + c;
    x.RR = slot(r + 1) * RW + c;
    x.Lp = x.L + 1;
    x.Lm = x.L - 1;
    x.Rp = x.R + 1;
    x.Rm = x.R - 1;
    const FaceFlux<R> F = GEN ? face_flux_gen<R, AXI>(S.K, S.P, x, false, false, inv_r)
                              : face_flux<R, AXI>(S.K, S.P, x, false, false, inv_r);
    const int s = slot(r);
    S.YF[0][s][lane] = P2<R>{F.Fh, F.Fp};
    S.YF[1][s][lane] = P2<R>{F.Fmt, F.Fmn};   // x-, y-momentum
    S.YF[2][s][lane] = P2<R>{F.Fc, F.un};
}

// Step 4 for the cell (r, x0 + lane).
template <class R, bool AXI>
__device__ __forceinline__ void cell_update(Smem<R>& S, int stage, int x0, int r, int row_in_chunk, int lane,
                                            R irc, int* flag) {
    const Consts<R>& K = S.K;
    const int gx = x0 + lane;
    const long long c = (long long)r * K.nx + gx + K.off;
    const int q = slot(r) * RW + lane + kHalo;
    const int qn = slot(r + 1) * RW + lane + kHalo, qs = slot(r - 1) * RW + lane + kHalo;
    const int sr = slot(r), sn = slot(r + 1);
    // Eq. 52; axisymmetric: the x-face fluxes carry their areas r_f, divided
    // here by the cell volume r_i = gx + 1/2 (per radian); irc = 1 / r_i
    R Rk[5], divu;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const P2<R> e = S.XF[k][row_in_chunk][lane + 1], w = S.XF[k][row_in_chunk][lane];
        const P2<R> n = S.YF[k][sn][lane], so = S.YF[k][sr][lane];
        const R dx0 = e.x - w.x, dx1 = e.y - w.y;
        const R d0 = -((AXI ? dx0 * irc : dx0) + (n.x - so.x));
        const R d1 = (AXI ? dx1 * irc : dx1) + (n.y - so.y);
        Rk[2 * k] = d0;
        if (k < 2) Rk[2 * k + 1] = -d1;
        else divu = d1;
    }
    const R divF1 = -Rk[1];   // div(rho cs^2 u), the pressure-flux divergence

    const Ring<R>& P = S.P;
    const P2<R> tc = (&P.tc[0][0])[q], rc = (&P.rc[0][0])[q], uv = (&P.uv[0][0])[q];
    const R T = tc.x, Cp = tc.y, rho = rc.x, C = rc.y, u = uv.x, v = uv.y;
    const R Fl = (&P.fl[0][0])[q];
    const P2<R>* RC = &P.rc[0][0];
    const P2<R>* PM = &P.pm[0][0];
    const R drx = R(0.5) * (RC[q + 1].x - RC[q - 1].x);
    const R dry = R(0.5) * (RC[qn].x - RC[qs].x);
    const R dmx = R(0.5) * (PM[q + 1].y - PM[q - 1].y);
    const R dmy = R(0.5) * (PM[qn].y - PM[qs].y);
    const Q4<R> cc = ld4(K.cellc);   // kv, g_x, g_y, 1 / dt
    R dfs;
    if (stage == 0) {   // reading R14: lagged dF_s/dt, fixed over the step
        R* Fsp = reinterpret_cast<R*>(K.Fsp);
        const R Fs = R(1) - Fl;
        dfs = (Fs - ld_l2(Fsp + c)) * cc.w;
        reinterpret_cast<R*>(K.dFs)[c] = dfs;
        Fsp[c] = Fs;
    } else {
        dfs = ld_l2(reinterpret_cast<const R*>(K.dFs) + c);
    }
    const R cs2 = R(1.0 / 3.0);
    const R D = solid_gate(K, C) * dfs;
    Rk[0] += Cp * T * divu;                                           // Eq. 51 row 1
    Rk[1] += u * (drx * cs2) + v * (dry * cs2) + rho * cs2 * cc.x * D;   // row 2
    Rk[2] += cs2 * (-Fl * C * dmx + rho * cc.y - rho * u * D);         // row 3 (R13)
    Rk[3] += cs2 * (-Fl * C * dmy + rho * cc.z - rho * v * D);         // row 4
    Rk[4] += C * cc.x * dfs;                                           // row 5 (R12: Eq. 40 / 47)
    const Q4<R> c2 = ld4(K.cellc2);   // dt, dt_f in z, w
    if (AXI)   // hoop stress Pi_thetatheta / r with the pressure advanced over dt_s (reading R24)
        Rk[2] += cs2 * (PM[q].x - c2.w * divF1 - R(2) * (&P.lm[0][0])[q].y * u * irc) * irc;

    // stage 0 reads W^n as its input: one load serves both
    const SV<R> wn = load_state(reinterpret_cast<const R*>(K.st[0]), K.plane, c);
    const SV<R> ws = stage == 0 ? wn : load_state(reinterpret_cast<const R*>(K.st[stage]), K.plane, c);
    SV<R> o;
    if constexpr (sizeof(R) == 8) {
        // Eq. 58 as written
        const R A = stage == 0 ? R(1) : (stage == 1 ? R(0.75) : R(1.0 / 3.0));
        const R B = stage == 0 ? R(0) : (stage == 1 ? R(0.25) : R(2.0 / 3.0));
        const R Cd = (stage == 0 ? R(1) : (stage == 1 ? R(0.25) : R(2.0 / 3.0))) * c2.z;
        o.Hh = A * wn.Hh + B * ws.Hh + Cd * Rk[0];
        o.p = A * wn.p + B * ws.p + Cd * Rk[1];
        o.mx = A * wn.mx + B * ws.mx + Cd * Rk[2];
        o.my = A * wn.my + B * ws.my + Cd * Rk[3];
        o.Ch = A * wn.Ch + B * ws.Ch + Cd * Rk[4];
        o.Hl = R(0);
        o.Cl = R(0);
    } else {
        // Eq. 58 as W^n + increment; H and C kept as compensated pairs.  TwoSum
        // for the sum and the renormalisation keeps every pair canonical.
        const R B = stage == 0 ? R(0) : (stage == 1 ? R(0.25) : R(2.0 / 3.0));
        const R Cd = (stage == 0 ? R(1) : (stage == 1 ? R(0.25) : R(2.0 / 3.0))) * c2.z;
        const R dH = B * ((ws.Hh - wn.Hh) + (ws.Hl - wn.Hl)) + Cd * Rk[0];
        const R dC = B * ((ws.Ch - wn.Ch) + (ws.Cl - wn.Cl)) + Cd * Rk[4];
        R s1, e1;
        two_sum(wn.Hh, dH, s1, e1);
        two_sum(s1, wn.Hl + e1, o.Hh, o.Hl);
        two_sum(wn.Ch, dC, s1, e1);
        two_sum(s1, wn.Cl + e1, o.Ch, o.Cl);
        o.p = wn.p + (B * (ws.p - wn.p) + Cd * Rk[1]);
        o.mx = wn.mx + (B * (ws.mx - wn.mx) + Cd * Rk[2]);
        o.my = wn.my + (B * (ws.my - wn.my) + Cd * Rk[3]);
    }
    if (K.zsv) {   // reading R15: no motion of the solid part
        R Tn, Fln;
        const R Cn = o.Ch + o.Cl;
        invert_enthalpy(K, o.Hh, o.Hl, clamp01(Cn), Tn, Fln);
        const R keep = R(1) - solid_gate(K, Cn) * (R(1) - Fln);
        o.mx *= keep;
        o.my *= keep;
    }
    if (!(isfinite(o.Hh) && isfinite(o.p) && isfinite(o.mx) && isfinite(o.my) && isfinite(o.Ch))) {
        atomicOr(flag, 1);      // solver-wide
        atomicOr(K.flag, 1);    // this domain
    }
    store_state(reinterpret_cast<R*>(K.st[stage == 2 ? 0 : stage + 1]), K.plane, c, o);
}

// One work item of Runge-Kutta stage `stage`: the strip segment
// [x0, x0 + 31) x [y0, y1) of the domain whose constants are in S.K (planar
// or axisymmetric, fixed per domain).  Returns false if a wait for an input
// tile gave up (the kernel then stops).
template <class R, bool AXI, bool GEN>
__device__ __forceinline__ bool sweep_item(Smem<R>& S, const StageLaunch& a, const int stage, TileIO& io, int x0,
                                           int y0, int y1) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const R* in = reinterpret_cast<const R*>(S.K.st[stage]);
    // a lane keeps its column through the item: in an axisymmetric domain
    // 1 / r of its cell centre (y-faces, cell volume) and of its x-face
    // (0 on the axis, where the face area is zero)
    const R ir_c = AXI ? wdiv(R(1), (R)(x0 + lane) + R(0.5)) : R(1);
    const R ir_f = (AXI && x0 + lane > 0) ? wdiv(R(1), (R)(x0 + lane)) : R(0);

    // prologue: rows y0-3 .. y0+2, mu_c of rows y0-2 .. y0+1, y-face row y0
    bool ok = true;
    if (tile_rows(S.K, x0, y0 - kHalo, 2 * kHalo)) {
        if (!S.pre) tile_fetch(S, a, stage, x0, y0 - kHalo);   // else copied during the previous item
        ok = tile_wait(S, io);
        load_rows_tile(S, x0, y0 - kHalo, 2 * kHalo);
    } else {
        load_rows(S, in, x0, y0 - kHalo, 2 * kHalo);
    }
    if (load_barrier_failed<R>(S, ok)) return tile_abort(S, io, a.flag);
    // the first chunk's rows arrive while the prologue computes
    if (tile_rows(S.K, x0, y0 + kHalo, kChunk)) tile_fetch(S, a, stage, x0, y0 + kHalo);
    if constexpr (sizeof(R) == 4)
        if (warp == NT / 32 - 1) prefetch_update_rows(S.K, stage, x0, y0, y1, lane);
    muc_rows<R, AXI>(S, x0, y0 - 2, 4);
    __syncthreads();
    if (warp == 0 && lane < kStripX) y_face<R, AXI, GEN>(S, y0, lane, AXI ? ir_c : R(0));
    // (the first chunk writes other ring rows: no barrier needed here)

    for (int j0 = y0; j0 < y1; j0 += kChunk) {
        // rows j0+3 .. j0+10: from the tile copied during the previous chunk,
        // or directly where boundary rules apply
        bool muc_done = false;
        if (tile_rows(S.K, x0, j0 + kHalo, kChunk)) {
            ok = tile_wait(S, io);
            if constexpr (sizeof(R) == 4) muc_done = muc_in_place(S.K, x0, j0 + 2, kChunk);
            load_rows_tile_muc<R, AXI>(S, x0, j0 + kHalo, muc_done);
        } else {
            load_rows(S, in, x0, j0 + kHalo, kChunk);
        }
        if (load_barrier_failed<R>(S, ok)) return tile_abort(S, io, a.flag);
        // the tile is free again: copy the next chunk's rows behind this one,
        // or after the last chunk the next work item's prologue rows
        if (j0 + kChunk < y1) {
            if (tile_rows(S.K, x0, j0 + kChunk + kHalo, kChunk)) tile_fetch(S, a, stage, x0, j0 + kChunk + kHalo);
        } else if constexpr (sizeof(R) == 4) {
            tile_prefetch_next(S, a);
        }
        // the next chunk's update rows into L2 (FP32C: the FP64 step is
        // bound by its FP64 arithmetic)
        if constexpr (sizeof(R) == 4)
            if (warp == NT / 32 - 1 && j0 + kChunk < y1) prefetch_update_rows(S.K, stage, x0, j0 + kChunk, y1, lane);
        if (!muc_done) {   // rows j0+2 .. j0+9
            muc_rows<R, AXI>(S, x0, j0 + 2, kChunk);
            __syncthreads();
        }
        // one face at a time per thread (x then y) keeps register use low
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
            if (k == 0) x_face<R, AXI, GEN>(S, x0, j0 + warp, warp, lane, ir_f);
            else if (lane < kStripX) y_face<R, AXI, GEN>(S, j0 + 1 + warp, lane, AXI ? ir_c : R(0));
        }
        __syncthreads();
        const int r = j0 + warp;
        if (r < y1 && lane < kStripX && x0 + lane < S.K.nx)
            cell_update<R, AXI>(S, stage, x0, r, warp, lane, ir_c, a.flag);
        __syncthreads();
    }
    return true;
}

}  // namespace

template <class R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) stage_kernel(StageLaunch a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<R>& S = *reinterpret_cast<Smem<R>*>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.cur_domain = -1;
        S.pre = 0;
        bar_init(&S.tile_bar);
    }
    __syncthreads();
    const Consts<R>* consts = static_cast<const Consts<R>*>(a.consts);
    TileIO io{0u};

    // Every item is claimed from the launch's counter, one item ahead (the
    // tile prefetch of the next item's prologue needs to know it).  In a
    // whole-step launch the items of stage 1 follow all of stage 0 and those
    // of stage 2 all of stage 1 (then stage 0 of the next step, when the
    // launch runs several), and an item waits for the items of the previous
    // stage it reads.  Only running CTAs hold items, and every item
    // waits only for items claimed before it, so the earliest unfinished
    // item can always proceed.
    int* const counter = a.work + (a.stages == 1 ? a.stage : 0);
    if (tid == 0) S.next = atomicAdd(counter, 1);
    __syncthreads();
    while (S.next < a.nitems * a.stages) {
        const int2 si = stage_item(a, S.next);
        const int4 item = a.items[si.y];
        const int prev = S.cur_domain;   // read by every thread before the barrier below
        __syncthreads();                 // the previous item is done with shared memory
        if (tid == 0) {
            S.next = atomicAdd(counter, 1);
            S.stage = si.x;
            S.item = si.y;
        }
        if (a.stages > 1 && si.x > 0) {
            if (tid < 32) {
                const bool ready = deps_ready(a, si.x, si.y, tid, true);
                if (tid == 0) S.ready = ready;
            }
            __syncthreads();
            if (!S.ready) return dep_abort(S, io, a.flag);
            // the rows this item copies by TMA were written through the generic proxy
            if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        if (item.x != prev) {
            const unsigned* src = reinterpret_cast<const unsigned*>(consts + item.x);
            unsigned* dst = reinterpret_cast<unsigned*>(&S.K);
            for (int k = tid; k < (int)(sizeof(Consts<R>) / 4); k += NT) dst[k] = src[k];
            if (tid == 0) S.cur_domain = item.x;
        }
        __syncthreads();                 // S.K
        const int x0 = item.y * kStripX;
        const int y0 = item.z, y1 = item.w;
        bool ok;
        if (S.K.gen) {   // some streaming step differs from 1/2 (reading R26)
            if (S.K.axi) ok = sweep_item<R, true, true>(S, a, si.x % 3, io, x0, y0, y1);
            else ok = sweep_item<R, false, true>(S, a, si.x % 3, io, x0, y0, y1);
        } else {
            if (S.K.axi) ok = sweep_item<R, true, false>(S, a, si.x % 3, io, x0, y0, y1);
            else ok = sweep_item<R, false, false>(S, a, si.x % 3, io, x0, y0, y1);
        }
        if (!ok) return;   // uniform: every thread saw the same __syncthreads_or
        if (a.stages > 1) {
            // publish: every thread's stores of this item, then its flag
            __syncthreads();
            if (tid == 0 && !a.dep_probe) {
                __threadfence();
                atomicExch(a.done + (size_t)S.stage * a.nitems + S.item, 1);
            }
        }
    }
}

// The dynamic shared-memory limit of stage_kernel<R> is a per-device
// attribute: it is set once for every device the kernel is launched on, under
// a lock, so that solvers on several devices and several host threads can
// launch it.
constexpr int kMaxAttrDevices = 64;

template <class R>
static cudaError_t configure_t() {
    static std::mutex m;
    static bool done[kMaxAttrDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxAttrDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(m);
    if (!done[dev]) {
        e = cudaFuncSetAttribute(stage_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<R>));
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

template <class R>
static cudaError_t launch_t(const StageLaunch& a, int grid, cudaStream_t s) {
    cudaError_t e = configure_t<R>();
    if (e != cudaSuccess) return e;
    stage_kernel<R><<<grid, NT, sizeof(Smem<R>), s>>>(a);
    return cudaGetLastError();
}

template <class R>
static int blocks_per_sm_t() {
    const size_t smem = sizeof(Smem<R>);
    if (configure_t<R>() != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<R>, NT, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_stage(int precision, const StageLaunch& a, int grid, cudaStream_t s) {
    return precision == 0 ? launch_t<double>(a, grid, s) : launch_t<float>(a, grid, s);
}

int stage_blocks_per_sm(int precision) { return precision == 0 ? blocks_per_sm_t<double>() : blocks_per_sm_t<float>(); }

size_t stage_smem_bytes(int precision) { return precision == 0 ? sizeof(Smem<double>) : sizeof(Smem<float>); }

}  // namespace eulbfs
