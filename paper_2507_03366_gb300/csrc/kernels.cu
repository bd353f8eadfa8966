// kernels.cu -- sm_103a kernels of the EULBFS explicit step (arXiv 2507.03366).
//
// The stage kernel is the hot path.  One CTA owns a 32 x TY tile of one domain
// of the batch and, per Runge-Kutta stage (Eq. 58):
//   A. loads the tile plus a 3-cell halo of the stage state, maps halo cells
//      through the boundary conditions, and derives the macroscopic fields
//      T, F_l, C_p, rho, lambda, mu (Eq. 5-7), u = m / (rho cs^2), p, C;
//   B. computes mu_c = 2 beta C(C-1)(2C-1) - kappa lap C (Sec. 2.3.1) in the tile;
//   C. computes the five flux moments of every face of the tile exactly once
//      (Eq. 54, 56, 9/29/33/42, 13/16, 35/37, 44/46, 53), shared through shared
//      memory by the two cells of the face;
//   D. forms R(W) = -div F + F_E (Eq. 51-52) per cell, takes the SSP-RK3 stage
//      and stores the new state (compensated for H and C in FP32C).
// Tiles come from a work list that spans every domain of the batch, so one
// launch advances all domains by one stage; the grid is persistent (a fixed
// number of CTAs per SM striding over the list).
//
// The face computation is written in the face frame (n, t): an x-face has
// n = x, t = y and a y-face n = y, t = x; D2Q9 is symmetric under the swap.
// With dt_s = 0.5 the surrounding points x_f - e_a dt_s of a face are the two
// cell centres (e_n = +-1, e_t = 0), the two cells' extrapolations half a cell
// along t (e_n = +-1, e_t = +-1), and three points on the face itself (e_n = 0),
// which take the mean of the two one-sided reconstructions.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "eulbfs.h"
#include "eulbfs_internal.h"

namespace eulbfs {

enum { BC_PERIODIC = 0, BC_DIRICHLET_T, BC_ADIABATIC, BC_NOSLIP, BC_SYMMETRY, BC_OUTLET, BC_NOFLUX, BC_WETTING };

template <class R> struct Prec;
template <> struct Prec<double> { static constexpr int NP = 5; };
template <> struct Prec<float> { static constexpr int NP = 7; };

// Working-precision copy of a domain's constants, held in shared memory.
template <class R>
struct Consts {
    R rho[3], mu[3], lam[3], cp[3];
    R L, Ts, Tl, beta, kappa, Qg, tau_g, Cref, kv, gx, gy, dt;
    R Tw[4], wet[4];
    int nx, ny, per_x, per_y, tiles_x, tile0, zsv;
    int bc_t[4], bc_f[4], bc_c[4];
    long long plane;
    const void* in;
    const void* base;
    void* out;
    void* Fsp;
    void* dFs;
};

template <class R>
__device__ void load_consts(const DomainDesc& d, int stage, Consts<R>& K) {
    for (int k = 0; k < 3; ++k) {
        K.rho[k] = (R)d.rho[k]; K.mu[k] = (R)d.mu[k]; K.lam[k] = (R)d.lam[k]; K.cp[k] = (R)d.cp[k];
    }
    K.L = (R)d.L; K.Ts = (R)d.Ts; K.Tl = (R)d.Tl; K.beta = (R)d.beta; K.kappa = (R)d.kappa;
    K.Qg = (R)d.Qg; K.tau_g = (R)d.tau_g; K.Cref = (R)d.Cref; K.kv = (R)d.kv;
    K.gx = (R)d.gx; K.gy = (R)d.gy; K.dt = (R)d.dt;
    for (int k = 0; k < 4; ++k) {
        K.Tw[k] = (R)d.Tw[k]; K.wet[k] = (R)d.wet[k];
        K.bc_t[k] = d.bc_t[k]; K.bc_f[k] = d.bc_f[k]; K.bc_c[k] = d.bc_c[k];
    }
    K.nx = d.nx; K.ny = d.ny; K.per_x = d.per_x; K.per_y = d.per_y;
    K.tiles_x = d.tiles_x; K.tile0 = d.tile0; K.zsv = d.zero_solid_velocity;
    K.plane = d.plane;
    K.in = d.st[stage];
    K.base = d.st[0];
    K.out = d.st[stage == 2 ? 0 : stage + 1];
    K.Fsp = d.Fsp;
    K.dFs = d.dFs;
}

// ---------------------------------------------------------------------------
// State access.  FP64: H p mx my C.  FP32C: Hhi Hlo p mx my Chi Clo.
// ---------------------------------------------------------------------------
template <class R>
struct SV { R Hh, Hl, p, mx, my, Ch, Cl; };

__device__ __forceinline__ SV<double> load_state(const double* b, long long P, long long c) {
    SV<double> s;
    s.Hh = b[c]; s.Hl = 0.0; s.p = b[P + c]; s.mx = b[2 * P + c]; s.my = b[3 * P + c];
    s.Ch = b[4 * P + c]; s.Cl = 0.0;
    return s;
}
__device__ __forceinline__ SV<float> load_state(const float* b, long long P, long long c) {
    SV<float> s;
    s.Hh = b[c]; s.Hl = b[P + c]; s.p = b[2 * P + c]; s.mx = b[3 * P + c]; s.my = b[4 * P + c];
    s.Ch = b[5 * P + c]; s.Cl = b[6 * P + c];
    return s;
}
__device__ __forceinline__ void store_state(double* b, long long P, long long c, const SV<double>& s) {
    b[c] = s.Hh; b[P + c] = s.p; b[2 * P + c] = s.mx; b[3 * P + c] = s.my; b[4 * P + c] = s.Ch;
}
__device__ __forceinline__ void store_state(float* b, long long P, long long c, const SV<float>& s) {
    b[c] = s.Hh; b[P + c] = s.Hl; b[2 * P + c] = s.p; b[3 * P + c] = s.mx; b[4 * P + c] = s.my;
    b[5 * P + c] = s.Ch; b[6 * P + c] = s.Cl;
}

// Knuth's TwoSum: s + e == a + b exactly.
template <class R>
__device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
    s = a + b;
    R bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <class R>
__device__ __forceinline__ R clamp01(R c) { return c < R(0) ? R(0) : (c > R(1) ? R(1) : c); }

// Eq. 5-6 with the readings of the oracle: uniform latent heat, Eq. 7 mixture
// heat capacity gated by clamp(C).  H = Hh + Hl (Hl = 0 in FP64); the
// differences H - H_s and H - H_l are formed from the pair without rounding H.
template <class R>
__device__ __forceinline__ void invert_enthalpy(const Consts<R>& K, R Hh, R Hl, R Ct, R& T, R& Fl) {
    const R cps = Ct * K.cp[0] + (R(1) - Ct) * K.cp[2];
    const R cpl = Ct * K.cp[1] + (R(1) - Ct) * K.cp[2];
    const R Hs = cps * K.Ts;
    const R HL = cpl * K.Tl + K.L;
    const R ds = (Hh - Hs) + Hl;
    const R dl = (Hh - HL) + Hl;
    if (ds < R(0)) {
        Fl = R(0);
        T = (Hh + Hl) / cps;
    } else if (dl > R(0)) {
        Fl = R(1);
        T = K.Tl + dl / cpl;
    } else if (HL > Hs) {
        Fl = ds / (HL - Hs);
        T = K.Ts + Fl * (K.Tl - K.Ts);
    } else {
        Fl = R(1);
        T = K.Tl;
    }
}

// Eq. 7 (reading R1): gamma = C~ [F_s g_s + F_l g_l] + (1 - C~) g_g.
template <class R>
__device__ __forceinline__ R mix(R Ct, R Fl, const R g[3]) {
    return Ct * ((R(1) - Fl) * g[0] + Fl * g[1]) + (R(1) - Ct) * g[2];
}

// Map a cell coordinate outside [0, n) through its boundary: periodic wrap or
// mirror about the wall (ghost layer k >= 1 mirrors interior cell k - 1).
__device__ __forceinline__ void map_axis(int g, int n, int per, int lo_side, int& s, int& k, int& side) {
    k = 0;
    side = lo_side;
    if (g >= 0 && g < n) { s = g; return; }
    if (per) { s = ((g % n) + n) % n; return; }
    if (g < 0) { k = -g; s = k - 1; side = lo_side; }
    else { k = g - n + 1; s = n - k; side = lo_side + 1; }
    s = s < 0 ? 0 : (s >= n ? n - 1 : s);   // layers deeper than the domain are never used
}

// Ghost value rules (boundary conditions on macroscopic variables).
template <class R>
struct Prim { R T, Fl, cp, rho, lam, mu, p, u, v, C; };

template <class R>
__device__ __forceinline__ void apply_ghost(const Consts<R>& K, int side, int k, bool x_normal, Prim<R>& q) {
    if (K.bc_t[side] == BC_DIRICHLET_T) q.T = R(2) * K.Tw[side] - q.T;
    const int f = K.bc_f[side];
    if (f == BC_OUTLET) q.p = -q.p;
    R& un = x_normal ? q.u : q.v;
    R& ut = x_normal ? q.v : q.u;
    if (f == BC_NOSLIP) { un = -un; ut = -ut; }
    else if (f == BC_SYMMETRY) { un = -un; }
    if (K.bc_c[side] == BC_WETTING) q.C = q.C + R(2 * k - 1) * K.wet[side] * q.C * (R(1) - q.C);
}

template <class R>
__device__ __forceinline__ Prim<R> derive(const Consts<R>& K, const SV<R>& w) {
    Prim<R> q;
    const R C = w.Ch + w.Cl;
    const R Ct = clamp01(C);
    invert_enthalpy(K, w.Hh, w.Hl, Ct, q.T, q.Fl);
    q.cp = mix(Ct, q.Fl, K.cp);
    q.rho = mix(Ct, q.Fl, K.rho);
    q.lam = mix(Ct, q.Fl, K.lam);
    q.mu = mix(Ct, q.Fl, K.mu);
    const R r3 = R(3) / q.rho;          // 1 / (rho cs^2)
    q.u = w.mx * r3;
    q.v = w.my * r3;
    q.p = w.p;
    q.C = C;
    return q;
}

// Shared-memory field indices of the tile.
enum { S_T, S_FL, S_CP, S_RHO, S_LAM, S_MU, S_P, S_U, S_V, S_C, S_MUC, S_NF };

template <class R, int TY>
struct Tile {
    static constexpr int RW = kTileX + 2 * kHalo;
    static constexpr int RH = TY + 2 * kHalo;
    static constexpr int RN = RW * RH;
    static constexpr int NXF = (kTileX + 1) * TY;     // x-faces
    static constexpr int NYF = kTileX * (TY + 1);     // y-faces
    static constexpr int NT = TY <= 8 ? 32 * TY : 256;
    static constexpr size_t bytes = sizeof(R) * (size_t)(S_NF * RN + 6 * (NXF + NYF));
};

template <class R>
struct FaceFlux { R Fh, Fp, Fmn, Fmt, Fc, un; };

// The 9 surrounding-point values of one field (Eq. 54; points on the face
// take the mean of the L and R reconstructions, reading R7).
template <class R>
__device__ __forceinline__ void points(const R* f, int L, int sn, int st, R o[9]) {
    const R l = f[L], r = f[L + sn];
    const R hnl = R(0.25) * (r - f[L - sn]);            // half-cell step of L along n
    const R hnr = R(0.25) * (f[L + 2 * sn] - l);
    const R htl = R(0.25) * (f[L + st] - f[L - st]);    // half-cell step along t
    const R htr = R(0.25) * (f[L + sn + st] - f[L + sn - st]);
    const R lf = l + hnl, rf = r - hnr;                 // one-sided values at the face
    o[0] = R(0.5) * (lf + rf);
    o[1] = l;
    o[2] = R(0.5) * ((lf - htl) + (rf - htr));
    o[3] = r;
    o[4] = R(0.5) * ((lf + htl) + (rf + htr));
    o[5] = l - htl;
    o[6] = r - htr;
    o[7] = r + htr;
    o[8] = l + htl;
}

template <class R>
__device__ __forceinline__ R point0(const R* f, int L, int sn) {
    const R l = f[L], r = f[L + sn];
    const R lf = l + R(0.25) * (r - f[L - sn]);
    const R rf = r - R(0.25) * (f[L + 2 * sn] - l);
    return R(0.5) * (lf + rf);
}

// Sec. 2.5 steps (2)-(4) and Eq. 53 for one face.
template <class R>
__device__ __forceinline__ FaceFlux<R> face_flux(const Consts<R>& K, const R* S, int RN, int L, int sn,
                                                 int st, int fUn, int fUt) {
    R un[9], ut[9], pp[9], rr[9], TT[9], cp[9], CC[9], mc[9];
    points(S + fUn * RN, L, sn, st, un);
    points(S + fUt * RN, L, sn, st, ut);
    points(S + S_P * RN, L, sn, st, pp);
    points(S + S_RHO * RN, L, sn, st, rr);
    points(S + S_T * RN, L, sn, st, TT);
    points(S + S_CP * RN, L, sn, st, cp);
    points(S + S_C * RN, L, sn, st, CC);
    points(S + S_MUC * RN, L, sn, st, mc);
    const R lamf = point0(S + S_LAM * RN, L, sn);
    const R muf = point0(S + S_MU * RN, L, sn);
    const R rho_f = rr[0];
    const R w0 = R(4.0 / 9.0), w1 = R(1.0 / 9.0), w5 = R(1.0 / 36.0);

    R pf = R(0), mn = R(0), mt = R(0), Cf = R(0);
    R Sh = R(0), Sg = R(0), Snn_p = R(0), Snn_q = R(0), Snt_p = R(0), Snt_q = R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int en = (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
        const int et = (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
        const R w = a == 0 ? w0 : (a < 5 ? w1 : w5);
        const R eu = R(en) * un[a] + R(et) * ut[a];
        const R uu = un[a] * un[a] + ut[a] * ut[a];
        // cs^2 (e.u/cs^2 + (e.u)^2/(2 cs^4) - u^2/(2 cs^2)) with cs^2 = 1/3
        const R q = eu + R(1.5) * eu * eu - R(0.5) * uu;
        const R f = w * (pp[a] + rr[a] * q);                 // Eq. 29
        pf += f;
        if (en != 0) mn += R(en) * f;
        if (et != 0) mt += R(et) * f;
        if (a == 0) {
            Cf += CC[0] - R(3) * mc[0] * K.Qg * (R(1) - w0);  // Eq. 42, alpha = 0
        } else {
            const R g = R(3) * w * (mc[a] * K.Qg + CC[a] * eu);   // Eq. 42
            Cf += g;
            if (en != 0) {
                Sg += R(en) * g;
                const R h = w * (K.Cref * TT[a] + R(3) * (cp[a] * TT[a]) * q);   // Eq. 9
                Sh += R(en) * h;
                // Eq. 33 (reading R8): w (p + rho_f q), kept as its p and q parts
                Snn_p += w * pp[a];
                Snn_q += w * q;
                if (et != 0) {
                    Snt_p += R(en * et) * w * pp[a];
                    Snt_q += R(en * et) * w * q;
                }
            }
        }
    }
    // Eq. 56: rho_f cs^2 u_f = sum e f^eq; tau from the face properties (R9)
    const R irf = R(1) / rho_f;
    const R unf = R(3) * mn * irf, utf = R(3) * mt * irf;
    const R th = R(6) * lamf * irf / K.Cref;    // tau_h - 0.5 = lambda / (rho C_ref cs^2 dt_s)
    const R tf = R(6) * muf * irf;              // tau_f - 0.5 = mu / (rho cs^2 dt_s)
    const R tg = K.tau_g - R(0.5);
    const R cs2 = R(1.0 / 3.0);
    FaceFlux<R> F;
    // h* = (1.5 - tau) h^eq(x_f) + (tau - 0.5) h^eq(x_f - e dt_s) (Eq. 13, 16);
    // the first moment of h^eq(x_f) is C_p T u at the face (Eq. 11).
    F.Fh = (R(1) - th) * (cp[0] * TT[0]) * unf + th * Sh;
    F.Fp = mn;                                   // sum e_n f^eq(x_f) = rho_f cs^2 u_n,f
    // f* = (1.5 - tau_f) f^eq(x_f) + (tau_f - 0.5) f^eq-m (Eq. 35, 37 with R3)
    F.Fmn = (R(1) - tf) * cs2 * (pf + rho_f * unf * unf) + tf * (Snn_p + rho_f * Snn_q);
    F.Fmt = (R(1) - tf) * cs2 * rho_f * unf * utf + tf * (Snt_p + rho_f * Snt_q);
    F.Fc = (R(1) - tg) * Cf * unf + tg * Sg;    // Eq. 44, 46
    F.un = unf;
    return F;
}

template <class R, int TY>
__global__ void __launch_bounds__(Tile<R, TY>::NT) stage_kernel(StageLaunch a) {
    using TL = Tile<R, TY>;
    constexpr int RW = TL::RW, RH = TL::RH, RN = TL::RN, NT = TL::NT;
    constexpr int XW = kTileX + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* S = reinterpret_cast<R*>(smem_raw);
    R* FX = S + S_NF * RN;           // 6 x NXF
    R* FY = FX + 6 * TL::NXF;        // 6 x NYF
    __shared__ Consts<R> K;
    __shared__ int cur_domain;
    const int tid = threadIdx.x;
    if (tid == 0) cur_domain = -1;
    __syncthreads();

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int d = a.tile_domain[tile];
        const int prev = cur_domain;   // read by every thread before the barrier below
        __syncthreads();               // previous tile fully consumed before smem is rewritten
        if (d != prev) {
            if (tid == 0) { load_consts(a.descs[d], a.stage, K); cur_domain = d; }
            __syncthreads();
        }
        const int local = tile - K.tile0;
        const int x0 = (local % K.tiles_x) * kTileX;
        const int y0 = (local / K.tiles_x) * TY;
        const R* in = reinterpret_cast<const R*>(K.in);
        const long long P = K.plane;

        // ---- A: halo load, boundary mapping, derived fields -------------------
        for (int idx = tid; idx < RN; idx += NT) {
            const int rx = idx % RW, ry = idx / RW;
            int sx, kx, sdx, sy, ky, sdy;
            map_axis(x0 + rx - kHalo, K.nx, K.per_x, XLO, sx, kx, sdx);
            map_axis(y0 + ry - kHalo, K.ny, K.per_y, YLO, sy, ky, sdy);
            const SV<R> w = load_state(in, P, (long long)sy * K.nx + sx);
            Prim<R> q = derive(K, w);
            if (kx) apply_ghost(K, sdx, kx, true, q);    // x sides first, then y (corners)
            if (ky) apply_ghost(K, sdy, ky, false, q);
            S[S_T * RN + idx] = q.T;
            S[S_FL * RN + idx] = q.Fl;
            S[S_CP * RN + idx] = q.cp;
            S[S_RHO * RN + idx] = q.rho;
            S[S_LAM * RN + idx] = q.lam;
            S[S_MU * RN + idx] = q.mu;
            S[S_P * RN + idx] = q.p;
            S[S_U * RN + idx] = q.u;
            S[S_V * RN + idx] = q.v;
            S[S_C * RN + idx] = q.C;
        }
        __syncthreads();

        // ---- B: chemical potential (R5), then mirror it into wall ghosts ------
        for (int idx = tid; idx < RN; idx += NT) {
            const int rx = idx % RW, ry = idx / RW;
            if (rx < 1 || rx >= RW - 1 || ry < 1 || ry >= RH - 1) continue;
            const R* Cs = S + S_C * RN;
            const R c = Cs[idx];
            const R lap = Cs[idx + 1] + Cs[idx - 1] + Cs[idx + RW] + Cs[idx - RW] - R(4) * c;
            S[S_MUC * RN + idx] = R(2) * K.beta * c * (c - R(1)) * (R(2) * c - R(1)) - K.kappa * lap;
        }
        __syncthreads();
        for (int idx = tid; idx < RN; idx += NT) {
            const int rx = idx % RW, ry = idx / RW;
            if (rx < 1 || rx >= RW - 1 || ry < 1 || ry >= RH - 1) continue;
            const int gx = x0 + rx - kHalo, gy = y0 + ry - kHalo;
            int mrx = rx, mry = ry;
            if (!K.per_x) {
                if (gx < 0) mrx = rx + (2 * (-gx) - 1);
                else if (gx >= K.nx) mrx = rx - (2 * (gx - K.nx + 1) - 1);
            }
            if (!K.per_y) {
                if (gy < 0) mry = ry + (2 * (-gy) - 1);
                else if (gy >= K.ny) mry = ry - (2 * (gy - K.ny + 1) - 1);
            }
            if ((mrx != rx || mry != ry) && mrx >= 1 && mrx < RW - 1 && mry >= 1 && mry < RH - 1)
                S[S_MUC * RN + idx] = S[S_MUC * RN + mry * RW + mrx];
        }
        __syncthreads();

        // ---- C: face fluxes, each face once ----------------------------------
        for (int f = tid; f < TL::NXF + TL::NYF; f += NT) {
            if (f < TL::NXF) {
                const int fx = f % XW, fy = f / XW;
                const int L = (fy + kHalo) * RW + (fx - 1 + kHalo);
                const FaceFlux<R> F = face_flux(K, S, RN, L, 1, RW, S_U, S_V);
                FX[0 * TL::NXF + f] = F.Fh;
                FX[1 * TL::NXF + f] = F.Fp;
                FX[2 * TL::NXF + f] = F.Fmn;   // x-momentum
                FX[3 * TL::NXF + f] = F.Fmt;   // y-momentum
                FX[4 * TL::NXF + f] = F.Fc;
                FX[5 * TL::NXF + f] = F.un;
            } else {
                const int g = f - TL::NXF;
                const int fx = g % kTileX, fy = g / kTileX;
                const int L = (fy - 1 + kHalo) * RW + (fx + kHalo);
                const FaceFlux<R> F = face_flux(K, S, RN, L, RW, 1, S_V, S_U);
                FY[0 * TL::NYF + g] = F.Fh;
                FY[1 * TL::NYF + g] = F.Fp;
                FY[2 * TL::NYF + g] = F.Fmt;   // x-momentum
                FY[3 * TL::NYF + g] = F.Fmn;   // y-momentum
                FY[4 * TL::NYF + g] = F.Fc;
                FY[5 * TL::NYF + g] = F.un;
            }
        }
        __syncthreads();

        // ---- D: residual, sources, Runge-Kutta stage, store -------------------
        for (int cidx = tid; cidx < kTileX * TY; cidx += NT) {
            const int tx = cidx % kTileX, ty = cidx / kTileX;
            const int gx = x0 + tx, gy = y0 + ty;
            if (gx >= K.nx || gy >= K.ny) continue;
            const long long c = (long long)gy * K.nx + gx;
            const int q = (ty + kHalo) * RW + tx + kHalo;
            const int fw = ty * XW + tx, fe = fw + 1;
            const int fs = ty * kTileX + tx, fn = fs + kTileX;
            R Rk[5];
#pragma unroll
            for (int k = 0; k < 5; ++k)
                Rk[k] = -((FX[k * TL::NXF + fe] - FX[k * TL::NXF + fw]) + (FY[k * TL::NYF + fn] - FY[k * TL::NYF + fs]));
            const R divu = (FX[5 * TL::NXF + fe] - FX[5 * TL::NXF + fw]) + (FY[5 * TL::NYF + fn] - FY[5 * TL::NYF + fs]);

            const R T = S[S_T * RN + q], Fl = S[S_FL * RN + q], Cp = S[S_CP * RN + q];
            const R rho = S[S_RHO * RN + q], u = S[S_U * RN + q], v = S[S_V * RN + q], C = S[S_C * RN + q];
            const R drx = R(0.5) * (S[S_RHO * RN + q + 1] - S[S_RHO * RN + q - 1]);
            const R dry = R(0.5) * (S[S_RHO * RN + q + RW] - S[S_RHO * RN + q - RW]);
            const R dmx = R(0.5) * (S[S_MUC * RN + q + 1] - S[S_MUC * RN + q - 1]);
            const R dmy = R(0.5) * (S[S_MUC * RN + q + RW] - S[S_MUC * RN + q - RW]);
            R dfs;
            if (a.stage == 0) {   // reading R14: lagged dF_s/dt, fixed over the step
                R* Fsp = reinterpret_cast<R*>(K.Fsp);
                const R Fs = R(1) - Fl;
                dfs = (Fs - Fsp[c]) / K.dt;
                reinterpret_cast<R*>(K.dFs)[c] = dfs;
                Fsp[c] = Fs;
            } else {
                dfs = reinterpret_cast<const R*>(K.dFs)[c];
            }
            const R cs2 = R(1.0 / 3.0);
            const R D = clamp01(C) * dfs;
            Rk[0] += Cp * T * divu;                                       // Eq. 51 row 1
            Rk[1] += u * (drx * cs2) + v * (dry * cs2) + rho * cs2 * K.kv * D;   // row 2
            Rk[2] += cs2 * (-Fl * C * dmx + rho * K.gx - rho * u * D);     // row 3 (R13)
            Rk[3] += cs2 * (-Fl * C * dmy + rho * K.gy - rho * v * D);     // row 4
            Rk[4] += C * K.kv * D;                                         // row 5 (R12)

            const SV<R> ws = load_state(in, P, c);
            const SV<R> wn = load_state(reinterpret_cast<const R*>(K.base), P, c);
            SV<R> o;
            if constexpr (sizeof(R) == 8) {
                // Eq. 58 as written
                const R A = a.stage == 0 ? R(1) : (a.stage == 1 ? R(0.75) : R(1.0 / 3.0));
                const R B = a.stage == 0 ? R(0) : (a.stage == 1 ? R(0.25) : R(2.0 / 3.0));
                const R Cd = (a.stage == 0 ? R(1) : (a.stage == 1 ? R(0.25) : R(2.0 / 3.0))) * K.dt;
                o.Hh = A * wn.Hh + B * ws.Hh + Cd * Rk[0];
                o.p = A * wn.p + B * ws.p + Cd * Rk[1];
                o.mx = A * wn.mx + B * ws.mx + Cd * Rk[2];
                o.my = A * wn.my + B * ws.my + Cd * Rk[3];
                o.Ch = A * wn.Ch + B * ws.Ch + Cd * Rk[4];
                o.Hl = R(0); o.Cl = R(0);
            } else {
                // Eq. 58 as W^n + increment; H and C kept as compensated pairs
                const R B = a.stage == 0 ? R(0) : (a.stage == 1 ? R(0.25) : R(2.0 / 3.0));
                const R Cd = (a.stage == 0 ? R(1) : (a.stage == 1 ? R(0.25) : R(2.0 / 3.0))) * K.dt;
                const R dH = B * ((ws.Hh - wn.Hh) + (ws.Hl - wn.Hl)) + Cd * Rk[0];
                const R dC = B * ((ws.Ch - wn.Ch) + (ws.Cl - wn.Cl)) + Cd * Rk[4];
                // TwoSum for both the sum and the renormalisation keeps every
                // pair canonical (hi = fl(hi + lo)) even where H or C cross zero,
                // so a pair survives a round trip through one double exactly.
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
                const R keep = R(1) - clamp01(Cn) * (R(1) - Fln);
                o.mx *= keep;
                o.my *= keep;
            }
            if (!(isfinite(o.Hh) && isfinite(o.p) && isfinite(o.mx) && isfinite(o.my) && isfinite(o.Ch)))
                atomicOr(a.flag, 1);
            store_state(reinterpret_cast<R*>(K.out), P, c, o);
        }
    }
}

template <class R, int TY>
static cudaError_t launch_stage_t(const StageLaunch& a, int grid, cudaStream_t s) {
    const size_t smem = Tile<R, TY>::bytes;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(stage_kernel<R, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    stage_kernel<R, TY><<<grid, Tile<R, TY>::NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <class R, int TY>
static int blocks_per_sm_t() {
    const size_t smem = Tile<R, TY>::bytes;
    cudaFuncSetAttribute(stage_kernel<R, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<R, TY>, Tile<R, TY>::NT, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_stage(int precision, int tile_y, const StageLaunch& a, int grid, cudaStream_t s) {
    if (precision == 0) {
        if (tile_y == 4) return launch_stage_t<double, 4>(a, grid, s);
        if (tile_y == 16) return launch_stage_t<double, 16>(a, grid, s);
        return launch_stage_t<double, 8>(a, grid, s);
    }
    if (tile_y == 4) return launch_stage_t<float, 4>(a, grid, s);
    if (tile_y == 16) return launch_stage_t<float, 16>(a, grid, s);
    return launch_stage_t<float, 8>(a, grid, s);
}

int stage_blocks_per_sm(int precision, int tile_y) {
    if (precision == 0) {
        if (tile_y == 4) return blocks_per_sm_t<double, 4>();
        if (tile_y == 16) return blocks_per_sm_t<double, 16>();
        return blocks_per_sm_t<double, 8>();
    }
    if (tile_y == 4) return blocks_per_sm_t<float, 4>();
    if (tile_y == 16) return blocks_per_sm_t<float, 16>();
    return blocks_per_sm_t<float, 8>();
}

size_t stage_smem_bytes(int precision, int tile_y) {
    if (precision == 0) return tile_y == 4 ? Tile<double, 4>::bytes : (tile_y == 16 ? Tile<double, 16>::bytes : Tile<double, 8>::bytes);
    return tile_y == 4 ? Tile<float, 4>::bytes : (tile_y == 16 ? Tile<float, 16>::bytes : Tile<float, 8>::bytes);
}

// ---------------------------------------------------------------------------
// Initial state, field output, checkpoints (double precision arithmetic).
// ---------------------------------------------------------------------------
// Inverse of Eq. 5-6 for the initial state (same rule as the oracle).
__device__ double enthalpy_of(const Consts<double>& K, double T, double Fl, double C) {
    const double Ct = clamp01(C);
    const double cps = Ct * K.cp[0] + (1.0 - Ct) * K.cp[2];
    const double cpl = Ct * K.cp[1] + (1.0 - Ct) * K.cp[2];
    const double Hs = cps * K.Ts;
    const double HL = cpl * K.Tl + K.L;
    if (T < K.Ts) return cps * T;
    if (T > K.Tl) return HL + cpl * (T - K.Tl);
    const double f = (K.Tl > K.Ts) ? (T - K.Ts) / (K.Tl - K.Ts) : Fl;
    if (f >= 1.0) return HL;
    if (f <= 0.0) return Hs;
    return Hs + f * (HL - Hs);
}

template <class R>
__device__ void put_pair(R& hi, R& lo, double x) {
    hi = (R)x;
    lo = (R)(x - (double)hi);
}

template <class R>
__global__ void init_kernel(const DomainDesc* dd, const double* T, const double* Fl, const double* C,
                            const double* u, const double* v, const double* p, long long n, int* bad) {
    __shared__ Consts<double> Kd;
    __shared__ Consts<R> K;
    if (threadIdx.x == 0) { load_consts(*dd, 0, Kd); load_consts(*dd, 0, K); }
    __syncthreads();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double Cc = C[c];
        if (!(isfinite(T[c]) && isfinite(Cc) && (!Fl || isfinite(Fl[c])) && (!u || isfinite(u[c])) &&
              (!v || isfinite(v[c])) && (!p || isfinite(p[c]))))
            atomicOr(bad, 1);
        const double H = enthalpy_of(Kd, T[c], Fl ? Fl[c] : 1.0, Cc);
        double Td, Fld;
        invert_enthalpy(Kd, H, 0.0, clamp01(Cc), Td, Fld);
        const double rho = mix(clamp01(Cc), Fld, Kd.rho);
        SV<R> s;
        if (sizeof(R) == 8) { s.Hh = (R)H; s.Hl = 0; s.Ch = (R)Cc; s.Cl = 0; }
        else { put_pair(s.Hh, s.Hl, H); put_pair(s.Ch, s.Cl, Cc); }
        s.p = (R)(p ? p[c] : 0.0);
        s.mx = (R)(u ? rho * (1.0 / 3.0) * u[c] : 0.0);
        s.my = (R)(v ? rho * (1.0 / 3.0) * v[c] : 0.0);
        store_state(reinterpret_cast<R*>(const_cast<void*>(K.base)), K.plane, c, s);
        // previous-step solid fraction from the stored state, in working precision (R14)
        R Tw, Flw;
        invert_enthalpy(K, s.Hh, s.Hl, clamp01(s.Ch + s.Cl), Tw, Flw);
        reinterpret_cast<R*>(K.Fsp)[c] = R(1) - Flw;
    }
}

template <class R>
__device__ __forceinline__ double pair_value(R hi, R lo) { return (double)hi + (double)lo; }

template <class R>
__global__ void fields_kernel(const DomainDesc* dd, long long n, double* H, double* T, double* Fl, double* C,
                              double* p, double* u, double* v) {
    __shared__ Consts<double> Kd;
    __shared__ const void* base;
    if (threadIdx.x == 0) { load_consts(*dd, 0, Kd); base = dd->st[0]; }
    __syncthreads();
    const R* b = reinterpret_cast<const R*>(base);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, Kd.plane, c);
        const double Hd = pair_value(w.Hh, w.Hl), Cd = pair_value(w.Ch, w.Cl);
        double Td, Fld;
        invert_enthalpy(Kd, Hd, 0.0, clamp01(Cd), Td, Fld);
        const double rho = mix(clamp01(Cd), Fld, Kd.rho);
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
    const long long P = dd->plane;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, P, c);
        if (H) H[c] = pair_value(w.Hh, w.Hl);
        if (p) p[c] = (double)w.p;
        if (mx) mx[c] = (double)w.mx;
        if (my) my[c] = (double)w.my;
        if (C) C[c] = pair_value(w.Ch, w.Cl);
        if (Fsp) Fsp[c] = (double)fs[c];
    }
}

template <class R>
__global__ void set_state_kernel(const DomainDesc* dd, long long n, const double* H, const double* p,
                                 const double* mx, const double* my, const double* C, const double* Fsp) {
    R* b = reinterpret_cast<R*>(dd->st[0]);
    R* fs = reinterpret_cast<R*>(dd->Fsp);
    const long long P = dd->plane;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        SV<R> w = load_state(b, P, c);
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
        store_state(b, P, c, w);
        if (Fsp) fs[c] = (R)Fsp[c];
    }
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
    if (threadIdx.x == 0) { load_consts(*dd, 0, Kd); base = dd->st[0]; }
    __syncthreads();
    const R* b = reinterpret_cast<const R*>(base);
    double acc[kDiagFields] = {0, 0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const SV<R> w = load_state(b, Kd.plane, c);
        const double H = pair_value(w.Hh, w.Hl), C = pair_value(w.Ch, w.Cl);
        double T, Fl;
        invert_enthalpy(Kd, H, 0.0, clamp01(C), T, Fl);
        const double rho = mix(clamp01(C), Fl, Kd.rho);
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
        const double rho = mix(clamp01(C), Fl, Kd.rho);
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

// Device address of g_noalloc_partials on the current device.  In host code
// the array's name is only a host-side stand-in, never a device address, so
// the address is resolved once per device (with that device current).
int noalloc_scratch(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(EULBFS_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(EULBFS_ECUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(EULBFS_ECUDA, "cudaGetSymbolAddress of the diagnostics scratch array failed");
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
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
    Consts<double> Kd = {};
    const eulbfs_phase* ph[3] = {&props->s, &props->l, &props->g};
    for (int k = 0; k < 3; ++k) { Kd.rho[k] = ph[k]->rho; Kd.cp[k] = ph[k]->cp; }
    Kd.Ts = props->Ts;
    Kd.Tl = props->Tl;
    Kd.L = props->L;
    Kd.plane = n;
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
