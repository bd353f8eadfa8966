// device_common.cuh -- device helpers shared by the stage kernel and the
// auxiliary kernels of libeulbfs: state access, compensated sums, the
// enthalpy closure (Eq. 5-7), boundary mapping and the derived fields.
#pragma once
#include <math.h>
#include <stdint.h>

#include "eulbfs_internal.h"

namespace eulbfs {

enum { BC_PERIODIC = 0, BC_DIRICHLET_T, BC_ADIABATIC, BC_NOSLIP, BC_SYMMETRY, BC_OUTLET, BC_NOFLUX, BC_WETTING,
       BC_WETTING_HYST };

template <class R> struct Prec;
template <> struct Prec<double> { static constexpr int NP = 5; };
template <> struct Prec<float> { static constexpr int NP = 7; };

// ---------------------------------------------------------------------------
// State access.  FP64: H p mx my C.  FP32C: Hhi Hlo p mx my Chi Clo.
// ---------------------------------------------------------------------------
template <class R>
struct SV { R Hh, Hl, p, mx, my, Ch, Cl; };

// Loads of data that other CTAs write during the same launch (a stage's
// output, read by the next stage of a whole-step launch; F_s and dF_s/dt)
// are cached in L2 only: an SM's L1 is not kept coherent with other SMs'
// stores, and a line it cached earlier in the launch could span cells that
// were written after it was read.
template <class T>
__device__ __forceinline__ T ld_l2(const T* p) { return __ldcg(p); }

__device__ __forceinline__ SV<double> load_state(const double* b, long long P, long long c) {
    SV<double> s;
    s.Hh = ld_l2(b + c); s.Hl = 0.0; s.p = ld_l2(b + P + c); s.mx = ld_l2(b + 2 * P + c);
    s.my = ld_l2(b + 3 * P + c); s.Ch = ld_l2(b + 4 * P + c); s.Cl = 0.0;
    return s;
}
__device__ __forceinline__ SV<float> load_state(const float* b, long long P, long long c) {
    SV<float> s;
    s.Hh = ld_l2(b + c); s.Hl = ld_l2(b + P + c); s.p = ld_l2(b + 2 * P + c); s.mx = ld_l2(b + 3 * P + c);
    s.my = ld_l2(b + 4 * P + c); s.Ch = ld_l2(b + 5 * P + c); s.Cl = ld_l2(b + 6 * P + c);
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

// Quotient in the working precision: correctly rounded in FP64; in FP32 the
// hardware approximate division (max error 2 ulp for |b| in [2^-126, 2^126]),
// which is far inside the FP32 path's tolerance and much cheaper than the
// IEEE division sequence.
__device__ __forceinline__ double wdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float wdiv(float a, float b) { return __fdividef(a, b); }

// Eq. 5-6 with the readings of the oracle: uniform latent heat, Eq. 7 mixture
// heat capacity gated by clamp(C).  H = Hh + Hl (Hl = 0 in FP64); the
// differences H - H_s and H - H_l are formed from the pair without rounding H.
// A constant group (Q4) of Consts: one 16-byte load in FP32.
template <class R>
__device__ __forceinline__ Q4<R> ld4(const Q4<R>& q) { return q; }
template <>
__device__ __forceinline__ Q4<float> ld4(const Q4<float>& q) {
    const float4 v = *reinterpret_cast<const float4*>(&q);
    return Q4<float>{v.x, v.y, v.z, v.w};
}

// The branches' heat capacities and H_l come from constant groups, so both
// readings run the same instructions: reading R1 mixes both heat capacities
// by C~ and H_l = C_p^liq T_l + L; with Eq. 7 as printed H_s = C_p,s T_s and
// H_l = C_p,l T_l + L with the pure phases' heat capacities, the solid
// branch's C_p is C_p,s (Eq. 7 at F_s = 1) and the liquid branch's Eq. 7 at
// F_s = 0 (as in R1).
template <class R>
__device__ __forceinline__ void invert_enthalpy(const Consts<R>& K, R Hh, R Hl, R Ct, R& T, R& Fl) {
    const Q4<R> cp = ld4(K.enthc), e = ld4(K.enth);
    const R cps = fma(Ct, cp.y, cp.x);     // R1: C~ cp_s + (1 - C~) cp_g
    const R cpl = fma(Ct, cp.w, cp.z);     // C~ cp_l + (1 - C~) cp_g
    const R HL = fma(cpl, K.hl[0], K.hl[1]);
    const R Hs = cps * e.x;
    const R ds = (Hh - Hs) + Hl;
    const R dl = (Hh - HL) + Hl;
    if (ds < R(0)) {
        Fl = R(0);
        T = wdiv(Hh + Hl, cps);
    } else if (dl > R(0)) {
        Fl = R(1);
        T = e.y + wdiv(dl, cpl);
    } else if (HL > Hs) {
        Fl = wdiv(ds, HL - Hs);
        T = fma(Fl, e.w, e.x);
    } else {
        Fl = R(1);
        T = e.y;
    }
}

// Eq. 7 as m.x + X (m.y + Y m.z).  Reading R1: gamma = C~ [F_s g_s + F_l g_l]
// + (1 - C~) g_g = g_g + C~ ((g_s - g_g) + F_l (g_l - g_s)), (X, Y) = (C~, F_l).
// As printed: F_s g_s + (1 - F_s)(C~ g_l + (1 - C~) g_g)
// = g_s + F_l ((g_g - g_s) + C~ (g_l - g_g)), (X, Y) = (F_l, C~).  The weights
// are swapped by the reading flag K.printed (0 or 1), without a branch.
template <class R>
struct MixW { R X, Y; };

template <class R>
__device__ __forceinline__ MixW<R> mix_weights(const Consts<R>& K, R Ct, R Fl) {
    const R p = K.printed;
    const R d = Fl - Ct;
    return MixW<R>{fma(p, d, Ct), fma(-p, d, Fl)};
}

template <class R>
__device__ __forceinline__ R mix(const MixW<R>& w, const Q4<R>& m) {
    return fma(w.X, fma(w.Y, m.z, m.y), m.x);
}

// The factor on F_s in the volume-change sources and the solid projection:
// C~ (reading R1), 1 with Eq. 7 as printed.
template <class R>
__device__ __forceinline__ R solid_gate(const Consts<R>& K, R C) {
    return fmax(clamp01(C), K.printed);
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

// map_axis along y for a slab of a split domain: rows within the halo
// ([-hlo, 0) and [ny, ny + hhi)) are read where they are, with no boundary
// rule (k = 0); rows beyond the halo are never used and are clamped into it.
template <class R>
__device__ __forceinline__ void map_row(const Consts<R>& K, int g, int& s, int& k, int& side) {
    if (g < 0 && K.hlo) { s = g < -K.hlo ? -K.hlo : g; k = 0; side = YLO; return; }
    if (g >= K.ny && K.hhi) { s = g > K.ny + K.hhi - 1 ? K.ny + K.hhi - 1 : g; k = 0; side = YHI; return; }
    map_axis(g, K.ny, K.per_y, YLO, s, k, side);
}

// Ghost value rules (boundary conditions on macroscopic variables).
template <class R>
struct Prim { R T, Fl, cp, rho, lam, mu, p, u, v, C; };

// Phase field C = C_hi + C_lo of cell c of a state buffer.
__device__ __forceinline__ double load_C(const double* b, long long P, long long c) { return ld_l2(b + 4 * P + c); }
__device__ __forceinline__ float load_C(const float* b, long long P, long long c) {
    return ld_l2(b + 5 * P + c) + ld_l2(b + 6 * P + c);
}

// Wetting coefficient 4 cos(theta) / xi of the wall position t of `side`
// (the row of an x side, the column of a y side; clamped into the domain or
// wrapped on a periodic axis).  WETTING: the fixed angle.  WETTING_HYST
// (contact-angle hysteresis): the apparent angle of the two wall layers,
// cos = dC/dn_out / |grad C| with dC/dn_out = C_0 - C_1 and the tangential
// central difference along layer 0 (one-sided at a walled end), clamped to
// [cos theta_adv, cos theta_rec]; the fixed angle where the wall cell carries
// no interface (C_0 (1 - C_0) < 1e-3: there the direction of grad C is
// round-off and the wetting correction, which scales with C (1 - C), is
// negligible).
template <class R>
__device__ __forceinline__ R wall_wetting(const Consts<R>& K, const R* in, int side, int t) {
    if (K.bc_c[side] != BC_WETTING_HYST) return K.wet[side];
    const bool xs = side < 2;
    const int n = xs ? K.ny : K.nx, m = xs ? K.nx : K.ny;
    const int per = xs ? K.per_y : K.per_x;
    // along a slab's halo rows the wall continues: the tangential range of an
    // x side reaches into the halo
    const int tlo = xs ? -K.hlo : 0, thi = xs ? n - 1 + K.hhi : n - 1;
    int tc, tp, tm;
    if (per) {
        tc = ((t % n) + n) % n;
        tp = tc + 1 == n ? 0 : tc + 1;
        tm = tc == 0 ? n - 1 : tc - 1;
    } else {
        tc = t < tlo ? tlo : (t > thi ? thi : t);
        tp = tc + 1 > thi ? thi : tc + 1;
        tm = tc - 1 < tlo ? tlo : tc - 1;
    }
    const int l0 = (side == XLO || side == YLO) ? 0 : m - 1;
    const int l1 = (side == XLO || side == YLO) ? 1 : m - 2;
    auto at = [&](int layer, int tt) -> R {
        const long long c = (xs ? (long long)tt * K.nx + layer : (long long)layer * K.nx + tt) + K.off;
        return load_C(in, K.plane, c);
    };
    const R c0 = at(l0, tc);
    if (!(c0 * (R(1) - c0) >= R(1e-3))) return K.wet[side];
    const R dn = c0 - at(l1, tc);
    const R dd = at(l0, tp) - at(l0, tm);
    const R dt = per ? R(0.5) * dd : wdiv(dd, (R)(tp - tm));
    const R g = sqrt(dn * dn + dt * dt);
    if (!(g > R(0))) return K.wet[side];
    R c = wdiv(dn, g);
    c = c < K.cos_adv[side] ? K.cos_adv[side] : (c > K.cos_rec[side] ? K.cos_rec[side] : c);
    return K.four_over_xi * c;
}

// Ghost layer k of `side` from the mirror cell's values; wet = the side's
// wetting coefficient at this wall position (wall_wetting).
template <class R>
__device__ __forceinline__ void apply_ghost(const Consts<R>& K, int side, int k, bool x_normal, R wet, Prim<R>& q) {
    if (K.bc_t[side] == BC_DIRICHLET_T) q.T = R(2) * K.Tw[side] - q.T;
    const int f = K.bc_f[side];
    if (f == BC_OUTLET) q.p = -q.p;
    R& un = x_normal ? q.u : q.v;
    R& ut = x_normal ? q.v : q.u;
    if (f == BC_NOSLIP) { un = -un; ut = -ut; }
    else if (f == BC_SYMMETRY) { un = -un; }
    if (K.bc_c[side] == BC_WETTING || K.bc_c[side] == BC_WETTING_HYST)
        q.C = q.C + R(2 * k - 1) * wet * q.C * (R(1) - q.C);
}

template <class R>
__device__ __forceinline__ Prim<R> derive(const Consts<R>& K, const SV<R>& w) {
    Prim<R> q;
    const R C = w.Ch + w.Cl;
    const R Ct = clamp01(C);
    invert_enthalpy(K, w.Hh, w.Hl, Ct, q.T, q.Fl);
    const MixW<R> mw = mix_weights(K, Ct, q.Fl);
    q.cp = mix(mw, ld4(K.mcp));
    q.rho = mix(mw, ld4(K.mrho));
    q.lam = mix(mw, ld4(K.mlam));
    q.mu = mix(mw, ld4(K.mmu));
    const R r3 = wdiv(R(3), q.rho);     // 1 / (rho cs^2)
    q.u = w.mx * r3;
    q.v = w.my * r3;
    q.p = w.p;
    q.C = C;
    return q;
}

template <class R>
__device__ __forceinline__ double pair_value(R hi, R lo) { return (double)hi + (double)lo; }

template <class R>
__device__ __forceinline__ void put_pair(R& hi, R& lo, double x) {
    hi = (R)x;
    lo = (R)(x - (double)hi);
}

}  // namespace eulbfs
