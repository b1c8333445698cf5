// cell.cuh -- per-cell device code of the difference-free conservative phase-field LBM
// (Zhao, Patel & Lee, arXiv:2407.12263): Lax-Wendroff pull, macroscopic stage, collisions.
//
// Storage (Q planes of N (f, g) pairs). Plane i >= 1 holds the populations shifted by their
// lattice weight times a reference level, f_i - t_i w0 (w0 = p0 / cs^2) and g_i - t_i phi_ref
// (phi_ref = 0 or 1, the bulk phase that fills most of the grid). Plane 0 holds the zeroth
// moments, sum_i f_i - w0 (FP32) and phi (the 32-bit fixed-point integer phi * 2^30), in place
// of the rest populations, which they fix exactly (f_0 = sum_i f_i - sum_{i>=1} f_i). These are
// exact changes of variables:
//  * propagation and collision are linear with weights summing to one, so the shift passes
//    through them, and every FP32 value is a deviation instead of a number of order t_i;
//  * the rest population does not move and the collision conserves the zeroth moment, so
//    phi_new(x) = phi*(x) + sum_{i>=1} [LW(g*_i)(x) - g*_i(x)] and the collision leaves it alone.
//    Held as an integer and advanced by integer face fluxes (see pull), sum phi is conserved
//    exactly, and no per-step rounding bias enters phi in any cell.
// The Lax-Wendroff update of the moving populations is evaluated in difference form: it
// returns a uniform field unchanged bit for bit. All arithmetic is FP32 with constants folded
// (1/cs^2 = 3, 1/(2 cs^4) = 4.5).
#pragma once

#include "lattice.cuh"
#include "lbm_internal.h"
#include "storage.cuh"

namespace lbm {

constexpr float kNormalGuard = 1e-24f;  // n = 0 where |K1|^2 (or |grad phi|^2) <= this

// Element offsets from a cell to its six face neighbours on the periodic grid.
struct Nbr {
    int xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nbr make_nbr(const Params& P, int x, int y, int z) {
    Nbr n;
    n.xm = (x == 0) ? P.nx - 1 : -1;
    n.xp = (x == P.nx - 1) ? -(P.nx - 1) : 1;
    n.ym = (y == 0) ? (P.ny - 1) * P.nx : -P.nx;
    n.yp = (y == P.ny - 1) ? -(P.ny - 1) * P.nx : P.nx;
    n.zm = (z == 0) ? (P.nz - 1) * P.nxy : -P.nxy;
    n.zp = (z == P.nz - 1) ? -(P.nz - 1) * P.nxy : P.nxy;
    return n;
}

// Cells on a wall side (walls lie half-way between the last cell and the next).
struct WallSide {
    bool xlo, xhi, ylo, yhi, zlo, zhi;
};

__device__ __forceinline__ WallSide make_wall_side(const Params& P, int x, int y, int z) {
    WallSide w;
    w.xlo = (P.walls & 1) && x == 0;
    w.xhi = (P.walls & 1) && x == P.nx - 1;
    w.ylo = (P.walls & 2) && y == 0;
    w.yhi = (P.walls & 2) && y == P.ny - 1;
    w.zlo = (P.walls & 4) && z == 0;
    w.zhi = (P.walls & 4) && z == P.nz - 1;
    return w;
}

// Whether x + s e_i lies beyond a wall.
template <int Q>
__device__ __forceinline__ bool crosses_wall(const WallSide& w, int i, int s) {
    const int ex = s * Lat<Q>::cx(i), ey = s * Lat<Q>::cy(i), ez = s * Lat<Q>::cz(i);
    return (ex < 0 && w.xlo) || (ex > 0 && w.xhi) || (ey < 0 && w.ylo) || (ey > 0 && w.yhi) || (ez < 0 && w.zlo) ||
           (ez > 0 && w.zhi);
}

// Offsets for gradients of phi with walls: across a wall the stencil reads the mirror image
// of the cell, i.e. the same index along that axis (zero normal gradient).
__device__ __forceinline__ Nbr mirror_at_walls(const Nbr& n, const WallSide& w) {
    Nbr m = n;
    if (w.xlo) m.xm = 0;
    if (w.xhi) m.xp = 0;
    if (w.ylo) m.ym = 0;
    if (w.yhi) m.yp = 0;
    if (w.zlo) m.zm = 0;
    if (w.zhi) m.zp = 0;
    return m;
}

// Offset of the cell x + s e_i (s = +1 or -1). Folds to two or three adds once unrolled.
template <int Q>
__device__ __forceinline__ int link_offset(const Nbr& n, int i, int s) {
    const int ex = s * Lat<Q>::cx(i), ey = s * Lat<Q>::cy(i), ez = s * Lat<Q>::cz(i);
    return (ex > 0 ? n.xp : ex < 0 ? n.xm : 0) + (ey > 0 ? n.yp : ey < 0 ? n.ym : 0) +
           (ez > 0 ? n.zp : ez < 0 ? n.zm : 0);
}

// Lax-Wendroff propagation (Sec. 2.2) into registers:
//   fbar_i(x) = f*_i(x) - c [f*_i(x) - f*_i(x - e_i)] - c(1-c)/2 [f*_i(x + e_i) - 2 f*_i(x) + f*_i(x - e_i)]
//             = f*_i(x) + lw_m [f*_i(x - e_i) - f*_i(x)] + lw_p [f*_i(x + e_i) - f*_i(x)],
// the same for g, and the zeroth moments fb[0] = sum fbar - w0, gb[0] = phi - phi_ref of the
// propagated state. Each load brings the (f_i, g_i) pair of one cell. With WALLS, a stencil
// point beyond a wall reads the opposite pair of this cell instead (half-way bounce-back; at
// c = 1 it is the usual bounce-back).
//
// phi itself advances in flux form: the same update reads
//   gbar_i(x) = g*_i(x) + F_i(x - e_i/2) - F_i(x + e_i/2),  F_i = lw_m g*_i(upwind) - lw_p g*_i(downwind),
// so phi_fx (phi * 2^30, the fixed-point plane-0 value) loses, across each face x + e_i/2, the
// net outflow of the pair (i, j = opposite of i) that crosses it,
//   N = F_i - F_j = lw_m [g*_i(x) - g*_j(x + e_i)] - lw_p [g*_i(x + e_i) - g*_j(x)],
// rounded to an integer. The cell on the other side evaluates the same expression with every
// difference negated; IEEE subtraction, products and round-to-nearest are odd in sign, so it
// gets -N bit for bit, the integers cancel in pairs and sum phi over the grid never changes.
// At a wall the two terms of N read the same values of this cell, so N = 0 exactly.
// Each load brings the words of an opposite pair (i, j) at one stencil cell (storage.cuh): at
// x - e_i the pair of i there and that of j at x + e_j, at x + e_i the reverse, so 3 loads serve
// both stencils. With walls, a stencil point beyond a wall takes the opposite pair of this cell
// instead (half-way bounce-back), from the word loaded at x. im, ip: the cell indices of x - e_i
// and x + e_i; with unsigned indices each address is one wide multiply-add on the plane's base
// (the FP32 step), the 16-bit steps, held at 96 registers, form them from signed offsets
// (Store<S>::kUnsignedIndex), which ran faster there.
// RAW: fb[i], gb[i] (i >= 1) stay in storage units (see storage.cuh); fb[0], gb[0] are always in
// population units. Every difference of two stored values is taken as (neighbour) - (FP32 of
// this cell's value) with one rounding; a difference a - b in the flux is written -(b - a),
// which is the same number.
template <int Q, bool WITH_F, int S, bool WALLS = false, bool RAW = false>
__device__ __forceinline__ void pull(const Params& P, const void* __restrict__ state, int c, const Nbr& nb,
                                     float (&fb)[Q], float (&gb)[Q], int& phi_fx,
                                     const WallSide& ws = WallSide{}) {
    using St = Store<S>;
    constexpr float sf = RAW ? 1.0f : St::kInvF, sg = RAW ? 1.0f : St::kInvG;
    float df = 0.f;                 // increment of sum f, storage units
    unsigned int dphi = 0u;         // increment of phi_fx (wraps; the true sum fits in 32 bits)
    const float fa = P.flux_as, fbk = P.flux_bs;  // flux_a, flux_b times the storage's kInvG
    const float2 lwm = make_float2(P.lw_m, P.lw_m), lwp = make_float2(P.lw_p, P.lw_p);
    const float2 nfa = make_float2(-fa, -fa), fbk2 = make_float2(fbk, fbk);
#pragma unroll
    for (int k = 0; k < Lat<Q>::kPairs; ++k) {
        const int i = Lat<Q>::pair_first(k), j = Lat<Q>::pair_second(k);
        // x - e_i and x + e_i; for j = opposite of i they are x + e_j and x - e_j
        const unsigned im = (unsigned)(c + link_offset<Q>(nb, i, -1)), ip = (unsigned)(c + link_offset<Q>(nb, i, +1));
        typename St::Raw rmi, r0i, rpi, rmj, r0j, rpj;
        {
            const typename St::Word* pw = pair_plane<S>(state, P.N, k);
            const typename St::Word* qm;
            const typename St::Word* qp;
            if constexpr (St::kUnsignedIndex) {
                qm = pw + im;
                qp = pw + ip;
            } else {
                qm = pw + c + ((int)im - c);
                qp = pw + c + ((int)ip - c);
            }
            const typename St::Word vm = __ldg(qm), v0 = __ldg(pw + c), vp = __ldg(qp);
            rmi = St::lo(vm);
            rpj = St::hi(vm);
            r0i = St::lo(v0);
            r0j = St::hi(v0);
            rpi = St::lo(vp);
            rmj = St::hi(vp);
            if (WALLS) {  // half-way bounce-back: beyond a wall, the opposite pair of this cell
                if (crosses_wall<Q>(ws, i, -1)) rmi = r0j;
                if (crosses_wall<Q>(ws, i, +1)) rpi = r0j;
                if (crosses_wall<Q>(ws, j, -1)) rmj = r0i;
                if (crosses_wall<Q>(ws, j, +1)) rpj = r0i;
            }
        }
        const float2 v0i = St::cvt(r0i), v0j = St::cvt(r0j);
        // the Lax-Wendroff corrections of (f_i, g_i) and (f_j, g_j), both members at once
        // (packed FP32 arithmetic, each lane rounded as its scalar form would be)
        const float2 ei = __ffma2_rn(lwm, St::sub2(rmi, v0i), __fmul2_rn(lwp, St::sub2(rpi, v0i)));
        const float2 ej = __ffma2_rn(lwm, St::sub2(rmj, v0j), __fmul2_rn(lwp, St::sub2(rpj, v0j)));
        const float2 bi = __fadd2_rn(v0i, ei), bj = __fadd2_rn(v0j, ej);
        gb[i] = bi.y * sg;
        gb[j] = bj.y * sg;
        // net outflow of phi across x + e_i/2 and across x - e_i/2 (= x + e_j/2):
        //   fa (g_i(x) - g_j(x + e_i)) + fbk (g_i(x + e_i) - g_j(x)), and the same with i, j swapped
        const float2 out = __ffma2_rn(nfa, make_float2(St::sub_g(rmj, v0i.y), St::sub_g(rmi, v0j.y)),
                                      __fmul2_rn(fbk2, make_float2(St::sub_g(rpi, v0j.y), St::sub_g(rpj, v0i.y))));
        dphi -= (unsigned int)__float2int_rn(out.x) + (unsigned int)__float2int_rn(out.y);
        if (WITH_F) {
            fb[i] = bi.x * sf;
            fb[j] = bj.x * sf;
            df += ei.x + ej.x;
        }
    }
    const float2 m0 = Store<S>::kUnsignedIndex ? __ldg(moment_plane(state) + (unsigned)c) : __ldg(moment_plane(state) + c);
    phi_fx = (int)((unsigned int)__float_as_int(m0.y) + dphi);
    gb[0] = __int2float_rn((int)((unsigned int)phi_fx - (unsigned int)P.phi_ref_fx)) * kPhiFxInvF;
    if (WITH_F) fb[0] = m0.x + df * St::kInvF;
}

struct Macro {
    float Phi;    // phi - phi_ref
    float phi, omphi, rho, inv_rho;
    float u[3];
    float n[3];
    float S[3];
    float gphi[3];
    float Pbar;   // sum fbar - w0
    float P;      // p / cs^2 - w0 = sum fbar - w0 + u . grad rho / 2
    float gnorm;  // |grad phi|
    float gsum[3];  // sum g_i e_i of the propagated g
};

// phi, rho, u (Sec. 2.3, Eq. momentum): rho u = sum fbar_i e_i + rho G / 2.
// U: the storage type whose units fb[i >= 1] are in (STORE_F32: population units).
template <int Q, bool GEN, int U = STORE_F32>
__device__ __forceinline__ void macro_flow(const Params& P, const float (&fb)[Q], const float (&gb)[Q], Macro& m) {
    m.Phi = gb[0];
    m.phi = P.phi_ref + m.Phi;
    m.omphi = (1.f - P.phi_ref) - m.Phi;  // 1 - phi, exact on the phi_ref side
    m.Pbar = fb[0];
    // first moments of f and g together, (sum f_i e_i, sum g_i e_i) per axis in packed FP32:
    // opposite velocities enter as one difference
    float2 s[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int k = 0; k < Lat<Q>::kPairs; ++k) {
        const int i = Lat<Q>::pair_first(k), j = Lat<Q>::pair_second(k);
        const float2 d = fsub2_rn(make_float2(fb[i], gb[i]), make_float2(fb[j], gb[j]));  // e_i (f_i - f_j)
        const int e[3] = {Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (e[a] > 0) s[a] = __fadd2_rn(s[a], d);
            if (e[a] < 0) s[a] = fsub2_rn(s[a], d);
        }
    }
    if constexpr (Store<U>::kInvF != 1.0f || Store<U>::kInvG != 1.0f) {  // to population units: exact
        const float2 inv = make_float2(Store<U>::kInvF, Store<U>::kInvG);  // powers of two
#pragma unroll
        for (int a = 0; a < 3; ++a) s[a] = __fmul2_rn(s[a], inv);
    }
    float jx = s[0].x, jy = s[1].x, jz = s[2].x;
    m.gsum[0] = s[0].y;
    m.gsum[1] = s[1].y;
    m.gsum[2] = s[2].y;
    if (GEN) {
        m.rho = P.rho2 + P.drho * m.phi;
        m.inv_rho = 1.0f / m.rho;
        jx += 0.5f * m.rho * P.G[0];
        jy += 0.5f * m.rho * P.G[1];
        jz += 0.5f * m.rho * P.G[2];
    } else {
        m.rho = P.rho2;
        m.inv_rho = 1.0f;  // rho2 = 1 and no density contrast
    }
    m.u[0] = jx * m.inv_rho;
    m.u[1] = jy * m.inv_rho;
    m.u[2] = jz * m.inv_rho;
}

// Interface normal, sharpening flux and gradients from the first central moment of g
// (Sec. 2.3, Eq. norm): K1 = sum g_i e_i - phi u, n = -K1/|K1|, S = 4 phi (1-phi)/delta n,
// grad phi = (tau_phi cs^2 S - K1) / ((tau_phi + 1/2) cs^2). The shift t_i phi_ref has no
// first moment, so the stored deviations give K1 directly.
template <int Q, int U = STORE_F32>
__device__ __forceinline__ void macro_interface_df(const Params& P, Macro& m) {
    float kx = m.gsum[0], ky = m.gsum[1], kz = m.gsum[2];  // sum g_i e_i from macro_flow
    kx -= m.phi * m.u[0];
    ky -= m.phi * m.u[1];
    kz -= m.phi * m.u[2];
    const float k2 = kx * kx + ky * ky + kz * kz;
    const float r = (k2 > kNormalGuard) ? -rsqrtf(k2) : 0.f;
    m.n[0] = kx * r;
    m.n[1] = ky * r;
    m.n[2] = kz * r;
    const float smag = P.four_over_delta * m.phi * m.omphi;
    m.S[0] = smag * m.n[0];
    m.S[1] = smag * m.n[1];
    m.S[2] = smag * m.n[2];
    m.gphi[0] = P.grad_s * m.S[0] - P.grad_k * kx;
    m.gphi[1] = P.grad_s * m.S[1] - P.grad_k * ky;
    m.gphi[2] = P.grad_s * m.S[2] - P.grad_k * kz;
}

// Finite-difference variant (Sec. 3.4): n = grad phi / |grad phi| with grad phi given.
__device__ __forceinline__ void macro_interface_fd(const Params& P, float gx, float gy, float gz, Macro& m) {
    m.gphi[0] = gx;
    m.gphi[1] = gy;
    m.gphi[2] = gz;
    const float g2 = gx * gx + gy * gy + gz * gz;
    const float r = (g2 > kNormalGuard) ? rsqrtf(g2) : 0.f;
    m.n[0] = gx * r;
    m.n[1] = gy * r;
    m.n[2] = gz * r;
    const float smag = P.four_over_delta * m.phi * m.omphi;
    m.S[0] = smag * m.n[0];
    m.S[1] = smag * m.n[1];
    m.S[2] = smag * m.n[2];
}

// Pressure (Eq. pressure): p/cs^2 = sum fbar_i + u . grad rho / 2, held as P = p/cs^2 - w0.
template <bool GEN>
__device__ __forceinline__ void macro_pressure(const Params& P, Macro& m) {
    m.P = m.Pbar;
    if (GEN) m.P += 0.5f * P.drho * (m.u[0] * m.gphi[0] + m.u[1] * m.gphi[1] + m.u[2] * m.gphi[2]);
    m.gnorm = sqrtf(m.gphi[0] * m.gphi[0] + m.gphi[1] * m.gphi[1] + m.gphi[2] * m.gphi[2]);
}

// Isotropic central difference of the propagated phi field (Sec. 3.4):
// grad phi = sum_{i != 0} t_i e_i [phi(x + e_i) - phi(x - e_i)] / (2 cs^2)
//          = 3 sum_{i != 0} t_i e_i phi(x + e_i)   (the velocity set is symmetric).
// The plane holds phi - phi_ref; the constant drops out of the difference.
template <int Q>
__device__ __forceinline__ void fd_gradient(const float* __restrict__ phi, int c, const Nbr& nb,
                                            float& gx, float& gy, float& gz) {
    gx = gy = gz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float v = Lat<Q>::w(i) * __ldg(phi + c + link_offset<Q>(nb, i, +1));
        if (Lat<Q>::cx(i) > 0) gx += v;
        if (Lat<Q>::cx(i) < 0) gx -= v;
        if (Lat<Q>::cy(i) > 0) gy += v;
        if (Lat<Q>::cy(i) < 0) gy -= v;
        if (Lat<Q>::cz(i) > 0) gz += v;
        if (Lat<Q>::cz(i) < 0) gz -= v;
    }
    gx *= 3.f;
    gy *= 3.f;
    gz *= 3.f;
}

template <int Q>
__device__ __forceinline__ float edot(int i, const float (&v)[3]) {
    float r = 0.f;
    if (Lat<Q>::cx(i) > 0) r += v[0];
    if (Lat<Q>::cx(i) < 0) r -= v[0];
    if (Lat<Q>::cy(i) > 0) r += v[1];
    if (Lat<Q>::cy(i) < 0) r -= v[1];
    if (Lat<Q>::cz(i) > 0) r += v[2];
    if (Lat<Q>::cz(i) < 0) r -= v[2];
    return r;
}

// Collisions, in place on fb / gb (shifted values, i >= 1):
//   f^eq_i - t_i w0 = t_i [P + rho gam_i - 4.5 Pi_s:(e_i e_i - cs^2 I)]            (Eq. geq_s,
//        gam_i = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2, the CSS term entering with a minus sign so that
//        the second moment is p I + rho u u - Pi_s as App. A requires)
//   Pi_s:(e e - cs^2 I) = sigma |grad phi| [|e|^2 - (e.n)^2 - cs^2 (D - |n|^2)]        (Eq. surface)
//   S_i = t_i gam_i (e_i - u) . grad rho                                                 (App. A)
//   R_i = t_i [3 (e_i - u) + 9 (e_i . u) e_i] . rho G                                    (Eq. body)
//   f*_i = fbar_i - omega_rho (fbar_i - f^eq_i + F_i/2) + F_i                           (Eq. c-n_m)
//   g^eq_i - t_i phi_ref = t_i [(phi - phi_ref) + phi gam_i + tau_phi e_i . S]          (Eq. geq)
//   g*_i = g_i - omega_g (g_i - g^eq_i)                                                  (Eq. c-n_c)
// Opposite velocities i and j (e_j = -e_i) share e.u, (e.n)^2 and e.S up to sign, so each pair
// splits into a part even in e (gam_even = 4.5 (e.u)^2 - 1.5 u^2, Pi_s term) and a part odd in
// e (3 e.u, e.S), evaluated once.
// Zeroth moments: the g collision conserves phi; sum_i f*_i = sum_i fbar_i + u . grad rho,
// because sum_i F_i = u . grad rho and sum_i f^eq_i = p / cs^2.
// U: the storage type whose units fb[i], gb[i] (i >= 1) are in; the weights t_i carry its
// scales, so f^eq, F and g^eq come out in the same units.
template <int Q, bool GEN, int U = STORE_F32>
__device__ __forceinline__ void collide(const Params& P, const Macro& m, float (&fb)[Q], float (&gb)[Q]) {
    constexpr int D = Lat<Q>::D;
    const float u2 = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
    const float sg = P.sigma * m.gnorm;
    const float trc = (float)D - (m.n[0] * m.n[0] + m.n[1] * m.n[1] + m.n[2] * m.n[2]);
    const float pi0 = -sg * (trc * (1.0f / 3.0f));  // sigma |grad phi| (|e|^2 - cs^2 trc) for |e|^2 = 0
    const float gr[3] = {P.drho * m.gphi[0], P.drho * m.gphi[1], P.drho * m.gphi[2]};
    const float rG[3] = {m.rho * P.G[0], m.rho * P.G[1], m.rho * P.G[2]};
    const float ugr = m.u[0] * gr[0] + m.u[1] * gr[1] + m.u[2] * gr[2];
    const float urG = m.u[0] * rG[0] + m.u[1] * rG[1] + m.u[2] * rG[2];
    float omega_f = P.omega_f;
    if (GEN) {
        const float tau = P.tau_f * (1.f + P.mu_m1 * m.phi) * m.inv_rho;  // eta(phi) / (rho cs^2)
        omega_f = 1.0f / (tau + 0.5f);
    }
    const float omega_g = P.omega_g;
    // f* = (1 - w_f) fbar + w_f f^eq + (1 - w_f/2) F and g* = (1 - w_g) g + w_g g^eq: the same
    // collisions, one multiply-add per population once the pair's parts are known. f and g of
    // a population travel together as the lanes of packed FP32 operations.
    const float a_f = 1.f - omega_f, c_f = 1.f - 0.5f * omega_f, a_g = 1.f - omega_g;
    const float2 a_fg = make_float2(a_f, a_g);
    const float u2h = 1.5f * u2;
    const float feq0 = m.P - 4.5f * pi0;  // P - 4.5 Pi_s term shared by every |e|^2 class
    const float rho3 = 3.f * m.rho, phi3 = 3.f * m.phi, urG3 = 3.f * urG;
    const float2 rho_phi = make_float2(m.rho, m.phi);
#pragma unroll
    for (int k = 0; k < Lat<Q>::kPairs; ++k) {
        const int i = Lat<Q>::pair_first(k), j = Lat<Q>::pair_second(k);
        const float t = Lat<Q>::w(i) * Store<U>::kScaleF;
        const float tg = Lat<Q>::w(i) * Store<U>::kScaleG;
        const float twg = tg * omega_g;
        const float eu = edot<Q>(i, m.u);
        const float en = edot<Q>(i, m.n);
        const float es = edot<Q>(i, m.S);
        const float even = 4.5f * eu * eu - u2h;                   // gam_i = even + 3 eu, gam_j = even - 3 eu
        const float pis = sg * ((float)Lat<Q>::e2(i) - en * en);  // Pi_s term minus its |e|^2 = 0 part
        // even parts of the equilibria over t and tg: f^eq_i = t (Xe + Xo), f^eq_j = t (Xe - Xo),
        //   Xe = P - 4.5 Pi_s term + rho even;  g^eq: Phi + phi even
        const float2 Xe = __ffma2_rn(rho_phi, make_float2(even, even), make_float2(feq0 - 4.5f * pis, m.Phi));
        // (w_f f^eq + (1 - w_f/2) F, w_g g^eq), split into parts even and odd in e
        float2 Ae, Ao;
        if (GEN) {
            // F_i = t (Ye + Yo), F_j = t (Ye - Yo), from e_j = -e_i in S_i and R_i:
            //   Ye = 3 eu (e.grad rho + 3 e.rho G) - even u.grad rho - 3 u.rho G
            //   Yo = even e.grad rho - 3 eu u.grad rho + 3 e.rho G
            const float egr = edot<Q>(i, gr);
            const float erG = edot<Q>(i, rG);
            const float odd = 3.f * eu;
            const float Ye = odd * (egr + 3.f * erG) - even * ugr - urG3;
            const float Yo = even * egr - odd * ugr + 3.f * erG;
            Ae = __fmul2_rn(make_float2(t, twg), make_float2(omega_f * Xe.x + c_f * Ye, Xe.y));
            Ao = __fmul2_rn(make_float2(t, twg), make_float2(omega_f * (rho3 * eu) + c_f * Yo, phi3 * eu + P.tau_phi * es));
        } else {
            const float tw = t * omega_f;  // uniform over the grid
            Ae = __fmul2_rn(make_float2(tw, twg), Xe);
            Ao = __fmul2_rn(make_float2(tw * rho3, twg), make_float2(eu, phi3 * eu + P.tau_phi * es));
        }
        const float2 qi = __ffma2_rn(a_fg, make_float2(fb[i], gb[i]), __fadd2_rn(Ae, Ao));
        const float2 qj = __ffma2_rn(a_fg, make_float2(fb[j], gb[j]), fsub2_rn(Ae, Ao));
        fb[i] = qi.x;
        gb[i] = qi.y;
        fb[j] = qj.x;
        gb[j] = qj.y;
    }
    fb[0] = GEN ? m.Pbar + ugr : m.Pbar;  // plane 0 keeps phi_fx: the collision conserves phi
}

// One whole time step of cell (x, y, z): propagate, macroscopic stage, collide, store the Q
// post-collision pairs into fg_out. The single-case step kernel and the batched kernel both run
// this, so a case gives the same bits whichever of them advances it.
template <int Q, int SCHEME, bool GEN, int S>
__device__ __forceinline__ void step_cell(const Params& P, const void* __restrict__ fg_in, void* __restrict__ fg_out,
                                          const float* __restrict__ phi_fd, int x, int y, int z) {
    const Nbr nb = make_nbr(P, x, y, z);
    const int c = (z * P.ny + y) * P.nx + x;
    const WallSide ws = GEN ? make_wall_side(P, x, y, z) : WallSide{};

    float fb[Q], gb[Q];
    int phi_fx;
    // Only warps holding a wall cell take the propagation with per-link wall tests. The choice is
    // per warp, so a warp never runs both versions; for a cell off the walls both read the same
    // addresses and give the same bits, so the result does not depend on it.
    const bool at_wall = GEN && (ws.xlo || ws.xhi || ws.ylo || ws.yhi || ws.zlo || ws.zhi);
    if (GEN && __any_sync(__activemask(), at_wall))
        pull<Q, true, S, true, true>(P, fg_in, c, nb, fb, gb, phi_fx, ws);
    else
        pull<Q, true, S, false, true>(P, fg_in, c, nb, fb, gb, phi_fx);

    // fb[i], gb[i] (i >= 1) stay in storage units until they are stored
    Macro m;
    macro_flow<Q, GEN, S>(P, fb, gb, m);
    if (SCHEME == SCHEME_DF) {
        macro_interface_df<Q, S>(P, m);
    } else {
        float gx, gy, gz;
        fd_gradient<Q>(phi_fd, c, GEN ? mirror_at_walls(nb, ws) : nb, gx, gy, gz);
        macro_interface_fd(P, gx, gy, gz, m);
    }
    macro_pressure<GEN>(P, m);
    collide<Q, GEN, S>(P, m, fb, gb);

    // streaming stores: the output is not re-read this step; one word per opposite pair
    __stcs(moment_plane(fg_out) + c, make_float2(fb[0], __int_as_float(phi_fx)));
#pragma unroll
    for (int k = 0; k < Lat<Q>::kPairs; ++k) {
        const int i = Lat<Q>::pair_first(k), j = Lat<Q>::pair_second(k);
        __stcs(pair_plane<S>(fg_out, P.N, k) + c, Store<S>::word(fb[i], gb[i], fb[j], gb[j]));
    }
}

}  // namespace lbm
