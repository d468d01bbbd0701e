// goc_step.cuh -- the fused GOC-LBM time step (one launch per time step).
//
// A persistent grid walks over TX x TY tiles.  For each tile, one thread
// issues TMA bulk-tensor copies (cp.async.bulk.tensor.3d, mbarrier completion)
// of the stored populations, the stored force and the MIE populations of the
// tile plus its halo into shared memory; the copy of the next tile is in
// flight while the current one is computed (two stages).  Per tile:
//   phase 1 pulls the populations of the tile and a halo of one node (two next
//           to a wall) -- pull streaming with boundary conditions, Appendix E
//           Step 6, Eq. 101/103 -- and forms the hydrodynamic fields
//           (Appendix E Step 7, with the stored force of the previous step);
//   phase 2 takes, per node, the second-order normal derivatives, the MIE part
//           (Appendix G Steps 1-3, all local), stresses and effective force
//           (Eq. Special1_Force_terms with the Lorentz force of Eq.
//           Lorentzforce-GOC in F_ext), the central-moment collision (Appendix E
//           Steps 1-5), and stores the post-collision populations and force.
// Tiles are of three kinds: interior (every pull source inside the lattice,
// no boundary logic), near a wall (TMA data, bounce-back logic), and tiles
// whose halo wraps across a periodic boundary (direct global loads).
//
// Precision: populations are held as deviations from a per-node reference
// built from the rest equilibrium at rho0,
//   f_rest = P^-1 (h1 h2 rho0, 0, 0, h2/h1 rho0 cs2, h1/h2 rho0 cs2, 0, 0, 0, rho0 cs2^2),
// and the geometric force of that rest state F_rest = -(h2 theta11, h1 theta22) rho0 cs2
// (Eq. Special1_Force_terms at U = 0): pre-collision populations relative to
// f_ref- = f_rest - F_rest/4 (e_a . unit) on links 1..4, post-collision ones
// relative to f_ref+ = f_rest + F_rest/4 (e_a . unit).  With these references
// the O(cs2 theta) rest-state streaming and force cancel analytically instead
// of in FP32 rounding.  The collision is written as
// f~ = f + P^-1 F(-U) B^-1 [Lambda (n^eq - n) + (I - Lambda/2) Psi], with
// n^eq - n expanded so that every term is small.  This is the same update as
// the paper's Eq. GOC-LBEcentralmoment, reorganised for FP32.
#pragma once

#include <cstddef>

#include "goc_device.cuh"

namespace goc {

#ifndef GOC_TILE_ROWS
#define GOC_TILE_ROWS 8        // tile height (rows); the tile width is one warp
#endif
#ifndef GOC_MIN_BLOCKS
#define GOC_MIN_BLOCKS 3       // resident blocks per SM asked of the register allocator (measured best)
#endif
constexpr int TX = 32, TY = GOC_TILE_ROWS, NT = TX * TY;
constexpr int MH = 2;                        // halo of the field arrays (one-sided stencils)
constexpr int HYS = 3;                       // halo rows of the staged tile (fields halo + pull)
template <class S> struct Tiling {
    static constexpr int HXS = 16 / (int)sizeof(S);     // TMA x origin must be 16-byte aligned
    static constexpr int BX = TX + 2 * HXS;
    static constexpr int BY = TY + 2 * HYS;
    static constexpr int BYG = TY + 2;                    // MIE populations: halo of one row
    static constexpr int align128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int F_BYTES = 9 * BY * BX * (int)sizeof(S);
    static constexpr int FF_BYTES = 2 * BY * BX * (int)sizeof(S);
    static constexpr int G_BYTES = 10 * BYG * BX * (int)sizeof(S);
    static constexpr int OFF_FF = align128(F_BYTES);
    static constexpr int OFF_G = OFF_FF + align128(FF_BYTES);
    static constexpr int STAGE_NSE = OFF_G;
    static constexpr int STAGE_MHD = OFF_G + align128(G_BYTES);
};

// ---- TMA / mbarrier primitives (inline PTX) ----------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.u32 %0, 1, 0, P;\n}" : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after 2^24 polls (each try_wait suspends for a
// while), records status 2 and reports failure so the block can return.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *flag) {
    for (uint32_t it = 0; it < (1u << 24); it++)
        if (mbar_try_wait(bar, parity)) return true;
    if (flag) atomicExch(flag, 2);
    return false;
}

// ---- where the stored values of a tile are read from --------------------------
template <class S> struct SrcGlobal {      // direct (read-only path) global loads
    const S *f, *F, *g;
    long long plane;
    int pitch;
    float sf, sF, sg;
    __device__ __forceinline__ float fv(int a, int i, int j) const {
        return scl<S>(Store<S>::ld(f + a * plane + (long long)j * pitch + i), sf);
    }
    __device__ __forceinline__ float Fv(int c, int i, int j) const {
        return scl<S>(Store<S>::ld(F + c * plane + (long long)j * pitch + i), sF);
    }
    __device__ __forceinline__ float gv(int k, int i, int j) const {
        return scl<S>(Store<S>::ld(g + k * plane + (long long)j * pitch + i), sg);
    }
};
template <class S> struct SrcSmem {        // the TMA-staged tile
    using T = Tiling<S>;
    const S *f, *F, *g;
    int ox, oy, oyg;                        // lattice coordinates of staged element (0, 0)
    float sf, sF, sg;
    __device__ __forceinline__ float fv(int a, int i, int j) const {
        return scl<S>(Store<S>::lds(f + (a * T::BY + (j - oy)) * T::BX + (i - ox)), sf);
    }
    __device__ __forceinline__ float Fv(int c, int i, int j) const {
        return scl<S>(Store<S>::lds(F + (c * T::BY + (j - oy)) * T::BX + (i - ox)), sF);
    }
    __device__ __forceinline__ float gv(int k, int i, int j) const {
        return scl<S>(Store<S>::lds(g + (k * T::BYG + (j - oyg)) * T::BX + (i - ox)), sg);
    }
};

// Pull the nine deviations arriving at node (i, j): the value stored at the
// source is relative to the source's f_ref+, the result relative to this
// node's f_ref-, so links 1..4 add f_ref+(source) - f_ref-(node) (the rm/rp
// tables; links 0 and 5..8 have the same reference everywhere).  A link whose
// source lies outside a wall axis is a half-way bounce-back of the node's own
// outgoing population, plus the moving-wall term f_a^eq(w) - f_abar^eq(w)
// (Eq. 101) = e1 rho_w cs2 u / (2 h2_w) across a S/N wall and
// e2 rho_w cs2 u / (2 h1_w) across a W/E wall (rho_w: this node's density at
// the time of the outgoing population).  CHECKS = false: every source is
// inside the lattice (interior tile).
template <bool CHECKS, class Src>
__device__ __forceinline__ void pull_node(const StepParams &p, const Src &src, int i, int j, float h1, float h2,
                                          float d[9]) {
    if (p.nopull) {
#pragma unroll
        for (int a = 0; a < 9; a++) d[a] = src.fv(a, i, j);
        return;
    }
    float rhow = 0.f;
    bool rhow_ready = false;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        int si = i - e1(a), sj = j - e2(a);
        bool ox = false, oy = false;
        if (CHECKS) {
            if (si < 0 || si >= p.nx) {
                if (p.per_x) si = wrapi(si, p.nx); else ox = true;
            }
            if (sj < 0 || sj >= p.ny) {
                if (p.per_y) sj = wrapi(sj, p.ny); else oy = true;
            }
        }
        float v;
        if (!ox && !oy) {
            v = src.fv(a, si, sj);
            if (a == 1) v += h2 * p.ax1.rm[i];
            if (a == 3) v += h2 * p.ax1.rp[i];
            if (a == 2) v += h1 * p.ax2.rm[j];
            if (a == 4) v += h1 * p.ax2.rp[j];
        } else {
            v = src.fv(opp(a), i, j);
            if (p.moving && (e1(a) != 0 && e2(a) != 0)) {
                int sy = e2(a) > 0 ? SIDE_S : SIDE_N;
                int sx = e1(a) > 0 ? SIDE_W : SIDE_E;
                float uy = oy ? p.uw[sy] : 0.f, ux = ox ? p.uw[sx] : 0.f;
                if (uy != 0.f || ux != 0.f) {
                    if (!rhow_ready) {
                        float s = 0.f;
#pragma unroll
                        for (int b = 0; b < 9; b++) s += src.fv(b, i, j);
                        rhow = p.rho0 + s / (h1 * h2);
                        rhow_ready = true;
                    }
                    if (uy != 0.f) v += e1(a) * rhow * p.cs2 * uy / (2.f * p.hwn[sy]);
                    if (ux != 0.f) v += e2(a) * rhow * p.cs2 * ux / (2.f * p.hwn[sx]);
                }
            }
        }
        d[a] = v;
    }
}

// Pull the MIE deviations of component c.  Storage references (the MIE
// analogue of f_ref-/+): pre-collision g_ref- = W H B_rest - e.M/2,
// post-collision g_ref+ = W H B_rest + e.M/2, with the rest-state first moments
// M = (csm2/2) B_rest (h1 H theta11, H h2 theta22) that the local gradient
// formula (Eqs. gradB1/gradB2) implies for a uniform field.  A link from
// inside adds g_ref+(source) - g_ref-(node) (dm/dp tables).  Outside a wall:
// anti-bounce-back g_a = -g~_abar + 2 W_a h_wall B_wall,c (Appendix G,
// boundary conditions), h_wall = h1,wall h2,wall, which in these variables is
// -s_abar + 2 W_a (h_wall B_wall - H B_rest) + e_a.M.
template <bool CHECKS, class Src>
__device__ __forceinline__ void pull_mie(const StepParams &p, const Src &src, int i, int j, float h1, float h2,
                                         int c, float d[5]) {
    const float H = h1 * h2;
    if (p.nopull) {
#pragma unroll
        for (int a = 0; a < 5; a++) d[a] = src.gv(c * 5 + a, i, j);
        return;
    }
    const float br = p.brest[c];
#pragma unroll
    for (int a = 0; a < 5; a++) {
        int si = i - g1(a), sj = j - g2(a);
        bool ox = false, oy = false;
        if (CHECKS) {
            if (si < 0 || si >= p.nx) {
                if (p.per_x) si = wrapi(si, p.nx); else ox = true;
            }
            if (sj < 0 || sj >= p.ny) {
                if (p.per_y) sj = wrapi(sj, p.ny); else oy = true;
            }
        }
        float v;
        if (!ox && !oy) {
            v = src.gv(c * 5 + a, si, sj);
            if (a == 1) v += br * h2 * p.ax1.dm[i];
            if (a == 3) v += br * h2 * p.ax1.dp[i];
            if (a == 2) v += br * h1 * p.ax2.dm[j];
            if (a == 4) v += br * h1 * p.ax2.dp[j];
        } else {
            int side = oy ? (g2(a) > 0 ? SIDE_S : SIDE_N) : (g1(a) > 0 ? SIDE_W : SIDE_E);
            float hw = oy ? h1 * p.hwn[side] : p.hwn[side] * h2;
            float eM = oy ? g2(a) * 0.5f * p.csm2 * H * h2 * p.ax2.th[j] * br
                          : g1(a) * 0.5f * p.csm2 * h1 * H * p.ax1.th[i] * br;
            v = -src.gv(c * 5 + gopp(a), i, j) + 2.f * p.W1 * (hw * p.bw[side][c] - H * br) + eM;
        }
        d[a] = v;
    }
}

// rho and U (Eq. GOChydrodynamicfields) from pre-collision deviations d and the
// previous step's F - F_rest: the -F_rest/2 momentum of f_ref- and the +F_rest/2
// of the force shift cancel, leaving U1 = (sum d e1 + (F1 - F1_rest)/2)/(rho h2).
__device__ __forceinline__ void fields_from(const StepParams &p, const float d[9], float F1p, float F2p,
                                            float ih1, float ih2, float &drho, float &U1, float &U2) {
    float k00 = 0.f;
#pragma unroll
    for (int a = 0; a < 9; a++) k00 += d[a];
    const float k10 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    const float k01 = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    drho = k00 * (ih1 * ih2);
    const float irho = __frcp_rn(p.rho0 + drho);
    U1 = (k10 + 0.5f * F1p) * irho * ih2;
    U2 = (k01 + 0.5f * F2p) * irho * ih1;
}

// Second-order derivative along an axis from values at offsets -2..2: central,
// or one-sided at the first and last node of a wall axis.
__device__ __forceinline__ float dfd(float vm2, float vm1, float v0, float vp1, float vp2, int k, int n,
                                     int per) {
    if (per || (k > 0 && k < n - 1)) return 0.5f * (vp1 - vm1);
    if (k == 0) return 0.5f * (-3.f * v0 + 4.f * vp1 - vp2);
    return 0.5f * (3.f * v0 - 4.f * vm1 + vm2);
}

struct FieldSmem {
    float rho[TY + 2 * MH][TX + 2 * MH], u1[TY + 2 * MH][TX + 2 * MH], u2[TY + 2 * MH][TX + 2 * MH];
};

// Phase 2 for node (i, j) = (i0 + tx, j0 + ty).
template <class S, bool MHD, bool CHECKS, class Src>
__device__ __forceinline__ void node_update(const StepParams &p, const Src &src, int i, int j, int tx, int ty,
                                            const FieldSmem &sm, const float (&d)[9], float F1p, float F2p,
                                            float h1, float h2, float ih1, float ih2) {
    const int ex = tx + MH, ey = ty + MH;
    const float t11 = p.ax1.th[i], t22 = p.ax2.th[j];
    const float H = h1 * h2, iH = ih1 * ih2;
    const float drho = sm.rho[ey][ex], U1 = sm.u1[ey][ex], U2 = sm.u2[ey][ex];
    const float rho = p.rho0 + drho;

    // normal derivatives (second-order finite differences)
    float dU1, dr1, dU2, dr2;
    if (CHECKS) {
        dU1 = dfd(sm.u1[ey][ex - 2], sm.u1[ey][ex - 1], U1, sm.u1[ey][ex + 1], sm.u1[ey][ex + 2], i, p.nx, p.per_x);
        dr1 = dfd(sm.rho[ey][ex - 2], sm.rho[ey][ex - 1], drho, sm.rho[ey][ex + 1], sm.rho[ey][ex + 2], i, p.nx, p.per_x);
        dU2 = dfd(sm.u2[ey - 2][ex], sm.u2[ey - 1][ex], U2, sm.u2[ey + 1][ex], sm.u2[ey + 2][ex], j, p.ny, p.per_y);
        dr2 = dfd(sm.rho[ey - 2][ex], sm.rho[ey - 1][ex], drho, sm.rho[ey + 1][ex], sm.rho[ey + 2][ex], j, p.ny, p.per_y);
    } else {
        dU1 = 0.5f * (sm.u1[ey][ex + 1] - sm.u1[ey][ex - 1]);
        dr1 = 0.5f * (sm.rho[ey][ex + 1] - sm.rho[ey][ex - 1]);
        dU2 = 0.5f * (sm.u2[ey + 1][ex] - sm.u2[ey - 1][ex]);
        dr2 = 0.5f * (sm.rho[ey + 1][ex] - sm.rho[ey - 1][ex]);
    }

    const long long idx = (long long)j * p.pitch + i;
    float FL1 = 0.f, FL2 = 0.f, B1 = 0.f, B2 = 0.f;

    // ---- MIE (Appendix G): local dB, J3, Lorentz force, SRT collision -------
    if constexpr (MHD) {
        S *gout = static_cast<S *>(p.gout);
        float gd[2][5], Bc[2], dBc[2], dB1[2], dB2[2], A1[2], A2[2];
#pragma unroll
        for (int c = 0; c < 2; c++) {
            pull_mie<CHECKS>(p, src, i, j, h1, h2, c, gd[c]);
            float s = gd[c][0] + gd[c][1] + gd[c][2] + gd[c][3] + gd[c][4];
            dBc[c] = s * iH;                    // h1 h2 B = sum g (Eq. 13_C, Y = 0); sum g_ref- = H B_rest
            Bc[c] = p.brest[c] + dBc[c];
        }
        B1 = Bc[0];
        B2 = Bc[1];
        const float U[2] = {U1, U2};
#pragma unroll
        for (int c = 0; c < 2; c++) {
            A1[c] = U1 * Bc[c] - Bc[0] * U[c];   // A_c1 (Eq. 2_C)
            A2[c] = U2 * Bc[c] - Bc[1] * U[c];   // A_c2
            // Eqs. gradB1/gradB2 with Lambda^(1) = sum e (g - g^eq(0)) (Eqs.
            // firstvelmomenttensor1/2); the rest-state moment M of g_ref- cancels
            // against the B_rest part of the curvature term.
            const float L1 = (gd[c][1] - gd[c][3]) - h2 * A1[c] + 0.5f * p.csm2 * h1 * H * t11 * dBc[c];
            const float L2 = (gd[c][2] - gd[c][4]) - h1 * A2[c] + 0.5f * p.csm2 * H * h2 * t22 * dBc[c];
            dB1[c] = -L1 * __frcp_rn(p.csm2 * (0.5f * H + (p.taum - 0.5f) * h2 * ih1));
            dB2[c] = -L2 * __frcp_rn(p.csm2 * (0.5f * H + (p.taum - 0.5f) * h1 * ih2));
        }
        // current density (Eq. currentdensity-GOC) and Lorentz force (Eq. Lorentzforce-GOC)
        const float J3 = p.imum * iH * (h2 * dB1[1] - h1 * dB2[0]);
        FL1 = -J3 * B2;
        FL2 = J3 * B1;
        // SRT collision (Eq. 12_C, S = 0 on straight grids) with g^eq of
        // Eq. EDF-MIE-base plus the correction of Eq. 42_C.  Relative to the
        // references: s = d - (d - G)/tau_m, G = g^eq - g_ref- without the
        // B_rest curvature part, which cancels with the change g_ref- -> g_ref+.
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const float lc1 = p.eta * (H - h2 * ih1) * dB1[c] + p.eta * h1 * H * t11 * dBc[c];
            const float lc2 = p.eta * (H - h1 * ih2) * dB2[c] + p.eta * H * h2 * t22 * dBc[c];
            const float x1 = (h2 * A1[c] + lc1) * p.icsm2;
            const float x2 = (h1 * A2[c] + lc2) * p.icsm2;
#pragma unroll
            for (int a = 0; a < 5; a++) {
                const float W = a == 0 ? p.W0 : p.W1;
                const float G = W * (H * dBc[c] + g1(a) * x1 + g2(a) * x2);
                const float gt = gd[c][a] - (gd[c][a] - G) * p.itaum;
                Store<S>::st(gout + (c * 5 + a) * p.plane + idx, scl<S>(gt, p.isg));
            }
        }
    }

    // ---- stresses and effective force (straight grid, Appendix B (i)) -------
    const float zeta = p.zeta, nu = p.nu, cs2 = p.cs2;
    const float tau11 = rho * ((zeta + nu) * ih1 * dU1 + (zeta - nu) * ih2 * dU2);
    const float tau22 = rho * ((zeta + nu) * ih2 * dU2 + (zeta - nu) * ih1 * dU1);
    // F = F_rest + F_dev, F_rest = -(h2, h1) rho0 cs2 (theta11, theta22) is the
    // geometric force of the rest state; only F_dev is stored.
    const float F1dev = h2 * (p.fext1 + FL1 - drho * cs2 * t11 + (tau11 - rho * U1 * U1) * t11);
    const float F2dev = h1 * (p.fext2 + FL2 - drho * cs2 * t22 + (tau22 - rho * U2 * U2) * t22);
    const float F1r = -h2 * p.rho0 * cs2 * t11, F2r = -h1 * p.rho0 * cs2 * t22;
    const float F1 = F1dev + F1r;
    const float F2 = F2dev + F2r;

    // ---- correction coefficients (Eqs. 83, 85; theta12 = theta21 = 0) ------
    const float r = h2 * ih1, s = h1 * ih2;               // h2/h1, h1/h2
    const float ics2 = p.ics2;
    const float a1 = p.gi * U1 * U1 * ics2, a2 = p.gi * U2 * U2 * ics2;
    const float r1 = r * ih1, s2 = s * ih2;               // h2/h1^2, h1/h2^2
    const float D31 = rho * (2.f * zeta - (zeta + nu) * r1 - (zeta - nu) * ih2
                             - zeta * (2.f - h2 * ics2 + (3.f * a1 + 1.f) * r1));
    const float D32 = rho * (2.f * zeta - (zeta + nu) * s2 - (zeta - nu) * ih1
                             - zeta * (2.f - h1 * ics2 + (3.f * a2 + 1.f) * s2));
    const float D33 = -zeta * ((3.f - a1) * r1 - h2 * ics2 - a2 * ih2) * U1;
    const float D34 = -zeta * ((3.f - a2) * s2 - h1 * ics2 - a1 * ih1) * U2;
    const float C3 = rho * zeta * (2.f * U1 * (a1 + 1.f) * r * t11 + 2.f * U2 * (a2 + 1.f) * s * t22);
    const float D41 = rho * (2.f * nu - (zeta + nu) * r1 + (zeta - nu) * ih2
                             - nu * (2.f - h2 * ics2 + (3.f * a1 + 1.f) * r1));
    const float D42 = rho * (-2.f * nu + (zeta + nu) * s2 - (zeta - nu) * ih1
                             - nu * (-2.f + h1 * ics2 - (3.f * a2 + 1.f) * s2));
    const float D43 = -nu * ((3.f - a1) * r1 - h2 * ics2 + a2 * ih2) * U1;
    const float D44 = -nu * (-(3.f - a2) * s2 + h1 * ics2 - a1 * ih1) * U2;
    const float C4 = rho * nu * (2.f * U1 * (a1 + 1.f) * r * t11 - 2.f * U2 * (a2 + 1.f) * s * t22);
    const float n3 = D31 * dU1 + D32 * dU2 + D33 * dr1 + D34 * dr2 + C3;
    const float n4 = D41 * dU1 + D42 * dU2 + D43 * dr1 + D44 * dr2 + C4;

    // ---- central moments of the deviations: c = F(U) P d -------------------
    const float k00 = d[0] + d[1] + d[2] + d[3] + d[4] + d[5] + d[6] + d[7] + d[8];
    const float k10 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    const float k01 = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    const float k20 = d[1] + d[3] + d[5] + d[6] + d[7] + d[8];
    const float k02 = d[2] + d[4] + d[5] + d[6] + d[7] + d[8];
    const float k11 = d[5] - d[6] + d[7] - d[8];
    const float k21 = d[5] + d[6] - d[7] - d[8];
    const float k12 = d[5] - d[6] - d[7] + d[8];
    const float k22 = d[5] + d[6] + d[7] + d[8];
    const float u = U1, v = U2, uu = u * u, vv = v * v, uv = u * v;
    // first raw moments of f - f_rest (f_ref- carries -F_rest/2 of momentum)
    const float K10 = k10 - 0.5f * F1r, K01 = k01 - 0.5f * F2r;
    const float c20 = k20 - 2.f * u * K10 + uu * k00;
    const float c02 = k02 - 2.f * v * K01 + vv * k00;
    const float c11 = k11 - v * K10 - u * K01 + uv * k00;
    const float c21 = k21 - 2.f * u * k11 + uu * K01 - v * k20 + 2.f * uv * K10 - uu * v * k00;
    const float c12 = k12 - 2.f * v * k11 + vv * K10 - u * k02 + 2.f * uv * K01 - u * vv * k00;
    const float c22 = k22 - 2.f * u * k12 + uu * k02 - 2.f * v * k21 + 4.f * uv * k11
                      - 2.f * uu * v * K01 + vv * k20 - 2.f * u * vv * K10 + uu * vv * k00;

    // ---- n^eq - n in the combined basis (rest parts cancelled) ---------------
    const float a0 = H * p.rho0, b0 = r * p.rho0 * cs2, c0 = s * p.rho0 * cs2;
    const float hm1 = h1 - 1.f, hm2 = h2 - 1.f;
    const float q20 = r * hm1 * hm1, q02 = s * hm2 * hm2, q11 = hm1 * hm2;
    const float q21 = -hm2 * hm1 * hm1 * ih1, q12 = -hm1 * hm2 * hm2 * ih2;
    const float e2s = (r + s) * cs2 * drho + q20 * rho * uu + q02 * rho * vv + n3 - (c20 + c02) - (uu + vv) * a0;
    const float e2d = (r - s) * cs2 * drho + q20 * rho * uu - q02 * rho * vv + n4 - (c20 - c02) - (uu - vv) * a0;
    const float e11 = q11 * rho * uv - c11 - uv * a0;
    const float e21 = q21 * rho * uu * v + (1.f - h2) * rho * cs2 * v * ih1 - c21 + v * b0 + uu * v * a0;
    const float e12 = q12 * rho * u * vv + (1.f - h1) * rho * cs2 * u * ih2 - c12 + u * c0 + u * vv * a0;
    const float e22 = cs2 * cs2 * drho - c22 - vv * b0 - uu * c0 - uu * vv * a0;

    // ---- sources (Eq. cmsourcesGOC) and relaxation ---------------------------
    const float w1 = ih1 - 1.f, w2 = ih2 - 1.f;
    const float s2s = 2.f * (w1 * F1 * u + w2 * F2 * v);
    const float s2d = 2.f * (w1 * F1 * u - w2 * F2 * v);
    const float s11 = w2 * F1 * v + w1 * F2 * u;
    const float *om = p.om;
    // k10^eq - k10 = F^{n-1}/2 exactly (definition of U), likewise k01.
    // D10d excludes F_rest, which the change of reference f_ref- -> f_ref+ absorbs.
    const float D10d = om[1] * 0.5f * F1p + (1.f - 0.5f * om[1]) * F1dev;
    const float D01d = om[2] * 0.5f * F2p + (1.f - 0.5f * om[2]) * F2dev;
    const float D10 = D10d + F1r, D01 = D01d + F2r;
    const float D2s = om[3] * e2s + (1.f - 0.5f * om[3]) * s2s;
    const float D2d = om[4] * e2d + (1.f - 0.5f * om[4]) * s2d;
    const float D20 = 0.5f * (D2s + D2d), D02 = 0.5f * (D2s - D2d);
    const float D11 = om[5] * e11 + (1.f - 0.5f * om[5]) * s11;
    const float D21 = om[6] * e21, D12 = om[7] * e12, D22 = om[8] * e22;

    // ---- back to raw moments with F(-U) (Delta k00 = 0) ----------------------
    const float R20 = D20 + 2.f * u * D10;
    const float R02 = D02 + 2.f * v * D01;
    const float R11 = D11 + v * D10 + u * D01;
    const float R21 = D21 + 2.f * u * D11 + uu * D01 + v * D20 + 2.f * uv * D10;
    const float R12 = D12 + 2.f * v * D11 + vv * D10 + u * D02 + 2.f * uv * D01;
    const float R22 = D22 + 2.f * u * D12 + uu * D02 + 2.f * v * D21 + 4.f * uv * D11
                      + 2.f * uu * v * D01 + vv * D20 + 2.f * u * vv * D10;

    // ---- P^-1 and store ------------------------------------------------------
    float o[9];
    o[0] = d[0] - R20 - R02 + R22;
    o[1] = d[1] + 0.5f * (D10d + R20 - R12 - R22);
    o[2] = d[2] + 0.5f * (D01d + R02 - R21 - R22);
    o[3] = d[3] + 0.5f * (-D10d + R20 + R12 - R22);
    o[4] = d[4] + 0.5f * (-D01d + R02 + R21 - R22);
    o[5] = d[5] + 0.25f * (R11 + R21 + R12 + R22);
    o[6] = d[6] + 0.25f * (-R11 + R21 - R12 + R22);
    o[7] = d[7] + 0.25f * (R11 - R21 - R12 + R22);
    o[8] = d[8] + 0.25f * (-R11 - R21 + R12 + R22);
    S *fout = static_cast<S *>(p.fout);
#pragma unroll
    for (int a = 0; a < 9; a++) Store<S>::st(fout + a * p.plane + idx, scl<S>(o[a], p.isf));
    S *Fout = static_cast<S *>(p.Fout);
    Store<S>::st(Fout + idx, scl<S>(F1dev, p.isF));
    Store<S>::st(Fout + p.plane + idx, scl<S>(F2dev, p.isF));

    if (p.uout) {
        p.uout[idx] = U1;
        p.uout[p.plane + idx] = U2;
        p.uout[2 * p.plane + idx] = B1;
        p.uout[3 * p.plane + idx] = B2;
    }
    if (p.flag) {   // divergence flag: one atomic per warp at most
        const bool bad = !(rho > 0.f && fabsf(U1) + fabsf(U2) < 1e30f);
        const unsigned m = __activemask();
        if (__any_sync(m, bad) && (threadIdx.x & 31) == (__ffs(m) - 1) && *((volatile int *)p.flag) == 0)
            atomicExch(p.flag, 1);
    }
}

// One tile of one lattice from a given source; KIND 0: interior (no boundary
// logic, fields halo 1), 1: near a boundary (fields halo 2 where inside).
// Every thread pulls its own node into registers (kept across the barrier for
// the collision); the ring of halo nodes around the tile is shared out over the
// threads.  Contains a block barrier: every thread of the block must call it.
template <class S, bool MHD, int KIND, class Src>
__device__ __forceinline__ void tile_compute(const StepParams &p, const Src &src, int i0, int j0, FieldSmem &sm) {
    constexpr bool CHECKS = KIND != 0;
    constexpr int W = KIND == 0 ? 1 : MH;                 // halo width of the fields
    constexpr int BAND = W * (TX + 2 * W);                // nodes in the top (or bottom) band
    constexpr int RING = 2 * BAND + 2 * W * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + tx, j = j0 + ty;
    const bool own = i < p.nx && j < p.ny;
    float d[9], F1p = 0.f, F2p = 0.f, h1 = 1.f, h2 = 1.f, ih1 = 1.f, ih2 = 1.f;
    {   // own node
        float drho = 0.f, U1 = 0.f, U2 = 0.f;
        if (own) {
            h1 = p.ax1.h[i];
            h2 = p.ax2.h[j];
            ih1 = p.ax1.ih[i];
            ih2 = p.ax2.ih[j];
            pull_node<CHECKS>(p, src, i, j, h1, h2, d);
            F1p = src.Fv(0, i, j);
            F2p = src.Fv(1, i, j);
            fields_from(p, d, F1p, F2p, ih1, ih2, drho, U1, U2);
        } else if (CHECKS) {   // ragged tile: past the last node of a periodic axis sits the wrapped node
            int ii = i, jj = j;
            bool in = true;
            if (ii >= p.nx) {
                if (p.per_x) ii = wrapi(ii, p.nx); else in = false;
            }
            if (jj >= p.ny) {
                if (p.per_y) jj = wrapi(jj, p.ny); else in = false;
            }
            if (in) {
                float dd[9];
                pull_node<CHECKS>(p, src, ii, jj, p.ax1.h[ii], p.ax2.h[jj], dd);
                fields_from(p, dd, src.Fv(0, ii, jj), src.Fv(1, ii, jj), p.ax1.ih[ii], p.ax2.ih[jj], drho, U1, U2);
            }
        }
        sm.rho[ty + MH][tx + MH] = drho;
        sm.u1[ty + MH][tx + MH] = U1;
        sm.u2[ty + MH][tx + MH] = U2;
    }
    // halo ring: top band, bottom band, left band, right band
    for (int r = tid; r < RING; r += NT) {
        int x, y;
        if (r < 2 * BAND) {
            const int b = r < BAND ? r : r - BAND;
            const int row = b / (TX + 2 * W);
            x = b - row * (TX + 2 * W) - W;
            y = r < BAND ? row - W : TY + row;
        } else {
            const int b = r - 2 * BAND;
            const int side = b / (W * TY), bb = b - side * (W * TY);
            const int col = bb / TY;
            y = bb - col * TY;
            x = side == 0 ? col - W : TX + col;
        }
        int ii = i0 + x, jj = j0 + y;
        bool in = true;
        if (CHECKS) {
            if (ii < 0 || ii >= p.nx) {
                if (p.per_x) ii = wrapi(ii, p.nx); else in = false;
            }
            if (jj < 0 || jj >= p.ny) {
                if (p.per_y) jj = wrapi(jj, p.ny); else in = false;
            }
        }
        float drho = 0.f, U1 = 0.f, U2 = 0.f;
        if (in) {
            float dd[9];
            pull_node<CHECKS>(p, src, ii, jj, p.ax1.h[ii], p.ax2.h[jj], dd);
            fields_from(p, dd, src.Fv(0, ii, jj), src.Fv(1, ii, jj), p.ax1.ih[ii], p.ax2.ih[jj], drho, U1, U2);
        }
        sm.rho[y + MH][x + MH] = drho;
        sm.u1[y + MH][x + MH] = U1;
        sm.u2[y + MH][x + MH] = U2;
    }
    __syncthreads();
    if (own) node_update<S, MHD, CHECKS>(p, src, i, j, tx, ty, sm, d, F1p, F2p, h1, h2, ih1, ih2);
}

// Kind of a tile: 0 interior (all pull sources of the tile and its fields
// halo inside the lattice), 1 near a wall (staged data suffices), 2 its halo
// wraps across a periodic boundary (direct global loads).
template <class S>
__device__ __forceinline__ int tile_kind(const StepParams &p, int i0, int j0) {
    using T = Tiling<S>;
    if (!p.use_tma) return 2;
    const bool wx = p.per_x && (i0 - T::HXS < 0 || i0 + TX + T::HXS > p.nx);
    const bool wy = p.per_y && (j0 - HYS < 0 || j0 + TY + HYS > p.ny);
    if (wx || wy) return 2;
    if (i0 >= 2 && i0 + TX + 2 <= p.nx && j0 >= 2 && j0 + TY + 2 <= p.ny) return 0;
    return 1;
}

template <class S>
__device__ __forceinline__ void issue_tile(const StepParams &p, int i0, int j0, unsigned char *stage, uint64_t *bar,
                                           bool mhd) {
    using T = Tiling<S>;
    const uint32_t bytes = T::F_BYTES + T::FF_BYTES + (mhd ? T::G_BYTES : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_3d(stage, &p.tm_f, i0 - T::HXS, j0 - HYS, 0, bar);
    tma_load_3d(stage + T::OFF_FF, &p.tm_F, i0 - T::HXS, j0 - HYS, 0, bar);
    if (mhd) tma_load_3d(stage + T::OFF_G, &p.tm_g, i0 - T::HXS, j0 - 1, 0, bar);
}

template <class S, bool MHD>
__device__ __forceinline__ void run_tile(const StepParams &p, int kind, int i0, int j0, const unsigned char *stage,
                                         FieldSmem &sm) {
    using T = Tiling<S>;
    if (kind == 2) {
        SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin), static_cast<const S *>(p.gin),
                         p.plane, p.pitch, p.sf, p.sF, p.sg};
        tile_compute<S, MHD, 1>(p, src, i0, j0, sm);
    } else {
        SrcSmem<S> src{reinterpret_cast<const S *>(stage), reinterpret_cast<const S *>(stage + T::OFF_FF),
                       reinterpret_cast<const S *>(stage + T::OFF_G), i0 - T::HXS, j0 - HYS, j0 - 1,
                       p.sf, p.sF, p.sg};
        if (kind == 0) tile_compute<S, MHD, 0>(p, src, i0, j0, sm);
        else tile_compute<S, MHD, 1>(p, src, i0, j0, sm);
    }
}

// Single lattice: persistent blocks stride over the tiles; TMA staging in two
// dynamic shared-memory stages.
template <class S, bool MHD>
__global__ void __launch_bounds__(NT, GOC_MIN_BLOCKS) step_kernel(const __grid_constant__ StepParams p) {
    using T = Tiling<S>;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ FieldSmem sm;
    constexpr int STAGE = MHD ? T::STAGE_MHD : T::STAGE_NSE;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY, ntiles = ntx * nty;
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    if (leader) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int t = blockIdx.x;
    if (leader && t < ntiles) {
        const int i0 = (t % ntx) * TX, j0 = (t / ntx) * TY;
        if (tile_kind<S>(p, i0, j0) != 2) issue_tile<S>(p, i0, j0, dyn, &bars[0], MHD);
    }
    uint32_t ph0 = 0, ph1 = 0;
    int stage = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (leader && tn < ntiles) {
            const int i0n = (tn % ntx) * TX, j0n = (tn / ntx) * TY;
            if (tile_kind<S>(p, i0n, j0n) != 2) {
                fence_proxy_async();   // generic reads of that stage (previous tile) precede the async writes
                issue_tile<S>(p, i0n, j0n, dyn + (stage ^ 1) * STAGE, &bars[stage ^ 1], MHD);
            }
        }
        const int i0 = (t % ntx) * TX, j0 = (t / ntx) * TY;
        const int kind = tile_kind<S>(p, i0, j0);
        if (kind != 2) {
            uint32_t &ph = stage ? ph1 : ph0;
            const bool ok = mbar_wait_bounded(&bars[stage], ph, p.flag);
            if (!__syncthreads_and(ok)) return;   // the whole block leaves together on a timeout
            ph ^= 1;
        }
        run_tile<S, MHD>(p, kind, i0, j0, dyn + stage * STAGE, sm);
        __syncthreads();   // the stage and the field arrays are reused by the next tile
        stage ^= 1;
    }
}

// Many lattices in one launch: work item t in [0, total) is a tile of the
// lattice k with tile_off[k] <= t < tile_off[k+1]; a persistent grid strides
// over the items.  Lattices with and without the MIE may be mixed (the stage
// is sized for the MIE when any member has it).
__device__ __forceinline__ int find_lattice(const int *tile_off, int nlat, int t) {
    int lo = 0, hi = nlat - 1;   // last k with tile_off[k] <= t
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class S, bool MHD>
__global__ void __launch_bounds__(NT, GOC_MIN_BLOCKS) batch_step_kernel(const StepParams *__restrict__ params,
                                                                        const int *__restrict__ tile_off, int nlat) {
    using T = Tiling<S>;
    constexpr int STAGE = MHD ? T::STAGE_MHD : T::STAGE_NSE;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ FieldSmem sm;
    __shared__ int s_item[2][3];   // per stage: lattice, i0, j0 of the staged item
    __shared__ __align__(16) unsigned char s_par[(offsetof(StepParams, tm_f) + 15) / 16 * 16];
    __shared__ int s_k;            // lattice whose parameters are in s_par
    const int total = tile_off[nlat];
    // contiguous range of work items per block: neighbouring tiles of one lattice
    const int per = (total + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per, t_end = min(total, t_begin + per);
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (leader) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_k = -1;
    }
    auto prefetch = [&](int t, int st) {
        const int k = find_lattice(tile_off, nlat, t);
        const StepParams &q = params[k];
        const int local = t - tile_off[k];
        const int ntx = (q.nx + TX - 1) / TX;
        const int i0 = (local % ntx) * TX, j0 = (local / ntx) * TY;
        s_item[st][0] = k;
        s_item[st][1] = i0;
        s_item[st][2] = j0;
        if (tile_kind<S>(q, i0, j0) != 2) {
            fence_proxy_async();
            issue_tile<S>(q, i0, j0, dyn + st * STAGE, &bars[st], MHD);
        }
    };
    if (leader && t_begin < t_end) prefetch(t_begin, 0);
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    int stage = 0;
    for (int t = t_begin; t < t_end; t++) {
        if (leader && t + 1 < t_end) prefetch(t + 1, stage ^ 1);
        const int k = s_item[stage][0], i0 = s_item[stage][1], j0 = s_item[stage][2];
        if (k != s_k) {   // parameters (up to the TMA descriptors) of a new lattice into shared memory
            const uint4 *src = reinterpret_cast<const uint4 *>(&params[k]);
            uint4 *dst = reinterpret_cast<uint4 *>(s_par);
            for (int w = tid; w < (int)(sizeof(s_par) / 16); w += NT) dst[w] = src[w];
            __syncthreads();
            if (leader) s_k = k;
        }
        const StepParams &p = *reinterpret_cast<const StepParams *>(s_par);
        const int kind = tile_kind<S>(p, i0, j0);
        if (kind != 2) {
            uint32_t &ph = stage ? ph1 : ph0;
            const bool ok = mbar_wait_bounded(&bars[stage], ph, p.flag);
            if (!__syncthreads_and(ok)) return;   // the whole block leaves together on a timeout
            ph ^= 1;
        }
        run_tile<S, MHD>(p, kind, i0, j0, dyn + stage * STAGE, sm);
        __syncthreads();   // stage, field arrays and s_item are reused
        stage ^= 1;
    }
}

}  // namespace goc
