// goc_step.cuh -- the fused GOC-LBM time step (one launch per time step).
//
// One thread block owns a TX x TY tile of nodes.  Phase 1 pulls the stored
// post-collision populations of the tile plus a halo of two nodes in each
// direction (pull streaming with boundary conditions, Appendix E Step 6,
// Eq. 101/103), forms the hydrodynamic fields (Appendix E Step 7, with the
// stored force of the previous step) and keeps them in shared memory.
// Phase 2 takes, per node, the second-order normal derivatives from shared
// memory, the MIE part (Appendix G Steps 1-3, all local), the stresses and the
// effective force (Eq. Special1_Force_terms with the Lorentz force of Eq.
// Lorentzforce-GOC in F_ext), the central-moment collision (Appendix E Steps
// 1-5), and stores the post-collision populations and the force.
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

#include "goc_device.cuh"

namespace goc {

constexpr int TX = 32, TY = 8, HX = 2, HY = 2;
constexpr int EW = TX + 2 * HX, EH = TY + 2 * HY, EXT = EW * EH, NT = TX * TY;

// Pull the nine deviations arriving at node (i, j): the value stored at the
// source is relative to the source's f_ref+, the result relative to this
// node's f_ref-, so links 1..4 add f_ref+(source) - f_ref-(node) (the rm/rp
// tables; links 0 and 5..8 have the same reference everywhere).  A link whose source lies outside a wall axis is a half-way
// bounce-back of the node's own outgoing population, plus the moving-wall
// term f_a^eq(w) - f_abar^eq(w) (Eq. 101) = e1 rho_w cs2 u / (2 h2_w) across a
// S/N wall and e2 rho_w cs2 u / (2 h1_w) across a W/E wall.
template <class S>
__device__ __forceinline__ void pull_node(const StepParams &p, int i, int j, float h1, float h2,
                                          float d[9]) {
    const S *fin = static_cast<const S *>(p.fin);
    const long long own = (long long)j * p.pitch + i;
    if (p.nopull) {
#pragma unroll
        for (int a = 0; a < 9; a++) d[a] = Store<S>::ld(fin + a * p.plane + own) * p.sf;
        return;
    }
    float rhow = 0.f;
    bool rhow_ready = false;
#pragma unroll
    for (int a = 0; a < 9; a++) {
        int si = i - e1(a), sj = j - e2(a);
        bool ox = false, oy = false;
        if (si < 0 || si >= p.nx) {
            if (p.per_x) si = wrapi(si, p.nx); else ox = true;
        }
        if (sj < 0 || sj >= p.ny) {
            if (p.per_y) sj = wrapi(sj, p.ny); else oy = true;
        }
        float v;
        if (!ox && !oy) {
            v = Store<S>::ld(fin + a * p.plane + (long long)sj * p.pitch + si) * p.sf;
            if (a == 1) v += h2 * p.ax1.rm[i];
            if (a == 3) v += h2 * p.ax1.rp[i];
            if (a == 2) v += h1 * p.ax2.rm[j];
            if (a == 4) v += h1 * p.ax2.rp[j];
        } else {
            v = Store<S>::ld(fin + opp(a) * p.plane + own) * p.sf;
            if (p.moving && (e1(a) != 0 && e2(a) != 0)) {
                int sy = e2(a) > 0 ? SIDE_S : SIDE_N;
                int sx = e1(a) > 0 ? SIDE_W : SIDE_E;
                float uy = oy ? p.uw[sy] : 0.f, ux = ox ? p.uw[sx] : 0.f;
                if (uy != 0.f || ux != 0.f) {
                    if (!rhow_ready) {   // rho of this node at the time of the outgoing population
                        float s = 0.f;
#pragma unroll
                        for (int b = 0; b < 9; b++) s += Store<S>::ld(fin + b * p.plane + own);
                        rhow = p.rho0 + s * p.sf / (h1 * h2);
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
template <class S>
__device__ __forceinline__ void pull_mie(const StepParams &p, int i, int j, float h1, float h2,
                                         int c, float d[5]) {
    const S *gin = static_cast<const S *>(p.gin);
    const long long own = (long long)j * p.pitch + i;
    const float H = h1 * h2;
    if (p.nopull) {
#pragma unroll
        for (int a = 0; a < 5; a++) d[a] = Store<S>::ld(gin + (c * 5 + a) * p.plane + own) * p.sg;
        return;
    }
    const float br = p.brest[c];
#pragma unroll
    for (int a = 0; a < 5; a++) {
        int si = i - g1(a), sj = j - g2(a);
        bool ox = false, oy = false;
        if (si < 0 || si >= p.nx) {
            if (p.per_x) si = wrapi(si, p.nx); else ox = true;
        }
        if (sj < 0 || sj >= p.ny) {
            if (p.per_y) sj = wrapi(sj, p.ny); else oy = true;
        }
        float v;
        if (!ox && !oy) {
            v = Store<S>::ld(gin + (c * 5 + a) * p.plane + (long long)sj * p.pitch + si) * p.sg;
            if (a == 1) v += br * h2 * p.ax1.dm[i];
            if (a == 3) v += br * h2 * p.ax1.dp[i];
            if (a == 2) v += br * h1 * p.ax2.dm[j];
            if (a == 4) v += br * h1 * p.ax2.dp[j];
        } else {
            int side = oy ? (g2(a) > 0 ? SIDE_S : SIDE_N) : (g1(a) > 0 ? SIDE_W : SIDE_E);
            float hw = oy ? h1 * p.hwn[side] : p.hwn[side] * h2;
            // e_a . M at this node (only the wall-normal component is non-zero here)
            float eM = oy ? g2(a) * 0.5f * p.csm2 * H * h2 * p.ax2.th[j] * br
                          : g1(a) * 0.5f * p.csm2 * h1 * H * p.ax1.th[i] * br;
            v = -Store<S>::ld(gin + (c * 5 + gopp(a)) * p.plane + own) * p.sg
                + 2.f * p.W1 * (hw * p.bw[side][c] - H * br) + eM;
        }
        d[a] = v;
    }
}

// rho and U (Eq. GOChydrodynamicfields) from pre-collision deviations d and the
// previous step's F - F_rest: the -F_rest/2 momentum of f_ref- and the +F_rest/2
// of the force shift cancel, leaving U1 = (sum d e1 + (F1 - F1_rest)/2)/(rho h2).
__device__ __forceinline__ void fields_from(const StepParams &p, const float d[9], float F1p, float F2p,
                                            float h1, float h2, float &drho, float &U1, float &U2) {
    float k00 = 0.f;
#pragma unroll
    for (int a = 0; a < 9; a++) k00 += d[a];
    float k10 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    float k01 = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    drho = k00 / (h1 * h2);
    float rho = p.rho0 + drho;
    U1 = (k10 + 0.5f * F1p) / (rho * h2);
    U2 = (k01 + 0.5f * F2p) / (rho * h1);
}

// Second-order derivative along an axis from shared-memory values
// vm2, vm1, v0, vp1, vp2 (offsets -2..2): central, or one-sided at the first
// and last node of a wall axis.
__device__ __forceinline__ float dfd(float vm2, float vm1, float v0, float vp1, float vp2, int k, int n,
                                     int per) {
    if (per || (k > 0 && k < n - 1)) return 0.5f * (vp1 - vm1);
    if (k == 0) return 0.5f * (-3.f * v0 + 4.f * vp1 - vp2);
    return 0.5f * (3.f * v0 - 4.f * vm1 + vm2);
}

struct TileSmem;
template <class S, bool MHD>
__device__ __forceinline__ void node_update(const StepParams &p, int i, int j, int tx, int ty,
                                            const TileSmem &sm);

struct TileSmem {
    float rho[EH][EW], u1[EH][EW], u2[EH][EW];
    float d[9][TY][TX];
    float F[2][TY][TX];
};

// One TX x TY tile (tile coordinates bx, by) of one lattice.  All threads of
// the block must call it (it contains a block barrier).
template <class S, bool MHD>
__device__ __forceinline__ void step_tile(const StepParams &p, int bx, int by, TileSmem &sm) {
    float (&s_rho)[EH][EW] = sm.rho;
    float (&s_u1)[EH][EW] = sm.u1;
    float (&s_u2)[EH][EW] = sm.u2;
    float (&s_d)[9][TY][TX] = sm.d;
    float (&s_F)[2][TY][TX] = sm.F;

    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = bx * TX, j0 = by * TY;
    const S *Fin = static_cast<const S *>(p.Fin);

    // ---- phase 1: fields on the tile and its halo --------------------------
    for (int e = tid; e < EXT; e += NT) {
        const int ey = e / EW, ex = e - ey * EW;
        int i = i0 - HX + ex, j = j0 - HY + ey;
        bool in = true;
        if (i < 0 || i >= p.nx) {
            if (p.per_x) i = wrapi(i, p.nx); else in = false;
        }
        if (j < 0 || j >= p.ny) {
            if (p.per_y) j = wrapi(j, p.ny); else in = false;
        }
        if (!in) {
            s_rho[ey][ex] = 0.f;
            s_u1[ey][ex] = 0.f;
            s_u2[ey][ex] = 0.f;
            continue;
        }
        const float h1 = p.ax1.h[i], h2 = p.ax2.h[j];
        float d[9];
        pull_node<S>(p, i, j, h1, h2, d);
        const long long idx = (long long)j * p.pitch + i;
        // stored force of the previous step, F - F_rest
        const float F1p = Store<S>::ld(Fin + idx) * p.sF;
        const float F2p = Store<S>::ld(Fin + p.plane + idx) * p.sF;
        float drho, U1, U2;
        fields_from(p, d, F1p, F2p, h1, h2, drho, U1, U2);
        s_rho[ey][ex] = drho;
        s_u1[ey][ex] = U1;
        s_u2[ey][ex] = U2;
        const int tx = ex - HX, ty = ey - HY;
        if (tx >= 0 && tx < TX && ty >= 0 && ty < TY && i0 + tx < p.nx && j0 + ty < p.ny) {
#pragma unroll
            for (int a = 0; a < 9; a++) s_d[a][ty][tx] = d[a];
            s_F[0][ty][tx] = F1p;
            s_F[1][ty][tx] = F2p;
        }
    }
    __syncthreads();

    // ---- phase 2: one node per thread ---------------------------------------
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + tx, j = j0 + ty;
    if (i < p.nx && j < p.ny) node_update<S, MHD>(p, i, j, tx, ty, sm);
}

// Phase 2 of step_tile for node (i, j) = (i0 + tx, j0 + ty).
template <class S, bool MHD>
__device__ __forceinline__ void node_update(const StepParams &p, int i, int j, int tx, int ty,
                                            const TileSmem &sm) {
    const float (&s_rho)[EH][EW] = sm.rho;
    const float (&s_u1)[EH][EW] = sm.u1;
    const float (&s_u2)[EH][EW] = sm.u2;
    const float (&s_d)[9][TY][TX] = sm.d;
    const float (&s_F)[2][TY][TX] = sm.F;
    const int ex = tx + HX, ey = ty + HY;

    const float h1 = p.ax1.h[i], h2 = p.ax2.h[j];
    const float ih1 = p.ax1.ih[i], ih2 = p.ax2.ih[j];
    const float t11 = p.ax1.th[i], t22 = p.ax2.th[j];
    const float H = h1 * h2;
    float d[9];
#pragma unroll
    for (int a = 0; a < 9; a++) d[a] = s_d[a][ty][tx];
    const float F1p = s_F[0][ty][tx], F2p = s_F[1][ty][tx];
    const float drho = s_rho[ey][ex], U1 = s_u1[ey][ex], U2 = s_u2[ey][ex];
    const float rho = p.rho0 + drho;

    // normal derivatives (second-order finite differences)
    const float dU1 = dfd(s_u1[ey][ex - 2], s_u1[ey][ex - 1], U1, s_u1[ey][ex + 1], s_u1[ey][ex + 2], i, p.nx, p.per_x);
    const float dr1 = dfd(s_rho[ey][ex - 2], s_rho[ey][ex - 1], drho, s_rho[ey][ex + 1], s_rho[ey][ex + 2], i, p.nx, p.per_x);
    const float dU2 = dfd(s_u2[ey - 2][ex], s_u2[ey - 1][ex], U2, s_u2[ey + 1][ex], s_u2[ey + 2][ex], j, p.ny, p.per_y);
    const float dr2 = dfd(s_rho[ey - 2][ex], s_rho[ey - 1][ex], drho, s_rho[ey + 1][ex], s_rho[ey + 2][ex], j, p.ny, p.per_y);

    const long long idx = (long long)j * p.pitch + i;
    float FL1 = 0.f, FL2 = 0.f, B1 = 0.f, B2 = 0.f;

    // ---- MIE (Appendix G): local dB, J3, Lorentz force, SRT collision -------
    if constexpr (MHD) {
        S *gout = static_cast<S *>(p.gout);
        float gd[2][5], Bc[2], dBc[2], dB1[2], dB2[2], A1[2], A2[2];
#pragma unroll
        for (int c = 0; c < 2; c++) {
            pull_mie<S>(p, i, j, h1, h2, c, gd[c]);
            float s = gd[c][0] + gd[c][1] + gd[c][2] + gd[c][3] + gd[c][4];
            dBc[c] = s / H;                     // h1 h2 B = sum g (Eq. 13_C, Y = 0); sum g_ref- = H B_rest
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
            dB1[c] = -L1 / (p.csm2 * (0.5f * H + (p.taum - 0.5f) * h2 * ih1));
            dB2[c] = -L2 / (p.csm2 * (0.5f * H + (p.taum - 0.5f) * h1 * ih2));
        }
        // current density (Eq. currentdensity-GOC) and Lorentz force (Eq. Lorentzforce-GOC)
        const float J3 = p.imum / H * (h2 * dB1[1] - h1 * dB2[0]);
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
                Store<S>::st(gout + (c * 5 + a) * p.plane + idx, gt * p.isg);
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
    const float ics2 = 1.f / cs2;
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
    for (int a = 0; a < 9; a++) Store<S>::st(fout + a * p.plane + idx, o[a] * p.isf);
    S *Fout = static_cast<S *>(p.Fout);
    Store<S>::st(Fout + idx, F1dev * p.isF);
    Store<S>::st(Fout + p.plane + idx, F2dev * p.isF);

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

// Single lattice: one block per tile.
template <class S, bool MHD>
__global__ void __launch_bounds__(NT, 2) step_kernel(const StepParams p) {
    __shared__ TileSmem sm;
    step_tile<S, MHD>(p, blockIdx.x, blockIdx.y, sm);
}

// Many lattices in one launch: work item t in [0, total) is a tile of the
// lattice k with tile_off[k] <= t < tile_off[k+1]; a persistent grid strides
// over the items.  Lattices with and without the MIE may be mixed.
template <class S>
__global__ void __launch_bounds__(NT, 2) batch_step_kernel(const StepParams *__restrict__ params,
                                                           const int *__restrict__ tile_off, int nlat) {
    __shared__ TileSmem sm;
    __shared__ int s_k;
    const int total = tile_off[nlat];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            int lo = 0, hi = nlat - 1;   // last k with tile_off[k] <= t
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
            }
            s_k = lo;
        }
        __syncthreads();
        const int k = s_k;
        const StepParams &p = params[k];
        const int local = t - tile_off[k];
        const int tiles_x = (p.nx + TX - 1) / TX;
        const int by = local / tiles_x, bx = local - by * tiles_x;
        if (p.gin) step_tile<S, true>(p, bx, by, sm);
        else step_tile<S, false>(p, bx, by, sm);
        __syncthreads();   // shared memory is reused by the next item
    }
}

}  // namespace goc
