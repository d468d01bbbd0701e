// goc_std.cuh -- the standard uniform-grid central-moment D2Q9 LBM, the
// matched-accuracy comparator of the GOC scheme.
//
// It is the GOC step specialised to h1 = h2 = 1 (theta = 0, c_s^2 = 1/3) with
// the cubic terms of Eqs. 83/85 dropped: there the normal-gradient corrections
// of Eqs. 82-85 vanish identically, the geometric force is zero, the
// metric-dependent parts of the central-moment equilibria (q20 ... q12) vanish
// and the force of every step is the constant body force.  What remains is a
// local cascaded central-moment collision with forcing and a pull from the
// eight neighbours: no finite differences, no stored force, no tables.  The
// populations are stored as deviations from w_a rho0 (the rest equilibrium),
// FP32 or a scaled 16-bit format.
#pragma once

#include "goc_device.cuh"

namespace goc {

constexpr int STD_BX = 128, STD_BY = 2;   // 256 threads: rows of 128 nodes

template <class S, bool CHECKS>
__device__ __forceinline__ void std_pull(const StepParams &p, const S *fin, int i, int j, float d[9]) {
    const long long idx = (long long)j * p.pitch + i;
    if (p.nopull) {
#pragma unroll
        for (int a = 0; a < 9; a++) d[a] = scl<S>(Store<S>::ld(fin + a * p.plane + idx), p.sf);
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
            v = scl<S>(Store<S>::ld(fin + a * p.plane + (long long)sj * p.pitch + si), p.sf);
        } else {   // half-way bounce-back of the node's own outgoing population, moving wall (Eq. 101)
            v = scl<S>(Store<S>::ld(fin + opp(a) * p.plane + idx), p.sf);
            if (p.moving && (e1(a) != 0 && e2(a) != 0)) {
                const int sy = e2(a) > 0 ? SIDE_S : SIDE_N;
                const int sx = e1(a) > 0 ? SIDE_W : SIDE_E;
                const float uy = oy ? p.uw[sy] : 0.f, ux = ox ? p.uw[sx] : 0.f;
                if (uy != 0.f || ux != 0.f) {
                    if (!rhow_ready) {
                        float s = 0.f;
#pragma unroll
                        for (int b = 0; b < 9; b++) s += scl<S>(Store<S>::ld(fin + b * p.plane + idx), p.sf);
                        rhow = p.rho0 + s;
                        rhow_ready = true;
                    }
                    if (uy != 0.f) v += e1(a) * rhow * p.cs2 * uy * 0.5f;
                    if (ux != 0.f) v += e2(a) * rhow * p.cs2 * ux * 0.5f;
                }
            }
        }
        d[a] = v;
    }
}

template <class S, bool CHECKS>
__device__ __forceinline__ void std_node(const StepParams &p, int i, int j) {
    const S *fin = static_cast<const S *>(p.fin);
    float d[9];
    std_pull<S, CHECKS>(p, fin, i, j, d);
    // fields; the force of the previous step is the body force (zero before the first step)
    const float F1p = p.nopull ? 0.f : p.fext1, F2p = p.nopull ? 0.f : p.fext2;
    float k00 = 0.f;
#pragma unroll
    for (int a = 0; a < 9; a++) k00 += d[a];
    const float k10 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    const float k01 = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    const float drho = k00, rho = p.rho0 + drho;
    const float irho = __frcp_rn(rho);
    const float u = (k10 + 0.5f * F1p) * irho, v = (k01 + 0.5f * F2p) * irho;
    const float uu = u * u, vv = v * v, uv = u * v, cs2 = p.cs2, r0 = p.rho0;

    // central moments about (u, v): 1D passes along xi1 per row, then along xi2
    float k0[3], k1[3], k2[3];
    {
        const float fm[3] = {d[7], d[3], d[6]}, f0[3] = {d[4], d[0], d[2]}, fp[3] = {d[8], d[1], d[5]};
#pragma unroll
        for (int y = 0; y < 3; y++) {
            const float s = fp[y] + fm[y], t = fp[y] - fm[y];
            k0[y] = s + f0[y];
            k1[y] = fmaf(-u, k0[y], t);
            k2[y] = fmaf(-u, t + k1[y], s);
        }
    }
    float c[3][3];
    {
        const float *kk[3] = {k0, k1, k2};
#pragma unroll
        for (int m = 0; m < 3; m++) {
            const float s = kk[m][2] + kk[m][0], t = kk[m][2] - kk[m][0];
            c[m][0] = s + kk[m][1];
            c[m][1] = fmaf(-v, c[m][0], t);
            c[m][2] = fmaf(-v, t + c[m][1], s);
        }
    }
    // equilibrium minus current central moments (rest parts cancelled), relaxation, forcing
    const float e2s = 2.f * cs2 * drho - (c[2][0] + c[0][2]) - (uu + vv) * r0;
    const float e2d = -(c[2][0] - c[0][2]) - (uu - vv) * r0;
    const float e11 = -c[1][1] - uv * r0;
    const float e21 = -c[2][1] + v * r0 * (cs2 + uu);
    const float e12 = -c[1][2] + u * r0 * (cs2 + vv);
    const float e22 = cs2 * cs2 * drho - c[2][2] - r0 * (cs2 * (uu + vv) + uu * vv);
    const float *om = p.om;
    const float D10 = om[1] * 0.5f * F1p + (1.f - 0.5f * om[1]) * p.fext1;
    const float D01 = om[2] * 0.5f * F2p + (1.f - 0.5f * om[2]) * p.fext2;
    const float D2s = om[3] * e2s, D2d = om[4] * e2d;
    const float g[3][3] = {{0.f, D01, 0.5f * (D2s - D2d)},
                           {D10, om[5] * e11, om[7] * e12},
                           {0.5f * (D2s + D2d), om[6] * e21, om[8] * e22}};
    // back to populations: inverse 1D passes along xi2, then xi1
    float r0_[3], rp[3], rn[3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const float m1 = fmaf(v, g[m][0], g[m][1]);
        const float m2 = fmaf(v, g[m][1] + m1, g[m][2]);
        r0_[m] = g[m][0] - m2;
        rp[m] = 0.5f * (m1 + m2);
        rn[m] = 0.5f * (m2 - m1);
    }
    const float *rows[3] = {r0_, rp, rn};   // e2 = 0, +1, -1
    float o0[3], op[3], on[3];
#pragma unroll
    for (int y = 0; y < 3; y++) {
        const float m1 = fmaf(u, rows[y][0], rows[y][1]);
        const float m2 = fmaf(u, rows[y][1] + m1, rows[y][2]);
        o0[y] = rows[y][0] - m2;
        op[y] = 0.5f * (m1 + m2);
        on[y] = 0.5f * (m2 - m1);
    }
    float o[9];
    o[0] = d[0] + o0[0];
    o[1] = d[1] + op[0];
    o[3] = d[3] + on[0];
    o[2] = d[2] + o0[1];
    o[5] = d[5] + op[1];
    o[6] = d[6] + on[1];
    o[4] = d[4] + o0[2];
    o[8] = d[8] + op[2];
    o[7] = d[7] + on[2];

    const long long idx = (long long)j * p.pitch + i;
    const bool sr = Store<S>::scaled && p.sr;
    uint32_t rng = sr ? node_seed((uint32_t)(idx + (long long)p.seed_row0 * p.pitch), *p.seed_rd) : 0u;
    S *fout = static_cast<S *>(p.fout);
#pragma unroll
    for (int a = 0; a < 9; a++) put<S>(fout + a * p.plane + idx, scl<S>(o[a], p.isf), sr, rng);
    if (p.uout) {
        __stcg(p.uout + idx, u);
        __stcg(p.uout + p.plane + idx, v);
        __stcg(p.uout + 2 * p.plane + idx, 0.f);
        __stcg(p.uout + 3 * p.plane + idx, 0.f);
    }
    if (p.flag) {
        const bool bad = !(rho > 0.f && fabsf(u) + fabsf(v) < 1e30f);
        const unsigned mk = __activemask();
        if (__any_sync(mk, bad) && (threadIdx.x & 31) == (__ffs(mk) - 1) && *((volatile int *)p.flag) == 0)
            atomicExch(p.flag, 1);
    }
}

// One thread per node; blocks of STD_BX x STD_BY.  Blocks whose pull sources
// all lie inside the lattice take the path without boundary logic.
template <class S>
__global__ void __launch_bounds__(STD_BX *STD_BY) std_step_kernel(const __grid_constant__ StepParams p) {
    const int i0 = blockIdx.x * STD_BX, j0 = blockIdx.y * STD_BY;
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    griddep_launch_dependents();
    griddep_wait();
    if (Store<S>::scaled && p.sr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        *p.seed_wr = *p.seed_rd + 1u;
    if (i >= p.nx || j >= p.ny) return;
    const bool interior = i0 >= 1 && i0 + STD_BX + 1 <= p.nx && j0 >= 1 && j0 + STD_BY + 1 <= p.ny;
    if (interior) std_node<S, false>(p, i, j);
    else std_node<S, true>(p, i, j);
}

}  // namespace goc
