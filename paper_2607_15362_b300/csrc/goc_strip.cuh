// goc_strip.cuh -- the fused GOC-LBM step by warp strips (no shared memory,
// no block barriers).
//
// A warp owns a strip of SW = 30 output columns and sh rows.  Lane l holds
// column c0 + l (c0 = the column left of the strip); lanes 1..30 update nodes,
// lanes 0 and 31 only supply the fields of the x-neighbours.  The warp sweeps
// the rows r0 - 1 .. r1 of its strip: at row r it pulls the populations of
// row r (pull streaming with the boundary conditions, Appendix E Step 6, Eq.
// 101/103) and forms rho, U (Appendix E Step 7, with the stored force of the
// previous step), then updates row r - 1, whose normal derivatives come from
// the fields of rows r - 2, r (kept in registers) along xi2 and from the
// neighbouring lanes (warp shuffles) along xi1.  A node's fields are formed
// once per strip, plus the two rows above and below the strip and the two halo
// columns.  At a wall row the one-sided stencil needs the fields two rows
// inward: row ny - 3 is in the sweep history; row 2 (south wall) is pulled
// once more.
//
// Every node runs the same functions as in the tile kernel (fields_from,
// dfd, collide); the results agree with it to FP32 rounding (the compiler may
// fuse multiply-adds differently in the two kernels).  Measured on a B300 the
// tile kernel is faster except for the MIE lattices at 4-row strips.
#pragma once

#include "goc_step.cuh"

namespace goc {

constexpr int SW = 30;                       // output columns per strip
#ifndef GOC_STRIP_WARPS
#define GOC_STRIP_WARPS 4                    // warps per block (independent strips)
#endif
#ifndef GOC_STRIP_MIN_BLOCKS
#define GOC_STRIP_MIN_BLOCKS 4
#endif
constexpr int STRIP_NT = 32 * GOC_STRIP_WARPS;

// column of lane 0 of strip sx: one left of the first output column; the last
// strip of a lattice at least 31 wide is moved left so that its lane 31 is the
// first column past the lattice (every wall node then has two inward lanes)
__host__ __device__ __forceinline__ int strip_c0(int sx, int nx) {
    const int c = SW * sx - 1;
    return (nx >= SW + 1 && c > nx - (SW + 1)) ? nx - (SW + 1) : c;
}
__host__ __device__ __forceinline__ int strips_x(int nx) { return (nx + SW - 1) / SW; }

// pull and fields of node (i, row r) if it exists (row wrapped on a periodic axis)
template <class S, bool CHECKS>
__device__ __forceinline__ bool strip_pull(const StepParams &p, const SrcGlobal<S> &src, int i, bool iv, float h1,
                                           float ih1, int r, float d[9], float &F1p, float &F2p, float &h2, float &ih2,
                                           float &drho, float &U1, float &U2) {
    int jr = r;
    bool nv = iv;
    if (CHECKS && (jr < 0 || jr >= p.ny)) {
        if (p.per_y) jr = wrapi(jr, p.ny); else nv = false;
    }
    F1p = F2p = 0.f;
    h2 = ih2 = 1.f;
    drho = U1 = U2 = 0.f;
    if (nv) {
        h2 = p.ax2.h[jr];
        ih2 = p.ax2.ih[jr];
        pull_node<CHECKS>(p, src, i, jr, h1, h2, d);
        F1p = src.Fv(0, i, jr);
        F2p = src.Fv(1, i, jr);
        fields_from(p, d, F1p, F2p, ih1, ih2, drho, U1, U2);
    } else {
#pragma unroll
        for (int a = 0; a < 9; a++) d[a] = 0.f;
    }
    return nv;
}

template <class S, bool MHD, bool CHECKS>
__device__ __forceinline__ void strip_run(const StepParams &p, int c0, int xlo, int xhi, int r0, int r1) {
    const SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin), static_cast<const S *>(p.gin),
                           p.plane, p.pitch, p.sf, p.sF, p.sg};
    const int lane = threadIdx.x & 31;
    const int col = c0 + lane;
    int i = col;
    bool iv = true;
    if (CHECKS && (i < 0 || i >= p.nx)) {
        if (p.per_x) i = wrapi(i, p.nx); else iv = false;
    }
    const bool outc = iv && col >= xlo && col < xhi;
    const int ic = iv ? i : 0;
    const float h1 = p.ax1.h[ic], ih1 = p.ax1.ih[ic];

    // sweep state: fields of rows r-3 (z), r-2 (a), r-1 (b); populations of row r-1
    float rz = 0.f, vz = 0.f, ra = 0.f, ua = 0.f, va = 0.f, rb = 0.f, ub = 0.f, vb = 0.f;
    float db[9], F1b = 0.f, F2b = 0.f, h2b = 1.f, ih2b = 1.f;
#pragma unroll
    for (int a = 0; a < 9; a++) db[a] = 0.f;
    bool nb = false;

    for (int r = r0 - 1; r <= r1; r++) {
        float dc[9], F1c, F2c, h2c, ih2c, rc, uc, vc;
        const bool nc = strip_pull<S, CHECKS>(p, src, i, iv, h1, ih1, r, dc, F1c, F2c, h2c, ih2c, rc, uc, vc);
        const int j = r - 1;
        if (j >= r0) {   // update row j (warp-uniform)
            const unsigned full = 0xffffffffu;
            const float um1 = __shfl_up_sync(full, ub, 1), up1 = __shfl_down_sync(full, ub, 1);
            const float qm1 = __shfl_up_sync(full, rb, 1), qp1 = __shfl_down_sync(full, rb, 1);
            float fl[7][1];
            fl[0][0] = rb;
            fl[1][0] = ub;
            fl[2][0] = vb;
            if (CHECKS) {
                const float um2 = __shfl_up_sync(full, ub, 2), up2 = __shfl_down_sync(full, ub, 2);
                const float qm2 = __shfl_up_sync(full, rb, 2), qp2 = __shfl_down_sync(full, rb, 2);
                fl[3][0] = dfd(um2, um1, ub, up1, up2, i, p.nx, p.per_x);
                fl[4][0] = dfd(qm2, qm1, rb, qp1, qp2, i, p.nx, p.per_x);
                // two rows inward of a wall row: row 2 (south) is pulled again; row ny - 3
                // (north) is in the sweep history unless the strip starts below it
                float rx = 0.f, vx = 0.f;
                const bool south = !p.per_y && j == 0;
                const bool north = !p.per_y && j == p.ny - 1 && j - 2 < r0 - 1;
                if (south || north) {
                    float dx[9], t1, t2, t3, t4, ux;
                    strip_pull<S, CHECKS>(p, src, i, iv, h1, ih1, south ? 2 : p.ny - 3, dx, t1, t2, t3, t4, rx, ux, vx);
                }
                const float vm2 = north ? vx : vz, rm2 = north ? rx : rz;
                const float vp2 = south ? vx : 0.f, rp2 = south ? rx : 0.f;
                fl[5][0] = dfd(vm2, va, vb, vc, vp2, j, p.ny, p.per_y);
                fl[6][0] = dfd(rm2, ra, rb, rc, rp2, j, p.ny, p.per_y);
            } else {
                fl[3][0] = 0.5f * (up1 - um1);
                fl[4][0] = 0.5f * (qp1 - qm1);
                fl[5][0] = 0.5f * (vc - va);
                fl[6][0] = 0.5f * (rc - ra);
            }
            if (outc && nb) {
                const int jj[1] = {j};
                const bool own[1] = {true};
                const float dn[1][9] = {{db[0], db[1], db[2], db[3], db[4], db[5], db[6], db[7], db[8]}};
                const float F1n[1] = {F1b}, F2n[1] = {F2b}, h2n[1] = {h2b}, ih2n[1] = {ih2b};
                collide<S, MHD, CHECKS, float>(p, src, i, jj, own, dn, F1n, F2n, h1, ih1, h2n, ih2n, fl);
            }
        }
        rz = ra;
        vz = va;
        ra = rb;
        ua = ub;
        va = vb;
        rb = rc;
        ub = uc;
        vb = vc;
#pragma unroll
        for (int a = 0; a < 9; a++) db[a] = dc[a];
        F1b = F1c;
        F2b = F2c;
        h2b = h2c;
        ih2b = ih2c;
        nb = nc;
    }
    (void)ua;
}

// One warp per strip; strips ordered along xi1 first.  Strips whose pull
// sources and stencils all lie inside the lattice take the path without
// boundary logic.
template <class S, bool MHD>
__global__ void __launch_bounds__(STRIP_NT, GOC_STRIP_MIN_BLOCKS) strip_kernel(const __grid_constant__ StepParams p) {
    griddep_launch_dependents();
    griddep_wait();
    if (Store<S>::scaled && p.sr && blockIdx.x == 0 && threadIdx.x == 0) *p.seed_wr = *p.seed_rd + 1u;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nsx = strips_x(p.nx), sh = p.strip_h;
    const int nsy = (p.ny + sh - 1) / sh;
    if (warp >= nsx * nsy) return;   // whole warps leave together
    const int sx = warp % nsx, sy = warp / nsx;
    const int c0 = strip_c0(sx, p.nx);
    const int xlo = SW * sx, xhi = min(xlo + SW, p.nx);
    const int r0 = sy * sh, r1 = min(r0 + sh, p.ny);
    const bool interior = c0 >= 1 && c0 + 32 <= p.nx - 1 && r0 >= 2 && r1 + 1 <= p.ny - 1;
    if (interior) strip_run<S, MHD, false>(p, c0, xlo, xhi, r0, r1);
    else strip_run<S, MHD, true>(p, c0, xlo, xhi, r0, r1);
}

}  // namespace goc
