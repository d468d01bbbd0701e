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
#include "goc_vec.cuh"

namespace goc {

#ifndef GOC_TILE_ROWS
#define GOC_TILE_ROWS 8        // tile height (rows); the tile width is one warp
#endif
#ifndef GOC_MIN_BLOCKS
#define GOC_MIN_BLOCKS 4       // resident blocks per SM asked of the register allocator, NSE kernels (64
                               // registers; measured best: 124.9 vs 139.7 us at 2048^2 with 3 blocks)
#endif
#ifndef GOC_MIE_STAGED
// 0 (default): the MIE populations are read through L1 and the NSE+MIE kernels
// run 3 blocks per SM (80 registers, 2 x 25 KB stages); 1: they are staged by
// TMA with the tile (2 x 41 KB stages, 2 blocks per SM).  Measured (B300,
// FP32 / FP16 us per step): Hartmann channel 256 x 1024 31.8 / 37.2 against
// 34.2 / 41.8 staged; 1024^2 cavity with the MIE 70.7 / 71.5 against 70.6 /
// 76.7; 2048^2 218 / 232 against 208 / 253.
#define GOC_MIE_STAGED 0
#endif
#ifndef GOC_MIN_BLOCKS_MHD
#define GOC_MIN_BLOCKS_MHD (GOC_MIE_STAGED ? 2 : 3)
#endif
#ifndef GOC_MIN_BLOCKS_MHD_STRAIGHT
// NSE+MIE kernels of straight grids: 4 blocks per SM (64 registers) measured
// faster than 3 (80 registers, no spills): Hartmann channel 256 x 1024
// 27.9 against 30.3-31.8 us per step, 2048^2 cavity with the MIE 181 against
// 207 us (FP32).  The curved-grid MIE kernels, with more terms, keep 3.
#define GOC_MIN_BLOCKS_MHD_STRAIGHT (GOC_MIE_STAGED ? 2 : 4)
#endif
#ifndef GOC_ROWS_PER_THREAD
#define GOC_ROWS_PER_THREAD 1  // nodes per thread (rows ty + r TY/RPT); 2 runs the collision on packed f32x2 (measured slower)
#endif
constexpr int TX = 32, TY = GOC_TILE_ROWS, RPT = GOC_ROWS_PER_THREAD, TYT = TY / RPT, NT = TX * TYT;
static_assert(TY % RPT == 0, "tile rows must be a multiple of the rows per thread");
template <int R> struct VecOf;
template <> struct VecOf<1> { using type = float; };
template <> struct VecOf<2> { using type = float2; };
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
    static constexpr int STAGE_MHD = GOC_MIE_STAGED ? OFF_G + align128(G_BYTES) : OFF_G;
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
// (A source may also say where a node's new populations go, out_slot below,
// and may carry the population sum of wall nodes, wall_sum: the in-place
// lattices of goc_aa.cuh.)
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
// Offset of the new population a of node (i, j) in the output buffer: its own
// node and link (two-buffer lattices; idx = j pitch + i).
template <class Src>
__device__ __forceinline__ long long out_slot(const Src &, const StepParams &p, int a, int, int, long long idx) {
    return a * p.plane + idx;
}
// The same for the MIE population of component c along link a (component-major).
template <class Src>
__device__ __forceinline__ long long out_slot_g(const Src &, const StepParams &p, int c, int a, int, int,
                                                long long idx) {
    return (c * 5 + a) * p.plane + idx;
}
// Sources that carry the population sums of the wall nodes (the moving-wall
// density below) define kWallSums = true.
template <class Src, class = void> struct HasWallSums { static constexpr bool value = false; };
template <class Src> struct HasWallSums<Src, decltype(void(Src::kWallSums))> { static constexpr bool value = Src::kWallSums; };
// Sources of lattices updated in place define kInPlace = true (their output
// slots follow out_slot / out_slot_g).
template <class Src, class = void> struct InPlaceSrc { static constexpr bool value = false; };
template <class Src> struct InPlaceSrc<Src, decltype(void(Src::kInPlace))> { static constexpr bool value = Src::kInPlace; };

template <class S> struct SrcSmem {        // the TMA-staged tile
    using T = Tiling<S>;
    const S *f, *F, *g;
    int ox, oy, oyg;                        // lattice coordinates of staged element (0, 0)
    float sf, sF, sg;
#if !GOC_MIE_STAGED
    long long plane;                        // g: the MIE populations in global memory
    int pitch;
#endif
    __device__ __forceinline__ float fv(int a, int i, int j) const {
        return scl<S>(Store<S>::lds(f + (a * T::BY + (j - oy)) * T::BX + (i - ox)), sf);
    }
    __device__ __forceinline__ float Fv(int c, int i, int j) const {
        return scl<S>(Store<S>::lds(F + (c * T::BY + (j - oy)) * T::BX + (i - ox)), sF);
    }
    __device__ __forceinline__ float gv(int k, int i, int j) const {
#if GOC_MIE_STAGED
        return scl<S>(Store<S>::lds(g + (k * T::BYG + (j - oyg)) * T::BX + (i - ox)), sg);
#else
        return scl<S>(Store<S>::ld(g + k * plane + (long long)j * pitch + i), sg);
#endif
    }
};

// The storage reference field of the MIE populations of row j: the per-row
// reference of 16-bit straight-grid storage (REF), else the uniform B_rest.
template <bool REF>
__device__ __forceinline__ float bref(const StepParams &p, int c, int j) {
    return REF ? GOC_BROW(p, c, j) : p.brest[c];
}

// Pull the nine deviations arriving at node (i, j): the value stored at the
// source is relative to the source's f_ref+, the result relative to this
// node's f_ref-, so links 1..4 add f_ref+(source) - f_ref-(node) (the rm/rp
// tables; links 0 and 5..8 have the same reference everywhere).  A link whose
// source lies outside a wall axis is a half-way bounce-back of the node's own
// outgoing population, plus the moving-wall term f_a^eq(w) - f_abar^eq(w)
// (Eq. 101) = e1 rho_w cs2 u / (2 h2_w) across a S/N wall and
// e2 rho_w cs2 u / (2 h1_w) across a W/E wall (rho_w: this node's density at
// the time of the outgoing population).  CHECKS = false: every source is
// inside the lattice (interior tile).  REF: the per-row storage reference of
// links 1 and 3 (half momentum ur1 = u1r[j]) is the same at the source and the
// node of an x link and cancels; a link bounced back at a W/E wall changes
// from link 1 to 3 (or back), whose references differ by 2 e1 ur1.
template <bool CHECKS, int GEOM = 0, bool REF = false, class Src>
__device__ __forceinline__ void pull_node(const StepParams &p, const Src &src, int i, int j, float h1, float h2,
                                          float d[9], float ur1 = 0.f) {
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
            if (GEOM == 2) {   // node table: full corrections per node and link
                if (a >= 1 && a <= 4) v += gm_at(p.gm, p.plane, p.pitch, 5 + a, i, j);
            } else {
                if (a == 1) v += GEOM ? p.ax1.rm[i] : h2 * p.ax1.rm[i];   // curvilinear: full corrections
                if (a == 3) v += GEOM ? p.ax1.rp[i] : h2 * p.ax1.rp[i];
                if (a == 2) v += h1 * p.ax2.rm[j];
                if (a == 4) v += h1 * p.ax2.rp[j];
            }
        } else {
            v = src.fv(opp(a), i, j);
            if (REF && (a == 1 || a == 3)) v -= 2.f * (float)e1(a) * ur1;
            if (p.moving && (e1(a) != 0 && e2(a) != 0)) {
                int sy = e2(a) > 0 ? SIDE_S : SIDE_N;
                int sx = e1(a) > 0 ? SIDE_W : SIDE_E;
                float uy = oy ? p.uw[sy] : 0.f, ux = ox ? p.uw[sx] : 0.f;
                if (uy != 0.f || ux != 0.f) {
                    if (!rhow_ready) {
                        float s = 0.f;
                        if constexpr (HasWallSums<Src>::value) {
                            s = src.wall_sum(i, j);   // the same sum, taken before this launch
                        } else {
#pragma unroll
                            for (int b = 0; b < 9; b++) s += src.fv(b, i, j);
                        }
                        rhow = p.rho0 + s / (h1 * h2);
                        rhow_ready = true;
                    }
                    const float hy = GEOM == 2 ? gm_wall(p.gm, p.plane, p.nx, p.ny, sy, i) : p.hwn[sy];
                    const float hx = GEOM == 2 ? gm_wall(p.gm, p.plane, p.nx, p.ny, sx, j) : p.hwn[sx];
                    if (uy != 0.f) v += e1(a) * rhow * p.cs2 * uy / (2.f * hy);
                    if (ux != 0.f) v += e2(a) * rhow * p.cs2 * ux / (2.f * hx);
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
// -s_abar + 2 W_a (h_wall B_wall - H B_rest) + e_a.M.  REF: B_rest is the
// row field Bref_c(j); links 2 and 4 come from another row and take their
// corrections from the per-row tables bpull.
template <bool CHECKS, int GEOM = 0, bool REF = false, class Src>
__device__ __forceinline__ void pull_mie(const StepParams &p, const Src &src, int i, int j, float h1, float h2,
                                         int c, float d[5]) {
    const float H = h1 * h2;
    if (p.nopull) {
#pragma unroll
        for (int a = 0; a < 5; a++) d[a] = src.gv(c * 5 + a, i, j);
        return;
    }
    const float br = bref<REF>(p, c, j);
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
            if (GEOM == 0) {   // curvilinear grids store g itself (B_rest = 0)
                if (a == 1) v += br * h2 * p.ax1.dm[i];
                if (a == 3) v += br * h2 * p.ax1.dp[i];
                if (REF) {
                    if (a == 2) v += h1 * GOC_BPULL(p, 0, c, j);
                    if (a == 4) v += h1 * GOC_BPULL(p, 1, c, j);
                } else {
                    if (a == 2) v += br * h1 * p.ax2.dm[j];
                    if (a == 4) v += br * h1 * p.ax2.dp[j];
                }
            }
        } else if (GEOM) {   // h_wall = h1 h2 at the wall point
            // (the column metric has bw premultiplied by the tangential factor,
            // which is constant along its radial walls)
            const int side = oy ? (g2(a) > 0 ? SIDE_S : SIDE_N) : (g1(a) > 0 ? SIDE_W : SIDE_E);
            const int k = oy ? i : j;
            const float hw = GEOM == 2 ? gm_wall(p.gm, p.plane, p.nx, p.ny, side, k) *
                                             gm_wall(p.gm, p.plane, p.nx, p.ny, 4 + side, k)
                                       : p.hwn[side];
            v = -src.gv(c * 5 + gopp(a), i, j) + 2.f * p.W1 * hw * p.bw[side][c];
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

// Metric factors (and their inverses) of node (i, j) for the grid kinds:
// GEOM 0 straight (h1(xi1), h2(xi2)), 1 curvilinear column (h1, h2 of xi1),
// 2 node table.
template <int GEOM>
__device__ __forceinline__ void node_metric(const StepParams &p, int i, int j, float &h1, float &h2, float &ih1,
                                            float &ih2) {
    if (GEOM == 2) {
        h1 = gm_at(p.gm, p.plane, p.pitch, 0, i, j);
        h2 = gm_at(p.gm, p.plane, p.pitch, 1, i, j);
        ih1 = 1.f / h1;
        ih2 = 1.f / h2;
    } else {
        h1 = p.ax1.h[i];
        ih1 = p.ax1.ih[i];
        h2 = GEOM == 1 ? curv_h2(p.ax1, i) : p.ax2.h[j];
        ih2 = GEOM == 1 ? curv_ih2(p.ax1, i) : p.ax2.ih[j];
    }
}

// Hardware reciprocal (rcp.approx: relative error below 2^-22, no refinement):
// rho is near rho0, far from zero, infinities and denormals.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// rho and U (Eq. GOChydrodynamicfields) from pre-collision deviations d and the
// previous step's F - F_rest: the -F_rest/2 momentum of f_ref- and the +F_rest/2
// of the force shift cancel, leaving U1 = (sum d e1 + (F1 - F1_rest)/2)/(rho h2).
// REF: links 1 and 3 of the reference carry 2 ur1 of momentum more.
template <bool REF = false>
__device__ __forceinline__ void fields_from(const StepParams &p, const float d[9], float F1p, float F2p,
                                            float ih1, float ih2, float &drho, float &U1, float &U2,
                                            float ur1 = 0.f) {
    float k00 = 0.f;
#pragma unroll
    for (int a = 0; a < 9; a++) k00 += d[a];
    const float k10 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    const float k01 = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    drho = k00 * (ih1 * ih2);
    const float irho = rcp_approx(p.rho0 + drho);
    if (REF) U1 = (k10 + fmaf(0.5f, F1p, 2.f * ur1)) * irho * ih2;
    else U1 = (k10 + 0.5f * F1p) * irho * ih2;
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

// Collision on raw moments in the storage variables: the raw-moment MRT of
// Appendix D (Steps 1-3: m = P f, relaxation of k00, k10, k01, k2s, k2d,
// k11, k21, k12, k22 with omega_0..8 towards Eq. GOCmomentequilibria with the
// corrections n3, n4 of Eqs. 82-85 on k2s, k2d, sources of Eq.
// GOCmomentsources, f~ = P^-1 m~), and, with every rate 1/tau and zeta = nu,
// the SRT of Appendix F (f~ = f + (f^eq - f)/tau + (1 - 1/(2 tau)) S, the same
// update written in velocity space: its Eq. 14D equilibria are these with
// the bare corrections (n3 +- n4)/2).  m = moments of f - f_rest (two passes
// of the 1D transform about zero velocity), Delta = omega (m^eq - m) + (1 -
// omega/2) Psi per moment with m^eq - m_rest, the change of reference f_ref-
// -> f_ref+ taken off the first moments (which leaves omega F^{n-1}/2 + (1 -
// omega/2) F_dev there, as in the central-moment path); o = d + P^-1 Delta.
// REF: f_ref- - f_rest also holds +-ur1 on links 1 and 3 (per-row reference).
template <bool REF, class V>
__device__ __forceinline__ void raw_relax(const StepParams &p, const V (&d)[9], V (&o)[9], V rho, V drho, V U1,
                                          V U2, V ih2, float ih1, V r, V s, V uu, V vv, V uv, V n3, V n4, V F1,
                                          V F2, V F1dev, V F2dev, V F1p, V F2p, V F1r, V F2r, V ur1) {
    const float *om = p.om, cs2 = p.cs2;
    // populations of f - f_rest by rows e2 = -1, 0, +1 at e1 = -1, 0, +1
    const V q1 = REF ? fmav(F1r, 0.25f, bc<V>(0.f) - ur1) : F1r * 0.25f, q2 = F2r * 0.25f;
    const V fm[3] = {d[7], d[3] + q1, d[6]};
    const V f0[3] = {d[4] + q2, d[0], d[2] - q2};
    const V fp[3] = {d[8], d[1] - q1, d[5]};
    V k0[3], k1[3], k2[3];                                // per row: orders 0, 1, 2 along xi1
#pragma unroll
    for (int y = 0; y < 3; y++) {
        const V sm_ = fp[y] + fm[y];
        k0[y] = sm_ + f0[y];
        k1[y] = fp[y] - fm[y];
        k2[y] = sm_;
    }
    V m[3][3];                                            // m[a][b]: order a along xi1, b along xi2
    {
        const V *kk[3] = {k0, k1, k2};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const V sm_ = kk[a][2] + kk[a][0];
            m[a][0] = sm_ + kk[a][1];
            m[a][1] = kk[a][2] - kk[a][0];
            m[a][2] = sm_;
        }
    }
    // m^eq - m_rest (Eq. 14D; m_rest = (H rho0, 0, 0, r rho0 cs2, s rho0 cs2, 0, 0, 0, rho0 cs2^2))
    const V csd = drho * cs2;
    const V E20 = fmav(r, fmav(rho, uu, csd), (n3 + n4) * 0.5f);
    const V E02 = fmav(s, fmav(rho, vv, csd), (n3 - n4) * 0.5f);
    const V E11 = rho * uv;
    const V E21 = rho * U2 * (uu + cs2) * ih1;
    const V E12 = rho * U1 * (vv + cs2) * ih2;
    const V E22 = fmav(csd, bc<V>(cs2), rho * fmav(uu, vv, (uu + vv) * cs2));
    V g[3][3];
    g[0][0] = bc<V>(0.f);
    g[1][0] = fmav(F1p, 0.5f * om[1], F1dev * (1.f - 0.5f * om[1]));
    g[0][1] = fmav(F2p, 0.5f * om[2], F2dev * (1.f - 0.5f * om[2]));
    {   // combined second-order diagonal moments k2s, k2d (rates omega_3, omega_4)
        const V a20 = E20 - m[2][0], a02 = E02 - m[0][2];
        const V s20 = F1 * U1 * (2.f * ih1), s02 = F2 * U2 * ih2 * 2.f;
        const V D2s = fmav(a20 + a02, om[3], (s20 + s02) * (1.f - 0.5f * om[3]));
        const V D2d = fmav(a20 - a02, om[4], (s20 - s02) * (1.f - 0.5f * om[4]));
        g[2][0] = (D2s + D2d) * 0.5f;
        g[0][2] = (D2s - D2d) * 0.5f;
    }
    g[1][1] = fmav(E11 - m[1][1], om[5], fmav(F1 * U2, ih2, F2 * U1 * ih1) * (1.f - 0.5f * om[5]));
    g[2][1] = (E21 - m[2][1]) * om[6];
    g[1][2] = (E12 - m[1][2]) * om[7];
    g[2][2] = (E22 - m[2][2]) * om[8];
    // P^-1: along xi2, then xi1; for raw moments (c0, c1, c2) the values at
    // e = 0, +1, -1 are c0 - c2, (c1 + c2)/2, (c2 - c1)/2
    V r0[3], rp[3], rn[3];                                // per xi1 order: rows e2 = 0, +1, -1
#pragma unroll
    for (int a = 0; a < 3; a++) {
        r0[a] = g[a][0] - g[a][2];
        rp[a] = (g[a][1] + g[a][2]) * 0.5f;
        rn[a] = (g[a][2] - g[a][1]) * 0.5f;
    }
    const V *rows[3] = {r0, rp, rn};
    V o0[3], op[3], on[3];
#pragma unroll
    for (int y = 0; y < 3; y++) {
        o0[y] = rows[y][0] - rows[y][2];
        op[y] = (rows[y][1] + rows[y][2]) * 0.5f;
        on[y] = (rows[y][2] - rows[y][1]) * 0.5f;
    }
    o[0] = d[0] + o0[0];
    o[1] = d[1] + op[0];
    o[3] = d[3] + on[0];
    o[2] = d[2] + o0[1];
    o[5] = d[5] + op[1];
    o[6] = d[6] + on[1];
    o[4] = d[4] + o0[2];
    o[8] = d[8] + op[2];
    o[7] = d[7] + on[2];
}

// ---- packed FP32 pairs (two lanes, one instruction: sm_100-family f32x2) ----
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float s) { return __fadd2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fma2(float2 a, float s, float2 c) { return __ffma2_rn(a, make_float2(s, s), c); }
__device__ __forceinline__ float2 fma2(float s, float2 b, float2 c) { return __ffma2_rn(make_float2(s, s), b, c); }
// a - b (the product b * (-1) is exact, so this is the rounded difference)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Central-moment collision of one node on a straight grid (theta12 = theta21
// = 0): the stresses and effective force (Appendix B (i), Eq.
// Special1_Force_terms), the corrections of Eqs. 82-85, the central-moment
// relaxation with sources (Appendix E Steps 1-5) and the return to
// populations -- the update of the central-moment path of collide() for
// GEOM 0, with the pairs of quantities its formulas treat alike along xi1 and
// xi2 (h1 and h2, U1 and U2, the two force components, the coefficient pairs
// of the corrections, the equilibrium pairs k21/k12 ...) computed together on
// packed FP32 pairs.  Inputs: pre-collision deviations d (relative to f_ref-),
// drho, U1, U2 and their normal derivatives, the metric of the node, the
// stored force of the previous step (F1p, F2p), the Lorentz force (FL1, FL2),
// the per-row storage reference ur1 (REF).  Outputs: o (relative to f_ref+)
// and the force deviation F - F_rest.
template <bool REF>
__device__ __forceinline__ void collide_straight(const StepParams &p, const float (&d)[9], float drho, float U1,
                                                 float U2, float dU1, float dr1, float dU2, float dr2, float h1,
                                                 float ih1, float t11, float h2, float ih2, float t22, float F1p,
                                                 float F2p, float FL1, float FL2, float ur1, float (&o)[9],
                                                 float &F1dev, float &F2dev) {
    const float cs2 = p.cs2, zeta = p.zeta, nu = p.nu;
    const float rho = drho + p.rho0, csd = drho * cs2;
    const float2 iM = f2(ih1, ih2), T = f2(t11, t22);
    const float2 Ms = f2(h2, h1), iMs = f2(ih2, ih1);     // swapped: (h2, h1), (1/h2, 1/h1)
    const float2 U = f2(U1, U2), Us = f2(U2, U1);
    // ---- stresses tau11, tau22 and the effective force ------------------------
    const float2 G = mul2(f2(dU1, dU2), iM);             // (dU1/(h1 dxi1), dU2/(h2 dxi2))
    const float2 tau = mul2(fma2(G, zeta + nu, mul2(f2(G.y, G.x), zeta - nu)), rho);
    const float2 UU = mul2(U, U);                         // (uu, vv)
    const float2 A = add2(fma2(-rho, UU, tau), -csd);     // tau_kk - rho U_k^2 - drho cs2
    // F = F_rest + F_dev with F_rest = -(h2 theta11, h1 theta22) rho0 cs2, the
    // geometric force of the rest state; only F_dev is stored
    const float2 Fdev = mul2(fma2(A, T, f2(FL1 + p.fext1, FL2 + p.fext2)), Ms);
    const float2 Fr = mul2(mul2(T, -p.rho0 * cs2), Ms);
    const float2 F = add2(Fdev, Fr);
    F1dev = Fdev.x;
    F2dev = Fdev.y;
    // ---- normal-gradient corrections (Eqs. 82-85 regrouped as in collide) ----
    const float2 RS = mul2(Ms, iM);                        // (r, s) = (h2/h1, h1/h2)
    const float2 R12 = mul2(RS, iM);                       // (h2/h1^2, h1/h2^2)
    const float uv = U1 * U2;
    const float2 a = mul2(UU, p.gic);                      // (a1, a2)
    const float2 P3 = sub2(fma2(Ms, p.zc, mul2(iMs, -p.zmn)), mul2(R12, fma2(a, 3.f * zeta, f2(p.A3, p.A3))));
    const float2 P4 = sub2(fma2(Ms, p.nc, mul2(iMs, p.zmn)), mul2(R12, fma2(a, 3.f * nu, f2(p.A4, p.A4))));   // (P41, -P42)
    const float2 X = fma2(add2(f2(-a.x, -a.y), 3.f), R12, mul2(Ms, -p.ics2));
    const float2 B = mul2(a, iM);                          // (b1, b2)
    const float2 Y = mul2(mul2(mul2(U, add2(a, 1.f)), RS), mul2(T, 2.f));
    const float2 PD3 = mul2(P3, f2(dU1, dU2)), PD4 = mul2(P4, f2(dU1, dU2));
    const float q3 = fmaf(Y.x + Y.y, zeta, PD3.x + PD3.y);
    const float q4 = fmaf(Y.x - Y.y, nu, PD4.x - PD4.y);
    const float2 V = mul2(U, f2(dr1, dr2));
    const float2 Bs = f2(B.y, B.x);
    const float2 W3 = mul2(V, sub2(X, Bs)), W4 = mul2(V, add2(X, Bs));
    const float n3 = fmaf(-zeta, W3.x + W3.y, rho * q3);
    const float n4 = fmaf(-nu, W4.x - W4.y, rho * q4);
    // ---- central moments c = F(U) P (f - f_rest): two passes of the 1D transform
    const float u = U1, v = U2, nu_ = -u, nv_ = -v;
    float k0[3], k1[3], k2[3];                            // per row e2 = -1, 0, +1
    {
        const float q1 = REF ? fmaf(Fr.x, 0.25f, -ur1) : Fr.x * 0.25f, q2 = Fr.y * 0.25f;
        const float fm[3] = {d[7], d[3] + q1, d[6]};
        const float f0[3] = {d[4] + q2, d[0], d[2] - q2};
        const float fp[3] = {d[8], d[1] - q1, d[5]};
#pragma unroll
        for (int y = 0; y < 3; y++) {
            const float sm_ = fp[y] + fm[y], tm_ = fp[y] - fm[y];
            k0[y] = sm_ + f0[y];
            k1[y] = fmaf(nu_, k0[y], tm_);
            k2[y] = fmaf(nu_, tm_ + k1[y], sm_);
        }
    }
    float c[3][3];                                        // c[m][n]: order m along xi1, n along xi2
    {
        const float *kk[3] = {k0, k1, k2};
#pragma unroll
        for (int m = 0; m < 3; m++) {
            const float sm_ = kk[m][2] + kk[m][0], tm_ = kk[m][2] - kk[m][0];
            c[m][0] = sm_ + kk[m][1];
            c[m][1] = fmaf(nv_, c[m][0], tm_);
            c[m][2] = fmaf(nv_, tm_ + c[m][1], sm_);
        }
    }
    // ---- n^eq - n in the combined basis (rest parts cancelled) ---------------
    const float a0 = h1 * h2 * p.rho0;
    const float2 BC = mul2(RS, p.rho0 * cs2);             // (b0, c0)
    const float2 HM = add2(f2(h1, h2), -1.f);              // (h1 - 1, h2 - 1)
    const float q11 = HM.x * HM.y;
    const float2 Q2 = mul2(mul2(RS, HM), HM);              // (q20, q02)
    const float2 Q3 = mul2(mul2(HM, iM), -q11);            // (q21, q12)
    const float2 E = sub2(fma2(RS, csd, mul2(mul2(Q2, UU), rho)), fma2(UU, a0, f2(c[2][0], c[0][2])));
    const float e2s = E.x + E.y + n3, e2d = E.x - E.y + n4;
    const float e11 = fmaf(rho, q11, -a0) * uv - c[1][1];
    const float2 inner = mul2(fma2(Q3, UU, mul2(mul2(f2(HM.y, HM.x), iM), -cs2)), rho);
    const float2 E3 = sub2(fma2(Us, fma2(UU, a0, BC), mul2(inner, Us)), f2(c[2][1], c[1][2]));   // (e21, e12)
    const float e22 = csd * cs2 - c[2][2] - fmaf(UU.y, BC.x, UU.x * BC.y) - UU.x * UU.y * a0;
    // ---- sources (Eq. cmsourcesGOC) and relaxation ---------------------------
    const float *om = p.om;
    const float2 FU = mul2(mul2(F, U), add2(iM, -1.f));   // (F1 U1 (1/h1 - 1), F2 U2 (1/h2 - 1))
    const float s2s = (FU.x + FU.y) * 2.f, s2d = (FU.x - FU.y) * 2.f;
    const float s11 = fmaf((ih2 - 1.f) * F.x, v, F.y * u * (ih1 - 1.f));
    // k10^eq - k10 = F^{n-1}/2 exactly (definition of U), likewise k01; the
    // first-moment change excludes F_rest, which the change of reference
    // f_ref- -> f_ref+ absorbs
    const float2 om12 = f2(om[1], om[2]);
    const float2 D1 = fma2(f2(F1p, F2p), mul2(om12, 0.5f), mul2(Fdev, fma2(om12, -0.5f, f2(1.f, 1.f))));
    const float2 D2 = fma2(f2(e2s, e2d), f2(om[3], om[4]),
                           mul2(f2(s2s, s2d), fma2(f2(om[3], om[4]), -0.5f, f2(1.f, 1.f))));   // (k2s, k2d)
    const float2 D20 = mul2(f2(D2.x + D2.y, D2.x - D2.y), 0.5f);                               // (D20, D02)
    const float D11 = fmaf(e11, om[5], s11 * (1.f - 0.5f * om[5]));
    const float2 D3 = mul2(E3, f2(om[6], om[7]));          // (D21, D12)
    const float D22 = e22 * om[8];
    // ---- back to populations: o = d + P^-1 F(-U) Delta - (f_ref+ - f_ref-) ----
    // (f_ref+ - f_ref- has raw moments (0, F1r, F2r, 0, ...), taken off in
    // central-moment space as in collide)
    {
        const float uv2 = uv * 2.f;
        const float2 G2 = fma2(mul2(U, 2.f), Fr, D20);                           // (g20, g02)
        const float2 G3 = fma2(-uv2, Fr, fma2(f2(-UU.x, -UU.y), f2(Fr.y, Fr.x), D3));   // (g21, g12)
        const float g[3][3] = {{0.f, D1.y, G2.y},
                               {D1.x, fmaf(v, Fr.x, fmaf(u, Fr.y, D11)), G3.y},
                               {G2.x, G3.x, fmaf(uv2, fmaf(u, Fr.y, v * Fr.x), D22)}};
        float r0[3], rp[3], rn[3];                        // per xi1 order m: rows e2 = 0, +1, -1
#pragma unroll
        for (int m = 0; m < 3; m++) {
            const float m1 = fmaf(v, g[m][0], g[m][1]);
            const float m2 = fmaf(v, g[m][1] + m1, g[m][2]);
            r0[m] = g[m][0] - m2;
            rp[m] = (m1 + m2) * 0.5f;
            rn[m] = (m2 - m1) * 0.5f;
        }
        const float *rows[3] = {r0, rp, rn};
        float o0[3], op[3], on[3];                        // values at e1 = 0, +1, -1 per row
#pragma unroll
        for (int y = 0; y < 3; y++) {
            const float m1 = fmaf(u, rows[y][0], rows[y][1]);
            const float m2 = fmaf(u, rows[y][1] + m1, rows[y][2]);
            o0[y] = rows[y][0] - m2;
            op[y] = (m1 + m2) * 0.5f;
            on[y] = (m2 - m1) * 0.5f;
        }
        o[0] = d[0] + o0[0];
        o[1] = d[1] + op[0];
        o[3] = d[3] + on[0];
        o[2] = d[2] + o0[1];
        o[5] = d[5] + op[1];
        o[6] = d[6] + on[1];
        o[4] = d[4] + o0[2];
        o[8] = d[8] + op[2];
        o[7] = d[7] + on[2];
    }
}

// Phase 2 for the R = Lanes<V>::R nodes (i, j[r]) of one thread, r = 0..R-1
// (one node with V = float, two with V = float2: every arithmetic step below
// runs once for both): the MIE, stresses, forces and the central-moment
// collision from the pulled deviations dn, the stored force of the previous
// step, the fields and their normal derivatives fl[k][r] (k: drho, U1, U2,
// dU1/dxi1, drho/dxi1, dU2/dxi2, drho/dxi2), and the stores.  own[r]: whether
// node r is a lattice node this thread updates.
template <class S, bool MHD, bool CHECKS, class V, bool SRT, int GEOM, class Src>
__device__ __forceinline__ void collide(const StepParams &p, const Src &src, int i, const int (&j)[Lanes<V>::R],
                                        const bool (&own)[Lanes<V>::R], const float (&dn)[Lanes<V>::R][9],
                                        const float (&F1pn)[Lanes<V>::R], const float (&F2pn)[Lanes<V>::R], float h1,
                                        float ih1, const float (&h2n)[Lanes<V>::R], const float (&ih2n)[Lanes<V>::R],
                                        const float (&fl)[7][Lanes<V>::R], const float (&ur1n)[Lanes<V>::R],
                                        const float *th_given = nullptr) {
    // th_given (straight grids, one node per thread): theta11, theta22 of the
    // node, already loaded by the caller
    constexpr int R = Lanes<V>::R;
    constexpr bool REF = Store<S>::scaled && GEOM == 0;   // per-row storage reference
    float th_[R];
#pragma unroll
    for (int r = 0; r < R; r++)   // theta22
        th_[r] = GEOM == 2 ? gm_at(p.gm, p.plane, p.pitch, 5, i, own[r] ? j[r] : j[0])
                           : (GEOM ? 0.f : (th_given ? th_given[1] : p.ax2.th[own[r] ? j[r] : j[0]]));
    const V drho = pack<V>(fl[0]), U1 = pack<V>(fl[1]), U2 = pack<V>(fl[2]);
    const V dU1 = pack<V>(fl[3]), dr1 = pack<V>(fl[4]), dU2 = pack<V>(fl[5]), dr2 = pack<V>(fl[6]);
    const V t22 = pack<V>(th_);
    const V h2 = pack<V>(h2n), ih2 = pack<V>(ih2n), F1p = pack<V>(F1pn), F2p = pack<V>(F2pn);
    static_assert(GEOM != 2 || R == 1, "the node-table metric runs one node per thread");
    const float t11 = GEOM == 2 ? gm_at(p.gm, p.plane, p.pitch, 2, i, j[0]) : (th_given ? th_given[0] : p.ax1.th[i]);
    V d[9];
#pragma unroll
    for (int a = 0; a < 9; a++) {
        float t[R];
#pragma unroll
        for (int r = 0; r < R; r++) t[r] = dn[r][a];
        d[a] = pack<V>(t);
    }
    const V rho = drho + p.rho0;
    const V H = h2 * h1, iH = ih2 * ih1;
    const float cs2 = p.cs2;
    long long idx[R];
#pragma unroll
    for (int r = 0; r < R; r++) idx[r] = (long long)j[r] * p.pitch + i;
    // random streams of the stochastic rounding (16-bit storage), one per node
    const bool sr = Store<S>::scaled && p.sr;
    uint32_t rng[R];
    {
        const uint32_t step = sr ? *p.seed_rd : 0u;
#pragma unroll
        for (int r = 0; r < R; r++)
            rng[r] = sr ? node_seed((uint32_t)(idx[r] + (long long)p.seed_row0 * p.pitch), step) : 0u;
    }
    V FL1 = bc<V>(0.f), FL2 = bc<V>(0.f), B1 = bc<V>(0.f), B2 = bc<V>(0.f);
    // theta12, theta21 of curvilinear grids (the column metric has theta12 = 0)
    float t21 = 0.f, t12 = 0.f;
    if constexpr (GEOM == 2) {
        t12 = gm_at(p.gm, p.plane, p.pitch, 3, i, j[0]);
        t21 = gm_at(p.gm, p.plane, p.pitch, 4, i, j[0]);
    } else if constexpr (GEOM == 1) {
        t21 = curv_t21(p.ax1, p.nx, i);
    }

    // ---- MIE (Appendix G): local dB, J3, Lorentz force, SRT collision -------
    if constexpr (MHD && GEOM == 0 && R == 1) {
        // The same MIE update for one node on a straight grid with the two
        // field components c = 0, 1 as the lanes of packed FP32 pairs (every
        // formula below is the same for both components).
        S *gout = static_cast<S *>(p.gout);
        float t[2][5];
#pragma unroll
        for (int c = 0; c < 2; c++) pull_mie<CHECKS, 0, REF>(p, src, i, j[0], h1, h2n[0], c, t[c]);
        float2 GD[5];
#pragma unroll
        for (int a = 0; a < 5; a++) GD[a] = f2(t[0][a], t[1][a]);
        // h1 h2 B = sum g (Eq. 13_C, Y = 0 on straight grids); sum g_ref- = H B_rest
        const float2 GMOV = add2(add2(GD[1], GD[3]), add2(GD[2], GD[4]));   // the four moving links
        const float2 GSUM = add2(GD[0], GMOV);
        const float2 DBC = mul2(GSUM, iH);
        B1 = DBC.x + bref<REF>(p, 0, j[0]);
        B2 = DBC.y + bref<REF>(p, 1, j[0]);
        // A_cd = U_d B_c - B_d U_c (Eq. 2_C): (A1[0], A1[1]) = (0, A12), (A2[0], A2[1]) = (-A12, 0)
        const float A12 = U1 * B2 - B1 * U2;
        const float2 A1 = f2(0.f, A12), A2 = f2(-A12, 0.f);
        // Eqs. gradB1/gradB2 with Lambda^(1) = sum e (g - g^eq(0))
        const float k1 = rcpv(fmaf(h2 * ih1, p.taum - 0.5f, H * 0.5f) * p.csm2);
        const float k2 = rcpv(fmaf(h1 * ih2, p.taum - 0.5f, H * 0.5f) * p.csm2);
        const float m1 = H * (0.5f * p.csm2 * h1 * t11), m2 = H * h2 * t22 * (0.5f * p.csm2);
        const float2 DB1 = mul2(fma2(DBC, m1, fma2(A1, -h2, sub2(GD[1], GD[3]))), -k1);
        const float2 DB2 = mul2(fma2(DBC, m2, fma2(A2, -h1, sub2(GD[2], GD[4]))), -k2);
        // current density (Eq. currentdensity-GOC) and Lorentz force (Eq. Lorentzforce-GOC)
        const float J3 = iH * (h2 * DB1.y - DB2.x * h1) * p.imum;
        FL1 = -J3 * B2;
        FL2 = J3 * B1;
        // SRT collision (Eq. 12_C) written as in the general form below
        const float e1c = (H - h2 * ih1) * p.eta, e2c = (H - h1 * ih2) * p.eta;
        const float m1e = H * (p.eta * h1 * t11), m2e = H * h2 * t22 * p.eta;
        const float2 X1 = mul2(fma2(A1, h2, fma2(DB1, e1c, mul2(DBC, m1e))), p.icsm2);
        const float2 X2 = mul2(fma2(A2, h1, fma2(DB2, e2c, mul2(DBC, m2e))), p.icsm2);
        float2 Geq[5];
        Geq[1] = mul2(add2(GSUM, X1), p.W1);
        Geq[2] = mul2(add2(GSUM, X2), p.W1);
        Geq[3] = mul2(sub2(GSUM, X1), p.W1);
        Geq[4] = mul2(sub2(GSUM, X2), p.W1);
        const float2 Q0 = sub2(GMOV, add2(add2(Geq[1], Geq[3]), add2(Geq[2], Geq[4])));   // g^eq_0 - g_0
        float2 GT[5];
        GT[0] = fma2(Q0, p.itaum, GD[0]);
#pragma unroll
        for (int a = 1; a < 5; a++) GT[a] = fma2(sub2(Geq[a], GD[a]), p.itaum, GD[a]);
        if (own[0]) {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                S *go = gout + c * 5 * p.plane + idx[0];
                float gt[5];
#pragma unroll
                for (int a = 0; a < 5; a++) gt[a] = c ? GT[a].y : GT[a].x;
                if constexpr (Store<S>::scaled && InPlaceSrc<Src>::value) {   // in place: slots of the layout
                    const float is = p.isg;
                    S *gs[5];
#pragma unroll
                    for (int a = 0; a < 5; a++) gs[a] = gout + out_slot_g(src, p, c, a, i, j[0], idx[0]);
                    put2<S>(gs[0], gs[1], gt[0] * is, gt[1] * is, sr, rng[0]);
                    put2<S>(gs[2], gs[3], gt[2] * is, gt[3] * is, sr, rng[0]);
                    put2<S>(gs[4], static_cast<S *>(nullptr), gt[4] * is, 0.f, sr, rng[0]);
                } else if constexpr (Store<S>::scaled) {   // pairs through one conversion each
                    const float is = p.isg;
                    const long long pl = p.plane;
                    put2<S>(go, go + pl, gt[0] * is, gt[1] * is, sr, rng[0]);
                    put2<S>(go + 2 * pl, go + 3 * pl, gt[2] * is, gt[3] * is, sr, rng[0]);
                    put2<S>(go + 4 * pl, static_cast<S *>(nullptr), gt[4] * is, 0.f, sr, rng[0]);
                } else if constexpr (InPlaceSrc<Src>::value) {   // (in-place lattices: slots of their layout)
#pragma unroll
                    for (int a = 0; a < 5; a++) put<S>(gout + out_slot_g(src, p, c, a, i, j[0], idx[0]), gt[a], sr, rng[0]);
                } else {
#pragma unroll
                    for (int a = 0; a < 5; a++) put<S>(go + a * p.plane, gt[a], sr, rng[0]);
                }
            }
        }
    } else if constexpr (MHD) {
        S *gout = static_cast<S *>(p.gout);
        V gd[2][5], dBc[2], dB1[2], dB2[2], gsum[2], gmov[2];
#pragma unroll
        for (int c = 0; c < 2; c++) {
            float t[R][5];
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (own[r]) pull_mie<CHECKS, GEOM, REF>(p, src, i, j[r], h1, h2n[r], c, t[r]);
                else {
#pragma unroll
                    for (int a = 0; a < 5; a++) t[r][a] = 0.f;
                }
            }
#pragma unroll
            for (int a = 0; a < 5; a++) {
                float u_[R];
#pragma unroll
                for (int r = 0; r < R; r++) u_[r] = t[r][a];
                gd[c][a] = pack<V>(u_);
            }
            // h1 h2 B = sum g - Y/2 (Eq. 13_C; Y = 0 on straight grids); sum g_ref- = H B_rest
            gmov[c] = (gd[c][1] + gd[c][3]) + (gd[c][2] + gd[c][4]);   // the four moving links
            gsum[c] = gd[c][0] + gmov[c];
            dBc[c] = gsum[c] * iH;
        }
        if constexpr (GEOM) {
            // curvilinear grids (B_rest = 0): Y_1 = H theta12 (U2 B1 - U1 B2),
            // Y_2 = H theta21 (U1 B2 - U2 B1) (Eq. 6ab_C) are linear in B, so
            // B = sum g / H - Y / (2 H) is a 2 x 2 solve at the node
            const V a11 = fmav(U2, 0.5f * t12, bc<V>(1.f)), a12 = U1 * (-0.5f * t12);
            const V a21 = U2 * (-0.5f * t21), a22 = fmav(U1, 0.5f * t21, bc<V>(1.f));
            const V idet = rcpv(a11 * a22 - a12 * a21);
            const V s0 = dBc[0], s1 = dBc[1];
            dBc[0] = (s0 * a22 - a12 * s1) * idet;
            dBc[1] = (a11 * s1 - a21 * s0) * idet;
        }
        {
            float b0_[R], b1_[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int jr = own[r] ? j[r] : j[0];
                b0_[r] = bref<REF>(p, 0, jr);
                b1_[r] = bref<REF>(p, 1, jr);
            }
            B1 = dBc[0] + pack<V>(b0_);
            B2 = dBc[1] + pack<V>(b1_);
        }
        // A_cd = U_d B_c - B_d U_c (Eq. 2_C): A_11 = A_22 = 0, A_21 = -A_12
        const V A12 = U1 * B2 - B1 * U2;
        const V A1[2] = {bc<V>(0.f), A12}, A2[2] = {bc<V>(0.f) - A12, bc<V>(0.f)};
        // Eqs. gradB1/gradB2 with Lambda^(1) = sum e (g - g^eq(0)) (Eqs.
        // firstvelmomenttensor1/2); the rest-state moment M of g_ref- cancels
        // against the B_rest part of the curvature term.
        const V k1 = rcpv(fmav(h2 * ih1, p.taum - 0.5f, H * 0.5f) * p.csm2);
        const V k2 = rcpv(fmav(h1 * ih2, p.taum - 0.5f, H * 0.5f) * p.csm2);
        // (theta11 + theta21, theta22 + theta12 on curvilinear grids)
        const V m1 = H * (0.5f * p.csm2 * h1 * (GEOM ? t11 + t21 : t11)), m2 = H * h2 * t22 * (0.5f * p.csm2);
        const V m2c = GEOM ? fmav(H * h2, 0.5f * p.csm2 * t12, m2) : m2;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const V L1 = fmav(m1, dBc[c], (gd[c][1] - gd[c][3]) - h2 * A1[c]);
            const V L2 = fmav(m2c, dBc[c], (gd[c][2] - gd[c][4]) - A2[c] * h1);
            dB1[c] = bc<V>(0.f) - L1 * k1;
            dB2[c] = bc<V>(0.f) - L2 * k2;
        }
        // current density (Eq. currentdensity-GOC) and Lorentz force (Eq. Lorentzforce-GOC)
        V J3 = iH * (h2 * dB1[1] - dB2[0] * h1) * p.imum;
        if constexpr (GEOM) J3 = fmav(fmav(B2, t21, B1 * (-t12)), p.imum, J3);   // + (B2 theta21 - B1 theta12)/mu
        FL1 = bc<V>(0.f) - J3 * B2;
        FL2 = J3 * B1;
        // SRT collision (Eq. 12_C, S = 0 on straight grids) with g^eq of
        // Eq. EDF-MIE-base plus the correction of Eq. 42_C, written as
        // g~ = g + (g^eq - g)/tau_m + S.  Relative to the references: g^eq -
        // g_ref- without the B_rest curvature part, which cancels with the change
        // g_ref- -> g_ref+.  The zeroth moment of g^eq is H B = sum g - Y/2 by
        // construction (the rest link takes H B minus the other four), so the
        // collision moves sum g by exactly -Y (Eq. 8a_C with its weight) up to
        // rounding; with the FP32 weights W0 + 4 W1 != 1 and a separate
        // 1 - 1/tau_m, B drifted by a fixed relative amount every step.  The
        // rest link (g_0 ~ H B, nearly all of the field) is updated by g^eq_0 -
        // g_0 = (sum of the moving links - Y/2) - (their g^eq), formed from the
        // small moving-link values only: near a steady state it is then close to
        // zero and leaves g_0 unchanged, where forming it from a sum that holds
        // g_0 itself repeated the same rounding of g_0 every step (a drift of
        // about one FP32 unit of B per step).
        const V e1c = (H - h2 * ih1) * p.eta, e2c = (H - h1 * ih2) * p.eta;
        const V m1e = H * (p.eta * h1 * (GEOM ? t11 + t21 : t11)), m2e = GEOM ? H * h2 * ((t22 + t12) * p.eta) : H * h2 * t22 * p.eta;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const V x1 = fmav(h2, A1[c], fmav(e1c, dB1[c], m1e * dBc[c])) * p.icsm2;
            const V x2 = fmav(h1, A2[c], fmav(e2c, dB2[c], m2e * dBc[c])) * p.icsm2;
            V base = gsum[c], mov = gmov[c];                   // H (B - B_rest) = sum g - Y/2
            V ys = bc<V>(0.f);
            if constexpr (GEOM) {   // source S_a = -W_a Y_c (Eq. 8a_C), weight (1 - 1/(2 tau_m)) in Eq. 12_C
                const V Y = c == 0 ? H * t12 * A2[0] : H * t21 * A1[1];
                base = fmav(Y, -0.5f, base);
                mov = fmav(Y, -0.5f, mov);
                ys = Y * (0.5f * p.itaum - 1.f);
            }
            V Geq[5];
            Geq[1] = (base + x1) * p.W1;
            Geq[2] = (base + x2) * p.W1;
            Geq[3] = (base - x1) * p.W1;
            Geq[4] = (base - x2) * p.W1;
            const V q0 = mov - ((Geq[1] + Geq[3]) + (Geq[2] + Geq[4]));   // g^eq_0 - g_0
            V Sa[5];
            if constexpr (GEOM) {
                const V s1 = ys * p.W1;
                Sa[1] = Sa[2] = Sa[3] = Sa[4] = s1;
                Sa[0] = fmav(s1, -4.f, ys);
            }
            V gt[5];
#pragma unroll
            for (int a = 0; a < 5; a++) {
                gt[a] = fmav(a == 0 ? q0 : Geq[a] - gd[c][a], p.itaum, gd[c][a]);
                if constexpr (GEOM) gt[a] = gt[a] + Sa[a];
            }
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!own[r]) continue;
                S *go = gout + c * 5 * p.plane + idx[r];
                if constexpr (Store<S>::scaled) {   // pairs through one conversion each
                    const float is = p.isg;
                    const long long pl = p.plane;
                    put2<S>(go, go + pl, lane(gt[0], r) * is, lane(gt[1], r) * is, sr, rng[r]);
                    put2<S>(go + 2 * pl, go + 3 * pl, lane(gt[2], r) * is, lane(gt[3], r) * is, sr, rng[r]);
                    put2<S>(go + 4 * pl, static_cast<S *>(nullptr), lane(gt[4], r) * is, 0.f, sr, rng[r]);
                } else {
#pragma unroll
                    for (int a = 0; a < 5; a++) put<S>(go + a * p.plane, scl<S>(lane(gt[a], r), p.isg), sr, rng[r]);
                }
            }
        }
    }

    V o[9], F1dev, F2dev;
    if constexpr (GEOM == 0 && !SRT && R == 1) {   // straight grid, central moments, one node per thread
        collide_straight<REF>(p, d, drho, U1, U2, dU1, dr1, dU2, dr2, h1, ih1, t11, h2, ih2, t22, F1p, F2p, FL1,
                              FL2, ur1n[0], o, F1dev, F2dev);
    } else {
    // ---- stresses and effective force (straight grid, Appendix B (i)) -------
    const float zeta = p.zeta, nu = p.nu;
    const V g1d = dU1 * ih1, g2d = dU2 * ih2;             // dU1/(h1 dxi1), dU2/(h2 dxi2)
    V tau11 = rho * fmav(g1d, zeta + nu, g2d * (zeta - nu));
    V tau22 = rho * fmav(g2d, zeta + nu, g1d * (zeta - nu));
    // F = F_rest + F_dev, F_rest = -(h2, h1) rho0 cs2 (theta11, theta22) is the
    // geometric force of the rest state; only F_dev is stored.
    V F1r, F2r, tc11 = bc<V>(0.f), tc22 = bc<V>(0.f);
    if constexpr (GEOM) {
        // curvilinear grids (theta12, theta21; the column metric has theta12 =
        // theta22 = 0): tau^c (Eq. tauc), the full effective force (Eqs.
        // bodyforce1/2) and the local shear stress of Appendix A; F_rest =
        // (h2 (theta21 - theta11), h1 (theta12 - theta22)) rho0 cs2
        tc11 = rho * fmav(U2, (zeta + nu) * t12, U1 * ((zeta - nu) * t21));
        tc22 = rho * fmav(U1, (zeta + nu) * t21, U2 * ((zeta - nu) * t12));
        tau11 = tau11 + tc11;
        tau22 = tau22 + tc22;
        const V csd_ = drho * cs2;
        const V A1 = tau11 - rho * (U1 * U1) - csd_, A2 = tau22 - rho * (U2 * U2) - csd_;
        const V ruv2 = rho * U1 * U2 * 2.f;
        const V Ft1d = h2 * (fmav(A1, t11, FL1 + p.fext1) - A2 * t21 - ruv2 * t12);
        const V Ft2d = h1 * (fmav(A2, t22, FL2 + p.fext2) - A1 * t12 - ruv2 * t21);
        F1r = h2 * ((t21 - t11) * p.rho0 * cs2);
        F2r = h1 * (t12 - t22) * (p.rho0 * cs2);
        const V k11 = d[5] - d[6] + d[7] - d[8];          // raw k11 of f (f_ref- has none)
        const float c5 = 1.f - 0.5f * p.om[5];
        const V tau12 = (bc<V>(0.f) - c5) *
                        (k11 + ((Ft1d + F1r) * U2 * ih2 + (Ft2d + F2r) * U1 * ih1) * 0.5f - rho * U1 * U2) *
                        rcpv(fmav(U1, c5 * t21, fmav(U2, c5 * t12, bc<V>(1.f))));
        F1dev = fmav(tau12, 2.f * t12 * h2, Ft1d);
        F2dev = fmav(tau12, 2.f * t21 * h1, Ft2d);
    } else {
        F1dev = h2 * fmav(tau11 - rho * (U1 * U1) - drho * cs2, t11, FL1 + p.fext1);
        F2dev = fmav(tau22 - rho * (U2 * U2) - drho * cs2, t22, FL2 + p.fext2) * h1;
        F1r = h2 * (-p.rho0 * cs2 * t11);
        F2r = t22 * (-p.rho0 * cs2 * h1);
    }
    const V F1 = F1dev + F1r;
    const V F2 = F2dev + F2r;

    // ---- normal-gradient corrections (Eqs. 82-85; theta12 = theta21 = 0) -----
    // The coefficients D3k, D4k, C3, C4 regrouped: with a1 = gi U1^2/cs2,
    // a2 = gi U2^2/cs2, r1 = h2/h1^2, s2 = h1/h2^2,
    //   D31 = rho [zeta h2/cs2 - (zeta-nu)/h2 - r1 (2 zeta + nu + 3 zeta a1)],
    //   D41 = rho [nu h2/cs2 + (zeta-nu)/h2 - r1 (zeta + 2 nu + 3 nu a1)],
    //   D33 = -zeta U1 (X1 - a2/h2), D43 = -nu U1 (X1 + a2/h2), X1 = (3 - a1) r1 - h2/cs2,
    // and the mirror images for D32, D42, D34, D44.
    const V r = h2 * ih1, s = ih2 * h1;                   // h2/h1, h1/h2
    const V r1 = r * ih1, s2 = s * ih2;                   // h2/h1^2, h1/h2^2
    const V uu = U1 * U1, vv = U2 * U2, uv = U1 * U2;
    const V a1 = uu * p.gic, a2 = vv * p.gic;
    V n3, n4;
    {
        const float zmn = p.zmn;
        const V P31 = fmav(h2, p.zc, ih2 * (-zmn)) - r1 * fmav(a1, 3.f * zeta, p.A3);
        const V P32 = bc<V>(p.zc * h1 - zmn * ih1) - s2 * fmav(a2, 3.f * zeta, p.A3);
        const V P41 = fmav(h2, p.nc, ih2 * zmn) - r1 * fmav(a1, 3.f * nu, p.A4);
        const V P42 = s2 * fmav(a2, 3.f * nu, p.A4) - (p.nc * h1 + zmn * ih1);
        const V X1 = fmav(3.f - a1, r1, h2 * (-p.ics2)), X2 = fmav(3.f - a2, s2, bc<V>(-h1 * p.ics2));
        const V b2 = a2 * ih2, b1 = a1 * ih1;
        const V Y1 = U1 * (a1 + 1.f) * r * (2.f * t11), Y2 = U2 * (a2 + 1.f) * s * t22 * 2.f;
        const V q3 = fmav(Y1 + Y2, zeta, fmav(P31, dU1, P32 * dU2));
        const V q4 = fmav(Y1 - Y2, nu, fmav(P41, dU1, P42 * dU2));
        n3 = rho * q3 - U1 * (X1 - b2) * dr1 * zeta - U2 * (X2 - b1) * dr2 * zeta;
        n4 = rho * q4 - U1 * (X1 + b2) * dr1 * nu + U2 * (X2 + b1) * dr2 * nu;
        if constexpr (GEOM) {   // tau^c and the theta21, theta12 parts of C3, C4
            const V Hc = H * p.ics2, a13 = fmav(a1, r, 3.f * r), a23 = fmav(a2, s, 3.f * s);   // (3 + a) h2/h1, h1/h2
            n3 = n3 - fmav(r, tc11, s * tc22) - rho * U1 * (t21 * zeta) * (a13 + s * 2.f - Hc)
                 - rho * U2 * (t12 * zeta) * (a23 + r * 2.f - Hc);
            n4 = n4 - (r * tc11 - s * tc22) - rho * U1 * (t21 * nu) * (a13 - s * 2.f - Hc)
                 - rho * U2 * (t12 * nu) * (r * 2.f + Hc - a23);
        }
    }

    if constexpr (SRT) {
        raw_relax<REF, V>(p, d, o, rho, drho, U1, U2, ih2, ih1, r, s, uu, vv, uv, n3, n4, F1, F2, F1dev, F2dev, F1p,
                          F2p, F1r, F2r, pack<V>(ur1n));
    } else {
    // ---- central moments c = F(U) P (f - f_rest) -----------------------------
    // f - f_rest = d + (f_ref- - f_rest), the latter -F_rest/4 (e . unit) on
    // links 1..4.  Central moments about (U1, U2) by two passes of the 1D
    // transform (values at e = -1, 0, +1 -> moments of orders 0, 1, 2 about the
    // velocity component): first along xi1 within each row of equal e2, then
    // along xi2 for each xi1 order.
    const V u = U1, v = U2;
    const V nu_ = bc<V>(0.f) - u, nv_ = bc<V>(0.f) - v;
    V k0[3], k1[3], k2[3];                                // per row e2 = -1, 0, +1
    {
        // (REF: f_ref- - f_rest also holds +-ur1 on links 1 and 3)
        const V q1 = REF ? fmav(F1r, 0.25f, bc<V>(0.f) - pack<V>(ur1n)) : F1r * 0.25f, q2 = F2r * 0.25f;
        const V fm[3] = {d[7], d[3] + q1, d[6]};
        const V f0[3] = {d[4] + q2, d[0], d[2] - q2};
        const V fp[3] = {d[8], d[1] - q1, d[5]};
#pragma unroll
        for (int y = 0; y < 3; y++) {
            const V sm_ = fp[y] + fm[y], tm_ = fp[y] - fm[y];
            k0[y] = sm_ + f0[y];
            k1[y] = fmav(nu_, k0[y], tm_);
            k2[y] = fmav(nu_, tm_ + k1[y], sm_);
        }
    }
    V c[3][3];                                            // c[m][n]: order m along xi1, n along xi2
    {
        const V *kk[3] = {k0, k1, k2};
#pragma unroll
        for (int m = 0; m < 3; m++) {
            const V sm_ = kk[m][2] + kk[m][0], tm_ = kk[m][2] - kk[m][0];
            c[m][0] = sm_ + kk[m][1];
            c[m][1] = fmav(nv_, c[m][0], tm_);
            c[m][2] = fmav(nv_, tm_ + c[m][1], sm_);
        }
    }
    const V c20 = c[2][0], c02 = c[0][2], c11 = c[1][1], c21 = c[2][1], c12 = c[1][2], c22 = c[2][2];

    // ---- n^eq - n in the combined basis (rest parts cancelled) ---------------
    const V a0 = H * p.rho0, b0 = r * (p.rho0 * cs2), c0 = s * (p.rho0 * cs2);
    const float hm1 = h1 - 1.f;
    const V hm2 = h2 - 1.f;
    const V q20 = r * (hm1 * hm1), q02 = s * hm2 * hm2, q11 = hm2 * hm1;
    const V q21 = hm2 * (-hm1 * hm1 * ih1), q12 = hm2 * hm2 * ih2 * (-hm1);
    const V rq20 = rho * q20 * uu, rq02 = rho * q02 * vv;
    const V csd = drho * cs2;
    const V e2s = fmav(r + s, csd, rq20 + rq02 + n3) - (c20 + c02) - (uu + vv) * a0;
    const V e2d = fmav(r - s, csd, rq20 - rq02 + n4) - (c20 - c02) - (uu - vv) * a0;
    const V e11 = (rho * q11 - a0) * uv - c11;
    const V e21 = fmav(v, b0 + (uu * a0), (rho * q21 * uu + rho * (1.f - h2) * ih1 * cs2) * v) - c21;
    const V e12 = fmav(u, c0 + (vv * a0), (rho * q12 * vv + rho * (1.f - h1) * ih2 * cs2) * u) - c12;
    const V e22 = csd * cs2 - c22 - vv * b0 - uu * c0 - uu * vv * a0;

    // ---- sources (Eq. cmsourcesGOC) and relaxation ---------------------------
    const float w1 = ih1 - 1.f;
    const V w2 = ih2 - 1.f;
    const V fu = F1 * u * w1, fv = F2 * v * w2;
    const V s2s = (fu + fv) * 2.f;
    const V s2d = (fu - fv) * 2.f;
    const V s11 = fmav(w2 * F1, v, F2 * u * w1);
    const float *om = p.om;
    // k10^eq - k10 = F^{n-1}/2 exactly (definition of U), likewise k01.
    // D10d excludes F_rest, which the change of reference f_ref- -> f_ref+ absorbs.
    const V D10d = fmav(F1p, 0.5f * om[1], F1dev * (1.f - 0.5f * om[1]));
    const V D01d = fmav(F2p, 0.5f * om[2], F2dev * (1.f - 0.5f * om[2]));
    const V D2s = fmav(e2s, om[3], s2s * (1.f - 0.5f * om[3]));
    const V D2d = fmav(e2d, om[4], s2d * (1.f - 0.5f * om[4]));
    const V D20 = (D2s + D2d) * 0.5f, D02 = (D2s - D2d) * 0.5f;
    const V D11 = fmav(e11, om[5], s11 * (1.f - 0.5f * om[5]));
    const V D21 = e21 * om[6], D12 = e12 * om[7], D22 = e22 * om[8];

    // ---- back to populations: o = d + P^-1 F(-U) Delta - (f_ref+ - f_ref-) ----
    // f_ref+ - f_ref- has raw moments r = (0, F1r, F2r, 0, ...); it is taken off
    // in central-moment space, Delta - F(U) r, whose terms are all small (first
    // moments D10d, D01d, higher ones shifted by O(U F_rest)).  The inverse
    // transform runs the 1D passes in reverse order: along xi2, then xi1; for
    // central moments (c0, c1, c2) about w, the raw moments are m1 = c1 + w c0,
    // m2 = c2 + 2 w c1 + w^2 c0 and the values at e = 0, +1, -1 are c0 - m2,
    // (m1 + m2)/2, (m2 - m1)/2.
    {
        const V uv2 = uv * 2.f;
        const V g[3][3] = {
            {bc<V>(0.f), D01d, fmav(v * 2.f, F2r, D02)},
            {D10d, fmav(v, F1r, fmav(u, F2r, D11)), D12 - vv * F1r - uv2 * F2r},
            {fmav(u * 2.f, F1r, D20), D21 - uu * F2r - uv2 * F1r, fmav(uv2, fmav(u, F2r, v * F1r), D22)}};
        V r0[3], rp[3], rn[3];                            // per xi1 order m: rows e2 = 0, +1, -1
#pragma unroll
        for (int m = 0; m < 3; m++) {
            const V m1 = fmav(v, g[m][0], g[m][1]);
            const V m2 = fmav(v, g[m][1] + m1, g[m][2]);
            r0[m] = g[m][0] - m2;
            rp[m] = (m1 + m2) * 0.5f;
            rn[m] = (m2 - m1) * 0.5f;
        }
        // rows e2 = 0 (links 3, 0, 1), +1 (6, 2, 5), -1 (7, 4, 8)
        const V *rows[3] = {r0, rp, rn};
        V o0[3], op[3], on[3];                            // values at e1 = 0, +1, -1 per row
#pragma unroll
        for (int y = 0; y < 3; y++) {
            const V m1 = fmav(u, rows[y][0], rows[y][1]);
            const V m2 = fmav(u, rows[y][1] + m1, rows[y][2]);
            o0[y] = rows[y][0] - m2;
            op[y] = (m1 + m2) * 0.5f;
            on[y] = (m2 - m1) * 0.5f;
        }
        o[0] = d[0] + o0[0];
        o[1] = d[1] + op[0];
        o[3] = d[3] + on[0];
        o[2] = d[2] + o0[1];
        o[5] = d[5] + op[1];
        o[6] = d[6] + on[1];
        o[4] = d[4] + o0[2];
        o[8] = d[8] + op[2];
        o[7] = d[7] + on[2];
    }
    }   // central-moment path
    }   // general collision
    S *fout = static_cast<S *>(p.fout);
    S *Fout = static_cast<S *>(p.Fout);
#pragma unroll
    for (int q = 0; q < R; q++) {
        if (!own[q]) continue;
        if constexpr (Store<S>::scaled && InPlaceSrc<Src>::value) {   // in place: slots of the layout
            S *Fo = Fout + idx[q];
            const float is = p.isf;
            S *fs[9];
#pragma unroll
            for (int a = 0; a < 9; a++) fs[a] = fout + out_slot(src, p, a, i, j[q], idx[q]);
#pragma unroll
            for (int a = 0; a < 8; a += 2)
                put2<S>(fs[a], fs[a + 1], lane(o[a], q) * is, lane(o[a + 1], q) * is, sr, rng[q]);
            put2<S>(fs[8], Fo, lane(o[8], q) * is, lane(F1dev, q) * p.isF, sr, rng[q]);
            put2<S>(Fo + p.plane, static_cast<S *>(nullptr), lane(F2dev, q) * p.isF, 0.f, sr, rng[q]);
        } else if constexpr (Store<S>::scaled) {   // pairs through one conversion each
            S *fo = fout + idx[q], *Fo = Fout + idx[q];
            const long long pl = p.plane;
            const float is = p.isf;
#pragma unroll
            for (int a = 0; a < 8; a += 2)
                put2<S>(fo + a * pl, fo + (a + 1) * pl, lane(o[a], q) * is, lane(o[a + 1], q) * is, sr, rng[q]);
            put2<S>(fo + 8 * pl, Fo, lane(o[8], q) * is, lane(F1dev, q) * p.isF, sr, rng[q]);
            put2<S>(Fo + pl, static_cast<S *>(nullptr), lane(F2dev, q) * p.isF, 0.f, sr, rng[q]);
        } else {
            for (int a = 0; a < 9; a++)
                put<S>(fout + out_slot(src, p, a, i, j[q], idx[q]), scl<S>(lane(o[a], q), p.isf), sr, rng[q]);
            put<S>(Fout + idx[q], scl<S>(lane(F1dev, q), p.isF), sr, rng[q]);
            put<S>(Fout + p.plane + idx[q], scl<S>(lane(F2dev, q), p.isF), sr, rng[q]);
        }
        if (p.uout) {
            __stcg(p.uout + idx[q], lane(U1, q));
            __stcg(p.uout + p.plane + idx[q], lane(U2, q));
            __stcg(p.uout + 2 * p.plane + idx[q], lane(B1, q));
            __stcg(p.uout + 3 * p.plane + idx[q], lane(B2, q));
        }
    }
    // divergence (non-positive density or non-finite velocity): the thread
    // that sees it sets the status word unless it is set already (no vote and
    // nothing kept across tiles: the test costs a compare and a branch)
#pragma unroll
    for (int q = 0; q < R; q++) {
        const float rq = lane(rho, q), uq = fabsf(lane(U1, q)) + fabsf(lane(U2, q));
        if (own[q] && !(rq > 0.f && uq < 1e30f) && p.flag && *((volatile int *)p.flag) == 0) atomicExch(p.flag, 1);
    }
}

// Normal derivatives of the fields from the tile's field arrays (second
// order: central, one-sided at the first and last node of a wall axis), then
// the collision.
template <class S, bool MHD, bool CHECKS, class V, bool SRT, int GEOM, class Src>
__device__ __forceinline__ void node_update(const StepParams &p, const Src &src, int i, int tx,
                                            const int (&j)[Lanes<V>::R], const int (&ty)[Lanes<V>::R],
                                            const bool (&own)[Lanes<V>::R], const FieldSmem &sm,
                                            const float (&dn)[Lanes<V>::R][9], const float (&F1pn)[Lanes<V>::R],
                                            const float (&F2pn)[Lanes<V>::R], float h1, float ih1,
                                            const float (&h2n)[Lanes<V>::R], const float (&ih2n)[Lanes<V>::R],
                                            const float (&ur1n)[Lanes<V>::R]) {
    constexpr int R = Lanes<V>::R;
    const int ex = tx + MH;
    float fl[7][R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int ey = ty[r] + MH;
        const float drho = sm.rho[ey][ex], U1 = sm.u1[ey][ex], U2 = sm.u2[ey][ex];
        fl[0][r] = drho;
        fl[1][r] = U1;
        fl[2][r] = U2;
        if (CHECKS) {
            fl[3][r] = dfd(sm.u1[ey][ex - 2], sm.u1[ey][ex - 1], U1, sm.u1[ey][ex + 1], sm.u1[ey][ex + 2], i, p.nx, p.per_x);
            fl[4][r] = dfd(sm.rho[ey][ex - 2], sm.rho[ey][ex - 1], drho, sm.rho[ey][ex + 1], sm.rho[ey][ex + 2], i, p.nx, p.per_x);
            fl[5][r] = dfd(sm.u2[ey - 2][ex], sm.u2[ey - 1][ex], U2, sm.u2[ey + 1][ex], sm.u2[ey + 2][ex], j[r], p.ny, p.per_y);
            fl[6][r] = dfd(sm.rho[ey - 2][ex], sm.rho[ey - 1][ex], drho, sm.rho[ey + 1][ex], sm.rho[ey + 2][ex], j[r], p.ny, p.per_y);
        } else {
            fl[3][r] = 0.5f * (sm.u1[ey][ex + 1] - sm.u1[ey][ex - 1]);
            fl[4][r] = 0.5f * (sm.rho[ey][ex + 1] - sm.rho[ey][ex - 1]);
            fl[5][r] = 0.5f * (sm.u2[ey + 1][ex] - sm.u2[ey - 1][ex]);
            fl[6][r] = 0.5f * (sm.rho[ey + 1][ex] - sm.rho[ey - 1][ex]);
        }
    }
    collide<S, MHD, CHECKS, V, SRT, GEOM>(p, src, i, j, own, dn, F1pn, F2pn, h1, ih1, h2n, ih2n, fl, ur1n);
}

// One tile of one lattice from a given source; KIND 0: interior (no boundary
// logic, fields halo 1), 1: near a boundary (fields halo 2 where inside).
// Each thread pulls its RPT nodes (column i0 + tx, rows ty + r TYT) into
// registers (kept across the barrier for the collision); the ring of halo
// nodes around the tile is shared out over the threads.  Contains a block
// barrier: every thread of the block must call it.  ok: this thread's wait
// for the staged copy succeeded; false (returned by every thread) when any
// thread's wait failed -- the block then leaves.
template <class S, bool MHD, int KIND, bool SRT, int GEOM, class Src>
__device__ __forceinline__ bool tile_compute(const StepParams &p, const Src &src, int i0, int j0, FieldSmem &sm,
                                             bool ok) {
    constexpr bool CHECKS = KIND != 0;
    constexpr bool REF = Store<S>::scaled && GEOM == 0;   // per-row storage reference
    constexpr int W = KIND == 0 ? 1 : MH;                 // halo width of the fields
    constexpr int BAND = W * (TX + 2 * W);                // nodes in the top (or bottom) band
    constexpr int RING = 2 * BAND + 2 * W * TY;
    constexpr int R = RPT;
    using V = typename VecOf<R>::type;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int tx = threadIdx.x;
    const int i = i0 + tx;
    const bool inx = i < p.nx;
    float h1 = 1.f, ih1 = 1.f;
    if (inx && GEOM != 2) {
        h1 = p.ax1.h[i];
        ih1 = p.ax1.ih[i];
    }
    int j[R], ty[R];
    bool own[R];
    float d[R][9], F1p[R], F2p[R], h2[R], ih2[R], ur1[R];
#pragma unroll
    for (int r = 0; r < R; r++) {   // own nodes
        ty[r] = threadIdx.y + r * TYT;
        j[r] = j0 + ty[r];
        own[r] = inx && j[r] < p.ny;
        float drho = 0.f, U1 = 0.f, U2 = 0.f;
        F1p[r] = F2p[r] = 0.f;
        h2[r] = ih2[r] = 1.f;
        ur1[r] = 0.f;
#pragma unroll
        for (int a = 0; a < 9; a++) d[r][a] = 0.f;
        if (own[r]) {
            node_metric<GEOM>(p, i, j[r], h1, h2[r], ih1, ih2[r]);   // (GEOM 2 runs one node per thread)
            if (REF) ur1[r] = GOC_U1R(p, j[r]);
            pull_node<CHECKS, GEOM, REF>(p, src, i, j[r], h1, h2[r], d[r], ur1[r]);
            F1p[r] = src.Fv(0, i, j[r]);
            F2p[r] = src.Fv(1, i, j[r]);
            fields_from<REF>(p, d[r], F1p[r], F2p[r], ih1, ih2[r], drho, U1, U2, ur1[r]);
        } else if (CHECKS) {   // ragged tile: past the last node of a periodic axis sits the wrapped node
            int ii = i, jj = j[r];
            bool in = true;
            if (ii >= p.nx) {
                if (p.per_x) ii = wrapi(ii, p.nx); else in = false;
            }
            if (jj >= p.ny) {
                if (p.per_y) jj = wrapi(jj, p.ny); else in = false;
            }
            if (in) {
                float dd[9], g1, g2, ig1, ig2;
                node_metric<GEOM>(p, ii, jj, g1, g2, ig1, ig2);
                const float u = REF ? GOC_U1R(p, jj) : 0.f;
                pull_node<CHECKS, GEOM, REF>(p, src, ii, jj, g1, g2, dd, u);
                fields_from<REF>(p, dd, src.Fv(0, ii, jj), src.Fv(1, ii, jj), ig1, ig2, drho, U1, U2, u);
            }
        }
        sm.rho[ty[r] + MH][tx + MH] = drho;
        sm.u1[ty[r] + MH][tx + MH] = U1;
        sm.u2[ty[r] + MH][tx + MH] = U2;
    }
    // halo ring: top band, bottom band, left band, right band (taken from the
    // last warp down: warp 0 also stages the next tile)
    for (int q = NT - 1 - tid; q < RING; q += NT) {
        int x, y;
        if (q < 2 * BAND) {
            const int b = q < BAND ? q : q - BAND;
            const int row = b / (TX + 2 * W);
            x = b - row * (TX + 2 * W) - W;
            y = q < BAND ? row - W : TY + row;
        } else {
            const int b = q - 2 * BAND;
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
            float dd[9], g1, g2, ig1, ig2;
            node_metric<GEOM>(p, ii, jj, g1, g2, ig1, ig2);
            const float u = REF ? GOC_U1R(p, jj) : 0.f;
            pull_node<CHECKS, GEOM, REF>(p, src, ii, jj, g1, g2, dd, u);
            fields_from<REF>(p, dd, src.Fv(0, ii, jj), src.Fv(1, ii, jj), ig1, ig2, drho, U1, U2, u);
        }
        sm.rho[y + MH][x + MH] = drho;
        sm.u1[y + MH][x + MH] = U1;
        sm.u2[y + MH][x + MH] = U2;
    }
    if (!__syncthreads_and(ok)) return false;
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; r++) any = any || own[r];
    if (any)
        node_update<S, MHD, CHECKS, V, SRT, GEOM>(p, src, i, tx, j, ty, own, sm, d, F1p, F2p, h1, ih1, h2, ih2, ur1);
    return true;
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

// The three tensor maps of a lattice's input buffers (populations, force, MIE).
struct TileMaps {
    const CUtensorMap *f, *F, *g;
};

template <class S>
__device__ __forceinline__ void issue_tile(const TileMaps &m, int i0, int j0, unsigned char *stage, uint64_t *bar,
                                           bool mhd) {
    using T = Tiling<S>;
    const uint32_t bytes = T::F_BYTES + T::FF_BYTES + (mhd && GOC_MIE_STAGED ? T::G_BYTES : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_3d(stage, m.f, i0 - T::HXS, j0 - HYS, 0, bar);
    tma_load_3d(stage + T::OFF_FF, m.F, i0 - T::HXS, j0 - HYS, 0, bar);
    if (mhd && GOC_MIE_STAGED) tma_load_3d(stage + T::OFF_G, m.g, i0 - T::HXS, j0 - 1, 0, bar);
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

template <class S, bool MHD, bool SRT = false, int GEOM = 0>
__device__ __forceinline__ bool run_tile(const StepParams &p, int kind, int i0, int j0, const unsigned char *stage,
                                         FieldSmem &sm, bool ok) {
    using T = Tiling<S>;
    if (kind == 2) {
        SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin), static_cast<const S *>(p.gin),
                         p.plane, p.pitch, p.sf, p.sF, p.sg};
        return tile_compute<S, MHD, 1, SRT, GEOM>(p, src, i0, j0, sm, ok);
    }
#if GOC_MIE_STAGED
    SrcSmem<S> src{reinterpret_cast<const S *>(stage), reinterpret_cast<const S *>(stage + T::OFF_FF),
                   reinterpret_cast<const S *>(stage + T::OFF_G), i0 - T::HXS, j0 - HYS, j0 - 1,
                   p.sf, p.sF, p.sg};
#else
    SrcSmem<S> src{reinterpret_cast<const S *>(stage), reinterpret_cast<const S *>(stage + T::OFF_FF),
                   static_cast<const S *>(p.gin), i0 - T::HXS, j0 - HYS, j0 - 1, p.sf, p.sF, p.sg, p.plane, p.pitch};
#endif
    if (kind == 0) return tile_compute<S, MHD, 0, SRT, GEOM>(p, src, i0, j0, sm, ok);
    return tile_compute<S, MHD, 1, SRT, GEOM>(p, src, i0, j0, sm, ok);
}

// The tiles of one lattice processed by one block with TMA staging in two
// dynamic shared-memory stages: the copy of the next tile is issued before
// the current one is computed.  Block b starts with tile first = b; the next
// tile is stride + the counter's next value (dynamic order, with ctr) or
// t + stride (static order).  Every thread of the block calls it; the barriers
// must be initialised.
template <class S, bool MHD, bool SRT, int GEOM>
__device__ __forceinline__ void lattice_tiles(const StepParams &p, const TileMaps &m, int *ctr, int first, int stride,
                                              unsigned char *dyn, uint64_t *bars, FieldSmem &sm, int4 *s_item,
                                              bool leader) {
    using T = Tiling<S>;
    constexpr int STAGE = MHD ? T::STAGE_MHD : T::STAGE_NSE;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY, ntiles = ntx * nty;
    // leader: record item t for stage st as (t, i0, j0, kind) and start its copy
    auto take = [&](int st, int t) {
        int4 it = make_int4(t, 0, 0, 0);
        if (t < ntiles) {
            it.y = (t % ntx) * TX;
            it.z = (t / ntx) * TY;
            it.w = tile_kind<S>(p, it.y, it.z);
            if (it.w != 2) {
                fence_proxy_async();   // generic reads of that stage (previous tile) precede the async writes
                issue_tile<S>(m, it.y, it.z, dyn + st * STAGE, &bars[st], MHD);
            }
        }
        s_item[st] = it;
    };
    // leader, dynamic queue, NSE: the counter value of the item after the
    // next one is fetched one tile ahead, so the atomic's round trip overlaps
    // a tile.  With the MIE (fewer, longer tiles per block) the reservation
    // would hold back an item a faster block could take.
    constexpr bool AHEAD = !MHD;
    int pend = 0;
    if (leader) {
        if (ctr && AHEAD) pend = atomicAdd(ctr, 1);
        take(0, first);
    }
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    int stage = 0;
    for (;;) {
        const int4 it = s_item[stage];
        const int t = it.x;
        if (t >= ntiles) break;   // uniform: every thread reads the same shared value
        if (leader) {
            int nt = t + stride;
            if (ctr && AHEAD) {
                nt = stride + pend;
                pend = atomicAdd(ctr, 1);
            } else if (ctr) {
                nt = stride + atomicAdd(ctr, 1);
            }
            take(stage ^ 1, nt);
        }
        const int i0 = it.y, j0 = it.z, kind = it.w;
        bool ok = true;   // every thread waits for the copy itself; the fields barrier gathers the outcome
        if (kind != 2) {
            uint32_t &ph = stage ? ph1 : ph0;
            ok = mbar_wait_bounded(&bars[stage], ph, p.flag);
            ph ^= 1;
        }
        if (MHD) {   // with the MIE the block gathers after the copy (measured faster there)
            if (!__syncthreads_and(ok)) return;
        }
        if (!run_tile<S, MHD, SRT, GEOM>(p, kind, i0, j0, dyn + stage * STAGE, sm, ok)) return;   // the block leaves together
        __syncthreads();   // the stage, the field arrays and s_item are reused by the next tile
        stage ^= 1;
    }
}

// Single lattice: persistent blocks take tiles from the lattice's queue.
// SRT (raw): the collision on raw moments -- Appendix D's raw-moment MRT, or
// Appendix F's SRT when every rate is 1/tau -- instead of the central-moment one.
// GEOM: 1 the curvilinear column metric (annular sector; h1, h2, theta11,
// theta21 functions of xi1), 2 the metric given node by node (general
// orthogonal grids), with the theta21 / theta12 terms of the force, tau^c,
// the corrections and the local shear stress (Appendix A) and, with the MIE,
// those of the gradient formula, g^corr and J3 and the source Y (Appendix G).
template <class S, bool MHD, bool SRT = false, int GEOM = 0>
__global__ void __launch_bounds__(NT, MHD ? (GEOM == 0 ? GOC_MIN_BLOCKS_MHD_STRAIGHT : GOC_MIN_BLOCKS_MHD) : GOC_MIN_BLOCKS)
    step_kernel(const __grid_constant__ StepParams p) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ FieldSmem sm;
    __shared__ int4 s_item[2];
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    if (leader) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    griddep_launch_dependents();
    griddep_wait();   // the previous step is complete: its populations may be read and overwritten
    if (leader && blockIdx.x == 0) {
        if (Store<S>::scaled && p.sr) *p.seed_wr = *p.seed_rd + 1u;   // next step's index
        if (p.tctr_next) *p.tctr_next = 0;                                  // next step's tile queue
    }
    const TileMaps m{&p.tm_f, &p.tm_F, &p.tm_g};
    lattice_tiles<S, MHD, SRT, GEOM>(p, m, p.tctr, blockIdx.x, gridDim.x, dyn, bars, sm, s_item, leader);
}

// Many lattices in one launch.  Their parameters travel in the kernel
// parameter space (up to kBatchMax lattices, 28 KB); the tensor maps sit in a
// global array.  Work items are the tiles of all member lattices (item t of
// lattice k for toff[k] <= t < toff[k+1]), handed out dynamically: the block
// leader takes the next item from a global counter while the current one is
// computed (its TMA copy goes into the other stage), so tiles of unequal cost
// (wall tiles, tiles on periodic seams read from global memory) balance out
// over the blocks.  Block b starts with item b; the counter of a step,
// ctr[parity], hands out the items from gridDim.x on; each launch zeroes the
// other counter for the next step.
constexpr int kBatchMax = 32;
struct BatchArgs {
    int n;                          // lattices in this launch
    int toff[kBatchMax + 1];        // first item of each lattice; toff[n] = items
    int parity;                     // this step's counter
    int *ctr;                       // [2] item counters in global memory
    const CUtensorMap *maps;        // [n][3] tensor maps of the input buffers, in global memory
    StepParams p[kBatchMax];        // (their tm_* members are not used)
};

__device__ __forceinline__ int batch_lattice(const BatchArgs &a, int t) {
    int lo = 0, hi = a.n - 1;       // last k with toff[k] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.toff[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// batch_step_kernel: see goc_lean.cuh (straight-grid members take the interior path there)

}  // namespace goc
