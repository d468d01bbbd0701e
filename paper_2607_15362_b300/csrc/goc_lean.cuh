// goc_lean.cuh -- the step kernel for straight grids (h1 = h1(xi1), h2 =
// h2(xi2): every grid of Sec. 6 and 7) with the central-moment collision:
// the same time step as step_kernel<S, MHD, false, 0> (Appendix E Steps 1-7,
// Appendix G with the MIE), organised to spend fewer instructions per node on
// everything around the collision.
//
//   * The metric of a column or a row is one 32-byte record (h, 1/h, theta,
//     the two pull corrections; float4 pairs, two vector loads) instead of
//     five loads from five tables.
//   * Interior tiles (every pull source and the fields halo inside the
//     lattice) take a path whose shared-memory addresses are fixed offsets
//     from one per-thread base, with the ring of halo nodes laid out once per
//     thread; tiles next to a wall or across a periodic seam take the general
//     tile path of goc_step.cuh.
//   * The post-collision values of one node are stored through one 64-bit
//     address per buffer and per-plane offsets kept for the whole launch.
#pragma once

#include "goc_step.cuh"

namespace goc {

// Metric record of node index k along an axis: rec[2k] = (h, 1/h, theta, rm),
// rec[2k + 1] = (rp, dm, dp, 0) (the rows of the per-axis tables, see Axis).
struct AxisRecord {
    float h, ih, th, rm, rp, dm, dp;
};
__device__ __forceinline__ AxisRecord axis_record(const float4 *rec, int k) {
    const float4 a = __ldg(rec + 2 * k), b = __ldg(rec + 2 * k + 1);
    return AxisRecord{a.x, a.y, a.z, a.w, b.x, b.y, b.z};
}

// Pull of the nine deviations arriving at an interior node whose stored value
// of link 0 sits at s (all sources inside the staged box), with the rest-state
// pull corrections of links 1..4 (rm/rp of the node's column and row).
template <class S, int BYS = Tiling<S>::BY>
__device__ __forceinline__ void lean_pull(const S *s, float sf, const AxisRecord &c, const AxisRecord &r,
                                          float d[9]) {
    using T = Tiling<S>;
    constexpr int BX = T::BX, PL = T::BX * BYS;
    d[0] = scl<S>(Store<S>::lds(s), sf);
    d[1] = fmaf(r.h, c.rm, scl<S>(Store<S>::lds(s + PL - 1), sf));            // source (i-1, j)
    d[2] = fmaf(c.h, r.rm, scl<S>(Store<S>::lds(s + 2 * PL - BX), sf));       // (i, j-1)
    d[3] = fmaf(r.h, c.rp, scl<S>(Store<S>::lds(s + 3 * PL + 1), sf));        // (i+1, j)
    d[4] = fmaf(c.h, r.rp, scl<S>(Store<S>::lds(s + 4 * PL + BX), sf));       // (i, j+1)
    d[5] = scl<S>(Store<S>::lds(s + 5 * PL - BX - 1), sf);                    // (i-1, j-1)
    d[6] = scl<S>(Store<S>::lds(s + 6 * PL - BX + 1), sf);                    // (i+1, j-1)
    d[7] = scl<S>(Store<S>::lds(s + 7 * PL + BX + 1), sf);                    // (i+1, j+1)
    d[8] = scl<S>(Store<S>::lds(s + 8 * PL + BX - 1), sf);                    // (i-1, j+1)
}

// One interior tile: the fields of the tile and of its ring (halo of one
// node) from the staged populations, then the collision of each node.  Every
// thread of the block calls it (it contains the fields barrier).  st: the
// stage (populations, then the stored force at Tiling<S>::OFF_FF).
template <class S, bool MHD, bool SEAM = false>
__device__ __forceinline__ bool lean_tile(const StepParams &p, const unsigned char *st, int i0, int j0,
                                          FieldSmem &sm, bool ok) {
    using T = Tiling<S>;
    constexpr bool REF = Store<S>::scaled;                // per-row storage reference (16-bit storage)
    constexpr int BX = T::BX, BAND = TX + 2, RING = 2 * BAND + 2 * TY;
    const S *sf_ = reinterpret_cast<const S *>(st);
    const S *sF_ = reinterpret_cast<const S *>(st + T::OFF_FF);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i = i0 + tx, j = j0 + ty;
    const float4 *rec1 = axis_records(p.ax1, p.nx), *rec2 = axis_records(p.ax2, p.ny);
    const AxisRecord c = axis_record(rec1, i), r = axis_record(rec2, j);
    // own node
    const int so = (ty + HYS) * BX + tx + T::HXS;
    float d[9], drho, U1, U2;
    const float ur1 = REF ? GOC_U1R(p, j) : 0.f;
    lean_pull<S>(sf_ + so, p.sf, c, r, d);
    const float F1p = scl<S>(Store<S>::lds(sF_ + so), p.sF);
    const float F2p = scl<S>(Store<S>::lds(sF_ + T::BX * T::BY + so), p.sF);
    fields_from<REF>(p, d, F1p, F2p, c.ih, r.ih, drho, U1, U2, ur1);
    sm.rho[ty + MH][tx + MH] = drho;
    sm.u1[ty + MH][tx + MH] = U1;
    sm.u2[ty + MH][tx + MH] = U2;
    // ring: rows -1 and TY (columns -1..TX), columns -1 and TX (rows 0..TY-1),
    // one node per thread from the last thread down (warp 0 also stages the
    // next tile)
    {
        const int q = NT - 1 - tid;
        if (q < RING) {
            int x, y;
            if (q < 2 * BAND) {
                y = q < BAND ? -1 : TY;
                x = (q < BAND ? q : q - BAND) - 1;
            } else {
                const int b = q - 2 * BAND;
                x = b < TY ? -1 : TX;
                y = b < TY ? b : b - TY;
            }
            const AxisRecord cq = axis_record(rec1, SEAM ? wrapi(i0 + x, p.nx) : i0 + x), rq = axis_record(rec2, j0 + y);
            const int sq = (y + HYS) * BX + x + T::HXS;
            float dd[9], a, u, v;
            lean_pull<S>(sf_ + sq, p.sf, cq, rq, dd);
            fields_from<REF>(p, dd, scl<S>(Store<S>::lds(sF_ + sq), p.sF),
                             scl<S>(Store<S>::lds(sF_ + T::BX * T::BY + sq), p.sF), cq.ih, rq.ih, a, u, v,
                             REF ? GOC_U1R(p, j0 + y) : 0.f);
            sm.rho[y + MH][x + MH] = a;
            sm.u1[y + MH][x + MH] = u;
            sm.u2[y + MH][x + MH] = v;
        }
    }
    if (!__syncthreads_and(ok)) return false;
    // central second-order differences (interior)
    const int ex = tx + MH, ey = ty + MH;
    const float fl[7][1] = {{drho}, {U1}, {U2},
                            {0.5f * (sm.u1[ey][ex + 1] - sm.u1[ey][ex - 1])},
                            {0.5f * (sm.rho[ey][ex + 1] - sm.rho[ey][ex - 1])},
                            {0.5f * (sm.u2[ey + 1][ex] - sm.u2[ey - 1][ex])},
                            {0.5f * (sm.rho[ey + 1][ex] - sm.rho[ey - 1][ex])}};
    const int jj[1] = {j};
    const bool own[1] = {true};
    const float dn[1][9] = {{d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8]}};
    const float F1n[1] = {F1p}, F2n[1] = {F2p}, h2n[1] = {r.h}, ih2n[1] = {r.ih}, urn[1] = {ur1};
    SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin), static_cast<const S *>(p.gin),
                     p.plane, p.pitch, p.sf, p.sF, p.sg};
    const float th[2] = {c.th, r.th};
    // (SEAM: the MIE pull wraps across the periodic seam)
    collide<S, MHD, SEAM, float, false, 0>(p, src, i, jj, own, dn, F1n, F2n, c.h, c.ih, h2n, ih2n, fl, urn, th);
    return true;
}

// Kind of a tile for the straight-grid kernel: tile_kind's 0 (interior), 1
// (near a wall), 2 (halo across a periodic seam, global loads), and 3: a full
// tile whose staged box crosses the periodic seam of xi1 only (inside the
// lattice and away from walls along xi2, nx a multiple of the tile width).
// Kind 3 is staged like kind 0 -- the copy fills the columns beyond the seam
// with zeros -- and those columns are then copied from the other side of the
// lattice (seam_fill), so the tile takes the interior path.  FP32 storage
// only: with 16-bit storage the general path on global loads and the interior
// path round the scaled values differently in the last bit (the compiler
// fuses different products), and the slabs of one lattice, whose seam tiles
// near a cut take the general path, must reproduce the lattice bitwise.
template <class S>
__device__ __forceinline__ int tile_kind_lean(const StepParams &p, int i0, int j0) {
    const int k = tile_kind<S>(p, i0, j0);
    if (Store<S>::scaled || k != 2 || !p.use_tma || p.nopull || !p.per_x || p.nx % TX) return k;
    const bool wy = p.per_y && (j0 - HYS < 0 || j0 + TY + HYS > p.ny);
    return !wy && j0 >= 2 && j0 + TY + 2 <= p.ny ? 3 : 2;
}

// Copy the columns of a kind-3 tile's stage that lie beyond the periodic seam
// of xi1 (zero-filled by the copy) from the other side of the lattice: per
// side, Tiling<S>::HXS columns (16 bytes) of each of the 11 planes and each
// staged row inside the lattice, one 16-byte load and store per segment.
// Called by every thread after the stage's copy has landed; the caller
// separates it from the reads with a block barrier.
template <class S>
__device__ __forceinline__ void seam_fill(const StepParams &p, unsigned char *st, int i0, int j0) {
    using T = Tiling<S>;
    constexpr int SEG = T::HXS, NSEG = 11 * T::BY;
    static_assert(SEG * sizeof(S) == 16, "a segment is 16 bytes");
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int q = tid; q < 2 * NSEG; q += NT) {
        const int side = q >= NSEG ? 1 : 0, k = q - side * NSEG;
        const int plane = k / T::BY, row = k - plane * T::BY;
        const int bx0 = side ? T::BX - SEG : 0;
        const int x0 = i0 - T::HXS + bx0, y = j0 - HYS + row;
        if ((x0 >= 0 && x0 < p.nx) || y < 0 || y >= p.ny) continue;
        const int xs = x0 < 0 ? x0 + p.nx : x0 - p.nx;
        const S *src = plane < 9 ? static_cast<const S *>(p.fin) + plane * p.plane
                                 : static_cast<const S *>(p.Fin) + (plane - 9) * p.plane;
        src += (long long)y * p.pitch + xs;
        unsigned char *dst = st + (plane < 9 ? 0 : T::OFF_FF) +
                             (((plane < 9 ? plane : plane - 9) * T::BY + row) * T::BX + bx0) * (int)sizeof(S);
        *reinterpret_cast<uint4 *>(dst) = __ldg(reinterpret_cast<const uint4 *>(src));
    }
}

template <class S, bool MHD, bool SEAMS = true>
__device__ __forceinline__ bool lean_run_tile(const StepParams &p, int kind, int i0, int j0,
                                              unsigned char *stage, FieldSmem &sm, bool ok) {
    if (kind == 0 && !p.nopull) return lean_tile<S, MHD>(p, stage, i0, j0, sm, ok);   // (the first step
                                                                                       // reads f^0 in place)
    if (SEAMS && kind == 3) {   // (never for the first step: tile_kind_lean)
        seam_fill<S>(p, stage, i0, j0);
        __syncthreads();
        return lean_tile<S, MHD, true>(p, stage, i0, j0, sm, ok);
    }
    return run_tile<S, MHD, false, 0>(p, kind, i0, j0, stage, sm, ok);
}

// Single lattice on a straight grid: persistent blocks take tiles from the
// lattice's queue, as step_kernel does.  SEAMS: the lattice has seam tiles of
// kind 3 (FP32, periodic along xi1, width a multiple of 32); the other
// lattices run an instantiation without that path.
template <class S, bool MHD, bool SEAMS>
__global__ void __launch_bounds__(NT, MHD ? GOC_MIN_BLOCKS_MHD_STRAIGHT : GOC_MIN_BLOCKS)
    lean_step_kernel(const __grid_constant__ StepParams p) {
    using T = Tiling<S>;
    constexpr int STAGE = MHD ? T::STAGE_MHD : T::STAGE_NSE;
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
    griddep_wait();
    if (leader && blockIdx.x == 0) {
        if (Store<S>::scaled && p.sr) *p.seed_wr = *p.seed_rd + 1u;
        if (p.tctr_next) *p.tctr_next = 0;
    }
    const TileMaps m{&p.tm_f, &p.tm_F, &p.tm_g};
    int *ctr = p.tctr;
    const int first = blockIdx.x, stride = gridDim.x;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY, ntiles = ntx * nty;
    auto take = [&](int stg, int t) {
        int4 it = make_int4(t, 0, 0, 0);
        if (t < ntiles) {
            it.y = (t % ntx) * TX;
            it.z = (t / ntx) * TY;
            it.w = SEAMS ? tile_kind_lean<S>(p, it.y, it.z) : tile_kind<S>(p, it.y, it.z);
            if (it.w != 2) {
                fence_proxy_async();
                issue_tile<S>(m, it.y, it.z, dyn + stg * STAGE, &bars[stg], MHD);
            }
        }
        s_item[stg] = it;
    };
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
        if (t >= ntiles) break;
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
        bool ok = true;
        if (it.w != 2) {
            uint32_t &ph = stage ? ph1 : ph0;
            ok = mbar_wait_bounded(&bars[stage], ph, p.flag);
            ph ^= 1;
        }
        if (MHD) {
            if (!__syncthreads_and(ok)) return;
        }
        if (!lean_run_tile<S, MHD, SEAMS>(p, it.w, it.y, it.z, dyn + stage * STAGE, sm, ok)) return;
        __syncthreads();
        stage ^= 1;
    }
}

// ---- 32 x 16 tiles, two rows per thread -------------------------------------
// The same step on tiles twice as tall: each thread updates the nodes of rows
// ty and ty + 8 of its column, so the per-tile work (item, copy, barriers,
// metric records of the column) and the ring of halo nodes are shared by twice
// the nodes.  Interior tiles are staged by TMA (box [9][22][BX] and [2][22][BX]:
// 16 rows and a halo of 3); tiles next to a wall or across a periodic seam run
// as two 32 x 8 tiles of the general path on direct global loads.  FP32 keeps
// one stage (released after the last read of the tile, then the next copy is
// issued), 16-bit storage two.
template <class S> struct Tiling2 {
    static constexpr int HXS = Tiling<S>::HXS, BX = Tiling<S>::BX, TYL = 2 * TY, BY = TYL + 2 * HYS;
    static constexpr int align128(int b) { return (b + 127) / 128 * 128; }
    static constexpr int F_BYTES = 9 * BY * BX * (int)sizeof(S);
    static constexpr int FF_BYTES = 2 * BY * BX * (int)sizeof(S);
    static constexpr int OFF_FF = align128(F_BYTES);
    static constexpr int STAGE = OFF_FF + align128(FF_BYTES);
    static constexpr int NSTAGE = sizeof(S) == 4 ? 1 : 2;
};
struct FieldSmem2 {
    float rho[2 * TY + 2 * MH][TX + 2 * MH], u1[2 * TY + 2 * MH][TX + 2 * MH], u2[2 * TY + 2 * MH][TX + 2 * MH];
};
static_assert(sizeof(FieldSmem2) >= sizeof(FieldSmem), "the general path's field arrays live in FieldSmem2");

// Kind of a 32 x 16 tile: 0 interior (staged), 1 anything else (general path,
// global loads).
template <class S>
__device__ __forceinline__ int tile_kind2(const StepParams &p, int i0, int j0) {
    using T = Tiling2<S>;
    if (!p.use_tma) return 1;
    const bool wx = p.per_x && (i0 - T::HXS < 0 || i0 + TX + T::HXS > p.nx);
    const bool wy = p.per_y && (j0 - HYS < 0 || j0 + T::TYL + HYS > p.ny);
    if (wx || wy) return 1;
    if (i0 >= 2 && i0 + TX + 2 <= p.nx && j0 >= 2 && j0 + T::TYL + 2 <= p.ny) return 0;
    return 1;
}

template <class S, bool MHD>
__device__ __forceinline__ void lean2_collide(const StepParams &p, int i, int j, const AxisRecord &c,
                                              const AxisRecord &r, const float (&d)[9], float F1p, float F2p,
                                              float drho, float U1, float U2, const FieldSmem2 &sm, int ex, int ey,
                                              float ur1) {
    const float fl[7][1] = {{drho}, {U1}, {U2},
                            {0.5f * (sm.u1[ey][ex + 1] - sm.u1[ey][ex - 1])},
                            {0.5f * (sm.rho[ey][ex + 1] - sm.rho[ey][ex - 1])},
                            {0.5f * (sm.u2[ey + 1][ex] - sm.u2[ey - 1][ex])},
                            {0.5f * (sm.rho[ey + 1][ex] - sm.rho[ey - 1][ex])}};
    const int jj[1] = {j};
    const bool own[1] = {true};
    const float dn[1][9] = {{d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8]}};
    const float F1n[1] = {F1p}, F2n[1] = {F2p}, h2n[1] = {r.h}, ih2n[1] = {r.ih}, urn[1] = {ur1};
    const float th[2] = {c.th, r.th};
    SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin), static_cast<const S *>(p.gin),
                     p.plane, p.pitch, p.sf, p.sF, p.sg};
    collide<S, MHD, false, float, false, 0>(p, src, i, jj, own, dn, F1n, F2n, c.h, c.ih, h2n, ih2n, fl, urn, th);
}

// One interior 32 x 16 tile from the stage st.  Every thread of the block
// calls it (fields barrier inside).  The populations of the upper node are
// pulled again after the barrier instead of being held through the lower
// node's collision.
template <class S, bool MHD>
__device__ __forceinline__ bool lean2_tile(const StepParams &p, const unsigned char *st, int i0, int j0,
                                           FieldSmem2 &sm, bool ok) {
    using T = Tiling2<S>;
    constexpr bool REF = Store<S>::scaled;
    constexpr int BX = T::BX, PLF = T::BX * T::BY, TYL = T::TYL, BAND = TX + 2, RING = 2 * BAND + 2 * TYL;
    const S *sf_ = reinterpret_cast<const S *>(st);
    const S *sF_ = reinterpret_cast<const S *>(st + T::OFF_FF);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i = i0 + tx, ja = j0 + ty, jb = ja + TY;
    const float4 *rec1 = axis_records(p.ax1, p.nx), *rec2 = axis_records(p.ax2, p.ny);
    const AxisRecord c = axis_record(rec1, i), ra = axis_record(rec2, ja), rb = axis_record(rec2, jb);
    const int sa = (ty + HYS) * BX + tx + T::HXS, sb = sa + TY * BX;
    // lower node: pulled, fields, kept; upper node: fields only
    float d[9], drho, U1, U2;
    const float ura = REF ? GOC_U1R(p, ja) : 0.f, urb = REF ? GOC_U1R(p, jb) : 0.f;
    lean_pull<S, T::BY>(sf_ + sa, p.sf, c, ra, d);
    const float F1p = scl<S>(Store<S>::lds(sF_ + sa), p.sF), F2p = scl<S>(Store<S>::lds(sF_ + PLF + sa), p.sF);
    fields_from<REF>(p, d, F1p, F2p, c.ih, ra.ih, drho, U1, U2, ura);
    sm.rho[ty + MH][tx + MH] = drho;
    sm.u1[ty + MH][tx + MH] = U1;
    sm.u2[ty + MH][tx + MH] = U2;
    {
        float db[9], a, u, v;
        lean_pull<S, T::BY>(sf_ + sb, p.sf, c, rb, db);
        fields_from<REF>(p, db, scl<S>(Store<S>::lds(sF_ + sb), p.sF), scl<S>(Store<S>::lds(sF_ + PLF + sb), p.sF),
                         c.ih, rb.ih, a, u, v, urb);
        sm.rho[ty + TY + MH][tx + MH] = a;
        sm.u1[ty + TY + MH][tx + MH] = u;
        sm.u2[ty + TY + MH][tx + MH] = v;
    }
    {   // ring, from the last thread down (warp 0 also stages the next tile)
        const int q = NT - 1 - tid;
        if (q < RING) {
            int x, y;
            if (q < 2 * BAND) {
                y = q < BAND ? -1 : TYL;
                x = (q < BAND ? q : q - BAND) - 1;
            } else {
                const int b = q - 2 * BAND;
                x = b < TYL ? -1 : TX;
                y = b < TYL ? b : b - TYL;
            }
            const AxisRecord cq = axis_record(rec1, i0 + x), rq = axis_record(rec2, j0 + y);
            const int sq = (y + HYS) * BX + x + T::HXS;
            float dd[9], a, u, v;
            lean_pull<S, T::BY>(sf_ + sq, p.sf, cq, rq, dd);
            fields_from<REF>(p, dd, scl<S>(Store<S>::lds(sF_ + sq), p.sF), scl<S>(Store<S>::lds(sF_ + PLF + sq), p.sF),
                             cq.ih, rq.ih, a, u, v, REF ? GOC_U1R(p, j0 + y) : 0.f);
            sm.rho[y + MH][x + MH] = a;
            sm.u1[y + MH][x + MH] = u;
            sm.u2[y + MH][x + MH] = v;
        }
    }
    if (!__syncthreads_and(ok)) return false;
    lean2_collide<S, MHD>(p, i, ja, c, ra, d, F1p, F2p, drho, U1, U2, sm, tx + MH, ty + MH, ura);
    {   // upper node: pulled again from the stage, its fields from the field arrays
        float db[9];
        lean_pull<S, T::BY>(sf_ + sb, p.sf, c, rb, db);
        const int ey = ty + TY + MH, ex = tx + MH;
        lean2_collide<S, MHD>(p, i, jb, c, rb, db, scl<S>(Store<S>::lds(sF_ + sb), p.sF),
                              scl<S>(Store<S>::lds(sF_ + PLF + sb), p.sF), sm.rho[ey][ex], sm.u1[ey][ex],
                              sm.u2[ey][ex], sm, ex, ey, urb);
    }
    return true;
}

template <class S>
__device__ __forceinline__ void issue_tile2(const TileMaps &m, int i0, int j0, unsigned char *stage, uint64_t *bar) {
    using T = Tiling2<S>;
    mbar_expect_tx(bar, T::F_BYTES + T::FF_BYTES);
    tma_load_3d(stage, m.f, i0 - T::HXS, j0 - HYS, 0, bar);
    tma_load_3d(stage + T::OFF_FF, m.F, i0 - T::HXS, j0 - HYS, 0, bar);
}

// Single lattice on a straight grid, 32 x 16 tiles (p.tm_f / p.tm_F must be
// the maps with the 22-row box).
template <class S, bool MHD>
__global__ void __launch_bounds__(NT, MHD ? GOC_MIN_BLOCKS_MHD_STRAIGHT : GOC_MIN_BLOCKS)
    lean2_step_kernel(const __grid_constant__ StepParams p) {
    using T = Tiling2<S>;
    constexpr int NS = T::NSTAGE;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ FieldSmem2 sm;
    __shared__ int4 s_item[2];
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    if (leader) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    griddep_launch_dependents();
    griddep_wait();
    if (leader && blockIdx.x == 0) {
        if (Store<S>::scaled && p.sr) *p.seed_wr = *p.seed_rd + 1u;
        if (p.tctr_next) *p.tctr_next = 0;
    }
    const TileMaps m{&p.tm_f, &p.tm_F, &p.tm_g};
    int *ctr = p.tctr;
    const int stride = gridDim.x;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + T::TYL - 1) / T::TYL, ntiles = ntx * nty;
    auto take = [&](int stg, int t) {
        int4 it = make_int4(t, 0, 0, 1);
        if (t < ntiles) {
            it.y = (t % ntx) * TX;
            it.z = (t / ntx) * T::TYL;
            it.w = p.nopull ? 1 : tile_kind2<S>(p, it.y, it.z);   // (the first step reads f^0 in place)
            if (it.w == 0) {
                fence_proxy_async();
                issue_tile2<S>(m, it.y, it.z, dyn + stg * T::STAGE, &bars[stg]);
            }
        }
        s_item[stg] = it;
    };
    auto next_index = [&](int t) { return ctr ? stride + atomicAdd(ctr, 1) : t + stride; };
    if (leader) take(0, blockIdx.x);
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    int stage = 0;
    for (;;) {
        const int4 it = s_item[stage];
        const int t = it.x;
        if (t >= ntiles) break;
        int nt = 0;
        if (leader) {
            nt = next_index(t);
            if (NS == 2) take(stage ^ 1, nt);
        }
        bool ok = true;
        if (it.w == 0) {
            uint32_t &ph = stage ? ph1 : ph0;
            ok = mbar_wait_bounded(&bars[stage], ph, p.flag);
            ph ^= 1;
            if (MHD) {
                if (!__syncthreads_and(ok)) return;
            }
            if (!lean2_tile<S, MHD>(p, dyn + stage * T::STAGE, it.y, it.z, sm, ok)) return;
        } else {   // two 32 x 8 tiles of the general path on global loads
            SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin),
                             static_cast<const S *>(p.gin), p.plane, p.pitch, p.sf, p.sF, p.sg};
            FieldSmem &sm1 = *reinterpret_cast<FieldSmem *>(&sm);
            if (!tile_compute<S, MHD, 1, false, 0>(p, src, it.y, it.z, sm1, true)) return;
            if (it.z + TY < p.ny) {
                __syncthreads();   // the field arrays are reused
                if (!tile_compute<S, MHD, 1, false, 0>(p, src, it.y, it.z + TY, sm1, true)) return;
            }
        }
        __syncthreads();   // the stage, the field arrays and s_item are reused
        if (NS == 1) {
            if (leader) take(0, nt);   // the single stage is free: copy the next tile
            __syncthreads();
        } else {
            stage ^= 1;
        }
    }
}

// Many lattices in one launch (BatchArgs, goc_step.cuh): the tiles of all
// members from one work queue; members on straight grids take the interior
// and seam paths of the straight-grid kernel, the others the general path.
template <class S, bool MHD, int GEOM = 0>
__global__ void __launch_bounds__(NT, MHD ? (GEOM == 0 ? GOC_MIN_BLOCKS_MHD_STRAIGHT : GOC_MIN_BLOCKS_MHD) : GOC_MIN_BLOCKS)
    batch_step_kernel(const __grid_constant__ BatchArgs a) {
    using T = Tiling<S>;
    constexpr int STAGE = MHD ? T::STAGE_MHD : T::STAGE_NSE;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ FieldSmem sm;
    __shared__ int4 s_item[2];   // per stage: item, i0, j0, 4 lattice + tile kind
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    const int items = a.toff[a.n];
    if (leader) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    griddep_launch_dependents();
    griddep_wait();   // the previous step of every member is complete
    // record item t for stage st and start its copy (leader only); block b
    // starts with item b, later items come from the counter
    auto take = [&](int st, int t) {
        int4 it = make_int4(t, 0, 0, 0);
        if (t < items) {
            const int k = batch_lattice(a, t);
            const StepParams &q = a.p[k];
            const int ntx = (q.nx + TX - 1) / TX, local = t - a.toff[k];
            it.y = (local % ntx) * TX;
            it.z = (local / ntx) * TY;
            const int kind = GEOM == 0 ? tile_kind_lean<S>(q, it.y, it.z) : tile_kind<S>(q, it.y, it.z);
            it.w = 4 * k + kind;
            if (kind != 2) {
                const TileMaps m{a.maps + 3 * k, a.maps + 3 * k + 1, a.maps + 3 * k + 2};
                fence_proxy_async();   // generic reads of that stage precede the async writes
                issue_tile<S>(m, it.y, it.z, dyn + st * STAGE, &bars[st], MHD);
            }
            if (local == 0 && Store<S>::scaled && q.sr) *q.seed_wr = *q.seed_rd + 1u;
        }
        s_item[st] = it;
    };
    constexpr bool AHEAD = !MHD;   // as in the single-lattice kernel
    int pend = 0;   // leader: counter value of the item after the next one (fetched one tile ahead)
    if (leader) {
        if (blockIdx.x == 0) a.ctr[a.parity ^ 1] = 0;   // the next step's counter
        if (AHEAD) pend = atomicAdd(&a.ctr[a.parity], 1);
        take(0, blockIdx.x);
    }
    __syncthreads();
    uint32_t ph0 = 0, ph1 = 0;
    int stage = 0;
    for (;;) {
        const int4 it = s_item[stage];
        if (it.x >= items) break;   // uniform: every thread reads the same shared value
        if (leader) {
            int nt;
            if (AHEAD) {
                nt = (int)gridDim.x + pend;
                pend = atomicAdd(&a.ctr[a.parity], 1);
            } else {
                nt = (int)gridDim.x + atomicAdd(&a.ctr[a.parity], 1);
            }
            take(stage ^ 1, nt);
        }
        const int k = it.w >> 2, kind = it.w & 3, i0 = it.y, j0 = it.z;
        const StepParams &p = a.p[k];
        bool ok = true;   // every thread waits for the copy itself; the fields barrier gathers the outcome
        if (kind != 2) {
            uint32_t &ph = stage ? ph1 : ph0;
            ok = mbar_wait_bounded(&bars[stage], ph, p.flag);
            ph ^= 1;
        }
        if (MHD) {
            if (!__syncthreads_and(ok)) return;
        }
        bool done;
        if constexpr (GEOM == 0) done = lean_run_tile<S, MHD>(p, kind, i0, j0, dyn + stage * STAGE, sm, ok);
        else done = run_tile<S, MHD, false, GEOM>(p, kind, i0, j0, dyn + stage * STAGE, sm, ok);
        if (!done) return;   // the block leaves together
        __syncthreads();   // the stage, the field arrays and s_item are reused
        stage ^= 1;
    }
}

}  // namespace goc
