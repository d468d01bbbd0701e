// goc_aa.cuh -- lattices that keep one population buffer and update it in
// place (FP32 storage, straight grids, central-moment collision, with or
// without the MIE).
//
// The step is the one of goc_step.cuh (Appendix E, Steps 1-7): pull
// streaming with the rest-state pull corrections and the wall conditions of
// Eqs. 101/103, the fields of Eq. GOChydrodynamicfields with the lagged
// force, second-order normal derivatives of the fields, the central-moment
// collision.  Only where the populations live changes.  Two access patterns
// alternate (the "AA" pattern), and in each of them every slot of the buffer
// is read and then written by one and the same node, so a launch can
// overwrite its input (the D2Q5 populations of the MIE, Appendix G, follow
// the same layouts with their own links):
//
//   layout AA_C   slot (x, a) holds the population of node x along link a:
//                 the initial state f^0, which the first step reads in place;
//   layout AA_S   the post-collision population of node x along link a sits
//                 at (x, opp(a)): its own node, the link reversed;
//   layout AA_T   it sits at (x + e_a, a), the node it streams to, or at
//                 (x, opp(a)) where x + e_a is outside the lattice (a wall).
//
// A step that reads AA_C or AA_T writes AA_S (node x reads and writes only
// its own slots); a step that reads AA_S writes AA_T (node x reads slot
// (x - e_a, opp(a)) -- or (x, a) where x - e_a is outside -- and writes the
// same slots: (z, c) belongs to node z - e_c, or to z where that is
// outside).  The normal derivatives need the fields of the neighbours at the
// same time level, which other nodes of the same launch overwrite, so each
// step is two launches: aa_fields_kernel stores rho, U1, U2 of every node
// (and the population sum of each wall node, which the moving-wall condition
// reads) without writing populations, then aa_collide_kernel pulls again,
// takes the neighbours' fields from that buffer and writes the new
// populations in place (the MIE update needs no neighbour values beyond its
// pulls).  The force F is read and written by its own node.
// Every value goes through the functions the two-buffer kernels use, in the
// same order, so the populations are bitwise those of the two-buffer step.
//
// Resident per node: 36 B populations + 8 B force + 12 B fields = 56 B
// (two-buffer lattices: 88 B); with the MIE 40 B more (two-buffer: 80 B
// more).  Moved per step: 44 B read and 12 B written by the fields pass,
// 44 B + 12 B read and 44 B written by the collision pass: 156 B (two-buffer
// step: 88 B); with the MIE 80 B more (the same as two buffers).
#pragma once

#include "goc_step.cuh"

namespace goc {

enum { AA_C = 0, AA_S = 1, AA_T = 2 };

// Population source of an in-place lattice in layout L.  WS: the population
// sums of the wall nodes come from the fields pass (wsum, [4][wn]: along W
// and E by row, along S and N by column) instead of being summed here.  CH:
// a node may lie on the lattice's edge (links leave it); false for the nodes
// of blocks whose nodes all have their eight neighbours inside.
template <class S, int L, bool WS, bool CH = true> struct SrcAA {
    static_assert(L == AA_C || L == AA_S || L == AA_T, "layout");
    static constexpr bool kWallSums = WS;
    static constexpr bool kInPlace = true;
    const S *f, *F, *g;
    long long plane;
    int pitch, nx, ny, per_x, per_y;
    const float *wsum;
    int wn;
    float sf, sF, sg;   // storage scales (1 for FP32)
    // the node a population of node (i, j) along link a streams to, and
    // whether it lies inside the lattice (periodic axes wrap)
    __device__ __forceinline__ bool dest(int a, int i, int j, int &ti, int &tj) const {
        ti = i + e1(a);
        tj = j + e2(a);
        bool in = true;
        if (!CH) return true;
        if (ti < 0 || ti >= nx) {
            if (per_x) ti = wrapi(ti, nx); else in = false;
        }
        if (tj < 0 || tj >= ny) {
            if (per_y) tj = wrapi(tj, ny); else in = false;
        }
        return in;
    }
    // the post-collision population of node (i, j) along link a
    __device__ __forceinline__ long long fslot(int a, int i, int j) const {
        const long long idx = (long long)j * pitch + i;
        if constexpr (L == AA_C) {
            return a * plane + idx;
        } else if constexpr (L == AA_S) {
            return opp(a) * plane + idx;
        } else {
            int ti, tj;
            if (dest(a, i, j, ti, tj)) return a * plane + (long long)tj * pitch + ti;
            return opp(a) * plane + idx;
        }
    }
    __device__ __forceinline__ float fv(int a, int i, int j) const { return scl<S>(Store<S>::ld(f + fslot(a, i, j)), sf); }
    __device__ __forceinline__ float Fv(int c, int i, int j) const {
        return scl<S>(Store<S>::ld(F + c * plane + (long long)j * pitch + i), sF);
    }
    // the post-collision MIE population k = 5 c + a of node (i, j) (D2Q5
    // links g1, g2; the same two layouts)
    __device__ __forceinline__ bool gdest(int a, int i, int j, int &ti, int &tj) const {
        ti = i + g1(a);
        tj = j + g2(a);
        bool in = true;
        if (!CH) return true;
        if (ti < 0 || ti >= nx) {
            if (per_x) ti = wrapi(ti, nx); else in = false;
        }
        if (tj < 0 || tj >= ny) {
            if (per_y) tj = wrapi(tj, ny); else in = false;
        }
        return in;
    }
    __device__ __forceinline__ long long gslot(int k, int i, int j) const {
        const int c = k / 5, a = k - 5 * c;
        const long long idx = (long long)j * pitch + i;
        if constexpr (L == AA_C) {
            return k * plane + idx;
        } else if constexpr (L == AA_S) {
            return (5 * c + gopp(a)) * plane + idx;
        } else {
            int ti, tj;
            if (gdest(a, i, j, ti, tj)) return k * plane + (long long)tj * pitch + ti;
            return (5 * c + gopp(a)) * plane + idx;
        }
    }
    __device__ __forceinline__ float gv(int k, int i, int j) const { return scl<S>(Store<S>::ld(g + gslot(k, i, j)), sg); }
    __device__ __forceinline__ float wall_sum(int i, int j) const {
        if (j == 0) return wsum[SIDE_S * wn + i];
        if (j == ny - 1) return wsum[SIDE_N * wn + i];
        if (i == 0) return wsum[SIDE_W * wn + j];
        return wsum[SIDE_E * wn + j];
    }
};

// Where a step writes the new population of node (i, j) along link a: AA_T
// after reading AA_S, else AA_S.
template <class S, int L, bool WS, bool CH>
__device__ __forceinline__ long long out_slot(const SrcAA<S, L, WS, CH> &s, const StepParams &p, int a, int i, int j,
                                              long long idx) {
    if constexpr (L == AA_S) {
        int ti, tj;
        if (s.dest(a, i, j, ti, tj)) return a * p.plane + (long long)tj * p.pitch + ti;
    }
    return opp(a) * p.plane + idx;
}

template <class S, int L, bool WS, bool CH>
__device__ __forceinline__ long long out_slot_g(const SrcAA<S, L, WS, CH> &s, const StepParams &p, int c, int a, int i,
                                                int j, long long idx) {
    if constexpr (L == AA_S) {
        int ti, tj;
        if (s.gdest(a, i, j, ti, tj)) return (5 * c + a) * p.plane + (long long)tj * p.pitch + ti;
    }
    return (5 * c + gopp(a)) * p.plane + idx;
}

template <class S, int L, bool WS, bool CH = true>
__device__ __forceinline__ SrcAA<S, L, WS, CH> aa_source(const StepParams &p, const float *wsum, int wn) {
    return SrcAA<S, L, WS, CH>{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin),
                               static_cast<const S *>(p.gin), p.plane, p.pitch, p.nx, p.ny, p.per_x, p.per_y,
                               wsum, wn, p.sf, p.sF, p.sg};
}

// The offset of the stored population of node (i, j) along D2Q9 link a
// (k = 5 c + a of the MIE with g5) in layout lay -- the same slots as the
// sources above, chosen at run time (the reference-row kernels).
__device__ __forceinline__ long long aa_slot(const StepParams &p, int lay, int a, int i, int j, bool g5 = false,
                                             int c = 0) {
    const long long idx = (long long)j * p.pitch + i;
    const int e1a = g5 ? g1(a) : e1(a), e2a = g5 ? g2(a) : e2(a);
    const int base = g5 ? 5 * c : 0, ro = g5 ? gopp(a) : opp(a);
    if (lay == AA_S) return (base + ro) * p.plane + idx;
    if (lay == AA_T) {
        int ti = i + e1a, tj = j + e2a;
        bool in = true;
        if (ti < 0 || ti >= p.nx) {
            if (p.per_x) ti = wrapi(ti, p.nx); else in = false;
        }
        if (tj < 0 || tj >= p.ny) {
            if (p.per_y) tj = wrapi(tj, p.ny); else in = false;
        }
        if (in) return (base + a) * p.plane + (long long)tj * p.pitch + ti;
        return (base + ro) * p.plane + idx;
    }
    return (base + a) * p.plane + idx;
}

// whether every node of this block has its eight neighbours inside the
// lattice (no wall, no wrap, no ragged edge): the nodes then take the paths
// without boundary logic, as the interior tiles of the two-buffer kernels do
__device__ __forceinline__ bool aa_block_interior(const StepParams &p) {
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    return i0 >= 1 && i0 + TX <= p.nx - 1 && j0 >= 1 && j0 + TY <= p.ny - 1;
}

// Fields pass: rho - rho0, U1, U2 of every node into fld ([3][plane]), and
// the population sum of every wall node into wsum (lattices with a moving
// wall).  Writes no population.
template <class S, int L, bool CH>
__device__ __forceinline__ void aa_fields_node(const StepParams &p, int i, int j, float *fld, float *wsum, int wn) {
    constexpr bool REF = Store<S>::scaled;   // per-row storage reference (16-bit storage)
    const SrcAA<S, L, false, CH> src = aa_source<S, L, false, CH>(p, nullptr, 0);
    float h1, h2, ih1, ih2, d[9], drho, U1, U2;
    const float ur1 = REF ? GOC_U1R(p, j) : 0.f;
    node_metric<0>(p, i, j, h1, h2, ih1, ih2);
    pull_node<CH, 0, REF>(p, src, i, j, h1, h2, d, ur1);
    fields_from<REF>(p, d, src.Fv(0, i, j), src.Fv(1, i, j), ih1, ih2, drho, U1, U2, ur1);
    const long long idx = (long long)j * p.pitch + i;
    fld[idx] = drho;
    fld[p.plane + idx] = U1;
    fld[2 * p.plane + idx] = U2;
    if (CH && p.moving && (i == 0 || i == p.nx - 1 || j == 0 || j == p.ny - 1)) {
        float s = 0.f;   // the sum pull_node takes at a moving wall, in the same order
#pragma unroll
        for (int b = 0; b < 9; b++) s += src.fv(b, i, j);
        if (j == 0) wsum[SIDE_S * wn + i] = s;
        if (j == p.ny - 1) wsum[SIDE_N * wn + i] = s;
        if (i == 0) wsum[SIDE_W * wn + j] = s;
        if (i == p.nx - 1) wsum[SIDE_E * wn + j] = s;
    }
}

// (6 blocks of 256 threads per SM, 40 registers: at 2048^2 the step took
// 166 us against 179 us at 4 blocks and 64 registers; 8 blocks spill heavily)
template <class S, int L>
__global__ void __launch_bounds__(NT, 6) aa_fields_kernel(const __grid_constant__ StepParams p, float *fld,
                                                                        float *wsum, int wn) {
    griddep_launch_dependents();
    griddep_wait();
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (aa_block_interior(p)) {
        aa_fields_node<S, L, false>(p, i, j, fld, wsum, wn);
    } else if (i < p.nx && j < p.ny) {
        aa_fields_node<S, L, true>(p, i, j, fld, wsum, wn);
    }
}

// the stored field c of node (ii, jj): wrapped on periodic axes, 0 outside
// a wall (as in the field arrays of the tile kernels)
__device__ __forceinline__ float aa_field(const StepParams &p, const float *fld, int c, int ii, int jj) {
    if (ii < 0 || ii >= p.nx) {
        if (!p.per_x) return 0.f;
        ii = wrapi(ii, p.nx);
    }
    if (jj < 0 || jj >= p.ny) {
        if (!p.per_y) return 0.f;
        jj = wrapi(jj, p.ny);
    }
    return fld[c * p.plane + (long long)jj * p.pitch + ii];
}

// Collision pass: pull, the fields of the node and its neighbours from the
// fields pass, normal derivatives, collision; the new populations go to the
// node's slots of the next layout, the force to the node.
template <class S, int L, bool MHD, bool CH>
__device__ __forceinline__ void aa_collide_node(const StepParams &p, int i, int j, const float *fld, const float *wsum,
                                                int wn) {
    constexpr bool REF = Store<S>::scaled;
    const SrcAA<S, L, true, CH> src = aa_source<S, L, true, CH>(p, wsum, wn);
    float h1, ih1;
    float h2[1], ih2[1], d[1][9], F1p[1], F2p[1], ur1[1] = {REF ? GOC_U1R(p, j) : 0.f};
    node_metric<0>(p, i, j, h1, h2[0], ih1, ih2[0]);
    pull_node<CH, 0, REF>(p, src, i, j, h1, h2[0], d[0], ur1[0]);
    F1p[0] = src.Fv(0, i, j);
    F2p[0] = src.Fv(1, i, j);
    const long long idx = (long long)j * p.pitch + i, pl = p.plane, pt = p.pitch;
    float fl[7][1];
    if constexpr (CH) {
        const float drho = aa_field(p, fld, 0, i, j), U1 = aa_field(p, fld, 1, i, j), U2 = aa_field(p, fld, 2, i, j);
        fl[0][0] = drho;
        fl[1][0] = U1;
        fl[2][0] = U2;
        fl[3][0] = dfd(aa_field(p, fld, 1, i - 2, j), aa_field(p, fld, 1, i - 1, j), U1, aa_field(p, fld, 1, i + 1, j),
                       aa_field(p, fld, 1, i + 2, j), i, p.nx, p.per_x);
        fl[4][0] = dfd(aa_field(p, fld, 0, i - 2, j), aa_field(p, fld, 0, i - 1, j), drho,
                       aa_field(p, fld, 0, i + 1, j), aa_field(p, fld, 0, i + 2, j), i, p.nx, p.per_x);
        fl[5][0] = dfd(aa_field(p, fld, 2, i, j - 2), aa_field(p, fld, 2, i, j - 1), U2, aa_field(p, fld, 2, i, j + 1),
                       aa_field(p, fld, 2, i, j + 2), j, p.ny, p.per_y);
        fl[6][0] = dfd(aa_field(p, fld, 0, i, j - 2), aa_field(p, fld, 0, i, j - 1), drho,
                       aa_field(p, fld, 0, i, j + 1), aa_field(p, fld, 0, i, j + 2), j, p.ny, p.per_y);
    } else {   // central differences, as the interior tiles take them
        fl[0][0] = fld[idx];
        fl[1][0] = fld[pl + idx];
        fl[2][0] = fld[2 * pl + idx];
        fl[3][0] = 0.5f * (fld[pl + idx + 1] - fld[pl + idx - 1]);
        fl[4][0] = 0.5f * (fld[idx + 1] - fld[idx - 1]);
        fl[5][0] = 0.5f * (fld[2 * pl + idx + pt] - fld[2 * pl + idx - pt]);
        fl[6][0] = 0.5f * (fld[idx + pt] - fld[idx - pt]);
    }
    const int jj[1] = {j};
    const bool own[1] = {true};
    collide<S, MHD, CH, float, false, 0>(p, src, i, jj, own, d, F1p, F2p, h1, ih1, h2, ih2, fl, ur1);
}

// Collision pass: pull, the fields of the node and its neighbours from the
// fields pass, normal derivatives, collision; the new populations go to the
// node's slots of the next layout, the force to the node.
template <class S, int L, bool MHD>
__global__ void __launch_bounds__(NT, MHD ? GOC_MIN_BLOCKS_MHD_STRAIGHT : GOC_MIN_BLOCKS)
    aa_collide_kernel(const __grid_constant__ StepParams p, const float *fld, const float *wsum, int wn) {
    griddep_launch_dependents();
    griddep_wait();
    // stochastic rounding: the step index of the next step, for the launch of
    // the other parity (as the two-buffer step kernels do)
    if (Store<S>::scaled && p.sr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        *p.seed_wr = *p.seed_rd + 1u;
    const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
    if (aa_block_interior(p)) {
        aa_collide_node<S, L, MHD, false>(p, i, j, fld, wsum, wn);
    } else if (i < p.nx && j < p.ny) {
        aa_collide_node<S, L, MHD, true>(p, i, j, fld, wsum, wn);
    }
}

// Macroscopic fields of an in-place lattice (as moments_kernel, FP64 output
// [5][ny][nx]; no MIE).
template <class S, int L, bool MHD>
__global__ void aa_moments_kernel(const StepParams p, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    constexpr bool REF = Store<S>::scaled;
    const SrcAA<S, L, false> src = aa_source<S, L, false>(p, nullptr, 0);
    float h1, h2, ih1, ih2, d[9], drho, U1, U2;
    const float ur1 = REF ? GOC_U1R(p, j) : 0.f;
    node_metric<0>(p, i, j, h1, h2, ih1, ih2);
    pull_node<true, 0, REF>(p, src, i, j, h1, h2, d, ur1);
    fields_from<REF>(p, d, src.Fv(0, i, j), src.Fv(1, i, j), ih1, ih2, drho, U1, U2, ur1);
    const long long N = (long long)p.nx * p.ny, n = (long long)j * p.nx + i;
    out[n] = (double)p.rho0 + (double)drho;
    out[N + n] = U1;
    out[2 * N + n] = U2;
    double B1 = 0.0, B2 = 0.0;
    if constexpr (MHD) {   // as moments_kernel on straight grids
        float gd[2][5];
        for (int c = 0; c < 2; c++) pull_mie<true, 0, REF>(p, src, i, j, h1, h2, c, gd[c]);
        const float s0 = (gd[0][0] + gd[0][1] + gd[0][2] + gd[0][3] + gd[0][4]) / (h1 * h2);
        const float s1 = (gd[1][0] + gd[1][1] + gd[1][2] + gd[1][3] + gd[1][4]) / (h1 * h2);
        B1 = (double)bref<REF>(p, 0, j) + (double)s0;
        B2 = (double)bref<REF>(p, 1, j) + (double)s1;
    }
    out[3 * N + n] = B1;
    out[4 * N + n] = B2;
}

}  // namespace goc
