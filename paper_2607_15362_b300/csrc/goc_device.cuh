// goc_device.cuh -- device-side data structures and helpers of the GOC-LBM
// kernels (sm_103a).  All arithmetic of the time step is FP32; the metric
// precompute and the reductions use FP64.
#pragma once

#include <cuda.h>   // CUtensorMap (type only; tensor maps are encoded through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace goc {

// D2Q9 velocities (Eq. 1a/1b) and D2Q5 velocities (Eq. D2Q5a/b).
__host__ __device__ constexpr int e1(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int e2(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5); }
__host__ __device__ constexpr int g1(int a) { return a == 1 ? 1 : (a == 3 ? -1 : 0); }
__host__ __device__ constexpr int g2(int a) { return a == 2 ? 1 : (a == 4 ? -1 : 0); }
__host__ __device__ constexpr int gopp(int a) { return a == 0 ? 0 : ((a + 1) & 3) + 1; }

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp");

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

// Per-axis FP32 tables (straight grids: h1 = h1(xi1), h2 = h2(xi2)).
struct Axis {
    const float *h;    // metric factor at the nodes
    const float *ih;   // 1/h
    const float *th;   // theta_kk = h'/h^2
    const float *rm;   // rest-state pull correction, source k-1: 0.5 rho0 cs2 (1/h(k-1) - 1/h(k))
    const float *rp;   // rest-state pull correction, source k+1: 0.5 rho0 cs2 (1/h(k+1) - 1/h(k))
    const float *dm;   // MIE pull corrections, source k-1: W1 (h(k-1) - h(k)) + csm2 (h^2 theta(k-1) + h^2 theta(k))/4
    const float *dp;   //                      source k+1: W1 (h(k+1) - h(k)) - csm2 (h^2 theta(k+1) + h^2 theta(k))/4
    // The table holds 8 rows of n values (7 on straight grids, plus a spare
    // row), then the same quantities per node index as records of two float4,
    // (h, ih, th, rm), (rp, dm, dp, 0), at h + 8 n (see axis_records).
    // Curvilinear column metric (annular sector; xi1 axis): rm/rp hold the
    // full pull corrections of links 1/3 (not per unit h2), and the rows dm,
    // dp, dp + n hold h2, 1/h2 and theta21 as functions of xi1 (the MIE then
    // stores its populations without a reference field and needs no dm/dp).
};

// the per-index records of an axis table of n entries
__device__ __forceinline__ const float4 *axis_records(const Axis &a, int n) {
    return reinterpret_cast<const float4 *>(a.h + 8 * (size_t)n);
}

// the node-by-node metric (StepParams.gm): plane k at node (i, j), and the
// wall metric at position k along wall `side` (0-3: the wall-normal factor at
// W, E, S, N; 4-7: the tangential one)
__device__ __forceinline__ float gm_at(const float *gm, long long plane, int pitch, int k, int i, int j) {
    return gm[k * plane + (long long)j * pitch + i];
}
__device__ __forceinline__ float gm_wall(const float *gm, long long plane, int nx, int ny, int side, int k) {
    return gm[10 * plane + (long long)side * (nx > ny ? nx : ny) + k];
}

// rows of the per-row storage reference table (StepParams.reft)
#define GOC_U1R(p, j) ((p).reft[(j)])
#define GOC_BROW(p, c, j) ((p).reft[(1 + (c)) * (p).ny + (j)])
#define GOC_BPULL(p, k, c, j) ((p).reft[(3 + 2 * (k) + (c)) * (p).ny + (j)])

// the curvilinear column metric of node column i (see Axis)
__device__ __forceinline__ float curv_h2(const Axis &a, int i) { return a.dm[i]; }
__device__ __forceinline__ float curv_ih2(const Axis &a, int i) { return a.dp[i]; }
__device__ __forceinline__ float curv_t21(const Axis &a, int n, int i) { return a.dp[n + i]; }

// Everything one step needs, passed by value.
struct StepParams {
    int nx, ny, pitch;         // pitch in elements (multiple of 32)
    long long plane;           // ny * pitch
    int per_x, per_y;          // periodic axes
    int curv;                  // 1: curvilinear column metric (h1, h2, theta11, theta21 functions of xi1);
                               // 2: metric given node by node (gm)
    // slab of a larger lattice (goc_create_slab): local rows [own0, own1) are
    // the lattice's own (reductions), seed_row0 is the global row of local row
    // 0 (random streams of stochastic rounding follow global node indices);
    // 0, ny, 0 for a whole lattice.  (Placed in alignment gaps: the batch
    // kernel carries 32 of these blocks in its 32 KB parameter space.)
    int own0;
    // node-by-node metric (curv = 2): FP32 planes [10][plane] h1, h2, theta11,
    // theta12, theta21, theta22 and the pull corrections of links 1..4 (into
    // the node), then [8][max(nx, ny)] the wall-normal metric along W, E, S, N
    // and the tangential one
    const float *gm;
    int nopull;                // 1: the input buffer holds pre-collision populations (the
                               // initial state f^0 of Appendix C.1): read them in place
    int seed_row0;
    const void *fin;           // [9][plane] stored post-collision deviations (input)
    void *fout;                // [9][plane] (output)
    const void *Fin;           // [2][plane] stored effective force of the previous step
    void *Fout;
    const void *gin;           // [10][plane] MIE vector populations (component-major)
    void *gout;
    Axis ax1, ax2;
    float rho0, cs2, ics2, nu, zeta;
    float om[9];
    float fext1, fext2;
    float gi;                  // 1: full correction coefficients, 0: cubic terms dropped
    // combinations of zeta, nu and 1/cs2 in the correction coefficients (Eqs. 83, 85)
    float zc, nc, zmn, A3, A4, gic;   // zeta/cs2, nu/cs2, zeta-nu, 2zeta+nu, zeta+2nu, gi/cs2
    float uw[4];               // tangential wall velocity per side
    float hwn[4];              // wall-normal metric factor at each wall (W/E: h1, S/N: h2)
    int moving;                // any moving wall
    float sf, isf;             // population storage scale and its inverse (1 for FP32)
    float sF, isF;             // force storage scale
    float sg, isg;             // MIE storage scale
    // MIE (Appendix G)
    float csm2, icsm2, taum, itaum, eta, imum, W0, W1;
    float brest[2];            // reference (storage) field
    float bw[4][2];            // wall fields
    // optional outputs
    float *uout;               // [4][plane]: U1, U2, B1, B2 of this step's time level (may be null)
    int *flag;                 // status flag (may be null): 1 divergence, 2 a TMA wait timed out
    // stochastic rounding of 16-bit stores: the step index of this launch is
    // read from *seed_rd and seed_rd + 1 written to *seed_wr (the counter the
    // launch of the other buffer parity reads)
    int sr;
    int constF;                // 1: no stored force; the force of every step is the body force
    // tile queue of the single-lattice step kernel: this launch takes tiles from
    // *tctr and zeroes *tctr_next for the launch of the other buffer parity
    // (tctr == null: static order, block b takes tiles b, b + grid, ...).
    // Every launch zeroes tctr_next, whether it takes tiles from a queue or
    // not, so that a change of tile order between steps finds it clean.
    int *tctr;
    int *tctr_next;
    const unsigned *seed_rd;
    unsigned *seed_wr;
    // Per-row storage reference of 16-bit storage on straight grids (null
    // otherwise): the stored deviations of links 1 and 3 are taken relative to
    // a reference that carries the momentum h2 rho0 A1(j) of a row velocity
    // A1(j), and the MIE populations relative to a row field Bref_c(j); both
    // are row means of the flow, refreshed every few hundred steps, so that at
    // a steady channel flow the stored values (and their rounding) shrink to
    // the part the row means do not capture.
    // One table of 7 rows of ny values (one pointer: the batch kernel carries
    // 32 of these parameter blocks in its parameter space):
    //   row 0           u1r[j] = h2 rho0 A1(j) / 2  (added on link 1, taken off link 3)
    //   rows 1, 2       brow[c][j] = Bref_c(j)
    //   rows 3 + 2k + c bpull[k][c][j]: pull correction of MIE link 2 (k = 0) or
    //                   4 (k = 1), per unit h1, for the source row j -+ 1
    const float *reft;
    // TMA descriptors of the input buffers (3D: [planes][ny][nx])
    int use_tma;
    int own1;                  // end of the owned rows (see own0)
    CUtensorMap tm_f;          // box [9][TY + 2 HYS][TX + 2 HXS]
    CUtensorMap tm_F;          // box [2][TY + 2 HYS][TX + 2 HXS]
    CUtensorMap tm_g;          // box [10][TY + 2][TX + 2 HXS]
};

// ---- storage formats (ld: global read-only path, lds: shared memory, st:
// global store -- st.global, so the compiler knows a store cannot alias shared
// memory) ---------------------------------------------------------------------
template <class S> struct Store;
template <> struct Store<float> {
    static constexpr bool scaled = false;   // FP32 is stored unscaled
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float lds(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { __stcg(p, v); }
    static __device__ __forceinline__ void st_sr(float *p, float v, uint32_t &) { __stcg(p, v); }
};
// Stochastic rounding (st_sr): u, uniform in [0, 2^k) with k the number of
// FP32 significand bits the format drops (13 for FP16, 16 for BF16), is added
// to the magnitude bits and the sum truncated toward zero, which rounds away
// from zero with probability equal to the dropped fraction (IEEE formats are
// sign-magnitude, so the same holds for negative values).  The random stream
// is a 32-bit LCG (multiplier 747796405, increment 2891336453) whose high bits
// are used.
__device__ __forceinline__ uint32_t lcg_next(uint32_t &r) {
    r = r * 747796405u + 2891336453u;
    return r;
}
template <> struct Store<__half> {
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float lds(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { __stcg(p, __float2half_rn(v)); }
    static __device__ __forceinline__ void st_sr(__half *p, float v, uint32_t &r) {
        __stcg(p, __float2half_rz(__uint_as_float(__float_as_uint(v) + (lcg_next(r) >> 19))));
    }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float lds(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { __stcg(p, __float2bfloat16_rn(v)); }
    static __device__ __forceinline__ void st_sr(__nv_bfloat16 *p, float v, uint32_t &r) {
        __stcg(p, __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + (lcg_next(r) >> 16))));
    }
};

// value * scale for 16-bit storage, value unchanged for FP32
template <class S> __device__ __forceinline__ float scl(float v, float s) { return Store<S>::scaled ? v * s : v; }

// Seed of a node's random stream: the 32-bit finaliser of MurmurHash3 applied
// to a mix of the node index and the step index.
__device__ __forceinline__ uint32_t node_seed(uint32_t idx, uint32_t step) {
    uint32_t h = idx * 0x9E3779B1u ^ (step * 0x85EBCA77u + 0x27D4EB2Fu);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Two values to a 16-bit format in one conversion, packed as (a << 16) | b:
// with sr stochastically rounded by the hardware (cvt.rs: random bits 31..16
// round a, bits 15..0 round b; each rounds away from zero with probability
// equal to the discarded fraction), else rounded to nearest; a value beyond
// the format's range saturates to its largest finite value (as the truncating
// conversion of the software rounding does), never to infinity.
template <class S> __device__ __forceinline__ uint32_t cvt2(float a, float b, bool sr, uint32_t rbits);
template <> __device__ __forceinline__ uint32_t cvt2<__half>(float a, float b, bool sr, uint32_t rbits) {
    uint32_t d;
    if (sr) asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    else asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(a), "f"(b));
    return d;
}
template <> __device__ __forceinline__ uint32_t cvt2<__nv_bfloat16>(float a, float b, bool sr, uint32_t rbits) {
    uint32_t d;
    if (sr) asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    else asm("cvt.rn.satfinite.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(a), "f"(b));
    return d;
}
// 32 random bits for one cvt2: the high halves of the next two LCG outputs
// (the low bits of an LCG have short periods)
__device__ __forceinline__ uint32_t rand_pair_bits(uint32_t &r) {
    const uint32_t w1 = lcg_next(r), w2 = lcg_next(r);
    return __byte_perm(w1, w2, 0x3276);   // (w1 & 0xffff0000) | (w2 >> 16)
}
// Store the two halves of a cvt2 result (pb may be null: the low half is dropped).
template <class S> __device__ __forceinline__ void st_pair(S *pa, S *pb, uint32_t d) {
    asm volatile("st.global.cg.b16 [%0], %1;" ::"l"(pa), "h"((unsigned short)(d >> 16)) : "memory");
    if (pb) asm volatile("st.global.cg.b16 [%0], %1;" ::"l"(pb), "h"((unsigned short)(d & 0xffffu)) : "memory");
}
// a and b (unscaled) stored at pa and pb through one cvt2, the random bits
// drawn from r when stochastic rounding is on
template <class S>
__device__ __forceinline__ void put2(S *pa, S *pb, float a, float b, bool sr, uint32_t &r) {
    if (sr) {
        st_pair<S>(pa, pb, cvt2<S>(a, b, true, rand_pair_bits(r)));
    } else {   // round to nearest: the scalar conversions
        Store<S>::st(pa, a);
        if (pb) Store<S>::st(pb, b);
    }
}

// store of one value: stochastic rounding for 16-bit storage when asked for
template <class S>
__device__ __forceinline__ void put(S *p, float v, bool sr, uint32_t &r) {
    if (Store<S>::scaled && sr) Store<S>::st_sr(p, v, r);
    else Store<S>::st(p, v);
}

// Programmatic dependent launch: a step kernel launched with programmatic
// stream serialisation may start while the previous step drains; it lets its
// own successor be scheduled (launch_dependents) and waits for the previous
// grid's completion and memory (wait) before touching any population.  Both
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int wrapi(int k, int n) {
    k %= n;
    return k < 0 ? k + n : k;
}

}  // namespace goc
