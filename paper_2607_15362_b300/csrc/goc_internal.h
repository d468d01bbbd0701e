// goc_internal.h -- host-side declarations shared by the translation units of
// libgoc: the lattice object, the launch helper and the per-storage-type
// kernel launchers (each storage type's kernels are compiled in a file of
// their own, goc_kernels_<type>.cu, so the library builds in parallel).
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>

#include "../../include/goc.h"
#include "goc_device.cuh"
#include "goc_step.cuh"
#include "goc_lean.cuh"

// Error reporting shared by every translation unit: records the message
// returned by goc_last_error() and returns st.
goc_status goc_fail(goc_status st, const char *fmt, ...);

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return goc_fail(GOC_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                            __FILE__, __LINE__);                                              \
    } while (0)

// Kernel launch with programmatic stream serialisation (the kernel may start
// while its predecessor drains; it waits in griddepcontrol.wait before
// touching data).  GOC_DISABLE_PDL=1 launches plainly.
inline bool pdl_enabled() {
    static const int on = std::getenv("GOC_DISABLE_PDL") ? 0 : 1;
    return on != 0;
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = (pdl && pdl_enabled()) ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

using goc::StepParams;

struct goc_lattice {
    goc_grid grid;
    goc_map map;
    goc_flow flow;
    goc_mhd mhd;
    int storage = GOC_FP32;
    cudaStream_t stream = nullptr;
    int device = 0;
    int check_every = 100;
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;
    // device memory
    void *f[2] = {nullptr, nullptr};
    void *F[2] = {nullptr, nullptr};
    void *g[2] = {nullptr, nullptr};
    float *tab1 = nullptr, *tab2 = nullptr;      // [8][nx] + records [nx][8], [8][ny] + records [ny][8]
    double *m1 = nullptr, *m2 = nullptr;         // FP64 h, theta per axis: [2][n+2]
    float *gm = nullptr;                         // node-table metric: [10][plane] + [4][max(nx, ny)]
    float *uout[2] = {nullptr, nullptr};
    int *flag = nullptr;
    double *red = nullptr;                       // 8 doubles
    double *mom = nullptr;                       // [5][ny][nx]
    size_t device_bytes = 0;
    // parameters
    double q = 1.0, cs2 = 1.0 / 3.0, nu = 0, zeta = 0, tau = 1, csm2 = 0, taum = 1, eta = 0;
    double hw[4] = {1, 1, 1, 1};
    StepParams sp;
    int cur = 0;
    long long steps = 0;
    double res_u = 0.0, res_b = 0.0;
    cudaGraphExec_t graph = nullptr;
    int graph_cur = 0;                           // buffer the captured graph starts from
    bool owns_stream = false;
    bool in_batch = false;                       // stepped only through goc_batch_step
    bool guard = false;                          // guard bands: padding columns and buffer tails hold a canary
    int *hflag = nullptr;                        // pinned host copy of flag[0], refreshed after each goc_step
    cudaEvent_t flag_ev = nullptr;               // completion of that copy
    bool fresh = false;                          // buffer holds f^0 (pre-collision): next step reads in place
    bool res_pending = false;                    // residual sums of a batch step wait in red[4..7]
    CUtensorMap tmf[2], tmF[2], tmg[2];          // TMA descriptors of both buffers
    CUtensorMap tmf2[2], tmF2[2];                // the same with the box of 32 x 16 tiles
    bool tma_ok = false;
    int rounding = 0;                            // goc_exec.rounding
    int scheme = 0;                              // goc_exec.scheme
    // launch configuration (results are bitwise the same under every choice):
    // tile queue (dynamic) or static tile order, programmatic dependent launch
    int cfg_dynamic = 1, cfg_pdl = 1;
    int cfg_balanced = 0;                        // grid: the fewest blocks taking the same rounds of tiles
    int cfg_rows = 1;                            // straight grids: tiles of 8 (1) or 16 (2) rows
    bool tuned = false;                          // chosen by the launch autotuner (or fixed)
    // Each single-lattice step kernel zeroes the tile queue of the other
    // buffer parity, which the next step uses; steps taken by a batch kernel
    // do not, and the next single-lattice launch zeroes both first.
    bool queues_dirty = false;
    int plateau_checks = 0;                      // goc_exec.plateau_checks
    // per-row storage reference (16-bit storage on straight grids; see goc_aux.cuh)
    double *ref64 = nullptr;                     // FP64 master rows [3][ny] (A1, Bref_1, Bref_2), then the next rows
    float *reft = nullptr;                       // FP32 tables u1r [ny], brow [2][ny], bpull [4][ny]
    int ref_every = 0;                           // steps between refreshes (0: the reference stays as created)
    long long ref_next = 0;                      // step count at which the next refresh is due
    // slab of a larger lattice (goc_create_slab): global rows [slab_r0, slab_r1)
    // owned, slab_glo / slab_ghi ghost rows below / above them
    bool slab = false;
    int slab_r0 = 0, slab_r1 = 0, slab_glo = 0, slab_ghi = 0;
    // in place (goc_exec.streaming = 1, goc_aa.cuh): f[1] and F[1] name the
    // single buffers f[0], F[0]; cur names the layout of the populations
    // (fresh: f^0; else 1 after odd steps, 0 after even ones)
    bool aa = false;
    float *aa_fld = nullptr;                     // [3][plane] rho - rho0, U1, U2 of the step in progress
    float *aa_wsum = nullptr;                    // [4][aa_wn] population sums of the wall nodes
    int aa_wn = 0;
};

// Per-storage-type launchers (S = float, __half, __nv_bfloat16), defined in
// goc_kernels_<type>.cu: one time step of a lattice, and the persistent grid
// and launch of the batch kernel of a group (mhd: MIE on, geom: grid kind).
template <class S> goc_status launch_step_t(goc_lattice *L, const StepParams &p);
template <class S> int batch_grid_t(int mhd, int geom, int *stage_bytes);
template <class S>
cudaError_t batch_launch_t(int mhd, int geom, dim3 gd, dim3 bd, size_t smem, cudaStream_t st, const goc::BatchArgs &a);
// in-place lattices (goc_kernels_<type>.cu): one step (fields pass, then
// collision pass), and the macroscopic fields into out ([5][ny][nx] FP64)
template <class S> goc_status launch_aa_step_t(goc_lattice *L, const StepParams &p);
template <class S> goc_status launch_aa_moments_t(goc_lattice *L, const StepParams &p, double *out);
#define GOC_DECLARE_LAUNCHERS(S)                                                                         \
    extern template goc_status launch_aa_step_t<S>(goc_lattice *, const StepParams &);                  \
    extern template goc_status launch_aa_moments_t<S>(goc_lattice *, const StepParams &, double *);     \
    extern template goc_status launch_step_t<S>(goc_lattice *, const StepParams &);                     \
    extern template int batch_grid_t<S>(int, int, int *);                                                \
    extern template cudaError_t batch_launch_t<S>(int, int, dim3, dim3, size_t, cudaStream_t, const goc::BatchArgs &);
GOC_DECLARE_LAUNCHERS(float)
GOC_DECLARE_LAUNCHERS(__half)
GOC_DECLARE_LAUNCHERS(__nv_bfloat16)
