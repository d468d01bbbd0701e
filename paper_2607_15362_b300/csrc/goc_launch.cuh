// goc_launch.cuh -- the kernel launchers of one storage type S (included by
// goc_kernels_<type>.cu, which instantiate them): the step kernels of a
// single lattice (straight, curvilinear-column and node-table grids; central-
// or raw-moment collisions; with or without the MIE), the standard uniform-
// grid comparator, and the batch kernels.
#pragma once

#include <algorithm>

#include "goc_aa.cuh"
#include "goc_internal.h"
#include "goc_lean.cuh"
#include "goc_std.cuh"

using namespace goc;

namespace {

// Persistent grid size of a tiled step kernel: resident blocks per SM x SMs
// (found once per kernel, `cached`), or with `balanced` the fewest blocks that
// take the same number of rounds of tiles (equal shares).
template <class K>
int persistent_grid(K kern, size_t bytes, int ntiles, bool balanced, int &cached) {
    if (cached < 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, bytes);
        cached = std::max(1, sms * std::max(1, per));
    }
    if (balanced) {
        const int rounds = (ntiles + cached - 1) / cached;
        return (ntiles + rounds - 1) / rounds;
    }
    return std::min(ntiles, cached);
}

// Dynamic shared memory of a step kernel (two stages) and its persistent grid size.
template <class S, bool MHD, bool SRT = false, int GEOM = 0>
int step_grid(int ntiles, size_t *smem, bool balanced = false) {
    using T = Tiling<S>;
    const size_t bytes = 2 * (size_t)(MHD ? T::STAGE_MHD : T::STAGE_NSE);
    *smem = bytes;
    static int cached = -1;
    return persistent_grid(step_kernel<S, MHD, SRT, GEOM>, bytes, ntiles, balanced, cached);
}

// The same for the straight-grid kernel lean_step_kernel.
template <class S, bool MHD, bool SEAMS>
int lean_grid(int ntiles, size_t *smem, bool balanced = false) {
    using T = Tiling<S>;
    const size_t bytes = 2 * (size_t)(MHD ? T::STAGE_MHD : T::STAGE_NSE);
    *smem = bytes;
    static int cached = -1;
    return persistent_grid(lean_step_kernel<S, MHD, SEAMS>, bytes, ntiles, balanced, cached);
}

// Launch lean_step_kernel with or without the seam path (kind-3 tiles exist
// only for FP32 lattices periodic along xi1 whose width is a multiple of 32).
template <class S, bool MHD>
cudaError_t launch_lean(goc_lattice *L, const StepParams &p, int ntiles, bool pdl) {
    size_t smem = 0;
    if constexpr (!Store<S>::scaled) {
        if (L->sp.per_x && L->nx % TX == 0) {
            const int grid = lean_grid<S, MHD, true>(ntiles, &smem, L->cfg_balanced != 0);
            return launch_pdl(pdl, lean_step_kernel<S, MHD, true>, dim3(grid), dim3(TX, TYT), smem, L->stream, p);
        }
    }
    const int grid = lean_grid<S, MHD, false>(ntiles, &smem, L->cfg_balanced != 0);
    return launch_pdl(pdl, lean_step_kernel<S, MHD, false>, dim3(grid), dim3(TX, TYT), smem, L->stream, p);
}

// The same for the 32 x 16 tile kernel lean2_step_kernel.
template <class S, bool MHD>
int lean2_grid(int ntiles, size_t *smem, bool balanced = false) {
    using T = Tiling2<S>;
    const size_t bytes = (size_t)T::NSTAGE * T::STAGE;
    *smem = bytes;
    static int cached = -1;
    return persistent_grid(lean2_step_kernel<S, MHD>, bytes, ntiles, balanced, cached);
}

// Straight grids with the central-moment collision run lean_step_kernel
// unless GOC_GENERAL_KERNEL is set (the general tile path of step_kernel, for
// comparisons).
inline bool lean_enabled() {
    static const bool on = std::getenv("GOC_GENERAL_KERNEL") == nullptr;
    return on;
}

template <class S>
goc_status launch_std_t(goc_lattice *L, const StepParams &p) {
    dim3 grid((L->nx + STD_BX - 1) / STD_BX, (L->ny + STD_BY - 1) / STD_BY), block(STD_BX, STD_BY);
    CU(launch_pdl(L->cfg_pdl != 0, std_step_kernel<S>, grid, block, 0, L->stream, p));
    return GOC_OK;
}

// Curved grids (GEOM 1, 2): the step kernel for the lattice's collision
// (central moments, or raw moments for schemes 2 and 3) and MIE setting.
template <class S, int GEOM>
cudaError_t launch_geom(goc_lattice *L, const StepParams &p, int ntiles) {
    size_t smem = 0;
    const bool pdl = L->cfg_pdl != 0, raw = L->scheme == 2 || L->scheme == 3;
    const dim3 block(TX, TYT);
    if (L->mhd.enabled && raw) {
        const int grid = step_grid<S, true, true, GEOM>(ntiles, &smem, L->cfg_balanced != 0);
        return launch_pdl(pdl, step_kernel<S, true, true, GEOM>, dim3(grid), block, smem, L->stream, p);
    }
    if (L->mhd.enabled) {
        const int grid = step_grid<S, true, false, GEOM>(ntiles, &smem, L->cfg_balanced != 0);
        return launch_pdl(pdl, step_kernel<S, true, false, GEOM>, dim3(grid), block, smem, L->stream, p);
    }
    if (raw) {
        const int grid = step_grid<S, false, true, GEOM>(ntiles, &smem, L->cfg_balanced != 0);
        return launch_pdl(pdl, step_kernel<S, false, true, GEOM>, dim3(grid), block, smem, L->stream, p);
    }
    const int grid = step_grid<S, false, false, GEOM>(ntiles, &smem, L->cfg_balanced != 0);
    return launch_pdl(pdl, step_kernel<S, false, false, GEOM>, dim3(grid), block, smem, L->stream, p);
}


template <class S, bool MHD, int GEOM>
int persistent_grid_t(int total, int *stage_bytes) {
    using T = Tiling<S>;
    const int stage = MHD ? T::STAGE_MHD : T::STAGE_NSE;
    *stage_bytes = stage;
    static int cached = -1;
    if (cached < 0) {
        cudaFuncSetAttribute(batch_step_kernel<S, MHD, GEOM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * stage);
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_step_kernel<S, MHD, GEOM>, NT, 2 * (size_t)stage);
        cached = std::max(1, sms * std::max(1, per));
    }
    return std::min(total, cached);
}


template <class S, int GEOM>
int batch_grid_g(int mhd, int *stage_bytes) {
    return mhd ? persistent_grid_t<S, true, GEOM>(1 << 30, stage_bytes)
               : persistent_grid_t<S, false, GEOM>(1 << 30, stage_bytes);
}

}  // namespace

template <class S>
goc_status launch_step_t(goc_lattice *L, const StepParams &p) {
    if (L->scheme == 1) return launch_std_t<S>(L, p);
    const int ntiles = ((L->nx + TX - 1) / TX) * ((L->ny + TY - 1) / TY);
    size_t smem = 0;
    const bool pdl = L->cfg_pdl != 0;
    if (L->sp.curv == 2) {   // node-table metric
        const cudaError_t e = launch_geom<S, 2>(L, p, ntiles);
        CU(e);
    } else if (L->sp.curv) {   // curvilinear column metric
        const cudaError_t e = launch_geom<S, 1>(L, p, ntiles);
        CU(e);
    } else if (L->scheme == 2 || L->scheme == 3) {   // collision on raw moments (Appendix F SRT, Appendix D MRT)
        if (L->mhd.enabled) {
            const int grid = step_grid<S, true, true>(ntiles, &smem, L->cfg_balanced != 0);
            CU(launch_pdl(pdl, step_kernel<S, true, true>, dim3(grid), dim3(TX, TYT), smem, L->stream, p));
        } else {
            const int grid = step_grid<S, false, true>(ntiles, &smem, L->cfg_balanced != 0);
            CU(launch_pdl(pdl, step_kernel<S, false, true>, dim3(grid), dim3(TX, TYT), smem, L->stream, p));
        }
    } else if (lean_enabled() && L->cfg_rows == 2 && L->tma_ok) {   // 32 x 16 tiles
        StepParams q = p;
        q.tm_f = L->tmf2[L->cur];
        q.tm_F = L->tmF2[L->cur];
        const int nt2 = ((L->nx + TX - 1) / TX) * ((L->ny + 2 * TY - 1) / (2 * TY));
        if (L->mhd.enabled) {
            const int grid = lean2_grid<S, true>(nt2, &smem, L->cfg_balanced != 0);
            CU(launch_pdl(pdl, lean2_step_kernel<S, true>, dim3(grid), dim3(TX, TYT), smem, L->stream, q));
        } else {
            const int grid = lean2_grid<S, false>(nt2, &smem, L->cfg_balanced != 0);
            CU(launch_pdl(pdl, lean2_step_kernel<S, false>, dim3(grid), dim3(TX, TYT), smem, L->stream, q));
        }
    } else if (lean_enabled() && L->mhd.enabled) {
        CU((launch_lean<S, true>(L, p, ntiles, pdl)));
    } else if (lean_enabled()) {
        CU((launch_lean<S, false>(L, p, ntiles, pdl)));
    } else if (L->mhd.enabled) {
        const int grid = step_grid<S, true>(ntiles, &smem, L->cfg_balanced != 0);
        CU(launch_pdl(pdl, step_kernel<S, true>, dim3(grid), dim3(TX, TYT), smem, L->stream, p));
    } else {
        const int grid = step_grid<S, false>(ntiles, &smem, L->cfg_balanced != 0);
        CU(launch_pdl(pdl, step_kernel<S, false>, dim3(grid), dim3(TX, TYT), smem, L->stream, p));
    }
    CU(cudaGetLastError());
    return GOC_OK;
}

template <class S>
int batch_grid_t(int mhd, int geom, int *stage_bytes) {
    return geom == 2 ? batch_grid_g<S, 2>(mhd, stage_bytes)
           : geom == 1 ? batch_grid_g<S, 1>(mhd, stage_bytes)
                       : batch_grid_g<S, 0>(mhd, stage_bytes);
}

template <class S>
cudaError_t batch_launch_t(int mhd, int geom, dim3 gd, dim3 bd, size_t smem, cudaStream_t st, const BatchArgs &a) {
    switch (2 * geom + (mhd ? 1 : 0)) {
        case 5: return launch_pdl(true, batch_step_kernel<S, true, 2>, gd, bd, smem, st, a);
        case 4: return launch_pdl(true, batch_step_kernel<S, false, 2>, gd, bd, smem, st, a);
        case 3: return launch_pdl(true, batch_step_kernel<S, true, 1>, gd, bd, smem, st, a);
        case 2: return launch_pdl(true, batch_step_kernel<S, false, 1>, gd, bd, smem, st, a);
        case 1: return launch_pdl(true, batch_step_kernel<S, true, 0>, gd, bd, smem, st, a);
        default: return launch_pdl(true, batch_step_kernel<S, false, 0>, gd, bd, smem, st, a);
    }
}

// In-place lattices (goc_aa.cuh): one step, a fields pass and a collision
// pass in the kernels of the layout the populations are in (f^0; the link
// reversed at the node, after odd steps; at the destination, after even ones).
template <class S, int LAY>
goc_status launch_aa_layout(goc_lattice *L, const StepParams &p) {
    const dim3 grid((L->nx + TX - 1) / TX, (L->ny + TY - 1) / TY), block(TX, TY);
    const bool pdl = L->cfg_pdl != 0;
    const float *fld = L->aa_fld, *wsum = L->aa_wsum;
    CU(launch_pdl(pdl, aa_fields_kernel<S, LAY>, grid, block, 0, L->stream, p, L->aa_fld, L->aa_wsum, L->aa_wn));
    if (L->mhd.enabled)
        CU(launch_pdl(pdl, aa_collide_kernel<S, LAY, true>, grid, block, 0, L->stream, p, fld, wsum, L->aa_wn));
    else
        CU(launch_pdl(pdl, aa_collide_kernel<S, LAY, false>, grid, block, 0, L->stream, p, fld, wsum, L->aa_wn));
    return GOC_OK;
}

template <class S>
goc_status launch_aa_step_t(goc_lattice *L, const StepParams &p) {
    if (L->fresh) return launch_aa_layout<S, AA_C>(L, p);
    return L->cur ? launch_aa_layout<S, AA_S>(L, p) : launch_aa_layout<S, AA_T>(L, p);
}

template <class S>
goc_status launch_aa_moments_t(goc_lattice *L, const StepParams &p, double *out) {
    const dim3 grid((L->nx + 127) / 128, L->ny), block(128);
    const int lay = L->fresh ? AA_C : (L->cur ? AA_S : AA_T);
    if (L->mhd.enabled) {
        if (lay == AA_C) aa_moments_kernel<S, AA_C, true><<<grid, block, 0, L->stream>>>(p, out);
        else if (lay == AA_S) aa_moments_kernel<S, AA_S, true><<<grid, block, 0, L->stream>>>(p, out);
        else aa_moments_kernel<S, AA_T, true><<<grid, block, 0, L->stream>>>(p, out);
    } else {
        if (lay == AA_C) aa_moments_kernel<S, AA_C, false><<<grid, block, 0, L->stream>>>(p, out);
        else if (lay == AA_S) aa_moments_kernel<S, AA_S, false><<<grid, block, 0, L->stream>>>(p, out);
        else aa_moments_kernel<S, AA_T, false><<<grid, block, 0, L->stream>>>(p, out);
    }
    CU(cudaGetLastError());
    return GOC_OK;
}

#define GOC_DEFINE_LAUNCHERS(S)                                                                   \
    template goc_status launch_aa_step_t<S>(goc_lattice *, const StepParams &);                  \
    template goc_status launch_aa_moments_t<S>(goc_lattice *, const StepParams &, double *);     \
    template goc_status launch_step_t<S>(goc_lattice *, const StepParams &);                     \
    template int batch_grid_t<S>(int, int, int *);                                                \
    template cudaError_t batch_launch_t<S>(int, int, dim3, dim3, size_t, cudaStream_t, const BatchArgs &);
