// goc_kernels_f32.cu -- the kernels of storage type float and their launchers,
// and those of the in-place lattices (FP32 only).
#include "goc_aa.cuh"
#include "goc_launch.cuh"

GOC_DEFINE_LAUNCHERS(float)

template <int LAY>
static goc_status launch_aa_layout(goc_lattice *L, const StepParams &p) {
    const dim3 grid((L->nx + TX - 1) / TX, (L->ny + TY - 1) / TY), block(TX, TY);
    const bool pdl = L->cfg_pdl != 0;
    const float *fld = L->aa_fld, *wsum = L->aa_wsum;
    CU(launch_pdl(pdl, aa_fields_kernel<LAY>, grid, block, 0, L->stream, p, L->aa_fld, L->aa_wsum, L->aa_wn));
    if (L->mhd.enabled)
        CU(launch_pdl(pdl, aa_collide_kernel<LAY, true>, grid, block, 0, L->stream, p, fld, wsum, L->aa_wn));
    else
        CU(launch_pdl(pdl, aa_collide_kernel<LAY, false>, grid, block, 0, L->stream, p, fld, wsum, L->aa_wn));
    return GOC_OK;
}

goc_status launch_aa_step(goc_lattice *L, const StepParams &p) {
    if (L->fresh) return launch_aa_layout<AA_C>(L, p);
    return L->cur ? launch_aa_layout<AA_S>(L, p) : launch_aa_layout<AA_T>(L, p);
}

goc_status launch_aa_moments(goc_lattice *L, const StepParams &p, double *out) {
    const dim3 grid((L->nx + 127) / 128, L->ny), block(128);
    const int lay = L->fresh ? AA_C : (L->cur ? AA_S : AA_T);
    if (L->mhd.enabled) {
        if (lay == AA_C) aa_moments_kernel<AA_C, true><<<grid, block, 0, L->stream>>>(p, out);
        else if (lay == AA_S) aa_moments_kernel<AA_S, true><<<grid, block, 0, L->stream>>>(p, out);
        else aa_moments_kernel<AA_T, true><<<grid, block, 0, L->stream>>>(p, out);
    } else {
        if (lay == AA_C) aa_moments_kernel<AA_C, false><<<grid, block, 0, L->stream>>>(p, out);
        else if (lay == AA_S) aa_moments_kernel<AA_S, false><<<grid, block, 0, L->stream>>>(p, out);
        else aa_moments_kernel<AA_T, false><<<grid, block, 0, L->stream>>>(p, out);
    }
    CU(cudaGetLastError());
    return GOC_OK;
}
