// goc_kernels_f32.cu -- the kernels of storage type float and their launchers,
// and those of the in-place lattices (FP32 only).
#include "goc_aa.cuh"
#include "goc_launch.cuh"

GOC_DEFINE_LAUNCHERS(float)

template <int LAY>
static goc_status launch_aa_layout(goc_lattice *L, const StepParams &p) {
    const dim3 grid((L->nx + TX - 1) / TX, (L->ny + TY - 1) / TY), block(TX, TY);
    const bool pdl = L->cfg_pdl != 0;
    CU(launch_pdl(pdl, aa_fields_kernel<LAY>, grid, block, 0, L->stream, p, L->aa_fld, L->aa_wsum, L->aa_wn));
    CU(launch_pdl(pdl, aa_collide_kernel<LAY>, grid, block, 0, L->stream, p, static_cast<const float *>(L->aa_fld),
                  static_cast<const float *>(L->aa_wsum), L->aa_wn));
    return GOC_OK;
}

goc_status launch_aa_step(goc_lattice *L, const StepParams &p) {
    if (L->fresh) return launch_aa_layout<AA_C>(L, p);
    return L->cur ? launch_aa_layout<AA_S>(L, p) : launch_aa_layout<AA_T>(L, p);
}

goc_status launch_aa_moments(goc_lattice *L, const StepParams &p, double *out) {
    const dim3 grid((L->nx + 127) / 128, L->ny), block(128);
    if (L->fresh) aa_moments_kernel<AA_C><<<grid, block, 0, L->stream>>>(p, out);
    else if (L->cur) aa_moments_kernel<AA_S><<<grid, block, 0, L->stream>>>(p, out);
    else aa_moments_kernel<AA_T><<<grid, block, 0, L->stream>>>(p, out);
    CU(cudaGetLastError());
    return GOC_OK;
}
