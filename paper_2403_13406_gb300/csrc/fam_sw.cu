// fam_sw.cu -- shallow water, D1Q2 (M = 2) and D2Q4 (M = 3).
#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_sw(int family, bool fp64, bool entropic, bool diag, const StageLaunch &L)
{
    if (family == FAM_SW1) return stage_family<ShallowWater<1>, 1>(fp64, entropic, diag, L);
    if (family == FAM_SW2) return stage_family<ShallowWater<2>, 2>(fp64, entropic, diag, L);
    return cudaErrorInvalidValue;
}

cudaError_t fused_sw(int family, bool fp64, bool entropic, const FusedLaunch &L)
{
    if (family == FAM_SW1) return fused_family<ShallowWater<1>>(fp64, entropic, L);
    return cudaErrorInvalidValue;
}

cudaError_t adjoint_sw(int family, bool fp64, bool entropic, const AdjointLaunch &L)
{
    if (family == FAM_SW1) return adjoint_family<ShallowWater<1>, 1>(fp64, entropic, L);
    if (family == FAM_SW2) return adjoint_family<ShallowWater<2>, 2>(fp64, entropic, L);
    return cudaErrorInvalidValue;
}

cudaError_t adjoint_init_sw(int family, bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                            const Params &P, cudaStream_t st)
{
    if (family == FAM_SW1) return adjoint_init_family<ShallowWater<1>>(fp64, u0, g, du0, ncell, P, st);
    if (family == FAM_SW2) return adjoint_init_family<ShallowWater<2>>(fp64, u0, g, du0, ncell, P, st);
    return cudaErrorInvalidValue;
}

cudaError_t batch_sw(int family, bool fp64, bool entropic, const BatchLaunch &L)
{
    if (family == FAM_SW2) return batch_family<ShallowWater<2>>(fp64, entropic, L);
    return cudaErrorInvalidValue;
}

int batch_occ_sw(int family, bool fp64, bool entropic)
{
    if (family == FAM_SW2) return batch_occ_family<ShallowWater<2>>(fp64, entropic);
    return 0;
}

cudaError_t init_sw(int family, bool fp64, const double *u0, void *f, int64_t ncell, const Params &P,
                    Counters *cnt, cudaStream_t st)
{
    if (family == FAM_SW1) return init_family<ShallowWater<1>>(fp64, u0, f, ncell, P, cnt, st);
    if (family == FAM_SW2) return init_family<ShallowWater<2>>(fp64, u0, f, ncell, P, cnt, st);
    return cudaErrorInvalidValue;
}

cudaError_t totals_sw(int family, bool fp64, const void *f, double *partials, double *out, int64_t nx, int64_t ny,
                      const Shift &sh, const Params &P, cudaStream_t st)
{
    if (family == FAM_SW1) return totals_family<ShallowWater<1>, 1>(fp64, f, partials, out, nx, ny, sh, P, st);
    if (family == FAM_SW2) return totals_family<ShallowWater<2>, 2>(fp64, f, partials, out, nx, ny, sh, P, st);
    return cudaErrorInvalidValue;
}

}  // namespace eslbm
