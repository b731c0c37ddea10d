// fam_sw1.cu -- shallow water D1Q2 (M = 2): kernels and launchers.
#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_sw1(bool fp64, int om, const StageLaunch &L)
{
    return stage_family<ShallowWater<1>, 1>(fp64, om, L);
}

cudaError_t fused_sw1(bool fp64, int om, const FusedLaunch &L)
{
    return fused_family<ShallowWater<1>>(fp64, om, L);
}

cudaError_t adjoint_sw1(bool fp64, int om, const AdjointLaunch &L)
{
    return adjoint_family<ShallowWater<1>, 1>(fp64, om, L);
}

cudaError_t adjoint_init_sw1(bool fp64, const double *u0, const void *g, double *du0, int64_t ncell, const Params &P,
                             cudaStream_t st)
{
    return adjoint_init_family<ShallowWater<1>>(fp64, u0, g, du0, ncell, P, st);
}

cudaError_t init_sw1(bool fp64, const double *u0, void *f, int64_t ncell, const Params &P, Counters *cnt,
                     cudaStream_t st)
{
    return init_family<ShallowWater<1>>(fp64, u0, f, ncell, P, cnt, st);
}

cudaError_t totals_sw1(bool fp64, const void *f, double *partials, double *out, int64_t nx, int64_t ny,
                       const Shift &sh, const Params &P, cudaStream_t st)
{
    return totals_family<ShallowWater<1>, 1>(fp64, f, partials, out, nx, ny, sh, P, st);
}

cudaError_t check_sw1(bool fp64, int om, const Params &P, Counters *cnt, cudaStream_t st)
{
    return check_family<ShallowWater<1>>(fp64, om, P, cnt, st);
}

}  // namespace eslbm
