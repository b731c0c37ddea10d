// fam_sw2.cu -- shallow water D2Q4 (M = 3): kernels and launchers.
#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_sw2(bool fp64, int om, const StageLaunch &L)
{
    return stage_family<ShallowWater<2>, 2>(fp64, om, L);
}

cudaError_t step2d_sw2(bool fp64, int om, const Step2dLaunch &L)
{
    return step2d_family<ShallowWater<2>>(fp64, om, L);
}

cudaError_t adjoint_sw2(bool fp64, int om, const AdjointLaunch &L)
{
    return adjoint_family<ShallowWater<2>, 2>(fp64, om, L);
}

cudaError_t adjoint_init_sw2(bool fp64, const double *u0, const void *g, double *du0, int64_t ncell, const Params &P,
                             cudaStream_t st)
{
    return adjoint_init_family<ShallowWater<2>>(fp64, u0, g, du0, ncell, P, st);
}

cudaError_t batch_sw2(bool fp64, int om, const BatchLaunch &L)
{
    return batch_family<ShallowWater<2>>(fp64, om, L);
}

int batch_occ_sw2(bool fp64, int om) { return batch_occ_family<ShallowWater<2>>(fp64, om); }

cudaError_t init_sw2(bool fp64, const double *u0, void *f, int64_t ncell, const Params &P, Counters *cnt,
                     cudaStream_t st)
{
    return init_family<ShallowWater<2>>(fp64, u0, f, ncell, P, cnt, st);
}

cudaError_t totals_sw2(bool fp64, const void *f, double *partials, double *out, int64_t nx, int64_t ny,
                       const Shift &sh, const Params &P, cudaStream_t st)
{
    return totals_family<ShallowWater<2>, 2>(fp64, f, partials, out, nx, ny, sh, P, st);
}

cudaError_t check_sw2(bool fp64, int om, const Params &P, Counters *cnt, cudaStream_t st)
{
    return check_family<ShallowWater<2>>(fp64, om, P, cnt, st);
}

cudaError_t batch_adjoint_sw2(bool fp64, int om, const BatchAdjointLaunch &L)
{
    return batch_adjoint_family<ShallowWater<2>>(fp64, om, L);
}

int batch_adjoint_occ_sw2(bool fp64, int om) { return batch_adjoint_occ_family<ShallowWater<2>>(fp64, om); }

}  // namespace eslbm
