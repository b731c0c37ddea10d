// fam_euler.cu -- Euler D2Q4 (M = 4, fixed omega): kernels and launchers.
#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_euler(bool fp64, const StageLaunch &L) { return stage_family<Euler2, 2>(fp64, OM_FIXED, L); }

cudaError_t step2d_euler(bool fp64, const Step2dLaunch &L) { return step2d_family<Euler2>(fp64, OM_FIXED, L); }

cudaError_t init_euler(bool fp64, const double *u0, void *f, int64_t ncell, const Params &P, Counters *cnt,
                       cudaStream_t st)
{
    return init_family<Euler2>(fp64, u0, f, ncell, P, cnt, st);
}

cudaError_t totals_euler(bool fp64, const void *f, double *partials, double *out, int64_t nx, int64_t ny,
                         const Shift &sh, const Params &P, cudaStream_t st)
{
    return totals_family<Euler2, 2>(fp64, f, partials, out, nx, ny, sh, P, st);
}

cudaError_t adjoint_euler(bool fp64, const AdjointLaunch &L) { return adjoint_family<Euler2, 2>(fp64, OM_FIXED, L); }

cudaError_t adjoint_init_euler(bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                               const Params &P, cudaStream_t st)
{
    return adjoint_init_family<Euler2>(fp64, u0, g, du0, ncell, P, st);
}

cudaError_t batch_euler(bool fp64, const BatchLaunch &L) { return batch_family<Euler2>(fp64, OM_FIXED, L); }

int batch_occ_euler(bool fp64) { return batch_occ_family<Euler2>(fp64, OM_FIXED); }

cudaError_t batch_adjoint_euler(bool fp64, const BatchAdjointLaunch &L)
{
    return batch_adjoint_family<Euler2>(fp64, OM_FIXED, L);
}

int batch_adjoint_occ_euler(bool fp64) { return batch_adjoint_occ_family<Euler2>(fp64, OM_FIXED); }

}  // namespace eslbm
