// fam_scalar.cu -- linear transport and Burgers (M = 1), D1Q2 and D2Q4.
#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_scalar(int family, bool fp64, int om, const StageLaunch &L)
{
    switch (family) {
    case FAM_LINEAR1: return stage_family<Scalar<1, false>, 1>(fp64, om, L);
    case FAM_LINEAR2: return stage_family<Scalar<2, false>, 2>(fp64, om, L);
    case FAM_BURGERS1: return stage_family<Scalar<1, true>, 1>(fp64, om, L);
    case FAM_BURGERS2: return stage_family<Scalar<2, true>, 2>(fp64, om, L);
    }
    return cudaErrorInvalidValue;
}

cudaError_t step2d_scalar(int family, bool fp64, int om, const Step2dLaunch &L)
{
    if (family == FAM_LINEAR2) return step2d_family<Scalar<2, false>>(fp64, om, L);
    if (family == FAM_BURGERS2) return step2d_family<Scalar<2, true>>(fp64, om, L);
    return cudaErrorInvalidValue;
}

cudaError_t fused_scalar(int family, bool fp64, int om, const FusedLaunch &L)
{
    if (family == FAM_LINEAR1) return fused_family<Scalar<1, false>>(fp64, om, L);
    if (family == FAM_BURGERS1) return fused_family<Scalar<1, true>>(fp64, om, L);
    return cudaErrorInvalidValue;
}

cudaError_t adjoint_scalar(int family, bool fp64, int om, const AdjointLaunch &L)
{
    switch (family) {
    case FAM_LINEAR1: return adjoint_family<Scalar<1, false>, 1>(fp64, om, L);
    case FAM_LINEAR2: return adjoint_family<Scalar<2, false>, 2>(fp64, om, L);
    case FAM_BURGERS1: return adjoint_family<Scalar<1, true>, 1>(fp64, om, L);
    case FAM_BURGERS2: return adjoint_family<Scalar<2, true>, 2>(fp64, om, L);
    }
    return cudaErrorInvalidValue;
}

cudaError_t adjoint_init_scalar(int family, bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                                const Params &P, cudaStream_t st)
{
    switch (family) {
    case FAM_LINEAR1: return adjoint_init_family<Scalar<1, false>>(fp64, u0, g, du0, ncell, P, st);
    case FAM_LINEAR2: return adjoint_init_family<Scalar<2, false>>(fp64, u0, g, du0, ncell, P, st);
    case FAM_BURGERS1: return adjoint_init_family<Scalar<1, true>>(fp64, u0, g, du0, ncell, P, st);
    case FAM_BURGERS2: return adjoint_init_family<Scalar<2, true>>(fp64, u0, g, du0, ncell, P, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_scalar(int family, bool fp64, int om, const BatchLaunch &L)
{
    if (family == FAM_LINEAR2) return batch_family<Scalar<2, false>>(fp64, om, L);
    if (family == FAM_BURGERS2) return batch_family<Scalar<2, true>>(fp64, om, L);
    return cudaErrorInvalidValue;
}

int batch_occ_scalar(int family, bool fp64, int om)
{
    if (family == FAM_LINEAR2) return batch_occ_family<Scalar<2, false>>(fp64, om);
    if (family == FAM_BURGERS2) return batch_occ_family<Scalar<2, true>>(fp64, om);
    return 0;
}

cudaError_t init_scalar(int family, bool fp64, const double *u0, void *f, int64_t ncell, const Params &P,
                        Counters *cnt, cudaStream_t st)
{
    switch (family) {
    case FAM_LINEAR1: return init_family<Scalar<1, false>>(fp64, u0, f, ncell, P, cnt, st);
    case FAM_LINEAR2: return init_family<Scalar<2, false>>(fp64, u0, f, ncell, P, cnt, st);
    case FAM_BURGERS1: return init_family<Scalar<1, true>>(fp64, u0, f, ncell, P, cnt, st);
    case FAM_BURGERS2: return init_family<Scalar<2, true>>(fp64, u0, f, ncell, P, cnt, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t totals_scalar(int family, bool fp64, const void *f, double *partials, double *out, int64_t nx,
                          int64_t ny, const Shift &sh, const Params &P, cudaStream_t st)
{
    switch (family) {
    case FAM_LINEAR1: return totals_family<Scalar<1, false>, 1>(fp64, f, partials, out, nx, ny, sh, P, st);
    case FAM_LINEAR2: return totals_family<Scalar<2, false>, 2>(fp64, f, partials, out, nx, ny, sh, P, st);
    case FAM_BURGERS1: return totals_family<Scalar<1, true>, 1>(fp64, f, partials, out, nx, ny, sh, P, st);
    case FAM_BURGERS2: return totals_family<Scalar<2, true>, 2>(fp64, f, partials, out, nx, ny, sh, P, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t check_scalar(int family, bool fp64, int om, const Params &P, Counters *cnt, cudaStream_t st)
{
    if (family == FAM_BURGERS1) return check_family<Scalar<1, true>>(fp64, om, P, cnt, st);
    if (family == FAM_BURGERS2) return check_family<Scalar<2, true>>(fp64, om, P, cnt, st);
    return cudaSuccess;
}

cudaError_t batch_adjoint_scalar(int family, bool fp64, int om, const BatchAdjointLaunch &L)
{
    if (family == FAM_LINEAR2) return batch_adjoint_family<Scalar<2, false>>(fp64, om, L);
    if (family == FAM_BURGERS2) return batch_adjoint_family<Scalar<2, true>>(fp64, om, L);
    return cudaErrorInvalidValue;
}

int batch_adjoint_occ_scalar(int family, bool fp64, int om)
{
    if (family == FAM_LINEAR2) return batch_adjoint_occ_family<Scalar<2, false>>(fp64, om);
    if (family == FAM_BURGERS2) return batch_adjoint_occ_family<Scalar<2, true>>(fp64, om);
    return 0;
}

}  // namespace eslbm
