// fam_misc.cu -- Euler (fixed omega), gathers, conversion and the dispatch
// entry points declared in launch.h.
#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_scalar(int, bool, bool, bool, const StageLaunch &);
cudaError_t stage_sw(int, bool, bool, bool, const StageLaunch &);
cudaError_t init_scalar(int, bool, const double *, void *, int64_t, const Params &, Counters *, cudaStream_t);
cudaError_t init_sw(int, bool, const double *, void *, int64_t, const Params &, Counters *, cudaStream_t);
cudaError_t totals_scalar(int, bool, const void *, double *, double *, int64_t, int64_t, const Shift &,
                          const Params &, cudaStream_t);
cudaError_t totals_sw(int, bool, const void *, double *, double *, int64_t, int64_t, const Shift &, const Params &,
                      cudaStream_t);

cudaError_t fused_scalar(int, bool, bool, const FusedLaunch &);
cudaError_t fused_sw(int, bool, bool, const FusedLaunch &);

cudaError_t launch_fused1d(int family, bool fp64, bool entropic, const FusedLaunch &L)
{
    if (family == FAM_SW1) return fused_sw(family, fp64, entropic, L);
    if (family == FAM_LINEAR1 || family == FAM_BURGERS1) return fused_scalar(family, fp64, entropic, L);
    return cudaErrorInvalidValue;
}

cudaError_t launch_stage(int family, bool fp64, bool entropic, bool diag, const StageLaunch &L)
{
    if (family == FAM_SW1 || family == FAM_SW2) return stage_sw(family, fp64, entropic, diag, L);
    if (family == FAM_EULER2) return stage_family<Euler2, 2>(fp64, false, false, L);
    return stage_scalar(family, fp64, entropic, diag, L);
}

cudaError_t launch_init_eq(int family, bool fp64, const double *u0, void *f, int64_t ncell, const Params &P,
                           Counters *cnt, cudaStream_t st)
{
    if (family == FAM_SW1 || family == FAM_SW2) return init_sw(family, fp64, u0, f, ncell, P, cnt, st);
    if (family == FAM_EULER2) return init_family<Euler2>(fp64, u0, f, ncell, P, cnt, st);
    return init_scalar(family, fp64, u0, f, ncell, P, cnt, st);
}

cudaError_t launch_totals(int family, bool fp64, const void *f, double *partials, double *out, int64_t nx,
                          int64_t ny, const Shift &sh, const Params &P, cudaStream_t st)
{
    if (family == FAM_SW1 || family == FAM_SW2) return totals_sw(family, fp64, f, partials, out, nx, ny, sh, P, st);
    if (family == FAM_EULER2) return totals_family<Euler2, 2>(fp64, f, partials, out, nx, ny, sh, P, st);
    return totals_scalar(family, fp64, f, partials, out, nx, ny, sh, P, st);
}

template <int DIM, class R, bool MOM>
static cudaError_t gather_t(const void *f, double *out, int64_t nx, int64_t ny, int M, int p0, int np,
                            const Shift &sh, cudaStream_t st)
{
    dim3 grid((unsigned)((nx + kBlock - 1) / kBlock), (unsigned)ny);
    k_gather<DIM, R, MOM><<<grid, kBlock, 0, st>>>((const R *)f, out, nx, ny, M, p0, np, sh);
    return cudaGetLastError();
}

cudaError_t launch_gather_moments(int dim, bool fp64, const void *f, double *out, int64_t nx, int64_t ny, int M,
                                  const Shift &sh, cudaStream_t st)
{
    if (dim == 1)
        return fp64 ? gather_t<1, double, true>(f, out, nx, ny, M, 0, 0, sh, st)
                    : gather_t<1, float, true>(f, out, nx, ny, M, 0, 0, sh, st);
    return fp64 ? gather_t<2, double, true>(f, out, nx, ny, M, 0, 0, sh, st)
                : gather_t<2, float, true>(f, out, nx, ny, M, 0, 0, sh, st);
}

cudaError_t launch_gather_planes(int dim, bool fp64, const void *f, double *out, int64_t nx, int64_t ny, int M,
                                 int plane0, int nplanes, const Shift &sh, cudaStream_t st)
{
    if (dim == 1)
        return fp64 ? gather_t<1, double, false>(f, out, nx, ny, M, plane0, nplanes, sh, st)
                    : gather_t<1, float, false>(f, out, nx, ny, M, plane0, nplanes, sh, st);
    return fp64 ? gather_t<2, double, false>(f, out, nx, ny, M, plane0, nplanes, sh, st)
                : gather_t<2, float, false>(f, out, nx, ny, M, plane0, nplanes, sh, st);
}

cudaError_t launch_set(bool fp64, const double *src, void *f, int64_t n, Counters *cnt, cudaStream_t st)
{
    const unsigned grid = (unsigned)((n + kBlock - 1) / kBlock);
    if (fp64) k_set<double><<<grid, kBlock, 0, st>>>(src, (double *)f, n, cnt);
    else k_set<float><<<grid, kBlock, 0, st>>>(src, (float *)f, n, cnt);
    return cudaGetLastError();
}

cudaError_t adjoint_scalar(int, bool, bool, const AdjointLaunch &);
cudaError_t adjoint_sw(int, bool, bool, const AdjointLaunch &);
cudaError_t adjoint_init_scalar(int, bool, const double *, const void *, double *, int64_t, const Params &,
                                cudaStream_t);
cudaError_t adjoint_init_sw(int, bool, const double *, const void *, double *, int64_t, const Params &, cudaStream_t);

cudaError_t launch_adjoint_stage(int family, bool fp64, bool entropic, const AdjointLaunch &L)
{
    if (family == FAM_SW1 || family == FAM_SW2) return adjoint_sw(family, fp64, entropic, L);
    if (family == FAM_EULER2) return adjoint_family<Euler2, 2>(fp64, false, L);
    return adjoint_scalar(family, fp64, entropic, L);
}

cudaError_t launch_adjoint_init(int family, bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                                const Params &P, cudaStream_t st)
{
    if (family == FAM_SW1 || family == FAM_SW2) return adjoint_init_sw(family, fp64, u0, g, du0, ncell, P, st);
    if (family == FAM_EULER2) return adjoint_init_family<Euler2>(fp64, u0, g, du0, ncell, P, st);
    return adjoint_init_scalar(family, fp64, u0, g, du0, ncell, P, st);
}

cudaError_t launch_adjoint_readout(int dim, bool fp64, const double *lam, void *g, int64_t nx, int64_t ny, int M,
                                   const Shift &sh, cudaStream_t st)
{
    dim3 grid((unsigned)((nx + kBlock - 1) / kBlock), (unsigned)ny);
    if (dim == 1) {
        if (fp64) k_adjoint_readout<1, double><<<grid, kBlock, 0, st>>>(lam, (double *)g, nx, ny, M, sh);
        else k_adjoint_readout<1, float><<<grid, kBlock, 0, st>>>(lam, (float *)g, nx, ny, M, sh);
    } else {
        if (fp64) k_adjoint_readout<2, double><<<grid, kBlock, 0, st>>>(lam, (double *)g, nx, ny, M, sh);
        else k_adjoint_readout<2, float><<<grid, kBlock, 0, st>>>(lam, (float *)g, nx, ny, M, sh);
    }
    return cudaGetLastError();
}

cudaError_t batch_scalar(int, bool, bool, const BatchLaunch &);
cudaError_t batch_sw(int, bool, bool, const BatchLaunch &);
int batch_occ_scalar(int, bool, bool);
int batch_occ_sw(int, bool, bool);

cudaError_t launch_batch_step(int family, bool fp64, bool entropic, const BatchLaunch &L)
{
    if (family == FAM_SW2) return batch_sw(family, fp64, entropic, L);
    if (family == FAM_EULER2) return batch_family<Euler2>(fp64, false, L);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return batch_scalar(family, fp64, entropic, L);
    return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int family, bool fp64, bool entropic)
{
    if (family == FAM_SW2) return batch_occ_sw(family, fp64, entropic);
    if (family == FAM_EULER2) return batch_occ_family<Euler2>(fp64, false);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return batch_occ_scalar(family, fp64, entropic);
    return 0;
}

int totals_blocks() { return kRedBlocks; }

}  // namespace eslbm
