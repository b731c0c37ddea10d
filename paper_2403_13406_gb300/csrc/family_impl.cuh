// family_impl.cuh -- launcher bodies shared by the per-family translation units.
#pragma once

#include "kernels.cuh"
#include "launch.h"

namespace eslbm {

template <class Sys, int DIM, class R, bool ENT, bool DIAG>
cudaError_t stage_one(const StageLaunch &L)
{
    StageArgs<R> a{(const R *)L.fin, (R *)L.fout, L.nx, L.ny, L.ncell, L.sh, L.kind, L.cnt};
    dim3 grid((unsigned)((L.nx + kBlock - 1) / kBlock), (unsigned)L.ny);
    k_stage<Sys, DIM, R, ENT, DIAG><<<grid, kBlock, 0, L.stream>>>(a, L.P);
    return cudaGetLastError();
}

template <class Sys, int DIM, class R>
cudaError_t stage_prec(bool entropic, bool diag, const StageLaunch &L)
{
    if constexpr (Sys::LINEAR || Sys::M == 4) {
        (void)entropic;
        (void)diag;
        return stage_one<Sys, DIM, R, false, false>(L);
    } else {
        if (!entropic) return stage_one<Sys, DIM, R, false, false>(L);
        if (diag) return stage_one<Sys, DIM, R, true, true>(L);
        return stage_one<Sys, DIM, R, true, false>(L);
    }
}

template <class Sys, int DIM>
cudaError_t stage_family(bool fp64, bool entropic, bool diag, const StageLaunch &L)
{
    return fp64 ? stage_prec<Sys, DIM, double>(entropic, diag, L) : stage_prec<Sys, DIM, float>(entropic, diag, L);
}

template <class Sys>
cudaError_t init_family(bool fp64, const double *u0, void *f, int64_t ncell, const Params &P, Counters *cnt,
                        cudaStream_t st)
{
    const unsigned grid = (unsigned)((ncell + kBlock - 1) / kBlock);
    if (fp64) k_init_eq<Sys, double><<<grid, kBlock, 0, st>>>(u0, (double *)f, ncell, P, cnt);
    else k_init_eq<Sys, float><<<grid, kBlock, 0, st>>>(u0, (float *)f, ncell, P, cnt);
    return cudaGetLastError();
}

template <class Sys, int DIM>
cudaError_t totals_family(bool fp64, const void *f, double *partials, double *out, int64_t nx, int64_t ny,
                          const Shift &sh, const Params &P, cudaStream_t st)
{
    if (fp64) k_totals_partial<Sys, DIM, double><<<kRedBlocks, kRedThreads, 0, st>>>((const double *)f, partials, nx, ny, sh, P);
    else k_totals_partial<Sys, DIM, float><<<kRedBlocks, kRedThreads, 0, st>>>((const float *)f, partials, nx, ny, sh, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_totals_final<2 + Sys::M><<<1, kRedThreads, 0, st>>>(partials, out, kRedBlocks);
    return cudaGetLastError();
}

}  // namespace eslbm
