// family_impl.cuh -- launcher bodies shared by the per-family translation units.
#pragma once

#include <algorithm>
#include <atomic>

#include "kernels.cuh"
#include "launch.h"
#include "check.cuh"
#include "step2d.cuh"

namespace eslbm {

// Launch settings that belong to a device (function attributes, occupancy, SM
// count) are cached per device: a process may drive several GPUs.
constexpr int kMaxDevices = 64;

inline int device_slot()
{
    int d = 0;
    cudaGetDevice(&d);
    return d < 0 ? 0 : d % kMaxDevices;
}

template <class Sys, int DIM, class R, int OM>
cudaError_t stage_one(const StageLaunch &L)
{
    constexpr int V4 = 16 / (int)sizeof(R);
    if constexpr (DIM == 2) {
        // rows start on 16-byte boundaries: stage the pulled rows with bulk copies
        if (L.nx % V4 == 0 && ((uintptr_t)L.fin & 15u) == 0) {
            constexpr int NP = Sys::Q * Sys::M;
            BulkArgs<R> b{(const R *)L.fin, (R *)L.fout, L.nx, L.ny, L.ncell, L.sh, L.kind, kRowTile + 2 * V4, L.cnt};
            const size_t smem = 128 + (size_t)NP * (size_t)b.slot * sizeof(R);
            static std::atomic<int> attr[kMaxDevices];
            const int d = device_slot();
            if (!attr[d].load()) {
                cudaFuncSetAttribute(k_stage_bulk<Sys, R, OM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(128 + 16 * (kRowTile + 4) * sizeof(double)));
                attr[d].store(1);
            }
            dim3 grid((unsigned)((L.nx + kRowTile - 1) / kRowTile), (unsigned)L.ny);
            k_stage_bulk<Sys, R, OM><<<grid, kRowThreads, smem, L.stream>>>(b, params_as<R>(L.P));
            return cudaGetLastError();
        }
    }
    StageArgs<R> a{(const R *)L.fin, (R *)L.fout, L.nx, L.ny, L.ncell, L.sh, L.kind, L.cnt};
    dim3 grid((unsigned)((L.nx + kBlock - 1) / kBlock), (unsigned)L.ny);
    k_stage<Sys, DIM, R, OM><<<grid, kBlock, 0, L.stream>>>(a, params_as<R>(L.P));
    return cudaGetLastError();
}

// Calls f.template operator()<OM>() for the kernel variant a (system, precision,
// omega mode) combination uses: fixed omega, and the linear and Euler systems,
// have a single variant (nothing to root-find or check); the mixed mode exists
// for FP32 storage only (FP64 storage already evaluates in FP64).  Diagnostics
// are a runtime flag of the same kernels (Params::diag).
template <class Sys, class R, class F> cudaError_t with_variant(int om, F &&f)
{
    if constexpr (Sys::LINEAR || Sys::M == 4) {
        (void)om;
        return f.template operator()<OM_FIXED>();
    } else {
        if (om == OM_FIXED) return f.template operator()<OM_FIXED>();
        if constexpr (sizeof(R) == 4)
            if (om == OM_MIXED) return f.template operator()<OM_MIXED>();
        return f.template operator()<OM_ENTROPIC>();
    }
}

template <class Sys, int DIM, class R>
cudaError_t stage_prec(int om, const StageLaunch &L)
{
    return with_variant<Sys, R>(om, [&]<int OM>() { return stage_one<Sys, DIM, R, OM>(L); });
}

template <class Sys, int DIM>
cudaError_t stage_family(bool fp64, int om, const StageLaunch &L)
{
    return fp64 ? stage_prec<Sys, DIM, double>(om, L) : stage_prec<Sys, DIM, float>(om, L);
}

// Tile of the temporally blocked 1D kernel: enough tiles to give every SM
// `bps` resident blocks in a single wave, with the window of a block taking
// at most its share of the SM's shared memory.
constexpr int kSmemPerSm = 220 * 1024;

inline int fused_tile(int64_t n, int halo, int bytes_per_cell, int bps)
{
    static std::atomic<int> sm_count[kMaxDevices];
    const int d = device_slot();
    int sms = sm_count[d].load();
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        sm_count[d].store(sms);
    }
    int64_t t = (n + (int64_t)bps * sms - 1) / ((int64_t)bps * sms);
    t = ((t + 31) / 32) * 32;
    if (t < 128) t = 128;
    const int64_t tmax = (kSmemPerSm / bps) / bytes_per_cell - 2 * halo;
    if (t > tmax) t = tmax;
    return (int)t;
}

template <class Sys, class R, int OM, bool REC>
cudaError_t fused_one_rec(const FusedLaunch &L)
{
    constexpr int NP = Sys::Q * Sys::M;
    if (!stage_list_ok(L.sl)) return cudaErrorInvalidValue;
    static std::atomic<int> bps_cache[kMaxDevices];  // resident blocks per SM allowed by the registers (<= 4)
    const int d = device_slot();
    int bps = bps_cache[d].load();
    if (!bps) {
        cudaFuncSetAttribute(k_step1d<Sys, R, OM, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemPerSm);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step1d<Sys, R, OM, REC>, kFusedBlock, 0) !=
            cudaSuccess)
            occ = 1;
        bps = occ < 1 ? 1 : (occ > 4 ? 4 : occ);
        bps_cache[d].store(bps);
    }
    const int tile = fused_tile(L.n, L.sl.halo, NP * (int)sizeof(R), bps);
    if (tile < 32) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(tile + 2 * L.sl.halo) * NP * sizeof(R);
    FusedArgs<R> a{(const R *)L.fin, (R *)L.fout, L.n, tile, L.cnt,
                   (R *)L.rec, L.rec_stride_bytes / (int64_t)sizeof(R), L.nrec};
    const unsigned grid = (unsigned)((L.n + tile - 1) / tile);
    k_step1d<Sys, R, OM, REC><<<grid, kFusedBlock, smem, L.stream>>>(a, L.sl, params_as<R>(L.P));
    return cudaGetLastError();
}

template <class Sys, class R>
cudaError_t fused_prec(int om, const FusedLaunch &L)
{
    if (L.rec) return with_variant<Sys, R>(om, [&]<int OM>() { return fused_one_rec<Sys, R, OM, true>(L); });
    return with_variant<Sys, R>(om, [&]<int OM>() { return fused_one_rec<Sys, R, OM, false>(L); });
}

template <class Sys>
cudaError_t fused_family(bool fp64, int om, const FusedLaunch &L)
{
    return fp64 ? fused_prec<Sys, double>(om, L) : fused_prec<Sys, float>(om, L);
}

template <class Sys, int DIM, class R>
cudaError_t adjoint_prec(int om, const AdjointLaunch &L)
{
    dim3 grid((unsigned)((L.nx + kBlock - 1) / kBlock), (unsigned)L.ny);
    const ParamsR<R> P = params_as<R>(L.P);
    return with_variant<Sys, R>(om, [&]<int OM>() {
        k_adjoint_stage<Sys, DIM, R, OM><<<grid, kBlock, 0, L.stream>>>((const R *)L.fin, (const R *)L.gout,
                                                                        (R *)L.gin, L.nx, L.ny, L.sh, L.kind, P);
        return cudaGetLastError();
    });
}

template <class Sys, int DIM>
cudaError_t adjoint_family(bool fp64, int om, const AdjointLaunch &L)
{
    return fp64 ? adjoint_prec<Sys, DIM, double>(om, L) : adjoint_prec<Sys, DIM, float>(om, L);
}

template <class Sys>
cudaError_t adjoint_init_family(bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                                const Params &P, cudaStream_t st)
{
    const unsigned grid = (unsigned)((ncell + kBlock - 1) / kBlock);
    if (fp64) k_adjoint_init<Sys, double><<<grid, kBlock, 0, st>>>(u0, (const double *)g, du0, ncell, params_as<double>(P));
    else k_adjoint_init<Sys, float><<<grid, kBlock, 0, st>>>(u0, (const float *)g, du0, ncell, params_as<float>(P));
    return cudaGetLastError();
}

template <class Sys, class R, int OM>
cudaError_t batch_one(const BatchLaunch &L)
{
    BatchArgs<R> a{{(R *)L.pool[0], (R *)L.pool[1]}, L.inst, L.items, L.n_items, L.side, L.cnt, (R *)L.rec,
                   L.pool_elems};
    StageList sl = L.sl;
    ParamsR<R> P = params_as<R>(L.P);
    void *args[] = {&a, &sl, &P};
    return cudaLaunchCooperativeKernel((const void *)k_batch_step<Sys, R, OM>, dim3((unsigned)L.grid), dim3(kBlock),
                                       args, 0, L.stream);
}

template <class Sys, class R>
cudaError_t batch_prec(int om, const BatchLaunch &L)
{
    return with_variant<Sys, R>(om, [&]<int OM>() { return batch_one<Sys, R, OM>(L); });
}

template <class Sys>
cudaError_t batch_family(bool fp64, int om, const BatchLaunch &L)
{
    return fp64 ? batch_prec<Sys, double>(om, L) : batch_prec<Sys, float>(om, L);
}

template <class Sys, class R>
int batch_occ_prec(int om)
{
    int n = 0;
    cudaError_t e = with_variant<Sys, R>(om, [&]<int OM>() {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<Sys, R, OM>, kBlock, 0);
    });
    return e == cudaSuccess ? n : 0;
}

template <class Sys>
int batch_occ_family(bool fp64, int om)
{
    return fp64 ? batch_occ_prec<Sys, double>(om) : batch_occ_prec<Sys, float>(om);
}

template <class Sys, class R>
cudaError_t batch_adjoint_prec(int om, const BatchAdjointLaunch &L)
{
    BatchAdjointArgs<R> a{(const R *)L.step_in, (const R *)L.rec, L.pool_elems, {(R *)L.cot[0], (R *)L.cot[1]},
                          L.side, L.inst, L.items, L.n_items};
    StageList sl = L.sl;
    ParamsR<R> P = params_as<R>(L.P);
    void *args[] = {&a, &sl, &P};
    return with_variant<Sys, R>(om, [&]<int OM>() {
        return cudaLaunchCooperativeKernel((const void *)k_batch_adjoint_step<Sys, R, OM>, dim3((unsigned)L.grid),
                                           dim3(kBlock), args, 0, L.stream);
    });
}

template <class Sys>
cudaError_t batch_adjoint_family(bool fp64, int om, const BatchAdjointLaunch &L)
{
    return fp64 ? batch_adjoint_prec<Sys, double>(om, L) : batch_adjoint_prec<Sys, float>(om, L);
}

template <class Sys, class R>
int batch_adjoint_occ_prec(int om)
{
    int n = 0;
    cudaError_t e = with_variant<Sys, R>(om, [&]<int OM>() {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_adjoint_step<Sys, R, OM>, kBlock, 0);
    });
    return e == cudaSuccess ? n : 0;
}

template <class Sys>
int batch_adjoint_occ_family(bool fp64, int om)
{
    return fp64 ? batch_adjoint_occ_prec<Sys, double>(om) : batch_adjoint_occ_prec<Sys, float>(om);
}

template <class Sys, class R, int OM>
cudaError_t step2d_one(const Step2dLaunch &L)
{
    if (!stage_list_ok(L.sl) || L.sl.n > kStep2dMaxStages) return cudaErrorInvalidValue;
    const Plan2d &pl = L.plan;
    if (pl.ring > kStep2dMaxRing || pl.smem > (size_t)kStep2dSmemBudget) return cudaErrorInvalidValue;
    // threads: a producer warp, and consumers over which the items of a tick spread evenly (at most
    // the variant's threads in all, at most kStep2dSlots items a consumer)
    constexpr int cmax = Step2dThreads<Sys, R, OM>::value - 32;
    const int nslots = (pl.items + cmax - 1) / cmax;
    if (nslots < 1 || nslots > kStep2dSlots) return cudaErrorInvalidValue;
    const int threads = 32 + ((pl.items + nslots - 1) / nslots + 31) / 32 * 32;
    static std::atomic<int> attr[kMaxDevices];
    const int d = device_slot();
    if (!attr[d].load()) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d<Sys, R, OM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kStep2dSmemBudget);
        if (e != cudaSuccess) return e;
        attr[d].store(1);
    }
    Step2dArgs<R> a{(const R *)L.fin, (R *)L.fout, L.nx, L.ny, L.ncell, pl.tx, pl.ly, pl.hl, pl.wx, pl.ring,
                    pl.prefetch, pl.nstrips, L.cnt};
    const unsigned grid = (unsigned)((int64_t)pl.nstrips * pl.nsegs);
    k_step2d<Sys, R, OM><<<grid, threads, pl.smem, L.stream>>>(a, L.sl, params_as<R>(L.P));
    return cudaGetLastError();
}

template <class Sys>
cudaError_t step2d_family(bool fp64, int om, const Step2dLaunch &L)
{
    if (fp64) return with_variant<Sys, double>(om, [&]<int OM>() { return step2d_one<Sys, double, OM>(L); });
    return with_variant<Sys, float>(om, [&]<int OM>() { return step2d_one<Sys, float, OM>(L); });
}

// the per-cell check of the relaxations recorded by the previous launch (diagnostics)
template <class Sys>
cudaError_t check_family(bool fp64, int om, const Params &P, Counters *cnt, cudaStream_t st)
{
    if constexpr (Sys::LINEAR || Sys::M == 4) {
        return cudaSuccess;  // nothing is recorded
    } else {
        if (!P.rec || om == OM_FIXED) return cudaSuccess;
        const int64_t n = (int64_t)P.rec_stages * P.rec_cells;
        const unsigned grid = (unsigned)std::min<int64_t>(4096, (n + kBlock - 1) / kBlock);
        const float tol = (!fp64 && om != OM_MIXED) ? 64.0f * 1.1920929e-7f : 64.0f * 2.220446e-16f;
        if (fp64) k_check<Sys, double><<<grid, kBlock, 0, st>>>(params_as<double>(P), tol, cnt);
        else k_check<Sys, float><<<grid, kBlock, 0, st>>>(params_as<float>(P), tol, cnt);
        return cudaGetLastError();
    }
}

template <class Sys>
cudaError_t init_family(bool fp64, const double *u0, void *f, int64_t ncell, const Params &P, Counters *cnt,
                        cudaStream_t st)
{
    const unsigned grid = (unsigned)((ncell + kBlock - 1) / kBlock);
    const ParamsR<double> Pd = params_as<double>(P);
    if (fp64) k_init_eq<Sys, double><<<grid, kBlock, 0, st>>>(u0, (double *)f, ncell, Pd, cnt);
    else k_init_eq<Sys, float><<<grid, kBlock, 0, st>>>(u0, (float *)f, ncell, Pd, cnt);
    return cudaGetLastError();
}

template <class Sys, int DIM>
cudaError_t totals_family(bool fp64, const void *f, double *partials, double *out, int64_t nx, int64_t ny,
                          const Shift &sh, const Params &P, cudaStream_t st)
{
    const ParamsR<double> Pd = params_as<double>(P);
    if (fp64) k_totals_partial<Sys, DIM, double><<<kRedBlocks, kRedThreads, 0, st>>>((const double *)f, partials, nx, ny, sh, Pd);
    else k_totals_partial<Sys, DIM, float><<<kRedBlocks, kRedThreads, 0, st>>>((const float *)f, partials, nx, ny, sh, Pd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_totals_final<2 + Sys::M><<<1, kRedThreads, 0, st>>>(partials, out, kRedBlocks);
    return cudaGetLastError();
}

}  // namespace eslbm
