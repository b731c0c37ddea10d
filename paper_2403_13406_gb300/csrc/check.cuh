// check.cuh -- diagnostics: the per-cell entropy check of Section 4 on the
// relaxations an entropic kernel recorded (Params::rec).
#pragma once

#include "kernels.cuh"

namespace eslbm {

// Change of the cell's microscopic entropy under R_omega relative to the entropy
// the relaxation can dissipate: F(omega - 1) / B(-1) with F(t) = B(t) - B(-1),
// B(t) = sum_k B_k(t delta_k) (eq. variableOmegaProblem), in double precision from
// the recorded moments and deviations, with the kernel's own constants.  -1 for
// omega = 1 (the projection), 0 at equilibrium, +inf for a non-trivial omega
// outside the convexity domain.
template <class Sys>
__device__ float entropy_excess(const ParamsR<double> &Pd, const double *u, const double *delta, double w)
{
    if (w == 1.0) return -1.0f;
    typename Sys::template Ctx<double> cx;
    Sys::template prepare<double>(Pd, u, delta, cx);
    double B0, d0, B1, d1;
    if (!Sys::template eval<double>(Pd, cx, -1.0, B0, d0)) return INFINITY;
    if (!(B0 > 0.0)) return 0.0f;
    if (!Sys::template eval<double>(Pd, cx, w - 1.0, B1, d1)) return INFINITY;
    const double r = (B1 - B0) / B0;
    return r == r ? float(r) : INFINITY;
}

// Records of one launch: n = rec_stages * rec_cells relaxations.  A cell counts
// as an entropy increase when F(omega - 1) > tol B(-1), tol = 64 unit roundoffs
// of the arithmetic that chose omega; the largest F / B(-1) and the range of
// omega go to the counters too (one atomic per warp).
template <class Sys, class R>
__global__ void __launch_bounds__(kBlock) k_check(ParamsR<R> P, float tol, Counters *cnt)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    const int64_t n = (int64_t)P.rec_stages * P.rec_cells;
    const ParamsR<double> Pd = promote(P);
    float wmin = INFINITY, wmax = 0.0f, emax = 0.0f;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;  // the whole warp runs every iteration
        bool inc = false;
        if (i < n) {
            const double w = double(P.rec[(M + Q * M) * n + i]);
            double u[M], delta[Q * M];
#pragma unroll
            for (int m = 0; m < M; ++m) u[m] = double(P.rec[m * n + i]);
#pragma unroll
            for (int k = 0; k < Q * M; ++k) delta[k] = double(P.rec[(M + k) * n + i]);
            const float ex = entropy_excess<Sys>(Pd, u, delta, w);
            inc = ex > tol;
            wmin = fminf(wmin, float(w));
            wmax = fmaxf(wmax, float(w));
            emax = fmaxf(emax, ex);
        }
        warp_count(inc, &cnt->entropy_increases);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wmin = fminf(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
        wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&cnt->omega_min_bits, __float_as_uint(wmin));
        atomicMax(&cnt->omega_max_bits, __float_as_uint(wmax));
        if (emax > 0.0f) atomicMax(&cnt->excess_max_bits, __float_as_uint(emax));
    }
}

}  // namespace eslbm
