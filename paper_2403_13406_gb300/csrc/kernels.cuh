// kernels.cuh -- CUDA kernels of the composite step, templated on the system
// (physics), the dimension and the storage precision.
//
// Data layout: structure of arrays, plane (k*M + m) of ncell = nx*ny cells,
// x fastest.  One thread owns one cell of the output; within a warp the cells
// are consecutive in x, so every plane access of a warp is one contiguous run
// of 32 elements (coalesced), also for the shifted pulls.
#pragma once

#include <cooperative_groups.h>

#include "systems.cuh"

namespace cg = cooperative_groups;

namespace eslbm {

constexpr int kBlock = 256;       // threads per block of the per-cell kernels
constexpr int kFusedBlock = 256;  // threads per block of the temporally blocked 1D kernel
constexpr int kRedBlocks = 1024;  // fixed grid of the totals reduction (deterministic order)
constexpr int kRedThreads = 256;

template <class R> struct StageArgs {
    const R *__restrict__ fin;
    R *__restrict__ fout;
    int64_t nx, ny, ncell;
    Shift sh;
    int kind;
    Counters *cnt;
};

__device__ __forceinline__ int64_t wrap_add(int64_t x, int64_t r, int64_t n)
{
    const int64_t s = x + r;
    return s >= n ? s - n : s;
}

// source cell of population k for output cell (x, y)
template <int DIM>
__device__ __forceinline__ int64_t src_cell(int k, int64_t x, int64_t y, int64_t nx, int64_t ny, const Shift &sh)
{
    if (Lattice<DIM>::axis(k) == 0) return y * nx + wrap_add(x, sh.roff[k], nx);
    return wrap_add(y, sh.roff[k], ny) * nx + x;
}

__device__ __forceinline__ void warp_count(bool flag, unsigned long long *counter)
{
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask && (threadIdx.x & 31) == 0) atomicAdd(counter, (unsigned long long)__popc(mask));
}

// Conserved moments u of the distributions held in f (f itself, or f - fbar in
// the shifted storage) and the relaxation target tgt_k = f^eq_k(u) minus what
// the storage subtracts, so that f^eq - f = tgt - (stored values) in both forms.
template <class Sys, class R>
__device__ __forceinline__ void moments_target(const ParamsR<R> &P, const R *f, R *u, R *tgt)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    R s[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        R a = f[m];
#pragma unroll
        for (int k = 1; k < Q; ++k) a += f[k * M + m];
        s[m] = a;
    }
    if (!P.shifted) {
#pragma unroll
        for (int m = 0; m < M; ++m) u[m] = s[m];
        Sys::template equilibrium<R>(P, u, tgt);
        return;
    }
    R du[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        du[m] = s[m] + P.cm[m];
        u[m] = P.ubar[m] + du[m];
    }
    Sys::template equilibrium_dev<R>(P, du, u, tgt);
#pragma unroll
    for (int i = 0; i < Q * M; ++i) tgt[i] += P.rdev[i];
}

// The deviations delta_k = f^eq_k - f_k of a cell, with the last population of each component
// taking minus the sum of the others: sum_k delta_k = 0 up to the rounding of that short sum of
// deviations (relative to |delta|), so that the relaxation f + omega delta moves the conserved
// moments only by the rounding of its own results.  With every delta_k from its equilibrium the
// moment sum u and the equilibria carried their roundings (relative to |f|) into sum_k delta_k,
// and where opposite equilibria straddle a binade edge those roundings are biased: a steady
// drift of the conserved totals (FP32 2D Burgers: 1.4e-4 of the mass over 2000 steps).  In exact
// arithmetic the two forms agree (sum_k f^eq_k = u = sum_k f_k).
// D1Q2 (Q = 2) keeps every delta_k from its own equilibrium: on the 1D shallow-water workload (FP32
// shifted storage, entropic omega, t = 0.05) the error against FP64 was 3.5e-6 that way and 1.7e-5
// with the conservative form (whose rounding then lands in the state rather than in the totals),
// while the 1D totals stay within the FP32 rounding of the state either way.
template <int Q, int M, class R> __host__ __device__ __forceinline__ void deviations(const R *feq, const R *f, R *delta)
{
    if constexpr (Q == 2) {
#pragma unroll
        for (int i = 0; i < Q * M; ++i) delta[i] = feq[i] - f[i];
        return;
    }
#pragma unroll
    for (int i = 0; i < (Q - 1) * M; ++i) delta[i] = feq[i] - f[i];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        R s = delta[m];
#pragma unroll
        for (int k = 1; k < Q - 1; ++k) s += delta[k * M + m];
        delta[(Q - 1) * M + m] = -s;
    }
}

// The kernel's constants in double precision, exactly as the kernel rounded them
// (a float kernel's g, 1 / (2V), ... promoted), for the FP64 evaluations of the
// mixed mode and of the diagnostics.
template <class R> __device__ __forceinline__ ParamsR<double> promote(const ParamsR<R> &p)
{
    ParamsR<double> q;
    q.V = p.V;
    q.inv2V = p.inv2V;
    q.a[0] = p.a[0];
    q.a[1] = p.a[1];
    q.c[0] = p.c[0];
    q.c[1] = p.c[1];
    q.g = p.g;
    q.gamma_m1 = p.gamma_m1;
    q.omega = p.omega;
    q.t_max = p.t_max;
    q.gV4 = p.gV4;
    q.inv16gV = p.inv16gV;
    q.shifted = p.shifted;
    q.rec = nullptr;
    q.rec_cells = 0;
    q.rec_stages = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        q.ubar[i] = p.ubar[i];
        q.cm[i] = p.cm[i];
        q.aux[i] = p.aux[i];
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        q.rdev[i] = p.rdev[i];
        q.fbar[i] = p.fbar[i];
    }
    return q;
}

// Entropic omega with the entropy difference in FP64 (FP32 storage).  The FP32
// root-find's t = omega - 1 is certified by evaluating, in double precision from
// the same moments and deviations (and the kernel's own constants),
// E0 = B(-1) = sum_k B_k(-delta_k) and the residual F(t) = B(t) - E0 at the
// returned root.  F(t) <= 0 keeps omega.  F(t) > 0 (the FP32 root fell above the
// root by its rounding) replaces t by the chord root through (0, -E0) and
// (t, F(t)), t E0 / B(t): on a convex F that chord lies above F, so its root never
// exceeds the root and the cell's microscopic entropy does not increase to FP64
// rounding (Section 4).  The result is rounded towards zero to FP32 (t, then
// omega = 1 + t), which keeps that side.  A cell that FP64 finds outside the
// convexity domain falls back to omega = 1 (counted).
template <class Sys, class R>
__device__ R mixed_omega(const ParamsR<R> &P, const R *u, const R *delta, R w, bool &fallback)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    if constexpr (sizeof(R) == 8) {
        return w;
    } else {
        if (fallback || w == R(1)) return w;
        const ParamsR<double> Pd = promote(P);
        double ud[M], dd[Q * M];
#pragma unroll
        for (int m = 0; m < M; ++m) ud[m] = double(u[m]);
#pragma unroll
        for (int i = 0; i < Q * M; ++i) dd[i] = double(delta[i]);
        typename Sys::template Ctx<double> cx;
        Sys::template prepare<double>(Pd, ud, dd, cx);
        double E0, dE0, Bt, dBt;
        if (!Sys::template eval<double>(Pd, cx, -1.0, E0, dE0)) {
            fallback = true;
            return R(1);
        }
        if (!(E0 > 0.0)) return w;  // at equilibrium: every omega leaves the cell unchanged
        const double t = double(w) - 1.0;
        if (!Sys::template eval<double>(Pd, cx, t, Bt, dBt)) {
            fallback = true;
            return R(1);
        }
        if (Bt - E0 <= 0.0) return w;
        const float tc = __double2float_rz(t * E0 / Bt);
        return __fadd_rz(1.0f, tc);
    }
}

// One relaxation of one cell (eq. relaxationDiscretizationOmega), in place.
// rec: this relaxation's record (diagnostics, see Params::rec) or null; the
// record only stores values the relaxation computes anyway.
template <class Sys, class R, int OM>
__device__ __forceinline__ void relax_cell(const ParamsR<R> &P, R *f, int kind, bool &fallback, R *rec)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    const int64_t fs = (int64_t)P.rec_stages * P.rec_cells;  // distance between the fields of a record
    R u[M], feq[Q * M];
    moments_target<Sys, R>(P, f, u, feq);
    fallback = false;
    R delta[Q * M];
    deviations<Q, M, R>(feq, f, delta);
    if (kind == KIND_PROJECT) {  // R_1: projection on the equilibrium (Section 6.1), f + delta
        if (rec) rec[(M + Q * M) * fs] = R(1);
#pragma unroll
        for (int i = 0; i < Q * M; ++i) f[i] += delta[i];
        return;
    }
    if (rec) {
#pragma unroll
        for (int m = 0; m < M; ++m) rec[m * fs] = u[m];
#pragma unroll
        for (int i = 0; i < Q * M; ++i) rec[(M + i) * fs] = delta[i];
    }
    R w = P.omega;
    if constexpr (OM != OM_FIXED && !Sys::LINEAR) {
        typename Sys::template Ctx<R> cx;
        Sys::template prepare<R>(P, u, delta, cx);
        w = entropic_omega<Sys, R>(P, cx, fallback);
        if constexpr (OM == OM_MIXED) w = mixed_omega<Sys, R>(P, u, delta, w, fallback);
    } else if constexpr (OM != OM_FIXED) {
        w = R(2);  // quadratic kinetic entropies: omega* = 2 exactly (Proposition 2)
    }
    if (rec) rec[(M + Q * M) * fs] = w;
#pragma unroll
    for (int i = 0; i < Q * M; ++i) f[i] += w * delta[i];
}

// Kernels that record their relaxations for the diagnostics (entropic omega,
// nonlinear system): the record of stage st of a launch at cell c, or null.
template <class Sys, int OM> constexpr bool checked() { return OM != OM_FIXED && !Sys::LINEAR; }

template <class Sys, class R, int OM>
__device__ __forceinline__ R *record_of(const ParamsR<R> &P, int st, int64_t cell, bool on)
{
    if constexpr (checked<Sys, OM>())
        return (P.rec && on) ? P.rec + (int64_t)st * P.rec_cells + cell : nullptr;
    return nullptr;
}

// Fused stage: pull-shift by sh (transport, eq. transportPhase) then relax.
template <class Sys, int DIM, class R, int OM>
__global__ void __launch_bounds__(kBlock) k_stage(StageArgs<R> a, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    const bool valid = x < a.nx;
    R f[Q * M];
    bool fb = false;
    if (valid) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int64_t s = src_cell<DIM>(k, x, y, a.nx, a.ny, a.sh);
#pragma unroll
            for (int m = 0; m < M; ++m) f[k * M + m] = a.fin[(int64_t)(k * M + m) * a.ncell + s];
        }
        const int64_t o = y * a.nx + x;
        relax_cell<Sys, R, OM>(P, f, a.kind, fb, record_of<Sys, R, OM>(P, 0, o, true));
#pragma unroll
        for (int i = 0; i < Q * M; ++i) a.fout[(int64_t)i * a.ncell + o] = f[i];
    }
    if constexpr (checked<Sys, OM>()) warp_count(valid && fb, &a.cnt->fallbacks);
}

// ---------------------------------------------------------------------------
// 2D fused stage with the pulled rows staged in shared memory by bulk copies
// (cp.async.bulk, completion counted on an mbarrier).  A block of 256 threads
// owns a row segment [x0, x0 + T) of row y, T <= 1024 cells (four per thread:
// with 4-plane states a block then keeps 16 KB of copies in flight, and enough
// blocks fit on an SM to cover the memory latency).  For every plane the source
// of the pull is one contiguous run of a single row: the same columns of row
// y + roff (vertical populations) or columns x0 + roff ... of row y, wrapping
// at the row end (horizontal populations).  Each run is copied from its 16-byte
// boundary (rounded down; the remainder becomes an offset into the plane's
// slot) as one or, when it wraps, two bulk copies; rows start on 16-byte
// boundaries because the launcher requires nx to be a multiple of
// 16 / sizeof(R).  One elected thread issues every copy; the block waits on the
// mbarrier with a bounded number of polls, and on time-out counts the event and
// skips the stage's arithmetic (the host reports it as an error).
// ---------------------------------------------------------------------------
constexpr int kRowTile = 1024;    // cells of a row segment
constexpr int kRowThreads = 256;  // threads of the block

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <class R> struct BulkArgs {
    const R *__restrict__ fin;
    R *__restrict__ fout;
    int64_t nx, ny, ncell;
    Shift sh;
    int kind;
    int slot;  // elements per plane slot in shared memory (kRowTile + 2 * 16 / sizeof(R))
    Counters *cnt;
};

template <class Sys, class R, int OM>
__global__ void __launch_bounds__(kRowThreads) k_stage_bulk(BulkArgs<R> a, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M, NP = Q * M;
    constexpr int V4 = 16 / (int)sizeof(R);  // elements per 16 bytes
    extern __shared__ __align__(128) unsigned char smem_bulk[];
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smem_bulk);
    R *sm = reinterpret_cast<R *>(smem_bulk + 128);
    __shared__ int s_off[NP];  // element offset of the run's first needed value in its slot
    const int64_t y = blockIdx.y;
    const int64_t x0 = (int64_t)blockIdx.x * kRowTile;
    const int T = (int)min((int64_t)kRowTile, a.nx - x0);
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // one bulk copy of n elements into shared memory, announced to the mbarrier first
        auto copy = [&](R *dst, const R *src, int64_t n) {
            const uint32_t nb = (uint32_t)(n * (int64_t)sizeof(R));
            asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(nb) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(dst)),
                "l"(src), "r"(nb), "r"(bar)
                : "memory");
        };
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int64_t r = a.sh.roff[k];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int p = k * M + m;
                const R *plane = a.fin + (int64_t)p * a.ncell;
                R *dst = sm + (int64_t)p * a.slot;
                if (Lattice<2>::axis(k) == 0) {
                    int64_t sx = x0 + r;
                    if (sx >= a.nx) sx -= a.nx;
                    const int64_t al = sx - (sx % V4);
                    const int off = (int)(sx - al);
                    const int64_t L = (off + T + V4 - 1) / V4 * V4;  // whole 16-byte units
                    const int64_t first = min(L, a.nx - al);
                    s_off[p] = off;
                    copy(dst, plane + y * a.nx + al, first);
                    if (first < L) copy(dst + first, plane + y * a.nx, L - first);  // wrap to the row start
                } else {
                    int64_t sy = y + r;
                    if (sy >= a.ny) sy -= a.ny;
                    s_off[p] = 0;
                    copy(dst, plane + sy * a.nx + x0, (T + V4 - 1) / V4 * V4);
                }
            }
        }
        unsigned long long state;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(bar) : "memory");
        (void)state;
    }
    __syncthreads();  // s_off visible
    // bounded wait for phase 0 of the mbarrier
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    }
    if (__syncthreads_or(!done)) {  // the whole block gives up together
        if (threadIdx.x == 0) atomicAdd(&a.cnt->copy_timeouts, 1ull);
        return;
    }
    for (int j0 = 0; j0 < kRowTile; j0 += kRowThreads) {  // same trip count for every thread
        const int j = j0 + threadIdx.x;
        const bool valid = j < T;
        bool fb = false;
        if (valid) {
            R f[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) f[p] = sm[(int64_t)p * a.slot + s_off[p] + j];
            const int64_t o = y * a.nx + x0 + j;
            relax_cell<Sys, R, OM>(P, f, a.kind, fb, record_of<Sys, R, OM>(P, 0, o, true));
#pragma unroll
            for (int p = 0; p < NP; ++p) a.fout[(int64_t)p * a.ncell + o] = f[p];
        }
        if constexpr (checked<Sys, OM>()) warp_count(fb, &a.cnt->fallbacks);
    }
}

// ---------------------------------------------------------------------------
// Temporally blocked 1D composite step.  One block owns an output tile of T
// cells and loads a window of W = T + 2H cells of every plane into shared
// memory, H = sum |s_i| over the fused stages.  In shared memory the transport
// is index arithmetic: population k of window cell j lives at circular slot
// (j - o_k) mod W, and a stage adds sign_k s_i to o_k before relaxing every
// cell in place (one thread per cell, so the in-place update is race free).
// Values wrapping around the window edges are wrong, but after the stages
// they have moved at most H cells inward, so the tile [H, H + T) is exact.
// Global traffic per fused step: one read (plus the 2H halo) and one write of
// the state instead of one per stage.
// ---------------------------------------------------------------------------

template <class R> struct FusedArgs {
    const R *__restrict__ fin;
    R *__restrict__ fout;
    int64_t n;       // cells
    int tile;        // T
    Counters *cnt;
    // recording (reverse mode): the output of stage i < nrec is also written, in the physical
    // layout, to rec + i * rec_stride
    R *rec;
    int64_t rec_stride;
    int nrec;
};

// Four resident blocks per SM (64 registers a thread) for the FP32 relaxation; two (128) where
// an FP64 evaluation joins it (FP64 storage, the mixed mode).
template <class R, int OM> constexpr int step1d_min_blocks() { return (sizeof(R) == 4 && OM != OM_MIXED) ? 4 : 2; }

template <class Sys, class R, int OM, bool RECORD = false>
__global__ void __launch_bounds__(kFusedBlock, step1d_min_blocks<R, OM>())
    k_step1d(FusedArgs<R> a, StageList sl, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M, NP = Q * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);
    const int64_t x0 = (int64_t)blockIdx.x * a.tile;
    const int T = (int)min((int64_t)a.tile, a.n - x0);
    const int H = sl.halo;
    const int W = T + 2 * H;
    // load the window (periodic)
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        int64_t gx = (x0 - H + j) % a.n;
        if (gx < 0) gx += a.n;
#pragma unroll
        for (int p = 0; p < NP; ++p) sm[p * W + j] = a.fin[(int64_t)p * a.n + gx];
    }
    __syncthreads();
    int off[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) off[k] = 0;
    int moved = 0;  // sum of |shift| over the stages so far
    for (int st = 0; st < sl.n; ++st) {
        const int s = sl.shift[st], kind = sl.kind[st];
#pragma unroll
        for (int k = 0; k < Q; ++k) off[k] += Lattice<1>::sign(k) * s;
        moved += s < 0 ? -s : s;
        // only window cells within the later stages' total shift (H - moved) of the tile can still
        // reach it: [moved, W - moved).  Their pulls read [moved - |s|, W - moved + |s|), the range
        // the previous stage computed.
        const int jlo = moved, cnt = W - 2 * moved;
        const int jend = ((cnt + 31) / 32) * 32;  // whole warps for the warp-level counters
        for (int jj = threadIdx.x; jj < jend; jj += blockDim.x) {
            const int j = jlo + jj;
            const bool valid = jj < cnt;
            bool fb = false;
            if (valid) {
                int slot[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    int i = j - off[k];
                    i = i < 0 ? i + W : (i >= W ? i - W : i);
                    slot[k] = i;
                }
                R f[NP];
#pragma unroll
                for (int k = 0; k < Q; ++k)
#pragma unroll
                    for (int m = 0; m < M; ++m) f[k * M + m] = sm[(k * M + m) * W + slot[k]];
                // only cells of the final tile count and record (each cell-stage once)
                const bool in_tile = j >= H && j < H + T;
                relax_cell<Sys, R, OM>(P, f, kind, fb, record_of<Sys, R, OM>(P, st, x0 + j - H, in_tile));
                fb = fb && in_tile;
#pragma unroll
                for (int k = 0; k < Q; ++k)
#pragma unroll
                    for (int m = 0; m < M; ++m) sm[(k * M + m) * W + slot[k]] = f[k * M + m];
            }
            if constexpr (checked<Sys, OM>()) warp_count(fb, &a.cnt->fallbacks);
        }
        __syncthreads();
        if constexpr (RECORD) {
            if (st < a.nrec) {  // the tile is exact after every stage
                R *dst = a.rec + (int64_t)st * a.rec_stride;
                for (int j = threadIdx.x; j < T; j += blockDim.x) {
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        int i = j + H - off[k];
                        i = i < 0 ? i + W : (i >= W ? i - W : i);
#pragma unroll
                        for (int m = 0; m < M; ++m) dst[(int64_t)(k * M + m) * a.n + x0 + j] = sm[(k * M + m) * W + i];
                    }
                }
                __syncthreads();  // the next stage rewrites the window in place
            }
        }
    }
    // write the exact tile
    for (int j = threadIdx.x; j < T; j += blockDim.x) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            int i = j + H - off[k];
            i = i < 0 ? i + W : (i >= W ? i - W : i);
#pragma unroll
            for (int m = 0; m < M; ++m) a.fout[(int64_t)(k * M + m) * a.n + x0 + j] = sm[(k * M + m) * W + i];
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint of one relaxation.  For f' = f + omega(f) delta, delta = f^eq(u) - f,
// u = sum_k f_k, E_k = d f^eq_k / d u:
//   J^T g'  at population j  =  (1 - omega) g'_j + omega sum_k E_k^T g'_k
//                                + grad_{f_j} omega (delta . g').
// For the entropic omega = 1 + t*, F(t*, f) = 0 with F(t, f) = B(t) - B(-1),
// B(t) = sum_k B_k(t delta_k; u), gives by the implicit function theorem
// grad_f t* = -grad_f F / F'(t*), where (Sigma_k delta_k = 0 removes the
// dependence through the dual p) grad_{f_j} F = t Delta_j(t) + Delta_j(-1)
//   - (1 + t) sum_k E_k^T Delta_k(t) and F'(t) = -sum_k Delta_k(t) . delta_k,
// Delta_k(t) = p - p'_k the dual deviation at h = t delta_k.  Cells at
// equilibrium, fallback cells (omega = 1) and quadratic entropies have a
// locally constant omega and no such term.
// ---------------------------------------------------------------------------
template <class Sys, class R, int OM>
__device__ __forceinline__ void relax_adjoint(const ParamsR<R> &P, const R *f, const R *gout, int kind, R *gin)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    R u[M], feq[Q * M];
    moments_target<Sys, R>(P, f, u, feq);
    R E[Q * M * M];
    Sys::template equilibrium_jacobian<R>(P, u, E);
    R a[M];  // sum_k E_k^T g'_k
#pragma unroll
    for (int n = 0; n < M; ++n) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < Q; ++k)
#pragma unroll
            for (int m = 0; m < M; ++m) s += E[(k * M + m) * M + n] * gout[k * M + m];
        a[n] = s;
    }
    if (kind == KIND_PROJECT) {
#pragma unroll
        for (int k = 0; k < Q; ++k)
#pragma unroll
            for (int n = 0; n < M; ++n) gin[k * M + n] = a[n];
        return;
    }
    R delta[Q * M];
    deviations<Q, M, R>(feq, f, delta);
    R w = P.omega;
    bool varying = false;
    typename Sys::template Ctx<R> cx;
    R Dm[Q * M];  // dual deviations at t = -1, from the root-find's own evaluation there
    if constexpr (OM != OM_FIXED && !Sys::LINEAR) {
        Sys::template prepare<R>(P, u, delta, cx);
        bool fb = false;
        R E0 = R(0);
        w = entropic_omega<Sys, R>(P, cx, fb, Dm, &E0);
        if constexpr (OM == OM_MIXED) w = mixed_omega<Sys, R>(P, u, delta, w, fb);
        varying = !fb && E0 > R(0);
    } else if constexpr (OM != OM_FIXED) {
        w = R(2);
    }
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int n = 0; n < M; ++n) gin[k * M + n] = (R(1) - w) * gout[k * M + n] + w * a[n];
    if constexpr (OM != OM_FIXED && !Sys::LINEAR) {
        if (varying) {
            const R t = w - R(1);
            R Dt[Q * M], B, dB;
            const bool ok = Sys::template eval<R>(P, cx, t, B, dB, Dt);
            R dg = R(0);
#pragma unroll
            for (int i = 0; i < Q * M; ++i) dg += delta[i] * gout[i];
            if (ok && dB > R(0) && dg != R(0)) {
                R c[M];  // sum_k E_k^T Delta_k(t)
#pragma unroll
                for (int n = 0; n < M; ++n) {
                    R s = R(0);
#pragma unroll
                    for (int k = 0; k < Q; ++k)
#pragma unroll
                        for (int m = 0; m < M; ++m) s += E[(k * M + m) * M + n] * Dt[k * M + m];
                    c[n] = s;
                }
                const R scale = -dg / dB;  // (delta . g') * (-1 / F'(t))
#pragma unroll
                for (int k = 0; k < Q; ++k)
#pragma unroll
                    for (int n = 0; n < M; ++n)
                        gin[k * M + n] += scale * (t * Dt[k * M + n] + Dm[k * M + n] - (R(1) + t) * c[n]);
            }
        }
    }
}

// Adjoint of a fused stage f_out(x) = R(f_in(src_k(x))): the cotangent of the
// stage input at src_k(x) is (J_R(x)^T g_out(x))_k (the reverse shift; src_k is
// a bijection, so every input cell receives exactly one contribution).
template <class Sys, int DIM, class R, int OM>
__global__ void __launch_bounds__(kBlock) k_adjoint_stage(const R *__restrict__ fin, const R *__restrict__ gout,
                                                          R *__restrict__ gin, int64_t nx, int64_t ny, Shift sh,
                                                          int kind, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    if (x >= nx) return;
    const int64_t ncell = nx * ny, o = y * nx + x;
    int64_t src[Q];
    R f[Q * M], go[Q * M], gi[Q * M];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        src[k] = src_cell<DIM>(k, x, y, nx, ny, sh);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            f[k * M + m] = fin[(int64_t)(k * M + m) * ncell + src[k]];
            go[k * M + m] = gout[(int64_t)(k * M + m) * ncell + o];
        }
    }
    relax_adjoint<Sys, R, OM>(P, f, go, kind, gi);
#pragma unroll
    for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int m = 0; m < M; ++m) gin[(int64_t)(k * M + m) * ncell + src[k]] = gi[k * M + m];
}

// Cotangent of the physical distributions from the cotangent of the moments
// u(x) = sum_k f_k(src_k(x)) read with the pending shift sh.
template <int DIM, class R>
__global__ void __launch_bounds__(kBlock) k_adjoint_readout(const double *__restrict__ lam, R *__restrict__ g,
                                                            int64_t nx, int64_t ny, int M, Shift sh)
{
    constexpr int Q = Lattice<DIM>::Q;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    if (x >= nx) return;
    const int64_t ncell = nx * ny, o = y * nx + x;
    for (int m = 0; m < M; ++m) {
        const R l = R(lam[(int64_t)m * ncell + o]);
#pragma unroll
        for (int k = 0; k < Q; ++k) g[(int64_t)(k * M + m) * ncell + src_cell<DIM>(k, x, y, nx, ny, sh)] = l;
    }
}

// dJ/du0 = sum_k E_k(u0)^T g_k for f_0 = f^eq(u0)
template <class Sys, class R>
__global__ void __launch_bounds__(kBlock) k_adjoint_init(const double *__restrict__ u0, const R *__restrict__ g,
                                                         double *__restrict__ du0, int64_t ncell, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    R u[M], E[Q * M * M];
#pragma unroll
    for (int m = 0; m < M; ++m) u[m] = R(u0[(int64_t)m * ncell + i]);
    Sys::template equilibrium_jacobian<R>(P, u, E);
#pragma unroll
    for (int n = 0; n < M; ++n) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < Q; ++k)
#pragma unroll
            for (int m = 0; m < M; ++m)
                s += double(E[(k * M + m) * M + n]) * double(g[(int64_t)(k * M + m) * ncell + i]);
        du0[(int64_t)n * ncell + i] = s;
    }
}

// ---------------------------------------------------------------------------
// Batched persistent step: every instance of a batch advances through all the
// stages of one composite step in a single cooperative launch.  A stage is a
// sweep of the blocks over the work items (row segments of all instances,
// each pulled periodically within its own instance); grid.sync() separates the
// stages (the cooperative launch guarantees that all blocks are resident, and
// fails instead of starting otherwise).  Ping-pong: stage i reads pool[i & 1]
// and writes pool[(i + 1) & 1] relative to the entry side.
// ---------------------------------------------------------------------------
template <class R> struct BatchArgs {
    R *pool[2];
    const BatchInstance *inst;
    const BatchItem *items;
    int n_items;
    int side;  // pool holding the state on entry
    Counters *cnt;
    // recording (reverse mode): when set, stage st reads pool[side] (st = 0) or rec + (st - 1) pool_elems
    // and writes rec + st pool_elems, so every stage's output is kept; the pools are not written
    R *rec;
    int64_t pool_elems;
};

template <class Sys, class R, int OM>
__global__ void __launch_bounds__(kBlock) k_batch_step(BatchArgs<R> a, StageList sl, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    cg::grid_group grid = cg::this_grid();
    int side = a.side;
    for (int st = 0; st < sl.n; ++st) {
        const R *__restrict__ fin = (a.rec && st > 0) ? a.rec + (int64_t)(st - 1) * a.pool_elems : a.pool[side];
        R *__restrict__ fout = a.rec ? a.rec + (int64_t)st * a.pool_elems : a.pool[side ^ 1];
        const int s = sl.shift[st], kind = sl.kind[st];
        for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
            const BatchItem w = a.items[it];
            const BatchInstance I = a.inst[w.inst];
            const int64_t ncell = I.nx * I.ny;
            const R *fi = fin + I.offset;
            R *fo = fout + I.offset;
            Shift sh;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int64_t n = Lattice<2>::axis(k) == 0 ? I.nx : I.ny;
                int64_t r = (-(int64_t)Lattice<2>::sign(k) * s) % n;
                sh.roff[k] = r < 0 ? r + n : r;
            }
            for (int j = threadIdx.x; j < ((w.nx + 31) / 32) * 32; j += blockDim.x) {
                const bool valid = j < w.nx;
                bool fb = false;
                if (valid) {
                    const int64_t x = w.x0 + j, y = w.y;
                    R f[Q * M];
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        const int64_t src = src_cell<2>(k, x, y, I.nx, I.ny, sh);
#pragma unroll
                        for (int m = 0; m < M; ++m) f[k * M + m] = fi[(int64_t)(k * M + m) * ncell + src];
                    }
                    const int64_t o = y * I.nx + x;
                    relax_cell<Sys, R, OM>(P, f, kind, fb, record_of<Sys, R, OM>(P, st, I.cell0 + o, true));
#pragma unroll
                    for (int i = 0; i < Q * M; ++i) fo[(int64_t)i * ncell + o] = f[i];
                }
                if constexpr (checked<Sys, OM>()) warp_count(fb, &a.cnt->fallbacks);
            }
        }
        side ^= 1;
        grid.sync();
    }
}

// Batched reverse mode: the adjoint stages of one composite step of every instance in one
// cooperative launch, in reverse stage order with a grid barrier between stages.  Stage st's
// forward input is step_in (st = 0) or the recorded output of stage st - 1; the cotangent
// ping-pongs between cot[side] (the step output's on entry) and cot[side ^ 1].  Per cell the
// arithmetic is that of k_adjoint_stage: the transposed relaxation Jacobian, scattered by the
// reverse shift (each input cell receives exactly one contribution).
template <class R> struct BatchAdjointArgs {
    const R *step_in;
    const R *rec;
    int64_t pool_elems;
    R *cot[2];
    int side;
    const BatchInstance *inst;
    const BatchItem *items;
    int n_items;
};

template <class Sys, class R, int OM>
__global__ void __launch_bounds__(kBlock) k_batch_adjoint_step(BatchAdjointArgs<R> a, StageList sl, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    cg::grid_group grid = cg::this_grid();
    int side = a.side;
    for (int st = sl.n - 1; st >= 0; --st) {
        const R *__restrict__ fin = st > 0 ? a.rec + (int64_t)(st - 1) * a.pool_elems : a.step_in;
        const R *__restrict__ gout = a.cot[side];
        R *__restrict__ gin = a.cot[side ^ 1];
        const int s = sl.shift[st], kind = sl.kind[st];
        for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
            const BatchItem w = a.items[it];
            const BatchInstance I = a.inst[w.inst];
            const int64_t ncell = I.nx * I.ny;
            Shift sh;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int64_t n = Lattice<2>::axis(k) == 0 ? I.nx : I.ny;
                int64_t r = (-(int64_t)Lattice<2>::sign(k) * s) % n;
                sh.roff[k] = r < 0 ? r + n : r;
            }
            for (int j = threadIdx.x; j < w.nx; j += blockDim.x) {
                const int64_t x = w.x0 + j, y = w.y, o = y * I.nx + x;
                int64_t src[Q];
                R f[Q * M], go[Q * M], gi[Q * M];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    src[k] = src_cell<2>(k, x, y, I.nx, I.ny, sh);
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        f[k * M + m] = fin[I.offset + (int64_t)(k * M + m) * ncell + src[k]];
                        go[k * M + m] = gout[I.offset + (int64_t)(k * M + m) * ncell + o];
                    }
                }
                relax_adjoint<Sys, R, OM>(P, f, go, kind, gi);
#pragma unroll
                for (int k = 0; k < Q; ++k)
#pragma unroll
                    for (int m = 0; m < M; ++m) gin[I.offset + (int64_t)(k * M + m) * ncell + src[k]] = gi[k * M + m];
            }
        }
        side ^= 1;
        grid.sync();
    }
}

// f_k = f^eq_k(u0) (Section 3.1) with the domain check of Section 1.2.
template <class Sys, class R>
__global__ void __launch_bounds__(kBlock) k_init_eq(const double *__restrict__ u0, R *__restrict__ f,
                                                    int64_t ncell, ParamsR<double> P, Counters *cnt)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false, nonfinite = false;
    if (i < ncell) {
        double u[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            u[m] = u0[(int64_t)m * ncell + i];
            nonfinite |= !isfinite(u[m]);
        }
        bad = !Sys::template admissible<double>(P, u);
        double feq[Q * M];
        Sys::template equilibrium<double>(P, u, feq);
#pragma unroll
        for (int j = 0; j < Q * M; ++j) f[(int64_t)j * ncell + i] = R(P.shifted ? feq[j] - P.fbar[j] : feq[j]);
    }
    warp_count(bad, &cnt->domain_violations);
    warp_count(nonfinite, &cnt->non_finite);
}

// distributions from double planes (rounded to the storage precision)
template <class R>
__global__ void __launch_bounds__(kBlock) k_set(const double *__restrict__ src, R *__restrict__ f, int64_t n,
                                                double offset, Counters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool nonfinite = false;
    if (i < n) {
        const double v = src[i];
        nonfinite = !isfinite(v);
        f[i] = R(v - offset);
    }
    warp_count(nonfinite, &cnt->non_finite);
}

// Moments u_m = sum_k f_k,m, or the planes [p0, p0 + np) of the logical
// distributions, as double planes (the pending shift sh is applied; in the
// shifted storage f = stored + fbar).
struct RefPlanes {
    double fbar[16];
};

template <int DIM, class R, bool MOMENTS>
__global__ void __launch_bounds__(kBlock) k_gather(const R *__restrict__ f, double *__restrict__ out, int64_t nx,
                                                   int64_t ny, int M, int p0, int np, Shift sh, RefPlanes ref)
{
    constexpr int Q = Lattice<DIM>::Q;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    if (x >= nx) return;
    const int64_t ncell = nx * ny, o = y * nx + x;
    if (MOMENTS) {
        for (int m = 0; m < M; ++m) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k)
                s += double(f[(int64_t)(k * M + m) * ncell + src_cell<DIM>(k, x, y, nx, ny, sh)]) + ref.fbar[k * M + m];
            out[(int64_t)m * ncell + o] = s;
        }
    } else {
        for (int p = p0; p < p0 + np; ++p)
            out[(int64_t)(p - p0) * ncell + o] =
                double(f[(int64_t)p * ncell + src_cell<DIM>(p / M, x, y, nx, ny, sh)]) + ref.fbar[p];
    }
}

// Sum of v over a block of kRedThreads threads in a fixed order (deterministic,
// independent of scheduling): a shuffle tree inside each warp, then the warp
// sums, in warp order, by a shuffle tree in the first warp.  The total is
// returned to thread 0; part holds kRedThreads / 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double *part)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < kRedThreads / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();  // part is reused by the next call
    return t;
}

// Totals (double precision): per cell Sigma(f) = S(u) + sum_k B_k(f_k - f^eq_k),
// S(u), and u.  Pass 1: fixed grid of kRedBlocks blocks, each reducing a fixed
// set of cells in a fixed tree order into partials[block][2 + M].
template <class Sys, int DIM, class R>
__global__ void __launch_bounds__(kRedThreads) k_totals_partial(const R *__restrict__ f, double *__restrict__ partials,
                                                                int64_t nx, int64_t ny, Shift sh, ParamsR<double> P)
{
    constexpr int Q = Sys::Q, M = Sys::M, NV = 2 + M;
    const int64_t ncell = nx * ny;
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = c / nx, x = c - y * nx;
        double fc[Q * M], u[M];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int64_t s = src_cell<DIM>(k, x, y, nx, ny, sh);
#pragma unroll
            for (int m = 0; m < M; ++m) fc[k * M + m] = double(f[(int64_t)(k * M + m) * ncell + s]) + P.fbar[k * M + m];
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            double s = fc[m];
#pragma unroll
            for (int k = 1; k < Q; ++k) s += fc[k * M + m];
            u[m] = s;
        }
        double feq[Q * M], delta[Q * M];
        Sys::template equilibrium<double>(P, u, feq);
        deviations<Q, M, double>(feq, fc, delta);
        const double S = Sys::template entropy<double>(P, u);
        typename Sys::template Ctx<double> cx;
        Sys::template prepare<double>(P, u, delta, cx);
        double E, dE;
        const bool ok = Sys::template eval<double>(P, cx, -1.0, E, dE);
        acc[0] += ok ? S + E : NAN;
        acc[1] += S;
#pragma unroll
        for (int m = 0; m < M; ++m) acc[2 + m] += u[m];
    }
    __shared__ double part[kRedThreads / 32];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double t = block_sum(acc[v], part);
        if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * NV + v] = t;
    }
}

// Pass 2: one block sums the partials in a fixed order.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_totals_final(const double *__restrict__ partials, double *__restrict__ out,
                                                              int nblocks)
{
    constexpr int nv = NV;
    __shared__ double part[kRedThreads / 32];
    for (int v = 0; v < nv; ++v) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += partials[(int64_t)b * nv + v];
        const double t = block_sum(a, part);
        if (threadIdx.x == 0) out[v] = t;
    }
}

}  // namespace eslbm
