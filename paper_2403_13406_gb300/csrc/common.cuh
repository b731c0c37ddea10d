// common.cuh -- shared device-side definitions of the sm_103a composite-step
// library: launch parameters, velocity sets and small helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace eslbm {

// Physical and numerical parameters of a run, passed by value to kernels.
struct Params {
    double V;        // lattice velocity
    double a[2];     // linear transport velocity
    double c[2];     // Burgers flux coefficients
    double g;        // gravity
    double gamma;    // Euler
    double omega;    // fixed relaxation parameter
    double t_max;    // entropic search interval for omega - 1
    // Shifted storage: the state holds g = f - fbar for a constant reference
    // equilibrium fbar_k = f^eq_k(u_ref) (rounded to the storage precision), so
    // that the storage rounding is relative to the deviation from the reference
    // state instead of to f.  The relaxation then works on deviations:
    // u = ubar + du with du = sum_k g_k + cm, and its target
    // f^eq_k(u) - fbar_k = [f^eq_k(u) - f^eq_k(ubar)] + rdev_k with the bracket in
    // deviation form (no cancellation).  ubar is sum_k fbar_k rounded to the
    // storage precision, cm that rounding's residual, rdev_k = f^eq_k(ubar) - fbar_k.
    int shifted;
    double fbar[16], ubar[4], cm[4], rdev[16];
    double aux[4];  // reference quantities of the deviation forms (velocities, pressure)
    // Diagnostics: when rec is set (a device buffer in the storage precision), an
    // entropic kernel records the inputs of every relaxation it performs -- the
    // moments u (M values), the deviations delta (q M) and the omega used -- at
    // rec[((i * rec_stages) + stage) * rec_cells + cell] for field i, and a separate
    // kernel checks them (k_check).  Recording only stores values the relaxation
    // holds anyway, behind a uniform branch: the arithmetic is the same with and
    // without it.  A projection records omega = 1 only.
    uint64_t rec;
    int64_t rec_cells;
    int rec_stages;
};

// The same parameters in the arithmetic type of a kernel (converted once on the
// host, so a float kernel executes no double-precision instruction), with the
// derived constants the kernels need.
template <class R> struct ParamsR {
    R V, inv2V, a[2], c[2], g, gamma_m1, omega, t_max;
    R gV4, inv16gV;  // 4 g V and 1 / (16 g V) (shallow water)
    int shifted;     // see Params
    R ubar[4], cm[4], rdev[16], fbar[16], aux[4];
    R *rec;          // see Params
    int64_t rec_cells;
    int rec_stages;
};

template <class R> inline ParamsR<R> params_as(const Params &P)
{
    ParamsR<R> q;
    q.V = R(P.V);
    q.inv2V = R(0.5 / P.V);
    q.a[0] = R(P.a[0]);
    q.a[1] = R(P.a[1]);
    q.c[0] = R(P.c[0]);
    q.c[1] = R(P.c[1]);
    q.g = R(P.g);
    q.gamma_m1 = R(P.gamma - 1.0);
    q.omega = R(P.omega);
    q.t_max = R(P.t_max);
    q.gV4 = R(4.0 * P.g * P.V);
    q.inv16gV = P.g > 0 ? R(1.0 / (16.0 * P.g * P.V)) : R(0);
    q.shifted = P.shifted;
    q.rec = reinterpret_cast<R *>(P.rec);
    q.rec_cells = P.rec_cells;
    q.rec_stages = P.rec_stages;
    for (int i = 0; i < 4; ++i) {
        q.ubar[i] = R(P.ubar[i]);
        q.cm[i] = R(P.cm[i]);
        q.aux[i] = R(P.aux[i]);
    }
    for (int i = 0; i < 16; ++i) {
        q.rdev[i] = R(P.rdev[i]);
        q.fbar[i] = R(P.fbar[i]);
    }
    return q;
}

enum { KIND_MAIN = 0, KIND_PROJECT = 1 };

// How a kernel chooses omega: the fixed value, the entropic root in the storage
// precision, or (FP32 storage only) the entropic root with the entropy
// difference evaluated in FP64.
enum OmegaMode { OM_FIXED = 0, OM_ENTROPIC = 1, OM_MIXED = 2 };

// Velocity sets of Section 1.2: D1Q2 = (+V, -V); D2Q4 = (+V,0), (0,+V), (-V,0), (0,-V).
template <int DIM> struct Lattice;
template <> struct Lattice<1> {
    static constexpr int Q = 2;
    __host__ __device__ static constexpr int axis(int) { return 0; }
    __host__ __device__ static constexpr int sign(int k) { return k == 0 ? 1 : -1; }
};
template <> struct Lattice<2> {
    static constexpr int Q = 4;
    __host__ __device__ static constexpr int axis(int k) { return k & 1; }
    __host__ __device__ static constexpr int sign(int k) { return k < 2 ? 1 : -1; }
};

// Pull offsets of one fused stage: population k at cell x reads the value at
// x + roff[k] (mod n) along its axis, i.e. x - sign_k * shift (eq. transportPhase).
struct Shift {
    int64_t roff[4];
};

// Stages fused into one launch of a temporally blocked kernel.  halo must equal
// the sum of |shift| over the stages: the kernels size their windows by it and
// compute, at each stage, only the cells that can still reach the output tile
// (the launchers reject a list whose halo differs).
constexpr int kMaxFusedStages = 64;
struct StageList {
    int n;                       // stages
    int halo;                    // sum of |shift|
    int shift[kMaxFusedStages];  // transport before each relaxation
    int kind[kMaxFusedStages];   // KIND_MAIN or KIND_PROJECT
};

// Limits of the temporally blocked 2D kernel (k_step2d): threads of a block,
// stages of one launch, rows of the ring (one mbarrier each, at the start of the
// dynamic shared memory) and dynamic shared memory of a block (227 KB per block
// on sm_103, less 2 KB for the kernel's static arrays).
#ifndef ESLBM_STEP2D_BLOCKS_PER_SM
#define ESLBM_STEP2D_BLOCKS_PER_SM 1
#endif
#ifndef ESLBM_STEP2D_PREFETCH
#define ESLBM_STEP2D_PREFETCH 3
#endif
#ifndef ESLBM_STEP2D_THREADS
#define ESLBM_STEP2D_THREADS 768
#endif
constexpr int kStep2dThreads = ESLBM_STEP2D_THREADS;             // threads of a block (most variants)
constexpr int kStep2dSlots = 8;                                   // items (stage, column) a thread owns
constexpr int kStep2dMaxItems = kStep2dSlots * (256 - 32);        // items of a tick (smallest block: 256)
constexpr int kStep2dBlocksPerSm = ESLBM_STEP2D_BLOCKS_PER_SM;  // resident blocks per SM (shared memory split)
constexpr int kStep2dPrefetch = ESLBM_STEP2D_PREFETCH;          // window rows loaded ahead of use
constexpr int kStep2dMaxStages = 32;
constexpr int kStep2dMaxRing = 64;
constexpr int kStep2dBarBytes = 8 * kStep2dMaxRing;
constexpr int kStep2dSmemBudget = 232448 / kStep2dBlocksPerSm - 2048;

// Launch plan of the temporally blocked 2D kernel (k_step2d) for one group of
// stages: a block owns tx x ly output cells and keeps `ring` rows of a window
// tx + 2 hl wide in shared memory (see step2d.cuh).
struct Plan2d {
    int tx, ly, hl, wx, ring, prefetch, nstrips, nsegs;
    int items;    // (stage, column) items of a tick: sum over the stages of tx + 2 (H - m_j)
    size_t smem;  // dynamic shared memory bytes
};

inline bool stage_list_ok(const StageList &sl)
{
    if (sl.n < 1 || sl.n > kMaxFusedStages) return false;
    long long h = 0;
    for (int i = 0; i < sl.n; ++i) h += sl.shift[i] < 0 ? -(long long)sl.shift[i] : sl.shift[i];
    return h == sl.halo;
}

// Batched execution: independent instances of one system on grids of their own
// size, packed in one pool per ping-pong side, cut into work items.
struct BatchInstance {
    int64_t nx, ny;
    int64_t offset;  // element offset of the instance's first plane in the pool
    int64_t cell0;   // index of the instance's first cell among the cells of all instances
};
struct BatchItem {
    int32_t inst;    // instance
    int32_t y;       // row
    int32_t x0, nx;  // segment [x0, x0 + nx) of the row
};

// Device counters (first 64 bytes of the workspace).
struct Counters {
    unsigned long long fallbacks;
    unsigned long long entropy_increases;
    unsigned int omega_min_bits;   // float bits of the smallest omega (positive floats order as ints)
    unsigned int omega_max_bits;
    unsigned long long domain_violations;
    unsigned long long non_finite;
    unsigned long long copy_timeouts;  // bulk-copy waits that gave up (never expected; reported as an error)
    unsigned int excess_max_bits;      // float bits of the largest per-cell F(omega - 1) / B(-1) seen (>= 0)
    unsigned int pad0;
    unsigned long long pad1;
};

template <class R> struct Tol;
// Newton stops when its last step is below this fraction of the iterate; one
// more evaluation then brings the error to the rounding level (quadratic
// convergence), and the final chord keeps the root on the non-increasing side.
template <> struct Tol<float> {
    static constexpr float newton = 1e-4f;
    static constexpr float inner = 2e-6f;
    static constexpr float inner_accept = 1e-4f;
    static constexpr int max_outer = 32;
    static constexpr int min_inner = 2;
    static constexpr int max_inner = 8;
};
template <> struct Tol<double> {
    static constexpr double newton = 1e-9;
    static constexpr double inner = 4e-16;
    static constexpr double inner_accept = 1e-12;
    static constexpr int max_outer = 64;
    static constexpr int min_inner = 2;
    static constexpr int max_inner = 12;
};

}  // namespace eslbm
