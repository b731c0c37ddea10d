// launch.h -- host-side launchers of the templated kernels, one translation
// unit per system family so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace eslbm {

struct StageLaunch {
    const void *fin;
    void *fout;
    int64_t nx, ny, ncell;
    Shift sh;
    int kind;
    Counters *cnt;
    Params P;
    cudaStream_t stream;
};

enum Family { FAM_LINEAR1, FAM_LINEAR2, FAM_BURGERS1, FAM_BURGERS2, FAM_SW1, FAM_SW2, FAM_EULER2 };

struct FusedLaunch {
    const void *fin;
    void *fout;
    int64_t n;
    StageList sl;
    Counters *cnt;
    Params P;
    cudaStream_t stream;
    void *rec = nullptr;         // optional: the outputs of the first nrec stages go to rec + i * rec_stride
    int64_t rec_stride_bytes = 0;
    int nrec = 0;
};

// temporally blocked 1D step (several stages in shared memory); 1D families only
cudaError_t launch_fused1d(int family, bool fp64, int om, const FusedLaunch &L);

struct Step2dLaunch {
    const void *fin;
    void *fout;
    int64_t nx, ny, ncell;
    StageList sl;  // the stages of this launch (halo = sum |shift|)
    Plan2d plan;   // from plan_step2d
    Counters *cnt;
    Params P;
    cudaStream_t stream;
};

// Plan of one launch of the temporally blocked 2D kernel for the stages sl on an
// nx x ny grid with `planes` planes of `elem`-byte values on `sms` SMs; false if
// the stages do not fit (rows not on 16-byte boundaries, ring or window too large).
bool plan_step2d(int64_t nx, int64_t ny, int planes, int elem, int sms, const StageList &sl, Plan2d &out);
// several fused stages of a 2D lattice in one launch (plan from plan_step2d)
cudaError_t launch_step2d(int family, bool fp64, int om, const Step2dLaunch &L);
// SMs of the current device (cached per device)
int device_sms();

// fused pull-shift + relaxation stage
cudaError_t launch_stage(int family, bool fp64, int om, const StageLaunch &L);
// Diagnostics: fields of one relaxation record (M moments, q M deviations, omega) and the
// per-cell check of the records the previous launch wrote (P.rec, rec_stages, rec_cells)
inline int record_fields(int q, int M) { return M + q * M + 1; }
cudaError_t launch_check(int family, bool fp64, int om, const Params &P, Counters *cnt, cudaStream_t st);
// f = f^eq(u0) with the domain check
cudaError_t launch_init_eq(int family, bool fp64, const double *u0, void *f, int64_t ncell, const Params &P,
                           Counters *cnt, cudaStream_t st);
// totals of Sigma, S and u in double precision into out[2 + M]
cudaError_t launch_totals(int family, bool fp64, const void *f, double *partials, double *out, int64_t nx,
                          int64_t ny, const Shift &sh, const Params &P, cudaStream_t st);
// gathers (pending shift applied) and conversion
// (fbar: the 16 reference distributions of the shifted storage, zeros otherwise)
cudaError_t launch_gather_moments(int dim, bool fp64, const void *f, double *out, int64_t nx, int64_t ny, int M,
                                  const Shift &sh, const double *fbar, cudaStream_t st);
cudaError_t launch_gather_planes(int dim, bool fp64, const void *f, double *out, int64_t nx, int64_t ny, int M,
                                 int plane0, int nplanes, const Shift &sh, const double *fbar, cudaStream_t st);
// f = src - offset rounded to the storage precision
cudaError_t launch_set(bool fp64, const double *src, void *f, int64_t n, double offset, Counters *cnt,
                       cudaStream_t st);
// Reference equilibrium of the shifted storage for u_ref (fills P.fbar, ubar, cm,
// rdev for the storage precision); false if u_ref is outside the domain.
bool reference_state(int family, bool fp64, const double *u_ref, Params &P);

struct AdjointLaunch {
    const void *fin;   // forward input of the stage (physical layout)
    const void *gout;  // cotangent of the stage output
    void *gin;         // cotangent of the stage input (written)
    int64_t nx, ny;
    Shift sh;
    int kind;
    Params P;
    cudaStream_t stream;
};

// reverse-mode stage (reverse shift + transposed relaxation Jacobian)
cudaError_t launch_adjoint_stage(int family, bool fp64, int om, const AdjointLaunch &L);
// cotangent of the distributions from the cotangent of the moments (pending shift sh)
cudaError_t launch_adjoint_readout(int dim, bool fp64, const double *lam, void *g, int64_t nx, int64_t ny, int M,
                                   const Shift &sh, cudaStream_t st);
// dJ/du0 from the cotangent of f_0 = f^eq(u0)
cudaError_t launch_adjoint_init(int family, bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                                const Params &P, cudaStream_t st);

struct BatchLaunch {
    void *pool[2];
    const BatchInstance *inst;  // device array
    const BatchItem *items;     // device array
    int n_items;
    int side;
    Counters *cnt;
    StageList sl;
    Params P;
    int grid;  // blocks (all resident: cooperative launch)
    cudaStream_t stream;
    void *rec = nullptr;     // reverse mode: keep every stage's output at rec + st * pool_elems
    int64_t pool_elems = 0;  // elements of one pool
};

// one composite step of every instance of a 2D batch (cooperative, grid.sync between stages)
cudaError_t launch_batch_step(int family, bool fp64, int om, const BatchLaunch &L);

struct BatchAdjointLaunch {
    const void *step_in;  // forward input of the step (a pool)
    const void *rec;      // outputs of its stages 0 .. n-2 (pools)
    int64_t pool_elems;
    void *cot[2];         // cotangent pools; cot[side] holds the step output's cotangent on entry
    int side;
    const BatchInstance *inst;
    const BatchItem *items;
    int n_items;
    StageList sl;
    Params P;
    int grid;
    cudaStream_t stream;
};

// the adjoint stages of one step of every instance (cooperative, reverse order)
cudaError_t launch_batch_adjoint_step(int family, bool fp64, int om, const BatchAdjointLaunch &L);
int batch_adjoint_blocks_per_sm(int family, bool fp64, int om);
// resident blocks per SM of that kernel (0 if the family has no batched kernel)
int batch_blocks_per_sm(int family, bool fp64, int om);

int totals_blocks();

}  // namespace eslbm
