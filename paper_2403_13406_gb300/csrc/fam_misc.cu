// fam_misc.cu -- Euler (fixed omega), gathers, conversion and the dispatch
// entry points declared in launch.h.
#include <algorithm>
#include <cmath>

#include "family_impl.cuh"

namespace eslbm {

cudaError_t stage_scalar(int, bool, int, const StageLaunch &);
cudaError_t stage_sw1(bool, int, const StageLaunch &);
cudaError_t stage_sw2(bool, int, const StageLaunch &);
cudaError_t init_scalar(int, bool, const double *, void *, int64_t, const Params &, Counters *, cudaStream_t);
cudaError_t init_sw1(bool, const double *, void *, int64_t, const Params &, Counters *, cudaStream_t);
cudaError_t init_sw2(bool, const double *, void *, int64_t, const Params &, Counters *, cudaStream_t);
cudaError_t totals_scalar(int, bool, const void *, double *, double *, int64_t, int64_t, const Shift &,
                          const Params &, cudaStream_t);
cudaError_t totals_sw1(bool, const void *, double *, double *, int64_t, int64_t, const Shift &, const Params &,
                       cudaStream_t);
cudaError_t totals_sw2(bool, const void *, double *, double *, int64_t, int64_t, const Shift &, const Params &,
                       cudaStream_t);

cudaError_t stage_euler(bool, const StageLaunch &);
cudaError_t step2d_euler(bool, const Step2dLaunch &);
cudaError_t step2d_scalar(int, bool, int, const Step2dLaunch &);
cudaError_t step2d_sw2(bool, int, const Step2dLaunch &);
cudaError_t init_euler(bool, const double *, void *, int64_t, const Params &, Counters *, cudaStream_t);
cudaError_t totals_euler(bool, const void *, double *, double *, int64_t, int64_t, const Shift &, const Params &,
                         cudaStream_t);
cudaError_t adjoint_euler(bool, const AdjointLaunch &);
cudaError_t adjoint_init_euler(bool, const double *, const void *, double *, int64_t, const Params &, cudaStream_t);
cudaError_t batch_euler(bool, const BatchLaunch &);
int batch_occ_euler(bool);

cudaError_t fused_scalar(int, bool, int, const FusedLaunch &);
cudaError_t fused_sw1(bool, int, const FusedLaunch &);

cudaError_t launch_fused1d(int family, bool fp64, int om, const FusedLaunch &L)
{
    if (family == FAM_SW1) return fused_sw1(fp64, om, L);
    if (family == FAM_LINEAR1 || family == FAM_BURGERS1) return fused_scalar(family, fp64, om, L);
    return cudaErrorInvalidValue;
}

cudaError_t launch_stage(int family, bool fp64, int om, const StageLaunch &L)
{
    if (family == FAM_SW1) return stage_sw1(fp64, om, L);
    if (family == FAM_SW2) return stage_sw2(fp64, om, L);
    if (family == FAM_EULER2) return stage_euler(fp64, L);
    return stage_scalar(family, fp64, om, L);
}

cudaError_t launch_init_eq(int family, bool fp64, const double *u0, void *f, int64_t ncell, const Params &P,
                           Counters *cnt, cudaStream_t st)
{
    if (family == FAM_SW1) return init_sw1(fp64, u0, f, ncell, P, cnt, st);
    if (family == FAM_SW2) return init_sw2(fp64, u0, f, ncell, P, cnt, st);
    if (family == FAM_EULER2) return init_euler(fp64, u0, f, ncell, P, cnt, st);
    return init_scalar(family, fp64, u0, f, ncell, P, cnt, st);
}

cudaError_t launch_totals(int family, bool fp64, const void *f, double *partials, double *out, int64_t nx,
                          int64_t ny, const Shift &sh, const Params &P, cudaStream_t st)
{
    if (family == FAM_SW1) return totals_sw1(fp64, f, partials, out, nx, ny, sh, P, st);
    if (family == FAM_SW2) return totals_sw2(fp64, f, partials, out, nx, ny, sh, P, st);
    if (family == FAM_EULER2) return totals_euler(fp64, f, partials, out, nx, ny, sh, P, st);
    return totals_scalar(family, fp64, f, partials, out, nx, ny, sh, P, st);
}

template <int DIM, class R, bool MOM>
static cudaError_t gather_t(const void *f, double *out, int64_t nx, int64_t ny, int M, int p0, int np,
                            const Shift &sh, const double *fbar, cudaStream_t st)
{
    RefPlanes ref;
    for (int i = 0; i < 16; ++i) ref.fbar[i] = fbar ? fbar[i] : 0.0;
    dim3 grid((unsigned)((nx + kBlock - 1) / kBlock), (unsigned)ny);
    k_gather<DIM, R, MOM><<<grid, kBlock, 0, st>>>((const R *)f, out, nx, ny, M, p0, np, sh, ref);
    return cudaGetLastError();
}

cudaError_t launch_gather_moments(int dim, bool fp64, const void *f, double *out, int64_t nx, int64_t ny, int M,
                                  const Shift &sh, const double *fbar, cudaStream_t st)
{
    if (dim == 1)
        return fp64 ? gather_t<1, double, true>(f, out, nx, ny, M, 0, 0, sh, fbar, st)
                    : gather_t<1, float, true>(f, out, nx, ny, M, 0, 0, sh, fbar, st);
    return fp64 ? gather_t<2, double, true>(f, out, nx, ny, M, 0, 0, sh, fbar, st)
                : gather_t<2, float, true>(f, out, nx, ny, M, 0, 0, sh, fbar, st);
}

cudaError_t launch_gather_planes(int dim, bool fp64, const void *f, double *out, int64_t nx, int64_t ny, int M,
                                 int plane0, int nplanes, const Shift &sh, const double *fbar, cudaStream_t st)
{
    if (dim == 1)
        return fp64 ? gather_t<1, double, false>(f, out, nx, ny, M, plane0, nplanes, sh, fbar, st)
                    : gather_t<1, float, false>(f, out, nx, ny, M, plane0, nplanes, sh, fbar, st);
    return fp64 ? gather_t<2, double, false>(f, out, nx, ny, M, plane0, nplanes, sh, fbar, st)
                : gather_t<2, float, false>(f, out, nx, ny, M, plane0, nplanes, sh, fbar, st);
}

cudaError_t launch_set(bool fp64, const double *src, void *f, int64_t n, double offset, Counters *cnt,
                       cudaStream_t st)
{
    const unsigned grid = (unsigned)((n + kBlock - 1) / kBlock);
    if (fp64) k_set<double><<<grid, kBlock, 0, st>>>(src, (double *)f, n, offset, cnt);
    else k_set<float><<<grid, kBlock, 0, st>>>(src, (float *)f, n, offset, cnt);
    return cudaGetLastError();
}

// Host side: f^eq and the domain check of the reference state are the device
// formulas compiled for the host (they are __host__ __device__).
// The kernels evaluate f^eq with the parameters rounded to their arithmetic
// type, so the reference residual rdev = f^eq(ubar) - fbar must be taken with
// those same rounded parameters: with the exact ones it would hold a constant
// inconsistency (for shallow water (g - fl(g)) hbar^2 / (4V)) that the
// relaxation re-injects at every stage.
static ParamsR<double> kernel_params(const Params &P, bool fp64)
{
    ParamsR<double> d = params_as<double>(P);
    if (fp64) return d;
    const ParamsR<float> f = params_as<float>(P);
    d.V = f.V;
    d.inv2V = f.inv2V;
    for (int j = 0; j < 2; ++j) {
        d.a[j] = f.a[j];
        d.c[j] = f.c[j];
    }
    d.g = f.g;
    d.gamma_m1 = f.gamma_m1;
    d.gV4 = f.gV4;
    d.inv16gV = f.inv16gV;
    return d;
}

template <class Sys>
static bool reference_for(bool fp64, const double *u_ref, Params &P)
{
    constexpr int Q = Sys::Q, M = Sys::M;
    P.shifted = 0;
    const ParamsR<double> Pd = kernel_params(P, fp64);
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < M; ++m) {
        u[m] = u_ref[m];
        if (!std::isfinite(u[m])) return false;
    }
    if (!Sys::template admissible<double>(Pd, u)) return false;
    auto storage = [fp64](double v) { return fp64 ? v : (double)(float)v; };
    double feq[16];
    Sys::template equilibrium<double>(Pd, u, feq);
    for (int i = 0; i < 16; ++i) P.fbar[i] = i < Q * M ? storage(feq[i]) : 0.0;
    double ub[4] = {0.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < M; ++m) {
        double s = 0.0;  // exact: a few values of the storage precision
        for (int k = 0; k < Q; ++k) s += P.fbar[k * M + m];
        ub[m] = storage(s);
        P.ubar[m] = ub[m];
        P.cm[m] = s - ub[m];
    }
    for (int m = M; m < 4; ++m) P.ubar[m] = P.cm[m] = 0.0;
    if (!Sys::template admissible<double>(Pd, ub)) return false;
    Sys::template equilibrium<double>(Pd, ub, feq);
    for (int i = 0; i < 16; ++i) P.rdev[i] = i < Q * M ? feq[i] - P.fbar[i] : 0.0;
    // reference velocity (and pressure) of the deviation forms, from the rounded ubar
    for (int i = 0; i < 4; ++i) P.aux[i] = 0.0;
    if (M >= 2) {
        for (int j = 0; j + 1 < M && j < 2; ++j) P.aux[j] = ub[1 + j] / ub[0];
        if (M == 4) P.aux[2] = Pd.gamma_m1 * (ub[3] - 0.5 * (ub[1] * P.aux[0] + ub[2] * P.aux[1]));
    }
    P.shifted = 1;
    return true;
}

bool reference_state(int family, bool fp64, const double *u_ref, Params &P)
{
    switch (family) {
    case FAM_LINEAR1: return reference_for<Scalar<1, false>>(fp64, u_ref, P);
    case FAM_LINEAR2: return reference_for<Scalar<2, false>>(fp64, u_ref, P);
    case FAM_BURGERS1: return reference_for<Scalar<1, true>>(fp64, u_ref, P);
    case FAM_BURGERS2: return reference_for<Scalar<2, true>>(fp64, u_ref, P);
    case FAM_SW1: return reference_for<ShallowWater<1>>(fp64, u_ref, P);
    case FAM_SW2: return reference_for<ShallowWater<2>>(fp64, u_ref, P);
    case FAM_EULER2: return reference_for<Euler2>(fp64, u_ref, P);
    }
    return false;
}

cudaError_t adjoint_scalar(int, bool, int, const AdjointLaunch &);
cudaError_t adjoint_sw1(bool, int, const AdjointLaunch &);
cudaError_t adjoint_sw2(bool, int, const AdjointLaunch &);
cudaError_t adjoint_init_scalar(int, bool, const double *, const void *, double *, int64_t, const Params &,
                                cudaStream_t);
cudaError_t adjoint_init_sw1(bool, const double *, const void *, double *, int64_t, const Params &, cudaStream_t);
cudaError_t adjoint_init_sw2(bool, const double *, const void *, double *, int64_t, const Params &, cudaStream_t);

cudaError_t launch_adjoint_stage(int family, bool fp64, int om, const AdjointLaunch &L)
{
    if (family == FAM_SW1) return adjoint_sw1(fp64, om, L);
    if (family == FAM_SW2) return adjoint_sw2(fp64, om, L);
    if (family == FAM_EULER2) return adjoint_euler(fp64, L);
    return adjoint_scalar(family, fp64, om, L);
}

cudaError_t launch_adjoint_init(int family, bool fp64, const double *u0, const void *g, double *du0, int64_t ncell,
                                const Params &P, cudaStream_t st)
{
    if (family == FAM_SW1) return adjoint_init_sw1(fp64, u0, g, du0, ncell, P, st);
    if (family == FAM_SW2) return adjoint_init_sw2(fp64, u0, g, du0, ncell, P, st);
    if (family == FAM_EULER2) return adjoint_init_euler(fp64, u0, g, du0, ncell, P, st);
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

cudaError_t batch_scalar(int, bool, int, const BatchLaunch &);
cudaError_t batch_sw2(bool, int, const BatchLaunch &);
int batch_occ_scalar(int, bool, int);
int batch_occ_sw2(bool, int);

cudaError_t launch_batch_step(int family, bool fp64, int om, const BatchLaunch &L)
{
    if (family == FAM_SW2) return batch_sw2(fp64, om, L);
    if (family == FAM_EULER2) return batch_euler(fp64, L);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return batch_scalar(family, fp64, om, L);
    return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int family, bool fp64, int om)
{
    if (family == FAM_SW2) return batch_occ_sw2(fp64, om);
    if (family == FAM_EULER2) return batch_occ_euler(fp64);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return batch_occ_scalar(family, fp64, om);
    return 0;
}

cudaError_t check_sw1(bool, int, const Params &, Counters *, cudaStream_t);
cudaError_t check_sw2(bool, int, const Params &, Counters *, cudaStream_t);
cudaError_t check_scalar(int, bool, int, const Params &, Counters *, cudaStream_t);

cudaError_t launch_check(int family, bool fp64, int om, const Params &P, Counters *cnt, cudaStream_t st)
{
    if (family == FAM_SW1) return check_sw1(fp64, om, P, cnt, st);
    if (family == FAM_SW2) return check_sw2(fp64, om, P, cnt, st);
    return check_scalar(family, fp64, om, P, cnt, st);
}

cudaError_t launch_step2d(int family, bool fp64, int om, const Step2dLaunch &L)
{
    if (family == FAM_SW2) return step2d_sw2(fp64, om, L);
    if (family == FAM_EULER2) return step2d_euler(fp64, L);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return step2d_scalar(family, fp64, om, L);
    return cudaErrorInvalidValue;
}

int device_sms()
{
    static std::atomic<int> sm_count[kMaxDevices];
    const int d = device_slot();
    int sms = sm_count[d].load();
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            (void)cudaGetLastError();  // no device (host-only use): plan for one SM, leave no error behind
            return 1;
        }
        sm_count[d].store(sms);
    }
    return sms;
}

bool plan_step2d(int64_t nx, int64_t ny, int planes, int elem, int sms, const StageList &sl, Plan2d &pl)
{
    if (!stage_list_ok(sl) || sl.n > kStep2dMaxStages || planes < 1 || (elem != 4 && elem != 8)) return false;
    const int V4 = 16 / elem;
    if (nx % V4) return false;
    const int H = sl.halo;
    // lags of the stages behind the load, and the ring that keeps every slot until its last reader
    int lag = 0, acc = 0, E = 0;
    int64_t items_margin = 0;
    int m = 0;
    for (int j = 0; j < sl.n; ++j) {
        const int s = sl.shift[j], as = s < 0 ? -s : s;
        lag += as + (j > 0 ? 1 : 0);
        acc += s;
        m += as;
        E = std::max(E, lag + (acc < 0 ? -acc : acc));
        items_margin += 2 * (H - m);
    }
    pl.prefetch = kStep2dPrefetch;
    pl.ring = E + pl.prefetch;
    if (pl.ring > kStep2dMaxRing) return false;
    pl.hl = (H + V4 - 1) / V4 * V4;
    const int64_t budget = kStep2dSmemBudget - kStep2dBarBytes;
    const int wx_max = (int)(budget / ((int64_t)pl.ring * planes * elem)) / V4 * V4;
    const int tx_max = wx_max - 2 * pl.hl;
    // a tick's items (about n tx) must fit the slots of the smallest block
    const int tx_cap = (int)std::min<int64_t>(tx_max, (kStep2dMaxItems - items_margin) / sl.n / V4 * V4);
    if (tx_cap < std::max(4 * V4, pl.hl)) return false;
    // strips as wide as the window allows, evened out over the row
    int64_t nstrips = (nx + tx_cap - 1) / tx_cap;
    const int64_t even = (nx + nstrips - 1) / nstrips;
    pl.tx = (int)((even + V4 - 1) / V4 * V4);
    nstrips = (nx + pl.tx - 1) / pl.tx;
    pl.nstrips = (int)nstrips;
    pl.wx = pl.tx + 2 * pl.hl;
    // rows per block: the time is (waves of kStep2dBlocksPerSm blocks per SM) x (ticks of a block)
    static const int cand[] = {32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 8192};
    double best = 0.0;
    pl.ly = 0;
    for (int ly : cand) {
        const int lye = (int)std::min<int64_t>(ly, ny);
        const int64_t nsegs = (ny + lye - 1) / lye;
        const int64_t blocks = nstrips * nsegs;
        const int64_t waves = (blocks + (int64_t)sms * kStep2dBlocksPerSm - 1) / ((int64_t)sms * kStep2dBlocksPerSm);
        const double cost = (double)waves * (double)(lye + H + lag);
        if (pl.ly == 0 || cost < best) {
            best = cost;
            pl.ly = lye;
            pl.nsegs = (int)nsegs;
        }
        if (ly >= ny) break;
    }
    if ((int64_t)pl.nstrips * pl.nsegs > 0x7fffffffLL) return false;
    pl.items = (int)((int64_t)sl.n * pl.tx + items_margin);
    pl.smem = (size_t)kStep2dBarBytes + (size_t)pl.ring * planes * pl.wx * elem;
    return pl.smem <= (size_t)kStep2dSmemBudget;
}

cudaError_t batch_adjoint_sw2(bool, int, const BatchAdjointLaunch &);
cudaError_t batch_adjoint_scalar(int, bool, int, const BatchAdjointLaunch &);
cudaError_t batch_adjoint_euler(bool, const BatchAdjointLaunch &);
int batch_adjoint_occ_sw2(bool, int);
int batch_adjoint_occ_scalar(int, bool, int);
int batch_adjoint_occ_euler(bool);

cudaError_t launch_batch_adjoint_step(int family, bool fp64, int om, const BatchAdjointLaunch &L)
{
    if (family == FAM_SW2) return batch_adjoint_sw2(fp64, om, L);
    if (family == FAM_EULER2) return batch_adjoint_euler(fp64, L);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return batch_adjoint_scalar(family, fp64, om, L);
    return cudaErrorInvalidValue;
}

int batch_adjoint_blocks_per_sm(int family, bool fp64, int om)
{
    if (family == FAM_SW2) return batch_adjoint_occ_sw2(fp64, om);
    if (family == FAM_EULER2) return batch_adjoint_occ_euler(fp64);
    if (family == FAM_LINEAR2 || family == FAM_BURGERS2) return batch_adjoint_occ_scalar(family, fp64, om);
    return 0;
}

int totals_blocks() { return kRedBlocks; }

}  // namespace eslbm
