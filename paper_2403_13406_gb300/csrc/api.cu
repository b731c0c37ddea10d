// api.cu -- host implementation of the C ABI declared in include/eslbm.h.
//
// The composite step is kept as the paper's operator list (transports T(s) and
// relaxations R) built from the rational composition weights; a small
// interpreter merges adjacent transports into the pull-shift of the next fused
// stage and carries the trailing transport as a pending shift, so a run of n
// steps of scheme I is T(1), then 18 n fused stages, then T(1) at readback.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/eslbm.h"
#include "host_schedule.h"
#include "launch.h"

using namespace eslbm;

namespace {

constexpr size_t kCountersBytes = 256;

eslbm_status validate(const eslbm_config *c)
{
    if (!c) return ESLBM_ERR_ARG;
    if (c->dim != 1 && c->dim != 2) return ESLBM_ERR_ARG;
    if (c->system < ESLBM_LINEAR || c->system > ESLBM_EULER) return ESLBM_ERR_ARG;
    if (c->precision != ESLBM_FP32 && c->precision != ESLBM_FP64 && c->precision != ESLBM_FP32_MIXED)
        return ESLBM_ERR_ARG;
    if (c->blocking < 0 || c->blocking > kStep2dMaxStages) return ESLBM_ERR_ARG;
    if (c->omega_mode != ESLBM_OMEGA_FIXED && c->omega_mode != ESLBM_OMEGA_ENTROPIC) return ESLBM_ERR_ARG;
    if (c->scheme < ESLBM_SCHEME_I || c->scheme > ESLBM_SCHEME_B) return ESLBM_ERR_ARG;
    if (c->kappa < 1 || c->kappa > 1024) return ESLBM_ERR_ARG;
    if (c->nx < 1 || c->ny < 1 || (c->dim == 1 && c->ny != 1)) return ESLBM_ERR_ARG;
    if (c->dim == 2 && c->ny > 65535) return ESLBM_ERR_ARG;  // one grid row of blocks per cell row
    if (c->nx > (int64_t(1) << 40) || c->nx * c->ny > (int64_t(1) << 40)) return ESLBM_ERR_ARG;
    if (!(c->V > 0.0) || !std::isfinite(c->V)) return ESLBM_ERR_ARG;
    if (c->omega_mode == ESLBM_OMEGA_FIXED && !(std::isfinite(c->omega))) return ESLBM_ERR_ARG;
    if (c->t_max < 0.0 || !std::isfinite(c->t_max)) return ESLBM_ERR_ARG;
    if (c->shifted != 0 && c->shifted != 1) return ESLBM_ERR_ARG;
    if (c->system == ESLBM_SHALLOW_WATER && !(c->g > 0.0)) return ESLBM_ERR_ARG;
    if (c->system == ESLBM_EULER) {
        if (c->dim != 2) return ESLBM_ERR_UNSUPPORTED;
        if (!(c->gamma > 1.0)) return ESLBM_ERR_ARG;
        if (c->omega_mode == ESLBM_OMEGA_ENTROPIC) return ESLBM_ERR_UNSUPPORTED;
    }
    if (c->system == ESLBM_LINEAR) {  // sub-characteristic condition (Examples 1 and 4)
        const double lim = c->dim == 1 ? c->V : 0.5 * c->V;
        for (int j = 0; j < c->dim; ++j)
            if (!(std::fabs(c->a[j]) < lim)) return ESLBM_ERR_DOMAIN;
    }
    return ESLBM_OK;
}

// steps fused into one launch of the 1D kernel: one composite step, or up to 24 steps of the
// short schemes
int64_t fused_group_of(int64_t stages_per_step)
{
    return stages_per_step >= 16 ? 1 : std::max<int64_t>(1, 24 / stages_per_step);
}

// Most stages of one launch of the temporally blocked 2D kernel: the configuration's limit, or with
// AUTO the fastest measured on GB300 -- two stages a launch for the 16-plane Euler state in FP32 with a
// fixed omega (3.28e9 against 3.03e9 site updates/s at 8192^2: the per-stage kernel is at the HBM
// roofline, the blocked one halves the traffic and is bound by instruction issue), one launch per
// stage otherwise (the blocked kernel was slower for the 4-plane states and for the entropic
// relaxations, whose arithmetic bounds both paths).
int max_group2d_of(const eslbm_config &c, int64_t planes)
{
    if (c.blocking >= 2) return c.blocking;
    if (c.blocking == ESLBM_BLOCKING_AUTO && c.dim == 2 && planes >= 16 && c.omega_mode == ESLBM_OMEGA_FIXED &&
        c.precision != ESLBM_FP64)
        return 2;
    return 0;
}

// 2D runs take the temporally blocked kernel when it applies (above) and rows start on 16-byte
// boundaries, else one launch per stage.
bool blocked2d_of(const eslbm_config &c, int64_t planes)
{
    return c.dim == 2 && max_group2d_of(c, planes) >= 2 && c.nx % (c.precision == ESLBM_FP64 ? 2 : 4) == 0;
}

// Stages one launch may run: the record buffer of the diagnostics holds that many.
int64_t max_launch_stages(const eslbm_config &c, int64_t stages_per_step, int64_t planes)
{
    if (c.dim == 1 && c.blocking != ESLBM_BLOCKING_OFF) return stages_per_step * fused_group_of(stages_per_step);
    if (blocked2d_of(c, planes))
        return std::min<int64_t>(stages_per_step, std::min(max_group2d_of(c, planes), kStep2dMaxStages));
    return 1;
}

// workspace: counters, FP64 reduction partials and totals, then the records (diagnostics)
constexpr size_t kRecordsOffset = kCountersBytes + sizeof(double) * 6 * 1024 + 256;

}  // namespace

struct eslbm_handle {
    eslbm_config cfg;
    eslbm_sizes sz;
    int family;
    bool fp64;
    int om;  // OmegaMode
    void *f[2];
    int cur;
    char *ws;
    cudaStream_t stream;
    int64_t pending;
    Params P;
    std::vector<Op> ops;
    uint64_t relaxations;
    std::string err;
    // graph replay of `graph_steps` steps entered with (graph_pending, graph_cur)
    bool use_graph;
    cudaGraphExec_t gexec;
    int64_t graph_pending;
    int graph_cur;
    int graph_steps;
    int graph_cur_after;
    int64_t graph_pending_after;

    Counters *counters() { return reinterpret_cast<Counters *>(ws); }
    double *partials() { return reinterpret_cast<double *>(ws + kCountersBytes); }
    double *totals_out()
    {
        return reinterpret_cast<double *>(ws + kCountersBytes + sizeof(double) * 6 * (size_t)totals_blocks());
    }
    void *records() { return ws + kRecordsOffset; }
    void *spare() { return f[1 - cur]; }
};

namespace {

eslbm_status fail(eslbm_handle *h, eslbm_status s, const std::string &msg)
{
    if (h) h->err = msg;
    return s;
}

eslbm_status cuda_fail(eslbm_handle *h, cudaError_t e, const char *where)
{
    return fail(h, ESLBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

// pull offsets that apply a transport by s cells to every population
Shift make_shift(const eslbm_handle *h, int64_t s)
{
    Shift sh;
    const int q = (int)h->sz.q;
    for (int k = 0; k < 4; ++k) sh.roff[k] = 0;
    for (int k = 0; k < q; ++k) {
        const int axis = h->cfg.dim == 1 ? 0 : (k & 1);
        const int sign = h->cfg.dim == 1 ? (k == 0 ? 1 : -1) : (k < 2 ? 1 : -1);
        const int64_t n = axis == 0 ? h->cfg.nx : h->cfg.ny;
        int64_t r = (-(int64_t)sign * s) % n;  // value at x comes from x - sign * s
        if (r < 0) r += n;
        sh.roff[k] = r;
    }
    return sh;
}

// kernel parameters of a launch of `stages` stages: with diagnostics the launch records its
// relaxations (Params::rec)
Params launch_params(const eslbm_handle *h, int stages)
{
    Params P = h->P;
    if (records_of(h->cfg)) {
        P.rec = (uint64_t)(uintptr_t)const_cast<eslbm_handle *>(h)->records();
        P.rec_cells = h->sz.ncell;
        P.rec_stages = stages;
    }
    return P;
}

// the per-cell check of what the launch recorded (diagnostics)
eslbm_status check_records(eslbm_handle *h, const Params &P)
{
    if (!P.rec) return ESLBM_OK;
    CK(launch_check(h->family, h->fp64, h->om, P, h->counters(), h->stream), "entropy check");
    return ESLBM_OK;
}

eslbm_status launch_one_stage(eslbm_handle *h, int64_t shift, int kind)
{
    StageLaunch L;
    L.fin = h->f[h->cur];
    L.fout = h->f[1 - h->cur];
    L.nx = h->cfg.nx;
    L.ny = h->cfg.ny;
    L.ncell = h->sz.ncell;
    L.sh = make_shift(h, shift);
    L.kind = kind;
    L.cnt = h->counters();
    L.P = launch_params(h, 1);
    L.stream = h->stream;
    CK(launch_stage(h->family, h->fp64, h->om, L), "stage launch");
    h->cur = 1 - h->cur;
    h->relaxations += (uint64_t)h->sz.ncell;
    return check_records(h, L.P);
}

eslbm_status run_ops(eslbm_handle *h)
{
    for (const Op &op : h->ops) {
        if (!op.relax) {
            h->pending += op.shift;
            continue;
        }
        eslbm_status s = launch_one_stage(h, h->pending, op.kind);
        if (s != ESLBM_OK) return s;
        h->pending = 0;
    }
    return ESLBM_OK;
}

// 1D runs use the temporally blocked kernel (unless blocking is off): the stages of
// `steps` consecutive steps (merged shifts, as in run_ops) in one launch.
bool fused_path(const eslbm_handle *h) { return h->cfg.dim == 1 && h->cfg.blocking != ESLBM_BLOCKING_OFF; }

int64_t fused_group(const eslbm_handle *h) { return fused_group_of(h->sz.stages_per_step); }

eslbm_status run_fused(eslbm_handle *h, int64_t steps)
{
    FusedLaunch L;
    L.sl.n = 0;
    L.sl.halo = 0;
    for (int64_t i = 0; i < steps; ++i) {
        for (const Op &op : h->ops) {
            if (!op.relax) {
                h->pending += op.shift;
                continue;
            }
            if (L.sl.n >= kMaxFusedStages) return fail(h, ESLBM_ERR_ARG, "too many fused stages");
            const int64_t s = h->pending;
            if (s > (1 << 20) || s < -(1 << 20)) return fail(h, ESLBM_ERR_ARG, "shift too large to fuse");
            L.sl.shift[L.sl.n] = (int)s;
            L.sl.kind[L.sl.n] = op.kind;
            L.sl.halo += (int)(s < 0 ? -s : s);
            L.sl.n += 1;
            h->pending = 0;
        }
    }
    if (L.sl.n == 0) return ESLBM_OK;
    L.fin = h->f[h->cur];
    L.fout = h->f[1 - h->cur];
    L.n = h->cfg.nx;
    L.cnt = h->counters();
    L.P = launch_params(h, L.sl.n);
    L.stream = h->stream;
    CK(launch_fused1d(h->family, h->fp64, h->om, L), "fused step launch");
    h->cur = 1 - h->cur;
    h->relaxations += (uint64_t)h->sz.ncell * (uint64_t)L.sl.n;
    return check_records(h, L.P);
}

// 2D runs use the temporally blocked 2D kernel (unless blocking is off) when rows start on
// 16-byte boundaries: the stages of a step in groups, each group one launch.
bool blocked2d_path(const eslbm_handle *h) { return blocked2d_of(h->cfg, h->sz.planes); }

int max_group2d(const eslbm_handle *h) { return max_group2d_of(h->cfg, h->sz.planes); }

struct Group2d {
    StageList sl;
    Plan2d plan;
};

// The stages of one step from `pending` (merged shifts, as in run_ops) in groups of at most
// max_group2d stages, split evenly; a group whose window does not fit is halved until it does.
bool step_groups2d(const eslbm_handle *h, int64_t pending, std::vector<Group2d> &out, int64_t *pending_after)
{
    std::vector<std::pair<int, int>> st;  // (shift, kind)
    for (const Op &op : h->ops) {
        if (!op.relax) {
            pending += op.shift;
            continue;
        }
        if (pending > 64 || pending < -64) return false;
        st.push_back({(int)pending, op.kind});
        pending = 0;
    }
    *pending_after = pending;
    out.clear();
    const int n = (int)st.size();
    const int gmax = std::max(1, std::min(max_group2d(h), kStep2dMaxStages));
    const int ngroups = (n + gmax - 1) / gmax;
    const int elem = h->fp64 ? 8 : 4;
    const int sms = device_sms();
    std::vector<std::pair<int, int>> spans;  // [first, count)
    for (int g = 0, first = 0; g < ngroups; ++g) {
        const int cnt = n / ngroups + (g < n % ngroups ? 1 : 0);
        spans.push_back({first, cnt});
        first += cnt;
    }
    for (size_t i = 0; i < spans.size(); ++i) {
        Group2d G;
        G.sl.n = spans[i].second;
        G.sl.halo = 0;
        for (int j = 0; j < G.sl.n; ++j) {
            G.sl.shift[j] = st[(size_t)(spans[i].first + j)].first;
            G.sl.kind[j] = st[(size_t)(spans[i].first + j)].second;
            G.sl.halo += std::abs(G.sl.shift[j]);
        }
        if (plan_step2d(h->cfg.nx, h->cfg.ny, (int)h->sz.planes, elem, sms, G.sl, G.plan)) {
            out.push_back(G);
        } else {
            if (G.sl.n == 1) return false;
            const int half = G.sl.n / 2;
            spans.insert(spans.begin() + (long)i + 1, {spans[i].first + half, G.sl.n - half});
            spans[i].second = half;
            --i;
        }
    }
    return true;
}

eslbm_status run_blocked2d(eslbm_handle *h)
{
    std::vector<Group2d> groups;
    int64_t after = 0;
    if (!step_groups2d(h, h->pending, groups, &after)) return run_ops(h);  // one launch per stage
    for (const Group2d &G : groups) {
        Step2dLaunch L;
        L.fin = h->f[h->cur];
        L.fout = h->f[1 - h->cur];
        L.nx = h->cfg.nx;
        L.ny = h->cfg.ny;
        L.ncell = h->sz.ncell;
        L.sl = G.sl;
        L.plan = G.plan;
        L.cnt = h->counters();
        L.P = launch_params(h, G.sl.n);
        L.stream = h->stream;
        CK(launch_step2d(h->family, h->fp64, h->om, L), "blocked 2D launch");
        h->cur = 1 - h->cur;
        h->relaxations += (uint64_t)h->sz.ncell * (uint64_t)G.sl.n;
        eslbm_status s = check_records(h, L.P);
        if (s != ESLBM_OK) return s;
    }
    h->pending = after;
    return ESLBM_OK;
}

// one unit of eslbm_step: a fused group of steps, or one step of per-stage launches
int64_t unit_steps(const eslbm_handle *h) { return fused_path(h) ? fused_group(h) : 1; }

eslbm_status run_unit(eslbm_handle *h, int64_t steps)
{
    if (fused_path(h)) return run_fused(h, steps);
    for (int64_t i = 0; i < steps; ++i) {
        eslbm_status s = blocked2d_path(h) ? run_blocked2d(h) : run_ops(h);
        if (s != ESLBM_OK) return s;
    }
    return ESLBM_OK;
}

// buffer swaps per unit from the current pending shift (the graph must return the ping-pong
// buffers to their start)
int64_t unit_swaps(const eslbm_handle *h)
{
    if (fused_path(h)) return 1;
    if (blocked2d_path(h)) {
        std::vector<Group2d> groups;
        int64_t after = 0;
        if (step_groups2d(h, h->pending, groups, &after)) return (int64_t)groups.size();
    }
    return h->sz.stages_per_step;
}

eslbm_status capture_graph(eslbm_handle *h)
{
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    const int64_t pend0 = h->pending;
    const int cur0 = h->cur;
    const uint64_t rel0 = h->relaxations;
    const int units = (unit_swaps(h) % 2 == 0) ? 1 : 2;
    const int nsteps = units * (int)unit_steps(h);
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    eslbm_status s = ESLBM_OK;
    for (int i = 0; i < units && s == ESLBM_OK; ++i) s = run_unit(h, unit_steps(h));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->graph_cur_after = h->cur;
    h->graph_pending_after = h->pending;
    h->pending = pend0;
    h->cur = cur0;
    h->relaxations = rel0;
    if (s != ESLBM_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    h->graph_pending = pend0;
    h->graph_cur = cur0;
    h->graph_steps = nsteps;
    return ESLBM_OK;
}

// ---- reverse mode -----------------------------------------------------------


struct GradLayout {
    int64_t n_outer, inner, stages;
    uint64_t stride, bytes;
};

GradLayout grad_layout(const eslbm_sizes &sz, int64_t n, int64_t K)
{
    GradLayout g;
    g.n_outer = n > 0 ? (n + K - 1) / K : 1;
    g.inner = std::min<int64_t>(K, std::max<int64_t>(n, 1));
    g.stages = sz.stages_per_step;
    g.stride = (sz.state_bytes + 255u) / 256u * 256u;
    g.bytes = g.stride * (uint64_t)(g.n_outer + g.inner + g.stages + 2);
    return g;
}

struct RecordedStage {
    const void *fin;
    int64_t shift;
    int kind;
};

eslbm_status stage_between(eslbm_handle *h, const void *fin, void *fout, int64_t shift, int kind)
{
    StageLaunch L;
    L.fin = fin;
    L.fout = fout;
    L.nx = h->cfg.nx;
    L.ny = h->cfg.ny;
    L.ncell = h->sz.ncell;
    L.sh = make_shift(h, shift);
    L.kind = kind;
    L.cnt = h->counters();
    L.P = h->P;
    L.stream = h->stream;
    CK(launch_stage(h->family, h->fp64, h->om, L), "stage launch");
    return ESLBM_OK;
}

}  // namespace

extern "C" {

int32_t eslbm_abi_version(void) { return ESLBM_ABI_VERSION; }

eslbm_status eslbm_gradient_workspace(const eslbm_config *cfg, int64_t n, int64_t K, uint64_t *bytes)
{
    if (!bytes || n < 0 || K < 1) return ESLBM_ERR_ARG;
    eslbm_sizes sz;
    eslbm_status s = eslbm_query(cfg, &sz);
    if (s != ESLBM_OK) return s;
    *bytes = grad_layout(sz, n, K).bytes;
    return ESLBM_OK;
}

eslbm_status eslbm_gradient(eslbm_handle *h, const double *u0, const double *dJ_duT, double *dJ_du0, int64_t n,
                            int64_t K, void *ws, uint64_t ws_bytes)
{
    if (!h || !u0 || !dJ_duT || !dJ_du0 || !ws || n < 0 || K < 1) return fail(h, ESLBM_ERR_ARG, "bad argument");
    const GradLayout G = grad_layout(h->sz, n, K);
    if (ws_bytes < G.bytes || ((uintptr_t)ws & 255u)) return fail(h, ESLBM_ERR_ARG, "gradient workspace too small");
    char *base = (char *)ws;
    auto outer = [&](int64_t i) { return (void *)(base + G.stride * (uint64_t)i); };
    auto inner = [&](int64_t i) { return (void *)(base + G.stride * (uint64_t)(G.n_outer + i)); };
    auto stage = [&](int64_t i) { return (void *)(base + G.stride * (uint64_t)(G.n_outer + G.inner + i)); };
    void *cot[2] = {base + G.stride * (uint64_t)(G.n_outer + G.inner + G.stages),
                    base + G.stride * (uint64_t)(G.n_outer + G.inner + G.stages + 1)};
    const size_t sb = (size_t)h->sz.state_bytes;

    // forward pass, checkpoint every K steps (physical state and its pending shift)
    eslbm_status s = eslbm_init_equilibrium(h, u0, 1);
    if (s != ESLBM_OK) return s;
    std::vector<int64_t> ck_pending((size_t)G.n_outer, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (i % K == 0) {
            CK(cudaMemcpyAsync(outer(i / K), h->f[h->cur], sb, cudaMemcpyDeviceToDevice, h->stream), "checkpoint");
            ck_pending[(size_t)(i / K)] = h->pending;
        }
        if ((s = run_unit(h, 1)) != ESLBM_OK) return s;  // the fused kernel where there is one
    }
    // cotangent of the final physical state from the cotangent of the moments
    int g = 0;
    CK(launch_adjoint_readout(h->cfg.dim, h->fp64, dJ_duT, cot[g], h->cfg.nx, h->cfg.ny, (int)h->sz.M,
                              make_shift(h, h->pending), h->stream),
       "adjoint readout");
    std::vector<int64_t> step_pending((size_t)G.inner, 0);
    std::vector<RecordedStage> rec;
    for (int64_t c = G.n_outer - 1; c >= 0 && n > 0; --c) {
        const int64_t s0 = c * K, s1 = std::min(n, s0 + K);
        // recompute the segment, keeping every step's starting state
        CK(cudaMemcpyAsync(h->f[h->cur], outer(c), sb, cudaMemcpyDeviceToDevice, h->stream), "restore");
        h->pending = ck_pending[(size_t)c];
        for (int64_t j = 0; j < s1 - s0; ++j) {
            CK(cudaMemcpyAsync(inner(j), h->f[h->cur], sb, cudaMemcpyDeviceToDevice, h->stream), "step state");
            step_pending[(size_t)j] = h->pending;
            if ((s = run_unit(h, 1)) != ESLBM_OK) return s;
        }
        for (int64_t j = s1 - s0 - 1; j >= 0; --j) {
            // recompute the step stage by stage, keeping every stage's input
            rec.clear();
            const void *in = inner(j);
            int64_t pend = step_pending[(size_t)j];
            if (fused_path(h)) {
                // one temporally blocked launch that also writes every stage's output but the last
                FusedLaunch L;
                L.sl.n = 0;
                L.sl.halo = 0;
                for (const Op &op : h->ops) {
                    if (!op.relax) {
                        pend += op.shift;
                        continue;
                    }
                    if (L.sl.n >= kMaxFusedStages || pend > (1 << 20) || pend < -(1 << 20))
                        return fail(h, ESLBM_ERR_ARG, "step cannot be fused");
                    rec.push_back({L.sl.n == 0 ? in : stage(L.sl.n - 1), pend, op.kind});
                    L.sl.shift[L.sl.n] = (int)pend;
                    L.sl.kind[L.sl.n] = op.kind;
                    L.sl.halo += (int)(pend < 0 ? -pend : pend);
                    L.sl.n += 1;
                    pend = 0;
                }
                L.fin = in;
                L.fout = stage(L.sl.n - 1);
                L.n = h->cfg.nx;
                L.cnt = h->counters();
                L.P = h->P;
                L.stream = h->stream;
                L.rec = stage(0);
                L.rec_stride_bytes = (int64_t)G.stride;
                L.nrec = L.sl.n - 1;
                CK(launch_fused1d(h->family, h->fp64, h->om, L), "recording step launch");
            } else {
                for (const Op &op : h->ops) {
                    if (!op.relax) {
                        pend += op.shift;
                        continue;
                    }
                    void *out = stage((int64_t)rec.size());
                    if ((s = stage_between(h, in, out, pend, op.kind)) != ESLBM_OK) return s;
                    rec.push_back({in, pend, op.kind});
                    in = out;
                    pend = 0;
                }
            }
            // reverse sweep of the stages: reverse shift and transposed relaxation Jacobian
            for (int64_t st = (int64_t)rec.size() - 1; st >= 0; --st) {
                AdjointLaunch A;
                A.fin = rec[(size_t)st].fin;
                A.gout = cot[g];
                A.gin = cot[1 - g];
                A.nx = h->cfg.nx;
                A.ny = h->cfg.ny;
                A.sh = make_shift(h, rec[(size_t)st].shift);
                A.kind = rec[(size_t)st].kind;
                A.P = h->P;
                A.stream = h->stream;
                CK(launch_adjoint_stage(h->family, h->fp64, h->om, A), "adjoint stage");
                g = 1 - g;
            }
        }
    }
    CK(launch_adjoint_init(h->family, h->fp64, u0, cot[g], dJ_du0, h->sz.ncell, h->P, h->stream), "adjoint init");
    // leave the handle on the final forward state
    h->pending = 0;
    s = eslbm_init_equilibrium(h, u0, 1);
    if (s != ESLBM_OK) return s;
    return eslbm_step(h, n);
}

const char *eslbm_status_string(eslbm_status s)
{
    switch (s) {
    case ESLBM_OK: return "ok";
    case ESLBM_ERR_ARG: return "invalid argument";
    case ESLBM_ERR_DOMAIN: return "outside the convexity / sub-characteristic domain";
    case ESLBM_ERR_CUDA: return "CUDA error";
    case ESLBM_ERR_NAN: return "non-finite values";
    case ESLBM_ERR_UNSUPPORTED: return "unsupported combination";
    case ESLBM_WARN_OMEGA_FALLBACK: return "entropic omega fell back to the projection in some cells";
    }
    return "unknown status";
}

eslbm_status eslbm_query(const eslbm_config *cfg, eslbm_sizes *out)
{
    if (!out) return ESLBM_ERR_ARG;
    eslbm_status s = validate(cfg);
    if (s != ESLBM_OK) return s;
    Params P;
    if ((s = params_of(*cfg, P)) != ESLBM_OK) return s;  // checks the reference state
    eslbm_sizes z;
    z.q = cfg->dim == 1 ? 2 : 4;
    z.M = num_M(*cfg);
    z.planes = z.q * z.M;
    z.ncell = cfg->nx * cfg->ny;
    z.state_bytes = (uint64_t)z.planes * (uint64_t)z.ncell * (cfg->precision == ESLBM_FP64 ? 8u : 4u);
    int64_t stages = 0;
    for (const Op &op : scheme_ops(cfg->scheme, cfg->kappa)) stages += op.relax ? 1 : 0;
    z.stages_per_step = stages;
    static_assert(kRecordsOffset == kCountersBytes + sizeof(double) * 6 * 1024 + 256, "workspace layout");
    z.workspace_bytes = kRecordsOffset;
    if (records_of(*cfg))  // diagnostics: one record of every relaxation of a launch
        z.workspace_bytes += (uint64_t)record_fields((int)z.q, (int)z.M) *
                             (uint64_t)max_launch_stages(*cfg, stages, z.planes) * (uint64_t)z.ncell *
                             (cfg->precision == ESLBM_FP64 ? 8u : 4u);
    z.step_cells = step_cells(cfg->scheme, cfg->kappa);
    z.launches_per_step = (double)stages;
    if (cfg->dim == 1 && cfg->blocking != ESLBM_BLOCKING_OFF) {
        z.launches_per_step = 1.0 / (double)fused_group_of(stages);
    } else if (blocked2d_of(*cfg, z.planes)) {
        eslbm_handle probe;  // the grouping needs the configuration, sizes and operator list
        probe.cfg = *cfg;
        probe.sz = z;
        probe.fp64 = cfg->precision == ESLBM_FP64;
        probe.family = family_of(*cfg);
        probe.om = omega_mode_of(*cfg);
        probe.ops = scheme_ops(cfg->scheme, cfg->kappa);
        int64_t pend = 0;
        for (const Op &op : probe.ops)  // the trailing shift that a step leaves pending
            pend = op.relax ? 0 : pend + op.shift;
        std::vector<Group2d> groups;
        int64_t after = 0;
        if (step_groups2d(&probe, pend, groups, &after)) z.launches_per_step = (double)groups.size();
    }
    *out = z;
    return ESLBM_OK;
}

eslbm_status eslbm_create(const eslbm_config *cfg, void *f_a, void *f_b, void *workspace, void *stream,
                          eslbm_handle **out)
{
    if (!out) return ESLBM_ERR_ARG;
    *out = nullptr;
    eslbm_sizes sz;
    eslbm_status s = eslbm_query(cfg, &sz);
    if (s != ESLBM_OK) return s;
    if (!f_a || !f_b || !workspace || f_a == f_b) return ESLBM_ERR_ARG;
    if (((uintptr_t)f_a | (uintptr_t)f_b | (uintptr_t)workspace) & 15u) return ESLBM_ERR_ARG;
    eslbm_handle *h = new (std::nothrow) eslbm_handle();
    if (!h) return ESLBM_ERR_ARG;
    h->cfg = *cfg;
    h->sz = sz;
    h->family = family_of(*cfg);
    h->fp64 = cfg->precision == ESLBM_FP64;
    h->om = omega_mode_of(*cfg);
    h->f[0] = f_a;
    h->f[1] = f_b;
    h->cur = 0;
    h->ws = (char *)workspace;
    h->stream = (cudaStream_t)stream;
    h->pending = 0;
    if ((s = params_of(*cfg, h->P)) != ESLBM_OK) {
        delete h;
        return s;
    }
    h->ops = scheme_ops(cfg->scheme, cfg->kappa);
    h->relaxations = 0;
    h->use_graph = false;
    h->gexec = nullptr;
    h->graph_steps = 0;
    s = eslbm_reset_diagnostics(h);
    if (s != ESLBM_OK) {
        delete h;
        return s;
    }
    *out = h;
    return ESLBM_OK;
}

eslbm_status eslbm_destroy(eslbm_handle *h)
{
    if (!h) return ESLBM_OK;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    delete h;
    return ESLBM_OK;
}

eslbm_status eslbm_set_stream(eslbm_handle *h, void *stream)
{
    if (!h) return ESLBM_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return ESLBM_OK;
}

const char *eslbm_last_error(const eslbm_handle *h) { return h ? h->err.c_str() : "null handle"; }

eslbm_status eslbm_init_equilibrium(eslbm_handle *h, const double *u0, int32_t u0_on_device)
{
    if (!h || !u0) return fail(h, ESLBM_ERR_ARG, "null argument");
    const size_t ubytes = sizeof(double) * (size_t)h->sz.M * (size_t)h->sz.ncell;
    const double *src = u0;
    if (!u0_on_device) {
        CK(cudaMemcpyAsync(h->spare(), u0, ubytes, cudaMemcpyHostToDevice, h->stream), "copy u0");
        src = (const double *)h->spare();
    }
    Counters *c = h->counters();
    CK(cudaMemsetAsync(&c->domain_violations, 0, 2 * sizeof(unsigned long long), h->stream), "clear flags");
    CK(launch_init_eq(h->family, h->fp64, src, h->f[h->cur], h->sz.ncell, h->P, c, h->stream), "init launch");
    unsigned long long flags[2];
    CK(cudaMemcpyAsync(flags, &c->domain_violations, sizeof(flags), cudaMemcpyDeviceToHost, h->stream),
       "read flags");
    CK(cudaStreamSynchronize(h->stream), "init sync");
    h->pending = 0;
    if (flags[1]) return fail(h, ESLBM_ERR_NAN, "non-finite initial data");
    if (flags[0]) {
        char buf[160];
        snprintf(buf, sizeof buf, "%llu cells violate the convexity / sub-characteristic condition", flags[0]);
        return fail(h, ESLBM_ERR_DOMAIN, buf);
    }
    return ESLBM_OK;
}

eslbm_status eslbm_init_distributions(eslbm_handle *h, const double *f0, int32_t on_device)
{
    if (!h || !f0) return fail(h, ESLBM_ERR_ARG, "null argument");
    Counters *c = h->counters();
    CK(cudaMemsetAsync(&c->non_finite, 0, sizeof(unsigned long long), h->stream), "clear flag");
    const int64_t n = h->sz.ncell;
    const size_t elem = h->fp64 ? 8 : 4;
    for (int64_t p = 0; p < h->sz.planes; ++p) {
        const double *src = f0 + p * n;
        if (!on_device) {
            CK(cudaMemcpyAsync(h->spare(), src, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->stream),
               "copy f0");
            src = (const double *)h->spare();
        }
        CK(launch_set(h->fp64, src, (char *)h->f[h->cur] + (size_t)p * (size_t)n * elem, n, h->P.fbar[p], c,
                      h->stream),
           "set");
    }
    unsigned long long nf = 0;
    CK(cudaMemcpyAsync(&nf, &c->non_finite, sizeof(nf), cudaMemcpyDeviceToHost, h->stream), "read flag");
    CK(cudaStreamSynchronize(h->stream), "sync");
    h->pending = 0;
    if (nf) return fail(h, ESLBM_ERR_NAN, "non-finite distributions");
    return ESLBM_OK;
}

eslbm_status eslbm_step(eslbm_handle *h, int64_t n)
{
    if (!h || n < 0) return fail(h, ESLBM_ERR_ARG, "bad step count");
    while (n > 0) {
        const bool graph_ok = h->use_graph && h->stream != nullptr;
        if (graph_ok) {
            const int64_t gsteps = ((unit_swaps(h) % 2 == 0) ? 1 : 2) * unit_steps(h);
            if (n >= gsteps) {
                if (!h->gexec || h->graph_pending != h->pending || h->graph_cur != h->cur) {
                    eslbm_status s = capture_graph(h);
                    if (s != ESLBM_OK) return s;
                }
                CK(cudaGraphLaunch(h->gexec, h->stream), "graph launch");
                h->cur = h->graph_cur_after;
                h->pending = h->graph_pending_after;
                h->relaxations += (uint64_t)h->sz.ncell * (uint64_t)(h->sz.stages_per_step * h->graph_steps);
                n -= h->graph_steps;
                continue;
            }
        }
        const int64_t k = std::min<int64_t>(n, unit_steps(h));
        eslbm_status s = run_unit(h, k);
        if (s != ESLBM_OK) return s;
        n -= k;
    }
    return ESLBM_OK;
}

eslbm_status eslbm_transport(eslbm_handle *h, int64_t s)
{
    if (!h) return ESLBM_ERR_ARG;
    h->pending += s;
    return ESLBM_OK;
}

eslbm_status eslbm_relax(eslbm_handle *h, int32_t kind)
{
    if (!h || (kind != ESLBM_RELAX_MAIN && kind != ESLBM_RELAX_PROJECT)) return fail(h, ESLBM_ERR_ARG, "bad kind");
    eslbm_status s = launch_one_stage(h, h->pending, kind == ESLBM_RELAX_PROJECT ? KIND_PROJECT : KIND_MAIN);
    if (s == ESLBM_OK) h->pending = 0;
    return s;
}

eslbm_status eslbm_read_moments(eslbm_handle *h, double *u_out, int32_t on_device)
{
    if (!h || !u_out) return fail(h, ESLBM_ERR_ARG, "null argument");
    double *dst = on_device ? u_out : (double *)h->spare();
    CK(launch_gather_moments(h->cfg.dim, h->fp64, h->f[h->cur], dst, h->cfg.nx, h->cfg.ny, (int)h->sz.M,
                             make_shift(h, h->pending), h->P.fbar, h->stream),
       "gather moments");
    if (!on_device) {
        CK(cudaMemcpyAsync(u_out, dst, sizeof(double) * (size_t)(h->sz.M * h->sz.ncell), cudaMemcpyDeviceToHost,
                           h->stream),
           "copy moments");
        CK(cudaStreamSynchronize(h->stream), "sync");
    }
    return ESLBM_OK;
}

eslbm_status eslbm_read_distributions(eslbm_handle *h, double *f_out, int32_t on_device)
{
    if (!h || !f_out) return fail(h, ESLBM_ERR_ARG, "null argument");
    const Shift sh = make_shift(h, h->pending);
    const int64_t n = h->sz.ncell;
    if (on_device) {
        CK(launch_gather_planes(h->cfg.dim, h->fp64, h->f[h->cur], f_out, h->cfg.nx, h->cfg.ny, (int)h->sz.M, 0,
                                (int)h->sz.planes, sh, h->P.fbar, h->stream),
           "gather planes");
        return ESLBM_OK;
    }
    // through the spare buffer, as many planes at a time as fit
    const int64_t per = std::max<int64_t>(1, (int64_t)(h->sz.state_bytes / (sizeof(double) * (uint64_t)n)));
    for (int64_t p = 0; p < h->sz.planes; p += per) {
        const int np = (int)std::min<int64_t>(per, h->sz.planes - p);
        CK(launch_gather_planes(h->cfg.dim, h->fp64, h->f[h->cur], (double *)h->spare(), h->cfg.nx, h->cfg.ny,
                                (int)h->sz.M, (int)p, np, sh, h->P.fbar, h->stream),
           "gather planes");
        CK(cudaMemcpyAsync(f_out + p * n, h->spare(), sizeof(double) * (size_t)(np * n), cudaMemcpyDeviceToHost,
                           h->stream),
           "copy planes");
    }
    CK(cudaStreamSynchronize(h->stream), "sync");
    return ESLBM_OK;
}

eslbm_status eslbm_read_totals(eslbm_handle *h, double *out, int32_t on_device)
{
    if (!h || !out) return fail(h, ESLBM_ERR_ARG, "null argument");
    double *dst = on_device ? out : h->totals_out();
    CK(launch_totals(h->family, h->fp64, h->f[h->cur], h->partials(), dst, h->cfg.nx, h->cfg.ny,
                     make_shift(h, h->pending), h->P, h->stream),
       "totals");
    if (!on_device) {
        CK(cudaMemcpyAsync(out, dst, sizeof(double) * (size_t)(2 + h->sz.M), cudaMemcpyDeviceToHost, h->stream),
           "copy totals");
        CK(cudaStreamSynchronize(h->stream), "sync");
    }
    return ESLBM_OK;
}

eslbm_status eslbm_get_diagnostics(eslbm_handle *h, eslbm_diagnostics *out)
{
    if (!h || !out) return fail(h, ESLBM_ERR_ARG, "null argument");
    Counters c;
    CK(cudaMemcpyAsync(&c, h->counters(), sizeof(c), cudaMemcpyDeviceToHost, h->stream), "read counters");
    CK(cudaStreamSynchronize(h->stream), "sync");
    out->relaxations = h->relaxations;
    out->fallbacks = c.fallbacks;
    out->entropy_increases = c.entropy_increases;
    float wmin, wmax;
    std::memcpy(&wmin, &c.omega_min_bits, sizeof(float));
    std::memcpy(&wmax, &c.omega_max_bits, sizeof(float));
    const bool seen = c.omega_min_bits != 0x7f800000u;
    out->omega_min = seen ? (double)wmin : NAN;
    out->omega_max = seen ? (double)wmax : NAN;
    float ex;
    std::memcpy(&ex, &c.excess_max_bits, sizeof(float));
    out->entropy_excess_max = (double)ex;
    if (c.copy_timeouts) return fail(h, ESLBM_ERR_CUDA, "a staged 2D stage gave up waiting for its bulk copies");
    return c.fallbacks ? ESLBM_WARN_OMEGA_FALLBACK : ESLBM_OK;
}

eslbm_status eslbm_reset_diagnostics(eslbm_handle *h)
{
    if (!h) return ESLBM_ERR_ARG;
    Counters c;
    std::memset(&c, 0, sizeof(c));
    c.omega_min_bits = 0x7f800000u;  // +inf
    c.omega_max_bits = 0u;
    static_assert(sizeof(Counters) <= kCountersBytes, "counters fit the reserved space");
    CK(cudaMemcpyAsync(h->counters(), &c, sizeof(c), cudaMemcpyHostToDevice, h->stream), "reset counters");
    CK(cudaStreamSynchronize(h->stream), "sync");
    h->relaxations = 0;
    return ESLBM_OK;
}

eslbm_status eslbm_use_graph(eslbm_handle *h, int32_t enable)
{
    if (!h) return ESLBM_ERR_ARG;
    h->use_graph = enable != 0;
    if (!h->use_graph && h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return ESLBM_OK;
}

}  // extern "C"
