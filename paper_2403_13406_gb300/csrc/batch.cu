// batch.cu -- C ABI of batched execution: many independent 2D lattices of
// uneven sizes advance together, one cooperative launch per composite step
// (all stages, grid.sync between them), optionally replayed from a CUDA graph.
// The work list (row segments of every instance) and the grid size come from a
// schedule that eslbm_batch_tune picks by timing candidates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/eslbm.h"
#include "host_schedule.h"
#include "launch.h"

using namespace eslbm;

namespace {

constexpr size_t kCounters = 256;
constexpr int64_t kMinSegment = 128;

uint64_t align256(uint64_t b) { return (b + 255u) / 256u * 256u; }

struct Layout {
    int64_t q, M, planes, total_cells, max_items;
    uint64_t elem, pool_bytes, inst_off, items_off, handle_ws_off, handle_ws_bytes, rec_off, ws_bytes;
    std::vector<BatchInstance> inst;
};

eslbm_status layout(const eslbm_config *base, int32_t count, const int64_t *nx, const int64_t *ny, Layout &L)
{
    if (!base || count < 1 || count > (1 << 20) || !nx || !ny) return ESLBM_ERR_ARG;
    if (base->dim != 2) return ESLBM_ERR_UNSUPPORTED;
    L.inst.resize((size_t)count);
    L.total_cells = 0;
    L.max_items = 0;
    uint64_t off = 0, handle_ws = 0;
    eslbm_sizes sz{};
    for (int32_t i = 0; i < count; ++i) {
        eslbm_config c = *base;
        c.nx = nx[i];
        c.ny = ny[i];
        eslbm_status s = eslbm_query(&c, &sz);  // validates every instance
        if (s != ESLBM_OK) return s;
        if (nx[i] > INT32_MAX) return ESLBM_ERR_ARG;  // work items hold 32-bit columns
        L.elem = base->precision == ESLBM_FP64 ? 8 : 4;
        L.inst[(size_t)i] = {nx[i], ny[i], (int64_t)(off / L.elem), L.total_cells};
        off += align256(sz.state_bytes);
        handle_ws = std::max<uint64_t>(handle_ws, sz.workspace_bytes);
        L.total_cells += sz.ncell;
        L.max_items += ny[i] * ((nx[i] + kMinSegment - 1) / kMinSegment);
    }
    if (L.max_items > (int64_t(1) << 31) - 1) return ESLBM_ERR_ARG;
    L.q = sz.q;
    L.M = sz.M;
    L.planes = sz.planes;
    L.pool_bytes = off;
    L.inst_off = kCounters;
    L.items_off = L.inst_off + align256(sizeof(BatchInstance) * (uint64_t)count);
    L.handle_ws_off = L.items_off + align256(sizeof(BatchItem) * (uint64_t)L.max_items);
    L.handle_ws_bytes = align256(handle_ws);
    L.rec_off = L.handle_ws_off + L.handle_ws_bytes;
    L.ws_bytes = L.rec_off;
    if (records_of(*base))  // diagnostics: one record of every relaxation of a step of every instance
        L.ws_bytes += (uint64_t)record_fields((int)L.q, (int)L.M) * (uint64_t)sz.stages_per_step *
                      (uint64_t)L.total_cells * L.elem;
    return ESLBM_OK;
}

}  // namespace

struct eslbm_batch {
    eslbm_config cfg;
    int32_t count;
    Layout L;
    int family;
    bool fp64;
    int om;  // OmegaMode
    void *pool[2];
    int side;
    char *ws;
    cudaStream_t stream;
    int64_t pending;
    Params P;
    std::vector<Op> ops;
    // schedule
    int64_t segment;
    int32_t blocks_per_sm, order;
    int n_items;
    int sms, max_bps;
    // graphs of `steps` consecutive steps entered on (side, pending): a small cache, as the
    // first step from pending = 0 enters differently from the later ones
    struct Graph {
        cudaGraphExec_t exec;
        int side;
        int64_t pending, steps;
    };
    bool use_graph;
    std::vector<Graph> graphs;
    std::string err;

    Counters *counters() { return reinterpret_cast<Counters *>(ws); }
    BatchInstance *d_inst() { return reinterpret_cast<BatchInstance *>(ws + L.inst_off); }
    BatchItem *d_items() { return reinterpret_cast<BatchItem *>(ws + L.items_off); }
    char *instance_ptr(int side_, int32_t i) { return (char *)pool[side_] + L.inst[(size_t)i].offset * L.elem; }
};

namespace {

#define BCK(call, where)                                                            \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            b->err = std::string(where) + ": " + cudaGetErrorString(e_);            \
            return ESLBM_ERR_CUDA;                                                  \
        }                                                                           \
    } while (0)

Shift shift_for(const eslbm_batch *b, int32_t i, int64_t s)
{
    Shift sh;
    for (int k = 0; k < 4; ++k) {
        const int axis = k & 1, sign = k < 2 ? 1 : -1;
        const int64_t n = axis == 0 ? b->L.inst[(size_t)i].nx : b->L.inst[(size_t)i].ny;
        int64_t r = (-(int64_t)sign * s) % n;
        sh.roff[k] = r < 0 ? r + n : r;
    }
    return sh;
}

void drop_graphs(eslbm_batch *b)
{
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

// Work list of the schedule: row segments of at most `segment` cells; order 0 walks the
// instances one after the other, order 1 interleaves rows of all instances round robin.
eslbm_status upload_schedule(eslbm_batch *b)
{
    std::vector<BatchItem> items;
    items.reserve((size_t)b->L.max_items);
    if (b->order == 0) {
        for (int32_t i = 0; i < b->count; ++i)
            for (int64_t y = 0; y < b->L.inst[(size_t)i].ny; ++y)
                for (int64_t x0 = 0; x0 < b->L.inst[(size_t)i].nx; x0 += b->segment)
                    items.push_back({i, (int32_t)y, (int32_t)x0,
                                     (int32_t)std::min<int64_t>(b->segment, b->L.inst[(size_t)i].nx - x0)});
    } else {
        int64_t ymax = 0;
        for (const BatchInstance &I : b->L.inst) ymax = std::max(ymax, I.ny);
        for (int64_t y = 0; y < ymax; ++y)
            for (int32_t i = 0; i < b->count; ++i) {
                if (y >= b->L.inst[(size_t)i].ny) continue;
                for (int64_t x0 = 0; x0 < b->L.inst[(size_t)i].nx; x0 += b->segment)
                    items.push_back({i, (int32_t)y, (int32_t)x0,
                                     (int32_t)std::min<int64_t>(b->segment, b->L.inst[(size_t)i].nx - x0)});
            }
    }
    if ((int64_t)items.size() > b->L.max_items) return ESLBM_ERR_ARG;
    b->n_items = (int)items.size();
    BCK(cudaMemcpyAsync(b->d_items(), items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                        b->stream),
        "upload work list");
    BCK(cudaStreamSynchronize(b->stream), "sync");
    drop_graphs(b);
    return ESLBM_OK;
}

eslbm_status run_step(eslbm_batch *b)
{
    BatchLaunch B;
    B.sl.n = 0;
    B.sl.halo = 0;
    for (const Op &op : b->ops) {
        if (!op.relax) {
            b->pending += op.shift;
            continue;
        }
        B.sl.shift[B.sl.n] = (int)b->pending;
        B.sl.kind[B.sl.n] = op.kind;
        B.sl.n += 1;
        b->pending = 0;
    }
    B.pool[0] = b->pool[0];
    B.pool[1] = b->pool[1];
    B.inst = b->d_inst();
    B.items = b->d_items();
    B.n_items = b->n_items;
    B.side = b->side;
    B.cnt = b->counters();
    B.P = b->P;
    if (records_of(b->cfg)) {  // diagnostics: record every relaxation, then check the records
        B.P.rec = (uint64_t)(uintptr_t)(b->ws + b->L.rec_off);
        B.P.rec_cells = b->L.total_cells;
        B.P.rec_stages = B.sl.n;
    }
    B.grid = std::max(1, std::min(b->n_items, b->sms * b->blocks_per_sm));
    B.stream = b->stream;
    BCK(launch_batch_step(b->family, b->fp64, b->om, B), "batch step launch");
    if (B.sl.n & 1) b->side ^= 1;
    if (B.P.rec) BCK(launch_check(b->family, b->fp64, b->om, B.P, b->counters(), b->stream), "entropy check");
    return ESLBM_OK;
}

constexpr int64_t kGraphSteps = 256;  // steps per captured graph
constexpr size_t kGraphCache = 4;

// Capture `steps` steps from the current (side, pending) and return the graph;
// the host bookkeeping ends where the replay will leave it.
eslbm_status capture(eslbm_batch *b, int64_t steps, cudaGraphExec_t *out)
{
    if (b->graphs.size() >= kGraphCache) drop_graphs(b);
    const int side0 = b->side;
    const int64_t pend0 = b->pending;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    eslbm_status s = ESLBM_OK;
    for (int64_t i = 0; i < steps && s == ESLBM_OK; ++i) s = run_step(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s != ESLBM_OK) {
        if (g) cudaGraphDestroy(g);
        b->side = side0;
        b->pending = pend0;
        return s;
    }
    BCK(e, "end capture");
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    b->side = side0;  // the caller replays and advances the bookkeeping
    b->pending = pend0;
    BCK(e, "graph instantiate");
    b->graphs.push_back({x, side0, pend0, steps});
    *out = x;
    return ESLBM_OK;
}

}  // namespace

extern "C" {

eslbm_status eslbm_batch_query(const eslbm_config *base, int32_t count, const int64_t *nx, const int64_t *ny,
                               eslbm_batch_sizes *out)
{
    if (!out) return ESLBM_ERR_ARG;
    Layout L;
    eslbm_status s = layout(base, count, nx, ny, L);
    if (s != ESLBM_OK) return s;
    out->count = count;
    out->q = L.q;
    out->M = L.M;
    out->planes = L.planes;
    out->total_cells = L.total_cells;
    out->pool_bytes = L.pool_bytes;
    out->workspace_bytes = L.ws_bytes;
    int64_t stages = 0;
    for (const Op &op : scheme_ops(base->scheme, base->kappa)) stages += op.relax ? 1 : 0;
    out->stages_per_step = stages;
    out->step_cells = step_cells(base->scheme, base->kappa);
    return ESLBM_OK;
}

eslbm_status eslbm_batch_create(const eslbm_config *base, int32_t count, const int64_t *nx, const int64_t *ny,
                                void *pool_a, void *pool_b, void *workspace, void *stream, eslbm_batch **out)
{
    if (!out) return ESLBM_ERR_ARG;
    *out = nullptr;
    Layout L;
    eslbm_status s = layout(base, count, nx, ny, L);
    if (s != ESLBM_OK) return s;
    if (!pool_a || !pool_b || !workspace || pool_a == pool_b) return ESLBM_ERR_ARG;
    if (((uintptr_t)pool_a | (uintptr_t)pool_b | (uintptr_t)workspace) & 255u) return ESLBM_ERR_ARG;
    eslbm_batch *b = new (std::nothrow) eslbm_batch();
    if (!b) return ESLBM_ERR_ARG;
    b->cfg = *base;
    b->count = count;
    b->L = L;
    b->family = family_of(*base);
    b->fp64 = base->precision == ESLBM_FP64;
    b->om = omega_mode_of(*base);
    b->pool[0] = pool_a;
    b->pool[1] = pool_b;
    b->side = 0;
    b->ws = (char *)workspace;
    b->stream = (cudaStream_t)stream;
    b->pending = 0;
    if ((s = params_of(*base, b->P)) != ESLBM_OK) {
        delete b;
        return s;
    }
    b->ops = scheme_ops(base->scheme, base->kappa);
    b->use_graph = false;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->max_bps = batch_blocks_per_sm(b->family, b->fp64, b->om);
    if (b->sms < 1 || b->max_bps < 1) {
        delete b;
        return ESLBM_ERR_CUDA;
    }
    b->segment = 256;
    b->blocks_per_sm = b->max_bps;
    b->order = 0;
    Counters c;
    std::memset(&c, 0, sizeof(c));
    c.omega_min_bits = 0x7f800000u;
    if (cudaMemcpyAsync(b->counters(), &c, sizeof(c), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d_inst(), L.inst.data(), sizeof(BatchInstance) * L.inst.size(), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess) {
        delete b;
        return ESLBM_ERR_CUDA;
    }
    s = upload_schedule(b);
    if (s != ESLBM_OK) {
        delete b;
        return s;
    }
    *out = b;
    return ESLBM_OK;
}

eslbm_status eslbm_batch_destroy(eslbm_batch *b)
{
    if (!b) return ESLBM_OK;
    drop_graphs(b);
    delete b;
    return ESLBM_OK;
}

const char *eslbm_batch_last_error(const eslbm_batch *b) { return b ? b->err.c_str() : "null batch"; }

eslbm_status eslbm_batch_init_equilibrium(eslbm_batch *b, const double *u0, int32_t on_device)
{
    if (!b || !u0) return ESLBM_ERR_ARG;
    const size_t ubytes = sizeof(double) * (size_t)b->L.M * (size_t)b->L.total_cells;
    const double *src = u0;
    if (!on_device) {  // stage through the spare pool (it holds at least M doubles per cell)
        if (ubytes > b->L.pool_bytes) return ESLBM_ERR_ARG;
        BCK(cudaMemcpyAsync(b->pool[1 - b->side], u0, ubytes, cudaMemcpyHostToDevice, b->stream), "copy u0");
        src = (const double *)b->pool[1 - b->side];
    }
    Counters *c = b->counters();
    BCK(cudaMemsetAsync(&c->domain_violations, 0, 2 * sizeof(unsigned long long), b->stream), "clear flags");
    int64_t cell0 = 0;
    for (int32_t i = 0; i < b->count; ++i) {
        const int64_t n = b->L.inst[(size_t)i].nx * b->L.inst[(size_t)i].ny;
        BCK(launch_init_eq(b->family, b->fp64, src + cell0 * b->L.M, b->instance_ptr(b->side, i), n, b->P, c,
                           b->stream),
            "init launch");
        cell0 += n;
    }
    unsigned long long flags[2];
    BCK(cudaMemcpyAsync(flags, &c->domain_violations, sizeof(flags), cudaMemcpyDeviceToHost, b->stream), "flags");
    BCK(cudaStreamSynchronize(b->stream), "sync");
    b->pending = 0;
    if (flags[1]) return ESLBM_ERR_NAN;
    if (flags[0]) return ESLBM_ERR_DOMAIN;
    return ESLBM_OK;
}

eslbm_status eslbm_batch_step(eslbm_batch *b, int64_t n)
{
    if (!b || n < 0) return ESLBM_ERR_ARG;
    if (b->use_graph && b->stream != nullptr) {
        while (n > 0) {
            const int64_t c = std::min(n, kGraphSteps);
            cudaGraphExec_t x = nullptr;
            for (const auto &g : b->graphs)
                if (g.side == b->side && g.pending == b->pending && g.steps == c) x = g.exec;
            if (!x) {
                eslbm_status s = capture(b, c, &x);
                if (s != ESLBM_OK) return s;
            }
            BCK(cudaGraphLaunch(x, b->stream), "graph launch");
            // advance the host bookkeeping by c steps without launching
            for (int64_t i = 0; i < c; ++i) {
                int stages = 0;
                for (const Op &op : b->ops) {
                    if (!op.relax) b->pending += op.shift;
                    else {
                        b->pending = 0;
                        ++stages;
                    }
                }
                if (stages & 1) b->side ^= 1;
            }
            n -= c;
        }
        return ESLBM_OK;
    }
    for (int64_t i = 0; i < n; ++i) {
        eslbm_status s = run_step(b);
        if (s != ESLBM_OK) return s;
    }
    return ESLBM_OK;
}

eslbm_status eslbm_batch_read_moments(eslbm_batch *b, double *u_out, int32_t on_device)
{
    if (!b || !u_out) return ESLBM_ERR_ARG;
    const size_t ubytes = sizeof(double) * (size_t)b->L.M * (size_t)b->L.total_cells;
    double *dst = u_out;
    if (!on_device) {
        if (ubytes > b->L.pool_bytes) return ESLBM_ERR_ARG;
        dst = (double *)b->pool[1 - b->side];
    }
    int64_t cell0 = 0;
    for (int32_t i = 0; i < b->count; ++i) {
        const BatchInstance &I = b->L.inst[(size_t)i];
        BCK(launch_gather_moments(2, b->fp64, b->instance_ptr(b->side, i), dst + cell0 * b->L.M, I.nx, I.ny,
                                  (int)b->L.M, shift_for(b, i, b->pending), b->P.fbar, b->stream),
            "gather moments");
        cell0 += I.nx * I.ny;
    }
    if (!on_device) {
        BCK(cudaMemcpyAsync(u_out, dst, ubytes, cudaMemcpyDeviceToHost, b->stream), "copy moments");
        BCK(cudaStreamSynchronize(b->stream), "sync");
    }
    return ESLBM_OK;
}

eslbm_status eslbm_batch_set_schedule(eslbm_batch *b, int64_t segment, int32_t blocks_per_sm, int32_t order)
{
    if (!b || segment < kMinSegment || segment > (1 << 20) || (order != 0 && order != 1)) return ESLBM_ERR_ARG;
    if (blocks_per_sm < 1 || blocks_per_sm > b->max_bps) return ESLBM_ERR_ARG;
    b->segment = segment;
    b->blocks_per_sm = blocks_per_sm;
    b->order = order;
    return upload_schedule(b);
}

eslbm_status eslbm_batch_get_schedule(const eslbm_batch *b, int64_t *segment, int32_t *blocks_per_sm, int32_t *order)
{
    if (!b || !segment || !blocks_per_sm || !order) return ESLBM_ERR_ARG;
    *segment = b->segment;
    *blocks_per_sm = b->blocks_per_sm;
    *order = b->order;
    return ESLBM_OK;
}

eslbm_status eslbm_batch_tune(eslbm_batch *b, void *scratch, uint64_t scratch_bytes, int32_t steps)
{
    if (!b || !scratch || steps < 1 || scratch_bytes < b->L.pool_bytes) return ESLBM_ERR_ARG;
    // keep the state: every candidate starts from it and it is restored at the end
    const int side0 = b->side;
    const int64_t pend0 = b->pending;
    BCK(cudaMemcpyAsync(scratch, b->pool[side0], b->L.pool_bytes, cudaMemcpyDeviceToDevice, b->stream), "save");
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    const int64_t segs[] = {128, 256, 512, 1024};
    int bps_opts[3] = {b->max_bps, std::max(1, b->max_bps / 2), 1};
    float best = 1e30f;
    int64_t best_seg = b->segment;
    int32_t best_bps = b->blocks_per_sm, best_order = b->order;
    const bool graph = b->use_graph;
    b->use_graph = false;
    eslbm_status s = ESLBM_OK;
    for (int64_t seg : segs) {
        for (int bi = 0; bi < 3 && s == ESLBM_OK; ++bi) {
            if (bi > 0 && bps_opts[bi] == bps_opts[bi - 1]) continue;
            for (int32_t order = 0; order < 2 && s == ESLBM_OK; ++order) {
                b->segment = seg;
                b->blocks_per_sm = bps_opts[bi];
                b->order = order;
                if ((s = upload_schedule(b)) != ESLBM_OK) break;
                BCK(cudaMemcpyAsync(b->pool[side0], scratch, b->L.pool_bytes, cudaMemcpyDeviceToDevice, b->stream),
                    "restore");
                b->side = side0;
                b->pending = pend0;
                if ((s = run_step(b)) != ESLBM_OK) break;  // warm-up
                BCK(cudaEventRecord(e0, b->stream), "record");
                for (int32_t i = 0; i < steps && s == ESLBM_OK; ++i) s = run_step(b);
                BCK(cudaEventRecord(e1, b->stream), "record");
                BCK(cudaEventSynchronize(e1), "sync");
                float ms = 0.f;
                BCK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
                if (ms < best) {
                    best = ms;
                    best_seg = seg;
                    best_bps = bps_opts[bi];
                    best_order = order;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->use_graph = graph;
    BCK(cudaMemcpyAsync(b->pool[side0], scratch, b->L.pool_bytes, cudaMemcpyDeviceToDevice, b->stream), "restore");
    b->side = side0;
    b->pending = pend0;
    if (s != ESLBM_OK) return s;
    b->segment = best_seg;
    b->blocks_per_sm = best_bps;
    b->order = best_order;
    return upload_schedule(b);
}

eslbm_status eslbm_batch_use_graph(eslbm_batch *b, int32_t enable)
{
    if (!b) return ESLBM_ERR_ARG;
    b->use_graph = enable != 0;
    if (!b->use_graph) drop_graphs(b);
    return ESLBM_OK;
}

}  // extern "C"

namespace {

// Workspace of the batched reverse mode, in pools (each the size of a state pool): the checkpoints
// of the forward pass every K steps, the starting states of the steps of one segment, the outputs of
// the stages of one step, and two cotangent pools.
struct BatchGradLayout {
    int64_t n_outer, inner, stages;
    uint64_t stride, bytes;
};

BatchGradLayout batch_grad_layout(const Layout &L, int64_t stages_per_step, int64_t n, int64_t K)
{
    BatchGradLayout g;
    g.n_outer = n > 0 ? (n + K - 1) / K : 1;
    g.inner = std::min<int64_t>(K, std::max<int64_t>(n, 1));
    g.stages = stages_per_step;
    g.stride = align256(L.pool_bytes);
    g.bytes = g.stride * (uint64_t)(g.n_outer + g.inner + g.stages + 2);
    return g;
}

int64_t batch_stages_per_step(const eslbm_config *base)
{
    int64_t n = 0;
    for (const Op &op : scheme_ops(base->scheme, base->kappa)) n += op.relax ? 1 : 0;
    return n;
}

// the stage list of one step entered with pending shift `pending` (merged transports), which is
// advanced to the step's trailing shift
StageList step_stage_list(const eslbm_batch *b, int64_t &pending)
{
    StageList sl;
    sl.n = 0;
    sl.halo = 0;
    for (const Op &op : b->ops) {
        if (!op.relax) {
            pending += op.shift;
            continue;
        }
        sl.shift[sl.n] = (int)pending;
        sl.kind[sl.n] = op.kind;
        sl.halo += (int)(pending < 0 ? -pending : pending);
        sl.n += 1;
        pending = 0;
    }
    return sl;
}

}  // namespace

extern "C" {

eslbm_status eslbm_batch_gradient_workspace(const eslbm_config *base, int32_t count, const int64_t *nx,
                                            const int64_t *ny, int64_t n, int64_t K, uint64_t *bytes)
{
    if (!bytes || n < 0 || K < 1) return ESLBM_ERR_ARG;
    Layout L;
    eslbm_status s = layout(base, count, nx, ny, L);
    if (s != ESLBM_OK) return s;
    *bytes = batch_grad_layout(L, batch_stages_per_step(base), n, K).bytes;
    return ESLBM_OK;
}

eslbm_status eslbm_batch_gradient(eslbm_batch *b, const double *u0, const double *dJ_duT, double *dJ_du0, int64_t n,
                                  int64_t K, void *ws, uint64_t ws_bytes)
{
    if (!b || !u0 || !dJ_duT || !dJ_du0 || !ws || n < 0 || K < 1) return ESLBM_ERR_ARG;
    const BatchGradLayout G = batch_grad_layout(b->L, batch_stages_per_step(&b->cfg), n, K);
    if (ws_bytes < G.bytes || ((uintptr_t)ws & 255u)) {
        b->err = "gradient workspace too small";
        return ESLBM_ERR_ARG;
    }
    char *base = (char *)ws;
    auto pool_at = [&](int64_t i) { return (void *)(base + G.stride * (uint64_t)i); };
    auto outer = [&](int64_t i) { return pool_at(i); };
    auto inner = [&](int64_t i) { return pool_at(G.n_outer + i); };
    auto stage = [&](int64_t i) { return pool_at(G.n_outer + G.inner + i); };
    void *cot[2] = {pool_at(G.n_outer + G.inner + G.stages), pool_at(G.n_outer + G.inner + G.stages + 1)};
    const size_t pb = (size_t)b->L.pool_bytes;
    const int64_t pool_elems = (int64_t)(G.stride / b->L.elem);
    auto inst_at = [&](void *pool, int32_t i) { return (void *)((char *)pool + b->L.inst[(size_t)i].offset * b->L.elem); };
    const int adj_bps = batch_adjoint_blocks_per_sm(b->family, b->fp64, b->om);
    if (adj_bps < 1) return ESLBM_ERR_CUDA;

    // forward pass with a checkpoint of every instance every K steps
    eslbm_status s = eslbm_batch_init_equilibrium(b, u0, 1);
    if (s != ESLBM_OK) return s;
    std::vector<int64_t> ck_pending((size_t)G.n_outer, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (i % K == 0) {
            BCK(cudaMemcpyAsync(outer(i / K), b->pool[b->side], pb, cudaMemcpyDeviceToDevice, b->stream), "checkpoint");
            ck_pending[(size_t)(i / K)] = b->pending;
        }
        if ((s = run_step(b)) != ESLBM_OK) return s;
    }
    // cotangent of the final distributions from the cotangent of the moments (pending shift applied)
    int64_t cell0 = 0;
    for (int32_t i = 0; i < b->count; ++i) {
        const BatchInstance &I = b->L.inst[(size_t)i];
        BCK(launch_adjoint_readout(2, b->fp64, dJ_duT + cell0 * b->L.M, inst_at(cot[0], i), I.nx, I.ny, (int)b->L.M,
                                   shift_for(b, i, b->pending), b->stream),
            "adjoint readout");
        cell0 += I.nx * I.ny;
    }
    int g = 0;
    std::vector<int64_t> step_pending((size_t)G.inner, 0);
    for (int64_t c = G.n_outer - 1; c >= 0 && n > 0; --c) {
        const int64_t s0 = c * K, s1 = std::min(n, s0 + K);
        // recompute the segment from its checkpoint, keeping every step's starting state
        BCK(cudaMemcpyAsync(b->pool[0], outer(c), pb, cudaMemcpyDeviceToDevice, b->stream), "restore");
        b->side = 0;
        b->pending = ck_pending[(size_t)c];
        for (int64_t j = 0; j < s1 - s0; ++j) {
            BCK(cudaMemcpyAsync(inner(j), b->pool[b->side], pb, cudaMemcpyDeviceToDevice, b->stream), "step state");
            step_pending[(size_t)j] = b->pending;
            if ((s = run_step(b)) != ESLBM_OK) return s;
        }
        for (int64_t j = s1 - s0 - 1; j >= 0; --j) {
            int64_t pend = step_pending[(size_t)j];
            const StageList sl = step_stage_list(b, pend);
            // the step again, one cooperative launch that keeps every stage's output
            BatchLaunch B;
            B.pool[0] = inner(j);
            B.pool[1] = stage(0);
            B.inst = b->d_inst();
            B.items = b->d_items();
            B.n_items = b->n_items;
            B.side = 0;
            B.cnt = b->counters();
            B.sl = sl;
            B.P = b->P;
            B.grid = std::max(1, std::min(b->n_items, b->sms * b->blocks_per_sm));
            B.stream = b->stream;
            B.rec = stage(0);
            B.pool_elems = pool_elems;
            BCK(launch_batch_step(b->family, b->fp64, b->om, B), "recording step launch");
            // its adjoint stages in reverse, one cooperative launch
            BatchAdjointLaunch A;
            A.step_in = inner(j);
            A.rec = stage(0);
            A.pool_elems = pool_elems;
            A.cot[0] = cot[0];
            A.cot[1] = cot[1];
            A.side = g;
            A.inst = b->d_inst();
            A.items = b->d_items();
            A.n_items = b->n_items;
            A.sl = sl;
            A.P = b->P;
            A.grid = std::max(1, std::min(b->n_items, b->sms * adj_bps));
            A.stream = b->stream;
            BCK(launch_batch_adjoint_step(b->family, b->fp64, b->om, A), "adjoint step launch");
            if (sl.n & 1) g ^= 1;
        }
    }
    // dJ/du0 = sum_k E_k(u0)^T g_k for f_0 = f^eq(u0)
    cell0 = 0;
    for (int32_t i = 0; i < b->count; ++i) {
        const BatchInstance &I = b->L.inst[(size_t)i];
        const int64_t off = cell0 * b->L.M;
        BCK(launch_adjoint_init(b->family, b->fp64, u0 + off, inst_at(cot[g], i), dJ_du0 + off, I.nx * I.ny, b->P,
                                b->stream),
            "adjoint init");
        cell0 += I.nx * I.ny;
    }
    // the pools now hold other states: start again from u0 on the next step
    b->side = 0;
    return eslbm_batch_init_equilibrium(b, u0, 1);
}

eslbm_status eslbm_batch_get_diagnostics(eslbm_batch *b, eslbm_diagnostics *out)
{
    if (!b || !out) return ESLBM_ERR_ARG;
    Counters c;
    BCK(cudaMemcpyAsync(&c, b->counters(), sizeof(c), cudaMemcpyDeviceToHost, b->stream), "counters");
    BCK(cudaStreamSynchronize(b->stream), "sync");
    std::memset(out, 0, sizeof(*out));
    out->fallbacks = c.fallbacks;
    out->entropy_increases = c.entropy_increases;
    float wmin, wmax, ex;
    std::memcpy(&wmin, &c.omega_min_bits, sizeof(float));
    std::memcpy(&wmax, &c.omega_max_bits, sizeof(float));
    std::memcpy(&ex, &c.excess_max_bits, sizeof(float));
    const bool seen = c.omega_min_bits != 0x7f800000u;
    out->omega_min = seen ? (double)wmin : NAN;
    out->omega_max = seen ? (double)wmax : NAN;
    out->entropy_excess_max = (double)ex;
    return c.fallbacks ? ESLBM_WARN_OMEGA_FALLBACK : ESLBM_OK;
}

}  // extern "C"
