// noalloc.cu -- totals of a caller-held state without any allocation.
//
// eslbm_read_totals needs a handle, and a handle needs a workspace that the
// caller allocates.  Some callers cannot allocate device memory at the point
// where they want the totals: code that runs while a CUDA graph is being
// captured (allocation calls are not allowed there), hosts that hand the
// library a fixed, pre-sized pool and forbid further cudaMalloc, and plug-ins
// that only borrow another framework's state buffer.  This entry point serves
// them: its scratch (the per-block partial sums of the two-pass reduction and
// the final totals) lives in a file-scope __device__ array that every device
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/eslbm.h"
#include "host_schedule.h"
#include "launch.h"

using namespace eslbm;

namespace {

// up to 8 totals (2 + M with M <= 6) for each of the fixed reduction blocks,
// then the 8 final totals: 8 * 1024 + 8 doubles = 64.06 KiB
constexpr int kMaxTotals = 8;
constexpr int kScratchDoubles = kMaxTotals * 1024 + kMaxTotals;

static __device__ __align__(256) double g_totals_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (set-up once per device).
// The address is cached for the life of the process: it is not looked up again
// after cudaDeviceReset or any other teardown of the device's primary context.
eslbm_status scratch_for_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ESLBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_totals_scratch) != cudaSuccess || !p) return ESLBM_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return ESLBM_OK;
}


}  // namespace

extern "C" eslbm_status eslbm_read_totals_noalloc(const eslbm_config *cfg, const void *f, int64_t pending_shift,
                                                  double *out, int32_t out_on_device, void *stream)
{
    eslbm_sizes sz;
    eslbm_status s = eslbm_query(cfg, &sz);
    if (s != ESLBM_OK) return s;
    if (!f || !out || ((uintptr_t)f & 15u)) return ESLBM_ERR_ARG;
    const int nv = 2 + (int)sz.M;
    if (nv > kMaxTotals || totals_blocks() * kMaxTotals + kMaxTotals > kScratchDoubles) return ESLBM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!out_on_device) {
        // the host copy ends with a stream synchronization, which stream capture forbids
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            (void)cudaGetLastError();  // leave no error behind for later launches
            return ESLBM_ERR_ARG;
        }
        if (cs != cudaStreamCaptureStatusNone) return ESLBM_ERR_ARG;
    }
    double *scratch = nullptr;
    s = scratch_for_current_device(&scratch);
    if (s != ESLBM_OK) return s;

    Params P;
    if ((s = params_of(*cfg, P)) != ESLBM_OK) return s;  // the reference of the shifted storage
    // pull offsets of T(pending_shift): population k at x reads x - sign_k * shift
    Shift sh;
    for (int k = 0; k < 4; ++k) sh.roff[k] = 0;
    for (int k = 0; k < (int)sz.q; ++k) {
        const int axis = cfg->dim == 1 ? 0 : (k & 1);
        const int sign = cfg->dim == 1 ? (k == 0 ? 1 : -1) : (k < 2 ? 1 : -1);
        const int64_t n = axis == 0 ? cfg->nx : cfg->ny;
        int64_t r = (-(int64_t)sign * pending_shift) % n;
        if (r < 0) r += n;
        sh.roff[k] = r;
    }
    double *partials = scratch;
    double *final_totals = scratch + (size_t)kMaxTotals * (size_t)totals_blocks();
    double *dst = out_on_device ? out : final_totals;
    // every block writes all of its partial sums and the final pass overwrites the totals,
    // so nothing in the scratch has to start at zero
    if (launch_totals(family_of(*cfg), cfg->precision == ESLBM_FP64, f, partials, dst, cfg->nx, cfg->ny, sh, P,
                      st) != cudaSuccess)
        return ESLBM_ERR_CUDA;
    if (!out_on_device) {
        if (cudaMemcpyAsync(out, final_totals, sizeof(double) * (size_t)nv, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return ESLBM_ERR_CUDA;
    }
    return ESLBM_OK;
}
