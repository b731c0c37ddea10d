// step2d.cuh -- temporally blocked 2D stages: several fused relax-plus-shift
// stages of D2Q4 in one launch, from a ring of rows in shared memory.
//
// A block owns the output cells [x0, x0 + tx) x [y0, y0 + ly) and sweeps its
// window along y.  The window is the strip widened by hl >= H columns on each
// side and H rows above and below, H = sum |s_j| over the G fused stages (a
// cell's value after G stages depends on cells at most H away along x or y).
// Rows of the window enter a ring of `ring` rows (all q*M planes of a row, one
// bulk copy per plane and contiguous run, completing on the slot's mbarrier),
// loaded `prefetch` rows ahead of use.
//
// Transport in shared memory is index arithmetic, as in the 1D kernel: after
// stages 1..j, with acc_j = s_1 + ... + s_j, population k of logical cell
// (row r, column c) lives at
//   +x: ring row r,          column c - acc_j      -x: ring row r,          column c + acc_j
//   +y: ring row r - acc_j,  column c              -y: ring row r + acc_j,  column c
// so a stage relaxes each cell in place (it reads and writes the same four
// slots).  Stage j handles one row per tick, lagging stage j - 1 by |s_j| + 1
// rows (stage 1 lags the load by |s_1|): every value it reads was written in an
// earlier tick, and one barrier per tick (among the consumer warps) orders the
// stages.  A consumer thread owns the same (stage, column) items every tick; a
// producer warp issues the rows' copies.  Stage j computes
// only the cells that can still reach the output (rows and columns within
// H - m_j of it, m_j = |s_1| + ... + |s_j|), which are exactly the cells whose
// inputs stage j - 1 computed.  The last stage writes the output rows straight
// to global memory.  A ring slot is reloaded only after its last reader
// (ring >= prefetch + max_j (lag_j + |acc_j|)).
//
// Global traffic per launch: (ly + 2H) (tx + 2 hl) / (ly tx) reads and one write
// of every distribution for G stages, against G reads and G writes when the
// stages run one launch each.
#pragma once

#include "kernels.cuh"

namespace eslbm {

template <class R> struct Step2dArgs {
    const R *__restrict__ fin;
    R *__restrict__ fout;
    int64_t nx, ny, ncell;
    int tx;        // output columns of a block (a multiple of 16 / sizeof(R))
    int ly;        // output rows of a block
    int hl;        // window margin on each side, >= H, a multiple of 16 / sizeof(R)
    int wx;        // shared-memory row stride: tx + 2 hl
    int ring;      // rows in the ring (<= kStep2dMaxRing)
    int prefetch;  // rows loaded ahead
    int nstrips;   // blocks along x
    Counters *cnt;
};

// Most threads of a block (one block per SM): as many as the registers of the relaxation allow
// -- FP32: 768 (85 registers a thread) for a fixed omega, 640 (102) for the entropic scalar
// relaxation, 512 (128) for the entropic shallow-water relaxation and 384 (170) with its FP64
// evaluation (the mixed mode); FP64 storage: 512, and 256 (255) for entropic shallow water.
template <class Sys, class R, int OM> struct Step2dThreads {
    static constexpr bool fp64 = sizeof(R) == 8;
    static constexpr int value = (OM == OM_FIXED || Sys::LINEAR) ? (fp64 ? 512 : kStep2dThreads)
                                 : Sys::M == 1                   ? (fp64 ? 512 : 640)
                                 : fp64                          ? 256
                                 : OM == OM_MIXED                ? 384
                                                                 : 512;
};

template <class Sys, class R, int OM>
__global__ void __launch_bounds__(Step2dThreads<Sys, R, OM>::value, kStep2dBlocksPerSm)
    k_step2d(Step2dArgs<R> a, StageList sl, ParamsR<R> P)
{
    constexpr int Q = Sys::Q, M = Sys::M, NP = Q * M;
    static_assert(Q == 4, "D2Q4 only");
    static_assert(NP <= 32, "one lane of the loading warp per plane");
    extern __shared__ __align__(128) unsigned char smem2d[];
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem2d);
    R *ring = reinterpret_cast<R *>(smem2d + kStep2dBarBytes);
    __shared__ int sLag[kStep2dMaxStages], sM[kStep2dMaxStages], sAcc[kStep2dMaxStages], sKind[kStep2dMaxStages];
    __shared__ int sOff[kStep2dMaxStages + 1];
    __shared__ int sTickDone, sFail, sIssued;  // ticks the consumers finished, failure flag, rows issued
    const int G = sl.n, H = sl.halo;
    const int64_t x0 = (int64_t)(blockIdx.x % a.nstrips) * a.tx;
    const int64_t y0 = (int64_t)(blockIdx.x / a.nstrips) * a.ly;
    const int tx = (int)min((int64_t)a.tx, a.nx - x0);
    const int ly = (int)min((int64_t)a.ly, a.ny - y0);
    const int wx = tx + 2 * a.hl;  // this block's window width (<= a.wx)
    const int nrows = ly + 2 * H;  // window rows
    const int rowstride = NP * a.wx;
    if (threadIdx.x == 0) {
        int lag = 0, m = 0, acc = 0, off = 0;
        for (int j = 0; j < G; ++j) {
            const int s = sl.shift[j], as = s < 0 ? -s : s;
            lag += as + (j > 0 ? 1 : 0);
            m += as;
            acc += s;
            sLag[j] = lag;
            sM[j] = m;
            sAcc[j] = acc;
            sKind[j] = sl.kind[j];
            sOff[j] = off;
            off += tx + 2 * (H - m);
        }
        sOff[G] = off;
        sTickDone = 0;
        sFail = 0;
        sIssued = 0;
        for (int i = 0; i < a.ring; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int items = sOff[G];
    const int ticks = ly + H + sLag[G - 1];
    int64_t gx0 = (x0 - a.hl) % a.nx;
    if (gx0 < 0) gx0 += a.nx;
    // r mod ring for 0 <= r < 2^16 and ring <= 64: (r * ceil(2^22 / ring)) >> 22 is the exact quotient
    const uint32_t ring_mul = ((1u << 22) + (uint32_t)a.ring - 1) / (uint32_t)a.ring;
    auto ring_row = [&](int r) { return r - (int)(((uint32_t)r * ring_mul) >> 22) * a.ring; };

    // window row r of every plane into ring slot r % ring, by the first warp: lane 0 announces the
    // bytes to the slot's mbarrier, lane p issues the bulk copies of plane p (one per contiguous run
    // of the row; two or more where the window wraps around the periodic row)
    auto load_row = [&](int r) {
        const int lane = threadIdx.x & 31;
        const int slot = ring_row(r);
        const uint32_t bar = smem_u32(&bars[slot]);
        int64_t gy = (y0 - H + r) % a.ny;
        if (gy < 0) gy += a.ny;
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(NP * wx * (int)sizeof(R));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        }
        __syncwarp();
        if (lane < NP) {
            R *dst = ring + (int64_t)slot * rowstride + lane * a.wx;
            const R *src = a.fin + (int64_t)lane * a.ncell + gy * a.nx;
            int done = 0;
            int64_t gx = gx0;
            while (done < wx) {
                const int len = (int)min((int64_t)(wx - done), a.nx - gx);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(dst + done)),
                    "l"(src + gx), "r"((uint32_t)(len * (int)sizeof(R))), "r"(bar)
                    : "memory");
                done += len;
                gx = 0;
            }
        }
    };
    // Warp 0 is the producer: it issues the rows' bulk copies, row r once the consumers have finished
    // tick r - prefetch (the last tick that reads the slot it overwrites; ring >= prefetch + the
    // longest lifetime of a row), which they publish in sTickDone (release / acquire).  The other
    // warps are the consumers: they wait for each row's copies on its mbarrier, relax, and meet at a
    // named barrier that only they use, once per tick.  All waits are bounded; a consumer that gives
    // up sets sFail before the tick's barrier, so that all consumers leave together.
    const int nconsumers = (int)blockDim.x - 32;
    int failed_tick = -1;
    if (threadIdx.x < 32) {
        for (int r = 0; r < nrows; ++r) {
            if (r >= a.prefetch) {
                int ok = 0;
                if (threadIdx.x == 0) {  // lane 0 waits; the decision is the warp's
                    for (int it = 0; it < (1 << 24) && !ok; ++it) {
                        int d, f;
                        asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];"
                                     : "=r"(d)
                                     : "r"(smem_u32(&sTickDone))
                                     : "memory");
                        asm volatile("ld.relaxed.cta.shared::cta.b32 %0, [%1];" : "=r"(f) : "r"(smem_u32(&sFail)) : "memory");
                        if (f) break;
                        ok = d >= r - a.prefetch + 1;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;  // the consumers gave up (or never got there): issue nothing more
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            load_row(r);
            if (threadIdx.x == 0) sIssued = r + 1;
        }
    } else {
        // The items of a tick (stage j, window column c) are the same every tick: consumer ct owns
        // items ct + s * nconsumers, s < kStep2dSlots, and keeps their stage and column in registers.
        const int ct = (int)threadIdx.x - 32;
        int slot_j[kStep2dSlots], slot_c[kStep2dSlots];
#pragma unroll
        for (int s = 0; s < kStep2dSlots; ++s) {
            const int idx = s * nconsumers + ct;
            int j = -1, c = 0;
            if (idx < items) {
                j = 0;
                while (idx >= sOff[j + 1]) ++j;
                c = a.hl - H + sM[j] + (idx - sOff[j]);
            }
            slot_j[s] = j;
            slot_c[s] = c;
        }
        const int nslots = (items + nconsumers - 1) / nconsumers;  // <= kStep2dSlots (launcher)
        for (int tau = 0; tau < ticks; ++tau) {
            // row tau of the window has arrived (bounded wait)
            uint32_t done = 1;
            if (tau < nrows) {
                const uint32_t bar = smem_u32(&bars[ring_row(tau)]);
                const uint32_t parity = (uint32_t)((tau / a.ring) & 1);
                done = 0;
                for (int it = 0; it < (1 << 22) && !done; ++it) {
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                        "selp.u32 %0, 1, 0, p;\n\t}"
                        : "=r"(done)
                        : "r"(bar), "r"(parity)
                        : "memory");
                }
                if (!done) atomicOr(&sFail, 1);
            }
#pragma unroll
            for (int s = 0; s < kStep2dSlots; ++s) {
                if (s >= nslots) break;  // uniform: every warp runs the same slots (warp-level counters)
                const int j = slot_j[s];
                const int r = j >= 0 ? tau - sLag[j] : -1;
                const bool valid = done && j >= 0 && r >= sM[j] && r < nrows - sM[j];
                bool fb = false, counted = false;
                if (valid) {
                    const int c = slot_c[s];
                    const int acc = sAcc[j];
                    // element offsets of the four populations' slots (plane 0 of each): rows r, r - acc,
                    // r + acc of the ring (r >= m_j >= |acc_j|), columns c -+ acc
                    const int b0 = ring_row(r) * rowstride;
                    int off[Q];
                    off[0] = b0 + c - acc;                       // +x
                    off[1] = ring_row(r - acc) * rowstride + c;  // +y
                    off[2] = b0 + c + acc;                       // -x
                    off[3] = ring_row(r + acc) * rowstride + c;  // -y
                    R f[NP];
#pragma unroll
                    for (int k = 0; k < Q; ++k)
#pragma unroll
                        for (int m = 0; m < M; ++m) f[k * M + m] = ring[off[k] + (k * M + m) * a.wx];
                    // output cells count and record (each cell-stage once over all blocks)
                    counted = r >= H && r < H + ly && c >= a.hl && c < a.hl + tx;
                    const int64_t cell = (y0 + r - H) * a.nx + (x0 + c - a.hl);
                    relax_cell<Sys, R, OM>(P, f, sKind[j], fb, record_of<Sys, R, OM>(P, j, cell, counted));
                    if (j == G - 1) {
#pragma unroll
                        for (int p = 0; p < NP; ++p) a.fout[(int64_t)p * a.ncell + cell] = f[p];
                    } else {
#pragma unroll
                        for (int k = 0; k < Q; ++k)
#pragma unroll
                            for (int m = 0; m < M; ++m) ring[off[k] + (k * M + m) * a.wx] = f[k * M + m];
                    }
                }
                if constexpr (checked<Sys, OM>()) warp_count(fb && counted, &a.cnt->fallbacks);
            }
            // every read and write of this tick is done
            asm volatile("bar.sync 1, %0;" ::"r"(nconsumers) : "memory");
            if (*(volatile int *)&sFail) {
                failed_tick = tau;
                break;
            }
            if (ct == 0) asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTickDone)), "r"(tau + 1) : "memory");
        }
    }
    __syncthreads();  // producer and consumers: every copy that will be issued has been issued
    if (failed_tick >= 0 && threadIdx.x == 32) {
        // a copy never arrived (not expected): report it, and before leaving wait (bounded) for the
        // copies still in flight into this block's shared memory
        atomicAdd(&a.cnt->copy_timeouts, 1ull);
        for (int r = failed_tick; r < sIssued; ++r) {
            const uint32_t bar = smem_u32(&bars[ring_row(r)]);
            const uint32_t parity = (uint32_t)((r / a.ring) & 1);
            uint32_t ok = 0;
            for (int it = 0; it < (1 << 22) && !ok; ++it) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                    "selp.u32 %0, 1, 0, p;\n\t}"
                    : "=r"(ok)
                    : "r"(bar), "r"(parity)
                    : "memory");
            }
        }
    }
}

}  // namespace eslbm
