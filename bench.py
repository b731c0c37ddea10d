#!/usr/bin/env python3
"""Throughput of the fourth-order entropy-stable composite step on GB300.

Headline workload: 2D compressible Euler (rho, rho u, rho v, E), gamma = 1.4,
vectorial D2Q4 per conserved variable (16 FP32 distributions per cell),
periodic 8192 x 8192, isentropic vortex (strength 5, background rho = p = 1,
velocity (1, 1)) on [0, 10]^2, V = 8, scheme I with omega = 2, 200 composite
steps of 18 fused stages.  One timed "step" is one whole solve through the C
ABI: init at equilibrium from the device-resident conserved fields, the
composite steps, and the readback of the moments and of the double-precision
totals.  value = site updates per second (cells x composite steps / time),
summed over ranks; with several GPUs every rank solves its own replica (the
path has no exchange between replicas).

The other workloads of the path are reported in the same line: 1D shallow
water at N = 2^20 to t = 0.05 (entropic omega, FP32), 2D Burgers 4096^2 for
2000 steps (entropic, past the shock), Euler 4096^2 random-interface Riemann
data (scheme III), 64 uneven batched 2D shallow-water instances for 500 steps
with the reverse mode, FP32 against FP64, the precision split, and the FP64
CPU oracle on the host cores.

--impl reference times the FP64 CPU oracle (OpenMP over the host cores) on a
bounded sample of the headline workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "composite-step site updates/s + HBM GB/s fraction; FP32 vs FP64 at stated L2 error"
UNIT = "site_updates/s"

# headline: Euler 8192^2 isentropic vortex, scheme I, omega = 2, FP32
EULER_N, EULER_V, EULER_GAMMA, EULER_STEPS = 8192, 8.0, 1.4, 200
# 1D shallow water (the 1D workload), 2D Burgers, batched shallow water
SW_N, SW_V, G, SW_T = 1 << 20, 4.0, 9.81, 0.05
SW_UREF = (1.0, 0.0)  # reference state of the shifted FP32 storage: the background depth at rest
BURGERS_N, BURGERS_V, BURGERS_STEPS = 4096, 3.0, 2000
RIEMANN_N, RIEMANN_STEPS = 4096, 500
BATCH_V, BATCH_STEPS, BATCH_K = 8.0, 500, 50
# FP32 ALU roofline of the 1D entropic kernel (an explanation next to the HBM model there):
# 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz, 415 FP32 flops per cell-stage (ncu count)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
SW_FLOPS_PER_CELL_STAGE = 415.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=EULER_N, help="headline grid (n x n)")
    p.add_argument("--composite-steps", type=int, default=EULER_STEPS, help="headline composite steps per solve")
    p.add_argument("--no-extras", action="store_true", help="headline only (no other workloads, no CPU baseline)")
    p.add_argument("--leg", default=None,
                   choices=["sw1d", "burgers2d", "riemann", "batched", "precision", "accuracy", "adjoint", "cpu",
                            "blocked2d", "profile", "batched_accuracy"],
                   help="run one secondary measurement alone and print its JSON")
    p.add_argument("--batch-count", type=int, default=64, help="instances of the batched leg")
    p.add_argument("--group", type=int, default=6, help="profile leg: stages per blocked 2D launch")
    p.add_argument("--case", default="euler",
                   choices=["euler", "euler_blocked", "sw1d", "burgers2d", "burgers2d_blocked", "batched"],
                   help="--leg profile: the workload of one short run (for ncu captures)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = str(gpu_index)
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[0] == self.idx:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def aggregate(total_ms, units_per_rank, dist=None, device=None):
    """Whole-job throughput: every rank times its own replica; the job time is the maximum over
    ranks and the value counts the units of all ranks.  Returns (value, max_ms)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * units_per_rank / (total_ms * 1e-3), total_ms


# DRAM bytes (read + write) per launch of the dominant kernels, from the ncu captures summarised under
# profiles/ (at a smaller size where noted, scaled by the cells a launch processes)
TRAFFIC = {
    "k_step2d_euler_8192_g2": (8.20e9, "profiles/k_step2d_euler_n2048_g2.txt: 513 MB at 2048^2, x 16"),
    "k_stage_bulk_euler_8192": (7.70e9, "profiles/k_stage_bulk_euler_n2048_fp32_fixed.txt: 481 MB at 2048^2, x 16"),
    "k_batch_step_sw2d_64": (47.0e9, "profiles/k_batch_step_sw2d_8inst_fp32_entropic.txt: 7.18 GB for 4.12 M cells, "
                                     "x 26.99 M / 4.12 M"),
}


def hbm_roofline(bytes_per_site_update, site_updates, seconds, kernel, launches, extra=None, traffic=None):
    """Per-stage traffic model of the path (every distribution read and written once per fused
    stage, 2 q M b bytes per cell-stage, 18 cell-stages per site update) over the dominant kernel's
    launches, timed back to back on one stream with CUDA events; `traffic` names the ncu-measured DRAM
    bytes per launch (TRAFFIC) where the kernel was captured."""
    peak, kind = peaks()
    achieved = bytes_per_site_update * site_updates / seconds / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
         "traffic": TRAFFIC[traffic][0] if traffic else None,
         "traffic_source": TRAFFIC[traffic][1] if traffic else None,
         "model": "per-stage: 18 x 2 q M b bytes per site update",
         "bytes_per_site_update": bytes_per_site_update, "peak_source": kind, "kernel": kernel,
         "launches": launches, "launch_us": seconds / max(launches, 1) * 1e6}
    if extra:
        r.update(extra)
    return r


# ---------------------------------------------------------------------------
# the FP64 CPU oracle on bounded samples (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_rate(workload, openmp):
    """Site updates per second of the FP64 oracle on a bounded sample of a workload (about 10 s of
    single-threaded work).  Returns (rate, seconds, sample description, threads)."""
    import oracle as O
    from paper_2403_13406_gb300 import inputs
    used = O.set_openmp(openmp)
    threads = (os.cpu_count() or 1) if (openmp and used) else 1
    if openmp and used:
        os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    if workload == "euler":
        n, steps = (1024, 2) if (openmp and used) else (384, 2)
        m = O.Model(2, "euler", n, n, V=EULER_V, gamma=EULER_GAMMA)
        f = O.init_equilibrium(m, inputs.euler_vortex_2d(n, n))
        desc = "Euler isentropic vortex %d^2, %d composite steps (scheme I, omega = 2)" % (n, steps)
        cells = n * n
    else:
        n, steps = (1 << 14, 2) if (openmp and used) else (1 << 11, 2)
        m = O.Model(1, "sw", n, V=SW_V, g=G, omega_mode="entropic")
        f = O.init_equilibrium(m, inputs.sw_sine_1d(n, 1.0, 0.1))
        desc = "1D shallow water N = %d, %d composite steps (entropic omega)" % (n, steps)
        cells = n
    t0 = time.perf_counter()
    O.composite_steps(m, f, steps)
    dt = time.perf_counter() - t0
    O.set_openmp(False)
    return cells * steps / dt, dt, desc, threads


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_rate("euler", True)
    rates, times = [], []
    desc, threads = "", 1
    for _ in range(args.steps):
        r, dt, desc, threads = oracle_rate("euler", True)
        rates.append(r)
        times.append(dt)
    value = statistics.mean(rates)
    sample = "FP64 C oracle (OpenMP, %d threads): %s" % (threads, desc)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": headline_config(args.n, args.composite_steps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def headline_config(n, steps):
    return {"workload": "euler2d_d2q4_vortex_n%d_steps%d" % (n, steps), "system": "euler", "lattice": "D2Q4",
            "nx": n, "ny": n, "M": 4, "V": EULER_V, "gamma": EULER_GAMMA, "scheme": "I", "omega": "fixed 2",
            "composite_steps": steps, "stages_per_step": 18, "precision": "fp32", "storage": "plain",
            "blocking": "auto: temporally blocked 2D kernel, 2 stages per launch (9 launches per step)",
            "initial_data": "isentropic vortex, strength 5, rho = p = 1, velocity (1, 1), on [0, 10]^2",
            "l2": "inputs larger than L2 (4.3 GB per state buffer); no flush needed"}


# ---------------------------------------------------------------------------
# headline: Euler 8192^2
# ---------------------------------------------------------------------------

def headline(torch, eslbm, inputs, stream, dev, args, world, dist, local):
    n, n_steps = args.n, args.composite_steps
    cfg = eslbm.make_config(2, "euler", n, n, V=EULER_V, gamma=EULER_GAMMA, precision="fp32", omega_mode="fixed")
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        sim.use_graph(True)
        u0_host = inputs.euler_vortex_2d(n, n)
        u0 = torch.from_numpy(u0_host).to(dev)
        u_out = torch.empty((sim.M, n, n), dtype=torch.float64, device=dev)
        tot = torch.empty(2 + sim.M, dtype=torch.float64, device=dev)
    sz = sim.sizes
    launches_step = float(sz.launches_per_step)

    def solve(ev=None):
        sim.init_equilibrium(u0)
        if ev:
            ev[0].record(stream)
        sim.step(n_steps)
        if ev:
            ev[1].record(stream)
        sim.moments(out=u_out)
        sim.totals(host=False, out=tot)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            solve()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        evs = []
        for _ in range(args.steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            solve(ev=(e[1], e[2]))
            e[3].record(stream)
            evs.append(e)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        if dist:
            dist.barrier()
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    kern_ms = [e[1].elapsed_time(e[2]) for e in evs]
    value, _ = aggregate(sum(step_ms), n * n * n_steps * args.steps, dist, dev)
    bytes_su = 18 * 2 * int(sz.planes) * 4
    kernel = "k_step2d<Euler2, float, fixed> (temporally blocked, %g launches per step)" % launches_step \
        if launches_step < 18 else "k_stage_bulk<Euler2, float, fixed> (one launch per stage)"
    traffic = None
    if n == 8192:
        traffic = "k_step2d_euler_8192_g2" if launches_step == 9 else \
            ("k_stage_bulk_euler_8192" if launches_step == 18 else None)
    roof = hbm_roofline(bytes_su, n * n * n_steps, statistics.mean(kern_ms) * 1e-3, kernel,
                        int(round(launches_step * n_steps)),
                        {"site_updates_per_s_kernel": n * n * n_steps / (statistics.mean(kern_ms) * 1e-3)},
                        traffic=traffic)
    with torch.cuda.stream(stream):
        # conservation over the run (FP64 totals) and the vortex after n steps: finite state
        t0 = np.asarray(sim.totals())
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    u0_pin = torch.from_numpy(u0_host).pin_memory()
    u_host = torch.empty((sim.M, n, n), dtype=torch.float64).pin_memory()
    tot_host = np.empty(2 + sim.M)
    lib = eslbm.lib()
    e2e_times, phases = [], {}
    with torch.cuda.stream(stream):
        for i in range(3):
            # run 0: each phase timed alone (synchronised), for the breakdown; runs 1, 2: timed end to end
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            sim._check(lib.eslbm_init_equilibrium(sim.h, u0_pin.data_ptr(), 0))
            if i == 0:
                torch.cuda.synchronize(dev)
                phases["h2d_and_init"] = time.perf_counter() - t
            t1 = time.perf_counter()
            sim.step(n_steps)
            if i == 0:
                torch.cuda.synchronize(dev)
                phases["steps"] = time.perf_counter() - t1
            t2 = time.perf_counter()
            sim._check(lib.eslbm_read_moments(sim.h, u_host.data_ptr(), 0))
            sim._check(lib.eslbm_read_totals(sim.h, tot_host.ctypes.data, 0))
            torch.cuda.synchronize(dev)
            if i == 0:
                phases["gather_d2h_and_totals"] = time.perf_counter() - t2
            else:
                e2e_times.append(time.perf_counter() - t)
    e2e_value = world * n * n * n_steps / statistics.mean(e2e_times)
    sim.close()
    launches = 1 + int(round(launches_step * n_steps)) + 1 + 2  # init, steps, gather, totals (two passes)
    return {"value": value, "ms_per_step": statistics.mean(step_ms), "roofline": roof, "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(sim.M * n * n * 8),
                    "d2h_bytes_per_step": int(sim.M * n * n * 8 + (2 + sim.M) * 8), "phases_s": phases},
            "gpu_launches": launches * args.steps, "mass_total": float(t0[2])}


# ---------------------------------------------------------------------------
# other workloads of the path
# ---------------------------------------------------------------------------

def timed_steps(torch, sim, stream, dev, n_steps, init=None):
    """CUDA-event time (ms) of n_steps composite steps from the given initial fields."""
    with torch.cuda.stream(stream):
        if init is not None:
            sim.init_equilibrium(init)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(n_steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1)


def sw1d_leg(torch, eslbm, inputs, stream, dev):
    """1D shallow water, N = 2^20, g = 9.81, V = 4, h0 = 1 + 0.1 sin 2 pi x, at rest, entropic omega,
    FP32 shifted by the state at rest, to t = 0.05 (8738 composite steps, one temporally blocked launch
    each): throughput and the per-stage HBM model, with the ALU view of the entropic root-find."""
    N = SW_N
    n_steps = inputs.steps_for(SW_T, 1.0 / N, SW_V)
    cfg = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision="fp32", omega_mode="entropic", u_ref=SW_UREF)
    u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        sim.use_graph(True)
        sim.init_equilibrium(u0)
        sim.step(4)
    ms = timed_steps(torch, sim, stream, dev, n_steps, init=u0)
    fb = int(sim.diagnostics()["fallbacks"])
    planes = int(sim.sizes.planes)
    sim.close()
    s = ms * 1e-3
    flops = SW_FLOPS_PER_CELL_STAGE * N * 18 * n_steps / s / 1e12
    roof = hbm_roofline(18 * 2 * planes * 4, N * n_steps, s, "k_step1d<ShallowWater<1>, float, entropic>",
                        n_steps, {"alu_view": {"achieved_tflops": flops, "peak_tflops": FP32_PEAK_TFLOPS,
                                               "frac": flops / FP32_PEAK_TFLOPS,
                                               "flops_per_cell_stage": SW_FLOPS_PER_CELL_STAGE}},
                        traffic=None)  # the capture predates the kernel's current D1Q2 deviations
    return {"sw1d": {"workload": "sw1d_d1q2_entropic_n%d_t%g" % (N, SW_T), "N": N, "V": SW_V, "g": G,
                     "t_final": n_steps * 24.0 / N / SW_V, "composite_steps": n_steps, "ms": ms,
                     "site_updates_per_s": N * n_steps / s, "roofline": roof, "fallbacks": fb,
                     "storage": "fp32, shifted, u_ref = (1, 0)", "cuda_graph": True,
                     "l2": "the 16 MB state is L2-resident within a step"}}


def burgers2d_leg(torch, eslbm, inputs, stream, dev):
    """2D Burgers 4096^2, u0 = 0.5 + 0.25 sin 2 pi x sin 2 pi y + 1e-3 N(0, 1), V = 3, entropic omega,
    FP32, 2000 composite steps (t = 3.9, past shock formation): throughput, per-stage HBM model,
    fallbacks, and the total microscopic entropy before and after (it may only decrease)."""
    n = BURGERS_N
    cfg = eslbm.make_config(2, "burgers", n, n, V=BURGERS_V, precision="fp32", omega_mode="entropic")
    u0 = torch.from_numpy(inputs.burgers_2d(n, n)).to(dev)
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        sim.use_graph(True)
        sim.init_equilibrium(u0)
        sim.step(2)
        sim.init_equilibrium(u0)
        sim.reset_diagnostics()
        t0 = sim.totals()
    ms = timed_steps(torch, sim, stream, dev, BURGERS_STEPS)
    with torch.cuda.stream(stream):
        t1 = sim.totals()
        fb = int(sim.diagnostics()["fallbacks"])
    lps = float(sim.sizes.launches_per_step)
    sim.close()
    s = ms * 1e-3
    kernel = ("k_step2d<Scalar<2, true>, float, entropic> (%g launches per step)" % lps if lps < 18
              else "k_stage_bulk<Scalar<2, true>, float, entropic>")
    return {"burgers2d": {"workload": "burgers2d_d2q4_entropic_n%d_steps%d" % (n, BURGERS_STEPS), "V": BURGERS_V,
                          "t_final": BURGERS_STEPS * 24.0 / n / BURGERS_V, "ms": ms,
                          "site_updates_per_s": n * n * BURGERS_STEPS / s,
                          "roofline": hbm_roofline(18 * 2 * 4 * 4, n * n * BURGERS_STEPS, s, kernel,
                                                   int(round(lps * BURGERS_STEPS))),
                          "fallbacks": fb, "sigma_total": [float(t0[0]), float(t1[0])],
                          "mass_total": [float(t0[2]), float(t1[2])]}}


def riemann_leg(torch, eslbm, inputs, stream, dev, omega=1.98):
    """Euler 4096^2 seeded random-interface Riemann data (four constant states with rho, p in
    [0.5, 1.5], u, v in [-0.5, 0.5]), V = 8, scheme III (the paper's Euler setting) with omega = 1.98,
    500 composite steps: throughput, and the state checked every 50 steps (finite, min rho, min p).
    With omega = 2 exactly the state loses finiteness after about 190 steps at this resolution (FP64
    as FP32, per stage as blocked)."""
    n = RIEMANN_N
    cfg = eslbm.make_config(2, "euler", n, n, V=EULER_V, gamma=EULER_GAMMA, precision="fp32", omega_mode="fixed",
                            omega=omega, scheme="III")
    u0 = torch.from_numpy(inputs.euler_riemann_2d(n, n)).to(dev)
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        sim.use_graph(True)
        sim.init_equilibrium(u0)
        sim.step(2)
    ms = timed_steps(torch, sim, stream, dev, RIEMANN_STEPS, init=u0)
    rows = []
    with torch.cuda.stream(stream):
        sim.init_equilibrium(u0)
        for k in range(RIEMANN_STEPS // 50):
            sim.step(50)
            u = sim.moments()
            rho = u[0]
            p = (EULER_GAMMA - 1) * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / rho)
            fin = bool(torch.isfinite(u).all())
            rows.append({"steps": 50 * (k + 1), "finite": fin, "rho_min": float(rho.min()), "p_min": float(p.min())})
            if not fin:
                break
    lps = float(sim.sizes.launches_per_step)
    sim.close()
    s = ms * 1e-3
    return {"euler_riemann": {"workload": "euler2d_d2q4_riemann_n%d_steps%d_schemeIII" % (n, RIEMANN_STEPS),
                              "omega": omega, "ms": ms, "site_updates_per_s": n * n * RIEMANN_STEPS / s,
                              "roofline": hbm_roofline(27 * 2 * 16 * 4, n * n * RIEMANN_STEPS, s,
                                                       ("k_step2d<Euler2, float, fixed> (temporally blocked, %g launches "
                                                        "per step)" % lps) if lps < 27 else "k_stage_bulk<Euler2, float, fixed>",
                                                       int(round(lps * RIEMANN_STEPS)),
                                                       {"model": "per-stage: 27 x 2 q M b bytes per step (scheme III)"}),
                              "state": rows}}


def blocked2d_leg(torch, eslbm, inputs, stream, dev, steps=10):
    """The temporally blocked 2D kernel (k_step2d, several stages per launch from a ring of rows in
    shared memory) against one launch per stage, on the headline Euler workload (8192^2, scheme I,
    FP32) and on 2D Burgers 4096^2 (fixed and entropic omega): site updates per second of each and
    the per-stage HBM model's fraction (the blocked kernel moves fewer bytes than that model)."""
    out = {}
    cases = (("euler_8192_fixed", "euler", EULER_N, dict(V=EULER_V, gamma=EULER_GAMMA), "fixed",
              lambda n: inputs.euler_vortex_2d(n, n), 64),
             ("burgers_4096_fixed", "burgers", BURGERS_N, dict(V=BURGERS_V), "fixed", lambda n: inputs.burgers_2d(n, n), 16),
             ("burgers_4096_entropic", "burgers", BURGERS_N, dict(V=BURGERS_V), "entropic",
              lambda n: inputs.burgers_2d(n, n), 16))
    for name, system, n, kw, mode, init, bpc in cases:
        row = {}
        for label, blocking in (("per_stage", False), ("blocked_2", 2), ("blocked_3", 3), ("blocked_6", 6)):
            cfg = eslbm.make_config(2, system, n, n, precision="fp32", omega_mode=mode, blocking=blocking, **kw)
            u0 = torch.from_numpy(init(n)).to(dev)
            with torch.cuda.stream(stream):
                sim = eslbm.Simulation(cfg, stream=stream, device=dev)
                sim.use_graph(True)
                sim.init_equilibrium(u0)
                sim.step(2)
            ms = timed_steps(torch, sim, stream, dev, steps)
            lps = float(sim.sizes.launches_per_step)
            sim.close()
            del u0
            sps = n * n * steps / (ms * 1e-3)
            peak, _ = peaks()
            row[label] = {"site_updates_per_s": sps, "launches_per_step": lps,
                          "per_stage_model_frac": sps * 18 * 2 * bpc / 1e9 / peak}
        for g in (2, 3, 6):
            row["blocked_%d_over_per_stage" % g] = (row["blocked_%d" % g]["site_updates_per_s"] /
                                                    row["per_stage"]["site_updates_per_s"])
        out[name] = row
    return {"blocked2d": out}


def precision_leg(torch, eslbm, inputs, stream, dev, N=1 << 18):
    """The precision split on the 1D shallow-water workload to t = 0.05: FP32 storage with the
    entropic omega in FP32, FP32 storage with the entropy difference in FP64 (mixed), against the
    all-FP64 path on the same grid: relative L2 error of the state at the final time and time per
    composite step, plus the per-cell entropy check (diagnostics) of each mode."""
    n_steps = inputs.steps_for(SW_T, 1.0 / N, SW_V)
    u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
    res = {}
    for name, prec, uref in (("fp64", "fp64", None), ("fp32", "fp32", None), ("fp32_shifted", "fp32", SW_UREF),
                             ("fp32_mixed_shifted", "fp32_mixed", SW_UREF)):
        cfg = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision=prec, omega_mode="entropic", u_ref=uref)
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            sim.init_equilibrium(u0)
            sim.step(2)
        ms = timed_steps(torch, sim, stream, dev, n_steps, init=u0)
        with torch.cuda.stream(stream):
            u = sim.moments().cpu().numpy()
        sim.close()
        # the per-cell check over the first 64 steps, in the same kernels
        cfg_d = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision=prec, omega_mode="entropic", u_ref=uref,
                                  diagnostics=True)
        with torch.cuda.stream(stream):
            simd = eslbm.Simulation(cfg_d, stream=stream, device=dev)
            simd.init_equilibrium(u0)
            simd.step(64)
            d = simd.diagnostics()
            simd.close()
        res[name] = {"u": u, "ms_per_step": ms / n_steps, "entropy_increases_64_steps": int(d["entropy_increases"]),
                     "entropy_excess_max": float(d["entropy_excess_max"])}
    ref = res["fp64"]["u"]
    out = {}
    for name, r in res.items():
        row = {"ms_per_composite_step": r["ms_per_step"], "entropy_increases_64_steps": r["entropy_increases_64_steps"],
               "entropy_excess_max": r["entropy_excess_max"]}
        if name != "fp64":
            a = r["u"]
            row["rel_l2_h"] = float(np.linalg.norm(a[0] - ref[0]) / np.linalg.norm(ref[0]))
            row["rel_l2_hu"] = float(np.linalg.norm(a[1] - ref[1]) / max(np.linalg.norm(ref[1]), 1e-300))
            row["rel_l2_state"] = float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
        out[name] = row
    return {"precision": {"workload": "sw1d entropic, N = %d, t = %.4f (%d composite steps)"
                                      % (N, n_steps * 24.0 / N / SW_V, n_steps),
                          "reference": "fp64 composite on the same grid", "modes": out}}


def fp32_vs_fp64_leg(torch, eslbm, inputs, stream, dev, N=SW_N, nsteps=60):
    """FP64 composite form and FP64 plain second-order form R T on the 1D shallow-water grid:
    throughput on a bounded number of steps."""
    out = {}
    u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
    for name, prec, scheme, steps in (("fp64_composite", "fp64", "I", nsteps), ("fp32_composite", "fp32", "I", nsteps),
                                      ("fp64_plain", "fp64", "plain", 24 * nsteps)):
        cfg = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision=prec,
                                omega_mode="entropic" if scheme == "I" else "fixed", scheme=scheme,
                                u_ref=SW_UREF if prec == "fp32" else None)
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            sim.init_equilibrium(u0)
            sim.step(2 if scheme == "I" else 48)
        ms = timed_steps(torch, sim, stream, dev, steps, init=u0)
        sim.close()
        site_steps = N * (steps if scheme == "I" else steps / 24.0)
        out[name] = {"site_updates_per_s": site_steps / (ms * 1e-3), "ms": ms, "steps": steps, "scheme": scheme,
                     "omega": "entropic" if scheme == "I" else "fixed 2"}
    return {"fp32_vs_fp64": {"N": N, **out}}


def accuracy_leg(torch, eslbm, inputs, stream, dev, n_ref=1 << 16, sizes=tuple(1 << k for k in range(8, 17)),
                 targets=(1e-5, 1e-6, 1e-7)):
    """Time to solution at a stated L2 error: the FP32 composite scheme (entropic omega) against the FP64
    plain second-order scheme R T (omega = 2, 24 plain steps per composite step, so both reach the same
    time t = 2 x 24 / (256 V) = 0.046875 on every grid), 1D shallow water h0 = 1 + 0.1 sin 2 pi x.  The
    error is the relative discrete L2 norm of h against the FP64 composite solution on 2^16 cells, sampled
    at the coarse points (cells at j dx on every grid).  Times are CUDA-event times of the steps alone."""
    def run(N, prec, scheme, n_comp):
        cfg = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision=prec,
                                omega_mode="entropic" if scheme == "I" else "fixed", omega=2.0, scheme=scheme,
                                u_ref=SW_UREF if prec == "fp32" else None)
        steps = n_comp if scheme == "I" else 24 * n_comp
        u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            sim.init_equilibrium(u0)
            sim.step(1)  # warm-up and graph capture
        ms = timed_steps(torch, sim, stream, dev, steps, init=u0)
        with torch.cuda.stream(stream):
            h = sim.moments().cpu().numpy()[0]
        sim.close()
        return h, ms

    n_at = lambda N: 2 * N // 256  # composite steps to t = 0.046875
    ref, _ = run(n_ref, "fp64", "I", n_at(n_ref))
    rows = []
    for N in sizes:
        r = ref[:: n_ref // N]
        row = {"N": N}
        for name, prec, scheme in (("fp32_composite", "fp32", "I"), ("fp64_plain", "fp64", "plain")):
            h, ms = run(N, prec, scheme, n_at(N))
            row[name] = {"rel_l2": float(np.linalg.norm(h - r) / np.linalg.norm(r)), "ms": ms}
        rows.append(row)
    best = {}
    for eps in targets:
        pick = {}
        for name in ("fp32_composite", "fp64_plain"):
            ok = [r for r in rows if r[name]["rel_l2"] <= eps]
            pick[name] = ({"N": ok[0]["N"], "ms": ok[0][name]["ms"], "rel_l2": ok[0][name]["rel_l2"]} if ok
                          else None)
        if pick["fp32_composite"] and pick["fp64_plain"]:
            pick["speedup_fp32_composite"] = pick["fp64_plain"]["ms"] / pick["fp32_composite"]["ms"]
        best["%g" % eps] = pick
    return {"time_to_accuracy": {"t": 2 * 24 / (256 * SW_V), "reference": "fp64 composite, N = %d" % n_ref,
                                 "sweep": rows, "at_target_rel_l2": best}}


def adjoint_leg(torch, eslbm, inputs, stream, dev, N=1 << 16, n=96, K=16):
    """Reverse mode against forward on the 1D shallow-water workload shape (FP32, entropic): one forward
    solve (init, n steps, moments) and one eslbm_gradient (forward with checkpoints every K steps,
    segment and step recomputation, adjoint stages)."""
    cfg = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision="fp32", omega_mode="entropic")
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
        lam = torch.ones((2, N), dtype=torch.float64, device=dev)
        times = {}
        for name in ("forward", "adjoint", "forward", "adjoint"):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            if name == "forward":
                sim.init_equilibrium(u0)
                sim.step(n)
                sim.moments()
            else:
                sim.gradient(u0, lam, n, K)
            torch.cuda.synchronize(dev)
            times[name] = time.perf_counter() - t0
        sim.close()
    return {"adjoint_vs_forward": {"N": N, "steps": n, "checkpoint_every": K, "forward_s": times["forward"],
                                   "adjoint_s": times["adjoint"], "ratio": times["adjoint"] / times["forward"]}}


def batch_leg(torch, eslbm, inputs, stream, dev, count=64, steps=BATCH_STEPS, K=BATCH_K, grad=True, grad_steps=None):
    """Batched form: `count` 2D shallow-water instances (D2Q4, FP32 shifted by the state at rest of depth
    1, entropic) of uneven seeded sizes in [256, 1024]^2 with 8-mode Fourier depth data, advanced by one
    cooperative launch per composite step replayed from CUDA graphs, after the autotuner has picked the
    schedule, for `steps` composite steps; then the reverse mode: the gradient of the L2 misfit of the
    final depth against a seeded target with respect to the initial depth of every instance,
    checkpoints every K steps (grad_steps composite steps: the full run by default, fewer in the
    default bench line to bound its time).  The FP32 error after the steps is stated against FP64
    single-lattice runs of two instances."""
    grad_steps = steps if grad_steps is None else grad_steps
    sizes = inputs.batched_sizes(count, 256, 1024)
    cfg = eslbm.make_config(2, "sw", 1, 1, V=BATCH_V, g=G, precision="fp32", omega_mode="entropic",
                            u_ref=(1.0, 0.0, 0.0))
    with torch.cuda.stream(stream):
        b = eslbm.Batch(cfg, sizes, stream=stream, device=dev)
        u0 = b.pack([inputs.sw_fourier_2d(nx, ny, seed=1000 + i) for i, (nx, ny) in enumerate(sizes)])
        b.init_equilibrium(u0)
        t0 = time.perf_counter()
        sched = b.tune(steps=2)
        tune_s = time.perf_counter() - t0
        b.use_graph(True)
        b.init_equilibrium(u0)
        b.step(2)  # warm-up: captures the graphs
        b.init_equilibrium(u0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        fallbacks = int(b.diagnostics()["fallbacks"])
        cells = b.total_cells
        fp32 = b.moments()
        errs = []
        for i in (0, 1):  # FP64 reference of two instances, same steps
            nx, ny = sizes[i]
            c64 = eslbm.make_config(2, "sw", nx, ny, V=BATCH_V, g=G, precision="fp64", omega_mode="entropic")
            s64 = eslbm.Simulation(c64, stream=stream, device=dev)
            s64.use_graph(True)
            s64.init_equilibrium(torch.from_numpy(inputs.sw_fourier_2d(nx, ny, seed=1000 + i)).to(dev))
            s64.step(steps)
            ref = s64.moments()
            s64.close()
            errs.append(float(torch.linalg.vector_norm(fp32[i][0] - ref[0]) / torch.linalg.vector_norm(ref[0])))
        out = {"instances": count, "total_cells": cells, "sizes": "seeded uniform nx, ny in [256, 1024]",
               "steps": steps, "ms": ms, "site_updates_per_s": cells * steps / (ms * 1e-3),
               "roofline": hbm_roofline(18 * 2 * 12 * 4, cells * steps, ms * 1e-3,
                                        "k_batch_step<ShallowWater<2>, float, entropic>", steps,
                                        traffic="k_batch_step_sw2d_64" if count == 64 else None),
               "schedule": {"segment": sched[0], "blocks_per_sm": sched[1], "order": sched[2]},
               "tune_s": tune_s, "cuda_graph": True, "fallbacks": fallbacks, "V": BATCH_V,
               "storage": "fp32, shifted, u_ref = (1, 0, 0)",
               "rel_l2_h_vs_fp64": {"instances": [list(sizes[0]), list(sizes[1])], "values": errs}}
        if grad:
            target = b.pack([inputs.sw_fourier_2d(nx, ny, seed=5000 + i) for i, (nx, ny) in enumerate(sizes)])
            torch.cuda.synchronize(dev)
            tf = time.perf_counter()
            b.init_equilibrium(u0)
            b.step(grad_steps)
            uT = b.moments_flat()
            torch.cuda.synchronize(dev)
            fwd_s = time.perf_counter() - tf
            lam = torch.zeros_like(uT)
            for v, (u, t) in enumerate(zip(b.unpack(uT), b.unpack(target))):
                b.unpack(lam)[v][0] = 2.0 * (u[0] - t[0])  # dJ/dh_T of J = sum (h_T - target)^2
            torch.cuda.synchronize(dev)
            ta = time.perf_counter()
            g = b.gradient(u0, lam, grad_steps, K)
            torch.cuda.synchronize(dev)
            adj_s = time.perf_counter() - ta
            out["adjoint"] = {"instances": count, "steps": grad_steps, "checkpoint_every": K, "forward_s": fwd_s,
                              "gradient_s": adj_s, "ratio": adj_s / fwd_s, "grad_norm": float(torch.linalg.vector_norm(g)),
                              "finite": bool(torch.isfinite(g).all())}
        b.close()
    return {"batched": out}


def batched_accuracy_leg(torch, eslbm, inputs, stream, dev, count=8, base=(32, 128), levels=(1, 2, 4, 8), ref_level=16,
                         n0=4, targets=(1e-4, 3e-5, 1e-5, 3e-6)):
    """Time to a stated L2 error in the batched form: `count` 2D shallow-water instances of uneven seeded
    sizes (base range, scaled by each refinement level) with the 8-mode Fourier depth data of the batched
    workload, advanced as one batch in FP32 by the composite scheme (entropic omega, shifted storage,
    one cooperative launch per composite step from CUDA graphs), against the same batch in FP64 by the
    plain second-order scheme R T (omega = 2, 24 plain steps per composite step: the same final time on
    every level and instance).  Level l runs l n0 composite steps.  The error of h is the relative L2
    norm over all instances against FP64 composite solutions at `ref_level` times the base resolution,
    sampled at the coarse cells (omega = 2: the composite scheme is fourth order with either relaxation on
    smooth data, and the fixed one spares the reference the FP64 root-find).  Times are CUDA-event times
    of the steps alone."""
    rng_sizes = [(max(4, a // 4 * 4), max(4, b // 4 * 4)) for a, b in inputs.batched_sizes(count, *base)]
    refs = []
    for i, (nx, ny) in enumerate(rng_sizes):
        c64 = eslbm.make_config(2, "sw", nx * ref_level, ny * ref_level, V=BATCH_V, g=G, precision="fp64",
                                omega_mode="fixed", omega=2.0)
        with torch.cuda.stream(stream):
            s64 = eslbm.Simulation(c64, stream=stream, device=dev)
            s64.use_graph(True)
            s64.init_equilibrium(torch.from_numpy(inputs.sw_fourier_2d(nx * ref_level, ny * ref_level,
                                                                       seed=1000 + i)).to(dev))
            s64.step(n0 * ref_level)
            refs.append(s64.moments()[0].cpu().numpy())
            s64.close()

    def run(level, prec, scheme):
        sizes = [(nx * level, ny * level) for nx, ny in rng_sizes]
        plain = scheme == "plain"
        cfg = eslbm.make_config(2, "sw", 1, 1, V=BATCH_V, g=G, precision=prec,
                                omega_mode="fixed" if plain else "entropic", omega=2.0, scheme=scheme,
                                u_ref=None if plain else (1.0, 0.0, 0.0))
        steps = n0 * level * (24 if plain else 1)
        with torch.cuda.stream(stream):
            b = eslbm.Batch(cfg, sizes, stream=stream, device=dev)
            u0 = b.pack([inputs.sw_fourier_2d(nx, ny, seed=1000 + i) for i, (nx, ny) in enumerate(sizes)])
            b.use_graph(True)
            b.init_equilibrium(u0)
            b.step(min(steps, 24))  # warm-up: captures the graphs
            b.init_equilibrium(u0)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            hs = [m[0].cpu().numpy() for m in b.moments()]
            cells = b.total_cells
            b.close()
        f = ref_level // level
        num = sum(float(np.sum((h - r[::f, ::f]) ** 2)) for h, r in zip(hs, refs))
        den = sum(float(np.sum(r[::f, ::f] ** 2)) for r in refs)
        return {"rel_l2": (num / den) ** 0.5, "ms": ms, "cells": cells, "steps": steps}

    rows = []
    for level in levels:
        rows.append({"level": level, "fp32_batched_composite": run(level, "fp32", "I"),
                     "fp64_batched_plain": run(level, "fp64", "plain")})
    best = {}
    for eps in targets:
        pick = {}
        for name in ("fp32_batched_composite", "fp64_batched_plain"):
            ok = [r for r in rows if r[name]["rel_l2"] <= eps]
            pick[name] = {"level": ok[0]["level"], **ok[0][name]} if ok else None
        if pick["fp32_batched_composite"] and pick["fp64_batched_plain"]:
            pick["speedup_fp32_batched"] = pick["fp64_batched_plain"]["ms"] / pick["fp32_batched_composite"]["ms"]
        best["%g" % eps] = pick
    return {"batched_time_to_accuracy": {
        "instances": count, "base_sizes": "seeded uniform nx, ny in [%d, %d], multiples of 4" % base,
        "levels": list(levels), "composite_steps_at_level_1": n0,
        "reference": "fp64 composite (omega = 2) per instance at %d x the base resolution" % ref_level,
        "sweep": rows, "at_target_rel_l2": best}}


def cpu_leg():
    """The FP64 oracle on the host cores: single-threaded and OpenMP over every core, on bounded samples
    of the headline and of the 1D workload (rates in site updates per second)."""
    out = {}
    for wl in ("euler", "sw1d"):
        for omp in (False, True):
            r, dt, desc, threads = oracle_rate(wl, omp)
            out["%s_%s" % (wl, "openmp" if omp else "single")] = {"site_updates_per_s": r, "seconds": dt,
                                                                   "threads": threads, "sample": desc}
    return {"cpu_oracle": out}


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def profile_leg(torch, eslbm, inputs, stream, dev, case="euler", n=None, steps=2, group=6):
    """One short run of a workload's kernels, for ncu captures (init, `steps` composite steps,
    moments): euler = the headline at n x n (default 2048, one launch per stage), euler_blocked =
    the same through the temporally blocked 2D kernel (`group` stages per launch), sw1d = the 1D workload
    at 2^20 cells, burgers2d[_blocked] = 2D Burgers entropic at n x n (default 4096), batched = 8 of
    the batched instances."""
    if case == "batched":
        sizes = inputs.batched_sizes(8, 256, 1024)
        cfg = eslbm.make_config(2, "sw", 1, 1, V=BATCH_V, g=G, precision="fp32", omega_mode="entropic",
                                u_ref=(1.0, 0.0, 0.0))
        b = eslbm.Batch(cfg, sizes, stream=stream, device=dev)
        with torch.cuda.stream(stream):
            b.init_equilibrium(b.pack([inputs.sw_fourier_2d(nx, ny, seed=1000 + i) for i, (nx, ny) in enumerate(sizes)]))
            b.step(steps)
            torch.cuda.synchronize(dev)
        b.close()
        return {"profile": case, "instances": len(sizes), "steps": steps}
    if case == "sw1d":
        N = SW_N
        cfg = eslbm.make_config(1, "sw", N, V=SW_V, g=G, precision="fp32", omega_mode="entropic", u_ref=SW_UREF)
        u0 = inputs.sw_sine_1d(N, 1.0, 0.1)
    elif case.startswith("euler"):
        N = n or 2048
        cfg = eslbm.make_config(2, "euler", N, N, V=EULER_V, gamma=EULER_GAMMA, precision="fp32", omega_mode="fixed",
                                blocking=group if case.endswith("blocked") else True)
        u0 = inputs.euler_vortex_2d(N, N)
    else:
        N = n or BURGERS_N
        cfg = eslbm.make_config(2, "burgers", N, N, V=BURGERS_V, precision="fp32", omega_mode="entropic",
                                blocking=group if case.endswith("blocked") else True)
        u0 = inputs.burgers_2d(N, N)
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        sim.init_equilibrium(torch.from_numpy(u0).to(dev))
        sim.step(steps)
        sim.moments()
        torch.cuda.synchronize(dev)
        sim.close()
    return {"profile": case, "n": N, "steps": steps}


LEGS = {"sw1d": sw1d_leg, "burgers2d": burgers2d_leg, "riemann": riemann_leg, "batched": batch_leg,
        "batched_accuracy": batched_accuracy_leg,
        "blocked2d": blocked2d_leg, "profile": profile_leg,
        "precision": precision_leg, "accuracy": accuracy_leg, "adjoint": adjoint_leg}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.leg == "cpu":
        print(json.dumps(cpu_leg()), flush=True)
        return
    import torch
    from paper_2403_13406_gb300 import eslbm, inputs
    if args.leg:
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        kw = {"count": args.batch_count} if args.leg == "batched" else {}
        if args.leg == "precision" and args.n != EULER_N:
            kw = {"N": args.n}  # e.g. --leg precision --n 1048576: the 1D grid of the 1D workload
        if args.leg == "profile":
            kw = {"case": args.case, "n": None if args.n == EULER_N else args.n, "group": args.group}
        print(json.dumps(LEGS[args.leg](torch, eslbm, inputs, stream, dev, **kw)), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", local if world > 1 else 0)
    stream = torch.cuda.Stream(device=dev)

    head = headline(torch, eslbm, inputs, stream, dev, args, world, dist, local)
    extras, cpu = {}, None
    if not args.no_extras and rank == 0:
        for leg in (sw1d_leg, burgers2d_leg, riemann_leg, blocked2d_leg, precision_leg, fp32_vs_fp64_leg,
                    accuracy_leg, batched_accuracy_leg, adjoint_leg):
            try:
                extras.update(leg(torch, eslbm, inputs, stream, dev))
            except Exception as e:  # a failing extra is reported, and does not take the headline line with it
                extras[leg.__name__] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
        extras.update(batch_leg(torch, eslbm, inputs, stream, dev, count=args.batch_count, grad_steps=100,
                                K=10))
    if rank == 0 and world == 1 and not args.no_extras:
        c = cpu_leg()["cpu_oracle"]
        extras["cpu_oracle"] = c
        e = c["euler_single"]
        cpu = {"value": e["site_updates_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "FP64 C oracle, single thread: %s, %.1f s" % (e["sample"], e["seconds"]),
               "openmp": {"value": c["euler_openmp"]["site_updates_per_s"], "cores": c["euler_openmp"]["threads"],
                          "sample": c["euler_openmp"]["sample"]}}
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(headline_config(args.n, args.composite_steps),
                               parallelism="replicas" if world > 1 else "single", cuda_graph=True),
                "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head["e2e"],
                "gpu_launches": head["gpu_launches"], "clocks": head["clocks"]}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
