#!/usr/bin/env python3
"""Throughput of the fourth-order entropy-stable composite step on GB300.

Workload: 1D shallow water (h, hu), g = 9.81, vectorial D1Q2 per conserved
variable (4 distributions per cell), periodic, h0 = 1 + 0.1 sin(2 pi x), u0 = 0,
N = 2^20 cells, V = 4, entropic relaxation parameter, FP32 distributions, run
to t = 0.05 (8738 composite steps of 18 fused stages).  One timed "step" is one
whole solve through the C ABI: init at equilibrium from the device-resident
conserved fields, the composite steps, and the readback of the moments and of
the double-precision entropy / mass totals.

value = site updates per second (cells x composite steps / time), summed over
ranks.  With several GPUs every rank solves its own replica (the path has no
exchange between replicas).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
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
N_CELLS = 1 << 20
V, G, T_FINAL = 4.0, 9.81, 0.05
L2_FLUSH_BYTES = 512 << 20
# FP32 roofline of the dominant kernel (the fused composite step k_step1d, entropic shallow water):
# 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz; and the FP32 operations of one cell-stage
# (FADD + FMUL + 2 FFMA counted by ncu on this workload: 12.5e9 flops per launch over
# 607 blocks x 1800 window cells x 18 stages)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FLOPS_PER_CELL_STAGE = 636.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_CELLS)
    p.add_argument("--t-final", type=float, default=T_FINAL)
    p.add_argument("--no-extras", action="store_true", help="skip the FP64 and CPU baseline legs")
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


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

def oracle_sample(n_cells=512, steps=1):
    import oracle as O
    from paper_2403_13406_gb300 import inputs
    m = O.Model(1, "sw", n_cells, V=V, g=G, omega_mode="entropic")
    f = O.init_equilibrium(m, inputs.sw_sine_1d(n_cells, 1.0, 0.1))
    t0 = time.perf_counter()
    O.composite_steps(m, f, steps)
    dt = time.perf_counter() - t0
    return n_cells * steps / dt, dt


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_cells = 512
    for _ in range(args.warmup):
        oracle_sample(n_cells)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = oracle_sample(n_cells)
        rates.append(r)
        times.append(dt)
    value = n_cells * args.steps / sum(times)
    sample = "oracle (FP64 C, single thread), 1 composite step of the 1D shallow-water workload on %d cells" % n_cells
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "sw1d_d1q2_entropic", "N_sample": n_cells, "V": V, "g": G},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    from paper_2403_13406_gb300 import eslbm, inputs

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

    N = args.n
    n_steps = inputs.steps_for(args.t_final, 1.0 / N, V)
    cfg = eslbm.make_config(1, "sw", N, V=V, g=G, precision="fp32", omega_mode="entropic")
    with torch.cuda.stream(stream):
        sim = eslbm.Simulation(cfg, stream=stream, device=dev)
        sim.use_graph(True)
        u0_host = inputs.sw_sine_1d(N, 1.0, 0.1)
        u0 = torch.from_numpy(u0_host).to(dev)
        u_out = torch.empty((sim.M, N), dtype=torch.float64, device=dev)
        tot = torch.empty(2 + sim.M, dtype=torch.float64, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stages = int(sim.sizes.stages_per_step) * n_steps
    launches_per_step = 1 + n_steps + 1 + 2  # init, one fused launch per composite step, gather, totals

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
            flush.fill_(1.0)  # write > L2 between timed steps (outside the events)
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
    stage_ms = [e[1].elapsed_time(e[2]) / stages for e in evs]
    value, total_ms = aggregate(sum(step_ms), N * n_steps * args.steps, dist, dev)

    # dominant kernel: the fused composite step (one launch per composite step of 18 stages); it is
    # bound by FP32 arithmetic (the entropic root-find), its global traffic being one read and one
    # write of the 16 MB state per launch
    stage_s = statistics.mean(stage_ms) * 1e-3
    launch_s = stage_s * int(sim.sizes.stages_per_step)
    flops = FLOPS_PER_CELL_STAGE * N * int(sim.sizes.stages_per_step)
    achieved = flops / launch_s / 1e12
    peak, peak_kind = peaks()
    hbm_bytes = 2 * int(sim.sizes.planes) * N * 4
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": 16.8e6,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "kernel": "k_step1d<ShallowWater<1>, float, entropic> (one composite step per launch)",
                "launch_us": launch_s * 1e6, "stage_us": stage_s * 1e6,
                "flops_per_cell_stage": FLOPS_PER_CELL_STAGE,
                "hbm_view": {"bytes_per_launch": hbm_bytes, "achieved_gbs": hbm_bytes / launch_s / 1e9,
                             "peak_gbs": peak, "frac": hbm_bytes / launch_s / 1e9 / peak,
                             "per_stage_model_gbs": 18 * hbm_bytes / launch_s / 1e9,
                             "peak_source": peak_kind}}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    u0_pin = torch.from_numpy(u0_host).pin_memory()
    u_host = torch.empty((sim.M, N), dtype=torch.float64).pin_memory()
    tot_host = np.empty(2 + sim.M)
    e2e_times = []
    with torch.cuda.stream(stream):
        for i in range(args.steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sim.init_equilibrium(u0_pin.numpy())
            sim.step(n_steps)
            lib = eslbm.lib()
            sim._check(lib.eslbm_read_moments(sim.h, u_host.data_ptr(), 0))
            sim._check(lib.eslbm_read_totals(sim.h, tot_host.ctypes.data, 0))
            torch.cuda.synchronize(dev)
            if i:
                e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * N * n_steps / statistics.mean(e2e_times)
    h2d = sim.M * N * 8
    d2h = sim.M * N * 8 + (2 + sim.M) * 8

    extras = {}
    if not args.no_extras and rank == 0:
        extras = fp64_leg(sim, torch, eslbm, inputs, stream, dev, N)
        extras.update(adjoint_leg(torch, eslbm, inputs, stream, dev))
    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        rate, dt = oracle_sample(2048)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "1 composite step of the same workload on 2048 cells (FP64 C oracle, %.1f s)" % dt}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "sw1d_d1q2_entropic_n%d_t%g" % (N, args.t_final), "system": "shallow_water",
                           "lattice": "D1Q2", "N": N, "V": V, "g": G, "t_final": args.t_final,
                           "composite_steps": n_steps, "stages": stages, "omega": "entropic", "precision": "fp32",
                           "cuda_graph": True, "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed between timed steps; the 16 MB state stays L2-resident inside a step"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_per_step * args.steps, "clocks": clk}
        line.update(extras)
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.destroy_process_group()


def fp64_leg(sim32, torch, eslbm, inputs, stream, dev, N, nsteps=60):
    """FP64 composite form and FP64 plain second-order form R T on the same grid: throughput on a
    bounded number of steps, and the FP32-vs-FP64 L2 difference of h after those steps."""
    out = {}
    u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
    res = {}
    for name, prec, scheme, steps in (("fp64_composite", "fp64", "I", nsteps), ("fp32_composite", "fp32", "I", nsteps),
                                      ("fp64_plain", "fp64", "plain", 24 * nsteps)):
        cfg = eslbm.make_config(1, "sw", N, V=V, g=G, precision=prec, omega_mode="entropic" if scheme == "I" else "fixed",
                                scheme=scheme)
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            sim.init_equilibrium(u0)
            sim.step(2 if scheme == "I" else 48)
            torch.cuda.synchronize(dev)
            sim.init_equilibrium(u0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            res[name] = sim.moments().cpu().numpy()
            sim.close()
        site_steps = N * (steps if scheme == "I" else steps / 24.0)
        out[name] = {"site_updates_per_s": site_steps / (ms * 1e-3), "ms": ms,
                     "steps": steps, "scheme": scheme, "omega": "entropic" if scheme == "I" else "fixed 2"}
    ref = res["fp64_composite"][0]
    nrm = np.linalg.norm(ref)
    out["fp32_composite"]["rel_l2_h_vs_fp64"] = float(np.linalg.norm(res["fp32_composite"][0] - ref) / nrm)
    out["fp64_plain"]["rel_l2_h_vs_fp64_composite"] = float(np.linalg.norm(res["fp64_plain"][0] - ref) / nrm)
    return {"fp32_vs_fp64": {"N": N, "t": nsteps * 24.0 / N / V, **out}}


def adjoint_leg(torch, eslbm, inputs, stream, dev, N=1 << 16, n=96, K=16):
    """Reverse mode against forward on the same workload shape (1D shallow water, FP32, entropic):
    one forward solve (init, n steps, moments) and one eslbm_gradient (forward with checkpoints
    every K steps, segment and step recomputation, adjoint stages)."""
    cfg = eslbm.make_config(1, "sw", N, V=V, g=G, precision="fp32", omega_mode="entropic")
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


if __name__ == "__main__":
    main()
