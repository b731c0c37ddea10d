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
U_REF = (1.0, 0.0)  # reference state of the shifted FP32 storage: the background depth at rest
BATCH_V = 8.0  # lattice velocity of the batched 2D shallow-water instances: sqrt(9.81 x 1.05) < V/2
L2_FLUSH_BYTES = 512 << 20
# FP32 roofline of the dominant kernel (the fused composite step k_step1d, entropic shallow water):
# 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz; and the FP32 operations of one cell-stage
# (FADD + FMUL + 2 FFMA counted by ncu on this workload: 7.98e9 flops per launch over the 19.25e6
# cell-stages a launch computes, 607 blocks x 31716).  The kernel is bound by instruction issue: 641 thread instructions
# per cell-stage against 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FLOPS_PER_CELL_STAGE = 415.0
ISSUE_PEAK_TINST = 152 * 4 * 32 * 2.07e9 / 1e12
INST_PER_CELL_STAGE = 641.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_CELLS)
    p.add_argument("--t-final", type=float, default=T_FINAL)
    p.add_argument("--no-extras", action="store_true", help="skip the FP64 and CPU baseline legs")
    p.add_argument("--leg", default=None, choices=["hbm2d", "batched", "fp32err"],
                   help="run one secondary measurement alone and print its JSON (for profiling)")
    p.add_argument("--hbm-steps", type=int, default=20, help="composite steps of the 2D streaming leg")
    p.add_argument("--hbm-case", default=None, help="one case of the 2D streaming leg (default: all)")
    p.add_argument("--batch-count", type=int, default=64, help="instances of the batched leg")
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
            "data": "synthetic",
            "config": {"workload": "sw1d_d1q2_entropic_n%d_t%g" % (args.n, args.t_final), "system": "shallow_water",
                       "lattice": "D1Q2", "N": args.n, "V": V, "g": G, "t_final": args.t_final, "omega": "entropic",
                       "N_sample": n_cells, "steps_per_sample": 1},
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
    if args.leg:
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        leg = {"hbm2d": hbm2d_leg, "batched": batch_leg, "fp32err": fp32err_leg}[args.leg]
        kw = ({"steps": args.hbm_steps, "only": args.hbm_case} if args.leg == "hbm2d" else
              {"N": args.n, "t_final": args.t_final} if args.leg == "fp32err" else {"count": args.batch_count})
        print(json.dumps(leg(torch, eslbm, inputs, stream, dev, **kw)), flush=True)
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

    N = args.n
    n_steps = inputs.steps_for(args.t_final, 1.0 / N, V)
    cfg = eslbm.make_config(1, "sw", N, V=V, g=G, precision="fp32", omega_mode="entropic", u_ref=U_REF)
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
    inst_rate = INST_PER_CELL_STAGE * N * int(sim.sizes.stages_per_step) / launch_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": 16.81e6,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "kernel": "k_step1d<ShallowWater<1>, float, entropic> (one composite step per launch)",
                "launch_us": launch_s * 1e6, "stage_us": stage_s * 1e6,
                "flops_per_cell_stage": FLOPS_PER_CELL_STAGE,
                "issue_view": {"inst_per_cell_stage": INST_PER_CELL_STAGE, "achieved_tinst_s": inst_rate,
                               "peak_tinst_s": ISSUE_PEAK_TINST, "frac": inst_rate / ISSUE_PEAK_TINST,
                               "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz"},
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
        extras.update(accuracy_leg(torch, eslbm, inputs, stream, dev))
        extras.update(adjoint_leg(torch, eslbm, inputs, stream, dev))
        extras.update(batch_leg(torch, eslbm, inputs, stream, dev))
        extras.update(hbm2d_leg(torch, eslbm, inputs, stream, dev))
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
                           "storage": "shifted, u_ref = (1, 0)",
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
                                scheme=scheme, u_ref=U_REF if prec == "fp32" else None)
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


def fp32err_leg(torch, eslbm, inputs, stream, dev, N=N_CELLS, t_final=T_FINAL):
    """Error of the FP32 composite solution against the FP64 composite solution of the bench workload
    (1D shallow water, entropic omega) at the final time, relative L2 of h and of hu, with the error after
    1/8, 1/4, 1/2 of the steps (rounding accumulates with the number of stages).  FP64 runs at 1/64 of
    the FP32 rate on this GPU, so the full-size case takes minutes."""
    n_steps = inputs.steps_for(t_final, 1.0 / N, V)
    marks = sorted(set([max(1, n_steps // 8), max(1, n_steps // 4), max(1, n_steps // 2), n_steps]))
    u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
    res = {}
    for prec in ("fp32", "fp32_shifted", "fp64"):
        cfg = eslbm.make_config(1, "sw", N, V=V, g=G, precision=prec[:4], omega_mode="entropic",
                                u_ref=U_REF if prec == "fp32_shifted" else None)
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            sim.init_equilibrium(u0)
            done, out = 0, []
            for mk in marks:
                sim.step(mk - done)
                done = mk
                out.append(sim.moments().cpu().numpy())
            res[prec] = out
            sim.close()
    rows = []
    for i, mk in enumerate(marks):
        b = res["fp64"][i]
        row = {"steps": mk, "t": mk * 24.0 / N / V}
        for name in ("fp32", "fp32_shifted"):
            a = res[name][i]
            row[name] = {"rel_l2_h": float(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])),
                         "rel_l2_hu": float(np.linalg.norm(a[1] - b[1]) / max(np.linalg.norm(b[1]), 1e-300)),
                         "rel_l2_state": float(np.linalg.norm(a - b) / np.linalg.norm(b))}
        rows.append(row)
    return {"fp32_error": {"N": N, "t_final": t_final, "reference": "fp64 composite (same scheme, same grid)",
                           "rows": rows}}


def accuracy_leg(torch, eslbm, inputs, stream, dev, n_ref=1 << 16, sizes=tuple(1 << k for k in range(8, 17)),
                 targets=(1e-5, 1e-6, 1e-7)):
    """Time to solution at a stated L2 error: the FP32 composite scheme (entropic omega) against the FP64
    plain second-order scheme R T (omega = 2, 24 plain steps per composite step, so both reach the same
    time t = 2 x 24 / (256 V) = 0.046875 on every grid), 1D shallow water h0 = 1 + 0.1 sin 2 pi x.  The
    error is the relative discrete L2 norm of h against the FP64 composite solution on 2^16 cells, sampled
    at the coarse points (cells at j dx on every grid).  Times are CUDA-event times of the steps alone."""
    def run(N, prec, scheme, n_comp):
        cfg = eslbm.make_config(1, "sw", N, V=V, g=G, precision=prec,
                                omega_mode="entropic" if scheme == "I" else "fixed", omega=2.0, scheme=scheme,
                                u_ref=U_REF if prec == "fp32" else None)
        steps = n_comp if scheme == "I" else 24 * n_comp
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            u0 = torch.from_numpy(inputs.sw_sine_1d(N, 1.0, 0.1)).to(dev)
            sim.init_equilibrium(u0)
            sim.step(1)  # warm-up and graph capture
            sim.init_equilibrium(u0)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            h = sim.moments().cpu().numpy()[0]
            sim.close()
        return h, e0.elapsed_time(e1)

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
    return {"time_to_accuracy": {"t": 2 * 24 / (256 * V), "reference": "fp64 composite, N = %d" % n_ref,
                                 "sweep": rows, "at_target_rel_l2": best}}


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


def batch_leg(torch, eslbm, inputs, stream, dev, count=64, steps=20, grad_instances=4, grad_n=50, grad_K=10):
    """Batched form: `count` 2D shallow-water instances (D2Q4, FP32, entropic) of uneven seeded sizes in
    [256, 1024]^2 with 8-mode Fourier depth data, advanced by one cooperative launch per composite step
    replayed from CUDA graphs, after the autotuner has picked the schedule; a bounded number of steps.
    The reverse mode is timed on the first `grad_instances` instances (L2 misfit of the final depth
    against a seeded target, checkpoints every grad_K steps).  FP32 storage shifted by the state at rest
    of depth 1; its error after the timed steps is stated against FP64 single-lattice runs of two
    instances."""
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
        b.step(steps)  # warm-up: captures the graphs
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
            s64.init_equilibrium(torch.from_numpy(inputs.sw_fourier_2d(nx, ny, seed=1000 + i)).to(dev))
            s64.step(steps)
            ref = s64.moments()
            s64.close()
            errs.append(float(torch.linalg.vector_norm(fp32[i][0] - ref[0]) / torch.linalg.vector_norm(ref[0])))
        b.close()
        # reverse mode on a bounded sample of the instances
        gs = sizes[:grad_instances]
        gb = eslbm.Batch(cfg, gs, stream=stream, device=dev)
        gu0 = gb.pack([inputs.sw_fourier_2d(nx, ny, seed=1000 + i) for i, (nx, ny) in enumerate(gs)])
        target = gb.pack([inputs.sw_fourier_2d(nx, ny, seed=5000 + i) for i, (nx, ny) in enumerate(gs)])
        torch.cuda.synchronize(dev)
        tf = time.perf_counter()
        gb.init_equilibrium(gu0)
        gb.step(grad_n)
        uT = gb.moments_flat()
        torch.cuda.synchronize(dev)
        fwd_s = time.perf_counter() - tf
        lam = torch.zeros_like(uT)
        for v, (u, t) in enumerate(zip(gb.unpack(uT), gb.unpack(target))):
            gb.unpack(lam)[v][0] = 2.0 * (u[0] - t[0])  # dJ/dh_T of J = sum (h_T - target)^2
        torch.cuda.synchronize(dev)
        ta = time.perf_counter()
        grad = gb.gradient(gu0, lam, grad_n, grad_K)
        torch.cuda.synchronize(dev)
        adj_s = time.perf_counter() - ta
        gnorm = float(torch.linalg.vector_norm(grad))
        gb.close()
    return {"batched": {"instances": count, "total_cells": cells, "sizes": "seeded uniform nx, ny in [256, 1024]",
                        "steps": steps, "ms": ms, "site_updates_per_s": cells * steps / (ms * 1e-3),
                        "schedule": {"segment": sched[0], "blocks_per_sm": sched[1], "order": sched[2]},
                        "tune_s": tune_s, "cuda_graph": True, "fallbacks": fallbacks, "V": BATCH_V,
                        "storage": "fp32, shifted, u_ref = (1, 0, 0)",
                        "rel_l2_h_vs_fp64": {"instances": [list(sizes[0]), list(sizes[1])], "values": errs},
                        "adjoint": {"instances": grad_instances, "steps": grad_n, "checkpoint_every": grad_K,
                                    "forward_s": fwd_s, "gradient_s": adj_s, "ratio": adj_s / fwd_s,
                                    "grad_norm": gnorm}}}


def hbm2d_leg(torch, eslbm, inputs, stream, dev, steps=20, only=None):
    """Per-stage streaming rate of the 2D stage kernel (one fused pull-shift + relax launch per stage,
    every distribution read and written once): D2Q4 Burgers 4096^2 FP32 (32 B per cell-stage) with
    omega = 2 and with the entropic omega, and D2Q4 Euler 8192^2 FP32 (128 B per cell-stage) with
    omega = 2 and scheme III (the paper's Euler setting).  Inputs are larger than L2 (268 MB and
    4.3 GB per state buffer), so every stage streams from HBM."""
    peak, kind = peaks()
    cases = [("burgers2d_4096_fixed", 2, "burgers", 4096, dict(V=3.0, c=(1.0, 1.0)), "fixed", "I", steps,
              lambda n: inputs.burgers_2d(n, n)),
             ("burgers2d_4096_entropic", 2, "burgers", 4096, dict(V=3.0, c=(1.0, 1.0)), "entropic", "I", steps,
              lambda n: inputs.burgers_2d(n, n)),
             ("euler2d_8192_fixed", 2, "euler", 8192, dict(V=8.0, gamma=1.4), "fixed", "III", max(1, steps // 10),
              lambda n: inputs.euler_vortex_2d(n, n))]
    out = {}
    for name, dim, system, n, kw, mode, scheme, nsteps, init in cases:
        if only and name != only:
            continue
        cfg = eslbm.make_config(dim, system, n, n, precision="fp32", omega_mode=mode, scheme=scheme, **kw)
        with torch.cuda.stream(stream):
            sim = eslbm.Simulation(cfg, stream=stream, device=dev)
            sim.use_graph(True)
            u0 = torch.from_numpy(init(n)).to(dev)
            sim.init_equilibrium(u0)
            del u0
            sim.step(1)  # warm-up and graph capture
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(nsteps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            stages = nsteps * int(sim.sizes.stages_per_step)
            bytes_stage = 2 * int(sim.sizes.state_bytes)
            fb = int(sim.diagnostics()["fallbacks"])
            sim.close()
        stage_s = ms * 1e-3 / stages
        out[name] = {"cells": n * n, "steps": nsteps, "stages": stages, "stage_us": stage_s * 1e6,
                     "bytes_per_stage": bytes_stage, "achieved_gbs": bytes_stage / stage_s / 1e9,
                     "frac_of_hbm_peak": bytes_stage / stage_s / 1e9 / peak, "peak_gbs": peak, "peak_source": kind,
                     "site_updates_per_s": n * n * nsteps / (ms * 1e-3), "fallbacks": fb,
                     "kernel": "%s<%s, 2, float, %s>" % ("k_stage_bulk" if n % 4 == 0 else "k_stage", system, mode)}
    return {"hbm2d": out}


if __name__ == "__main__":
    main()
