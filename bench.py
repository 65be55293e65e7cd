"""Benchmark: batched forward + adjoint gradient of the RT CNOP hot path.

Workload (one step, the default): rt_gradient on a batch of 32 instances of
the 256x768 Rayleigh-Taylor box (gamma 1.4, g_y -0.1, rho 2 over 1, h_s 0.01,
p 2.5 at y = 0, periodic x / reflecting y, PLM minmod + HLLC + SSP-RK2,
CFL 0.4), horizon T = 2.0, FP32 state with FP64 reductions, seeded i.i.d.
(vx, vy) perturbations scaled to C = 1e-4, sqrt(N) checkpointing. One step
is one gradient evaluation of every instance: forward to T, recomputation,
adjoint.

Metric: cell-updates/s of forward+adjoint (cells x RK2 steps of all
instances / device time of the gradient call). Also reported: gradient
evaluations/s, the same metric end to end through the C ABI with host
buffers, an FP64 single-instance gradient at the same horizon, the roofline
of the dominant kernel, and the FP64 CPU oracle's rate on a bounded sample
(all host cores, and one core).

Other configurations (--config):
  uneven64  64 instances of uneven grids (32 x 128x384, 24 x 256x768,
            8 x 512x1536), T = 2, delta cycling over 1e-5, 1e-4, 1e-3;
  hires     one 1024x3072 instance, T = 6 (about 58k steps), revolve
            checkpointing capped at 40 GB.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--config default|uneven64|hires]
Under torchrun every rank runs its own batch (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rt_inputs as I  # noqa: E402

NX, NY = 256, 768
T_HORIZON = 2.0
DELTA = 1e-4
METRIC = "cell-updates/s fwd+adjoint; CNOP gradient evals/s at 256x768, batch 32, vs FP64"
UNIT = "cell-updates/s"
# algorithmic bytes per cell per adjoint launch (FP32): stage-2 adjoint reads
# U1, lam^{n+1}, writes lam1 (12 s); stage-1 adjoint reads U^n, lam1,
# lam^{n+1}, writes lam^n (16 s); s = 4 bytes; the two launches of a step
# alternate, so the mean is 14 s.
ADJ_BYTES_PER_CELL = {"stage2_adjoint": 12 * 4, "stage1_adjoint": 16 * 4, "mean": 14 * 4}
# DRAM traffic of k_adjoint<float, minmod> per cell per launch (read + write),
# from one ncu capture of 16 instances of the benchmark grid (traffic grows in
# proportion to the cells); None while the kernel differs from the profiled one.
ADJ_TRAFFIC_BYTES_PER_CELL = 49.62
STEP_BYTES_PER_CELL_UPDATE = 68 * 4  # forward 20s + segment recompute 20s (U1 kept) + adjoint 12s + 16s (sqrt checkpointing)
# Warp instructions k_adjoint<float, minmod> executes per cell per launch
# (ncu sm__inst_executed.sum / cells, 16 instances of the benchmark grid, mean
# of the two adjoint stages). The kernel is bound by instruction issue: the
# issue roofline divides its executed instructions per second by the issue
# peak of 148 SMs x 4 schedulers x 1 warp instruction per clock at the
# sampled SM clock.
ADJ_WARP_INSTR_PER_CELL = 34.95
ISSUE_PER_SM_PER_CLK = 4
KERNEL_TIMING_EVERY = 8


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return summarise_clocks(list(self.rows))


def summarise_clocks(rows):
    """Median SM clock under load, the highest max-clock reading and the
    throttle reasons seen, from nvidia-smi rows (index, clocks.sm,
    clocks.max.sm, power.draw, active mask, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap). Non-numeric clock fields are skipped."""
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- configurations
class Config:
    """A benchmark workload: the problems of one rank's batch, each instance's
    seed and budget, and the context options."""

    def __init__(self, name, workload, problems, seeds, deltas, ckpt, cap_bytes=0.0):
        self.name, self.workload = name, workload
        self.problems, self.seeds, self.deltas = problems, seeds, deltas
        self.ckpt, self.cap_bytes = ckpt, cap_bytes


def make_config(name, rank):
    import paper_2608_04085_b300 as rt
    if name == "default":
        n = 32
        return Config(name, "rt-box 256x768 x32 instances, T=2.0, FP32 state + FP64 reductions, rt_gradient "
                            "(fwd+ckpt recompute+adjoint)",
                      [I.single_256().replace(T=T_HORIZON) for _ in range(n)],
                      list(range(rank * n, rank * n + n)), [DELTA] * n, rt.RT_CKPT_SQRT)
    if name == "uneven64":
        grids = [(128, 384)] * 32 + [(256, 768)] * 24 + [(512, 1536)] * 8
        deltas = [(1e-5, 1e-4, 1e-3)[i % 3] for i in range(64)]
        return Config(name, "rt-box uneven batch: 32 x 128x384 + 24 x 256x768 + 8 x 512x1536, T=2.0, "
                            "delta cycling 1e-5/1e-4/1e-3, FP32 state + FP64 reductions, rt_gradient",
                      [I.rt_box(nx, ny, T=2.0) for nx, ny in grids], list(range(rank * 64, rank * 64 + 64)),
                      deltas, rt.RT_CKPT_SQRT)
    if name == "hires":
        return Config(name, "rt-box 1024x3072 x1 instance, T=6.0, FP32 state + FP64 reductions, revolve "
                            "checkpointing capped at 40 GB, rt_gradient",
                      [I.rt_box(1024, 3072, T=6.0)], [rank], [DELTA], rt.RT_CKPT_REVOLVE, 40e9)
    raise ValueError(name)


def config_inputs(cfg):
    """Seeded (vx, vy) fields of the batch, instance after instance."""
    return np.concatenate([I.gaussian_field(s, 2, w.ny, w.nx).ravel() for s, w in zip(cfg.seeds, cfg.problems)])


def reduce_timing(ms_total, cells_total, world, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the cell
    updates); identity on one rank. Weak scaling: every rank advances its
    own batch, so the only collective is this reduction of two scalars."""
    if world <= 1:
        return ms_total, cells_total
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_total, cells_total], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def host_cpu():
    """The host the CPU baseline ran on: logical CPUs and the CPU model name
    (None where /proc/cpuinfo does not say)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"host_cpus": os.cpu_count(), "cpu_model": model}


def cpu_oracle_sample(n_steps, threads):
    """FP64 CPU oracle on a bounded sample of the workload: one 256x768
    instance, n_steps CFL steps forward plus the reverse sweep, on `threads`
    host threads (the oracle's row loops; the same values for any count).
    Returns (cell-updates/s, seconds, threads used, sample description)."""
    import oracle
    oracle.set_threads(threads)
    w = I.single_256().replace(nsteps=n_steps)
    v = oracle.scale_to_budget(w, I.gaussian_field(0, 2, NY, NX), DELTA)
    t0 = time.perf_counter()
    out = oracle.forward(w, v)
    oracle.gradient(w, v, out["dt"])
    dt = time.perf_counter() - t0
    used = oracle.get_threads()
    oracle.set_threads(1)
    cells = NX * NY * out["nsteps"]
    return cells / dt, dt, used, (f"1 instance 256x768 FP64, {out['nsteps']} CFL steps forward + reverse sweep, "
                                  f"{used} thread(s)")


def all_cores():
    import oracle
    return max(1, oracle.num_procs())


def cpu_baseline_block():
    """The oracle's rate on all host cores (value) and on one core."""
    n = all_cores()
    rate, secs, used, desc = cpu_oracle_sample(50, n)
    r1, s1, _, d1 = cpu_oracle_sample(4, 1)
    return {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc, "seconds": secs,
            "single_core": {"value": r1, "sample": d1, "seconds": s1}, **host_cpu()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n = all_cores()
    for _ in range(args.warmup):
        cpu_oracle_sample(2, n)
    vals, secs = [], 0.0
    desc, used = "", n
    for _ in range(args.steps):
        v, s, used, desc = cpu_oracle_sample(2, n)
        vals.append(v)
        secs += s
    value = float(np.mean(vals))
    cfg_workload = "rt-box 256x768 x32 instances, T=2.0, FP32 state + FP64 reductions, rt_gradient"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg_workload + " (oracle: bounded sample per step)", "grid": [NX, NY],
                   "T": T_HORIZON},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc,
                         **host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def fp64_single_instance(v_first, steps_fp32):
    """FP64 single-instance gradient of the benchmark grid at the full
    horizon (instance 0's input): one warm-up call, one timed call."""
    import paper_2608_04085_b300 as rt
    p64 = [I.single_256().replace(T=T_HORIZON)]
    with rt.Context(p64, precision=rt.RT_FP64, ckpt=rt.RT_CKPT_SQRT) as c64:
        v64 = v_first[: c64.total].copy()
        c64.gradient(v64)
        _, _, s64 = c64.gradient(v64)
    rate64 = s64["cell_updates"] / (s64["ms"] * 1e-3)
    return {"cell_updates_per_s": rate64, "steps": s64["steps"], "T": T_HORIZON, "ms": s64["ms"],
            "grad_evals_per_s": 1e3 / s64["ms"], "measured": "full horizon, one timed gradient"}


def run_ours(args):
    import torch
    import paper_2608_04085_b300 as rt

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    cfg = make_config(args.config, rank)
    n_inst = len(cfg.problems)
    xi = config_inputs(cfg)
    ctx = rt.Context(cfg.problems, precision=rt.RT_FP32_STATE, ckpt=cfg.ckpt, ckpt_cap_bytes=cfg.cap_bytes)
    # scale each instance onto C = delta (Eq. constraint) with the library's projection kernel
    v_host = ctx.project(xi, cfg.deltas, to_budget=True)
    # the stage-kernel variant the autotuner kept, and its timings
    variant, tuning = ctx.stage_kernel()
    stage_name = {rt.RT_STAGE_SWEEP: "sweep", rt.RT_STAGE_TILE8: "tile8", rt.RT_STAGE_TILE: "tile",
                  rt.RT_STAGE_TILE32: "tile32"}.get(variant, str(variant))
    stage_tuning = {k: round(float(t), 4) for k, t in tuning.items()}
    adj_rows, adj_t = ctx.adjoint_rows()
    adj_tuning = {str(k): round(float(t), 4) for k, t in adj_t.items()}
    v_dev = torch.from_numpy(v_host).to(dev)
    g_dev = torch.empty_like(v_dev)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.gradient(v_dev, out=g_dev)
    # timed region: kernel-timing instrumentation off, CUDA graphs on
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ms_total, cells_total, launches, segs = 0.0, 0.0, 0, []
    for _ in range(args.steps):
        J, _, st = ctx.gradient(v_dev, out=g_dev)
        ms_total += st["ms"]
        cells_total += st["cell_updates"]
        launches += st["launches"]
        segs.append(st["segments"])
    barrier()
    clk = clocks.stop()
    steps_run = st["steps"]
    cells_per_step = st["cell_updates"]

    # per-kernel launch times: a separate gradient of the same workload with
    # every KERNEL_TIMING_EVERY-th time-step launch bracketed by CUDA events
    ctx.set_kernel_timing(KERNEL_TIMING_EVERY)
    ctx.gradient(v_dev, out=g_dev)
    ktimes = ctx.kernel_times()
    ctx.set_kernel_timing(0)

    # end to end through the C ABI with host buffers in pinned memory (the
    # host-to-device copy of v and the device-to-host copy of the gradient and
    # J happen inside every call)
    v_pin = torch.from_numpy(v_host).pin_memory()
    g_pin = torch.zeros(ctx.total, dtype=torch.float64).pin_memory()
    e2e_s = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        _, _, st_h = ctx.gradient(v_pin, out=g_pin)
        e2e_s.append(time.perf_counter() - t0)
    e2e_rate = st_h["cell_updates"] / statistics.mean(e2e_s)

    t_max, cells_total = reduce_timing(ms_total, cells_total, world, dev)

    fp64 = None
    if rank == 0 and args.config == "default" and not args.no_fp64:
        fp64 = fp64_single_instance(v_host, steps_run)

    if rank == 0:
        value = cells_total / (t_max * 1e-3)
        grad_evals = n_inst * world * args.steps / (t_max * 1e-3)
        peak, peak_kind = measured_peaks()
        adj_ms, _, adj_launches = ktimes["adjoint"]
        st1_ms, st2_ms = ktimes["stage1"][0], ktimes["stage2"][0]
        # cells swept by one adjoint launch, on average: every reverse step
        # runs two adjoint launches over the cells of the instances still active
        cells_per_adj_launch = 2.0 * cells_per_step / adj_launches
        sm_max = clk.get("sm_max_mhz") or 2032.0  # fallback: B300 maximum SM clock
        fma32, fma64 = rt.fma_peak()  # measured FMA throughput, outside the timed region
        issue_peak = 148 * ISSUE_PER_SM_PER_CLK * sm_max * 1e6
        achieved = ADJ_BYTES_PER_CELL["mean"] * cells_per_adj_launch / (adj_ms * 1e-3) / 1e9
        traffic = (ADJ_TRAFFIC_BYTES_PER_CELL * cells_per_adj_launch
                   if ADJ_TRAFFIC_BYTES_PER_CELL is not None else None)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg.workload, "name": cfg.name, "instances_per_gpu": n_inst,
                       "grids": sorted({(w.nx, w.ny) for w in cfg.problems}),
                       "T": sorted({w.T for w in cfg.problems}), "rk2_steps_max": steps_run,
                       "checkpointing": {rt.RT_CKPT_SQRT: "sqrt(N)", rt.RT_CKPT_REVOLVE: "revolve"}[cfg.ckpt],
                       "checkpoint_cap_bytes": cfg.cap_bytes or None,
                       "l2": "working set > L2 (no flush)",
                       "stage_kernel": stage_name, "stage_tuning_ms_per_step": stage_tuning,
                       "adjoint_tile_rows": adj_rows, "adjoint_tuning_ms_per_launch": adj_tuning,
                       "tile_loads": "tma"},
            "grad_evals_per_s": grad_evals,
            "e2e": {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(ctx.total * 8),
                    "d2h_bytes_per_step": int(ctx.total * 8 + n_inst * 8), "calls": len(e2e_s),
                    "seconds_per_call": statistics.mean(e2e_s), "host_buffers": "pinned"},
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": {"bound": "hbm", "kernel": "k_adjoint<float>", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_kind + " hbm_gbs",
                         "algorithmic_bytes_per_cell": ADJ_BYTES_PER_CELL["mean"],
                         "cells_per_launch": cells_per_adj_launch,
                         "mean_launch_ms": {"adjoint": adj_ms, "stage1": st1_ms, "stage2": st2_ms},
                         "launch_times": "CUDA events around every %dth time-step launch of one gradient "
                                         "run after the timed region (same stream, graphs bypassed)"
                                         % KERNEL_TIMING_EVERY},
            "issue_roofline": {"bound": "issue", "kernel": "k_adjoint<float>",
                               "achieved": ADJ_WARP_INSTR_PER_CELL * cells_per_adj_launch / (adj_ms * 1e-3),
                               "peak": issue_peak, "unit": "warp-instr/s",
                               "frac": ADJ_WARP_INSTR_PER_CELL * cells_per_adj_launch / (adj_ms * 1e-3)
                               / issue_peak,
                               "warp_instr_per_cell": ADJ_WARP_INSTR_PER_CELL,
                               "peak_source": "148 SMs x 4 issue/clk x %.0f MHz (sampled max SM clock)" % sm_max,
                               "measured_fma_tflops": {"f32": fma32, "f64": fma64}},
            "step_roofline": {"bytes_per_cell_update": STEP_BYTES_PER_CELL_UPDATE,
                              "achieved_gbs": value * STEP_BYTES_PER_CELL_UPDATE / 1e9,
                              "frac": value * STEP_BYTES_PER_CELL_UPDATE / 1e9 / peak},
        }
        if cfg.ckpt == rt.RT_CKPT_REVOLVE:
            line["revolve_recomputed_steps"] = -segs[-1]
        if fp64:
            line["fp64_single_instance"] = fp64
            line["speedup_vs_fp64_single"] = grad_evals / world / fp64["grad_evals_per_s"]
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline_block()
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """Small case for ncu captures: 16 instances of the benchmark grid with a
    short horizon (T = 0.01, about 25 RK2 steps), the benchmark's sqrt(N)
    checkpointing and its stage kernel (32-row tiles), so one gradient
    launches the same kernel mix as a benchmark step (about 130 launches
    instead of about 29,000); about 1 GB on the device, each kernel's working
    set (4 x 50 MB) still larger than L2."""
    import paper_2608_04085_b300 as rt
    nb = 16
    probs = [I.single_256().replace(T=0.01) for _ in range(nb)]
    # the tile variant with 32-row tiles, which the autotuner keeps for the
    # benchmark batch: under a profiler the autotuner's timings are distorted
    # and could pick another
    with rt.Context(probs, precision=rt.RT_FP32_STATE, ckpt=rt.RT_CKPT_SQRT, stage_kernel=rt.RT_STAGE_TILE32) as ctx:
        v = ctx.project(I.gaussian_batch(range(nb), 2, NY, NX).reshape(-1), DELTA, to_budget=True)
        for k in range(3):
            ctx.set_kernel_timing(1 if k == 2 else 0)
            _, _, st = ctx.gradient(v)
            rec = {"profile_case": k, **st}
            if k == 2:
                rec["kernel_ms"] = {name: t[0] for name, t in ctx.kernel_times().items()}
            print(json.dumps(rec), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["default", "uneven64", "hires"], default="default")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 single-instance gradient")
    ap.add_argument("--profile-case", action="store_true", help="short-horizon case sized for ncu captures")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
