"""Benchmark: u-series energy + forces + potentials on the membrane-shaped slab.

One step = one evaluation of the ~64,000-charge membrane slab (80 x 80 x 100 A,
64 x 64 x 80 grid, C1 b = 2 series) at every cutoff of the sweep
r_c = 8, 9, 10, 11, 12, 13 A, inputs resident in HBM.  value = atom-evals/s
(charges x evaluations / second, device time from CUDA events on the
evaluation stream, L2 flushed between steps by writing a 512 MB buffer).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torch.distributed.run): every rank evaluates its own replica of
the workload (independent systems, no collective), value sums all ranks over
the slowest rank's time.  --impl reference times the FP64 oracle on the host
cores instead (the reference arm).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "u-series E+F atom-evals/s at rms rel force err ≤1e-4; serving p50/p99 ms"
UNIT = "atom-evals/s"
WORKLOAD = "membrane_slab"
SWEEP = (8.0, 9.0, 10.0, 11.0, 12.0, 13.0)
KERNELS_PER_EVAL = 10          # bin_count, scan, place, cell_sort, near, spread, conv x/y/z, gather
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
FLOPS_PER_PAIR = 2 * 12 + 20   # Horner value+derivative (degree 12) + rsqrt/Newton, 1/r^3, accumulation


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_oracle_eval(w, r_c, targets=None):
    import oracle as O
    from paper_1911_01377_gb300 import usr
    s = usr.usr_series_preset("C1_B2")
    return O.evaluate(O.Series(s.b, s.r0, s.w0, s.s0), r_c, w.box, w.xyzq[:, :3], w.xyzq[:, 3], targets=targets)


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, bounded samples."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from paper_1911_01377_gb300 import workloads as W
    w = W.get(WORKLOAD)
    rng = np.random.default_rng(7)
    n_t = 2048
    times = []
    for step in range(args.warmup + args.steps):
        r_c = SWEEP[step % len(SWEEP)]
        targets = rng.choice(w.n, size=n_t, replace=False)
        t0 = time.perf_counter()
        cpu_oracle_eval(w, r_c, targets=targets)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n_t * len(times) / total
    sample = (f"FP64 oracle (direct near sum + exact k-space far sum) on {W.get(WORKLOAD).n} charges, "
              f"forces+potentials for {n_t} random target atoms per step, r_c cycling {SWEEP[0]:g}-{SWEEP[-1]:g} A")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " 63,996 charges, 80x80x100 A, r_c 8-13 A"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1911_01377_gb300 import build as B
    B.build()
    import oracle as O
    from paper_1911_01377_gb300 import usr
    from paper_1911_01377_gb300 import workloads as W

    w = W.get(WORKLOAD)
    n = w.n
    x = torch.from_numpy(w.xyzq).to(dev)
    ctxs = [usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=n) for r_c in SWEEP]
    outs = [torch.empty((n, 4), dtype=torch.float32, device=dev) for _ in SWEEP]
    ens = [torch.empty(4, dtype=torch.float64, device=dev) for _ in SWEEP]
    # algorithmic pair counts (unique pairs within r_c) per cutoff, outside the timed region
    pairs = []
    for c in ctxs:
        cnt, _ = c.debug_pairs(x)
        pairs.append(int(cnt.sum().item()) // 2)
    for c in ctxs:
        usr.usr_set_profiling(c.ctx, True)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        for c, o, e in zip(ctxs, outs, ens):
            usr.usr_eval(c.ctx, n, x.data_ptr(), o.data_ptr(), e.data_ptr(), stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    for c in ctxs:
        if usr.usr_last_device_status(c.ctx) != 0:
            raise RuntimeError("device status error during warm-up")

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    sampler = ClockSampler(ids[local] if local < len(ids) else str(local))
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stage_ms = [[0.0] * usr.USR_NSTAGES for _ in SWEEP]
    step_ms = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(float(_ % 7))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, c in enumerate(ctxs):
            for s, v in enumerate(usr.usr_stage_times(c.ctx)):
                stage_ms[k][s] += v
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    evals = n * len(SWEEP) * args.steps * ws
    value = evals / (total_ms / 1e3)

    # end to end through the host-buffer entry point (pinned memory, copies inside)
    xh = torch.from_numpy(w.xyzq).pin_memory()
    oh = [torch.empty((n, 4), dtype=torch.float32).pin_memory() for _ in SWEEP]
    eh = [torch.empty(4, dtype=torch.float64).pin_memory() for _ in SWEEP]
    for c in ctxs:
        usr.usr_set_profiling(c.ctx, False)
    for _ in range(max(1, args.warmup)):
        for c, o, e in zip(ctxs, oh, eh):
            usr.usr_eval_host(c.ctx, n, xh.data_ptr(), o.data_ptr(), e.data_ptr(), stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for c, o, e in zip(ctxs, oh, eh):
            usr.usr_eval_host(c.ctx, n, xh.data_ptr(), o.data_ptr(), e.data_ptr(), stream)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(t.item())
    e2e_value = evals / t_e2e

    if rank != 0:
        return
    # per-stage averages and the dominant kernel's roofline
    per_stage = [sum(stage_ms[k][s] for k in range(len(SWEEP))) / (len(SWEEP) * args.steps)
                 for s in range(usr.USR_NSTAGES)]
    dom = max(range(usr.USR_NSTAGES), key=lambda s: per_stage[s])
    infos = [c.info for c in ctxs]
    G = w.grid[0] * w.grid[1] * w.grid[2]
    P = 12

    def stage_flops(s, k):
        inf = infos[k]
        if usr.STAGES[s] == "near":
            return pairs[k] * FLOPS_PER_PAIR
        if usr.STAGES[s].startswith("conv"):
            ax = "xyz".index(usr.STAGES[s][-1])
            return 2.0 * G * inf.n_terms * w.grid[ax]
        if usr.STAGES[s] in ("spread", "gather"):
            return n * P ** 3 * (2 if usr.STAGES[s] == "spread" else 8)
        return None

    flops = [stage_flops(dom, k) for k in range(len(SWEEP))]
    roof = None
    if flops[0] is not None:
        t_dom = [stage_ms[k][dom] / args.steps for k in range(len(SWEEP))]
        achieved = sum(flops) / (sum(t_dom) / 1e3) / 1e12
        roof = {"kernel": usr.STAGES[dom], "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz max SM clock"}

    # CPU baseline: the FP64 oracle, one full evaluation at r_c = 8 A, also giving the error
    import numpy as np  # noqa: F811
    t0 = time.perf_counter()
    ref = cpu_oracle_eval(w, SWEEP[0])
    t_cpu = time.perf_counter() - t0
    g_out = outs[0].double().cpu().numpy()
    g_E = float(ens[0][0].item())
    err_f = O.rms_rel(g_out[:, :3], ref.F)
    err_e = abs(g_E / ref.E - 1.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: {n} charges (2133 12-bead chains + 12800 waters), "
                               f"80x80x100 A, 64x64x80 grid, C1 b=2, r_c sweep 8-13 A (6 evals/step)",
                   "global_batch": n * len(SWEEP) * ws, "parallelism": f"replicas x{ws}",
                   "l2": "flushed between steps (512 MB write)", "wall_s_timed": t_wall},
        "roofline": roof,
        "stage_ms_mean": dict(zip(usr.STAGES, per_stage)),
        "accuracy_rc8": {"rms_force_rel_err": err_f, "energy_rel_err": err_e},
        "cpu_baseline": {"value": n / t_cpu, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"one full FP64 oracle evaluation (E, all forces and potentials) of the "
                                   f"{n}-charge slab at r_c = 8 A, {t_cpu:.1f} s"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * n * len(SWEEP),
                "d2h_bytes_per_step": (16 * n + 32) * len(SWEEP)},
        "clocks": clocks,
        "gpu_launches": KERNELS_PER_EVAL * len(SWEEP) * args.steps,
        "pairs_per_rc": dict(zip([str(r) for r in SWEEP], pairs)),
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
