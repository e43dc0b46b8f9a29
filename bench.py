"""Throughput of the BaB-ND bounding hot path on GB300.

One step = one branch-and-bound iteration (Algorithm 2) on the pushing-scale
workload: prune the pool against the FP64 incumbent, pick out 2048 boxes and
bisect them (4096 children), search every child with 1024 uniform rollouts of
H = 20 steps (upper bounds, FP64 re-score of the best plan), and bound every
child from below (interval bounds + CROWN + concretization, outward margin).
All of it runs in libbab's kernels through the C-ABI binding; the pool stays
in device memory and the iteration chains its calls through device counts,
with no host synchronisation.

Metric: CROWN subdomain-bounds/s (children bounded per second, whole job);
rollout-steps/s is reported beside it.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.

Multi-GPU (torchrun): each rank runs an independent planning problem (seed +
rank) on its own GPU; no data-path collective; value = all ranks' boxes / the
slowest rank's time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pushing"
N_PICK = 2048          # parents per iteration -> 4096 children bounded per iteration (--boxes changes it)
SEED = 2024
METRIC = "CROWN subdomain-bounds/s & rollout-steps/s at H=20"
PRECISION = "bf16x3"   # rollout arithmetic (--precision)


def workload_config():
    from paper_2412_09584_gb300 import workloads as W
    c = W.CONFIGS[WORKLOAD]
    return {"workload": "pushing-scale BaB iteration: state 8, action 2, MLP 10-128-128-128-8 ReLU residual, H=20, "
                        "rho=0.01, 4096 children bounded per iteration (2048 picked, widest-dim bisection), "
                        "1024 uniform rollouts per child",
            "rollout_arithmetic": {"fp32": "FP32 CUDA cores", "bf16x3": "tcgen05, 3-term BF16 split, FP32 accumulate",
                                   "bf16": "tcgen05, BF16 operands, FP32 accumulate, FP32 re-score"}[PRECISION],
            "bound_arithmetic": "FP32 CUDA cores, outward-rounded intervals, margin-corrected CROWN",
            "boxes_per_step": 2 * N_PICK, "samples_per_box": c["samples"], "H": c["H"],
            "initial_pool": "4096-box grid over [-1,1]^40", "l2": "flushed between steps (256 MiB write)"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        for line in open(self.file.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


PRECISIONS = {"fp32": 0, "bf16x3": 1, "bf16": 2}


def fp32_alu_peak_tflops(sm_mhz):
    """Dense FP32 FMA peak: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class BabIteration:
    """Device-resident BaB state and one iteration = prune/pick/split, rollouts, bounds."""

    def __init__(self, seed, device):
        import torch
        from paper_2412_09584_gb300 import binding as B
        from paper_2412_09584_gb300 import workloads as W
        self.torch, self.B = torch, B
        self.dev = device
        c = W.CONFIGS[WORKLOAD]
        self.p = W.config_problem(WORKLOAD, seed)
        self.H, self.rho, self.M = c["H"], c["rho"], c["samples"]
        self.d = self.p["k"] * self.H
        self.nb = 2 * N_PICK
        self.seed = seed
        self.ctx = B.bab_load_dynamics(self.p["dims"], self.p["params"], self.p["s"], self.p["k"])
        f = dict(device=device, dtype=torch.float32)
        self.x0 = torch.as_tensor(self.p["x0"]).to(**f)
        self.goal = torch.as_tensor(self.p["goal"]).to(**f)
        lo, hi, ids = W.grid_boxes(self.d, int(np.log2(self.nb)))  # 4096 boxes = the 12-level grid
        self.cap = 4096 + 64 * N_PICK  # enough for 60+ iterations of pool growth
        self.pool = [self._alloc(), self._alloc()]
        self.cur = 0
        P = self.pool[0]
        n0 = lo.shape[0]
        P["lo"][:n0] = torch.as_tensor(lo).to(**f)
        P["hi"][:n0] = torch.as_tensor(hi).to(**f)
        P["id"][:n0] = torch.as_tensor(ids.astype(np.int64)).to(device)
        self.n_max = n0
        self.best_u = torch.empty(max(self.nb, n0), self.d, **f)
        self.keep = torch.empty(self.cap, dtype=torch.uint8, device=device)
        self.counts = torch.zeros(3, dtype=torch.int32, device=device)
        self.inc_val = torch.full((1,), float("inf"), dtype=torch.float64, device=device)
        self.inc_u = torch.zeros(self.d, **f)
        self.margin = torch.empty(max(self.nb, n0), **f)
        self.n_live_dev = torch.tensor([n0], dtype=torch.int32, device=device)
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
        # initial search and bound of the starting pool (Algorithm 2, lines 2-3)
        self.search_and_bound(P, n0, None)
        self.launches_per_step = 2 + 4 + 2  # prune/branch 2, rollout 4, interval bounds + CROWN 2
        self.ev = []

    def _alloc(self):
        torch = self.torch
        f = dict(device=self.dev, dtype=torch.float32)
        return {"lo": torch.empty(self.cap, self.d, **f), "hi": torch.empty(self.cap, self.d, **f),
                "lb": torch.empty(self.cap, **f), "ub": torch.empty(self.cap, **f),
                "id": torch.empty(self.cap, dtype=torch.int64, device=self.dev)}

    def search_and_bound(self, P, n, d_n, time_rollout=False):
        B, torch = self.B, self.torch
        if time_rollout:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
        B.bab_rollout(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], P["id"], n, self.M,
                      self.seed, PRECISIONS[PRECISION], P["ub"], self.best_u, self.inc_val, self.inc_u, d_n=d_n)
        if time_rollout:
            e1.record()
            e2 = torch.cuda.Event(enable_timing=True)
        B.bab_bound_crown(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], n, P["lb"],
                          margin=self.margin, d_n=d_n)
        if time_rollout:
            e2.record()
            self.ev.append((e0, e1, e2))

    def step(self, timed=False):
        B = self.B
        src, dst = self.pool[self.cur], self.pool[self.cur ^ 1]
        B.bab_prune_branch(self.ctx, self.d, src["lo"], src["hi"], src["lb"], src["ub"], src["id"], self.n_max,
                           self.inc_val, N_PICK, 0.75, self.cap, dst["lo"], dst["hi"], dst["lb"], dst["ub"],
                           dst["id"], self.keep, self.counts, d_n=self.n_live_dev)
        self.n_max = min(self.n_max + N_PICK, self.cap - N_PICK)
        self.search_and_bound(dst, self.nb, self.counts[0:1], time_rollout=timed)
        self.n_live_dev.copy_(self.counts[2:3])
        self.cur ^= 1

    def flush_l2(self):
        self.flush.fill_(1.0)

    def close(self):
        self.B.bab_destroy(self.ctx)


def run_ours(args):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    it = BabIteration(SEED + rank, dev)
    for _ in range(args.warmup):
        it.step()
        it.flush_l2()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0.record()
        for _ in range(args.steps):
            it.step(timed=True)
            it.flush_l2()
        t1.record()
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    roll_ms = [a.elapsed_time(b) for a, b, _ in it.ev]
    crown_ms = [b.elapsed_time(c) for _, b, c in it.ev]
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    clocks = clk.summary()

    # end to end through the C-ABI: each step copies its batch of boxes in from pinned host memory and the
    # next batch plus the bounds and incumbent back out
    e2e = run_e2e(it, args.steps)
    inc = float(it.inc_val.item())
    it.close()

    boxes = it.nb * args.steps * ws
    value = boxes / (ms / 1e3)
    rsteps = boxes * it.M * it.H / (ms / 1e3)
    macs = sum(a * b for a, b in zip(it.p["dims"][1:], it.p["dims"][:-1]))
    flops_roll = 2.0 * it.nb * it.M * it.H * macs
    roll_avg = statistics.mean(roll_ms) / 1e3
    achieved = flops_roll / roll_avg / 1e12
    if PRECISION == "fp32":
        roof = {"kernel": "k_rollout_fp32 (bab_rollout)", "bound": "alu", "peak": fp32_alu_peak_tflops(2070.0),
                "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz max SM clock"}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        pk = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {"kernel": "k_rollout_tc (bab_rollout)", "bound": "tensor", "peak": pk,
                "peak_note": ("of measured bf16 sustained (MEASURED_PEAKS.json)" if peaks else "of fallback") +
                             "; achieved counts algorithmic FLOPs (2 x MACs of the network); the tensor pipe "
                             "executes " + ("3x that (3-term BF16 split)" if PRECISION == "bf16x3" else
                                            "the same (BF16 operands)") + " plus padding to multiples of 16"}
    roof.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / roof["peak"], "traffic": None})
    if rank != 0:
        return
    out = {"metric": METRIC, "value": value, "unit": "subdomain-bounds/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16x3", "bf16": "bf16"}[PRECISION],
           "data": "synthetic (seeded random network, start and goal)",
           "config": dict(workload_config(), parallelism=f"independent problems x{ws}" if ws > 1 else "single GPU"),
           "rollout_steps_per_s": rsteps,
           "kernel_ms": {"rollout": statistics.mean(roll_ms), "bound_crown": statistics.mean(crown_ms)},
           "crown_subdomain_bounds_per_s_kernel_only": it.nb / (statistics.mean(crown_ms) / 1e3),
           "incumbent_fp64": inc,
           "roofline": roof,
           "clocks": clocks, "e2e": e2e, "gpu_launches": it.launches_per_step * args.steps}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_e2e(it, steps):
    """Same iteration with the batch of boxes crossing the host boundary every step."""
    torch, B = it.torch, it.B
    nb, d = it.nb, it.d
    h_lo = torch.empty(nb, d, dtype=torch.float32, pin_memory=True)
    h_hi = torch.empty_like(h_lo, pin_memory=True)
    h_id = torch.empty(nb, dtype=torch.int64, pin_memory=True)
    h_lb = torch.empty(nb, dtype=torch.float32, pin_memory=True)
    h_ub = torch.empty_like(h_lb, pin_memory=True)
    h_inc = torch.empty(1, dtype=torch.float64, pin_memory=True)
    src = it.pool[it.cur]
    h_lo.copy_(src["lo"][:nb])
    h_hi.copy_(src["hi"][:nb])
    h_id.copy_(src["id"][:nb])
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        P = it.pool[it.cur]
        P["lo"][:nb].copy_(h_lo, non_blocking=True)
        P["hi"][:nb].copy_(h_hi, non_blocking=True)
        P["id"][:nb].copy_(h_id, non_blocking=True)
        it.search_and_bound(P, nb, None)
        h_lb.copy_(P["lb"][:nb], non_blocking=True)
        h_ub.copy_(P["ub"][:nb], non_blocking=True)
        dst = it.pool[it.cur ^ 1]
        B.bab_prune_branch(it.ctx, d, P["lo"], P["hi"], P["lb"], P["ub"], P["id"], it.n_max, it.inc_val, N_PICK,
                           0.75, it.cap, dst["lo"], dst["hi"], dst["lb"], dst["ub"], dst["id"], it.keep, it.counts,
                           d_n=it.n_live_dev)
        it.n_max = min(it.n_max + N_PICK, it.cap - N_PICK)
        it.n_live_dev.copy_(it.counts[2:3])
        h_lo.copy_(dst["lo"][:nb], non_blocking=True)
        h_hi.copy_(dst["hi"][:nb], non_blocking=True)
        h_id.copy_(dst["id"][:nb], non_blocking=True)
        h_inc.copy_(it.inc_val, non_blocking=True)
        it.cur ^= 1
        it.flush_l2()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    h2d = nb * (2 * d * 4 + 8)
    d2h = nb * (2 * 4) + nb * (2 * d * 4 + 8) + 8
    return {"value": nb * steps / (ms / 1e3), "unit": "subdomain-bounds/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def oracle_sample_step(problem, lo, hi, ids, M, n_roll, n_bound, pool_n):
    """The oracle on a bounded sample of one iteration: rollouts of n_roll boxes, bounds of n_bound boxes and
    prune/branch of a pool of pool_n boxes. Returns seconds per box for search and bound, and prune seconds."""
    from oracle import oracle as O
    t = time.perf_counter()
    O.rollout(problem, lo[:n_roll], hi[:n_roll], ids[:n_roll], M, SEED)
    t_roll = (time.perf_counter() - t) / n_roll
    t = time.perf_counter()
    O.crown(problem, lo[:n_bound], hi[:n_bound])
    t_bound = (time.perf_counter() - t) / n_bound
    rng = np.random.default_rng(0)
    lb = rng.normal(10, 3, pool_n).astype(np.float32)
    ub = (lb + 1).astype(np.float32)
    reps = (pool_n + lo.shape[0] - 1) // lo.shape[0]
    plo = np.tile(lo, (reps, 1))[:pool_n]
    phi = np.tile(hi, (reps, 1))[:pool_n]
    pid = np.arange(1, pool_n + 1, dtype=np.uint64)
    t = time.perf_counter()
    O.prune_branch(plo, phi, lb, ub, pid, 11.0, N_PICK)
    t_prune = time.perf_counter() - t
    return t_roll, t_bound, t_prune


def cpu_baseline(budget_s=20.0):
    from paper_2412_09584_gb300 import workloads as W
    c = W.CONFIGS[WORKLOAD]
    p = W.config_problem(WORKLOAD, SEED)
    lo, hi, ids = W.grid_boxes(c["H"] * p["k"], c["grid_dims"])
    # calibrate on one box, then size the sample to the budget
    t_roll, t_bound, t_prune = oracle_sample_step(p, lo, hi, ids, c["samples"], 1, 4, 4096)
    n_roll = max(1, min(64, int(0.7 * budget_s / max(t_roll, 1e-6))))
    n_bound = max(4, min(4096, int(0.2 * budget_s / max(t_bound, 1e-6))))
    t_roll, t_bound, t_prune = oracle_sample_step(p, lo, hi, ids, c["samples"], n_roll, n_bound, 4096 + N_PICK)
    step_s = 2 * N_PICK * (t_roll + t_bound) + t_prune
    return {"value": 2 * N_PICK / step_s, "unit": "subdomain-bounds/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 C oracle, single thread: rollouts of {n_roll} boxes x {c['samples']} samples x H={c['H']}, "
                      f"CROWN of {n_bound} boxes, prune/branch of a {4096 + N_PICK}-box pool; per-box times scaled to "
                      f"one {2 * N_PICK}-box iteration ({step_s:.1f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2412_09584_gb300 import workloads as W
    O.build()
    c = W.CONFIGS[WORKLOAD]
    p = W.config_problem(WORKLOAD, SEED)
    lo, hi, ids = W.grid_boxes(c["H"] * p["k"], c["grid_dims"])
    n_roll, n_bound = 2, 2
    for _ in range(args.warmup):
        oracle_sample_step(p, lo, hi, ids, c["samples"], n_roll, n_bound, 1024)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(p, lo, hi, ids, c["samples"], n_roll, n_bound, 1024)
    sec = (time.perf_counter() - t) / args.steps
    value = n_bound / sec
    sample = (f"per step: FP64 C oracle on {n_roll} boxes (1024 rollouts of H=20 each, then CROWN) and prune/branch "
              f"of a 1024-box pool, single thread")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "subdomain-bounds/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(),
           "cpu_baseline": {"value": value, "unit": "subdomain-bounds/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "subdomain-bounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    global N_PICK, PRECISION
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default=PRECISION,
                    help="rollout arithmetic: fp32 (CUDA cores), bf16x3 (tcgen05, 3-term split), bf16 (tcgen05)")
    ap.add_argument("--boxes", type=int, default=2 * N_PICK,
                    help="children bounded per iteration; smaller values make small cases for profiler captures")
    args = ap.parse_args()
    N_PICK = args.boxes // 2
    PRECISION = args.precision
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
