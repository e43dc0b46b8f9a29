"""Throughput of the BaB-ND bounding hot path on GB300.

One step = one branch-and-bound iteration (Algorithm 2) on the pushing-scale
workload: prune the pool against the FP64 incumbent, pick out 2048 boxes and
bisect them (4096 children), search every child with 1024 uniform rollouts of
H = 20 steps (upper bounds, FP64 re-score of the best plan), and bound every
child from below (interval bounds + CROWN + concretization, outward margin).
All of it runs in libbab's kernels through the C-ABI binding; the pool stays
in device memory, the iteration chains its calls through device counts with
no host synchronisation, and the timed steps replay the iteration as a CUDA
graph.

Metric: CROWN subdomain-bounds/s (children bounded per second, whole job);
rollout-steps/s is reported beside it, and a time-to-gap comparison (alpha-CROWN
with split precision vs plain FP32 CROWN+IBP BaB) on the 4096-box alpha
workload.  `--impl reference` times the FP64 CPU oracle on a bounded sample of
the same workload instead.

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

SEED = 2024
METRIC = "CROWN subdomain-bounds/s & rollout-steps/s at H=20"
PRECISIONS = {"fp32": 0, "bf16x3": 1, "bf16": 2}
BOUND_PRECISIONS = {"fp32": 0, "bf16x3": 1, "tf32x3": 3}
ARITH = {"fp32": "FP32 CUDA cores", "bf16x3": "tcgen05, 3-term BF16 split, FP32 accumulate",
         "bf16": "tcgen05, BF16 operands, FP32 accumulate, FP32 re-score of each box's pick",
         "tf32x3": "tcgen05, 3-term TF32 split, FP32 accumulate"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank):
    """Each rank plans its own independent problem (weak scaling, no data-path collective)."""
    return SEED + rank


def max_over_ranks(ms, device):
    """The slowest rank's time: the whole job takes as long as its last rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * ws / (ms / 1e3)


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
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # nvidia-smi takes a while to start: wait (at most 5 s) for its first row so the samples cover the
        # whole timed region that follows
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.file.name) > 0:
                break
            time.sleep(0.01)
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


_FP32_PEAK = None


def fp32_peak_measured():
    """The FP32 FMA rate measured on this GPU by the library's probe kernel (best of scalar and paired FMAs),
    TFLOP/s; measured once per process."""
    global _FP32_PEAK
    if _FP32_PEAK is None:
        from paper_2412_09584_gb300 import binding as B
        scalar, paired = B.bab_probe_fp32_peak()
        _FP32_PEAK = {"tflops": max(scalar, paired), "scalar": scalar, "paired": paired}
    return _FP32_PEAK


def bf16_peaks():
    """Measured BF16 GEMM rates of the GB300s (burst, sustained) in TFLOP/s, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        return pk.get("bf16_tflops", 1900.0), pk.get("bf16_tflops_sustained", 1700.0), "measured"
    return 1900.0, 1700.0, "fallback"


def rollout_roofline(precision, p, nb, M, H, roll_ms):
    """Roofline of the rollout kernel: algorithmic FLOPs (2 x the network's MACs per rollout-step) per launch over
    its CUDA-event duration, against the measured FP32 FMA rate (CUDA cores) or the measured BF16 burst rate (the
    kernel is timed on its own); for the tensor-core paths also what the pipe executes (3 MMAs per product for the
    3-term split, layers padded to multiples of 16)."""
    macs = sum(a * b for a, b in zip(p["dims"][1:], p["dims"][:-1]))
    achieved = 2.0 * nb * M * H * macs / (roll_ms / 1e3) / 1e12
    if precision == "fp32":
        pk = fp32_peak_measured()
        roof = {"kernel": "k_rollout_fp32 (bab_rollout)", "bound": "alu", "peak": pk["tflops"],
                "peak_note": "of measured FP32 FMA rate (bab_probe_fp32_peak on this GPU, best of scalar "
                             f"{pk['scalar']:.1f} and paired {pk['paired']:.1f} TFLOP/s)"}
    else:
        burst, _, kind = bf16_peaks()
        fused = precision == "bf16" and len(p["dims"]) >= 4
        roof = {"kernel": ("k_rollout_tcf" if fused else "k_rollout_tc") + " (bab_rollout)", "bound": "tensor",
                "peak": burst,
                "peak_note": f"of {kind} bf16 burst (MEASURED_PEAKS.json): the kernel is timed on its own with CUDA "
                             "events; achieved counts algorithmic FLOPs (2 x MACs of the network); the tensor pipe "
                             "executes " + ("3x that (3-term BF16 split)" if precision == "bf16x3" else "the same") +
                             " plus padding to multiples of 16" +
                             ("; the fused step (output layer and next first layer as one product over [a | u x], "
                              "the bias by one more K = 16 step) executes more" if fused else "")}
    roof.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / roof["peak"]})
    if precision != "fp32":
        dims = p["dims"]
        pad16 = lambda v: (v + 15) // 16 * 16
        L = len(dims) - 1
        K = [0] + [pad16(8 + p["s"] if l == 1 else dims[l - 1]) for l in range(1, L + 1)]
        Nn = [0] + [pad16(dims[l]) for l in range(1, L + 1)]
        if precision == "bf16" and L >= 3:
            # per rollout: layer 1 of step 0 once; per step layers 2 .. L-1 and the fused product, each with its
            # bias step (K + 16)
            per_step = sum((K[l] + 16) * Nn[l] for l in range(2, L)) + (K[L] + K[1] + 16) * (Nn[1] + Nn[L])
            ex = per_step + ((K[1] + 16) * Nn[1]) / H
        else:
            ex = sum(K[l] * Nn[l] for l in range(1, L + 1))
        ratio = (3 if precision == "bf16x3" else 1) * ex / macs
        roof.update({"executed_per_algorithmic": ratio, "executed": achieved * ratio,
                     "executed_frac": achieved * ratio / roof["peak"]})
    return roof


class BabState:
    """Device-resident BaB pool and one iteration: prune/pick/split, rollouts, bounds (plain or alpha-CROWN).

    Every call of an iteration reads its live counts from the device, so an iteration can be captured as a
    CUDA graph; with `fixed_launch` the pool calls are sized for the largest pool so every replay launches
    the same grids."""

    def __init__(self, workload, seed, device, n_pick, rollout_prec="bf16x3", bound_prec="fp32", alpha_steps=0,
                 alpha_lr=0.1, samples=None, fixed_launch=False, pool_iters=64, autotune=False, search_stop=None,
                 heuristics=None, cem=None, cost=None, interval_prec="fp32", rescore_topk=0):
        import torch
        from paper_2412_09584_gb300 import binding as B
        from paper_2412_09584_gb300 import workloads as W
        self.torch, self.B = torch, B
        self.dev = device
        c = W.CONFIGS[workload]
        self.p = W.config_problem(workload, seed)
        self.H, self.rho = c["H"], c["rho"]
        self.M = samples or c["samples"]
        self.d = self.p["k"] * self.H
        self.sumh = sum(self.p["dims"][1:-1])
        self.n_pick = n_pick
        self.nb = 2 * n_pick
        self.seed = seed
        self.rprec, self.bprec = PRECISIONS[rollout_prec], BOUND_PRECISIONS[bound_prec]
        self.alpha_steps, self.alpha_lr = alpha_steps, alpha_lr
        self.ctx = B.bab_load_dynamics(self.p["dims"], self.p["params"], self.p["s"], self.p["k"])
        self.iprec = interval_prec
        if interval_prec != "fp32":
            # interval bounds on tensor cores (3-term BF16 or TF32 split products with a computed margin)
            B.bab_set_interval_precision(self.ctx, BOUND_PRECISIONS[interval_prec])
        if rescore_topk:
            # BF16 rollouts: re-score only the boxes of the rescore_topk smallest BF16 upper bounds in FP32
            B.bab_set_rescore_topk(self.ctx, rescore_topk)
        if cost is not None:
            # the pushing-with-obstacles state cost (Appendix D.4) instead of the squared distance
            B.bab_set_cost(self.ctx, B.COST_PUSHING_OBSTACLES, cost["w"], cost["lam"], cost["obstacles"], cost["p0"])
        f = dict(device=device, dtype=torch.float32)
        self.x0 = torch.as_tensor(self.p["x0"]).to(**f)
        self.goal = torch.as_tensor(self.p["goal"]).to(**f)
        levels = min(int(np.log2(self.nb)), self.d)
        lo, hi, ids = W.grid_boxes(self.d, levels)
        n0 = lo.shape[0]
        self.cap = n0 + pool_iters * n_pick
        self.pool = [self._alloc(), self._alloc()]
        self.cur = 0
        P = self.pool[0]
        P["lo"][:n0] = torch.as_tensor(lo).to(**f)
        P["hi"][:n0] = torch.as_tensor(hi).to(**f)
        P["id"][:n0] = torch.as_tensor(ids.astype(np.int64)).to(device)
        self.fixed = fixed_launch
        self.n_max = self.cap - n_pick if fixed_launch else n0
        nbuf = max(self.nb, n0)
        self.best_u = torch.empty(nbuf, self.d, **f)
        self.margin = torch.empty(nbuf, **f)
        self.keep = torch.empty(self.cap, dtype=torch.uint8, device=device)
        self.counts = torch.zeros(3, dtype=torch.int32, device=device)
        self.counts[2] = n0
        self.inc_val = torch.full((1,), float("inf"), dtype=torch.float64, device=device)
        self.inc_u = torch.zeros(self.d, **f)
        self.n_live_dev = torch.tensor([n0], dtype=torch.int32, device=device)
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
        self.ev = []
        self.side = torch.cuda.Stream(device=device)
        # the paper's bounding (search-integrated bounds, propagation early-stop at step search_stop): FP32 rollouts
        # record the bounds, CROWN uses them
        self.search_stop = search_stop
        if search_stop is not None:
            nb_ = max(self.nb, n0)
            self.emp = [torch.empty(nb_, self.H, self.sumh, **f), torch.empty(nb_, self.H, self.sumh, **f),
                        torch.empty(nb_, self.H + 1, self.p["s"], **f), torch.empty(nb_, self.H + 1, self.p["s"], **f)]
        # the paper's branching heuristics (Section 3.1): softmax pick-out at temperature T and split dimensions
        # from the imbalance of the top w% samples; None: smallest lb and widest dimension
        self.heur = heuristics
        self.it = 0
        # cross-entropy search (Section 3.3) instead of uniform samples: dict(iters, elites, jitter), samples per
        # iteration = M / iters; every pool row carries its best input, the warm start of its children
        self.cem = cem
        if cem is not None:
            for Q in self.pool:
                Q["bu"] = torch.zeros(self.cap, self.d, **f)
            if heuristics is None:
                self.heur = {"T": None, "w": 1.0, "split": False}
            for Q in self.pool:
                Q.setdefault("sd", torch.full((self.cap,), -1, dtype=torch.int32, device=device))
        if heuristics is not None:
            for Q in self.pool:
                Q["sd"] = torch.full((self.cap,), -1, dtype=torch.int32, device=device)
            self.costs = torch.empty(max(self.nb, n0), self.M, **f)
        self.variants = None
        if autotune:
            # tile shapes timed on the starting pool (outside any timed region)
            B.bab_autotune(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], P["id"], n0, self.M,
                           alpha_steps=alpha_steps)
            names = {"rollout_fp32": B.KERNEL_ROLLOUT_FP32, "alpha_fused": B.KERNEL_ALPHA_FUSED,
                     "rollout_tc_tiles_per_cta": B.KERNEL_ROLLOUT_TC, "crown_tc_tiles_per_cta": B.KERNEL_CROWN_TC}
            self.variants = {k: B.bab_get_variant(self.ctx, v) for k, v in names.items()}
        # Algorithm 2 starts by searching and bounding the starting pool
        self.search_and_bound(P, n0, None)
        fused = alpha_steps and self.bprec == B.PREC_FP32 and (self.variants or {}).get("alpha_fused", -1) != -2
        # prune/branch 2, rollout 4 (keys, rollout, finalize, incumbent) plus the FP32 re-score of BF16 rollouts (and
        # the top-k selection before it), bound 2 (or the alpha loop)
        bf16 = self.rprec == PRECISIONS["bf16"]
        roll = 4 + (1 if bf16 else 0) + (1 if bf16 and rescore_topk else 0)
        self.launches_per_step = 2 + roll + (2 if not alpha_steps else (2 if fused else 3 + alpha_steps * 3))

    def snapshot(self):
        """Device copies of the BaB state (both pools, counts, incumbent), to rerun the same iterations."""
        keys = ("counts", "inc_val", "inc_u", "n_live_dev")
        return {"pool": [{k: v.clone() for k, v in P.items()} for P in self.pool], "cur": self.cur, "it": self.it,
                **{k: getattr(self, k).clone() for k in keys}}

    def restore(self, snap):
        """Back to a snapshot, in place (captured graphs keep their buffers)."""
        for P, Q in zip(self.pool, snap["pool"]):
            for k, v in Q.items():
                P[k].copy_(v)
        for k in ("counts", "inc_val", "inc_u", "n_live_dev"):
            getattr(self, k).copy_(snap[k])
        self.cur, self.it = snap["cur"], snap["it"]

    def _alloc(self):
        torch = self.torch
        f = dict(device=self.dev, dtype=torch.float32)
        return {"lo": torch.empty(self.cap, self.d, **f), "hi": torch.empty(self.cap, self.d, **f),
                "lb": torch.empty(self.cap, **f), "ub": torch.empty(self.cap, **f),
                "id": torch.empty(self.cap, dtype=torch.int64, device=self.dev)}

    def search_and_bound(self, P, n, d_n, events=False):
        B, torch = self.B, self.torch
        if events:
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
        if self.cem is not None:
            c = self.cem
            warm = P["bu"] if self.it > 0 else None   # the starting pool has no parents
            B.bab_rollout_cem(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], P["id"], n,
                              self.M // c["iters"], c["iters"], c["elites"], c["jitter"], self.seed + self.it,
                              self.rprec, P["ub"], P["bu"], warm_u=warm, d_n=d_n)
        elif self.heur is not None:
            B.bab_rollout_split(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], P["id"], n, self.M,
                                self.seed, self.rprec, self.heur["w"], P["ub"], P["sd"], best_u=self.best_u,
                                costs=self.costs, d_n=d_n)
        elif self.search_stop is None:
            B.bab_rollout(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], P["id"], n, self.M,
                          self.seed, self.rprec, P["ub"], self.best_u, d_n=d_n)
        else:
            B.bab_rollout_search_bounds(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], P["id"], n,
                                        self.M, self.seed, P["ub"], *self.emp, best_u=self.best_u, d_n=d_n)
        if events:
            e[1].record()
        # the FP64 incumbent re-score runs on a side stream, beside the bounds of the same boxes
        main = torch.cuda.current_stream()
        self.side.wait_stream(main)
        with torch.cuda.stream(self.side):
            B.bab_update_incumbent(self.ctx, self.x0, self.goal, self.H, self.rho, P["ub"],
                                   P["bu"] if self.cem is not None else self.best_u, n, self.inc_val, self.inc_u,
                                   d_n=d_n)
        if self.search_stop is not None:
            B.bab_bound_crown_given(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], n, *self.emp,
                                    self.search_stop, P["lb"], d_n=d_n)
        elif not self.alpha_steps:
            B.bab_bound_crown(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], n, P["lb"],
                              precision=self.bprec, margin=self.margin, d_n=d_n)
        else:
            B.bab_alpha_optimize(self.ctx, self.x0, self.goal, self.H, self.rho, P["lo"], P["hi"], n,
                                 self.alpha_steps, self.alpha_lr, P["lb"][:n], precision=self.bprec, d_n=d_n)
        if events:
            e[2].record()
            self.ev.append(e)
        main.wait_stream(self.side)  # the next prune reads the incumbent

    def step(self, events=False):
        B = self.B
        src, dst = self.pool[self.cur], self.pool[self.cur ^ 1]
        if self.heur is None:
            B.bab_prune_branch(self.ctx, self.d, src["lo"], src["hi"], src["lb"], src["ub"], src["id"], self.n_max,
                               self.inc_val, self.n_pick, 0.75, self.cap, dst["lo"], dst["hi"], dst["lb"], dst["ub"],
                               dst["id"], self.keep, self.counts, d_n=self.n_live_dev)
        else:
            # children come first in dst and get their split dimensions from their own search below
            rule = B.PICK_SOFTMAX if self.heur["T"] is not None else B.PICK_LB
            B.bab_prune_branch_heuristic(self.ctx, self.d, src["lo"], src["hi"], src["lb"], src["ub"], src["id"],
                                         self.n_max, self.inc_val, self.n_pick, 0.75, rule, self.heur["T"] or 1.0,
                                         self.seed * 1000003 + self.it, self.cap, dst["lo"], dst["hi"], dst["lb"],
                                         dst["ub"], dst["id"], self.keep, self.counts,
                                         split_dim=src["sd"] if self.heur["split"] else None,
                                         out_split_dim=dst["sd"], row_u=src.get("bu"), out_row_u=dst.get("bu"),
                                         d_n=self.n_live_dev)
        self.it += 1
        if not self.fixed:
            self.n_max = min(self.n_max + self.n_pick, self.cap - self.n_pick)
        self.search_and_bound(dst, self.nb, self.counts[0:1], events=events)
        self.n_live_dev.copy_(self.counts[2:3])
        self.cur ^= 1

    def gap(self):
        """Incumbent (FP64) minus the smallest lower bound of the live pool (synchronises)."""
        n = int(self.counts[2].item())
        P = self.pool[self.cur]
        lbmin = float(P["lb"][:n].min().item()) if n > 0 else float("inf")
        return float(self.inc_val.item()) - lbmin, n

    def flush_l2(self):
        self.flush.fill_(1.0)

    def close(self):
        self.B.bab_destroy(self.ctx)


def capture_graphs(st):
    """CUDA graphs of one iteration for each pool parity (the pool ping-pongs between two buffers)."""
    torch = st.torch
    graphs = []
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            st.step()
        torch.cuda.synchronize()
        for _ in range(2):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                st.step()
            graphs.append(g)
    torch.cuda.current_stream().wait_stream(s)
    return graphs


# DRAM bytes (read + write) per launch of the BF16 tensor-core rollout (the fused-step kernel) at 4096 boxes x
# 1024 samples, from one ncu capture of this bench (dram__bytes_read.sum + dram__bytes_write.sum); valid only for
# the kernel sources it was taken on, so it is reported only while their digest (comments and whitespace removed)
# matches.
ROLLOUT_TC_TRAFFIC = {"bytes": 1949440, "precision": "bf16", "boxes": 4096, "samples": 1024,
                      "sources_sha1": "acaf47e420a87e8b2e2dd1b3bc427a83bbfb5ee1"}
ROLLOUT_TC_SOURCES = ("rollout_tc.cu", "tc_ptx.cuh", "kernels.cuh", "bab_internal.cuh")


def code_digest(texts):
    """SHA-1 of source texts with their comments and whitespace removed (a comment edit keeps the capture valid)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for t in texts:
        t = re.sub(r"/\*.*?\*/", " ", t, flags=re.S)
        t = re.sub(r"//[^\n]*", " ", t)
        h.update(" ".join(t.split()).encode())
    return h.hexdigest()


def rollout_sources_sha1():
    texts = []
    for name in ROLLOUT_TC_SOURCES:
        with open(os.path.join(ROOT, "paper_2412_09584_gb300", "csrc", name)) as f:
            texts.append(f.read())
    return code_digest(texts)


def rollout_traffic(precision, boxes, samples):
    t = ROLLOUT_TC_TRAFFIC
    if (precision, boxes, samples) != (t["precision"], t["boxes"], t["samples"]):
        return None
    return t["bytes"] if rollout_sources_sha1() == t["sources_sha1"] else None


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
    n_pick = args.boxes // 2
    st = BabState("pushing", rank_seed(rank), dev, n_pick, args.precision, args.bound_precision,
                  interval_prec=args.interval_precision,
                  fixed_launch=not args.no_graph, autotune=not args.no_autotune)
    for _ in range(args.warmup):
        st.step()
        st.flush_l2()
    graphs = None if args.no_graph else capture_graphs(st)
    torch.cuda.synchronize()
    snap = st.snapshot()  # the end-to-end run below starts from the same pool as the timed region
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0.record()
        for i in range(args.steps):
            if graphs is not None:
                graphs[st.cur].replay()
                st.cur ^= 1
            else:
                st.step()
            st.flush_l2()
        t1.record()
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    if ws > 1:
        ms = max_over_ranks(ms, dev)
    clocks = clk.summary()
    # per-kernel times on the launching stream (eager steps, same shapes)
    for _ in range(3):
        st.step(events=True)
        st.flush_l2()
    torch.cuda.synchronize()
    roll_ms = [e[0].elapsed_time(e[1]) for e in st.ev]
    bound_ms = [e[1].elapsed_time(e[2]) for e in st.ev]
    # end to end through the C-ABI with host buffers, from the timed region's starting pool (the pool grows every
    # iteration, and with it the prune/branch plan); whole-job rate over the slowest rank, as the device timing
    st.restore(snap)
    del snap
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e2e = run_e2e(st, args.steps)
    ms_e2e = e2e.pop("ms")
    if ws > 1:
        ms_e2e = max_over_ranks(ms_e2e, dev)
    e2e["value"] = job_rate(st.nb * args.steps, ws, ms_e2e)
    inc = float(st.inc_val.item())
    st.close()
    # the single-GPU comparisons run at N = 1 only (a multi-rank run reports the scaled iteration alone)
    extra = ws == 1
    ttg = time_to_gap(dev) if extra and not args.no_time_to_gap else None
    ttg_push = time_to_gap_pushing(dev) if extra and not args.no_time_to_gap else None
    tiny = tiny_latency(dev) if extra and not args.no_time_to_gap else None
    batched = batched_bab(dev) if extra and not args.no_batched else None
    manip = manip_scale(dev) if extra and not args.no_manip else None
    paper_bounds = paper_bounding_comparison(dev) if extra and not args.no_time_to_gap else None
    heuristics = heuristics_comparison(dev) if extra and not args.no_time_to_gap else None
    cem_cmp = cem_comparison(dev) if extra and not args.no_time_to_gap else None
    synth = synthetic_sweep(dev) if extra and not args.no_time_to_gap else None
    obst = obstacle_bab(dev) if extra and not args.no_time_to_gap else None

    boxes = st.nb * args.steps * ws
    value = job_rate(st.nb * args.steps, ws, ms)
    rsteps = boxes * st.M * st.H / (ms / 1e3)
    roof = rollout_roofline(args.precision, st.p, st.nb, st.M, st.H, statistics.mean(roll_ms))
    roof["traffic"] = rollout_traffic(args.precision, st.nb, st.M)
    # the same iteration with the rollouts in the other arithmetics: all-FP32 (the configuration as named) and
    # plain BF16 with each box's pick re-scored in FP32 (the search precision the method's plan prescribes)
    lines = precision_lines(dev, rank_seed(rank), n_pick, args.precision, args.bound_precision,
                            args.interval_precision) \
        if ws == 1 and not args.no_precision_lines else None
    if rank != 0:
        return
    cfg = {"workload": "pushing-scale BaB iteration: state 8, action 2, MLP 10-128-128-128-8 ReLU residual, H=20, "
                       f"rho=0.01, {st.nb} children bounded per iteration ({n_pick} picked, widest-dim bisection), "
                       f"{st.M} uniform rollouts per child",
           "rollout_arithmetic": ARITH[args.precision],
           "bound_arithmetic": {"bf16x3": "interval bounds on tcgen05 (3-term BF16 split, computed margin)",
                                "tf32x3": "interval bounds on tcgen05 (3-term TF32 split, computed margin)",
                                "fp32": "outward-rounded FP32 intervals"}[args.interval_precision] +
                               "; CROWN products " +
                               {"bf16x3": "on tcgen05, 3-term BF16 split", "tf32x3": "on tcgen05, 3-term TF32 split",
                                "fp32": "in FP32 on CUDA cores"}[args.bound_precision] + ", margin-corrected",
           "boxes_per_step": st.nb, "samples_per_box": st.M, "H": st.H,
           "initial_pool": f"{st.nb}-box grid over [-1,1]^{st.d}", "l2": "flushed between steps (256 MiB write)",
           "timed_region": "CUDA-graph replays of the whole iteration" if graphs is not None else "eager launches",
           "launch_variants": st.variants or "built-in heuristic",
           "parallelism": f"independent problems x{ws}" if ws > 1 else "single GPU"}
    out = {"metric": METRIC, "value": value, "unit": "subdomain-bounds/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": args.precision, "data": "synthetic (seeded random network, start and goal)",
           "config": cfg, "rollout_steps_per_s": rsteps,
           "kernel_ms": {"rollout": statistics.mean(roll_ms), "bound": statistics.mean(bound_ms)},
           "crown_subdomain_bounds_per_s_kernel_only": st.nb / (statistics.mean(bound_ms) / 1e3),
           "incumbent_fp64": inc, "roofline": roof, "clocks": clocks, "e2e": e2e,
           "gpu_launches": st.launches_per_step * args.steps, "time_to_gap": ttg, "time_to_gap_pushing": ttg_push, "batched": batched, "manip_scale": manip,
           "paper_bounding": paper_bounds, "heuristics": heuristics, "cem_search": cem_cmp,
           "synthetic_objective": synth, "obstacle_cost": obst, "tiny_latency": tiny, "precision_lines": lines,
           "fp32_peak_measured": fp32_peak_measured()}
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def precision_lines(dev, seed, n_pick, headline, bound_precision, interval_precision="fp32", steps=3):
    """The bench iteration with the rollouts in each arithmetic other than the headline's, and with the headline's
    rollouts and the other CROWN arithmetic: CUDA-graph replays of the same pushing-scale iteration, L2 flushed
    between steps, per-kernel times by CUDA events after the timed region; each with its rollout roofline (FP32
    against the measured FP32 FMA rate)."""
    import torch
    out = {}
    other_bound = "fp32" if bound_precision == "bf16x3" else "bf16x3"
    other_int = "fp32" if interval_precision == "bf16x3" else "bf16x3"
    combos = [(p, bound_precision, interval_precision) for p in ("fp32", "bf16x3", "bf16") if p != headline]
    combos += [(headline, other_bound, interval_precision), (headline, bound_precision, other_int)]
    if bound_precision != "tf32x3":
        combos.append((headline, "tf32x3", interval_precision))
    if interval_precision != "tf32x3":
        combos.append((headline, bound_precision, "tf32x3"))
    for prec, bprec, iprec in combos:
        key = prec if bprec == bound_precision else f"{prec}, {bprec} CROWN products"
        if iprec != interval_precision:
            key = f"{prec}, {iprec} interval bounds"
        st = BabState("pushing", seed, dev, n_pick, prec, bprec, fixed_launch=True, interval_prec=iprec)
        for _ in range(3):
            st.step()
            st.flush_l2()
        graphs = capture_graphs(st)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(steps):
            graphs[st.cur].replay()
            st.cur ^= 1
            st.flush_l2()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        st.ev = []
        for _ in range(2):
            st.step(events=True)
            st.flush_l2()
        torch.cuda.synchronize()
        roll = statistics.mean(e[0].elapsed_time(e[1]) for e in st.ev)
        bound = statistics.mean(e[1].elapsed_time(e[2]) for e in st.ev)
        out[key] = {"rollout_arithmetic": ARITH[prec], "bound_arithmetic": bprec, "interval_arithmetic": iprec,
                    "ms_per_step": ms,
                    "subdomain_bounds_per_s": st.nb / (ms / 1e3),
                    "rollout_steps_per_s": st.nb * st.M * st.H / (ms / 1e3),
                    "kernel_ms": {"rollout": roll, "bound": bound},
                    "roofline": rollout_roofline(prec, st.p, st.nb, st.M, st.H, roll), "steps": steps}
        del graphs
        st.close()
    return out


def run_e2e(st, steps):
    """Same iteration with the batch of boxes crossing the host boundary every step: the batch is copied in
    from pinned host memory, searched and bounded, pruned and branched, and the next batch plus the bounds and
    the incumbent are copied back out."""
    torch, B = st.torch, st.B
    nb, d = st.nb, st.d
    h_lo = torch.empty(nb, d, dtype=torch.float32, pin_memory=True)
    h_hi = torch.empty_like(h_lo, pin_memory=True)
    h_id = torch.empty(nb, dtype=torch.int64, pin_memory=True)
    h_lb = torch.empty(nb, dtype=torch.float32, pin_memory=True)
    h_ub = torch.empty_like(h_lb, pin_memory=True)
    h_inc = torch.empty(1, dtype=torch.float64, pin_memory=True)
    src = st.pool[st.cur]
    h_lo.copy_(src["lo"][:nb])
    h_hi.copy_(src["hi"][:nb])
    h_id.copy_(src["id"][:nb])
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        P = st.pool[st.cur]
        P["lo"][:nb].copy_(h_lo, non_blocking=True)
        P["hi"][:nb].copy_(h_hi, non_blocking=True)
        P["id"][:nb].copy_(h_id, non_blocking=True)
        st.search_and_bound(P, nb, None)
        h_lb.copy_(P["lb"][:nb], non_blocking=True)
        h_ub.copy_(P["ub"][:nb], non_blocking=True)
        dst = st.pool[st.cur ^ 1]
        B.bab_prune_branch(st.ctx, d, P["lo"], P["hi"], P["lb"], P["ub"], P["id"], st.n_max, st.inc_val,
                           st.n_pick, 0.75, st.cap, dst["lo"], dst["hi"], dst["lb"], dst["ub"], dst["id"], st.keep,
                           st.counts, d_n=st.n_live_dev)
        st.n_live_dev.copy_(st.counts[2:3])
        h_lo.copy_(dst["lo"][:nb], non_blocking=True)
        h_hi.copy_(dst["hi"][:nb], non_blocking=True)
        h_id.copy_(dst["id"][:nb], non_blocking=True)
        h_inc.copy_(st.inc_val, non_blocking=True)
        st.cur ^= 1
        st.flush_l2()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    h2d = nb * (2 * d * 4 + 8)
    d2h = nb * (2 * 4) + nb * (2 * d * 4 + 8) + 8
    return {"value": nb * steps / (ms / 1e3), "unit": "subdomain-bounds/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms": ms}


def manip_scale(dev, reps=3):
    """Object-manipulation scale (MLP 36-256x4-32, H = 40, 16384 boxes of [-1, 1]^160): 4 BF16 tensor-core
    rollouts per box (65536 in all, each box's best re-scored in FP32, the incumbent in FP64), interval bounds
    and the 3-term BF16 tensor-core CROWN, both with the weights streamed through shared memory.  CUDA events
    around each call after a warm-up; returns milliseconds and rates."""
    import torch
    from paper_2412_09584_gb300 import binding as B
    from paper_2412_09584_gb300 import workloads as W
    c = W.CONFIGS["manip"]
    p = W.config_problem("manip", SEED)
    n, M, H = c["boxes"], c["samples"], c["H"]
    d = p["k"] * H
    lo, hi, ids = W.grid_boxes(d, c["grid_dims"])
    ctx = B.bab_load_dynamics(p["dims"], p["params"], p["s"], p["k"])
    f = dict(device=dev, dtype=torch.float32)
    x0, goal = torch.as_tensor(p["x0"]).to(**f), torch.as_tensor(p["goal"]).to(**f)
    tlo, thi = torch.as_tensor(lo).to(**f), torch.as_tensor(hi).to(**f)
    tid = torch.as_tensor(ids.astype(np.int64)).to(dev)
    ub, best_u = torch.empty(n, **f), torch.empty(n, d, **f)
    inc_val = torch.full((1,), float("inf"), dtype=torch.float64, device=dev)
    inc_u = torch.zeros(d, **f)
    lb, lb32 = torch.empty(n, **f), torch.empty(n, **f)
    B.bab_set_rescore_topk(ctx, 64)  # the configuration re-scores the top 64 BF16 rollouts in FP32

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_roll = timed(lambda: B.bab_rollout(ctx, x0, goal, H, p["rho"], tlo, thi, tid, n, M, SEED, B.PREC_BF16, ub,
                                         best_u, inc_val, inc_u))
    t_ibp = timed(lambda: B.bab_bound_ibp(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb32))
    t_tc = timed(lambda: B.bab_bound_crown(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb, precision=B.PREC_BF16X3))
    t_32 = timed(lambda: B.bab_bound_crown(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb32))
    sound = bool((lb <= ub).all().item())
    # the interval bounds on tensor cores (3-term BF16 split with a computed margin: sound, wider)
    lb_f = lb.clone()
    B.bab_set_interval_precision(ctx, B.PREC_BF16X3)
    t_ibp_tc = timed(lambda: B.bab_bound_ibp(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb32))
    t_tc_tc = timed(lambda: B.bab_bound_crown(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb, precision=B.PREC_BF16X3))
    sound = sound and bool((lb <= ub).all().item())
    # how much of the bound the wider intervals give up, relative to the bound's magnitude (median over boxes)
    loss = float(((lb_f - lb).abs() / lb_f.abs().clamp_min(1.0)).median().item())
    # the same with TF32 halves (a smaller margin per layer)
    B.bab_set_interval_precision(ctx, B.PREC_TF32X3)
    t_ibp_tf = timed(lambda: B.bab_bound_ibp(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb32))
    t_tc_tf = timed(lambda: B.bab_bound_crown(ctx, x0, goal, H, p["rho"], tlo, thi, n, lb, precision=B.PREC_BF16X3))
    sound = sound and bool((lb <= ub).all().item())
    loss_tf = float(((lb_f - lb).abs() / lb_f.abs().clamp_min(1.0)).median().item())
    B.bab_set_interval_precision(ctx, B.PREC_FP32)
    B.bab_destroy(ctx)
    macs = sum(a * b for a, b in zip(p["dims"][1:], p["dims"][:-1]))
    bwd_flop = 2.0 * macs * H * n  # algorithmic backward products of one CROWN call (the pipe runs 3x for the split)
    return {"workload": f"MLP 36-256x4-32, H={H}, rho={p['rho']}, {n} boxes (2^{c['grid_dims']} grid of [-1,1]^{d}), "
                        f"{M} BF16 rollouts per box, top 64 re-scored in FP32, incumbent in FP64",
            "rollout_bf16_ms": t_roll,
            "rollout_steps_per_s": n * M * H / (t_roll / 1e3), "ibp_ms": t_ibp,
            "bound_bf16x3_ms": t_tc, "bound_fp32_ms": t_32,
            "subdomain_bounds_per_s_bf16x3": n / (t_tc / 1e3), "subdomain_bounds_per_s_fp32": n / (t_32 / 1e3),
            "crown_backward_tflops_bf16x3": bwd_flop / ((t_tc - t_ibp) / 1e3) / 1e12,
            "ibp_tensor_core_ms": t_ibp_tc, "bound_bf16x3_tc_intervals_ms": t_tc_tc,
            "subdomain_bounds_per_s_tc_intervals": n / (t_tc_tc / 1e3),
            "tc_intervals_bound_loss_median": loss,
            "ibp_tensor_core_tf32_ms": t_ibp_tf, "bound_bf16x3_tf32_intervals_ms": t_tc_tf,
            "subdomain_bounds_per_s_tf32_intervals": n / (t_tc_tf / 1e3),
            "tf32_intervals_bound_loss_median": loss_tf,
            "note": "bound times include the interval bounds (ibp_ms); backward TFLOP/s = algorithmic 2 x MACs x H x "
                    "boxes over (bound - ibp) time; weights streamed through shared memory (they exceed it); "
                    "tc_intervals: the interval bounds on tensor cores (3-term BF16 split, computed margin), the "
                    "bound's median loss against FP32 intervals relative to its magnitude; tf32_intervals: the same "
                    "with 3-term TF32 halves",
            "bounds_below_sampled_ub": sound,
            "iteration": manip_iteration(dev)}


def manip_iteration(dev, steps=4):
    """The object-manipulation configuration as whole BaB iterations: prune + pick-out + bisect of the pool (8192
    picked, 16384 children), 4 BF16 rollouts per child with the top 64 re-scored in FP32 and the FP64 incumbent on a
    side stream, interval bounds + 3-term BF16 CROWN; CUDA-graph replays, CUDA events, the pool and its intervals
    far beyond L2.  With FP32 intervals, then with the intervals on tensor cores (BF16, then TF32 halves)."""
    import torch
    out = {"workload": "MLP 36-256x4-32, H=40, rho=0.01, 16384 children per iteration (8192 picked, widest-dim "
                       "bisection), 4 BF16 rollouts each, top 64 re-scored in FP32, FP64 incumbent, CROWN on tcgen05 "
                       "(3-term BF16 split)"}
    keys = {"fp32": "fp32_intervals", "bf16x3": "tensor_core_intervals", "tf32x3": "tensor_core_tf32_intervals"}
    for iprec in ("fp32", "bf16x3", "tf32x3"):
        st = BabState("manip", SEED, dev, 8192, "bf16", "bf16x3", fixed_launch=True, pool_iters=steps + 10,
                      interval_prec=iprec, rescore_topk=64)
        graphs = capture_graphs(st)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(steps):
            graphs[st.cur].replay()
            st.cur ^= 1
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        out[keys[iprec]] = {
            "ms_per_iteration": ms, "subdomain_bounds_per_s": st.nb / (ms / 1e3),
            "rollout_steps_per_s": st.nb * st.M * st.H / (ms / 1e3), "steps": steps,
            "status": st.B.bab_status(st.ctx)}
        del graphs
        st.close()
    return out



def batched_bab(dev, iters=50, n_pick=64, samples=None, alpha_steps=None, P=None, picks_choices=(8, 16, 32, 64, 128, 160)):
    """Many concurrent plans: P problems of the tiny architecture (own weights, start, goal; horizons uniform in
    10..80), each pool starting as a 256-box grid; per iteration, per problem: prune against its incumbent, pick
    a problem- and iteration-dependent number of boxes (drawn from picks_choices, so that the live pools spread
    over about 256-8192 rows and change size every iteration; n_pick for all when picks_choices is None), split
    them, search (BF16x3 tensor-core rollouts) and bound (interval bounds + alpha-CROWN) the children.  Every
    iteration is one CUDA-graph replay (one launch per kernel for all problems) after a device-side copy of that
    iteration's pick counts.  Returns timing, live-pool sizes, pruned rows and gaps."""
    import torch
    from paper_2412_09584_gb300 import binding as B
    from paper_2412_09584_gb300 import workloads as W
    c = W.CONFIGS["batched"]
    P = P or c["problems"]
    samples = samples or c["samples"]
    alpha_steps = c["alpha_steps"] if alpha_steps is None else alpha_steps
    probs, _ = W.batch_problems(P, SEED, H_lo=c["H_lo"], H_hi=c["H_hi"])
    params, x0, goal, Hs, rho = W.pack_batch(probs)
    k = probs[0]["k"]
    Hmax = int(Hs.max())
    d = k * Hmax
    ctx = B.bab_load_dynamics_batch(probs[0]["dims"], params, probs[0]["s"], k)
    f = dict(device=dev, dtype=torch.float32)
    i32 = dict(device=dev, dtype=torch.int32)
    tx0, tgoal, tH, trho = (torch.as_tensor(x0).to(**f), torch.as_tensor(goal).to(**f),
                            torch.as_tensor(Hs).to(**i32), torch.as_tensor(rho).to(**f))
    lo, hi, ids, prob = W.batch_grid_boxes(probs, 8, d)
    n0 = lo.shape[0]
    if picks_choices is not None:
        rng = np.random.default_rng(SEED + 5)
        sched_np = rng.choice(np.asarray(picks_choices, dtype=np.int32), size=(iters + 4, P))
        n_pick = int(max(picks_choices))
    else:
        sched_np = np.full((iters + 4, P), n_pick, dtype=np.int32)
    per_iter = P * n_pick
    cap = n0 + (iters + 8) * per_iter
    nb = 2 * per_iter

    def alloc():
        return {"lo": torch.zeros(cap, d, **f), "hi": torch.zeros(cap, d, **f), "lb": torch.empty(cap, **f),
                "ub": torch.empty(cap, **f), "id": torch.zeros(cap, dtype=torch.int64, device=dev),
                "prob": torch.zeros(cap, **i32)}
    pool = [alloc(), alloc()]
    P0 = pool[0]
    P0["lo"][:n0] = torch.as_tensor(lo).to(**f)
    P0["hi"][:n0] = torch.as_tensor(hi).to(**f)
    P0["id"][:n0] = torch.as_tensor(ids.astype(np.int64)).to(dev)
    P0["prob"][:n0] = torch.as_tensor(prob).to(**i32)
    best_u = torch.empty(max(nb, n0), d, **f)
    inc_val = torch.full((P,), float("inf"), dtype=torch.float64, device=dev)
    inc_u = torch.zeros(P, d, **f)
    keep = torch.empty(cap, dtype=torch.uint8, device=dev)
    counts = torch.zeros(3, **i32)
    n_live = torch.tensor([n0], **i32)
    picks = torch.full((P,), n_pick, **i32)
    sched = torch.as_tensor(sched_np).to(**i32)
    # tile shapes timed on problem 0's starting boxes (the grid rows are grouped by problem)
    r0, d0 = int((prob == 0).sum()), k * int(Hs[0])
    B.bab_autotune(ctx, tx0[0].contiguous(), tgoal[0].contiguous(), int(Hs[0]), float(rho[0]),
                   P0["lo"][:r0, :d0].contiguous(), P0["hi"][:r0, :d0].contiguous(), P0["id"][:r0], r0, samples)

    def search_and_bound(Q, n, d_n):
        B.bab_rollout_batch(ctx, tx0, tgoal, tH, trho, Hmax, d, Q["lo"], Q["hi"], Q["id"], Q["prob"], n, samples,
                            SEED, Q["ub"], best_u, inc_val, inc_u, d_n=d_n, precision=B.PREC_BF16X3)
        B.bab_bound_batch(ctx, tx0, tgoal, tH, trho, Hmax, d, Q["lo"], Q["hi"], Q["prob"], n, Q["lb"],
                          alpha_steps=alpha_steps, lr=c["alpha_lr"], d_n=d_n)

    state = {"cur": 0, "it": 0}
    n_max = cap - per_iter

    def step():
        src, dst = pool[state["cur"]], pool[state["cur"] ^ 1]
        B.bab_prune_branch_batch(ctx, d, tH, Hmax, src["lo"], src["hi"], src["lb"], src["ub"], src["id"],
                                 src["prob"], n_max, inc_val, picks, per_iter, 0.75, cap, dst["lo"], dst["hi"],
                                 dst["lb"], dst["ub"], dst["id"], dst["prob"], keep, counts, d_n=n_live)
        search_and_bound(dst, nb, counts[0:1])
        n_live.copy_(counts[2:3])
        state["cur"] ^= 1

    search_and_bound(P0, n0, None)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for i in range(2):  # warm-up (loads every kernel), then one graph per pool parity
            picks.copy_(sched[i])
            step()
        torch.cuda.synchronize()
        graphs = []
        for i in range(2):
            picks.copy_(sched[2 + i])
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                step()
            graphs.append(g)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    done = 2 + 2  # iterations run so far (two eager warm-up steps and the two captured ones)
    picked = sched_np[:done].sum(axis=0).astype(np.int64)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for i in range(done, iters):
        picks.copy_(sched[i])  # this iteration's quota per problem, read by the graph's prune/branch
        graphs[state["cur"]].replay()
        state["cur"] ^= 1
    t1.record()
    picked += sched_np[done:iters].sum(axis=0)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / (iters - done)
    status = B.bab_status(ctx)
    n = int(counts[2].item())
    Q = pool[state["cur"]]
    lbmin = torch.full((P,), float("inf"), **f).scatter_reduce(0, Q["prob"][:n].long(), Q["lb"][:n], "amin")
    live = torch.bincount(Q["prob"][:n].long(), minlength=P).cpu().numpy()
    gaps = (inc_val - lbmin.double()).cpu().numpy()
    B.bab_destroy(ctx)
    # every pick replaces a box by its two children (+1 row), every prune removes one: rows created minus live
    start = np.bincount(prob, minlength=P)
    pruned = start + picked - live
    quota = ("per problem and iteration drawn from " + str(list(picks_choices))) if picks_choices is not None \
        else f"{n_pick} per problem per iteration"
    children = 2.0 * float(sched_np[done:iters].sum()) / (iters - done)  # children bounded per timed iteration
    return {"workload": f"{P} problems of MLP 6-32-32-4 (own weights, start, goal), horizons uniform in "
                        f"[{c['H_lo']}, {c['H_hi']}], 256-box starting grid each, boxes picked and split {quota}, "
                        f"{samples} BF16x3 tensor-core rollouts per child, interval bounds + alpha-CROWN "
                        f"({alpha_steps} Adam steps) per child",
            "iterations": iters, "ms_per_iteration": ms, "children_per_iteration_mean": children,
            "launch_rows_per_iteration": nb,
            "subdomain_bounds_per_s": children / (ms / 1e3),
            "rollout_steps_per_s": children * samples * float(np.mean(Hs)) / (ms / 1e3),
            "launches_per_iteration": 3 + 4 + 2 + 1, "timed_region": "CUDA-graph replays, one launch per kernel, "
                                                                    "after a device copy of the iteration's quotas",
            "live_rows_end": n, "live_rows_per_problem_end": {"min": int(live.min()), "median": float(np.median(live)),
                                                               "max": int(live.max())},
            "pruned_rows": {"total": int(pruned.sum()), "problems_with_pruning": int((pruned > 0).sum())},
            "gap_end": {"min": float(gaps.min()), "median": float(np.median(gaps)), "max": float(gaps.max())},
            "device_status": status}



def paper_bounding_comparison(dev, iters=30, stops=(0, 2)):
    """The paper's bounding (search-integrated bounds + propagation early-stop) against sound bounds in the same
    BaB loop (alpha workload: tiny network, H = 5, 4096 children per iteration, 256 FP32 rollouts each): the
    incumbent reached (the plan's objective, exact in FP64), the live pool left (how much was pruned) and the
    time per iteration.  The estimated bounds are not sound, so they certify no gap."""
    import torch
    out = {"workload": "alpha: MLP 6-32-32-4, H=5, 4096 children per iteration, 256 FP32 rollouts each, "
                       f"{iters} iterations"}
    variants = {"sound_ibp_crown": None}
    variants.update({f"search_bounds_stop_{t}": t for t in stops})
    for name, stop in variants.items():
        for warm in (True, False):
            st = BabState("alpha", SEED, dev, 2048, "fp32", "fp32", pool_iters=iters + 2, search_stop=stop)
            torch.cuda.synchronize()
            t = time.perf_counter()
            curve = []
            for _ in range(2 if warm else iters):
                st.step()
                if not warm:
                    curve.append(float(st.inc_val.item()))
            torch.cuda.synchronize()
            sec = time.perf_counter() - t
            n_live = int(st.counts[2].item())
            st.close()
        out[name] = {"incumbent": curve[-1], "incumbent_curve": [round(v, 6) for v in curve],
                     "live_pool_end": n_live, "ms_per_iteration": 1e3 * sec / iters,
                     "bound": "sound (interval + CROWN, margin)" if stop is None else
                              f"estimate: search-integrated bounds, early stop at step {stop}"}
    return out



def heuristics_comparison(dev, iters=30):
    """The paper's branching heuristics (Section 3.1; T = 0.05, w = 1%, eta = 0.75 as in its hyper-parameter
    study) against the deterministic pick-out and widest-dimension split, in the same sound BaB loop: incumbent
    and gap per iteration, live pool, time per iteration.  Two workloads: the small alpha network (H = 5, where
    the pool prunes) and the pushing network (H = 20)."""
    import torch
    work = {"alpha": ("MLP 6-32-32-4, H=5, 4096 children per iteration, 256 FP32 rollouts each", 2048, "fp32"),
            "pushing": ("MLP 10-128-128-128-8, H=20, 512 children per iteration, 1024 BF16x3 rollouts each", 256,
                        "bf16x3")}
    variants = {"lb_pick_widest_split": None, "softmax_pick_widest_split": {"T": 0.05, "w": 1.0, "split": False},
                "lb_pick_imbalance_split": {"T": None, "w": 1.0, "split": True},
                "softmax_pick_imbalance_split": {"T": 0.05, "w": 1.0, "split": True}}
    out = {"bound": f"sound (interval + CROWN, FP32, margin); {iters} iterations; the gap needs one host sync per "
                    "iteration (included in the time)"}
    for wl, (desc, n_pick, rprec) in work.items():
        res = {"workload": f"{wl}: {desc}"}
        # one untimed pass first, so that no variant is timed while the clocks ramp up
        for name, h in [("warm-up", None)] + list(variants.items()):
            for warm in (True, False):
                st = BabState(wl, SEED, dev, n_pick, rprec, "fp32", pool_iters=iters + 2, heuristics=h)
                torch.cuda.synchronize()
                t = time.perf_counter()
                inc, gaps = [], []
                for _ in range(2 if warm else iters):
                    st.step()
                    if not warm:
                        g, _ = st.gap()
                        inc.append(float(st.inc_val.item()))
                        gaps.append(g)
                torch.cuda.synchronize()
                sec = time.perf_counter() - t
                n_live = int(st.counts[2].item())
                st.close()
            if name == "warm-up":
                continue
            res[name] = {"incumbent": inc[-1], "gap": gaps[-1],
                         "incumbent_every_5": [round(v, 5) for v in inc[4::5]],
                         "gap_every_5": [round(v, 5) for v in gaps[4::5]],
                         "live_pool_end": n_live, "ms_per_iteration": 1e3 * sec / iters}
        out[wl] = res
    return out


def cem_comparison(dev, iters=30):
    """Cross-entropy search (Section 3.3; each child warm-started from its parent's best input, 10 elites as in the
    paper's CEM settings) against uniform samples with the same number of rollouts per box, in the same sound BaB
    loop: incumbent and gap per iteration, time per iteration."""
    import torch
    work = {"alpha": ("MLP 6-32-32-4, H=5, 4096 children per iteration, 256 FP32 rollouts each", 2048, "fp32"),
            "pushing": ("MLP 10-128-128-128-8, H=20, 512 children per iteration, 1024 BF16x3 rollouts each", 256,
                        "bf16x3")}
    variants = {"uniform": None, "cem_4x": {"iters": 4, "elites": 10, "jitter": 1e-3},
                "cem_8x": {"iters": 8, "elites": 10, "jitter": 1e-3}}
    out = {"bound": f"sound (interval + CROWN, FP32, margin); {iters} iterations; the same rollouts per box "
                    "(CEM: samples / iterations per iteration); deterministic pick-out and widest split"}
    for wl, (desc, n_pick, rprec) in work.items():
        res = {"workload": f"{wl}: {desc}"}
        for name, c in [("warm-up", None)] + list(variants.items()):
            for warm in (True, False):
                st = BabState(wl, SEED, dev, n_pick, rprec, "fp32", pool_iters=iters + 2, cem=c)
                torch.cuda.synchronize()
                t = time.perf_counter()
                inc, gaps = [], []
                for _ in range(2 if warm else iters):
                    st.step()
                    if not warm:
                        g, _ = st.gap()
                        inc.append(float(st.inc_val.item()))
                        gaps.append(g)
                torch.cuda.synchronize()
                sec = time.perf_counter() - t
                n_live = int(st.counts[2].item())
                st.close()
            if name == "warm-up":
                continue
            res[name] = {"incumbent": inc[-1], "gap": gaps[-1],
                         "incumbent_every_5": [round(v, 6) for v in inc[4::5]],
                         "live_pool_end": n_live, "ms_per_iteration": 1e3 * sec / iters}
        out[wl] = res
    return out


SYNTH_G_STAR = -0.98033911  # per-coordinate minimum of 5 u^2 + cos(50 u) (the oracle pins it to 1e-6)


def synthetic_bab(dev, d=100, iters=1000, n_pick=512, samples=256, cem_iters=0, levels=10, eta=0.75):
    """Algorithm 2 on the paper's synthetic objective (Section 4): f(u) = sum 5 u_i^2 + cos(50 u_i) over
    [-1, 1]^d, d = 100.  Search: `samples` uniform draws per child, or the cross-entropy search (cem_iters
    iterations of samples / cem_iters, 10 elites, each child warm-started from its parent's best input); bound:
    the sound per-term interval minima; prune / pick-out / widest-dimension bisection on the device.  Reports the
    incumbent against f* = d g*, the certified gap and the coordinates in the global basin."""
    import torch
    from paper_2412_09584_gb300 import binding as B
    from paper_2412_09584_gb300 import workloads as W
    ctx = B.bab_context_create()
    f = dict(device=dev, dtype=torch.float32)
    lo, hi, ids = W.grid_boxes(d, levels)
    n0 = lo.shape[0]
    cap = n0 + (iters + 2) * n_pick
    pools = [{"lo": torch.empty(cap, d, **f), "hi": torch.empty(cap, d, **f), "lb": torch.empty(cap, **f),
              "ub": torch.empty(cap, **f), "id": torch.empty(cap, dtype=torch.int64, device=dev),
              "bu": torch.empty(cap, d, **f)} for _ in range(2)]
    P = pools[0]
    P["lo"][:n0] = torch.as_tensor(lo).to(**f)
    P["hi"][:n0] = torch.as_tensor(hi).to(**f)
    P["id"][:n0] = torch.as_tensor(ids.astype(np.int64)).to(dev)
    iv = torch.full((1,), float("inf"), dtype=torch.float64, device=dev)
    iu = torch.zeros(d, **f)
    keep = torch.empty(cap, dtype=torch.uint8, device=dev)
    counts = torch.zeros(3, dtype=torch.int32, device=dev)
    live = torch.tensor([n0], dtype=torch.int32, device=dev)
    m_it = samples // cem_iters if cem_iters else samples

    def search(Q, n, d_n, seed, warm):
        B.bab_synth_search(ctx, d, Q["lo"], Q["hi"], Q["id"], n, m_it, seed, Q["ub"], Q["bu"], iters=cem_iters,
                           elites=10, jitter=1e-3, warm_u=warm, inc_val=iv, inc_u=iu, d_n=d_n)
        B.bab_synth_bound(ctx, d, Q["lo"], Q["hi"], n, Q["lb"], d_n=d_n)

    search(P, n0, None, 1, None)
    cur, nmax = 0, n0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(iters):
        src, dst = pools[cur], pools[cur ^ 1]
        B.bab_prune_branch_heuristic(ctx, d, src["lo"], src["hi"], src["lb"], src["ub"], src["id"], nmax, iv,
                                     n_pick, eta, B.PICK_LB, 1.0, 0, cap, dst["lo"], dst["hi"], dst["lb"],
                                     dst["ub"], dst["id"], keep, counts, row_u=src["bu"], out_row_u=dst["bu"],
                                     d_n=live)
        nmax = min(nmax + n_pick, cap - n_pick)
        search(dst, 2 * n_pick, counts[0:1], 2 + it, dst["bu"] if cem_iters else None)
        live.copy_(counts[2:3])
        cur ^= 1
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    nl = int(counts[2].item())
    lbmin = float(pools[cur]["lb"][:nl].min().item()) if nl else float("inf")
    inc = float(iv.item())
    u = iu.cpu().numpy().astype(np.float64)
    g = 5 * u * u + np.cos(50 * u)
    status = B.bab_status(ctx)
    B.bab_destroy(ctx)
    return {"d": d, "f_star": d * SYNTH_G_STAR, "incumbent": inc, "gap_to_f_star": inc - d * SYNTH_G_STAR,
            "certified_gap": inc - min(lbmin, inc), "coordinates_in_global_basin": int((g < SYNTH_G_STAR + 0.05).sum()),
            "iterations": iters, "children_per_iteration": 2 * n_pick, "eta": eta,
            "search": f"cross-entropy {cem_iters} x {m_it}, warm-started" if cem_iters else f"{samples} uniform",
            "live_pool_end": nl, "ms_per_iteration": 1e3 * sec / iters, "status": status}


def synthetic_sweep(dev):
    """The synthetic objective at d = 10, 30 and 100 (the paper's figure spans d <= 100): warm-started
    cross-entropy search (4 x 64 per child), eta = 0.25, 1024 children per iteration."""
    out = {}
    for d, iters in ((10, 300), (30, 600), (100, 1000)):
        out[f"d{d}"] = synthetic_bab(dev, d=d, iters=iters, cem_iters=4, eta=0.25, levels=min(10, d))
    return out


def obstacle_bab(dev, iters=30):
    """Algorithm 2 with the pushing-with-obstacles cost (Appendix D.4: weighted norm to the target, w_t = t / H,
    plus lambda = 10 times the obstacle penalties of the pusher and the 4 keypoints; 3 obstacles) on the pushing
    network: 512 children per iteration, 1024 BF16x3 rollouts each (uniform, or the warm-started cross-entropy
    search 4 x 256 in FP32), sound FP32 interval + CROWN bounds, or alpha-CROWN (20 Adam steps per iteration); and
    the headline arithmetic (BF16 rollouts with the picks re-scored in FP32, CROWN on tensor cores)."""
    import torch
    from paper_2412_09584_gb300 import workloads as W
    p = W.config_problem("pushing", SEED)
    cost = W.obstacle_cost(p["H"], SEED)
    out = {"workload": "pushing network, H=20, 3 obstacles, lambda 10, w_t = t/H; sound FP32 bounds (CROWN, or "
                       f"alpha-CROWN with 20 Adam steps); {iters} iterations",
           "obstacles": [[round(v, 4) for v in o] for o in cost["obstacles"]]}
    variants = (("uniform_bf16x3", dict(rollout_prec="bf16x3")),
                ("cem_fp32_4x256", dict(rollout_prec="fp32", cem={"iters": 4, "elites": 10, "jitter": 1e-3})),
                ("uniform_bf16x3_alpha20", dict(rollout_prec="bf16x3", alpha_steps=20)),
                ("uniform_bf16_tc_crown", dict(rollout_prec="bf16", bound_prec="bf16x3")))
    # one untimed pass first, so that no variant is timed while the clocks ramp up
    for name, kw in (("warm-up", variants[0][1]),) + variants:
        for warm in (True, False):
            kw2 = dict(bound_prec="fp32", **kw) if "bound_prec" not in kw else kw
            st = BabState("pushing", SEED, dev, 256, pool_iters=iters + 2, cost=cost, **kw2)
            torch.cuda.synchronize()
            t = time.perf_counter()
            inc, gaps = [], []
            for _ in range(2 if warm else iters):
                st.step()
                if not warm:
                    g, _ = st.gap()
                    inc.append(float(st.inc_val.item()))
                    gaps.append(g)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t
            n_live = int(st.counts[2].item())
            status = st.B.bab_status(st.ctx)
            st.close()
        if name == "warm-up":
            continue
        out[name] = {"incumbent": inc[-1], "gap": gaps[-1], "incumbent_every_5": [round(v, 5) for v in inc[4::5]],
                     "live_pool_end": n_live, "ms_per_iteration": 1e3 * sec / iters, "status": status}
    return out


def tiny_latency(dev, reps=200):
    """Configuration 1 (the small sanity case): MLP 6-32-32-4, H = 5, 64 children per iteration (32 picked),
    256 FP32 rollouts each, FP32 interval + CROWN bounds.  Latency-bound: microseconds per BaB iteration as a
    CUDA-graph replay (and as eager launches), inputs resident."""
    import torch
    out = {"workload": "tiny: MLP 6-32-32-4, H=5, 64 children per iteration, 256 FP32 rollouts each, FP32 bounds"}
    st = BabState("tiny", SEED, dev, 32, "fp32", "fp32", fixed_launch=True, pool_iters=2 * reps + 64)
    for _ in range(3):
        st.step()
    graphs = capture_graphs(st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graphs[st.cur].replay()
        st.cur ^= 1
    e1.record()
    torch.cuda.synchronize()
    out["us_per_iteration_graph"] = 1e3 * e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps // 4):
        st.step()
    e1.record()
    torch.cuda.synchronize()
    out["us_per_iteration_eager"] = 1e3 * e0.elapsed_time(e1) / (reps // 4)
    for _ in range(5):
        st.step(events=True)
    torch.cuda.synchronize()
    out["us_rollout"] = 1e3 * float(np.mean([e[0].elapsed_time(e[1]) for e in st.ev[-5:]]))
    out["us_bound"] = 1e3 * float(np.mean([e[1].elapsed_time(e[2]) for e in st.ev[-5:]]))
    out["launches_per_iteration"] = st.launches_per_step
    out["status"] = st.B.bab_status(st.ctx)
    st.close()
    return out


def time_to_gap(dev, workload="alpha", n_pick=2048, iters=20, max_iters=60, variants=None):
    """Wall time for alpha-optimised and split-precision BaB variants to reach the optimality gap that plain FP32
    CROWN+IBP BaB reaches after `iters` iterations.  Gap = FP64 incumbent - smallest lower bound of the live pool
    (read back every iteration by every variant alike)."""
    import torch

    def run(rprec, bprec, alpha_steps, n_iter, target=None, iprec="fp32"):
        st = BabState(workload, SEED, dev, n_pick, rprec, bprec, alpha_steps=alpha_steps,
                      pool_iters=max_iters + 2, autotune=True, interval_prec=iprec)
        torch.cuda.synchronize()
        t = time.perf_counter()
        hist = []
        for it in range(n_iter):
            st.step()
            g, n = st.gap()
            hist.append((time.perf_counter() - t, g, n))
            if target is not None and g <= target:
                break
        st.close()
        run.variants = st.variants
        return hist

    # plain: FP32 rollouts and FP32 CROWN; split: 3-term BF16 tensor-core rollouts and CROWN; alpha_split: split
    # plus 5 Adam steps per iteration (alpha_split_20: 20), each a tensor-core CROWN + adjoint + Adam launch;
    # alpha_fused: 3-term BF16 rollouts plus the 20-step alpha-CROWN loop in one FP32 launch per iteration;
    # alpha_fused_5, alpha_fused_2: the same with 5 or 2 Adam steps (the bound gains most in the first steps);
    # *_tc_intervals (*_tf32_intervals): the interval bounds on tensor cores as well, BF16 (TF32) halves;
    # headline*: the bench's own arithmetic (BF16 rollouts with the picks re-scored in FP32, tensor-core CROWN),
    # plain or with 2 tensor-core Adam steps
    if variants is None:
        variants = {"plain_fp32": ("fp32", "fp32", 0), "split": ("bf16x3", "bf16x3", 0),
                    "alpha_split": ("bf16x3", "bf16x3", 5), "alpha_split_20": ("bf16x3", "bf16x3", 20),
                    "alpha_fused": ("bf16x3", "fp32", 20), "alpha_fused_5": ("bf16x3", "fp32", 5),
                    "alpha_fused_2": ("bf16x3", "fp32", 2), "alpha_split_2": ("bf16x3", "bf16x3", 2),
                    "split_tc_intervals": ("bf16x3", "bf16x3", 0, "bf16x3"),
                    "alpha_split_tc_intervals": ("bf16x3", "bf16x3", 5, "bf16x3"),
                    "headline": ("bf16", "bf16x3", 0), "headline_alpha_2": ("bf16", "bf16x3", 2)}
    def go(v, **kw):  # a variant: (rollout, CROWN products, Adam steps[, interval bounds])
        return run(*v[:3], iprec=v[3] if len(v) > 3 else "fp32", **kw)

    for v in variants.values():  # load every kernel and size every scratch buffer before timing
        go(v, n_iter=2)
    plain = go(variants["plain_fp32"], n_iter=iters)
    target = plain[-1][1]
    c = W_CONFIGS()[workload]
    dims = "-".join(str(x) for x in [c["s"] + c["k"]] + list(c["hidden"]) + [c["s"]])
    out = {"workload": f"{workload}: MLP {dims}, H={c['H']}, {2 * n_pick} children per iteration, "
                       f"{c['samples']} rollouts each; gap = FP64 incumbent - min lower bound of the live pool; "
                       f"target = plain FP32 BaB's gap after {iters} iterations", "target_gap": target}
    plain_variants = run.variants
    for name, v in variants.items():
        h = plain if name == "plain_fp32" else go(v, n_iter=max_iters, target=target)
        reached = h[-1][1] <= target
        out[name] = {"seconds": h[-1][0], "iterations": len(h), "reached": reached,
                     "ms_per_iteration": 1e3 * h[-1][0] / len(h), "gap_curve": [round(x[1], 6) for x in h],
                     "rollout": v[0], "bound": v[1], "alpha_steps": v[2], "intervals": v[3] if len(v) > 3 else "fp32",
                     "launch_variants": plain_variants if name == "plain_fp32" else run.variants}
        if name != "plain_fp32":
            out[name]["speedup_vs_plain"] = plain[-1][0] / h[-1][0] if reached else None
    return out


def W_CONFIGS():
    from paper_2412_09584_gb300 import workloads as W
    return W.CONFIGS


def time_to_gap_pushing(dev):
    """Time-to-gap on the pushing network (MLP 10-128-128-128-8, H = 20), 512 children per iteration."""
    variants = {"plain_fp32": ("fp32", "fp32", 0), "split": ("bf16x3", "bf16x3", 0),
                "split_fp32_bound": ("bf16x3", "fp32", 0), "alpha_fused": ("bf16x3", "fp32", 20),
                "alpha_fused_5": ("bf16x3", "fp32", 5), "alpha_split": ("bf16x3", "bf16x3", 5),
                "alpha_fused_2": ("bf16x3", "fp32", 2), "alpha_split_2": ("bf16x3", "bf16x3", 2),
                "split_tc_intervals": ("bf16x3", "bf16x3", 0, "bf16x3"),
                "alpha_split_tc_intervals": ("bf16x3", "bf16x3", 5, "bf16x3"),
                "headline": ("bf16", "bf16x3", 0), "headline_alpha_2": ("bf16", "bf16x3", 2),
                "headline_tc_intervals": ("bf16", "bf16x3", 0, "bf16x3"),
                "headline_tf32_intervals": ("bf16", "bf16x3", 0, "tf32x3")}
    return time_to_gap(dev, "pushing", n_pick=256, iters=10, max_iters=30, variants=variants)


def oracle_sample_step(problem, lo, hi, ids, M, n_roll, n_bound, pool_n, n_pick):
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
    O.prune_branch(plo, phi, lb, ub, pid, 11.0, n_pick)
    t_prune = time.perf_counter() - t
    return t_roll, t_bound, t_prune


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker_init():
    from oracle import oracle as O
    O.lib()


def _oracle_boxes(job):
    """One worker's share of the all-cores baseline: the oracle's rollouts and CROWN bounds of a few boxes."""
    problem, lo, hi, ids, M = job
    from oracle import oracle as O
    O.rollout(problem, lo, hi, ids, M, SEED)
    O.crown(problem, lo, hi)
    return lo.shape[0]


def oracle_pool(cores):
    """A pool of `cores` fresh interpreters (spawned, so it is safe after CUDA is initialised), warmed up."""
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init)
    pool.map(abs, range(cores))
    return pool


def oracle_boxes_parallel(pool, cores, problem, lo, hi, ids, M, per_worker):
    """Wall seconds for `cores` workers to search and bound `per_worker` distinct boxes each."""
    jobs = [(problem, lo[w * per_worker:(w + 1) * per_worker], hi[w * per_worker:(w + 1) * per_worker],
             ids[w * per_worker:(w + 1) * per_worker], M) for w in range(cores)]
    t = time.perf_counter()
    done = sum(pool.map(_oracle_boxes, jobs))
    assert done == cores * per_worker
    return time.perf_counter() - t


def cpu_baseline(budget_s=20.0, n_pick=2048):
    """The FP64 oracle, as it stands, on the host: one process over every host core (independent boxes split
    across spawned workers), and one thread; bounded samples scaled to one iteration of 2 n_pick children."""
    from paper_2412_09584_gb300 import workloads as W
    c = W.CONFIGS["pushing"]
    p = W.config_problem("pushing", SEED)
    lo, hi, ids = W.grid_boxes(c["H"] * p["k"], c["grid_dims"])
    # calibrate on one box, then size the sample to the budget
    t_roll, t_bound, t_prune = oracle_sample_step(p, lo, hi, ids, c["samples"], 1, 4, 4096, n_pick)
    single_budget = 0.5 * budget_s
    n_roll = max(1, min(64, int(0.7 * single_budget / max(t_roll, 1e-6))))
    n_bound = max(4, min(4096, int(0.2 * single_budget / max(t_bound, 1e-6))))
    t_roll, t_bound, t_prune = oracle_sample_step(p, lo, hi, ids, c["samples"], n_roll, n_bound, 4096 + n_pick,
                                                  n_pick)
    step_s = 2 * n_pick * (t_roll + t_bound) + t_prune
    single = {"value": 2 * n_pick / step_s, "cores": 1,
              "sample": f"rollouts of {n_roll} boxes x {c['samples']} samples x H={c['H']}, CROWN of {n_bound} "
                        f"boxes, prune/branch of a {4096 + n_pick}-box pool; per-box times scaled to one "
                        f"{2 * n_pick}-box iteration ({step_s:.1f} s)"}
    cores = host_cores()
    per_worker = max(1, min(lo.shape[0] // cores, int(0.5 * budget_s / max(t_roll + t_bound, 1e-6))))
    pool = oracle_pool(cores)
    try:
        wall = oracle_boxes_parallel(pool, cores, p, lo, hi, ids, c["samples"], per_worker)
    finally:
        pool.close()
        pool.join()
    step_all = 2 * n_pick * wall / (cores * per_worker) + t_prune
    return {"value": 2 * n_pick / step_all, "unit": "subdomain-bounds/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle in {cores} spawned processes: {cores} x {per_worker} distinct boxes, each "
                      f"{c['samples']} rollouts of H={c['H']} then CROWN ({wall:.1f} s wall), plus one prune/branch of "
                      f"a {4096 + n_pick}-box pool; scaled to one {2 * n_pick}-box iteration ({step_all:.1f} s)",
            "single_thread": single}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2412_09584_gb300 import workloads as W
    O.build()
    c = W.CONFIGS["pushing"]
    p = W.config_problem("pushing", SEED)
    lo, hi, ids = W.grid_boxes(c["H"] * p["k"], c["grid_dims"])
    # one box per host core per step (independent boxes in spawned workers), then prune/branch in this process
    cores = host_cores()
    pool = oracle_pool(cores)
    rng = np.random.default_rng(0)
    pool_n = 1024
    lb = rng.normal(10, 3, pool_n).astype(np.float32)
    ub = (lb + 1).astype(np.float32)
    plo, phi = lo[:pool_n], hi[:pool_n]
    pid = np.arange(1, pool_n + 1, dtype=np.uint64)

    def step(i):
        off = (i * cores) % (lo.shape[0] - cores)
        oracle_boxes_parallel(pool, cores, p, lo[off:], hi[off:], ids[off:], c["samples"], 1)
        O.prune_branch(plo, phi, lb, ub, pid, 11.0, args.boxes // 2)

    try:
        for i in range(args.warmup):
            step(i)
        t = time.perf_counter()
        for i in range(args.steps):
            step(args.warmup + i)
        sec = (time.perf_counter() - t) / args.steps
    finally:
        pool.close()
        pool.join()
    value = cores / sec
    sample = (f"per step: FP64 C oracle on {cores} boxes, one per spawned process (1024 rollouts of H=20 each, then "
              f"CROWN), and prune/branch of a {pool_n}-box pool")
    cfg = {"workload": "pushing-scale BaB iteration: state 8, action 2, MLP 10-128-128-128-8 ReLU residual, H=20, "
                       "rho=0.01, 1024 uniform rollouts per child (bounded sample per step)",
           "boxes_per_step": cores, "samples_per_box": c["samples"], "H": c["H"]}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "subdomain-bounds/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": "subdomain-bounds/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "subdomain-bounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-gap", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of CUDA-graph replays")
    ap.add_argument("--no-autotune", action="store_true", help="built-in launch heuristics instead of bab_autotune")
    ap.add_argument("--no-batched", action="store_true", help="skip the many-problem BaB section")
    ap.add_argument("--no-manip", action="store_true", help="skip the object-manipulation-scale section")
    ap.add_argument("--no-precision-lines", action="store_true",
                    help="skip the same iteration with the rollouts in the other arithmetics")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--interval-precision", choices=["fp32", "bf16x3", "tf32x3"], default="fp32",
                    help="interval bounds: fp32 (directed rounding, CUDA cores), bf16x3 or tf32x3 (tcgen05, 3-term "
                         "split, computed margin)")
    ap.add_argument("--bound-precision", choices=sorted(BOUND_PRECISIONS), default="bf16x3",
                    help="CROWN products: fp32 (CUDA cores), bf16x3 or tf32x3 (tcgen05, 3-term split, "
                         "margin-corrected)")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="bf16",
                    help="rollout arithmetic: fp32 (CUDA cores), bf16x3 (tcgen05, 3-term split), bf16 (tcgen05)")
    ap.add_argument("--boxes", type=int, default=4096,
                    help="children bounded per iteration; smaller values make small cases for profiler captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
