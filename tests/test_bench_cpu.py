"""Host arithmetic of bench.py, checked on the CPU against hand counts: the rollout roofline's algorithmic and
executed FLOPs, the source digest that keeps a DRAM-traffic capture tied to the kernel it was taken on, and the
command line's precision choices."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

PUSHING = {"dims": [10, 128, 128, 128, 8], "s": 8}  # MLP 10-128-128-128-8, state 8, action 2


def test_rollout_roofline_counts_algorithmic_flops():
    """2 x MACs x rollout-steps over the kernel time: the pushing network has 10*128 + 2*128*128 + 128*8 = 35,072
    MACs per step, so 4096 boxes x 1024 samples x 20 steps in 10 ms are 0.5884 PFLOP / 10 ms = 588.4 TFLOP/s."""
    import bench
    r = bench.rollout_roofline("bf16x3", PUSHING, 4096, 1024, 20, 10.0)
    assert r["achieved"] == pytest.approx(2 * 35072 * 4096 * 1024 * 20 / 1e-2 / 1e12, rel=1e-12)
    assert r["unit"] == "TFLOP/s" and r["bound"] == "tensor"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)


def test_rollout_roofline_executed_work_of_the_split_kernel():
    """Layer by layer, each layer's K and N padded to 16 (layer 1 reads the 16-wide row [u_t | x_t], 8 + 8):
    16*128 + 128*128 + 128*128 + 128*16 = 36,864 executed MACs per step, three times for the 3-term split."""
    import bench
    r = bench.rollout_roofline("bf16x3", PUSHING, 4096, 1024, 20, 10.0)
    assert r["executed_per_algorithmic"] == pytest.approx(3 * 36864 / 35072, rel=1e-12)
    assert r["executed"] == pytest.approx(r["achieved"] * 3 * 36864 / 35072, rel=1e-12)


def test_rollout_roofline_executed_work_of_the_fused_step_kernel():
    """The BF16 fused step: layers 2 and 3 with their bias step ((128 + 16) x 128 each), the fused product of the
    output layer and the next first layer over [a | u x] plus its bias step ((128 + 16 + 16) x (128 + 16)), and
    layer 1 of step 0 once per rollout ((16 + 16) x 128 / H): 59,904 + 204.8 MACs per step."""
    import bench
    r = bench.rollout_roofline("bf16", PUSHING, 4096, 1024, 20, 10.0)
    per_step = 2 * 144 * 128 + 160 * 144 + 32 * 128 / 20
    assert per_step == pytest.approx(60108.8)
    assert r["executed_per_algorithmic"] == pytest.approx(per_step / 35072, rel=1e-12)
    assert r["kernel"].startswith("k_rollout_tcf")


def test_traffic_digest_ignores_comments_and_whitespace_only():
    """A DRAM-traffic capture stays valid across comment and layout edits of the kernel sources, and not across
    code edits."""
    import bench
    a = "int f(int x) {\n  return x + 1; // one more\n}\n"
    b = "/* header */ int f(int x)\n{\n    return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_digest([a]) == bench.code_digest([b])
    assert bench.code_digest([a]) != bench.code_digest([c])


def test_traffic_reported_only_for_its_workload():
    """The stored capture is for BF16 rollouts at 4096 boxes x 1024 samples; any other workload reports none."""
    import bench
    t = bench.ROLLOUT_TC_TRAFFIC
    assert bench.rollout_traffic("bf16", 2048, 1024) is None
    assert bench.rollout_traffic("bf16x3", t["boxes"], t["samples"]) is None
    got = bench.rollout_traffic("bf16", t["boxes"], t["samples"])
    assert got is None or got == t["bytes"]


def test_job_rate_is_whole_job_throughput():
    """Units per rank x ranks over the slowest rank's time."""
    import bench
    assert bench.job_rate(4096, 1, 10.0) == pytest.approx(409600.0)
    assert bench.job_rate(4096, 4, 20.0) == pytest.approx(819200.0)


def test_precision_names_match_the_binding():
    """The bench's precision names map to the header's BAB_PREC_* values."""
    import bench
    from paper_2412_09584_gb300 import binding as B
    assert bench.PRECISIONS == {"fp32": B.PREC_FP32, "bf16x3": B.PREC_BF16X3, "bf16": B.PREC_BF16}
    assert bench.BOUND_PRECISIONS == {"fp32": B.PREC_FP32, "bf16x3": B.PREC_BF16X3, "tf32x3": B.PREC_TF32X3}
