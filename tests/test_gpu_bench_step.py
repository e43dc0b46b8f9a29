"""One BaB iteration (Algorithm 2) exactly as bench.py times it: the pushing-scale iteration with 2048 boxes picked
and split into 4096 children, 1024 tensor-core rollouts per child (BF16 with each child's pick re-scored in FP32,
the bench's default, or the 3-term BF16 split) and interval + CROWN bounds (the CROWN products on tensor cores with
the 3-term BF16 split, the bench's default, or in FP32), replayed from the bench's own CUDA graph.  The new pool's boxes, identifiers and carried bounds are bit-exact against the
oracle's prune/pick-out/bisection of the previous pool; sampled children's upper and lower bounds are compared with
the oracle's, and the incumbent with its FP64 objective."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

REL_BF16X3 = 1e-5  # upper bounds from the 3-term BF16 split: about 2^-16 per product, FP32 accumulation
REL = 1e-5         # FP32 bounds, relative to the oracle's sum of |terms| (at least 1)
REL_TC = 5e-5      # CROWN with 3-term BF16 split products, relative to the same scale


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("precision,bound_precision", [("bf16", "bf16x3"), ("bf16x3", "fp32")])
def test_bench_iteration_matches_oracle(oracle, precision, bound_precision):
    import bench
    dev = torch.device("cuda:0")
    st = bench.BabState("pushing", bench.rank_seed(0), dev, 2048, precision, bound_precision, fixed_launch=True)
    try:
        graphs = bench.capture_graphs(st)
        torch.cuda.synchronize()
        src = st.pool[st.cur]
        n = int(st.counts[2].item())
        snap = {k: src[k][:n].cpu().numpy() for k in ("lo", "hi", "lb", "ub")}
        snap["id"] = src["id"][:n].cpu().numpy().astype(np.uint64)
        inc = float(st.inc_val.item())
        graphs[st.cur].replay()
        st.cur ^= 1
        torch.cuda.synchronize()
        dst = st.pool[st.cur]
        nc, nr, tot = (int(x) for x in st.counts.cpu().numpy())
        o = oracle.prune_branch(snap["lo"], snap["hi"], snap["lb"], snap["ub"], snap["id"], inc, 2048, 0.75)
        assert (nc, nr) == (o["n_children"], o["n_rest"]) and tot == nc + nr
        assert nc == 4096
        got = {k: dst[k][:tot].cpu().numpy() for k in ("lo", "hi", "lb", "ub")}
        got_id = dst["id"][:tot].cpu().numpy().astype(np.uint64)
        for k in ("lo", "hi"):
            assert np.array_equal(got[k].view(np.uint32), o[k].view(np.uint32)), k
        assert np.array_equal(got_id, o["id"])
        # unpicked rows keep their bounds; the children's come from this iteration's search and bound
        for k in ("lb", "ub"):
            assert np.array_equal(got[k][nc:].view(np.uint32), o[k][nc:].view(np.uint32)), k
        rows = [0, 1, nc // 2, nc - 1]
        lo_c, hi_c, id_c = got["lo"][rows], got["hi"][rows], got_id[rows]
        ub_o, _, _ = oracle.rollout(st.p, lo_c, hi_c, id_c, st.M, st.seed)
        if precision == "bf16x3":
            np.testing.assert_allclose(got["ub"][rows], ub_o, rtol=REL_BF16X3, atol=0)
        else:
            # BF16 picks a sample; its ub is that sample's FP32 objective: never below the best of the same samples
            f_pick = np.array([oracle.objective(st.p, u.astype(np.float64)) for u in st.best_u[:nc].cpu().numpy()[rows]])
            np.testing.assert_allclose(got["ub"][rows], f_pick, rtol=REL, atol=0)
            assert np.all(got["ub"][rows] >= ub_o * (1 - REL))
            np.testing.assert_allclose(got["ub"][rows], ub_o, rtol=1e-2)
        oc = oracle.crown(st.p, lo_c, hi_c)
        margin = st.margin[:nc].cpu().numpy()[rows]
        scale = np.maximum(oc["scale"], 1.0)
        tol = REL_TC if bound_precision == "bf16x3" else REL
        assert np.all(np.abs(got["lb"][rows] + margin - oc["lb"]) <= tol * scale)
        assert np.all(got["lb"][rows] <= oc["lb"])
        # every child: its lower bound below its sampled upper bound
        assert np.all(got["lb"][:nc] <= got["ub"][:nc])
        inc_u = st.inc_u.cpu().numpy().astype(np.float64)
        assert float(st.inc_val.item()) == pytest.approx(oracle.objective(st.p, inc_u), rel=1e-10)
        assert float(st.inc_val.item()) <= inc
    finally:
        st.close()
