"""Batched problems (several planning problems of one architecture, uneven horizons, rows of all problems in one
launch): every row must match the single-problem path on its own problem bit for bit, and the FP64 oracle within
the FP32 tolerances; prune / pick-out / split per problem must be bit-exact against the oracle run per problem."""
import numpy as np
import pytest
import torch

from paper_2412_09584_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


class Batch:
    def __init__(self, P=5, seed=3, H_lo=2, H_hi=7):
        from gpu_util import T
        from paper_2412_09584_gb300 import binding as B
        self.B = B
        self.probs, _ = W.batch_problems(P, seed, H_lo=H_lo, H_hi=H_hi)
        params, x0, goal, Hs, rho = W.pack_batch(self.probs)
        self.Hs = Hs
        self.Hmax = int(Hs.max())
        self.k = self.probs[0]["k"]
        self.dst = self.k * self.Hmax
        self.ctx = B.bab_load_dynamics_batch(self.probs[0]["dims"], params, self.probs[0]["s"], self.k)
        self.x0, self.goal, self.tH, self.trho = T(x0), T(goal), T(Hs, torch.int32), T(rho)
        self.P = P

    def close(self):
        self.B.bab_destroy(self.ctx)

    def dp(self, p):
        return self.k * int(self.Hs[p])


def _rows(bt, seed, counts):
    return W.batch_random_boxes(bt.probs, counts, bt.dst, seed)


@pytest.mark.parametrize("prec_name,M", [("fp32", 64), ("bf16x3", 200), ("bf16", 130)])
def test_batch_rollout_matches_single_and_oracle(oracle, prec_name, M):
    """FP32 on CUDA cores, or tensor cores with each tile streaming its own problem's weights: every row equals
    the single-problem call on its problem bit for bit (the single-problem BF16 call taken layer by layer, as the
    batched kernel runs; its default fused-step kernel is compared with it in test_gpu_variants)."""
    from gpu_util import DEV, GpuProblem, T, ids_t
    bt = Batch()
    B = bt.B
    prec = {"fp32": B.PREC_FP32, "bf16x3": B.PREC_BF16X3, "bf16": B.PREC_BF16}[prec_name]
    try:
        lo, hi, ids, prob = _rows(bt, 1, [7, 3, 9, 5, 6])
        n, seed = lo.shape[0], 11
        ub = torch.empty(n, device=DEV)
        best_u = torch.empty(n, bt.dst, device=DEV)
        inc_val = torch.full((bt.P,), np.inf, dtype=torch.float64, device=DEV)
        inc_u = torch.zeros(bt.P, bt.dst, device=DEV)
        B.bab_rollout_batch(bt.ctx, bt.x0, bt.goal, bt.tH, bt.trho, bt.Hmax, bt.dst, T(lo), T(hi), ids_t(ids),
                            T(prob, torch.int32), n, M, seed, ub, best_u, inc_val, inc_u, precision=prec)
        torch.cuda.synchronize()
        ub, best_u = ub.cpu().numpy(), best_u.cpu().numpy()
        inc_val, inc_u = inc_val.cpu().numpy(), inc_u.cpu().numpy()
        for p in range(bt.P):
            rows = np.nonzero(prob == p)[0]
            dp = bt.dp(p)
            g = GpuProblem(bt.probs[p])
            try:
                B.bab_set_variant(g.ctx, B.KERNEL_ROLLOUT_TC, 4)  # two tiles per CTA, layer by layer
                r = g.rollout(lo[rows, :dp], hi[rows, :dp], ids[rows], M=M, seed=seed, precision=prec)
            finally:
                g.close()
            assert np.array_equal(ub[rows].view(np.uint32), r["ub"].view(np.uint32))
            assert np.array_equal(best_u[rows, :dp].view(np.uint32), r["best_u"].view(np.uint32))
            assert np.all(best_u[rows, dp:] == 0)
            ub_o, _, _ = oracle.rollout(bt.probs[p], lo[rows, :dp], hi[rows, :dp], ids[rows], M, seed)
            if prec_name == "bf16":  # each row's best BF16 sample, re-scored in FP32
                f_b = np.array([oracle.objective(bt.probs[p], u[:dp].astype(np.float64)) for u in best_u[rows]])
                np.testing.assert_allclose(ub[rows], f_b, rtol=REL)
            else:
                np.testing.assert_allclose(ub[rows], ub_o, rtol=REL, atol=0)
            f = oracle.objective(bt.probs[p], inc_u[p, :dp].astype(np.float64))
            assert inc_val[p] == pytest.approx(f, rel=1e-10)
            assert inc_val[p] <= ub[rows].min() * (1 + 2 * REL)
    finally:
        bt.close()


@pytest.mark.parametrize("steps", [0, 4])
def test_batch_bound_matches_single_and_oracle(oracle, steps):
    from gpu_util import DEV, GpuProblem, T
    bt = Batch(seed=5)
    B = bt.B
    try:
        lo, hi, ids, prob = _rows(bt, 2, [4, 8, 2, 6, 5])
        n = lo.shape[0]
        lb = torch.empty(n, device=DEV)
        lb_ibp = torch.empty(n, device=DEV)
        B.bab_bound_batch(bt.ctx, bt.x0, bt.goal, bt.tH, bt.trho, bt.Hmax, bt.dst, T(lo), T(hi),
                          T(prob, torch.int32), n, lb, alpha_steps=steps, lr=0.1, lb_ibp=lb_ibp)
        torch.cuda.synchronize()
        lb, lb_ibp = lb.cpu().numpy(), lb_ibp.cpu().numpy()
        for p in range(bt.P):
            rows = np.nonzero(prob == p)[0]
            dp = bt.dp(p)
            plo, phi = lo[rows, :dp], hi[rows, :dp]
            g = GpuProblem(bt.probs[p])
            try:
                ibp_lb, _, _, _, _ = g.ibp(plo, phi)
                assert np.array_equal(lb_ibp[rows].view(np.uint32), ibp_lb.view(np.uint32))
                if steps == 0:
                    single = g.crown(plo, phi)["lb"]
                else:
                    best = torch.empty(len(rows), device=DEV)
                    B.bab_alpha_optimize(g.ctx, g.x0, g.goal, g.H, g.rho, T(plo), T(phi), len(rows), steps, 0.1, best)
                    single = best.cpu().numpy()
            finally:
                g.close()
            assert np.array_equal(lb[rows].view(np.uint32), single.view(np.uint32))
            o = oracle.crown(bt.probs[p], plo, phi)
            scale = np.maximum(o["scale"], 1.0)
            if steps == 0:
                assert np.all(np.abs(lb[rows] - o["lb"]) <= 2 * REL * scale)
            else:
                best_o, _, _, _ = oracle.alpha_optimize(bt.probs[p], plo, phi, steps, 0.1)
                assert np.all(np.abs(lb[rows] - best_o) <= 1e-3 * scale)
            assert np.all(lb[rows] <= (o["lb"] if steps == 0 else best_o) + 1e-12 * scale)
    finally:
        bt.close()


@pytest.mark.parametrize("seed,n_pick", [(1, [2, 0, 5, 9, 3]), (4, [40, 40, 40, 40, 40]), (7, [1, 2, 3, 4, 5])])
def test_batch_prune_branch_bit_exact(oracle, seed, n_pick):
    from gpu_util import DEV, T, ids_t
    bt = Batch(seed=seed)
    B = bt.B
    try:
        lo, hi, ids, prob = _rows(bt, seed, [12, 30, 7, 19, 25])
        n = lo.shape[0]
        lb, ub = W.pool_values(n, seed=seed, nan_frac=0.02, tie_frac=0.1)
        inc = np.array([np.median(lb[prob == p][~np.isnan(lb[prob == p])]) for p in range(bt.P)], dtype=np.float64)
        tot = int(sum(n_pick))
        cap = n + tot + 1
        f = dict(device=DEV)
        out = [torch.full((cap, bt.dst), np.nan, **f), torch.full((cap, bt.dst), np.nan, **f),
               torch.empty(cap, **f), torch.empty(cap, **f), torch.zeros(cap, dtype=torch.int64, **f),
               torch.full((cap,), -1, dtype=torch.int32, **f)]
        keep = torch.empty(n, dtype=torch.uint8, **f)
        counts = torch.zeros(3, dtype=torch.int32, **f)
        pcounts = torch.zeros(bt.P, 2, dtype=torch.int32, **f)
        B.bab_status(bt.ctx)
        B.bab_prune_branch_batch(bt.ctx, bt.dst, bt.tH, bt.Hmax, T(lo), T(hi), T(lb), T(ub), ids_t(ids),
                                 T(prob, torch.int32), n, torch.tensor(inc, dtype=torch.float64, **f),
                                 T(np.array(n_pick), torch.int32), tot, 0.75, cap, *out, keep, counts, pcounts)
        assert B.bab_status(bt.ctx) == (-6 if np.isnan(lb).any() else 0)  # NaN bounds are kept and reported
        o_lo, o_hi, o_lb, o_ub, o_id, o_pr = [x.cpu().numpy() for x in out]
        keep, counts, pcounts = keep.cpu().numpy(), counts.cpu().numpy(), pcounts.cpu().numpy()
        exp = [oracle.prune_branch(lo[prob == p, :bt.dp(p)], hi[prob == p, :bt.dp(p)], lb[prob == p], ub[prob == p],
                                   ids[prob == p], inc[p], n_pick[p]) for p in range(bt.P)]
        tc = sum(e["n_children"] for e in exp)
        tr = sum(e["n_rest"] for e in exp)
        assert list(counts) == [tc, tr, tc + tr]
        row = 0
        for part in ("children", "rest"):
            for p, e in enumerate(exp):
                m = e["n_children"] if part == "children" else e["n_rest"]
                sl = slice(0, e["n_children"]) if part == "children" else slice(e["n_children"], e["n_children"] + m)
                dp = bt.dp(p)
                rr = slice(row, row + m)
                assert np.array_equal(o_lo[rr, :dp].view(np.uint32), e["lo"][sl].view(np.uint32))
                assert np.array_equal(o_hi[rr, :dp].view(np.uint32), e["hi"][sl].view(np.uint32))
                assert np.all(o_lo[rr, dp:] == 0) and np.all(o_hi[rr, dp:] == 0)
                assert np.array_equal(o_lb[rr].view(np.uint32), e["lb"][sl].view(np.uint32))
                assert np.array_equal(o_ub[rr].view(np.uint32), e["ub"][sl].view(np.uint32))
                assert np.array_equal(o_id[rr].astype(np.uint64), e["id"][sl])
                assert np.all(o_pr[rr] == p)
                if part == "children":
                    assert pcounts[p, 0] * 2 == m
                else:
                    assert pcounts[p, 1] == m
                row += m
        for p, e in enumerate(exp):
            assert np.array_equal(keep[prob == p], e["keep"])
    finally:
        bt.close()
