"""Helpers for the GPU tests: run the CUDA path through the C-ABI binding on numpy inputs."""
import numpy as np
import torch

from paper_2412_09584_gb300 import binding as B

DEV = torch.device("cuda:0")


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def ids_t(ids):
    return torch.as_tensor(np.asarray(ids, dtype=np.uint64).astype(np.int64)).to(DEV)


class GpuProblem:
    """A loaded context plus the problem tensors on cuda:0."""

    def __init__(self, problem):
        self.p = problem
        self.ctx = B.bab_load_dynamics(problem["dims"], problem["params"], problem["s"], problem["k"])
        self.x0 = T(problem["x0"])
        self.goal = T(problem["goal"])
        self.H = int(problem["H"])
        self.rho = float(problem["rho"])
        self.d = problem["k"] * self.H
        self.sumh = int(sum(problem["dims"][1:-1]))

    def close(self):
        B.bab_destroy(self.ctx)

    def rollout(self, lo, hi, ids, M, seed, precision=B.PREC_FP32, incumbent=False):
        n = lo.shape[0]
        ub = torch.empty(n, device=DEV)
        best_u = torch.empty(n, self.d, device=DEV)
        inc_val = torch.full((1,), np.inf, dtype=torch.float64, device=DEV) if incumbent else None
        inc_u = torch.zeros(self.d, device=DEV) if incumbent else None
        B.bab_rollout(self.ctx, self.x0, self.goal, self.H, self.rho, T(lo), T(hi), ids_t(ids), n, M, seed,
                      precision, ub, best_u, inc_val, inc_u)
        torch.cuda.synchronize()
        out = {"ub": ub.cpu().numpy(), "best_u": best_u.cpu().numpy()}
        if incumbent:
            out["inc_val"] = float(inc_val.item())
            out["inc_u"] = inc_u.cpu().numpy()
        return out

    def ibp(self, lo, hi):
        n = lo.shape[0]
        lb = torch.empty(n, device=DEV)
        pl = torch.empty(n, self.H, max(self.sumh, 1), device=DEV)
        pu = torch.empty_like(pl)
        xl = torch.empty(n, self.H + 1, self.p["s"], device=DEV)
        xu = torch.empty_like(xl)
        B.bab_bound_ibp(self.ctx, self.x0, self.goal, self.H, self.rho, T(lo), T(hi), n, lb, pl, pu, xl, xu)
        torch.cuda.synchronize()
        return lb.cpu().numpy(), pl.cpu().numpy()[:, :, :self.sumh], pu.cpu().numpy()[:, :, :self.sumh], \
            xl.cpu().numpy(), xu.cpu().numpy()

    def crown(self, lo, hi, alpha=None, precision=B.PREC_FP32):
        n = lo.shape[0]
        lb = torch.empty(n, device=DEV)
        mg = torch.empty(n, device=DEV)
        mu = torch.empty(n, self.d, device=DEV)
        cst = torch.empty(n, device=DEV)
        B.bab_bound_crown(self.ctx, self.x0, self.goal, self.H, self.rho, T(lo), T(hi), n, lb,
                          alpha=None if alpha is None else T(alpha), precision=precision, margin=mg, lin_coef=mu,
                          lin_const=cst)
        torch.cuda.synchronize()
        return {"lb": lb.cpu().numpy(), "margin": mg.cpu().numpy(), "lin_coef": mu.cpu().numpy(),
                "lin_const": cst.cpu().numpy()}

    def alpha_init(self, lo, hi):
        n = lo.shape[0]
        alpha = torch.empty(n, self.H, self.sumh, device=DEV)
        B.bab_alpha_init(self.ctx, self.x0, self.goal, self.H, self.rho, T(lo), T(hi), n, alpha)
        return alpha

    def alpha_steps(self, lo, hi, steps, lr, alpha=None, precision=B.PREC_FP32):
        n = lo.shape[0]
        tlo, thi = T(lo), T(hi)
        alpha = self.alpha_init(lo, hi) if alpha is None else T(alpha)
        m = torch.zeros_like(alpha)
        v = torch.zeros_like(alpha)
        lb_best = torch.full((n,), -np.inf, device=DEV)
        lb = torch.empty(n, device=DEV)
        g = torch.empty_like(alpha)
        hist = []
        for step in range(1, steps + 1):
            B.bab_alpha_step(self.ctx, self.x0, self.goal, self.H, self.rho, tlo, thi, n, alpha, m, v, step, lr,
                             lb=lb, lb_best=lb_best, grad_alpha=g, precision=precision)
            hist.append({"lb": lb.cpu().numpy(), "grad": g.cpu().numpy(), "alpha": alpha.cpu().numpy()})
        torch.cuda.synchronize()
        return lb_best.cpu().numpy(), alpha.cpu().numpy(), hist

    def prune_branch(self, lo, hi, lb, ub, ids, inc_val, n_pick, eta=0.75):
        n, d = lo.shape
        cap = n + n_pick + 1
        out = [torch.full((cap, d), np.nan, device=DEV), torch.full((cap, d), np.nan, device=DEV),
               torch.empty(cap, device=DEV), torch.empty(cap, device=DEV),
               torch.zeros(cap, dtype=torch.int64, device=DEV)]
        keep = torch.empty(max(n, 1), dtype=torch.uint8, device=DEV)
        counts = torch.zeros(3, dtype=torch.int32, device=DEV)
        inc = torch.tensor([inc_val], dtype=torch.float64, device=DEV)
        B.bab_prune_branch(self.ctx, d, T(lo), T(hi), T(lb), T(ub), ids_t(ids), n, inc, n_pick, eta, cap, *out,
                           keep, counts)
        torch.cuda.synchronize()
        nc, nr, tot = (int(x) for x in counts.cpu().numpy())
        assert tot == nc + nr
        m = nc + nr
        return {"keep": keep.cpu().numpy()[:n], "n_children": nc, "n_rest": nr, "lo": out[0].cpu().numpy()[:m],
                "hi": out[1].cpu().numpy()[:m], "lb": out[2].cpu().numpy()[:m], "ub": out[3].cpu().numpy()[:m],
                "id": out[4].cpu().numpy()[:m].astype(np.uint64)}
