"""torch.autograd wrapper of the solve-and-evaluate map (argument marshalling only).

forward:  planar plan from the nodes xi (N x 2; xi' and xi'' fixed), the bordered
          solve A [sigma; a] = [2 g; 0] (Sec. 5) and u at the targets (Eq. u_multi);
backward: [sbar; abar] = C^T ubar, the adjoint solve A^T lam = C^T ubar (transposed
          FMM inside GMRES), dL/dg from lbf_gradient_data and dL/dxi from
          lbf_gradient_nodes.
Every step runs in the CUDA library; this module only moves tensors.
"""
from __future__ import annotations

import torch

from . import lbfmm as L


class SolveEvaluate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, xi, dxi, d2xi, centres, targets, island_ptr, opt):
        plan = L.lbf_plan_create_planar(island_ptr, xi.detach().contiguous(), dxi, d2xi, centres,
                                        opt=opt)
        N, M = plan.N, plan.M
        dev = g.device
        sigma = torch.empty(N, dtype=torch.float64, device=dev)
        a = torch.empty(M, dtype=torch.float64, device=dev)
        rc, _, _ = L.lbf_gmres_solve(plan, g.detach().contiguous(), sigma, a)
        if rc != L.LBF_OK:
            raise L.LbfError(rc, "lbf_gmres_solve")
        T = targets.numel() // 3
        u = torch.empty(T, dtype=torch.float64, device=dev)
        L.lbf_evaluate(plan, sigma, a, targets, u)
        ctx.plan = plan
        ctx.save_for_backward(sigma, a, targets)
        return u

    @staticmethod
    def backward(ctx, ubar):
        plan = ctx.plan
        sigma, a, targets = ctx.saved_tensors
        N, M = plan.N, plan.M
        ub = ubar.detach().contiguous()
        r = torch.empty(N + M, dtype=torch.float64, device=ub.device)
        L.lbf_evaluate_transpose(plan, targets, ub, r[:N], r[N:])
        lam = torch.empty_like(r)
        rc, _, _ = L.lbf_gmres_solve_transpose(plan, r, lam)
        if rc != L.LBF_OK:
            raise L.LbfError(rc, "lbf_gmres_solve_transpose")
        grad_g = None
        if ctx.needs_input_grad[0]:
            grad_g = torch.empty(N, dtype=torch.float64, device=ub.device)
            L.lbf_gradient_data(plan, lam, grad_g)
        grad_xi = None
        if ctx.needs_input_grad[1]:
            grad_xi = torch.empty((N, 2), dtype=torch.float64, device=ub.device)
            L.lbf_gradient_nodes(plan, sigma, a, lam, targets, ub, grad_xi)
        return grad_g, grad_xi, None, None, None, None, None, None


def solve_evaluate(g, xi, dxi, d2xi, centres, targets, island_ptr, opt=None):
    """u at the targets (T) from Dirichlet data g (N) and planar nodes xi (N x 2)."""
    return SolveEvaluate.apply(g, xi, dxi, d2xi, centres, targets, island_ptr, opt)
