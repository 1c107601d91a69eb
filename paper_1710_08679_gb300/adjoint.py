"""Gradient of a surface-observation misfit through the solver (no counterpart in
the paper; built on its batched solver).

Forward model: K_bc(m) u_k = f_k for K sources (one batched solve, the Green's
functions of Sec. 5), u = sum_k a_k u_k, u_obs = P u with P the observation
interpolation. For J = J(u_obs) the adjoint state is K_bc lambda = P^T dJ/du_obs
(K is symmetric, so the same solver serves) and
    dJ/dm_e = -lambda^T (dK_bc/dm_e) u   (fe_adjoint_grad, m_e = log E_e)
    dJ/da_k = lambda . f_k.
The solves, the element sensitivity kernel and every product run in libfe; torch
ops here only combine the K Green's functions, apply the sparse observation
operator and take dot products of vectors.
"""
from __future__ import annotations

import numpy as np

from . import fe


class Observation:
    """Sparse observation operator on the device: u_obs[p, c] = sum_j w[p, j] u[node[p, j], c]."""

    def __init__(self, node: np.ndarray, weight: np.ndarray, device="cuda"):
        import torch
        self.node = torch.from_numpy(np.ascontiguousarray(node, dtype=np.int64)).to(device)
        self.weight = torch.from_numpy(np.ascontiguousarray(weight, dtype=np.float64)).to(device)

    def apply(self, u):
        """u [N, 3] -> [P, 3]."""
        return (self.weight[:, :, None] * u[self.node]).sum(dim=1)

    def adjoint(self, g, n_nodes: int):
        """g [P, 3] -> P^T g as [N, 3]."""
        import torch
        out = torch.zeros((n_nodes, 3), dtype=g.dtype, device=g.device)
        out.index_add_(0, self.node.reshape(-1), (self.weight[:, :, None] * g[:, None, :]).reshape(-1, 3))
        return out


def _solve(mesh: "fe.Mesh", f, opts):
    u, stats, st = mesh.solve(f, **opts)
    return u, stats


def make_adjoint_solve():
    import torch

    class AdjointSolve(torch.autograd.Function):
        """(logE [E], a [K]) -> u_obs [P, 3], gradients by the adjoint method."""

        @staticmethod
        def forward(ctx, logE, a, mesh, sources, obs, opts):
            mesh.set_log_young(logE.detach().contiguous())
            G, _ = _solve(mesh, sources, opts)                  # Green's functions [N, K, 3]
            u = torch.einsum("nkc,k->nc", G, a.detach())
            ctx.mesh, ctx.obs, ctx.opts = mesh, obs, opts
            ctx.save_for_backward(u, sources)
            return obs.apply(u)

        @staticmethod
        def backward(ctx, g_obs):
            u, sources = ctx.saved_tensors
            mesh, obs = ctx.mesh, ctx.obs
            rhs = (obs.adjoint(g_obs.contiguous(), mesh.n_nodes) * mesh.free)[:, None, :].contiguous()
            lam, _ = _solve(mesh, rhs, ctx.opts)
            g_logE = mesh.adjoint_grad(u[:, None, :].contiguous(), lam)
            g_a = torch.einsum("nkc,nc->k", sources * mesh.free[:, None, :], lam[:, 0, :])
            return g_logE, g_a, None, None, None, None

    return AdjointSolve


def misfit_and_grad(mesh, logE, a, sources, obs, d, opts):
    """J = 1/2 |u_obs - d|^2 and its gradient (dJ/dlogE, dJ/da) via autograd."""
    import torch
    AdjointSolve = make_adjoint_solve()
    logE = logE.detach().clone().requires_grad_(True)
    a = a.detach().clone().requires_grad_(True)
    u_obs = AdjointSolve.apply(logE, a, mesh, sources, obs, opts)
    J = 0.5 * torch.sum((u_obs - d) ** 2)
    J.backward()
    return float(J.item()), logE.grad.detach(), a.grad.detach()


def misfit(mesh, logE, a, sources, obs, d, opts) -> float:
    import torch
    mesh.set_log_young(logE.contiguous())
    G, _ = _solve(mesh, sources, opts)
    u = torch.einsum("nkc,k->nc", G, a)
    r = obs.apply(u) - d
    return float(0.5 * torch.sum(r * r).item())
