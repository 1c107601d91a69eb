"""Gradient of a surface-observation misfit through the solver (no counterpart in
the paper; built on its batched solver).

Forward model: K_bc(m) u_k = f_k for K sources (one batched solve, the Green's
functions of Sec. 5), u = sum_k a_k u_k, u_obs = Obs u with Obs the observation
interpolation. For J = J(u_obs) the adjoint state is K_bc lambda = P Obs^T dJ/du_obs
(K is symmetric, so the same solver serves) and
    dJ/dm_e = -lambda^T (dK_bc/dm_e) u   (fe_adjoint_grad, m_e = log E_e)
    dJ/da_k = (P f_k) . lambda           (fe_case_dots).
Every step runs in libfe: the solves, the combination of the Green's functions
(fe_combine_cases), the observation operator and its transpose (fe_obs_apply,
fe_obs_adjoint), the element sensitivities and the source dots. This module
marshals arguments and wires them into torch.autograd; the misfit J itself is the
caller's torch expression of u_obs.
"""
from __future__ import annotations

from . import fe

Observation = fe.Observation


def _solve(mesh: "fe.Mesh", f, opts):
    u, stats, st = mesh.solve(f, **opts)
    return u, stats


def _ensure_moduli(mesh: "fe.Mesh", logE):
    """Make the mesh hold exp(logE) (it may have changed since, e.g. by a second forward)."""
    import torch
    cur = getattr(mesh, "log_young", None)
    if cur is None or cur.shape != logE.shape or not torch.equal(cur, logE):
        mesh.set_log_young(logE.contiguous())


def make_adjoint_solve():
    import torch

    class AdjointSolve(torch.autograd.Function):
        """(logE [E], a [K]) -> u_obs [P, 3], gradients by the adjoint method."""

        @staticmethod
        def forward(ctx, logE, a, mesh, sources, obs, opts):
            logE = logE.detach().contiguous()
            _ensure_moduli(mesh, logE)
            G, _ = _solve(mesh, sources, opts)                  # Green's functions [N, K, 3]
            u = mesh.combine_cases(G, a.detach().contiguous())
            ctx.mesh, ctx.obs, ctx.opts = mesh, obs, opts
            ctx.save_for_backward(u, sources, logE)
            return obs.apply(u)

        @staticmethod
        def backward(ctx, g_obs):
            u, sources, logE = ctx.saved_tensors
            mesh, obs = ctx.mesh, ctx.obs
            _ensure_moduli(mesh, logE)                          # the moduli of the forward pass
            rhs = obs.adjoint(g_obs.contiguous())[:, None, :].contiguous()
            lam, _ = _solve(mesh, rhs, ctx.opts)
            g_logE = mesh.adjoint_grad(u[:, None, :].contiguous(), lam)
            g_a = mesh.case_dots(sources.contiguous(), lam[:, 0, :].contiguous())
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
    _ensure_moduli(mesh, logE.detach().contiguous())
    G, _ = _solve(mesh, sources, opts)
    u = mesh.combine_cases(G, a.contiguous())
    r = obs.apply(u) - d
    return float(0.5 * torch.sum(r * r).item())
