"""Differentiable solve: p = pressure part of A(theta, lambda, mu)^{-1} b as a
``torch.autograd.Function`` whose backward pass is one adjoint solve with the same
multigrid-preconditioned FGMRES (A is symmetric) and the library's gradient kernel
(``bmg_adjoint_gradient``).  theta is the per-triangle log-permeability (float32,
shape (2, n, n): lower-left then upper-right triangles, indexed [j, i]).

All arithmetic runs in the library; this module only moves tensors between the (2, n, n)
parameter shape and the library's padded layout.
"""
from __future__ import annotations

import torch

from . import (assemble_logk, setup_hierarchy, pitch, vector_len)


class PressureSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, lam, mu, b, cfg: dict):
        n = theta.shape[-1]
        P = pitch(n)
        dev = theta.device
        th = torch.zeros(2, n + 1, P, dtype=torch.float32, device=dev)
        th[:, :n, :n] = theta.detach().to(torch.float32)
        s = assemble_logk(n, float(lam), float(mu), th.reshape(-1), cfg.get("tau", 1.0),
                          cfg.get("alpha", 1.0), cfg.get("inv_M", 1.0))
        h = setup_hierarchy(s, cfg.get("smoother", "vanka"), cfg.get("nu1", 1), cfg.get("nu2", 1),
                            omega=cfg.get("omega", 0.7), omega_J=cfg.get("omega_J", 1.0),
                            n_coarse=cfg.get("n_coarse", 8), precision=cfg.get("precision", "fp64"))
        x = torch.zeros(vector_len(n), dtype=torch.float64, device=dev)
        info = h.fgmres_solve(b.detach(), x, rtol=cfg.get("rtol", 1e-10), restart=cfg.get("restart", 50),
                              maxit=cfg.get("maxit", 2000))
        if info["status"] != "converged":
            raise RuntimeError(f"forward solve did not converge: {info}")
        ctx.state = (s, h, x, n, P, cfg, theta.dtype, lam, mu)
        ctx.forward_info = info
        return x.view(10, n + 1, P)[8:10, :n, :n].clone()

    @staticmethod
    def backward(ctx, gp):
        s, h, x, n, P, cfg, tdt, lam, mu = ctx.state
        dev = x.device
        g = torch.zeros(10, n + 1, P, dtype=torch.float64, device=dev)
        g[8:10, :n, :n] = gp.to(torch.float64)
        g = g.reshape(-1)
        xi = torch.zeros_like(x)
        info = h.fgmres_solve(g, xi, rtol=cfg.get("rtol", 1e-10), restart=cfg.get("restart", 50),
                              maxit=cfg.get("maxit", 2000))
        if info["status"] != "converged":
            raise RuntimeError(f"adjoint solve did not converge: {info}")
        dth = torch.empty(2 * (n + 1) * P, dtype=torch.float64, device=dev)
        dl = torch.empty(2, dtype=torch.float64, device=dev)
        s.adjoint_gradient(x, xi, dth, dl)
        dtheta = dth.view(2, n + 1, P)[:, :n, :n].to(tdt)
        glam = dl[0].to(lam.dtype) if torch.is_tensor(lam) else None
        gmu = dl[1].to(mu.dtype) if torch.is_tensor(mu) else None
        return dtheta, glam, gmu, xi, None


def pressure_solve(theta, lam, mu, b, **cfg):
    """p (2, n, n) float64 from theta (2, n, n), scalar tensors lam, mu and the right-hand
    side b (float64 CUDA vector in the library layout); differentiable in theta, lam, mu, b."""
    return PressureSolve.apply(theta, lam, mu, b, cfg)
