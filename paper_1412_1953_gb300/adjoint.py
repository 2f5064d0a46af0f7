"""Differentiation form: gradients of the amplitude J = <g|u> by one adjoint MG-CCCS solve.

u solves the Temkin-Poet problem (H - E)u = f with V1 + V2 = -Z/x - Z/y, V12 = 1/max(x,y)
plus a real per-node perturbation dV, f held fixed.  J = sum_k w_k g_k u_k (bilinear,
ECS quadrature weights).  W(H - E) is complex symmetric (Sec. 2.5), so the adjoint
problem is the forward problem with right-hand side g, solved by the same MG-CCCS
(GMRES) solver; the forward solution is kept (checkpointed) for the backward pass
instead of any per-cycle state.  Every numerical step runs in the CUDA library; this
module only orders the calls and applies the chain rule to the real and imaginary parts.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import inputs
from . import mgcccs as M


def _solve(solver, rhs, rtol, max_iter):
    x = torch.zeros_like(rhs)
    its, rr = solver.solve(x, rhs, rtol=rtol, max_iter=max_iter)
    return x, its, rr


def setup_tp(E, Z, dV, geom, solver_kw):
    """Solver for the TP problem at (E, Z, dV); geom = dict(n, L, R0, theta)."""
    n, L, R0, th = geom["n"], geom["L"], geom["R0"], geom["theta"]
    _, z = inputs.node_coordinates(n, L, R0, th)
    zi = z[1:-1]
    v1 = (-float(Z) / zi).astype(np.complex128)
    base = inputs.temkin_poet(n, L=L, R0=R0, theta=th, E=float(E), Z=float(Z), noise_amplitude=0.0)
    v12 = torch.as_tensor(base.v12).to("cuda")
    if dV is not None:
        v12 = v12 + dV.detach().to(torch.complex128).reshape(v12.shape)
    p = M.make_params(n, n, L, L, R0, R0, th, float(E), **solver_kw)
    return M.Solver(p, v1, v1.copy(), v12.contiguous())


def amplitude_and_gradients(E, Z, dV, f, g, geom, solver_kw, rtol=1e-12, max_iter=2000):
    """J and the holomorphic derivatives dJ/dE, dJ/dZ (complex scalars) and dJ/d(dV_k)
    (complex array), from one forward and one adjoint solve."""
    solver = setup_tp(E, Z, dV, geom, solver_kw)
    u, its_f, _ = _solve(solver, f, rtol, max_iter)
    mu, its_a, _ = _solve(solver, g, rtol, max_iter)
    out = torch.zeros(4, dtype=torch.complex128, device="cuda")
    dAdZ = torch.as_tensor(inputs.tp_charge_derivative(geom["n"], geom["L"], geom["R0"], geom["theta"])).to("cuda")
    solver.weighted_dot(g, u, out[0:1])
    solver.weighted_dot(mu, u, out[1:2])                   # dJ/dE  (d(H-E)/dE = -I)
    solver.weighted_dot(mu, u, out[2:3], d=dAdZ, scale=-1.0)  # dJ/dZ
    ddV = torch.empty_like(u)
    solver.weighted_product(mu, u, ddV, scale=-1.0)          # dJ/d(dV_k)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return {"J": o[0], "dE": o[1], "dZ": o[2], "ddV": ddV, "u": u, "mu": mu, "its": (its_f, its_a)}


class TPAmplitude(torch.autograd.Function):
    """(Re J, Im J) as a differentiable function of (E, Z, dV) with real E, Z and real
    per-node dV; backward runs one adjoint MG-CCCS solve with the checkpointed u."""

    @staticmethod
    def forward(ctx, E, Z, dV, f, g, geom, solver_kw, rtol=1e-12, max_iter=1000):
        solver = setup_tp(E.item(), Z.item(), dV, geom, solver_kw)
        u, _, _ = _solve(solver, f, rtol, max_iter)
        J = torch.zeros(1, dtype=torch.complex128, device="cuda")
        solver.weighted_dot(g, u, J)
        ctx.save_for_backward(u)
        ctx.solver, ctx.g, ctx.geom, ctx.rtol, ctx.max_iter = solver, g, geom, rtol, max_iter
        ctx.dV_shape = dV.shape
        return J.real[0].clone(), J.imag[0].clone()

    @staticmethod
    def backward(ctx, g_re, g_im):
        (u,) = ctx.saved_tensors
        solver, geom = ctx.solver, ctx.geom
        mu, _, _ = _solve(solver, ctx.g, ctx.rtol, ctx.max_iter)
        out = torch.zeros(2, dtype=torch.complex128, device="cuda")
        dAdZ = torch.as_tensor(inputs.tp_charge_derivative(geom["n"], geom["L"], geom["R0"], geom["theta"])).to("cuda")
        solver.weighted_dot(mu, u, out[0:1])
        solver.weighted_dot(mu, u, out[1:2], d=dAdZ, scale=-1.0)
        ddV = torch.empty_like(u)
        solver.weighted_product(mu, u, ddV, scale=-1.0)
        gE = g_re * out[0].real + g_im * out[0].imag
        gZ = g_re * out[1].real + g_im * out[1].imag
        gdV = (g_re * ddV.real + g_im * ddV.imag).reshape(ctx.dV_shape)
        return gE, gZ, gdV, None, None, None, None, None, None
