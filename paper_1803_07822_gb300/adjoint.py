"""Gradients of a wall force with respect to the wall deformation.

The library's adjoint (cslbm_adjoint_*, cslbm_step_backward) sits behind a
torch.autograd.Function that takes the metric inputs of a lattice (g6, dg18,
J9 as CUDA tensors) to the objective e . F, F the force of the fluid on one
wall after a number of steps from rest; its backward pass walks the steps
back with checkpoints every few steps (the states of a segment are
recomputed from the segment's checkpoint and kept while the segment is
reversed).  The deformation-to-metric map of the channel chart is written in
torch below, so that gradients reach the deformation's Fourier coefficients
by ordinary autograd: that map is the caller's parametrization (the shell),
the LBM steps and their adjoint run in the library's kernels.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _abi
from ._abi import call
from .inputs import LAYOUT, SYM, fourier_modes, grid  # noqa: F401  (fourier_modes: the modes of chart_from_coeffs)


def chart_from_coeffs(coeffs, n, modes, scale, layout=LAYOUT):
    """(g6 [6, N], dg18 [18, N], J9 [9, N]) of the channel chart whose top-wall
    displacement is d = scale * H * sum_m c_m cos(2 pi k_m s / L_s + 2 pi l_m p / L_p + phi_m)
    (periodic span and flow), as differentiable torch functions of coeffs
    (a float64 tensor on the target device).  Same arithmetic as
    inputs.fourier_deformation + inputs.channel_chart."""
    import torch
    dev = coeffs.device
    w, a_p, a_s = layout
    r = [torch.as_tensor(v, dtype=torch.float64, device=dev) for v in grid(n)]
    p, s, xw = r[a_p], r[a_s], r[w]
    H = n[w] - 1
    Ls, Lp = n[a_s], n[a_p]
    k, l, phi = (torch.as_tensor(np.asarray(v, dtype=np.float64), device=dev) for v in modes)
    ks = 2.0 * math.pi * k / Ls
    lp = 2.0 * math.pi * l / Lp
    th = ks[:, None] * s[None, :] + lp[:, None] * p[None, :] + phi[:, None]
    cth, sth = torch.cos(th), torch.sin(th)
    c = coeffs[:, None] * (scale * H)
    d = (c * cth).sum(0)
    ds = -(c * ks[:, None] * sth).sum(0)
    dp = -(c * lp[:, None] * sth).sum(0)
    dss = -(c * (ks * ks)[:, None] * cth).sum(0)
    dpp = -(c * (lp * lp)[:, None] * cth).sum(0)
    dps = -(c * (ks * lp)[:, None] * cth).sum(0)
    N = xw.numel()
    zero, one = torch.zeros(N, dtype=torch.float64, device=dev), torch.ones(N, dtype=torch.float64, device=dev)
    Jrows = [[one if a == i else zero for i in range(3)] for a in range(3)]
    Jrows[w][w] = 1.0 + d / H
    Jrows[w][a_p] = xw * dp / H
    Jrows[w][a_s] = xw * ds / H
    J = torch.stack([torch.stack(row) for row in Jrows])  # [a, i, N]
    Hs = [[[zero for _ in range(3)] for _ in range(3)] for _ in range(3)]

    def put(j, kk, val):
        Hs[w][j][kk] = val
        Hs[w][kk][j] = val

    put(w, a_p, dp / H)
    put(w, a_s, ds / H)
    put(a_p, a_p, xw * dpp / H)
    put(a_p, a_s, xw * dps / H)
    put(a_s, a_s, xw * dss / H)
    # g_ij = sum_a J^a_i J^a_j and d_k g_ij = sum_a (H^a_ki J^a_j + J^a_i H^a_kj), written out as
    # elementwise products (a batched 3 x 3 contraction per node is no GEMM)
    Hess = torch.stack([torch.stack([torch.stack(Hs[a][j]) for j in range(3)]) for a in range(3)])  # [a, j, k, N]
    g6 = torch.stack([(J[:, i] * J[:, j]).sum(0) for i, j in SYM])
    dg18 = torch.stack([(Hess[:, kk, i] * J[:, j] + J[:, i] * Hess[:, kk, j]).sum(0)
                        for kk in range(3) for i, j in SYM])
    return g6, dg18, J.reshape(9, N)


class Adjoint:
    """Adjoint fields of one CurvedLattice (FP32 or FP64 storage, walls at
    rest and periodic faces)."""

    def __init__(self, lat):
        import torch
        self.lat = lat
        nb = ctypes.c_size_t(0)
        call("cslbm_adjoint_workspace_bytes", lat.ctx, ctypes.byref(nb))
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=lat.device)
        call("cslbm_adjoint_attach", lat.ctx, self.workspace.data_ptr(), nb.value)

    def seed_wall_force(self, axis, side, e3):
        e = (ctypes.c_double * 3)(*[float(v) for v in e3])
        call("cslbm_adjoint_seed_wall_force", self.lat.ctx, int(axis), int(side), e)

    def step_backward(self):
        call("cslbm_step_backward", self.lat.ctx)

    def init_backward(self):
        call("cslbm_adjoint_init_backward", self.lat.ctx)

    def metric_grad(self, g6, dg18):
        """(grad g6, grad dg18, grad J9), FP64 CUDA tensors."""
        import torch
        N = self.lat.N
        g6 = g6.detach().to(self.lat.device, torch.float64).contiguous()
        dg18 = dg18.detach().to(self.lat.device, torch.float64).contiguous()
        o6 = torch.empty((6, N), dtype=torch.float64, device=self.lat.device)
        o18 = torch.empty((18, N), dtype=torch.float64, device=self.lat.device)
        o9 = torch.empty((9, N), dtype=torch.float64, device=self.lat.device)
        call("cslbm_adjoint_metric_grad", self.lat.ctx, g6.data_ptr(), dg18.data_ptr(), o6.data_ptr(),
             o18.data_ptr(), o9.data_ptr())
        return o6, o18, o9


def wall_force_objective(lat, g6, dg18, J9, steps, every=20, axis=2, side=1, e3=(0.0, 1.0, 0.0)):
    """e3 . F after `steps` steps from rest (F: force of the fluid on wall
    (axis, side), Cartesian), differentiable in g6, dg18, J9 (CUDA tensors)."""
    return _WallForce.apply(g6, dg18, J9, lat, int(steps), int(every), int(axis), int(side), tuple(e3))


def _make_function():
    import torch

    class WallForce(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g6, dg18, J9, lat, steps, every, axis, side, e3):
            lat.set_metric(g6.detach(), dg18.detach())
            lat.set_jacobian(J9.detach())
            lat.init_equilibrium()
            ckpts = []
            done = 0
            while done < steps:
                k = min(every, steps - done)
                ckpts.append((done, k, lat.save_state()))
                lat.step(k)
                done += k
            final = lat.save_state()
            F = lat.wall_force(axis, side)
            ctx.lat, ctx.ckpts, ctx.final = lat, ckpts, final
            ctx.axis, ctx.side, ctx.e3 = axis, side, e3
            ctx.save_for_backward(g6.detach(), dg18.detach())
            return torch.tensor(float(np.dot(e3, F)), dtype=torch.float64, device=g6.device)

        @staticmethod
        def backward(ctx, gout):
            g6, dg18 = ctx.saved_tensors
            lat = ctx.lat
            adj = getattr(lat, "_adjoint", None)
            if adj is None:
                adj = lat._adjoint = Adjoint(lat)
            else:
                call("cslbm_adjoint_attach", lat.ctx, adj.workspace.data_ptr(), adj.workspace.numel())
            scale = float(gout)
            lat.load_state(ctx.final)
            adj.seed_wall_force(ctx.axis, ctx.side, [scale * v for v in ctx.e3])
            for t0, k, ck in reversed(ctx.ckpts):
                lat.load_state(ck)
                states = []
                for _ in range(k):
                    states.append(lat.save_state())
                    lat.step(1)
                for st in reversed(states):
                    lat.load_state(st)
                    adj.step_backward()
            adj.init_backward()
            o6, o18, o9 = adj.metric_grad(g6, dg18)
            return o6, o18, o9, None, None, None, None, None, None

    return WallForce


class _Lazy:
    fn = None

    @staticmethod
    def apply(*a):
        if _Lazy.fn is None:
            _Lazy.fn = _make_function()
        return _Lazy.fn.apply(*a)


_WallForce = _Lazy
