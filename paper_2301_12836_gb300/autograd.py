"""Differentiable receiver data of the LS forward model (torch.autograd.Function).

d[f, r, :] = u_f(x_r), u_f solving A_f u_f = u0_f(M) (Sec. 2-3) at each angular frequency w_f,
for a moment tensor M at a fixed source position and receivers on grid nodes.  The backward
pass is the discrete adjoint: lambda_f = A_f^{-H} R^T g_f (lsm_solve_adjoint), then the
contrast gradients (lsm_gradient, accumulated over frequencies) and the moment-tensor gradient
Re<lambda_f, du0/dM> (lsm_source_gradient).  All arithmetic runs in the library's kernels; this
module only marshals tensors (receiver gather and scatter are index operations).

For a real loss L, torch hands backward g = dL/dRe(d) + i dL/dIm(d), and
dL = Re<g, dd> = Re<lambda, du0 + K(Dv dC eps(u) + w^2 drho u)>.
"""
from __future__ import annotations

import torch

from . import lsm


class ReceiverModel:
    """Forward model at fixed grid, background, frequencies, source position and receivers.

    n: (nx, ny, nz); dx [m]; lam0, mu0, rho0: background; freqs_hz: frequencies; xs: source
    position [m]; receivers: integer tensor/array (k, 3) of node indices (ix, iy, iz).
    dC0, drho0: an initial contrast (device float64) used to create the handles.
    checkpoint: keep no wavefield between forward and backward; the backward pass solves the
    forward systems again (twice the forward solves, nf * 3N complex values less memory).
    """

    def __init__(self, n, dx, lam0, mu0, rho0, dC0, drho0, freqs_hz, xs, receivers, precision=lsm.LSM_FP64,
                 tol=1e-10, maxit=2000, checkpoint=False, max_outer=8):
        import numpy as np
        self.n = tuple(int(v) for v in n)
        nx, ny, nz = self.n
        self.N = nx * ny * nz
        self.xs = [float(v) for v in xs]
        opts = lsm.lsm_default_opts(precision=precision, tol=tol, maxit=maxit, max_outer=max_outer)
        ws = [2.0 * np.pi * float(f) for f in freqs_hz]
        self.base = lsm.lsm_create(self.n, dx, lam0, mu0, rho0, dC0, drho0, ws[0], opts)
        self.handles = [self.base] + [lsm.lsm_create_shared(self.base, w) for w in ws[1:]]
        rec = torch.as_tensor(np.asarray(receivers), dtype=torch.long)
        self.ridx = (rec[:, 2] * ny * nx + rec[:, 1] * nx + rec[:, 0]).to(dC0.device)
        self.device = dC0.device
        self.checkpoint = bool(checkpoint)
        self.last_iters = []

    def __call__(self, dC, drho, M):
        return _LSReceivers.apply(dC, drho, M, self)


def _forward_field(model, h, Mv):
    """u solving A u = u0(M) at the handle's frequency (from a zero initial guess)."""
    b = torch.empty(3 * model.N, dtype=torch.complex128, device=model.device)
    lsm.lsm_source(h, Mv, model.xs, b)
    x = torch.zeros_like(b)
    _, model._it, _ = lsm.lsm_solve(h, b, x)
    return x


class _LSReceivers(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dC, drho, M, model):
        dC = dC.detach().contiguous()
        drho = drho.detach().contiguous()
        lsm.lsm_set_contrast(model.base, dC, drho)
        Mv = [float(v) for v in M.detach().cpu().tolist()]
        N = model.N
        nf, nr = len(model.handles), model.ridx.numel()
        out = torch.empty((nf, nr, 3), dtype=torch.complex128, device=model.device)
        us = []
        model.last_iters = []
        for f, h in enumerate(model.handles):
            x = _forward_field(model, h, Mv)
            model.last_iters.append(model._it)
            if not model.checkpoint:
                us.append(x)
            out[f] = x.view(3, N)[:, model.ridx].transpose(0, 1)
        ctx.model = model
        ctx.us = us
        ctx.Mv = Mv
        ctx.save_for_backward(dC, drho)
        return out

    @staticmethod
    def backward(ctx, g):
        model = ctx.model
        dC, drho = ctx.saved_tensors
        lsm.lsm_set_contrast(model.base, dC, drho)   # the handles may have seen another contrast since
        N = model.N
        gC = torch.zeros(21 * N, dtype=torch.float64, device=model.device)
        grho = torch.zeros(N, dtype=torch.float64, device=model.device)
        gM = torch.zeros(6, dtype=torch.float64)
        g = g.to(torch.complex128)
        for f, h in enumerate(model.handles):
            rhs = torch.zeros(3 * N, dtype=torch.complex128, device=model.device)
            rhs.view(3, N)[:, model.ridx] = g[f].transpose(0, 1)
            lam = torch.zeros_like(rhs)
            lsm.lsm_solve_adjoint(h, rhs, lam)
            u = _forward_field(model, h, ctx.Mv) if model.checkpoint else ctx.us[f]
            lsm.lsm_gradient(h, u, lam, gC, grho, accumulate=True)
            gM += torch.tensor(lsm.lsm_source_gradient(h, model.xs, lam), dtype=torch.float64)
        return gC.view_as(dC), grho.view_as(drho), gM.to(dtype=torch.float64), None
