"""Differentiable region-of-interest dose.

RoiDose.apply(weights [S], spectrum [G], density [V]) -> J = sum_v roi(v) D(v)
with D the dose tally of the forward solve.  The forward pass and the
gradients run in libdoctors: doctors_solve + doctors_dose forward, and
doctors_adjoint_solve (adjoint sweeps, ray back-projection) backward.  The
only torch arithmetic is the explicit density factor of the dose itself,
d D(v)/d rho(v) at fixed fluence = sum_g k[mat v][g] phi[g](v), and the
response r[g][v] = roi(v) k[mat v][g] rho(v) handed to the adjoint.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as C


class DoseProblem:
    """Holds a DoctorsProblem, the base sources and the dose tables."""

    def __init__(self, prob, roi, k=None, tol=1e-6, max_iters=500):
        from .solver import DoctorsProblem
        self.prob = prob
        self.solver = DoctorsProblem(prob, tol=tol, max_iters=max_iters)
        self.k = np.ascontiguousarray(prob.k_dep if k is None else k, np.float64)
        self.mat = torch.as_tensor(prob.mat.astype(np.int64), device="cuda")
        self.k_t = torch.as_tensor(self.k, device="cuda")                     # [nmat][G]
        self.roi = torch.as_tensor(np.asarray(roi, np.float64), device="cuda")  # [V]

    def set_inputs(self, weights, spectrum, density):
        srcs = []
        w = weights.detach().double().cpu().numpy()
        chi = spectrum.detach().double().cpu().numpy()
        for s, ws in zip(self.prob.sources, w):
            q = type(s)(**{**s.__dict__})
            q.weight = float(ws)
            q.spectrum = chi.copy()
            srcs.append(q)
        self.solver.set_sources(srcs)
        rho = density.detach().float().contiguous()
        self.solver.set_materials(self.mat.to(torch.uint8), rho, self.prob.sigma_t, self.prob.sigma_s)


class RoiDose(torch.autograd.Function):
    @staticmethod
    def forward(ctx, weights, spectrum, density, dp: DoseProblem):
        dp.set_inputs(weights, spectrum, density)
        dp.solver.solve()
        dose = dp.solver.dose(dp.k)
        ctx.dp = dp
        ctx.devices = (weights.device, spectrum.device)
        ctx.save_for_backward(density)
        return (dp.roi * dose).sum().to(weights.device)

    @staticmethod
    def backward(ctx, gJ):
        dp = ctx.dp
        (density,) = ctx.saved_tensors
        kv = dp.k_t[dp.mat].T                                      # [G][V]
        rho = density.detach().double()
        response = (kv * (dp.roi * rho)[None, :]).contiguous()
        g = dp.solver.adjoint(response)
        phi = dp.solver.fluence(C.DOCTORS_FLUENCE_TOTAL).double()
        explicit = dp.roi * (kv * phi).sum(dim=0)
        d_rho = g["density"] + explicit
        gJ = gJ.to(torch.float64)
        return (gJ * g["weights"]).to(ctx.devices[0]), (gJ * g["spectrum"]).to(ctx.devices[1]), \
            (gJ * d_rho).to(density.dtype), None
