"""Differentiable region-of-interest dose.

RoiDose.apply(weights [S], spectrum [G], density [V]) -> J = sum_v roi(v) D(v)
with D the dose tally of the forward solve.  Every step runs in libdoctors:
doctors_solve + doctors_roi_dose forward (J summed in FP64 on the device), and
doctors_roi_gradients backward (the adjoint response, adjoint sweeps, ray
back-projection and the dose's own density factor, all on the device).  This
module only moves the inputs into the problem and scales the returned
gradients by the incoming gradient of J.
"""
from __future__ import annotations

import numpy as np
import torch


class DoseProblem:
    """Holds a DoctorsProblem, the base sources and the dose tables."""

    def __init__(self, prob, roi, k=None, tol=1e-6, max_iters=500):
        from .solver import DoctorsProblem
        self.prob = prob
        self.solver = DoctorsProblem(prob, tol=tol, max_iters=max_iters)
        self.k = np.ascontiguousarray(prob.k_dep if k is None else k, np.float64)
        self.mat = torch.as_tensor(prob.mat.astype(np.uint8), device="cuda")
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
        self.solver.set_materials(self.mat, rho, self.prob.sigma_t, self.prob.sigma_s)


class RoiDose(torch.autograd.Function):
    @staticmethod
    def forward(ctx, weights, spectrum, density, dp: DoseProblem):
        dp.set_inputs(weights, spectrum, density)
        dp.solver.solve()
        J = dp.solver.roi_dose(dp.k, dp.roi)
        ctx.dp = dp
        ctx.meta = (weights.device, spectrum.device, density.dtype)
        return torch.tensor(J, dtype=torch.float64, device=weights.device)

    @staticmethod
    def backward(ctx, gJ):
        dp = ctx.dp
        dev_w, dev_s, dtype_rho = ctx.meta
        g = dp.solver.roi_gradients(dp.k, dp.roi)
        gJ = gJ.to(torch.float64)
        return (gJ * g["weights"]).to(dev_w), (gJ * g["spectrum"]).to(dev_s), \
            (gJ * g["density"]).to(dtype_rho), None
