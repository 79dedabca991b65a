"""torch.autograd.Function over the library: receiver fields as a differentiable function of the
particle centres, radii and the frequency (inverse scattering, Sec. 7.5).

Forward: ms_setup at the given parameters, ms_solve for the incidences, ms_fields at the receivers.
Backward: ms_grad with w = grad_output.  For a complex output u, PyTorch hands backward the tensor g
with dL = Re sum conj(g) du for a real loss L, which is exactly the w of ms_grad.
"""
from __future__ import annotations

import numpy as np
import torch

from . import MS_PREC_FP64, Solver


class ScatteredFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, centres: torch.Tensor, radii: torch.Tensor, omega: torch.Tensor, spec: dict):
        s = Solver(centres.detach().cpu().numpy(), radii.detach().cpu().numpy(), spec["bc"], spec["media"],
                   float(omega.detach().cpu()), spec["p"], **spec.get("options", {}))
        gamma, info = s.solve(spec["kinds"], spec["angles"], tol=spec.get("tol", 1e-12),
                              prec=spec.get("prec", MS_PREC_FP64))
        u = s.fields(gamma, spec["receivers"])
        ctx.solver, ctx.gamma, ctx.spec = s, gamma, spec
        ctx.devices = (centres.device, radii.device, omega.device)
        return u

    @staticmethod
    def backward(ctx, gu: torch.Tensor):
        spec = ctx.spec
        gc, gr, go, info = ctx.solver.grad(spec["kinds"], spec["angles"], ctx.gamma, gu.contiguous(),
                                           spec["receivers"], tol=spec.get("grad_tol", 1e-10),
                                           prec=spec.get("prec", MS_PREC_FP64), want_omega=True)
        dc, dr, dw = ctx.devices
        return gc.to(dc), gr.to(dr), torch.tensor(go, dtype=torch.float64, device=dw), None


def scattered_fields(centres, radii, omega, bc, media, p, kinds, angles, receivers, **kw):
    """u (nrhs, R, 2) complex128 on the GPU; differentiable in centres (M,2), radii (M,), omega ()."""
    spec = {"bc": np.asarray(bc, dtype=np.int32), "media": media, "p": int(p), "kinds": np.asarray(kinds),
            "angles": np.asarray(angles, dtype=np.float64), "receivers": np.asarray(receivers, dtype=np.float64)}
    spec.update(kw)
    return ScatteredFields.apply(centres, radii, omega, spec)
