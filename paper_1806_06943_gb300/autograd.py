"""torch.autograd bridge to lb_grad: the observable J of the state after a
number of steps, as a differentiable function of the coupling constants and
relaxation times theta = (G_AB, G1, G2, tau_A, tau_B).

Forward and backward both run in liblb.so (the FP64 or FP32 step and the
hand-written FP64 discrete adjoint); this module only moves theta and the
gradient between torch tensors and the C-ABI."""
from __future__ import annotations

import numpy as np
import torch

from . import lb

THETA = ("G_AB", "G1", "G2", "tau_A", "tau_B")


class LBObservable(torch.autograd.Function):
    """J = LBObservable.apply(theta, spec) with theta a float64 tensor of 5
    and spec a dict: nx, ny, rho (numpy [2][ny][nx]), nsteps, ckpt_every,
    objective (lb.LB_OBJ_MU_R or lb.LB_OBJ_DP), and optionally g, walls,
    wall_mode, wall_rho, probe (cx, cy, R), precision (lb.LB_FP64, the
    default, or lb.LB_FP32 for an FP32 forward with the FP64 adjoint)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, spec: dict) -> torch.Tensor:
        th = theta.detach().cpu().double().numpy()
        kw = {k: spec[k] for k in ("g", "walls", "wall_mode", "wall_rho") if k in spec}
        lat = lb.Lattice(spec["nx"], spec["ny"], G_AB=th[0], G1=th[1], G2=th[2], tau=(th[3], th[4]),
                         precision=spec.get("precision", lb.LB_FP64), **kw)
        try:
            lat.set_fields(np.ascontiguousarray(spec["rho"], dtype=np.float64))
            if "probe" in spec:
                lat.set_probe(*spec["probe"])
            J, dJ = lat.grad(spec["nsteps"], spec["ckpt_every"], spec.get("objective", lb.LB_OBJ_MU_R))
        finally:
            lat.close()
        ctx.save_for_backward(torch.as_tensor(dJ, dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (dJ,) = ctx.saved_tensors
        return grad_out * dJ, None


def observable(theta: torch.Tensor, spec: dict) -> torch.Tensor:
    return LBObservable.apply(theta, spec)
