"""torch.autograd.Function around the discrete adjoint of the C ABI.

``final_state_objective(theta, layout, n_steps, ...)`` returns
J = w_solid mean h(psi_T) + w_centroid y_c(T)/L_y as a 0-d tensor that is
differentiable with respect to theta = (eps_s, Omega, sigma).  The forward
runs pf_adjoint_step (forward sweep with checkpoints every K steps, reverse
sweep with recomputation in between) and keeps dJ/dtheta for backward.
Marshalling only: every step runs in the CUDA kernels of libpf.so.
"""
from __future__ import annotations

import torch

from . import pf

PARAMS = ("eps_s", "Omega", "sigma")


class FinalStateObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, layout, n_steps, w_solid, w_centroid, checkpoint_every,
                precision):
        th = theta.detach().double().cpu().tolist()
        params = dict(layout.params, **dict(zip(PARAMS, th)))
        sim = pf.Simulation([(layout.nx, layout.ny)], params, precision)
        try:
            sim.init_fields(0, layout.seeds, layout.R_s, layout.bubbles)
            J, g = sim.adjoint_step(int(n_steps), w_solid, w_centroid, int(checkpoint_every))
        finally:
            sim.close()
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None


def final_state_objective(theta: torch.Tensor, layout, n_steps: int, w_solid: float = 1.0,
                          w_centroid: float = 1.0, checkpoint_every: int = 100,
                          precision: str = "fp32") -> torch.Tensor:
    return FinalStateObjective.apply(theta, layout, n_steps, w_solid, w_centroid,
                                     checkpoint_every, precision)
