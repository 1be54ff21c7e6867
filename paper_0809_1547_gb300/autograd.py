"""torch.autograd binding of the adjoint gradient (``mb_adjoint_energy_zface``).

``emitted_energy(eps_r, pump, realization)`` returns the energy (J) that
crosses a z plane in +z during ``realization.n_steps`` steps started from the
initial state (fields zero, N0 = N_a), as a differentiable function of the
per-cell permittivity map and the pump rate.  The forward call runs the
library's forward sweep and its reverse-time adjoint in one C call (both on
the GPU); backward only scales the saved gradients.  Argument marshalling
only: every step runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .binding import MBSimulation, mb_params


@dataclass
class Realization:
    """Everything but eps_r and W_p that defines the run."""
    grid: tuple
    dx: float
    dt: float
    gain_mask: np.ndarray
    N_a: float
    seed: int
    n_steps: int
    ckpt_every: int = 200
    z_plane: int = -1
    params: mb_params | None = None
    sources: list = field(default_factory=list)   # (ijk, comp, lam, t0, tau, amp)


class EmittedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r: torch.Tensor, pump: torch.Tensor, r: Realization):
        sim = MBSimulation(r.grid, r.dx, r.dt, r.params)
        try:
            eps_h = eps_r.detach().to("cpu", torch.float32).numpy()
            sim.set_material(eps_h, r.gain_mask, r.N_a, float(pump))
            sim.set_seed(r.seed)
            for s in r.sources:
                sim.set_source(*s)
            J, g, gp = sim.adjoint_energy_zface(r.n_steps, r.ckpt_every, r.z_plane)
        finally:
            sim.close()
        ctx.save_for_backward(g.to(eps_r.device, eps_r.dtype).reshape(eps_r.shape),
                              torch.tensor(gp, dtype=torch.float64))
        ctx.pump_dtype = pump.dtype
        ctx.pump_device = pump.device
        return torch.tensor(J, dtype=torch.float64, device=eps_r.device)

    @staticmethod
    def backward(ctx, gJ):
        g, gp = ctx.saved_tensors
        g_eps = (gJ.to(g.dtype) * g) if ctx.needs_input_grad[0] else None
        g_pump = (gJ.double().cpu() * gp).to(ctx.pump_device, ctx.pump_dtype) \
            if ctx.needs_input_grad[1] else None
        return g_eps, g_pump, None


def emitted_energy(eps_r: torch.Tensor, pump: torch.Tensor, realization: Realization) -> torch.Tensor:
    """Differentiable energy through the z plane (float64 scalar tensor)."""
    return EmittedEnergy.apply(eps_r, pump, realization)
