"""PyTorch autograd wrapper: the MBD@rsSCS energy as a differentiable function of
coordinates and free-atom parameters.

forward  = the library's device evaluation (TS scaling, screening, Q, Newton-Schulz,
           energy), inputs and output on the GPU;
backward = the library's hand-written reverse pass (mbd_backward_dev: the MBD pair pass
           on Q^{-1/2}, the chain through the screened parameters, the adjoint
           screening solves and pair pass, the TS chain), scaled on the device by the
           incoming gradient.
No arithmetic of the method runs in PyTorch; PyTorch provides device memory, the
stream and the autograd graph.
"""
from __future__ import annotations

import torch

from . import binding


class MBDEnergyFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, alpha0_ref, c6_ref, rvdw_ref, ratio, calc):
        ins = [t.detach().contiguous() for t in (coords, alpha0_ref, c6_ref, rvdw_ref, ratio)]
        energy = torch.empty(1, dtype=torch.float64, device=coords.device)
        calc.evaluate_dev(*ins, energy)
        ctx.calc = calc
        ctx.evaluation = calc.evaluation_count()
        ctx.save_for_backward(*ins)
        return energy[0]

    @staticmethod
    def backward(ctx, grad_e):
        ins = ctx.saved_tensors
        N = ins[0].shape[0]
        need_r = ctx.needs_input_grad[0]
        need_p = any(ctx.needs_input_grad[1:5])
        gR = torch.empty(N, 3, dtype=torch.float64, device=ins[0].device) if need_r else None
        gp = torch.empty(4, N, dtype=torch.float64, device=ins[0].device) if need_p else None
        ge = grad_e.detach().to(torch.float64).reshape(1).contiguous()
        if ctx.calc.evaluation_count() != ctx.evaluation:
            # another forward on the same context has replaced this one's device state (e.g.
            # E = f(x1) + f(x2)): evaluate these inputs again before differentiating
            ctx.calc.evaluate_dev(*ins, torch.empty(1, dtype=torch.float64, device=ins[0].device))
            ctx.evaluation = ctx.calc.evaluation_count()
        ctx.calc.backward_dev(*ins, grad_energy=ge, grad_coords=gR, grad_params=gp, evaluation=ctx.evaluation)
        out = [gR] + ([gp[k] for k in range(4)] if need_p else [None] * 4)
        return (*out, None)


class MBDEnergy(torch.nn.Module):
    """Holds one library context for systems of a fixed atom count on one device."""

    def __init__(self, n_atoms: int, device: int = 0, **options):
        super().__init__()
        import numpy as np
        self.calc = binding.MBD(device, **options)
        self.calc.set_geometry(np.zeros((n_atoms, 3)) + np.arange(n_atoms)[:, None])
        self.n_atoms = n_atoms

    def forward(self, coords, alpha0_ref, c6_ref, rvdw_ref, ratio):
        if coords.shape[0] != self.n_atoms:
            raise ValueError("atom count differs from the module's")
        return MBDEnergyFunction.apply(coords, alpha0_ref, c6_ref, rvdw_ref, ratio, self.calc)


def mbd_energy(coords, alpha0_ref, c6_ref, rvdw_ref, ratio, calc):
    """Functional form: calc is a binding.MBD whose geometry size matches coords."""
    return MBDEnergyFunction.apply(coords, alpha0_ref, c6_ref, rvdw_ref, ratio, calc)
