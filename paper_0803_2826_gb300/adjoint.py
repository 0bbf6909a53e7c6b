"""torch.autograd wrapper around the library's reverse pass.

``kinetic_energy(force, lattice, nsteps, lo, hi, checkpoint_every)`` returns
L = 1/2 sum_{box} |j|^2 / rho after ``nsteps`` deterministic (kT = 0) steps
from the lattice's current state, as a differentiable function of the force
field.  Forward and reverse passes both run in the CUDA library
(``lb_adjoint_kinetic``: forward steps with a checkpoint every
``checkpoint_every`` steps, then the hand-written adjoint with recomputation
inside each segment); this module only moves the field into the handle's
force buffer and hands the gradient to autograd.
"""
from __future__ import annotations

import torch

from . import lbfluct as L


class KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, force, lattice, nsteps, lo, hi, checkpoint_every):
        if lattice.force is None:
            raise ValueError("the lattice needs a force field buffer (Lattice(..., force=tensor))")
        lattice.force.copy_(force.detach())
        grad = torch.empty_like(lattice.force)
        loss = torch.zeros(1, dtype=torch.float64, device=lattice.force.device)
        L.lb_adjoint_kinetic(lattice.h, nsteps, checkpoint_every, lo, hi, grad, loss)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad * grad_out.to(grad.dtype), None, None, None, None, None


def kinetic_energy(force, lattice, nsteps, lo, hi, checkpoint_every=50):
    return KineticEnergy.apply(force, lattice, nsteps, tuple(lo), tuple(hi), checkpoint_every)
