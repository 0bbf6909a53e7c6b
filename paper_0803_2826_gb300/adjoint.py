"""torch.autograd wrapper around the library's reverse pass.

``kinetic_energy(force, lattice, nsteps, lo, hi, checkpoint_every)`` returns
L = 1/2 sum_{box} |j|^2 / rho after ``nsteps`` deterministic (kT = 0) steps
from the lattice's current state, as a differentiable function of the force
field.  Forward and reverse passes both run in the CUDA library: the
autograd forward calls ``lb_adjoint_forward`` (the steps, a checkpoint every
``checkpoint_every`` steps, L and its seed), and only a backward call runs
``lb_adjoint_backward`` (the hand-written adjoint with recomputation inside
each segment); this module only moves the field into the handle's force
buffer and hands the gradient to autograd.
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
        loss = torch.zeros(1, dtype=torch.float64, device=lattice.force.device)
        L.lb_adjoint_forward(lattice.h, nsteps, checkpoint_every, lo, hi, loss)
        ctx.lattice = lattice
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        lattice = ctx.lattice
        grad = torch.empty_like(lattice.force)
        L.lb_adjoint_backward(lattice.h, grad)
        return grad * grad_out.to(grad.dtype), None, None, None, None, None


def kinetic_energy(force, lattice, nsteps, lo, hi, checkpoint_every=50):
    return KineticEnergy.apply(force, lattice, nsteps, tuple(lo), tuple(hi), checkpoint_every)


class CoupledKineticEnergy(torch.autograd.Function):
    """The same loss after ``nsteps`` coupled steps (free particles at kT = 0:
    ``lb_couple_particles`` then ``lb_step``), differentiable in the force
    field and the particles' initial positions and momenta
    (``lb_adjoint_kinetic_coupled``).  The particle tensors are advanced in
    place by the forward pass, as the coupled steps do."""

    @staticmethod
    def forward(ctx, force, pos, mom, lattice, cp, mass0, gamma0, nsteps, lo, hi, checkpoint_every):
        if lattice.force is None:
            raise ValueError("the lattice needs a force field buffer (Lattice(..., force=tensor))")
        lattice.force.copy_(force.detach())
        n = pos.shape[0]
        parts = L.particles(n, pos.detach(), mom.detach(), mass0=mass0, gamma0=gamma0)
        grad = torch.empty_like(lattice.force)
        gpos = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        gmom = torch.empty_like(gpos)
        loss = torch.zeros(1, dtype=torch.float64, device=lattice.force.device)
        L.lb_adjoint_kinetic_coupled(lattice.h, parts, cp, nsteps, checkpoint_every, lo, hi, grad, gpos, gmom, loss)
        ctx.save_for_backward(grad, gpos, gmom)
        ctx.dtypes = (pos.dtype, mom.dtype)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        grad, gpos, gmom = ctx.saved_tensors
        s = grad_out.to(grad.dtype)
        return (grad * s, (gpos * s).to(ctx.dtypes[0]), (gmom * s).to(ctx.dtypes[1]),
                None, None, None, None, None, None, None, None)


def coupled_kinetic_energy(force, pos, mom, lattice, cp, nsteps, lo, hi, *, mass0=1.0, gamma0=1.0,
                           checkpoint_every=50):
    """pos: device FP64 [n][3], mom: device FP32 [n][3] (advanced in place)."""
    return CoupledKineticEnergy.apply(force, pos, mom, lattice, cp, mass0, gamma0, nsteps, tuple(lo), tuple(hi),
                                      checkpoint_every)
