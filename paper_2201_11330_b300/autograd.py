"""torch.autograd bridge for the hand-written adjoint of the LBM step.

``kinetic_energy(lattice, force, lid, T, K)`` returns the final-time kinetic
energy J = rho0/2 sum_x |u(x, T)|^2 of a run started from equilibrium, as a
differentiable function of the body-force field (d, N) and the moving-wall
velocity (3,).  The forward runs T fused steps with checkpoints every K
steps (lbm_adjoint_forward); the backward recomputes between checkpoints and
runs the reverse collide-stream kernels (lbm_adjoint_backward).  Both are
CUDA work in liblbm.so; this module only routes tensors.
"""
from __future__ import annotations

import torch


class LBMKineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, force, lid, lattice, T, K, p0=None, u0=None):
        lattice.set_force(force.detach().to(torch.float32).contiguous())
        lattice.set_lid([float(v) for v in lid.detach().cpu().tolist()])
        lattice.init(p0, u0)  # the stored state includes the first collision, with this force
        J = lattice.adjoint_forward(int(T), int(K))
        ctx.lattice = lattice
        ctx.force_meta = (force.dtype, force.device, force.shape)
        ctx.lid_meta = (lid.dtype, lid.device)
        return torch.tensor(J, dtype=torch.float64, device=force.device)

    @staticmethod
    def backward(ctx, grad_J):
        gF, gU = ctx.lattice.adjoint_backward()
        dt, dev, shape = ctx.force_meta
        gF = (gF * grad_J.to(gF.device)).to(dt).reshape(shape).to(dev)
        ldt, ldev = ctx.lid_meta
        gU = (gU.to(grad_J.device) * grad_J).to(ldt).to(ldev)
        return gF, gU, None, None, None, None, None


def kinetic_energy(lattice, force, lid, T, K, p0=None, u0=None):
    """Differentiable J(force, lid) on `lattice` (a Lattice created with has_force=True)."""
    return LBMKineticEnergy.apply(force, lid, lattice, T, K, p0, u0)
