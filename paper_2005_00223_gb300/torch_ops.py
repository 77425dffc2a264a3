"""torch.autograd.Function around the library's hand-written adjoint.

``dp_energy(model, nlist, coord, box, prec)`` returns the total energy as a
differentiable function of the coordinates (a CUDA float64 tensor [n, 3]).
The forward pass runs dp_compute_dev, which evaluates the energy and, in
the same pass, its adjoint (forces); backward returns -grad_out * F without
re-evaluating anything.  The virial and per-atom energies are returned as
non-differentiable extras.  PyTorch only provides the device buffers and
the stream: every arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import _lib


class DPEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coord, model_h, nlist_h, box, prec):
        if not coord.is_cuda or coord.dtype != torch.float64:
            raise TypeError("coord must be a CUDA float64 tensor")
        coord = coord.contiguous()
        n = coord.shape[0]
        energy = torch.empty(1, dtype=torch.float64, device=coord.device)
        atom_energy = torch.empty(n, dtype=torch.float64, device=coord.device)
        force = torch.empty((n, 3), dtype=torch.float64, device=coord.device)
        virial = torch.empty((3, 3), dtype=torch.float64, device=coord.device)
        stream = torch.cuda.current_stream(coord.device)
        _lib.dp_compute_dev(model_h, nlist_h, coord, box, prec, energy, atom_energy, force, virial, stream)
        ctx.save_for_backward(force)
        ctx.mark_non_differentiable(atom_energy, force, virial)
        return energy[0], atom_energy, force, virial

    @staticmethod
    def backward(ctx, g_energy, g_atom_energy, g_force, g_virial):
        (force,) = ctx.saved_tensors
        return -g_energy * force, None, None, None, None


def dp_energy(model, nlist, coord, box, prec="fp64"):
    """E, E_i, F, W with E differentiable w.r.t. coord (autograd uses F = -dE/dr)."""
    return DPEnergy.apply(coord, model.h, nlist.h, box, prec)
