"""Differentiable energies: a torch.autograd.Function around the library's
forward (flr_energy_forces_uncertainty_batch) and its hand-written backward
(flr_energy_backward).

    E = energies(pos, beta, batch_model)   # [n_atoms], differentiable
    (w * E).sum().backward()               # pos.grad, beta.grad

pos.grad = -(forces of the weighted energy) comes from the force kernel with
the per-atom weights applied to g = dE/dB; beta.grad_s = sum_i u_i d_i d_i^T
comes from a block kernel over the compact descriptor rows.  Descriptors,
radial values and harmonics are recomputed in the backward call, not stored.
"""
from __future__ import annotations

import numpy as np
import torch

from . import flare as F


class BatchModel:
    """What stays fixed across forward calls: the context (hyperparameters,
    precision), Sigma, species, cells and structure offsets."""

    def __init__(self, ff: F.FlareGB, sigma, species, offsets, cells, pbc):
        self.ff = ff
        self.sigma = np.ascontiguousarray(sigma, np.float64)
        self.species = torch.as_tensor(species, dtype=torch.int32, device="cuda").contiguous()
        self.offsets = np.ascontiguousarray(offsets, np.int32)
        self.cells = np.ascontiguousarray(np.asarray(cells, np.float64).reshape(-1, 9))
        self.pbc = np.ascontiguousarray(np.asarray(pbc, np.int32).reshape(-1, 3))
        self.nl = ff.nbrlist(int(self.offsets[-1]))

    @staticmethod
    def from_structures(ff, sigma, structs):
        sp = np.concatenate([np.asarray(s.species, np.int32) for s in structs])
        offsets = np.concatenate([[0], np.cumsum([len(s.species) for s in structs])]).astype(np.int32)
        return BatchModel(ff, sigma, sp, offsets, np.stack([np.asarray(s.cell).ravel() for s in structs]),
                          np.stack([np.asarray(s.pbc, np.int32) for s in structs]))

    def batch(self, pos4):
        return F.Batch(pos4, self.species, self.offsets, self.cells, self.pbc)


class _EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, beta, model: BatchModel):
        n = pos.shape[0]
        pos4 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        pos4[:, :3] = pos.detach().to(torch.float32)
        model.ff.set_model(beta.detach().to("cpu", torch.float64).numpy(), model.sigma)
        b = model.batch(pos4)
        F.build_neighbors_batch(model.ff, b, model.nl)
        out = F.energy_forces_uncertainty_batch(model.ff, b, model.nl)
        ctx.model = model
        ctx.pos4 = pos4
        ctx.beta_meta = (beta.dtype, beta.device)
        ctx.mark_non_differentiable(out["forces"], out["sigma"])
        return out["energy"], out["forces"], out["sigma"]

    @staticmethod
    def backward(ctx, g_energy, g_forces, g_sigma):
        model = ctx.model
        if g_energy is None:
            return None, None, None
        b = model.batch(ctx.pos4)
        want_beta = ctx.needs_input_grad[1]
        gpos, gbeta = F.energy_backward(model.ff, b, model.nl, g_energy, want_beta=want_beta)
        dt, dev = ctx.beta_meta
        gpos = gpos if ctx.needs_input_grad[0] else None
        gb = gbeta.to(device=dev, dtype=dt) if gbeta is not None else None
        return gpos, gb, None


def energies(pos: torch.Tensor, beta: torch.Tensor, model: BatchModel):
    """Per-atom energies [n] (differentiable in pos [n, 3] and beta
    [n_species, d, d]); also returns forces [n, 3] and sigma [n] as
    non-differentiable tensors."""
    return _EnergyFn.apply(pos, beta, model)
