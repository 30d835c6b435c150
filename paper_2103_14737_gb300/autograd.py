"""torch.autograd binding of the simulation: dense cell energies as a
differentiable function of the layer-fraction table and the shape weights.

Forward is ``fcs_simulate_events`` (dense cells), backward is
``fcs_simulate_backward``: with the seed fixed, each hit keeps its task,
count, shape bin and cell, and the parameters move only the hit energies
E f / n (Sec. 4) and, through the likelihood ratio of the drawn shape bin,
the weight of each hit.  The parameters are pushed into the library with
``fcs_update_params`` whenever the tensors changed since the last push.
"""
from __future__ import annotations

import torch

from .fcs import MODE_ATOMIC, Simulator


class _Pushed:
    """Remembers which tensor versions the library holds."""

    def __init__(self):
        self.key = None


def _push(sim: Simulator, frac: torch.Tensor, shape_w: torch.Tensor):
    key = (frac.data_ptr(), frac._version, shape_w.data_ptr(), shape_w._version)
    state = sim.__dict__.setdefault("_pushed", _Pushed())
    if state.key != key:
        sim.update_params(frac=frac.detach().contiguous().reshape(-1),
                          shape_w=shape_w.detach().contiguous().reshape(-1))
        state.key = key


class SimulateCells(torch.autograd.Function):
    """cells[n_events][n_cells] = simulate(frac, shape_w; particles, seed)."""

    @staticmethod
    def forward(ctx, frac, shape_w, sim: Simulator, dparts, seed: int, first_event: int = 0):
        _push(sim, frac, shape_w)
        n_events = dparts["event_offsets"].numel() - 1
        cells = torch.empty((n_events, sim.n_cells), dtype=torch.float32, device=dparts["E"].device)
        sim.simulate(dparts, seed, first_event, mode=MODE_ATOMIC, outputs=dict(cells=cells))
        ctx.sim, ctx.dparts, ctx.seed, ctx.first_event = sim, dparts, seed, first_event
        ctx.frac_shape, ctx.w_shape = frac.shape, shape_w.shape
        ctx.save_for_backward(frac, shape_w)
        return cells

    @staticmethod
    def backward(ctx, grad_cells):
        frac, shape_w = ctx.saved_tensors
        _push(ctx.sim, frac, shape_w)
        g = ctx.sim.backward(ctx.dparts, ctx.seed, grad_cells.float().contiguous(), ctx.first_event)
        return (g["d_frac"].view(ctx.frac_shape), g["d_shape_w"].view(ctx.w_shape), None, None, None, None)


def simulate_cells(sim: Simulator, frac: torch.Tensor, shape_w: torch.Tensor, dparts, seed: int,
                   first_event: int = 0) -> torch.Tensor:
    return SimulateCells.apply(frac, shape_w, sim, dparts, seed, first_event)
