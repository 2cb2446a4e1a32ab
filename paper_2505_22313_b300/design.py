"""Design loop: the recipe of the paper's toy example (Sec. 3.2) on this library's adjoint.

Adam on the height map (doe_adam_step), gradients from doe_grad against a target intensity
(the L2 loss of Eq. 4 stands in for the supplement's task losses), the learning rate decayed
to zero with a cosine schedule, and the heights kept in the fabricable range [0, h_max] after
every step.  Every step runs in the library's kernels; this module only sequences the calls
and keeps the per-step losses on the device until the end.

    from paper_2505_22313_b300 import design, api
    h, losses = design.optimize(h0, geom, target, iters=3000)

The broadband design of Sec. 5.4 keeps the phase radially symmetric through a polynomial in the
radius; ``optimize_radial`` runs the same loop on the coefficients of that polynomial
(doe_radial_heights, then doe_grad, then doe_radial_grad, then Adam on the coefficients).
"""
from __future__ import annotations

import math

import torch

from . import _lib, api
from .inputs import HMAX


def cosine_lr(lr0: float, t: int, iters: int) -> float:
    """Learning rate of step t = 1..iters: lr0 (1 + cos(pi (t - 1) / iters)) / 2, from lr0 down
    to (almost) zero at the last step."""
    return 0.5 * lr0 * (1.0 + math.cos(math.pi * (t - 1) / iters))


def optimize(h0: torch.Tensor, geom: api.Geometry, target: torch.Tensor, iters: int, lr0: float | None = None,
             h_max: float = HMAX, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             stream=None):
    """Returns (heights, losses): the optimised heights (a new tensor) and the loss before each
    step, float64 [iters] on the device.  lr0 defaults to 1e-2 h_max: the paper's initial
    rate 1e-2 read on heights normalised to the fabricable range."""
    h = h0.detach().clone().to(torch.float32)
    m = torch.zeros_like(h)
    v = torch.zeros_like(h)
    g = torch.empty_like(h)
    losses = torch.empty((iters,), dtype=torch.float64, device=h.device)
    ws = api.workspace(api.workspace_bytes(geom, _lib.DOE_OP_GRAD), h.device)
    lr0 = 1e-2 * h_max if lr0 is None else lr0
    for t in range(1, iters + 1):
        api.grad(h, geom, target, out=g, loss=losses[t - 1:t], ws=ws, stream=stream)
        api.adam_step(h, g, m, v, cosine_lr(lr0, t, iters), t, beta1, beta2, eps, 0.0, h_max, stream=stream)
    return h, losses


def optimize_radial(c0: torch.Tensor, geom: api.Geometry, target: torch.Tensor, iters: int, lr0: float,
                    beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
    """Returns (coefficients, losses): the optimised radial coefficients c (float32 [n_c], a new
    tensor; heights h = sum_k c[k] (rho / R)^(2k) on the geometry's height grid) and the loss
    before each step, float64 [iters] on the device.  The coefficients are not projected: the
    phase wraps, so heights outside [0, h_max] only cost fabrication range, not correctness."""
    c = c0.detach().clone().to(torch.float32)
    n_c, n = c.numel(), geom.NL
    m = torch.zeros_like(c)
    v = torch.zeros_like(c)
    gc = torch.empty_like(c)
    h = torch.empty((n, n), dtype=torch.float32, device=c.device)
    gh = torch.empty_like(h)
    losses = torch.empty((iters,), dtype=torch.float64, device=c.device)
    ws = api.workspace(api.workspace_bytes(geom, _lib.DOE_OP_GRAD), c.device)
    wr = api.workspace(_lib.load().doe_radial_workspace_bytes(n_c), c.device)
    inf = float("inf")
    for t in range(1, iters + 1):
        api.radial_heights(c, n, out=h, stream=stream)
        api.grad(h, geom, target, out=gh, loss=losses[t - 1:t], ws=ws, stream=stream)
        api.radial_grad(gh, n_c, out=gc, ws=wr, stream=stream)
        api.adam_step(c, gc, m, v, cosine_lr(lr0, t, iters), t, beta1, beta2, eps, -inf, inf, stream=stream)
    return c, losses
