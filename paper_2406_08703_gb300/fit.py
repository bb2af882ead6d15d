"""Staged gradient-descent fit (Sec. 4 of the paper): Adam (Kingma & Ba) on the
parameter groups of a loss-and-gradient plan, every state tensor on the device.

The paper fits the positions, fluxes and aberrations first with the pixel
response frozen, then the pixel response alone.  A stage here is a number of
epochs and one learning rate per parameter group; a zero (or absent) rate
freezes the group for that stage, and each group keeps its own Adam step count,
so a group that starts learning in a later stage starts with bias-corrected
moments.  One epoch is one dlx_loss_grad over the whole model followed by one
dlx_adam per active group; nothing is copied to the host until the fit ends.
"""

from __future__ import annotations

from typing import Optional, Sequence

from . import dlx_adam, dlx_loss_grad, empty_grads

# parameter group -> (parameter key, gradient key)
GROUPS = {
    "zern": ("zern_coeff", "d_zern"),
    "opd_pix": ("opd_pix", "d_opd_pix"),
    "flat": ("flat", "d_flat"),
    "flux": ("flux", "d_flux"),
    "pos": ("pos", "d_pos"),
}


def paper_schedule(lr: dict, epochs_psf: int = 100, epochs_prf: int = 50) -> list:
    """The paper's two stages: the PSF parameters (positions, fluxes, aberrations)
    with the pixel-response rate at zero, then the pixel response alone."""
    psf = {k: v for k, v in lr.items() if k != "flat"}
    return [(epochs_psf, psf), (epochs_prf, {"flat": lr["flat"]})]


def staged_fit(plan, params: dict, data, stages: Sequence, stream=None, beta1: float = 0.9, beta2: float = 0.999,
               eps: float = 1e-8, losses: Optional[object] = None) -> object:
    """Runs the stages in place on `params` (float32 device tensors, updated in
    place).  `stages` is a list of (n_epochs, {group: learning rate}).  Returns
    the float64 device tensor of the loss of every epoch (evaluated before that
    epoch's update)."""
    import torch

    n_total = sum(int(n) for n, _ in stages)
    dev = f"cuda:{plan.device}"
    if losses is None:
        losses = torch.empty(n_total, dtype=torch.float64, device=dev)
    used = {g for _, lrs in stages for g, lr in lrs.items() if lr}
    for g in used:
        if g not in GROUPS:
            raise KeyError(f"unknown parameter group {g!r}")
        if params.get(GROUPS[g][0]) is None:
            raise ValueError(f"group {g!r} has no parameter tensor")
    grads = empty_grads(plan)
    state = {g: [torch.zeros_like(params[GROUPS[g][0]]), torch.zeros_like(params[GROUPS[g][0]]), 0] for g in used}
    i = 0
    for n, lrs in stages:
        for _ in range(int(n)):
            dlx_loss_grad(plan, params, data, loss=losses[i:i + 1], grads=grads, stream=stream)
            for g, lr in lrs.items():
                if not lr:
                    continue
                pk, gk = GROUPS[g]
                st = state[g]
                st[2] += 1
                dlx_adam(params[pk], grads[gk], st[0], st[1], float(lr), st[2], beta1, beta2, eps, stream=stream)
            i += 1
    return losses
