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


def new_state(params: dict, groups=GROUPS) -> dict:
    """Adam state of every group: {group: [m, v, steps]} (device tensors shaped like the parameter)."""
    import torch

    return {g: [torch.zeros_like(params[GROUPS[g][0]]), torch.zeros_like(params[GROUPS[g][0]]), 0]
            for g in groups if params.get(GROUPS[g][0]) is not None}


def checkpoint(params: dict, state: dict) -> dict:
    """Host copy of a fit: every parameter tensor and each group's Adam moments and step count.
    `restore` turns it back into device tensors; continuing from it repeats the uninterrupted fit
    bit for bit (every kernel here sums in a fixed order)."""
    out = {"param/" + k: v.detach().cpu().numpy().copy() for k, v in params.items() if v is not None}
    for g, (m, v, t) in state.items():
        out["m/" + g] = m.detach().cpu().numpy().copy()
        out["v/" + g] = v.detach().cpu().numpy().copy()
        out["t/" + g] = t
    return out


def restore(ckpt: dict, device: str = "cuda") -> tuple:
    """(params, state) as device tensors from `checkpoint`'s host copy."""
    import torch

    params = {k[6:]: torch.as_tensor(v, device=device).clone() for k, v in ckpt.items() if k.startswith("param/")}
    state = {}
    for k, v in ckpt.items():
        if k.startswith("m/"):
            g = k[2:]
            state[g] = [torch.as_tensor(v, device=device).clone(), torch.as_tensor(ckpt["v/" + g], device=device).clone(),
                        int(ckpt["t/" + g])]
    return params, state


def staged_fit(plan, params: dict, data, stages: Sequence, stream=None, beta1: float = 0.9, beta2: float = 0.999,
               eps: float = 1e-8, losses: Optional[object] = None, state: Optional[dict] = None) -> object:
    """Runs the stages in place on `params` (float32 device tensors, updated in
    place).  `stages` is a list of (n_epochs, {group: learning rate}).  `state`
    (from `new_state`, or `restore` of a checkpoint) carries each group's Adam
    moments and step count across calls and is updated in place; without it a
    fresh state is used.  Returns the float64 device tensor of the loss of every
    epoch (evaluated before that epoch's update)."""
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
    if state is None:
        state = new_state(params, used)
    for g in used:
        if g not in state:
            state[g] = new_state(params, [g])[g]
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
