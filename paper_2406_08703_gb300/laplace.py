"""Laplace-approximation errors (Sec. 4): the curvature of the Poisson
likelihood over the source positions, fluxes and Zernike coefficients, with the
pixel response held fixed, and the 1-sigma errors sqrt(diag(H^-1)) marginalised
over all of those parameters.

Three curvature matrices are offered (`kind`):
  "hessian"      -- the Hessian of the negative log-likelihood sum (m - d ln m),
                    H = J^T diag(d/m^2) J + sum_p (1 - d_p/m_p) d^2 m_p;
  "gauss_newton" -- its first term alone;
  "fisher"       -- the expected information J^T diag(1/m) J.

Every column of J = dm/dtheta is exact up to rounding, with no step size to tune:
  position theta_{s,x|y}: dlx_model_jvp along the pupil coordinate x or y
      (the tilt of source s), on a plan of that one source;
  Zernike c_j: dlx_model_jvp along the basis map Z_j, every source;
  flux F_s: the model of source s alone with unit flux (the model is linear
      in each flux).
The second-order term comes column by column from dlx_model_vjp_jvp (positions,
Zernikes) and dlx_model_vjp with unit flux (fluxes), all with the cotangent
1 - d/m held fixed.  A source's position and flux columns touch only that
source's images, so they run on a one-source plan at 1/n_src of the cost.
The Gram products run in dlx_fisher_gram; only the inversion of the small
(n_par x n_par) matrix runs on the host, in float64.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

from . import (dlx_fisher_gram, dlx_forward, dlx_make_mft, dlx_model_jvp, dlx_model_vjp, dlx_model_vjp_jvp,
               dlx_nll_cotangent, empty_grads, GRAM_MAX_PAR)

GROUPS = ("pos", "flux", "zern")
KINDS = ("hessian", "gauss_newton", "fisher")


def labels(n_src: int, n_zern: int, groups: Sequence[str] = GROUPS) -> list:
    """Parameter order of the matrices: ("pos", s, axis), ("flux", s), ("zern", j)."""
    out = []
    for g in groups:
        if g == "pos":
            out += [("pos", s, a) for s in range(n_src) for a in (0, 1)]
        elif g == "flux":
            out += [("flux", s) for s in range(n_src)]
        elif g == "zern":
            out += [("zern", j) for j in range(n_zern)]
        else:
            raise KeyError(f"unknown parameter group {g!r}")
    return out


class Laplace:
    """Curvature and errors of one plan's model.  Builds (once) the one-source
    plan of the same shape and form for the per-source columns."""

    def __init__(self, plan, groups: Sequence[str] = GROUPS):
        import torch

        self.plan = plan
        self.groups = tuple(groups)
        i = plan.info
        self.ns, self.nz, self.ni = i.n_src, i.n_zern, i.n_pupil
        self.shape = (i.n_exp, i.n_det, i.n_det)
        self.labels = labels(self.ns, self.nz, self.groups)
        if len(self.labels) > GRAM_MAX_PAR:
            raise ValueError(f"{len(self.labels)} parameters; dlx_fisher_gram takes at most {GRAM_MAX_PAR}")
        self.dev = f"cuda:{plan.device}"
        if self.ns == 1:
            self.single = plan
        else:
            self.single = dlx_make_mft(dataclasses.replace(plan.desc, n_src=1), plan.device)
        # pupil coordinates (metres) as optical-path tangents of a tilt: t[ny][nx] = x_nx or y_ny
        d = plan.desc.diameter_m / self.ni
        x = ((torch.arange(self.ni, dtype=torch.float64) - 0.5 * (self.ni - 1)) * d).to(torch.float32)
        self.tx = x[None, :].expand(self.ni, self.ni).contiguous().to(self.dev)
        self.ty = x[:, None].expand(self.ni, self.ni).contiguous().to(self.dev)
        self.k_max = 2.0 * math.pi / min(plan.desc.lambdas)

    def _alpha(self, t) -> float:
        """Step of the central difference: largest phase change of the tangent near 1 rad (the
        difference is exact for any step; this keeps both models far above their rounding)."""
        a = self.k_max * float(t.abs().max())
        return 1.0 / a if a > 0 else 1.0

    def _source(self, params: dict, s: int, unit_flux: bool = False) -> dict:
        import torch

        q = dict(params)
        q["pos"] = params["pos"][s:s + 1].contiguous()
        q["flux"] = torch.ones(1, dtype=torch.float32, device=self.dev) if unit_flux else \
            params["flux"][s:s + 1].contiguous()
        return q

    def _tangent(self, params: dict, lab):
        """(plan, params, t_map, src_mask) of a position or Zernike column."""
        if lab[0] == "pos":
            return self.single, self._source(params, lab[1]), (self.tx if lab[2] == 0 else self.ty), 1
        return self.plan, params, params["zern_basis"][lab[1]], (1 << self.ns) - 1 if self.ns < 32 else 0xffffffff

    def jacobian(self, params: dict, stream=None):
        """J [n_par][n_exp Nd Nd] float32 on the device, rows in `labels` order."""
        import torch

        J = torch.empty((len(self.labels), int(np.prod(self.shape))), dtype=torch.float32, device=self.dev)
        work = torch.empty(self.shape, dtype=torch.float32, device=self.dev)
        for k, lab in enumerate(self.labels):
            row = J[k].view(self.shape)
            if lab[0] == "flux":
                dlx_forward(self.single, self._source(params, lab[1], unit_flux=True), model=row, stream=stream)
            else:
                plan, prm, t, mask = self._tangent(params, lab)
                dlx_model_jvp(plan, prm, t, mask, self._alpha(t), jvp=row, work=work, stream=stream)
        return J

    def _second_order(self, params: dict, cot, stream=None):
        """R = sum_p cot_p d^2 m_p over the parameter pairs (float64 device [n_par][n_par]), symmetrised."""
        import torch

        n = len(self.labels)
        index = {lab: k for k, lab in enumerate(self.labels)}
        R = torch.zeros((n, n), dtype=torch.float64, device=self.dev)
        which = ("d_zern", "d_flux", "d_pos")
        g_full, w_full = empty_grads(self.plan, which), empty_grads(self.plan, which)
        g_one, w_one = empty_grads(self.single, which), empty_grads(self.single, which)

        def scatter(col, g, src):
            # src None: gradients of the full plan; else of the one-source plan (its row 0 = source src)
            parts, rows = [], []
            ss = list(range(self.ns)) if src is None else [src]
            sel = slice(None) if src is None else slice(0, 1)
            for grp in self.groups:
                if grp == "pos":
                    parts.append(g["d_pos"][sel].reshape(-1))
                    rows += [index[("pos", s, a)] for s in ss for a in (0, 1)]
                elif grp == "flux":
                    parts.append(g["d_flux"][sel])
                    rows += [index[("flux", s)] for s in ss]
                elif self.nz:
                    parts.append(g["d_zern"])
                    rows += [index[("zern", j)] for j in range(self.nz)]
            R[torch.tensor(rows, device=self.dev), col] = torch.cat(parts).double()

        for k, lab in enumerate(self.labels):
            if lab[0] == "flux":
                # d^2 m / (d theta dF_s) = d(m of source s at unit flux) / d theta;  d^2 m / dF^2 = 0
                dlx_model_vjp(self.single, self._source(params, lab[1], unit_flux=True), cot, grads=g_one,
                              stream=stream)
                scatter(k, g_one, lab[1])
                R[k, k] = 0.0
                continue
            plan, prm, t, mask = self._tangent(params, lab)
            if lab[0] == "pos":
                dlx_model_vjp_jvp(plan, prm, cot, t, mask, self._alpha(t), grads=g_one, work=w_one, stream=stream)
                scatter(k, g_one, lab[1])
            else:
                dlx_model_vjp_jvp(plan, prm, cot, t, mask, self._alpha(t), grads=g_full, work=w_full,
                                  stream=stream)
                scatter(k, g_full, None)
        return 0.5 * (R + R.T)

    def information(self, params: dict, data=None, kind: str = "hessian", stream=None):
        """Curvature matrix (float64 device [n_par][n_par]) of the kind named in KINDS."""
        if kind not in KINDS:
            raise KeyError(f"kind must be one of {KINDS}")
        if kind != "fisher" and data is None:
            raise ValueError(f"kind {kind!r} needs the data")
        model = dlx_forward(self.plan, params, stream=stream)
        J = self.jacobian(params, stream=stream)
        flat_m = model.view(-1)
        if kind == "fisher":
            return dlx_fisher_gram(J, flat_m, None, stream=stream)
        H = dlx_fisher_gram(J, flat_m, data.view(-1), stream=stream)
        if kind == "hessian":
            cot = dlx_nll_cotangent(model, data, stream=stream)
            H = H + self._second_order(params, cot, stream=stream)
        return H

    def errors(self, params: dict, data=None, kind: str = "hessian", stream=None) -> dict:
        """1-sigma errors sqrt(diag(H^-1)), marginalised over every parameter of the groups."""
        H = self.information(params, data, kind, stream=stream).cpu().numpy()
        return errors_from_information(H, self.labels, self.ns, self.nz)


def errors_from_information(H: np.ndarray, labs: list, n_src: int, n_zern: int) -> dict:
    """Inverse of the curvature after scaling it to unit diagonal (float64, host)."""
    d = np.sqrt(np.abs(np.diag(H)))
    d[d == 0] = 1.0
    Hs = H / np.outer(d, d)
    cov = np.linalg.inv(Hs) / np.outer(d, d)
    var = np.diag(cov)
    sigma = np.where(var > 0, np.sqrt(np.abs(var)), np.nan)
    out = dict(labels=labs, information=H, cov=cov, sigma=sigma, sigma_pos=np.full((n_src, 2), np.nan),
               sigma_flux=np.full(n_src, np.nan), sigma_zern=np.full(n_zern, np.nan))
    for k, lab in enumerate(labs):
        if lab[0] == "pos":
            out["sigma_pos"][lab[1], lab[2]] = sigma[k]
        elif lab[0] == "flux":
            out["sigma_flux"][lab[1]] = sigma[k]
        else:
            out["sigma_zern"][lab[1]] = sigma[k]
    return out


def laplace_errors(plan, params: dict, data=None, kind: str = "hessian", groups: Sequence[str] = GROUPS,
                   stream=None) -> dict:
    """One-call form of Laplace(plan, groups).errors(params, data, kind)."""
    return Laplace(plan, groups).errors(params, data, kind, stream=stream)
